// Plain-data description of a persistent batched step (FP32-bulk forms),
// shared by the kernel (kernels_batch.cuh) and the C ABI that builds it.
#pragma once
#include "common.cuh"

namespace atdns {

// Members of a batch the persistent step takes (the tile descriptions of all
// of them fit the constant bank of its module).
constexpr int kBatchConstMembers = 64;

// What a tile of one member reads: the same description a standalone step
// passes to the paired kernel as parameters.  The persistent step keeps the
// members' descriptions in constant memory and indexes them with a CTA-uniform
// member number, so the tile body takes its coefficients from the constant
// bank exactly as the standalone kernel takes them from its parameters.
struct TileDesc {
  Geom g;
  Coef<float> K;
  CoefPair KP;
  StepArgs<float> A;
};

// What one member's step needs besides (built on the host, read from global
// memory).
struct BatchMember {
  Geom g;
  Coef<float> K;
  CoefPair KP;
  StepArgs<float> A;            // as for a single step: A.ds is the member's device step state
  int mode, L, tl, cr;          // delay mode and parameters (Sec. 3.1)
  uint32_t k0, k1;              // key of the delay stream
  float* GH[3];                 // ghost arrays per direction
  double* ring[3];              // FP64 slab ring per direction
  const float* xst;             // staged x-face slabs (or null)
  long long xst_half;
  long long ghost_cnt[3];       // ghost points per direction
  long long nblk;               // tiles (rows of A.partial)
  double* sums;                 // [kNumStat] final statistics sums
};

// Ghost points of one ghost work item.
constexpr int kBatchGhostChunk = 1024;

struct BatchSched {
  const BatchMember* m;
  int count;
  unsigned* gdone;                // [count] ghost items finished (monotone over launches)
  unsigned* tdone;                // [count] tiles finished (monotone over launches)
  int* err;                       // set when a wait gave up
  unsigned epoch;                 // launches since the counters were cleared, this one included
};

// Persistent batched step on (TX, TY) paired tiles: the number of CTAs that
// are resident together (grid of the cooperative launch), the upload of the
// members' tile descriptions, shapes {ZC, tiles_x, tiles_y, ghost items} and
// the prefix sums of their ghost items and of their tiles to constant memory
// (stream ordered; count <= kBatchConstMembers), and the launch.
cudaError_t batch_resident_ctas(int TX, int TY, int* ctas);
cudaError_t upload_batch_tiles(const TileDesc* desc, const int (*shape)[4], const long long* ghost_prefix,
                               const long long* tile_prefix, int count, cudaStream_t st);
cudaError_t launch_batch_step(int TX, int TY, const BatchSched& S, int ctas, cudaStream_t st);
// The persistent step's bounded wait, run on a count that nothing advances
// with at most 2^log2_polls polls: *gave_up = 1 when it returned unsatisfied.
cudaError_t batch_wait_selftest(int log2_polls, int* gave_up);

}  // namespace atdns
