// Persistent batched step (FP32-bulk forms): one cooperative launch advances
// every member of an ensemble of independent runs by one AB2 step.
//
// The work items: first the ghost items of every member (chunks of its AT
// ghost points: Table B extrapolation, Appendix B, with the delays of
// Sec. 3.1 computed in place from the counter-based generator, and the ring
// slabs of the current level -- the work of the delay-map and ghost kernels
// of a single step), then the tiles of every member on the paired fused
// kernel (kernels_fused2.cuh).  Items are dealt round-robin to the CTAs (item
// = CTA + k * grid), each CTA taking its items in increasing order; a tile
// waits (bounded) until its own member's ghost items are done, so the tiles
// of the members whose ghosts finished first start while other CTAs still
// assemble ghosts.  Every wait is for items of lower index, so the lowest
// unfinished item can always proceed and the launch cannot deadlock.  The
// member of an item is found by a search of constant-memory prefix sums with
// a CTA-uniform index, and the tile body reads its member's description from
// constant memory.  The CTA that finishes a member's last tile sums the
// member's statistics partials in a fixed order and advances the member's
// step state.
//
// Members may differ in grid, PEs, Mach number, viscosity, precision form
// (P32 or P32C) and z chunk; they share the tile shape (TX, TY) of the
// launch and the delay mode of the step.
#pragma once
#include "batch.h"
#include "kernels_fused2.cuh"

namespace atdns {

// The members' tile descriptions, their shapes {ZC, tiles_x, tiles_y, ghost
// items} and the prefix sums of their ghost items and of their tiles.
__constant__ TileDesc c_tiles[kBatchConstMembers];
__constant__ int c_shape[kBatchConstMembers][4];
__constant__ long long c_gitems[kBatchConstMembers + 1];
__constant__ long long c_items[kBatchConstMembers + 1];

// Member of work item v given the prefix sums pre[0 .. count] (v uniform
// over the CTA, pre in constant memory).
__device__ __forceinline__ int member_of(const long long* pre, int count, long long v) {
  int lo = 0, hi = count;   // pre[lo] <= v < pre[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pre[mid] <= v) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Bounded wait of one thread until *ctr == target: at most max_polls polls
// about 64 ns apart; false when it gave up.
constexpr long long kBatchWaitPolls = 1LL << 26;   // seconds: far beyond any ghost item
__device__ __forceinline__ bool wait_count(const unsigned* ctr, unsigned target, long long max_polls) {
  const volatile unsigned* c = ctr;
  long long polls = 0;
  while (*c != target) {
    if (++polls > max_polls) return false;
    __nanosleep(64);
  }
  __threadfence();
  return true;
}

// Self-test of the bounded wait: one thread waits for a count that nothing
// advances; *out = 1 when the wait gave up (the expected result), 0 if not.
__global__ void k_wait_selftest(const unsigned* ctr, long long max_polls, int* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = wait_count(ctr, 1u, max_polls) ? 0 : 1;
}

template <int TX, int TY>
__global__ void __launch_bounds__(TX * TY / 2, (TX * TY / 2 <= 128) ? 2 : 1) k_batch_step(BatchSched S) {
  extern __shared__ __align__(16) unsigned char fused_smem[];
  __shared__ int s_flag;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int count = S.count;
  const long long gitems_all = c_gitems[count];
  const long long items = gitems_all + c_items[count];
  for (long long item = blockIdx.x; item < items; item += gridDim.x) {
    if (item < gitems_all) {
      const int mi = member_of(c_gitems, count, item);
      const BatchMember& m = S.m[mi];
      const long long local = item - c_gitems[mi];
      // ---- a ghost item: kBatchGhostChunk of the member's ghost points
      if (local == 0 && tid == 0) {   // the step's max/min keys, before any tile of the member
        m.A.words[0] = (unsigned long long)LLONG_MIN;
        m.A.words[1] = (unsigned long long)LLONG_MAX;
        m.A.words[2] = (unsigned long long)LLONG_MAX;
      }
      const long long gtot = m.ghost_cnt[0] + m.ghost_cnt[1] + m.ghost_cnt[2];
      const long long j0 = local * kBatchGhostChunk;
      const long long j1 = j0 + kBatchGhostChunk < gtot ? j0 + kBatchGhostChunk : gtot;
      const long long n = m.A.ds->n;
      auto delay = [&](int p, int face) { return delay_of(m.mode, n, p, face, m.L, m.tl, m.cr, m.k0, m.k1); };
      for (long long j = j0 + tid; j < j1; j += nt)
        ghost_point<float, 2>(m.g, m.K, m.A.Ub[0], m.A.Ub[1], m.A.Ulob[0], m.A.Ulob[1], m.A.ds, nullptr, m.GH[0],
                              m.GH[1], m.GH[2], m.ring[0], m.ring[1], m.ring[2], m.xst, m.xst_half, delay, n,
                              m.ghost_cnt[0], m.ghost_cnt[1], m.ghost_cnt[2], j);
      __threadfence();
      __syncthreads();
      if (tid == 0) atomicAdd(S.gdone + mi, 1u);
      continue;
    }
    // ---- a tile: after the member's ghost items of this step
    const long long tv = item - gitems_all;
    const int mi = member_of(c_items, count, tv);
    const BatchMember& m = S.m[mi];
    if (tid == 0) {
      s_flag = wait_count(S.gdone + mi, S.epoch * (unsigned)c_shape[mi][3], kBatchWaitPolls);
      if (!s_flag) atomicExch(S.err, 1);
    }
    __syncthreads();
    if (!s_flag) return;
    const long long t = tv - c_items[mi];
    const int tiles_x = c_shape[mi][1], tiles_y = c_shape[mi][2];
    const int bx = (int)(t % tiles_x);
    const int by = (int)((t / tiles_x) % tiles_y);
    const int bz = (int)(t / ((long long)tiles_x * tiles_y));
    fused2_tile<TX, TY>(c_tiles[mi].g, c_tiles[mi].K, c_tiles[mi].KP, c_tiles[mi].A, c_shape[mi][0], bx, by, bz, t,
                        fused_smem);
    // the member's last tile: statistics in a fixed order, then the step advance
    __threadfence();
    __syncthreads();
    if (tid == 0) s_flag = atomicAdd(S.tdone + mi, 1u) + 1u == S.epoch * (unsigned)m.nblk;
    __syncthreads();
    if (s_flag) {
      __threadfence();
      if (m.A.do_stats && tid < kNumStat) {
        double a = 0.0;
        for (long long b = 0; b < m.nblk; ++b) a += m.A.partial[b * kNumStat + tid];
        m.sums[tid] = a;
      }
      if (tid == 0) {
        DevState* ds = const_cast<DevState*>(m.A.ds);
        ds->n += 1;
        ds->first = 0;
        ds->cur = 1 - ds->cur;
      }
    }
    __syncthreads();
  }
}

}  // namespace atdns
