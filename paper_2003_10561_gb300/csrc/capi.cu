// C ABI of the AT-DNS library (include/at_dns.h): handle, allocation, state
// transfer, step orchestration and the small kernels around the step (delay
// map, ring fill, forcing, wave speed, final reductions).
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <algorithm>
#include <array>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/at_dns.h"
#include "batch.h"
#include "common.cuh"
#include "launch.h"

using namespace atdns;

namespace {

thread_local std::string g_create_error;

struct Mode3 { int kx, ky, kz; };

}  // namespace

struct at_dns {
  at_dns_config_t cfg{};
  Geom g{};
  Phys ph{};
  cudaStream_t st = nullptr;
  bool p64 = true;
  size_t ssize = 8;            // bytes of the scalar type
  // device buffers (scalar type S unless noted)
  void* U[2] = {nullptr, nullptr};
  void* Ulo[2] = {nullptr, nullptr};   // compensated form: low words of U
  bool comp = false;
  int cur = 0;
  void* PQ = nullptr;
  void* G = nullptr;
  void* Rprev = nullptr;
  void* GH[3] = {nullptr, nullptr, nullptr};
  void* ring[3] = {nullptr, nullptr, nullptr};
  void* xst = nullptr;         // FP32 forms: x-face slabs of the state [hi, lo][5][2M P_x][plane_x]
  long long xst_half = 0;      // elements from its hi half to its lo half (compensated form; else 0)
  double* stage = nullptr;     // [5][npts] FP64 staging / rhs output
  uint8_t* dmap = nullptr;     // [P][6]
  double* partial = nullptr;   // [main_blocks][kNumStat]
  double* sums = nullptr;      // [kNumStat]
  unsigned long long* words = nullptr;  // [4]
  // forcing
  int nmodes = 0, fK = 0;
  Mode3* modes = nullptr;      // device
  double2* fhat = nullptr;     // [nmodes][3]
  void* fB = nullptr;          // vec2<S> [(K+1)][3][n2][n1]
  void* fX = nullptr;          // vec2<S> [(K+1)][n0]
  // state
  bool has_state = false, first = true, stats_valid = false;
  long long n = 0;
  double t = 0.0, dt = 0.0;
  long long stats_step = 0;
  double stats_time = 0.0;
  size_t bytes = 0;
  // caller-provided device memory: every allocation is carved from it
  char* pool = nullptr;
  size_t pool_size = 0, pool_used = 0;
  std::string err;
  DevState* ds = nullptr;       // device copy of (n, first, cur)
  // captured one-step graphs per delay mode (replayed by at_dns_step)
  cudaGraphExec_t gexec[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double gdt[5] = {0, 0, 0, 0, 0};    // dt the graphs were captured with
  bool use_graphs = true;
  // kernel path: fused single pass on TX x TY tiles marching ZC planes, or multi-pass
  bool fused = false;
  bool paired = false;         // fused pass with two points per thread (FP32 forms)
  int TX = 0, TY = 0, ZC = 0;
  long long nblk_step = 0;     // blocks of the kernel that writes the statistics partials
  // per-kernel event timing
  bool prof = false;
  struct Rec { int kind; cudaEvent_t a, b; };
  std::vector<Rec> recs;
};

// ---------------------------------------------------------------------------
// NVTX ranges around the public calls (host side: the kernels a call enqueues
// fall in its range, so a profiler can select them by the call's name; the
// calls cost nothing measurable when no tool is attached)
namespace {
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace

// ---------------------------------------------------------------------------
// small kernels
namespace {

__global__ void k_delay_map(uint8_t* out, int P, long long n, const DevState* ds, int mode, int L, int tl, int cr,
                            uint32_t k0, uint32_t k1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P * 6) return;
  if (ds) n = ds->n;
  out[i] = (uint8_t)delay_of(mode, n, i / 6, i % 6, L, tl, cr, k0, k1);
}

__global__ void k_set_state(DevState* ds, long long n, int first, int cur) {
  ds->n = n;
  ds->first = first;
  ds->cur = cur;
}

// Between two RK3 stages: the stage state is in the other buffer.
__global__ void k_flip_state(DevState* ds) { ds->cur = 1 - ds->cur; }

// End of a step: level n+1 is in the other buffer and the next step is AB2.
__global__ void k_advance_state(DevState* ds) {
  ds->n += 1;
  ds->first = 0;
  ds->cur = 1 - ds->cur;
}

template <typename S>
__global__ void k_from_double(const double* __restrict__ in, S* __restrict__ out, long long count) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < count) out[i] = (S)in[i];
}

template <typename S>
__global__ void k_to_double(const S* __restrict__ in, double* __restrict__ out, long long count) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < count) out[i] = (double)in[i];
}

// Compensated form: FP64 value -> FP32 high word + FP32 low word (the rest).
__global__ void k_split_double(const double* __restrict__ in, float* __restrict__ hi, float* __restrict__ lo,
                               long long count) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double v = in[i];
  const float h = (float)v;
  hi[i] = h;
  lo[i] = (float)(v - (double)h);
}

__global__ void k_join_double(const float* __restrict__ hi, const float* __restrict__ lo, double* __restrict__ out,
                              long long count) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < count) out[i] = (double)hi[i] + (double)lo[i];
}

// Write the PE-boundary slabs of the FP64 field U ([5][npts]) into ring slot
// `slot` (the ring is FP64 in every precision form): the M layers next to each
// face, slab index 2M pe + t (t < M: local t, t >= M: local nl - 2M + t).
// The PE-boundary slabs of an FP64 field into the ring slots first_slot,
// first_slot + 1, ... (count slots, mod the ring length), one read of the
// field for all of them.  One thread per slab point in the ring's own order
// (direction d's cnt_d points: slab sp = 2M pe + t, plane point pl), so the
// ring writes are coalesced, and so are the field reads of the y- and z-faces.
__global__ void k_ring_store(Geom g, const double* __restrict__ U, double* r0, double* r1, double* r2, long long cnt0,
                             long long cnt1, long long cnt2, int first_slot, int count, const DevState* ds) {
  long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int d = 0;
  if (j >= cnt0) {
    j -= cnt0;
    d = 1;
    if (j >= cnt1) {
      j -= cnt1;
      d = 2;
      if (j >= cnt2) return;
    }
  }
  const long long plane = g.plane[d];
  const long long sp = j / plane, pl = j - sp * plane;
  const int M = g.M, pe = (int)(sp / (2 * M)), t = (int)(sp - 2LL * M * pe);
  const int cd = pe * g.nl[d] + (t < M ? t : g.nl[d] - 2 * M + t);
  int x, y, z;
  if (d == 0) {
    x = cd;
    z = (int)(pl / g.n[1]);
    y = (int)(pl - (long long)z * g.n[1]);
  } else if (d == 1) {
    y = cd;
    z = (int)(pl / g.n[0]);
    x = (int)(pl - (long long)z * g.n[0]);
  } else {
    z = cd;
    y = (int)(pl / g.n[0]);
    x = (int)(pl - (long long)y * g.n[0]);
  }
  const long long idx = checked(((long long)z * g.n[1] + y) * g.n[0] + x, g.npts, ds, CHK_STATE);
  double* ring = d == 0 ? r0 : (d == 1 ? r1 : r2);
  const long long PS = 2LL * M * g.pes[d];
  const long long spp = checked(sp * plane + pl, PS * plane, ds, CHK_RING);
  for (int v = 0; v < 5; ++v) {
    const double val = U[v * g.npts + idx];
    for (int s = 0, slot = first_slot; s < count; ++s, slot = slot + 1 == g.nlev ? 0 : slot + 1)
      ring[((long long)slot * 5 + v) * PS * plane + spp] = val;
  }
}

// max over points and directions of (|u_d| + c) / dx_d  (FP64 input), as an ordered key.
__global__ void k_wave(Geom g, Phys ph, const double* __restrict__ U, unsigned long long* word) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double s = 0.0;
  if (idx < g.npts) {
    const long long N = g.npts;
    const double r = U[idx], inv = 1.0 / r;
    const double u[3] = {U[N + idx] * inv, U[2 * N + idx] * inv, U[3 * N + idx] * inv};
    const double p = ph.eform ? ph.gm1 * U[4 * N + idx]
                              : ph.gm1 * (U[4 * N + idx] - 0.5 * r * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
    const double c = sqrt(ph.gamma * p * inv);
    for (int d = 0; d < 3; ++d) s = fmax(s, (fabs(u[d]) + c) * g.inv_dx[d]);
  }
  for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  if ((threadIdx.x & 31) == 0) atomicMax((long long*)word, ordered_key(s));
}

// Reset the max/min keys; the health word only when asked (it stays sticky
// across the steps of one at_dns_step call).
__global__ void k_reset_words(unsigned long long* w, int health_too) {
  w[0] = (unsigned long long)LLONG_MIN;
  w[1] = (unsigned long long)LLONG_MAX;
  w[2] = (unsigned long long)LLONG_MAX;
  if (health_too) w[3] = 0ULL;
}

// Fixed-order sum of the block partials: block s sums statistic s.
__global__ void k_stats_final(const double* __restrict__ partial, long long nb, double* sums) {
  __shared__ double sh[256];
  const int s = blockIdx.x;
  double acc = 0.0;
  for (long long b = threadIdx.x; b < nb; b += blockDim.x) acc += partial[b * kNumStat + s];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[s] = sh[0];
}

// Ornstein-Uhlenbeck forcing coefficients on the half set of modes:
// f^0 = amp P(xi^0), f^s = a f^{s-1} + b P(xi^s), b = amp sqrt(1 - a^2),
// xi from Box-Muller on Philox4x32-10 words 0, 1 of counter (s, m, c, 0x464F);
// P removes the component along the wavevector.  One thread per mode runs the
// recursion from step `from` to step `to` (from = 0 starts it).
__global__ void k_force_advance(const Mode3* __restrict__ modes, int nmodes, double2* fhat, long long from,
                                long long to, const DevState* ds, double a, double b, double amp, uint32_t k0,
                                uint32_t k1) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nmodes) return;
  if (ds) from = to = ds->n;   // advance to the current step only
  const Mode3 md = modes[m];
  const double kv[3] = {(double)md.kx, (double)md.ky, (double)md.kz};
  const double k2 = kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2];
  double fr[3], fi[3];
  for (int c = 0; c < 3; ++c) { fr[c] = fhat[m * 3 + c].x; fi[c] = fhat[m * 3 + c].y; }
  for (long long s = from; s <= to; ++s) {
    double xr[3], xi[3];
    for (int c = 0; c < 3; ++c) {
      const uint4 w = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)m, (uint32_t)c, kForceTag), k0, k1);
      const double u1 = ((double)w.x + 0.5) * 2.3283064365386963e-10;   // 2^-32
      const double u2 = ((double)w.y + 0.5) * 2.3283064365386963e-10;
      const double r = sqrt(-2.0 * log(u1));
      double sn, cs;
      sincos(2.0 * M_PI * u2, &sn, &cs);
      xr[c] = r * cs;
      xi[c] = r * sn;
    }
    const double kr = (kv[0] * xr[0] + kv[1] * xr[1] + kv[2] * xr[2]) / k2;
    const double ki = (kv[0] * xi[0] + kv[1] * xi[1] + kv[2] * xi[2]) / k2;
    for (int c = 0; c < 3; ++c) {
      const double pr = xr[c] - kv[c] * kr, pi = xi[c] - kv[c] * ki;
      if (s == 0) { fr[c] = amp * pr; fi[c] = amp * pi; }
      else { fr[c] = a * fr[c] + b * pr; fi[c] = a * fi[c] + b * pi; }
    }
  }
  for (int c = 0; c < 3; ++c) fhat[m * 3 + c] = make_double2(fr[c], fi[c]);
}

// Line sums B[kx][c](y, z) = sum over modes with this kx of
// 2 f_hat[m][c] exp(i (ky y dy + kz z dz)), so that at a point
// f_c = sum_kx Re(B[kx][c] exp(i kx x dx)).
template <typename S>
__global__ void k_force_lines(Geom g, const Mode3* __restrict__ modes, int nmodes, const double2* __restrict__ fhat,
                              int K, vec2_t<S>* B) {
  const long long ln = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long lines = (long long)g.n[2] * g.n[1];
  if (ln >= lines) return;
  const int z = (int)(ln / g.n[1]), y = (int)(ln - (long long)z * g.n[1]);
  const double dy = 2.0 * M_PI / g.n[1], dz = 2.0 * M_PI / g.n[2];
  double br[kMaxKf + 1][3], bi[kMaxKf + 1][3];
  for (int kx = 0; kx <= K; ++kx)
    for (int c = 0; c < 3; ++c) br[kx][c] = bi[kx][c] = 0.0;
  for (int m = 0; m < nmodes; ++m) {
    const Mode3 md = modes[m];
    double sn, cs;
    sincos(md.ky * y * dy + md.kz * z * dz, &sn, &cs);
    for (int c = 0; c < 3; ++c) {
      const double2 f = fhat[m * 3 + c];
      br[md.kx][c] += 2.0 * (f.x * cs - f.y * sn);
      bi[md.kx][c] += 2.0 * (f.x * sn + f.y * cs);
    }
  }
  for (int kx = 0; kx <= K; ++kx)
    for (int c = 0; c < 3; ++c) {
      vec2_t<S> v;
      v.x = (S)br[kx][c];
      v.y = (S)bi[kx][c];
      B[((long long)kx * 3 + c) * lines + ln] = v;
    }
}

template <typename S>
__global__ void k_force_xtab(int n0, int K, vec2_t<S>* X) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (K + 1) * n0) return;
  const int kx = i / n0, x = i - kx * n0;
  double sn, cs;
  sincos(kx * x * (2.0 * M_PI / n0), &sn, &cs);
  vec2_t<S> v;
  v.x = (S)cs;
  v.y = (S)sn;
  X[i] = v;
}

inline unsigned nblk(long long n, int b = kBlock) { return (unsigned)((n + b - 1) / b); }

const char* const kKernelNames[] = {"delay_map", "prim", "ghost", "grad", "force_lines",
                                    "main", "stats_final", "force_advance"};
enum { KD_DELAY, KD_PRIM, KD_GHOST, KD_GRAD, KD_FLINES, KD_MAIN, KD_STATS, KD_FADV, KD_COUNT };

// Event pair around one launch when profiling is on.
struct Timed {
  at_dns* h;
  int kind;
  cudaEvent_t b = nullptr;
  Timed(at_dns* h_, int k) : h(h_), kind(k) {
    if (!h->prof) return;
    cudaEvent_t a;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, h->st);
    h->recs.push_back({kind, a, b});
  }
  ~Timed() {
    if (h->prof && b) cudaEventRecord(b, h->st);
  }
};

int fail(at_dns* h, int code, const std::string& msg);

// Bounds-checked builds: report (and clear) the index checks that failed in
// the handle's kernels since the last report; ordinary builds: nothing.
int report_checks(at_dns* h) {
#ifdef AT_DNS_CHECKS
  unsigned long long c = 0;
  if (cudaMemcpyAsync(&c, &h->ds->check, sizeof(c), cudaMemcpyDeviceToHost, h->st) != cudaSuccess ||
      cudaStreamSynchronize(h->st) != cudaSuccess)
    return fail(h, AT_DNS_E_CUDA, "cannot read the index checks");
  if (c) {
    cudaMemsetAsync(&h->ds->check, 0, sizeof(c), h->st);
    return fail(h, AT_DNS_E_BOUNDS, "index checks failed in the kernels (bounds-checked build), classes " +
                                        std::to_string(c));
  }
#else
  (void)h;
#endif
  return AT_DNS_OK;
}

int fail(at_dns* h, int code, const std::string& msg) {
  h->err = msg;
  return code;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(h, AT_DNS_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

int dev_alloc(at_dns* h, void** p, size_t bytes) {
  if (bytes == 0) { *p = nullptr; return AT_DNS_OK; }
  if (h->pool) {   // bump allocation from the caller's region, 256-byte aligned
    const size_t at = (h->pool_used + 255) & ~(size_t)255;
    if (at + bytes > h->pool_size) {
      *p = nullptr;
      return fail(h, AT_DNS_E_OOM, "device pool of " + std::to_string(h->pool_size) + " bytes is too small (needs " +
                                       std::to_string(at + bytes) + " so far)");
    }
    *p = h->pool + at;
    h->pool_used = at + bytes;
    h->bytes += bytes;
    return AT_DNS_OK;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    (void)cudaGetLastError();
    return fail(h, AT_DNS_E_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
  }
  h->bytes += bytes;
  return AT_DNS_OK;
}

// FP64 staging buffer for host transfers, allocated on first use (a caller
// that only passes device pointers never pays its 40 bytes per point).
int get_stage(at_dns* h) {
  if (h->stage) return AT_DNS_OK;
  return dev_alloc(h, (void**)&h->stage, 5 * (size_t)h->g.npts * sizeof(double));
}

double key_to_double(unsigned long long k) {
  long long b = (long long)k;
  b ^= (b >> 63) & 0x7FFFFFFFFFFFFFFFLL;
  double v;
  std::memcpy(&v, &b, 8);
  return v;
}

// Decode an order-preserving key of a float (FP32 form) written as int64.
double fkey_to_double(unsigned long long k) {
  int b = (int)(long long)k;
  b ^= (b >> 31) & 0x7FFFFFFF;
  float v;
  std::memcpy(&v, &b, 4);
  return (double)v;
}

std::vector<Mode3> forcing_modes(double kf) {
  std::vector<Mode3> out;
  const int K = (int)std::floor(kf);
  for (int kz = -K; kz <= K; ++kz)
    for (int ky = -K; ky <= K; ++ky)
      for (int kx = -K; kx <= K; ++kx) {
        const int k2 = kx * kx + ky * ky + kz * kz;
        if (k2 == 0 || k2 > kf * kf + 1e-12) continue;
        if (kx > 0 || (kx == 0 && ky > 0) || (kx == 0 && ky == 0 && kz > 0)) out.push_back({kx, ky, kz});
      }
  return out;
}

// The x-face slabs of the current FP32 state (and its low words) into the
// staging buffer the ghost kernel reads: slab sp = 2M pe + t (t < M: local t,
// t >= M: local nl - 2M + t), plane index z n1 + y.
template <typename S>
__global__ void k_xstage_fill(Geom g, const S* __restrict__ U, const S* __restrict__ Ulo, S* xst, long long half) {
  const long long P2 = 2LL * g.M * g.pes[0], cnt = P2 * g.plane[0];
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= cnt) return;
  const int sp = (int)(j / g.plane[0]);
  const long long pl = j - (long long)sp * g.plane[0];
  const int pe = sp / (2 * g.M), t = sp - pe * 2 * g.M;
  const int x = pe * g.nl[0] + (t < g.M ? t : g.nl[0] - 2 * g.M + t);
  const long long src = pl * g.n[0] + x;   // pl = z n1 + y
  for (int v = 0; v < 5; ++v) {
    xst[v * cnt + j] = U[v * g.npts + src];
    if (half) xst[half + v * cnt + j] = Ulo ? Ulo[v * g.npts + src] : S(0);
  }
}

// The PE-boundary slabs of an FP64 level on the device into ring slot `slot`.
int ring_store(at_dns* h, const double* field, int first_slot, int count) {
  long long cnt[3];
  for (int d = 0; d < 3; ++d) cnt[d] = h->g.pes[d] > 1 ? 2LL * h->g.M * h->g.pes[d] * h->g.plane[d] : 0;
  const long long total = cnt[0] + cnt[1] + cnt[2];
  if (!total) return AT_DNS_OK;
  k_ring_store<<<nblk(total), kBlock, 0, h->st>>>(h->g, field, (double*)h->ring[0], (double*)h->ring[1],
                                                  (double*)h->ring[2], cnt[0], cnt[1], cnt[2], first_slot, count,
                                                  h->ds);
  CK(cudaGetLastError());
  return AT_DNS_OK;
}

// ---------------------------------------------------------------------------
// typed operations
template <typename S>
struct Ops {
  static S* U(at_dns* h, int i) { return (S*)h->U[i]; }

  // Upload an FP64 level into dst (S); *dev_src receives the FP64 copy of it
  // on the device (the caller's buffer, or the staging buffer).
  static int upload_field(at_dns* h, const double* src, int where, S* dst, const double** dev_src) {
    const long long cnt = 5 * h->g.npts;
    const double* dsrc = src;
    if (where == AT_DNS_HOST && sizeof(S) == sizeof(double)) {
      // FP64: straight into the state (no staging buffer, no device copy)
      CK(cudaMemcpyAsync(dst, src, cnt * sizeof(double), cudaMemcpyHostToDevice, h->st));
      *dev_src = (const double*)dst;
      return AT_DNS_OK;
    }
    if (where == AT_DNS_HOST) {
      int rc;
      if ((rc = get_stage(h))) return rc;
      CK(cudaMemcpyAsync(h->stage, src, cnt * sizeof(double), cudaMemcpyHostToDevice, h->st));
      dsrc = h->stage;
    }
    *dev_src = dsrc;
    if (sizeof(S) == sizeof(double)) {
      if ((const void*)dsrc != (const void*)dst)
        CK(cudaMemcpyAsync(dst, dsrc, cnt * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    } else if (h->comp) {
      k_split_double<<<nblk(cnt), kBlock, 0, h->st>>>(dsrc, (float*)dst, (float*)h->Ulo[h->cur], cnt);
      CK(cudaGetLastError());
    } else {
      k_from_double<S><<<nblk(cnt), kBlock, 0, h->st>>>(dsrc, dst, cnt);
      CK(cudaGetLastError());
    }
    return AT_DNS_OK;
  }


  static int download(at_dns* h, double* out, int where) {
    const long long cnt = 5 * h->g.npts;
    if (where == AT_DNS_HOST && sizeof(S) == sizeof(double)) {
      // FP64: straight from the state (no staging buffer, no device copy)
      CK(cudaMemcpyAsync(out, U(h, h->cur), cnt * sizeof(double), cudaMemcpyDeviceToHost, h->st));
      CK(cudaStreamSynchronize(h->st));
      return AT_DNS_OK;
    }
    if (where == AT_DNS_HOST) {
      int rc;
      if ((rc = get_stage(h))) return rc;
    }
    double* dst = where == AT_DNS_DEVICE ? out : h->stage;
    if (sizeof(S) == sizeof(double)) {
      CK(cudaMemcpyAsync(dst, U(h, h->cur), cnt * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    } else if (h->comp) {
      k_join_double<<<nblk(cnt), kBlock, 0, h->st>>>((const float*)U(h, h->cur), (const float*)h->Ulo[h->cur], dst,
                                                    cnt);
      CK(cudaGetLastError());
    } else {
      k_to_double<S><<<nblk(cnt), kBlock, 0, h->st>>>(U(h, h->cur), dst, cnt);
      CK(cudaGetLastError());
    }
    if (where == AT_DNS_HOST) {
      CK(cudaMemcpyAsync(out, h->stage, cnt * sizeof(double), cudaMemcpyDeviceToHost, h->st));
      CK(cudaStreamSynchronize(h->st));
    }
    return AT_DNS_OK;
  }

  // Queue one RHS evaluation at the device level n on stream `st`: update
  // (a step, advancing the device step state) or write R to Rout.  Touches no
  // host-side state, so it can be captured into a graph.
  //
  // rkstage >= 0: that stage of the low-storage RK3 (Williamson 1980; the
  // step counter advances after stage 2).
  static int launch_step(at_dns* h, int mode, bool update, double* Rout, bool stats, bool reset_health,
                         cudaStream_t st, int rkstage = -1) {
    const Geom& g = h->g;
    const int P = g.pes[0] * g.pes[1] * g.pes[2];
    const uint64_t seed = h->cfg.seed;
    {
      Timed t(h, KD_DELAY);
      k_delay_map<<<nblk(P * 6), kBlock, 0, st>>>(h->dmap, P, 0, h->ds, mode, h->cfg.max_delay, g.M + 1,
                                                 h->cfg.comm_period, (uint32_t)seed, (uint32_t)(seed >> 32));
    }
    CK(cudaGetLastError());
    const S* U0 = U(h, 0);
    const S* U1 = U(h, 1);
    const Coef<S> K = make_coef<S>(g, h->ph, h->dt);
    S* GH[3] = {(S*)h->GH[0], (S*)h->GH[1], (S*)h->GH[2]};
    double* ring[3] = {(double*)h->ring[0], (double*)h->ring[1], (double*)h->ring[2]};
    if (!h->fused) { Timed t(h, KD_PRIM); CK(launch_prim<S>(g, K, U0, U1, h->ds, (S*)h->PQ, st)); }
    if (g.pes[0] > 1 || g.pes[1] > 1 || g.pes[2] > 1) {
      Timed t(h, KD_GHOST);
      CK(launch_ghost<S>(g, K, U0, U1, h->comp ? (S*)h->Ulo[0] : nullptr, h->comp ? (S*)h->Ulo[1] : nullptr, h->ds,
                         h->fused ? nullptr : (S*)h->PQ, GH, ring, (const S*)h->xst, h->xst_half, h->dmap, 0, st));
    }
    if (!h->fused) { Timed t(h, KD_GRAD); CK(launch_grad<S>(g, K, (S*)h->PQ, GH, (S*)h->G, st)); }
    if (h->cfg.forcing) {
      const long long lines = (long long)g.n[2] * g.n[1];
      {
        Timed t(h, KD_FLINES);
        k_force_lines<S><<<nblk(lines, 128), 128, 0, st>>>(g, h->modes, h->nmodes, h->fhat, h->fK, (vec2_t<S>*)h->fB);
      }
      CK(cudaGetLastError());
    }
    k_reset_words<<<1, 1, 0, st>>>(h->words, reset_health ? 1 : 0);
    CK(cudaGetLastError());
    StepArgs<S> a{};
    a.Ub[0] = U0;
    a.Ub[1] = U1;
    a.Ulob[0] = h->comp ? (S*)h->Ulo[0] : nullptr;
    a.Ulob[1] = h->comp ? (S*)h->Ulo[1] : nullptr;
    a.ds = h->ds;
    a.PQ = (S*)h->PQ;
    a.G = (S*)h->G;
    for (int d = 0; d < 3; ++d) a.GH[d] = GH[d];
    a.xst = (S*)h->xst;
    a.xst_half = h->xst_half;
    a.Rprev = (S*)h->Rprev;
    a.Rout = Rout;
    a.partial = h->partial;
    a.words = h->words;
    a.fB = h->cfg.forcing ? (const vec2_t<S>*)h->fB : nullptr;
    a.fX = (const vec2_t<S>*)h->fX;
    a.fK = h->fK;
    a.dt = h->dt;
    a.do_update = update ? 1 : 0;
    a.do_stats = stats ? 1 : 0;
    if (rkstage >= 0) {
      static const double kA[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
      static const double kB[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};
      a.rk = 1;
      a.rkA = (S)kA[rkstage];
      a.rkB = (S)kB[rkstage];
    }
    if (h->fused) {
      Timed t(h, KD_MAIN);
      if constexpr (sizeof(S) == 4) {
        if (h->paired) CK(launch_fused2(g, K, a, h->TX, h->TY, h->ZC, st));
        else CK(launch_fused<S>(g, K, a, h->TX, h->TY, h->ZC, st));
      } else {
        CK(launch_fused<S>(g, K, a, h->TX, h->TY, h->ZC, st));
      }
    } else {
      Timed t(h, KD_MAIN);
      CK(launch_main<S>(g, K, a, st));
    }
    if (stats) {
      { Timed t(h, KD_STATS); k_stats_final<<<kNumStat, 256, 0, st>>>(h->partial, h->nblk_step, h->sums); }
      CK(cudaGetLastError());
    }
    if (update && rkstage >= 0 && rkstage < 2) {
      k_flip_state<<<1, 1, 0, st>>>(h->ds);
      CK(cudaGetLastError());
    } else if (update) {
      k_advance_state<<<1, 1, 0, st>>>(h->ds);
      CK(cudaGetLastError());
      if (h->cfg.forcing) {
        const double a_ = std::exp(-h->dt / h->cfg.f_tcorr);
        const double b_ = h->cfg.f_amp * std::sqrt(1.0 - a_ * a_);
        {
          Timed t(h, KD_FADV);
          k_force_advance<<<nblk(h->nmodes, 64), 64, 0, st>>>(h->modes, h->nmodes, h->fhat, 0, 0, h->ds, a_, b_,
                                                             h->cfg.f_amp, (uint32_t)h->cfg.f_seed,
                                                             (uint32_t)(h->cfg.f_seed >> 32));
        }
        CK(cudaGetLastError());
      }
    }
    return AT_DNS_OK;
  }

  // Host-side bookkeeping of one queued evaluation (mirrors the device state).
  static void account(at_dns* h, bool update, bool stats) {
    if (stats) {
      h->stats_valid = true;
      h->stats_step = h->n;
      h->stats_time = h->t;
    }
    if (update) {
      h->cur = 1 - h->cur;
      h->first = false;
      h->n += 1;
      h->t += h->dt;
    }
  }

  // One time step on `st`: one AB2 update, or the three stages of the
  // low-storage RK3 (statistics of U^n from the first stage).
  static int launch_update(at_dns* h, int mode, bool stats, bool reset_health, cudaStream_t st) {
    if (h->cfg.integrator != AT_DNS_RK3) return launch_step(h, mode, true, nullptr, stats, reset_health, st);
    for (int s = 0; s < 3; ++s) {
      const int rc = launch_step(h, mode, true, nullptr, stats && s == 0, reset_health && s == 0, st, s);
      if (rc) return rc;
    }
    return AT_DNS_OK;
  }

  static int evaluate_step(at_dns* h, int mode, bool stats, bool reset_health) {
    int rc = launch_update(h, mode, stats, reset_health, h->st);
    if (rc) return rc;
    account(h, true, stats);
    return AT_DNS_OK;
  }

  static int evaluate(at_dns* h, int mode, bool update, double* Rout, bool stats, bool reset_health) {
    int rc = launch_step(h, mode, update, Rout, stats, reset_health, h->st);
    if (rc) return rc;
    account(h, update, stats);
    return AT_DNS_OK;
  }

  // Stage the x-face slabs of the current state (FP32 forms with x-faces).
  static int xstage_fill(at_dns* h) {
    if (!h->xst) return AT_DNS_OK;
    const long long cnt = 2LL * h->g.M * h->g.pes[0] * h->g.plane[0];
    k_xstage_fill<S><<<nblk(cnt), kBlock, 0, h->st>>>(h->g, U(h, h->cur), h->comp ? (const S*)h->Ulo[h->cur] : nullptr,
                                                      (S*)h->xst, h->xst_half);
    CK(cudaGetLastError());
    return AT_DNS_OK;
  }

  static int xtab(at_dns* h) {
    const int cnt = (h->fK + 1) * h->g.n[0];
    k_force_xtab<S><<<nblk(cnt), kBlock, 0, h->st>>>(h->g.n[0], h->fK, (vec2_t<S>*)h->fX);
    CK(cudaGetLastError());
    return AT_DNS_OK;
  }
};

// Tile shape of the fused path, or false if it does not apply: the fused
// kernel runs the 4th-order scheme; tiles must not straddle PE faces, hold a
// multiple of 32 points (at most 256) and be at least 8 wide in x and y (the
// one-sided mixed stencils reach 4 points into a PE).
bool pick_fused_shape(const Geom& g, int& TX, int& TY, int& ZC) {
  TX = TY = ZC = 0;
  if (g.M != 2) return false;
  int ext[3];
  for (int d = 0; d < 3; ++d) ext[d] = g.pes[d] > 1 ? g.nl[d] : g.n[d];
  TX = TY = ZC = 0;
  for (int t : {32, 16, 8})
    if (ext[0] % t == 0) { TX = t; break; }
  if (!TX) return false;
  // compiled tile shapes: 32x8, 16x16, 16x8, 8x32, 8x16, 8x8
  for (int t : {32, 16, 8})
    if (TX * t <= 256 && (TX * t) % 32 == 0 && ext[1] % t == 0 && !(TX == 32 && t != 8)) { TY = t; break; }
  if (!TY) return false;
  if (ext[2] <= 64) ZC = ext[2];
  else
    for (int t = 64; t >= 8; --t)
      if (ext[2] % t == 0) { ZC = t; break; }
  return ZC > 0;
}

void drop_graphs(at_dns* h) {
  for (int m = 0; m < 5; ++m)
    if (h->gexec[m]) {
      cudaGraphExecDestroy(h->gexec[m]);
      h->gexec[m] = nullptr;
    }
}

// Capture (once per delay mode and dt) the kernels of one step into a graph.
int step_graph(at_dns* h, int mode, bool stats) {
  if (h->gexec[mode] && h->gdt[mode] == h->dt) return AT_DNS_OK;
  if (h->gexec[mode]) { cudaGraphExecDestroy(h->gexec[mode]); h->gexec[mode] = nullptr; }
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed));
  const int rc = h->p64 ? Ops<double>::launch_update(h, mode, stats, false, h->st)
                        : Ops<float>::launch_update(h, mode, stats, false, h->st);
  const cudaError_t e = cudaStreamEndCapture(h->st, &graph);
  if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
  if (e != cudaSuccess) return fail(h, AT_DNS_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  const cudaError_t e2 = cudaGraphInstantiate(&h->gexec[mode], graph, 0);
  cudaGraphDestroy(graph);
  if (e2 != cudaSuccess) {
    h->gexec[mode] = nullptr;
    return fail(h, AT_DNS_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e2));
  }
  h->gdt[mode] = h->dt;
  return AT_DNS_OK;
}

// Switch the kernel path of a handle (allocating the multi-pass work arrays
// on first use); captured graphs are dropped.
int set_path(at_dns* h, bool fused, int TX, int TY, int ZC, bool paired = false) {
  const Geom& g = h->g;
  if (!fused && !h->PQ) {
    const size_t N = (size_t)g.npts;
    int rc;
    if ((rc = dev_alloc(h, &h->PQ, (size_t)kNumQ * N * h->ssize)) ||
        (rc = dev_alloc(h, &h->G, (size_t)kNumGrad * N * h->ssize))) {
      if (h->PQ && !h->pool) cudaFree(h->PQ);
      h->PQ = nullptr;
      return rc;
    }
  }
  h->fused = fused;
  h->paired = fused && paired;
  h->TX = fused ? TX : 0;
  h->TY = fused ? TY : 0;
  h->ZC = fused ? ZC : 0;
  h->nblk_step = fused ? (long long)(g.n[0] / TX) * (g.n[1] / TY) * (g.n[2] / ZC) : main_blocks(g);
  drop_graphs(h);
  return AT_DNS_OK;
}

struct Candidate { bool fused; int TX, TY, ZC; bool paired; };

// Kernel-path candidates of the autotuner: the multi-pass path and every
// compiled fused tile shape that fits the PE extents, with whole-PE, half and
// quarter z chunks (at least 8 planes).
std::vector<Candidate> tune_candidates(const Geom& g, bool p64) {
  std::vector<Candidate> out;
  out.push_back({false, 0, 0, 0, false});
  if (g.M != 2) return out;   // the fused kernel runs the 4th-order scheme only
  int ext[3];
  for (int d = 0; d < 3; ++d) ext[d] = g.pes[d] > 1 ? g.nl[d] : g.n[d];
  // 32x16 (one CTA of 512 threads per SM) is compiled for the FP32 forms only:
  // its FP64 window does not fit in shared memory
  const int shapes[7][2] = {{32, 8}, {16, 16}, {16, 8}, {8, 32}, {8, 16}, {8, 8}, {32, 16}};
  int zmax = 0;
  if (ext[2] <= 64) zmax = ext[2];
  else
    for (int t = 64; t >= 8; --t)
      if (ext[2] % t == 0) { zmax = t; break; }
  for (auto& sh : shapes) {
    if (ext[0] % sh[0] || ext[1] % sh[1]) continue;
    if (p64 && sh[1] == 16 && sh[0] == 32) continue;
    for (int div : {1, 2, 4}) {
      const int zc = zmax / div;
      if (zc < 8 || zmax % div || ext[2] % zc) continue;
      out.push_back({true, sh[0], sh[1], zc, false});
    }
  }
  // the paired kernel (FP32 forms): two points per thread, packed arithmetic
  const int pshapes[4][2] = {{32, 8}, {32, 16}, {16, 16}, {16, 8}};
  for (auto& sh : pshapes) {
    if (p64 || ext[0] % sh[0] || ext[1] % sh[1]) continue;
    for (int div : {1, 2, 4}) {
      const int zc = zmax / div;
      if (zc < 8 || zmax % div || ext[2] % zc) continue;
      out.push_back({true, sh[0], sh[1], zc, true});
    }
  }
  return out;
}

int force_reset(at_dns* h, long long step) {
  if (!h->cfg.forcing) return AT_DNS_OK;
  const double a_ = std::exp(-h->dt / h->cfg.f_tcorr);
  const double b_ = h->cfg.f_amp * std::sqrt(1.0 - a_ * a_);
  k_force_advance<<<nblk(h->nmodes, 64), 64, 0, h->st>>>(h->modes, h->nmodes, h->fhat, 0, step, nullptr, a_, b_,
                                                        h->cfg.f_amp, (uint32_t)h->cfg.f_seed,
                                                        (uint32_t)(h->cfg.f_seed >> 32));
  CK(cudaGetLastError());
  return AT_DNS_OK;
}

// dt from the CFL number and the state U^step (FP64, device memory).
int set_dt(at_dns* h, const double* U) {
  if (h->cfg.dt > 0) { h->dt = h->cfg.dt; return AT_DNS_OK; }
  k_reset_words<<<1, 1, 0, h->st>>>(h->words, 1);
  CK(cudaGetLastError());
  k_wave<<<nblk(h->g.npts), kBlock, 0, h->st>>>(h->g, h->ph, U, h->words);
  CK(cudaGetLastError());
  unsigned long long w = 0;
  CK(cudaMemcpyAsync(&w, h->words, sizeof(w), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  const double s = key_to_double(w);
  if (!(s > 0) || !std::isfinite(s)) return fail(h, AT_DNS_E_INVALID_ARG, "state has no finite positive wave speed");
  h->dt = h->cfg.cfl / s;
  return AT_DNS_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// checkpoints: the run state of a handle in one self-describing buffer
namespace {

struct CkptHeader {
  char magic[8];                     // "ATDNSCK1"
  int32_t version;
  // the configuration the run state belongs to (compared on load)
  int32_t n[3], pes[3];
  int32_t precision, order, energy_form, visc_law, integrator, forcing, max_delay, comm_period;
  int32_t extrapolate_state;
  uint64_t seed, f_seed;
  double gamma, prandtl, mu0, visc_exp, sutherland_s, kf, f_amp, f_tcorr;
  // the run state's scalars
  int64_t step, stats_step;
  int32_t first, stats_valid;
  double dt, t, stats_time;
  // byte offsets of the sections (-1: absent) and the total size
  int64_t off_U, off_Ulo, off_R, off_ring[3], off_fhat, off_sums, off_words, total;
};

size_t ck_align(size_t x) { return (x + 255) / 256 * 256; }

// Bytes of the FP64 slab ring of direction d (as allocated).
size_t ring_bytes(const at_dns* h, int d) {
  return (size_t)h->g.nlev * 5 * (2ull * h->g.M * h->g.pes[d] * (size_t)h->g.plane[d]) * sizeof(double);
}

// The configuration fields and the section layout of handle h.
void ckpt_layout(const at_dns* h, CkptHeader& H) {
  std::memset(&H, 0, sizeof(H));
  std::memcpy(H.magic, "ATDNSCK1", 8);
  H.version = 1;
  const at_dns_config_t& c = h->cfg;
  for (int d = 0; d < 3; ++d) { H.n[d] = h->g.n[d]; H.pes[d] = h->g.pes[d]; }
  H.precision = c.precision;
  H.order = 2 * h->g.M;
  H.energy_form = c.energy_form;
  H.visc_law = c.visc_law;
  H.integrator = c.integrator;
  H.forcing = c.forcing;
  H.max_delay = c.max_delay;
  H.comm_period = c.comm_period;
  H.extrapolate_state = c.extrapolate_state;
  H.seed = c.seed;
  H.f_seed = c.f_seed;
  H.gamma = c.gamma;
  H.prandtl = c.prandtl;
  H.mu0 = c.mu0;
  H.visc_exp = c.visc_exp;
  H.sutherland_s = c.sutherland_s;
  H.kf = c.kf;
  H.f_amp = c.f_amp;
  H.f_tcorr = c.f_tcorr;
  const size_t field = 5 * (size_t)h->g.npts * h->ssize;
  size_t off = ck_align(sizeof(CkptHeader));
  H.off_U = (int64_t)off;
  off = ck_align(off + field);
  H.off_Ulo = h->comp ? (int64_t)off : -1;
  if (h->comp) off = ck_align(off + field);
  H.off_R = (int64_t)off;
  off = ck_align(off + field);
  for (int d = 0; d < 3; ++d) {
    H.off_ring[d] = h->ring[d] ? (int64_t)off : -1;
    if (h->ring[d]) off = ck_align(off + ring_bytes(h, d));
  }
  H.off_fhat = h->nmodes ? (int64_t)off : -1;
  if (h->nmodes) off = ck_align(off + (size_t)h->nmodes * 3 * sizeof(double2));
  H.off_sums = (int64_t)off;
  off = ck_align(off + kNumStat * sizeof(double));
  H.off_words = (int64_t)off;
  off = ck_align(off + 4 * sizeof(unsigned long long));
  H.total = (int64_t)off;
}

// The first configuration field in which a saved header differs from this
// handle's, or null.
const char* ckpt_mismatch(const CkptHeader& a, const CkptHeader& b) {
  for (int d = 0; d < 3; ++d) {
    if (a.n[d] != b.n[d]) return "grid";
    if (a.pes[d] != b.pes[d]) return "pes";
  }
  if (a.precision != b.precision) return "precision";
  if (a.order != b.order) return "order";
  if (a.energy_form != b.energy_form) return "energy_form";
  if (a.visc_law != b.visc_law) return "visc_law";
  if (a.integrator != b.integrator) return "integrator";
  if (a.forcing != b.forcing) return "forcing";
  if (a.max_delay != b.max_delay) return "max_delay";
  if (a.comm_period != b.comm_period) return "comm_period";
  if (a.extrapolate_state != b.extrapolate_state) return "extrapolate_state";
  if (a.seed != b.seed) return "seed";
  if (a.f_seed != b.f_seed) return "f_seed";
  if (a.gamma != b.gamma || a.prandtl != b.prandtl || a.mu0 != b.mu0 || a.visc_exp != b.visc_exp ||
      a.sutherland_s != b.sutherland_s)
    return "physical constants";
  if (a.kf != b.kf || a.f_amp != b.f_amp || a.f_tcorr != b.f_tcorr) return "forcing constants";
  if (a.total != b.total) return "layout";
  return nullptr;
}

}  // namespace

extern "C" {

int at_dns_checkpoint_size(const at_dns_t* h, int64_t* bytes) {
  if (!h || !bytes) return AT_DNS_E_INVALID_ARG;
  CkptHeader H;
  ckpt_layout(h, H);
  *bytes = H.total;
  return AT_DNS_OK;
}

int at_dns_checkpoint_save(at_dns_t* h, void* buf, int where) {
  NvtxRange nvtx_range("at_dns_checkpoint_save");
  if (!h) return AT_DNS_E_INVALID_ARG;
  h->err.clear();
  if (!buf) return fail(h, AT_DNS_E_INVALID_ARG, "buf is NULL");
  if (where != AT_DNS_HOST && where != AT_DNS_DEVICE) return fail(h, AT_DNS_E_INVALID_ARG, "bad where");
  if (!h->has_state) return fail(h, AT_DNS_E_STATE, "no state set");
  CkptHeader H;
  ckpt_layout(h, H);
  DevState dsv;   // the step counter, start-up flag and state buffer as the device has them
  CK(cudaMemcpyAsync(&dsv, h->ds, sizeof(dsv), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  H.step = dsv.n;
  H.first = dsv.first;
  H.stats_step = h->stats_step;
  H.stats_valid = h->stats_valid ? 1 : 0;
  H.dt = h->dt;
  H.t = h->t;
  H.stats_time = h->stats_time;
  const cudaMemcpyKind kind = where == AT_DNS_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  char* out = (char*)buf;
  const size_t field = 5 * (size_t)h->g.npts * h->ssize;
  CK(cudaMemcpyAsync(out + H.off_U, h->U[dsv.cur], field, kind, h->st));
  if (H.off_Ulo >= 0) CK(cudaMemcpyAsync(out + H.off_Ulo, h->Ulo[dsv.cur], field, kind, h->st));
  CK(cudaMemcpyAsync(out + H.off_R, h->Rprev, field, kind, h->st));
  for (int d = 0; d < 3; ++d)
    if (H.off_ring[d] >= 0) CK(cudaMemcpyAsync(out + H.off_ring[d], h->ring[d], ring_bytes(h, d), kind, h->st));
  if (H.off_fhat >= 0)
    CK(cudaMemcpyAsync(out + H.off_fhat, h->fhat, (size_t)h->nmodes * 3 * sizeof(double2), kind, h->st));
  CK(cudaMemcpyAsync(out + H.off_sums, h->sums, kNumStat * sizeof(double), kind, h->st));
  CK(cudaMemcpyAsync(out + H.off_words, h->words, 4 * sizeof(unsigned long long), kind, h->st));
  if (where == AT_DNS_HOST) std::memcpy(out, &H, sizeof(H));
  else CK(cudaMemcpyAsync(out, &H, sizeof(H), cudaMemcpyHostToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));
  return AT_DNS_OK;
}

int at_dns_checkpoint_load(at_dns_t* h, const void* buf, int where) {
  NvtxRange nvtx_range("at_dns_checkpoint_load");
  if (!h) return AT_DNS_E_INVALID_ARG;
  h->err.clear();
  if (!buf) return fail(h, AT_DNS_E_INVALID_ARG, "buf is NULL");
  if (where != AT_DNS_HOST && where != AT_DNS_DEVICE) return fail(h, AT_DNS_E_INVALID_ARG, "bad where");
  CkptHeader S, H;
  if (where == AT_DNS_HOST) std::memcpy(&S, buf, sizeof(S));
  else CK(cudaMemcpy(&S, buf, sizeof(S), cudaMemcpyDeviceToHost));
  if (std::memcmp(S.magic, "ATDNSCK1", 8) != 0 || S.version != 1)
    return fail(h, AT_DNS_E_INVALID_ARG, "not a checkpoint of this library");
  ckpt_layout(h, H);
  if (const char* what = ckpt_mismatch(S, H))
    return fail(h, AT_DNS_E_INVALID_ARG, std::string("checkpoint of another configuration: ") + what + " differs");
  if (S.step < 0 || !(S.dt > 0)) return fail(h, AT_DNS_E_INVALID_ARG, "checkpoint holds no run state");
  const cudaMemcpyKind kind = where == AT_DNS_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const char* in = (const char*)buf;
  const size_t field = 5 * (size_t)h->g.npts * h->ssize;
  h->cur = 0;
  CK(cudaMemcpyAsync(h->U[0], in + H.off_U, field, kind, h->st));
  if (H.off_Ulo >= 0) CK(cudaMemcpyAsync(h->Ulo[0], in + H.off_Ulo, field, kind, h->st));
  CK(cudaMemcpyAsync(h->Rprev, in + H.off_R, field, kind, h->st));
  for (int d = 0; d < 3; ++d)
    if (H.off_ring[d] >= 0) CK(cudaMemcpyAsync(h->ring[d], in + H.off_ring[d], ring_bytes(h, d), kind, h->st));
  if (H.off_fhat >= 0)
    CK(cudaMemcpyAsync(h->fhat, in + H.off_fhat, (size_t)h->nmodes * 3 * sizeof(double2), kind, h->st));
  CK(cudaMemcpyAsync(h->sums, in + H.off_sums, kNumStat * sizeof(double), kind, h->st));
  CK(cudaMemcpyAsync(h->words, in + H.off_words, 4 * sizeof(unsigned long long), kind, h->st));
  h->n = S.step;
  h->first = S.first != 0;
  h->dt = S.dt;
  h->t = S.t;
  h->stats_step = S.stats_step;
  h->stats_time = S.stats_time;
  h->stats_valid = S.stats_valid != 0;
  h->has_state = true;
  k_set_state<<<1, 1, 0, h->st>>>(h->ds, S.step, S.first, 0);
  CK(cudaGetLastError());
  // the x-face slabs of U^n that the next ghost kernel reads (FP32 forms)
  const int rc = h->p64 ? AT_DNS_OK : Ops<float>::xstage_fill(h);
  if (rc) return rc;
  CK(cudaStreamSynchronize(h->st));
  return AT_DNS_OK;
}

}  // extern "C"

extern "C" {

int at_dns_config_default(at_dns_config_t* c) {
  if (!c) return AT_DNS_E_INVALID_ARG;
  std::memset(c, 0, sizeof(*c));
  for (int d = 0; d < 3; ++d) { c->n[d] = 32; c->pes[d] = 1; }
  c->gamma = 1.4;
  c->prandtl = 0.7;
  c->mu0 = 0.01;
  c->visc_exp = 0.76;
  c->dt = 0.0;
  c->cfl = 0.5;
  c->max_delay = 2;
  c->comm_period = 3;
  c->seed = 0;
  c->forcing = 0;
  c->kf = 2.0;
  c->f_amp = 0.0;
  c->f_tcorr = 1.0;
  c->f_seed = 0;
  c->precision = AT_DNS_P64;
  c->stats_every = 1;
  c->stream = nullptr;
  c->order = 4;
  c->energy_form = AT_DNS_ENERGY_TOTAL;
  c->visc_law = AT_DNS_VISC_POWER;
  c->sutherland_s = 0.368;
  c->integrator = AT_DNS_AB2;
  c->extrapolate_state = 0;
  return AT_DNS_OK;
}

static int create_fail(at_dns* h, int code) {
  g_create_error = h->err;
  at_dns_destroy(h);
  return code;
}

int at_dns_create(const at_dns_config_t* cfg, at_dns_t** out) {
  if (!cfg || !out) { g_create_error = "NULL argument"; return AT_DNS_E_INVALID_ARG; }
  *out = nullptr;
  const at_dns_config_t& c = *cfg;
  std::string bad;
  const int M = c.order == 6 ? 3 : 2;
  if (c.order != 4 && c.order != 6) bad = "order must be 4 or 6";
  for (int d = 0; d < 3 && bad.empty(); ++d) {
    if (c.n[d] < 2 * M + 1 || c.n[d] > 32768) bad = "n[d] must be in [order + 1, 32768]";
    else if (c.pes[d] < 1 || c.n[d] % c.pes[d] != 0) bad = "pes[d] must divide n[d]";
    else if (c.pes[d] > 1 && c.n[d] / c.pes[d] < 2 * M + 1) bad = "n[d]/pes[d] must be >= order + 1 when pes[d] > 1";
  }
  if (bad.empty()) {
    if (!(c.gamma > 1.0)) bad = "gamma must be > 1";
    else if (!(c.prandtl > 0)) bad = "prandtl must be > 0";
    else if (!(c.mu0 >= 0)) bad = "mu0 must be >= 0";
    else if (!std::isfinite(c.gamma) || !std::isfinite(c.prandtl) || !std::isfinite(c.mu0) ||
             !std::isfinite(c.visc_exp))
      bad = "gamma, prandtl, mu0 and visc_exp must be finite";
    else if (c.max_delay < 0 || c.max_delay > 64) bad = "max_delay must be in [0, 64]";
    else if (c.comm_period < 1) bad = "comm_period must be >= 1";
    else if (c.precision != AT_DNS_P64 && c.precision != AT_DNS_P32 && c.precision != AT_DNS_P32C)
      bad = "unknown precision";
    else if (!(c.dt > 0) && !(c.cfl > 0)) bad = "need dt > 0 or cfl > 0";
    else if (c.forcing && (!(c.kf >= 1.0) || c.kf > kMaxKf)) bad = "kf must be in [1, 4]";
    else if (c.forcing && !(c.f_tcorr > 0)) bad = "f_tcorr must be > 0";
    else if (c.stats_every != 0 && c.stats_every != 1) bad = "stats_every must be 0 or 1";
    else if (c.kernel_path < 0 || c.kernel_path > 3) bad = "unknown kernel_path";
    else if (c.kernel_path == AT_DNS_PATH_PAIRED && c.precision == AT_DNS_P64)
      bad = "the paired path runs the FP32 forms only";
    else if (c.energy_form != AT_DNS_ENERGY_TOTAL && c.energy_form != AT_DNS_ENERGY_INTERNAL) bad = "unknown energy_form";
    else if (c.visc_law != AT_DNS_VISC_POWER && c.visc_law != AT_DNS_VISC_SUTHERLAND) bad = "unknown visc_law";
    else if (c.visc_law == AT_DNS_VISC_SUTHERLAND && !(c.sutherland_s > 0)) bad = "sutherland_s must be > 0";
    else if (c.integrator != AT_DNS_AB2 && c.integrator != AT_DNS_RK3) bad = "unknown integrator";
    else if (c.extrapolate_state != 0 && c.extrapolate_state != 1) bad = "extrapolate_state must be 0 or 1";
    else if (c.pool && ((uintptr_t)c.pool & 255)) bad = "pool must be 256-byte aligned";
  }
  if (bad.empty() && (long long)c.n[0] * c.n[1] * c.n[2] >= (1LL << 31)) bad = "grids must hold fewer than 2^31 points";
  if (!bad.empty()) { g_create_error = bad; return AT_DNS_E_INVALID_ARG; }

  at_dns* h = new at_dns();
  h->cfg = c;
  if (c.pool) {
    h->pool = (char*)c.pool;
    h->pool_size = c.pool_bytes;
  }
  h->st = (cudaStream_t)c.stream;
  h->p64 = c.precision == AT_DNS_P64;
  h->comp = c.precision == AT_DNS_P32C;
  h->ssize = h->p64 ? 8 : 4;
  Geom& g = h->g;
  g.npts = 1;
  g.xstate = c.extrapolate_state;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = c.n[d];
    g.pes[d] = c.pes[d];
    g.nl[d] = c.n[d] / c.pes[d];
    g.npts *= c.n[d];
  }
  g.stride[0] = 1;
  g.stride[1] = g.n[0];
  g.stride[2] = (long long)g.n[0] * g.n[1];
  for (int d = 0; d < 3; ++d) g.plane[d] = g.npts / g.n[d];
  set_stencils(g, M);
  g.nlev = c.max_delay + M + 1;   // L + T_l levels
  Phys& ph = h->ph;
  ph.gamma = c.gamma;
  ph.gm1 = c.gamma - 1.0;
  ph.prandtl = c.prandtl;
  ph.eform = c.energy_form;
  ph.vlaw = c.visc_law;
  ph.suth_s = c.sutherland_s;
  ph.mu0 = c.mu0;
  ph.omega = c.visc_exp;
  ph.cp_over_pr = 1.0 / ((c.gamma - 1.0) * c.prandtl);

  const size_t S = h->ssize;
  const size_t N = (size_t)g.npts;
  int rc;
  const bool can_fuse = pick_fused_shape(g, h->TX, h->TY, h->ZC);
  if (c.kernel_path == AT_DNS_PATH_FUSED && !can_fuse) {
    h->err = M != 2 ? "the fused path runs the 4th-order scheme only"
                    : "the fused path needs PE (or grid) extents that are multiples of 8 in x and y";
    return create_fail(h, AT_DNS_E_UNSUPPORTED);
  }
  if (c.kernel_path == AT_DNS_PATH_PAIRED) {
    // the first paired candidate of the tuner's list (largest tile, whole-PE z chunk)
    bool found = false;
    for (const Candidate& cd : tune_candidates(g, h->p64))
      if (cd.paired) { h->TX = cd.TX; h->TY = cd.TY; h->ZC = cd.ZC; found = true; break; }
    if (!found) {
      h->err = M != 2 ? "the paired path runs the 4th-order scheme only"
                      : "the paired path needs PE (or grid) extents that are multiples of 16 in x and 8 in y";
      return create_fail(h, AT_DNS_E_UNSUPPORTED);
    }
    h->paired = true;
  }
  // AUTO takes the faster path on GB300 at the benchmark workload (at_dns_tune
  // can switch): a fused one for the FP32 forms (one pass over U, no work
  // arrays; the paired kernel where its tiles fit), the multi-pass one for
  // FP64 (bound by the FP64 pipe, where the fused path's halo recompute costs
  // more than the work arrays' traffic)
  if (c.kernel_path == AT_DNS_PATH_AUTO && !h->p64 && M == 2) {
    // AUTO for the FP32 forms: the paired fused kernel where its tiles fit
    // (faster than the one-point kernel at the benchmark workload on GB300)
    for (const Candidate& cd : tune_candidates(g, h->p64))
      if (cd.paired) { h->TX = cd.TX; h->TY = cd.TY; h->ZC = cd.ZC; h->paired = true; break; }
  }
  h->fused = h->paired ||
             (can_fuse && (c.kernel_path == AT_DNS_PATH_FUSED || (c.kernel_path == AT_DNS_PATH_AUTO && !h->p64)));
  if (!h->fused) h->TX = h->TY = h->ZC = 0;
  h->nblk_step = h->fused ? (long long)(g.n[0] / h->TX) * (g.n[1] / h->TY) * (g.n[2] / h->ZC) : main_blocks(g);
  if ((rc = dev_alloc(h, &h->U[0], 5 * N * S)) || (rc = dev_alloc(h, &h->U[1], 5 * N * S)) ||
      (rc = dev_alloc(h, &h->Rprev, 5 * N * S)))
    return create_fail(h, rc);
  if (!h->fused) {
    if ((rc = dev_alloc(h, &h->PQ, (size_t)kNumQ * N * S)) || (rc = dev_alloc(h, &h->G, (size_t)kNumGrad * N * S)))
      return create_fail(h, rc);
  }
  if (h->comp) {
    if ((rc = dev_alloc(h, &h->Ulo[0], 5 * N * S)) || (rc = dev_alloc(h, &h->Ulo[1], 5 * N * S)))
      return create_fail(h, rc);
  }
  for (int d = 0; d < 3; ++d) {
    if (g.pes[d] == 1) continue;
    const size_t gpts = 2ull * M * g.pes[d] * (size_t)g.plane[d];
    if ((rc = dev_alloc(h, &h->GH[d], (size_t)kNumGhostQ * gpts * S)) ||
        (rc = dev_alloc(h, &h->ring[d], (size_t)g.nlev * 5 * gpts * sizeof(double))))
      return create_fail(h, rc);
    if (d == 0 && !h->p64) {
      // x-face slabs staged by the step kernels for the next ghost kernel
      const size_t halves = h->comp ? 2 : 1;
      if ((rc = dev_alloc(h, &h->xst, halves * 5 * gpts * S))) return create_fail(h, rc);
      h->xst_half = h->comp ? (long long)(5 * gpts) : 0;
    }
  }
  const int P = g.pes[0] * g.pes[1] * g.pes[2];
  if ((rc = dev_alloc(h, (void**)&h->ds, sizeof(DevState))) || (rc = dev_alloc(h, (void**)&h->dmap, (size_t)P * 6)) ||
      (rc = dev_alloc(h, (void**)&h->partial, (size_t)main_blocks(g) * kNumStat * sizeof(double))) ||
      (rc = dev_alloc(h, (void**)&h->sums, kNumStat * sizeof(double))) ||
      (rc = dev_alloc(h, (void**)&h->words, 4 * sizeof(unsigned long long))))
    return create_fail(h, rc);
  if (cudaMemsetAsync(h->ds, 0, sizeof(DevState), h->st) != cudaSuccess) {
    (void)cudaGetLastError();
    return create_fail(h, AT_DNS_E_CUDA);
  }
  // forcing tables (allocated even without forcing: the x-table is tiny)
  std::vector<Mode3> modes = forcing_modes(c.forcing ? c.kf : 1.0);
  h->nmodes = c.forcing ? (int)modes.size() : 0;
  h->fK = c.forcing ? (int)std::floor(c.kf) : 0;
  const size_t lines = (size_t)g.n[2] * g.n[1];
  const size_t v2 = 2 * S;
  if ((rc = dev_alloc(h, &h->fX, (size_t)(h->fK + 1) * g.n[0] * v2))) return create_fail(h, rc);
  if (c.forcing) {
    if ((rc = dev_alloc(h, (void**)&h->modes, modes.size() * sizeof(Mode3))) ||
        (rc = dev_alloc(h, (void**)&h->fhat, modes.size() * 3 * sizeof(double2))) ||
        (rc = dev_alloc(h, &h->fB, (size_t)(h->fK + 1) * 3 * lines * v2)))
      return create_fail(h, rc);
    if (cudaMemcpy(h->modes, modes.data(), modes.size() * sizeof(Mode3), cudaMemcpyHostToDevice) != cudaSuccess)
      { h->err = "copy of forcing modes failed"; return create_fail(h, AT_DNS_E_CUDA); }
  }
  rc = h->p64 ? Ops<double>::xtab(h) : Ops<float>::xtab(h);
  if (rc) return create_fail(h, rc);
  if (cudaStreamSynchronize(h->st) != cudaSuccess) { h->err = "initialisation failed"; return create_fail(h, AT_DNS_E_CUDA); }
  *out = h;
  return AT_DNS_OK;
}

int at_dns_set_history(at_dns_t* h, const double* levels, int32_t nlevels, int64_t step, int where) {
  NvtxRange nvtx_range("at_dns_set_history");
  if (!h) return AT_DNS_E_INVALID_ARG;
  h->err.clear();
  if (!levels) return fail(h, AT_DNS_E_INVALID_ARG, "levels is NULL");
  if (where != AT_DNS_HOST && where != AT_DNS_DEVICE) return fail(h, AT_DNS_E_INVALID_ARG, "bad where");
  if (nlevels < 1 || nlevels > h->g.nlev) return fail(h, AT_DNS_E_INVALID_ARG, "nlevels must be in [1, L + T_l]");
  if (step < 0) return fail(h, AT_DNS_E_INVALID_ARG, "step must be >= 0");
  const long long cnt = 5 * h->g.npts;
  int rc;
  // older levels first so that U[cur] ends up holding U^step; each given level
  // is uploaded once and stored into its ring slot (the oldest one also into
  // the slots of the older levels that were not given: levels last .. l sit
  // in consecutive slots from that of level `last`)
  const double* dev_level0 = nullptr;   // U^step in FP64 on the device
  for (int l = nlevels - 1; l >= 0; --l) {
    const double* lv = levels + (size_t)l * cnt;
    const int last = l == nlevels - 1 ? h->g.nlev - 1 : l;
    const double* dev_lv = nullptr;   // the level in FP64 on the device
    if (h->p64) {
      if ((rc = Ops<double>::upload_field(h, lv, where, Ops<double>::U(h, h->cur), &dev_lv))) return rc;
    } else {
      if ((rc = Ops<float>::upload_field(h, lv, where, Ops<float>::U(h, h->cur), &dev_lv))) return rc;
    }
    const int first_slot = (int)(((step - last) % h->g.nlev + h->g.nlev) % h->g.nlev);
    if ((rc = ring_store(h, dev_lv, first_slot, last - l + 1))) return rc;
    if (l == 0) dev_level0 = dev_lv;
  }
  // the x-face slabs of U^step for the first ghost kernel (FP32 forms)
  rc = h->p64 ? AT_DNS_OK : Ops<float>::xstage_fill(h);
  if (rc) return rc;
  // U^step in FP64 on the device for the CFL reduction: the caller's level 0,
  // the state (FP64 form) or the staging buffer the host path filled with it
  if (!(h->has_state && h->dt > 0) || step == 0) {
    if ((rc = set_dt(h, dev_level0))) return rc;
  }
  h->n = step;
  h->t = step * h->dt;
  h->first = true;
  h->has_state = true;
  k_set_state<<<1, 1, 0, h->st>>>(h->ds, step, 1, h->cur);
  CK(cudaGetLastError());
  h->stats_valid = false;
  if ((rc = force_reset(h, step))) return rc;
  CK(cudaStreamSynchronize(h->st));
  return report_checks(h);
}

int at_dns_set_state(at_dns_t* h, const double* u, int where) {
  if (!h) return AT_DNS_E_INVALID_ARG;
  h->has_state = false;
  return at_dns_set_history(h, u, 1, 0, where);
}

int at_dns_get_state(at_dns_t* h, double* u_out, int where) {
  NvtxRange nvtx_range("at_dns_get_state");
  if (!h) return AT_DNS_E_INVALID_ARG;
  h->err.clear();
  if (!u_out) return fail(h, AT_DNS_E_INVALID_ARG, "u_out is NULL");
  if (where != AT_DNS_HOST && where != AT_DNS_DEVICE) return fail(h, AT_DNS_E_INVALID_ARG, "bad where");
  if (!h->has_state) return fail(h, AT_DNS_E_STATE, "no state set");
  return h->p64 ? Ops<double>::download(h, u_out, where) : Ops<float>::download(h, u_out, where);
}

static int check_mode(at_dns* h, int mode) {
  if (mode != AT_DNS_SYNC && mode != AT_DNS_PERIODIC && mode != AT_DNS_RANDOM && mode != AT_DNS_FIXED &&
      mode != AT_DNS_ORDERED)
    return fail(h, AT_DNS_E_INVALID_ARG, "unknown delay mode");
  if (h->cfg.integrator == AT_DNS_RK3 && mode != AT_DNS_SYNC)
    return fail(h, AT_DNS_E_UNSUPPORTED, "the RK3 integrator runs synchronous steps only");
  if (mode == AT_DNS_PERIODIC && h->cfg.comm_period - 1 > h->cfg.max_delay)
    return fail(h, AT_DNS_E_INVALID_ARG, "periodic delays need comm_period - 1 <= max_delay");
  return AT_DNS_OK;
}

int at_dns_rhs(at_dns_t* h, int32_t delay_mode, double* rhs_out, int where) {
  NvtxRange nvtx_range("at_dns_rhs");
  if (!h) return AT_DNS_E_INVALID_ARG;
  h->err.clear();
  int rc;
  if ((rc = check_mode(h, delay_mode))) return rc;
  if (!rhs_out) return fail(h, AT_DNS_E_INVALID_ARG, "rhs_out is NULL");
  if (where != AT_DNS_HOST && where != AT_DNS_DEVICE) return fail(h, AT_DNS_E_INVALID_ARG, "bad where");
  if (!h->has_state) return fail(h, AT_DNS_E_STATE, "no state set");
  if (where == AT_DNS_HOST && (rc = get_stage(h))) return rc;
  double* dst = where == AT_DNS_DEVICE ? rhs_out : h->stage;
  rc = h->p64 ? Ops<double>::evaluate(h, delay_mode, false, dst, true, true)
              : Ops<float>::evaluate(h, delay_mode, false, dst, true, true);
  if (rc) return rc;
  if (where == AT_DNS_HOST)
    CK(cudaMemcpyAsync(rhs_out, h->stage, 5 * h->g.npts * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return report_checks(h);
}

int at_dns_step(at_dns_t* h, int32_t nsteps, int32_t delay_mode) {
  NvtxRange nvtx_range("at_dns_step");
  if (!h) return AT_DNS_E_INVALID_ARG;
  h->err.clear();
  int rc;
  if ((rc = check_mode(h, delay_mode))) return rc;
  if (nsteps < 0) return fail(h, AT_DNS_E_INVALID_ARG, "nsteps must be >= 0");
  if (!h->has_state) return fail(h, AT_DNS_E_STATE, "no state set");
  const bool stats = h->cfg.stats_every == 1;
  // replay a captured one-step graph when the handle runs on its own stream
  // (the legacy default stream cannot be captured) and no per-launch event
  // timing is requested; otherwise launch kernel by kernel
  const bool graph = h->use_graphs && h->st != nullptr && !h->prof && nsteps > 1;
  if (graph) {
    if ((rc = step_graph(h, delay_mode, stats))) return rc;
    k_reset_words<<<1, 1, 0, h->st>>>(h->words, 1);
    CK(cudaGetLastError());
    for (int s = 0; s < nsteps; ++s) {
      CK(cudaGraphLaunch(h->gexec[delay_mode], h->st));
      if (h->p64) Ops<double>::account(h, true, stats); else Ops<float>::account(h, true, stats);
    }
  } else {
    for (int s = 0; s < nsteps; ++s) {
      rc = h->p64 ? Ops<double>::evaluate_step(h, delay_mode, stats, s == 0)
                  : Ops<float>::evaluate_step(h, delay_mode, stats, s == 0);
      if (rc) return rc;
    }
  }
  if (!stats) h->stats_valid = false;
  if ((rc = report_checks(h))) return rc;
  if (nsteps > 0) {
    unsigned long long w = 0;
    CK(cudaMemcpyAsync(&w, h->words + 3, sizeof(w), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (w) return fail(h, AT_DNS_E_UNSTABLE, "non-finite value, rho <= 0 or p <= 0 in the last step (flags " +
                                                 std::to_string(w) + ")");
  }
  return AT_DNS_OK;
}

int at_dns_stats(at_dns_t* h, at_dns_stats_t* out) {
  NvtxRange nvtx_range("at_dns_stats");
  if (!h) return AT_DNS_E_INVALID_ARG;
  h->err.clear();
  if (!out) return fail(h, AT_DNS_E_INVALID_ARG, "out is NULL");
  if (!h->has_state) return fail(h, AT_DNS_E_STATE, "no state set");
  int rc;
  if (!h->stats_valid) {
    rc = h->p64 ? Ops<double>::evaluate(h, AT_DNS_SYNC, false, nullptr, true, true)
                : Ops<float>::evaluate(h, AT_DNS_SYNC, false, nullptr, true, true);
    if (rc) return rc;
  }
  double s[kNumStat];
  unsigned long long w[4];
  CK(cudaMemcpyAsync(s, h->sums, sizeof(s), cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(w, h->words, sizeof(w), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  const double N = (double)h->g.npts;
  std::memset(out, 0, sizeof(*out));
  out->step = h->stats_step;
  out->time = h->stats_time;
  out->dt = h->dt;
  out->mass = s[ST_RHO] / N;
  out->mom[0] = s[ST_M0] / N;
  out->mom[1] = s[ST_M1] / N;
  out->mom[2] = s[ST_M2] / N;
  out->energy = s[ST_E] / N;
  out->tke = s[ST_KE] / N;
  out->dissipation = s[ST_SIGS] / N;
  out->grad_m2 = s[ST_G2] / (3 * N);
  out->grad_m3 = s[ST_G3] / (3 * N);
  out->grad_m4 = s[ST_G4] / (3 * N);
  out->skewness = out->grad_m3 / std::pow(out->grad_m2, 1.5);
  out->flatness = out->grad_m4 / (out->grad_m2 * out->grad_m2);
  out->enstrophy = s[ST_ENST] / N;
  out->pressure_dilatation = s[ST_PTHETA] / N;
  out->forcing_power = s[ST_FPOW] / N;
  out->urms = std::sqrt(s[ST_U2] / N / 3.0);
  out->mach_t = std::sqrt(s[ST_U2] / N) / (s[ST_C] / N);
  double (*dec)(unsigned long long) = h->p64 ? key_to_double : fkey_to_double;
  out->max_wave_speed = dec(w[0]);
  out->min_rho = dec(w[1]);
  out->min_p = dec(w[2]);
  out->unstable = (int32_t)w[3];
  return AT_DNS_OK;
}

int at_dns_get_delay_map(at_dns_t* h, int64_t step, int32_t mode, uint8_t* out) {
  if (!h) return AT_DNS_E_INVALID_ARG;
  h->err.clear();
  int rc;
  if ((rc = check_mode(h, mode))) return rc;
  if (!out) return fail(h, AT_DNS_E_INVALID_ARG, "out is NULL");
  if (step < 0) return fail(h, AT_DNS_E_INVALID_ARG, "step must be >= 0");
  const Geom& g = h->g;
  const int P = g.pes[0] * g.pes[1] * g.pes[2];
  // the step's own map buffer: every step rebuilds it before use
  k_delay_map<<<nblk(P * 6), kBlock, 0, h->st>>>(h->dmap, P, step, nullptr, mode, h->cfg.max_delay, g.M + 1,
                                                h->cfg.comm_period, (uint32_t)h->cfg.seed,
                                                (uint32_t)(h->cfg.seed >> 32));
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, h->dmap, (size_t)P * 6, cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return fail(h, AT_DNS_E_CUDA, std::string("delay map: ") + cudaGetErrorString(e));
  return AT_DNS_OK;
}

int at_dns_get_info(at_dns_t* h, at_dns_info_t* out) {
  if (!h || !out) return AT_DNS_E_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->step = h->n;
  out->time = h->t;
  out->dt = h->dt;
  out->n_levels = h->g.nlev;
  long long nt = 1, ni = 1;
  for (int d = 0; d < 3; ++d) { nt *= h->g.nl[d]; ni *= (h->g.nl[d] - 2 * h->g.M); }
  out->boundary_fraction = (double)(nt - ni) / (double)nt;
  out->device_bytes = h->bytes;
  const bool ghost = h->g.pes[0] > 1 || h->g.pes[1] > 1 || h->g.pes[2] > 1;
  // delay map, word reset, main kernel, step-state advance (+ derived fields
  // and gradients on the multi-pass path)
  out->kernels_per_step = (h->fused ? 4 : 6) + (ghost ? 1 : 0) + (h->cfg.stats_every ? 1 : 0) +
                          (h->cfg.forcing ? 2 : 0);
  out->kernel_path = h->paired ? AT_DNS_PATH_PAIRED : (h->fused ? AT_DNS_PATH_FUSED : AT_DNS_PATH_MULTIPASS);
  out->tile[0] = h->TX;
  out->tile[1] = h->TY;
  out->tile[2] = h->ZC;
  out->order = 2 * h->g.M;
  return AT_DNS_OK;
}

static void clear_recs(at_dns* h) {
  for (auto& r : h->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  h->recs.clear();
}

int at_dns_profile(at_dns_t* h, int32_t enable) {
  if (!h) return AT_DNS_E_INVALID_ARG;
  if (enable) {
    cudaStreamSynchronize(h->st);
    clear_recs(h);
  }
  h->prof = enable != 0;
  return AT_DNS_OK;
}

int at_dns_kernel_times(at_dns_t* h, at_dns_kernel_time_t* out, int32_t max, int32_t* count) {
  if (!h || !out || !count || max < 0) return AT_DNS_E_INVALID_ARG;
  h->err.clear();
  CK(cudaStreamSynchronize(h->st));
  long long n[KD_COUNT] = {0};
  double ms[KD_COUNT] = {0};
  for (auto& r : h->recs) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, r.a, r.b));
    n[r.kind] += 1;
    ms[r.kind] += t;
  }
  int c = 0;
  for (int k = 0; k < KD_COUNT; ++k) {
    if (!n[k]) continue;
    if (c < max) {
      std::memset(&out[c], 0, sizeof(out[c]));
      std::strncpy(out[c].name, kKernelNames[k], sizeof(out[c].name) - 1);
      out[c].launches = n[k];
      out[c].total_ms = ms[k];
    }
    ++c;
  }
  *count = c < max ? c : max;
  return AT_DNS_OK;
}

int at_dns_tune(at_dns_t* h, int32_t delay_mode, int32_t trials, double* best_ms) {
  NvtxRange nvtx_range("at_dns_tune");
  if (!h) return AT_DNS_E_INVALID_ARG;
  h->err.clear();
  int rc;
  if ((rc = check_mode(h, delay_mode))) return rc;
  if (trials < 1) return fail(h, AT_DNS_E_INVALID_ARG, "trials must be >= 1");
  if (!h->has_state) return fail(h, AT_DNS_E_STATE, "no state set");
  const bool was_prof = h->prof;
  h->prof = false;
  const bool stats = h->cfg.stats_every == 1;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  double best = 1e300;
  Candidate pick{h->fused, h->TX, h->TY, h->ZC, h->paired};
  for (const Candidate& c : tune_candidates(h->g, h->p64)) {
    if (set_path(h, c.fused, c.TX, c.TY, c.ZC, c.paired) != AT_DNS_OK) continue;   // e.g. no memory for work arrays
    // one untimed evaluation, then `trials` timed right-hand sides (no state change)
    for (int t = 0; t <= trials; ++t) {
      if (t == 1) CK(cudaEventRecord(e0, h->st));
      rc = h->p64 ? Ops<double>::launch_step(h, delay_mode, false, nullptr, stats, true, h->st)
                  : Ops<float>::launch_step(h, delay_mode, false, nullptr, stats, true, h->st);
      if (rc) break;
    }
    if (rc) { h->err.clear(); rc = AT_DNS_OK; continue; }
    CK(cudaEventRecord(e1, h->st));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms / trials < best) { best = ms / trials; pick = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if ((rc = set_path(h, pick.fused, pick.TX, pick.TY, pick.ZC, pick.paired))) return rc;
  h->stats_valid = false;
  h->prof = was_prof;
  if (best_ms) *best_ms = best;
  return AT_DNS_OK;
}

int at_dns_set_kernel_path(at_dns_t* h, int32_t path, const int32_t tile[3]) {
  if (!h) return AT_DNS_E_INVALID_ARG;
  h->err.clear();
  if (path == AT_DNS_PATH_MULTIPASS) return set_path(h, false, 0, 0, 0);
  if ((path != AT_DNS_PATH_FUSED && path != AT_DNS_PATH_PAIRED) || !tile)
    return fail(h, AT_DNS_E_INVALID_ARG, "path must be MULTIPASS, or FUSED or PAIRED with a tile");
  const bool paired = path == AT_DNS_PATH_PAIRED;
  for (const Candidate& c : tune_candidates(h->g, h->p64))
    if (c.fused && c.paired == paired && c.TX == tile[0] && c.TY == tile[1] && c.ZC == tile[2])
      return set_path(h, true, c.TX, c.TY, c.ZC, paired);
  return fail(h, AT_DNS_E_UNSUPPORTED, "tile is not a fused-path candidate for this handle");
}

int at_dns_synchronize(at_dns_t* h) {
  if (!h) return AT_DNS_E_INVALID_ARG;
  CK(cudaStreamSynchronize(h->st));
  return AT_DNS_OK;
}

const char* at_dns_last_error(const at_dns_t* h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

void at_dns_destroy(at_dns_t* h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st); else cudaDeviceSynchronize();
  drop_graphs(h);
  void* ptrs[] = {h->ds, h->U[0], h->U[1], h->Ulo[0], h->Ulo[1], h->PQ, h->G, h->Rprev, h->GH[0], h->GH[1], h->GH[2],
                  h->ring[0], h->ring[1], h->ring[2], h->xst, h->stage, h->dmap, h->partial, h->sums, h->words,
                  h->modes, h->fhat, h->fB, h->fX};
  if (!h->pool)
    for (void* p : ptrs)
      if (p) cudaFree(p);
  clear_recs(h);
  delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched ensembles: independent members, one graph launch per step
struct at_dns_batch {
  std::vector<at_dns*> m;
  std::vector<cudaStream_t> ms;       // one stream per member (owned)
  std::vector<cudaEvent_t> ev;        // per-member ordering / join events
  cudaEvent_t fork = nullptr, done = nullptr;
  cudaStream_t st = nullptr;          // batch stream
  bool own_st = false;
  cudaGraphExec_t gexec[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  std::vector<std::string> gkey[5];   // member path + dt each graph was captured with
  std::string err;
  // persistent single-launch step (eligible FP32 batches)
  bool allow_persistent = false;      // the persistent single-launch step is opt-in
  int ptx = 0, pty = 0;               // its tile (0: not eligible)
  int ctas = 0;                       // CTAs resident together (the cooperative grid)
  atdns::BatchMember* dmem = nullptr; // device member table
  unsigned* dctr = nullptr;           // [2][count]: ghost items, tiles finished per member
  unsigned epoch = 0;                 // persistent launches since the counters were cleared
  int* derr = nullptr;                // a wait gave up
  std::string pkey;                   // mode + members' dt the table was built with
  // the members' tile descriptions for constant memory (uploaded when this
  // batch is not the one whose tables are there)
  std::vector<atdns::TileDesc> htiles;
  std::vector<std::array<int, 4>> hshape;
  std::vector<long long> hgitems, hitems;   // prefix sums of the ghost items and of the tiles
  unsigned long long table_gen = 0;
};

namespace {

// Constant memory holds the tile descriptions of one batch at a time: the
// batch (and table generation) whose tables are there, and an event after
// the last persistent launch that read them (an upload for another batch
// waits for it).
std::mutex g_const_mu;
const at_dns_batch* g_const_owner = nullptr;
unsigned long long g_const_gen = 0;
cudaEvent_t g_const_last = nullptr;

std::string member_key(const at_dns* h) {
  char buf[128];
  std::snprintf(buf, sizeof(buf), "%d:%d:%d:%d:%.17g", (int)h->fused, h->TX, h->TY, h->ZC, h->dt);
  return buf;
}

int batch_fail(at_dns_batch* b, int code, const std::string& msg) {
  b->err = msg;
  return code;
}

void batch_drop(at_dns_batch* b) {
  for (int k = 0; k < 5; ++k)
    if (b->gexec[k]) { cudaGraphExecDestroy(b->gexec[k]); b->gexec[k] = nullptr; }
}

// z chunk of a paired tile: the z extent itself up to 64 planes, else its
// largest divisor in [8, 64] (0: none)
int z_chunk(const at_dns* h) {
  const int ext = h->g.pes[2] > 1 ? h->g.nl[2] : h->g.n[2];
  if (ext <= 64) return ext;
  for (int t = 64; t >= 8; --t)
    if (ext % t == 0) return t;
  return 0;
}

// The paired tile every member can run (16x16 preferred, then 32x8), or
// false when some member cannot take the persistent step (FP64, 6th order,
// RK3, forcing, extents that fit no common tile).
bool batch_persistent_tile(const at_dns_batch* b, int& TX, int& TY) {
  const int shapes[2][2] = {{16, 16}, {32, 8}};
  for (auto& sh : shapes) {
    bool ok = true;
    for (const at_dns* h : b->m) {
      int ext[3];
      for (int d = 0; d < 3; ++d) ext[d] = h->g.pes[d] > 1 ? h->g.nl[d] : h->g.n[d];
      if (b->m.size() > (size_t)atdns::kBatchConstMembers || h->p64 || h->g.M != 2 ||
          h->cfg.integrator != AT_DNS_AB2 || h->cfg.forcing || ext[0] % sh[0] || ext[1] % sh[1] || !z_chunk(h)) {
        ok = false;
        break;
      }
    }
    if (ok) { TX = sh[0]; TY = sh[1]; return true; }
  }
  return false;
}

// Build (or keep) the device member table of the persistent step for mode.
int batch_table(at_dns_batch* b, int mode) {
  const int M = (int)b->m.size();
  std::string key = std::to_string(mode) + "/" + std::to_string(b->ptx) + "x" + std::to_string(b->pty);
  for (const at_dns* h : b->m) key += ":" + std::to_string(h->dt);
  if (b->dmem && key == b->pkey) return AT_DNS_OK;
  if (!b->dmem) {
    if (cudaMalloc(&b->dmem, M * sizeof(atdns::BatchMember)) != cudaSuccess ||
        cudaMalloc(&b->dctr, 2 * M * sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&b->derr, sizeof(int)) != cudaSuccess) {
      (void)cudaGetLastError();
      return batch_fail(b, AT_DNS_E_OOM, "cannot allocate the persistent step's tables");
    }
    if (cudaMemsetAsync(b->derr, 0, sizeof(int), b->st) != cudaSuccess)
      return batch_fail(b, AT_DNS_E_CUDA, "cannot clear the persistent step's error flag");
  }
  // the table and counters are rewritten after every earlier launch that read
  // them has finished; the counters restart with the table
  if (cudaStreamSynchronize(b->st) != cudaSuccess ||
      cudaMemsetAsync(b->dctr, 0, 2 * M * sizeof(unsigned), b->st) != cudaSuccess)
    return batch_fail(b, AT_DNS_E_CUDA, "cannot clear the persistent step's counters");
  b->epoch = 0;
  std::vector<atdns::BatchMember> hm(M);
  b->htiles.assign(M, atdns::TileDesc{});
  b->hshape.assign(M, std::array<int, 4>{0, 0, 0, 0});
  b->hgitems.assign(M + 1, 0);
  b->hitems.assign(M + 1, 0);
  for (int i = 0; i < M; ++i) {
    const at_dns* h = b->m[i];
    const Geom& g = h->g;
    atdns::BatchMember& m = hm[i];
    std::memset(&m, 0, sizeof(m));
    m.g = g;
    m.K = make_coef<float>(g, h->ph, h->dt);
    m.KP = make_coef_pair(m.K);
    StepArgs<float>& a = m.A;
    a.Ub[0] = (const float*)h->U[0];
    a.Ub[1] = (const float*)h->U[1];
    a.Ulob[0] = h->comp ? (float*)h->Ulo[0] : nullptr;
    a.Ulob[1] = h->comp ? (float*)h->Ulo[1] : nullptr;
    a.ds = h->ds;
    for (int d = 0; d < 3; ++d) a.GH[d] = (const float*)h->GH[d];
    a.Rprev = (float*)h->Rprev;
    a.partial = h->partial;
    a.words = h->words;
    a.fB = nullptr;
    a.fX = (const vec2_t<float>*)h->fX;
    a.dt = h->dt;
    a.do_update = 1;
    a.do_stats = h->cfg.stats_every == 1 ? 1 : 0;
    a.xst = (float*)h->xst;
    a.xst_half = h->xst_half;
    const int ZC = z_chunk(h), tiles_x = g.n[0] / b->ptx, tiles_y = g.n[1] / b->pty;
    m.nblk = (long long)tiles_x * tiles_y * (g.n[2] / ZC);
    m.mode = mode;
    m.L = h->cfg.max_delay;
    m.tl = g.M + 1;
    m.cr = h->cfg.comm_period;
    m.k0 = (uint32_t)h->cfg.seed;
    m.k1 = (uint32_t)(h->cfg.seed >> 32);
    for (int d = 0; d < 3; ++d) {
      m.GH[d] = (float*)h->GH[d];
      m.ring[d] = (double*)h->ring[d];
      m.ghost_cnt[d] = g.pes[d] > 1 ? 2LL * g.M * g.pes[d] * g.plane[d] : 0;
    }
    m.xst = (const float*)h->xst;
    m.xst_half = h->xst_half;
    m.sums = h->sums;
    // ghost items (at least one: it also resets the step's max/min keys)
    const long long gtot = m.ghost_cnt[0] + m.ghost_cnt[1] + m.ghost_cnt[2];
    const long long gitems = std::max(1LL, (gtot + atdns::kBatchGhostChunk - 1) / atdns::kBatchGhostChunk);
    b->htiles[i].g = m.g;
    b->htiles[i].K = m.K;
    b->htiles[i].KP = m.KP;
    b->htiles[i].A = m.A;
    b->hshape[i] = {ZC, tiles_x, tiles_y, (int)gitems};
    b->hgitems[i + 1] = b->hgitems[i] + gitems;
    b->hitems[i + 1] = b->hitems[i] + m.nblk;
  }
  if (cudaMemcpy(b->dmem, hm.data(), M * sizeof(atdns::BatchMember), cudaMemcpyHostToDevice) != cudaSuccess)
    return batch_fail(b, AT_DNS_E_CUDA, "cannot upload the persistent step's tables");
  b->pkey = key;
  ++b->table_gen;
  return AT_DNS_OK;
}

// Whether the next batch step runs as the persistent single launch (and its tile).
bool batch_uses_persistent(at_dns_batch* b) {
  if (!b->allow_persistent) return false;
  int TX = 0, TY = 0;
  if (!batch_persistent_tile(b, TX, TY)) return false;
  if (TX != b->ptx || TY != b->pty || !b->ctas) {
    int ctas = 0;
    if (batch_resident_ctas(TX, TY, &ctas) != cudaSuccess) {
      (void)cudaGetLastError();
      return false;
    }
    b->ptx = TX;
    b->pty = TY;
    b->ctas = ctas;
    b->pkey.clear();
  }
  return true;
}

}  // namespace

extern "C" {

void at_dns_batch_destroy(at_dns_batch_t* b);

int at_dns_batch_create(const at_dns_config_t* cfgs, int32_t count, void* stream, at_dns_batch_t** out) {
  if (!cfgs || !out || count < 1) { g_create_error = "bad batch arguments"; return AT_DNS_E_INVALID_ARG; }
  *out = nullptr;
  at_dns_batch* b = new at_dns_batch();
  if (stream) b->st = (cudaStream_t)stream;
  else {
    if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) {
      g_create_error = "cannot create the batch stream";
      delete b;
      return AT_DNS_E_CUDA;
    }
    b->own_st = true;
  }
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess) {
    g_create_error = "cannot create events";
    at_dns_batch_destroy(b);
    return AT_DNS_E_CUDA;
  }
  for (int i = 0; i < count; ++i) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      g_create_error = "cannot create member streams";
      at_dns_batch_destroy(b);
      return AT_DNS_E_CUDA;
    }
    b->ms.push_back(s);
    b->ev.push_back(e);
    at_dns_config_t c = cfgs[i];
    c.stream = s;
    at_dns* h = nullptr;
    const int rc = at_dns_create(&c, &h);
    if (rc) {
      g_create_error = "member " + std::to_string(i) + ": " + g_create_error;
      at_dns_batch_destroy(b);
      return rc;
    }
    b->m.push_back(h);
  }
  *out = b;
  return AT_DNS_OK;
}

int at_dns_batch_member(at_dns_batch_t* b, int32_t i, at_dns_t** out) {
  if (!b || !out || i < 0 || i >= (int)b->m.size()) return AT_DNS_E_INVALID_ARG;
  *out = b->m[i];
  return AT_DNS_OK;
}

int at_dns_batch_step(at_dns_batch_t* b, int32_t nsteps, int32_t delay_mode) {
  NvtxRange nvtx_range("at_dns_batch_step");
  if (!b) return AT_DNS_E_INVALID_ARG;
  b->err.clear();
  if (nsteps < 0 || delay_mode < 0 || delay_mode > 4) return batch_fail(b, AT_DNS_E_INVALID_ARG, "bad arguments");
  const int M = (int)b->m.size();
  std::vector<std::string> key(M);
  for (int i = 0; i < M; ++i) {
    at_dns* h = b->m[i];
    if (!h->has_state) return batch_fail(b, AT_DNS_E_STATE, "member " + std::to_string(i) + " has no state");
    if (check_mode(h, delay_mode)) return batch_fail(b, AT_DNS_E_INVALID_ARG, "member " + std::to_string(i) + ": " + h->err);
    key[i] = member_key(h);
  }
  if (nsteps == 0) return AT_DNS_OK;
  if (batch_uses_persistent(b)) {
    int rc;
    if ((rc = batch_table(b, delay_mode))) return rc;
    // order after each member's own stream; reset the health words
    for (int i = 0; i < M; ++i) {
      k_reset_words<<<1, 1, 0, b->ms[i]>>>(b->m[i]->words, 1);
      cudaEventRecord(b->ev[i], b->ms[i]);
      cudaStreamWaitEvent(b->st, b->ev[i], 0);
    }
    atdns::BatchSched S;
    S.m = b->dmem;
    S.count = M;
    S.gdone = b->dctr;
    S.tdone = b->dctr + M;
    S.err = b->derr;
    {
      std::lock_guard<std::mutex> lock(g_const_mu);
      if (g_const_owner != b || g_const_gen != b->table_gen) {
        if (!g_const_last && cudaEventCreateWithFlags(&g_const_last, cudaEventDisableTiming) != cudaSuccess)
          return batch_fail(b, AT_DNS_E_CUDA, "cannot create the constant-table event");
        if (g_const_owner) cudaStreamWaitEvent(b->st, g_const_last, 0);
        const cudaError_t e = atdns::upload_batch_tiles(
            b->htiles.data(), reinterpret_cast<const int(*)[4]>(b->hshape.data()), b->hgitems.data(), b->hitems.data(), M,
            b->st);
        if (e != cudaSuccess) {
          g_const_owner = nullptr;
          return batch_fail(b, AT_DNS_E_CUDA, std::string("persistent step tables: ") + cudaGetErrorString(e));
        }
        g_const_owner = b;
        g_const_gen = b->table_gen;
      }
      for (int s = 0; s < nsteps; ++s) {
        S.epoch = ++b->epoch;
        const cudaError_t e = launch_batch_step(b->ptx, b->pty, S, b->ctas, b->st);
        if (e != cudaSuccess) {
          cudaEventRecord(g_const_last, b->st);
          return batch_fail(b, AT_DNS_E_CUDA, std::string("persistent step: ") + cudaGetErrorString(e));
        }
        for (int i = 0; i < M; ++i) {
          at_dns* h = b->m[i];
          Ops<float>::account(h, true, h->cfg.stats_every == 1);
        }
      }
      cudaEventRecord(g_const_last, b->st);
    }
    int gave_up = 0;
    if (cudaMemcpyAsync(&gave_up, b->derr, sizeof(int), cudaMemcpyDeviceToHost, b->st) != cudaSuccess ||
        cudaStreamSynchronize(b->st) != cudaSuccess)
      return batch_fail(b, AT_DNS_E_CUDA, "persistent step failed");
    if (gave_up) {
      cudaMemsetAsync(b->derr, 0, sizeof(int), b->st);
      return batch_fail(b, AT_DNS_E_TIMEOUT, "a wait of the persistent step for a member's ghost items gave up");
    }
  } else {
  cudaGraphExec_t& ge = b->gexec[delay_mode];
  if (!ge || b->gkey[delay_mode] != key) {
    if (ge) { cudaGraphExecDestroy(ge); ge = nullptr; }
    // one step of every member, each on its own branch of the graph; the
    // branches are captured largest member first, so that the small members'
    // kernels fill the SMs the large ones leave idle rather than the reverse
    std::vector<int> order(M);
    for (int i = 0; i < M; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return b->m[x]->g.npts > b->m[y]->g.npts; });
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(b->st, cudaStreamCaptureModeRelaxed) != cudaSuccess)
      return batch_fail(b, AT_DNS_E_CUDA, "graph capture failed to start");
    int rc = AT_DNS_OK;
    cudaEventRecord(b->fork, b->st);
    for (int k = 0; k < M && !rc; ++k) {
      const int i = order[k];
      at_dns* h = b->m[i];
      cudaStreamWaitEvent(b->ms[i], b->fork, 0);
      const bool stats = h->cfg.stats_every == 1;
      rc = h->p64 ? Ops<double>::launch_update(h, delay_mode, stats, false, b->ms[i])
                  : Ops<float>::launch_update(h, delay_mode, stats, false, b->ms[i]);
      cudaEventRecord(b->ev[i], b->ms[i]);
      cudaStreamWaitEvent(b->st, b->ev[i], 0);
    }
    const cudaError_t e = cudaStreamEndCapture(b->st, &graph);
    if (rc) { if (graph) cudaGraphDestroy(graph); return batch_fail(b, rc, "capture: " + b->m[0]->err); }
    if (e != cudaSuccess) return batch_fail(b, AT_DNS_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    const cudaError_t e2 = cudaGraphInstantiate(&ge, graph, 0);
    cudaGraphDestroy(graph);
    if (e2 != cudaSuccess) { ge = nullptr; return batch_fail(b, AT_DNS_E_CUDA, "graph instantiate failed"); }
    b->gkey[delay_mode] = key;
  }
  // order after each member's own stream, reset the health words, replay
  for (int i = 0; i < M; ++i) {
    k_reset_words<<<1, 1, 0, b->ms[i]>>>(b->m[i]->words, 1);
    cudaEventRecord(b->ev[i], b->ms[i]);
    cudaStreamWaitEvent(b->st, b->ev[i], 0);
  }
  for (int s = 0; s < nsteps; ++s) {
    const cudaError_t e = cudaGraphLaunch(ge, b->st);
    if (e != cudaSuccess) return batch_fail(b, AT_DNS_E_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    for (int i = 0; i < M; ++i) {
      at_dns* h = b->m[i];
      const bool stats = h->cfg.stats_every == 1;
      if (h->p64) Ops<double>::account(h, true, stats); else Ops<float>::account(h, true, stats);
    }
  }
  }
  cudaEventRecord(b->done, b->st);
  std::vector<unsigned long long> w(M, 0);
  for (int i = 0; i < M; ++i) {
    cudaStreamWaitEvent(b->ms[i], b->done, 0);
    cudaMemcpyAsync(&w[i], b->m[i]->words + 3, sizeof(unsigned long long), cudaMemcpyDeviceToHost, b->ms[i]);
  }
  for (int i = 0; i < M; ++i) {
    const cudaError_t e = cudaStreamSynchronize(b->ms[i]);
    if (e != cudaSuccess) return batch_fail(b, AT_DNS_E_CUDA, std::string("batch step: ") + cudaGetErrorString(e));
  }
  for (int i = 0; i < M; ++i)
    if (report_checks(b->m[i])) return batch_fail(b, AT_DNS_E_BOUNDS, "member " + std::to_string(i) + ": " + b->m[i]->err);
  for (int i = 0; i < M; ++i)
    if (w[i]) return batch_fail(b, AT_DNS_E_UNSTABLE, "member " + std::to_string(i) + " became unstable");
  return AT_DNS_OK;
}

int at_dns_batch_tune(at_dns_batch_t* b, int32_t delay_mode, int32_t trials) {
  NvtxRange nvtx_range("at_dns_batch_tune");
  if (!b) return AT_DNS_E_INVALID_ARG;
  b->err.clear();
  if (trials < 1 || delay_mode < 0 || delay_mode > 4) return batch_fail(b, AT_DNS_E_INVALID_ARG, "bad arguments");
  const int M = (int)b->m.size();
  for (int i = 0; i < M; ++i)
    if (!b->m[i]->has_state) return batch_fail(b, AT_DNS_E_STATE, "member " + std::to_string(i) + " has no state");
  auto path_of = [](const at_dns* h) { return Candidate{h->fused, h->TX, h->TY, h->ZC, h->paired}; };
  auto same = [](const Candidate& a, const Candidate& c) {
    return a.fused == c.fused && a.paired == c.paired && a.TX == c.TX && a.TY == c.TY && a.ZC == c.ZC;
  };
  std::vector<std::vector<Candidate>> plans(1, std::vector<Candidate>(M));
  for (int i = 0; i < M; ++i) plans[0][i] = path_of(b->m[i]);   // the members' paths now
  // each member's own pick, timed alone (right-hand sides: no state change)
  {
    std::vector<Candidate> own(M);
    for (int i = 0; i < M; ++i) {
      const int rc = at_dns_tune(b->m[i], delay_mode, trials, nullptr);
      if (rc) return batch_fail(b, rc, "member " + std::to_string(i) + ": " + b->m[i]->err);
      own[i] = path_of(b->m[i]);
    }
    plans.push_back(own);
  }
  // the run states, so that the timed batch steps below leave them as they are
  std::vector<void*> saved(M, nullptr);
  auto release = [&]() {
    for (void*& p : saved)
      if (p) { cudaFree(p); p = nullptr; }
  };
  for (int i = 0; i < M; ++i) {
    int64_t bytes = 0;
    at_dns_checkpoint_size(b->m[i], &bytes);
    if (cudaMalloc(&saved[i], (size_t)bytes) != cudaSuccess) {
      // no room for the checkpoints: keep each member's own pick
      (void)cudaGetLastError();
      release();
      batch_drop(b);
      return AT_DNS_OK;
    }
    if (at_dns_checkpoint_save(b->m[i], saved[i], AT_DNS_DEVICE)) {
      release();
      return batch_fail(b, AT_DNS_E_CUDA, "member " + std::to_string(i) + ": " + b->m[i]->err);
    }
  }
  auto restore = [&]() {
    for (int i = 0; i < M; ++i)
      if (at_dns_checkpoint_load(b->m[i], saved[i], AT_DNS_DEVICE)) return false;
    return true;
  };
  // uniform shapes: every member on the same tile shape where it has one (its
  // largest z chunk), else on its own pick
  {
    std::vector<Candidate> shapes;
    for (int i = 0; i < M; ++i)
      for (const Candidate& c : tune_candidates(b->m[i]->g, b->m[i]->p64)) {
        bool seen = false;
        for (const Candidate& s : shapes)
          seen = seen || (s.fused == c.fused && s.paired == c.paired && s.TX == c.TX && s.TY == c.TY);
        if (!seen) shapes.push_back(c);
      }
    for (const Candidate& s : shapes) {
      std::vector<Candidate> cfg = plans[1];
      for (int i = 0; i < M; ++i)
        for (const Candidate& c : tune_candidates(b->m[i]->g, b->m[i]->p64))
          if (c.fused == s.fused && c.paired == s.paired && c.TX == s.TX && c.TY == s.TY) { cfg[i] = c; break; }
      bool dup = false;
      for (const auto& k : plans) {
        bool eq = true;
        for (int i = 0; i < M; ++i) eq = eq && same(k[i], cfg[i]);
        dup = dup || eq;
      }
      if (!dup) plans.push_back(cfg);
    }
  }
  // time one batch step of every configuration (graph form), from the saved states
  const bool was_persistent = b->allow_persistent;
  b->allow_persistent = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e300;
  size_t pick = 0;
  for (size_t k = 0; k < plans.size(); ++k) {
    bool ok = true;
    for (int i = 0; i < M && ok; ++i) {
      const Candidate& c = plans[k][i];
      ok = set_path(b->m[i], c.fused, c.TX, c.TY, c.ZC, c.paired) == AT_DNS_OK;
    }
    ok = ok && at_dns_batch_step(b, 1, delay_mode) == AT_DNS_OK;   // captures the graph
    if (ok) {
      cudaEventRecord(e0, b->st);
      ok = at_dns_batch_step(b, trials, delay_mode) == AT_DNS_OK;
      cudaEventRecord(e1, b->st);
      cudaEventSynchronize(e1);
    }
    float ms = 0.f;
    if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms / trials < best) {
      best = ms / trials;
      pick = k;
    }
    b->err.clear();
    if (!restore()) {
      b->allow_persistent = was_persistent;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      release();
      return batch_fail(b, AT_DNS_E_CUDA, "cannot restore the members' states");
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->allow_persistent = was_persistent;
  for (int i = 0; i < M; ++i) {
    const Candidate& c = plans[pick][i];
    if (set_path(b->m[i], c.fused, c.TX, c.TY, c.ZC, c.paired) != AT_DNS_OK) {
      release();
      return batch_fail(b, AT_DNS_E_CUDA, "member " + std::to_string(i) + ": " + b->m[i]->err);
    }
  }
  release();
  batch_drop(b);
  return AT_DNS_OK;
}

int at_dns_batch_persistent(at_dns_batch_t* b, int32_t enable, int32_t* persistent) {
  if (!b) return AT_DNS_E_INVALID_ARG;
  b->err.clear();
  if (enable >= 0) b->allow_persistent = enable != 0;
  if (persistent) *persistent = batch_uses_persistent(b) ? 1 : 0;
  return AT_DNS_OK;
}

int at_dns_wait_selftest(int32_t log2_polls, int32_t* gave_up) {
  if (!gave_up || log2_polls < 0 || log2_polls > 26) return AT_DNS_E_INVALID_ARG;
  int g = -1;
  if (atdns::batch_wait_selftest(log2_polls, &g) != cudaSuccess) return AT_DNS_E_CUDA;
  *gave_up = g;
  return AT_DNS_OK;
}

const char* at_dns_batch_last_error(const at_dns_batch_t* b) { return b ? b->err.c_str() : g_create_error.c_str(); }

void at_dns_batch_destroy(at_dns_batch_t* b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  {
    std::lock_guard<std::mutex> lock(g_const_mu);
    if (g_const_owner == b) g_const_owner = nullptr;   // a later batch at this address uploads its own
  }
  batch_drop(b);
  for (void* p : {(void*)b->dmem, (void*)b->dctr, (void*)b->derr})
    if (p) cudaFree(p);
  for (at_dns* h : b->m) at_dns_destroy(h);
  for (cudaStream_t s : b->ms) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->done) cudaEventDestroy(b->done);
  if (b->own_st) cudaStreamDestroy(b->st);
  delete b;
}

}  // extern "C"
