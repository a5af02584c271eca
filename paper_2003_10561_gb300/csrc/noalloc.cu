// at_dns_rhs_noalloc: a right-hand side evaluation that allocates no device
// memory, for callers that cannot call cudaMalloc -- code that runs while
// another component owns every allocation on the device (a host framework
// with its own caching allocator or a fixed memory budget), code called from
// inside a region that must not allocate (a real-time loop, or a callback
// where an allocation would synchronise the device), or a plugin loaded into
// a process that forbids new allocations after start-up.
//
// The caller passes the state and the output; the per-point work arrays the
// kernels need (derived fields, gradients, reduction words) live in one
// file-scope __device__ array of fixed size, so every GPU that loads this
// library holds it (about 59 MB) until the process exits.
#include <climits>
#include <cmath>
#include <cstring>

#include "../../include/at_dns.h"
#include "common.cuh"
#include "launch.h"

using namespace atdns;

namespace {

constexpr long long kMaxPts = AT_DNS_NOALLOC_MAX_POINTS;
constexpr long long kWordDoubles = 4;   // max/min keys and the health word
constexpr long long kScratchDoubles = (long long)(kNumQ + kNumGrad) * kMaxPts + kWordDoubles;

// Shared by every call on a device; contents persist between calls.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

__global__ void k_noalloc_reset(unsigned long long* w) {
  w[0] = (unsigned long long)LLONG_MIN;
  w[1] = (unsigned long long)LLONG_MAX;
  w[2] = (unsigned long long)LLONG_MAX;
  w[3] = 0ULL;
}

// Device address of the scratch array on the current device (host code only
// sees a stand-in for it).  Looked up on every call, with the caller's device
// current: the lookup is a host-side query, not a stream operation, and it
// stays right after a cudaDeviceReset has rebuilt the device's context (the
// array can then sit at another address).  The first call on a device loads
// the library's device code there.
cudaError_t scratch_on_current_device(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = (double*)p;
  return cudaSuccess;
}

}  // namespace

extern "C" int at_dns_rhs_noalloc(const int32_t n[3], double gamma, double prandtl, double mu0, double visc_exp,
                                  const double* u_dev, double* rhs_dev, void* stream) {
  if (!n || !u_dev || !rhs_dev) return AT_DNS_E_INVALID_ARG;
  long long npts = 1;
  for (int d = 0; d < 3; ++d) {
    if (n[d] < 5 || n[d] > 32768) return AT_DNS_E_INVALID_ARG;
    npts *= n[d];
  }
  if (npts > kMaxPts) return AT_DNS_E_TOO_LARGE;
  if (!(gamma > 1.0) || !(prandtl > 0) || !(mu0 >= 0) || !std::isfinite(gamma) || !std::isfinite(prandtl) ||
      !std::isfinite(mu0) || !std::isfinite(visc_exp))
    return AT_DNS_E_INVALID_ARG;
  double* base = nullptr;
  if (scratch_on_current_device(&base) != cudaSuccess) return AT_DNS_E_CUDA;

  // one PE, periodic in every direction: no faces, no delays, no ring
  Geom g{};
  g.npts = npts;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = n[d];
    g.pes[d] = 1;
    g.nl[d] = n[d];
  }
  g.stride[0] = 1;
  g.stride[1] = g.n[0];
  g.stride[2] = (long long)g.n[0] * g.n[1];
  for (int d = 0; d < 3; ++d) g.plane[d] = g.npts / g.n[d];
  set_stencils(g, 2);   // 4th-order scheme
  g.nlev = 3;
  Phys ph{};
  ph.gamma = gamma;
  ph.gm1 = gamma - 1.0;
  ph.prandtl = prandtl;
  ph.mu0 = mu0;
  ph.omega = visc_exp;
  ph.cp_over_pr = 1.0 / ((gamma - 1.0) * prandtl);
  const Coef<double> K = make_coef<double>(g, ph, 0.0);

  // carve the array for this problem size
  double* PQ = base;
  double* G = base + (long long)kNumQ * npts;
  unsigned long long* words = (unsigned long long*)(base + (long long)(kNumQ + kNumGrad) * npts);
  cudaStream_t st = (cudaStream_t)stream;
  double* const GH[3] = {nullptr, nullptr, nullptr};

  k_noalloc_reset<<<1, 1, 0, st>>>(words);   // the words must start cleared
  if (cudaGetLastError() != cudaSuccess) return AT_DNS_E_CUDA;
  if (launch_prim<double>(g, K, u_dev, u_dev, nullptr, PQ, st) != cudaSuccess) return AT_DNS_E_CUDA;
  if (launch_grad<double>(g, K, PQ, GH, G, st) != cudaSuccess) return AT_DNS_E_CUDA;
  StepArgs<double> a{};
  a.U = u_dev;
  a.PQ = PQ;
  a.G = G;
  a.Rout = rhs_dev;
  a.words = words;
  a.do_update = 0;
  a.do_stats = 0;
  if (launch_main<double>(g, K, a, st) != cudaSuccess) return AT_DNS_E_CUDA;
  return AT_DNS_OK;
}
