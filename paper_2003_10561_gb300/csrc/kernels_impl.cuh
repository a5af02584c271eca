// Definitions of the launchers for one scalar type and stencil half width;
// included by kernels_p64.cu, kernels_p32.cu (M = 2) and kernels_p64_o6.cu,
// kernels_p32_o6.cu (M = 3) with AT_DNS_SCALAR and AT_DNS_HALF_WIDTH set.
#include "kernels.cuh"
#include "launch.h"

namespace atdns {

using S = AT_DNS_SCALAR;
constexpr int kM = AT_DNS_HALF_WIDTH;

#if AT_DNS_HALF_WIDTH == 2
template <>
cudaError_t launch_prim<S>(const Geom& g, const Coef<S>& K, const S* U0, const S* U1, const DevState* ds, S* PQ,
                           cudaStream_t st) {
  const unsigned nb = (unsigned)((g.npts + kBlock - 1) / kBlock);
  k_prim<S><<<nb, kBlock, 0, st>>>(g, K, U0, U1, ds, PQ);
  return cudaGetLastError();
}
#endif

template <>
cudaError_t launch_ghost_m<S, kM>(const Geom& g, const Coef<S>& K, const S* U0, const S* U1, const S* Ulo0,
                                  const S* Ulo1, const DevState* ds, const S* PQ, S* const GH[3],
                                  double* const ring[3], const S* xst, long long xst_half, const uint8_t* dmap,
                                  long long n, cudaStream_t st) {
  long long cnt[3];
  for (int d = 0; d < 3; ++d) cnt[d] = g.pes[d] > 1 ? 2LL * kM * g.pes[d] * g.plane[d] : 0;
  const long long tot = cnt[0] + cnt[1] + cnt[2];
  if (tot == 0) return cudaSuccess;
  const unsigned nb = (unsigned)((tot + kBlock - 1) / kBlock);
  k_ghost<S, kM><<<nb, kBlock, 0, st>>>(g, K, U0, U1, Ulo0, Ulo1, ds, PQ, GH[0], GH[1], GH[2], ring[0], ring[1],
                                        ring[2], xst, xst_half, dmap, n, cnt[0], cnt[1], cnt[2]);
  return cudaGetLastError();
}

template <>
cudaError_t launch_grad_m<S, kM>(const Geom& g, const Coef<S>& K, const S* PQ, S* const GH[3], S* G,
                                 cudaStream_t st) {
  const unsigned nb = (unsigned)((g.npts + kBlock - 1) / kBlock);
  k_grad<S, kM><<<nb, kBlock, 0, st>>>(g, K, PQ, GH[0], GH[1], GH[2], G);
  return cudaGetLastError();
}

template <>
cudaError_t launch_main_m<S, kM>(const Geom& g, const Coef<S>& K, const StepArgs<S>& a, cudaStream_t st) {
  const unsigned nb = (unsigned)main_blocks(g);
  k_main<S, kM><<<nb, kBlock, 0, st>>>(g, K, a);
  return cudaGetLastError();
}

}  // namespace atdns
