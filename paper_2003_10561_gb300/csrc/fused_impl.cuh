// Launcher of the fused step kernel for one scalar type; included by
// kernels_fused_p64.cu and kernels_fused_p32.cu with AT_DNS_SCALAR set.
#include "kernels_fused.cuh"
#include "launch.h"

namespace atdns {

using S = AT_DNS_SCALAR;

template <int TX, int TY>
static cudaError_t run_fused(const Geom& g, const Coef<S>& K, const StepArgs<S>& a, int ZC, cudaStream_t st) {
  const size_t smem = fused_smem_bytes<S>(TX, TY);
  cudaError_t e = cudaFuncSetAttribute(k_fused<S, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();   // a tile too large for this precision: not a sticky error
    return e;
  }
  const dim3 grid((unsigned)(g.n[0] / TX), (unsigned)(g.n[1] / TY), (unsigned)(g.n[2] / ZC));
  const dim3 block((unsigned)TX, (unsigned)TY);
  k_fused<S, TX, TY><<<grid, block, smem, st>>>(g, K, a, ZC);
  return cudaGetLastError();
}

template <>
cudaError_t launch_fused<S>(const Geom& g, const Coef<S>& K, const StepArgs<S>& a, int TX, int TY, int ZC,
                            cudaStream_t st) {
  if (TX == 32 && TY == 8) return run_fused<32, 8>(g, K, a, ZC, st);
  if constexpr (sizeof(S) == 4)
    if (TX == 32 && TY == 16) return run_fused<32, 16>(g, K, a, ZC, st);
  if (TX == 16 && TY == 16) return run_fused<16, 16>(g, K, a, ZC, st);
  if (TX == 16 && TY == 8) return run_fused<16, 8>(g, K, a, ZC, st);
  if (TX == 8 && TY == 32) return run_fused<8, 32>(g, K, a, ZC, st);
  if (TX == 8 && TY == 16) return run_fused<8, 16>(g, K, a, ZC, st);
  if (TX == 8 && TY == 8) return run_fused<8, 8>(g, K, a, ZC, st);
  return cudaErrorInvalidValue;
}

}  // namespace atdns
