// Launcher of the paired fused step kernel (FP32-bulk forms).
#include "kernels_fused2.cuh"
#include "launch.h"

namespace atdns {

template <int TX, int TY, bool PLAIN>
static cudaError_t run_fused2_as(const Geom& g, const Coef<float>& K, const StepArgs<float>& a, int ZC,
                                 cudaStream_t st) {
  const size_t smem = fused_smem_bytes<float>(TX, TY);
  cudaError_t e =
      cudaFuncSetAttribute(k_fused2<TX, TY, PLAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return e;
  }
  const dim3 grid((unsigned)(g.n[0] / TX), (unsigned)(g.n[1] / TY), (unsigned)(g.n[2] / ZC));
  k_fused2<TX, TY, PLAIN><<<grid, TX * TY / 2, smem, st>>>(g, K, make_coef_pair(K), a, ZC);
  return cudaGetLastError();
}

// The common configuration (an unforced AB2 step that updates the state, in
// the total-energy form with the power-law viscosity) runs the kernel
// compiled for it alone; every other configuration runs the general one.
template <int TX, int TY>
static cudaError_t run_fused2(const Geom& g, const Coef<float>& K, const StepArgs<float>& a, int ZC,
                              cudaStream_t st) {
  const bool plain = !K.eform && !K.vlaw && !a.fB && !a.rk && a.do_update && !a.Rout;
  return plain ? run_fused2_as<TX, TY, true>(g, K, a, ZC, st) : run_fused2_as<TX, TY, false>(g, K, a, ZC, st);
}

cudaError_t launch_fused2(const Geom& g, const Coef<float>& K, const StepArgs<float>& a, int TX, int TY, int ZC,
                          cudaStream_t st) {
  if (TX == 32 && TY == 8) return run_fused2<32, 8>(g, K, a, ZC, st);
  if (TX == 32 && TY == 16) return run_fused2<32, 16>(g, K, a, ZC, st);
  if (TX == 16 && TY == 16) return run_fused2<16, 16>(g, K, a, ZC, st);
  if (TX == 16 && TY == 8) return run_fused2<16, 8>(g, K, a, ZC, st);
  return cudaErrorInvalidValue;
}

}  // namespace atdns
