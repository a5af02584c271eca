// Launchers of the templated step kernels; each precision is instantiated in
// its own translation unit (kernels_p64.cu, kernels_p32.cu).
#pragma once
#include "common.cuh"

namespace atdns {

constexpr int kBlock = 256;

template <typename S>
cudaError_t launch_prim(const Geom& g, const Coef<S>& K, const S* U0, const S* U1, const DevState* ds, S* PQ,
                        cudaStream_t st);

template <typename S>
cudaError_t launch_ghost(const Geom& g, const Coef<S>& K, const S* U0, const S* U1, const DevState* ds,
                         const S* PQ, S* const GH[3],
                         S* const ring[3], const uint8_t* dmap, long long n, cudaStream_t st);

template <typename S>
cudaError_t launch_grad(const Geom& g, const Coef<S>& K, const S* PQ, S* const GH[3], S* G, cudaStream_t st);

template <typename S>
cudaError_t launch_main(const Geom& g, const Coef<S>& K, const StepArgs<S>& a, cudaStream_t st);

// Fused single-pass step kernel on TX x TY tiles marching ZC planes in z.
template <typename S>
cudaError_t launch_fused(const Geom& g, const Coef<S>& K, const StepArgs<S>& a, int TX, int TY, int ZC,
                         cudaStream_t st);

// Number of blocks k_main is launched with (size of the partial-sum array).
inline long long main_blocks(const Geom& g) { return (g.npts + kBlock - 1) / kBlock; }

}  // namespace atdns
