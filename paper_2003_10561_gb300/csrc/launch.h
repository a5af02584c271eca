// Launchers of the templated step kernels.
#pragma once
#include "common.cuh"

namespace atdns {

constexpr int kBlock = 256;

template <typename S>
cudaError_t launch_prim(const Geom& g, const Coef<S>& K, const S* U0, const S* U1, const DevState* ds, S* PQ,
                        cudaStream_t st);

// The ghost, gradient and main kernels for stencil half width M (2: 4th
// order, 3: 6th order); each (S, M) pair is compiled in its own translation
// unit (kernels_p64.cu, kernels_p32.cu, kernels_p64_o6.cu, kernels_p32_o6.cu).
// The ghost kernel also writes level n of the state (FP64: the state, or the
// compensated form's hi + lo; Ulo0 / Ulo1 null otherwise) into the ring.
template <typename S, int M>
cudaError_t launch_ghost_m(const Geom& g, const Coef<S>& K, const S* U0, const S* U1, const S* Ulo0, const S* Ulo1,
                           const DevState* ds, const S* PQ, S* const GH[3], double* const ring[3], const S* xst,
                           long long xst_half, const uint8_t* dmap, long long n, cudaStream_t st);

template <typename S, int M>
cudaError_t launch_grad_m(const Geom& g, const Coef<S>& K, const S* PQ, S* const GH[3], S* G, cudaStream_t st);

template <typename S, int M>
cudaError_t launch_main_m(const Geom& g, const Coef<S>& K, const StepArgs<S>& a, cudaStream_t st);

template <typename S>
inline cudaError_t launch_ghost(const Geom& g, const Coef<S>& K, const S* U0, const S* U1, const S* Ulo0,
                                const S* Ulo1, const DevState* ds, const S* PQ, S* const GH[3],
                                double* const ring[3], const S* xst, long long xst_half, const uint8_t* dmap,
                                long long n, cudaStream_t st) {
  return g.M == 3 ? launch_ghost_m<S, 3>(g, K, U0, U1, Ulo0, Ulo1, ds, PQ, GH, ring, xst, xst_half, dmap, n, st)
                  : launch_ghost_m<S, 2>(g, K, U0, U1, Ulo0, Ulo1, ds, PQ, GH, ring, xst, xst_half, dmap, n, st);
}

template <typename S>
inline cudaError_t launch_grad(const Geom& g, const Coef<S>& K, const S* PQ, S* const GH[3], S* G, cudaStream_t st) {
  return g.M == 3 ? launch_grad_m<S, 3>(g, K, PQ, GH, G, st) : launch_grad_m<S, 2>(g, K, PQ, GH, G, st);
}

template <typename S>
inline cudaError_t launch_main(const Geom& g, const Coef<S>& K, const StepArgs<S>& a, cudaStream_t st) {
  return g.M == 3 ? launch_main_m<S, 3>(g, K, a, st) : launch_main_m<S, 2>(g, K, a, st);
}

// Fused single-pass step kernel on TX x TY tiles marching ZC planes in z.
template <typename S>
cudaError_t launch_fused(const Geom& g, const Coef<S>& K, const StepArgs<S>& a, int TX, int TY, int ZC,
                         cudaStream_t st);

// Paired fused step kernel (two x-adjacent points per thread, packed FP32
// arithmetic; FP32 forms only): tiles 32x8, 32x16, 16x16, 16x8.
cudaError_t launch_fused2(const Geom& g, const Coef<float>& K, const StepArgs<float>& a, int TX, int TY, int ZC,
                          cudaStream_t st);

// Number of blocks k_main is launched with (size of the partial-sum array).
inline long long main_blocks(const Geom& g) { return (g.npts + kBlock - 1) / kBlock; }

}  // namespace atdns
