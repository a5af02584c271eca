// Launcher of the persistent batched step (cooperative launch).
#include "kernels_batch.cuh"

namespace atdns {

template <int TX, int TY>
static cudaError_t batch_prepare(int* ctas) {
  const size_t smem = fused_smem_bytes<float>(TX, TY);
  cudaError_t e = cudaFuncSetAttribute(k_batch_step<TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_step<TX, TY>, TX * TY / 2, smem)) != cudaSuccess)
    return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  *ctas = per_sm * sms;
  return per_sm > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

cudaError_t batch_resident_ctas(int TX, int TY, int* ctas) {
  if (TX == 16 && TY == 16) return batch_prepare<16, 16>(ctas);
  if (TX == 32 && TY == 8) return batch_prepare<32, 8>(ctas);
  return cudaErrorInvalidValue;
}

cudaError_t upload_batch_tiles(const TileDesc* desc, const int (*shape)[4], const long long* ghost_prefix,
                               const long long* tile_prefix, int count, cudaStream_t st) {
  if (count < 1 || count > kBatchConstMembers) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemcpyToSymbolAsync(c_tiles, desc, count * sizeof(TileDesc), 0, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyToSymbolAsync(c_shape, shape, count * sizeof(int[4]), 0, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyToSymbolAsync(c_gitems, ghost_prefix, (count + 1) * sizeof(long long), 0, cudaMemcpyHostToDevice,
                                st);
  if (e == cudaSuccess)
    e = cudaMemcpyToSymbolAsync(c_items, tile_prefix, (count + 1) * sizeof(long long), 0, cudaMemcpyHostToDevice, st);
  return e;
}

template <int TX, int TY>
static cudaError_t batch_launch(const BatchSched& S, int ctas, cudaStream_t st) {
  const size_t smem = fused_smem_bytes<float>(TX, TY);
  BatchSched arg = S;
  void* args[] = {&arg};
  return cudaLaunchCooperativeKernel((const void*)k_batch_step<TX, TY>, dim3((unsigned)ctas), dim3(TX * TY / 2), args,
                                     smem, st);
}

cudaError_t batch_wait_selftest(int log2_polls, int* gave_up) {
  unsigned* ctr = nullptr;
  int* out = nullptr;
  cudaError_t e = cudaMalloc(&ctr, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(ctr, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(out, 0xff, sizeof(int));
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 32>>>(ctr, 1LL << log2_polls, out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(gave_up, out, sizeof(int), cudaMemcpyDeviceToHost);
  if (ctr) cudaFree(ctr);
  if (out) cudaFree(out);
  return e;
}

cudaError_t launch_batch_step(int TX, int TY, const BatchSched& S, int ctas, cudaStream_t st) {
  if (TX == 16 && TY == 16) return batch_launch<16, 16>(S, ctas, st);
  if (TX == 32 && TY == 8) return batch_launch<32, 8>(S, ctas, st);
  return cudaErrorInvalidValue;
}

}  // namespace atdns
