// Internal launchers of the batched-ensemble kernels (batch.cu), used by batch_api.cu.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dirac {
struct BatchArgs;
struct InitArgs;
struct NormArgs;
bool batch_supported(int fp32, int K, int P);
cudaError_t launch_batch(const BatchArgs &b, int fp32, int K, int P, int blocks, cudaStream_t s);
cudaError_t batch_occupancy(int fp32, int K, int P, int *blocks_per_sm);
cudaError_t launch_batch_init(const InitArgs &ia, int fp32, cudaStream_t s);
cudaError_t launch_batch_norm(const NormArgs &na, int64_t nchunks, const int64_t *chunk_off, int nruns, double vol,
                              double *norm, int fp32, cudaStream_t s);
}  // namespace dirac
