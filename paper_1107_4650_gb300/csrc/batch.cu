// Instantiations and launchers of the batched-ensemble kernels.
#include "batch_kernels.cuh"
#include "batch_internal.cuh"

namespace dirac {

namespace {
template <typename T, int K, int P>
cudaError_t launch_batch_t(const BatchArgs &b, int blocks, cudaStream_t s) {
    const int smem = ring_smem_bytes<T, K, P>(4);
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<T, K, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    batch_kernel<T, K, P><<<blocks, 128, smem, s>>>(b);
    return cudaGetLastError();
}
template <typename T, int K, int P>
cudaError_t occupancy_t(int *blocks_per_sm) {
    const int smem = ring_smem_bytes<T, K, P>(4);
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<T, K, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, batch_kernel<T, K, P>, 128, smem);
}
}  // namespace

#define DIRAC_BATCH_CASES(X)              \
    X(double, 1, 2) X(double, 1, 4) X(double, 2, 2) \
    X(float, 1, 2) X(float, 1, 4) X(float, 2, 2) X(float, 2, 4) X(float, 4, 2)

bool batch_supported(int fp32, int K, int P) {
#define X(T, k, p) if ((fp32 != 0) == (sizeof(T) == 4) && K == k && P == p) return true;
    DIRAC_BATCH_CASES(X)
#undef X
    return false;
}

cudaError_t launch_batch(const BatchArgs &b, int fp32, int K, int P, int blocks, cudaStream_t s) {
#define X(T, k, p) if ((fp32 != 0) == (sizeof(T) == 4) && K == k && P == p) return launch_batch_t<T, k, p>(b, blocks, s);
    DIRAC_BATCH_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t batch_occupancy(int fp32, int K, int P, int *blocks_per_sm) {
#define X(T, k, p) if ((fp32 != 0) == (sizeof(T) == 4) && K == k && P == p) return occupancy_t<T, k, p>(blocks_per_sm);
    DIRAC_BATCH_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch_init(const InitArgs &ia, int fp32, cudaStream_t s) {
    const int blocks = 152 * 8;
    if (fp32) batch_init_kernel<float><<<blocks, 256, 0, s>>>(ia);
    else batch_init_kernel<double><<<blocks, 256, 0, s>>>(ia);
    return cudaGetLastError();
}

cudaError_t launch_batch_norm(const NormArgs &na, int64_t nchunks, const int64_t *chunk_off, int nruns, double vol,
                              double *norm, int fp32, cudaStream_t s) {
    if (nchunks <= 0) return cudaSuccess;
    if (fp32) batch_norm_partial_kernel<float><<<(unsigned)nchunks, 256, 0, s>>>(na);
    else batch_norm_partial_kernel<double><<<(unsigned)nchunks, 256, 0, s>>>(na);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    batch_norm_fold_kernel<<<(nruns + 127) / 128, 128, 0, s>>>(chunk_off, nruns, na.partial, vol, norm);
    return cudaGetLastError();
}

}  // namespace dirac
