// Observables and face-flux accumulation (Sec. 5.2.1: R and T are integrals of |psi|^2).
// All sums are FP64 and deterministic: fixed grid size, fixed per-thread order, fixed trees.
#include "dirac_internal.cuh"

namespace dirac {

namespace {

constexpr int OBS_THREADS = 256;

__device__ __forceinline__ double abs2(double re, double im) { return __dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im)); }

template <typename T>
__device__ __forceinline__ double rho_at(const T *p, double) {
    double s = abs2((double)p[0], (double)p[1]);
    s = __dadd_rn(s, abs2((double)p[2], (double)p[3]));
    s = __dadd_rn(s, abs2((double)p[4], (double)p[5]));
    return __dadd_rn(s, abs2((double)p[6], (double)p[7]));
}
// fixed-point state: each component q scale (scale a power of two: exact)
__device__ __forceinline__ double rho_at(const long long *p, double sc) {
    double v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = __dmul_rn(__ll2double_rn(p[c]), sc);
    double s = abs2(v[0], v[1]);
    s = __dadd_rn(s, abs2(v[2], v[3]));
    s = __dadd_rn(s, abs2(v[4], v[5]));
    return __dadd_rn(s, abs2(v[6], v[7]));
}

// Sums v over the block into lane 0 of warp 0 in a fixed order.
__device__ __forceinline__ void block_sum5(double v[5], double *sh /* [32][5] */) {
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] = __dadd_rn(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 5; ++k) sh[warp * 5 + k] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            double x = lane < nw ? sh[lane * 5 + k] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x = __dadd_rn(x, __shfl_xor_sync(0xffffffffu, x, o));
            v[k] = x;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(OBS_THREADS) obs_partial_kernel(const ObsArgs a) {
    __shared__ double sh[32 * 5];
    const T *psi = static_cast<const T *>(a.psi);
    const int64_t N = a.nx * a.ny * a.nz;
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += (int64_t)gridDim.x * blockDim.x) {
        const double rho = rho_at(psi + idx * 8, a.scale);
        const int64_t i = idx % a.nx;
        const int64_t t = idx / a.nx;
        const int64_t j = t % a.ny;
        const int64_t k = t / a.ny;
        v[0] = __dadd_rn(v[0], rho);
        if (a.face >= 0 && i >= a.face) v[1] = __dadd_rn(v[1], rho);
        v[2] = __dadd_rn(v[2], __dmul_rn(__dadd_rn(a.x0, __dmul_rn((double)i, a.dx)), rho));
        v[3] = __dadd_rn(v[3], __dmul_rn(__dadd_rn(a.y0, __dmul_rn((double)j, a.dx)), rho));
        v[4] = __dadd_rn(v[4], __dmul_rn(__dadd_rn(a.z0, __dmul_rn((double)k, a.dx)), rho));
        if (a.density) a.density[idx] = rho;
    }
    block_sum5(v, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 5; ++k) a.partial[blockIdx.x * 5 + k] = v[k];
}

__global__ void __launch_bounds__(OBS_THREADS) obs_final_kernel(const double *partial, int nblocks, double *out) {
    __shared__ double sh[32 * 5];
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < 5; ++k) v[k] = __dadd_rn(v[k], partial[b * 5 + k]);
    block_sum5(v, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 5; ++k) out[k] = v[k];
}

}  // namespace

cudaError_t launch_observables(const ObsArgs &a, int precision, int nblocks, cudaStream_t s) {
    if (precision == 1)
        obs_partial_kernel<float><<<nblocks, OBS_THREADS, 0, s>>>(a);
    else if (precision == 2)
        obs_partial_kernel<long long><<<nblocks, OBS_THREADS, 0, s>>>(a);
    else
        obs_partial_kernel<double><<<nblocks, OBS_THREADS, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    obs_final_kernel<<<1, OBS_THREADS, 0, s>>>(a.partial, nblocks, a.out);
    return cudaGetLastError();
}

}  // namespace dirac
