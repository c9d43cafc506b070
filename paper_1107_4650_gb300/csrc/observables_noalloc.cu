// dirac_observables_noalloc: the observables reduction for a state in caller-owned device memory,
// with its block partials kept in a fixed file-scope device array instead of memory allocated per
// grid.  It serves callers that cannot allocate device memory themselves: for example a host
// framework that owns the whole device budget through its own pool, or a latency-critical loop that
// must not pay the device synchronisation cudaMalloc/cudaFree can imply.  It calls no cudaMalloc,
// cudaFree or other allocating routine.
//
// Scratch: kNoAllocMaxBlocks x 5 doubles (640 KiB), held by every device that loads the library
// until the process exits.  Each block reduces a fixed run of kNoAllocCellsPerBlock cells, so the
// summation order does not depend on the device; grids above kNoAllocMaxBlocks x
// kNoAllocCellsPerBlock cells are rejected with DIRAC_ERR_ARG.  Every call writes the partials it
// reads, so nothing needs clearing between calls, but all calls share the one array: calls whose
// kernels overlap on the GPU (different streams, or different host threads) race on it.  The result is
// written to the caller's device buffer asynchronously, so the call cannot report a non-finite state:
// a state holding NaN or Inf gives a NaN or Inf norm in out[0], which the caller checks.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/dirac.h"
#include "dirac_internal.cuh"

namespace dirac {

dirac_status set_thread_error(dirac_status st, const std::string &msg);  // dirac_api.cu

namespace {

constexpr int kNoAllocThreads = 256;
constexpr int64_t kNoAllocCellsPerBlock = DIRAC_NOALLOC_CELLS_PER_BLOCK;
constexpr int64_t kNoAllocMaxBlocks = DIRAC_NOALLOC_MAX_BLOCKS;
constexpr int kMaxDevices = 64;

// Device-side scratch.  Host code must not pass this symbol to a kernel (on the host it names a
// stand-in, not a device address); the per-device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks * 5];

std::mutex g_setup_mutex;
double *g_partials_addr[kMaxDevices] = {};

__device__ __forceinline__ double abs2_na(double re, double im) {
    return __dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im));
}

__device__ __forceinline__ void block_sum5_na(double v[5], double *sh) {
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

// Block b sums cells [b * kNoAllocCellsPerBlock, (b+1) * kNoAllocCellsPerBlock) into partials[b*5 .. b*5+4]:
// rho, rho right of the face, x rho, y rho, z rho.
template <typename T>
__global__ void __launch_bounds__(kNoAllocThreads) noalloc_partial_kernel(const T *psi, int64_t nx, int64_t ny,
                                                                           int64_t N, double dx, double x0, double y0,
                                                                           double z0, int64_t face, double *partials) {
    __shared__ double sh[32 * 5];
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const int64_t begin = (int64_t)blockIdx.x * kNoAllocCellsPerBlock;
    const int64_t end = min(begin + kNoAllocCellsPerBlock, N);
    for (int64_t idx = begin + threadIdx.x; idx < end; idx += blockDim.x) {
        const T *p = psi + idx * 8;
        double rho = abs2_na((double)p[0], (double)p[1]);
        rho = __dadd_rn(rho, abs2_na((double)p[2], (double)p[3]));
        rho = __dadd_rn(rho, abs2_na((double)p[4], (double)p[5]));
        rho = __dadd_rn(rho, abs2_na((double)p[6], (double)p[7]));
        const int64_t i = idx % nx;
        const int64_t t = idx / nx;
        const int64_t j = t % ny;
        const int64_t k = t / ny;
        v[0] = __dadd_rn(v[0], rho);
        if (face >= 0 && i >= face) v[1] = __dadd_rn(v[1], rho);
        v[2] = __dadd_rn(v[2], __dmul_rn(__dadd_rn(x0, __dmul_rn((double)i, dx)), rho));
        v[3] = __dadd_rn(v[3], __dmul_rn(__dadd_rn(y0, __dmul_rn((double)j, dx)), rho));
        v[4] = __dadd_rn(v[4], __dmul_rn(__dadd_rn(z0, __dmul_rn((double)k, dx)), rho));
    }
    block_sum5_na(v, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 5; ++k) partials[blockIdx.x * 5 + k] = v[k];
}

// Folds the first nblocks partials in a fixed order; out = {norm, norm_right, cx, cy, cz}.
__global__ void __launch_bounds__(kNoAllocThreads) noalloc_final_kernel(const double *partials, int64_t nblocks,
                                                                         double vol, double *out) {
    __shared__ double sh[32 * 5];
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < 5; ++k) v[k] = __dadd_rn(v[k], partials[b * 5 + k]);
    block_sum5_na(v, sh);
    if (threadIdx.x == 0) {
        const double s = v[0];
        out[0] = __dmul_rn(s, vol);
        out[1] = __dmul_rn(v[1], vol);
        out[2] = s > 0.0 ? __ddiv_rn(v[2], s) : 0.0;
        out[3] = s > 0.0 ? __ddiv_rn(v[3], s) : 0.0;
        out[4] = s > 0.0 ? __ddiv_rn(v[4], s) : 0.0;
    }
}

// Device address of the scratch array on the current device.  Outside a stream capture it is looked up
// (cudaGetSymbolAddress, a host call that allocates nothing) on every call and recorded for the device, so a
// module reloaded at another address after cudaDeviceReset or a new primary context is picked up at once.
// Inside a capture the recorded address is used: the first call on a device must come before any capture.
cudaError_t partials_address(cudaStream_t s, double **addr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_partials_addr[dev] = static_cast<double *>(p);
    } else if (!g_partials_addr[dev]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *addr = g_partials_addr[dev];
    return cudaSuccess;
}

}  // namespace

}  // namespace dirac

extern "C" dirac_status dirac_observables_noalloc(const void *psi, int precision, int ndim, const int64_t n[3],
                                                  double dx, const double x_min[3], int64_t flux_face, void *stream,
                                                  double *out) {
    using namespace dirac;
    if (!psi || !n || !x_min || !out) return set_thread_error(DIRAC_ERR_ARG, "dirac_observables_noalloc: null argument");
    if (precision != DIRAC_FP64 && precision != DIRAC_FP32)
        return set_thread_error(DIRAC_ERR_ARG, "dirac_observables_noalloc: precision must be DIRAC_FP64 or DIRAC_FP32");
    if (ndim != 2 && ndim != 3) return set_thread_error(DIRAC_ERR_ARG, "dirac_observables_noalloc: ndim must be 2 or 3");
    if (n[0] < 1 || n[1] < 1 || n[2] < 1 || (ndim == 2 && n[1] != 1))
        return set_thread_error(DIRAC_ERR_ARG, "dirac_observables_noalloc: bad grid sizes");
    if (!(dx > 0)) return set_thread_error(DIRAC_ERR_ARG, "dirac_observables_noalloc: dx must be > 0");
    const double cells = (double)n[0] * (double)n[1] * (double)n[2];
    if (cells > (double)(kNoAllocMaxBlocks * kNoAllocCellsPerBlock))
        return set_thread_error(DIRAC_ERR_ARG,
                                "dirac_observables_noalloc: grid of " + std::to_string((long long)cells) +
                                    " cells exceeds the fixed scratch limit of " +
                                    std::to_string((long long)(kNoAllocMaxBlocks * kNoAllocCellsPerBlock)) +
                                    " cells (" + std::to_string((long long)kNoAllocMaxBlocks) + " blocks of " +
                                    std::to_string((long long)kNoAllocCellsPerBlock) + "); use dirac_observables");
    const int64_t N = n[0] * n[1] * n[2];
    const int64_t nblocks = (N + kNoAllocCellsPerBlock - 1) / kNoAllocCellsPerBlock;
    double *partials = nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = partials_address(s, &partials);
    if (e != cudaSuccess)
        return set_thread_error(DIRAC_ERR_CUDA, std::string("dirac_observables_noalloc: cudaGetSymbolAddress: ") +
                                                    cudaGetErrorString(e) +
                                                    " (inside a stream capture the first call on a device must come first)");
    const double x0 = x_min[0] + 0.5 * dx, y0 = x_min[1] + 0.5 * dx, z0 = x_min[2] + 0.5 * dx;
    if (precision == DIRAC_FP32)
        noalloc_partial_kernel<float><<<(unsigned)nblocks, kNoAllocThreads, 0, s>>>(
            static_cast<const float *>(psi), n[0], n[1], N, dx, x0, y0, z0, flux_face, partials);
    else
        noalloc_partial_kernel<double><<<(unsigned)nblocks, kNoAllocThreads, 0, s>>>(
            static_cast<const double *>(psi), n[0], n[1], N, dx, x0, y0, z0, flux_face, partials);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        const double vol = (ndim == 3) ? dx * dx * dx : dx * dx;
        noalloc_final_kernel<<<1, kNoAllocThreads, 0, s>>>(partials, nblocks, vol, out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return set_thread_error(DIRAC_ERR_CUDA, std::string("dirac_observables_noalloc: launch: ") + cudaGetErrorString(e));
    return DIRAC_OK;
}
