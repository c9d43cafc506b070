// Launcher body shared by the FP64 and FP32 instantiation units.
#pragma once
#include "step_kernels.cuh"

namespace dirac {

template <typename T, int K, int P, int MODE>
static cudaError_t launch_one(const SweepArgs &a, int wpb, cudaStream_t s) {
    const int64_t warps = a.nstrips * a.nsegs * a.nplanes;
    const int64_t blocks = (warps + wpb - 1) / wpb;
    if (blocks <= 0) return cudaSuccess;
    sweep_kernel<T, K, P, MODE><<<(unsigned)blocks, 32 * wpb, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_zphase(const ZArgs &a, int threads, cudaStream_t s) {
    const int64_t n = a.nx * a.ny * a.nsegs;
    const int64_t blocks = (n + threads - 1) / threads;
    if (blocks <= 0) return cudaSuccess;
    zphase_kernel<T><<<(unsigned)blocks, threads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace dirac
