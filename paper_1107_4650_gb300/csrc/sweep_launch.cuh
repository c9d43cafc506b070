// Launcher body shared by the FP64 and FP32 instantiation units.
#pragma once
#include "step_kernels.cuh"

namespace dirac {

template <typename T, int K, int P, int MODE>
static cudaError_t launch_one(const SweepArgs &a, int wpb, cudaStream_t s) {
    const int64_t warps = a.nstrips * a.nsegs * a.nplanes;
    const int64_t blocks = (warps + wpb - 1) / wpb;
    if (blocks <= 0) return cudaSuccess;
    const int smem = ring_smem_bytes<T, Levels<K, MODE>::value, P, HistSmem<T, K, P, MODE>::value>(wpb);
    // opt in to > 48 KB of dynamic shared memory, once per device and block size
    static std::atomic<unsigned long long> done[4];
    const int slot = (wpb == 4) ? 0 : (wpb == 2) ? 1 : (wpb == 8) ? 2 : 3;
    if (slot == 3) done[3].store(0, std::memory_order_relaxed);  // other block sizes: every launch
    cudaError_t e = optin_smem(sweep_kernel<T, K, P, MODE>, smem, done[slot]);
    if (e != cudaSuccess) return e;
    sweep_kernel<T, K, P, MODE><<<(unsigned)blocks, 32 * wpb, smem, s>>>(a);
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
