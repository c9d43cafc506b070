// Arithmetic issue-rate probe: the denominators of the ALU roofline the FP64 step kernels are held to.
// Every thread runs 8 independent dependency chains of DFMA, DADD, FFMA or FADD in registers (enough
// independent work per SM to hide the pipe latency) and stores one sum, so the timed launch is pure
// issue.  Prints lane-instructions per second and per SM per clock at the device's maximum SM clock.
// Also: 64-bit integer adds (chains q += q of the neighbouring chain) and int64 <-> FP64 conversion pairs
// (q -> double -> q + 1), the operations of a fixed-point evaluation of the sweeps.  And binary64 additions
// on the integer units (iadd_rn), alone and interleaved with hardware DADD chains, to see whether the two
// pipes overlap.
#include <cstdio>
#include <cuda_runtime.h>

#include "iadd64.cuh"

namespace {

template <typename T, bool FMA>
__global__ void chains(T *out, int iters) {
    T a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = T(1e-3) * T(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (sizeof(T) == 8)
                a[k] = FMA ? (T)__fma_rn((double)a[k], 0.9999999, 1e-7) : (T)__dadd_rn((double)a[k], 1e-7);
            else
                a[k] = FMA ? (T)__fmaf_rn((float)a[k], 0.9999999f, 1e-7f) : (T)__fadd_rn((float)a[k], 1e-7f);
        }
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// OP 0: 64-bit integer add; OP 1: int64 -> FP64 -> int64 conversion pair (counted as two instructions)
template <int OP>
__global__ void int_chains(long long *out, int iters) {
    long long q[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) q[k] = (long long)(threadIdx.x + 1) * (k + 3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (OP == 0)
                q[k] += q[k ^ 1];
            else
                q[k] = __double2ll_rn(__ll2double_rn(q[k])) + 1;
        }
    }
    long long s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += q[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// ND hardware DADD chains and NS integer-unit addition chains per thread, interleaved
template <int ND, int NS>
__global__ void mixed_chains(double *out, int iters) {
    double a[ND > 0 ? ND : 1], b[NS > 0 ? NS : 1];
#pragma unroll
    for (int k = 0; k < ND; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
#pragma unroll
    for (int k = 0; k < NS; ++k) b[k] = 1.0 + 1e-3 * (threadIdx.x + 2 * k + 1);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < (ND > NS ? ND : NS); ++k) {
            if (k < ND) a[k] = __dadd_rn(a[k], 1e-7);
            if (k < NS) b[k] = dirac::iadd_rn(b[k], (k & 1) ? -3e-8 : 1e-7);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < ND; ++k) s += a[k];
#pragma unroll
    for (int k = 0; k < NS; ++k) s += b[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int ND, int NS>
double run_mixed(const char *name, int blocks, int threads, int iters, double sms, double clk_hz) {
    double *out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(double)) != cudaSuccess) return -1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {  // first launch is a warm-up
        cudaEventRecord(e0);
        mixed_chains<ND, NS><<<blocks, threads>>>(out, iters);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    const double adds = (double)blocks * threads * (double)(ND + NS) * iters;
    const double rate = adds / (best * 1e-3);
    std::printf("{\"op\": \"%s\", \"dadd_chains\": %d, \"int_unit_chains\": %d, \"ms\": %.4f, \"adds_per_s\": %.4e, "
                "\"adds_per_sm_per_clk\": %.3f}\n",
                name, ND, NS, best, rate, rate / (sms * clk_hz));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return rate;
}

template <int OP>
double run_int(const char *name, int blocks, int threads, int iters, double per_iter, double sms, double clk_hz) {
    long long *out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(long long)) != cudaSuccess) return -1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {  // first launch is a warm-up
        cudaEventRecord(e0);
        int_chains<OP><<<blocks, threads>>>(out, iters);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    const double instr = (double)blocks * threads * 8.0 * iters * per_iter;
    const double rate = instr / (best * 1e-3);
    std::printf("{\"op\": \"%s\", \"ms\": %.4f, \"lane_instr_per_s\": %.4e, \"per_sm_per_clk\": %.3f}\n", name, best, rate,
                rate / (sms * clk_hz));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return rate;
}

template <typename T, bool FMA>
double run(const char *name, int blocks, int threads, int iters, double sms, double clk_hz) {
    T *out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(T)) != cudaSuccess) return -1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {  // first launch is a warm-up
        cudaEventRecord(e0);
        chains<T, FMA><<<blocks, threads>>>(out, iters);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    const double instr = (double)blocks * threads * 8.0 * iters;
    const double rate = instr / (best * 1e-3);
    std::printf("{\"op\": \"%s\", \"ms\": %.4f, \"lane_instr_per_s\": %.4e, \"per_sm_per_clk\": %.3f}\n", name, best, rate,
                rate / (sms * clk_hz));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return rate;
}

}  // namespace

int main() {
    int sms = 0, clk_khz = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
    const double clk = clk_khz > 0 ? clk_khz * 1e3 : 2.07e9;
    const int threads = 256, blocks = sms * 8;
    run<double, true>("DFMA", blocks, threads, 4096, sms, clk);
    run<double, false>("DADD", blocks, threads, 4096, sms, clk);
    run<float, true>("FFMA", blocks, threads, 65536, sms, clk);
    run<float, false>("FADD", blocks, threads, 65536, sms, clk);
    run_int<0>("IADD64", blocks, threads, 16384, 1.0, sms, clk);
    run_int<1>("CVT_S64_F64_PAIR", blocks, threads, 1024, 2.0, sms, clk);
    run_mixed<8, 0>("ADD_MIX", blocks, threads, 1024, sms, clk);
    run_mixed<0, 8>("ADD_MIX", blocks, threads, 1024, sms, clk);
    run_mixed<8, 2>("ADD_MIX", blocks, threads, 1024, sms, clk);
    run_mixed<8, 4>("ADD_MIX", blocks, threads, 1024, sms, clk);
    run_mixed<8, 8>("ADD_MIX", blocks, threads, 1024, sms, clk);
    const cudaError_t e = cudaGetLastError();
    std::printf("{\"sms\": %d, \"clock_hz\": %.4e, \"status\": \"%s\"}\n", sms, clk, cudaGetErrorString(e));
    return e == cudaSuccess ? 0 : 1;
}
