// Arithmetic issue-rate probe: the denominators of the ALU roofline the FP64 step kernels are held to.
// Every thread runs 8 independent dependency chains of DFMA, DADD, FFMA or FADD in registers (enough
// independent work per SM to hide the pipe latency) and stores one sum, so the timed launch is pure
// issue.  Prints lane-instructions per second and per SM per clock at the device's maximum SM clock.
#include <cstdio>
#include <cuda_runtime.h>

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
    const cudaError_t e = cudaGetLastError();
    std::printf("{\"sms\": %d, \"clock_hz\": %.4e, \"status\": \"%s\"}\n", sms, clk, cudaGetErrorString(e));
    return e == cudaSuccess ? 0 : 1;
}
