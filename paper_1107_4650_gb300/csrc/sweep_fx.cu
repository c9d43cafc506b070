// 64-bit fixed-point instantiations of the step kernels (storage DIRAC_FX64: the 2-D step, and the 3-D x-y
// pass and z/phase pass) and the state conversions.
//
// The state is q = round(psi 2^S) in int64 with S chosen from the state's discrete L2 norm A (the square
// root of the sum of |psi_c|^2 over all cells and components): each sweep with its 1/2 and the phase are
// contractions in that norm, so a component after j sweeps without the 1/2 is at most 2^j A; with
// A 2^S < 2^60 in 2-D (2^59 in 3-D) every value of a step stays below 2^62 and every sum of two
// components below 2^62.5.  The sweeps then add exactly; the phase (Eq. sol_dis_4, coefficients
// round(p 2^62) carrying the sweeps' 1/4, or 1/8) rounds each output component once.
#include "sweep_launch.cuh"

namespace dirac {

cudaError_t launch_sweep_fx(const SweepArgs &a, int mode, int K, int P, int wpb, cudaStream_t s) {
    if (mode == 0) {
        if (K == 1 && P == 1) return launch_one<long long, 1, 1, 0>(a, wpb, s);
        if (K == 1 && P == 2) return launch_one<long long, 1, 2, 0>(a, wpb, s);
        if (K == 1 && P == 4) return launch_one<long long, 1, 4, 0>(a, wpb, s);
        if (K == 2 && P == 2) return launch_one<long long, 2, 2, 0>(a, wpb, s);
    } else if (mode == 2) {  // 2-D second-order step
        if (K == 1 && P == 1) return launch_one<long long, 1, 1, 2>(a, wpb, s);
        if (K == 1 && P == 2) return launch_one<long long, 1, 2, 2>(a, wpb, s);
    } else if (mode == 1) {  // 3-D x-y pass (the z sweep and phase follow in launch_zphase_fx)
        if (K == 1 && P == 1) return launch_one<long long, 1, 1, 1>(a, wpb, s);
        if (K == 1 && P == 2) return launch_one<long long, 1, 2, 1>(a, wpb, s);
        if (K == 1 && P == 4) return launch_one<long long, 1, 4, 1>(a, wpb, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_zphase_fx(const ZArgs &a, int threads, cudaStream_t s) { return launch_zphase<long long>(a, threads, s); }

bool sweep_supported_fx(int mode, int K, int P) {
    if (mode == 1) return K == 1 && (P == 1 || P == 2 || P == 4);
    if (mode == 2) return K == 1 && (P == 1 || P == 2);
    return mode == 0 && ((K == 1 && (P == 1 || P == 2 || P == 4)) || (K == 2 && P == 2));
}

namespace {

__global__ void fx_encode_kernel(const double *x, long long *q, int64_t n, int S) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        q[i] = __double2ll_rn(scalbn(x[i], S));
}

__global__ void fx_decode_kernel(const long long *q, double *x, int64_t n, int S) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = scalbn(__ll2double_rn(q[i]), -S);
}

unsigned grid_for(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

cudaError_t launch_fx_encode(const double *x, long long *q, int64_t n, int S, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    fx_encode_kernel<<<grid_for(n), 256, 0, s>>>(x, q, n, S);
    return cudaGetLastError();
}

cudaError_t launch_fx_decode(const long long *q, double *x, int64_t n, int S, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    fx_decode_kernel<<<grid_for(n), 256, 0, s>>>(q, x, n, S);
    return cudaGetLastError();
}

}  // namespace dirac
