// Instantiations of the characteristic-shift step kernel (c dt = S dx, S = 2, 3, 4; with and without a uniform
// vector potential).
#include "shift_kernels.cuh"

namespace dirac {

template <typename T>
static cudaError_t launch_shift_t(const SweepArgs &a, int S, int P, int wpb, cudaStream_t s) {
    if (P == 2) {
        if (S == 2) return launch_shift_one<T, 2, 2>(a, wpb, s);
        if (S == 3) return launch_shift_one<T, 3, 2>(a, wpb, s);
        if (S == 4) return launch_shift_one<T, 4, 2>(a, wpb, s);
    } else if (P == 1) {
        if (S == 2) return launch_shift_one<T, 2, 1>(a, wpb, s);
        if (S == 3) return launch_shift_one<T, 3, 1>(a, wpb, s);
        if (S == 4) return launch_shift_one<T, 4, 1>(a, wpb, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_shift(const SweepArgs &a, int fp32, int S, int P, int wpb, cudaStream_t s) {
    return fp32 ? launch_shift_t<float>(a, S, P, wpb, s) : launch_shift_t<double>(a, S, P, wpb, s);
}

bool shift_supported(int S, int P) { return (S >= 2 && S <= 4) && (P == 1 || P == 2); }

}  // namespace dirac
