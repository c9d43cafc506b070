// FP64 instantiations of the fused sweep kernels.
#include "sweep_launch.cuh"

namespace dirac {

cudaError_t launch_sweep_f64(const SweepArgs &a, int mode, int K, int P, int wpb, cudaStream_t s) {
    if (mode == 0) {
        if (K == 1 && P == 1) return launch_one<double, 1, 1, 0>(a, wpb, s);
        if (K == 1 && P == 2) return launch_one<double, 1, 2, 0>(a, wpb, s);
        if (K == 1 && P == 4) return launch_one<double, 1, 4, 0>(a, wpb, s);
        if (K == 2 && P == 2) return launch_one<double, 2, 2, 0>(a, wpb, s);
    } else if (mode == 2) {
        if (K == 1 && P == 2) return launch_one<double, 1, 2, 2>(a, wpb, s);
        if (K == 1 && P == 1) return launch_one<double, 1, 1, 2>(a, wpb, s);
    } else if (mode == 5) {
        if (K == 1 && P == 1) return launch_one<double, 1, 1, 5>(a, wpb, s);
        if (K == 1 && P == 2) return launch_one<double, 1, 2, 5>(a, wpb, s);
    } else if (mode == 3) {
        if (K == 1 && P == 1) return launch_one<double, 1, 1, 3>(a, wpb, s);
        if (K == 1 && P == 2) return launch_one<double, 1, 2, 3>(a, wpb, s);
    } else {
        if (K == 1 && P == 1) return launch_one<double, 1, 1, 1>(a, wpb, s);
        if (K == 1 && P == 2) return launch_one<double, 1, 2, 1>(a, wpb, s);
        if (K == 1 && P == 4) return launch_one<double, 1, 4, 1>(a, wpb, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_zphase_f64(const ZArgs &a, int threads, cudaStream_t s) { return launch_zphase<double>(a, threads, s); }

}  // namespace dirac
