// FP32-storage instantiations of the fused sweep kernels.
#include "sweep_launch.cuh"

namespace dirac {

cudaError_t launch_sweep_f32(const SweepArgs &a, int mode, int K, int P, int wpb, cudaStream_t s) {
    if (mode == 0) {
        if (K == 1 && P == 1) return launch_one<float, 1, 1, 0>(a, wpb, s);
        if (K == 1 && P == 2) return launch_one<float, 1, 2, 0>(a, wpb, s);
        if (K == 1 && P == 4) return launch_one<float, 1, 4, 0>(a, wpb, s);
        if (K == 2 && P == 2) return launch_one<float, 2, 2, 0>(a, wpb, s);
        if (K == 2 && P == 4) return launch_one<float, 2, 4, 0>(a, wpb, s);
        if (K == 4 && P == 2) return launch_one<float, 4, 2, 0>(a, wpb, s);
        if (K == 4 && P == 4) return launch_one<float, 4, 4, 0>(a, wpb, s);
    } else if (mode == 2) {
        if (K == 1 && P == 2) return launch_one<float, 1, 2, 2>(a, wpb, s);
        if (K == 1 && P == 4) return launch_one<float, 1, 4, 2>(a, wpb, s);
        if (K == 2 && P == 2) return launch_one<float, 2, 2, 2>(a, wpb, s);
        if (K == 1 && P == 1) return launch_one<float, 1, 1, 2>(a, wpb, s);
    } else if (mode == 5) {
        if (K == 1 && P == 1) return launch_one<float, 1, 1, 5>(a, wpb, s);
        if (K == 1 && P == 2) return launch_one<float, 1, 2, 5>(a, wpb, s);
    } else if (mode == 3) {
        if (K == 1 && P == 1) return launch_one<float, 1, 1, 3>(a, wpb, s);
        if (K == 1 && P == 2) return launch_one<float, 1, 2, 3>(a, wpb, s);
        if (K == 2 && P == 2) return launch_one<float, 2, 2, 3>(a, wpb, s);
    } else {
        if (K == 1 && P == 1) return launch_one<float, 1, 1, 1>(a, wpb, s);
        if (K == 1 && P == 2) return launch_one<float, 1, 2, 1>(a, wpb, s);
        if (K == 1 && P == 4) return launch_one<float, 1, 4, 1>(a, wpb, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_zphase_f32(const ZArgs &a, int threads, cudaStream_t s) { return launch_zphase<float>(a, threads, s); }

bool sweep_supported(int fp32, int mode, int K, int P) {
    if (mode == 1) return K == 1 && (P == 1 || P == 2 || P == 4);
    if (mode == 2) return (K == 1 && (P == 1 || P == 2 || (fp32 && P == 4))) || (fp32 && K == 2 && P == 2);
    if (mode == 3) return (K == 1 && (P == 1 || P == 2)) || (fp32 && K == 2 && P == 2);
    if (mode == 5) return K == 1 && (P == 1 || P == 2);
    if (K == 1) return P == 1 || P == 2 || P == 4;
    if (!fp32) return K == 2 && P == 2;
    if (K == 2) return P == 2 || P == 4;
    if (K == 4) return P == 2 || P == 4;
    return false;
}

}  // namespace dirac
