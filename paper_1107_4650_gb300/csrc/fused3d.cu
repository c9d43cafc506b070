// Instantiations of the fused 3-D step kernels: one step per pass (8 or 16 warps per block: 6 or 14 owned
// rows per tile) and two steps per pass (FP32: 16 warps, 12 owned rows; FP64: 8 warps, 4 owned rows), with
// and without a uniform vector potential.
#include "fused3d_kernels.cuh"

namespace dirac {

cudaError_t launch_fused3d(const SweepArgs &a, int precision, int warps, int steps, int64_t ny, int64_t nz,
                           int64_t nstrips, int64_t nytiles, int64_t nzsegs, int64_t zseg_h, cudaStream_t s) {
    const int fp32 = precision == 1;
    Fused3DArgs A{};
    A.s = a;
    A.ny = ny;
    A.nz = nz;
    A.nstrips = nstrips;
    A.nytiles = nytiles;
    A.nzsegs = nzsegs;
    A.zseg_h = zseg_h;
    const bool field = a.ucoef != nullptr && a.ucoef_n > 0;
    if (precision == 2) {  // 64-bit fixed point: one step per pass, no vector potential
        if (steps != 1 || field) return cudaErrorInvalidValue;
        if (warps == 16) return launch_fused3d_one<long long, 16, false>(A, s);
        if (warps == 8) return launch_fused3d_one<long long, 8, false>(A, s);
        return cudaErrorInvalidValue;
    }
    if (steps == 2) {
        // two steps per pass: FP32 with 16-warp blocks, FP64 with 8 (its register budget)
        if (fp32 && warps == 16)
            return field ? launch_fused3d2_one<float, 16, true>(A, s) : launch_fused3d2_one<float, 16, false>(A, s);
        if (!fp32 && warps == 8)
            return field ? launch_fused3d2_one<double, 8, true>(A, s) : launch_fused3d2_one<double, 8, false>(A, s);
        return cudaErrorInvalidValue;
    }
    if (steps != 1) return cudaErrorInvalidValue;
    if (field) {
        if (warps == 16) return fp32 ? launch_fused3d_one<float, 16, true>(A, s) : launch_fused3d_one<double, 16, true>(A, s);
        if (warps == 8) return fp32 ? launch_fused3d_one<float, 8, true>(A, s) : launch_fused3d_one<double, 8, true>(A, s);
    } else {
        if (warps == 16) return fp32 ? launch_fused3d_one<float, 16, false>(A, s) : launch_fused3d_one<double, 16, false>(A, s);
        if (warps == 8) return fp32 ? launch_fused3d_one<float, 8, false>(A, s) : launch_fused3d_one<double, 8, false>(A, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dirac
