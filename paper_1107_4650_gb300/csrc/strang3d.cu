// Instantiations of the fused passes of the 3-D second-order step: the x-y-x (half step) and x-y-x-x-y-x
// (two half steps) passes with 16 or 32 warps per block, the z-phase-z pass with and without a uniform
// vector potential; FP64, FP32 and 64-bit fixed-point states (fixed point: no vector potential).
#include "strang3d_kernels.cuh"

namespace dirac {

template <typename T>
static cudaError_t launch_strang_xy_t(const StrangXYArgs &A, int warps, int nh, cudaStream_t s) {
    if (nh == 1 && warps == 16) return launch_strang_xy_one<T, 16, 1>(A, s);
    if (nh == 1 && warps == 32) return launch_strang_xy_one<T, 32, 1>(A, s);
    if (nh == 2 && warps == 16) return launch_strang_xy_one<T, 16, 2>(A, s);
    if (nh == 2 && warps == 32) return launch_strang_xy_one<T, 32, 2>(A, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_strang_xy(const SweepArgs &a, int precision, int warps, int nh, int64_t ny, int64_t nz,
                             int64_t nstrips, int64_t nytiles, int64_t nzsegs, int64_t zseg_h, const double fscale[4],
                             int rshift_mid, int rshift_end, cudaStream_t s) {
    StrangXYArgs A{};
    A.s = a;
    A.ny = ny;
    A.nz = nz;
    A.nstrips = nstrips;
    A.nytiles = nytiles;
    A.nzsegs = nzsegs;
    A.zseg_h = zseg_h;
    for (int q = 0; q < 4; ++q) A.fscale[q] = fscale[q];
    A.rshift_mid = rshift_mid;
    A.rshift_end = rshift_end;
    if (precision == 1) return launch_strang_xy_t<float>(A, warps, nh, s);
    if (precision == 2) return launch_strang_xy_t<long long>(A, warps, nh, s);
    return launch_strang_xy_t<double>(A, warps, nh, s);
}

cudaError_t launch_strang_z(const void *in, void *out, const void *table, int64_t nx, int64_t ny, int64_t nz,
                            int periodic, int full_table, const double *ucoef, int64_t ucoef_n, int64_t step0,
                            int64_t nsegs, int64_t seg_h, int precision, cudaStream_t s) {
    StrangZArgs a{};
    a.in = in;
    a.out = out;
    a.table = table;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.seg_h = seg_h;
    a.periodic = periodic;
    a.full_table = full_table;
    a.ucoef = ucoef;
    a.ucoef_n = ucoef_n;
    a.step0 = step0;
    const bool field = ucoef != nullptr && ucoef_n > 0;
    if (precision == 2) return field ? cudaErrorInvalidValue : launch_strang_z_one<long long, false>(a, nsegs, s);
    const bool fp32 = precision == 1;
    if (field) return fp32 ? launch_strang_z_one<float, true>(a, nsegs, s) : launch_strang_z_one<double, true>(a, nsegs, s);
    return fp32 ? launch_strang_z_one<float, false>(a, nsegs, s) : launch_strang_z_one<double, false>(a, nsegs, s);
}

}  // namespace dirac
