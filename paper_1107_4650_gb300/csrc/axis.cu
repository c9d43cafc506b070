// Launchers of the single-sweep kernels used by the 3-D second-order step.
#include "axis_kernels.cuh"

namespace dirac {

// the phase-matrix variant exists for floating-point states only
template <typename T> static void launch_axis_field(const AxisArgs &a, int blocks, cudaStream_t s) {
    axis_kernel<T, 2, true, 1><<<blocks, 256, 0, s>>>(a);
}
template <> void launch_axis_field<long long>(const AxisArgs &, int, cudaStream_t) {}

template <typename T>
static cudaError_t launch_axis_t(const AxisArgs &a, int axis, int phase, int blocks, cudaStream_t s) {
    const bool field = a.ucoef != nullptr && a.ucoef_n > 0;
    if (sizeof(T) == 8 && (T)0.5 == (T)0 && field) return cudaErrorInvalidValue;  // fixed point: no phase matrix
    if (axis == 0 && !phase) axis_kernel<T, 0, false, 0><<<blocks, 256, 0, s>>>(a);
    else if (axis == 1 && !phase) axis_kernel<T, 1, false, 0><<<blocks, 256, 0, s>>>(a);
    else if (axis == 2 && !phase) axis_kernel<T, 2, false, 0><<<blocks, 256, 0, s>>>(a);
    else if (axis == 2 && phase && !field) axis_kernel<T, 2, true, 0><<<blocks, 256, 0, s>>>(a);
    else if (axis == 2 && phase && field) launch_axis_field<T>(a, blocks, s);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_axis_cellfield(const AxisArgs &a, int precision, int blocks, cudaStream_t s) {
    if (precision == 1)
        axis_kernel<float, 2, true, 2><<<blocks, 256, 0, s>>>(a);
    else if (precision == 0)
        axis_kernel<double, 2, true, 2><<<blocks, 256, 0, s>>>(a);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_axis(const void *in, void *out, const void *table, int64_t nx, int64_t ny, int64_t nz, int axis,
                        int64_t shift, int periodic, int full_table, int phase, int64_t flux_face, double fscale,
                        double vol, double *flux_part, double *flux_cum, unsigned *ticket, const double *ucoef,
                        int64_t ucoef_n, int64_t step0, int precision, int rshift, int blocks, cudaStream_t s) {
    AxisArgs a{};
    a.rshift = rshift;
    a.ucoef = ucoef;
    a.ucoef_n = ucoef_n;
    a.step0 = step0;
    a.in = in;
    a.out = out;
    a.table = table;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.shift = shift;
    a.periodic = periodic;
    a.full_table = full_table;
    a.flux_face = axis == 0 ? flux_face : -1;
    a.fscale = fscale;
    a.vol = vol;
    a.flux_part = flux_part;
    a.flux_cum = flux_cum;
    a.ticket = ticket;
    if (precision == 1) return launch_axis_t<float>(a, axis, phase, blocks, s);
    if (precision == 2) return launch_axis_t<long long>(a, axis, phase, blocks, s);
    return launch_axis_t<double>(a, axis, phase, blocks, s);
}

}  // namespace dirac
