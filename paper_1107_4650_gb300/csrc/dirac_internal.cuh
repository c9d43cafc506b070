// Internal declarations shared by the translation units of libdirac.
// Not part of the public ABI (that is include/dirac.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dirac {

// Arguments of the fused sweep kernels (step_kernels.cuh).
//
// The kernel treats the data as `nplanes` independent planes of `nr` rows of `nx` cells.
//   mode 0 (2-D step):   plane = the x-z grid, rows run along z; one launch runs K full steps
//                        (x sweep, z sweep, phase), the sweeps' 1/2 factors folded into the
//                        phase table as 1/4.
//   mode 3 (2-D step with a uniform vector potential): as mode 0 with the full phase matrix.
//   mode 4 (2-D step with characteristic shift S > 1): shift_kernels.cuh, one step per launch.
//   mode 1 (3-D, x-y):   planes = z slices, rows run along y; x sweep then y sweep, no phase,
//                        output left at 4x the swept state (exact scaling, no rounding).
// Each warp owns an x strip of `strip_w` cells and a segment of `seg_h` rows of one plane.
struct SweepArgs {
    const void *in;
    void *out;
    const void *table;     // mode 0: 4 values (pu.re, pu.im, pd.re, pd.im) per x column (full_table
                           //         = 0) or per cell (full_table = 1), element type = storage type
    int64_t nx, nr, nplanes;
    int64_t strip_w, nstrips, nsegs, seg_h;
    int64_t flux_face;     // x face index or -1
    double *flux_part;     // [K][nplanes*nsegs] per-step face-flux partial sums (unscaled)
    double *flux_cum;      // cumulative flux; the last block of a launch adds vol * (sum of each step)
    unsigned *ticket;      // block-completion counter, 0 between launches (the last block resets it)
    unsigned *err;         // set non-zero by a kernel whose bounded wait ran out
    double vol;            // cell volume dx^d
    int periodic;
    int full_table;
    // mode 3 (uniform vector potential): per-step entries of U (Sec. 2.3) as 6 complex values
    // (Dup, Ddn, Ez, -Ez, Ep, Em) = 12 doubles per step; level s of a launch uses step (step0 + s) mod ucoef_n
    const double *ucoef;
    int64_t ucoef_n;
    int64_t step0;
    // failure-detection test hook (DIRAC_INJECT_STALL): the launch's first warp makes its first row-copy
    // wait run out, so the kernel reports DIRAC_ERR_TIMEOUT through *err
    int inject_stall;
    // multiplies the face-flux sums: 1 for floating-point states, 2^-2S for a fixed-point state q = psi 2^S
    double flux_unit = 1.0;
};

// Arguments of the 3-D z-sweep + phase kernel: the input is 4x the x-y swept state, the table is
// pre-scaled by 1/8 so the output is the true state after a full step.
struct ZArgs {
    const void *in;
    void *out;
    const void *table;     // per x column (full_table = 0) or per cell (full_table = 1)
    int64_t nx, ny, nz;
    int64_t nsegs, seg_h;
    int periodic;
    int full_table;
};

// Arguments of the single-sweep kernels (axis_kernels.cuh): one sweep of the whole grid along one axis with
// the characteristics moved `shift` cells, optionally followed by the phase.
struct AxisArgs {
    const void *in;
    void *out;
    const void *table;   // phase epilogue: (pu, pd) per x column or per cell, pre-scaled
    int64_t nx, ny, nz;
    int64_t shift;
    int periodic;
    int full_table;
    int64_t flux_face;   // x sweeps: face index, or -1
    double fscale;       // multiplies the summed |.|^2 of the face cells
    double vol;          // cell volume
    double *flux_part;   // [gridDim.x]
    double *flux_cum;
    unsigned *ticket;
    // uniform vector potential (phase epilogue only): 12 doubles of U entries per step, this launch's step
    const double *ucoef;
    int64_t ucoef_n, step0;
    // fixed-point states: the output divided by 2^rshift, rounded to nearest (halves up); 0 = none
    int rshift;
    // field varying in space and time (phase epilogue of the cell-field plan): profiles a (3 per cell) and w (1 per
    // cell), V dt per cell (fvdt_full) or per x column, absorber per x column (each nullable), this step's envelope
    // integrals F = (F_x, F_y, F_z, F_V), mu = m c^2 dt and the power-of-two scale of the sweeps' halves
    const double *fa, *fw, *fvdt, *fabs;
    int fvdt_full;
    double fenv[4];
    double fmu, fscale_phase;
};
// The z sweep with the cell-field phase epilogue (precision DIRAC_FP64 or DIRAC_FP32).
cudaError_t launch_axis_cellfield(const AxisArgs &a, int precision, int blocks, cudaStream_t s);

// Launchers: return cudaErrorInvalidValue for an unsupported (K, P) pair.
cudaError_t launch_sweep_f64(const SweepArgs &a, int mode, int K, int P, int warps_per_block, cudaStream_t s);
cudaError_t launch_sweep_f32(const SweepArgs &a, int mode, int K, int P, int warps_per_block, cudaStream_t s);
// 64-bit fixed-point state (DIRAC_FX64): mode 0 (2-D step) and mode 1 (3-D x-y pass) with the z/phase pass
cudaError_t launch_sweep_fx(const SweepArgs &a, int mode, int K, int P, int warps_per_block, cudaStream_t s);
cudaError_t launch_zphase_fx(const ZArgs &a, int threads, cudaStream_t s);
bool sweep_supported_fx(int mode, int K, int P);
// Fixed-point state conversion: q[i] = round-to-nearest-even(x[i] 2^S), and x[i] = q[i] 2^-S (n values each)
cudaError_t launch_fx_encode(const double *x, long long *q, int64_t n, int S, cudaStream_t s);
cudaError_t launch_fx_decode(const long long *q, double *x, int64_t n, int S, cudaStream_t s);
cudaError_t launch_zphase_f64(const ZArgs &a, int threads, cudaStream_t s);
cudaError_t launch_zphase_f32(const ZArgs &a, int threads, cudaStream_t s);

// Observables: per-block FP64 partial sums of (rho, rho right of face, x rho, y rho, z rho) over the
// grid, then one block folds the partials in a fixed order into out[5].  rho per cell is written to
// density when non-null.
struct ObsArgs {
    const void *psi;
    double scale;           // fixed-point state: psi = q scale (unused for floating-point states)
    int64_t nx, ny, nz;
    double dx, x0, y0, z0;  // x0 = x_min + dx/2 etc. (first cell centre)
    int64_t face;
    double *density;
    double *partial;        // [nblocks][5]
    double *out;            // [5]
};
// precision: DIRAC_FP64, DIRAC_FP32 or DIRAC_FX64 (the state then is int64 q, psi = q * a.scale)
cudaError_t launch_observables(const ObsArgs &a, int precision, int nblocks, cudaStream_t s);

// Instantiated (K, P) pairs of the sweep kernels.
bool sweep_supported(int fp32, int mode, int K, int P);

// Characteristic-shift step kernel (mode 4: 2-D first-order step with c dt = S dx, one step per launch,
// strips of 32 P - 2 S owned cells); S in 2..4, P in {1, 2}.
cudaError_t launch_shift(const SweepArgs &a, int fp32, int S, int P, int warps_per_block, cudaStream_t s);
bool shift_supported(int S, int P);

// One sweep of the whole grid along `axis` with the characteristics moved `shift` cells (output 2x the
// swept state), optionally followed by the phase from `table` (z sweeps only); x sweeps accumulate the face
// flux scaled by fscale when flux_face >= 0 (parts: one per block).  Used by the 3-D second-order step.
// With ucoef (12 doubles per step, ucoef_n steps) the phase is the vector-potential matrix of step step0.
// precision: DIRAC_FP64, DIRAC_FP32 or DIRAC_FX64 (int64 state; no vector potential; rshift > 0 divides the
// output by 2^rshift with rounding to nearest, halves up).
cudaError_t launch_axis(const void *in, void *out, const void *table, int64_t nx, int64_t ny, int64_t nz, int axis,
                        int64_t shift, int periodic, int full_table, int phase, int64_t flux_face, double fscale,
                        double vol, double *flux_part, double *flux_cum, unsigned *ticket, const double *ucoef,
                        int64_t ucoef_n, int64_t step0, int precision, int rshift, int blocks, cudaStream_t s);

// Fused 3-D step (x, y, z sweeps and phase in one pass, `steps` = 1 or 2 steps per launch): blocks of
// `warps` warps own a (32 - 2 steps)-cell x strip and warps - 2 steps rows along y and stream a z segment of
// zseg_h planes (steps 1: 8 or 16 warps; steps 2: 16 warps in FP32, 8 in FP64; 64-bit fixed point: steps 1,
// no vector potential).  precision: 0 FP64, 1 FP32, 2 int64 fixed point.  Flux parts:
// [steps][nzsegs * nytiles * warps] (a.nsegs * a.nplanes must equal nzsegs * nytiles * warps).
cudaError_t launch_fused3d(const SweepArgs &a, int precision, int warps, int steps, int64_t ny, int64_t nz,
                           int64_t nstrips, int64_t nytiles, int64_t nzsegs, int64_t zseg_h, cudaStream_t s);

// 3-D second-order step as fused passes (strang3d_kernels.cuh).  x-y-x pass (nh = 1: half a step) or
// x-y-x-x-y-x pass (nh = 2: the second half of one step and the first half of the next): blocks of `warps`
// (16 or 32) warps own a (32 - 4 nh)-cell x strip and warps - 4 nh rows along y over a z segment of zseg_h
// planes; fscale[s] scales the face flux of its x sweep s; flux parts [2 nh][nzsegs * nytiles * warps]
// (a.nsegs * a.nplanes must equal nzsegs * nytiles * warps).  z-phase-z pass: one thread per column and
// plane parity over nsegs segments of seg_h planes, the phase from `table` (or, with ucoef, the
// vector-potential matrix of step step0).
// precision: 0 FP64, 1 FP32, 2 64-bit fixed point (rshift_mid / rshift_end: the step's final division by 2^r,
// rounded, between the halves of an NH = 2 pass / after the pass's last sweep; 0 for floating-point states).
cudaError_t launch_strang_xy(const SweepArgs &a, int precision, int warps, int nh, int64_t ny, int64_t nz,
                             int64_t nstrips, int64_t nytiles, int64_t nzsegs, int64_t zseg_h, const double fscale[4],
                             int rshift_mid, int rshift_end, cudaStream_t s);
cudaError_t launch_strang_z(const void *in, void *out, const void *table, int64_t nx, int64_t ny, int64_t nz,
                            int periodic, int full_table, const double *ucoef, int64_t ucoef_n, int64_t step0,
                            int64_t nsegs, int64_t seg_h, int precision, cudaStream_t s);

// Entries of the U matrix of Sec. 2.3 for mu = m c^2 dt and the field integral At (12 doubles:
// Dup, Ddn, Ez, -Ez, Ep, Em as (re, im)); A = sqrt(((mu^2 + At_x^2) + At_y^2) + At_z^2), sin(A)/A -> 1 at A = 0.
void u_entries(double mu, const double At[3], double out[12]);

// Phase coefficients of Eq. sol_dis_4 at A = 0 for potential energy v, times `scale`:
// out = (cos t_up, -sin t_up, cos t_dn, -sin t_dn), t_up = mu + v dt, t_dn = v dt - mu (FP64, libm).
void phase_coeffs(double mu, double v, double dt, double scale, double out[4]);
// The same coefficients times an absorbing-layer factor a (a = 1: identical to phase_coeffs):
// out = (cos t_up * a, -sin t_up * a, ...) * scale.
void phase_coeffs_masked(double mu, double v, double dt, double a, double scale, double out[4]);
// FP32 pair for (c, s): the float neighbours whose squared modulus is closest to 1.
void round_unitary(double c, double s, float &cf, float &sf);

}  // namespace dirac
