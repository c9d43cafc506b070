/*
 * dirac.h - C ABI of libdirac, a GB300 (sm_103a) implementation of the
 * split-operator / method-of-characteristics scheme for the time-dependent
 * Dirac equation of Fillion-Gourdeau, Lorin and Bandrauk (arXiv:1107.4650).
 *
 * One time step (first-order splitting, Sec. 2.1, Eqs. split1-split4, in the
 * discrete form of Sec. 2.3, Eqs. sol_dis_1-sol_dis_4, with c dt = dx, K = 1):
 *   x sweep   psi <- 1/2 {(I + alpha_x) psi(i-1) + (I - alpha_x) psi(i+1)}
 *   y sweep   (3-D only, Eq. sol_dis_2)
 *   z sweep   (Eq. sol_dis_3)
 *   phase     psi <- exp(-i beta m c^2 dt - i V dt) psi   (Eq. sol_dis_4, A = 0)
 * "2-D" is the x-z plane (Sec. 2.4).  Units are the caller's (atomic units in
 * the paper: m = 1, c = 137.0359895).
 *
 * Conventions for every call:
 *   - every call returns a dirac_status; nothing is thrown and nothing exits;
 *   - on an error the message is kept in the grid (dirac_last_error) when a
 *     grid exists, otherwise in a thread-local buffer (dirac_last_error(NULL));
 *   - host buffers passed in are copied before the call returns; device buffers
 *     passed in are read or written on the grid's stream;
 *   - a grid is used by one host thread at a time;
 *   - the state is stored point-major, psi[z][y][x][c][re,im], c = 0..3 the four
 *     spinor components in the Dirac representation (Eq. dirac_mat): 64 bytes a
 *     cell in FP64 storage, 32 bytes in FP32 storage.
 */
#ifndef DIRAC_H
#define DIRAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dirac_grid dirac_grid; /* opaque, library-owned */

typedef enum {
    DIRAC_OK = 0,
    DIRAC_ERR_ARG = 1,       /* invalid argument (null pointer, bad size, bad enum) */
    DIRAC_ERR_OOM = 2,       /* device or host allocation failed */
    DIRAC_ERR_CUDA = 3,      /* a CUDA runtime call failed; see dirac_last_error */
    DIRAC_ERR_NONFINITE = 4, /* the state holds NaN or Inf (reported by dirac_observables) */
    DIRAC_ERR_TIMEOUT = 5,   /* a bounded device wait ran out */
    DIRAC_ERR_STATE = 6      /* call not valid in the grid's current state */
} dirac_status;

/* storage precision.  DIRAC_FX64: 64-bit fixed point, q = round(psi 2^S) per real component in int64, for
 * first-order steps (2-D: the fused step kernel, k = 1 or 2; 3-D: the fused single pass, points_per_lane 0,
 * or the x-y pass + z/phase pass) and second-order steps (2-D: one per launch; 3-D: the fused passes, eight
 * single sweeps, or single sweeps with one z-phase-z pass, the phase carrying the first four halves and the
 * step's last x sweep dividing by 16 with rounding): the sweeps' additions are exact and each step
 * rounds once (twice in 3-D second order), in the phase (a 128-bit product with the coefficients held as
 * round(p 2^62)).  dirac_set_state picks S from the state's discrete norm (dirac_info.fx_shift); states go
 * in and out as complex128.  No vector potential or char_shift > 1. */
enum { DIRAC_FP64 = 0, DIRAC_FP32 = 1, DIRAC_FX64 = 2 };
enum { DIRAC_BC_ZERO = 0, DIRAC_BC_PERIODIC = 1 };    /* boundary */
enum { DIRAC_V_NONE = 0, DIRAC_V_X_ONLY = 1, DIRAC_V_FULL = 2 }; /* potential layout */
enum { DIRAC_LIE = 0, DIRAC_STRANG = 1 };             /* splitting order */

typedef struct {
    int ndim;             /* 2 (x-z plane, n[1] must be 1) or 3 */
    int64_t n[3];         /* cells along x, y, z */
    double dx;            /* cell edge a; the time step is dt = dx / c (c dt = a, Sec. 2.3) */
    double c;             /* speed of light */
    double m;             /* particle mass */
    double x_min[3];      /* lower corner: cell (i,j,k) has centre x_min + (i+1/2) dx (Sec. 2.3) */
    int precision;        /* DIRAC_FP64 or DIRAC_FP32 storage of the state */
    int boundary;         /* DIRAC_BC_ZERO: cells outside the grid are zero at every sub-step
                             (Dirichlet condition of Sec. 5); DIRAC_BC_PERIODIC: wrap */
    int64_t flux_face;    /* x face index i_s in [1, nx-1] whose crossing probability is accumulated
                             every step (between cells i_s-1 and i_s), or -1 for none.  With periodic
                             boundaries and char_shift K > 1 it must lie in [K, nx-K], so that the K
                             cells each side of the face whose characteristics cross it are grid cells
                             (DIRAC_ERR_ARG otherwise) */
    void *stream;         /* cudaStream_t the grid's work is enqueued on (NULL = legacy stream) */
    int device;           /* CUDA device ordinal */
    int steps_per_launch; /* steps fused in one kernel launch (temporal block depth).  2-D: 1 or 2 for FP64,
                             1, 2 or 4 for FP32.  3-D first order: 1 or 2, 2 only in the fused pass
                             (points_per_lane 0); 3-D second order: 1.  0 = library choice (3-D: 2 for FP32
                             storage, 1 for FP64) */
    int use_graphs;       /* 1: replay dirac_step's steady-state launches from a captured CUDA graph */
    int points_per_lane;  /* x cells per lane of the step kernel: 1, 2 or 4 (K = 2 needs 2 in FP64);
                             0 = library choice */
    int splitting;        /* DIRAC_LIE: first-order steps x, (y,) z, phase with dt = dx / c (Sec. 2.1);
                             DIRAC_STRANG: second-order steps (Sec. 2.4).  2-D: x, z, phase(dt), z, x with
                             dt = 2 dx / c, so each half-step sweep is the one-cell shift; steps_per_launch
                             1 (FP64) or 1, 2 (FP32).  3-D: A B A C D C A B A with dt = 4 dx / c, x sweeps
                             moving one cell and y, z sweeps two (c dt/2 = 2 dx), run as eight single-sweep
                             launches per step (points_per_lane 1), as six single sweeps with C D C in one
                             z-phase-z pass (points_per_lane 4: the same bits) or as fused passes
                             (points_per_lane 2): a run of m steps (one dirac_step call, or a captured graph
                             of 32 steps) is x-y-x, m z-phase-z passes separated by m - 1 x-y-x-x-y-x
                             passes, then x-y-x, so the state in memory is at a step boundary only between
                             runs; 0 = library choice (fused passes for FP32 and fixed-point storage, the
                             z-phase-z plan for FP64; char_shift > 1: eight single sweeps) */
    int char_shift;       /* characteristic shift K of Sec. 2.3: c dt = K dx, each sweep moves the
                             characteristics by K cells.  0 or 1: the paper's K = 1; 2, 3 or 4 (FP64 or FP32
                             storage, one step per launch): 2-D first order (dt = K dx / c, the fused
                             shift kernel), 3-D first order (dt = K dx / c) and 2-D second order
                             (dt = 2 K dx / c) as single-sweep launches, 3-D second order (dt = 4 K dx / c,
                             x sweeps moving K cells and y, z sweeps 2 K) as eight single sweeps; a vector
                             potential is allowed with each of them */
    void *ext_state[2];   /* optional caller-owned device buffers used as the grid's two ping-pong state
                             buffers (both NULL: the grid allocates its own).  Each holds one state,
                             nx ny nz x 8 values of the storage type (double, float, or int64 for DIRAC_FX64),
                             on cfg.device, 16-byte aligned, not overlapping.  The grid adopts ext_state[0] as
                             its current state as it stands (nothing is copied or cleared; for DIRAC_FX64 the
                             values are q with shift 0 until a dirac_set_state), reads and writes both buffers
                             on its stream while it lives (steps, dirac_get_state's decoding, autotuning),
                             never frees them, and does not count them in dirac_info.device_bytes.  The caller
                             keeps them alive until dirac_destroy and orders its own writes to them before the
                             grid's next call on its stream; dirac_info.state_index says which one holds the
                             current state. */
} dirac_config;

/* Fills cfg with defaults: ndim 2, n = {256,1,256}, dx = 10/8192, c = 137.0359895, m = 1,
 * x_min centred, FP64, zero boundary, no flux face, legacy stream, device 0, library k, graphs on,
 * first-order splitting. */
void dirac_default_config(dirac_config *cfg);

/* Creates a grid: validates cfg, allocates two state buffers (ping-pong; none when cfg->ext_state
 * supplies them), the phase table and scratch on cfg->device, zero state (the contents of ext_state[0]
 * when given), V = 0.  Errors: DIRAC_ERR_ARG for an invalid config (including one ext_state pointer
 * without the other, a buffer that is not device memory of cfg->device, not 16-byte aligned, or two
 * buffers closer than one state's size), DIRAC_ERR_OOM when allocation fails (nothing is leaked),
 * DIRAC_ERR_CUDA otherwise.  The grid owns the device memory it allocated; free it with dirac_destroy. */
dirac_status dirac_create_grid(const dirac_config *cfg, dirac_grid **out);

/* Releases every resource of the grid (waits for its stream first).  NULL is accepted. */
dirac_status dirac_destroy(dirac_grid *g);

/* Static scalar potential energy V (so that V~ = V dt in Eq. field_dis2), host pointer, copied.
 * layout DIRAC_V_NONE (V ignored, V = 0), DIRAC_V_X_ONLY (count = nx values, V depends on x only)
 * or DIRAC_V_FULL (count = nx*ny*nz values in [z][y][x] order).  The phase coefficients
 * exp(-i (+-m c^2 dt + V dt)) (Eq. sol_dis_4 at A = 0) are formed in FP64 on the host and copied to
 * the device.  Errors: DIRAC_ERR_ARG on a bad layout/count/null V. */
dirac_status dirac_set_potential(dirac_grid *g, const double *V, int layout, int64_t count);

/* Copies a state in (layout above, storage precision of the grid; complex128 or complex64 per
 * component; complex128 for DIRAC_FX64, encoded on the device with a new shift S).  on_device != 0: psi is
 * a device pointer on the grid's device, read on the grid's stream.  Resets the step counter and the
 * cumulative flux to 0.  DIRAC_FX64 synchronises the stream (S is chosen on the host) and returns
 * DIRAC_ERR_NONFINITE for a state holding NaN or Inf. */
dirac_status dirac_set_state(dirac_grid *g, const void *psi, int on_device);

/* Copies the current state out (same layout; DIRAC_FX64 decodes it to complex128).  Host copies are
 * complete when the call returns; device copies are ordered on the grid's stream. */
dirac_status dirac_get_state(dirac_grid *g, void *psi, int on_device);

/* DIRAC_FX64 grids: the fixed-point state itself, int64 q = round(psi 2^shift) in the layout above (8 values
 * per cell), in or out without conversion (exact checkpoints).  set: the caller's shift must keep the
 * discrete L2 norm of q below 2^60 in 2-D, 2^59 in 3-D first order and 2^57 in 3-D second order (the
 * shifts dirac_set_state picks; see DIRAC_FX64); resets the counters like dirac_set_state.  Errors:
 * DIRAC_ERR_ARG for another precision or a null pointer. */
dirac_status dirac_set_state_fx(dirac_grid *g, const int64_t *q, int shift, int on_device);
dirac_status dirac_get_state_fx(dirac_grid *g, int64_t *q, int *shift, int on_device);

/* Device pointer of the current state buffer (valid until the next dirac_step / dirac_destroy; with
 * cfg.ext_state it is ext_state[dirac_info.state_index]).
 * DIRAC_FX64: the int64 fixed-point values q (psi = q 2^-S, S = dirac_info.fx_shift). */
dirac_status dirac_state_ptr(dirac_grid *g, void **dev_ptr);

/* Advances nsteps >= 0 time steps (asynchronous on the grid's stream): x sweep, (y sweep), z sweep,
 * phase per step, fused into kernels that each run steps_per_launch steps. */
dirac_status dirac_step(dirac_grid *g, int64_t nsteps);

typedef struct {
    double norm;        /* sum rho dx^d, rho = sum_c |psi_c|^2 */
    double norm_right;  /* the same over cells with i >= flux_face (0 without a face) */
    double flux_cum;    /* probability carried across flux_face since the last set_state */
    double centroid[3]; /* sum x rho / sum rho per axis */
    int64_t step;       /* steps taken since the last set_state */
} dirac_obs;

/* Reductions of the current state (Sec. 5.2.1: R and T are integrals of |psi|^2), accumulated in
 * FP64, deterministic.  density (nullable) receives rho per cell in FP64, [z][y][x], on the device
 * when density_on_device != 0, else on the host.  Synchronises the grid's stream.
 * Returns DIRAC_ERR_NONFINITE (obs still filled) when the norm is NaN or Inf, and DIRAC_ERR_TIMEOUT when
 * a step kernel gave up waiting for a row copy since the last dirac_set_state (every such wait is bounded
 * by about one second; the state is then invalid and dirac_set_state clears the report).  Setting the
 * environment variable DIRAC_INJECT_STALL before dirac_create_grid makes every zero-boundary step launch of
 * that grid stall one copy on purpose, to test this path. */
dirac_status dirac_observables(dirac_grid *g, dirac_obs *obs, double *density, int density_on_device);

/* Absorbing layer (an addition to the paper's scheme, which names absorbing boundaries as future work):
 * factors a(x) in (0, 1] per x column (count = nx, host pointer) multiplied into the phase coefficients,
 * so the state is damped by a(x) every step.  The zero boundary of Sec. 5 partially reflects a massive
 * wave; layers a few dozen columns deep with a(x) rising smoothly to 1 absorb it instead.  count = 0 or
 * a = NULL removes the layer.  Rebuilds the phase table from the last potential set. */
dirac_status dirac_set_absorber(dirac_grid *g, const double *a, int64_t count);

/* Uniform vector potential (dipole approximation of a laser field): the phase step becomes the full
 * matrix of Eq. sol_dis_4, psi <- U exp(-i V dt) psi, with U the 4x4 matrix of Sec. 2.3 built from
 * mu = m c^2 dt and the field integral At_n = e * int_{t_n}^{t_{n+1}} A(t) dt of Eq. field_dis1.
 *   A_tilde: host array of 3 * nsteps_table doubles, (At_x, At_y, At_z) of step n at [3n, 3n+3); the caller
 *            evaluates the integrals (analytically or by quadrature; e = -1 for an electron in a.u.).
 *   Step n is counted by the grid's step counter (0 after dirac_set_state, set by dirac_set_counters).
 * Copied; the entries of U are formed once per step on the host in FP64 and applied on the device.
 * First-order (DIRAC_LIE) grids, 2-D or 3-D (3-D steps then run the fused single pass), and second-order
 * (DIRAC_STRANG) grids, whose phase spans the whole step dt (2 dx / c in 2-D, 4 dx / c in 3-D; At_n its
 * integral over it), and 2-D grids with char_shift > 1 (dt = K dx / c).  NULL or nsteps_table = 0 removes
 * the field.  Errors: DIRAC_ERR_ARG for a negative count or a non-finite entry.
 * dirac_step returns DIRAC_ERR_ARG, enqueuing nothing, when the step counter would pass the table's end.
 * Steps with a field are launched one block of steps_per_launch at a time (no graph replay: each launch
 * takes its step index); the phase costs 48 instead of 16 FP64 instructions per point-step. */
dirac_status dirac_set_vector_potential(dirac_grid *g, const double *A_tilde, int64_t nsteps_table);

/* Fields varying in space and time (Sec. 2.3: the phase matrix U(i) of Eq. sol_dis_4 with the field integral
 * At(i) = e int_{t_n}^{t_{n+1}} A(t, x_i) dt of Eq. field_dis1 at every cell, and the scalar integral
 * V~(i) = int V(t, x_i) dt of Eq. field_dis2), for fields of the separable form
 *     e A_d(t, x) = f_d(t) a_d(x)   (d = x, y, z)     and     V(t, x) = V(x) + f_V(t) w(x),
 * V(x) the static potential of dirac_set_potential, whose integrals over step n are exactly
 *     At_d(i) = F_d^n a_d(i)     and     V~(i) = V(i) dt + F_V^n w(i),
 * F^n = int_{t_n}^{t_{n+1}} f(t) dt the envelopes' integrals over the step (the caller evaluates them,
 * analytically or by quadrature).  Per cell and step the phase is psi <- U(At(i)) exp(-i V~(i)) psi, U the
 * closed form of Sec. 2.3 with mu = m c^2 dt, formed on the device in FP64 (its sin and cos agree with the
 * host's to an ulp or two, so FP64 results agree with an FP64 evaluation on the host to about 1e-15 per step
 * rather than bit for bit).  Arguments (host buffers, copied):
 *   a  3 doubles per cell, [z][y][x][d] (NULL: no vector potential);
 *   w  1 double per cell, [z][y][x] (NULL: no time-dependent scalar potential);
 *   F  4 doubles per step, (F_x, F_y, F_z, F_V) of step n at [4n, 4n+4); step n is counted by the grid's step
 *      counter, as for dirac_set_vector_potential; NULL or nsteps_table = 0 removes the field.
 * Every step form runs with it (2-D and 3-D, first and second order, whose phase spans the whole step dt, and
 * char_shift 1-4) as single-sweep launches (DIRAC_PLAN_FIELD_SWEEPS), one step per block, no graph replay;
 * FP64 and FP32 storage.  Errors: DIRAC_ERR_ARG for a non-finite entry, a negative count or a DIRAC_FX64 grid,
 * DIRAC_ERR_STATE while a uniform vector potential is set (the two are exclusive: a(i) = (1, 1, 1) is the
 * uniform field).  dirac_step returns DIRAC_ERR_ARG, enqueuing nothing, when the step counter would pass the
 * table's end. */
dirac_status dirac_set_field(dirac_grid *g, const double *a, const double *w, const double *F, int64_t nsteps_table);

/* Checkpoint support: sets the step counter and cumulative flux (after dirac_set_state). */
dirac_status dirac_set_counters(dirac_grid *g, int64_t step, double flux_cum);

typedef struct {
    int steps_per_launch;   /* temporal block depth k in use */
    int points_per_lane;    /* x cells per lane in the step kernel */
    int64_t launch_warps;   /* warps in one step launch */
    int64_t strip_width;    /* x cells written by one warp */
    int64_t segment_rows;   /* rows written by one warp */
    int graphs;             /* 1 when dirac_step replays a CUDA graph */
    int64_t kernel_launches;/* kernels enqueued by this grid so far (all kinds) */
    size_t device_bytes;    /* device memory owned by the grid */
    int plan;               /* DIRAC_PLAN_*: which kernels one step runs */
    int fx_shift;           /* DIRAC_FX64: the state's fixed-point shift S (psi = q 2^-S); 0 otherwise */
    int state_index;        /* 0 or 1: the ping-pong buffer (ext_state[i] when given) holding the current state */
} dirac_info;

/* dirac_info.plan */
enum {
    DIRAC_PLAN_STEP_2D = 0,      /* fused 2-D first-order step, k steps per launch */
    DIRAC_PLAN_STRANG_2D = 1,    /* fused 2-D second-order step */
    DIRAC_PLAN_FIELD_2D = 2,     /* 2-D first-order step with the vector-potential phase matrix */
    DIRAC_PLAN_SHIFT_2D = 3,     /* 2-D first-order step with characteristic shift > 1 */
    DIRAC_PLAN_3D_TWO_PASS = 4,  /* 3-D x-y pass + z/phase pass */
    DIRAC_PLAN_3D_FUSED = 5,     /* 3-D single pass */
    DIRAC_PLAN_3D_STRANG = 6,    /* 3-D second-order step: eight single-sweep launches */
    DIRAC_PLAN_STRANG_FIELD_2D = 7, /* 2-D second-order step with the vector-potential phase matrix */
    DIRAC_PLAN_3D_STRANG_FUSED = 8, /* 3-D second-order steps: x-y-x, z-phase-z, x-y-x-x-y-x, ... passes */
    DIRAC_PLAN_SHIFT_SWEEPS = 9,    /* char_shift > 1 as single-sweep launches: 3-D first order x y z+phase,
                                       2-D second order x z+phase z x */
    DIRAC_PLAN_FIELD_SWEEPS = 10,   /* a field varying in space and time (dirac_set_field): single-sweep launches */
    DIRAC_PLAN_3D_STRANG_ZPASS = 11 /* 3-D second-order step: x y x single sweeps, one z-phase-z pass, x y x */
};

dirac_status dirac_get_info(const dirac_grid *g, dirac_info *info);

/* Chooses steps_per_launch and points_per_lane by timing candidate launches on this grid (the state
 * is saved and restored around the trial).  Synchronises.  The choice holds until destroy. */
dirac_status dirac_autotune(dirac_grid *g);

/* ---------------------------------------------------------------------------------------------
 * Batched ensemble: many independent 2-D Klein-step scattering runs (Sec. 5.2) of uneven grid sizes
 * and step counts, advanced together by one persistent kernel per block of steps_per_launch steps
 * (warps take (run, strip, segment) tasks from an atomic queue), the launch sequence replayed from a
 * CUDA graph.  Each run is the single-grid scheme of dirac_step on a side x side x-z grid with the
 * zero boundary, the tanh step V(x) = V0/2 [1 + tanh(x/L)] centred on its flux face (x = 0 there)
 * and the Gaussian packet [1, 0, 0, C] e^{i p0 x} exp(-((x-x0)^2 + z^2)/(4 width^2)) of Sec. 5.2.2
 * (z = 0 mid-grid).  The result of a run is its transmission T = cumulative face flux / initial norm
 * (R = 1 - T: the boundary is outflowing).  Cell (i, k) of a run has centre
 * ((i - face + 1/2) dx, (k - side/2 + 1/2) dx).
 * --------------------------------------------------------------------------------------------- */
typedef struct dirac_batch dirac_batch; /* opaque, library-owned */

typedef struct {
    int64_t side;   /* cells per side, >= 8 */
    int64_t face;   /* flux face / step position, in [1, side-1] */
    int64_t nsteps; /* time steps of this run, >= 0 */
    double V0;      /* step height (potential energy) */
    double L;       /* step width, > 0 */
    double p0;      /* packet momentum along x */
    double width;   /* packet width, > 0 */
    double x0;      /* packet centre along x (the step is at x = 0) */
    int64_t absorb; /* absorbing-layer columns at each x edge (0: none); the initial packet is zero there */
    double eta;     /* layer strength: factor exp(-eta s^2) per step, s = depth into the layer / absorb */
} dirac_klein_run;

typedef struct {
    int precision;          /* DIRAC_FP32 (the ensemble's storage) or DIRAC_FP64 */
    double dx, c, m;        /* as in dirac_config; dt = dx / c */
    void *stream;           /* cudaStream_t (NULL = legacy stream) */
    int device;
    int steps_per_launch;   /* 0 = library choice */
    int points_per_lane;    /* 0 = library choice */
    int64_t segment_rows;   /* rows per task; 0 = library choice */
    int use_graphs;         /* 1: the launch sequence of dirac_batch_run is captured once and replayed */
} dirac_batch_config;

/* Defaults: FP32, dx = 10/8192, c = 137.0359895, m = 1, legacy stream, device 0, library tiles, graphs. */
void dirac_batch_default_config(dirac_batch_config *cfg);

/* Validates the runs, allocates every run's ping-pong state, phase table and flux scratch on the device
 * and writes the initial packets.  Errors: DIRAC_ERR_ARG (bad run or config), DIRAC_ERR_OOM. */
dirac_status dirac_batch_create(const dirac_klein_run *runs, int nruns, const dirac_batch_config *cfg,
                                dirac_batch **out);
dirac_status dirac_batch_destroy(dirac_batch *b);

/* Writes the initial packets again and clears the fluxes (the batch can then run again). */
dirac_status dirac_batch_reset(dirac_batch *b);

/* Replaces run `run`'s initial state (layout of dirac_set_state, side x 1 x side cells) before
 * dirac_batch_run; host buffers are copied before the call returns. */
dirac_status dirac_batch_set_state(dirac_batch *b, int run, const void *psi, int on_device);

/* Replaces run `run`'s x-only potential (side values, host pointer) by V; coefficients as in
 * dirac_set_potential, times the run's absorbing-layer factors. */
dirac_status dirac_batch_set_potential(dirac_batch *b, int run, const double *V, int64_t count);

/* Replaces run `run`'s absorbing-layer factors by a (side values in (0, 1], host pointer); they multiply the
 * phase coefficients from the next dirac_batch_set_potential on. */
dirac_status dirac_batch_set_absorber(dirac_batch *b, int run, const double *a, int64_t count);

/* Advances every run by its nsteps (asynchronous on the batch stream); measures each run's initial norm
 * first.  A second call needs dirac_batch_reset in between (DIRAC_ERR_STATE otherwise). */
dirac_status dirac_batch_run(dirac_batch *b);

/* Per-run results after dirac_batch_run (synchronises): T[r] = flux[r] / norm0[r]; any pointer may be NULL. */
dirac_status dirac_batch_results(dirac_batch *b, double *T, double *flux, double *norm0);

/* Copies run `run`'s current state out (after dirac_batch_run: its final state). */
dirac_status dirac_batch_get_state(dirac_batch *b, int run, void *psi, int on_device);

/* Chooses steps_per_launch, points_per_lane and segment_rows by timing trial launches on this batch, then
 * writes the initial packets again (a state set with dirac_batch_set_state is lost). */
dirac_status dirac_batch_autotune(dirac_batch *b);

typedef struct {
    int steps_per_launch, points_per_lane;
    int64_t segment_rows;
    int64_t launches;       /* kernel launches of one dirac_batch_run */
    int64_t max_tasks;      /* tasks of the fullest launch */
    int64_t point_steps;    /* sum over runs of side^2 x nsteps */
    int blocks;             /* resident blocks of the persistent kernel */
    size_t device_bytes;
} dirac_batch_info;
dirac_status dirac_batch_get_info(const dirac_batch *b, dirac_batch_info *info);
const char *dirac_batch_last_error(const dirac_batch *b);

/* One call: create, autotune (when cfg->steps_per_launch == 0), run, results, destroy.
 * T_out and R_out (nullable) receive nruns values each. */
dirac_status dirac_batch_klein(const dirac_klein_run *runs, int nruns, const dirac_batch_config *cfg, double *T_out,
                               double *R_out);

/* ---------------------------------------------------------------------------------------------
 * Transmission surrogate: an MLP 3 -> 256 -> 256 -> 256 -> 256 -> 1 (tanh hidden layers, sigmoid output)
 * with BF16 weights and FP32 accumulation, trained on GPU by the library's own forward, backward and
 * Adam kernels on transmissions the solver produced.  The hidden-layer products run on the tensor cores
 * (tcgen05, accumulator in tensor memory); train, predict and gradient return DIRAC_ERR_TIMEOUT if one
 * of their bounded (about one second) waits for the tensor cores ran out.  Inputs are reduced run parameters
 * q = (V0 / m c^2, p0 / m c, width / dx), mapped linearly from the training box [lo, hi] to [-1, 1]^3.
 * Queries outside the box are answered by the batched solver (the surrogate's fallback).
 * --------------------------------------------------------------------------------------------- */
typedef struct dirac_surrogate dirac_surrogate; /* opaque */

/* Creates an untrained network (Xavier-uniform weights from a splitmix64 stream of `seed`, zero biases)
 * for the box lo[3], hi[3] of reduced parameters.  max_batch bounds the training / inference batch. */
dirac_status dirac_surrogate_create(const double lo[3], const double hi[3], uint64_t seed, int max_batch, void *stream,
                                    int device, dirac_surrogate **out);
dirac_status dirac_surrogate_destroy(dirac_surrogate *s);

/* Adam training on n samples (X: n x 3 reduced parameters, T: n targets in [0, 1]), host buffers: `epochs`
 * passes over a fresh shuffle each (splitmix64 of the seed and the epoch), mini-batches of `batch`,
 * learning rate lr with cosine decay to lr/20.  The first call on freshly created parameters sets the
 * output bias to the logit of the mean target (not after dirac_surrogate_set_params).  loss_out (nullable) receives the last epoch's mean squared
 * error.  Synchronises. */
dirac_status dirac_surrogate_train(dirac_surrogate *s, const double *X, const double *T, int64_t n, int epochs,
                                   int batch, double lr, double *loss_out);

/* Network prediction for n points (host buffers), no range check: one fused kernel launch per max_batch
 * points (128 points per CTA: tensor-core layers, weights staged by bulk copies), the same rounding points
 * and results as the training forward pass.  Synchronises; DIRAC_ERR_TIMEOUT if a bounded wait (weights
 * copied in, tensor-core products done; about one second each) ran out, the outputs then invalid.  Setting
 * DIRAC_INJECT_STALL before dirac_surrogate_create makes every prediction launch of that network stall one
 * weight wait on purpose, to test this path. */
dirac_status dirac_surrogate_predict(dirac_surrogate *s, const double *X, int64_t n, double *T_out);

/* Gradient of mean((y - T)^2) over the n <= max_batch samples with respect to every parameter (FP32, the
 * parameter layout of dirac_surrogate_get_params), without updating; loss_out receives the loss. */
dirac_status dirac_surrogate_gradient(dirac_surrogate *s, const double *X, const double *T, int64_t n, float *grad_out,
                                      double *loss_out);

/* Number of parameters (198657) and FP32 master parameters in the order W1[256][3], b1, W2[256][256], b2,
 * W3, b3, W4, b4, w5[256], b5 (host buffers). */
int64_t dirac_surrogate_num_params(void);
dirac_status dirac_surrogate_get_params(dirac_surrogate *s, float *params);
dirac_status dirac_surrogate_set_params(dirac_surrogate *s, const float *params);

/* Checkpoint of the network at `path` (a file; the surrogate counterpart of a training run's checkpoint
 * path): the box lo/hi, the FP32 master parameters, the Adam moments and step and the shuffle seed, so that
 * training resumes where it stopped.  save overwrites the file; load replaces the surrogate's box, seed,
 * parameters and optimizer state (max_batch, stream and device stay).  Errors: DIRAC_ERR_ARG for a file that cannot be opened, a
 * short or foreign file, or a checkpoint of another parameter count. */
dirac_status dirac_surrogate_save(dirac_surrogate *s, const char *path);
dirac_status dirac_surrogate_load(dirac_surrogate *s, const char *path);

/* Transmission for n queries: the network inside the box, the batched solver (geometry of the Klein
 * ensemble: 64-column absorbing layers (eta 0.1) at both x edges, side = smallest of 256, 384, 512, 768,
 * 1024 holding 8 width + 264 cells (1024 at most), face 8 width + 8 cells right of the left layer and at
 * least 192 cells from the right edge, packet 4 widths left of the step, L = 4 dx, steps = time for the
 * packet to travel 8 widths at its group velocity + 200, clamped to [2000, 6000]) outside it, with
 * solver_cfg's precision.  used_solver (nullable) receives 1 for the points the solver answered. */
dirac_status dirac_surrogate_query(dirac_surrogate *s, const double *X, int64_t n, const dirac_batch_config *solver_cfg,
                                   double *T_out, int *used_solver);

/* Ensemble geometry of one reduced query q (same rule as the fallback above), for callers that build
 * their own batches. */
dirac_status dirac_klein_run_from_reduced(const double q[3], double dx, double c, double m, dirac_klein_run *run);

/* Last error of s (or of this thread for calls without a surrogate). Never NULL. */
const char *dirac_surrogate_last_error(const dirac_surrogate *s);

/* Allocation-free observables.  The paper has no counterpart: this serves callers that cannot
 * allocate device memory, such as a host framework that owns the whole device budget through its own
 * pool, or a latency-critical loop that must not pay the device synchronisation that cudaMalloc and
 * cudaFree can imply.  It computes what dirac_observables computes (to FP64 rounding: the block
 * partition differs) for a state in caller-owned device memory and allocates nothing: its block
 * partials live in one fixed device array of DIRAC_NOALLOC_MAX_BLOCKS x 5 doubles (640 KiB), defined
 * in the library and held by every device that loads it until the process exits.
 *   psi        device pointer on the current device, layout psi[z][y][x][c][re,im]; `precision` is
 *              DIRAC_FP64 (complex128) or DIRAC_FP32 (complex64) only: a fixed-point (DIRAC_FX64) state,
 *              such as dirac_state_ptr returns for a DIRAC_FX64 grid, is rejected with DIRAC_ERR_ARG
 *   n, ndim    grid as in dirac_config (n[1] == 1 when ndim == 2); at most
 *              DIRAC_NOALLOC_MAX_BLOCKS * DIRAC_NOALLOC_CELLS_PER_BLOCK cells, else DIRAC_ERR_ARG
 *   dx, x_min  cell edge and lower corner; flux_face as in dirac_config (-1: norm_right = 0)
 *   stream     cudaStream_t the two kernels are enqueued on (NULL = legacy stream); asynchronous
 *   out        device pointer to 5 doubles: norm, norm_right, centroid x, y, z
 * A call outside a stream capture looks up the array's device address (cudaGetSymbolAddress, which
 * allocates nothing) with the current device, so after cudaDeviceReset the next such call finds the
 * reloaded array; a call inside a capture uses the address the last uncaptured call on that device
 * found, so make the first call on a device before any stream capture (DIRAC_ERR_CUDA otherwise).
 * Every call shares the array and overwrites the partials it reads, so nothing needs clearing, but
 * calls whose kernels overlap on the GPU (different streams or host threads) race on it.  The result
 * is written asynchronously, so unlike dirac_observables this call never returns DIRAC_ERR_NONFINITE:
 * a state holding NaN or Inf leaves a NaN or Inf norm in out[0].  Errors go to dirac_last_error(NULL). */
#define DIRAC_NOALLOC_MAX_BLOCKS 16384
#define DIRAC_NOALLOC_CELLS_PER_BLOCK 8192
dirac_status dirac_observables_noalloc(const void *psi, int precision, int ndim, const int64_t n[3], double dx,
                                       const double x_min[3], int64_t flux_face, void *stream, double *out);

/* Last error message for g (or of this thread when g == NULL). Never NULL. */
const char *dirac_last_error(const dirac_grid *g);

/* Library version string. */
const char *dirac_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DIRAC_H */
