/*
 * FP64 CPU oracle for the split-operator / method-of-characteristics Dirac
 * scheme (Fillion-Gourdeau, Lorin, Bandrauk, "Numerical solution of the
 * time-dependent Dirac equation in coordinate space without fermion-doubling").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow statement of what the
 * scheme computes.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load it; the product library never does.  It shares no code,
 * header or table with the CUDA path.
 *
 * Grid and storage.  P0 finite volumes of edge a = dx (Sec. 2.3, Eq. discr_psi);
 * cell (i,j,k) has centre x_min + (i+1/2)dx.  The state is stored point-major as
 * psi[((k*ny + j)*nx + i)*4 + c] complex (re, im interleaved), c = 0..3 for the
 * four spinor components.  "2-D" is the x-z plane (ny = 1, the y sweep omitted,
 * Sec. 2.4 last paragraph).
 *
 * Boundary.  ZERO: cells outside the N cells are zero at every sub-step (the
 * Dirichlet condition psi|dOmega = 0 of Sec. 5).  PERIODIC: indices wrap (the
 * setting of the Fourier argument of Sec. 3).
 *
 * Arithmetic order (shared convention, written out on each side independently):
 *   - each sweep forms 1/2 {(I + alpha) psi(i-1) + (I - alpha) psi(i+1)} with the
 *     two bracketed rows added first and the sum then multiplied by 1/2;
 *   - the phase multiplies by p = (cos t, -sin t) with t = m*c*c*dt + V*dt for
 *     components 1,2 and t = V*dt - m*c*c*dt for components 3,4, the complex
 *     product taken as re = fma(z.re, p.re, -(z.im*p.im)),
 *     im = fma(z.re, p.im, z.im*p.re);
 *   - with a uniform vector potential the phase is the 4x4 matrix U exp(-i V dt): each entry of U times
 *     g = (cos(V dt), -sin(V dt)) as the complex product above, then psi'_a = sum over b = 1..4 in order of
 *     M_ab psi_b, accumulated from zero as re = fma(z.re, p.re, fma(-z.im, p.im, re)),
 *     im = fma(z.re, p.im, fma(z.im, p.re, im)) with z = psi_b, p = M_ab.
 * Compiled with -ffp-contract=off so that no other contraction happens.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { double re, im; } cplx;

static inline cplx c_add(cplx a, cplx b) { cplx r = {a.re + b.re, a.im + b.im}; return r; }
static inline cplx c_sub(cplx a, cplx b) { cplx r = {a.re - b.re, a.im - b.im}; return r; }
/* a + i*b and a - i*b, with i*b = (-b.im, b.re) */
static inline cplx c_add_ib(cplx a, cplx b) { cplx r = {a.re - b.im, a.im + b.re}; return r; }
static inline cplx c_sub_ib(cplx a, cplx b) { cplx r = {a.re + b.im, a.im - b.re}; return r; }
static inline cplx c_half(cplx a) { cplx r = {0.5 * a.re, 0.5 * a.im}; return r; }
static inline cplx c_mul(cplx z, cplx p) {
    cplx r;
    r.re = fma(z.re, p.re, -(z.im * p.im));
    r.im = fma(z.re, p.im, z.im * p.re);
    return r;
}
static inline double c_abs2(cplx a) { return a.re * a.re + a.im * a.im; }

/* Returns a pointer to the 4 components of cell (i,j,k), or NULL for a ghost
 * cell outside the grid under the ZERO boundary. */
static const cplx *cell(const cplx *psi, const int64_t n[3], int periodic,
                        int64_t i, int64_t j, int64_t k) {
    if (periodic) {
        i = ((i % n[0]) + n[0]) % n[0];
        j = ((j % n[1]) + n[1]) % n[1];
        k = ((k % n[2]) + n[2]) % n[2];
    } else if (i < 0 || i >= n[0] || j < 0 || j >= n[1] || k < 0 || k >= n[2]) {
        return NULL;
    }
    return psi + ((k * n[1] + j) * n[0] + i) * 4;
}

static const cplx ZERO4[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};

/* One directional sub-step, Eqs. sol_dis_1 (axis 0), sol_dis_2 (axis 1),
 * sol_dis_3 (axis 2): out(i) = 1/2 {(I + alpha_d) L + (I - alpha_d) R} with
 * L = psi(i - e_d), R = psi(i + e_d).  Dirac representation (Eq. dirac_mat):
 *   alpha_x psi = ( psi4,   psi3,   psi2,   psi1)
 *   alpha_y psi = (-i psi4, i psi3, -i psi2, i psi1)
 *   alpha_z psi = ( psi3,  -psi4,   psi1,  -psi2)
 * Components are 0-based below (psi1 -> [0]). */
static void sweep_cell(cplx *o, const cplx *L, const cplx *R, int axis) {
    if (axis == 0) {
        o[0] = c_half(c_add(c_add(L[0], L[3]), c_sub(R[0], R[3])));
        o[1] = c_half(c_add(c_add(L[1], L[2]), c_sub(R[1], R[2])));
        o[2] = c_half(c_add(c_add(L[1], L[2]), c_sub(R[2], R[1])));
        o[3] = c_half(c_add(c_add(L[0], L[3]), c_sub(R[3], R[0])));
    } else if (axis == 1) {
        o[0] = c_half(c_add(c_sub_ib(L[0], L[3]), c_add_ib(R[0], R[3])));
        o[1] = c_half(c_add(c_add_ib(L[1], L[2]), c_sub_ib(R[1], R[2])));
        o[2] = c_half(c_add(c_sub_ib(L[2], L[1]), c_add_ib(R[2], R[1])));
        o[3] = c_half(c_add(c_add_ib(L[3], L[0]), c_sub_ib(R[3], R[0])));
    } else {
        o[0] = c_half(c_add(c_add(L[0], L[2]), c_sub(R[0], R[2])));
        o[1] = c_half(c_add(c_sub(L[1], L[3]), c_add(R[1], R[3])));
        o[2] = c_half(c_add(c_add(L[0], L[2]), c_sub(R[2], R[0])));
        o[3] = c_half(c_add(c_sub(L[3], L[1]), c_add(R[1], R[3])));
    }
}

/* Characteristic shift K (Sec. 2.3): with c dt = K a the solution of each directional equation moves the
 * characteristics by K cells, so L = psi(i - K e_d), R = psi(i + K e_d).  The paper takes K = 1; any
 * K >= 1 is exact in each direction.  Set by oracle_set_shift (default 1); dt = K dx / c in the steps. */
static int64_t g_shift = 1;

void oracle_set_shift(int64_t K) { g_shift = K >= 1 ? K : 1; }

/* Sweep along `axis` (0 = x, 1 = y, 2 = z) of the whole grid, in place, with neighbours `shift` cells away. */
static int sweep_shift(double *psi_d, const int64_t n[3], int axis, int periodic, int64_t shift) {
    cplx *psi = (cplx *)psi_d;
    int64_t total = n[0] * n[1] * n[2];
    cplx *out = (cplx *)malloc((size_t)total * 4 * sizeof(cplx));
    if (!out) return -1;
    int64_t d[3] = {0, 0, 0};
    d[axis] = shift;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n[2]; ++k)
        for (int64_t j = 0; j < n[1]; ++j)
            for (int64_t i = 0; i < n[0]; ++i) {
                const cplx *L = cell(psi, n, periodic, i - d[0], j - d[1], k - d[2]);
                const cplx *R = cell(psi, n, periodic, i + d[0], j + d[1], k + d[2]);
                sweep_cell(out + ((k * n[1] + j) * n[0] + i) * 4, L ? L : ZERO4, R ? R : ZERO4, axis);
            }
    memcpy(psi, out, (size_t)total * 4 * sizeof(cplx));
    free(out);
    return 0;
}

/* Sweep along `axis` with the characteristic shift set by oracle_set_shift. */
int oracle_sweep(double *psi_d, const int64_t n[3], int axis, int periodic) {
    return sweep_shift(psi_d, n, axis, periodic, g_shift);
}

/* Potential energy at cell (i,j,k): layout 0 = none (V = 0), 1 = one value per
 * x column (nx entries), 2 = one value per cell. */
static double potential(const double *V, int layout, const int64_t n[3], int64_t i, int64_t j, int64_t k) {
    if (layout == 1) return V[i];
    if (layout == 2) return V[(k * n[1] + j) * n[0] + i];
    return 0.0;
}

/* Mass and scalar-potential step, Eq. sol_dis_4 with A = 0:
 * psi <- exp(-i beta m c^2 dt - i V dt) psi, i.e. components 1,2 multiplied by
 * exp(-i (m c^2 dt + V dt)) and components 3,4 by exp(-i (V dt - m c^2 dt)).
 * (The U matrix of Sec. 2.3 at A = 0 is diag(e^{-i mu}, e^{-i mu}, e^{i mu}, e^{i mu}).) */
static const double *g_absorb = NULL;  /* optional per-x-column damping factor, see oracle_set_absorber */

/* Absorbing layer (not part of the paper's scheme): a factor a(x) in (0, 1] per x column multiplied into
 * both phase coefficients of that column, i.e. psi <- a(x) exp(-i ...) psi each step.  NULL removes it. */
void oracle_set_absorber(const double *a) { g_absorb = a; }

int oracle_phase(double *psi_d, const int64_t n[3], double m, double c, double dt,
                 const double *V, int layout) {
    cplx *psi = (cplx *)psi_d;
    double mu = m * c * c * dt;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n[2]; ++k)
        for (int64_t j = 0; j < n[1]; ++j)
            for (int64_t i = 0; i < n[0]; ++i) {
                double vdt = potential(V, layout, n, i, j, k) * dt;
                double t_up = mu + vdt;
                double t_dn = vdt - mu;
                cplx p_up = {cos(t_up), -sin(t_up)};
                cplx p_dn = {cos(t_dn), -sin(t_dn)};
                if (g_absorb) {
                    const double a = g_absorb[i];
                    p_up.re = p_up.re * a; p_up.im = p_up.im * a;
                    p_dn.re = p_dn.re * a; p_dn.im = p_dn.im * a;
                }
                cplx *q = psi + ((k * n[1] + j) * n[0] + i) * 4;
                q[0] = c_mul(q[0], p_up);
                q[1] = c_mul(q[1], p_up);
                q[2] = c_mul(q[2], p_dn);
                q[3] = c_mul(q[3], p_dn);
            }
    return 0;
}

/* Probability carried across the face between cells face-1 and face during one
 * x sweep (Sec. 2.2 and App. A): the +c characteristics (psi1+psi4, psi2+psi3)/sqrt2
 * of cells face-K .. face-1 move right across it, the -c characteristics
 * (psi1-psi4, psi2-psi3)/sqrt2 of cells face .. face+K-1 move left across it (shift K).
 * A whole cell's characteristic content moves, so the probability is the density
 * times the cell volume dx^d, summed over all (j,k) in index order (cells in
 * increasing i within a row). */
static double face_flux(const cplx *psi, const int64_t n[3], int periodic, int64_t face, double vol) {
    double f = 0.0;
    for (int64_t k = 0; k < n[2]; ++k)
        for (int64_t j = 0; j < n[1]; ++j) {
            double right = 0.0, left = 0.0;
            for (int64_t i = face - g_shift; i < face; ++i) {
                const cplx *a = cell(psi, n, periodic, i, j, k);
                a = a ? a : ZERO4;
                right += 0.5 * (c_abs2(c_add(a[0], a[3])) + c_abs2(c_add(a[1], a[2])));
            }
            for (int64_t i = face; i < face + g_shift; ++i) {
                const cplx *b = cell(psi, n, periodic, i, j, k);
                b = b ? b : ZERO4;
                left += 0.5 * (c_abs2(c_sub(b[0], b[3])) + c_abs2(c_sub(b[1], b[2])));
            }
            f += right - left;
        }
    return f * vol;
}

/* Uniform vector potential (not needed by the paper's runs, Sec. 2.3 states the general step).  When a
 * table is set, step s of oracle_step (counted from step0) applies the full matrix of Eq. sol_dis_4,
 *   psi <- U exp(-i V dt) psi,  U = exp(-i beta m c^2 dt + i alpha.At),
 * with At = (At_x, At_y, At_z) = g_avec[3 (step0 + s) ..] the time integral of e A over the step
 * (Eq. field_dis1, supplied by the caller).  NULL removes it. */
static const double *g_avec = NULL;
static int64_t g_avec_n = 0, g_avec_step0 = 0;

void oracle_set_vector_potential(const double *At, int64_t nsteps_table, int64_t step0) {
    g_avec = At;
    g_avec_n = nsteps_table;
    g_avec_step0 = step0;
}

/* acc + z p, taken as re = fma(z.re, p.re, fma(-z.im, p.im, acc.re)), im = fma(z.re, p.im, fma(z.im, p.re, acc.im)) */
static inline cplx c_mac(cplx acc, cplx z, cplx p) {
    cplx r;
    r.re = fma(z.re, p.re, fma(-z.im, p.im, acc.re));
    r.im = fma(z.re, p.im, fma(z.im, p.re, acc.im));
    return r;
}

/* The 4x4 matrix U of Sec. 2.3 (the closed form of exp(i(beta F + alpha.F)) with F = -m c^2 dt and
 * F = At), written out entry by entry as the paper prints it:
 *   diagonal:  cos(A) -+ i (m c^2 dt / A) sin(A)   (- for components 1,2, + for 3,4)
 *   (1,3), (3,1):  i At_z sin(A)/A        (2,4), (4,2):  -i At_z sin(A)/A
 *   (1,4), (3,2):  (i At_x + At_y) sin(A)/A     (2,3), (4,1):  (i At_x - At_y) sin(A)/A
 * A = sqrt((m c^2 dt)^2 + At.At), summed as ((mu^2 + At_x^2) + At_y^2) + At_z^2; sin(A)/A -> 1 at A = 0. */
static void u_matrix(double mu, const double At[3], cplx U[4][4]) {
    const double A = sqrt(((mu * mu + At[0] * At[0]) + At[1] * At[1]) + At[2] * At[2]);
    const double sA = A > 0.0 ? sin(A) / A : 1.0;
    const double cA = cos(A);
    const double ax = At[0] * sA, ay = At[1] * sA, az = At[2] * sA, ms = mu * sA;
    memset(U, 0, 16 * sizeof(cplx));
    U[0][0].re = cA; U[0][0].im = -ms;
    U[1][1].re = cA; U[1][1].im = -ms;
    U[2][2].re = cA; U[2][2].im = ms;
    U[3][3].re = cA; U[3][3].im = ms;
    U[0][2].im = az;  U[2][0].im = az;
    U[1][3].im = -az; U[3][1].im = -az;
    U[0][3].re = ay;  U[0][3].im = ax;  U[2][1].re = ay;  U[2][1].im = ax;
    U[1][2].re = -ay; U[1][2].im = ax;  U[3][0].re = -ay; U[3][0].im = ax;
}

/* q <- M q for one cell with M = U g: each entry multiplied by g first (complex product), then
 * q'_a = sum_b M_ab q_b over b = 1..4 in order, accumulated with c_mac from zero. */
static void apply_ug(cplx *q, cplx U[4][4], cplx g) {
    cplx o[4];
    for (int a = 0; a < 4; ++a) {
        cplx acc = {0.0, 0.0};
        for (int b = 0; b < 4; ++b) acc = c_mac(acc, q[b], c_mul(U[a][b], g));
        o[a] = acc;
    }
    for (int a = 0; a < 4; ++a) q[a] = o[a];
}

/* Eq. sol_dis_4 with a uniform vector potential: psi <- (U exp(-i V dt)) psi per cell, the scalar factor
 * g = (cos(V dt), -sin(V dt)) (times the absorbing-layer factor when one is set) multiplied into every
 * entry first (M = U g as a complex product), then psi'_a = sum_b M_ab psi_b over b = 1..4 in order,
 * accumulated with c_mac from zero. */
static int oracle_phase_A(double *psi_d, const int64_t n[3], double m, double c, double dt,
                          const double *V, int layout, const double At[3]) {
    cplx *psi = (cplx *)psi_d;
    const double mu = m * c * c * dt;
    cplx U[4][4];
    u_matrix(mu, At, U);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n[2]; ++k)
        for (int64_t j = 0; j < n[1]; ++j)
            for (int64_t i = 0; i < n[0]; ++i) {
                const double vdt = potential(V, layout, n, i, j, k) * dt;
                cplx g = {cos(vdt), -sin(vdt)};
                if (g_absorb) {
                    g.re = g.re * g_absorb[i];
                    g.im = g.im * g_absorb[i];
                }
                apply_ug(psi + ((k * n[1] + j) * n[0] + i) * 4, U, g);
            }
    return 0;
}

/* Fields that vary in space and time (Sec. 2.3: the phase matrix U(i) of Eq. sol_dis_4 built from the field
 * integral At(i) of Eq. field_dis1 at each cell, and the scalar integral V~(i) of Eq. field_dis2), for fields
 * of the separable form
 *   e A_d(t, x) = f_d(t) a_d(x)  (d = x, y, z)   and   V(t, x) = V(x) + f_V(t) w(x),
 * whose integrals over step n are exactly  At_d(i) = F_d a_d(i)  and  V~(i) = V(i) dt + F_V w(i)  with
 * F = (F_x, F_y, F_z, F_V) the integrals of the envelopes over the step (supplied by the caller: row
 * step0 + s of its table for step s of a call) and the profiles a (3 per cell, [z][y][x][d]) and w (1 per
 * cell).  A NULL profile is zero.  Per cell: psi <- (U(At(i)) g) psi with g = (cos V~, -sin V~) (times the
 * absorber factor), U and the product as for the uniform field. */
static const double *g_fa = NULL, *g_fw = NULL, *g_fenv = NULL;
static int64_t g_fenv_n = 0, g_fenv_step0 = 0;

void oracle_set_field(const double *a, const double *w, const double *F, int64_t nsteps_table, int64_t step0) {
    g_fa = a;
    g_fw = w;
    g_fenv = F;
    g_fenv_n = nsteps_table;
    g_fenv_step0 = step0;
}

static int oracle_phase_field(double *psi_d, const int64_t n[3], double m, double c, double dt,
                              const double *V, int layout, const double F[4]) {
    cplx *psi = (cplx *)psi_d;
    const double mu = m * c * c * dt;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n[2]; ++k)
        for (int64_t j = 0; j < n[1]; ++j)
            for (int64_t i = 0; i < n[0]; ++i) {
                const int64_t cidx = (k * n[1] + j) * n[0] + i;
                double At[3] = {0.0, 0.0, 0.0};
                if (g_fa)
                    for (int d = 0; d < 3; ++d) At[d] = F[d] * g_fa[3 * cidx + d];
                double vt = potential(V, layout, n, i, j, k) * dt;
                if (g_fw) vt = vt + F[3] * g_fw[cidx];
                cplx U[4][4];
                u_matrix(mu, At, U);
                cplx g = {cos(vt), -sin(vt)};
                if (g_absorb) {
                    g.re = g.re * g_absorb[i];
                    g.im = g.im * g_absorb[i];
                }
                apply_ug(psi + cidx * 4, U, g);
            }
    return 0;
}

/* The phase sub-step of step s of a call: the space-time field when one is set, else the uniform vector
 * potential when one is set, else Eq. sol_dis_4 at A = 0.  Returns -2 when the field's table ends before it. */
static int phase_step(double *psi, const int64_t n[3], double m, double c, double dt, const double *V, int layout,
                      int64_t s) {
    if (g_fenv) {
        const int64_t t = g_fenv_step0 + s;
        if (t < 0 || t >= g_fenv_n) return -2;
        return oracle_phase_field(psi, n, m, c, dt, V, layout, g_fenv + 4 * t);
    }
    if (g_avec) {
        const int64_t t = g_avec_step0 + s;
        if (t < 0 || t >= g_avec_n) return -2;
        return oracle_phase_A(psi, n, m, c, dt, V, layout, g_avec + 3 * t);
    }
    return oracle_phase(psi, n, m, c, dt, V, layout);
}

/* nsteps steps of the first-order splitting, Eqs. split1-split4 in the discrete
 * form sol_dis_1-sol_dis_4: x sweep, y sweep (3-D only), z sweep, phase.  dt = dx/c
 * (c dt = a, K = 1, Sec. 2.3).  If flux_face >= 0 the probability crossing that x
 * face in each x sweep is added to *flux_cum. */
int oracle_step(double *psi, const int64_t n[3], int ndim, int periodic, double m, double c,
                double dx, const double *V, int layout, int64_t nsteps, int64_t flux_face,
                double *flux_cum) {
    double dt = (double)g_shift * dx / c;
    double vol = (ndim == 3) ? dx * dx * dx : dx * dx;
    for (int64_t s = 0; s < nsteps; ++s) {
        if (flux_face >= 0 && flux_cum) *flux_cum += face_flux((const cplx *)psi, n, periodic, flux_face, vol);
        if (oracle_sweep(psi, n, 0, periodic)) return -1;
        if (ndim == 3 && oracle_sweep(psi, n, 1, periodic)) return -1;
        if (oracle_sweep(psi, n, 2, periodic)) return -1;
        if (phase_step(psi, n, m, c, dt, V, layout, s)) return -2;
    }
    return 0;
}

/* ---- 64-bit fixed-point evaluation of the first-order step ----
 * The same scheme (x sweep, y sweep in 3-D, z sweep, phase: Eqs. sol_dis_1 - sol_dis_4 at A = 0) evaluated
 * on an int64 state q = psi 2^S (re, im interleaved, the layout above), as the GPU's fixed-point storage does:
 *   - each sweep forms the bracketed sums of its equation without the 1/2; integer sums are exact (a
 *     step's values stay below 2^62 while the input's discrete L2 norm times 2^S is below 2^60 in 2-D,
 *     2^59 in 3-D: each sweep with its 1/2 and the phase do not raise that norm, so j sweeps without
 *     the 1/2 leave every component below 2^j times it);
 *   - the phase coefficient p (as in oracle_phase, FP64, absorber factor included) times the deferred
 *     halves (1/4 in 2-D, 1/8 in 3-D) is held as P = round(p / 4 * 2^62) (resp. p / 8), rounded to
 *     nearest with ties to even;
 *   - each output component is the exact 128-bit value z.re P.re - z.im P.im (resp. z.re P.im + z.im P.re),
 *     scaled by 2^-62 and rounded to the nearest integer with halves upward.
 * ZERO / PERIODIC boundaries as above.  dt = dx / c. */
typedef struct { int64_t re, im; } qcplx;
static const qcplx QZERO4[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};

static const qcplx *qcell(const qcplx *q, const int64_t n[3], int periodic, int64_t i, int64_t j, int64_t k) {
    if (periodic) {
        i = (i % n[0] + n[0]) % n[0];
        j = (j % n[1] + n[1]) % n[1];
        k = (k % n[2] + n[2]) % n[2];
    } else if (i < 0 || i >= n[0] || j < 0 || j >= n[1] || k < 0 || k >= n[2]) {
        return NULL;
    }
    return q + ((k * n[1] + j) * n[0] + i) * 4;
}

static int64_t q_round62(__int128 v) { return (int64_t)((v + ((__int128)1 << 61)) >> 62); }

static int64_t q_coef(double p, double halves) { return (int64_t)nearbyint(ldexp(p * halves, 62)); }

/* x sweep (Eq. sol_dis_1 without the 1/2), characteristics moved sh cells: in -> out */
static void fx_sweep_x(const qcplx *in, qcplx *out, const int64_t n[3], int periodic, int64_t sh) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n[2]; ++k)
        for (int64_t j = 0; j < n[1]; ++j)
            for (int64_t i = 0; i < n[0]; ++i) {
                const qcplx *L = qcell(in, n, periodic, i - sh, j, k), *R = qcell(in, n, periodic, i + sh, j, k);
                if (!L) L = QZERO4;
                if (!R) R = QZERO4;
                qcplx *o = out + ((k * n[1] + j) * n[0] + i) * 4;
                o[0].re = (L[0].re + L[3].re) + (R[0].re - R[3].re); o[0].im = (L[0].im + L[3].im) + (R[0].im - R[3].im);
                o[1].re = (L[1].re + L[2].re) + (R[1].re - R[2].re); o[1].im = (L[1].im + L[2].im) + (R[1].im - R[2].im);
                o[2].re = (L[1].re + L[2].re) + (R[2].re - R[1].re); o[2].im = (L[1].im + L[2].im) + (R[2].im - R[1].im);
                o[3].re = (L[0].re + L[3].re) + (R[3].re - R[0].re); o[3].im = (L[0].im + L[3].im) + (R[3].im - R[0].im);
            }
}

/* y sweep (Eq. sol_dis_2 without the 1/2; i b = (-b.im, b.re)), sh cells: in -> out */
static void fx_sweep_y(const qcplx *in, qcplx *out, const int64_t n[3], int periodic, int64_t sh) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n[2]; ++k)
        for (int64_t j = 0; j < n[1]; ++j)
            for (int64_t i = 0; i < n[0]; ++i) {
                const qcplx *L = qcell(in, n, periodic, i, j - sh, k), *R = qcell(in, n, periodic, i, j + sh, k);
                if (!L) L = QZERO4;
                if (!R) R = QZERO4;
                qcplx *o = out + ((k * n[1] + j) * n[0] + i) * 4;
                /* (L1 - i L4) + (R1 + i R4) */
                o[0].re = (L[0].re + L[3].im) + (R[0].re - R[3].im); o[0].im = (L[0].im - L[3].re) + (R[0].im + R[3].re);
                /* (L2 + i L3) + (R2 - i R3) */
                o[1].re = (L[1].re - L[2].im) + (R[1].re + R[2].im); o[1].im = (L[1].im + L[2].re) + (R[1].im - R[2].re);
                /* (L3 - i L2) + (R3 + i R2) */
                o[2].re = (L[2].re + L[1].im) + (R[2].re - R[1].im); o[2].im = (L[2].im - L[1].re) + (R[2].im + R[1].re);
                /* (L4 + i L1) + (R4 - i R1) */
                o[3].re = (L[3].re - L[0].im) + (R[3].re + R[0].im); o[3].im = (L[3].im + L[0].re) + (R[3].im - R[0].re);
            }
}

/* z sweep (Eq. sol_dis_3 without the 1/2), sh cells: in -> out */
static void fx_sweep_z(const qcplx *in, qcplx *out, const int64_t n[3], int periodic, int64_t sh) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n[2]; ++k)
        for (int64_t j = 0; j < n[1]; ++j)
            for (int64_t i = 0; i < n[0]; ++i) {
                const qcplx *L = qcell(in, n, periodic, i, j, k - sh), *R = qcell(in, n, periodic, i, j, k + sh);
                if (!L) L = QZERO4;
                if (!R) R = QZERO4;
                qcplx *z = out + ((k * n[1] + j) * n[0] + i) * 4;
                z[0].re = (L[0].re + L[2].re) + (R[0].re - R[2].re); z[0].im = (L[0].im + L[2].im) + (R[0].im - R[2].im);
                z[1].re = (L[1].re - L[3].re) + (R[1].re + R[3].re); z[1].im = (L[1].im - L[3].im) + (R[1].im + R[3].im);
                z[2].re = (L[0].re + L[2].re) + (R[2].re - R[0].re); z[2].im = (L[0].im + L[2].im) + (R[2].im - R[0].im);
                z[3].re = (L[3].re - L[1].re) + (R[1].re + R[3].re); z[3].im = (L[3].im - L[1].im) + (R[1].im + R[3].im);
            }
}

/* Phase (Eq. sol_dis_4 at A = 0) over dt, in place: P = round(p * halves * 2^62), each output component
 * round((z.re P.re - z.im P.im) 2^-62) (resp. z.re P.im + z.im P.re) from the exact 128-bit value. */
static void fx_phase(qcplx *q, const int64_t n[3], double m, double c, double dt, const double *V, int layout,
                     double halves) {
    const double mu = m * c * c * dt;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n[2]; ++k)
        for (int64_t j = 0; j < n[1]; ++j)
            for (int64_t i = 0; i < n[0]; ++i) {
                const double vdt = potential(V, layout, n, i, j, k) * dt;
                const double t_up = mu + vdt, t_dn = vdt - mu;
                double pu_re = cos(t_up), pu_im = -sin(t_up), pd_re = cos(t_dn), pd_im = -sin(t_dn);
                if (g_absorb) {
                    const double a = g_absorb[i];
                    pu_re = pu_re * a; pu_im = pu_im * a; pd_re = pd_re * a; pd_im = pd_im * a;
                }
                const int64_t P[4] = {q_coef(pu_re, halves), q_coef(pu_im, halves), q_coef(pd_re, halves),
                                      q_coef(pd_im, halves)};
                qcplx *o = q + ((k * n[1] + j) * n[0] + i) * 4;
                for (int cc = 0; cc < 4; ++cc) {
                    const int64_t pr = P[cc < 2 ? 0 : 2], pi = P[cc < 2 ? 1 : 3];
                    const qcplx z = o[cc];
                    o[cc].re = q_round62((__int128)z.re * pr - (__int128)z.im * pi);
                    o[cc].im = q_round62((__int128)z.re * pi + (__int128)z.im * pr);
                }
            }
}

/* nsteps first-order steps (x, y in 3-D, z, phase), dt = dx / c. */
int oracle_step_fx(int64_t *q_d, const int64_t n[3], int ndim, int periodic, double m, double c, double dx,
                   const double *V, int layout, int64_t nsteps) {
    if ((ndim != 2 && ndim != 3) || (ndim == 2 && n[1] != 1)) return -3;
    qcplx *q = (qcplx *)q_d;
    const int64_t total = n[0] * n[1] * n[2];
    qcplx *t = (qcplx *)malloc((size_t)total * 4 * sizeof(qcplx));
    qcplx *u = (qcplx *)malloc((size_t)total * 4 * sizeof(qcplx));
    if (!t || !u) {
        free(t);
        free(u);
        return -1;
    }
    const double halves = ndim == 3 ? 0.125 : 0.25;
    for (int64_t s = 0; s < nsteps; ++s) {
        fx_sweep_x(q, t, n, periodic, 1);
        if (ndim == 3) {
            fx_sweep_y(t, u, n, periodic, 1);
            memcpy(t, u, (size_t)total * 4 * sizeof(qcplx));
        }
        fx_sweep_z(t, q, n, periodic, 1);
        fx_phase(q, n, m, c, dx / c, V, layout, halves);
    }
    free(t);
    free(u);
    return 0;
}

/* nsteps second-order steps in the x-z plane (Sec. 2.4): x, z, phase over dt = 2 dx / c with the four
 * sweeps' halves (1/16) in its coefficients, z, x.  The phase output is a quarter of the state (rounded at
 * that scale); the last two sweeps double it twice, exactly. */
int oracle_step_strang2d_fx(int64_t *q_d, const int64_t n[3], int periodic, double m, double c, double dx,
                            const double *V, int layout, int64_t nsteps) {
    if (n[1] != 1) return -3;
    qcplx *q = (qcplx *)q_d;
    const int64_t total = n[0] * n[2];
    qcplx *t = (qcplx *)malloc((size_t)total * 4 * sizeof(qcplx));
    if (!t) return -1;
    for (int64_t s = 0; s < nsteps; ++s) {
        fx_sweep_x(q, t, n, periodic, 1);
        fx_sweep_z(t, q, n, periodic, 1);
        fx_phase(q, n, m, c, 2.0 * dx / c, V, layout, 0.0625);
        fx_sweep_z(q, t, n, periodic, 1);
        fx_sweep_x(t, q, n, periodic, 1);
    }
    free(t);
    return 0;
}

/* nsteps second-order 3-D steps (Sec. 2.4): A(1) B(2) A(1) C(2) D C(2) A(1) B(2) A(1), the cells moved
 * by each sweep in parentheses, dt = 4 dx / c.  The state entering the phase is 16 times the true one; the
 * phase coefficients carry those four halves (1/16), so its output is the true state, rounded at that
 * scale; the last four sweeps leave 16 times it, divided back by 16 with rounding to nearest (halves up). */
int oracle_step_strang3d_fx(int64_t *q_d, const int64_t n[3], int periodic, double m, double c, double dx,
                            const double *V, int layout, int64_t nsteps) {
    qcplx *q = (qcplx *)q_d;
    const int64_t total = n[0] * n[1] * n[2];
    qcplx *t = (qcplx *)malloc((size_t)total * 4 * sizeof(qcplx));
    if (!t) return -1;
    for (int64_t s = 0; s < nsteps; ++s) {
        fx_sweep_x(q, t, n, periodic, 1);
        fx_sweep_y(t, q, n, periodic, 2);
        fx_sweep_x(q, t, n, periodic, 1);
        fx_sweep_z(t, q, n, periodic, 2);
        fx_phase(q, n, m, c, 4.0 * dx / c, V, layout, 1.0 / 16.0);
        fx_sweep_z(q, t, n, periodic, 2);
        fx_sweep_x(t, q, n, periodic, 1);
        fx_sweep_y(q, t, n, periodic, 2);
        fx_sweep_x(t, q, n, periodic, 1);
        for (int64_t e = 0; e < total * 8; ++e) q_d[e] = (q_d[e] + 8) >> 4;
    }
    free(t);
    return 0;
}

/* nsteps steps of the second-order (Strang) splitting of Sec. 2.4 in the x-z plane: with B omitted and
 * consecutive A steps merged, one step is A(dt/2) C(dt/2) D(dt) C(dt/2) A(dt/2) (D with the full phase
 * matrix when a vector potential is set: row step0 + s of its table is the integral over the whole step).  Each half-step sweep is
 * the one-cell characteristic shift when c dt/2 = dx, so dt = 2 dx / c here.  The face flux is added at
 * both x sweeps of a step. */
int oracle_step_strang2d(double *psi, const int64_t n[3], int periodic, double m, double c, double dx,
                         const double *V, int layout, int64_t nsteps, int64_t flux_face, double *flux_cum) {
    double dt = 2.0 * (double)g_shift * dx / c;
    double vol = dx * dx;
    for (int64_t s = 0; s < nsteps; ++s) {
        if (flux_face >= 0 && flux_cum) *flux_cum += face_flux((const cplx *)psi, n, periodic, flux_face, vol);
        if (oracle_sweep(psi, n, 0, periodic)) return -1;
        if (oracle_sweep(psi, n, 2, periodic)) return -1;
        /* a field's phase matrix spans the whole step dt */
        if (phase_step(psi, n, m, c, dt, V, layout, s)) return -2;
        if (oracle_sweep(psi, n, 2, periodic)) return -1;
        if (flux_face >= 0 && flux_cum) *flux_cum += face_flux((const cplx *)psi, n, periodic, flux_face, vol);
        if (oracle_sweep(psi, n, 0, periodic)) return -1;
    }
    return 0;
}

/* nsteps steps of the second-order splitting of Sec. 2.4 in 3-D: A(dt/4) B(dt/2) A(dt/4) C(dt/2) D(dt)
 * C(dt/2) A(dt/4) B(dt/2) A(dt/4).  With c dt/4 = K dx (K = the characteristic shift) each A sweep moves
 * the characteristics by K cells and each B and C sweep by 2K cells, so dt = 4 K dx / c.  The face flux is
 * added at each of the four x sweeps of a step (shift K). */
int oracle_step_strang3d(double *psi, const int64_t n[3], int periodic, double m, double c, double dx,
                         const double *V, int layout, int64_t nsteps, int64_t flux_face, double *flux_cum) {
    const double dt = 4.0 * (double)g_shift * dx / c;
    const double vol = dx * dx * dx;
    const int axes[9] = {0, 1, 0, 2, -1, 2, 0, 1, 0};
    for (int64_t s = 0; s < nsteps; ++s) {
        for (int q = 0; q < 9; ++q) {
            const int ax = axes[q];
            if (ax < 0) {  /* a field's phase matrix spans the whole step dt */
                if (phase_step(psi, n, m, c, dt, V, layout, s)) return -2;
                continue;
            }
            if (ax == 0 && flux_face >= 0 && flux_cum)
                *flux_cum += face_flux((const cplx *)psi, n, periodic, flux_face, vol);
            if (sweep_shift(psi, n, ax, periodic, ax == 0 ? g_shift : 2 * g_shift)) return -1;
        }
    }
    return 0;
}

/* Observables, summed in index order:
 *   out[0] = norm        = sum rho dx^d,  rho = sum_c |psi_c|^2
 *   out[1] = norm_right  = sum over cells with i >= flux_face of rho dx^d (0 if flux_face < 0)
 *   out[2..4] = centroid = sum x rho / sum rho, x = x_min + (i+1/2) dx per axis */
int oracle_observables(const double *psi_d, const int64_t n[3], int ndim, double dx,
                       const double x_min[3], int64_t flux_face, double out[5]) {
    const cplx *psi = (const cplx *)psi_d;
    double vol = (ndim == 3) ? dx * dx * dx : dx * dx;
    double s = 0.0, sr = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    for (int64_t k = 0; k < n[2]; ++k)
        for (int64_t j = 0; j < n[1]; ++j)
            for (int64_t i = 0; i < n[0]; ++i) {
                const cplx *q = psi + ((k * n[1] + j) * n[0] + i) * 4;
                double rho = c_abs2(q[0]) + c_abs2(q[1]) + c_abs2(q[2]) + c_abs2(q[3]);
                s += rho;
                if (flux_face >= 0 && i >= flux_face) sr += rho;
                sx += (x_min[0] + (i + 0.5) * dx) * rho;
                sy += (x_min[1] + (j + 0.5) * dx) * rho;
                sz += (x_min[2] + (k + 0.5) * dx) * rho;
            }
    out[0] = s * vol;
    out[1] = sr * vol;
    out[2] = s > 0 ? sx / s : 0.0;
    out[3] = s > 0 ? sy / s : 0.0;
    out[4] = s > 0 ? sz / s : 0.0;
    return 0;
}
