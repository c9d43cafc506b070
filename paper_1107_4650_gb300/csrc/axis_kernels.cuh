// One directional sweep of the whole grid per launch, with the characteristics moved by `shift` cells
// (Eqs. sol_dis_1-sol_dis_3 with c dt = shift * dx), optionally followed by the phase (Eq. sol_dis_4).
// Used for the 3-D second-order splitting of Sec. 2.4, whose nine sub-steps mix one-cell (x) and
// two-cell (y, z) shifts.
//
// One thread per output cell (grid-stride loop over a grid of a few blocks per SM): it loads the two
// cells `shift` away along the axis (zero outside the grid, or wrapped) and forms, with no 1/2,
//   x: o1 = (L1+L4) + (R1-R4), o2 = (L2+L3) + (R2-R3), o3 = (L2+L3) + (R3-R2), o4 = (L1+L4) + (R4-R1)
//   y: o1 = (L1-iL4) + (R1+iR4), o2 = (L2+iL3) + (R2-iR3), o3 = (L3-iL2) + (R3+iR2), o4 = (L4+iL1) + (R4-iR1)
//   z: o1 = (L1+L3) + (R1-R3), o2 = (L2-L4) + (R2+R4), o3 = (L1+L3) + (R3-R1), o4 = (L4-L2) + (R2+R4)
// (the order in which the sums are taken is fixed).  The output is 2x the swept state; the caller folds
// the factors of 2 into the phase table.  Reads hit L1/L2 for the second use of every cell (neighbouring
// threads, neighbouring rows, planes a few MB apart), so HBM sees about one read and one write per cell.
// Face flux (x sweeps): threads whose cell lies in [face - shift, face) add |u14|^2 + |u23|^2 of the state
// entering the sweep, those in [face, face + shift) subtract |w14|^2 + |w23|^2; the block's sum times
// `fscale` (1/2 over the square of the state's scale) is its part, and the last block folds the parts.
#pragma once

#include "step_kernels.cuh"

namespace dirac {

// psi'_a = sum_b M_ab psi_b over the non-zero entries of M = U g (Dup, Ddn, Ez, -Ez, Ep, Em), columns in order,
// accumulated with cmac from zero (a product with a zero entry would add exactly nothing).
template <typename T> __device__ __forceinline__ void apply_m6(Cx<T> (&o)[4], const Cx<T> (&m6)[6]) {
    const Cx<T> z0 = {T(0), T(0)};
    const Cx<T> n0 = cmac(cmac(cmac(z0, o[0], m6[0]), o[2], m6[2]), o[3], m6[4]);
    const Cx<T> n1 = cmac(cmac(cmac(z0, o[1], m6[0]), o[2], m6[5]), o[3], m6[3]);
    const Cx<T> n2 = cmac(cmac(cmac(z0, o[0], m6[2]), o[1], m6[4]), o[2], m6[1]);
    const Cx<T> n3 = cmac(cmac(cmac(z0, o[0], m6[5]), o[1], m6[3]), o[3], m6[1]);
    o[0] = n0;
    o[1] = n1;
    o[2] = n2;
    o[3] = n3;
}

// Entries of M = U(At) g for cell c (column i) of a field varying in space and time (Sec. 2.3, Eqs. sol_dis_4,
// field_dis1, field_dis2): At_d = F_d a_d(c), V~ = V dt + F_V w(c), U the closed form of exp(i(beta F + alpha.F))
// with F = -m c^2 dt and At, A = sqrt(((mu^2 + At_x^2) + At_y^2) + At_z^2), sin(A)/A -> 1 at A = 0, g =
// (cos V~, -sin V~) times the absorber factor and the power-of-two scale of the sweeps' halves.  All in FP64
// (CUDA's sin and cos, within an ulp or two of the host's), then rounded to the storage type.
template <typename T>
__device__ __forceinline__ void cell_field_matrix(const AxisArgs &a, int64_t c, int64_t i, Cx<T> (&m6)[6]) {
    double At[3] = {0.0, 0.0, 0.0};
    if (a.fa)
#pragma unroll
        for (int d = 0; d < 3; ++d) At[d] = __dmul_rn(a.fenv[d], __ldg(a.fa + 3 * c + d));
    double vt = a.fvdt ? __ldg(a.fvdt + (a.fvdt_full ? c : i)) : 0.0;
    if (a.fw) vt = __dadd_rn(vt, __dmul_rn(a.fenv[3], __ldg(a.fw + c)));
    const double mu = a.fmu;
    const double A2 = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(mu, mu), __dmul_rn(At[0], At[0])), __dmul_rn(At[1], At[1])),
                                __dmul_rn(At[2], At[2]));
    const double A = __dsqrt_rn(A2);
    double sA = 1.0, cA = 1.0;
    if (A > 0.0) {
        double sn;
        sincos(A, &sn, &cA);
        sA = __ddiv_rn(sn, A);
    }
    const double ax = __dmul_rn(At[0], sA), ay = __dmul_rn(At[1], sA), az = __dmul_rn(At[2], sA), ms = __dmul_rn(mu, sA);
    double sv, cv;
    sincos(vt, &sv, &cv);
    Cx<double> g = {cv, -sv};
    if (a.fabs) {
        const double f = __ldg(a.fabs + i);
        g = {__dmul_rn(g.re, f), __dmul_rn(g.im, f)};
    }
    g = {__dmul_rn(g.re, a.fscale_phase), __dmul_rn(g.im, a.fscale_phase)};
    const Cx<double> U6[6] = {{cA, -ms}, {cA, ms}, {0.0, az}, {0.0, -az}, {ay, ax}, {-ay, ax}};
#pragma unroll
    for (int e = 0; e < 6; ++e) {
        const Cx<double> p = cmulp(U6[e], g);
        m6[e] = Cx<T>{(T)p.re, (T)p.im};
    }
}


template <typename T, int AXIS, bool PHASE, int FLD>
__global__ void __launch_bounds__(256) axis_kernel(const AxisArgs a) {
    constexpr bool FIELD = FLD == 1;
    const int64_t nx = a.nx, ny = a.ny, nz = a.nz, S = a.shift;
    const int64_t ncells = nx * ny * nz;
    const bool per = a.periodic != 0;
    const T *in = static_cast<const T *>(a.in);
    T *out = static_cast<T *>(a.out);
    const T *tab = static_cast<const T *>(a.table);
    const int64_t stride = AXIS == 0 ? 1 : (AXIS == 1 ? nx : nx * ny);
    const int64_t n_ax = AXIS == 0 ? nx : (AXIS == 1 ? ny : nz);
    double facc = 0.0;
    Cx<T> UM[FIELD ? 6 : 1];  // U entries of this step: Dup, Ddn, Ez, -Ez, Ep, Em (Sec. 2.3)
    if (FIELD) {
        const double *u = a.ucoef + (a.step0 % a.ucoef_n) * 12;
#pragma unroll
        for (int e = 0; e < (FIELD ? 6 : 1); ++e) UM[e] = Cx<T>{(T)__ldg(u + 2 * e), (T)__ldg(u + 2 * e + 1)};
    }
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += (int64_t)gridDim.x * blockDim.x) {
        int64_t i, t;
        if (ncells <= 0x7fffffff) {  // 32-bit index arithmetic when the grid allows it (uniform branch)
            const uint32_t c32 = (uint32_t)c, nx32 = (uint32_t)nx, ny32 = (uint32_t)ny;
            i = c32 % nx32;
            t = (AXIS == 0) ? i : (AXIS == 1 ? (c32 / nx32) % ny32 : c32 / (nx32 * ny32));
        } else {
            i = c % nx;
            t = (AXIS == 0) ? i : (AXIS == 1 ? (c / nx) % ny : c / (nx * ny));
        }
        Cx<T> L[4], R[4];
        const int64_t tl = t - S, tr = t + S;
        if (per || tl >= 0) {
            const int64_t tw = per ? pmod(tl, n_ax) : tl;
            load_pt(in + (c + (tw - t) * stride) * 8, L);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) L[q] = {T(0), T(0)};
        }
        if (per || tr < n_ax) {
            const int64_t tw = per ? pmod(tr, n_ax) : tr;
            load_pt(in + (c + (tw - t) * stride) * 8, R);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) R[q] = {T(0), T(0)};
        }
        Cx<T> o[4];
        if (AXIS == 0) {
            const Cx<T> u14 = cadd(L[0], L[3]), u23 = cadd(L[1], L[2]);
            o[0] = cadd(u14, csub(R[0], R[3]));
            o[1] = cadd(u23, csub(R[1], R[2]));
            o[2] = cadd(u23, csub(R[2], R[1]));
            o[3] = cadd(u14, csub(R[3], R[0]));
            if (a.flux_face >= 0) {
                const int64_t f = a.flux_face;
                if (i >= f - S && i < f + S) {
                    Cx<T> s[4];
                    load_pt(in + c * 8, s);
                    const Cx<T> p14 = (i < f) ? cadd(s[0], s[3]) : csub(s[0], s[3]);
                    const Cx<T> p23 = (i < f) ? cadd(s[1], s[2]) : csub(s[1], s[2]);
                    const double v = __dadd_rn(abs2d(p14), abs2d(p23));
                    facc = (i < f) ? __dadd_rn(facc, v) : __dsub_rn(facc, v);
                }
            }
        } else if (AXIS == 1) {
            o[0] = cadd(csub_ib(L[0], L[3]), cadd_ib(R[0], R[3]));
            o[1] = cadd(cadd_ib(L[1], L[2]), csub_ib(R[1], R[2]));
            o[2] = cadd(csub_ib(L[2], L[1]), cadd_ib(R[2], R[1]));
            o[3] = cadd(cadd_ib(L[3], L[0]), csub_ib(R[3], R[0]));
        } else {
            o[0] = cadd(cadd(L[0], L[2]), csub(R[0], R[2]));
            o[1] = cadd(csub(L[1], L[3]), cadd(R[1], R[3]));
            o[2] = cadd(cadd(L[0], L[2]), csub(R[2], R[0]));
            o[3] = cadd(csub(L[3], L[1]), cadd(R[1], R[3]));
        }
        if (PHASE) {
            Cx<T> pu, pd;
            load_tab(tab + (a.full_table ? c : i) * 4, pu, pd);
            if (FLD == 2) {
                // a field varying in space and time: this cell's U(At(i)) exp(-i V~(i)) times the sweeps' scale
                Cx<T> m6[6];
                cell_field_matrix<T>(a, c, i, m6);
                apply_m6(o, m6);
            } else if (FIELD) {
                // (U_ab g) psi_b over the non-zero entries, columns in order, g = the table's exp(-i V dt)
                Cx<T> m6[FIELD ? 6 : 1];
#pragma unroll
                for (int e = 0; e < (FIELD ? 6 : 1); ++e) m6[e] = cmulp(UM[e], pu);
                const Cx<T> z0 = {T(0), T(0)};
                const Cx<T> n0 = cmac(cmac(cmac(z0, o[0], m6[0]), o[2], m6[2]), o[3], m6[4]);
                const Cx<T> n1 = cmac(cmac(cmac(z0, o[1], m6[0]), o[2], m6[5]), o[3], m6[3]);
                const Cx<T> n2 = cmac(cmac(cmac(z0, o[0], m6[2]), o[1], m6[4]), o[2], m6[1]);
                const Cx<T> n3 = cmac(cmac(cmac(z0, o[0], m6[5]), o[1], m6[3]), o[3], m6[1]);
                o[0] = n0;
                o[1] = n1;
                o[2] = n2;
                o[3] = n3;
            } else {
                o[0] = cmulp(o[0], pu);
                o[1] = cmulp(o[1], pu);
                o[2] = cmulp(o[2], pd);
                o[3] = cmulp(o[3], pd);
            }
        }
        if (a.rshift > 0) round_shift(o, a.rshift);
        store_pt(out + c * 8, o);
    }
    if (AXIS == 0 && a.flux_face >= 0) {
        // block part in a fixed order (warp xor tree, then warps in index order), then the last-block fold
        __shared__ double wpart[8];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) facc = __dadd_rn(facc, __shfl_xor_sync(0xffffffffu, facc, o));
        if ((threadIdx.x & 31) == 0) wpart[threadIdx.x >> 5] = facc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = __dadd_rn(b, wpart[w]);
            a.flux_part[blockIdx.x] = __dmul_rn(a.fscale, b);
        }
        __shared__ unsigned s_last;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = (atomicAdd(a.ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
        __syncthreads();
        if (s_last && threadIdx.x == 0) {
            __threadfence();
            double f = 0.0;
            for (unsigned q = 0; q < gridDim.x; ++q) f = __dadd_rn(f, __ldcg(a.flux_part + q));
            *a.flux_cum = __dadd_rn(__ldcg(a.flux_cum), __dmul_rn(f, a.vol));
            __threadfence();
            *a.ticket = 0u;
        }
    }
}

}  // namespace dirac
