// First-order 2-D step with a characteristic shift S > 1 (c dt = S dx, Sec. 2.3): the x sweep takes the
// cells i - S and i + S, the z sweep the rows q - S and q + S, then the phase over dt = S dx / c.
//
// One warp = one x strip of 32 P - 2 S owned cells (S halo cells each side) and a segment of rows, one step
// per launch.  Rows stream through registers: the "+z" characteristic sums of the last 2 S x-swept rows
// sit in a register ring indexed by (row - first row) mod 2 S; the row loop is unrolled by 2 S so every
// index into the ring is a compile-time constant.  Arithmetic order is that of the S = 1 kernel:
//   sweep:  u = a + b, w = a - b;  a' = u(-S) + w(+S), b' = u(-S) - w(+S)   (1/2 factors deferred)
//   phase:  re = fma(z.re, p.re, -(z.im p.im)),  im = fma(z.re, p.im, z.im p.re), p carrying 1/4.
// The face flux of a row is the +c characteristics of cells face-S..face-1 minus the -c characteristics
// of cells face..face+S-1 (each 1/2 (|u14|^2 + |u23|^2) or 1/2 (|w14|^2 + |w23|^2)), evaluated by the
// strip that owns the face: each lane holds at most one cell of each range (S < 32), adds its value to a
// partial in the storage type, and folds the partial into an FP64 sum every 32 rows, so the face warp's
// extra work stays a few instructions per row (FP64 issues far slower than FP32 on this GPU); the 1/2 is
// applied once to the warp's sum (exact power-of-two scaling).
#pragma once

#include "step_kernels.cuh"

namespace dirac {

// FIELD: a uniform vector potential; the phase is U(step) exp(-i V dt) applied as in the one-cell field mode.
template <typename T, int S, int P, bool FIELD>
__device__ __forceinline__ void shift_warp(const SweepArgs &a, const int64_t wid, const int lane) {
    const int64_t seg = wid / a.nstrips;
    const int64_t strip = wid - seg * a.nstrips;
    const int64_t nx = a.nx, nr = a.nr;
    const bool per = a.periodic != 0;
    const int64_t x_own0 = strip * a.strip_w;
    const int64_t x_own1 = min(x_own0 + a.strip_w, nx);
    const int64_t xa = x_own0 - S;
    const int64_t r_begin = seg * a.seg_h;
    const int64_t r_end = min(r_begin + a.seg_h, nr);
    const T *in = static_cast<const T *>(a.in);
    T *out = static_cast<T *>(a.out);
    const T *tab = static_cast<const T *>(a.table);

    int64_t xl[P];
    bool xin[P];
#pragma unroll
    for (int j = 0; j < P; ++j) {
        const int64_t x = xa + 32 * j + lane;
        xin[j] = (x >= 0 && x < nx);
        xl[j] = per ? pmod(x, nx) : min(max(x, (int64_t)0), nx - 1);
    }
    Cx<T> pu[P], pd[P];
    if (!a.full_table) {
#pragma unroll
        for (int j = 0; j < P; ++j) load_tab(tab + xl[j] * 4, pu[j], pd[j]);
    }
    Cx<T> UM[FIELD ? 6 : 1];  // U entries of this launch's step (Dup, Ddn, Ez, -Ez, Ep, Em)
    if (FIELD) {
        const double *u = a.ucoef + (a.step0 % a.ucoef_n) * 12;
#pragma unroll
        for (int e = 0; e < (FIELD ? 6 : 1); ++e) UM[e] = Cx<T>{(T)__ldg(u + 2 * e), (T)__ldg(u + 2 * e + 1)};
    }
    const int64_t face = a.flux_face;
    const bool has_face = face >= x_own0 && face < x_own1;
    double facc = 0.0;
    T fpart = T(0);
    int jr = -1, jl = -1;  // point group of this lane's cell in [face - S, face) and in [face, face + S)
#pragma unroll
    for (int j = 0; j < P; ++j) {
        const int64_t x = xa + 32 * j + lane;
        if (x >= face - S && x < face) jr = j;
        if (x >= face && x < face + S) jl = j;
    }

    Cx<T> UH[2 * S][P][2];
#pragma unroll
    for (int t = 0; t < 2 * S; ++t)
#pragma unroll
        for (int j = 0; j < P; ++j) {
            UH[t][j][0] = {T(0), T(0)};
            UH[t][j][1] = {T(0), T(0)};
        }
    const int src_prev = (lane + 32 - S) & 31, src_next = (lane + S) & 31;
    const int64_t r_first = r_begin - S, r_last = r_end + S;

    // row r of the state (zero outside the grid under the zero boundary)
    auto load_row = [&](int64_t r, Cx<T> (*dst)[4]) {
        const bool row_ok = per || (r >= 0 && r < nr);
        const int64_t rl = per ? pmod(r, nr) : r;
#pragma unroll
        for (int j = 0; j < P; ++j) {
            if (row_ok && (per || xin[j])) {
                load_pt(in + (rl * nx + xl[j]) * 8, dst[j]);
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c) dst[j][c] = {T(0), T(0)};
            }
        }
    };
    // FP32 storage is bandwidth-bound: the next row's loads are issued before this row's arithmetic
    constexpr bool PREFETCH = sizeof(T) == 4;
    Cx<T> nxt[PREFETCH ? P : 1][4];
    if (PREFETCH) load_row(r_first, nxt);

    for (int64_t r0 = r_first; r0 < r_last; r0 += 2 * S) {
#pragma unroll
        for (int t = 0; t < 2 * S; ++t) {
            const int64_t r = r0 + t;
            if (r >= r_last) break;
            Cx<T> st[P][4];
            if (PREFETCH) {
#pragma unroll
                for (int j = 0; j < P; ++j)
#pragma unroll
                    for (int c = 0; c < 4; ++c) st[j][c] = nxt[PREFETCH ? j : 0][c];
                if (r + 1 < r_last) load_row(r + 1, nxt);
            } else {
                load_row(r, st);
            }
            // x characteristics; u of cell x - S and w of cell x + S by shuffle (lanes < S take the previous
            // point group, lanes >= 32 - S the next one)
            Cx<T> u14[P], u23[P], w14[P], w23[P];
#pragma unroll
            for (int j = 0; j < P; ++j) {
                u14[j] = cadd(st[j][0], st[j][3]);
                w14[j] = csub(st[j][0], st[j][3]);
                u23[j] = cadd(st[j][1], st[j][2]);
                w23[j] = csub(st[j][1], st[j][2]);
            }
            Cx<T> pu14[P], pu23[P], nw14[P], nw23[P];
#pragma unroll
            for (int j = 0; j < P; ++j) {
                pu14[j] = shfl_c(u14[j], src_prev);
                pu23[j] = shfl_c(u23[j], src_prev);
                nw14[j] = shfl_c(w14[j], src_next);
                nw23[j] = shfl_c(w23[j], src_next);
            }
            if (has_face && r >= r_begin && r < r_end) {
                if (jr >= 0 || jl >= 0) {
                    Cx<T> ra = {T(0), T(0)}, rb = ra, la = ra, lb = ra;
#pragma unroll
                    for (int j = 0; j < P; ++j) {
                        if (j == jr) {
                            ra = u14[j];
                            rb = u23[j];
                        }
                        if (j == jl) {
                            la = w14[j];
                            lb = w23[j];
                        }
                    }
                    const T vr = Ar<T>::fma(ra.re, ra.re, Ar<T>::fma(ra.im, ra.im, Ar<T>::fma(rb.re, rb.re, Ar<T>::mul(rb.im, rb.im))));
                    const T vl = Ar<T>::fma(la.re, la.re, Ar<T>::fma(la.im, la.im, Ar<T>::fma(lb.re, lb.re, Ar<T>::mul(lb.im, lb.im))));
                    fpart = Ar<T>::add(fpart, Ar<T>::sub(vr, vl));
                }
                if (((r - r_begin) & 31) == 31 || r == r_end - 1) {
                    facc = __dadd_rn(facc, (double)fpart);
                    fpart = T(0);
                }
            }
            const int64_t q = r - S;  // output row: rows q - S (ring slot t) and q + S (this row)
            const bool out_row = q >= r_begin && q < r_end;
#pragma unroll
            for (int j = 0; j < P; ++j) {
                const int jp = j > 0 ? j - 1 : 0;
                const int jn = j < P - 1 ? j + 1 : P - 1;
                const Cx<T> lu14 = (lane < S) ? pu14[jp] : pu14[j];
                const Cx<T> lu23 = (lane < S) ? pu23[jp] : pu23[j];
                const Cx<T> rw14 = (lane >= 32 - S) ? nw14[jn] : nw14[j];
                const Cx<T> rw23 = (lane >= 32 - S) ? nw23[jn] : nw23[j];
                // x sweep (Eq. sol_dis_1 with neighbours at -+S), x2
                const Cx<T> b0 = cadd(lu14, rw14);
                const Cx<T> b3 = csub(lu14, rw14);
                const Cx<T> b1 = cadd(lu23, rw23);
                const Cx<T> b2 = csub(lu23, rw23);
                // z sweep (Eq. sol_dis_3 with rows -+S): +z movers (b1+b3, b2-b4), -z movers (b1-b3, b2+b4)
                const Cx<T> U13 = cadd(b0, b2), U24 = csub(b1, b3);
                if (out_row) {
                    const Cx<T> W13 = csub(b0, b2), W24 = cadd(b1, b3);
                    Cx<T> o[4];
                    o[0] = cadd(UH[t][j][0], W13);
                    o[2] = csub(UH[t][j][0], W13);
                    o[1] = cadd(UH[t][j][1], W24);
                    o[3] = csub(W24, UH[t][j][1]);
                    Cx<T> qu, qd;
                    if (a.full_table) {
                        load_tab(tab + (q * nx + xl[j]) * 4, qu, qd);
                    } else {
                        qu = pu[j];
                        qd = pd[j];
                    }
                    if (FIELD) {
                        Cx<T> m6[FIELD ? 6 : 1];
#pragma unroll
                        for (int e = 0; e < (FIELD ? 6 : 1); ++e) m6[e] = cmulp(UM[e], qu);
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
                        o[0] = cmulp(o[0], qu);
                        o[1] = cmulp(o[1], qu);
                        o[2] = cmulp(o[2], qd);
                        o[3] = cmulp(o[3], qd);
                    }
                    const int64_t x = xa + 32 * j + lane;
                    if (x >= x_own0 && x < x_own1) store_pt(out + (q * nx + x) * 8, o);
                }
                UH[t][j][0] = U13;
                UH[t][j][1] = U24;
            }
        }
    }
    if (has_face) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) facc = __dadd_rn(facc, __shfl_xor_sync(0xffffffffu, facc, o));
        if (lane == 0) a.flux_part[seg] = __dmul_rn(0.5, facc);
    }
}

template <typename T, int S, int P, bool FIELD>
__global__ void __launch_bounds__(128) shift_kernel(const SweepArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wid < a.nstrips * a.nsegs) shift_warp<T, S, P, FIELD>(a, wid, lane);
    if (a.flux_face >= 0) finish_flux<1>(a);
}

template <typename T, int S, int P>
static cudaError_t launch_shift_one(const SweepArgs &a, int wpb, cudaStream_t s) {
    const int64_t warps = a.nstrips * a.nsegs;
    const int64_t blocks = (warps + wpb - 1) / wpb;
    if (blocks <= 0) return cudaSuccess;
    if (a.ucoef != nullptr && a.ucoef_n > 0)
        shift_kernel<T, S, P, true><<<(unsigned)blocks, 32 * wpb, 0, s>>>(a);
    else
        shift_kernel<T, S, P, false><<<(unsigned)blocks, 32 * wpb, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace dirac
