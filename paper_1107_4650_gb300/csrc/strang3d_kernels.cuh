// Fused passes of the 3-D second-order step (Sec. 2.4, dt = 4 dx / c):
//   A(1) B(2) A(1) | C(2) D C(2) | A(1) B(2) A(1)     (cells moved per sweep in parentheses)
// A run of m steps is 2m + 1 passes over HBM instead of 8m single-sweep launches:
//   x-y-x, then m times z-phase-z, separated by x-y-x-x-y-x passes (the second half of one step and the
// first half of the next), then x-y-x.  Arithmetic is that of the single-sweep kernels (axis_kernels.cuh),
// operation by operation, so the result is the same bit for bit in either storage precision; only where the
// intermediate states live changes (registers and shared memory instead of HBM).
//
// x-y-x pass (NH = 1 half step) and x-y-x-x-y-x pass (NH = 2), per z plane (planes are independent): a block
// of W warps owns an x strip of 32 - 4 NH cells (lane l holds cell x0 - 2 NH + l: one halo cell each side per
// x sweep) and W - 4 NH rows along y (warp w holds row y0 - 2 NH + w: two halo rows each side per two-cell
// y sweep).  Per plane and half step:
//   * the warps x-sweep their row with shuffles and write its y characteristics to shared memory; after a
//     block barrier the warps two rows inside y-sweep their row from rows y - 2 ("+y" movers) and y + 2
//     ("-y" movers), zero the cells outside the grid (zero boundary), x-sweep again;
//   * NH = 2: that state (zeroed outside the grid) starts the next half step the same way, two rows further in.
// The owned lanes of the owned rows store.  NH = 1 double-buffers its shared rows by plane (one barrier per
// plane); NH = 2 has two barriers per plane, which order every reuse of its two single buffers.
// Face flux: every x sweep adds, on the face strip's owned rows, 1/2 (|u14|^2 + |u23|^2) of cell face - 1 and
// subtracts 1/2 (|w14|^2 + |w23|^2) of cell face, of the state entering it, times 1 / s^2 for the state's
// scale s (fscale); one part per (sweep, z segment, y tile, warp), folded by the last block.
// 64-bit fixed-point state (q = psi 2^S): the sweeps are exact integer sums, the face terms are formed in FP64
// (fscale carries 2^-2S), and the step's final division by 16 (rounded to nearest, halves up: the phase carries
// only the first four halves) follows the step's last x sweep: at the end of a pass that ends a step and between
// the halves of an x-y-x-x-y-x pass (rshift_end, rshift_mid; 0 for floating-point states).
//
// z-phase-z pass: the two-cell z sweeps couple plane k only with planes k - 2 and k + 2, and the phase is
// pointwise, so even and odd planes form two independent chains.  One thread per (x, y) column and plane
// parity streams its chain over a segment of planes (plus four halo planes each side).  Input plane k
// gives the characteristic sums U = (s1 + s3, s2 - s4) and W = (s1 - s3, s2 + s4); the first sweep's output
// at plane j = k - 2 is U(j - 2) + W(j + 2) (U of the chain's last two planes in a register ring), the phase
// of Eq. sol_dis_4 (table carrying the eight sweeps' 1/256, its entries loaded with the state's planes
// ahead of use) follows, cells outside the grid are zeroed, and the second sweep's output at plane k - 4 is
// formed the same way from a second ring.  The loop takes two chain planes per iteration so every ring
// index is a constant.
#pragma once

#include "step_kernels.cuh"

namespace dirac {

struct StrangXYArgs {
    SweepArgs s;          // in, out, flux fields; flux parts [2 NH][nzsegs * nytiles * W]
    int64_t ny, nz;
    int64_t nstrips, nytiles, nzsegs, zseg_h;
    double fscale[4];     // per x sweep: 1/2 over the square of the scale of the state entering it
    int rshift_mid;       // fixed point, NH = 2: divide by 2^rshift_mid (rounded) after the first half's last sweep
    int rshift_end;       // fixed point: divide by 2^rshift_end (rounded) after the pass's last sweep
};

struct StrangZArgs {
    const void *in;
    void *out;
    const void *table;
    int64_t nx, ny, nz;
    int64_t seg_h;        // planes per z segment (blockIdx.y = 2 segment + plane parity)
    int periodic, full_table;
    const double *ucoef;  // uniform vector potential: U entries per step (12 doubles), or null
    int64_t ucoef_n, step0;
};

// resident blocks per SM the register budget is fitted to: two 16-warp blocks in FP32
template <typename T, int W> struct XYMinBlocks { static constexpr int value = (sizeof(T) == 4 && W == 16) ? 2 : 1; };
// z-phase-z pass: 128-thread blocks per SM the register budget is fitted to
template <typename T, bool FIELD> struct ZMinBlocks { static constexpr int value = sizeof(T) == 4 ? 4 : 3; };

// type the face terms are summed in: the state's own floating-point type, FP64 for a fixed-point state
template <typename T> struct FaceAcc { using type = T; };
template <> struct FaceAcc<long long> { using type = double; };
// plane index type of the z loops: 32-bit for floating-point states (grid dimensions stay below 2^31), 64-bit for
// the fixed-point state
template <typename T> struct PlaneIdx { using type = int; };
template <> struct PlaneIdx<long long> { using type = int64_t; };

template <typename T>
__device__ __forceinline__ typename FaceAcc<T>::type face_term(Cx<T> p14, Cx<T> p23) {
    return Ar<T>::fma(p14.re, p14.re, Ar<T>::fma(p14.im, p14.im, Ar<T>::fma(p23.re, p23.re, Ar<T>::mul(p23.im, p23.im))));
}
template <> __device__ __forceinline__ double face_term<long long>(Cx<long long> p14, Cx<long long> p23) {
    const double a = (double)p14.re, b = (double)p14.im, c = (double)p23.re, d = (double)p23.im;
    return __fma_rn(a, a, __fma_rn(b, b, __fma_rn(c, c, __dmul_rn(d, d))));
}

// A: x sweep, one cell (Eq. sol_dis_1), of a row held one cell per lane; the output (2x the swept state) is
// valid on lanes whose two neighbours hold valid cells.  The face lanes add their term of the entering state.
template <typename T>
__device__ __forceinline__ void xsweep_row(const Cx<T> s[4], Cx<T> o[4], int lane, bool fl_u, bool fl_w,
                                           typename FaceAcc<T>::type &fp) {
    using F = typename FaceAcc<T>::type;
    const Cx<T> u14 = cadd(s[0], s[3]), w14 = csub(s[0], s[3]);
    const Cx<T> u23 = cadd(s[1], s[2]), w23 = csub(s[1], s[2]);
    if (fl_u) fp = Ar<F>::add(fp, face_term(u14, u23));
    if (fl_w) fp = Ar<F>::sub(fp, face_term(w14, w23));
    const Cx<T> lu14 = shfl_c(u14, (lane + 31) & 31), lu23 = shfl_c(u23, (lane + 31) & 31);
    const Cx<T> rw14 = shfl_c(w14, (lane + 1) & 31), rw23 = shfl_c(w23, (lane + 1) & 31);
    o[0] = cadd(lu14, rw14);
    o[3] = csub(lu14, rw14);
    o[1] = cadd(lu23, rw23);
    o[2] = csub(lu23, rw23);
}

// y characteristics of row w (Eq. sol_dis_2): "+y" movers (a1 - i a4, a2 + i a3), "-y" movers (a1 + i a4, a2 - i a3)
template <typename T>
__device__ __forceinline__ void ywrite_row(Cx<T> *buf, int w, int lane, const Cx<T> a[4]) {
    buf[(w * 4 + 0) * 32 + lane] = csub_ib(a[0], a[3]);
    buf[(w * 4 + 1) * 32 + lane] = cadd_ib(a[1], a[2]);
    buf[(w * 4 + 2) * 32 + lane] = cadd_ib(a[0], a[3]);
    buf[(w * 4 + 3) * 32 + lane] = csub_ib(a[1], a[2]);
}

// B: y sweep, two cells, of row w: "+y" movers of row w - 2, "-y" movers of row w + 2
template <typename T>
__device__ __forceinline__ void ysweep_row(const Cx<T> *buf, int w, int lane, Cx<T> q[4]) {
    const Cx<T> U14 = buf[((w - 2) * 4 + 0) * 32 + lane], U23 = buf[((w - 2) * 4 + 1) * 32 + lane];
    const Cx<T> W14 = buf[((w + 2) * 4 + 2) * 32 + lane], W23 = buf[((w + 2) * 4 + 3) * 32 + lane];
    q[0] = cadd(U14, W14);
    q[3] = cmul_i(csub(U14, W14));
    q[1] = cadd(U23, W23);
    q[2] = cmul_mi(csub(U23, W23));
}

template <typename T>
__device__ __forceinline__ void zero_pt(Cx<T> q[4]) {
#pragma unroll
    for (int c = 0; c < 4; ++c) q[c] = {T(0), T(0)};
}

// One block's planes.  FLUX: the block's strip holds the face (the face terms are formed only here); EDGE:
// the block's cells reach outside the grid under the zero boundary (only here are cells zeroed).
template <typename T, int W, int NH, bool FLUX, bool EDGE>
__device__ __forceinline__ void strang_xy_block(const StrangXYArgs &A, const int64_t strip, const int64_t ytile,
                                                const int64_t zseg, Cx<T> *ych) {
    constexpr int HX = 2 * NH;       // halo lanes (x) and halo rows (y) on each side
    constexpr int OWN = 32 - 2 * HX;
    constexpr int H = W - 2 * HX;
    constexpr int NS = 2 * NH;       // x sweeps per pass
    const SweepArgs &a = A.s;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nx = a.nx, ny = A.ny, nz = A.nz;
    const bool per = a.periodic != 0;
    const int64_t x_own0 = strip * OWN, x_own1 = min(x_own0 + OWN, nx);
    const int64_t x = x_own0 - HX + lane;
    const int64_t y = ytile * H - HX + w;
    const bool owned_row = w >= HX && w < W - HX && y < ny;
    const bool mid_row = w >= 2 && w < W - 2;  // NH = 2: rows of the first half step's second sweep pair
    const bool own_lane = x >= x_own0 && x < x_own1;
    using ZI = typename PlaneIdx<T>::type;
    const ZI z_begin = (ZI)(zseg * A.zseg_h), z_end = (ZI)min((int64_t)z_begin + A.zseg_h, nz);
    const bool ghost = EDGE && !(x >= 0 && x < nx && y >= 0 && y < ny);  // outside the grid (zero boundary)
    const int64_t xl = per ? pmod(x, nx) : min(max(x, (int64_t)0), nx - 1);
    const int64_t yl = per ? pmod(y, ny) : min(max(y, (int64_t)0), ny - 1);
    // this lane's cell in plane z_begin (owned lanes of owned rows: xl = x, yl = y); planes nx ny 8 apart
    const int64_t plane = nx * ny * 8;
    const T *src = static_cast<const T *>(a.in) + ((z_begin * ny + yl) * nx + xl) * 8;
    T *dst = static_cast<T *>(a.out) + ((z_begin * ny + yl) * nx + xl) * 8;

    const int64_t face = a.flux_face;
    const bool fw = FLUX && owned_row;  // warp-uniform
    const bool fl_u = fw && x == face - 1, fl_w = fw && x == face;
    using FA = typename FaceAcc<T>::type;
    double facc[NS];
    FA fp[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        facc[q] = 0.0;
        fp[q] = FA(0);
    }
    auto sweep_x = [&](const Cx<T> in4[4], Cx<T> out4[4], FA &acc) {
        if (FLUX && fw) {
            xsweep_row(in4, out4, lane, fl_u, fl_w, acc);
        } else {
            xsweep_row(in4, out4, lane, false, false, acc);
        }
    };

    // planes in flight: two ahead in FP32 (bandwidth-bound), one in FP64 and fixed point
    constexpr int LA = sizeof(T) == 4 ? 2 : 1;
    Cx<T> ring[LA][4];
#pragma unroll
    for (int j = 0; j < LA; ++j) {
        if (z_begin + j < z_end) {
            if (!ghost) {
                load_pt(src + j * plane, ring[j]);
            } else {
                zero_pt(ring[j]);
            }
        }
    }
    const T *ld = src + LA * plane;

    for (ZI k = z_begin; k < z_end; ++k, ld += plane, dst += plane) {
        Cx<T> st[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) st[c] = ring[0][c];
#pragma unroll
        for (int j = 0; j + 1 < LA; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) ring[j][c] = ring[j + 1][c];
        if (k + LA < z_end) {
            if (!ghost) {
                load_pt(ld, ring[LA - 1]);
            } else {
                zero_pt(ring[LA - 1]);
            }
        }

        Cx<T> t[4], q[4];
        sweep_x(st, t, fp[0]);
        Cx<T> *buf1 = NH == 1 ? ych + (size_t)((k - z_begin) & 1) * (W * 4 * 32) : ych;
        ywrite_row(buf1, w, lane, t);
        __syncthreads();
        if (NH == 1) {
            if (owned_row) {
                ysweep_row(buf1, w, lane, q);
                if (ghost) zero_pt(q);
                sweep_x(q, t, fp[1]);
                if (A.rshift_end > 0) round_shift(t, A.rshift_end);
                if (own_lane) store_pt(dst, t);
            }
        } else {
            Cx<T> *buf2 = ych + W * 4 * 32;
            if (mid_row) {
                ysweep_row(buf1, w, lane, q);
                if (ghost) zero_pt(q);
                sweep_x(q, t, fp[1]);
                if (A.rshift_mid > 0) round_shift(t, A.rshift_mid);  // fixed point: the end of a step
                if (ghost) zero_pt(t);  // the state between the two half steps
                sweep_x(t, q, fp[NS > 2 ? 2 : 0]);
                ywrite_row(buf2, w, lane, q);
            }
            __syncthreads();
            if (owned_row) {
                ysweep_row(buf2, w, lane, q);
                if (ghost) zero_pt(q);
                sweep_x(q, t, fp[NS > 3 ? 3 : 0]);
                if (A.rshift_end > 0) round_shift(t, A.rshift_end);
                if (own_lane) store_pt(dst, t);
            }
        }
        if (FLUX && fw && (fl_u || fl_w) && (((k - z_begin) & 31) == 31 || k == z_end - 1)) {
#pragma unroll
            for (int s2 = 0; s2 < NS; ++s2) {
                facc[s2] = __dadd_rn(facc[s2], (double)fp[s2]);
                fp[s2] = FA(0);
            }
        }
    }
    if (FLUX) {
        // one part per (sweep, z segment, y tile, warp) of the strip that owns the face; other warps write 0
        const int64_t nparts = A.nzsegs * A.nytiles * W;
        const int64_t qi = (zseg * A.nytiles + ytile) * W + w;
#pragma unroll
        for (int s2 = 0; s2 < NS; ++s2) {
            double f = facc[s2];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) f = __dadd_rn(f, __shfl_xor_sync(0xffffffffu, f, o));
            if (lane == 0) a.flux_part[s2 * nparts + qi] = __dmul_rn(A.fscale[s2], f);
        }
    }
}

template <typename T, int W, int NH>
__global__ void __launch_bounds__(32 * W, XYMinBlocks<T, W>::value) strang_xy_kernel(const StrangXYArgs A) {
    constexpr int HX = 2 * NH;
    constexpr int OWN = 32 - 2 * HX;
    constexpr int H = W - 2 * HX;
    const SweepArgs &a = A.s;
    const int64_t b = blockIdx.x;
    const int64_t strip = b % A.nstrips;
    const int64_t rest = b / A.nstrips;
    const int64_t ytile = rest % A.nytiles;
    const int64_t zseg = rest / A.nytiles;
    const int64_t nx = a.nx, ny = A.ny;
    const int64_t x0 = strip * OWN - HX, y0 = ytile * H - HX;  // the block's first lane cell and row
    const int64_t face = a.flux_face;
    const bool fblk = face >= 0 && face >= strip * OWN && face < min(strip * OWN + OWN, nx);
    const bool eblk = a.periodic == 0 && (x0 < 0 || x0 + 32 > nx || y0 < 0 || y0 + W > ny);
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    Cx<T> *ych = reinterpret_cast<Cx<T> *>(dyn_smem);  // [2][W][4][32]
    if (fblk) {
        if (eblk) strang_xy_block<T, W, NH, true, true>(A, strip, ytile, zseg, ych);
        else strang_xy_block<T, W, NH, true, false>(A, strip, ytile, zseg, ych);
    } else {
        if (eblk) strang_xy_block<T, W, NH, false, true>(A, strip, ytile, zseg, ych);
        else strang_xy_block<T, W, NH, false, false>(A, strip, ytile, zseg, ych);
    }
    if (face >= 0) finish_flux<2 * NH>(a);
}

template <typename T, bool FIELD>
__global__ void __launch_bounds__(128, ZMinBlocks<T, FIELD>::value) strang_z_kernel(const StrangZArgs a) {
    const int64_t nx = a.nx, ny = a.ny, nz = a.nz;
    const int64_t ncol = nx * ny;
    const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncol) return;
    const bool per = a.periodic != 0;
    const int par = (int)(blockIdx.y & 1);
    using ZI = typename PlaneIdx<T>::type;
    const ZI z_begin = (ZI)((int64_t)(blockIdx.y >> 1) * a.seg_h), z_end = (ZI)min((int64_t)z_begin + a.seg_h, nz);
    const T *in = static_cast<const T *>(a.in);
    T *out = static_cast<T *>(a.out);
    const T *tab = static_cast<const T *>(a.table);
    const int64_t xi = col % nx;
    Cx<T> pu, pd;
    if (!a.full_table) load_tab(tab + xi * 4, pu, pd);
    Cx<T> UM[FIELD ? 6 : 1];  // U entries of this step: Dup, Ddn, Ez, -Ez, Ep, Em (Sec. 2.3)
    if (FIELD) {
        const double *u = a.ucoef + (a.step0 % a.ucoef_n) * 12;
#pragma unroll
        for (int e = 0; e < (FIELD ? 6 : 1); ++e) UM[e] = Cx<T>{(T)__ldg(u + 2 * e), (T)__ldg(u + 2 * e + 1)};
    }
    const int64_t plane = ncol * 8;
    auto load_plane = [&](ZI k, Cx<T> s[4]) {
        if (per || (k >= 0 && k < nz)) {
            const int64_t kl = per ? pmod((int64_t)k, nz) : (int64_t)k;
            load_pt(in + kl * plane + col * 8, s);
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) s[c] = {T(0), T(0)};
        }
    };
    // "+z" sums of the chain's last two input planes (first sweep) and last two phased planes (second)
    Cx<T> R1[2][2], R2[2][2];
#pragma unroll
    for (int t = 0; t < 2; ++t) R1[t][0] = R1[t][1] = R2[t][0] = R2[t][1] = Cx<T>{T(0), T(0)};
    // planes of this thread's parity from z_begin - 4 (or - 3) to z_end + 3 (or + 2)
    const ZI k_first = z_begin - 4 + ((par - z_begin) & 1);
    const ZI k_last = z_end + 3 - (((z_end + 3) - par) & 1);
    constexpr int LA = sizeof(T) == 4 ? 2 : 1;
    // the phase at plane j = k - 2 takes the table entry loaded with input plane k
    auto load_phase = [&](ZI k, Cx<T> &qu, Cx<T> &qd) {
        const ZI j = k - 2;
        if (a.full_table && (per || (j >= 0 && j < nz))) load_tab(tab + ((per ? pmod(j, nz) : j) * ncol + col) * 4, qu, qd);
    };
    Cx<T> pre[LA][4], tpu[LA], tpd[LA];
#pragma unroll
    for (int j = 0; j < LA; ++j) {
        load_plane(k_first + 2 * j, pre[j]);
        tpu[j] = pu;
        tpd[j] = pd;
        load_phase(k_first + 2 * j, tpu[j], tpd[j]);
    }

    for (ZI k0 = k_first; k0 <= k_last; k0 += 4) {
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const ZI k = k0 + 2 * t;
            if (k > k_last) break;
            Cx<T> s[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) s[c] = pre[0][c];
            const Cx<T> qu = tpu[0], qd = tpd[0];
#pragma unroll
            for (int j = 0; j + 1 < LA; ++j) {
#pragma unroll
                for (int c = 0; c < 4; ++c) pre[j][c] = pre[j + 1][c];
                tpu[j] = tpu[j + 1];
                tpd[j] = tpd[j + 1];
            }
            if (k + 2 * LA <= k_last) {
                load_plane(k + 2 * LA, pre[LA - 1]);
                load_phase(k + 2 * LA, tpu[LA - 1], tpd[LA - 1]);
            }
            // C: z sweep, two cells (Eq. sol_dis_3): output plane j = k - 2 from U(k - 4) and W(k)
            const Cx<T> U13 = cadd(s[0], s[2]), U24 = csub(s[1], s[3]);
            const Cx<T> W13 = csub(s[0], s[2]), W24 = cadd(s[1], s[3]);
            Cx<T> o[4];
            o[0] = cadd(R1[t][0], W13);
            o[2] = csub(R1[t][0], W13);
            o[1] = cadd(R1[t][1], W24);
            o[3] = csub(W24, R1[t][1]);
            R1[t][0] = U13;
            R1[t][1] = U24;
            // D: phase of Eq. sol_dis_4 at plane j (zero outside the grid under the zero boundary)
            const ZI j = k - 2;
            if (per || (j >= 0 && j < nz)) {
                if (FIELD) {
                    // (U_ab g) psi_b over the non-zero entries, columns in order, g = the table's exp(-i V dt)
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
                    o[0] = cmulp4(o[0], qu);
                    o[1] = cmulp4(o[1], qu);
                    o[2] = cmulp4(o[2], qd);
                    o[3] = cmulp4(o[3], qd);
                }
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c) o[c] = {T(0), T(0)};
            }
            // C: z sweep, two cells: output plane m = j - 2 from the phased U(j - 4) and W(j)
            const Cx<T> V13 = cadd(o[0], o[2]), V24 = csub(o[1], o[3]);
            const Cx<T> X13 = csub(o[0], o[2]), X24 = cadd(o[1], o[3]);
            Cx<T> r[4];
            r[0] = cadd(R2[t][0], X13);
            r[2] = csub(R2[t][0], X13);
            r[1] = cadd(R2[t][1], X24);
            r[3] = csub(X24, R2[t][1]);
            R2[t][0] = V13;
            R2[t][1] = V24;
            const ZI m = k - 4;
            if (m >= z_begin && m < z_end) store_pt(out + m * plane + col * 8, r);
        }
    }
}

template <typename T, int W, int NH>
static cudaError_t launch_strang_xy_one(const StrangXYArgs &A, cudaStream_t s) {
    const int64_t blocks = A.nstrips * A.nytiles * A.nzsegs;
    if (blocks <= 0) return cudaSuccess;
    const int smem = 2 * W * 4 * 32 * (int)sizeof(Cx<T>);
    static std::atomic<unsigned long long> done{0};
    cudaError_t e = optin_smem(strang_xy_kernel<T, W, NH>, smem, done);
    if (e != cudaSuccess) return e;
    strang_xy_kernel<T, W, NH><<<(unsigned)blocks, 32 * W, smem, s>>>(A);
    return cudaGetLastError();
}

template <typename T, bool FIELD>
static cudaError_t launch_strang_z_one(const StrangZArgs &a, int64_t nsegs, cudaStream_t s) {
    const int64_t ncol = a.nx * a.ny;
    if (ncol <= 0 || nsegs <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((ncol + 127) / 128), (unsigned)(2 * nsegs));  // y: segment x plane parity
    strang_z_kernel<T, FIELD><<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace dirac
