// Fused 3-D first-order step: x sweep, y sweep, z sweep and phase (Eqs. sol_dis_1-sol_dis_4) in one pass
// over HBM, one step per launch.
//
// A block of W warps owns an x strip of 30 cells (one halo cell each side, lane l holds cell xa + l) and
// a tile of W - 2 rows along y; warp w handles row y0 - 1 + w, so warps 0 and W-1 carry the y halo rows.
// The block streams the planes of its z segment (plus one halo plane each side):
//   * each warp loads its row of the plane, x-sweeps it with warp shuffles and writes the row's y
//     characteristics (U = "+y" movers, W = "-y" movers) to shared memory (double-buffered by plane);
//   * after one block barrier the owned warps y-sweep their row from the rows above and below;
//   * the z sweep keeps the "+z" sums of the two previous planes per cell in registers (output plane
//     k - 1 = U(k - 2) + W(k)), then the phase with the table pre-scaled by 1/8, and the store.
// Arithmetic order is that of the two-kernel 3-D path (x-y pass at 4x scale, then z sweep and phase), so
// the FP64 result is the same bit for bit.  Face flux: the lanes holding cells face-1 and face of owned
// rows and planes add 1/2 (|u14|^2+|u23|^2) and subtract 1/2 (|w14|^2+|w23|^2) of the state entering the x
// sweep, to a storage-type partial folded into FP64 every 32 planes.
// FIELD: a uniform vector potential; the phase is the 4 x 4 matrix U(step) exp(-i V dt) of Eq. sol_dis_4
// (table entry g = exp(-i V dt) / 8 times each entry of U, then the column-ordered fma chains of the 2-D
// kernel), one launch = one step whose index selects the row of the U table.
// 64-bit fixed-point states (T = long long): the sweeps are exact integer sums, so any order gives the bits
// of the two-kernel path; the phase is the rounded 128-bit product (the table holding round(p 2^62) with the
// 1/8); the face terms are formed in FP64 from the converted values and scaled by the state's 2^-2S.
#pragma once

#include "step_kernels.cuh"

namespace dirac {

struct Fused3DArgs {
    SweepArgs s;          // in, out, table, flux fields; s.nsegs * s.nplanes = flux parts
    int64_t ny, nz;
    int64_t nstrips, nytiles, nzsegs, zseg_h;
};

// accumulator type of the face terms: the storage type, FP64 for fixed-point states
template <typename T> struct FaceAcc { using type = T; };
template <> struct FaceAcc<long long> { using type = double; };
// plane index type of the z loop: 32-bit for floating-point states (grid dimensions stay below 2^31), 64-bit for
// the fixed-point state (register budget)
template <typename T> struct PlaneIdx { using type = int; };
template <> struct PlaneIdx<long long> { using type = int64_t; };

// |p14|^2 + |p23|^2 as a fused chain in the accumulator type
template <typename T>
__device__ __forceinline__ typename FaceAcc<T>::type face_sq(Cx<T> p14, Cx<T> p23) {
    using F = typename FaceAcc<T>::type;
    return Ar<F>::fma((F)p14.re, (F)p14.re,
                      Ar<F>::fma((F)p14.im, (F)p14.im, Ar<F>::fma((F)p23.re, (F)p23.re, Ar<F>::mul((F)p23.im, (F)p23.im))));
}

template <typename T, int W, bool FIELD>
__global__ void __launch_bounds__(32 * W, 1) fused3d_kernel(const Fused3DArgs A) {
    constexpr int H = W - 2;
    const SweepArgs &a = A.s;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t b = blockIdx.x;
    const int64_t strip = b % A.nstrips;
    const int64_t rest = b / A.nstrips;
    const int64_t ytile = rest % A.nytiles;
    const int64_t zseg = rest / A.nytiles;
    const int64_t nx = a.nx, ny = A.ny, nz = A.nz;
    const bool per = a.periodic != 0;
    const int64_t x_own0 = strip * 30, x_own1 = min(x_own0 + 30, nx);
    const int64_t x = x_own0 - 1 + lane;
    const int64_t y = ytile * H - 1 + w;
    const bool owned_row = w >= 1 && w <= H && y < ny;
    using ZI = typename PlaneIdx<T>::type;
    const ZI z_begin = (ZI)(zseg * A.zseg_h), z_end = (ZI)min((int64_t)z_begin + A.zseg_h, nz);
    const bool xin = x >= 0 && x < nx, yin = y >= 0 && y < ny;
    const int64_t xl = per ? pmod(x, nx) : min(max(x, (int64_t)0), nx - 1);
    const int64_t yl = per ? pmod(y, ny) : min(max(y, (int64_t)0), ny - 1);
    const T *in = static_cast<const T *>(a.in);
    T *out = static_cast<T *>(a.out);
    const T *tab = static_cast<const T *>(a.table);

    extern __shared__ __align__(16) unsigned char dyn_smem[];
    Cx<T> *ych = reinterpret_cast<Cx<T> *>(dyn_smem);  // [2][W][4][32]

    Cx<T> pu, pd;
    if (!a.full_table) load_tab(tab + xl * 4, pu, pd);
    Cx<T> UM[FIELD ? 6 : 1];  // entries of U for this launch's step: Dup, Ddn, Ez, -Ez, Ep, Em
    if (FIELD) {
        const double *u = a.ucoef + (a.step0 % a.ucoef_n) * 12;
#pragma unroll
        for (int e = 0; e < (FIELD ? 6 : 1); ++e) UM[e] = Cx<T>{(T)__ldg(u + 2 * e), (T)__ldg(u + 2 * e + 1)};
    }
    const int64_t face = a.flux_face;
    const bool face_lane = owned_row && face >= x_own0 && face < x_own1 && (x == face - 1 || x == face);
    double facc = 0.0;
    typename FaceAcc<T>::type fpart = 0;

    Cx<T> UA[2] = {{T(0), T(0)}, {T(0), T(0)}}, UB[2] = {{T(0), T(0)}, {T(0), T(0)}};

    // cell (xl, yl) of a plane: plane k at (k nx ny + cell) (periodic: halo planes wrap)
    const int64_t plane_cells = nx * ny, cell = yl * nx + xl;
    auto wrap_z = [&](ZI k) -> int64_t {
        if (per && (k < 0 || k >= nz)) return pmod((int64_t)k, nz);
        return k;
    };
    auto load_row = [&](ZI k, Cx<T> s[4]) {
        const bool ok = per || (yin && k >= 0 && k < nz && xin);
        if (ok) {
            load_pt(in + (wrap_z(k) * plane_cells + cell) * 8, s);
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) s[c] = {T(0), T(0)};
        }
    };
    // rows of the next planes in flight: one ahead in FP64 (bound by the FP64 pipe), two in FP32 (three or
    // four measured no faster at 256^3 and 384^3: the per-plane block barrier is the limit there)
    constexpr int LA = sizeof(T) == 4 ? 2 : 1;
    Cx<T> ring[LA][4];
#pragma unroll
    for (int j = 0; j < LA; ++j)
        if (z_begin - 1 + j <= z_end) load_row(z_begin - 1 + j, ring[j]);

    // per-cell table entries of the next output plane, loaded one plane ahead (full table only)
    Cx<T> tu = pu, td = pd, tu_next = pu, td_next = pd;

    for (ZI k = z_begin - 1; k <= z_end; ++k) {
        if (a.full_table && owned_row) {
            tu = tu_next;
            td = td_next;
            if (k >= z_begin && k < z_end) load_tab(tab + ((int64_t)k * plane_cells + cell) * 4, tu_next, td_next);
        }
        Cx<T> st[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) st[c] = ring[0][c];
#pragma unroll
        for (int j = 0; j + 1 < LA; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) ring[j][c] = ring[j + 1][c];
        if (k + LA <= z_end) load_row(k + LA, ring[LA - 1]);
        // x characteristics and the x sweep (neighbours by shuffle; lanes 0 and 31 are halo cells)
        const Cx<T> u14 = cadd(st[0], st[3]), w14 = csub(st[0], st[3]);
        const Cx<T> u23 = cadd(st[1], st[2]), w23 = csub(st[1], st[2]);
        if (face_lane && k >= z_begin && k < z_end) {
            using F = typename FaceAcc<T>::type;
            const F v = (x == face - 1) ? face_sq(u14, u23) : -face_sq(w14, w23);
            fpart = Ar<F>::add(fpart, v);
            if (((k - z_begin) & 31) == 31 || k == z_end - 1) {
                facc = __dadd_rn(facc, (double)fpart);
                fpart = 0;
            }
        }
        const Cx<T> lu14 = shfl_c(u14, (lane + 31) & 31), lu23 = shfl_c(u23, (lane + 31) & 31);
        const Cx<T> rw14 = shfl_c(w14, (lane + 1) & 31), rw23 = shfl_c(w23, (lane + 1) & 31);
        const Cx<T> b0 = cadd(lu14, rw14), b3 = csub(lu14, rw14);
        const Cx<T> b1 = cadd(lu23, rw23), b2 = csub(lu23, rw23);
        // y characteristics (Eq. sol_dis_2): "+y" movers (b1 - i b4, b2 + i b3), "-y" movers (b1 + i b4, b2 - i b3)
        Cx<T> *buf = ych + (size_t)((k - z_begin + 1) & 1) * (W * 4 * 32);
        buf[(w * 4 + 0) * 32 + lane] = csub_ib(b0, b3);
        buf[(w * 4 + 1) * 32 + lane] = cadd_ib(b1, b2);
        buf[(w * 4 + 2) * 32 + lane] = cadd_ib(b0, b3);
        buf[(w * 4 + 3) * 32 + lane] = csub_ib(b1, b2);
        __syncthreads();
        if (owned_row) {
            // y sweep of row y: "+y" movers of row y-1, "-y" movers of row y+1 (x2 again: 4x the state)
            const Cx<T> U14 = buf[((w - 1) * 4 + 0) * 32 + lane], U23 = buf[((w - 1) * 4 + 1) * 32 + lane];
            const Cx<T> W14 = buf[((w + 1) * 4 + 2) * 32 + lane], W23 = buf[((w + 1) * 4 + 3) * 32 + lane];
            Cx<T> s[4];
            s[0] = cadd(U14, W14);
            s[3] = cmul_i(csub(U14, W14));
            s[1] = cadd(U23, W23);
            s[2] = cmul_mi(csub(U23, W23));
            // z sweep (Eq. sol_dis_3): +z movers (s1+s3, s2-s4) of plane k-2, -z movers (s1-s3, s2+s4) of plane k
            const Cx<T> U13 = cadd(s[0], s[2]), U24 = csub(s[1], s[3]);
            const Cx<T> W13 = csub(s[0], s[2]), W24 = cadd(s[1], s[3]);
            const ZI zo = k - 1;
            if (zo >= z_begin && zo < z_end) {
                Cx<T> o[4];
                o[0] = cadd(UA[0], W13);
                o[2] = csub(UA[0], W13);
                o[1] = cadd(UA[1], W24);
                o[3] = csub(W24, UA[1]);
                const Cx<T> qu = a.full_table ? tu : pu, qd = a.full_table ? td : pd;
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
                if (x >= x_own0 && x < x_own1) store_pt(out + ((int64_t)zo * plane_cells + cell) * 8, o);
            }
            UA[0] = UB[0];
            UA[1] = UB[1];
            UB[0] = U13;
            UB[1] = U24;
        }
    }
    if (face >= 0 && face >= x_own0 && face < x_own1) {
        // one flux part per (y tile, z segment, warp) of the strip that owns the face; halo warps write 0
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) facc = __dadd_rn(facc, __shfl_xor_sync(0xffffffffu, facc, o));
        if (lane == 0) a.flux_part[(zseg * A.nytiles + ytile) * W + w] = __dmul_rn(0.5 * a.flux_unit, facc);
    }
    if (face >= 0) finish_flux<1>(a);
}

// Two first-order steps per pass (temporal block k = 2): HBM is read and written once per two steps.
// The block's strip is 28 cells (two halo lanes each side) by W - 4 rows (two halo rows each side), and
// the block streams its z segment plus two halo planes each side.  Per input plane k:
//   * step 1: every warp x-sweeps its row and writes its y characteristics to shared memory; after a
//     barrier the rows one inside the halo y-sweep, z-sweep (register history of the "+z" sums of the
//     previous two planes) and take the phase: the state after step 1 at plane k - 1, zeroed outside the
//     grid (zero boundary: cells outside are zero at every sub-step);
//   * step 2: those rows x-sweep it and write its y characteristics; after a second barrier the owned
//     rows y-sweep, z-sweep (their own history) and take the phase of step 2: plane k - 2, stored.
// Each step's arithmetic is that of the one-step kernel, so the result equals two one-step launches bit for
// bit.  Both steps' face flux is taken on the state entering their x sweep (parts [2][nzsegs nytiles W]).
// FIELD: the phase matrices of steps step0 and step0 + 1.
template <typename T, int W, bool FIELD>
__global__ void __launch_bounds__(32 * W, 1) fused3d2_kernel(const Fused3DArgs A) {
    constexpr int H = W - 4;
    const SweepArgs &a = A.s;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t b = blockIdx.x;
    const int64_t strip = b % A.nstrips;
    const int64_t rest = b / A.nstrips;
    const int64_t ytile = rest % A.nytiles;
    const int64_t zseg = rest / A.nytiles;
    const int64_t nx = a.nx, ny = A.ny, nz = A.nz;
    const bool per = a.periodic != 0;
    const int64_t x_own0 = strip * 28, x_own1 = min(x_own0 + 28, nx);
    const int64_t x = x_own0 - 2 + lane;
    const int64_t y = ytile * H - 2 + w;
    const bool owned_row = w >= 2 && w < W - 2 && y < ny;
    const bool mid_row = w >= 1 && w < W - 1;
    const bool own_lane = x >= x_own0 && x < x_own1;
    using ZI = typename PlaneIdx<T>::type;
    const ZI z_begin = (ZI)(zseg * A.zseg_h), z_end = (ZI)min((int64_t)z_begin + A.zseg_h, nz);
    const bool xin = x >= 0 && x < nx, yin = y >= 0 && y < ny;
    const bool ghost_xy = !per && !(xin && yin);
    const int64_t xl = per ? pmod(x, nx) : min(max(x, (int64_t)0), nx - 1);
    const int64_t yl = per ? pmod(y, ny) : min(max(y, (int64_t)0), ny - 1);
    const T *in = static_cast<const T *>(a.in);
    T *out = static_cast<T *>(a.out);
    const T *tab = static_cast<const T *>(a.table);

    extern __shared__ __align__(16) unsigned char dyn_smem[];
    Cx<T> *buf1 = reinterpret_cast<Cx<T> *>(dyn_smem);  // [W][4][32] step 1's y characteristics
    Cx<T> *buf2 = buf1 + W * 4 * 32;                    // [W][4][32] step 2's

    Cx<T> pu = {T(0), T(0)}, pd = {T(0), T(0)};
    if (!a.full_table) load_tab(tab + xl * 4, pu, pd);
    Cx<T> UM[2][FIELD ? 6 : 1];  // entries of U for the two steps: Dup, Ddn, Ez, -Ez, Ep, Em
    if (FIELD) {
#pragma unroll
        for (int st = 0; st < 2; ++st) {
            const double *u = a.ucoef + ((a.step0 + st) % a.ucoef_n) * 12;
#pragma unroll
            for (int e = 0; e < (FIELD ? 6 : 1); ++e)
                UM[st][e] = Cx<T>{(T)__ldg(u + 2 * e), (T)__ldg(u + 2 * e + 1)};
        }
    }
    const int64_t face = a.flux_face;
    const bool face_warp = owned_row && face >= x_own0 && face < x_own1;
    const bool fl_u = face_warp && x == face - 1, fl_w = face_warp && x == face;
    double facc[2] = {0.0, 0.0};
    T fp[2] = {T(0), T(0)};

    // cell (xl, yl) of a plane: plane k at (k nx ny + cell) (periodic: halo planes wrap)
    const int64_t plane_cells = nx * ny, cell = yl * nx + xl;
    auto wrap_z = [&](ZI k) -> int64_t {
        if (per && (k < 0 || k >= nz)) return pmod((int64_t)k, nz);
        return k;
    };
    auto load_row = [&](ZI k, Cx<T> s[4]) {
        const bool ok = per || (yin && k >= 0 && k < nz && xin);
        if (ok) {
            load_pt(in + (wrap_z(k) * plane_cells + cell) * 8, s);
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) s[c] = {T(0), T(0)};
        }
    };
    auto face_term = [&](Cx<T> p14, Cx<T> p23) -> T {
        return Ar<T>::fma(p14.re, p14.re, Ar<T>::fma(p14.im, p14.im, Ar<T>::fma(p23.re, p23.re, Ar<T>::mul(p23.im, p23.im))));
    };
    // x sweep of a row held one cell per lane (valid where both neighbours are); face terms of its input
    auto xsweep = [&](const Cx<T> s[4], Cx<T> o[4], T &acc, bool count) {
        const Cx<T> u14 = cadd(s[0], s[3]), w14 = csub(s[0], s[3]);
        const Cx<T> u23 = cadd(s[1], s[2]), w23 = csub(s[1], s[2]);
        if (count && fl_u) acc = Ar<T>::add(acc, face_term(u14, u23));
        if (count && fl_w) acc = Ar<T>::sub(acc, face_term(w14, w23));
        const Cx<T> lu14 = shfl_c(u14, (lane + 31) & 31), lu23 = shfl_c(u23, (lane + 31) & 31);
        const Cx<T> rw14 = shfl_c(w14, (lane + 1) & 31), rw23 = shfl_c(w23, (lane + 1) & 31);
        o[0] = cadd(lu14, rw14);
        o[3] = csub(lu14, rw14);
        o[1] = cadd(lu23, rw23);
        o[2] = csub(lu23, rw23);
    };
    // y characteristics (Eq. sol_dis_2): "+y" movers (b1 - i b4, b2 + i b3), "-y" movers (b1 + i b4, b2 - i b3)
    auto ywrite = [&](Cx<T> *buf, const Cx<T> b4[4]) {
        buf[(w * 4 + 0) * 32 + lane] = csub_ib(b4[0], b4[3]);
        buf[(w * 4 + 1) * 32 + lane] = cadd_ib(b4[1], b4[2]);
        buf[(w * 4 + 2) * 32 + lane] = cadd_ib(b4[0], b4[3]);
        buf[(w * 4 + 3) * 32 + lane] = csub_ib(b4[1], b4[2]);
    };
    // y sweep from rows w - 1 and w + 1, z sweep against the history (output plane = input plane - 1), phase
    auto yz_phase = [&](const Cx<T> *buf, Cx<T> (&HA)[2], Cx<T> (&HB)[2], Cx<T> qu, Cx<T> qd, int st, Cx<T> o[4]) {
        const Cx<T> U14 = buf[((w - 1) * 4 + 0) * 32 + lane], U23 = buf[((w - 1) * 4 + 1) * 32 + lane];
        const Cx<T> W14 = buf[((w + 1) * 4 + 2) * 32 + lane], W23 = buf[((w + 1) * 4 + 3) * 32 + lane];
        Cx<T> s[4];
        s[0] = cadd(U14, W14);
        s[3] = cmul_i(csub(U14, W14));
        s[1] = cadd(U23, W23);
        s[2] = cmul_mi(csub(U23, W23));
        const Cx<T> U13 = cadd(s[0], s[2]), U24 = csub(s[1], s[3]);
        const Cx<T> W13 = csub(s[0], s[2]), W24 = cadd(s[1], s[3]);
        o[0] = cadd(HA[0], W13);
        o[2] = csub(HA[0], W13);
        o[1] = cadd(HA[1], W24);
        o[3] = csub(W24, HA[1]);
        HA[0] = HB[0];
        HA[1] = HB[1];
        HB[0] = U13;
        HB[1] = U24;
        if (FIELD) {
            Cx<T> m6[FIELD ? 6 : 1];
#pragma unroll
            for (int e = 0; e < (FIELD ? 6 : 1); ++e) m6[e] = cmulp(UM[st][e], qu);
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
    };

    constexpr int LA = sizeof(T) == 4 ? 2 : 1;
    const ZI k_first = z_begin - 2, k_last = z_end + 1;
    Cx<T> ring[LA][4];
#pragma unroll
    for (int j = 0; j < LA; ++j)
        if (k_first + j <= k_last) load_row(k_first + j, ring[j]);
    Cx<T> H1A[2] = {{T(0), T(0)}, {T(0), T(0)}}, H1B[2] = {{T(0), T(0)}, {T(0), T(0)}};
    Cx<T> H2A[2] = {{T(0), T(0)}, {T(0), T(0)}}, H2B[2] = {{T(0), T(0)}, {T(0), T(0)}};
    // per-cell table entries (full table): step 1 at plane k - 1 (rows one inside the halo), step 2 at k - 2
    auto table_at = [&](ZI j, Cx<T> &qu, Cx<T> &qd) {
        qu = pu;
        qd = pd;
        if (a.full_table && (per || (j >= 0 && j < nz)))
            load_tab(tab + (wrap_z(j) * plane_cells + cell) * 4, qu, qd);
    };
    Cx<T> t1u, t1d, t2u, t2d;
    table_at(k_first - 1, t1u, t1d);
    table_at(k_first - 2, t2u, t2d);

    for (ZI k = k_first; k <= k_last; ++k) {
        Cx<T> st[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) st[c] = ring[0][c];
#pragma unroll
        for (int j = 0; j + 1 < LA; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) ring[j][c] = ring[j + 1][c];
        if (k + LA <= k_last) load_row(k + LA, ring[LA - 1]);
        const Cx<T> q1u = t1u, q1d = t1d, q2u = t2u, q2d = t2d;
        if (mid_row) table_at(k, t1u, t1d);            // step 1's next plane
        if (owned_row) table_at(k - 1, t2u, t2d);      // step 2's next plane

        // step 1: x sweep of input plane k
        Cx<T> b4[4];
        xsweep(st, b4, fp[0], k >= z_begin && k < z_end);
        ywrite(buf1, b4);
        __syncthreads();
        const ZI j1 = k - 1;  // step 1's output plane
        if (mid_row) {
            Cx<T> o[4];
            yz_phase(buf1, H1A, H1B, q1u, q1d, 0, o);
            if (ghost_xy || (!per && (j1 < 0 || j1 >= nz))) {
#pragma unroll
                for (int c = 0; c < 4; ++c) o[c] = {T(0), T(0)};
            }
            // step 2: x sweep of plane j1
            xsweep(o, b4, fp[1], j1 >= z_begin && j1 < z_end);
            ywrite(buf2, b4);
        }
        __syncthreads();
        const ZI m = k - 2;  // step 2's output plane
        if (owned_row) {
            Cx<T> o[4];
            yz_phase(buf2, H2A, H2B, q2u, q2d, 1, o);
            if (own_lane && m >= z_begin && m < z_end) store_pt(out + ((int64_t)m * plane_cells + cell) * 8, o);
        }
        if ((fl_u || fl_w) && (((k - k_first) & 31) == 31 || k == k_last)) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                facc[q] = __dadd_rn(facc[q], (double)fp[q]);
                fp[q] = T(0);
            }
        }
    }
    if (face >= 0 && face >= x_own0 && face < x_own1) {
        // one part per (step, z segment, y tile, warp) of the strip that owns the face; other warps write 0
        const int64_t nparts = A.nzsegs * A.nytiles * W;
        const int64_t q = (zseg * A.nytiles + ytile) * W + w;
#pragma unroll
        for (int st = 0; st < 2; ++st) {
            double f = facc[st];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) f = __dadd_rn(f, __shfl_xor_sync(0xffffffffu, f, o));
            if (lane == 0) a.flux_part[st * nparts + q] = __dmul_rn(0.5, f);
        }
    }
    if (face >= 0) finish_flux<2>(a);
}

template <typename T, int W, bool FIELD>
static cudaError_t launch_fused3d2_one(const Fused3DArgs &A, cudaStream_t s) {
    const int64_t blocks = A.nstrips * A.nytiles * A.nzsegs;
    if (blocks <= 0) return cudaSuccess;
    const int smem = 2 * W * 4 * 32 * (int)sizeof(Cx<T>);
    static std::atomic<unsigned long long> done{0};
    cudaError_t e = optin_smem(fused3d2_kernel<T, W, FIELD>, smem, done);
    if (e != cudaSuccess) return e;
    fused3d2_kernel<T, W, FIELD><<<(unsigned)blocks, 32 * W, smem, s>>>(A);
    return cudaGetLastError();
}

template <typename T, int W, bool FIELD>
static cudaError_t launch_fused3d_one(const Fused3DArgs &A, cudaStream_t s) {
    const int64_t blocks = A.nstrips * A.nytiles * A.nzsegs;
    if (blocks <= 0) return cudaSuccess;
    const int smem = 2 * W * 4 * 32 * (int)sizeof(Cx<T>);
    static std::atomic<unsigned long long> done{0};
    cudaError_t e = optin_smem(fused3d_kernel<T, W, FIELD>, smem, done);
    if (e != cudaSuccess) return e;
    fused3d_kernel<T, W, FIELD><<<(unsigned)blocks, 32 * W, smem, s>>>(A);
    return cudaGetLastError();
}

}  // namespace dirac
