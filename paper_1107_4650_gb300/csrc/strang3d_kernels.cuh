// Fused passes of the 3-D second-order step (Sec. 2.4, dt = 4 dx / c):
//   A(1) B(2) A(1) | C(2) D C(2) | A(1) B(2) A(1)     (cells moved per sweep in parentheses)
// run as three passes over HBM instead of eight single-sweep launches: an x-y-x pass, a z-phase-z pass and
// the x-y-x pass again.  Arithmetic is that of the single-sweep kernels (axis_kernels.cuh), operation by
// operation, so the result is the same bit for bit in either storage precision; only where the
// intermediate states live changes (registers and shared memory instead of HBM).
//
// x-y-x pass (per z plane; planes are independent): a block of W warps owns a 28-cell x strip (lane l
// holds cell x0 - 2 + l: two halo cells each side, one per x sweep) and W - 4 rows along y (warp w holds
// row y0 - 2 + w: two halo rows each side for the two-cell y sweep).  Per plane:
//   * every warp loads its row, x-sweeps it with shuffles (valid on lanes 1..30) and writes the row's
//     y characteristics to shared memory (double-buffered by plane: one block barrier per plane);
//   * the owned warps y-sweep their row from rows y - 2 ("+y" movers) and y + 2 ("-y" movers), zero the
//     cells outside the grid (zero boundary), x-sweep again (valid on lanes 2..29) and store.
// Face flux: both x sweeps add, on the face strip's owned rows, 1/2 (|u14|^2 + |u23|^2) of cell face - 1
// and subtract 1/2 (|w14|^2 + |w23|^2) of cell face, of the state entering that sweep, times 1 / s^2 for
// the state's scale s; one part per (sweep, z segment, y tile, warp), folded by the last block.
//
// z-phase-z pass: the two-cell z sweeps couple plane k only with planes k - 2 and k + 2, and the phase is
// pointwise, so even and odd planes form two independent chains.  One thread per (x, y) column and plane
// parity streams its chain over a segment of planes (plus four halo planes each side).  Input plane k
// gives the characteristic sums U = (s1 + s3, s2 - s4) and W = (s1 - s3, s2 + s4); the first sweep's output
// at plane j = k - 2 is U(j - 2) + W(j + 2) (U of the chain's last two planes in a register ring), the phase
// of Eq. sol_dis_4 (table carrying the eight sweeps' 1/256) follows, cells outside the grid are zeroed,
// and the second sweep's output at plane k - 4 is formed the same way from a second ring.  The loop takes
// two chain planes per iteration so every ring index is a constant.
#pragma once

#include "step_kernels.cuh"

namespace dirac {

struct StrangXYArgs {
    SweepArgs s;          // in, out, flux fields; flux parts [2][nzsegs * nytiles * W]
    int64_t ny, nz;
    int64_t nstrips, nytiles, nzsegs, zseg_h;
    double fscale0, fscale1;  // 1/2 over the square of the scale of the state entering each x sweep
};

struct StrangZArgs {
    const void *in;
    void *out;
    const void *table;
    int64_t nx, ny, nz;
    int64_t seg_h;        // planes per z segment (blockIdx.y = segment)
    int periodic, full_table;
    const double *ucoef;  // uniform vector potential: U entries per step (12 doubles), or null
    int64_t ucoef_n, step0;
};

// resident blocks per SM the register budget is fitted to: two 16-warp blocks in FP32
template <typename T, int W> struct XYMinBlocks { static constexpr int value = (sizeof(T) == 4 && W == 16) ? 2 : 1; };
// z-phase-z pass: 128-thread blocks per SM the register budget is fitted to
template <typename T, bool FIELD> struct ZMinBlocks { static constexpr int value = sizeof(T) == 4 ? (FIELD ? 4 : 5) : (FIELD ? 3 : 4); };

template <typename T, int W>
__global__ void __launch_bounds__(32 * W, XYMinBlocks<T, W>::value) strang_xy_kernel(const StrangXYArgs A) {
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
    const bool own_lane = x >= x_own0 && x < x_own1;
    const int64_t z_begin = zseg * A.zseg_h, z_end = min(z_begin + A.zseg_h, nz);
    const bool xin = x >= 0 && x < nx, yin = y >= 0 && y < ny;
    const int64_t xl = per ? pmod(x, nx) : min(max(x, (int64_t)0), nx - 1);
    const int64_t yl = per ? pmod(y, ny) : min(max(y, (int64_t)0), ny - 1);
    const T *in = static_cast<const T *>(a.in);
    T *out = static_cast<T *>(a.out);

    extern __shared__ __align__(16) unsigned char dyn_smem[];
    Cx<T> *ych = reinterpret_cast<Cx<T> *>(dyn_smem);  // [2][W][4][32]

    const int64_t face = a.flux_face;
    const bool face_warp = owned_row && face >= x_own0 && face < x_own1;
    const bool fl_u = face_warp && x == face - 1, fl_w = face_warp && x == face;
    double facc0 = 0.0, facc1 = 0.0;
    T fp0 = T(0), fp1 = T(0);

    const bool row_ok = per || (yin && xin);
    auto load_row = [&](int64_t k, Cx<T> s[4]) {
        if (row_ok) {
            load_pt(in + ((k * ny + yl) * nx + xl) * 8, s);
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) s[c] = {T(0), T(0)};
        }
    };
    // planes in flight: two ahead in FP32 (bandwidth-bound), one in FP64
    constexpr int LA = sizeof(T) == 4 ? 2 : 1;
    Cx<T> ring[LA][4];
#pragma unroll
    for (int j = 0; j < LA; ++j)
        if (z_begin + j < z_end) load_row(z_begin + j, ring[j]);

    auto face_term = [&](Cx<T> p14, Cx<T> p23) -> T {
        return Ar<T>::fma(p14.re, p14.re, Ar<T>::fma(p14.im, p14.im, Ar<T>::fma(p23.re, p23.re, Ar<T>::mul(p23.im, p23.im))));
    };

    for (int64_t k = z_begin; k < z_end; ++k) {
        Cx<T> st[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) st[c] = ring[0][c];
#pragma unroll
        for (int j = 0; j + 1 < LA; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) ring[j][c] = ring[j + 1][c];
        if (k + LA < z_end) load_row(k + LA, ring[LA - 1]);

        // A: x sweep, one cell (Eq. sol_dis_1)
        const Cx<T> u14 = cadd(st[0], st[3]), w14 = csub(st[0], st[3]);
        const Cx<T> u23 = cadd(st[1], st[2]), w23 = csub(st[1], st[2]);
        if (fl_u) fp0 = Ar<T>::add(fp0, face_term(u14, u23));
        if (fl_w) fp0 = Ar<T>::sub(fp0, face_term(w14, w23));
        const Cx<T> lu14 = shfl_c(u14, (lane + 31) & 31), lu23 = shfl_c(u23, (lane + 31) & 31);
        const Cx<T> rw14 = shfl_c(w14, (lane + 1) & 31), rw23 = shfl_c(w23, (lane + 1) & 31);
        const Cx<T> a0 = cadd(lu14, rw14), a3 = csub(lu14, rw14);
        const Cx<T> a1 = cadd(lu23, rw23), a2 = csub(lu23, rw23);
        // y characteristics (Eq. sol_dis_2): "+y" movers (a1 - i a4, a2 + i a3), "-y" movers (a1 + i a4, a2 - i a3)
        Cx<T> *buf = ych + (size_t)((k - z_begin) & 1) * (W * 4 * 32);
        buf[(w * 4 + 0) * 32 + lane] = csub_ib(a0, a3);
        buf[(w * 4 + 1) * 32 + lane] = cadd_ib(a1, a2);
        buf[(w * 4 + 2) * 32 + lane] = cadd_ib(a0, a3);
        buf[(w * 4 + 3) * 32 + lane] = csub_ib(a1, a2);
        __syncthreads();
        if (owned_row) {
            // B: y sweep, two cells: "+y" movers of row y - 2, "-y" movers of row y + 2
            const Cx<T> U14 = buf[((w - 2) * 4 + 0) * 32 + lane], U23 = buf[((w - 2) * 4 + 1) * 32 + lane];
            const Cx<T> W14 = buf[((w + 2) * 4 + 2) * 32 + lane], W23 = buf[((w + 2) * 4 + 3) * 32 + lane];
            Cx<T> q[4];
            q[0] = cadd(U14, W14);
            q[3] = cmul_i(csub(U14, W14));
            q[1] = cadd(U23, W23);
            q[2] = cmul_mi(csub(U23, W23));
            if (!per && !xin) {
#pragma unroll
                for (int c = 0; c < 4; ++c) q[c] = {T(0), T(0)};
            }
            // A: x sweep, one cell
            const Cx<T> v14 = cadd(q[0], q[3]), x14 = csub(q[0], q[3]);
            const Cx<T> v23 = cadd(q[1], q[2]), x23 = csub(q[1], q[2]);
            if (fl_u) fp1 = Ar<T>::add(fp1, face_term(v14, v23));
            if (fl_w) fp1 = Ar<T>::sub(fp1, face_term(x14, x23));
            const Cx<T> lv14 = shfl_c(v14, (lane + 31) & 31), lv23 = shfl_c(v23, (lane + 31) & 31);
            const Cx<T> rx14 = shfl_c(x14, (lane + 1) & 31), rx23 = shfl_c(x23, (lane + 1) & 31);
            Cx<T> o[4];
            o[0] = cadd(lv14, rx14);
            o[3] = csub(lv14, rx14);
            o[1] = cadd(lv23, rx23);
            o[2] = csub(lv23, rx23);
            if (own_lane) store_pt(out + ((k * ny + y) * nx + x) * 8, o);
        }
        if ((fl_u || fl_w) && (((k - z_begin) & 31) == 31 || k == z_end - 1)) {
            facc0 = __dadd_rn(facc0, (double)fp0);
            facc1 = __dadd_rn(facc1, (double)fp1);
            fp0 = T(0);
            fp1 = T(0);
        }
    }
    if (face >= 0 && face >= x_own0 && face < x_own1) {
        // one part per (sweep, z segment, y tile, warp) of the strip that owns the face; other warps write 0
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            facc0 = __dadd_rn(facc0, __shfl_xor_sync(0xffffffffu, facc0, o));
            facc1 = __dadd_rn(facc1, __shfl_xor_sync(0xffffffffu, facc1, o));
        }
        const int64_t nparts = A.nzsegs * A.nytiles * W;
        const int64_t q = (zseg * A.nytiles + ytile) * W + w;
        if (lane == 0) {
            a.flux_part[q] = __dmul_rn(A.fscale0, facc0);
            a.flux_part[nparts + q] = __dmul_rn(A.fscale1, facc1);
        }
    }
    if (face >= 0) finish_flux<2>(a);
}

template <typename T, bool FIELD>
__global__ void __launch_bounds__(128, ZMinBlocks<T, FIELD>::value) strang_z_kernel(const StrangZArgs a) {
    const int64_t nx = a.nx, ny = a.ny, nz = a.nz;
    const int64_t ncol = nx * ny;
    const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncol) return;
    const bool per = a.periodic != 0;
    const int par = (int)(blockIdx.y & 1);
    const int64_t z_begin = (int64_t)(blockIdx.y >> 1) * a.seg_h, z_end = min(z_begin + a.seg_h, nz);
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
    auto load_plane = [&](int64_t k, Cx<T> s[4]) {
        if (per || (k >= 0 && k < nz)) {
            const int64_t kl = per ? pmod(k, nz) : k;
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
    const int64_t k_first = z_begin - 4 + ((par - z_begin) & 1);
    const int64_t k_last = z_end + 3 - (((z_end + 3) - par) & 1);
    constexpr int LA = sizeof(T) == 4 ? 2 : 1;
    Cx<T> pre[LA][4];
#pragma unroll
    for (int j = 0; j < LA; ++j) load_plane(k_first + 2 * j, pre[j]);

    for (int64_t k0 = k_first; k0 <= k_last; k0 += 4) {
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int64_t k = k0 + 2 * t;
            if (k > k_last) break;
            Cx<T> s[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) s[c] = pre[0][c];
#pragma unroll
            for (int j = 0; j + 1 < LA; ++j)
#pragma unroll
                for (int c = 0; c < 4; ++c) pre[j][c] = pre[j + 1][c];
            if (k + 2 * LA <= k_last) load_plane(k + 2 * LA, pre[LA - 1]);
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
            const int64_t j = k - 2;
            if (per || (j >= 0 && j < nz)) {
                Cx<T> qu = pu, qd = pd;
                if (a.full_table) load_tab(tab + ((per ? pmod(j, nz) : j) * ncol + col) * 4, qu, qd);
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
                    o[0] = cmulp(o[0], qu);
                    o[1] = cmulp(o[1], qu);
                    o[2] = cmulp(o[2], qd);
                    o[3] = cmulp(o[3], qd);
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
            const int64_t m = k - 4;
            if (m >= z_begin && m < z_end) store_pt(out + m * plane + col * 8, r);
        }
    }
}

template <typename T, int W>
static cudaError_t launch_strang_xy_one(const StrangXYArgs &A, cudaStream_t s) {
    const int64_t blocks = A.nstrips * A.nytiles * A.nzsegs;
    if (blocks <= 0) return cudaSuccess;
    const int smem = 2 * W * 4 * 32 * (int)sizeof(Cx<T>);
    static unsigned long long done = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 64 || !(done & (1ull << dev))) {
        cudaError_t e = cudaFuncSetAttribute(strang_xy_kernel<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        if (dev < 64) done |= 1ull << dev;
    }
    strang_xy_kernel<T, W><<<(unsigned)blocks, 32 * W, smem, s>>>(A);
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
