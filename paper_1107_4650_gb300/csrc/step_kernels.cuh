// Fused sweep kernels of the split-operator Dirac scheme (Sec. 2.3, Eqs. sol_dis_1-sol_dis_4).
//
// Design (one warp = one independent strip, no shared memory, no block barrier):
//   * a warp owns `strip_w` consecutive x cells of one plane and a segment of rows; it loads
//     32*P cells per row (lane l holds cells xa + 32 j + l, j < P), i.e. K halo cells on each side;
//   * it streams the rows of its segment (plus K halo rows at each end) through K pipelined
//     levels held in registers: level s turns the step-(s-1) state of row q into the step-s state
//     of row q-1, so one pass over HBM advances K steps (temporal blocking);
//   * the x sweep needs cells x-1 and x+1: the characteristic sums u = a+b of the left neighbour
//     and w = a-b of the right neighbour come from warp shuffles;
//   * the second sweep (z in 2-D, y in the 3-D x-y pass) needs rows q-1 and q+1: each level keeps
//     the "+" characteristic sums of the two previous rows in registers;
//   * the ghost-zero boundary is imposed on every level's output (cells outside the grid are 0
//     at every sub-step); a zero row stays zero through the x sweep, so one mask per level is
//     exact.
// Arithmetic order is fixed (explicit round-to-nearest intrinsics, no contraction):
//   sweep:  u = a + b, w = a - b;  a' = u(-) + w(+), b' = u(-) - w(+)   (1/2 factors deferred)
//   phase:  re = fma(z.re, p.re, -(z.im p.im)),  im = fma(z.re, p.im, z.im p.re)
// with p carrying the deferred 1/4 (exact power-of-two scaling).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <type_traits>

#include "dirac_internal.cuh"

// Compile-time tunables of the 2-D step kernels: resident 4-warp blocks per SM the register budget is fitted to
// (fixed point k = 1, P = 1; FP32 k = 2, P = 2; FP64 k = 1, P = 2 and 4), and rows per loop iteration of the
// fixed-point kernel.  Fixed point: 4 blocks with two rows per iteration fit 128 registers without spilling (33.1
// against 26.7 G point-steps/s at 150 registers and 3 blocks, 2048^2).  FP32 k = 2, P = 2 (and the second-order
// step at k = 1, P = 2): 4 blocks fit once the z sweep's history lives in shared memory (HistSmem below).
#ifndef FX_MIN_BLOCKS
#define FX_MIN_BLOCKS 4
#endif
#ifndef F32_MIN_BLOCKS
#define F32_MIN_BLOCKS 4
#endif
#ifndef F64_MIN_BLOCKS
#define F64_MIN_BLOCKS 1
#endif
#ifndef FX_ROW_UNROLL
#define FX_ROW_UNROLL 2
#endif

namespace dirac {

// Opts `kernel` in to `smem` bytes of dynamic shared memory, once per device (bit `dev` of `done`; devices
// past 63 set the attribute on every launch).  Concurrent first launches may both set it: harmless.
template <typename K>
static cudaError_t optin_smem(K *kernel, int smem, std::atomic<unsigned long long> &done) {
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
    if (bit && (done.load(std::memory_order_relaxed) & bit)) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_relaxed);
    return e;
}

template <typename T> struct Ar;
template <> struct Ar<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
};
template <> struct Ar<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
};

// 64-bit fixed point (storage DIRAC_FX64): the state is q = psi 2^S in int64, so the sweeps' additions are
// exact; only the phase product rounds (cmulp below).
template <> struct Ar<long long> {
    static __device__ __forceinline__ long long add(long long a, long long b) { return a + b; }
    static __device__ __forceinline__ long long sub(long long a, long long b) { return a - b; }
    static __device__ __forceinline__ long long mul(long long a, long long b) { return a * b; }
    static __device__ __forceinline__ long long fma(long long a, long long b, long long c) { return a * b + c; }
};

template <typename T> struct Cx { T re, im; };

template <typename T> __device__ __forceinline__ Cx<T> cadd(Cx<T> a, Cx<T> b) {
    return {Ar<T>::add(a.re, b.re), Ar<T>::add(a.im, b.im)};
}
template <typename T> __device__ __forceinline__ Cx<T> csub(Cx<T> a, Cx<T> b) {
    return {Ar<T>::sub(a.re, b.re), Ar<T>::sub(a.im, b.im)};
}
// a + i b and a - i b
template <typename T> __device__ __forceinline__ Cx<T> cadd_ib(Cx<T> a, Cx<T> b) {
    return {Ar<T>::sub(a.re, b.im), Ar<T>::add(a.im, b.re)};
}
template <typename T> __device__ __forceinline__ Cx<T> csub_ib(Cx<T> a, Cx<T> b) {
    return {Ar<T>::add(a.re, b.im), Ar<T>::sub(a.im, b.re)};
}
// i z and -i z (exact)
template <typename T> __device__ __forceinline__ Cx<T> cmul_i(Cx<T> a) { return {-a.im, a.re}; }
template <typename T> __device__ __forceinline__ Cx<T> cmul_mi(Cx<T> a) { return {a.im, -a.re}; }
template <typename T> __device__ __forceinline__ Cx<T> cmulp(Cx<T> z, Cx<T> p) {
    return {Ar<T>::fma(z.re, p.re, -Ar<T>::mul(z.im, p.im)), Ar<T>::fma(z.re, p.im, Ar<T>::mul(z.im, p.re))};
}
// Fixed point: the phase coefficient p is held as round(p 2^62) (|p| <= 1/4: the sweeps' deferred 1/4 rides
// in it), each output component is the exact 128-bit value z.re p.re - z.im p.im (resp. z.re p.im +
// z.im p.re), rounded once to the nearest integer after the 2^-62 (halves upward).  The exact values come
// from three products instead of four (k1 = p.re (z.re + z.im), k2 = z.re (p.im - p.re), k3 = z.im (p.re +
// p.im); re = k1 - k3, im = k1 + k2): integer arithmetic, so the same bits.  |z| < 2^62 and |p| <= 2^60
// keep the sums inside int64.
// The rounding offset 2^61 is added to k1 once, for both outputs: the same integers as rounding each.
template <> __device__ __forceinline__ Cx<long long> cmulp<long long>(Cx<long long> z, Cx<long long> p) {
    const __int128 k1 = (__int128)p.re * (z.re + z.im) + ((__int128)1 << 61);
    const __int128 k2 = (__int128)z.re * (p.im - p.re);
    const __int128 k3 = (__int128)z.im * (p.re + p.im);
    return {(long long)((k1 - k3) >> 62), (long long)((k1 + k2) >> 62)};
}
// The same product with four multiplies for the fixed-point state: each output from two independent 128-bit
// products (re = z.re p.re - z.im p.im, im = z.re p.im + z.im p.re, each rounded as in cmulp, so the same
// integers).  More instructions but no shared sum ahead of the products: measured faster in the 3-D
// second-order z-phase-z pass (12.40 against 12.10 G point-steps/s at 256^3), slower in the 2-D step (31.0
// against 33.2).  Floating-point states take cmulp.
template <typename T> __device__ __forceinline__ Cx<T> cmulp4(Cx<T> z, Cx<T> p) { return cmulp(z, p); }
template <> __device__ __forceinline__ Cx<long long> cmulp4<long long>(Cx<long long> z, Cx<long long> p) {
    const __int128 a = (__int128)z.re * p.re + ((__int128)1 << 61), b = (__int128)z.im * p.im;
    const __int128 c = (__int128)z.re * p.im + ((__int128)1 << 61), d = (__int128)z.im * p.re;
    return {(long long)((a - b) >> 62), (long long)((c + d) >> 62)};
}
// Fixed point: o / 2^r rounded to nearest, halves upward (floating-point states never ask for it).
template <typename T> __device__ __forceinline__ void round_shift(Cx<T> (&)[4], int) {}
template <> __device__ __forceinline__ void round_shift<long long>(Cx<long long> (&o)[4], int r) {
    const long long half = 1ll << (r - 1);
#pragma unroll
    for (int q = 0; q < 4; ++q) o[q] = Cx<long long>{(o[q].re + half) >> r, (o[q].im + half) >> r};
}
// acc + z p with re = fma(z.re, p.re, fma(-z.im, p.im, acc.re)), im = fma(z.re, p.im, fma(z.im, p.re, acc.im))
template <typename T> __device__ __forceinline__ Cx<T> cmac(Cx<T> acc, Cx<T> z, Cx<T> p) {
    return {Ar<T>::fma(z.re, p.re, Ar<T>::fma(-z.im, p.im, acc.re)), Ar<T>::fma(z.re, p.im, Ar<T>::fma(z.im, p.re, acc.im))};
}
template <typename T> __device__ __forceinline__ double abs2d(Cx<T> a) {
    double r = (double)a.re, i = (double)a.im;
    return __dadd_rn(__dmul_rn(r, r), __dmul_rn(i, i));
}

template <typename T> __device__ __forceinline__ Cx<T> shfl_c(Cx<T> v, int src) {
    return {__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src)};
}

// ---- point load/store: 4 complex components, 64 B (FP64) or 32 B (FP32)
__device__ __forceinline__ void load_pt(const double *p, Cx<double> s[4]) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        double2 v = q[c];
        s[c] = {v.x, v.y};
    }
}
__device__ __forceinline__ void load_pt(const float *p, Cx<float> s[4]) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
    float4 a = q[0], b = q[1];
    s[0] = {a.x, a.y};
    s[1] = {a.z, a.w};
    s[2] = {b.x, b.y};
    s[3] = {b.z, b.w};
}
__device__ __forceinline__ void store_pt(double *p, const Cx<double> s[4]) {
    double2 *q = reinterpret_cast<double2 *>(p);
#pragma unroll
    for (int c = 0; c < 4; ++c) q[c] = make_double2(s[c].re, s[c].im);
}
__device__ __forceinline__ void store_pt(float *p, const Cx<float> s[4]) {
    float4 *q = reinterpret_cast<float4 *>(p);
    q[0] = make_float4(s[0].re, s[0].im, s[1].re, s[1].im);
    q[1] = make_float4(s[2].re, s[2].im, s[3].re, s[3].im);
}
__device__ __forceinline__ void load_pt(const long long *p, Cx<long long> s[4]) {
    const longlong2 *q = reinterpret_cast<const longlong2 *>(p);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        longlong2 v = q[c];
        s[c] = {v.x, v.y};
    }
}
__device__ __forceinline__ void store_pt(long long *p, const Cx<long long> s[4]) {
    longlong2 *q = reinterpret_cast<longlong2 *>(p);
#pragma unroll
    for (int c = 0; c < 4; ++c) q[c] = make_longlong2(s[c].re, s[c].im);
}
__device__ __forceinline__ void load_tab(const long long *p, Cx<long long> &pu, Cx<long long> &pd) {
    const longlong2 *q = reinterpret_cast<const longlong2 *>(p);
    longlong2 a = q[0], b = q[1];
    pu = {a.x, a.y};
    pd = {b.x, b.y};
}
__device__ __forceinline__ void load_tab(const double *p, Cx<double> &pu, Cx<double> &pd) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
    double2 a = q[0], b = q[1];
    pu = {a.x, a.y};
    pd = {b.x, b.y};
}
__device__ __forceinline__ void load_tab(const float *p, Cx<float> &pu, Cx<float> &pd) {
    float4 a = *reinterpret_cast<const float4 *>(p);
    pu = {a.x, a.y};
    pd = {a.z, a.w};
}

__device__ __forceinline__ int64_t pmod(int64_t a, int64_t n) {
    int64_t r = a % n;
    return r < 0 ? r + n : r;
}

// Rows per iteration of the row loop (1 or 2; measured per variant: two rows let the history registers
// alternate instead of moving, which pays where the loop body is short).
template <typename T, int K, int MODE> struct RowUnroll {
    static constexpr bool FX = sizeof(T) == 8 && (T)0.5 == (T)0;  // the int64 fixed-point state
    static constexpr int value = (sizeof(T) == 4 && K == 1 && MODE == 0) ? 2 : ((FX && K == 1 && MODE == 0) ? FX_ROW_UNROLL : 1);
};
// Whether the z sweep's history (the "+" sums of the two previous rows per level) lives in the warp's shared
// memory instead of registers, one slot per row parity so that nothing moves.  Measured for the single-grid
// FP32 kernels with P = 2: at k = 2 the registers it frees let four blocks (16 warps) per SM run without
// spilling, 114.5 against 105.0 G point-steps/s at 2048^2; at k = 4 it takes the kernel from 208 to 128
// registers, 105.3 against 67.1 G; in the second-order step (mode 2) 150 -> 114 registers at k = 1 and
// 197 -> 126 at k = 2, the best plan 60.8 against 56.8 G; the same bits every time.  The batched kernel, which
// runs the same warp routine, keeps the history in registers (107.5 against 116.0 G with it in shared memory).
template <typename T, int K, int P, int MODE> struct HistSmem {
    static constexpr bool value =
        sizeof(T) == 4 && P == 2 && ((MODE == 0 && (K == 2 || K == 4)) || (MODE == 2 && (K == 1 || K == 2)));
};
template <typename T, int K, int P, int MODE, int UNR = RowUnroll<T, K, MODE>::value, bool HS = false>
__device__ __forceinline__ void sweep_warp(const SweepArgs &a, const int64_t wid, const int lane, unsigned char *wsmem);
template <int K>
__device__ __forceinline__ void finish_flux(const SweepArgs &a);
template <typename T, int K, int P, bool HS = false> struct Ring;

// Pipelined levels of one launch: K steps, or 2K levels for the second-order splitting (mode 2).
template <int K, int MODE> struct Levels { static constexpr int value = (MODE == 2 || MODE == 5) ? 2 * K : K; };

// MODE 0: 2-D first-order step (x sweep, z sweep, phase), K steps per launch.
// MODE 1: 3-D x-y pass (x sweep, y sweep), K must be 1.
// MODE 2: 2-D second-order (Strang) step x, z, phase(dt), z, x (Sec. 2.4), K steps = 2K levels per launch;
//         the four sweeps' 1/2 factors ride in the phase coefficients as 1/16.
// MODE 3: 2-D first-order step with a uniform vector potential: the phase is the full 4x4 matrix of
//         Eq. sol_dis_4, U(step) exp(-i V dt), with the table holding g = exp(-i V dt) / 4 per column or cell.
// MODE 5: MODE 2 with a uniform vector potential (the phase of each step's first level is the matrix, the
//         table holding g = exp(-i V dt) / 16).
// Resident 4-warp blocks per SM the register budget is fitted to (1: the compiler's choice).
template <typename T, int K, int P, int MODE> struct SweepMinBlocks {
    static constexpr bool FX = sizeof(T) == 8 && (T)0.5 == (T)0;
    static constexpr bool F64 = sizeof(T) == 8 && !FX;
    static constexpr int value = (FX && K == 1 && P == 1 && MODE == 0)                  ? FX_MIN_BLOCKS
                                 : (sizeof(T) == 4 && K == 2 && P == 2 && MODE == 0)   ? F32_MIN_BLOCKS
                                 : (sizeof(T) == 4 && K == 1 && P == 2 && MODE == 2)   ? F32_MIN_BLOCKS
                                 : (F64 && K == 1 && (P == 2 || P == 4) && MODE == 0) ? F64_MIN_BLOCKS
                                                                                       : 1;
};

template <typename T, int K, int P, int MODE>
__global__ void __launch_bounds__(128, SweepMinBlocks<T, K, P, MODE>::value) sweep_kernel(const SweepArgs a) {
    constexpr int L = Levels<K, MODE>::value;
    constexpr bool HS = HistSmem<T, K, P, MODE>::value;
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t per_plane = a.nstrips * a.nsegs;
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    unsigned char *wsmem = dyn_smem + (threadIdx.x >> 5) * Ring<T, L, P, HS>::WARP_BYTES;
    // Warps past the end skip the work but still reach the block-completion ticket below.
    if (wid < per_plane * a.nplanes) sweep_warp<T, K, P, MODE, RowUnroll<T, K, MODE>::value, HS>(a, wid, lane, wsmem);
    if (a.flux_face >= 0) finish_flux<L>(a);
}

// Last-block fold of the per-warp flux partials: every block takes a ticket after its partials are
// visible; the block that takes the last ticket sums them in a fixed order (step by step, parts in
// index order), adds vol * sum to the cumulative flux and resets the ticket.  No block waits.
template <int K>
__device__ __forceinline__ void finish_flux(const SweepArgs &a) {
    __shared__ unsigned s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(a.ticket, 1u);
        s_last = (t == gridDim.x - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        const int64_t nparts = a.nsegs * a.nplanes;
        double F = __ldcg(a.flux_cum);
        for (int s = 0; s < K; ++s) {
            double f = 0.0;
            for (int64_t q = 0; q < nparts; ++q) f = __dadd_rn(f, __ldcg(a.flux_part + s * nparts + q));
            F = __dadd_rn(F, __dmul_rn(f, a.vol));
        }
        *a.flux_cum = F;
        __threadfence();
        *a.ticket = 0u;
    }
}

// ---- TMA bulk-copy row ring (per warp).  Lane 0 issues one cp.async.bulk per row into a ring slot,
// armed with mbarrier expect_tx; every lane waits on the slot's mbarrier phase before reading it.
// All waits are bounded: on expiry the kernel raises a flag in *a.err and drains its own copies.
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_inval(uint32_t bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for the phase with the given parity to complete: gives up after about one second of the
// global timer (checked every 64 polls), or after 2^24 polls whatever the timer says.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (int it = 0; it < (1 << 24); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it > 32) __nanosleep(64);
        if ((it & 63) == 63 && global_ns() - t0 > 1000000000ull) return false;
    }
    return false;
}

// Per-warp shared memory: 128 B of mbarriers, the row ring, the flux hand-off area (K levels x 8 values x 32
// lanes), then with HS the sweep history ([row parity 2][level K][lane 32][point P][2] complex values; the ring
// keeps three rows so that four blocks fit).
template <typename T, int K, int P, bool HS> struct Ring {
    static constexpr int ROW_BYTES = 32 * P * 8 * (int)sizeof(T);  // one warp row: 32P cells
    static constexpr int SLOTS = (HS || ROW_BYTES >= 8192) ? 3 : 4;
    static constexpr int FLUX_BYTES = K * 8 * 32 * (int)sizeof(T);
    static constexpr int HIST_BYTES = HS ? 2 * K * 32 * P * 2 * 2 * (int)sizeof(T) : 0;
    static constexpr int WARP_BYTES = 128 + SLOTS * ROW_BYTES + FLUX_BYTES + HIST_BYTES;
};

// Dynamic shared memory a block of `wpb` warps needs.
template <typename T, int K, int P, bool HS = false> constexpr int ring_smem_bytes(int wpb) {
    return wpb * Ring<T, K, P, HS>::WARP_BYTES;
}

// Records row q's "+" sums in the two-slot history: with two rows per iteration into the slot that held row
// q - 2 (`older`); with one, slot 0 takes slot 1 (row q - 1) and slot 1 takes row q.
template <typename T, int UNR>
__device__ __forceinline__ void push_row(Cx<T> (&s0)[2], Cx<T> (&s1)[2], Cx<T> (&older)[2], Cx<T> v0, Cx<T> v1) {
    if (UNR == 2) {
        older[0] = v0;
        older[1] = v1;
    } else {
        s0[0] = s1[0];
        s0[1] = s1[1];
        s1[0] = v0;
        s1[1] = v1;
    }
}

// x characteristics of a row (u = a + b travels +x, w = a - b travels -x) and the neighbours the x sweep
// takes: u of the left cell and w of the right cell (warp shuffles; lane 0 and lane 31 take them from the
// adjacent point of lanes 31 and 0).
template <typename T, int P>
__device__ __forceinline__ void x_characteristics(const Cx<T> (*s)[4], int lane, int src_prev, int src_next, Cx<T> *u14,
                                                  Cx<T> *u23, Cx<T> *w14, Cx<T> *w23, Cx<T> *lu14, Cx<T> *lu23,
                                                  Cx<T> *rw14, Cx<T> *rw23) {
#pragma unroll
    for (int j = 0; j < P; ++j) {
        u14[j] = cadd(s[j][0], s[j][3]);
        w14[j] = csub(s[j][0], s[j][3]);
        u23[j] = cadd(s[j][1], s[j][2]);
        w23[j] = csub(s[j][1], s[j][2]);
    }
    Cx<T> pu14[P], pu23[P], nw14[P], nw23[P];
#pragma unroll
    for (int j = 0; j < P; ++j) {
        pu14[j] = shfl_c(u14[j], src_prev);
        pu23[j] = shfl_c(u23[j], src_prev);
        nw14[j] = shfl_c(w14[j], src_next);
        nw23[j] = shfl_c(w23[j], src_next);
    }
#pragma unroll
    for (int j = 0; j < P; ++j) {
        const int jp = j > 0 ? j - 1 : 0;
        const int jn = j < P - 1 ? j + 1 : P - 1;
        lu14[j] = (lane == 0) ? pu14[jp] : pu14[j];
        lu23[j] = (lane == 0) ? pu23[jp] : pu23[j];
        rw14[j] = (lane == 31) ? nw14[jn] : nw14[j];
        rw23[j] = (lane == 31) ? nw23[jn] : nw23[j];
    }
}

// One row of the face flux: the face lane's 8 values go to lane (row % 32) of the hand-off area; at every 32nd
// row (or the segment's last) all lanes fold their rows: scale (|u14|^2 + |u23|^2) - scale (|w14|^2 + |w23|^2),
// scale = 1/2 for a state at its true size, 2 for one held at half size.
template <typename T, int P>
__device__ __forceinline__ void flux_row(const Cx<T> *lu14, const Cx<T> *lu23, const Cx<T> *w14, const Cx<T> *w23,
                                         int face_j, int face_lane, int lane, int64_t row_in_seg, bool last_row, T *g,
                                         double scale, double &facc) {
    T v[8] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int j = 0; j < P; ++j) {
        if (j == face_j) {
            v[0] = lu14[j].re; v[1] = lu14[j].im; v[2] = lu23[j].re; v[3] = lu23[j].im;
            v[4] = w14[j].re;  v[5] = w14[j].im;  v[6] = w23[j].re;  v[7] = w23[j].im;
        }
    }
    const int t = (int)(row_in_seg & 31);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const T x = __shfl_sync(0xffffffffu, v[k], face_lane);
        if (lane == t) g[k * 32 + t] = x;
    }
    if (t == 31 || last_row) {
        __syncwarp();
        if (lane <= t) {
            const T *gl = g + lane;
            const double right = __dmul_rn(scale, __dadd_rn(abs2d(Cx<T>{gl[0], gl[32]}), abs2d(Cx<T>{gl[64], gl[96]})));
            const double left = __dmul_rn(scale, __dadd_rn(abs2d(Cx<T>{gl[128], gl[160]}), abs2d(Cx<T>{gl[192], gl[224]})));
            facc = __dadd_rn(facc, __dsub_rn(right, left));
        }
        __syncwarp();
    }
}

template <typename T, int K, int P, int MODE, int UNR, bool HS>
__device__ __forceinline__ void sweep_warp(const SweepArgs &a, const int64_t wid, const int lane, unsigned char *wsmem) {
    constexpr int L = Levels<K, MODE>::value;  // pipelined levels (one row and one x cell of halo each)
    const int64_t per_plane = a.nstrips * a.nsegs;
    const int64_t plane = wid / per_plane;
    const int64_t rem = wid - plane * per_plane;
    const int64_t seg = rem / a.nstrips;
    const int64_t strip = rem - seg * a.nstrips;
    const int64_t nx = a.nx, nr = a.nr;
    const bool per = a.periodic != 0;
    const bool ring = !per;  // periodic grids wrap the strip: plain loads
    const int64_t x_own0 = strip * a.strip_w;
    const int64_t x_own1 = min(x_own0 + a.strip_w, nx);
    const int64_t xa = x_own0 - L;
    // Row indices fit 32 bits (the host limits every grid dimension below 2^31).  The floating-point kernels run
    // their row loop on 32-bit indices (FP32 k = 2: 105 against 94 G point-steps/s at 2048^2); the fixed-point
    // kernel keeps 64-bit ones, with which it fits its 128-register budget without spilling (33.2 against 31.5 G).
    using RI = typename std::conditional<RowUnroll<T, K, MODE>::FX, int64_t, int>::type;
    const RI nr32 = (RI)nr;
    const RI r_begin = (RI)(seg * a.seg_h);
    const RI r_end = (RI)min((int64_t)r_begin + a.seg_h, nr);
    const T *in = static_cast<const T *>(a.in) + plane * nr * nx * 8;
    T *out = static_cast<T *>(a.out) + plane * nr * nx * 8;

    // every lane's cells lie inside the grid (or wrap): output rows inside the grid need no ghost-zero mask
    const bool strip_in = per || (xa >= 0 && xa + 32 * P <= nx);
    int64_t xl[P];
    bool xin[P], own[P];  // own: the cell is in this warp's strip (it stores it)
#pragma unroll
    for (int j = 0; j < P; ++j) {
        const int64_t x = xa + 32 * j + lane;
        xin[j] = (x >= 0 && x < nx);
        own[j] = x >= x_own0 && x < x_own1;
        xl[j] = per ? pmod(x, nx) : min(max(x, (int64_t)0), nx - 1);
    }
    // phase coefficients per x column (mode 0, x-only table)
    Cx<T> pu[P], pd[P];
    if (MODE != 1 && !a.full_table) {
#pragma unroll
        for (int j = 0; j < P; ++j) load_tab(static_cast<const T *>(a.table) + xl[j] * 4, pu[j], pd[j]);
    }
    // MODES 3 and 5: entries of U for each step of the launch (Dup, Ddn, Ez, -Ez, Ep, Em; Sec. 2.3), and with
    // an x-only table the entries times this lane's g per cell (M = U g, formed once per task)
    constexpr bool FLD = MODE == 3 || MODE == 5;
    constexpr int LA = FLD ? K : 1;
    Cx<T> UM[LA][6];
    Cx<T> MA[LA][FLD ? P : 1][6];
    if (FLD) {
#pragma unroll
        for (int st = 0; st < LA; ++st) {
            const double *u = a.ucoef + ((a.step0 + st) % a.ucoef_n) * 12;
#pragma unroll
            for (int e = 0; e < 6; ++e) UM[st][e] = Cx<T>{(T)__ldg(u + 2 * e), (T)__ldg(u + 2 * e + 1)};
            if (!a.full_table)
#pragma unroll
                for (int j = 0; j < (FLD ? P : 1); ++j)
#pragma unroll
                    for (int e = 0; e < 6; ++e) MA[st][j][e] = cmulp(UM[st][e], pu[j]);
        }
    }
    // Flux through the face (owned by this strip): per row, 1/2(|u14|^2+|u23|^2) at face-1 minus
    // 1/2(|w14|^2+|w23|^2) at face.  The face lane's 8 values of row q are handed to lane (q - r_begin) % 32;
    // every 32 rows all lanes evaluate their row at once, so the FP64 work runs SIMT-wide (1/32 of the FP64
    // issue a single lane would need).  Each lane accumulates its rows in FP64; a fixed xor tree adds lanes.
    const bool has_face = a.flux_face >= x_own0 && a.flux_face < x_own1;
    const int face_off = (int)(a.flux_face - xa);
    const int face_lane = face_off & 31, face_j = face_off >> 5;
    double facc[L];
#pragma unroll
    for (int s = 0; s < L; ++s) facc[s] = 0.0;

    // "+" characteristic sums of the two previous rows per level: rows q-2 (A) and q-1 (B)
    // The two previous rows' sums per level sit in two register slots.  With rows taken in pairs (UNR = 2),
    // row q of level lev reads slot (pair position + lev) & 1, which holds row q - 2, and overwrites it with
    // row q: the slot indices are compile-time constants and nothing moves.  With UNR = 1, slot 0 holds row
    // q - 2 and slot 1 row q - 1, shifted down after each row.
    Cx<T> UH[2][L][P][2];
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int s = 0; s < L; ++s)
#pragma unroll
            for (int j = 0; j < P; ++j)
#pragma unroll
                for (int h = 0; h < 2; ++h) UH[t][s][j][h] = {T(0), T(0)};

    const int src_prev = (lane + 31) & 31, src_next = (lane + 1) & 31;

    // Row ring: the copied span of a row is the strip's cells clipped to the grid.
    using RG = Ring<T, L, P, HS>;
    // HS: the sweep history in shared memory, slot = parity of the row it holds, zero at the task's start
    Cx<T> *hist = reinterpret_cast<Cx<T> *>(wsmem + 128 + RG::SLOTS * RG::ROW_BYTES + RG::FLUX_BYTES);
    if (HS) {
#pragma unroll
        for (int t = 0; t < 2 * L * P * 2; ++t)
            hist[((t / (L * P * 2) * L + (t / (P * 2)) % L) * 32 + lane) * P * 2 + t % (P * 2)] = Cx<T>{T(0), T(0)};
    }
    T *gsm = reinterpret_cast<T *>(wsmem + 128 + RG::SLOTS * RG::ROW_BYTES);  // flux hand-off [K][8][32]
    const int64_t cx0 = max(xa, (int64_t)0), cx1 = min(xa + 32 * P, nx);
    const uint32_t copy_bytes = (uint32_t)((cx1 - cx0) * 8 * (int64_t)sizeof(T));
    const uint32_t bar0 = smem_u32(wsmem);
    const uint32_t slot0 = smem_u32(wsmem + 128);
    const uint32_t dst_off = (uint32_t)((cx0 - xa) * 8 * (int64_t)sizeof(T));
    const RI r_first = r_begin - L, r_last = r_end + L;  // rows [r_first, r_last) are read
    uint32_t phase_bits = 0, pending = 0;
    bool aborted = false;
    if (ring) {
        if (lane == 0) {
#pragma unroll
            for (int sl = 0; sl < RG::SLOTS; ++sl) mbar_init(bar0 + 8 * sl, 1);
            mbar_fence_init();
        }
        __syncwarp();
        bool stall = a.inject_stall && wid == 0;
#pragma unroll
        for (int sl = 0; sl < RG::SLOTS; ++sl) {
            const RI r = r_first + sl;
            if (r < r_last && r >= 0 && r < nr32) {
                if (lane == 0) {
                    // failure-detection test hook: the first warp of the launch announces 16 bytes more than
                    // its first row copy delivers, so that slot's phase never completes and its bounded wait
                    // runs out (the copy itself completes normally)
                    if (stall)
                        asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], 16;" ::"r"(bar0 + 8 * sl)
                                     : "memory");
                    bulk_load(slot0 + sl * RG::ROW_BYTES + dst_off, in + ((int64_t)r * nx + cx0) * 8, copy_bytes,
                              bar0 + 8 * sl);
                }
                stall = false;
                pending |= 1u << sl;
            }
        }
    }

    int sl = 0;
    for (RI r0 = r_first; r0 < r_last && !aborted; r0 += UNR) {
#pragma unroll
    for (int par = 0; par < UNR; ++par) {
        const RI r = r0 + par;
        if (r >= r_last) break;
        Cx<T> st[P][4];
        const bool row_ok = per || (r >= 0 && r < nr32);
        const int64_t rl = per ? pmod(r, nr) : r;
        if (ring) {
            if (row_ok) {
                if (!mbar_wait(bar0 + 8 * sl, (phase_bits >> sl) & 1u)) {
                    aborted = true;
                    break;
                }
                phase_bits ^= 1u << sl;
                pending &= ~(1u << sl);
            }
            const T *srow = reinterpret_cast<const T *>(wsmem + 128 + sl * RG::ROW_BYTES);
#pragma unroll
            for (int j = 0; j < P; ++j) {
                if (row_ok && xin[j]) {
                    load_pt(srow + (32 * j + lane) * 8, st[j]);
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c) st[j][c] = {T(0), T(0)};
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < P; ++j) {
                if (row_ok && (per || xin[j])) {
                    load_pt(in + (rl * nx + xl[j]) * 8, st[j]);
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c) st[j][c] = {T(0), T(0)};
                }
            }
        }
#pragma unroll
        for (int lev = 0; lev < L; ++lev) {
            const RI q = r - lev;  // row of the level-lev state in st
            // rows of level lev+1 that later levels (or the store) use: [r_first + lev + 1, r_last - lev - 1)
            const bool need_out = (q - 1 >= r_first + lev + 1) && (q - 1 < r_last - lev - 1);
            if ((MODE == 2 || MODE == 5) && (lev & 1)) {
                // second half of a Strang step: z sweep of rows q-2 and q into row q-1, then the x sweep of
                // row q-1.  The input is 1/4 of the state (the phase carried 1/16), the z-swept row 1/2 of it.
                const bool zrow_ok = per || (q - 1 >= 0 && q - 1 < nr32);
                Cx<T> zs[P][4];
#pragma unroll
                for (int j = 0; j < P; ++j) {
                    const Cx<T> U13 = cadd(st[j][0], st[j][2]), U24 = csub(st[j][1], st[j][3]);
                    const Cx<T> W13 = csub(st[j][0], st[j][2]), W24 = cadd(st[j][1], st[j][3]);
                    Cx<T>(&UO)[2] = UH[UNR == 2 ? (par + lev) & 1 : 0][lev][j];  // row q - 2
                    Cx<T> *hq = hist + ((((int)(q & 1) * L + lev) * 32 + lane) * P + j) * 2;  // HS: its slot
                    const Cx<T> o0 = HS ? hq[0] : UO[0], o1 = HS ? hq[1] : UO[1];
                    zs[j][0] = cadd(o0, W13);
                    zs[j][2] = csub(o0, W13);
                    zs[j][1] = cadd(o1, W24);
                    zs[j][3] = csub(W24, o1);
                    if (HS) {
                        hq[0] = U13;
                        hq[1] = U24;
                    } else {
                        push_row<T, UNR>(UH[0][lev][j], UH[1][lev][j], UO, U13, U24);
                    }
                    if (!zrow_ok)
#pragma unroll
                        for (int c = 0; c < 4; ++c) zs[j][c] = Cx<T>{T(0), T(0)};
                }
                if (!need_out) {
#pragma unroll
                    for (int j = 0; j < P; ++j)
#pragma unroll
                        for (int c = 0; c < 4; ++c) st[j][c] = Cx<T>{T(0), T(0)};
                    continue;
                }
                Cx<T> u14[P], u23[P], w14[P], w23[P], lu14[P], lu23[P], rw14[P], rw23[P];
                x_characteristics<T, P>(zs, lane, src_prev, src_next, u14, u23, w14, w23, lu14, lu23, rw14, rw23);
                if (has_face && q - 1 >= r_begin && q - 1 < r_end)
                    flux_row<T, P>(lu14, lu23, w14, w23, face_j, face_lane, lane, q - 1 - r_begin, q - 1 == r_end - 1,
                                   gsm + lev * 8 * 32, 2.0 * a.flux_unit, facc[lev]);
#pragma unroll
                for (int j = 0; j < P; ++j) {
                    const bool keep = per || (zrow_ok && xin[j]);
                    const Cx<T> b0 = cadd(lu14[j], rw14[j]), b3 = csub(lu14[j], rw14[j]);
                    const Cx<T> b1 = cadd(lu23[j], rw23[j]), b2 = csub(lu23[j], rw23[j]);
                    st[j][0] = keep ? b0 : Cx<T>{T(0), T(0)};
                    st[j][1] = keep ? b1 : Cx<T>{T(0), T(0)};
                    st[j][2] = keep ? b2 : Cx<T>{T(0), T(0)};
                    st[j][3] = keep ? b3 : Cx<T>{T(0), T(0)};
                }
                continue;
            }
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
            Cx<T> lu14[P], lu23[P], rw14[P], rw23[P];
#pragma unroll
            for (int j = 0; j < P; ++j) {
                const int jp = j > 0 ? j - 1 : 0;
                const int jn = j < P - 1 ? j + 1 : P - 1;
                lu14[j] = (lane == 0) ? pu14[jp] : pu14[j];
                lu23[j] = (lane == 0) ? pu23[jp] : pu23[j];
                rw14[j] = (lane == 31) ? nw14[jn] : nw14[j];
                rw23[j] = (lane == 31) ? nw23[jn] : nw23[j];
            }
            if (has_face && q >= r_begin && q < r_end)
                flux_row<T, P>(lu14, lu23, w14, w23, face_j, face_lane, lane, q - r_begin, q == r_end - 1,
                               gsm + lev * 8 * 32, 0.5 * a.flux_unit, facc[lev]);
            const bool out_row_ok = per || (q - 1 >= 0 && q - 1 < nr32);
#pragma unroll
            for (int j = 0; j < P; ++j) {
                // x sweep (Eq. sol_dis_1), x2
                const Cx<T> b0 = cadd(lu14[j], rw14[j]);
                const Cx<T> b3 = csub(lu14[j], rw14[j]);
                const Cx<T> b1 = cadd(lu23[j], rw23[j]);
                const Cx<T> b2 = csub(lu23[j], rw23[j]);
                Cx<T> o[4];
                if (MODE != 1) {
                    // z sweep (Eq. sol_dis_3): +z movers (b1+b3, b2-b4), -z movers (b1-b3, b2+b4)
                    const Cx<T> U13 = cadd(b0, b2), U24 = csub(b1, b3);
                    // row q - 2's sums: the slot of q's parity (HS) or the register slot
                    Cx<T> *hp = hist + ((((int)(q & 1) * L + lev) * 32 + lane) * P + j) * 2;
                    Cx<T> h0, h1;
                    if (HS) {
                        h0 = hp[0];
                        h1 = hp[1];
                    } else {
                        h0 = UH[UNR == 2 ? (par + lev) & 1 : 0][lev][j][0];
                        h1 = UH[UNR == 2 ? (par + lev) & 1 : 0][lev][j][1];
                    }
                    if (need_out) {
                        const Cx<T> W13 = csub(b0, b2), W24 = cadd(b1, b3);
                        o[0] = cadd(h0, W13);
                        o[2] = csub(h0, W13);
                        o[1] = cadd(h1, W24);
                        o[3] = csub(W24, h1);
                        // phase (Eq. sol_dis_4) with the deferred 1/4
                        Cx<T> qu, qd;
                        if (a.full_table) {
                            const int64_t rr = per ? pmod(q - 1, nr) : (int64_t)min(max(q - 1, (RI)0), nr32 - 1);
                            load_tab(static_cast<const T *>(a.table) + (plane * nr * nx + rr * nx + xl[j]) * 4, qu, qd);
                        } else {
                            qu = pu[j];
                            qd = pd[j];
                        }
                        if (FLD) {
                            // psi'_a = sum_b (U_ab g) psi_b over the non-zero entries, columns in order
                            constexpr int SPL = MODE == 5 ? 2 : 1;  // levels per step
                            Cx<T> m6[6];
#pragma unroll
                            for (int e = 0; e < 6; ++e)
                                m6[e] = a.full_table ? cmulp(UM[FLD ? lev / SPL : 0][e], qu)
                                                     : MA[FLD ? lev / SPL : 0][FLD ? j : 0][e];
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
                    }
                    if (HS) {  // row q's sums replace row q - 2's
                        hp[0] = U13;
                        hp[1] = U24;
                    } else {
                        push_row<T, UNR>(UH[0][lev][j], UH[1][lev][j], UH[UNR == 2 ? (par + lev) & 1 : 0][lev][j], U13, U24);
                    }
                } else {
                    // y sweep (Eq. sol_dis_2): +y movers (b1 - i b4, b2 + i b3), -y movers (b1 + i b4, b2 - i b3)
                    const Cx<T> U14 = csub_ib(b0, b3), U23 = cadd_ib(b1, b2);
                    if (need_out) {
                        const Cx<T> W14 = cadd_ib(b0, b3), W23 = csub_ib(b1, b2);
                        o[0] = cadd(UH[UNR == 2 ? (par + lev) & 1 : 0][lev][j][0], W14);
                        o[3] = cmul_i(csub(UH[UNR == 2 ? (par + lev) & 1 : 0][lev][j][0], W14));
                        o[1] = cadd(UH[UNR == 2 ? (par + lev) & 1 : 0][lev][j][1], W23);
                        o[2] = cmul_mi(csub(UH[UNR == 2 ? (par + lev) & 1 : 0][lev][j][1], W23));
                    }
                    push_row<T, UNR>(UH[0][lev][j], UH[1][lev][j], UH[UNR == 2 ? (par + lev) & 1 : 0][lev][j], U14, U23);
                }
                if (need_out) {
                    if (strip_in && out_row_ok) {  // warp-uniform: no cell of this row is a ghost cell
#pragma unroll
                        for (int c = 0; c < 4; ++c) st[j][c] = o[c];
                    } else {
                        const bool keep = per || (out_row_ok && xin[j]);
#pragma unroll
                        for (int c = 0; c < 4; ++c) st[j][c] = keep ? o[c] : Cx<T>{T(0), T(0)};
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c) st[j][c] = Cx<T>{T(0), T(0)};
                }
            }
        }
        const RI ro = r - L;
        if (ro >= r_begin && ro < r_end) {
            if constexpr (sizeof(RI) == 8) {
#pragma unroll
                for (int j = 0; j < P; ++j) {
                    const int64_t x = xa + 32 * j + lane;
                    if (x >= x_own0 && x < x_own1) store_pt(out + (ro * nx + x) * 8, st[j]);
                }
            } else {
                T *orow = out + (int64_t)ro * nx * 8;
#pragma unroll
                for (int j = 0; j < P; ++j)
                    if (own[j]) store_pt(orow + (xa + 32 * j + lane) * 8, st[j]);
            }
        }
        if (ring) {
            // refill this slot with row r + SLOTS once every lane has read it
            __syncwarp();
            const RI rn = r + RG::SLOTS;
            if (rn < r_last && rn >= 0 && rn < nr32) {
                if (lane == 0) {
                    fence_proxy_async();
                    bulk_load(slot0 + sl * RG::ROW_BYTES + dst_off, in + ((int64_t)rn * nx + cx0) * 8, copy_bytes,
                              bar0 + 8 * sl);
                }
                pending |= 1u << sl;
            }
            sl = (sl + 1 == RG::SLOTS) ? 0 : sl + 1;
        }
    }
    }
    if (aborted) {
        // a copy never completed: report, then wait (bounded) for this warp's copies still in flight
        if (lane == 0) atomicOr(a.err, 1u);
#pragma unroll
        for (int s2 = 0; s2 < RG::SLOTS; ++s2)
            if (pending & (1u << s2)) mbar_wait(bar0 + 8 * s2, (phase_bits >> s2) & 1u);
    }
    if (ring) {
        // release the barriers so the next task of this warp can initialise them again
        __syncwarp();
        if (lane == 0)
#pragma unroll
            for (int s2 = 0; s2 < RG::SLOTS; ++s2) mbar_inval(bar0 + 8 * s2);
        __syncwarp();
    }
    if (aborted) return;
    if (has_face) {
#pragma unroll
        for (int s = 0; s < L; ++s) {
            double v = facc[s];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0) a.flux_part[(int64_t)s * a.nsegs * a.nplanes + plane * a.nsegs + seg] = v;
        }
    }
}

// 3-D z sweep + phase: one thread per (x, y) column and z segment; the input is 4x the x-y swept
// state, the table carries 1/8, so the output is the state after the full step.
template <typename T>
__global__ void __launch_bounds__(128) zphase_kernel(const ZArgs a) {
    const int64_t ncol = a.nx * a.ny;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= ncol * a.nsegs) return;
    const int64_t seg = tid / ncol;
    const int64_t col = tid - seg * ncol;
    const int64_t x = col % a.nx;
    const int64_t nz = a.nz;
    const bool per = a.periodic != 0;
    const int64_t z_begin = seg * a.seg_h;
    const int64_t z_end = min(z_begin + a.seg_h, nz);
    const T *in = static_cast<const T *>(a.in);
    T *out = static_cast<T *>(a.out);
    const T *tab = static_cast<const T *>(a.table);
    Cx<T> pu, pd;
    if (!a.full_table) load_tab(tab + x * 4, pu, pd);
    Cx<T> UA[2] = {{T(0), T(0)}, {T(0), T(0)}}, UB[2] = {{T(0), T(0)}, {T(0), T(0)}};
    for (int64_t z = z_begin - 1; z <= z_end; ++z) {
        Cx<T> s[4];
        const bool ok = per || (z >= 0 && z < nz);
        if (ok) {
            const int64_t zl = per ? pmod(z, nz) : z;
            load_pt(in + (zl * ncol + col) * 8, s);
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) s[c] = {T(0), T(0)};
        }
        const Cx<T> U13 = cadd(s[0], s[2]), U24 = csub(s[1], s[3]);
        const Cx<T> W13 = csub(s[0], s[2]), W24 = cadd(s[1], s[3]);
        const int64_t zo = z - 1;
        if (zo >= z_begin && zo < z_end) {
            Cx<T> o[4];
            o[0] = cadd(UA[0], W13);
            o[2] = csub(UA[0], W13);
            o[1] = cadd(UA[1], W24);
            o[3] = csub(W24, UA[1]);
            Cx<T> qu = pu, qd = pd;
            if (a.full_table) load_tab(tab + (zo * ncol + col) * 4, qu, qd);
            o[0] = cmulp(o[0], qu);
            o[1] = cmulp(o[1], qu);
            o[2] = cmulp(o[2], qd);
            o[3] = cmulp(o[3], qd);
            store_pt(out + (zo * ncol + col) * 8, o);
        }
        UA[0] = UB[0];
        UA[1] = UB[1];
        UB[0] = U13;
        UB[1] = U24;
    }
}

}  // namespace dirac
