// Batched ensemble of independent 2-D Klein-step runs (uneven grid sizes and step counts) advanced
// by one persistent kernel per block of K steps.
//
// Work: every active run is cut into (strip, segment) tasks exactly as the single-grid step kernel
// cuts its grid; the tasks of all active runs form one list.  Resident warps take tasks from an
// atomic counter until the list is exhausted (dynamic balance across runs of different sizes) and
// run each task with the single-grid warp routine (sweep_warp), so the arithmetic, boundary and
// flux handling are identical to dirac_step's.  The last block to finish folds every active run's
// per-step face-flux partials into that run's cumulative flux (fixed order) and resets the counter.
//
// Runs are ordered so that the active set of every launch is a prefix of an order array; the task
// list's prefix offsets are precomputed per order, and a warp finds its run by binary search.
#pragma once

#include "step_kernels.cuh"

namespace dirac {

struct BatchRunDev {
    void *psi[2];           // ping-pong state buffers
    const void *table;      // x-only phase table, 4 values per column (pre-scaled by 1/4)
    int64_t side;           // nx = nz = side
    int64_t face;           // flux face index
    int64_t nsegs, seg_h;   // row segments
    double *flux_part;      // [K][nsegs]
    double *flux_cum;       // cumulative flux of this run
    int64_t parity_base;    // parity offset of the remainder phase (number of K-step launches)
};

struct BatchArgs {
    const BatchRunDev *runs;
    const int *order;       // run index per position; the active runs are order[0 .. n_active)
    const int64_t *task_off;// prefix task offsets along `order` (for this launch's K), n_active + 1 used
    int n_active;
    int parity_mode;        // 0: parity = launch & 1 (K-step phase); 1: (parity_base + launch) & 1
    int64_t launch;
    unsigned *counter;      // task counter, 0 between launches
    unsigned *ticket;       // block-completion ticket, 0 between launches
    unsigned *err;
    double vol;
};

template <typename T, int K, int P>
__global__ void __launch_bounds__(128) batch_kernel(const BatchArgs b) {
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    const int lane = threadIdx.x & 31;
    unsigned char *wsmem = dyn_smem + (threadIdx.x >> 5) * Ring<T, K, P>::WARP_BYTES;
    const int64_t total = b.task_off[b.n_active];
    for (;;) {
        unsigned task = 0;
        if (lane == 0) task = atomicAdd(b.counter, 1u);
        task = __shfl_sync(0xffffffffu, task, 0);
        if ((int64_t)task >= total) break;
        int lo = 0, hi = b.n_active;  // task_off[lo] <= task < task_off[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (b.task_off[mid] <= (int64_t)task) lo = mid; else hi = mid;
        }
        const BatchRunDev &R = b.runs[b.order[lo]];
        const int parity = (int)((b.parity_mode ? R.parity_base + b.launch : b.launch) & 1);
        SweepArgs a{};
        a.in = R.psi[parity];
        a.out = R.psi[parity ^ 1];
        a.table = R.table;
        a.nx = R.side;
        a.nr = R.side;
        a.nplanes = 1;
        a.strip_w = 32 * P - 2 * K;
        a.nstrips = (R.side + a.strip_w - 1) / a.strip_w;
        a.nsegs = R.nsegs;
        a.seg_h = R.seg_h;
        a.flux_face = R.face;
        a.flux_part = R.flux_part;
        a.flux_cum = R.flux_cum;
        a.ticket = nullptr;
        a.err = b.err;
        a.vol = b.vol;
        a.periodic = 0;
        a.full_table = 0;
        a.flux_unit = 1.0;  // floating-point states
        sweep_warp<T, K, P, 0, 2>(a, (int64_t)task - b.task_off[lo], lane, wsmem);  // two rows per iteration: measured faster here
    }
    // last block folds the flux partials of every active run and resets the counters
    __shared__ unsigned s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(b.ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int i = threadIdx.x; i < b.n_active; i += blockDim.x) {
            const BatchRunDev &R = b.runs[b.order[i]];
            double F = __ldcg(R.flux_cum);
            for (int s = 0; s < K; ++s) {
                double f = 0.0;
                for (int64_t q = 0; q < R.nsegs; ++q) f = __dadd_rn(f, __ldcg(R.flux_part + s * R.nsegs + q));
                F = __dadd_rn(F, __dmul_rn(f, b.vol));
            }
            *R.flux_cum = F;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            *b.counter = 0u;
            *b.ticket = 0u;
        }
    }
}

// Gaussian packet N [1, 0, 0, C] e^{i k0 x} exp(-((x-x0)^2 + z^2)/(4 w^2)) (Sec. 5.2.2) written for every run,
// unnormalised (the transmitted fraction divides by the measured initial norm).  One thread per cell of the
// concatenated runs; cell_off holds each run's first cell.
struct InitArgs {
    const BatchRunDev *runs;
    const int64_t *cell_off;   // [nruns + 1]
    const double *x0, *k0, *width, *spinC;  // per run
    const int64_t *absorb;     // absorbing-layer columns per run: the packet is zero there
    int nruns;
    double dx;
};

template <typename T>
__global__ void batch_init_kernel(const InitArgs ia) {
    const int64_t total = ia.cell_off[ia.nruns];
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = ia.nruns;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (ia.cell_off[mid] <= g) lo = mid; else hi = mid;
        }
        const BatchRunDev &R = ia.runs[lo];
        const int64_t c = g - ia.cell_off[lo];
        const int64_t i = c % R.side, k = c / R.side;
        const double x = (double)(i - R.face) * ia.dx + 0.5 * ia.dx;         // step face at x = 0
        const double z = (double)(k - R.side / 2) * ia.dx + 0.5 * ia.dx;     // packet centred in z
        const double w = ia.width[lo];
        const double dxx = x - ia.x0[lo];
        const double amp = exp(-(dxx * dxx + z * z) / (4.0 * w * w));
        double sn, cs;
        sincos(ia.k0[lo] * x, &sn, &cs);
        const double C = ia.spinC[lo];
        T *p = static_cast<T *>(R.psi[0]) + c * 8;
        if (i < ia.absorb[lo] || i >= R.side - ia.absorb[lo]) {
#pragma unroll
            for (int q = 0; q < 8; ++q) p[q] = T(0);
            continue;
        }
        p[0] = (T)(amp * cs);
        p[1] = (T)(amp * sn);
        p[2] = T(0); p[3] = T(0); p[4] = T(0); p[5] = T(0);
        p[6] = (T)(C * amp * cs);
        p[7] = (T)(C * amp * sn);
    }
}

// Per-run norm: block b of the launch reduces cells [b*chunk, (b+1)*chunk) of the concatenated runs that
// belong to one run (chunks never straddle runs: run boundaries are chunk-aligned in chunk_off).
struct NormArgs {
    const BatchRunDev *runs;
    const int64_t *chunk_off;  // first chunk of each run, [nruns + 1]
    int nruns;
    int64_t chunk;             // cells per chunk
    double *partial;           // one per chunk
    int parity_from_base;      // 1: read psi[(parity_base + remainder) & 1] via final_parity
    const int *final_parity;   // per run (used when parity_from_base)
};

template <typename T>
__global__ void batch_norm_partial_kernel(const NormArgs na) {
    __shared__ double sh[32];
    const int64_t ch = blockIdx.x;
    int lo = 0, hi = na.nruns;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (na.chunk_off[mid] <= ch) lo = mid; else hi = mid;
    }
    const BatchRunDev &R = na.runs[lo];
    const int par = na.parity_from_base ? na.final_parity[lo] : 0;
    const T *psi = static_cast<const T *>(R.psi[par]);
    const int64_t n = R.side * R.side;
    const int64_t c0 = (ch - na.chunk_off[lo]) * na.chunk;
    const int64_t c1 = min(c0 + na.chunk, n);
    double s = 0.0;
    for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        const T *p = psi + c * 8;
        double r = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) r = __dadd_rn(r, __dmul_rn((double)p[q], (double)p[q]));
        s = __dadd_rn(s, r);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = __dadd_rn(s, __shfl_xor_sync(0xffffffffu, s, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) na.partial[ch] = v;
    }
}

static __global__ void batch_norm_fold_kernel(const int64_t *chunk_off, int nruns, const double *partial, double vol,
                                       double *norm) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nruns; r += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t c = chunk_off[r]; c < chunk_off[r + 1]; ++c) s = __dadd_rn(s, partial[c]);
        norm[r] = __dmul_rn(s, vol);
    }
}

}  // namespace dirac
