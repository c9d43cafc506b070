// Host runtime of the batched Klein ensemble (include/dirac.h, dirac_batch_*).
//
// Launch schedule.  With K steps per launch, run r needs floor(n_r / K) K-step launches and
// n_r mod K single-step launches.  K-step launch l advances the runs with floor(n_r/K) > l: sorted by
// floor(n_r/K) descending (order_main) they are a prefix.  The single-step launches come after all
// K-step launches; launch j advances the runs with (n_r mod K) > j, a prefix of order_rem (sorted by
// n_r mod K descending), at parity (floor(n_r/K) + j) mod 2.  Each order has its own prefix offsets of
// the task list (tasks depend on the strip width 32P - 2K).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/dirac.h"
#include "batch_internal.cuh"
#include "batch_kernels.cuh"
#include "dirac_internal.cuh"

using namespace dirac;

namespace {
thread_local std::string g_batch_err;
constexpr int64_t kNormChunk = 65536;
}  // namespace

struct dirac_batch {
    dirac_batch_config cfg{};
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    int fp32 = 1;
    size_t elem = 4;
    int nruns = 0;
    std::vector<dirac_klein_run> runs;
    std::vector<BatchRunDev> hrun;
    std::vector<int64_t> state_off;  // element offset of each run's first buffer in the pool
    BatchRunDev *drun = nullptr;
    void *state_pool = nullptr;
    size_t state_bytes = 0;
    void *table_pool = nullptr;
    double *flux_part_pool = nullptr;
    size_t flux_part_n = 0;
    double *flux_cum = nullptr;
    double *norm0 = nullptr;
    double *norm_partial = nullptr;
    int64_t *d_chunk_off = nullptr;
    int64_t nchunks = 0;
    int64_t *d_cell_off = nullptr;
    double *d_init = nullptr;  // x0, k0, width, C per run
    int64_t *d_absorb = nullptr;
    std::vector<std::vector<double>> mask;  // absorbing-layer factors per run (side values)
    unsigned *counters = nullptr;  // counter, ticket, err, pad
    int *d_order_main = nullptr, *d_order_rem = nullptr;
    int64_t *d_off_main = nullptr, *d_off_rem = nullptr;
    std::vector<int> nact_main, nact_rem;
    int K = 2, P = 2, blocks = 0, sm_count = 152;
    int64_t seg_rows = 64, max_tasks = 0;
    cudaGraphExec_t graph = nullptr;
    bool ran = false;
    int64_t launches = 0;
    size_t device_bytes = 0;
    std::string err;
};

namespace {

dirac_status bfail(dirac_batch *b, dirac_status st, const std::string &m) {
    if (b) b->err = m; else g_batch_err = m;
    return st;
}
dirac_status bcuda(dirac_batch *b, cudaError_t e, const char *where) {
    return bfail(b, e == cudaErrorMemoryAllocation ? DIRAC_ERR_OOM : DIRAC_ERR_CUDA,
                 std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}
#define BCK(b, expr)                                           \
    do {                                                       \
        cudaError_t e_ = (expr);                               \
        if (e_ != cudaSuccess) return bcuda((b), e_, #expr);   \
    } while (0)

template <typename P>
dirac_status balloc(dirac_batch *b, P **p, size_t bytes) {
    cudaError_t e = cudaMalloc((void **)p, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) return bcuda(b, e, "cudaMalloc");
    b->device_bytes += std::max<size_t>(bytes, 16);
    return DIRAC_OK;
}

void drop_graph(dirac_batch *b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

// Tasks of run r for a launch with `k` steps per launch.
int64_t run_tasks(const dirac_batch *b, int r, int k) {
    const int64_t side = b->runs[r].side;
    const int64_t sw = 32 * b->P - 2 * k;
    return ((side + sw - 1) / sw) * b->hrun[r].nsegs;
}

// (Re)builds the launch plan for the current (K, P, seg_rows): segments, orders, task offsets, active counts.
dirac_status plan(dirac_batch *b) {
    drop_graph(b);
    const int n = b->nruns;
    for (int r = 0; r < n; ++r) {
        BatchRunDev &R = b->hrun[r];
        R.seg_h = std::min<int64_t>(b->seg_rows, R.side);
        R.nsegs = (R.side + R.seg_h - 1) / R.seg_h;
        R.parity_base = b->runs[r].nsteps / b->K;
    }
    // flux partials: K x nsegs per run
    size_t need = 0;
    for (int r = 0; r < n; ++r) need += (size_t)b->K * b->hrun[r].nsegs;
    if (need > b->flux_part_n) {
        if (b->flux_part_pool) {
            cudaFree(b->flux_part_pool);
            b->device_bytes -= b->flux_part_n * sizeof(double);
        }
        b->flux_part_pool = nullptr;
        dirac_status st = balloc(b, &b->flux_part_pool, need * sizeof(double));
        if (st != DIRAC_OK) return st;
        b->flux_part_n = need;
    }
    size_t off = 0;
    for (int r = 0; r < n; ++r) {
        b->hrun[r].flux_part = b->flux_part_pool + off;
        off += (size_t)b->K * b->hrun[r].nsegs;
    }
    std::vector<int> om(n), orr(n);
    std::iota(om.begin(), om.end(), 0);
    std::iota(orr.begin(), orr.end(), 0);
    const int K = b->K;
    std::stable_sort(om.begin(), om.end(), [&](int x, int y) { return b->runs[x].nsteps / K > b->runs[y].nsteps / K; });
    std::stable_sort(orr.begin(), orr.end(), [&](int x, int y) { return b->runs[x].nsteps % K > b->runs[y].nsteps % K; });
    std::vector<int64_t> offm(n + 1, 0), offr(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        offm[i + 1] = offm[i] + run_tasks(b, om[i], K);
        offr[i + 1] = offr[i] + run_tasks(b, orr[i], 1);
    }
    const int64_t Lmain = n ? b->runs[om[0]].nsteps / K : 0;
    b->nact_main.assign(Lmain, 0);
    for (int64_t l = 0; l < Lmain; ++l) {
        int c = 0;
        while (c < n && b->runs[om[c]].nsteps / K > l) ++c;
        b->nact_main[l] = c;
    }
    b->nact_rem.clear();
    for (int j = 0; j < K - 1; ++j) {
        int c = 0;
        while (c < n && b->runs[orr[c]].nsteps % K > j) ++c;
        if (c > 0) b->nact_rem.push_back(c);
    }
    b->max_tasks = offm[n];
    BCK(b, cudaMemcpyAsync(b->d_order_main, om.data(), n * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaMemcpyAsync(b->d_order_rem, orr.data(), n * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaMemcpyAsync(b->d_off_main, offm.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaMemcpyAsync(b->d_off_rem, offr.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaMemcpyAsync(b->drun, b->hrun.data(), n * sizeof(BatchRunDev), cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    int per_sm = 0;
    BCK(b, batch_occupancy(b->fp32, b->K, b->P, &per_sm));
    b->blocks = std::max(1, per_sm) * b->sm_count;
    return DIRAC_OK;
}

dirac_status upload_tables(dirac_batch *b, int only = -1) {
    const double dx = b->cfg.dx, c = b->cfg.c, m = b->cfg.m, dt = dx / c;
    const double mu = m * c * c * dt;
    for (int r = 0; r < b->nruns; ++r) {
        if (only >= 0 && r != only) continue;
        const dirac_klein_run &kr = b->runs[r];
        std::vector<double> V(kr.side);
        for (int64_t i = 0; i < kr.side; ++i) {
            const double x = (double)(i - kr.face) * dx + 0.5 * dx;
            V[i] = 0.5 * kr.V0 * (1.0 + std::tanh(x / kr.L));
        }
        dirac_status st = dirac_batch_set_potential(b, r, V.data(), kr.side);
        if (st != DIRAC_OK) return st;
    }
    (void)mu;
    return DIRAC_OK;
}

dirac_status init_states(dirac_batch *b) {
    InitArgs ia{};
    ia.runs = b->drun;
    ia.cell_off = b->d_cell_off;
    ia.x0 = b->d_init;
    ia.k0 = b->d_init + b->nruns;
    ia.width = b->d_init + 2 * b->nruns;
    ia.spinC = b->d_init + 3 * b->nruns;
    ia.absorb = b->d_absorb;
    ia.nruns = b->nruns;
    ia.dx = b->cfg.dx;
    BCK(b, launch_batch_init(ia, b->fp32, b->stream));
    b->launches++;
    BCK(b, cudaMemsetAsync(b->flux_cum, 0, b->nruns * sizeof(double), b->stream));
    b->ran = false;
    return DIRAC_OK;
}

dirac_status enqueue_schedule(dirac_batch *b, cudaStream_t s, int64_t max_main = -1) {
    BatchArgs a{};
    a.runs = b->drun;
    a.counter = b->counters;
    a.ticket = b->counters + 1;
    a.err = b->counters + 2;
    a.vol = b->cfg.dx * b->cfg.dx;
    const int64_t Lm = (max_main >= 0) ? std::min<int64_t>(max_main, b->nact_main.size()) : (int64_t)b->nact_main.size();
    for (int64_t l = 0; l < Lm; ++l) {
        a.order = b->d_order_main;
        a.task_off = b->d_off_main;
        a.n_active = b->nact_main[l];
        a.parity_mode = 0;
        a.launch = l;
        BCK(b, launch_batch(a, b->fp32, b->K, b->P, b->blocks, s));
        b->launches++;
    }
    if (max_main >= 0) return DIRAC_OK;
    for (size_t j = 0; j < b->nact_rem.size(); ++j) {
        a.order = b->d_order_rem;
        a.task_off = b->d_off_rem;
        a.n_active = b->nact_rem[j];
        a.parity_mode = 1;
        a.launch = (int64_t)j;
        BCK(b, launch_batch(a, b->fp32, 1, b->P, b->blocks, s));
        b->launches++;
    }
    return DIRAC_OK;
}

dirac_status enqueue_norm(dirac_batch *b, cudaStream_t s) {
    NormArgs na{};
    na.runs = b->drun;
    na.chunk_off = b->d_chunk_off;
    na.nruns = b->nruns;
    na.chunk = kNormChunk;
    na.partial = b->norm_partial;
    na.parity_from_base = 0;
    na.final_parity = nullptr;
    BCK(b, launch_batch_norm(na, b->nchunks, b->d_chunk_off, b->nruns, b->cfg.dx * b->cfg.dx, b->norm0, b->fp32, s));
    b->launches += 2;
    return DIRAC_OK;
}

int final_parity(const dirac_batch *b, int r) {
    const int64_t n = b->runs[r].nsteps;
    return (int)(((n / b->K) + (n % b->K)) & 1);
}

void release(dirac_batch *b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    drop_graph(b);
    void *ptrs[] = {b->drun, b->state_pool, b->table_pool, b->flux_part_pool, b->flux_cum, b->norm0, b->norm_partial,
                    b->d_chunk_off, b->d_cell_off, b->d_init, b->counters, b->d_order_main, b->d_order_rem,
                    b->d_off_main, b->d_off_rem};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
}

}  // namespace

extern "C" {

void dirac_batch_default_config(dirac_batch_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->precision = DIRAC_FP32;
    cfg->dx = 10.0 / 8192.0;
    cfg->c = 137.0359895;
    cfg->m = 1.0;
    cfg->use_graphs = 1;
}

const char *dirac_batch_last_error(const dirac_batch *b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

dirac_status dirac_batch_create(const dirac_klein_run *runs, int nruns, const dirac_batch_config *cfg,
                                dirac_batch **out) {
    if (!runs || !cfg || !out || nruns < 1) return bfail(nullptr, DIRAC_ERR_ARG, "dirac_batch_create: bad arguments");
    *out = nullptr;
    if (cfg->precision != DIRAC_FP32 && cfg->precision != DIRAC_FP64)
        return bfail(nullptr, DIRAC_ERR_ARG, "precision must be DIRAC_FP32 or DIRAC_FP64");
    if (!(cfg->dx > 0) || !(cfg->c > 0) || !std::isfinite(cfg->m))
        return bfail(nullptr, DIRAC_ERR_ARG, "dx, c must be > 0 and m finite");
    for (int r = 0; r < nruns; ++r) {
        const dirac_klein_run &k = runs[r];
        if (k.side < 8 || k.side > 65536 || k.face < 1 || k.face > k.side - 1 || k.nsteps < 0 || !(k.L > 0) ||
            !(k.width > 0) || !std::isfinite(k.V0) || !std::isfinite(k.p0) || !std::isfinite(k.x0) ||
            k.absorb < 0 || 2 * k.absorb > k.side || !(k.eta >= 0) || !std::isfinite(k.eta))
            return bfail(nullptr, DIRAC_ERR_ARG, "run " + std::to_string(r) + " has an invalid field");
    }
    const int fp32 = cfg->precision == DIRAC_FP32;
    int K = cfg->steps_per_launch > 0 ? cfg->steps_per_launch : 2;
    int P = cfg->points_per_lane > 0 ? cfg->points_per_lane : 2;
    if (!batch_supported(fp32, K, P) || !batch_supported(fp32, 1, P))
        return bfail(nullptr, DIRAC_ERR_ARG, "unsupported (steps_per_launch, points_per_lane) for this precision");
    dirac_batch *b = new (std::nothrow) dirac_batch();
    if (!b) return bfail(nullptr, DIRAC_ERR_OOM, "host allocation failed");
    b->cfg = *cfg;
    b->stream = static_cast<cudaStream_t>(cfg->stream);
    b->fp32 = fp32;
    b->elem = fp32 ? 4 : 8;
    b->nruns = nruns;
    b->runs.assign(runs, runs + nruns);
    b->K = K;
    b->P = P;
    b->seg_rows = cfg->segment_rows > 0 ? cfg->segment_rows : 64;
    auto fail_release = [&](dirac_status st) {
        std::string m = b->err;
        release(b);
        return bfail(nullptr, st, m);
    };
    cudaError_t e = cudaSetDevice(cfg->device);
    if (e != cudaSuccess) return fail_release(bcuda(b, e, "cudaSetDevice"));
    cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, cfg->device);
    if (b->sm_count <= 0) b->sm_count = 152;
    e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail_release(bcuda(b, e, "cudaStreamCreate"));
    // state pool and tables
    size_t cells = 0, tab = 0;
    b->state_off.resize(nruns);
    for (int r = 0; r < nruns; ++r) {
        b->state_off[r] = (int64_t)cells * 8;
        cells += (size_t)2 * runs[r].side * runs[r].side;
        tab += (size_t)runs[r].side * 4;
    }
    dirac_status st;
    if ((st = balloc(b, &b->state_pool, cells * 8 * b->elem)) != DIRAC_OK) return fail_release(st);
    if ((st = balloc(b, &b->table_pool, tab * b->elem)) != DIRAC_OK) return fail_release(st);
    if ((st = balloc(b, &b->drun, nruns * sizeof(BatchRunDev))) != DIRAC_OK) return fail_release(st);
    if ((st = balloc(b, &b->flux_cum, nruns * sizeof(double))) != DIRAC_OK) return fail_release(st);
    if ((st = balloc(b, &b->norm0, nruns * sizeof(double))) != DIRAC_OK) return fail_release(st);
    if ((st = balloc(b, &b->counters, 4 * sizeof(unsigned))) != DIRAC_OK) return fail_release(st);
    if ((st = balloc(b, &b->d_order_main, nruns * sizeof(int))) != DIRAC_OK) return fail_release(st);
    if ((st = balloc(b, &b->d_order_rem, nruns * sizeof(int))) != DIRAC_OK) return fail_release(st);
    if ((st = balloc(b, &b->d_off_main, (nruns + 1) * sizeof(int64_t))) != DIRAC_OK) return fail_release(st);
    if ((st = balloc(b, &b->d_off_rem, (nruns + 1) * sizeof(int64_t))) != DIRAC_OK) return fail_release(st);
    if ((st = balloc(b, &b->d_cell_off, (nruns + 1) * sizeof(int64_t))) != DIRAC_OK) return fail_release(st);
    if ((st = balloc(b, &b->d_chunk_off, (nruns + 1) * sizeof(int64_t))) != DIRAC_OK) return fail_release(st);
    if ((st = balloc(b, &b->d_init, 4 * nruns * sizeof(double))) != DIRAC_OK) return fail_release(st);
    if ((st = balloc(b, &b->d_absorb, nruns * sizeof(int64_t))) != DIRAC_OK) return fail_release(st);
    std::vector<int64_t> absorb(nruns);
    b->mask.resize(nruns);
    for (int r = 0; r < nruns; ++r) {
        const dirac_klein_run &k = runs[r];
        absorb[r] = k.absorb;
        b->mask[r].assign(k.side, 1.0);
        for (int64_t i = 0; i < k.side && k.absorb > 0; ++i) {
            const double sl = std::min(1.0, std::max(0.0, (double)(k.absorb - i) / (double)k.absorb));
            const double sr = std::min(1.0, std::max(0.0, (double)(i - (k.side - k.absorb) + 1) / (double)k.absorb));
            const double sv = std::max(sl, sr);
            b->mask[r][i] = std::exp(-k.eta * sv * sv);
        }
    }
    std::vector<int64_t> cell_off(nruns + 1, 0), chunk_off(nruns + 1, 0);
    std::vector<double> init(4 * nruns);
    b->hrun.resize(nruns);
    size_t toff = 0;
    for (int r = 0; r < nruns; ++r) {
        const dirac_klein_run &k = runs[r];
        BatchRunDev &R = b->hrun[r];
        char *base = static_cast<char *>(b->state_pool) + (size_t)b->state_off[r] * b->elem;
        R.psi[0] = base;
        R.psi[1] = base + (size_t)k.side * k.side * 8 * b->elem;
        R.table = static_cast<char *>(b->table_pool) + toff * b->elem;
        toff += (size_t)k.side * 4;
        R.side = k.side;
        R.face = k.face;
        R.flux_cum = b->flux_cum + r;
        cell_off[r + 1] = cell_off[r] + k.side * k.side;
        chunk_off[r + 1] = chunk_off[r] + (k.side * k.side + kNormChunk - 1) / kNormChunk;
        init[r] = k.x0;
        init[nruns + r] = k.p0;
        init[2 * nruns + r] = k.width;
        init[3 * nruns + r] = cfg->c * k.p0 / (cfg->m * cfg->c * cfg->c + std::sqrt(cfg->m * cfg->m * cfg->c * cfg->c * cfg->c * cfg->c + cfg->c * cfg->c * k.p0 * k.p0));
    }
    b->nchunks = chunk_off[nruns];
    if ((st = balloc(b, &b->norm_partial, b->nchunks * sizeof(double))) != DIRAC_OK) return fail_release(st);
    e = cudaMemcpy(b->d_cell_off, cell_off.data(), (nruns + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_chunk_off, chunk_off.data(), (nruns + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_init, init.data(), 4 * nruns * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_absorb, absorb.data(), nruns * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->counters, 0, 4 * sizeof(unsigned));
    if (e != cudaSuccess) return fail_release(bcuda(b, e, "batch setup copies"));
    if ((st = plan(b)) != DIRAC_OK) return fail_release(st);
    if ((st = upload_tables(b)) != DIRAC_OK) return fail_release(st);
    if ((st = init_states(b)) != DIRAC_OK) return fail_release(st);
    e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return fail_release(bcuda(b, e, "batch init"));
    *out = b;
    return DIRAC_OK;
}

dirac_status dirac_batch_destroy(dirac_batch *b) {
    if (!b) return DIRAC_OK;
    cudaSetDevice(b->cfg.device);
    release(b);
    return DIRAC_OK;
}

dirac_status dirac_batch_reset(dirac_batch *b) {
    if (!b) return bfail(nullptr, DIRAC_ERR_ARG, "null batch");
    BCK(b, cudaSetDevice(b->cfg.device));
    return init_states(b);
}

dirac_status dirac_batch_set_state(dirac_batch *b, int run, const void *psi, int on_device) {
    if (!b || !psi || run < 0 || run >= (b ? b->nruns : 0)) return bfail(b, DIRAC_ERR_ARG, "dirac_batch_set_state: bad argument");
    if (b->ran) return bfail(b, DIRAC_ERR_STATE, "dirac_batch_set_state after dirac_batch_run: reset first");
    BCK(b, cudaSetDevice(b->cfg.device));
    const size_t bytes = (size_t)b->runs[run].side * b->runs[run].side * 8 * b->elem;
    BCK(b, cudaMemcpyAsync(b->hrun[run].psi[0], psi, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           b->stream));
    if (!on_device) BCK(b, cudaStreamSynchronize(b->stream));
    return DIRAC_OK;
}

dirac_status dirac_batch_set_potential(dirac_batch *b, int run, const double *V, int64_t count) {
    if (!b || !V || run < 0 || run >= (b ? b->nruns : 0)) return bfail(b, DIRAC_ERR_ARG, "dirac_batch_set_potential: bad argument");
    if (count != b->runs[run].side) return bfail(b, DIRAC_ERR_ARG, "dirac_batch_set_potential: count must equal side");
    BCK(b, cudaSetDevice(b->cfg.device));
    const double dt = b->cfg.dx / b->cfg.c;
    const double mu = b->cfg.m * b->cfg.c * b->cfg.c * dt;
    const int64_t side = b->runs[run].side;
    if (b->fp32) {
        std::vector<float> h(side * 4);
        for (int64_t i = 0; i < side; ++i) {
            if (!std::isfinite(V[i])) return bfail(b, DIRAC_ERR_ARG, "potential holds a non-finite value");
            double p[4];
            phase_coeffs(mu, V[i], dt, 1.0, p);
            float cu, su, cd, sd;
            const double a = b->mask[run][i];
            if (a == 1.0) {
                round_unitary(p[0], p[1], cu, su);
                round_unitary(p[2], p[3], cd, sd);
            } else {
                cu = (float)(p[0] * a);
                su = (float)(p[1] * a);
                cd = (float)(p[2] * a);
                sd = (float)(p[3] * a);
            }
            h[i * 4 + 0] = cu * 0.25f;
            h[i * 4 + 1] = su * 0.25f;
            h[i * 4 + 2] = cd * 0.25f;
            h[i * 4 + 3] = sd * 0.25f;
        }
        BCK(b, cudaMemcpy(const_cast<void *>(b->hrun[run].table), h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice));
    } else {
        std::vector<double> h(side * 4);
        for (int64_t i = 0; i < side; ++i) {
            if (!std::isfinite(V[i])) return bfail(b, DIRAC_ERR_ARG, "potential holds a non-finite value");
            phase_coeffs_masked(mu, V[i], dt, b->mask[run][i], 0.25, &h[i * 4]);
        }
        BCK(b, cudaMemcpy(const_cast<void *>(b->hrun[run].table), h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    return DIRAC_OK;
}

dirac_status dirac_batch_set_absorber(dirac_batch *b, int run, const double *a, int64_t count) {
    if (!b || !a || run < 0 || run >= (b ? b->nruns : 0)) return bfail(b, DIRAC_ERR_ARG, "dirac_batch_set_absorber: bad argument");
    if (count != b->runs[run].side) return bfail(b, DIRAC_ERR_ARG, "dirac_batch_set_absorber: count must equal side");
    for (int64_t i = 0; i < count; ++i)
        if (!(a[i] > 0.0 && a[i] <= 1.0)) return bfail(b, DIRAC_ERR_ARG, "absorber factors must lie in (0, 1]");
    b->mask[run].assign(a, a + count);
    return DIRAC_OK;
}

dirac_status dirac_batch_run(dirac_batch *b) {
    if (!b) return bfail(nullptr, DIRAC_ERR_ARG, "null batch");
    if (b->ran) return bfail(b, DIRAC_ERR_STATE, "dirac_batch_run twice without dirac_batch_reset");
    BCK(b, cudaSetDevice(b->cfg.device));
    dirac_status st = enqueue_norm(b, b->stream);
    if (st != DIRAC_OK) return st;
    if (b->cfg.use_graphs) {
        if (!b->graph) {
            const int64_t l0 = b->launches;
            BCK(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeRelaxed));
            st = enqueue_schedule(b, b->cap_stream);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
            b->launches = l0;
            if (st != DIRAC_OK) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            if (e != cudaSuccess) return bcuda(b, e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&b->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return bcuda(b, e, "cudaGraphInstantiate");
        }
        BCK(b, cudaGraphLaunch(b->graph, b->stream));
        b->launches += (int64_t)b->nact_main.size() + (int64_t)b->nact_rem.size();
    } else {
        st = enqueue_schedule(b, b->stream);
        if (st != DIRAC_OK) return st;
    }
    b->ran = true;
    return DIRAC_OK;
}

dirac_status dirac_batch_results(dirac_batch *b, double *T, double *flux, double *norm0) {
    if (!b) return bfail(nullptr, DIRAC_ERR_ARG, "null batch");
    if (!b->ran) return bfail(b, DIRAC_ERR_STATE, "dirac_batch_results before dirac_batch_run");
    BCK(b, cudaSetDevice(b->cfg.device));
    std::vector<double> F(b->nruns), N(b->nruns);
    unsigned kerr = 0;
    BCK(b, cudaMemcpyAsync(F.data(), b->flux_cum, b->nruns * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaMemcpyAsync(N.data(), b->norm0, b->nruns * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaMemcpyAsync(&kerr, b->counters + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    if (kerr) return bfail(b, DIRAC_ERR_TIMEOUT, "a batch kernel's bounded wait for a row copy ran out");
    for (int r = 0; r < b->nruns; ++r) {
        if (T) T[r] = N[r] > 0 ? F[r] / N[r] : 0.0;
        if (flux) flux[r] = F[r];
        if (norm0) norm0[r] = N[r];
    }
    return DIRAC_OK;
}

dirac_status dirac_batch_get_state(dirac_batch *b, int run, void *psi, int on_device) {
    if (!b || !psi || run < 0 || run >= (b ? b->nruns : 0)) return bfail(b, DIRAC_ERR_ARG, "dirac_batch_get_state: bad argument");
    BCK(b, cudaSetDevice(b->cfg.device));
    const int par = b->ran ? final_parity(b, run) : 0;
    const size_t bytes = (size_t)b->runs[run].side * b->runs[run].side * 8 * b->elem;
    BCK(b, cudaMemcpyAsync(psi, b->hrun[run].psi[par], bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           b->stream));
    if (!on_device) BCK(b, cudaStreamSynchronize(b->stream));
    return DIRAC_OK;
}

dirac_status dirac_batch_autotune(dirac_batch *b) {
    if (!b) return bfail(nullptr, DIRAC_ERR_ARG, "null batch");
    BCK(b, cudaSetDevice(b->cfg.device));
    struct Cand { int K, P; int64_t seg; };
    std::vector<Cand> cands;
    const int Ks[] = {1, 2, 4}, Ps[] = {2, 4};
    const int64_t segs[] = {64, 128, 256};
    for (int K : Ks)
        for (int P : Ps)
            for (int64_t sg : segs)
                if (batch_supported(b->fp32, K, P) && batch_supported(b->fp32, 1, P)) cands.push_back({K, P, sg});
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const Cand keep = {b->K, b->P, b->seg_rows};
    Cand best = keep;
    double best_t = 1e300;
    dirac_status st = DIRAC_OK;
    for (const Cand &c : cands) {
        b->K = c.K;
        b->P = c.P;
        b->seg_rows = c.seg;
        if ((st = plan(b)) != DIRAC_OK) break;
        const int64_t L = std::max<int64_t>(1, 16 / c.K);  // ~16 steps of every (long enough) run
        if ((st = enqueue_schedule(b, b->stream, L)) != DIRAC_OK) break;  // warm-up
        cudaEventRecord(e0, b->stream);
        if ((st = enqueue_schedule(b, b->stream, L)) != DIRAC_OK) break;
        cudaEventRecord(e1, b->stream);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        // point-steps advanced: runs active at each of the L launches, K steps each
        int64_t ps = 0;
        for (int r = 0; r < b->nruns; ++r) {
            const int64_t act = std::min<int64_t>(L, b->runs[r].nsteps / c.K);
            ps += act * c.K * b->runs[r].side * b->runs[r].side;
        }
        const double per = ps > 0 ? ms / (double)ps : 1e300;
        if (per < best_t) {
            best_t = per;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->K = best.K;
    b->P = best.P;
    b->seg_rows = best.seg;
    dirac_status st2 = plan(b);
    if (st == DIRAC_OK) st = st2;
    if (st == DIRAC_OK) st = upload_tables(b);
    if (st == DIRAC_OK) st = init_states(b);
    return st;
}

dirac_status dirac_batch_get_info(const dirac_batch *b, dirac_batch_info *info) {
    if (!b || !info) return bfail(nullptr, DIRAC_ERR_ARG, "null argument");
    info->steps_per_launch = b->K;
    info->points_per_lane = b->P;
    info->segment_rows = b->seg_rows;
    info->launches = (int64_t)b->nact_main.size() + (int64_t)b->nact_rem.size();
    info->max_tasks = b->max_tasks;
    int64_t ps = 0;
    for (const auto &r : b->runs) ps += r.side * r.side * r.nsteps;
    info->point_steps = ps;
    info->blocks = b->blocks;
    info->device_bytes = b->device_bytes;
    return DIRAC_OK;
}

dirac_status dirac_batch_klein(const dirac_klein_run *runs, int nruns, const dirac_batch_config *cfg, double *T_out,
                               double *R_out) {
    dirac_batch *b = nullptr;
    dirac_status st = dirac_batch_create(runs, nruns, cfg, &b);
    if (st != DIRAC_OK) return st;
    if (cfg->steps_per_launch == 0) st = dirac_batch_autotune(b);
    if (st == DIRAC_OK) st = dirac_batch_run(b);
    std::vector<double> T(nruns);
    if (st == DIRAC_OK) st = dirac_batch_results(b, T.data(), nullptr, nullptr);
    if (st == DIRAC_OK) {
        for (int r = 0; r < nruns; ++r) {
            if (T_out) T_out[r] = T[r];
            if (R_out) R_out[r] = 1.0 - T[r];
        }
    } else {
        g_batch_err = b->err;
    }
    dirac_batch_destroy(b);
    return st;
}

}  // extern "C"
