// Host runtime of the transmission surrogate (include/dirac.h, dirac_surrogate_*).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dirac.h"
#include "mlp_internal.cuh"

using namespace dirac::mlp;

namespace {
thread_local std::string g_sur_err;

// splitmix64 (Steele, Lea, Flood 2014): one 64-bit output per counter value.
uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double unit(uint64_t seed, uint64_t i) { return (double)(splitmix64(seed * 0x100000001B3ull + i) >> 11) * 0x1.0p-53; }

__global__ void gather_kernel(const float *X, const float *T, const int *idx, float *xb, float *tb, int Bn) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= Bn) return;
    const int i = idx[b];
    xb[b * 3 + 0] = X[i * 3 + 0];
    xb[b * 3 + 1] = X[i * 3 + 1];
    xb[b * 3 + 2] = X[i * 3 + 2];
    if (T) tb[b] = T[i];
}

}  // namespace

struct dirac_surrogate {
    double lo[3], hi[3];
    uint64_t seed = 0;
    int max_batch = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    Net net;
    Acts acts{};
    float *grad = nullptr;
    float *xb = nullptr, *tb = nullptr;
    int *idx = nullptr;
    float *host_pinned = nullptr;  // staging: max_batch * 4 floats
    unsigned *flag_pinned = nullptr;  // the tensor-wait flag, read back with a prediction's outputs
    bool packed = false;  // net.wpack holds the current W2-W4 (cleared whenever the weights change)
    int inject_stall = 0;  // DIRAC_INJECT_STALL set at creation: every prediction launch stalls one wait
    int64_t step = 0;
    bool bias_set = false;  // output bias already chosen (trained or loaded parameters)
    std::vector<void *> owned;
    std::string err;
};

namespace {

dirac_status sfail(dirac_surrogate *s, dirac_status st, const std::string &m) {
    if (s) s->err = m; else g_sur_err = m;
    return st;
}
dirac_status scuda(dirac_surrogate *s, cudaError_t e, const char *w) {
    return sfail(s, e == cudaErrorMemoryAllocation ? DIRAC_ERR_OOM : DIRAC_ERR_CUDA,
                 std::string(w) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}
#define SCK(s, expr)                                          \
    do {                                                      \
        cudaError_t e_ = (expr);                              \
        if (e_ != cudaSuccess) return scuda((s), e_, #expr);  \
    } while (0)

template <typename T>
cudaError_t salloc(dirac_surrogate *s, T **p, size_t bytes) {
    cudaError_t e = cudaMalloc((void **)p, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess) s->owned.push_back(*p);
    return e;
}

void normalise(const dirac_surrogate *s, const double *q, float *out) {
    for (int d = 0; d < 3; ++d) out[d] = (float)(2.0 * (q[d] - s->lo[d]) / (s->hi[d] - s->lo[d]) - 1.0);
}

bool in_box(const dirac_surrogate *s, const double *q) {
    for (int d = 0; d < 3; ++d)
        if (!(q[d] >= s->lo[d] && q[d] <= s->hi[d])) return false;
    return true;
}

// Uploads normalised inputs (and targets) of points [i0, i0 + nb) into the batch buffers.
dirac_status stage(dirac_surrogate *s, const double *X, const double *T, int64_t i0, int nb) {
    float *h = s->host_pinned;
    // large batches: the per-query divisions on all host cores (each query's arithmetic unchanged)
#pragma omp parallel for schedule(static) if (nb >= 32768)
    for (int b = 0; b < nb; ++b) normalise(s, X + (i0 + b) * 3, h + b * 3);
    SCK(s, cudaMemcpyAsync(s->xb, h, (size_t)nb * 3 * sizeof(float), cudaMemcpyHostToDevice, s->stream));
    if (T) {
        float *ht = h + (size_t)s->max_batch * 3;
        for (int b = 0; b < nb; ++b) ht[b] = (float)T[i0 + b];
        SCK(s, cudaMemcpyAsync(s->tb, ht, (size_t)nb * sizeof(float), cudaMemcpyHostToDevice, s->stream));
    }
    return DIRAC_OK;
}

// Reads (and clears) the flag a GEMM sets when its bounded wait for the tensor cores ran out.
dirac_status check_tensor_waits(dirac_surrogate *s) {
    unsigned flag = 0;
    SCK(s, cudaMemcpy(&flag, s->net.err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (!flag) return DIRAC_OK;
    SCK(s, cudaMemset(s->net.err, 0, sizeof(unsigned)));
    return sfail(s, DIRAC_ERR_TIMEOUT, "a tensor-core GEMM's bounded wait ran out; results are invalid");
}

}  // namespace

extern "C" {

int64_t dirac_surrogate_num_params(void) { return NPARAM; }

dirac_status dirac_surrogate_create(const double lo[3], const double hi[3], uint64_t seed, int max_batch, void *stream,
                                    int device, dirac_surrogate **out) {
    if (!lo || !hi || !out || max_batch < 1 || max_batch > (1 << 20))
        return sfail(nullptr, DIRAC_ERR_ARG, "dirac_surrogate_create: bad arguments");
    for (int d = 0; d < 3; ++d)
        if (!(hi[d] > lo[d]) || !std::isfinite(lo[d]) || !std::isfinite(hi[d]))
            return sfail(nullptr, DIRAC_ERR_ARG, "dirac_surrogate_create: box needs lo < hi, finite");
    *out = nullptr;
    dirac_surrogate *s = new (std::nothrow) dirac_surrogate();
    if (!s) return sfail(nullptr, DIRAC_ERR_OOM, "host allocation failed");
    std::memcpy(s->lo, lo, sizeof(s->lo));
    std::memcpy(s->hi, hi, sizeof(s->hi));
    s->seed = seed;
    s->max_batch = max_batch;
    s->inject_stall = std::getenv("DIRAC_INJECT_STALL") ? 1 : 0;
    s->stream = static_cast<cudaStream_t>(stream);
    s->device = device;
    auto bail = [&](dirac_status st) {
        std::string m = s->err;
        dirac_surrogate_destroy(s);
        return sfail(nullptr, st, m);
    };
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return bail(scuda(s, e, "cudaSetDevice"));
    layout(s->net);
    const size_t B = (size_t)max_batch;
    e = salloc(s, &s->net.p, NPARAM * sizeof(float));
    if (e == cudaSuccess) e = salloc(s, &s->net.m, NPARAM * sizeof(float));
    if (e == cudaSuccess) e = salloc(s, &s->net.v, NPARAM * sizeof(float));
    if (e == cudaSuccess) e = salloc(s, &s->net.wb, NPARAM * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = salloc(s, &s->net.wpack, WPACK_BYTES);
    if (e == cudaSuccess) e = salloc(s, &s->grad, NPARAM * sizeof(float));
    for (int l = 0; l < 4 && e == cudaSuccess; ++l) {
        e = salloc(s, &s->acts.h[l], B * HID * sizeof(float));
        if (e == cudaSuccess) e = salloc(s, &s->acts.hb[l], B * HID * sizeof(__nv_bfloat16));
    }
    if (e == cudaSuccess) e = salloc(s, &s->acts.y, B * sizeof(float));
    if (e == cudaSuccess) e = salloc(s, &s->acts.dz5, B * sizeof(float));
    if (e == cudaSuccess) e = salloc(s, &s->acts.sqerr, B * sizeof(float));
    if (e == cudaSuccess) e = salloc(s, &s->acts.dz, B * HID * sizeof(float));
    if (e == cudaSuccess) e = salloc(s, &s->acts.dh, B * HID * sizeof(float));
    if (e == cudaSuccess) e = salloc(s, &s->acts.dzb, B * HID * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = salloc(s, &s->xb, B * 3 * sizeof(float));
    if (e == cudaSuccess) e = salloc(s, &s->tb, B * sizeof(float));
    if (e == cudaSuccess) e = salloc(s, &s->idx, B * sizeof(int));
    if (e == cudaSuccess) e = salloc(s, &s->net.err, 16);
    if (e == cudaSuccess) e = cudaMemset(s->net.err, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMallocHost(&s->host_pinned, B * 4 * sizeof(float));
    if (e == cudaSuccess) e = cudaMallocHost(&s->flag_pinned, 16);
    if (e != cudaSuccess) return bail(scuda(s, e, "surrogate allocation"));
    // Xavier-uniform weights, zero biases
    std::vector<float> p(NPARAM, 0.f);
    const int fan[5][2] = {{IN, HID}, {HID, HID}, {HID, HID}, {HID, HID}, {HID, 1}};
    for (int l = 0; l < 5; ++l) {
        const double a = std::sqrt(6.0 / (fan[l][0] + fan[l][1]));
        const int64_t cnt = (int64_t)fan[l][0] * fan[l][1];
        for (int64_t i = 0; i < cnt; ++i) p[s->net.off_w[l] + i] = (float)(a * (2.0 * unit(seed, s->net.off_w[l] + i) - 1.0));
    }
    dirac_status st = dirac_surrogate_set_params(s, p.data());
    if (st != DIRAC_OK) return bail(st);
    s->bias_set = false;
    *out = s;
    return DIRAC_OK;
}

dirac_status dirac_surrogate_destroy(dirac_surrogate *s) {
    if (!s) return DIRAC_OK;
    cudaSetDevice(s->device);
    cudaStreamSynchronize(s->stream);
    for (void *p : s->owned) cudaFree(p);
    if (s->host_pinned) cudaFreeHost(s->host_pinned);
    if (s->flag_pinned) cudaFreeHost(s->flag_pinned);
    delete s;
    return DIRAC_OK;
}

dirac_status dirac_surrogate_set_params(dirac_surrogate *s, const float *params) {
    if (!s || !params) return sfail(s, DIRAC_ERR_ARG, "null argument");
    SCK(s, cudaSetDevice(s->device));
    SCK(s, cudaMemcpyAsync(s->net.p, params, NPARAM * sizeof(float), cudaMemcpyHostToDevice, s->stream));
    SCK(s, cudaMemsetAsync(s->net.m, 0, NPARAM * sizeof(float), s->stream));
    SCK(s, cudaMemsetAsync(s->net.v, 0, NPARAM * sizeof(float), s->stream));
    s->packed = false;
    SCK(s, refresh_bf16(s->net, s->stream));
    SCK(s, cudaStreamSynchronize(s->stream));
    s->step = 0;
    s->bias_set = true;
    return DIRAC_OK;
}

dirac_status dirac_surrogate_get_params(dirac_surrogate *s, float *params) {
    if (!s || !params) return sfail(s, DIRAC_ERR_ARG, "null argument");
    SCK(s, cudaSetDevice(s->device));
    SCK(s, cudaMemcpyAsync(params, s->net.p, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
    SCK(s, cudaStreamSynchronize(s->stream));
    return DIRAC_OK;
}

// Checkpoint file: "DIRACNN1", uint32 version 1, uint32 parameter count, the box lo[3], hi[3] (FP64), int64 Adam
// step, uint64 shuffle seed, then the FP32 parameters, Adam first and second moments (NPARAM floats each), host
// byte order.
namespace {
constexpr char kCkptMagic[8] = {'D', 'I', 'R', 'A', 'C', 'N', 'N', '1'};
}

dirac_status dirac_surrogate_save(dirac_surrogate *s, const char *path) {
    if (!s || !path) return sfail(s, DIRAC_ERR_ARG, "dirac_surrogate_save: null argument");
    SCK(s, cudaSetDevice(s->device));
    std::vector<float> buf((size_t)3 * NPARAM);
    SCK(s, cudaMemcpyAsync(buf.data(), s->net.p, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
    SCK(s, cudaMemcpyAsync(buf.data() + NPARAM, s->net.m, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
    SCK(s, cudaMemcpyAsync(buf.data() + 2 * NPARAM, s->net.v, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
    SCK(s, cudaStreamSynchronize(s->stream));
    std::FILE *f = std::fopen(path, "wb");
    if (!f) return sfail(s, DIRAC_ERR_ARG, std::string("dirac_surrogate_save: cannot open ") + path);
    const uint32_t head[2] = {1u, (uint32_t)NPARAM};
    const int64_t step = s->step;
    bool ok = std::fwrite(kCkptMagic, 1, 8, f) == 8 && std::fwrite(head, sizeof(uint32_t), 2, f) == 2 &&
              std::fwrite(s->lo, sizeof(double), 3, f) == 3 && std::fwrite(s->hi, sizeof(double), 3, f) == 3 &&
              std::fwrite(&step, sizeof(int64_t), 1, f) == 1 && std::fwrite(&s->seed, sizeof(uint64_t), 1, f) == 1 &&
              std::fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return sfail(s, DIRAC_ERR_ARG, std::string("dirac_surrogate_save: write to ") + path + " failed");
    return DIRAC_OK;
}

dirac_status dirac_surrogate_load(dirac_surrogate *s, const char *path) {
    if (!s || !path) return sfail(s, DIRAC_ERR_ARG, "dirac_surrogate_load: null argument");
    std::FILE *f = std::fopen(path, "rb");
    if (!f) return sfail(s, DIRAC_ERR_ARG, std::string("dirac_surrogate_load: cannot open ") + path);
    char magic[8];
    uint32_t head[2];
    double lo[3], hi[3];
    int64_t step = 0;
    uint64_t seed = 0;
    std::vector<float> buf((size_t)3 * NPARAM);
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kCkptMagic, 8) == 0 &&
              std::fread(head, sizeof(uint32_t), 2, f) == 2 && head[0] == 1u && head[1] == (uint32_t)NPARAM &&
              std::fread(lo, sizeof(double), 3, f) == 3 && std::fread(hi, sizeof(double), 3, f) == 3 &&
              std::fread(&step, sizeof(int64_t), 1, f) == 1 && std::fread(&seed, sizeof(uint64_t), 1, f) == 1 &&
              std::fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    std::fclose(f);
    if (!ok) return sfail(s, DIRAC_ERR_ARG, std::string("dirac_surrogate_load: ") + path + " is not a checkpoint of this network");
    for (int d = 0; d < 3; ++d)
        if (!(hi[d] > lo[d]) || !std::isfinite(lo[d]) || !std::isfinite(hi[d]) || step < 0)
            return sfail(s, DIRAC_ERR_ARG, "dirac_surrogate_load: bad box or step in the checkpoint");
    SCK(s, cudaSetDevice(s->device));
    SCK(s, cudaMemcpyAsync(s->net.p, buf.data(), NPARAM * sizeof(float), cudaMemcpyHostToDevice, s->stream));
    SCK(s, cudaMemcpyAsync(s->net.m, buf.data() + NPARAM, NPARAM * sizeof(float), cudaMemcpyHostToDevice, s->stream));
    SCK(s, cudaMemcpyAsync(s->net.v, buf.data() + 2 * NPARAM, NPARAM * sizeof(float), cudaMemcpyHostToDevice, s->stream));
    s->packed = false;
    SCK(s, refresh_bf16(s->net, s->stream));
    SCK(s, cudaStreamSynchronize(s->stream));
    for (int d = 0; d < 3; ++d) {
        s->lo[d] = lo[d];
        s->hi[d] = hi[d];
    }
    s->step = step;
    s->seed = seed;
    s->bias_set = true;
    return DIRAC_OK;
}

dirac_status dirac_surrogate_gradient(dirac_surrogate *s, const double *X, const double *T, int64_t n, float *grad_out,
                                      double *loss_out) {
    if (!s || !X || !T || !grad_out || n < 1 || n > s->max_batch) return sfail(s, DIRAC_ERR_ARG, "bad arguments");
    SCK(s, cudaSetDevice(s->device));
    dirac_status st = stage(s, X, T, 0, (int)n);
    if (st != DIRAC_OK) return st;
    SCK(s, forward(s->net, s->acts, s->xb, (int)n, s->stream));
    SCK(s, backward(s->net, s->acts, s->xb, s->tb, s->grad, (int)n, s->stream));
    std::vector<float> sq(n);
    SCK(s, cudaMemcpyAsync(grad_out, s->grad, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
    SCK(s, cudaMemcpyAsync(sq.data(), s->acts.sqerr, n * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
    SCK(s, cudaStreamSynchronize(s->stream));
    st = check_tensor_waits(s);
    if (st != DIRAC_OK) return st;
    if (loss_out) {
        double L = 0;
        for (float v : sq) L += v;
        *loss_out = L / (double)n;
    }
    return DIRAC_OK;
}

dirac_status dirac_surrogate_train(dirac_surrogate *s, const double *X, const double *T, int64_t n, int epochs,
                                   int batch, double lr, double *loss_out) {
    if (!s || !X || !T || n < 1 || epochs < 0 || batch < 1 || batch > s->max_batch || !(lr > 0))
        return sfail(s, DIRAC_ERR_ARG, "dirac_surrogate_train: bad arguments");
    SCK(s, cudaSetDevice(s->device));
    s->packed = false;  // the Adam steps change the weights
    float *dX = nullptr, *dT = nullptr;
    int *dIdx = nullptr;
    std::vector<float> hx((size_t)n * 3), ht(n);
    for (int64_t i = 0; i < n; ++i) {
        normalise(s, X + i * 3, &hx[i * 3]);
        ht[i] = (float)T[i];
    }
    cudaError_t e = cudaMalloc(&dX, hx.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dT, ht.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dIdx, (size_t)n * sizeof(int));
    auto cleanup = [&]() {
        cudaFree(dX);
        cudaFree(dT);
        cudaFree(dIdx);
    };
    if (e != cudaSuccess) {
        cleanup();
        return scuda(s, e, "training buffers");
    }
    e = cudaMemcpy(dX, hx.data(), hx.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dT, ht.data(), ht.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !s->bias_set) {
        // first training call: start the output at the mean target (bias = logit of the mean), so the
        // sigmoid does not begin in a saturated region where the squared-error gradient vanishes
        double mean = 0.0;
        for (int64_t i = 0; i < n; ++i) mean += T[i];
        mean = std::min(1.0 - 1e-4, std::max(1e-4, mean / (double)n));
        const float b5 = (float)std::log(mean / (1.0 - mean));
        e = cudaMemcpy(s->net.p + s->net.off_b[4], &b5, sizeof(float), cudaMemcpyHostToDevice);
        s->bias_set = true;
    }
    std::vector<int> perm(n);
    const int64_t nb = n / batch;  // full batches per epoch (at least one: a smaller n trains on all of it)
    const int64_t per_epoch = std::max<int64_t>(1, nb);
    const int bsz = nb > 0 ? batch : (int)n;
    const int64_t total = per_epoch * epochs;
    std::vector<float> sq(bsz);
    double last = 0.0;
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
        for (int64_t i = 0; i < n; ++i) perm[i] = (int)i;
        for (int64_t i = n - 1; i > 0; --i) {  // Fisher-Yates
            const int64_t j = (int64_t)(unit(s->seed ^ 0xA5A5A5A5ull, (uint64_t)ep * (uint64_t)n + i) * (i + 1));
            std::swap(perm[i], perm[std::min<int64_t>(j, i)]);
        }
        e = cudaMemcpyAsync(dIdx, perm.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, s->stream);
        double ep_loss = 0.0;
        for (int64_t bi = 0; bi < per_epoch && e == cudaSuccess; ++bi) {
            gather_kernel<<<(bsz + 255) / 256, 256, 0, s->stream>>>(dX, dT, dIdx + bi * bsz, s->xb, s->tb, bsz);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = forward(s->net, s->acts, s->xb, bsz, s->stream);
            if (e == cudaSuccess) e = backward(s->net, s->acts, s->xb, s->tb, s->grad, bsz, s->stream);
            const double t = (double)s->step / (double)std::max<int64_t>(1, total);
            const double lr_t = lr / 20.0 + 0.5 * (lr - lr / 20.0) * (1.0 + std::cos(M_PI * t));
            ++s->step;
            if (e == cudaSuccess) e = adam(s->net, s->grad, (float)lr_t, s->step, s->stream);
            if (e == cudaSuccess && ep == epochs - 1) {
                e = cudaMemcpyAsync(sq.data(), s->acts.sqerr, bsz * sizeof(float), cudaMemcpyDeviceToHost, s->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
                for (float v : sq) ep_loss += v;
            }
        }
        if (ep == epochs - 1) last = ep_loss / (double)(per_epoch * bsz);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cleanup();
    if (e != cudaSuccess) return scuda(s, e, "training step");
    dirac_status st = check_tensor_waits(s);
    if (st != DIRAC_OK) return st;
    if (loss_out) *loss_out = last;
    return DIRAC_OK;
}

dirac_status dirac_surrogate_predict(dirac_surrogate *s, const double *X, int64_t n, double *T_out) {
    if (!s || !X || !T_out || n < 0) return sfail(s, DIRAC_ERR_ARG, "bad arguments");
    SCK(s, cudaSetDevice(s->device));
    if (!s->packed) {
        SCK(s, pack_weights(s->net, s->stream));
        s->packed = true;
    }
    std::vector<float> y(s->max_batch);
    *s->flag_pinned = 0;
    for (int64_t i0 = 0; i0 < n; i0 += s->max_batch) {
        const int nb = (int)std::min<int64_t>(s->max_batch, n - i0);
        dirac_status st = stage(s, X, nullptr, i0, nb);
        if (st != DIRAC_OK) return st;
        SCK(s, infer(s->net, s->xb, s->acts.y, nb, s->stream, s->inject_stall));
        SCK(s, cudaMemcpyAsync(y.data(), s->acts.y, nb * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
        if (i0 + nb >= n)  // the flag a timed-out tensor-core wait sets, read with the last outputs
            SCK(s, cudaMemcpyAsync(s->flag_pinned, s->net.err, sizeof(unsigned), cudaMemcpyDeviceToHost, s->stream));
        SCK(s, cudaStreamSynchronize(s->stream));
#pragma omp parallel for schedule(static) if (nb >= 32768)
        for (int b = 0; b < nb; ++b) T_out[i0 + b] = y[b];
    }
    if (*s->flag_pinned) {
        SCK(s, cudaMemset(s->net.err, 0, sizeof(unsigned)));
        return sfail(s, DIRAC_ERR_TIMEOUT, "a tensor-core wait of the inference kernel ran out; results are invalid");
    }
    return DIRAC_OK;
}

dirac_status dirac_klein_run_from_reduced(const double q[3], double dx, double c, double m, dirac_klein_run *run) {
    if (!q || !run || !(dx > 0) || !(c > 0) || !(m > 0) || !(q[2] > 0) || !(q[1] > 0) || !std::isfinite(q[0]))
        return sfail(nullptr, DIRAC_ERR_ARG, "dirac_klein_run_from_reduced: bad arguments");
    static const int64_t sides[] = {256, 384, 512, 768, 1024};
    const double wc = q[2];
    const int64_t absorb = 64;   // absorbing-layer columns at each x edge
    const int64_t beyond = 128;  // cells between the step face and the right absorbing layer
    const double need = 8.0 * wc + 8.0 + (double)(beyond + 2 * absorb);
    int64_t side = 1024;
    for (int64_t sd : sides)
        if ((double)sd >= need) {
            side = sd;
            break;
        }
    const double p0 = q[1] * m * c;
    const double E = std::sqrt(p0 * p0 * c * c + m * m * c * c * c * c);
    const double vg = p0 * c / E;
    const double steps = std::ceil(8.0 * wc / vg) + 200.0;
    run->side = side;
    run->face = std::min<int64_t>((int64_t)std::ceil(8.0 * wc) + 8 + absorb, side - beyond - absorb);
    run->nsteps = (int64_t)std::min(6000.0, std::max(2000.0, steps));
    run->V0 = q[0] * m * c * c;
    run->L = 4.0 * dx;
    run->p0 = p0;
    run->width = wc * dx;
    run->x0 = -4.0 * wc * dx;
    run->absorb = absorb;
    run->eta = 0.1;
    return DIRAC_OK;
}

dirac_status dirac_surrogate_query(dirac_surrogate *s, const double *X, int64_t n, const dirac_batch_config *solver_cfg,
                                   double *T_out, int *used_solver) {
    if (!s || !X || !T_out || n < 0 || !solver_cfg) return sfail(s, DIRAC_ERR_ARG, "bad arguments");
    std::vector<int64_t> inside, outside;
    for (int64_t i = 0; i < n; ++i) (in_box(s, X + i * 3) ? inside : outside).push_back(i);
    if (!inside.empty()) {
        std::vector<double> xi(inside.size() * 3), ti(inside.size());
        for (size_t k = 0; k < inside.size(); ++k) std::memcpy(&xi[k * 3], X + inside[k] * 3, 3 * sizeof(double));
        dirac_status st = dirac_surrogate_predict(s, xi.data(), (int64_t)inside.size(), ti.data());
        if (st != DIRAC_OK) return st;
        for (size_t k = 0; k < inside.size(); ++k) {
            T_out[inside[k]] = ti[k];
            if (used_solver) used_solver[inside[k]] = 0;
        }
    }
    if (!outside.empty()) {
        std::vector<dirac_klein_run> runs(outside.size());
        for (size_t k = 0; k < outside.size(); ++k) {
            dirac_status st = dirac_klein_run_from_reduced(X + outside[k] * 3, solver_cfg->dx, solver_cfg->c, solver_cfg->m, &runs[k]);
            if (st != DIRAC_OK) return sfail(s, st, "query " + std::to_string(outside[k]) + ": invalid parameters");
        }
        std::vector<double> T(outside.size());
        dirac_status st = dirac_batch_klein(runs.data(), (int)runs.size(), solver_cfg, T.data(), nullptr);
        if (st != DIRAC_OK) return sfail(s, st, std::string("fallback solver: ") + dirac_batch_last_error(nullptr));
        for (size_t k = 0; k < outside.size(); ++k) {
            T_out[outside[k]] = T[k];
            if (used_solver) used_solver[outside[k]] = 1;
        }
    }
    return DIRAC_OK;
}

const char *dirac_surrogate_last_error(const dirac_surrogate *s) { return s ? s->err.c_str() : g_sur_err.c_str(); }

}  // extern "C"
