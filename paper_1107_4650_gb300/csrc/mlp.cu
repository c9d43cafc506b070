// Surrogate network kernels: MLP 3 -> 256 -> 256 -> 256 -> 256 -> 1 (tanh hidden layers, sigmoid
// output) with BF16 weights and FP32 accumulation; forward, backward and Adam.
//
// Rounding points (the CPU gradient oracle mirrors them):
//   layer 1:        z1 = x . bf16(W1)^T + b1 in FP32 (K = 3, CUDA cores)
//   layers 2..4:    z = bf16(h) . bf16(W)^T + b, BF16 tensor-core products, FP32 accumulation
//   output:         z5 = bf16(h4) . bf16(w5) + b5 (FP32 dot), y = sigmoid(z5)
//   backward:       dz5 = 2 (y - t) y (1 - y) / B; dW5 = sum_b dz5 bf16(h4); dh4 = dz5 bf16(w5);
//                   dz = dh (1 - h^2);  dW = bf16(dz)^T . bf16(h_prev) and dh_prev = bf16(dz) . bf16(W)
//                   (tensor cores); db = sum_b dz (FP32); dW1 = dz1^T . x (FP32)
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlp_internal.cuh"

namespace dirac {
namespace mlp {

namespace {

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// C[M x N] (FP32, row-major, ldc) = sum_k A(m,k) B(k,n), A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn]
// (BF16, arbitrary strides).  Block tile 64 x 64, K tile 32; 4 warps, each a 32 x 32 sub-tile made of
// 2 x 4 mma.sync.m16n8k16 tiles.  Tiles are staged in shared memory element by element (the strided
// reads cover the transposed operands of the backward pass).
constexpr int TM = 64, TN = 64, TK = 32;

__global__ void __launch_bounds__(128) gemm_bf16_kernel(const __nv_bfloat16 *A, int64_t sam, int64_t sak,
                                                        const __nv_bfloat16 *B, int64_t sbk, int64_t sbn, float *C,
                                                        int64_t ldc, int M, int N, int K, int accumulate) {
    __shared__ __nv_bfloat16 As[TM][TK + 8];
    __shared__ __nv_bfloat16 Bs[TN][TK + 8];  // stored [n][k]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    for (int k0 = 0; k0 < K; k0 += TK) {
        for (int e = tid; e < TM * TK; e += blockDim.x) {
            const int r = e / TK, c = e % TK;
            const int m = m0 + r, k = k0 + c;
            As[r][c] = (m < M && k < K) ? A[(int64_t)m * sam + (int64_t)k * sak] : zero;
        }
        for (int e = tid; e < TN * TK; e += blockDim.x) {
            const int r = e / TK, c = e % TK;
            const int n = n0 + r, k = k0 + c;
            Bs[r][c] = (n < N && k < K) ? B[(int64_t)k * sbk + (int64_t)n * sbn] : zero;
        }
        __syncthreads();
        const int g = lane >> 2, t = lane & 3;
#pragma unroll
        for (int kk = 0; kk < TK; kk += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16;
                af[i][0] = pack_bf16(As[r + g][kk + 2 * t], As[r + g][kk + 2 * t + 1]);
                af[i][1] = pack_bf16(As[r + g + 8][kk + 2 * t], As[r + g + 8][kk + 2 * t + 1]);
                af[i][2] = pack_bf16(As[r + g][kk + 2 * t + 8], As[r + g][kk + 2 * t + 9]);
                af[i][3] = pack_bf16(As[r + g + 8][kk + 2 * t + 8], As[r + g + 8][kk + 2 * t + 9]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn + j * 8;
                bfr[j][0] = pack_bf16(Bs[c + g][kk + 2 * t], Bs[c + g][kk + 2 * t + 1]);
                bfr[j][1] = pack_bf16(Bs[c + g][kk + 2 * t + 8], Bs[c + g][kk + 2 * t + 9]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                        "{%0,%1,%2,%3};"
                        : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                        : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bfr[j][0]), "r"(bfr[j][1]));
        }
        __syncthreads();
    }
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = m0 + wm + i * 16 + g + (q >= 2 ? 8 : 0);
                const int n = n0 + wn + j * 8 + 2 * t + (q & 1);
                if (m < M && n < N) {
                    float *p = C + (int64_t)m * ldc + n;
                    *p = accumulate ? (*p + acc[i][j][q]) : acc[i][j][q];
                }
            }
}

// z1 = x . bf16(W1)^T + b1, h1 = tanh(z1); x is [B][3] FP32, W1 [256][3] BF16.
__global__ void layer1_fwd_kernel(const float *x, const __nv_bfloat16 *W1, const float *b1, float *h, __nv_bfloat16 *hb,
                                  int Bn) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)Bn * HID) return;
    const int b = (int)(e / HID), j = (int)(e % HID);
    float z = b1[j];
    z = fmaf(x[b * 3 + 0], __bfloat162float(W1[j * 3 + 0]), z);
    z = fmaf(x[b * 3 + 1], __bfloat162float(W1[j * 3 + 1]), z);
    z = fmaf(x[b * 3 + 2], __bfloat162float(W1[j * 3 + 2]), z);
    const float y = tanhf(z);
    h[e] = y;
    hb[e] = __float2bfloat16(y);
}

// h = tanh(z + b) in place on z (FP32), plus the BF16 copy.
__global__ void bias_tanh_kernel(float *z, const float *bias, __nv_bfloat16 *hb, int Bn) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)Bn * HID) return;
    const float y = tanhf(z[e] + bias[e % HID]);
    z[e] = y;
    hb[e] = __float2bfloat16(y);
}

// y = sigmoid(bf16(h4) . bf16(w5) + b5): one warp per sample.
__global__ void out_fwd_kernel(const __nv_bfloat16 *h4b, const __nv_bfloat16 *w5, const float *b5, float *y, int Bn) {
    const int lane = threadIdx.x & 31;
    const int b = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (b >= Bn) return;
    float s = 0.f;
    for (int j = lane; j < HID; j += 32) s = fmaf(__bfloat162float(h4b[(int64_t)b * HID + j]), __bfloat162float(w5[j]), s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[b] = 1.f / (1.f + expf(-(s + b5[0])));
}

// dz5 = 2 (y - t) y (1 - y) / B, and the per-sample squared error.
__global__ void out_bwd_kernel(const float *y, const float *t, float *dz5, float *sqerr, int Bn) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= Bn) return;
    const float d = y[b] - t[b];
    dz5[b] = 2.f * d * y[b] * (1.f - y[b]) / (float)Bn;
    sqerr[b] = d * d;
}

// dW5[j] = sum_b dz5[b] bf16(h4)[b][j], db5 = sum_b dz5[b] (block j = HID handles db5); then dh4 = dz5 w5.
__global__ void out_wgrad_kernel(const float *dz5, const __nv_bfloat16 *h4b, float *gW5, float *gb5, int Bn) {
    __shared__ float sh[32];
    const int j = blockIdx.x;
    float s = 0.f;
    for (int b = threadIdx.x; b < Bn; b += blockDim.x)
        s += dz5[b] * (j < HID ? __bfloat162float(h4b[(int64_t)b * HID + j]) : 1.f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[w];
        if (j < HID) gW5[j] = v; else gb5[0] = v;
    }
}

// dz = dh (1 - h^2) with dh = dz5 (x) w5 for the last hidden layer (from_out = 1) or dh given (from_out = 0);
// writes FP32 dz and its BF16 copy.
__global__ void tanh_bwd_kernel(const float *dh, const float *dz5, const __nv_bfloat16 *w5, const float *h, float *dz,
                                __nv_bfloat16 *dzb, int Bn, int from_out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)Bn * HID) return;
    const float g = from_out ? dz5[e / HID] * __bfloat162float(w5[e % HID]) : dh[e];
    const float y = h[e];
    const float v = g * (1.f - y * y);
    dz[e] = v;
    dzb[e] = __float2bfloat16(v);
}

// db[j] = sum_b dz[b][j] (FP32), one block per column.
__global__ void colsum_kernel(const float *dz, float *db, int Bn, int ncol) {
    __shared__ float sh[32];
    const int j = blockIdx.x;
    float s = 0.f;
    for (int b = threadIdx.x; b < Bn; b += blockDim.x) s += dz[(int64_t)b * ncol + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[w];
        db[j] = v;
    }
}

// dW1[j][i] = sum_b dz1[b][j] x[b][i] (FP32), one block per (j, i).
__global__ void layer1_wgrad_kernel(const float *dz1, const float *x, float *gW1, int Bn) {
    __shared__ float sh[32];
    const int j = blockIdx.x / 3, i = blockIdx.x % 3;
    float s = 0.f;
    for (int b = threadIdx.x; b < Bn; b += blockDim.x) s += dz1[(int64_t)b * HID + j] * x[b * 3 + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[w];
        gW1[j * 3 + i] = v;
    }
}

// Adam on the FP32 master parameters; refreshes the BF16 copies of the weight entries.
__global__ void adam_kernel(float *p, const float *g, float *m, float *v, __nv_bfloat16 *pb, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float upd = lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    const float np = p[i] - upd;
    p[i] = np;
    pb[i] = __float2bfloat16(np);
}

__global__ void to_bf16_kernel(const float *p, __nv_bfloat16 *pb, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pb[i] = __float2bfloat16(p[i]);
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

cudaError_t gemm_bf16(const __nv_bfloat16 *A, int64_t sam, int64_t sak, const __nv_bfloat16 *B, int64_t sbk, int64_t sbn,
                      float *C, int64_t ldc, int M, int N, int K, int accumulate, cudaStream_t s) {
    dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM);
    gemm_bf16_kernel<<<grid, 128, 0, s>>>(A, sam, sak, B, sbk, sbn, C, ldc, M, N, K, accumulate);
    return cudaGetLastError();
}

// Forward pass for a batch: fills the activation buffers and y.
cudaError_t forward(const Net &n, const Acts &a, const float *x, int Bn, cudaStream_t s) {
    const int64_t E = (int64_t)Bn * HID;
    layer1_fwd_kernel<<<nblk(E, 256), 256, 0, s>>>(x, n.wb + n.off_w[0], n.p + n.off_b[0], a.h[0], a.hb[0], Bn);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int l = 1; l < 4; ++l) {
        // z_l[b][j] = sum_k bf16(h_{l-1})[b][k] bf16(W_l)[j][k]
        e = gemm_bf16(a.hb[l - 1], HID, 1, n.wb + n.off_w[l], 1, HID, a.h[l], HID, Bn, HID, HID, 0, s);
        if (e != cudaSuccess) return e;
        bias_tanh_kernel<<<nblk(E, 256), 256, 0, s>>>(a.h[l], n.p + n.off_b[l], a.hb[l], Bn);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    out_fwd_kernel<<<nblk((int64_t)Bn * 32, 256), 256, 0, s>>>(a.hb[3], n.wb + n.off_w[4], n.p + n.off_b[4], a.y, Bn);
    return cudaGetLastError();
}

// Backward pass (after forward): gradients of mean((y - t)^2) into g (same layout as the parameters).
cudaError_t backward(const Net &n, const Acts &a, const float *x, const float *t, float *g, int Bn, cudaStream_t s) {
    const int64_t E = (int64_t)Bn * HID;
    out_bwd_kernel<<<nblk(Bn, 256), 256, 0, s>>>(a.y, t, a.dz5, a.sqerr, Bn);
    out_wgrad_kernel<<<HID + 1, 256, 0, s>>>(a.dz5, a.hb[3], g + n.off_w[4], g + n.off_b[4], Bn);
    tanh_bwd_kernel<<<nblk(E, 256), 256, 0, s>>>(nullptr, a.dz5, n.wb + n.off_w[4], a.h[3], a.dz, a.dzb, Bn, 1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int l = 3; l >= 1; --l) {
        // dW_l[j][k] = sum_b bf16(dz)[b][j] bf16(h_{l-1})[b][k]:  A(m=j, k=b) = dzb[b*HID + j], B(k=b, n=k) = hb[b*HID + k]
        e = gemm_bf16(a.dzb, 1, HID, a.hb[l - 1], HID, 1, g + n.off_w[l], HID, HID, HID, Bn, 0, s);
        if (e != cudaSuccess) return e;
        colsum_kernel<<<HID, 256, 0, s>>>(a.dz, g + n.off_b[l], Bn, HID);
        // dh_{l-1}[b][k] = sum_j bf16(dz)[b][j] bf16(W_l)[j][k]:  A(m=b, k=j) = dzb[b*HID + j], B(k=j, n=k) = W[j*HID + k]
        e = gemm_bf16(a.dzb, HID, 1, n.wb + n.off_w[l], HID, 1, a.dh, HID, Bn, HID, HID, 0, s);
        if (e != cudaSuccess) return e;
        tanh_bwd_kernel<<<nblk(E, 256), 256, 0, s>>>(a.dh, nullptr, nullptr, a.h[l - 1], a.dz, a.dzb, Bn, 0);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    layer1_wgrad_kernel<<<HID * 3, 256, 0, s>>>(a.dz, x, g + n.off_w[0], Bn);
    colsum_kernel<<<HID, 256, 0, s>>>(a.dz, g + n.off_b[0], Bn, HID);
    return cudaGetLastError();
}

cudaError_t adam(const Net &n, const float *g, float lr, int64_t step, cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<nblk(NPARAM, 256), 256, 0, s>>>(n.p, g, n.m, n.v, n.wb, NPARAM, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t refresh_bf16(const Net &n, cudaStream_t s) {
    to_bf16_kernel<<<nblk(NPARAM, 256), 256, 0, s>>>(n.p, n.wb, NPARAM);
    return cudaGetLastError();
}

}  // namespace mlp
}  // namespace dirac
