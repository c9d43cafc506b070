// Internal declarations of the surrogate network (mlp.cu, surrogate_api.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dirac {
namespace mlp {

constexpr int IN = 3;
constexpr int HID = 256;
// Parameter layout (FP32 master, its BF16 copy and the gradient share it):
// W1 [256][3], b1 [256], W2 [256][256], b2, W3, b3, W4, b4, w5 [256], b5 [1].
constexpr int64_t NPARAM = (int64_t)HID * IN + HID + 3 * ((int64_t)HID * HID + HID) + HID + 1;

struct Net {
    float *p = nullptr;           // FP32 master parameters
    float *m = nullptr, *v = nullptr;  // Adam moments
    __nv_bfloat16 *wb = nullptr;  // BF16 copy of p
    unsigned *err = nullptr;      // set by a GEMM whose bounded tensor-core wait ran out
    unsigned char *wpack = nullptr;  // BF16 W2, W3, W4 in the tensor core's shared-memory layout (inference)
    int64_t off_w[5], off_b[5];
};

struct Acts {
    float *h[4];              // tanh outputs per hidden layer [B][256] (FP32)
    __nv_bfloat16 *hb[4];     // their BF16 copies
    float *y, *dz5, *sqerr;   // [B]
    float *dz, *dh;           // [B][256]
    __nv_bfloat16 *dzb;       // [B][256]
};

inline void layout(Net &n) {
    int64_t o = 0;
    n.off_w[0] = o; o += (int64_t)HID * IN;
    n.off_b[0] = o; o += HID;
    for (int l = 1; l < 4; ++l) {
        n.off_w[l] = o; o += (int64_t)HID * HID;
        n.off_b[l] = o; o += HID;
    }
    n.off_w[4] = o; o += HID;
    n.off_b[4] = o; o += 1;
}

// C = A . B (+ C) on the tensor cores (tcgen05, accumulator in tensor memory); see mlp.cu.
cudaError_t gemm_bf16(const __nv_bfloat16 *A, int64_t sam, int64_t sak, const __nv_bfloat16 *B, int64_t sbk, int64_t sbn,
                      float *C, int64_t ldc, int M, int N, int K, int accumulate, unsigned *err, cudaStream_t s);
cudaError_t forward(const Net &n, const Acts &a, const float *x, int Bn, cudaStream_t s);
// Inference only: y = network(x) for Bn queries in one fused launch, with the same rounding points as forward.
// It reads W2-W4 from n.wpack, which pack_weights fills from n.wb (again after every change of the weights).
constexpr int64_t WPACK_BYTES = 3 * (int64_t)HID * HID * 2;
cudaError_t pack_weights(const Net &n, cudaStream_t s);
// inject_stall (tests): the first CTA's first weight wait runs out, as a stuck copy would make it.
cudaError_t infer(const Net &n, const float *x, float *y, int Bn, cudaStream_t s, int inject_stall);
cudaError_t backward(const Net &n, const Acts &a, const float *x, const float *t, float *g, int Bn, cudaStream_t s);
cudaError_t adam(const Net &n, const float *g, float lr, int64_t step, cudaStream_t s);
cudaError_t refresh_bf16(const Net &n, cudaStream_t s);

}  // namespace mlp
}  // namespace dirac
