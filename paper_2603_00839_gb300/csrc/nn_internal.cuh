// Internal interface of the warm-start network kernels (k_nn.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rtg {
namespace nn {

// C = op(A) op(B) (+ bias), BF16 operands, FP32 result; a_cm: A stored
// transposed; b_t: B stored N x K.  splits > 1 splits K (part: splits*M*N floats).
cudaError_t gemm(bool a_cm, bool b_t, const __nv_bfloat16* A, const __nv_bfloat16* B, float* C,
                 const float* bias, int M, int N, int K, int lda, int ldb, int splits, float* part,
                 cudaStream_t s);
cudaError_t im2col(const float* x, __nv_bfloat16* A, int N, int H, int W, int C, int stride, cudaStream_t s);
cudaError_t col2im(const float* dA, float* dx, int N, int H, int W, int C, int stride, cudaStream_t s);
cudaError_t relu_skip(const float* z, float* r, const float* skip, float* out, int64_t n, cudaStream_t s);
cudaError_t mask_grad(const float* dy, const float* mask, float* dz, __nv_bfloat16* dzb, int64_t n, cudaStream_t s);
cudaError_t colsum(const float* dz, float* db, int64_t rows, int cols, cudaStream_t s);
cudaError_t up2(const float* x, float* y, int N, int H, int W, int C, cudaStream_t s);
cudaError_t up2_back(const float* dy, float* dx, int N, int H, int W, int C, bool acc, cudaStream_t s);
cudaError_t add(const float* a, const float* b, float* out, int64_t n, cudaStream_t s);
cudaError_t to_nhwc(const float* src, float* dst, int N, int H, int W, int C, cudaStream_t s);
cudaError_t from_nhwc_add(const float* src, const float* base, float* dst, int N, int H, int W, int C,
                          cudaStream_t s);
// part: N * 32 * C floats of scratch
cudaError_t pool_head(const float* e, const float* w, const float* b, float* g, float* loglam, float* part, int N,
                      int HW, int C, cudaStream_t s);
// Implicit-GEMM 3x3 convolution forward with fused bias, ReLU and skip:
// r = act(conv(x) + b) (if r), out = r + skip (if out; skip may be null).
// H x W is the grid the convolution reads; up: x is stored at H/2 x W/2 and
// read through its nearest x2 up-sampling.  part (part_floats floats, may be
// null) lets small layers split K across CTAs.
cudaError_t conv_fwd(const float* x, const __nv_bfloat16* w, const float* bias, float* r, const float* skip,
                     float* out, int N, int H, int W, int C, int stride, int cout, bool relu, bool up,
                     float* part, int64_t part_floats, cudaStream_t s);
cudaError_t loss(const float* X0, const float* Xs, const float* loglam, const float* logmu, float* dout,
                 float* dloglam, double* out, int N, int H, int W, int C, cudaStream_t s);
cudaError_t head_back(const float* g, const float* dll, const float* w, float* dw, float* db, float* de, int N,
                      int HW, int C, cudaStream_t s);
cudaError_t adam(float* p, const float* g, float* m, float* v, __nv_bfloat16* pb, int64_t n, float lr, float b1,
                 float b2, float eps, float c1, float c2, cudaStream_t s);
cudaError_t to_bf16(const float* x, __nv_bfloat16* y, int64_t n, cudaStream_t s);

}  // namespace nn
}  // namespace rtg
