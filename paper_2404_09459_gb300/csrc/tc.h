// Tensor-core (tcgen05 / TMA) products of the sketch, power and projection steps.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gsvdr {

// True when the device is sm_103 / sm_100 class and the tcgen05 kernels were built.
bool tc_available(int device);

// Y (M x l, ld ldy, float) = G (M x n, float) * X, X given K-major as Xt (lx x n, ld ldx).
// prec selects TF32, TF32X3 or BF16 operands; accumulation is FP32.
// gnorm_part: per-CTA FP64 partial sums of G^2 (nullptr to skip), tc_gx_ctas(M) entries.
cudaError_t tc_gemm_gx(int prec, const float* G, int64_t ldg, int64_t M, int64_t n, const float* Xt,
                       int64_t ldx, int l, float* Y, int64_t ldy, double* gnorm_part, cudaStream_t st);
int tc_gx_ctas(int64_t M);

// Split-K partials of Z = G^T Q: part[z][c][j] (FP32), *splits receives the split count.
cudaError_t tc_gemm_gtq(int prec, const float* G, int64_t ldg, int64_t M, int64_t n, const float* Q,
                        int64_t ldq, int l, float* part, int64_t lp, int* splits, int64_t max_part_elems,
                        cudaStream_t st);
int64_t tc_gtq_part_elems(int64_t M, int64_t n, int l);

}  // namespace gsvdr
