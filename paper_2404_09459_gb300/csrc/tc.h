// Tensor-core (tcgen05 / TMA) products of the sketch, power and projection steps.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace gsvdr {

// True when the device is sm_103 and the driver exposes tensor-map encoding.
bool tc_available(int device);
// TMA addressing constraints: 16-byte aligned base, row stride (ldg elements of eb bytes)
// a multiple of 16 bytes, l <= 256.
bool tc_shape_ok(const void* G, int64_t ldg, int l, int eb = 4);

// Y (M x l, ld ldy) = G (M x n, ld ldg) X with X given K-major as Xt (round_up(l,16) x n,
// ld ldx, rows l.. zero).  TF32 operands, FP32 accumulation.  gnorm_part (or nullptr):
// per-CTA FP64 sums of G^2, tc_gx_ctas(M) entries.  A timed-out pipeline wait sets
// TIMEOUT in st_dev.
cudaError_t tc_gemm_gx(int prec, const float* G, int64_t ldg, int64_t M, int64_t n, const float* Xt, int64_t ldx,
                       int l, float* Y, int64_t ldy, double* gnorm_part, DevStatus* st_dev, cudaStream_t st);
int tc_gx_ctas(int64_t M);

// Split-K partials of Z = G^T Q with Q given transposed as Qt (round_up(l,16) x M, ld ldq,
// rows l.. zero): part[z][c][j] (FP32, ld lp); *splits receives the split count.
cudaError_t tc_gemm_gtq(int prec, const float* G, int64_t ldg, int64_t M, int64_t n, const float* Qt, int64_t ldq,
                        int l, float* part, int64_t lp, int* splits, int64_t max_part_elems, DevStatus* st_dev,
                        cudaStream_t st);
int64_t tc_gtq_part_elems(int64_t M, int64_t n, int l);

// BF16 data (G row-major BF16, ld a multiple of 8): Y = G X with X given K-major as BF16
// halves Xh (+ Xl, or nullptr for one product), each round_up(l,16) x n with ld ldx
// (a multiple of 8), padding rows zero.  FP32 accumulation.
cudaError_t tc_gemm_gx_bf16(const void* G, int64_t ldg, int64_t M, int64_t n, const void* Xh, const void* Xl,
                            int64_t ldx, int l, float* Y, int64_t ldy, double* gnorm_part, DevStatus* st_dev,
                            cudaStream_t st);
// Split-K partials of Z = G^T Q with Q^T given as BF16 halves Qh (+ Ql), round_up(l,16) x M
// with ld ldq (a multiple of 8), padding rows zero.
cudaError_t tc_gemm_gtq_bf16(const void* G, int64_t ldg, int64_t M, int64_t n, const void* Qh, const void* Ql,
                             int64_t ldq, int l, float* part, int64_t lp, int* splits, int64_t max_part_elems,
                             DevStatus* st_dev, cudaStream_t st);
int tc_gtq_splits_bf16(int64_t M, int64_t n, bool split);

// ---- grouped persistent products (many independent problems, one launch) ----
// One problem: G (M x n, row-major FP32, ld ldg, TMA-aligned) times a K-major B operand
// Bt with ld ldb: mode 0 (GX) Y = G X with Bt = X^T (round_up(l,16) x n, padding rows
// zero), out = Y (M x l, ld ldo), gnorm_part (or nullptr) receives tc_group_norm_parts()
// partial sums of G^2 per 128-row tile; mode 1 (GTQ) split-K partials of G^T Q with Bt = Q^T
// (round_up(l,16) x M), `splits` row ranges of rps rows (a multiple of 32), partial z
// at out + z * split_stride (n x l, ld ldo).
// transpose_out (mode 0): Y stored column-major, out[c * ldo + row].
struct TcGroupSpec {
  const float* G;
  int64_t ldg, M, n;
  const float* Bt;
  int64_t ldb;
  int l;
  float* out;
  int64_t ldo;
  int splits;
  int64_t rps, split_stride;
  double* gnorm_part;
  int transpose_out;
  const int* stop;  // null, or the problem's stop word: its tiles are left out once it is non-zero
  // mode 0, 3xTF32: null, or Bt - tf32(Bt) in Bt's layout, loaded by TMA beside Bt (the preparation
  // warps then form only A's low half)
  const float* Bt_lo;
};
int tc_group_norm_parts();
// Tiles of a grouped launch (128-row tiles in mode 0; column tiles x splits in mode 1).
int64_t tc_group_tiles(int mode, const TcGroupSpec* specs, int nprob);
// Bytes of the device table: the problems, then the tile list.
size_t tc_group_table_bytes(int nprob, int64_t ntiles);
// Writes the table into `host` (tc_group_table_bytes bytes; the caller copies it to the
// device, 256-byte aligned): tensor maps per problem, tiles longest first.
bool tc_group_build(int mode, const TcGroupSpec* specs, int nprob, void* host, int* nmma_max);
// Deepest pipeline for per_sm CTAs per SM.
int tc_group_max_stages(int mode, int prec, int nmma_max, int per_sm);
// One persistent launch over every tile of the table (prec 3 = 3xTF32, else TF32;
// norm: mode 0 with the fused sum of G^2).  A timed-out wait sets TIMEOUT in st_dev.
cudaError_t tc_group_launch(int mode, int prec, bool norm, const void* dev_table, int nprob, int64_t ntiles,
                            int nmma_max, int stages, int per_sm, DevStatus* st_dev, cudaStream_t st,
                            const void* dev_filtered = nullptr);
// Problems with stop words: tc_group_filter writes into dev_filtered (tc_group_filter_bytes)
// the tiles of the problems whose stop word is zero, in table order, and their count; a
// launch given dev_filtered runs those tiles only (every role walks the same list).
size_t tc_group_filter_bytes(int64_t ntiles);
cudaError_t tc_group_filter(const void* dev_table, int nprob, int64_t ntiles, void* dev_filtered, cudaStream_t st);

}  // namespace gsvdr
