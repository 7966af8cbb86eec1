// Internal launchers of the randomized-GSV library (host side, C++).
// Every launcher enqueues on `st` and returns the cudaError_t of the launch.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace gsvdr {

// ---- Gaussian test matrices (Algorithm 1 "Omega_i"; Theorem 3) -------------
// Raw Philox words, out[4t + w].
cudaError_t launch_philox_words(uint32_t* out, uint64_t count, uint64_t seed, uint32_t pair,
                                uint32_t side, uint32_t stream, cudaStream_t st);
// Omega (n x l) row-major FP64 (ld = l): the public definition.
cudaError_t launch_gaussian_rowmajor(double* out, int64_t n, int64_t l, uint64_t seed, uint32_t pair,
                                     uint32_t side, uint32_t stream, cudaStream_t st);
// Omega^T stored K-major for the sketch product: Xt[j * ldx + i] = Omega[i][j],
// j < lrows (rows l..lrows-1 are zero), i < n (columns n..ldx-1 are zero).
// Complex pairs: rho(Omega) of the complex n x l test matrix Omega[j][c] = g(2 (j l + c)) +
// i g(2 (j l + c) + 1) (g the real stream of an n x 2l matrix), written K-major like
// launch_gaussian_kmajor with n2 = 2n, l2 = 2l; and R = rho(G) (2M x 2n, row stride ldr) of a
// complex M x n matrix stored as interleaved (re, im) pairs with row stride ldg complex entries.
template <typename T>
cudaError_t launch_gaussian_kmajor_cplx(T* Xt, int64_t ldx, int64_t n2, int l2, int lrows, uint64_t seed,
                                        uint32_t pair, uint32_t side, uint32_t stream, cudaStream_t st);
template <typename T>
cudaError_t launch_realify(const T* G, int64_t ldg, int64_t M, int64_t n, T* R, int64_t ldr, cudaStream_t st);
cudaError_t launch_widen(const float* G, int64_t ldg, int64_t M, int64_t n, double* D, int64_t ldd, cudaStream_t st);
// dst (rows x n, row stride ldd) = src (rows x n, contiguous)
cudaError_t launch_repitch(const float* src, int64_t rows, int64_t n, float* dst, int64_t ldd, cudaStream_t st);
template <typename T>
cudaError_t launch_gaussian_kmajor(T* Xt, int64_t ldx, int64_t n, int l, int lrows, uint64_t seed,
                                   uint32_t pair, uint32_t side, uint32_t stream, cudaStream_t st);

// The same in BF16 (FP64 Gaussian -> nearest FP32 -> nearest BF16), ld a multiple of 8.
cudaError_t launch_gaussian_kmajor_bf16(void* Xt, int64_t ldx, int64_t n, int l, int lrows, uint64_t seed,
                                        uint32_t pair, uint32_t side, uint32_t stream, cudaStream_t st);
// Qt[j * ldq + i] = Y[i * ldy + j] for i < M, j < l.
template <typename T>
cudaError_t launch_transpose(const T* Y, int64_t ldy, int64_t M, int l, T* Qt, int64_t ldq, cudaStream_t st);
// BF16 halves of an FP32 matrix (rows x cols, ld lds): hi = bf16(x), lo = bf16(x - hi)
// (lo may be nullptr), ld ldd.  Columns cols.. of the destination are not written.
cudaError_t launch_split_bf16(const float* src, int64_t lds, int64_t rows, int64_t cols, void* hi, void* lo,
                              int64_t ldd, cudaStream_t st);

// ---- sketch / power products on CUDA cores (Algorithm 1 line "G Omega") ----
// Y (M x l, ld ldy) = G (M x n) * X where X is given K-major as Xt (l x n, ld ldx).
// If gnorm_part != nullptr, CTA b of column-tile 0 writes sum of G^2 over its
// rows to gnorm_part[b] (FP64; double-float accumulation for float data).
template <typename T>
cudaError_t launch_gemm_gx_simt(const T* G, int64_t ldg, int64_t M, int64_t n, const T* Xt,
                                int64_t ldx, int l, T* Y, int64_t ldy, double* gnorm_part,
                                cudaStream_t st);
int gemm_gx_simt_ctas(int64_t M);

// Split-K partials of G^T Q: part[z][c][j] (z < splits, c < n, j < l, ld lp)
// over the rows of split z.  Returns the number of splits used via *splits.
template <typename T, typename TP>
cudaError_t launch_gemm_gtq_simt(const T* G, int64_t ldg, int64_t M, int64_t n, const T* Q,
                                 int64_t ldq, int l, TP* part, int64_t lp, int splits,
                                 cudaStream_t st);
int gemm_gtq_splits(int64_t M, int64_t n, int l, int64_t max_part_elems);

// Sum the split partials in split order (deterministic), in FP64, into
//   transpose_out == 0: Z[c * ldz + j]   (n x l)
//   transpose_out == 1: Z[j * ldz + c]   (l x n, the projection B = Q^T G)
// If sq_part != nullptr, block b writes its sum of squares of the outputs.
template <typename TP, typename T>
cudaError_t launch_reduce_splits(const TP* part, int splits, int64_t n, int l, int64_t lp, T* Z,
                                 int64_t ldz, int transpose_out, double* sq_part, int* sq_blocks,
                                 cudaStream_t st);

// ---- CholeskyQR2 with shift (orthonormalisation of the sketch) -------------
// Gram partials of Y (M x l): part[c][i][j] over row chunk c (FP64 output).
template <typename T>
cudaError_t launch_gram_partial(const T* Y, int64_t ldy, int64_t M, int l, double* part, int chunks,
                                int64_t rows_per_chunk, cudaStream_t st);
int gram_chunks(int64_t M, int l, int64_t* rows_per_chunk);
// W = sum_c part[c] (FP64, chunk order).
cudaError_t launch_gram_reduce(const double* part, int chunks, int l, double* W, cudaStream_t st);

// Cholesky of W + s I (s = shift_coef * trace(W), 0 for no shift), one CTA,
// and the explicit inverse of the factor: Rinv (l x l, row-major, upper
// triangular, TC).  A pivot d_k <= tau_rel * (W + sI)_kk is numerically
// dependent: its column is dropped (column k of Rinv is zero, so column k of
// Q = Y Rinv is zero).  All columns dropped -> BREAKDOWN; non-finite -> NONFINITE.
// scratch: chol_scratch_elems(l) TC values (used when shared memory is too small).
int64_t chol_scratch_elems(int l);
// ldt > 0 (l > 64 only): the inverse factor transposed, Rinv[j * ldt + c] = R^{-1}[c][j] (the K-major
// operand of a tensor-core Q = Y R^{-1})
template <typename TC>
cudaError_t launch_chol_shift(const double* W, int l, double shift_coef, double tau_rel, TC* Rinv,
                              TC* scratch, DevStatus* st_dev, int stage, cudaStream_t st, int ldt = 0);
// The same factorisation of two Grams of equal width at once (two CTAs: the two sides of a
// pair), each with its own shift, floor, destination, scratch and status stage; 64 < l <= 256.
struct CholPairArgs {
  const double* W[2];
  float* Rinv[2];
  float* scratch[2];
  double shift_coef[2], tau_rel[2];
  int stage[2];
};
cudaError_t launch_chol_shift_pair(const CholPairArgs& a, int l, DevStatus* st_dev, cudaStream_t st, int ldt);

// Q = Y Rinv (upper triangular) per tile of rows, optional Gram partials of Q
// per CTA (part != nullptr, one chunk per CTA), optional transposed output
// Qt[j * ldq + row].
template <typename T, typename TC>
cudaError_t launch_apply_rinv(const T* Y, int64_t ldy, int64_t M, int l, const TC* Rinv, T* Q, int64_t ldq,
                              int transpose_out, double* part, cudaStream_t st);
int apply_ctas(int64_t M, int l, int elem_bytes);
// Whether the CholeskyQR passes take the Gram of Q from Q = Y R^{-1} (partials per row tile).
bool apply_fuses_gram(int l);
int64_t apply_rows_per_cta(int l, int elem_bytes);

// ---- small FP64 dense kernels (compressed-pair GSVD) -----------------------
// C (Mr x Nc) = op(A) * op(B) in FP64 accumulation; op(X) = X or X^T.
// df: double-float arithmetic (each operand as an FP32 hi + lo pair, error-free products and
// TwoSum accumulation, about 2^-48 relative) in place of FP64 FMAs: several times faster on GB300,
// for the mixed-precision paths; operands must lie inside FP32's exponent range (launch_pow2_scale).
// A: if !ta, Mr x K with lda; else K x Mr.  B: if !tb, K x Nc with ldb; else Nc x K.
// Split-K partials go to `work` (splits * Mr * Nc doubles) then a reduce writes
// C = alpha * sum + beta * C.  Returns cudaErrorInvalidValue if work too small.
template <typename TA, typename TB>
cudaError_t launch_dgemm_small(int Mr, int Nc, int K, const TA* A, int64_t lda, int ta, const TB* B,
                               int64_t ldb, int tb, double* C, int64_t ldc, double alpha, double beta,
                               double* work, int64_t work_elems, cudaStream_t st, bool df = false);

// One-CTA cyclic Jacobi eigensolver in FP32 (parallel round-robin order) on the
// symmetric N x N FP64 matrix A (scaled internally).  Writes the eigenvector
// matrix V (N x N, FP64, columns) and eigenvalues lam (FP64, unsorted).
// scratch: 2*N*N floats + N*N... (see jacobi_scratch_floats).
int64_t jacobi_scratch_floats(int N);
cudaError_t launch_jacobi_f32(const double* A, int N, double* V, double* lam, float* scratch,
                              int max_sweeps, DevStatus* st_dev, cudaStream_t st);

// All eigenpairs of the symmetric N x N FP64 matrix A in FP32, one CTA
// (tridiagonalisation, bisection, twisted factorisation, back-transformation,
// two-pass MGS with cluster replacement): X (N x N, FP64, orthonormal columns),
// lam (N, ascending).  scratch: eig_scratch_floats(N) floats.
int64_t eig_scratch_floats(int N);
// noise_rel > 0 (N <= 128): eigenvectors of eigenvalues with |lambda| <= noise_rel ||A||, which FP32
// cannot resolve, are replaced by an orthonormal basis of the complement of the others.
cudaError_t launch_eig_f32(const double* A, int N, double* X, double* lam, float* scratch, cudaStream_t st,
                           double noise_rel = 0.0);

// One Ogita-Aishima refinement step of the eigenvectors X (N x N) of the
// symmetric A, in FP64: R = I - X^T X, S = X^T A X, lam_i = s_ii/(1 - r_ii),
// F_ij = (s_ij + lam_j r_ij)/(lam_j - lam_i) (|lam_i - lam_j| > delta) or r_ij/2,
// X <- X + X F.  work: 4*N*N + splitK scratch doubles.
cudaError_t launch_oa_refine(const double* A, int N, double* X, double* lam, double* work,
                             int64_t work_elems, cudaStream_t st, bool df = false);

// Gather the r leading eigenvectors (by lam, descending; NaN last) of X (N x N)
// into Zr (N x r); order receives the permutation.
// CholeskyQR2 of M x l (l <= 64) as one cooperative persistent kernel (k_cholqr.cu).
// plan: the CTA count (0 when the shape does not fit: then use the separate
// kernels) and the rows per CTA.  part needs ctas * l * l doubles; bar is
// cholqr2_fused_bar_bytes() of device memory, zeroed once before first use.
size_t cholqr2_fused_bar_bytes();
int cholqr2_fused_max_ctas();
template <typename T, typename TC>
int cholqr2_fused_plan(int64_t M, int l, int64_t* rows_per);
template <typename T, typename TC>
cudaError_t launch_cholqr2_fused(const T* Y, int64_t ldy, int64_t M, int l, int ctas, int64_t rows_per, T* Q,
                                 int64_t ldq, int transpose_out, double* part, double* W, void* bar,
                                 double shift_coef, double tau_rel, DevStatus* st_dev, int stage, cudaStream_t st);

// Up to two problems (the two sides of a pair) in one cooperative launch: the CTAs of
// problem i follow those of problem i - 1; each problem has its own barrier word, partials
// and W.  The total CTA count must not exceed cholqr2_fused_max_total_ctas().
struct FqProb {
  const void* Y;
  int64_t ldy, M, rows_per;
  void* Q;
  int64_t ldq;
  double* part;
  double* W;
  void* bar;
  double shift_coef, tau_rel;
  int l, ctas, transpose_out, stage;
};
struct FqBatch {
  FqProb p[2];
  int nprob, pad;
};
template <typename T, typename TC>
cudaError_t launch_cholqr2_fused_n(const FqBatch& b, DevStatus* st_dev, cudaStream_t st);
template <typename T, typename TC>
int cholqr2_fused_max_total_ctas();

// The cluster of eigenvalues (within the last refinement step's delta) that
// straddles the cut between the r-th and (r+1)-th largest: its block of
// X^T A X is diagonalised (FP32 Jacobi, shifted and scaled) and its columns of
// X rotated.  Uses the work buffer of the preceding launch_oa_refine call.
// jscr: FP32 scratch of eig_scratch_floats(N) floats for clusters of more than CUT_CMAX columns
// (solved by the packed-triangle eigensolver in a second launch), or null to clip clusters there.
cudaError_t launch_oa_cut_cluster(int N, int r, double* X, const double* lam, double* work, int64_t work_elems,
                                  float* jscr, cudaStream_t st);
// Cut clusters: up to CUT_CMAX columns by FP32 Jacobi inside the detection kernel, larger ones
// (up to CUT_BIG_NMAX) by the packed-triangle FP32 eigensolver, whose descriptor the detection
// kernel leaves in the P block of the refinement work: an EigB at double offset CUT_EIGB_OFF
// (N = 0 when there is nothing to solve) and the block's eigenvalues from CUT_LAM_OFF.
constexpr int CUT_CMAX = 128;
constexpr int CUT_BIG_NMAX = 512;
constexpr int CUT_EIGB_OFF = 260;
constexpr int CUT_LAM_OFF = 512;
// The second launch: pblock is the P block of one problem (max_N its N), or the batched table.
cudaError_t launch_eig_cut_big(const double* pblock, int max_N, cudaStream_t st);
cudaError_t launch_eig_cut_big_b(const struct OaB* tab, int nprob, int max_N, cudaStream_t st);
cudaError_t launch_select_topr(const double* X, const double* lam, int N, int r, double* Zr,
                               int* order, cudaStream_t st);

// Comparative quantities of Section 1.
cudaError_t launch_metrics(const double* alpha, const double* beta, int r, int N, int pad_mode,
                           double* theta, double* rho, double* P1, double* P2, double* D,
                           cudaStream_t st);

// GSV pairs from U1 = Z1 W (l1 x r) and U2 = Z2 W (l2 x r): alpha_i = ||U1[:, i]||,
// beta_i = ||U2[:, i]||, normalised to alpha^2 + beta^2 = 1, sorted (eq. (ab)).
cudaError_t launch_cs_norms(const double* U1, int l1, const double* U2, int l2, int r, double* alpha,
                            double* beta, cudaStream_t st);

// GSVD factors of a solve (the recovery after Algorithm 2, rank-revealing reading): from
// U1 = [Z1; Z2] W (2 l x r, FP64), the bases Q_s (M_s x l, Q_s(i, j) = Q_s[i rs_s + j cs_s],
// element type float or double as tsize) and the stack S = [B1; B2] (2 l x n, row stride ldn,
// same type): column c of U (V) is Q_1 Z1 w_i / ||Z1 w_i|| (Q_2 Z2 w_i / ||Z2 w_i||, zero for a
// zero norm) and row c of R is ||[Z1; Z2] w_i|| w_i^T [Z1; Z2]^T S, where i is the column of
// descending-alpha rank c (the order of launch_cs_norms).  scr: 4 r doubles of device scratch.
// U (M_1 x r, ldu), V (M_2 x r, ldv), R (r x n, ldr): FP64 device, any of them may be null.
cudaError_t launch_gsvd_factors(int tsize, const void* Q1, int64_t rs1, int64_t cs1, int64_t M1, const void* Q2,
                                int64_t rs2, int64_t cs2, int64_t M2, int l, int r, const double* U1,
                                const void* S, int64_t ldn, int64_t n, double* scr, double* U, int64_t ldu,
                                double* V, int64_t ldv, double* R, int64_t ldr, cudaStream_t st);

// Residual (cumulated form): resid[s] = sqrt(max(g2 - b2, 0) / g2).
cudaError_t launch_residual(const double* gpart, int ng, const double* bpart, int nb, double* out,
                            cudaStream_t st);

// ---- learned (k, q) proposal (k_mlp.cu) ----------------------------------------
// Features of one side from W1 = Y^T Y, W2 = Z^T Z (16 x 16 FP64, full) and the
// sketch's partial sums of G^2 (gcount entries): 32 floats.
// The probe features of many sides in one launch (a CTA of 64 threads each).
struct ProbeFeatB {
  const double *W, *gpart;
  float* feats;
  int gcount, pad;
};
cudaError_t launch_probe_features_b(const ProbeFeatB* tab, int nprob, cudaStream_t st);
cudaError_t launch_probe_features(const double* W, const double* gpart, int gcount, float* feats, cudaStream_t st);
int64_t mlp_param_count();
int64_t mlp_scratch_floats(int B);
// Logits (B x 37) of X (B x 64); bf16: weight matrices rounded to BF16.
cudaError_t mlp_forward(const float* P, const float* norm, const float* X, int B, int bf16, float* logits,
                        float* scratch, cudaStream_t st);
// Mean loss (one float) and its gradient (mlp_param_count() floats) over rows
// `rows` (B indices, or nullptr for 0..B-1) of X, yk, yq.
cudaError_t mlp_loss_grad(const float* P, const float* norm, const float* X, const int* yk, const int* yq,
                          const int* rows, int B, float* grad, float* loss, float* scratch, cudaStream_t st);
cudaError_t mlp_adam(float* P, float* m, float* v, const float* grad, int t, float lr, float b1, float b2, float eps,
                     cudaStream_t st);
// The (k, q) plan of B rows of logits on the device: plan[3 i] = k (the top of the smallest k
// bucket whose cumulative softmax probability reaches quantile, clipped to kcap[i] and to
// lmax[i] - os[i]; any of the three arrays may be null), plan[3 i + 1] = q (argmax),
// plan[3 i + 2] = the k bucket.
cudaError_t launch_mlp_plan(const float* logits, int B, float quantile, const int* kcap, const int* lmax,
                            const int* os, int* plan, cudaStream_t st);

// ---- batched forms: one launch for many problems ------------------------------
// Each launcher takes a table of per-problem arguments in device memory (nprob
// entries) and the largest extent over the problems, which sizes the grid.
struct GaussB {  // Omega^T of one side, K-major FP32 (as launch_gaussian_kmajor)
  float* Xt;
  int64_t ldx, n;
  int l, lrows;
  uint64_t seed;
  uint32_t pair, side, stream, pad;
  float* lo;  // null, or Xt - tf32(Xt) in the same layout (the low half of a 3xTF32 B operand)
};
cudaError_t launch_gaussian_kmajor_b(const GaussB* tab, int nprob, int64_t max_ldx, int max_lrows, cudaStream_t st);

struct ReduceB {  // as launch_reduce_splits<float, float>; sq_part gets cdiv(n l, 256) sums
  const float* part;
  int splits, l;
  int64_t n, lp;
  float* Z;
  int64_t ldz;
  int transpose_out, pad;
  double* sq_part;
};
cudaError_t launch_reduce_splits_b(const ReduceB* tab, int nprob, int64_t max_nl, cudaStream_t st);

struct GramB {  // Gram partials of Y (M x l, FP32, l <= 128) over `chunks` chunks of rpc rows
  const float* Y;
  int64_t ldy, M, rpc;
  int l, chunks;
  double* part;
  const int* stop;  // null, or a stop word: the entry is skipped once it is non-zero
};
struct GramRedB {  // W = sum of the chunk partials
  const double* part;
  int chunks, l;
  double* W;
  const int* stop;
};
// The whole upper triangle of a chunk's Y^T Y in one CTA (register blocks, FP32 FMA over
// the chunk's rows), then the chunk sums in FP64 a thread per entry (both deterministic).
cudaError_t launch_gram_blocks_b(const GramB* tab, int nprob, int max_chunks, int max_l, cudaStream_t st);
cudaError_t launch_gram_sum_b(const GramRedB* tab, int nprob, int max_l, cudaStream_t st);

struct CholB {  // shifted Cholesky with the inverse factor (FP32 factor), as launch_chol_shift
  const double* W;
  double shift_coef, tau_rel;
  float* Rinv;   // ldt == 0: R^{-1} row-major (l x l); ldt > 0: its transpose, Rinv[j * ldt + c] = R^{-1}[c][j]
  DevStatus* st;
  int l, stage, ldt, pad;
  const int* stop;  // null, or a stop word: the entry is skipped once it is non-zero
};
// dst = src - tf32(src) over rows x cols (row strides lds, ldd), one entry per problem.
struct LoHalfB {
  const float* src;
  float* dst;
  int64_t rows, cols, ld;
  const int* stop;
};
cudaError_t launch_low_half_b(const LoHalfB* tab, int nprob, int64_t max_elems, cudaStream_t st);

// max_l <= 64: the register-resident elimination; <= 128: the shared-memory one.
cudaError_t launch_chol_b(const CholB* tab, int nprob, int max_l, cudaStream_t st);


// ---- grouped Algorithm 1 (k_adapt.cu) -------------------------------------------------
// Blocks of b <= ADAPT_BMAX columns, bases of at most ADAPT_CMAX columns per side.  Every
// table entry carries the side's stop word (0 while it adds blocks, then its column count):
// entries of stopped sides return at once.
constexpr int ADAPT_BMAX = 32;
constexpr int ADAPT_CMAX = 128;
struct AdaptB {  // Y (M x bi, ld ldy) <- Y - Q (Q^T Y), Q the first c rows of Qt (K-major, ld ldq)
  const float* Qt;
  int64_t ldq, M;
  float* Y;
  int64_t ldy;
  int c, bi;
  double* C;      // c x bi: Q^T Y (FP64 sums of FP32 chunk products)
  double* xpart;  // adapt_xpart_elems(M, c, bi) chunk partials
  const int* stop;
};
int64_t adapt_xpart_elems(int64_t M, int c, int bi);
// The projection of every entry (max_bi <= ADAPT_BMAX, max_c <= ADAPT_CMAX): three launches.
cudaError_t launch_adapt_project_b(const AdaptB* tab, int nprob, int64_t max_M, int max_c, int max_bi,
                                   cudaStream_t st);
struct AdaptEnergyB {  // ||P^T G||_F^2 of the block P = rows [c, c + bi) of Qt, on the CUDA cores
  const float* G;
  int64_t ldg, M, n;
  const float* Qt;
  int64_t ldq;
  int c, bi;
  float* part;    // adapt_energy_part_elems(M, n, bi) chunk partials
  double* epart;  // cdiv(n bi, 256) partial sums of squares (then zeros up to nb_out)
  const int* stop;
  int nb_out;     // slots of epart to fill (0: cdiv(n bi, 256))
};
int64_t adapt_energy_part_elems(int64_t M, int64_t n, int bi);
cudaError_t launch_adapt_energy_b(const AdaptEnergyB* tab, int nprob, int64_t max_M, int64_t max_n, int max_bi,
                                  cudaStream_t st);
struct AdaptStopB {  // the stop test of a side after one block
  const double* gpart;  // first block: the ng partial sums of ||G||_F^2
  const double* bpart;  // this block: the nb partial sums of ||P_i^T G||_F^2
  double* state;        // ||G||^2, running sum, estimate
  int* stop;
  double tol;
  int ng, nb, cols, first, last;  // cols: columns after this block; last: the cap is reached
  double* resid_out;              // the pair's residual slot of this side (the estimate)
  DevStatus* st;                  // TOL_MISS when the cap is reached above tol
};
cudaError_t launch_adapt_stop_b(const AdaptStopB* tab, int nprob, cudaStream_t st);
struct AdaptMaskB {  // rows [*stop, cap) of Qt (ld ldq) set to zero
  float* Qt;
  int64_t ldq;
  int cap, pad;
  const int* stop;
};
cudaError_t launch_adapt_mask_b(const AdaptMaskB* tab, int nprob, int64_t max_elems, cudaStream_t st);
// A pair of a grouped adaptive solve holds r_act = min(r, stop1 + stop2) pairs; the compressed-pair
// GSVD runs with the static r.  mode 0: columns [r_act, r) of Zr (L x r) to zero after the top-r
// selection; mode 1: C1[j][j] = -1 for j >= r_act after C1 = Z1^T Z1, so that those columns stay
// apart from every real eigenvector and end as pairs of zero norm (cs_norms marks them -1, last).
struct AdaptTrimB {
  double* Zr;
  double* C1;
  int L, r;
  const int* stop1;
  const int* stop2;
};
cudaError_t launch_adapt_trim_b(const AdaptTrimB* tab, int nprob, int max_L, int max_r, int mode, cudaStream_t st);

struct ResidB {  // cumulated residual of one side
  const double* gpart;
  const double* bpart;
  double* out;
  int ng, nb;
};
cudaError_t launch_residual_b(const ResidB* tab, int nprob, cudaStream_t st);

// C = alpha op(A) op(B) + beta C in FP64 accumulation (A and B FP32 or FP64), one
// 32 x 32 tile of C per CTA (no split-K: the batch fills the GPU).  C must not alias
// A or B.
struct DgemmB {
  const void* A;
  const void* B;
  double* C;
  int64_t lda, ldb, ldc;
  double alpha, beta;
  int Mr, Nc, K, ta, tb;
  int sym;  // the result is symmetric (Mr == Nc): upper tiles computed and mirrored
};
// df: 0 FP64, 1 double-float, 2 FP32 products of the high parts (the refinement's increment)
template <typename TA, typename TB>
cudaError_t launch_dgemm_b(const DgemmB* tab, int nprob, int max_Mr, int max_Nc, cudaStream_t st, int df = 0);

// One Ogita-Aishima step per problem (as launch_oa_refine), and the cut cluster after it.
struct OaB {
  const double* A;
  double* X;
  double* lam;
  double* XtX;  // N x N work matrices
  double* P;
  double* S;
  double* F;
  double* part;  // 3 sums
  int N, r;
  float* jscr;   // FP32 eigensolver scratch for a large cut cluster (eig_scratch_floats(N)), or null
  // double-float refinement (launch_oa_refine_b with df): N x N (hi, lo) copies of A, X, P and F
  // that the products read; null for the FP64 form
  float2 *Adf = nullptr, *Xdf = nullptr, *Pdf = nullptr, *Fdf = nullptr;
};
// The four products of a step use `dg` (4 * nprob DgemmB entries, filled by oa_b_tables).
void oa_b_tables(const OaB* hostOa, int nprob, DgemmB* dg);
cudaError_t launch_oa_refine_b(const OaB* tab, const DgemmB* dg, int nprob, int max_N, cudaStream_t st,
                               bool df = false);
cudaError_t launch_oa_cut_cluster_b(const OaB* tab, int nprob, int max_N, cudaStream_t st);

struct SelB {
  const double* X;
  const double* lam;
  double* Zr;
  int* order;
  int N, r;
};
cudaError_t launch_select_topr_b(const SelB* tab, int nprob, int max_N, cudaStream_t st);

struct CsB {
  const double* U1;
  const double* U2;
  double* alpha;
  double* beta;
  int l1, l2, r, pad;
};
cudaError_t launch_cs_norms_b(const CsB* tab, int nprob, int max_r, cudaStream_t st);

struct ScatterB {  // dst[0..count) = src[0..count)
  const double* src;
  double* dst;
  int count, pad;
};
cudaError_t launch_scatter_b(const ScatterB* tab, int n, cudaStream_t st);

// A (N x N) times the power of two that puts its largest |diagonal entry| in [1, 2) (exact).
cudaError_t launch_pow2_scale(double* A, int N, cudaStream_t st);
struct EigB;
cudaError_t launch_pow2_scale_b(const EigB* tab, int nprob, cudaStream_t st);  // each entry's A and N
struct EigB {
  const double* A;
  double* X;
  double* lam;
  float* scratch;
  float noise_rel;
  int N;
};
// All problems of the table have N <= 128 (eig128) or 128 < N <= 318 (the packed-triangle
// solver with the triangle in shared memory).
cudaError_t launch_eig_f32_b(const EigB* tab, int nprob, int max_N, cudaStream_t st);

}  // namespace gsvdr
