/*
 * gsvd_rand.h — C ABI of the GB300 randomized generalized-singular-value library.
 *
 * Method: Xu, Shen, Li, Gao, Li, "Randomized algorithms for GSVs" (arXiv:2404.09459).
 * For a matrix pair {G1 (m x n), G2 (p x n)} (Section 1, eq. (gsvd1):
 * G1 = U Sigma1 R, G2 = V Sigma2 R, alpha_i^2 + beta_i^2 = 1) the library
 *   1. extracts orthonormal bases Q1, Q2 of the column spaces of G1, G2 with a
 *      Gaussian sketch Y = G Omega (Theorem 3: Omega has k + p columns) and q
 *      power (subspace) iterations, re-orthonormalising with shifted CholeskyQR2;
 *   2. projects B_s = Q_s^T G_s (Algorithm 2, the compressed pair);
 *   3. computes the GSVs of the compressed pair (Algorithm 2; the reduced QR of
 *      the stack is taken rank-revealing, truncated to k pairs) in FP64;
 *   4. evaluates the comparative quantities of Section 1 (angular distance,
 *      relative significance, generalized fractions, generalized entropy).
 * Every step runs in this library's own CUDA kernels (sm_103a).
 *
 * Conventions shared by all entry points
 *   - Matrices are row-major with a leading dimension in ELEMENTS (ld >= cols).
 *   - Pointers may be device pointers or host pointers; the library detects
 *     which with cudaPointerGetAttributes.  Host inputs are copied to device
 *     workspace inside the call; host outputs are written after a stream sync.
 *   - Inputs are read-only and owned by the caller.  Outputs are caller-owned.
 *   - The library owns its device workspace, allocated on first use and grown
 *     on demand (cudaMalloc); it is freed by gsvd_rand_destroy.
 *   - Work is enqueued on cfg->stream.  gsvd_rand_solve and gsvd_rand_metrics
 *     synchronise that stream before returning so that they can report a
 *     status (breakdown, non-finite input) read back from the device.
 *   - Return value: GSVD_RAND_OK (0) or a negative GSVD_RAND_ERR_* code;
 *     gsvd_rand_last_error() gives a one-line message.  Nothing traps the GPU:
 *     device-side problems are reported through status words.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef GSVD_RAND_H
#define GSVD_RAND_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GSVD_RAND_OK 0
#define GSVD_RAND_ERR_ARG (-1)         /* bad shape, pointer, or parameter */
#define GSVD_RAND_ERR_OOM (-2)         /* device allocation failed */
#define GSVD_RAND_ERR_CUDA (-3)        /* a CUDA runtime call failed */
#define GSVD_RAND_ERR_NONFINITE (-4)   /* NaN/Inf in the input or an intermediate */
#define GSVD_RAND_ERR_BREAKDOWN (-5)   /* Cholesky failed even after the shift (e.g. G = 0) */
#define GSVD_RAND_ERR_TOL_MISS (-6)    /* adaptive basis reached its column cap above tol */
#define GSVD_RAND_ERR_TIMEOUT (-7)     /* a bounded device-side wait ran out */
#define GSVD_RAND_ERR_UNSUPPORTED (-8) /* option not built / not available on this device */
#define GSVD_RAND_ERR_TOO_LARGE (-9)   /* size above the fixed limit of gsvd_rand_metrics_noalloc */

/* Arithmetic of the sketch, power and projection products.
 *   FP64   : G is double; all products in FP64 (the plain path).
 *   TF32   : G is float; products on tensor cores with TF32 inputs and FP32
 *            accumulation; CholeskyQR2 in FP32 data with an FP64-reduced Gram;
 *            small GSVD in FP64.
 *   TF32X3 : as TF32, with each operand split hi + lo and three tensor products
 *            (hi*hi + hi*lo + lo*hi), about FP32 accuracy.
 *   BF16   : G is bfloat16; products on tensor cores (kind::f16) with FP32
 *            accumulation.  G is read in place when its base is 16-byte aligned and
 *            its row stride a multiple of 8 elements, else copied into the workspace.  Omega is
 *            the FP64 Gaussian rounded to the nearest FP32 and then to the nearest
 *            BF16, so the sketch G Omega is exact up to FP32 accumulation.  The power
 *            steps round their FP32 operand (Q, then Z) to BF16, or split it into
 *            BF16 hi + lo halves (two products) under GSVD_RAND_FLAG_BF16_SPLIT_POWER;
 *            the projection Q^T G always takes Q as hi + lo.  CholeskyQR2 and the
 *            small GSVD as in TF32.  Adaptive mode is not available in BF16.
 *   FP32   : G is float; products with FP32 CUDA-core FMAs (no tensor cores).  */
typedef enum {
  GSVD_RAND_FP64 = 0,
  GSVD_RAND_TF32 = 1,
  GSVD_RAND_BF16 = 2,
  GSVD_RAND_TF32X3 = 3,
  GSVD_RAND_FP32 = 4
} gsvd_rand_prec;

/* Philox stream ids (fourth counter word) of the Gaussian test matrices. */
#define GSVD_RAND_STREAM_FIXED 0u          /* the n x (k+p) Omega of the fixed-rank solve */
#define GSVD_RAND_STREAM_ADAPTIVE 0x10000u /* + block index i: Omega_i of Algorithm 1 */
#define GSVD_RAND_STREAM_PROBE 0x20000u    /* the 64-column probe sketch */

typedef struct gsvd_rand_ctx *gsvd_rand_t;

typedef struct {
  int device;        /* CUDA device ordinal the context is bound to */
  void *stream;      /* cudaStream_t to enqueue on; NULL = the legacy default stream */
  int prec;          /* gsvd_rand_prec */
  int adaptive;      /* 0: fixed rank k + oversample (Theorem 3) with q power steps;
                        1: bases by Algorithm 1 (blocks of block_b columns until the cumulated
                        relative residual is <= tol, at most min(M, n, 256) columns per side) */
  int block_b;       /* Algorithm 1 block size b (paper: 100), 1..256 (FP64: ..224) */
  double tol;        /* Algorithm 1 relative residual tolerance.  The cumulated residual of
                        Section 2 cancels below about sqrt(u) of ||G||_F (u of the basis'
                        orthonormality): tolerances below ~1e-7 (FP64) or ~1e-3 (FP32 data)
                        may not be certified and end in GSVD_RAND_ERR_TOL_MISS */
  int use_learned;   /* 1: k and q of the fixed-rank solve from the learned proposal (probe
                        features -> network), with Algorithm 1 (block_b, tol) as the fallback
                        when the proposed bases miss tol; k of gsvd_rand_solve is then the
                        output capacity and the cap on the proposed k */
  const char *mlp_path; /* network file for use_learned (see gsvd_rand_mlp_load), or NULL
                           to set the network later with gsvd_rand_mlp_set */
  int flags;         /* GSVD_RAND_FLAG_* */
} gsvd_rand_config;

/* flags */
#define GSVD_RAND_FLAG_CHOL_FP64 1 /* mixed precisions: run the CholeskyQR factorisations in FP64
                                      (without it, a solve whose FP32 factors break down is repeated
                                      in this form: gsvd_rand_chol64_retries) */
#define GSVD_RAND_FLAG_PROFILE 2   /* time each stage with CUDA events on the solve stream */
#define GSVD_RAND_FLAG_BF16_SPLIT_POWER 4 /* BF16: power-step operands as hi + lo (two products) */
#define GSVD_RAND_FLAG_BASIS_ONLY 8 /* bases and residuals only: no compressed-pair GSVD, alpha and
                                       beta may be NULL and are not written, *r_out = 0 */
#define GSVD_RAND_FLAG_ACC_RESID 16 /* grouped fixed-rank solves: the residual's ||Q^T G||_F^2 summed
                                       on the CUDA cores (one more pass over G) instead of taken from
                                       the tensor-core projection, whose long accumulation chains
                                       lose ~1e-4 of it (an estimate floor near 1e-2) */

/* Stages timed under GSVD_RAND_FLAG_PROFILE. */
#define GSVD_RAND_STAGE_SKETCH 0 /* Y = G X products (sketch and power steps) */
#define GSVD_RAND_STAGE_GTQ 1    /* Z = G^T Q products incl. the projection B = Q^T G */
#define GSVD_RAND_STAGE_ORTH 2   /* shifted CholeskyQR2 (Gram, Cholesky, triangular apply) */
#define GSVD_RAND_STAGE_SMALL 3  /* compressed-pair GSVD (FP64), all of it */
#define GSVD_RAND_STAGE_SMALL_GRAM 4   /* ... of which K = S S^T */
#define GSVD_RAND_STAGE_SMALL_JACOBI 5 /* ... the FP32 Jacobi eigensolve of K */
#define GSVD_RAND_STAGE_SMALL_REFINE 6 /* ... the FP64 eigenvector refinement of K */
#define GSVD_RAND_STAGE_SMALL_CS 7     /* ... the CS step (C1, C2 and their eigensolve) */
#define GSVD_RAND_STAGE_SETUP 8        /* grouped solves: status resets and the Gaussian test matrices */
#define GSVD_RAND_STAGE_PROPOSAL 9     /* learned grouped solves: the probes, the network and the plans */
#define GSVD_RAND_NUM_STAGES 10

/* Fill *cfg with defaults: device 0, default stream, TF32, fixed rank, b = 100, tol = 1e-4. */
int gsvd_rand_config_init(gsvd_rand_config *cfg);

/* Create a context on cfg->device.  *out receives the handle.
 * Errors: ARG (NULL pointers, bad prec), CUDA (device cannot be set). */
int gsvd_rand_create(gsvd_rand_t *out, const gsvd_rand_config *cfg);

/* Release the context and its workspace.  NULL is accepted. */
int gsvd_rand_destroy(gsvd_rand_t h);

/* Message of the last failing call on this context ("" if none). Owned by the context. */
const char *gsvd_rand_last_error(gsvd_rand_t h);

/* Randomized GSVs of {G1, G2} (Algorithm 2 with the fixed-rank basis of
 * Theorem 3 and q power iterations).
 *   G1, ld1 : m x n matrix, element type double (FP64) or float (other precs)
 *   G2, ld2 : p x n matrix, same element type
 *   k       : number of GSV pairs returned, 1 <= k
 *   oversample : extra sketch columns (the paper's p); l = k + oversample must
 *             satisfy l <= min(m, p, n) and l <= 256
 *   q       : power iterations, 0 <= q <= 16
 *   seed    : Philox key; side s in {0, 1} uses counter words (t, 0, s, 0)
 *   alpha   : k doubles, non-increasing (eq. (ab)); beta: k doubles, non-decreasing
 *   r_out   : may be NULL; receives k
 *   resid_out : may be NULL; receives 2 doubles, the relative residual
 *             ||(I - Q_s Q_s^T) G_s||_F / ||G_s||_F of each side in the
 *             cumulated form sqrt(||G_s||_F^2 - ||Q_s^T G_s||_F^2) (Section 2)
 * With cfg->adaptive = 1 the bases come from Algorithm 1 instead (Omega_i from
 * counter words (t, 0, s, 0x10000 + i)); oversample and q are not used, k is the
 * capacity of alpha/beta and min(k, l1 + l2) pairs are returned (*r_out), and
 * resid_out receives the final cumulated estimates.  When a side reaches its
 * column cap above tol the results are still written and TOL_MISS is returned.
 * Errors: ARG, OOM, CUDA, NONFINITE, BREAKDOWN, TOL_MISS (adaptive).
 * Synchronises cfg->stream. */
int gsvd_rand_solve(gsvd_rand_t h, const void *G1, int64_t m, int64_t ld1, const void *G2,
                    int64_t p, int64_t ld2, int64_t n, int k, int oversample, int q,
                    uint64_t seed, double *alpha, double *beta, int *r_out, double *resid_out);

/* Randomized GSVs of a complex pair.  Section 1 states the GSVD over C (eq. (gsvd1):
 * G1 = U Sigma1 R, G2 = V Sigma2 R with unitary U, V) and the synthetic experiments of
 * Section 4.1 are complex; the method is Algorithm 2 with the fixed-rank bases as in
 * gsvd_rand_solve, with conjugate transposes and a complex Gaussian test matrix
 *     Omega[j][c] = g(2 (j l + c)) + i g(2 (j l + c) + 1),  l = k + oversample,
 * g the real stream of gsvd_rand_gaussian for an n x 2l matrix (the real and imaginary parts
 * are the two normals of one Box-Muller pair), per side s counter words (t, 0, s, 0).
 *   G1, G2 : complex m x n and p x n, row-major, each entry an interleaved (re, im) pair:
 *            complex128 (two doubles) for FP64, complex64 (two floats) for TF32, TF32X3 and
 *            FP32; ld1, ld2 >= n in complex entries; device or host (read only).
 *   alpha, beta, r_out, resid_out : as gsvd_rand_solve (the GSVs of a complex pair are real).
 * The library solves the realified pair: each entry a + ib becomes the real 2 x 2 block
 * [[a, -b], [b, a]], a map that carries products and conjugate transposes over, so the real
 * method on the realified pair with the realified Omega (and k, oversample doubled) runs the
 * complex method's arithmetic and returns each complex GSV twice; one of each two is returned.
 * The realified matrices (4 m n and 4 p n reals) live in device memory owned by h, grown on
 * demand and freed by gsvd_rand_destroy.  k + oversample <= min(m, p, n) and <= 112 (FP64) or
 * 128 (the others).  gsvd_rand_factors is not available after a complex solve.
 * Errors: ARG, OOM, CUDA, UNSUPPORTED (BF16, adaptive, learned or basis-only contexts),
 * NONFINITE, BREAKDOWN.  Synchronises cfg->stream. */
int gsvd_rand_solve_complex(gsvd_rand_t h, const void *G1, int64_t m, int64_t ld1, const void *G2,
                            int64_t p, int64_t ld2, int64_t n, int k, int oversample, int q,
                            uint64_t seed, double *alpha, double *beta, int *r_out, double *resid_out);

/* One pair of a batched solve: the arguments of gsvd_rand_solve, the Philox counter word
 * 'pair' (side s of this pair uses counter words (t, pair, s, stream)), and the
 * per-pair return code written by gsvd_rand_solve_batched. */
typedef struct {
  const void *G1;
  int64_t m, ld1;
  const void *G2;
  int64_t p, ld2;
  int64_t n;
  int k, oversample, q;
  uint64_t seed;
  uint32_t pair;
  double *alpha, *beta; /* capacity k each */
  int *r_out;           /* may be NULL */
  double *resid_out;    /* may be NULL (2 doubles) */
  int status;           /* out: GSVD_RAND_OK or the pair's error code */
} gsvd_rand_pair;

/* Many independent pairs at once (the batched form of gsvd_rand_solve, with h's
 * configuration).  The pairs are spread over `workers` concurrent solves (<= 0: 8;
 * at most 64), each a sub-context of h with its own stream and workspace, kept
 * for later calls; while one pair runs its single-SM small GSVD, others use the
 * rest of the GPU.  Pairs are taken largest first.  Every pair's result and
 * status are written; returns GSVD_RAND_OK when all succeeded, else the status
 * of the first failing pair (by index).  Synchronises the worker streams (not
 * cfg->stream).  Errors: ARG, OOM, CUDA, and any per-pair error. */
int gsvd_rand_solve_batched(gsvd_rand_t h, int npairs, gsvd_rand_pair *pairs, int workers);

/* Many independent pairs solved as one group (fixed-rank solves, cfg->prec TF32 or
 * TF32X3): every step runs once for all pairs, so each launch holds the work of the
 * whole batch (Algorithms 1 and 2 of Section 2 per pair, as gsvd_rand_solve):
 *   - the products Y = G X, G^T Q and Q^T G of all sides are persistent grouped
 *     tcgen05 launches over one tile table (per-problem tensor maps, tiles longest
 *     first, tensor-memory accumulators); their pipeline depth and CTAs per SM are
 *     picked by a built-in autotuner (timed on the first batch of each size bucket;
 *     the choice does not change the results; the environment variable
 *     GSVD_RAND_GROUP_PIPELINE="stages,ctas_per_sm" pins it where that shape fits);
 *   - the shifted CholeskyQR3 passes, the split reductions, the residuals and the
 *     compressed-pair GSVDs run as batched kernels (one table entry per problem).
 * The whole launch sequence is captured into a CUDA graph and replayed while the
 * pairs' inputs (pointers, shapes, k, oversample, q, seed, pair word) stay the same;
 * the first call of a new batch builds the plan, uploads the tables, tunes and
 * captures (it costs several solves).  Results go to each pair's alpha / beta
 * (device or host; resid_out and r_out as in gsvd_rand_solve).  Per pair:
 * l = k + oversample <= min(m, p, n) and <= 128, q <= 16, G1 and G2 FP32: device matrices
 * with 16-byte aligned rows are read in place; host matrices (any ld >= n) are copied on
 * cfg->stream, every call, into device memory owned by h (rows padded to 16 bytes, kept
 * for later calls, freed by gsvd_rand_destroy) and solved from there; a fixed-rank group of at
 * least 16 pairs from host buffers then runs as chunks (two, or one per 64 pairs up to four),
 * each chunk's inputs copied while the chunk before it is solved (the results are those of one
 * group); pairs may differ in every size and in q.  A pair that breaks
 * these rules gets status ARG and is left out; the others are solved.  The grouped
 * path chunks its Gram sums differently from gsvd_rand_solve, so results agree with it
 * to rounding (not bit for bit); repeated calls are bit-identical.  The plan, tables
 * and graph live in device memory owned by h (freed by gsvd_rand_destroy).
 * With cfg->adaptive = 1 every side's basis comes from Algorithm 1 (BasisExt with the
 * cumulated-residual stop of Section 2) instead: blocks of b = cfg->block_b <= 32 Gaussian
 * columns (Omega_i from counter words (t, pair, s, 0x10000 + i), as gsvd_rand_solve), each
 * projected twice against the basis so far, orthonormalised, projected and orthonormalised
 * again, until sqrt(||G||_F^2 - sum_i ||P_i^T G||_F^2) <= tol ||G||_F or the basis has
 * min(m, p, n, 128) columns (then TOL_MISS, results still written).  Every block is one step
 * for the whole batch; the stop test runs on the device, where each side has a stop word that
 * makes the later blocks skip it (no host read between blocks).  oversample and q are not
 * used; each pair returns min(k, l1 + l2) pairs (*r_out; alpha / beta need min(k, 2 cap)
 * entries, those past *r_out are set to -1); gsvd_rand_grouped_basis_cols gives l1, l2.
 * With cfg->use_learned = 1 (and a network loaded) the learned proposal runs for the whole
 * group: the 64-column probe sketch of every pair on the device (no host read between pairs),
 * one network forward over the batch (BF16 weights) and every pair's (k, q) plan on the device
 * (as gsvd_rand_solve's learned form; k capped by the pair's k, which is the capacity of alpha
 * and beta), read back once; the pairs then run as one fixed-rank group with their own k and q,
 * the residual summed on the CUDA cores (the tensor-core products' estimate has a floor near
 * 1e-2), and the pairs whose residual misses tol on either side run again as one Algorithm 1
 * group (cfg->block_b <= 32).  gsvd_rand_grouped_plans gives each pair's (k, q, fallback).
 * A pair whose FP32 Cholesky factors overflow (NONFINITE) or vanish (BREAKDOWN), as they can
 * when the sketch's rank is well below l and the noise is under FP32 resolution, is solved again
 * on its own with FP64 Cholesky factors and its own Philox words (gsvd_rand_solve's form; counted
 * by gsvd_rand_chol64_retries); its status is that solve's.
 * Returns GSVD_RAND_OK when all pairs succeeded, else the status of the first
 * failing pair.  Ordered after and before cfg->stream; synchronises.
 * Errors: ARG, OOM, CUDA, UNSUPPORTED (precision, basis-only contexts, no sm_103 tensor
 * cores), and per-pair NONFINITE, BREAKDOWN, TIMEOUT, TOL_MISS (adaptive). */
int gsvd_rand_solve_grouped(gsvd_rand_t h, int npairs, gsvd_rand_pair *pairs);

/* The plans of the last learned grouped solve on h: plans[3 i] = k, plans[3 i + 1] = q,
 * plans[3 i + 2] = 1 when pair i fell back to Algorithm 1.  Errors: ARG (no learned grouped
 * solve of npairs pairs). */
int gsvd_rand_grouped_plans(gsvd_rand_t h, int *plans, int npairs);

/* The probe features of the last learned grouped solve on h: feats[64 i .. 64 i + 63] for pair i
 * (GSVD_RAND_MLP_IN per pair, as gsvd_rand_probe_features gives them for the pair's own Philox
 * word; zeros for pairs the probes left out), host memory.  The group's probes run as one grouped
 * pass whose Gram sums are chunked differently from a single probe's: the features agree with it
 * to rounding.  Errors: ARG (no learned grouped solve of npairs pairs). */
int gsvd_rand_grouped_features(gsvd_rand_t h, float *feats, int npairs);

/* The basis columns of each side of the last grouped solve on h with cfg->adaptive = 1
 * (Algorithm 1 in grouped form, see gsvd_rand_solve_grouped): cols[2 i + s] for pair i,
 * side s (0 for pairs left out); npairs entries of the last call's array.  Errors: ARG. */
int gsvd_rand_grouped_basis_cols(gsvd_rand_t h, int *cols, int npairs);

/* The last grouped plan of h: tuned[6] = (stages, CTAs per SM) of the first sketch,
 * the power-step sketch and the G^T Q / projection products; the graph captures and
 * replays so far and the kernel launches per replay.  Any pointer may be NULL. */
int gsvd_rand_grouped_info(gsvd_rand_t h, int *tuned, int64_t *captures, int64_t *replays, int64_t *launches);

/* The GSVD factors of the last fixed-rank gsvd_rand_solve on h (not basis-only), as the
 * recovery that follows Algorithm 2 in Section 2 gives them, in the rank-revealing reading:
 * with S = [Q1^T G1; Q2^T G2] = Zr Sigma Wr^T truncated to r = k and W the eigenvectors of
 * Z1^T Z1 (Z1, Z2 the two blocks of Zr),
 *     U = Q1 Z1 W diag(1 / ||Z1 w_i||)   (m x r),    V = Q2 Z2 W diag(1 / ||Z2 w_i||)   (p x r),
 *     R = diag(||Zr w_i||) W^T Zr^T S   (r x n),
 * so that G1 ~ U diag(alpha) R and G2 ~ V diag(beta) R with the solve's alpha, beta (column and
 * row i pair with alpha_i, beta_i; U and V have orthonormal columns where alpha, beta > 0; a
 * column whose alpha (beta) is zero is zero).  The product U diag(alpha) R does not depend on
 * the rotations of the bases.  U, V, R: device FP64 row-major with ldu, ldv >= r and ldr >= n;
 * any may be NULL.  The factors are taken from the solve's workspace: any later call on h that
 * uses it (a solve, gsvd_rand_metrics, ...) makes them unavailable.  Synchronises cfg->stream.
 * Errors: ARG (NULL handle, no such solve, host pointers, memory of another GPU or short leading
 * dimensions), CUDA. */
int gsvd_rand_factors(gsvd_rand_t h, double *U, int64_t ldu, double *V, int64_t ldv, double *R, int64_t ldr);

/* The pipeline shapes of the last gsvd_rand_solve on h whose products of both sides ran as
 * grouped tensor-core launches (fixed rank, TF32 / TF32X3, k + oversample <= 128):
 * shapes[6] = (stages, CTAs per SM) of the first sketch, the power-step sketch and the
 * G^T Q / projection products, as the built-in tuner picked them (zeros before such a
 * solve).  Errors: ARG (NULL handle or shapes). */
int gsvd_rand_product_shapes(gsvd_rand_t h, int *shapes);

/* Comparative quantities of Section 1 for r GSV pairs (alpha non-increasing,
 * beta non-decreasing):
 *   theta[i] = atan2(alpha_i, beta_i) - pi/4      (antisymmetric angular distance)
 *   rho[i]   = alpha_i / beta_i, +inf if beta_i = 0 (relative significance)
 *   P1[i] = alpha_i^2 / sum alpha^2, P2[i] = beta_i^2 / sum beta^2
 *   D[0], D[1] = -(1/log N) sum P log P, 0 log 0 = 0 (generalized entropy)
 * pad_to_n = 0: N = r.  pad_to_n > r: pad to N = pad_to_n pairs as Algorithm 2
 * does — pad_mode 0 appends (alpha, beta) = (0, 1), pad_mode 1 prepends (1, 0).
 * theta, rho, P1, P2 hold N doubles; D holds 2.  Any output may be NULL.
 * Errors: ARG (r < 1, N < 2, NULL alpha/beta).  Synchronises cfg->stream. */
int gsvd_rand_metrics(gsvd_rand_t h, const double *alpha, const double *beta, int r,
                      int pad_to_n, int pad_mode, double *theta, double *rho, double *P1,
                      double *P2, double *D);

/* Largest pair count N (after padding) that gsvd_rand_metrics_noalloc accepts. */
#define GSVD_RAND_NOALLOC_MAX_N 32768

/* gsvd_rand_metrics for callers that cannot let a library allocate device
 * memory.  The paper has no counterpart: this is a service entry point.
 * Outputs and arguments are those of gsvd_rand_metrics (same formulas, same
 * padding); results agree with it to rounding (the entropy sums are added in
 * another order).  Differences:
 *   - No handle: `device` is the GPU to run on and `stream` a cudaStream_t
 *     (NULL = the legacy default stream).  The caller's current device is
 *     restored before returning.
 *   - Nothing is allocated (no cudaMalloc, no pinned host memory).  Scratch is
 *     one fixed array of about 1.5 MiB in the library's static device memory,
 *     held on every GPU that loads the library until the process exits.
 *     Device pointers are used in place; host inputs and outputs pass through
 *     that scratch.  Its block counter is cleared on the stream at each call.
 *   - N = max(r, pad_to_n) <= GSVD_RAND_NOALLOC_MAX_N, else
 *     GSVD_RAND_ERR_TOO_LARGE and nothing is enqueued.
 *   - Every call looks up the scratch address on `device` (cudaGetSymbolAddress,
 *     which allocates nothing), so the entry point stays valid after the
 *     device's context is reset; the first call on a device also loads the
 *     library's device code there: make that first call before any stream capture.
 *   - All calls on one device share the one scratch array: calls that overlap
 *     in time (from several host threads, or on several streams) race and can
 *     return wrong results.  Each call synchronises `stream` before it returns.
 * Errors: ARG (as gsvd_rand_metrics, or a bad device), TOO_LARGE, CUDA.
 * There is no message string: the return code is the whole report. */
int gsvd_rand_metrics_noalloc(int device, void *stream, const double *alpha, const double *beta,
                              int r, int pad_to_n, int pad_mode, double *theta, double *rho,
                              double *P1, double *P2, double *D);

/* The Gaussian test matrix the solver draws: out (n x l, row-major, ld = l)
 * with out[i][j] from Philox4x32-10 (Salmon et al., SC'11) and Box-Muller:
 *   e = i*l + j, t = e >> 1; counter (t, pair, side, stream), key (seed lo, seed hi);
 *   words x0..x3: u1 = ((x0 >> 5) 2^26 + (x1 >> 6) + 0.5) 2^-53,
 *                 u2 = ((x2 >> 5) 2^26 + (x3 >> 6)) 2^-53,
 *   r = sqrt(-2 ln u1), a = 2 pi u2; even e -> r cos a, odd e -> r sin a.
 * Computed in FP64.  Errors: ARG, OOM, CUDA. */
int gsvd_rand_gaussian(gsvd_rand_t h, int64_t n, int64_t l, uint64_t seed, uint32_t pair,
                       uint32_t side, uint32_t stream, double *out);

/* The raw Philox4x32-10 words for counters (t, pair, side, stream), t = 0..count-1:
 * out[4 t + w] = word w.  Errors: ARG, OOM, CUDA. */
int gsvd_rand_philox(gsvd_rand_t h, uint64_t count, uint64_t seed, uint32_t pair, uint32_t side,
                     uint32_t stream, uint32_t *out);

/* Accumulated device time (ms, from CUDA events on the solve stream) and call
 * count of one stage since creation or the last reset; only filled while the
 * context has GSVD_RAND_FLAG_PROFILE.  In grouped solves the compressed-pair
 * GSVDs of pairs with L = 2l > 128 run as a branch concurrent with the others',
 * each step timed on its own branch: there the stage totals overlap and can sum
 * to more than the solve's elapsed time.  Errors: ARG (bad stage). */
int gsvd_rand_profile_get(gsvd_rand_t h, int stage, double *total_ms, int64_t *calls);
int gsvd_rand_profile_reset(gsvd_rand_t h);

/* Columns of the two bases used by the last gsvd_rand_solve on h: k + oversample each on
 * the fixed path, the Algorithm 1 block counts times block_b (or the cap) on the adaptive
 * path.  Errors: ARG (NULL handle). */
int gsvd_rand_basis_cols(gsvd_rand_t h, int *l1, int *l2);

/* Number of solves on h and its gsvd_rand_solve_batched workers that were repeated with FP64
 * Cholesky factors (the GSVD_RAND_FLAG_CHOL_FP64 form) because the FP32 factors of their
 * CholeskyQR broke down (NONFINITE or BREAKDOWN): FP32 data whose sketch is conditioned
 * beyond about 1e6, where the first shifted pass leaves Q1 too ill-conditioned for an FP32
 * Gram.  The repeated solve's result is the one returned.  Errors: ARG (NULL handle). */
int gsvd_rand_chol64_retries(gsvd_rand_t h, int64_t *count);

/* Total number of CUDA kernels this library has launched in this process. */
uint64_t gsvd_rand_launch_count(void);

/* ---------------------------------------------------------------------------
 * Learned (k, q) proposal.  The paper has no learned component: Algorithm 1
 * (Section 2) chooses the basis size adaptively, the fixed-rank method of
 * Section 3 needs k (and the power steps q) given.  A small classifier maps
 * cheap probe features of the pair to (k bucket, q) for the fixed-rank solve;
 * Algorithm 1 labels its training pairs and takes over whenever the proposed
 * bases miss the tolerance.
 *
 * Features (64 floats, side 1 then side 2): with Omega_p the n x 64 Gaussian
 * of Philox stream GSVD_RAND_STREAM_PROBE and Y = G Omega_p, log10 of the 1st,
 * 3rd, ..., 63rd largest eigenvalues of Y^T Y / (64 ||G||_F^2), clipped to
 * [-12, 1] (32 per side).  A 64-column probe shows where the energy of each side
 * falls off for ranks up to about 64 (a 16-column one, only up to 16).
 * Network: x^ = (x - mean) / std, h1 = relu(x^ W1 + b1), h2 = relu(h1 W2 + b2),
 * z = h2 W3 + b3; W1 64 x 128, W2 128 x 128, W3 128 x 37, row-major; params is
 * W1 | b1 | W2 | b2 | W3 | b3 (GSVD_RAND_MLP_PARAMS floats), norm is mean | std
 * (128 floats).  z[0:32]: k bucket b (k = 4b+1 .. 4b+4; the solve takes 4b+4 of the
 * smallest bucket whose cumulative softmax probability reaches GSVD_RAND_MLP_KQUANTILE),
 * z[32:37]: q = 0..4 (the solve takes the argmax).  Loss: softmax cross-entropy of each head, batch means,
 * summed.  All network pointers are device pointers unless stated.
 * --------------------------------------------------------------------------- */
#define GSVD_RAND_MLP_IN 64
#define GSVD_RAND_MLP_HID 128
#define GSVD_RAND_MLP_KCLS 32
#define GSVD_RAND_MLP_QCLS 5
#define GSVD_RAND_MLP_KBUCKET 4
#define GSVD_RAND_MLP_PROBE 64
#define GSVD_RAND_MLP_KQUANTILE 0.9 /* the learned solve takes the smallest k bucket whose
                                       cumulative softmax probability reaches this level */
#define GSVD_RAND_MLP_PARAMS (64 * 128 + 128 + 128 * 128 + 128 + 128 * 37 + 37)

/* The 64 probe features of {G1, G2} (layouts and precision as gsvd_rand_solve;
 * the Philox pair word is 0).  feats: 64 floats, device or host.  Errors: ARG
 * (m, p or n below 64), OOM, CUDA. */
int gsvd_rand_probe_features(gsvd_rand_t h, const void *G1, int64_t m, int64_t ld1, const void *G2, int64_t p,
                             int64_t ld2, int64_t n, uint64_t seed, float *feats);

/* Logits (B x 37) of the features X (B x 64); bf16 != 0 rounds the weight matrices
 * to BF16 (the inference form), else FP32.  Errors: ARG, OOM, CUDA. */
int gsvd_rand_mlp_forward(gsvd_rand_t h, const float *params, const float *norm, const float *X, int B, int bf16,
                          float *logits);

/* Mean loss (*loss, one device float) and its gradient (GSVD_RAND_MLP_PARAMS floats)
 * over the batch X (B x 64) with labels yk (k bucket) and yq (q), FP32.
 * Errors: ARG, OOM, CUDA. */
int gsvd_rand_mlp_loss_grad(gsvd_rand_t h, const float *params, const float *norm, const float *X, const int *yk,
                            const int *yq, int B, float *grad, float *loss);

/* One Adam step t >= 1 (Kingma & Ba 2015, bias-corrected) on params with moments m, v.
 * Errors: ARG, CUDA. */
int gsvd_rand_mlp_adam(gsvd_rand_t h, float *params, float *m, float *v, const float *grad, int t, float lr,
                       float beta1, float beta2, float eps);

/* `steps` minibatch steps of B rows each: step i uses rows order[i B .. i B + B - 1] of
 * X, yk, yq, then Adam (beta 0.9, 0.999, eps 1e-8) at step t0 + i + 1; loss_hist[i]
 * receives its loss.  Errors: ARG, OOM, CUDA. */
int gsvd_rand_mlp_train(gsvd_rand_t h, float *params, float *m, float *v, const float *norm, const float *X,
                        const int *yk, const int *yq, const int *order, int steps, int B, int t0, float lr,
                        float *loss_hist);

/* The network of the learned solve: params and norm copied from device or host
 * memory.  Errors: ARG, OOM, CUDA. */
int gsvd_rand_mlp_set(gsvd_rand_t h, const float *params, const float *norm);

/* The network from a file: "GSVDMLP1", int32 {64, 128, 32, 5}, then norm (128
 * floats) and params, little-endian.  Errors: ARG (missing or malformed file). */
int gsvd_rand_mlp_load(gsvd_rand_t h, const char *path);

/* The learned solve's (k, q) plan of B rows of network outputs (logits: device, B x 37 row-major,
 * as gsvd_rand_mlp_forward writes them), on the device: plan[3 i] = the top k of the smallest k
 * bucket whose cumulative softmax probability reaches `quantile` (GSVD_RAND_MLP_KQUANTILE in the
 * learned solves), plan[3 i + 1] = the most probable q (first on ties), plan[3 i + 2] = that k
 * bucket.  plan: 3 B ints, device or host.  The learned solves apply the same rule and then clip
 * k to their limits.  Synchronises cfg->stream.  Errors: ARG, CUDA. */
int gsvd_rand_mlp_plan(gsvd_rand_t h, const float *logits, int B, double quantile, int *plan);

/* k and q of the last learned solve, and fallback = 1 when Algorithm 1 solved it. */
int gsvd_rand_last_plan(gsvd_rand_t h, int *k, int *q, int *fallback);

#ifdef __cplusplus
}
#endif
#endif /* GSVD_RAND_H */
