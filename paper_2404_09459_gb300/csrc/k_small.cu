// Small dense kernels of the compressed-pair GSVD (Algorithm 2 after the basis
// extraction) and of the comparative metrics (Section 1).
//
// GB300 runs FP64 at about 1/57 of its FP32 rate (measured: 7.95 GFLOP/s per
// SM FP64 vs 457 GFLOP/s FP32), so no FP64 work here is sequential on one SM:
//   * FP64 products (the Gram K = S S^T, the refinement products) are split-K
//     GEMMs spread over the whole GPU;
//   * the eigensolver itself is a one-CTA FP32 cyclic Jacobi, and its result is
//     lifted to FP64 accuracy by Ogita-Aishima refinement (Ogita & Aishima,
//     "Iterative refinement for symmetric eigenvalue decomposition", Japan J.
//     Indust. Appl. Math. 35, 2018), whose work is FP64 GEMMs again.
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "kernels.h"

namespace gsvdr {

// ============================================================================
// FP64 split-K GEMM for small operands: C = alpha op(A) op(B) + beta C.
// ============================================================================
constexpr int SG_T = 32, SG_BK = 32;
// The tile loader maps e -> (e / 32, e % 32) onto both operand tiles: square 32 x 32.
static_assert(SG_T == 32 && SG_BK == 32, "dgemm_small_kernel's loader assumes 32 x 32 tiles");
constexpr int SG_KGRAIN = 8;  // split-K chunks are multiples of 8 (partial tiles are zero-filled)

// ----------------------------------------------------------------------------
// Double-float arithmetic (the mixed-precision paths).  GB300 runs FP32 at 64x its FP64 rate,
// so the refinement products of the mixed paths (1e-4 target) keep each operand as an
// unevaluated sum hi + lo of two FP32 numbers (Dekker, Numer. Math. 18, 1971) and accumulate
// with error-free transformations: the FP32 product of the high parts with its exact rounding
// error from an FMA, the cross terms hi*lo, and Knuth's TwoSum for the running sum (Knuth,
// TAOCP vol. 2, 4.2.2).  Relative precision about 2^-48 per product, against 2^-53 in FP64; the
// plain FP64 path keeps FP64.  The _rn intrinsics keep the compiler from contracting the
// TwoSum steps into FMAs, which would break their exactness.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void df_fma(const float2 a, const float2 b, float& sh, float& sl) {
  const float ph = __fmul_rn(a.x, b.x);
  const float pe = fmaf(a.x, b.x, -ph);                 // exact rounding error of a.x b.x
  const float pl = fmaf(a.x, b.y, fmaf(a.y, b.x, pe));  // plus the cross terms
  const float s = __fadd_rn(sh, ph);
  const float bb = __fsub_rn(s, sh);
  const float e = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(ph, bb));  // sh + ph - s exactly
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(e, pl));
}
// (sh, sl) back to |sl| <= ulp(sh) / 2 (Dekker's fast two-sum; |sh| >= |sl| by construction).
__device__ __forceinline__ void df_renorm(float& sh, float& sl) {
  const float s = __fadd_rn(sh, sl);
  sl = __fsub_rn(sl, __fsub_rn(s, sh));
  sh = s;
}
// One operand element into a tile slot: FP64 as is, or (DF) as its hi + lo FP32 pair stored in
// the same 8 bytes (hi = nearest FP32, lo = nearest FP32 to the remainder).
template <bool DF, typename T>
__device__ __forceinline__ void sg_put(double* slot, T v) {
  if constexpr (DF) {
    float h, l;
    if constexpr (std::is_same<T, float>::value) {
      h = v;
      l = 0.f;
    } else {
      h = __double2float_rn(v);
      l = __double2float_rn(v - (double)h);
    }
    *reinterpret_cast<float2*>(slot) = make_float2(h, l);
  } else {
    *slot = (double)v;
  }
}
// The 2 x 2 outputs of a thread over one k-tile (kk < kk_end): FP64 FMAs, or double-float.
template <bool DF>
__device__ __forceinline__ void sg_tile(const double (*As)[SG_T + 1], const double (*Bs)[SG_T + 1], int kk_end,
                                        int ty, int tx, double (&acc)[2][2], float (&dh)[2][2], float (&dl)[2][2]) {
  if constexpr (DF) {
#pragma unroll 4
    for (int kk = 0; kk < kk_end; ++kk) {
      const float2 a0 = *reinterpret_cast<const float2*>(&As[kk][ty * 2]);
      const float2 a1 = *reinterpret_cast<const float2*>(&As[kk][ty * 2 + 1]);
      const float2 b0 = *reinterpret_cast<const float2*>(&Bs[kk][tx * 2]);
      const float2 b1 = *reinterpret_cast<const float2*>(&Bs[kk][tx * 2 + 1]);
      df_fma(a0, b0, dh[0][0], dl[0][0]);
      df_fma(a0, b1, dh[0][1], dl[0][1]);
      df_fma(a1, b0, dh[1][0], dl[1][0]);
      df_fma(a1, b1, dh[1][1], dl[1][1]);
    }
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int q = 0; q < 2; ++q) df_renorm(dh[m][q], dl[m][q]);
  } else {
#pragma unroll 8
    for (int kk = 0; kk < kk_end; ++kk) {
      const double a0 = As[kk][ty * 2], a1 = As[kk][ty * 2 + 1];
      const double b0 = Bs[kk][tx * 2], b1 = Bs[kk][tx * 2 + 1];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
  }
}
template <bool DF>
__device__ __forceinline__ double sg_out(const double (&acc)[2][2], const float (&dh)[2][2], const float (&dl)[2][2],
                                         int m, int q) {
  return DF ? (double)dh[m][q] + (double)dl[m][q] : acc[m][q];
}

// A (N x N, ld N) scaled by the power of two that brings its largest |diagonal entry| into
// [1, 2): exact, and it keeps a Gram of any scale inside FP32's exponent range for the
// double-float products (the eigenvectors do not depend on the scale).  One CTA per problem.
__device__ __forceinline__ void pow2_scale_body(double* A, int N) {
  __shared__ double s_m[8];
  double m = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) m = fmax(m, fabs(A[(int64_t)i * N + i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
  __syncthreads();
  double mx = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, s_m[w]);
  if (!(mx > 0.0) || !isfinite(mx)) return;
  const double f = ldexp(1.0, -ilogb(mx));
  for (int64_t e = threadIdx.x; e < (int64_t)N * N; e += blockDim.x) A[e] *= f;
}
__global__ __launch_bounds__(256) void pow2_scale_kernel(double* A, int N) { pow2_scale_body(A, N); }
__global__ __launch_bounds__(256) void pow2_scale_b_kernel(const EigB* __restrict__ tab) {
  const EigB& e = tab[blockIdx.x];
  pow2_scale_body(const_cast<double*>(e.A), e.N);
}
cudaError_t launch_pow2_scale(double* A, int N, cudaStream_t st) {
  if (N < 1) return cudaSuccess;
  pow2_scale_kernel<<<1, 256, 0, st>>>(A, N);
  return launched();
}
cudaError_t launch_pow2_scale_b(const EigB* tab, int nprob, cudaStream_t st) {
  if (nprob < 1) return cudaSuccess;
  pow2_scale_b_kernel<<<nprob, 256, 0, st>>>(tab);
  return launched();
}

template <typename TA, typename TB, bool DF>
__global__ __launch_bounds__(256) void dgemm_small_kernel(int Mr, int Nc, int K, const TA* __restrict__ A,
                                                          int64_t lda, int ta, const TB* __restrict__ B,
                                                          int64_t ldb, int tb, double* __restrict__ part,
                                                          int kchunk) {
  __shared__ double As[SG_BK][SG_T + 1];
  __shared__ double Bs[SG_BK][SG_T + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.x * SG_T, j0 = blockIdx.y * SG_T, z = blockIdx.z;
  const int kb = z * kchunk, ke = min(K, kb + kchunk);
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  float dh[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, dl[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int k0 = kb; k0 < ke; k0 += SG_BK) {
    for (int e = tid; e < SG_T * SG_BK; e += 256) {
      int a = e / 32, b = e % 32;
      // A element (i, k)
      int i, kk;
      if (!ta) { i = a; kk = b; } else { kk = a; i = b; }
      int gi = i0 + i, gk = k0 + kk;
      TA va = TA(0);
      if (gi < Mr && gk < ke) va = ta ? A[(int64_t)gk * lda + gi] : A[(int64_t)gi * lda + gk];
      sg_put<DF>(&As[kk][i], va);
      // B element (k, j)
      int j;
      if (!tb) { kk = a; j = b; } else { j = a; kk = b; }
      int gj = j0 + j;
      gk = k0 + kk;
      TB vb = TB(0);
      if (gj < Nc && gk < ke) vb = tb ? B[(int64_t)gj * ldb + gk] : B[(int64_t)gk * ldb + gj];
      sg_put<DF>(&Bs[kk][j], vb);
    }
    __syncthreads();
    sg_tile<DF>(As, Bs, min(SG_BK, ke - k0), ty, tx, acc, dh, dl);
    __syncthreads();
  }
  double* P = part + (int64_t)z * Mr * Nc;
  for (int m = 0; m < 2; ++m)
    for (int q = 0; q < 2; ++q) {
      int i = i0 + ty * 2 + m, j = j0 + tx * 2 + q;
      if (i < Mr && j < Nc) P[(int64_t)i * Nc + j] = sg_out<DF>(acc, dh, dl, m, q);
    }
}

__global__ void dgemm_reduce_kernel(const double* __restrict__ part, int splits, int Mr, int Nc,
                                    double* C, int64_t ldc, double alpha, double beta) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)Mr * Nc) return;
  int i = (int)(e / Nc), j = (int)(e % Nc);
  double s = 0.0;
  for (int z = 0; z < splits; ++z) s += part[(int64_t)z * Mr * Nc + e];
  double* c = C + (int64_t)i * ldc + j;
  *c = beta == 0.0 ? alpha * s : alpha * s + beta * (*c);
}

template <typename TA, typename TB>
cudaError_t launch_dgemm_small(int Mr, int Nc, int K, const TA* A, int64_t lda, int ta, const TB* B,
                               int64_t ldb, int tb, double* C, int64_t ldc, double alpha, double beta,
                               double* work, int64_t work_elems, cudaStream_t st, bool df) {
  if (Mr <= 0 || Nc <= 0) return cudaSuccess;
  int tiles = (int)(cdiv(Mr, SG_T) * cdiv(Nc, SG_T));
  int kslices = (int)cdiv(std::max(K, 1), SG_KGRAIN);
  int splits = std::max(1, std::min(kslices, (2 * 152 + tiles - 1) / tiles));
  while (splits > 1 && (int64_t)splits * Mr * Nc > work_elems) --splits;
  if ((int64_t)Mr * Nc > work_elems) return cudaErrorInvalidValue;
  int kchunk = (int)round_up(cdiv(std::max(K, 1), splits), SG_KGRAIN);
  splits = (int)cdiv(std::max(K, 1), kchunk);
  dim3 grid((unsigned)cdiv(Mr, SG_T), (unsigned)cdiv(Nc, SG_T), (unsigned)splits);
  if (df)
    dgemm_small_kernel<TA, TB, true><<<grid, 256, 0, st>>>(Mr, Nc, K, A, lda, ta, B, ldb, tb, work, kchunk);
  else
    dgemm_small_kernel<TA, TB, false><<<grid, 256, 0, st>>>(Mr, Nc, K, A, lda, ta, B, ldb, tb, work, kchunk);
  cudaError_t e = launched();
  if (e != cudaSuccess) return e;
  dgemm_reduce_kernel<<<(unsigned)cdiv((int64_t)Mr * Nc, 256), 256, 0, st>>>(work, splits, Mr, Nc, C, ldc,
                                                                              alpha, beta);
  return launched();
}
template cudaError_t launch_dgemm_small<double, double>(int, int, int, const double*, int64_t, int,
                                                        const double*, int64_t, int, double*, int64_t,
                                                        double, double, double*, int64_t, cudaStream_t, bool);
template cudaError_t launch_dgemm_small<float, float>(int, int, int, const float*, int64_t, int,
                                                      const float*, int64_t, int, double*, int64_t,
                                                      double, double, double*, int64_t, cudaStream_t, bool);

// ============================================================================
// One-CTA cyclic Jacobi in FP32 with the round-robin (circle) ordering: every
// round applies N'/2 disjoint rotations (N' = N rounded up to even; pairs with
// the dummy index are skipped), N'-1 rounds form a sweep.  Rotation angles as
// in Golub & Van Loan, Algorithm 8.5.1 (sym.schur2).  A and V live in shared
// memory when they fit, else in the global scratch (L2-resident).
// ============================================================================
int64_t jacobi_scratch_floats(int N) { return 2ll * N * (N | 1); }

__global__ __launch_bounds__(1024) void jacobi_f32_kernel(const double* __restrict__ Ain, int N,
                                                          double* __restrict__ Vout,
                                                          double* __restrict__ lam, float* scratch,
                                                          int use_smem, int max_sweeps,
                                                          DevStatus* st_dev) {
  extern __shared__ float sm[];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarp = nt >> 5;
  const int Np = N + (N & 1), m = Np / 2;
  const int lda = N | 1;  // odd row stride: column walks are bank-conflict free
  float* A = use_smem ? sm : scratch;
  float* V = A + (int64_t)N * lda;
  __shared__ int s_p[256], s_q[256];
  __shared__ float s_c[256], s_s[256];
  __shared__ float s_scale;
  __shared__ unsigned s_off;  // max |a_pq| of the sweep (scaled A), as float bits
  if (tid == 0) {
    double mx = 0.0;
    for (int i = 0; i < N; ++i) mx = fmax(mx, fabs(Ain[(int64_t)i * N + i]));
    s_scale = (float)(mx > 0.0 && isfinite(mx) ? mx : 1.0);
  }
  __syncthreads();
  const float inv = 1.0f / s_scale;
  for (int i = warp; i < N; i += nwarp)
    for (int j = lane; j < N; j += 32) {
      A[(int64_t)i * lda + j] = (float)(Ain[(int64_t)i * N + j] * (double)inv);
      V[(int64_t)i * lda + j] = (i == j) ? 1.0f : 0.0f;
    }
  __syncthreads();
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) s_off = 0u;
    __syncthreads();
    for (int rnd = 0; rnd < Np - 1; ++rnd) {
      // phase A: the round's disjoint pairs (circle method: slot Np-1 fixed;
      // pairs (rnd, Np-1) and ((rnd + k) mod (Np-1), (rnd - k) mod (Np-1)); every
      // pair meets once in Np-1 rounds) and their rotation parameters.
      for (int k = tid; k < m; k += nt) {
        int a, b;
        if (k == 0) {
          a = rnd;
          b = Np - 1;
        } else {
          a = (rnd + k) % (Np - 1);
          b = (rnd - k + (Np - 1)) % (Np - 1);
        }
        const int p = min(a, b), q = max(a, b);
        float c = 1.f, s = 0.f;
        if (q < N) {
          float apq = A[(int64_t)p * lda + q], app = A[(int64_t)p * lda + p], aqq = A[(int64_t)q * lda + q];
          // A is scaled to max |a_ii| = 1: an absolute off-diagonal test.  The FP32
          // result only needs absolute accuracy ~u ||A|| (the FP64 refinement
          // takes it from there); a relative test would never stop on the
          // noise-level eigenvalues that FP32 cannot resolve.
          float off = fabsf(apq);
          atomicMax(&s_off, __float_as_uint(off));
          if (off > 1e-10f) {
            float tau = (aqq - app) / (2.f * apq);
            float t = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            c = rsqrtf(1.f + t * t);
            s = t * c;
          }
        }
        s_p[k] = p;
        s_q[k] = q;
        s_c[k] = c;
        s_s[k] = s;
      }
      __syncthreads();
      // phase B: columns p, q of A and V (A <- A J, V <- V J); warp per pair, lane per row
      for (int k = warp; k < m; k += nwarp) {
        const float c = s_c[k], s = s_s[k];
        if (s == 0.f) continue;
        const int p = s_p[k], q = s_q[k];
        for (int i = lane; i < N; i += 32) {
          float* ai = A + (int64_t)i * lda;
          float x = ai[p], y = ai[q];
          ai[p] = c * x - s * y;
          ai[q] = s * x + c * y;
          float* vi = V + (int64_t)i * lda;
          x = vi[p];
          y = vi[q];
          vi[p] = c * x - s * y;
          vi[q] = s * x + c * y;
        }
      }
      __syncthreads();
      // phase C: rows p, q of A (A <- J^T A); the annihilated entries are set to zero
      for (int k = warp; k < m; k += nwarp) {
        const float c = s_c[k], s = s_s[k];
        if (s == 0.f) continue;
        const int p = s_p[k], q = s_q[k];
        float* ap = A + (int64_t)p * lda;
        float* aq = A + (int64_t)q * lda;
        for (int j = lane; j < N; j += 32) {
          float x = ap[j], y = aq[j];
          ap[j] = (j == q) ? 0.f : c * x - s * y;
          aq[j] = (j == p) ? 0.f : s * x + c * y;
        }
      }
      __syncthreads();
    }
    // every thread reads the sweep's maximum before anyone resets it
    const float off = __uint_as_float(s_off);
    __syncthreads();
    if (off < 1e-7f) break;
  }
  if (sweep == max_sweeps && tid == 0 && st_dev) {
    // not converged to FP32 level: the refinement still improves it; counted only
    atomicAdd(&st_dev->pad, 1);
  }
  for (int i = warp; i < N; i += nwarp)
    for (int j = lane; j < N; j += 32) Vout[(int64_t)i * N + j] = (double)V[(int64_t)i * lda + j];
  for (int i = tid; i < N; i += nt) lam[i] = (double)A[(int64_t)i * lda + i] * (double)s_scale;
}

cudaError_t launch_jacobi_f32(const double* A, int N, double* V, double* lam, float* scratch,
                              int max_sweeps, DevStatus* st_dev, cudaStream_t st) {
  if (N < 1 || N > 512) return cudaErrorInvalidValue;
  size_t need = (size_t)jacobi_scratch_floats(N) * sizeof(float);
  int use_smem = need <= 200 * 1024;
  size_t smem = use_smem ? need : 0;
  cudaFuncSetAttribute(jacobi_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  jacobi_f32_kernel<<<1, 1024, smem, st>>>(A, N, V, lam, scratch, use_smem, max_sweeps, st_dev);
  return launched();
}

// ============================================================================
// Ogita-Aishima refinement (FP64).  X = X + X F with
//   R = I - X^T X, S = X^T A X, lam_i = s_ii / (1 - r_ii),
//   delta = 2 (||S - diag(lam)||_F + ||A||_F ||R||_F),
//   F_ij = (s_ij + lam_j r_ij) / (lam_j - lam_i) if |lam_i - lam_j| > delta, else r_ij / 2,
//   F_ii = r_ii / 2.
// ============================================================================
// Partial Frobenius sums of A, R = I - X^T X and S - diag(lam) per CTA; CTA 0
// also writes lam_i = s_ii / (x_i^T x_i) (= s_ii / (1 - r_ii)).
__global__ void oa_norms_kernel(const double* __restrict__ A, int N, const double* __restrict__ XtX,
                                const double* __restrict__ S, double* __restrict__ part,
                                double* __restrict__ lam) {
  __shared__ double red[3][8];
  const int64_t nn = (int64_t)N * N;
  double a2 = 0.0, r2 = 0.0, s2 = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / N), j = (int)(e % N);
    const double a = A[e];
    const double r = (i == j ? 1.0 : 0.0) - XtX[e];
    double sd = S[e];
    if (i == j) sd -= S[e] / XtX[e];
    a2 += a * a;
    r2 += r * r;
    s2 += sd * sd;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a2 += __shfl_down_sync(0xffffffffu, a2, o);
    r2 += __shfl_down_sync(0xffffffffu, r2, o);
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a2;
    red[1][threadIdx.x >> 5] = r2;
    red[2][threadIdx.x >> 5] = s2;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
    part[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = t;
  }
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < N; i += blockDim.x) lam[i] = S[(int64_t)i * N + i] / XtX[(int64_t)i * N + i];
}

// F_ij = (s_ij + lam_j r_ij) / (lam_j - lam_i) if |lam_i - lam_j| > delta else r_ij / 2,
// delta = 2 (||S - D||_F + ||A||_F ||R||_F) from the partial sums.
__global__ void oa_form_kernel(int N, const double* __restrict__ XtX, const double* __restrict__ S,
                               const double* __restrict__ part, int nparts, const double* __restrict__ lam,
                               double* __restrict__ F) {
  __shared__ double s_delta;
  if (threadIdx.x == 0) {
    double A2 = 0, R2 = 0, S2 = 0;
    for (int b = 0; b < nparts; ++b) {
      A2 += part[b];
      R2 += part[nparts + b];
      S2 += part[2 * nparts + b];
    }
    s_delta = 2.0 * (sqrt(S2) + sqrt(A2) * sqrt(R2));
  }
  __syncthreads();
  const double delta = s_delta;
  const int64_t nn = (int64_t)N * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / N), j = (int)(e % N);
    const double r = (i == j ? 1.0 : 0.0) - XtX[e];
    double f;
    if (i == j) {
      f = 0.5 * r;
    } else {
      const double d = lam[j] - lam[i];
      f = (fabs(d) > delta) ? (S[e] + lam[j] * r) / d : 0.5 * r;
    }
    F[e] = f;
  }
}

cudaError_t launch_oa_refine(const double* A, int N, double* X, double* lam, double* work,
                             int64_t work_elems, cudaStream_t st, bool df) {
  const int64_t nn = (int64_t)N * N;
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(128, cdiv(nn, 1024)));
  if (work_elems < 4 * nn + 3 * nb + nn) return cudaErrorInvalidValue;
  double* XtX = work;
  double* P = work + nn;
  double* S = work + 2 * nn;
  double* F = work + 3 * nn;
  double* part = work + 4 * nn;
  double* sk = part + 3 * nb;
  const int64_t skn = work_elems - 4 * nn - 3 * nb;
  cudaError_t e;
  if ((e = launch_dgemm_small<double, double>(N, N, N, X, N, 1, X, N, 0, XtX, N, 1.0, 0.0, sk, skn, st, df)))
    return e;
  if ((e = launch_dgemm_small<double, double>(N, N, N, A, N, 0, X, N, 0, P, N, 1.0, 0.0, sk, skn, st, df)))
    return e;
  if ((e = launch_dgemm_small<double, double>(N, N, N, X, N, 1, P, N, 0, S, N, 1.0, 0.0, sk, skn, st, df)))
    return e;
  oa_norms_kernel<<<nb, 256, 0, st>>>(A, N, XtX, S, part, lam);
  if ((e = launched())) return e;
  oa_form_kernel<<<nb, 256, 0, st>>>(N, XtX, S, part, nb, lam, F);
  if ((e = launched())) return e;
  // X <- X + X F   (the reduce of the split-K product reads and writes X elementwise)
  return launch_dgemm_small<double, double>(N, N, N, X, N, 0, F, N, 0, X, N, 1.0, 1.0, sk, skn, st, df);
}

// ============================================================================
// The cluster across the cut.  The Ogita-Aishima step only orthogonalises
// eigenvector pairs whose eigenvalues lie within delta of each other; with an
// FP32 start, delta stays near the start's error, so such a cluster is never
// split.  Only a cluster that straddles the cut between the r-th and
// (r+1)-th largest eigenvalue changes the selected span, so that one block of
// S = X^T A X (from the last refinement step) is diagonalised here: shifted
// by its mean and scaled to unit size, which resolves the block's own
// spread, by parallel cyclic Jacobi in FP32 (round-robin pairs).  Its columns
// of X are then rotated, X_c <- X_c V_c, and the following refinement steps
// re-orthogonalise in FP64 and separate them.  A cluster of more than
// CUT_CMAX columns (a dense run of eigenvalues below FP32 resolution, e.g. a
// slowly decaying tail) is not clipped: its shifted and scaled block is left
// in XtX (no longer needed by then) for the packed-triangle FP32 eigensolver,
// a second launch that reads the block's size from the descriptor this
// kernel writes (launch_eig_cut_big).
// Work layout (as launch_oa_refine): XtX, P, S, F (N x N each), part (3 nb).
// V_c goes to F, the cluster's column indices and size to P (ints 0 .. c);
// for a large cluster P also holds the eigensolver's descriptor (EigB at double
// offset CUT_EIGB_OFF) and the block's eigenvalues (from CUT_LAM_OFF).
// ============================================================================

__device__ __forceinline__ void oa_cut_cluster_body(int N, int r, double* XtX, const double* __restrict__ S,
                                                    const double* __restrict__ part, int nparts,
                                                    const double* __restrict__ lam, double* __restrict__ Vc,
                                                    int* __restrict__ cinfo, float* jscr, double null_rel) {
  extern __shared__ float cut_sm[];
  __shared__ int s_ord[512];
  __shared__ double s_dg[CUT_BIG_NMAX];  // Rayleigh quotients s_ii / x_i^T x_i of the cluster
  __shared__ double s_wmax[32];
  __shared__ int s_lo, s_c;
  __shared__ double s_delta, s_mu, s_scale;
  __shared__ int s_p[CUT_CMAX / 2], s_q[CUT_CMAX / 2];
  __shared__ float s_cs[CUT_CMAX / 2], s_sn[CUT_CMAX / 2];
  __shared__ unsigned s_off;
  __shared__ int s_null;
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nwarp = nt >> 5;
  // clusters beyond CUT_CMAX columns go to the second launch when its scratch is given
  const bool big_ok = jscr != nullptr && N > CUT_CMAX;
  const int cap = big_ok ? CUT_BIG_NMAX : CUT_CMAX;
  EigB* eb = big_ok ? reinterpret_cast<EigB*>(reinterpret_cast<double*>(cinfo) + CUT_EIGB_OFF) : nullptr;
  if (tid == 0) {
    double A2 = 0, R2 = 0, S2 = 0;
    for (int b = 0; b < nparts; ++b) {
      A2 += part[b];
      R2 += part[nparts + b];
      S2 += part[2 * nparts + b];
    }
    s_delta = 2.0 * (sqrt(S2) + sqrt(A2) * sqrt(R2));
  }
  // descending rank of every eigenvalue (NaN last, ties by index): s_ord[rank] = index
  for (int i = tid; i < N; i += nt) {
    const double li = isnan(lam[i]) ? -INFINITY : lam[i];
    int rank = 0;
    for (int j = 0; j < N; ++j) {
      const double lj = isnan(lam[j]) ? -INFINITY : lam[j];
      rank += (lj > li) || (lj == li && j < i);
    }
    s_ord[min(rank, N - 1)] = i;
  }
  __syncthreads();
  if (tid == 0) {
    const double d = s_delta;
    auto lm = [&](int rk) { return lam[s_ord[rk]]; };
    int lo = r - 1, hi = r + 1;  // ranks [lo, hi)
    // no cluster when the gap at the cut is resolved, or (null_rel > 0) when the last kept
    // eigenvalue lies below null_rel of the largest: the cut is then in the numerical null space
    // of K (directions of the bases beyond the pair's rank, at the FP32 data's noise level), where
    // any split is as good as another
    if (r < 1 || r >= N || !(lm(r - 1) - lm(r) <= d) || (null_rel > 0.0 && lm(r - 1) <= null_rel * lm(0))) {
      lo = 0;
      hi = 0;
    } else {
      while (lo > 0 && lm(lo - 1) - lm(lo) <= d && hi - lo < cap) --lo;
      while (hi < N && lm(hi - 1) - lm(hi) <= d && hi - lo < cap) ++hi;
    }
    s_lo = lo;
    s_c = hi - lo;
    // the cluster reaches into the numerical null space of K (null_rel > 0): its block is then
    // taken unshifted, so that the null eigenvalues sit at zero, where the big eigensolver takes
    // them as noise (an orthonormal complement of the other columns: their orientation inside
    // the null space is arbitrary) instead of separating a many-fold eigenvalue column by column
    s_null = null_rel > 0.0 && hi > lo && lm(hi - 1) <= null_rel * lm(0);
    cinfo[0] = hi - lo;
    if (eb) eb->N = 0;  // no second eigensolve unless the cluster is large (below)
  }
  __syncthreads();
  const int c = s_c, lo = s_lo;
  if (c < 2) return;
  for (int a = tid; a < c; a += nt) {
    const int ia = s_ord[lo + a];
    cinfo[1 + a] = ia;
    s_dg[a] = S[(int64_t)ia * N + ia] / XtX[(int64_t)ia * N + ia];
  }
  __syncthreads();
  if (tid == 0) {
    double mu = 0.0;
    for (int a = 0; a < c; ++a) mu += s_dg[a];
    s_mu = s_null ? 0.0 : mu / c;
  }
  __syncthreads();
  {  // scale: the largest |entry| of the shifted block (parallel max)
    double mx = 0.0;
    for (int e = tid; e < c * c; e += nt) {
      const int a = e / c, b = e % c;
      mx = fmax(mx, a == b ? fabs(s_dg[a] - s_mu) : fabs(S[(int64_t)s_ord[lo + a] * N + s_ord[lo + b]]));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) s_wmax[warp] = mx;
    __syncthreads();
    if (tid == 0) {
      double m = 0.0;
      for (int w = 0; w < nwarp; ++w) m = fmax(m, s_wmax[w]);
      s_scale = (m > 0.0 && isfinite(m)) ? m : 1.0;
    }
    __syncthreads();
  }
  const double inv = 1.0 / s_scale, mu = s_mu;
  if (c > CUT_CMAX) {
    // the block (FP64, c x c) into XtX, read by nothing else from here on; the eigensolver
    // writes its eigenvectors (V_c) into Vc and its eigenvalues after the descriptor
    for (int e = tid; e < c * c; e += nt) {
      const int a = e / c, b = e % c, ia = s_ord[lo + a], ib = s_ord[lo + b];
      XtX[e] = (a == b ? s_dg[a] - mu : 0.5 * (S[(int64_t)ia * N + ib] + S[(int64_t)ib * N + ia])) * inv;
    }
    if (tid == 0) {
      eb->A = XtX;
      eb->X = Vc;
      eb->lam = reinterpret_cast<double*>(cinfo) + CUT_LAM_OFF;
      eb->scratch = jscr;
      eb->noise_rel = s_null ? 1e-6f : 0.f;  // FP32 resolution of the unit-scaled block
      eb->N = c;
    }
    return;
  }
  const int lda = c | 1;
  float* T = cut_sm;
  float* V = cut_sm + c * lda;
  for (int e = tid; e < c * c; e += nt) {
    const int a = e / c, b = e % c, ia = s_ord[lo + a], ib = s_ord[lo + b];
    double t = 0.5 * (S[(int64_t)ia * N + ib] + S[(int64_t)ib * N + ia]);
    if (a == b) t = s_dg[a] - mu;
    T[a * lda + b] = (float)(t * inv);
    V[a * lda + b] = a == b ? 1.f : 0.f;
  }
  __syncthreads();
  const int cp = c + (c & 1), m = cp / 2;
  for (int sweep = 0; sweep < 30; ++sweep) {
    if (tid == 0) s_off = 0u;
    __syncthreads();
    for (int rnd = 0; rnd < cp - 1; ++rnd) {
      for (int k = tid; k < m; k += nt) {
        int a = k == 0 ? rnd : (rnd + k) % (cp - 1);
        int b = k == 0 ? cp - 1 : (rnd - k + (cp - 1)) % (cp - 1);
        const int p = min(a, b), q = max(a, b);
        float cs = 1.f, sn = 0.f;
        if (q < c) {
          const float apq = T[p * lda + q], app = T[p * lda + p], aqq = T[q * lda + q];
          atomicMax(&s_off, __float_as_uint(fabsf(apq)));
          if (fabsf(apq) > 1e-12f) {
            const float tau = (aqq - app) / (2.f * apq);
            const float t = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            cs = rsqrtf(1.f + t * t);
            sn = t * cs;
          }
        }
        s_p[k] = p;
        s_q[k] = q;
        s_cs[k] = cs;
        s_sn[k] = sn;
      }
      __syncthreads();
      for (int k = warp; k < m; k += nwarp) {  // columns p, q of T and V
        const float cs = s_cs[k], sn = s_sn[k];
        if (sn == 0.f) continue;
        const int p = s_p[k], q = s_q[k];
        for (int i = lane; i < c; i += 32) {
          float x = T[i * lda + p], y = T[i * lda + q];
          T[i * lda + p] = cs * x - sn * y;
          T[i * lda + q] = sn * x + cs * y;
          x = V[i * lda + p];
          y = V[i * lda + q];
          V[i * lda + p] = cs * x - sn * y;
          V[i * lda + q] = sn * x + cs * y;
        }
      }
      __syncthreads();
      for (int k = warp; k < m; k += nwarp) {  // rows p, q of T
        const float cs = s_cs[k], sn = s_sn[k];
        if (sn == 0.f) continue;
        const int p = s_p[k], q = s_q[k];
        for (int j = lane; j < c; j += 32) {
          const float x = T[p * lda + j], y = T[q * lda + j];
          T[p * lda + j] = (j == q) ? 0.f : cs * x - sn * y;
          T[q * lda + j] = (j == p) ? 0.f : sn * x + cs * y;
        }
      }
      __syncthreads();
    }
    const float off = __uint_as_float(s_off);
    __syncthreads();
    if (off < 1e-6f) break;
  }
  for (int e = tid; e < c * c; e += nt) Vc[e] = (double)V[(e / c) * lda + e % c];
}

__global__ __launch_bounds__(1024) void oa_cut_cluster_kernel(int N, int r, double* XtX,
                                                              const double* __restrict__ S,
                                                              const double* __restrict__ part, int nparts,
                                                              const double* __restrict__ lam,
                                                              double* __restrict__ Vc, int* __restrict__ cinfo,
                                                              float* jscr) {
  oa_cut_cluster_body(N, r, XtX, S, part, nparts, lam, Vc, cinfo, jscr, 0.0);
}

// X[:, idx] <- X[:, idx] V_c, one CTA per row of X.
__device__ __forceinline__ void cut_rotate_body(int N, double* __restrict__ X, const double* __restrict__ Vc,
                                                const int* __restrict__ cinfo, int i) {
  __shared__ double row[CUT_BIG_NMAX];
  const int c = cinfo[0];
  if (c < 2) return;
  for (int b = threadIdx.x; b < c; b += blockDim.x) row[b] = X[(int64_t)i * N + cinfo[1 + b]];
  __syncthreads();
  for (int a = threadIdx.x; a < c; a += blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < c; ++b) t += row[b] * Vc[(int64_t)b * c + a];
    X[(int64_t)i * N + cinfo[1 + a]] = t;
  }
}

__global__ __launch_bounds__(128) void cut_rotate_kernel(int N, double* __restrict__ X, const double* __restrict__ Vc,
                                                         const int* __restrict__ cinfo) {
  cut_rotate_body(N, X, Vc, cinfo, (int)blockIdx.x);
}

cudaError_t launch_oa_cut_cluster(int N, int r, double* X, const double* lam, double* work, int64_t work_elems,
                                  float* jscr, cudaStream_t st) {
  const int64_t nn = (int64_t)N * N;
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(128, cdiv(nn, 1024)));
  if (N > CUT_BIG_NMAX || work_elems < 4 * nn + 3 * nb + nn) return cudaErrorInvalidValue;
  double* XtX = work;
  int* cinfo = reinterpret_cast<int*>(work + nn);
  const double* S = work + 2 * nn;
  double* Vc = work + 3 * nn;
  const double* part = work + 4 * nn;
  const int cmax = std::min(N, CUT_CMAX);
  const size_t smem = (size_t)2 * cmax * (cmax | 1) * sizeof(float);
  // a fixed cap (the largest cluster block): concurrent launches must not lower it
  cudaFuncSetAttribute(oa_cut_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(2 * CUT_CMAX * (CUT_CMAX | 1) * sizeof(float)));
  oa_cut_cluster_kernel<<<1, 1024, smem, st>>>(N, r, XtX, S, part, nb, lam, Vc, cinfo, jscr);
  cudaError_t e = launched();
  if (e) return e;
  if (jscr && N > CUT_CMAX && (e = launch_eig_cut_big(work + nn, N, st))) return e;
  cut_rotate_kernel<<<N, 128, 0, st>>>(N, X, Vc, cinfo);
  return launched();
}

// ============================================================================
// Leading-r selection and the CS step.
// ============================================================================
// Sort key with a strict total order: NaN sorts below every number, ties by index,
// so the ranks below always form a permutation of 0..N-1.
__device__ __forceinline__ double sort_key(double x) { return isnan(x) ? -INFINITY : x; }

__device__ __forceinline__ void select_topr_body(const double* __restrict__ X, const double* __restrict__ lam, int N,
                                                 int r, double* __restrict__ Zr, int* __restrict__ order) {
  extern __shared__ int s_ord[];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < N; i += nt) {
    double li = sort_key(lam[i]);
    int rank = 0;
    for (int j = 0; j < N; ++j) {
      double lj = sort_key(lam[j]);
      rank += (lj > li) || (lj == li && j < i);
    }
    s_ord[min(max(rank, 0), N - 1)] = i;
  }
  __syncthreads();
  for (int i = tid; i < N; i += nt) order[i] = s_ord[i];
  for (int64_t e = tid; e < (int64_t)N * r; e += nt) {
    int row = (int)(e / r), t = (int)(e % r);
    int c = min(max(s_ord[t], 0), N - 1);
    Zr[e] = X[(int64_t)row * N + c];
  }
}

__global__ void select_topr_kernel(const double* __restrict__ X, const double* __restrict__ lam, int N,
                                   int r, double* __restrict__ Zr, int* __restrict__ order) {
  select_topr_body(X, lam, N, r, Zr, order);
}

cudaError_t launch_select_topr(const double* X, const double* lam, int N, int r, double* Zr, int* order,
                               cudaStream_t st) {
  select_topr_kernel<<<1, 512, (size_t)N * sizeof(int), st>>>(X, lam, N, r, Zr, order);
  return launched();
}

// alpha_i = ||U1[:, i]||, beta_i = ||U2[:, i]|| (U1 = Z1 W, U2 = Z2 W), normalised to
// alpha^2 + beta^2 = 1, sorted by alpha non-increasing (eq. (ab)).
__device__ __forceinline__ void cs_norms_body(const double* __restrict__ U1, int l1, const double* __restrict__ U2,
                                              int l2, int r, double* __restrict__ alpha, double* __restrict__ beta) {
  extern __shared__ double sab[];
  double* sa = sab;
  double* sb = sab + r;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < r; i += nt) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < l1; ++k) a = fma(U1[(int64_t)k * r + i], U1[(int64_t)k * r + i], a);
    for (int k = 0; k < l2; ++k) b = fma(U2[(int64_t)k * r + i], U2[(int64_t)k * r + i], b);
    double nn = sqrt(a + b);
    // a column of zero norm is no pair (the unused columns of a grouped adaptive solve):
    // marked -1, which sorts after every pair
    sa[i] = nn > 0.0 ? sqrt(a) / nn : -1.0;
    sb[i] = nn > 0.0 ? sqrt(b) / nn : -1.0;
  }
  __syncthreads();
  for (int i = tid; i < r; i += nt) {
    double ai = isnan(sa[i]) ? -1.0 : sa[i];
    int rank = 0;
    for (int j = 0; j < r; ++j) {
      double aj = isnan(sa[j]) ? -1.0 : sa[j];
      rank += (aj > ai) || (aj == ai && j < i);
    }
    rank = min(max(rank, 0), r - 1);
    alpha[rank] = sa[i];
    beta[rank] = sb[i];
  }
}

__global__ void cs_norms_kernel(const double* __restrict__ U1, int l1, const double* __restrict__ U2, int l2,
                                int r, double* __restrict__ alpha, double* __restrict__ beta) {
  cs_norms_body(U1, l1, U2, l2, r, alpha, beta);
}

cudaError_t launch_cs_norms(const double* U1, int l1, const double* U2, int l2, int r, double* alpha,
                            double* beta, cudaStream_t st) {
  cs_norms_kernel<<<1, 256, (size_t)2 * r * sizeof(double), st>>>(U1, l1, U2, l2, r, alpha, beta);
  return launched();
}


// ---------------------------------------------------------------------------
// GSVD factors (the recovery that follows Algorithm 2): the column order and scales first,
// with the same arithmetic and ranking as cs_norms_body, so that factor column c pairs with
// alpha[c], beta[c] of the solve.
// ---------------------------------------------------------------------------
__global__ void factor_prep_kernel(const double* __restrict__ U1, int l, int r, double* __restrict__ scr) {
  extern __shared__ double fsm[];
  double* sa = fsm;       // alpha of column i
  double* ua = fsm + r;   // 1 / ||Z1 w_i||
  double* ub = ua + r;    // 1 / ||Z2 w_i||
  double* un = ub + r;    // ||[Z1; Z2] w_i||
  const double* U2 = U1 + (int64_t)l * r;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < r; i += nt) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < l; ++k) a = fma(U1[(int64_t)k * r + i], U1[(int64_t)k * r + i], a);
    for (int k = 0; k < l; ++k) b = fma(U2[(int64_t)k * r + i], U2[(int64_t)k * r + i], b);
    const double nn = sqrt(a + b);
    sa[i] = nn > 0.0 ? sqrt(a) / nn : 0.0;
    ua[i] = a > 0.0 ? 1.0 / sqrt(a) : 0.0;
    ub[i] = b > 0.0 ? 1.0 / sqrt(b) : 0.0;
    un[i] = nn;
  }
  __syncthreads();
  // scr: perm (as doubles) | 1 / ||Z1 w|| | 1 / ||Z2 w|| | ||[Z1; Z2] w||, by rank
  for (int i = tid; i < r; i += nt) {
    const double ai = isnan(sa[i]) ? -1.0 : sa[i];
    int rank = 0;
    for (int j = 0; j < r; ++j) {
      const double aj = isnan(sa[j]) ? -1.0 : sa[j];
      rank += (aj > ai) || (aj == ai && j < i);
    }
    rank = min(max(rank, 0), r - 1);
    scr[rank] = (double)i;
    scr[r + rank] = ua[i];
    scr[2 * r + rank] = ub[i];
    scr[3 * r + rank] = un[i];
  }
}

// out[i][c] = sc[c] sum_j Q(i, j) Uh[j][perm[c]]: a thread per row, a grid row per column.  A cold
// path (gsvd_rand_factors, on request after a solve, never inside the timed solves): Q is re-read
// once per output column and, in the row-major layout, with a stride of lp elements between
// neighbouring threads; it costs O(M l r) strided loads, a small multiple of one solve's products.
template <typename T>
__global__ void factor_side_kernel(const T* __restrict__ Q, int64_t rs, int64_t cs, int64_t M, int l,
                                   const double* __restrict__ Uh, int r, const double* __restrict__ scr, int which,
                                   double* __restrict__ out, int64_t ldo) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (i >= M) return;
  const int src = (int)scr[c];
  const double sc = scr[(1 + which) * r + c];
  double s = 0.0;
  for (int j = 0; j < l; ++j) s = fma((double)Q[i * rs + (int64_t)j * cs], Uh[(int64_t)j * r + src], s);
  out[i * ldo + c] = sc * s;
}

// R[c][j] = nn[c] sum_k U1[k][perm[c]] S[k][j]: a thread per column of S, a grid row per row of R
template <typename T>
__global__ void factor_r_kernel(const double* __restrict__ U1, int L, int r, const double* __restrict__ scr,
                                const T* __restrict__ S, int64_t ldn, int64_t n, double* __restrict__ R, int64_t ldr) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (j >= n) return;
  const int src = (int)scr[c];
  double s = 0.0;
  for (int k = 0; k < L; ++k) s = fma(U1[(int64_t)k * r + src], (double)S[(int64_t)k * ldn + j], s);
  R[(int64_t)c * ldr + j] = scr[3 * r + c] * s;
}

template <typename T>
cudaError_t gsvd_factors_t(const T* Q1, int64_t rs1, int64_t cs1, int64_t M1, const T* Q2, int64_t rs2, int64_t cs2,
                           int64_t M2, int l, int r, const double* U1, const T* S, int64_t ldn, int64_t n, double* scr,
                           double* U, int64_t ldu, double* V, int64_t ldv, double* R, int64_t ldr, cudaStream_t st) {
  if (r < 1 || r > 65535 || l < 1) return cudaErrorInvalidValue;
  factor_prep_kernel<<<1, 256, (size_t)4 * r * sizeof(double), st>>>(U1, l, r, scr);
  int nl = 1;
  if (U) {
    factor_side_kernel<T><<<dim3((unsigned)cdiv(M1, 128), (unsigned)r), 128, 0, st>>>(Q1, rs1, cs1, M1, l, U1, r,
                                                                                      scr, 0, U, ldu);
    ++nl;
  }
  if (V) {
    factor_side_kernel<T><<<dim3((unsigned)cdiv(M2, 128), (unsigned)r), 128, 0, st>>>(
        Q2, rs2, cs2, M2, l, U1 + (int64_t)l * r, r, scr, 1, V, ldv);
    ++nl;
  }
  if (R) {
    factor_r_kernel<T><<<dim3((unsigned)cdiv(n, 128), (unsigned)r), 128, 0, st>>>(U1, 2 * l, r, scr, S, ldn, n, R,
                                                                                  ldr);
    ++nl;
  }
  return launched(nl);
}

cudaError_t launch_gsvd_factors(int tsize, const void* Q1, int64_t rs1, int64_t cs1, int64_t M1, const void* Q2,
                                int64_t rs2, int64_t cs2, int64_t M2, int l, int r, const double* U1,
                                const void* S, int64_t ldn, int64_t n, double* scr, double* U, int64_t ldu,
                                double* V, int64_t ldv, double* R, int64_t ldr, cudaStream_t st) {
  if (tsize == 8)
    return gsvd_factors_t<double>(static_cast<const double*>(Q1), rs1, cs1, M1, static_cast<const double*>(Q2), rs2,
                                  cs2, M2, l, r, U1, static_cast<const double*>(S), ldn, n, scr, U, ldu, V, ldv, R,
                                  ldr, st);
  if (tsize == 4)
    return gsvd_factors_t<float>(static_cast<const float*>(Q1), rs1, cs1, M1, static_cast<const float*>(Q2), rs2, cs2,
                                 M2, l, r, U1, static_cast<const float*>(S), ldn, n, scr, U, ldu, V, ldv, R, ldr, st);
  return cudaErrorInvalidValue;
}

// ============================================================================
// Comparative quantities (Section 1): theta, rho, P1, P2, D1, D2.
// ============================================================================
__device__ __forceinline__ void pair_at(const double* alpha, const double* beta, int r, int N,
                                        int pad_mode, int i, double& a, double& b) {
  if (pad_mode == 0) {
    if (i < r) {
      a = alpha[i];
      b = beta[i];
    } else {
      a = 0.0;
      b = 1.0;
    }
  } else {
    int off = N - r;
    if (i < off) {
      a = 1.0;
      b = 0.0;
    } else {
      a = alpha[i - off];
      b = beta[i - off];
    }
  }
}

__global__ __launch_bounds__(1024) void metrics_kernel(const double* __restrict__ alpha,
                                                       const double* __restrict__ beta, int r, int N,
                                                       int pad_mode, double* theta, double* rho,
                                                       double* P1, double* P2, double* D) {
  __shared__ double red[2][32];
  __shared__ double s_tot[2];
  const int tid = threadIdx.x, nt = blockDim.x;
  const double quarter_pi = 0.78539816339744830962;
  double sa = 0.0, sb = 0.0;
  for (int i = tid; i < N; i += nt) {
    double a, b;
    pair_at(alpha, beta, r, N, pad_mode, i, a, b);
    sa += a * a;
    sb += b * b;
    if (theta) theta[i] = atan2(a, b) - quarter_pi;
    if (rho) rho[i] = (b == 0.0) ? __longlong_as_double(0x7ff0000000000000ll) : a / b;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sa += __shfl_down_sync(0xffffffffu, sa, o);
    sb += __shfl_down_sync(0xffffffffu, sb, o);
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = sa;
    red[1][tid >> 5] = sb;
  }
  __syncthreads();
  if (tid == 0) {
    double ta = 0, tb = 0;
    for (int w = 0; w < (nt + 31) / 32; ++w) {
      ta += red[0][w];
      tb += red[1][w];
    }
    s_tot[0] = ta;
    s_tot[1] = tb;
  }
  __syncthreads();
  const double ta = s_tot[0], tb = s_tot[1];
  double h1 = 0.0, h2 = 0.0;
  for (int i = tid; i < N; i += nt) {
    double a, b;
    pair_at(alpha, beta, r, N, pad_mode, i, a, b);
    double p1 = ta > 0 ? a * a / ta : 0.0, p2 = tb > 0 ? b * b / tb : 0.0;
    if (P1) P1[i] = p1;
    if (P2) P2[i] = p2;
    if (p1 > 0) h1 += p1 * log(p1);
    if (p2 > 0) h2 += p2 * log(p2);
  }
  __syncthreads();
  for (int o = 16; o > 0; o >>= 1) {
    h1 += __shfl_down_sync(0xffffffffu, h1, o);
    h2 += __shfl_down_sync(0xffffffffu, h2, o);
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = h1;
    red[1][tid >> 5] = h2;
  }
  __syncthreads();
  if (tid == 0 && D) {
    double a = 0, b = 0;
    for (int w = 0; w < (nt + 31) / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    double lg = log((double)N);
    D[0] = -a / lg;
    D[1] = -b / lg;
  }
}

cudaError_t launch_metrics(const double* alpha, const double* beta, int r, int N, int pad_mode,
                           double* theta, double* rho, double* P1, double* P2, double* D,
                           cudaStream_t st) {
  metrics_kernel<<<1, 1024, 0, st>>>(alpha, beta, r, N, pad_mode, theta, rho, P1, P2, D);
  return launched();
}

// One warp: lane-strided partial sums, then a fixed shuffle tree (deterministic).
__global__ void residual_kernel(const double* gpart, int ng, const double* bpart, int nb, double* out) {
  const int lane = threadIdx.x;
  double g = 0.0, b = 0.0;
  for (int i = lane; i < ng; i += 32) g += gpart[i];
  for (int i = lane; i < nb; i += 32) b += bpart[i];
  for (int o = 16; o > 0; o >>= 1) {
    g += __shfl_xor_sync(0xffffffffu, g, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (lane == 0) *out = g > 0.0 ? sqrt(fmax(g - b, 0.0) / g) : 0.0;
}

cudaError_t launch_residual(const double* gpart, int ng, const double* bpart, int nb, double* out,
                            cudaStream_t st) {
  residual_kernel<<<1, 32, 0, st>>>(gpart, ng, bpart, nb, out);
  return launched();
}


// ============================================================================
// Batched forms for the compressed-pair GSVDs of a grouped solve: one launch
// per step for all pairs (tables in device memory, see kernels.h).
// ============================================================================
template <typename TA, typename TB, bool DF>
__global__ __launch_bounds__(256) void dgemm_b_kernel(const DgemmB* __restrict__ tab) {
  const DgemmB& g = tab[blockIdx.z];
  const int i0 = blockIdx.x * SG_T, j0 = blockIdx.y * SG_T;
  if (i0 >= g.Mr || j0 >= g.Nc) return;
  // symmetric result: the upper tiles only, mirrored on the way out
  if (g.sym && blockIdx.x > blockIdx.y) return;
  __shared__ double As[SG_BK][SG_T + 1];
  __shared__ double Bs[SG_BK][SG_T + 1];
  const TA* __restrict__ A = static_cast<const TA*>(g.A);
  const TB* __restrict__ B = static_cast<const TB*>(g.B);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int K = g.K, ta = g.ta, tb = g.tb;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  float dh[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, dl[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int k0 = 0; k0 < K; k0 += SG_BK) {
    for (int e = tid; e < SG_T * SG_BK; e += 256) {
      const int a = e / 32, b = e % 32;
      int i, kk;
      if (!ta) { i = a; kk = b; } else { kk = a; i = b; }
      int gi = i0 + i, gk = k0 + kk;
      sg_put<DF>(&As[kk][i], (gi < g.Mr && gk < K) ? (ta ? A[(int64_t)gk * g.lda + gi] : A[(int64_t)gi * g.lda + gk])
                                                  : TA(0));
      int j;
      if (!tb) { kk = a; j = b; } else { j = a; kk = b; }
      const int gj = j0 + j;
      gk = k0 + kk;
      sg_put<DF>(&Bs[kk][j], (gj < g.Nc && gk < K) ? (tb ? B[(int64_t)gj * g.ldb + gk] : B[(int64_t)gk * g.ldb + gj])
                                                  : TB(0));
    }
    __syncthreads();
    // threads whose rows and columns all lie past the edge skip the arithmetic (the SM's
    // FP64 units, ~1/64 of its FP32 rate, then go to the threads with real outputs)
    if (i0 + ty * 2 < g.Mr && j0 + tx * 2 < g.Nc) sg_tile<DF>(As, Bs, min(SG_BK, K - k0), ty, tx, acc, dh, dl);
    __syncthreads();
  }
  for (int m = 0; m < 2; ++m)
    for (int q = 0; q < 2; ++q) {
      const int i = i0 + ty * 2 + m, j = j0 + tx * 2 + q;
      if (i < g.Mr && j < g.Nc) {
        double* c = g.C + (int64_t)i * g.ldc + j;
        const double r = sg_out<DF>(acc, dh, dl, m, q);
        const double v = g.beta == 0.0 ? g.alpha * r : g.alpha * r + g.beta * (*c);
        *c = v;
        if (g.sym && blockIdx.x < blockIdx.y) g.C[(int64_t)j * g.ldc + i] = v;
      }
    }
}

// The double-float form of the batched product: the same 32 x 32 output tiles, 64 threads with
// 4 x 4 outputs each (rows 4 ty .. 4 ty + 3, columns 4 tx .. 4 tx + 3), the operands staged as
// (hi, lo) FP32 pairs in rows padded to 16-byte multiples so that each thread reads its four A
// and four B pairs of a k with four 16-byte loads (a 2 x 2 register tile needs one load per
// product; the 4 x 4 tile, one per four).  Each output is the same double-float chain over k as
// in dgemm_b_kernel<.., true> (df_fma per k, renormalised after each 32-k stage).
constexpr int DF_T = 32, DF_BK = 32, DF_THREADS = 64, DF_LD = DF_T + 2;
static_assert(DF_T == SG_T, "the double-float tiles share the grid of dgemm_b_kernel");
template <typename T>
__device__ __forceinline__ float2 df_split(T v) {
  if constexpr (std::is_same<T, float>::value) {
    return make_float2(v, 0.f);
  } else if constexpr (std::is_same<T, float2>::value) {
    return v;  // already a (hi, lo) pair
  } else {
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - (double)h));
  }
}
template <typename T>
__device__ __forceinline__ T df_zero() {
  if constexpr (std::is_same<T, float2>::value)
    return make_float2(0.f, 0.f);
  else
    return T(0);
}
// LOW: plain FP32 products of the operands' high parts (the Ogita-Aishima increment X F, whose
// entries are of the size of the current error: FP32's relative 6e-8 of an increment of 1e-7 is
// far below what the next step corrects).
template <typename TA, typename TB, bool LOW>
__global__ __launch_bounds__(DF_THREADS) void dfgemm_b_kernel(const DgemmB* __restrict__ tab) {
  const DgemmB& g = tab[blockIdx.z];
  const int i0 = blockIdx.x * DF_T, j0 = blockIdx.y * DF_T;
  if (i0 >= g.Mr || j0 >= g.Nc) return;
  if (g.sym && blockIdx.x > blockIdx.y) return;  // symmetric result: upper tiles, mirrored
  __shared__ __align__(16) float2 As[DF_BK][DF_LD];
  __shared__ __align__(16) float2 Bs[DF_BK][DF_LD];
  const TA* __restrict__ A = static_cast<const TA*>(g.A);
  const TB* __restrict__ B = static_cast<const TB*>(g.B);
  const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
  const int K = g.K, ta = g.ta, tb = g.tb;
  const bool active = i0 + 4 * ty < g.Mr && j0 + 4 * tx < g.Nc;
  float sh[4][4], sl[4][4];
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int q = 0; q < 4; ++q) sh[m][q] = sl[m][q] = 0.f;
  for (int k0 = 0; k0 < K; k0 += DF_BK) {
    for (int e = tid; e < DF_T * DF_BK; e += DF_THREADS) {
      const int a = e / 32, b = e % 32;  // consecutive threads along the contiguous index
      int i, kk;
      if (!ta) { i = a; kk = b; } else { kk = a; i = b; }
      int gi = i0 + i, gk = k0 + kk;
      As[kk][i] = df_split((gi < g.Mr && gk < K) ? (ta ? A[(int64_t)gk * g.lda + gi] : A[(int64_t)gi * g.lda + gk])
                                                : df_zero<TA>());
      int j;
      if (!tb) { kk = a; j = b; } else { j = a; kk = b; }
      const int gj = j0 + j;
      gk = k0 + kk;
      Bs[kk][j] = df_split((gj < g.Nc && gk < K) ? (tb ? B[(int64_t)gj * g.ldb + gk] : B[(int64_t)gk * g.ldb + gj])
                                                : df_zero<TB>());
    }
    __syncthreads();
    if (active) {
      const int kend = min(DF_BK, K - k0);
#pragma unroll 2
      for (int kk = 0; kk < kend; ++kk) {
        const float4 a01 = *reinterpret_cast<const float4*>(&As[kk][4 * ty]);
        const float4 a23 = *reinterpret_cast<const float4*>(&As[kk][4 * ty + 2]);
        const float4 b01 = *reinterpret_cast<const float4*>(&Bs[kk][4 * tx]);
        const float4 b23 = *reinterpret_cast<const float4*>(&Bs[kk][4 * tx + 2]);
        const float2 av[4] = {make_float2(a01.x, a01.y), make_float2(a01.z, a01.w), make_float2(a23.x, a23.y),
                              make_float2(a23.z, a23.w)};
        const float2 bv[4] = {make_float2(b01.x, b01.y), make_float2(b01.z, b01.w), make_float2(b23.x, b23.y),
                              make_float2(b23.z, b23.w)};
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (LOW)
              sh[m][q] = fmaf(av[m].x, bv[q].x, sh[m][q]);
            else
              df_fma(av[m], bv[q], sh[m][q], sl[m][q]);
          }
      }
      if (!LOW) {
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
          for (int q = 0; q < 4; ++q) df_renorm(sh[m][q], sl[m][q]);
      }
    }
    __syncthreads();
  }
  if (!active) return;
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + 4 * ty + m, j = j0 + 4 * tx + q;
      if (i < g.Mr && j < g.Nc) {
        double* c = g.C + (int64_t)i * g.ldc + j;
        const double r = (double)sh[m][q] + (double)sl[m][q];
        const double v = g.beta == 0.0 ? g.alpha * r : g.alpha * r + g.beta * (*c);
        *c = v;
        if (g.sym && blockIdx.x < blockIdx.y) g.C[(int64_t)j * g.ldc + i] = v;
      }
    }
}

template <typename TA, typename TB>
cudaError_t launch_dgemm_b(const DgemmB* tab, int nprob, int max_Mr, int max_Nc, cudaStream_t st, int df) {
  if (nprob <= 0) return cudaSuccess;
  const dim3 grid((unsigned)cdiv(max_Mr, SG_T), (unsigned)cdiv(max_Nc, SG_T), (unsigned)nprob);
  if (df == 2)
    dfgemm_b_kernel<TA, TB, true><<<grid, DF_THREADS, 0, st>>>(tab);
  else if (df)
    dfgemm_b_kernel<TA, TB, false><<<grid, DF_THREADS, 0, st>>>(tab);
  else
    dgemm_b_kernel<TA, TB, false><<<grid, 256, 0, st>>>(tab);
  return launched();
}
template cudaError_t launch_dgemm_b<float, float>(const DgemmB*, int, int, int, cudaStream_t, int);
template cudaError_t launch_dgemm_b<double, double>(const DgemmB*, int, int, int, cudaStream_t, int);

// The refinement's operands as (hi, lo) FP32 pairs, converted once per product instead of in
// every tile that loads them (FP64 conversions run at the FP64 rate: each N x N operand is loaded
// by N / 32 tiles).  which: 0 A, 1 X, 2 P, 3 F.
__global__ void oa_to_df_b_kernel(const OaB* __restrict__ tab, int which) {
  const OaB& o = tab[blockIdx.y];
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)o.N * o.N) return;
  const double* src = which == 0 ? o.A : which == 1 ? o.X : which == 2 ? o.P : o.F;
  float2* dst = which == 0 ? o.Adf : which == 1 ? o.Xdf : which == 2 ? o.Pdf : o.Fdf;
  const double v = src[e];
  const float h = __double2float_rn(v);
  dst[e] = make_float2(h, __double2float_rn(v - (double)h));
}

// Frobenius sums of A, R = I - X^T X and S - diag(lam) (part[0..2]) and lam, one CTA per problem.
__global__ __launch_bounds__(256) void oa_norms_b_kernel(const OaB* __restrict__ tab) {
  const OaB& o = tab[blockIdx.x];
  __shared__ double red[3][8];
  const int N = o.N;
  const int64_t nn = (int64_t)N * N;
  double a2 = 0.0, r2 = 0.0, s2 = 0.0;
  for (int64_t e = threadIdx.x; e < nn; e += blockDim.x) {
    const int i = (int)(e / N), j = (int)(e % N);
    const double a = o.A[e];
    const double r = (i == j ? 1.0 : 0.0) - o.XtX[e];
    double sd = o.S[e];
    if (i == j) sd -= o.S[e] / o.XtX[e];
    a2 += a * a;
    r2 += r * r;
    s2 += sd * sd;
  }
  for (int off = 16; off > 0; off >>= 1) {
    a2 += __shfl_down_sync(0xffffffffu, a2, off);
    r2 += __shfl_down_sync(0xffffffffu, r2, off);
    s2 += __shfl_down_sync(0xffffffffu, s2, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a2;
    red[1][threadIdx.x >> 5] = r2;
    red[2][threadIdx.x >> 5] = s2;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
    o.part[threadIdx.x] = t;
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) o.lam[i] = o.S[(int64_t)i * N + i] / o.XtX[(int64_t)i * N + i];
}

// F as in oa_form_kernel, delta from the three sums.
__global__ void oa_form_b_kernel(const OaB* __restrict__ tab) {
  const OaB& o = tab[blockIdx.z];
  const int N = o.N;
  const int64_t nn = (int64_t)N * N;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nn) return;
  const double delta = 2.0 * (sqrt(o.part[2]) + sqrt(o.part[0]) * sqrt(o.part[1]));
  const int i = (int)(e / N), j = (int)(e % N);
  const double r = (i == j ? 1.0 : 0.0) - o.XtX[e];
  double f;
  if (i == j) {
    f = 0.5 * r;
  } else {
    const double d = o.lam[j] - o.lam[i];
    f = (fabs(d) > delta) ? (o.S[e] + o.lam[j] * r) / d : 0.5 * r;
  }
  o.F[e] = f;
}

// X += P (P = X F of the step).
__global__ void oa_update_b_kernel(const OaB* __restrict__ tab) {
  const OaB& o = tab[blockIdx.z];
  const int64_t nn = (int64_t)o.N * o.N;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nn) o.X[e] += o.P[e];
}

void oa_b_tables(const OaB* h, int nprob, DgemmB* dg) {
  for (int i = 0; i < nprob; ++i) {
    const OaB& o = h[i];
    const int N = o.N;
    auto mk = [&](const void* A, int ta, const void* B, int tb, double* C) {
      DgemmB g;
      memset(&g, 0, sizeof(g));
      g.A = A;
      g.B = B;
      g.C = C;
      g.lda = g.ldb = g.ldc = N;
      g.alpha = 1.0;
      g.beta = 0.0;
      g.Mr = g.Nc = g.K = N;
      g.ta = ta;
      g.tb = tb;
      return g;
    };
    // double-float form (o.Xdf set): the operands are the (hi, lo) pair copies
    const bool d2 = o.Xdf != nullptr;
    const void* X = d2 ? (const void*)o.Xdf : (const void*)o.X;
    dg[i] = mk(X, 1, X, 0, o.XtX);                   // X^T X (symmetric)
    dg[i].sym = 1;
    dg[nprob + i] = mk(d2 ? (const void*)o.Adf : (const void*)o.A, 0, X, 0, o.P);  // A X
    dg[2 * nprob + i] = mk(X, 1, d2 ? (const void*)o.Pdf : (const void*)o.P, 0, o.S);  // X^T (A X) (symmetric: A is)
    dg[2 * nprob + i].sym = 1;
    dg[3 * nprob + i] = mk(X, 0, d2 ? (const void*)o.Fdf : (const void*)o.F, 0, o.P);  // X F
  }
}

cudaError_t launch_oa_refine_b(const OaB* tab, const DgemmB* dg, int nprob, int max_N, cudaStream_t st, bool df) {
  if (nprob <= 0) return cudaSuccess;
  cudaError_t e;
  const dim3 g2((unsigned)cdiv((int64_t)max_N * max_N, 256), 1, (unsigned)nprob);
  const dim3 gc((unsigned)cdiv((int64_t)max_N * max_N, 256), (unsigned)nprob);
  const dim3 gd((unsigned)cdiv(max_N, SG_T), (unsigned)cdiv(max_N, SG_T), (unsigned)nprob);
  if (df) {
    // operands converted once to (hi, lo) pairs (oa_b_tables points the products at them)
    for (int w = 0; w < 2; ++w) {
      oa_to_df_b_kernel<<<gc, 256, 0, st>>>(tab, w);
      if ((e = launched())) return e;
    }
    for (int k = 0; k < 2; ++k) {
      dfgemm_b_kernel<float2, float2, false><<<gd, DF_THREADS, 0, st>>>(dg + (int64_t)k * nprob);
      if ((e = launched())) return e;
    }
    oa_to_df_b_kernel<<<gc, 256, 0, st>>>(tab, 2);
    if ((e = launched())) return e;
    dfgemm_b_kernel<float2, float2, false><<<gd, DF_THREADS, 0, st>>>(dg + 2ll * nprob);
    if ((e = launched())) return e;
  } else {
    for (int k = 0; k < 3; ++k)
      if ((e = launch_dgemm_b<double, double>(dg + (int64_t)k * nprob, nprob, max_N, max_N, st, 0))) return e;
  }
  oa_norms_b_kernel<<<nprob, 256, 0, st>>>(tab);
  if ((e = launched())) return e;
  oa_form_b_kernel<<<g2, 256, 0, st>>>(tab);
  if ((e = launched())) return e;
  // the increment X F: FP32 products on the mixed paths (its entries are of the error's size)
  if (df) {
    oa_to_df_b_kernel<<<gc, 256, 0, st>>>(tab, 3);
    if ((e = launched())) return e;
    dfgemm_b_kernel<float2, float2, true><<<gd, DF_THREADS, 0, st>>>(dg + 3ll * nprob);
    if ((e = launched())) return e;
  } else if ((e = launch_dgemm_b<double, double>(dg + 3ll * nprob, nprob, max_N, max_N, st, 0))) {
    return e;
  }
  oa_update_b_kernel<<<g2, 256, 0, st>>>(tab);
  return launched();
}

// Cut cluster of each problem (XtX and S of the step just taken; V_c in F, the
// cluster's indices in P), then the rotation of its columns of X.
__global__ __launch_bounds__(1024) void oa_cut_cluster_b_kernel(const OaB* __restrict__ tab) {
  const OaB& o = tab[blockIdx.x];
  // grouped solves run FP32 data only: eigenvalues below 1e-12 of the largest (singular values
  // below 1e-6 of the stack's) are beyond what those bases resolve
  oa_cut_cluster_body(o.N, o.r, o.XtX, o.S, o.part, 1, o.lam, o.F, reinterpret_cast<int*>(o.P), o.jscr, 1e-12);
}
__global__ __launch_bounds__(128) void cut_rotate_b_kernel(const OaB* __restrict__ tab) {
  const OaB& o = tab[blockIdx.z];
  if ((int)blockIdx.x >= o.N) return;
  cut_rotate_body(o.N, o.X, o.F, reinterpret_cast<const int*>(o.P), (int)blockIdx.x);
}

cudaError_t launch_oa_cut_cluster_b(const OaB* tab, int nprob, int max_N, cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  if (max_N > 512) return cudaErrorInvalidValue;
  const int cmax = std::min(max_N, CUT_CMAX);
  const size_t smem = (size_t)2 * cmax * (cmax | 1) * sizeof(float);
  cudaFuncSetAttribute(oa_cut_cluster_b_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(2 * CUT_CMAX * (CUT_CMAX | 1) * sizeof(float)));
  oa_cut_cluster_b_kernel<<<nprob, 1024, smem, st>>>(tab);
  cudaError_t e = launched();
  if (e) return e;
  if (max_N > CUT_CMAX && (e = launch_eig_cut_big_b(tab, nprob, max_N, st))) return e;
  cut_rotate_b_kernel<<<dim3((unsigned)max_N, 1, (unsigned)nprob), 128, 0, st>>>(tab);
  return launched();
}

__global__ void select_topr_b_kernel(const SelB* __restrict__ tab) {
  const SelB& a = tab[blockIdx.x];
  select_topr_body(a.X, a.lam, a.N, a.r, a.Zr, a.order);
}

cudaError_t launch_select_topr_b(const SelB* tab, int nprob, int max_N, cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  select_topr_b_kernel<<<nprob, 512, (size_t)max_N * sizeof(int), st>>>(tab);
  return launched();
}

__global__ void cs_norms_b_kernel(const CsB* __restrict__ tab) {
  const CsB& a = tab[blockIdx.x];
  cs_norms_body(a.U1, a.l1, a.U2, a.l2, a.r, a.alpha, a.beta);
}

cudaError_t launch_cs_norms_b(const CsB* tab, int nprob, int max_r, cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  cs_norms_b_kernel<<<nprob, 256, (size_t)2 * max_r * sizeof(double), st>>>(tab);
  return launched();
}

__global__ void residual_b_kernel(const ResidB* __restrict__ tab, int nprob) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nprob) return;
  const ResidB& a = tab[i];
  double g = 0.0, b = 0.0;
  for (int t = 0; t < a.ng; ++t) g += a.gpart[t];
  for (int t = 0; t < a.nb; ++t) b += a.bpart[t];
  *a.out = g > 0.0 ? sqrt(fmax(g - b, 0.0) / g) : 0.0;
}

cudaError_t launch_residual_b(const ResidB* tab, int nprob, cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  residual_b_kernel<<<(unsigned)cdiv(nprob, 128), 128, 0, st>>>(tab, nprob);
  return launched();
}

__global__ void scatter_b_kernel(const ScatterB* __restrict__ tab) {
  const ScatterB& a = tab[blockIdx.x];
  for (int i = threadIdx.x; i < a.count; i += blockDim.x) a.dst[i] = a.src[i];
}

cudaError_t launch_scatter_b(const ScatterB* tab, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  scatter_b_kernel<<<n, 128, 0, st>>>(tab);
  return launched();
}

}  // namespace gsvdr
