// All eigenpairs of a small symmetric matrix in FP32, one CTA: the start that
// the FP64 Ogita-Aishima refinement of the compressed-pair GSVD lifts to FP64.
//
//   1. Householder tridiagonalisation T = Q^T A Q (Golub & Van Loan, Alg. 8.3.1),
//      the matrix-vector product one warp per row;
//   2. every eigenvalue of T by Sturm-count bisection, one thread each;
//   3. its eigenvector of T from the twisted factorisation of T - lambda I
//      (stationary L D L^T from the top, U D U^T from the bottom, twist index
//      at the smallest |gamma_k|; Dhillon & Parlett, Lin. Alg. Appl. 387, 2004),
//      one thread each, rescaled on the fly against overflow;
//   4. back-transformation X = Q Z, one warp per column;
//   5. two-pass modified Gram-Schmidt: the columns that are numerically
//      dependent (eigenvectors of a tight cluster) are set aside in the first
//      pass and replaced in the second by pseudo-random vectors orthogonalised
//      against all the others, so they span the cluster's invariant subspace.
#include <algorithm>

#include "kernels.h"

namespace gsvdr {

namespace {

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum; every thread receives the total.
__device__ float block_sum_f(float v, float* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, ln = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (ln == 0) red[w] = v;
  __syncthreads();
  float s = 0.f;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

// Block max; every thread receives the result.
__device__ float block_max_f(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, ln = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (ln == 0) red[w] = v;
  __syncthreads();
  float m = 0.f;
  for (int i = 0; i < nw; ++i) m = fmaxf(m, red[i]);
  return m;
}

// Columns whose largest entry is below this (in a matrix scaled to unit size) are taken as
// zero by the reflectors: their squares would fall into the denormal range.
constexpr float NRM_TINY = 1e-36f;

// sqrt(sum_i x(i)^2) for i = i0, i0 + 1, .. N - 1 over one warp (lane t), scaled by the largest
// |x(i)| before squaring (as the reference BLAS nrm2 scales), so that a column of tiny entries
// (the rounding-level rows of a nearly singular matrix) keeps the relative accuracy of its
// norm: unscaled, squares below 1e-38 turn denormal or vanish, the norm no longer matches the
// entries, and a reflector built from it is not orthogonal.  Returns 0 for a column whose
// largest entry is below NRM_TINY, NaN or inf when an entry is.
template <typename F>
__device__ __forceinline__ float warp_nrm2(int i0, int N, int t, F x) {
  float mx = 0.f;
  bool bad = false;
  for (int i = i0 + t; i < N; i += 32) {
    const float a = fabsf(x(i));
    bad = bad || !(a <= 3.0e38f);
    mx = fmaxf(mx, a);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (__any_sync(0xffffffffu, bad)) return __int_as_float(0x7fc00000);
  if (!(mx >= NRM_TINY)) return 0.f;
  const float sc = 1.f / mx;
  float sg = 0.f;
  for (int i = i0 + t; i < N; i += 32) {
    const float y = x(i) * sc;
    sg = fmaf(y, y, sg);
  }
  for (int o = 16; o > 0; o >>= 1) sg += __shfl_xor_sync(0xffffffffu, sg, o);
  return mx * sqrtf(sg);
}

// Number of eigenvalues of T (d, e2 = e^2) smaller than x.
__device__ int sturm_count(const float* d, const float* e2, int N, float x, float pivmin) {
  int c = 0;
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  c += q < 0.f;
  for (int i = 1; i < N; ++i) {
    q = d[i] - x - e2[i - 1] / q;
    if (fabsf(q) < pivmin) q = -pivmin;
    c += q < 0.f;
  }
  return c;
}

__device__ __forceinline__ float hash_unit(uint32_t a, uint32_t b) {
  uint32_t h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  h *= 0x297A2D39u;
  h ^= h >> 15;
  return (float)(h >> 8) * 5.9604645e-08f - 0.5f;
}

// A replacement for set-aside vector j of eigenvalue lambda_j: one step of inverse iteration
// on T - lambda_j I from a pseudo-random start (one thread).  T - lambda I = U D U^T with the
// backward pivots dm (dm_{N-1} = d_{N-1} - lambda, dm_i = d_i - lambda - e_i^2 / dm_{i+1}),
// U unit upper bidiagonal with U_{i,i+1} = e_i / dm_{i+1}: U y = b from the bottom, then
// x_0 = y_0 / dm_0, x_{i+1} = (y_{i+1} - e_i x_i) / dm_{i+1}.  The result lies, to the gap
// ratio, in T's eigenspace at lambda_j, so the vectors set aside from an exactly multiple
// eigenvalue are replaced within their own eigenspace.  Values growing past 2^60 rescale the
// whole vector (the same system with a scaled right-hand side).  A non-finite result falls
// back to the pseudo-random start itself.  x has stride xs.
// from_x: the right-hand side is x itself (a further step of inverse iteration on a vector from
// which the accepted columns were projected out: the step amplifies the missing eigenvector
// of the cluster, where a first step from a random start is dominated by an accepted one).
__device__ void inverse_iteration_start(const float* __restrict__ e, const float* __restrict__ dm, int N,
                                        uint32_t j, float* x, int64_t xs, bool from_x = false) {
  if (!from_x) x[(int64_t)(N - 1) * xs] = hash_unit(j, (uint32_t)(N - 1));
  for (int i = N - 2; i >= 0; --i) {
    const float rhs = from_x ? x[(int64_t)i * xs] : hash_unit(j, (uint32_t)i);
    float y = rhs - (e[i] / dm[i + 1]) * x[(int64_t)(i + 1) * xs];
    if (fabsf(y) > 1.15e18f) {
      for (int u = i + 1; u < N; ++u) x[(int64_t)u * xs] *= 8.67e-19f;
      y *= 8.67e-19f;
    }
    x[(int64_t)i * xs] = y;
  }
  float xv = x[0] / dm[0];
  x[0] = xv;
  bool ok = isfinite(xv);
  for (int i = 0; i + 1 < N; ++i) {
    xv = (x[(int64_t)(i + 1) * xs] - e[i] * xv) / dm[i + 1];
    if (fabsf(xv) > 1.15e18f) {
      for (int u = 0; u < N; ++u) x[(int64_t)u * xs] *= 8.67e-19f;
      xv *= 8.67e-19f;
    }
    x[(int64_t)(i + 1) * xs] = xv;
    ok = ok && isfinite(xv);
  }
  if (!ok)
    for (int i = 0; i < N; ++i) x[(int64_t)i * xs] = hash_unit(j, (uint32_t)i);
}

}  // namespace

int64_t eig_big_scratch_floats(int N);
int64_t eig_scratch_floats(int N) {
  const int lda = N | 1;
  return std::max<int64_t>(2ll * N * lda + 8ll * N + 2ll * N * N, eig_big_scratch_floats(N));
}

__global__ __launch_bounds__(1024) void eig_f32_kernel(const double* __restrict__ Ain, int N,
                                                       double* __restrict__ Xout, double* __restrict__ lam,
                                                       float* __restrict__ gscr, int use_smem) {
  extern __shared__ float sm[];
  __shared__ float red[32];
  __shared__ float s_scale, s_bound[2];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarp = nt >> 5;
  const int lda = N | 1;  // odd stride: column walks are bank-conflict free
  float* base = use_smem ? sm : gscr;
  float* A = base;                       // N x lda: A, then the reflectors; later scratch
  float* Z = A + (int64_t)N * lda;       // N x lda: eigenvectors (column j)
  float* d = Z + (int64_t)N * lda;       // N
  float* e = d + N;                      // N
  float* e2 = e + N;                     // N
  float* beta = e2 + N;                  // N
  float* v = beta + N;                   // N  (reflector / projection coefficients)
  float* p = v + N;                      // N
  float* cf = p + N;                     // N  (MGS coefficients)
  float* nrm = cf + N;                   // N  (column flags)
  float* LU = use_smem ? gscr : base + 2ll * N * lda + 8ll * N;  // 2 N x N per-thread pivots

  if (tid == 0) {
    double mx = 0.0;
    for (int i = 0; i < N; ++i) mx = fmax(mx, fabs(Ain[(int64_t)i * N + i]));
    s_scale = (float)(mx > 0.0 && isfinite(mx) ? mx : 1.0);
  }
  __syncthreads();
  const float inv = 1.0f / s_scale;
  for (int i = warp; i < N; i += nwarp)
    for (int j = lane; j < N; j += 32) A[(int64_t)i * lda + j] = (float)(Ain[(int64_t)i * N + j] * (double)inv);
  __syncthreads();

  // ---- 1. tridiagonalisation: reflector k zeroes A[k+2:, k] ------------------
  for (int k = 0; k + 2 < N; ++k) {
    const int m = N - k - 1;
    const float x0 = A[(int64_t)(k + 1) * lda + k];
    float amax = 0.f;
    for (int i = tid; i < m; i += nt) amax = fmaxf(amax, fabsf(A[(int64_t)(k + 1 + i) * lda + k]));
    const float mx = block_max_f(amax, red);  // scaled sum of squares (see warp_nrm2)
    const float isc = mx >= NRM_TINY ? 1.f / mx : 0.f;
    float part = 0.f;
    for (int i = tid; i < m; i += nt) {
      const float xi = A[(int64_t)(k + 1 + i) * lda + k] * isc;
      part += xi * xi;
    }
    const float sig2 = block_sum_f(part, red);
    const float sig = mx >= NRM_TINY ? mx * sqrtf(sig2) : (isfinite(sig2) ? 0.f : sig2);
    const float alpha = x0 >= 0.f ? -sig : sig;  // H x = alpha e1
    // normalised reflector (v_0 = 1, tau in [1, 2]): bounded for any scale of the column
    const bool refl = sig > 0.f && isfinite(sig);
    const float bk = refl ? (alpha - x0) / alpha : 0.f;
    const float vs = refl ? 1.f / (x0 - alpha) : 0.f;
    for (int i = tid; i < m; i += nt) v[i] = (i == 0) ? 1.f : A[(int64_t)(k + 1 + i) * lda + k] * vs;
    if (tid == 0) {
      beta[k] = bk;
      e[k] = (bk > 0.f) ? alpha : x0;
    }
    __syncthreads();
    if (bk > 0.f) {
      // p = bk A22 v, one warp per row
      for (int i = warp; i < m; i += nwarp) {
        const float* ai = A + (int64_t)(k + 1 + i) * lda + (k + 1);
        float s = 0.f;
        for (int j = lane; j < m; j += 32) s = fmaf(ai[j], v[j], s);
        s = warp_sum(s);
        if (lane == 0) p[i] = bk * s;
      }
      __syncthreads();
      float pv = 0.f;
      for (int i = tid; i < m; i += nt) pv += p[i] * v[i];
      const float kk = 0.5f * bk * block_sum_f(pv, red);
      for (int i = tid; i < m; i += nt) p[i] -= kk * v[i];  // p := w = p - (bk/2)(p^T v) v
      __syncthreads();
      for (int i = warp; i < m; i += nwarp) {
        float* ai = A + (int64_t)(k + 1 + i) * lda + (k + 1);
        const float vi = v[i], wi = p[i];
        for (int j = lane; j < m; j += 32) ai[j] -= vi * p[j] + wi * v[j];
      }
    }
    // keep the reflector in column k below the diagonal
    for (int i = tid; i < m; i += nt) A[(int64_t)(k + 1 + i) * lda + k] = v[i];
    __syncthreads();
  }
  for (int i = tid; i < N; i += nt) d[i] = A[(int64_t)i * lda + i];
  if (tid == 0) {
    if (N >= 2) e[N - 2] = A[(int64_t)(N - 1) * lda + (N - 2)];
    for (int k = (N >= 2 ? N - 2 : 0); k < N; ++k) beta[k] = 0.f;
  }
  __syncthreads();
  for (int i = tid; i < N - 1; i += nt) e2[i] = e[i] * e[i];
  if (tid == 0) {
    float lo = d[0], hi = d[0];
    for (int i = 0; i < N; ++i) {
      float rad = (i > 0 ? fabsf(e[i - 1]) : 0.f) + (i < N - 1 ? fabsf(e[i]) : 0.f);
      lo = fminf(lo, d[i] - rad);
      hi = fmaxf(hi, d[i] + rad);
    }
    float pad = 1e-6f * fmaxf(fabsf(lo), fabsf(hi)) + 1e-30f;
    s_bound[0] = lo - pad;
    s_bound[1] = hi + pad;
  }
  __syncthreads();
  const float tnorm = fmaxf(fabsf(s_bound[0]), fabsf(s_bound[1]));
  const float pivmin = fmaxf(1e-30f, 1e-12f * tnorm);
  const float atol = 4.f * 5.96e-8f * tnorm;

  // ---- 2 + 3. eigenvalue j (ascending) and its tridiagonal eigenvector -------
  for (int j = tid; j < N; j += nt) {
    float lo = s_bound[0], hi = s_bound[1];
    for (int it = 0; it < 64; ++it) {
      const float mid = 0.5f * (lo + hi);
      if (mid <= lo || mid >= hi || hi - lo <= atol) break;
      if (sturm_count(d, e2, N, mid, pivmin) > j)
        hi = mid;
      else
        lo = mid;
    }
    const float lm = 0.5f * (lo + hi);
    lam[j] = (double)lm * (double)s_scale;
    float* L = LU + (int64_t)j * N;
    float* U = LU + (int64_t)N * N + (int64_t)j * N;
    float dp = d[0] - lm;
    if (fabsf(dp) < pivmin) dp = -pivmin;
    L[0] = dp;
    for (int i = 0; i + 1 < N; ++i) {
      dp = d[i + 1] - lm - (e[i] / dp) * e[i];
      if (fabsf(dp) < pivmin) dp = -pivmin;
      L[i + 1] = dp;
    }
    float dm = d[N - 1] - lm;
    if (fabsf(dm) < pivmin) dm = -pivmin;
    U[N - 1] = dm;
    for (int i = N - 2; i >= 0; --i) {
      dm = d[i] - lm - (e[i] / dm) * e[i];
      if (fabsf(dm) < pivmin) dm = -pivmin;
      U[i] = dm;
    }
    int kt = 0;
    float best = 3.4e38f;
    for (int i = 0; i < N; ++i) {
      const float g = fabsf(L[i] + U[i] - (d[i] - lm));
      if (g < best) {
        best = g;
        kt = i;
      }
    }
    // z_kt = 1; z_i = -(e_i / d+_i) z_{i+1} upward; z_{i+1} = -(e_i / d-_{i+1}) z_i downward.
    // Entries are rescaled when they grow past 2^60 (the direction is what matters).
    Z[(int64_t)kt * lda + j] = 1.f;
    float z = 1.f;
    for (int i = kt - 1; i >= 0; --i) {
      z = -(e[i] / L[i]) * z;
      if (fabsf(z) > 1.15e18f) {
        for (int t = i + 1; t <= kt; ++t) Z[(int64_t)t * lda + j] *= 8.67e-19f;
        z *= 8.67e-19f;
      }
      Z[(int64_t)i * lda + j] = z;
    }
    z = Z[(int64_t)kt * lda + j];
    for (int i = kt; i + 1 < N; ++i) {
      z = -(e[i] / U[i + 1]) * z;
      if (fabsf(z) > 1.15e18f) {
        for (int t = 0; t <= i; ++t) Z[(int64_t)t * lda + j] *= 8.67e-19f;
        z *= 8.67e-19f;
      }
      Z[(int64_t)(i + 1) * lda + j] = z;
    }
    float s = 0.f;
    for (int i = 0; i < N; ++i) s = fmaf(Z[(int64_t)i * lda + j], Z[(int64_t)i * lda + j], s);
    const bool ok = s > 0.f && isfinite(s);
    const float sc = ok ? rsqrtf(s) : 0.f;
    for (int i = 0; i < N; ++i) Z[(int64_t)i * lda + j] = ok ? Z[(int64_t)i * lda + j] * sc : (i == j ? 1.f : 0.f);
  }
  __syncthreads();

  // ---- 4. X = H_0 ... H_{N-3} Z, one warp per column (no block barriers) -----
  for (int j = warp; j < N; j += nwarp) {
    for (int k = N - 3; k >= 0; --k) {
      const float bk = beta[k];
      if (bk == 0.f) continue;
      const int m = N - k - 1;
      float s = 0.f;
      for (int i = lane; i < m; i += 32) s = fmaf(A[(int64_t)(k + 1 + i) * lda + k], Z[(int64_t)(k + 1 + i) * lda + j], s);
      s = warp_sum(s) * bk;
      for (int i = lane; i < m; i += 32) Z[(int64_t)(k + 1 + i) * lda + j] -= s * A[(int64_t)(k + 1 + i) * lda + k];
      __syncwarp();
    }
  }
  __syncthreads();

  // ---- 5. two-pass MGS on the columns, dependent ones replaced last ----------
  // pass 0 orthonormalises the independent columns and flags the others (nrm = -1);
  // pass 1 replaces each flagged column by a pseudo-random vector orthogonalised
  // (twice) against every column already accepted.
  for (int pass = 0; pass < 2; ++pass) {
    for (int j = 0; j < N; ++j) {
      if (pass == 1) {
        if (nrm[j] >= 0.f) continue;
        for (int i = tid; i < N; i += nt) Z[(int64_t)i * lda + j] = hash_unit((uint32_t)j, (uint32_t)i);
        __syncthreads();
      }
      float n0 = 0.f;
      for (int i = tid; i < N; i += nt) n0 = fmaf(Z[(int64_t)i * lda + j], Z[(int64_t)i * lda + j], n0);
      n0 = block_sum_f(n0, red);
      for (int rep = 0; rep < 2; ++rep) {
        // coefficients against accepted columns c (pass 0: c < j; pass 1: all c != j not flagged)
        for (int c = warp; c < N; c += nwarp) {
          const bool acc = (c != j) && (pass == 0 ? (c < j && nrm[c] >= 0.f) : (nrm[c] >= 0.f));
          float s = 0.f;
          if (acc)
            for (int i = lane; i < N; i += 32) s = fmaf(Z[(int64_t)i * lda + c], Z[(int64_t)i * lda + j], s);
          s = warp_sum(s);
          if (lane == 0) cf[c] = acc ? s : 0.f;
        }
        __syncthreads();
        for (int i = tid; i < N; i += nt) {
          float s = 0.f;
          for (int c = 0; c < N; ++c) s = fmaf(Z[(int64_t)i * lda + c], cf[c], s);
          p[i] = s;
        }
        __syncthreads();
        for (int i = tid; i < N; i += nt) Z[(int64_t)i * lda + j] -= p[i];
        __syncthreads();
      }
      float n1 = 0.f;
      for (int i = tid; i < N; i += nt) n1 = fmaf(Z[(int64_t)i * lda + j], Z[(int64_t)i * lda + j], n1);
      n1 = block_sum_f(n1, red);
      // dependent if less than ~1e-3 of its length survives the projection
      const bool dep = !(n1 > 1e-6f * n0) || !(n1 > 0.f);
      if (pass == 0 && dep) {
        if (tid == 0) nrm[j] = -1.f;
        for (int i = tid; i < N; i += nt) Z[(int64_t)i * lda + j] = 0.f;
      } else {
        const float sc = rsqrtf(n1 > 0.f ? n1 : 1.f);
        for (int i = tid; i < N; i += nt) Z[(int64_t)i * lda + j] *= sc;
        if (tid == 0) nrm[j] = 1.f;
      }
      __syncthreads();
    }
  }
  for (int i = warp; i < N; i += nwarp)
    for (int j = lane; j < N; j += 32) Xout[(int64_t)i * N + j] = (double)Z[(int64_t)i * lda + j];
}

// ============================================================================
// The same method for N <= 128 with the matrix in registers.  Thread (w, t)
// of a 32 x 32 grid (warp w, lane t) holds entries (w + 32 r, t + 32 c),
// r, c < 4, of A during the reduction and entries (t + 32 r, w + 32 c) of the
// eigenvector matrix during the back-transformation, so that a row sum (the
// product A v) and a column sum (v^T Z) are warp sums and the updates stay in
// registers; shared memory carries only vectors, the reflectors and Z.
//   1. Householder tridiagonalisation, two barriers per step;
//   2. eigenvalues by multisection: 4 threads per eigenvalue evaluate Sturm
//      counts at 4 interior points, shrinking the bracket 5-fold per pass;
//      eigenvectors of T by the twisted factorisation, one thread each;
//   3. within each cluster of eigenvalues (gap below 1e-3 of ||T||) the
//      vectors are orthogonalised by classical Gram-Schmidt applied twice,
//      column by column with the whole CTA; a column with less than 1e-3 of
//      its length left is set aside and replaced at the end by one step of
//      inverse iteration at its eigenvalue from a pseudo-random start (so it
//      stays in that eigenspace even when several multiple eigenvalues lose
//      vectors), orthogonalised against every accepted column;
//   4. X = H_0 ... H_{N-3} Z, reflector by reflector, no block barriers.
// ============================================================================
namespace {
constexpr int E_NMAX = 128;
constexpr float E_CLUSTER = 1e-3f;

template <int R, int C>
__device__ __forceinline__ float pick(const float (&a)[R][C], int r, int c) {
  float v = 0.f;
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < C; ++j)
      if (i == r && j == c) v = a[i][j];
  return v;
}
}  // namespace

__device__ __forceinline__ void eig128_body(const double* __restrict__ Ain, int N, double* __restrict__ Xout,
                                            double* __restrict__ lam, float* __restrict__ Ug, float noise_rel) {
  extern __shared__ float esm[];
  __shared__ float s_d[E_NMAX], s_e[E_NMAX], s_beta[E_NMAX], s_col[2][E_NMAX], s_p[E_NMAX], s_lam[E_NMAX];
  __shared__ float2 s_de[E_NMAX];
  __shared__ float s_cf[E_NMAX], s_flag[E_NMAX];
  __shared__ int s_cstart[E_NMAX], s_prev[E_NMAX], s_np, s_npan;
  __shared__ float s_scale, s_bound[2], s_nrm, s_before;
  __shared__ int s_retry;
  const int tid = threadIdx.x, w = tid >> 5, t = tid & 31;
  const int lda = N | 1;
  float* Vref = esm;                       // N x 128: reflector k in row k (zero up to row k)
  float* Zs = esm + (size_t)N * E_NMAX;    // N x lda: eigenvectors of T, column j
  float* Us = Zs + (size_t)N * lda;        // N x lda: U pivots of the twisted factorisation, row j

  if (w == 0) {
    double mx = 0.0;
    for (int i = t; i < N; i += 32) mx = fmax(mx, fabs(Ain[(int64_t)i * N + i]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (t == 0) s_scale = (float)(mx > 0.0 && isfinite(mx) ? mx : 1.0);
  }
  __syncthreads();
  const float inv = 1.0f / s_scale;
  float a[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = w + 32 * r, j = t + 32 * c;
      a[r][c] = (i < N && j < N) ? (float)(Ain[(int64_t)i * N + j] * (double)inv) : 0.f;
    }

  // ---- 1. tridiagonalisation ------------------------------------------------
  for (int k = 0; k + 2 < N; ++k) {
    float* col = s_col[k & 1];
    if (t == (k & 31)) {  // column k of the current matrix, rows w + 32 r
      switch (k >> 5) {
#define EIG_COL(C) \
  case C:          \
    for (int r = 0; r < 4; ++r) col[w + 32 * r] = a[r][C]; \
    break;
        EIG_COL(0) EIG_COL(1) EIG_COL(2) EIG_COL(3)
#undef EIG_COL
      }
    }
    __syncthreads();
    if (w == 0) {
      // reflector H = I - tau v v^T with H x = alpha e_1, x = column k below row k, in the
      // normalised form v_0 = 1, v_i = x_i / (x0 - alpha), tau = (alpha - x0) / alpha in
      // [1, 2]: bounded for any scale of x (an unnormalised 2 / v^T v overflows on tiny columns)
      const float x0 = col[k + 1];
      const float sig = warp_nrm2(k + 1, N, t, [&](int i) { return col[i]; });
      const float alpha = x0 >= 0.f ? -sig : sig;
      const bool refl = sig > 0.f && isfinite(sig);
      const float bk = refl ? (alpha - x0) / alpha : 0.f;
      const float vs = refl ? 1.f / (x0 - alpha) : 0.f;
      for (int i = t; i < E_NMAX; i += 32)
        Vref[(size_t)k * E_NMAX + i] = (refl && i > k && i < N) ? (i == k + 1 ? 1.f : col[i] * vs) : 0.f;
      if (t == 0) {
        s_beta[k] = bk;
        s_e[k] = bk > 0.f ? alpha : x0;
        s_d[k] = col[k];
      }
    }
    __syncthreads();
    const float bk = s_beta[k];
    if (bk == 0.f) continue;  // uniform: nothing to annihilate
    const float* vk = Vref + (size_t)k * E_NMAX;
    float vr[4], vc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      vr[q] = vk[w + 32 * q];
      vc[q] = vk[t + 32 * q];
    }
    // p = beta A v over the active rows; per-warp share of p^T v
    float pvw = 0.f;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      float sr = 0.f;
      if (w + 32 * r > k) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (32 * c + 31 > k) sr = fmaf(a[r][c], vc[c], sr);
        for (int o = 16; o > 0; o >>= 1) sr += __shfl_xor_sync(0xffffffffu, sr, o);
        sr *= bk;
        pvw = fmaf(sr, vr[r], pvw);
      }
      if (t == 0) s_p[w + 32 * r] = sr;
    }
    if (t == 0) s_cf[w] = pvw;
    __syncthreads();
    // w = p - (beta/2)(p^T v) v ;  A <- A - v w^T - w v^T
    float pv = s_cf[t];
    for (int o = 16; o > 0; o >>= 1) pv += __shfl_xor_sync(0xffffffffu, pv, o);
    const float kk = 0.5f * bk * pv;
    float wr[4], wc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      wr[q] = s_p[w + 32 * q] - kk * vr[q];
      wc[q] = s_p[t + 32 * q] - kk * vc[q];
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (w + 32 * r > k) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (32 * c + 31 > k) a[r][c] -= vr[r] * wc[c] + wr[r] * vc[c];
      }
  }
  // the trailing 2 x 2 (or 1 x 1) block
  if (N >= 2) {
    if (t == ((N - 2) & 31) && w == ((N - 2) & 31)) s_d[N - 2] = pick(a, (N - 2) >> 5, (N - 2) >> 5);
    if (t == ((N - 2) & 31) && w == ((N - 1) & 31)) s_e[N - 2] = pick(a, (N - 1) >> 5, (N - 2) >> 5);
    if (tid == 0) s_beta[N - 2] = 0.f;
  }
  if (t == ((N - 1) & 31) && w == ((N - 1) & 31)) s_d[N - 1] = pick(a, (N - 1) >> 5, (N - 1) >> 5);
  if (tid == 0) s_beta[N - 1] = 0.f;
  __syncthreads();

  // ---- 2. eigenvalues (multisection) and eigenvectors of T ------------------
  if (w == 0) {
    float lo = 3.4e38f, hi = -3.4e38f;
    for (int i = t; i < N; i += 32) {
      const float rad = (i > 0 ? fabsf(s_e[i - 1]) : 0.f) + (i < N - 1 ? fabsf(s_e[i]) : 0.f);
      lo = fminf(lo, s_d[i] - rad);
      hi = fmaxf(hi, s_d[i] + rad);
      s_de[i] = make_float2(s_d[i], i > 0 ? s_e[i - 1] * s_e[i - 1] : 0.f);
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (t == 0) {
      const float pad = 1e-6f * fmaxf(fabsf(lo), fabsf(hi)) + 1e-30f;
      s_bound[0] = lo - pad;
      s_bound[1] = hi + pad;
    }
  }
  __syncthreads();
  const float tnorm = fmaxf(fabsf(s_bound[0]), fabsf(s_bound[1]));
  const float pivmin = fmaxf(1e-30f, 1e-12f * tnorm);
  if (tid < 4 * E_NMAX) {  // 4 points per eigenvalue: the bracket shrinks 5-fold per pass
    const int j = min(tid >> 2, N - 1), sub = tid & 3;
    float lo = s_bound[0], hi = s_bound[1];
    for (int it = 0; it < 10; ++it) {
      const float wd = hi - lo;
      const float x = lo + wd * (float)(sub + 1) * 0.2f;
      int cnt = 0;
      float q = 1.f;
      for (int i = 0; i < N; ++i) {
        const float2 de = s_de[i];
        q = (de.x - x) - (i > 0 ? __fdividef(de.y, q) : 0.f);
        if (fabsf(q) < pivmin) q = -pivmin;
        cnt += q < 0.f;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, cnt > j);
      const unsigned bits = (bal >> (t & 28)) & 0xfu;
      const int sl = bits ? __ffs(bits) - 1 : 4;
      const float nlo = sl == 0 ? lo : lo + wd * (float)sl * 0.2f;
      const float nhi = sl == 4 ? hi : lo + wd * (float)(sl + 1) * 0.2f;
      lo = nlo;
      hi = fmaxf(nhi, nlo);
    }
    if (sub == 0 && (tid >> 2) < N) {
      const float lm = 0.5f * (lo + hi);
      s_lam[j] = lm;
      lam[j] = (double)lm * (double)s_scale;
    }
  }
  __syncthreads();
  if (tid < N) {  // eigenvector j of T: twisted factorisation (L in Zs column j, U in Us row j)
    const int j = tid;
    const float lm = s_lam[j];
    float* U = Us + (size_t)j * lda;
    float dp = s_d[0] - lm;
    if (fabsf(dp) < pivmin) dp = -pivmin;
    Zs[j] = dp;
    for (int i = 0; i + 1 < N; ++i) {
      dp = s_d[i + 1] - lm - __fdividef(s_e[i], dp) * s_e[i];
      if (fabsf(dp) < pivmin) dp = -pivmin;
      Zs[(size_t)(i + 1) * lda + j] = dp;
    }
    float dm = s_d[N - 1] - lm;
    if (fabsf(dm) < pivmin) dm = -pivmin;
    U[N - 1] = dm;
    int kt = N - 1;
    float best = fabsf(Zs[(size_t)(N - 1) * lda + j] + dm - (s_d[N - 1] - lm));
    for (int i = N - 2; i >= 0; --i) {
      dm = s_d[i] - lm - __fdividef(s_e[i], dm) * s_e[i];
      if (fabsf(dm) < pivmin) dm = -pivmin;
      U[i] = dm;
      const float g = fabsf(Zs[(size_t)i * lda + j] + dm - (s_d[i] - lm));
      if (g < best) {
        best = g;
        kt = i;
      }
    }
    // z_kt = 1; upward z_i = -(e_i / L_i) z_{i+1} (L_i read just before it is overwritten);
    // downward z_{i+1} = -(e_i / U_{i+1}) z_i; entries are rescaled when they grow past 2^60
    float zkt = 1.f, z = 1.f;
    for (int i = kt - 1; i >= 0; --i) {
      z = -__fdividef(s_e[i], Zs[(size_t)i * lda + j]) * z;
      if (fabsf(z) > 1.15e18f) {
        for (int u = i + 1; u < kt; ++u) Zs[(size_t)u * lda + j] *= 8.67e-19f;
        zkt *= 8.67e-19f;
        z *= 8.67e-19f;
      }
      Zs[(size_t)i * lda + j] = z;
    }
    Zs[(size_t)kt * lda + j] = zkt;
    z = zkt;
    for (int i = kt; i + 1 < N; ++i) {
      z = -__fdividef(s_e[i], U[i + 1]) * z;
      if (fabsf(z) > 1.15e18f) {
        for (int u = 0; u <= i; ++u) Zs[(size_t)u * lda + j] *= 8.67e-19f;
        z *= 8.67e-19f;
      }
      Zs[(size_t)(i + 1) * lda + j] = z;
    }
  }
  __syncthreads();
  // normalise the columns and mark the cluster starts
  for (int j = w; j < N; j += 32) {
    float s2 = 0.f;
    for (int i = t; i < N; i += 32) s2 = fmaf(Zs[(size_t)i * lda + j], Zs[(size_t)i * lda + j], s2);
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    const bool ok = s2 > 0.f && isfinite(s2);
    const float sc = ok ? rsqrtf(s2) : 0.f;
    for (int i = t; i < N; i += 32) Zs[(size_t)i * lda + j] = ok ? Zs[(size_t)i * lda + j] * sc : (i == j ? 1.f : 0.f);
  }
  // flags: 1 accepted, -1 set aside (dependent), 2 noise (|lambda| below noise_rel ||T||: filled
  // at the end with the orthogonal complement of the other columns)
  if (tid == 0) {
    int st = 0;
    for (int j = 0; j < N; ++j) {
      if (j > 0 && !(s_lam[j] - s_lam[j - 1] <= E_CLUSTER * tnorm)) st = j;
      s_cstart[j] = st;
      s_flag[j] = (noise_rel > 0.f && fabsf(s_lam[j]) <= noise_rel * tnorm) ? 2.f : 1.f;
    }
  }
  __syncthreads();

  // ---- 3. clustered columns: CGS2 against the accepted columns of the cluster -
  for (int pass = 0; pass < 2; ++pass) {
    for (int j = 0; j < N; ++j) {
      const int cs = pass == 0 ? s_cstart[j] : 0;
      if (s_flag[j] == 2.f) continue;      // noise column: filled by the complement below
      if (pass == 0 && cs == j) continue;  // first of its cluster (or a singleton)
      if (pass == 1 && s_flag[j] >= 0.f) continue;
      // pass 1: the replacement by inverse iteration; when it falls (nearly) inside the span of
      // the accepted columns (an eigenvalue of T closer to accepted ones than to the missing
      // one), a second attempt from a plain pseudo-random start, which keeps the basis orthonormal
      for (int att = 0; att < (pass == 1 ? 3 : 1); ++att) {
      if (pass == 1) {
        // U pivots of the twisted factorisation at lambda_j are still in row j of Us; attempt 1
        // repeats inverse iteration on the projected residual, attempt 2 a plain random start
        if (tid == 0) {
          if (att < 2)
            inverse_iteration_start(s_e, Us + (size_t)j * lda, N, (uint32_t)j, Zs + j, lda, att == 1);
          else
            for (int i = 0; i < N; ++i) Zs[(size_t)i * lda + j] = hash_unit((uint32_t)j ^ 0x5bd1e995u, (uint32_t)i);
        }
        __syncthreads();
        if (w == 0) {  // the length before the projection
          float s2 = 0.f;
          for (int i = t; i < N; i += 32) s2 = fmaf(Zs[(size_t)i * lda + j], Zs[(size_t)i * lda + j], s2);
          for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
          if (t == 0) s_before = s2;
        }
        __syncthreads();
      }
      const int ce = pass == 0 ? j : N;
      for (int rep = 0; rep < 2; ++rep) {
        for (int c = cs + w; c < ce; c += 32) {
          const bool acc = c != j && s_flag[c] == 1.f;
          float s = 0.f;
          if (acc)
            for (int i = t; i < N; i += 32) s = fmaf(Zs[(size_t)i * lda + c], Zs[(size_t)i * lda + j], s);
          for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          if (t == 0) s_cf[c] = acc ? s : 0.f;
        }
        __syncthreads();
        {
          const int i = tid >> 3, part = tid & 7;
          float s = 0.f;
          if (i < N)
            for (int c = cs + part; c < ce; c += 8) s = fmaf(Zs[(size_t)i * lda + c], s_cf[c], s);
          s += __shfl_xor_sync(0xffffffffu, s, 1);
          s += __shfl_xor_sync(0xffffffffu, s, 2);
          s += __shfl_xor_sync(0xffffffffu, s, 4);
          __syncthreads();
          if (i < N && part == 0) Zs[(size_t)i * lda + j] -= s;
        }
        __syncthreads();
      }
      if (w == 0) {
        float s2 = 0.f;
        for (int i = t; i < N; i += 32) s2 = fmaf(Zs[(size_t)i * lda + j], Zs[(size_t)i * lda + j], s2);
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        // the column was unit length (pass 0) or of length^2 s_before (pass 1) before the projection
        const float before = pass == 0 ? 1.f : s_before;
        const bool dep = !(s2 > 1e-6f * before) || !(s2 > 0.f);
        if (t == 0) {
          s_nrm = dep && pass == 0 ? 0.f : rsqrtf(s2 > 0.f ? s2 : 1.f);
          s_flag[j] = dep && pass == 0 ? -1.f : 1.f;
          s_retry = (pass == 1 && att < 2 && dep) ? 1 : 0;
        }
      }
      __syncthreads();
      if (s_retry) continue;
      const float sc = s_nrm;
      for (int i = tid; i < N; i += 1024) Zs[(size_t)i * lda + j] *= sc;
      __syncthreads();
      break;
      }
    }
  }

  // ---- 3c. noise columns: orthonormal complement of the other columns --------
  // Householder QR of the n_nn other columns (copied into Us): the reflectors
  // H_0 .. H_{n_nn-1} applied to the unit vectors e_{n_nn} .. e_{N-1} span the
  // orthogonal complement of those columns, orthonormal by construction.
  if (tid == 0) {
    int nn = 0, nz = 0;
    for (int j = 0; j < N; ++j) {
      if (s_flag[j] == 2.f)
        s_prev[nz++] = j;  // noise columns
      else
        s_cstart[nn++] = j;  // the others (cluster starts are no longer needed)
    }
    s_np = nn;
    s_npan = nz;
  }
  __syncthreads();
  if (s_npan > 0) {
    const int nn = s_np, nz = s_npan;
    float* V = Us;  // N x lda, column c = other column s_cstart[c]
    for (int e = tid; e < N * nn; e += 1024) {
      const int i = e / nn, c = e % nn;
      V[(size_t)i * lda + c] = Zs[(size_t)i * lda + s_cstart[c]];
    }
    __syncthreads();
    for (int k = 0; k < nn; ++k) {
      if (w == 0) {
        const float sig = warp_nrm2(k, N, t, [&](int i) { return V[(size_t)i * lda + k]; });
        const float x0 = V[(size_t)k * lda + k];
        const float alpha = x0 >= 0.f ? -sig : sig;
        const float den = sig * (sig + fabsf(x0));  // v^T v / 2 for v = x - alpha e_k
        const float bk = (den >= NRM_TINY && isfinite(den)) ? 1.f / den : 0.f;
        __syncwarp();
        if (t == 0) {
          V[(size_t)k * lda + k] = x0 - alpha;  // v_k in place (rows k..N-1)
          s_cf[k] = bk;
        }
      }
      __syncthreads();
      const float bk = s_cf[k];
      for (int j = k + 1 + w; j < nn && bk != 0.f; j += 32) {
        float d = 0.f;
        for (int i = k + t; i < N; i += 32) d = fmaf(V[(size_t)i * lda + k], V[(size_t)i * lda + j], d);
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        d *= bk;
        for (int i = k + t; i < N; i += 32) V[(size_t)i * lda + j] -= d * V[(size_t)i * lda + k];
      }
      __syncthreads();
    }
    // Q e_{nn + q} into noise column q, reflectors in reverse order, a warp per column
    for (int q = w; q < nz; q += 32) {
      const int col = s_prev[q];
      for (int i = t; i < N; i += 32) Zs[(size_t)i * lda + col] = (i == nn + q) ? 1.f : 0.f;
      __syncwarp();
      for (int k = nn - 1; k >= 0; --k) {
        const float bk = s_cf[k];
        if (bk == 0.f) continue;
        float d = 0.f;
        for (int i = k + t; i < N; i += 32) d = fmaf(V[(size_t)i * lda + k], Zs[(size_t)i * lda + col], d);
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        d *= bk;
        for (int i = k + t; i < N; i += 32) Zs[(size_t)i * lda + col] -= d * V[(size_t)i * lda + k];
        __syncwarp();
      }
    }
    __syncthreads();
  }

  // ---- 4. back-transformation with Z in registers ---------------------------
  float z[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = t + 32 * r, j = w + 32 * c;
      z[r][c] = (i < N && j < N) ? Zs[(size_t)i * lda + j] : 0.f;
    }
  for (int k = N - 3; k >= 0; --k) {
    const float bk = s_beta[k];
    if (bk == 0.f) continue;
    float v[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) v[r] = Vref[(size_t)k * E_NMAX + t + 32 * r];
    // the four column sums reduced together (independent shuffle chains)
    float sc[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      sc[c] = 0.f;
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (32 * r + 31 > k) sc[c] = fmaf(v[r], z[r][c], sc[c]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int c = 0; c < 4; ++c) sc[c] += __shfl_xor_sync(0xffffffffu, sc[c], o);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float sb = sc[c] * bk;
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (32 * r + 31 > k) z[r][c] -= sb * v[r];
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = t + 32 * r, j = w + 32 * c;
      if (i < N && j < N) Zs[(size_t)i * lda + j] = z[r][c];
    }
  __syncthreads();
  for (int e = tid; e < N * N; e += 1024) Xout[e] = (double)Zs[(size_t)(e / N) * lda + e % N];
}

// ============================================================================
// The same method for 128 < N <= 512, one CTA of 1024 threads.  The launch
// gives the CTA dyn_floats floats of dynamic shared memory; the matrix is kept
//   - full (row-major, both triangles) in shared memory when N^2 floats fit
//     (N <= 227), else
//   - as its packed lower triangle, Ap[i (i + 1) / 2 + j] = A_ij (j <= i), in
//     shared memory when that fits (N <= 318), else
//   - full in global scratch (rows read and written whole, coalesced).
// The full forms apply the rank-2 update to (i, j) and (j, i) as the same
// correctly rounded value, so the stored matrix stays exactly symmetric and the
// row i right of the diagonal serves as column i.  The reflector of step k is
// stored contiguously (row k of RT) for the back-transformation.  From step 2
// on the eigenvectors of T live column-major in shared memory when N^2 floats
// fit (the matrix is no longer needed), else in global scratch; their
// factorisation pivots and the complement's reflectors stay in global scratch.
//   1. Householder tridiagonalisation, three barriers per step: the reflector
//      (one warp), p = beta A v (a warp per row), then the rank-2 update;
//   2.-3c. as in eig128 (multisection, twisted factorisation, cluster CGS2,
//      orthonormal complement of the noise columns);
//   4. X = H_0 ... H_{N-3} Z, a warp per column of Z held in registers.
// ============================================================================
namespace {
constexpr int EB_NMAX = 512;
constexpr int EB_SMEM_NMAX = 318;  // N (N + 1) / 2 floats = 202,884 bytes: with ~24 KB static, within 227 KB
constexpr int EB_DYN_FLOATS = 202 * 1024 / 4;  // the dynamic shared memory cap of the eig_big launches
__device__ __forceinline__ int pk(int i, int j) { return ((i * (i + 1)) >> 1) + j; }  // j <= i
// Dynamic shared memory (floats) for problems up to N: the full matrix when it fits, else the
// packed triangle when that fits, else none.
int eb_dyn_floats(int N) {
  const int64_t full = (int64_t)N * N, packed = (int64_t)N * (N + 1) / 2;
  return full <= EB_DYN_FLOATS ? (int)full : (packed <= EB_DYN_FLOATS ? (int)packed : 0);
}
}  // namespace

int64_t eig_big_scratch_floats(int N) { return 6ll * N * N + N + 64; }

// Column j of X = H_0 ... H_{N-3} Z (Z column-major in ZT, reflector k in row k of RT, its scalar
// in beta[k]; zero: no reflector), by one warp (lane t), written to Xout in FP64.
__device__ __forceinline__ void eig_big_back_col(int j, int N, const float* ZT, const float* __restrict__ RT,
                                                 const float* beta, double* __restrict__ Xout, int t) {
  constexpr int NR = EB_NMAX / 32;
  const float* Zc = ZT + (size_t)j * N;
  float z[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int i = t + 32 * r;
    z[r] = i < N ? Zc[i] : 0.f;
  }
  for (int k = N - 3; k >= 0; --k) {
    const float bk = beta[k];
    if (bk == 0.f) continue;
    float v[NR];
    float s = 0.f;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int i = t + 32 * r;
      v[r] = (i > k && i < N) ? RT[(size_t)k * N + i] : 0.f;
      s = fmaf(v[r], z[r], s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    s *= bk;
#pragma unroll
    for (int r = 0; r < NR; ++r) z[r] -= s * v[r];
  }
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int i = t + 32 * r;
    if (i < N) Xout[(int64_t)i * N + j] = (double)z[r];
  }
}

__device__ __forceinline__ void eig_big_body(const double* __restrict__ Ain, int N, double* __restrict__ Xout,
                                             double* __restrict__ lam, float* __restrict__ gscr, float noise_rel,
                                             int dyn_floats, int back = 1) {
  extern __shared__ float ebsm[];
  __shared__ float s_d[EB_NMAX], s_e[EB_NMAX], s_beta[EB_NMAX], s_v[EB_NMAX], s_p[EB_NMAX], s_lam[EB_NMAX];
  __shared__ float s_cf[EB_NMAX], s_flag[EB_NMAX];
  __shared__ float2 s_de[EB_NMAX];
  __shared__ int s_cstart[EB_NMAX], s_prev[EB_NMAX], s_np, s_npan;
  __shared__ float s_red[32], s_scale, s_bound[2], s_nrm, s_before;
  __shared__ int s_retry;
  const int tid = threadIdx.x, w = tid >> 5, t = tid & 31;
  const size_t NN = (size_t)N * N;
  const bool z_smem = (int64_t)NN <= dyn_floats;  // full matrix, then Z, in shared memory
  const bool packed = !z_smem && (int64_t)N * (N + 1) / 2 <= dyn_floats;
  float* LT = gscr + NN;      // N x N column-major: L pivots of eigenvalue j in column j
  float* UT = gscr + 2 * NN;  // N x N column-major: U pivots
  float* VT = gscr + 3 * NN;  // N x N column-major: the complement's Householder columns
  float* RT = gscr + 4 * NN;  // N x N: reflector k in row k (entries k + 1 .. N - 1)
  float* Af = z_smem ? ebsm : gscr + 5 * NN;  // the full forms' matrix (row-major)
  float* Ap = ebsm;                           // the packed form's triangle
  float* ZT = z_smem ? ebsm : gscr;  // from step 2 on: eigenvectors of T, then of A (column-major)

  if (w == 0) {
    double mx = 0.0;
    for (int i = t; i < N; i += 32) mx = fmax(mx, fabs(Ain[(int64_t)i * N + i]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (t == 0) s_scale = (float)(mx > 0.0 && isfinite(mx) ? mx : 1.0);
  }
  __syncthreads();
  const float inv = 1.0f / s_scale;
  if (packed) {
    for (int i = w; i < N; i += 32)
      for (int j = t; j <= i; j += 32) Ap[pk(i, j)] = (float)(Ain[(int64_t)i * N + j] * (double)inv);
  } else {  // both triangles from the lower one: exactly symmetric
    for (int i = w; i < N; i += 32)
      for (int j = t; j < N; j += 32)
        Af[(size_t)i * N + j] = (float)(Ain[(int64_t)max(i, j) * N + min(i, j)] * (double)inv);
  }
  for (int i = tid; i < N; i += 1024) s_v[i] = 0.f;
  __syncthreads();

  // ---- 1. tridiagonalisation ------------------------------------------------
  if (packed) {
  for (int k = 0; k + 2 < N; ++k) {
    if (w == 0) {
      const float x0 = Ap[pk(k + 1, k)];
      const float sig = warp_nrm2(k + 1, N, t, [&](int i) { return Ap[pk(i, k)]; });
      const float alpha = x0 >= 0.f ? -sig : sig;
      const bool refl = sig > 0.f && isfinite(sig);
      const float bk = refl ? (alpha - x0) / alpha : 0.f;  // normalised reflector, v_0 = 1, bk in [1, 2]
      const float vs = refl ? 1.f / (x0 - alpha) : 0.f;
      if (refl)
        for (int i = k + 1 + t; i < N; i += 32) {
          const float v = i == k + 1 ? 1.f : Ap[pk(i, k)] * vs;
          s_v[i] = v;
          RT[(size_t)k * N + i] = v;  // kept for the back-transformation
        }
      if (t == 0) {
        s_beta[k] = bk;
        s_e[k] = bk > 0.f ? alpha : x0;
        s_d[k] = Ap[pk(k, k)];
        s_v[k] = 0.f;
      }
    }
    __syncthreads();
    const float bk = s_beta[k];
    if (bk == 0.f) continue;  // uniform: nothing to annihilate
    // p = bk A22 v (rows k+1 .. N-1), per-warp share of p^T v
    float pvw = 0.f;
    for (int i = k + 1 + w; i < N; i += 32) {
      float s = 0.f;
      for (int j = k + 1 + t; j < N; j += 32) s = fmaf(j <= i ? Ap[pk(i, j)] : Ap[pk(j, i)], s_v[j], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      s *= bk;
      pvw = fmaf(s, s_v[i], pvw);
      if (t == 0) s_p[i] = s;
    }
    if (t == 0) s_red[w] = pvw;
    __syncthreads();
    float pv = s_red[t];
    for (int o = 16; o > 0; o >>= 1) pv += __shfl_xor_sync(0xffffffffu, pv, o);
    const float kk = 0.5f * bk * pv;
    // A22 <- A22 - v w^T - w v^T with w = p - kk v, on the packed lower triangle
    for (int i = k + 1 + w; i < N; i += 32) {
      const float vi = s_v[i], wi = s_p[i] - kk * vi;
      float* row = Ap + pk(i, 0);
      for (int j = k + 1 + t; j <= i; j += 32) {
        const float vj = s_v[j], wj = s_p[j] - kk * vj;
        row[j] -= vi * wj + wi * vj;
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (N >= 2) {
      s_d[N - 2] = Ap[pk(N - 2, N - 2)];
      s_e[N - 2] = Ap[pk(N - 1, N - 2)];
      s_beta[N - 2] = 0.f;
    }
    s_d[N - 1] = Ap[pk(N - 1, N - 1)];
    s_beta[N - 1] = 0.f;
  }
  } else {
  for (int k = 0; k + 2 < N; ++k) {
    const float* Ak = Af + (size_t)k * N;  // row k right of the diagonal = column k below it
    if (w == 0) {
      const float x0 = Ak[k + 1];
      const float sig = warp_nrm2(k + 1, N, t, [&](int i) { return Ak[i]; });
      const float alpha = x0 >= 0.f ? -sig : sig;
      const bool refl = sig > 0.f && isfinite(sig);
      const float bk = refl ? (alpha - x0) / alpha : 0.f;  // normalised reflector, v_0 = 1, bk in [1, 2]
      const float vs = refl ? 1.f / (x0 - alpha) : 0.f;
      if (refl)
        for (int i = k + 1 + t; i < N; i += 32) {
          const float v = i == k + 1 ? 1.f : Ak[i] * vs;
          s_v[i] = v;
          RT[(size_t)k * N + i] = v;  // kept for the back-transformation
        }
      if (t == 0) {
        s_beta[k] = bk;
        s_e[k] = bk > 0.f ? alpha : x0;
        s_d[k] = Ak[k];
        s_v[k] = 0.f;
      }
    }
    __syncthreads();
    const float bk = s_beta[k];
    if (bk == 0.f) continue;  // uniform: nothing to annihilate
    // p = bk A22 v (rows k+1 .. N-1, each read whole), per-warp share of p^T v
    float pvw = 0.f;
    for (int i = k + 1 + w; i < N; i += 32) {
      const float* row = Af + (size_t)i * N;
      float s = 0.f;
      for (int j = k + 1 + t; j < N; j += 32) s = fmaf(row[j], s_v[j], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      s *= bk;
      pvw = fmaf(s, s_v[i], pvw);
      if (t == 0) s_p[i] = s;
    }
    if (t == 0) s_red[w] = pvw;
    __syncthreads();
    float pv = s_red[t];
    for (int o = 16; o > 0; o >>= 1) pv += __shfl_xor_sync(0xffffffffu, pv, o);
    const float kk = 0.5f * bk * pv;
    // A22 <- A22 - v w^T - w v^T with w = p - kk v: (i, j) and (j, i) get the same value
    // (two correctly rounded products and their correctly rounded sum, in either order)
    for (int i = k + 1 + w; i < N; i += 32) {
      const float vi = s_v[i], wi = s_p[i] - kk * vi;
      float* row = Af + (size_t)i * N;
      for (int j = k + 1 + t; j < N; j += 32) {
        const float vj = s_v[j], wj = s_p[j] - kk * vj;
        row[j] -= __fadd_rn(__fmul_rn(vi, wj), __fmul_rn(wi, vj));
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (N >= 2) {
      s_d[N - 2] = Af[(size_t)(N - 2) * N + N - 2];
      s_e[N - 2] = Af[(size_t)(N - 1) * N + N - 2];
      s_beta[N - 2] = 0.f;
    }
    s_d[N - 1] = Af[(size_t)(N - 1) * N + N - 1];
    s_beta[N - 1] = 0.f;
  }
  }
  __syncthreads();  // the matrix is dead from here on (Z may take its shared memory)

  // ---- 2. eigenvalues (multisection) and eigenvectors of T ------------------
  if (w == 0) {
    float lo = 3.4e38f, hi = -3.4e38f;
    for (int i = t; i < N; i += 32) {
      const float rad = (i > 0 ? fabsf(s_e[i - 1]) : 0.f) + (i < N - 1 ? fabsf(s_e[i]) : 0.f);
      lo = fminf(lo, s_d[i] - rad);
      hi = fmaxf(hi, s_d[i] + rad);
      s_de[i] = make_float2(s_d[i], i > 0 ? s_e[i - 1] * s_e[i - 1] : 0.f);
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (t == 0) {
      const float pad = 1e-6f * fmaxf(fabsf(lo), fabsf(hi)) + 1e-30f;
      s_bound[0] = lo - pad;
      s_bound[1] = hi + pad;
    }
  }
  __syncthreads();
  const float tnorm = fmaxf(fabsf(s_bound[0]), fabsf(s_bound[1]));
  const float pivmin = fmaxf(1e-30f, 1e-12f * tnorm);
  for (int base = 0; base < N; base += 256) {  // 4 points per eigenvalue, 256 eigenvalues per round
    const int j0 = base + (tid >> 2), sub = tid & 3;
    const int j = min(j0, N - 1);
    float lo = s_bound[0], hi = s_bound[1];
    for (int it = 0; it < 10; ++it) {
      const float wd = hi - lo;
      const float x = lo + wd * (float)(sub + 1) * 0.2f;
      int cnt = 0;
      float q = 1.f;
      for (int i = 0; i < N; ++i) {
        const float2 de = s_de[i];
        q = (de.x - x) - (i > 0 ? __fdividef(de.y, q) : 0.f);
        if (fabsf(q) < pivmin) q = -pivmin;
        cnt += q < 0.f;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, cnt > j);
      const unsigned bits = (bal >> (t & 28)) & 0xfu;
      const int sl = bits ? __ffs(bits) - 1 : 4;
      const float nlo = sl == 0 ? lo : lo + wd * (float)sl * 0.2f;
      const float nhi = sl == 4 ? hi : lo + wd * (float)(sl + 1) * 0.2f;
      lo = nlo;
      hi = fmaxf(nhi, nlo);
    }
    if (sub == 0 && j0 < N) {
      const float lm = 0.5f * (lo + hi);
      s_lam[j0] = lm;
      lam[j0] = (double)lm * (double)s_scale;
    }
  }
  __syncthreads();
  for (int j = tid; j < N; j += 1024) {  // eigenvector j of T by the twisted factorisation
    const float lm = s_lam[j];
    float* Z = ZT + (size_t)j * N;
    float* Lc = LT + (size_t)j * N;
    float* U = UT + (size_t)j * N;
    float dp = s_d[0] - lm;
    if (fabsf(dp) < pivmin) dp = -pivmin;
    Lc[0] = dp;
    for (int i = 0; i + 1 < N; ++i) {
      dp = s_d[i + 1] - lm - __fdividef(s_e[i], dp) * s_e[i];
      if (fabsf(dp) < pivmin) dp = -pivmin;
      Lc[i + 1] = dp;
    }
    float dm = s_d[N - 1] - lm;
    if (fabsf(dm) < pivmin) dm = -pivmin;
    U[N - 1] = dm;
    int kt = N - 1;
    float best = fabsf(Lc[N - 1] + dm - (s_d[N - 1] - lm));
    for (int i = N - 2; i >= 0; --i) {
      dm = s_d[i] - lm - __fdividef(s_e[i], dm) * s_e[i];
      if (fabsf(dm) < pivmin) dm = -pivmin;
      U[i] = dm;
      const float g = fabsf(Lc[i] + dm - (s_d[i] - lm));
      if (g < best) {
        best = g;
        kt = i;
      }
    }
    // z_kt = 1; upward z_i = -(e_i / L_i) z_{i+1}; downward z_{i+1} = -(e_i / U_{i+1}) z_i;
    // entries are rescaled when they grow past 2^60
    float zkt = 1.f, z = 1.f;
    for (int i = kt - 1; i >= 0; --i) {
      z = -__fdividef(s_e[i], Lc[i]) * z;
      if (fabsf(z) > 1.15e18f) {
        for (int u = i + 1; u < kt; ++u) Z[u] *= 8.67e-19f;
        zkt *= 8.67e-19f;
        z *= 8.67e-19f;
      }
      Z[i] = z;
    }
    Z[kt] = zkt;
    z = zkt;
    for (int i = kt; i + 1 < N; ++i) {
      z = -__fdividef(s_e[i], U[i + 1]) * z;
      if (fabsf(z) > 1.15e18f) {
        for (int u = 0; u <= i; ++u) Z[u] *= 8.67e-19f;
        z *= 8.67e-19f;
      }
      Z[i + 1] = z;
    }
  }
  __syncthreads();
  for (int j = w; j < N; j += 32) {  // normalise the columns
    float* Z = ZT + (size_t)j * N;
    float s2 = 0.f;
    for (int i = t; i < N; i += 32) s2 = fmaf(Z[i], Z[i], s2);
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    const bool ok = s2 > 0.f && isfinite(s2);
    const float sc = ok ? rsqrtf(s2) : 0.f;
    for (int i = t; i < N; i += 32) Z[i] = ok ? Z[i] * sc : (i == j ? 1.f : 0.f);
  }
  // flags: 1 accepted, -1 set aside (dependent), 2 noise (filled with the complement)
  if (tid == 0) {
    int st = 0;
    for (int j = 0; j < N; ++j) {
      if (j > 0 && !(s_lam[j] - s_lam[j - 1] <= E_CLUSTER * tnorm)) st = j;
      s_cstart[j] = st;
      s_flag[j] = (noise_rel > 0.f && fabsf(s_lam[j]) <= noise_rel * tnorm) ? 2.f : 1.f;
    }
  }
  __syncthreads();

  // ---- 3. clustered columns: CGS2 against the accepted columns of the cluster -
  for (int pass = 0; pass < 2; ++pass) {
    for (int j = 0; j < N; ++j) {
      const int cs = pass == 0 ? s_cstart[j] : 0;
      if (s_flag[j] == 2.f) continue;
      if (pass == 0 && cs == j) continue;
      float* Zj = ZT + (size_t)j * N;
      if (pass == 1 && s_flag[j] >= 0.f) continue;
      // pass 1: inverse iteration, then (when that falls inside the accepted span) a plain
      // pseudo-random start, as in eig128
      for (int att = 0; att < (pass == 1 ? 3 : 1); ++att) {
      if (pass == 1) {
        // U pivots of the twisted factorisation at lambda_j are still in column j of UT; attempt 1
        // repeats inverse iteration on the projected residual, attempt 2 a plain random start
        if (tid == 0) {
          if (att < 2)
            inverse_iteration_start(s_e, UT + (size_t)j * N, N, (uint32_t)j, Zj, 1, att == 1);
          else
            for (int i = 0; i < N; ++i) Zj[i] = hash_unit((uint32_t)j ^ 0x5bd1e995u, (uint32_t)i);
        }
        __syncthreads();
        if (w == 0) {  // the length before the projection
          float s2 = 0.f;
          for (int i = t; i < N; i += 32) s2 = fmaf(Zj[i], Zj[i], s2);
          for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
          if (t == 0) s_before = s2;
        }
        __syncthreads();
      }
      const int ce = pass == 0 ? j : N;
      for (int rep = 0; rep < 2; ++rep) {
        for (int c = cs + w; c < ce; c += 32) {
          const bool acc = c != j && s_flag[c] == 1.f;
          float s = 0.f;
          if (acc) {
            const float* Zc = ZT + (size_t)c * N;
            for (int i = t; i < N; i += 32) s = fmaf(Zc[i], Zj[i], s);
          }
          for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          if (t == 0) s_cf[c] = acc ? s : 0.f;
        }
        __syncthreads();
        for (int i0 = 0; i0 < N; i0 += 128) {
          const int i = i0 + (tid >> 3), part = tid & 7;
          float s = 0.f;
          if (i < N)
            for (int c = cs + part; c < ce; c += 8) s = fmaf(ZT[(size_t)c * N + i], s_cf[c], s);
          s += __shfl_xor_sync(0xffffffffu, s, 1);
          s += __shfl_xor_sync(0xffffffffu, s, 2);
          s += __shfl_xor_sync(0xffffffffu, s, 4);
          if (i < N && part == 0) Zj[i] -= s;
        }
        __syncthreads();
      }
      if (w == 0) {
        float s2 = 0.f;
        for (int i = t; i < N; i += 32) s2 = fmaf(Zj[i], Zj[i], s2);
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        const float before = pass == 0 ? 1.f : s_before;
        const bool dep = !(s2 > 1e-6f * before) || !(s2 > 0.f);
        if (t == 0) {
          s_nrm = dep && pass == 0 ? 0.f : rsqrtf(s2 > 0.f ? s2 : 1.f);
          s_flag[j] = dep && pass == 0 ? -1.f : 1.f;
          s_retry = (pass == 1 && att < 2 && dep) ? 1 : 0;
        }
      }
      __syncthreads();
      if (s_retry) continue;
      const float sc = s_nrm;
      for (int i = tid; i < N; i += 1024) Zj[i] *= sc;
      __syncthreads();
      break;
      }
    }
  }

  // ---- 3c. noise columns: orthonormal complement of the other columns --------
  if (tid == 0) {
    int nn = 0, nz = 0;
    for (int j = 0; j < N; ++j) {
      if (s_flag[j] == 2.f)
        s_prev[nz++] = j;
      else
        s_cstart[nn++] = j;
    }
    s_np = nn;
    s_npan = nz;
  }
  __syncthreads();
  if (s_npan > 0) {
    const int nn = s_np, nz = s_npan;
    for (int c = w; c < nn; c += 32) {
      const float* src = ZT + (size_t)s_cstart[c] * N;
      float* dst = VT + (size_t)c * N;
      for (int i = t; i < N; i += 32) dst[i] = src[i];
    }
    __syncthreads();
    for (int k = 0; k < nn; ++k) {
      float* Vk = VT + (size_t)k * N;
      if (w == 0) {
        const float sig = warp_nrm2(k, N, t, [&](int i) { return Vk[i]; });
        const float x0 = Vk[k];
        const float alpha = x0 >= 0.f ? -sig : sig;
        const float den = sig * (sig + fabsf(x0));  // v^T v / 2 for v = x - alpha e_k
        const float bk = (den >= NRM_TINY && isfinite(den)) ? 1.f / den : 0.f;
        __syncwarp();
        if (t == 0) {
          Vk[k] = x0 - alpha;
          s_cf[k] = bk;
        }
      }
      __syncthreads();
      const float bk = s_cf[k];
      for (int j = k + 1 + w; j < nn && bk != 0.f; j += 32) {
        float* Vj = VT + (size_t)j * N;
        float d = 0.f;
        for (int i = k + t; i < N; i += 32) d = fmaf(Vk[i], Vj[i], d);
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        d *= bk;
        for (int i = k + t; i < N; i += 32) Vj[i] -= d * Vk[i];
      }
      __syncthreads();
    }
    for (int q = w; q < nz; q += 32) {
      float* Zc = ZT + (size_t)s_prev[q] * N;
      for (int i = t; i < N; i += 32) Zc[i] = (i == nn + q) ? 1.f : 0.f;
      __syncwarp();
      for (int k = nn - 1; k >= 0; --k) {
        const float bk = s_cf[k];
        if (bk == 0.f) continue;
        const float* Vk = VT + (size_t)k * N;
        float d = 0.f;
        for (int i = k + t; i < N; i += 32) d = fmaf(Vk[i], Zc[i], d);
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        d *= bk;
        for (int i = k + t; i < N; i += 32) Zc[i] -= d * Vk[i];
        __syncwarp();
      }
    }
    __syncthreads();
  }

  // ---- 4. back-transformation, a warp per column of Z in registers -----------
  if (!back) {  // a separate launch spreads the columns over CTAs (eig_big_back_kernel)
    for (int k = tid; k < N; k += 1024) gscr[6 * NN + k] = s_beta[k];
    return;
  }
  for (int j = w; j < N; j += 32) eig_big_back_col(j, N, ZT, RT, s_beta, Xout, t);
}

// X = H_0 ... H_{N-3} Z for columns spread over CTAs, a warp per column: the last step of
// eig_big_body when that ran with back = 0 (Z, the reflectors and their scalars in scratch).
__global__ __launch_bounds__(256) void eig_big_back_kernel(int N, const float* __restrict__ gscr,
                                                           double* __restrict__ Xout) {
  __shared__ float s_beta[EB_NMAX];
  const size_t NN = (size_t)N * N;
  for (int k = threadIdx.x; k < N; k += 256) s_beta[k] = gscr[6 * NN + k];
  __syncthreads();
  const int j = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (j < N) eig_big_back_col(j, N, gscr, gscr + 4 * NN, s_beta, Xout, threadIdx.x & 31);
}

__global__ __launch_bounds__(1024) void eig128_kernel(const double* __restrict__ Ain, int N,
                                                      double* __restrict__ Xout, double* __restrict__ lam,
                                                      float* __restrict__ Ug, float noise_rel) {
  eig128_body(Ain, N, Xout, lam, Ug, noise_rel);
}

__global__ __launch_bounds__(1024) void eig_big_kernel(const double* __restrict__ Ain, int N,
                                                       double* __restrict__ Xout, double* __restrict__ lam,
                                                       float* __restrict__ gscr, float noise_rel, int dyn_floats,
                                                       int back) {
  eig_big_body(Ain, N, Xout, lam, gscr, noise_rel, dyn_floats, back);
}

// Batched: one CTA per problem (the grouped solve's compressed pairs).
__global__ __launch_bounds__(1024) void eig128_b_kernel(const EigB* __restrict__ tab) {
  const EigB& a = tab[blockIdx.x];
  eig128_body(a.A, a.N, a.X, a.lam, a.scratch, a.noise_rel);
}
__global__ __launch_bounds__(1024) void eig_big_b_kernel(const EigB* __restrict__ tab, int dyn_floats) {
  const EigB& a = tab[blockIdx.x];
  eig_big_body(a.A, a.N, a.X, a.lam, a.scratch, a.noise_rel, dyn_floats);
}

// A cut cluster of more than CUT_CMAX columns (the descriptor written by the cut-cluster
// detection kernel into the P block of the refinement work; N = 0: nothing to solve).  The
// launch gives dyn_floats floats of dynamic shared memory.
__device__ __forceinline__ void eig_cut_big_body(const double* __restrict__ pblock, int dyn_floats) {
  const EigB* e = reinterpret_cast<const EigB*>(pblock + CUT_EIGB_OFF);
  const int c = e->N;
  if (c <= CUT_CMAX || c > EB_NMAX) return;
  eig_big_body(e->A, c, e->X, e->lam, e->scratch, e->noise_rel, dyn_floats);
}

__global__ __launch_bounds__(1024) void eig_cut_big_kernel(const double* __restrict__ pblock, int dyn_floats) {
  eig_cut_big_body(pblock, dyn_floats);
}

__global__ __launch_bounds__(1024) void eig_cut_big_b_kernel(const OaB* __restrict__ tab, int dyn_floats) {
  const OaB& o = tab[blockIdx.x];
  if (o.N <= CUT_CMAX || !o.jscr) return;  // no room for a descriptor, or no scratch: clipped clusters only
  eig_cut_big_body(o.P, dyn_floats);
}

cudaError_t launch_eig_cut_big(const double* pblock, int max_N, cudaStream_t st) {
  if (max_N <= CUT_CMAX) return cudaSuccess;
  const int dyn = eb_dyn_floats(std::min(max_N, EB_SMEM_NMAX));
  cudaFuncSetAttribute(eig_cut_big_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, EB_DYN_FLOATS * 4);
  eig_cut_big_kernel<<<1, 1024, (size_t)dyn * sizeof(float), st>>>(pblock, dyn);
  return launched();
}

cudaError_t launch_eig_cut_big_b(const OaB* tab, int nprob, int max_N, cudaStream_t st) {
  if (nprob <= 0 || max_N <= CUT_CMAX) return cudaSuccess;
  const int dyn = eb_dyn_floats(std::min(max_N, EB_SMEM_NMAX));
  cudaFuncSetAttribute(eig_cut_big_b_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, EB_DYN_FLOATS * 4);
  eig_cut_big_b_kernel<<<nprob, 1024, (size_t)dyn * sizeof(float), st>>>(tab, dyn);
  return launched();
}

cudaError_t launch_eig_f32_b(const EigB* tab, int nprob, int max_N, cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  if (max_N < 1 || max_N > EB_SMEM_NMAX) return cudaErrorInvalidValue;
  if (max_N <= E_NMAX) {
    const size_t smem = ((size_t)max_N * E_NMAX + 2 * (size_t)max_N * (max_N | 1)) * sizeof(float);
    cudaFuncSetAttribute(eig128_b_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    eig128_b_kernel<<<nprob, 1024, smem, st>>>(tab);
    return launched();
  }
  const int dyn = eb_dyn_floats(max_N);
  cudaFuncSetAttribute(eig_big_b_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, EB_DYN_FLOATS * 4);
  eig_big_b_kernel<<<nprob, 1024, (size_t)dyn * sizeof(float), st>>>(tab, dyn);
  return launched();
}

cudaError_t launch_eig_f32(const double* A, int N, double* X, double* lam, float* scratch, cudaStream_t st,
                           double noise_rel) {
  if (N < 1 || N > 1024) return cudaErrorInvalidValue;
  const int lda = N | 1;
  if (N <= E_NMAX) {
    const size_t smem = ((size_t)N * E_NMAX + 2 * (size_t)N * lda) * sizeof(float);
    // a fixed cap (N = 128 needs 197,632 bytes): concurrent launches must not lower it
    cudaFuncSetAttribute(eig128_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    eig128_kernel<<<1, 1024, smem, st>>>(A, N, X, lam, scratch, (float)noise_rel);
    return launched();
  }
  if (N <= EB_NMAX) {
    const int dyn = eb_dyn_floats(N);
    // a fixed cap: concurrent launches must not lower it
    cudaFuncSetAttribute(eig_big_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, EB_DYN_FLOATS * 4);
    // Z in global scratch (N^2 floats beyond the shared memory): its back-transformation runs as
    // a second launch over ceil(N / 8) CTAs of 8 warps instead of on this CTA's 32 warps
    const int back = (int64_t)N * N <= dyn ? 1 : 0;
    eig_big_kernel<<<1, 1024, (size_t)dyn * sizeof(float), st>>>(A, N, X, lam, scratch, (float)noise_rel, dyn,
                                                                 back);
    cudaError_t e = launched();
    if (e || back) return e;
    eig_big_back_kernel<<<(unsigned)((N + 7) / 8), 256, 0, st>>>(N, scratch, X);
    return launched();
  }
  const size_t smem = (2ull * N * lda + 8ull * N) * sizeof(float);
  const int use_smem = smem <= 200 * 1024;
  cudaFuncSetAttribute(eig_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  eig_f32_kernel<<<1, 1024, use_smem ? smem : 0, st>>>(A, N, X, lam, scratch, use_smem);
  return launched();
}

}  // namespace gsvdr
