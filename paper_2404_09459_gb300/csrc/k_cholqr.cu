// CholeskyQR2 of a tall M x l block (l <= 64) as one cooperative, persistent
// kernel: the re-orthonormalisation of the basis extraction (the "reduced QR"
// of Algorithm 1, done as shifted CholeskyQR2).
//
// One CTA per SM holds up to 160 rows of Y in shared memory for the whole
// call, so the intermediate Q1 = Y R1^{-1} never goes to HBM.  Per pass:
//   1. Gram partial of the CTA's rows (accumulated in the data type over the
//      CTA's rows, stored in FP64);
//   2. grid barrier; every CTA sums a slice of the l x l entries over all
//      partials in CTA order (deterministic) into W;
//   3. grid barrier; every CTA factors the same W (shifted on the first pass)
//      with the register-resident elimination on [W | I] and keeps R^{-1} in
//      shared memory: all CTAs take the same decisions, so none waits for
//      another;
//   4. the CTA's rows times R^{-1}, in place; a third pass runs when the second
//      factor is ill-conditioned (see below); the last pass writes Q.
// The grid barrier is a sense-reversing counter with a bounded spin: after
// about 2^22 polls a CTA sets GSVD_RAND_ERR_TIMEOUT and an abort flag that
// releases every other waiting CTA.  The launch is cooperative, so all CTAs
// are resident.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "kernels.h"

namespace gsvdr {

namespace {

constexpr int FQ_THREADS = 256;
constexpr int FQ_LP = 64;         // padded columns
constexpr int FQ_ROWS = 160;      // rows per CTA at most
constexpr int FQ_LS = FQ_LP + 4;  // row stride of the tile (16-byte rows for vector loads)
constexpr int FQ_RT = FQ_ROWS / 16;
constexpr long long FQ_SPIN_LIMIT = 1ll << 22;

struct GridBar {
  unsigned count;
  unsigned gen;
  int abort;
  int pad;
};

// Barrier over the `nctas` CTAs of one problem of the launch.
__device__ bool grid_barrier(GridBar* b, DevStatus* st, int stage, unsigned nctas) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &b->gen;
    volatile int* vab = &b->abort;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(&b->count, 1u);
    int ok = 1;
    if (arrived == nctas - 1) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      long long spins = 0;
      while (*vgen == g) {
        if (*vab) {
          ok = 0;
          break;
        }
        if (++spins > FQ_SPIN_LIMIT) {
          ok = 0;
          atomicExch(&b->abort, 1);
          set_status(st, -7, stage, -1);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    s_ok = ok && !*vab;
  }
  __syncthreads();
  return s_ok != 0;
}

// Shifted Cholesky of W (read from L2) with the inverse factor, 8 warps, the
// augmented rows in registers (as chol64_kernel).  Writes R^{-1} (zero padded to
// FQ_LP x FQ_LP, type T) to Rs.  Returns false when the factorisation failed;
// every CTA computes the same result.
template <typename T, typename TC>
__device__ bool chol_block(const double* W, int l, double shift, double tau_rel, T* Rs, DevStatus* st_dev,
                           int stage, bool report, float* cond2_out) {
  __shared__ float s_cond2;
  __shared__ TC s_row[2][128];
  __shared__ TC s_odiag[64], s_scale[64];
  __shared__ int s_bad, s_kept;
  __shared__ double s_tr;
  const int tid = threadIdx.x, w = tid >> 5, t = tid & 31;
  if (tid == 0) {
    s_bad = 0;
    s_kept = 0;
  }
  if (w == 0) {
    double tr = 0.0;
    for (int i = t; i < l; i += 32) tr += __ldcg(W + (int64_t)i * l + i);
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    if (t == 0) s_tr = tr;
  }
  __syncthreads();
  const double sh = shift * s_tr;
  TC a[8][4];
  bool bad = false;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = w + 8 * r;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int j = t + 32 * c;
      double v = (i < l && j < l) ? __ldcg(W + (int64_t)i * l + j) : 0.0;
      bad |= !isfinite(v);
      if (i == j && i < l) {
        v += sh;
        s_odiag[i] = (TC)v;
      }
      a[r][c] = (TC)v;
      a[r][2 + c] = (i == j && i < l) ? TC(1) : TC(0);
    }
  }
  if (bad) s_bad = 2;
  __syncthreads();
  // effective pivot: d when above tau times the column's own (shifted) diagonal, else that
  // floor (the column keeps its direction in the span; a later pass re-orthonormalises it);
  // 0 (column dropped) only when the floor itself is zero (a zero column)
  auto pivot = [&](int k, TC d) -> TC {
    const TC fl = (TC)tau_rel * s_odiag[k];
    return d > fl ? d : (fl > TC(0) ? fl : TC(0));
  };
  // publish row k of the augmented matrix into s_row[k & 1] (its owner warp)
  auto publish = [&](int k) {
    TC* row = s_row[k & 1];
    switch (k >> 3) {
#define FQ_PUB(R) \
  case R:          \
    for (int c = 0; c < 4; ++c) row[t + 32 * c] = a[R][c]; \
    break;
      FQ_PUB(0) FQ_PUB(1) FQ_PUB(2) FQ_PUB(3) FQ_PUB(4) FQ_PUB(5) FQ_PUB(6) FQ_PUB(7)
#undef FQ_PUB
    }
  };
  int bad_k = -1;
  if (s_bad == 0) {
    if (w == 0) publish(0);
    for (int k = 0; k < l; ++k) {
      __syncthreads();
      const TC* row = s_row[k & 1];
      const TC d = row[k];
      if (!isfinite(d)) {
        bad_k = k;
        break;
      }
      const int k1 = k + 1, w1 = k1 & 7;
      const TC pv = pivot(k, d);
      if (pv == TC(0)) {
        if (w == w1 && k1 < l) publish(k1);  // row k + 1 is unchanged by a dropped pivot
        continue;
      }
      const TC dinv = sizeof(TC) == 4 ? (TC)__frcp_rn((float)pv) : TC(1) / pv;
      TC rc[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) rc[c] = row[t + 32 * c];
      bool live[4];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        live[c] = sizeof(TC) == 4 || (32 * c < l && 32 * c + 31 > k);
        live[2 + c] = sizeof(TC) == 4 || (32 * c < l && 32 * c <= k);
      }
      if (sizeof(TC) == 4) {
        // FP32: no branches in the row loop, so its loads and FMAs overlap (f = 0 is exact)
        TC f[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int i = w + 8 * r;
          f[r] = (i > k && i < l) ? row[i] * dinv : TC(0);
        }
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) a[r][c] -= f[r] * rc[c];
      } else {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int i = w + 8 * r;
          if (i > k && i < l) {
            const TC f = row[i] * dinv;
#pragma unroll
            for (int c = 0; c < 4; ++c)
              if (live[c]) a[r][c] -= f * rc[c];
          }
        }
      }
      if (w == w1 && k1 < l) publish(k1);
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = w + 8 * r;
#pragma unroll
    for (int c = 0; c < 2; ++c)
      if (i < l && t + 32 * c == i) s_row[0][i] = a[r][c];
  }
  __syncthreads();
  if (w == 0 && bad_k < 0 && s_bad == 0) {
    int kept = 0;
    float dmin = 3.4e38f, dmax = 0.f;
    for (int i = t; i < l; i += 32) {
      const TC d = s_row[0][i];
      const TC pv = pivot(i, d);
      const bool dr = pv == TC(0);
      s_scale[i] = dr ? TC(0) : TC(1) / sqrt(pv);
      kept += dr ? 0 : 1;
      if (!dr) {
        dmin = fminf(dmin, (float)pv);
        dmax = fmaxf(dmax, (float)pv);
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      kept += __shfl_xor_sync(0xffffffffu, kept, o);
      dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
      dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    }
    if (t == 0) {
      s_kept = kept;
      s_cond2 = dmin > 0.f ? dmax / dmin : 3.4e38f;  // (max / min kept diagonal of R)^2
    }
  }
  __syncthreads();
  if (cond2_out) *cond2_out = s_cond2;
  if (bad_k >= 0 || s_bad || s_kept == 0) {
    if (report && tid == 0) set_status(st_dev, (s_bad == 2 || bad_k >= 0) ? -4 : -5, stage, bad_k);
    return false;
  }
  for (int e = tid; e < FQ_LP * FQ_LP; e += FQ_THREADS) Rs[e] = T(0);
  __syncthreads();
  // R^{-1}[c][j] = L^{-1}[j][c] / sqrt(d_j) for c <= j
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int j = w + 8 * r;
    if (j >= l) continue;
    const TC sj = s_scale[j];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int cc = t + 32 * c;
      if (cc <= j) Rs[cc * FQ_LP + j] = (T)(a[r][2 + c] * sj);
    }
  }
  __syncthreads();
  return true;
}

template <typename T, typename TC>
__global__ __launch_bounds__(FQ_THREADS, 2) void cholqr2_fused_kernel(FqBatch bt, DevStatus* st_dev) {
  // CTAs [0, p[0].ctas) work on problem 0, the next p[1].ctas on problem 1 (the two sides of
  // a pair share one launch: two CTAs per SM)
  const int pi = (bt.nprob > 1 && (int)blockIdx.x >= bt.p[0].ctas) ? 1 : 0;
  const FqProb& pr = bt.p[pi];
  const unsigned bx = blockIdx.x - (pi ? (unsigned)bt.p[0].ctas : 0u);
  const unsigned nb = (unsigned)pr.ctas;
  const T* __restrict__ Y = static_cast<const T*>(pr.Y);
  T* __restrict__ Q = static_cast<T*>(pr.Q);
  const int64_t ldy = pr.ldy, M = pr.M, rows_per = pr.rows_per, ldq = pr.ldq;
  const int l = pr.l, transpose_out = pr.transpose_out, stage = pr.stage;
  double* part = pr.part;
  double* W = pr.W;
  GridBar* bar = static_cast<GridBar*>(pr.bar);
  const double shift_coef = pr.shift_coef, tau_rel = pr.tau_rel;
  extern __shared__ __align__(16) unsigned char fq_smem[];
  T* Ys = reinterpret_cast<T*>(fq_smem);  // FQ_ROWS x FQ_LS: Y, then Q1
  T* Rs = Ys + FQ_ROWS * FQ_LS;           // FQ_LP x FQ_LP: R^{-1} of the current pass
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t r0 = (int64_t)bx * rows_per;
  const int64_t left = M - r0;
  const int rows = (int)(left < 0 ? 0 : (left < rows_per ? left : rows_per));
  for (int e = tid; e < FQ_ROWS * FQ_LP; e += FQ_THREADS) {
    const int r = e / FQ_LP, j = e % FQ_LP;
    Ys[r * FQ_LS + j] = (r < rows && j < l) ? Y[(r0 + r) * ldy + j] : T(0);
  }
  __syncthreads();
  const int64_t ll = (int64_t)l * l;
  // shifted CholeskyQR, then CholeskyQR; a third pass (as in shifted CholeskyQR3, Fukaya et
  // al. 2020) when the second factor shows that Q1 was far from orthonormal, so that Q2 can
  // be off by kappa(R2)^2 u: above ~1e-12 (FP64) or ~1e-6 (FP32)
  const float cond2_max = sizeof(T) == 8 ? 1e4f : 16.f;
  bool third = false;
  for (int pass = 0; pass < 3; ++pass) {
    if (pass == 2 && !third) break;
    // 1. Gram partial of the tile: thread (ty, tx) forms the 4 x 4 block (4 ty.., 4 tx..);
    //    the upper blocks are stored
    {
      const int i0 = ty * 4, j0 = tx * 4;
      T g[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) g[a][b] = T(0);
#pragma unroll 4
      for (int r = 0; r < rows; ++r) {
        const T* yr = Ys + r * FQ_LS;
        T x[4], y[4];
        if (sizeof(T) == 4) {
          const float4 xv = *reinterpret_cast<const float4*>(yr + i0);
          const float4 yv = *reinterpret_cast<const float4*>(yr + j0);
          x[0] = xv.x; x[1] = xv.y; x[2] = xv.z; x[3] = xv.w;
          y[0] = yv.x; y[1] = yv.y; y[2] = yv.z; y[3] = yv.w;
        } else {
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            x[a] = yr[i0 + a];
            y[a] = yr[j0 + a];
          }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) g[a][b] = fma(x[a], y[b], g[a][b]);
      }
      if (tx >= ty) {
        double* P = part + (int64_t)bx * ll;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int i = i0 + a, j = j0 + b;
            if (i < l && j < l && j >= i) P[(int64_t)i * l + j] = (double)g[a][b];
          }
      }
    }
    if (!grid_barrier(bar, st_dev, stage + pass, nb)) return;
    // 2. W = sum of the partials (upper entries, mirrored): a warp per entry, lanes over
    //    the partials, a fixed shuffle tree (deterministic)
    {
      const int warp = tid >> 5, lane = tid & 31;
      for (int64_t e = (int64_t)bx * (FQ_THREADS / 32) + warp; e < ll; e += (int64_t)nb * (FQ_THREADS / 32)) {
        const int i = (int)(e / l), j = (int)(e % l);
        if (j < i) continue;
        double s = 0.0;
        for (unsigned c = lane; c < nb; c += 32) s += __ldcg(part + (int64_t)c * ll + e);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
          W[(int64_t)i * l + j] = s;
          W[(int64_t)j * l + i] = s;
        }
      }
    }
    if (!grid_barrier(bar, st_dev, stage + pass, nb)) return;
    // 3. R^{-1} in every CTA (every CTA takes the same decisions).  When the third
    //    pass finds Q2 orthonormal to first order (max |W - I| <= 0.05), one
    //    Newton-Schulz step X = (3 I - W) / 2 (error O(||W - I||^2)) takes the place
    //    of the Cholesky; a Q2 further off (clamped pivots) gets a full CholeskyQR.
    bool newton = false;
    if (pass == 2) {
      __shared__ float s_dev[FQ_THREADS / 32];
      float dv = 0.f;
      for (int64_t e = tid; e < ll; e += FQ_THREADS) {
        const int i = (int)(e / l), j = (int)(e % l);
        dv = fmaxf(dv, (float)fabs(__ldcg(W + e) - (i == j ? 1.0 : 0.0)));
      }
      for (int o = 16; o > 0; o >>= 1) dv = fmaxf(dv, __shfl_xor_sync(0xffffffffu, dv, o));
      if ((tid & 31) == 0) s_dev[tid >> 5] = dv;
      __syncthreads();
      float mx = 0.f;
      for (int q = 0; q < FQ_THREADS / 32; ++q) mx = fmaxf(mx, s_dev[q]);
      newton = mx <= 0.05f;
      __syncthreads();
    }
    if (!newton) {
      float cond2 = 0.f;
      if (!chol_block<T, TC>(W, l, pass == 0 ? shift_coef : 0.0, tau_rel, Rs, st_dev, stage + (pass > 0),
                             bx == 0, &cond2))
        return;
      if (pass == 1) third = cond2 > cond2_max;
    } else {
      for (int e = tid; e < FQ_LP * FQ_LP; e += FQ_THREADS) {
        const int i = e / FQ_LP, j = e % FQ_LP;
        double v = 0.0;
        if (i < l && j < l) v = (i == j ? 1.5 : 0.0) - 0.5 * __ldcg(W + (int64_t)i * l + j);
        Rs[e] = (T)v;
      }
      __syncthreads();
    }
    // 4. rows x R^{-1}
    T acc[FQ_RT][4];
#pragma unroll
    for (int a = 0; a < FQ_RT; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    for (int i = 0; i < l; ++i) {
      T bv[4];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Rs[i * FQ_LP + tx * 4 + b];
#pragma unroll
      for (int a = 0; a < FQ_RT; ++a) {
        const T av = Ys[(ty + 16 * a) * FQ_LS + i];
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av, bv[b], acc[a][b]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < FQ_RT; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) Ys[(ty + 16 * a) * FQ_LS + tx * 4 + b] = acc[a][b];
    __syncthreads();
  }
  if (transpose_out) {
    for (int e = tid; e < rows * l; e += FQ_THREADS) {
      const int j = e / rows, r = e % rows;
      Q[(int64_t)j * ldq + r0 + r] = Ys[r * FQ_LS + j];
    }
  } else {
    for (int e = tid; e < rows * l; e += FQ_THREADS) {
      const int r = e / l, j = e % l;
      Q[(r0 + r) * ldq + j] = Ys[r * FQ_LS + j];
    }
  }
}

template <typename T>
size_t fq_smem_bytes() {
  return ((size_t)FQ_ROWS * FQ_LS + (size_t)FQ_LP * FQ_LP) * sizeof(T);
}

}  // namespace

size_t cholqr2_fused_bar_bytes() { return sizeof(GridBar); }
int cholqr2_fused_max_ctas() { return 160; }

template <typename T, typename TC>
int cholqr2_fused_plan(int64_t M, int l, int64_t* rows_per) {
  if (l < 1 || l > FQ_LP) return 0;
  // per device: SM count and resident CTAs per SM of this instantiation, looked up once
  // under a lock (the batched workers call this concurrently)
  static std::mutex mu;
  static int cached[64][2] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  int sms_c, per_c;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (cached[dev][0] == 0) {
      int sms = 0, per_sm = 0;
      const size_t smem = fq_smem_bytes<T>();
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          cudaFuncSetAttribute(cholqr2_fused_kernel<T, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
              cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cholqr2_fused_kernel<T, TC>, FQ_THREADS, smem) !=
              cudaSuccess) {
        cudaGetLastError();
        cached[dev][0] = -1;
      } else {
        cached[dev][1] = per_sm;
        cached[dev][0] = sms;
      }
    }
    sms_c = cached[dev][0];
    per_c = cached[dev][1];
  }
  if (sms_c <= 0 || per_c < 1) return 0;
  const int64_t max_ctas = std::min<int64_t>((int64_t)sms_c * per_c, cholqr2_fused_max_ctas());
  // FP64 tiles stay short: at the FP64 rate a full tile is too slow for one SM
  const int64_t row_cap = sizeof(T) == 8 ? 32 : FQ_ROWS;
  int64_t ctas = std::min<int64_t>(std::min<int64_t>(sms_c, max_ctas), cdiv(M, 16));
  const int64_t rp = cdiv(M, ctas);
  if (rp > row_cap) return 0;
  *rows_per = rp;
  return (int)cdiv(M, rp);
}

template <typename T, typename TC>
cudaError_t launch_cholqr2_fused_n(const FqBatch& bt, DevStatus* st_dev, cudaStream_t st) {
  const size_t smem = fq_smem_bytes<T>();
  FqBatch b = bt;
  int ctas = 0;
  for (int i = 0; i < b.nprob; ++i) ctas += b.p[i].ctas;
  void* args[] = {(void*)&b, (void*)&st_dev};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)cholqr2_fused_kernel<T, TC>, dim3((unsigned)ctas),
                                              dim3(FQ_THREADS), args, smem, st);
  if (e != cudaSuccess) return e;
  return launched();
}

template <typename T, typename TC>
cudaError_t launch_cholqr2_fused(const T* Y, int64_t ldy, int64_t M, int l, int ctas, int64_t rows_per, T* Q,
                                 int64_t ldq, int transpose_out, double* part, double* W, void* bar,
                                 double shift_coef, double tau_rel, DevStatus* st_dev, int stage, cudaStream_t st) {
  FqBatch b;
  memset(&b, 0, sizeof(b));
  b.nprob = 1;
  b.p[0] = FqProb{Y, ldy, M, rows_per, Q, ldq, part, W, bar, shift_coef, tau_rel, l, ctas, transpose_out, stage};
  return launch_cholqr2_fused_n<T, TC>(b, st_dev, st);
}

template <typename T, typename TC>
int cholqr2_fused_max_total_ctas() {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, cholqr2_fused_kernel<T, TC>, FQ_THREADS, fq_smem_bytes<T>()) !=
          cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return sms * per;
}

template int cholqr2_fused_plan<float, float>(int64_t, int, int64_t*);
template int cholqr2_fused_plan<float, double>(int64_t, int, int64_t*);
template int cholqr2_fused_plan<double, double>(int64_t, int, int64_t*);
template cudaError_t launch_cholqr2_fused_n<float, float>(const FqBatch&, DevStatus*, cudaStream_t);
template cudaError_t launch_cholqr2_fused_n<float, double>(const FqBatch&, DevStatus*, cudaStream_t);
template cudaError_t launch_cholqr2_fused_n<double, double>(const FqBatch&, DevStatus*, cudaStream_t);
template int cholqr2_fused_max_total_ctas<float, float>();
template int cholqr2_fused_max_total_ctas<float, double>();
template int cholqr2_fused_max_total_ctas<double, double>();
template cudaError_t launch_cholqr2_fused<float, float>(const float*, int64_t, int64_t, int, int, int64_t, float*,
                                                        int64_t, int, double*, double*, void*, double, double,
                                                        DevStatus*, int, cudaStream_t);
template cudaError_t launch_cholqr2_fused<float, double>(const float*, int64_t, int64_t, int, int, int64_t, float*,
                                                         int64_t, int, double*, double*, void*, double, double,
                                                         DevStatus*, int, cudaStream_t);
template cudaError_t launch_cholqr2_fused<double, double>(const double*, int64_t, int64_t, int, int, int64_t,
                                                          double*, int64_t, int, double*, double*, void*, double,
                                                          double, DevStatus*, int, cudaStream_t);

}  // namespace gsvdr
