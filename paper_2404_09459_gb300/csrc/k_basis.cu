// Basis-extraction kernels on CUDA cores: Gaussian test matrices, the sketch
// and power products (the FP64 / FP32 paths), split-K reduction, the Gram
// matrix, the shifted Cholesky factorisation and the triangular apply of
// CholeskyQR2.  Tensor-core products live in k_tc.cu.
#include <algorithm>

#include "kernels.h"

namespace gsvdr {

// ============================================================================
// Gaussian test matrices
// ============================================================================
__global__ void philox_words_kernel(uint32_t* out, uint64_t count, uint32_t k0, uint32_t k1,
                                    uint32_t pair, uint32_t side, uint32_t stream) {
  uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  Philox4 w = philox4x32_10((uint32_t)t, pair, side, stream, k0, k1);
  uint4 v = make_uint4(w.x[0], w.x[1], w.x[2], w.x[3]);
  reinterpret_cast<uint4*>(out)[t] = v;
}

cudaError_t launch_philox_words(uint32_t* out, uint64_t count, uint64_t seed, uint32_t pair,
                                uint32_t side, uint32_t stream, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  unsigned blocks = (unsigned)cdiv((int64_t)count, 256);
  philox_words_kernel<<<blocks, 256, 0, st>>>(out, count, (uint32_t)seed, (uint32_t)(seed >> 32), pair,
                                              side, stream);
  return launched();
}

__global__ void gaussian_rowmajor_kernel(double* out, int64_t total, uint32_t k0, uint32_t k1,
                                         uint32_t pair, uint32_t side, uint32_t stream) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * t >= total) return;
  Philox4 w = philox4x32_10((uint32_t)t, pair, side, stream, k0, k1);
  double z0, z1;
  box_muller_f64(w, z0, z1);
  out[2 * t] = z0;
  if (2 * t + 1 < total) out[2 * t + 1] = z1;
}

cudaError_t launch_gaussian_rowmajor(double* out, int64_t n, int64_t l, uint64_t seed, uint32_t pair,
                                     uint32_t side, uint32_t stream, cudaStream_t st) {
  int64_t total = n * l;
  if (total == 0) return cudaSuccess;
  int64_t pairs = (total + 1) / 2;
  gaussian_rowmajor_kernel<<<(unsigned)cdiv(pairs, 256), 256, 0, st>>>(
      out, total, (uint32_t)seed, (uint32_t)(seed >> 32), pair, side, stream);
  return launched();
}

template <typename T>
__device__ __forceinline__ T gaussian_at(int64_t e, uint32_t k0, uint32_t k1, uint32_t pair,
                                         uint32_t side, uint32_t stream);
template <>
__device__ __forceinline__ double gaussian_at<double>(int64_t e, uint32_t k0, uint32_t k1,
                                                      uint32_t pair, uint32_t side, uint32_t stream) {
  Philox4 w = philox4x32_10((uint32_t)(e >> 1), pair, side, stream, k0, k1);
  double z0, z1;
  box_muller_f64(w, z0, z1);
  return (e & 1) ? z1 : z0;
}
template <>
__device__ __forceinline__ float gaussian_at<float>(int64_t e, uint32_t k0, uint32_t k1,
                                                    uint32_t pair, uint32_t side, uint32_t stream) {
  Philox4 w = philox4x32_10((uint32_t)(e >> 1), pair, side, stream, k0, k1);
  float z0, z1;
  box_muller_f32(w, z0, z1);
  return (e & 1) ? z1 : z0;
}

template <typename T>
__global__ void gaussian_kmajor_kernel(T* Xt, int64_t ldx, int64_t n, int l, int lrows, uint32_t k0,
                                       uint32_t k1, uint32_t pair, uint32_t side, uint32_t stream) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // column of Xt (row of Omega)
  int j = blockIdx.y;                                          // row of Xt (column of Omega)
  if (i >= ldx || j >= lrows) return;
  T v = T(0);
  if (i < n && j < l) v = gaussian_at<T>(i * (int64_t)l + j, k0, k1, pair, side, stream);
  Xt[(int64_t)j * ldx + i] = v;
}

template <typename T>
cudaError_t launch_gaussian_kmajor(T* Xt, int64_t ldx, int64_t n, int l, int lrows, uint64_t seed,
                                   uint32_t pair, uint32_t side, uint32_t stream, cudaStream_t st) {
  dim3 grid((unsigned)cdiv(ldx, 256), (unsigned)lrows);
  gaussian_kmajor_kernel<T><<<grid, 256, 0, st>>>(Xt, ldx, n, l, lrows, (uint32_t)seed,
                                                  (uint32_t)(seed >> 32), pair, side, stream);
  return launched();
}
template cudaError_t launch_gaussian_kmajor<double>(double*, int64_t, int64_t, int, int, uint64_t,
                                                    uint32_t, uint32_t, uint32_t, cudaStream_t);
template cudaError_t launch_gaussian_kmajor<float>(float*, int64_t, int64_t, int, int, uint64_t,
                                                   uint32_t, uint32_t, uint32_t, cudaStream_t);

// ============================================================================
// Sum of squares accumulators: FP64 for double data, double-float (Knuth
// TwoSum on exact FMA products) for float data, so that ||G||_F^2 keeps about
// 44 bits while the arithmetic stays on the FP32 pipes.
// ============================================================================
template <typename T>
struct SqAcc;
template <>
struct SqAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s = fma(v, v, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct SqAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float v) {
    float p = v * v;
    float e = fmaf(v, v, -p);
    float t = hi + p;
    float z = t - hi;
    float err = (hi - (t - z)) + (p - z);
    hi = t;
    lo += err + e;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

__device__ double block_sum_double(double v) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  __syncthreads();
  if (ln == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) s += red[i];
  }
  return s;  // valid in thread 0
}

// ============================================================================
// Y = G X on CUDA cores.  64 x 64 output tile per CTA, 16-deep K slices.
// ============================================================================
constexpr int GX_BM = 64, GX_BN = 64, GX_BK = 16;

template <typename T>
__global__ __launch_bounds__(256) void gemm_gx_kernel(const T* __restrict__ G, int64_t ldg, int64_t M,
                                                      int64_t n, const T* __restrict__ Xt, int64_t ldx,
                                                      int l, T* __restrict__ Y, int64_t ldy,
                                                      double* gnorm_part) {
  __shared__ T As[GX_BK][GX_BM + 1];
  __shared__ T Bs[GX_BK][GX_BN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t row0 = (int64_t)blockIdx.x * GX_BM;
  const int col0 = blockIdx.y * GX_BN;
  const bool do_norm = gnorm_part != nullptr && blockIdx.y == 0;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  SqAcc<T> sq;
  for (int64_t k0 = 0; k0 < n; k0 += GX_BK) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int r = (tid >> 4) + 16 * i, c = tid & 15;
      int64_t gr = row0 + r, gc = k0 + c;
      T v = (gr < M && gc < n) ? G[gr * ldg + gc] : T(0);
      As[c][r] = v;
      if (do_norm) sq.add(v);
      int64_t gj = col0 + r;
      Bs[c][r] = (gj < l && gc < n) ? Xt[gj * ldx + gc] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GX_BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) a[m] = As[kk][ty * 4 + m];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = Bs[kk][tx * 4 + q];
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[m][q] = fma(a[m], b[q], acc[m][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    int64_t r = row0 + ty * 4 + m;
    if (r >= M) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int c = col0 + tx * 4 + q;
      if (c < l) Y[r * ldy + c] = acc[m][q];
    }
  }
  if (do_norm) {
    double s = block_sum_double(sq.value());
    if (threadIdx.x == 0) gnorm_part[blockIdx.x] = s;
  }
}

int gemm_gx_simt_ctas(int64_t M) { return (int)cdiv(M, GX_BM); }

template <typename T>
cudaError_t launch_gemm_gx_simt(const T* G, int64_t ldg, int64_t M, int64_t n, const T* Xt,
                                int64_t ldx, int l, T* Y, int64_t ldy, double* gnorm_part,
                                cudaStream_t st) {
  dim3 grid((unsigned)cdiv(M, GX_BM), (unsigned)cdiv(l, GX_BN));
  gemm_gx_kernel<T><<<grid, 256, 0, st>>>(G, ldg, M, n, Xt, ldx, l, Y, ldy, gnorm_part);
  return launched();
}
template cudaError_t launch_gemm_gx_simt<double>(const double*, int64_t, int64_t, int64_t,
                                                 const double*, int64_t, int, double*, int64_t,
                                                 double*, cudaStream_t);
template cudaError_t launch_gemm_gx_simt<float>(const float*, int64_t, int64_t, int64_t,
                                                const float*, int64_t, int, float*, int64_t, double*,
                                                cudaStream_t);

// ============================================================================
// Split-K partials of Z = G^T Q on CUDA cores.  Output tile 64 (columns of G)
// x 64 (columns of Q); K runs over the rows of one split, 16 rows per slice.
// ============================================================================
constexpr int GT_BC = 64, GT_BJ = 64, GT_BK = 16;

template <typename T, typename TP>
__global__ __launch_bounds__(256) void gemm_gtq_kernel(const T* __restrict__ G, int64_t ldg, int64_t M,
                                                       int64_t n, const T* __restrict__ Q, int64_t ldq,
                                                       int l, TP* __restrict__ part, int64_t lp,
                                                       int64_t rows_per_split) {
  __shared__ T Gs[GT_BK][GT_BC + 1];
  __shared__ T Qs[GT_BK][GT_BJ + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t c0 = (int64_t)blockIdx.x * GT_BC;
  const int j0 = blockIdx.y * GT_BJ;
  const int z = blockIdx.z;
  const int64_t rbeg = (int64_t)z * rows_per_split;
  const int64_t rend = min(M, rbeg + rows_per_split);
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int64_t r0 = rbeg; r0 < rend; r0 += GT_BK) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int rr = (tid >> 6) + 4 * i, cc = tid & 63;
      int64_t gr = r0 + rr;
      bool rok = gr < rend;
      int64_t gc = c0 + cc;
      Gs[rr][cc] = (rok && gc < n) ? G[gr * ldg + gc] : T(0);
      int gj = j0 + cc;
      Qs[rr][cc] = (rok && gj < l) ? Q[gr * ldq + gj] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GT_BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) a[m] = Gs[kk][ty * 4 + m];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = Qs[kk][tx * 4 + q];
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[m][q] = fma(a[m], b[q], acc[m][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    int64_t c = c0 + ty * 4 + m;
    if (c >= n) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int j = j0 + tx * 4 + q;
      if (j < l) part[((int64_t)z * n + c) * lp + j] = (TP)acc[m][q];
    }
  }
}

int gemm_gtq_splits(int64_t M, int64_t n, int l, int64_t max_part_elems) {
  int64_t tiles = cdiv(n, GT_BC) * cdiv(l, GT_BJ);
  int64_t want = std::max<int64_t>(1, (4 * 152) / tiles);
  int64_t maxs = std::max<int64_t>(1, cdiv(M, 128));
  int64_t s = std::min(want, maxs);
  int64_t lp = round_up(l, 4);
  while (s > 1 && s * n * lp > max_part_elems) --s;
  return (int)std::min<int64_t>(s, 1024);
}

template <typename T, typename TP>
cudaError_t launch_gemm_gtq_simt(const T* G, int64_t ldg, int64_t M, int64_t n, const T* Q,
                                 int64_t ldq, int l, TP* part, int64_t lp, int splits,
                                 cudaStream_t st) {
  int64_t rps = round_up(cdiv(M, splits), GT_BK);
  dim3 grid((unsigned)cdiv(n, GT_BC), (unsigned)cdiv(l, GT_BJ), (unsigned)splits);
  gemm_gtq_kernel<T, TP><<<grid, 256, 0, st>>>(G, ldg, M, n, Q, ldq, l, part, lp, rps);
  return launched();
}
template cudaError_t launch_gemm_gtq_simt<double, double>(const double*, int64_t, int64_t, int64_t,
                                                          const double*, int64_t, int, double*,
                                                          int64_t, int, cudaStream_t);
template cudaError_t launch_gemm_gtq_simt<float, float>(const float*, int64_t, int64_t, int64_t,
                                                        const float*, int64_t, int, float*, int64_t,
                                                        int, cudaStream_t);

// Deterministic split reduction (FP64 accumulation, split order).
template <typename TP, typename T>
__global__ void reduce_splits_kernel(const TP* __restrict__ part, int splits, int64_t n, int l,
                                     int64_t lp, T* __restrict__ Z, int64_t ldz, int transpose_out,
                                     double* sq_part) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t total = n * l;
  double v = 0.0;
  double sq = 0.0;
  if (e < total) {
    int64_t c, j;
    if (transpose_out) {  // thread order along c for coalesced writes of B (l x n)
      j = e / n;
      c = e % n;
    } else {
      c = e / l;
      j = e % l;
    }
    const TP* p = part + c * lp + j;
    for (int z = 0; z < splits; ++z) v += (double)p[(int64_t)z * n * lp];
    T out = (T)v;
    if (transpose_out)
      Z[j * ldz + c] = out;
    else
      Z[c * ldz + j] = out;
    sq = (double)out * (double)out;
  }
  if (sq_part) {
    double s = block_sum_double(sq);
    if (threadIdx.x == 0) sq_part[blockIdx.x] = s;
  }
}

template <typename TP, typename T>
cudaError_t launch_reduce_splits(const TP* part, int splits, int64_t n, int l, int64_t lp, T* Z,
                                 int64_t ldz, int transpose_out, double* sq_part, int* sq_blocks,
                                 cudaStream_t st) {
  int64_t total = n * l;
  unsigned blocks = (unsigned)cdiv(total, 256);
  if (sq_blocks) *sq_blocks = (int)blocks;
  reduce_splits_kernel<TP, T><<<blocks, 256, 0, st>>>(part, splits, n, l, lp, Z, ldz, transpose_out,
                                                      sq_part);
  return launched();
}
template cudaError_t launch_reduce_splits<double, double>(const double*, int, int64_t, int, int64_t,
                                                          double*, int64_t, int, double*, int*,
                                                          cudaStream_t);
template cudaError_t launch_reduce_splits<float, float>(const float*, int, int64_t, int, int64_t,
                                                        float*, int64_t, int, double*, int*,
                                                        cudaStream_t);

// ============================================================================
// Gram partials W_c = Y_c^T Y_c over row chunks; 64 x 64 output tiles, upper
// tiles only (ti <= tj).  Accumulation in T over one chunk, FP64 across chunks.
// ============================================================================
constexpr int GR_T = 64, GR_BK = 16;

template <typename T>
__global__ __launch_bounds__(256) void gram_partial_kernel(const T* __restrict__ Y, int64_t ldy,
                                                           int64_t M, int l, double* __restrict__ part,
                                                           int64_t rows_per_chunk) {
  const int ti = blockIdx.y, tj = blockIdx.z;
  if (ti > tj) return;
  __shared__ T As[GR_BK][GR_T + 1];
  __shared__ T Bs[GR_BK][GR_T + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int c = blockIdx.x;
  const int64_t rbeg = (int64_t)c * rows_per_chunk, rend = min(M, rbeg + rows_per_chunk);
  const int i0 = ti * GR_T, j0 = tj * GR_T;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int64_t r0 = rbeg; r0 < rend; r0 += GR_BK) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int rr = (tid >> 6) + 4 * i, cc = tid & 63;
      int64_t gr = r0 + rr;
      bool rok = gr < rend;
      As[rr][cc] = (rok && i0 + cc < l) ? Y[gr * ldy + i0 + cc] : T(0);
      Bs[rr][cc] = (rok && j0 + cc < l) ? Y[gr * ldy + j0 + cc] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GR_BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) a[m] = As[kk][ty * 4 + m];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = Bs[kk][tx * 4 + q];
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[m][q] = fma(a[m], b[q], acc[m][q]);
    }
    __syncthreads();
  }
  double* P = part + (int64_t)c * l * l;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    int i = i0 + ty * 4 + m;
    if (i >= l) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int j = j0 + tx * 4 + q;
      if (j < l && j >= i) P[(int64_t)i * l + j] = (double)acc[m][q];
    }
  }
}

int gram_chunks(int64_t M, int l, int64_t* rows_per_chunk) {
  int64_t t = cdiv(l, GR_T);
  int64_t upper = t * (t + 1) / 2;
  int64_t chunks = std::max<int64_t>(1, (2 * 152) / upper);
  chunks = std::min<int64_t>(chunks, std::max<int64_t>(1, cdiv(M, 64)));
  // keep the partial buffer <= 8M doubles
  while (chunks > 1 && chunks * (int64_t)l * l > (8ll << 20)) --chunks;
  int64_t rpc = round_up(cdiv(M, chunks), GR_BK);
  chunks = (int)cdiv(M, rpc);
  *rows_per_chunk = rpc;
  return (int)chunks;
}

template <typename T>
cudaError_t launch_gram_partial(const T* Y, int64_t ldy, int64_t M, int l, double* part, int chunks,
                                int64_t rows_per_chunk, cudaStream_t st) {
  int t = (int)cdiv(l, GR_T);
  dim3 grid((unsigned)chunks, (unsigned)t, (unsigned)t);
  gram_partial_kernel<T><<<grid, 256, 0, st>>>(Y, ldy, M, l, part, rows_per_chunk);
  return launched();
}
template cudaError_t launch_gram_partial<double>(const double*, int64_t, int64_t, int, double*, int,
                                                 int64_t, cudaStream_t);
template cudaError_t launch_gram_partial<float>(const float*, int64_t, int64_t, int, double*, int,
                                                int64_t, cudaStream_t);

// W[i][j] = W[j][i] = sum_c part[c][min(i,j)][max(i,j)], one warp per entry
// (fixed lane/shuffle order: deterministic).
__global__ void gram_reduce_kernel(const double* __restrict__ part, int chunks, int l,
                                   double* __restrict__ W) {
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= (int64_t)l * l) return;
  const int i = (int)(wid / l), j = (int)(wid % l);
  if (j < i) return;
  const double* p = part + (int64_t)i * l + j;
  double s = 0.0;
  for (int c = lane; c < chunks; c += 32) s += p[(int64_t)c * l * l];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) {
    W[(int64_t)i * l + j] = s;
    W[(int64_t)j * l + i] = s;
  }
}

cudaError_t launch_gram_reduce(const double* part, int chunks, int l, double* W, cudaStream_t st) {
  const int64_t threads = (int64_t)l * l * 32;
  gram_reduce_kernel<<<(unsigned)cdiv(threads, 256), 256, 0, st>>>(part, chunks, l, W);
  return launched();
}

// ============================================================================
// Shifted Cholesky, one CTA of 32 x 32 threads, full storage (odd stride) in
// shared memory: right-looking with the unscaled pivot row, one barrier per
// step.  Then R^{-1} by back substitution, one warp per column.
// ============================================================================
template <typename TC>
__global__ __launch_bounds__(1024) void chol_shift_kernel(const double* __restrict__ W, int l,
                                                          double shift_coef, double tau_rel,
                                                          TC* __restrict__ Rinv, DevStatus* st_dev,
                                                          int stage, TC* gscr, int use_smem) {
  extern __shared__ unsigned char smem_raw[];
  const int lda = l | 1;
  TC* A = use_smem ? reinterpret_cast<TC*>(smem_raw) : gscr;  // l x lda: A, later R
  TC* X = A + (int64_t)l * lda;                               // l x lda: R^{-1}
  __shared__ double s_shift;
  __shared__ int s_bad;
  __shared__ TC s_odiag[256];
  __shared__ unsigned char s_drop[256];
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  if (tid == 0) {
    double tr = 0.0;
    bool fin = true;
    for (int i = 0; i < l; ++i) {
      double d = W[(int64_t)i * l + i];
      tr += d;
      fin = fin && isfinite(d);
    }
    s_shift = shift_coef * tr;
    s_bad = fin ? 0 : 2;
  }
  __syncthreads();
  const double sh = s_shift;
  for (int i = ty; i < l; i += 32)
    for (int j = tx; j < l; j += 32) {
      double v = W[(int64_t)i * l + j] + (i == j ? sh : 0.0);
      if (!isfinite(v)) s_bad = 2;
      A[(int64_t)i * lda + j] = (TC)v;
      if (i == j) {
        s_odiag[i] = (TC)v;
        s_drop[i] = 0;
      }
    }
  __syncthreads();
  int bad_k = -1;
  if (s_bad == 0) {
    for (int k = 0; k < l; ++k) {
      const TC d = A[(int64_t)k * lda + k];
      if (!isfinite(d)) {
        bad_k = k;
        break;
      }
      // A pivot not above the Gram's resolution relative to its own column is
      // numerically dependent on the previous columns: drop it (its column of
      // Q becomes zero and adds a zero row to Q^T G).
      if (!(d > (TC)tau_rel * s_odiag[k])) {
        if (tid == 0) s_drop[k] = 1;
        continue;
      }
      const TC dinv = TC(1) / d;
      const TC* rowk = A + (int64_t)k * lda;
      for (int i = k + 1 + ty; i < l; i += 32) {
        const TC aki = rowk[i] * dinv;
        TC* ai = A + (int64_t)i * lda;
        for (int j = k + 1 + tx; j < l; j += 32)
          if (j >= i) ai[j] -= aki * rowk[j];
      }
      __syncthreads();
    }
  }
  __syncthreads();
  int kept = 0;
  for (int i = 0; i < l; ++i) kept += s_drop[i] ? 0 : 1;
  if (bad_k >= 0 || s_bad || kept == 0) {
    if (tid == 0) set_status(st_dev, (s_bad == 2 || bad_k >= 0) ? -4 : -5, stage, bad_k);
    return;
  }
  // R = rows scaled by 1/sqrt(pivot) (rows of dropped pivots = e_k), in place
  for (int i = ty; i < l; i += 32) {
    const bool dr = s_drop[i] != 0;
    const TC rk = dr ? TC(1) : sqrt(A[(int64_t)i * lda + i]);
    for (int j = tx; j < l; j += 32) {
      TC v = TC(0);
      if (j == i) v = rk;
      else if (j > i && !dr) v = A[(int64_t)i * lda + j] / rk;
      // written after every thread has read its pivot: separate pass below
      X[(int64_t)i * lda + j] = v;
    }
  }
  __syncthreads();
  for (int i = ty; i < l; i += 32)
    for (int j = tx; j < l; j += 32) A[(int64_t)i * lda + j] = X[(int64_t)i * lda + j];
  __syncthreads();
  // R^{-1}: column j by back substitution, X[i][j] = -(sum_{k=i+1..j} R[i][k] X[k][j]) / R[i][i]
  for (int j = ty; j < l; j += 32) {
    for (int i = j + 1 + tx; i < l; i += 32) X[(int64_t)i * lda + j] = TC(0);
    if (tx == 0) X[(int64_t)j * lda + j] = TC(1) / A[(int64_t)j * lda + j];
    __syncwarp();
    for (int i = j - 1; i >= 0; --i) {
      TC s = TC(0);
      for (int k = i + 1 + tx; k <= j; k += 32) s += A[(int64_t)i * lda + k] * X[(int64_t)k * lda + j];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (tx == 0) X[(int64_t)i * lda + j] = -s / A[(int64_t)i * lda + i];
      __syncwarp();
    }
  }
  __syncthreads();
  // dropped columns of Y contribute nothing: zero column k of R^{-1}
  for (int i = ty; i < l; i += 32)
    for (int j = tx; j < l; j += 32) {
      TC v = (j >= i && !s_drop[j]) ? X[(int64_t)i * lda + j] : TC(0);
      Rinv[(int64_t)i * l + j] = v;
    }
}

int64_t chol_scratch_elems(int l) { return 2ll * l * (l | 1); }

template <typename TC>
cudaError_t launch_chol_shift(const double* W, int l, double shift_coef, double tau_rel, TC* Rinv,
                              TC* scratch, DevStatus* st_dev, int stage, cudaStream_t st) {
  if (l < 1 || l > 256) return cudaErrorInvalidValue;
  size_t smem = (size_t)chol_scratch_elems(l) * sizeof(TC);
  int use_smem = smem <= 200 * 1024;
  cudaFuncSetAttribute(chol_shift_kernel<TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  chol_shift_kernel<TC><<<1, 1024, use_smem ? smem : 0, st>>>(W, l, shift_coef, tau_rel, Rinv, st_dev, stage,
                                                              scratch, use_smem);
  return launched();
}
template cudaError_t launch_chol_shift<double>(const double*, int, double, double, double*, double*,
                                               DevStatus*, int, cudaStream_t);
template cudaError_t launch_chol_shift<float>(const double*, int, double, double, float*, float*,
                                              DevStatus*, int, cudaStream_t);

// ============================================================================
// Q = Y R^{-1} (R^{-1} upper triangular, staged in shared memory) over a tile
// of rows per CTA; optional Gram partial of the produced rows (one chunk per
// CTA) and optional transposed store Qt[j * ldq + row].
// ============================================================================
int64_t apply_rows_per_cta(int l) { return l <= 64 ? 128 : (l <= 128 ? 64 : 32); }
int apply_ctas(int64_t M, int l) { return (int)cdiv(M, apply_rows_per_cta(l)); }

template <typename T, typename TC>
__global__ __launch_bounds__(256) void apply_rinv_kernel(const T* __restrict__ Y, int64_t ldy, int64_t M, int l,
                                                         const TC* __restrict__ Rinv, T* Q, int64_t ldq,
                                                         int transpose_out, double* part, int64_t rpc,
                                                         int r_smem) {
  extern __shared__ unsigned char smem_raw[];
  const int ls = l | 1;
  // R^{-1} in shared memory when it fits next to the tiles, else read through L1
  const int rld = r_smem ? ls : l;
  TC* Rsm = reinterpret_cast<TC*>(smem_raw);
  const TC* Rs = r_smem ? Rsm : Rinv;
  T* Ys = reinterpret_cast<T*>(smem_raw + (r_smem ? (size_t)l * ls * sizeof(TC) : 0));  // rpc x ls
  T* Qs = Ys + rpc * ls;                                                                 // rpc x ls
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * rpc;
  const int rows = (int)(rpc < M - r0 ? rpc : M - r0);
  if (r_smem)
    for (int e = tid; e < l * l; e += nt) {
      int i = e / l, j = e % l;
      Rsm[i * ls + j] = Rinv[e];
    }
  for (int e = tid; e < rows * l; e += nt) {
    int r = e / l, j = e % l;
    Ys[r * ls + j] = Y[(r0 + r) * ldy + j];
  }
  __syncthreads();
  // q[r][j] = sum_{i <= j} y[r][i] Rinv[i][j]; thread -> (r, j) with j fastest
  for (int e = tid; e < rows * l; e += nt) {
    const int r = e / l, j = e % l;
    const T* y = Ys + r * ls;
    T a0 = T(0), a1 = T(0);
    int i = 0;
    for (; i + 1 <= j; i += 2) {
      a0 = fma(y[i], (T)Rs[i * rld + j], a0);
      a1 = fma(y[i + 1], (T)Rs[(i + 1) * rld + j], a1);
    }
    if (i <= j) a0 = fma(y[i], (T)Rs[i * rld + j], a0);
    Qs[r * ls + j] = a0 + a1;
  }
  __syncthreads();
  if (transpose_out) {
    for (int e = tid; e < rows * l; e += nt) {
      int j = e / rows, r = e % rows;
      Q[(int64_t)j * ldq + r0 + r] = Qs[r * ls + j];
    }
  } else {
    for (int e = tid; e < rows * l; e += nt) {
      int r = e / l, j = e % l;
      Q[(r0 + r) * ldq + j] = Qs[r * ls + j];
    }
  }
  if (part) {
    double* P = part + (int64_t)blockIdx.x * l * l;
    for (int e = tid; e < l * l; e += nt) {
      int i = e / l, j = e % l;
      if (j < i) continue;
      T s0 = T(0), s1 = T(0);
      int r = 0;
      for (; r + 1 < rows; r += 2) {
        s0 = fma(Qs[r * ls + i], Qs[r * ls + j], s0);
        s1 = fma(Qs[(r + 1) * ls + i], Qs[(r + 1) * ls + j], s1);
      }
      if (r < rows) s0 = fma(Qs[r * ls + i], Qs[r * ls + j], s0);
      P[e] = (double)s0 + (double)s1;
    }
  }
}

template <typename T, typename TC>
cudaError_t launch_apply_rinv(const T* Y, int64_t ldy, int64_t M, int l, const TC* Rinv, T* Q, int64_t ldq,
                              int transpose_out, double* part, cudaStream_t st) {
  int64_t rpc = apply_rows_per_cta(l);
  const int ls = l | 1;
  const size_t tiles = 2 * (size_t)rpc * ls * sizeof(T);
  const size_t rbytes = (size_t)l * ls * sizeof(TC);
  const int r_smem = tiles + rbytes <= 200 * 1024;
  const size_t smem = tiles + (r_smem ? rbytes : 0);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  cudaFuncSetAttribute(apply_rinv_kernel<T, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  unsigned blocks = (unsigned)cdiv(M, rpc);
  apply_rinv_kernel<T, TC><<<blocks, 256, smem, st>>>(Y, ldy, M, l, Rinv, Q, ldq, transpose_out, part, rpc,
                                                      r_smem);
  return launched();
}
template cudaError_t launch_apply_rinv<double, double>(const double*, int64_t, int64_t, int, const double*,
                                                       double*, int64_t, int, double*, cudaStream_t);
template cudaError_t launch_apply_rinv<float, float>(const float*, int64_t, int64_t, int, const float*, float*,
                                                     int64_t, int, double*, cudaStream_t);
template cudaError_t launch_apply_rinv<float, double>(const float*, int64_t, int64_t, int, const double*, float*,
                                                      int64_t, int, double*, cudaStream_t);

}  // namespace gsvdr
