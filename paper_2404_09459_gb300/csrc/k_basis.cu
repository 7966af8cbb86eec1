// Basis-extraction kernels on CUDA cores: Gaussian test matrices, the sketch
// and power products (the FP64 / FP32 paths), split-K reduction, the Gram
// matrix, the shifted Cholesky factorisation and the triangular apply of
// CholeskyQR2.  Tensor-core products live in k_tc.cu.
#include <cuda_bf16.h>

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

// The real 2n x 2l test matrix of a complex pair (K-major, as gaussian_kmajor_kernel writes
// it): rho(Omega), Omega (n x l) complex with Omega[j][c] = g(e) + i g(e + 1), e = 2 (j l + c),
// g the real Philox/Box-Muller stream of an n x 2l matrix; each complex entry a + ib becomes the
// 2 x 2 block [[a, -b], [b, a]] (rows 2j, 2j + 1 and columns 2c, 2c + 1 of rho(Omega)).
template <typename T>
__global__ void gaussian_kmajor_cplx_kernel(T* Xt, int64_t ldx, int64_t n2, int l2, int lrows, uint32_t k0,
                                            uint32_t k1, uint32_t pair, uint32_t side, uint32_t stream) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // column of Xt (row of rho(Omega))
  int j = blockIdx.y;                                          // row of Xt (column of rho(Omega))
  if (i >= ldx || j >= lrows) return;
  T v = T(0);
  if (i < n2 && j < l2) {
    const int64_t e = (i >> 1) * (int64_t)l2 + (j & ~1);  // complex entry (i / 2, j / 2): real part
    const int a = (int)(i & 1), b = j & 1;
    v = a == b ? gaussian_at<T>(e, k0, k1, pair, side, stream) : gaussian_at<T>(e + 1, k0, k1, pair, side, stream);
    if (a == 0 && b == 1) v = -v;
  }
  Xt[(int64_t)j * ldx + i] = v;
}

template <typename T>
cudaError_t launch_gaussian_kmajor_cplx(T* Xt, int64_t ldx, int64_t n2, int l2, int lrows, uint64_t seed,
                                        uint32_t pair, uint32_t side, uint32_t stream, cudaStream_t st) {
  if ((n2 & 1) || (l2 & 1)) return cudaErrorInvalidValue;
  dim3 grid((unsigned)cdiv(ldx, 256), (unsigned)lrows);
  gaussian_kmajor_cplx_kernel<T><<<grid, 256, 0, st>>>(Xt, ldx, n2, l2, lrows, (uint32_t)seed,
                                                       (uint32_t)(seed >> 32), pair, side, stream);
  return launched();
}
template cudaError_t launch_gaussian_kmajor_cplx<double>(double*, int64_t, int64_t, int, int, uint64_t,
                                                         uint32_t, uint32_t, uint32_t, cudaStream_t);
template cudaError_t launch_gaussian_kmajor_cplx<float>(float*, int64_t, int64_t, int, int, uint64_t,
                                                        uint32_t, uint32_t, uint32_t, cudaStream_t);

// R = rho(G): G (M x n complex, interleaved (re, im) pairs of T, row stride ldg complex entries)
// into the real 2M x 2n matrix R (row stride ldr), entry a + ib as the block [[a, -b], [b, a]].
// A thread per complex entry; rows 2i and 2i + 1 of R are written as pairs.
template <typename T>
__global__ void realify_kernel(const T* __restrict__ G, int64_t ldg, int64_t M, int64_t n, T* __restrict__ R,
                               int64_t ldr) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = blockIdx.y;
  if (j >= n || i >= M) return;
  const T a = G[2 * (i * ldg + j)], b = G[2 * (i * ldg + j) + 1];
  T* r0 = R + (2 * i) * ldr + 2 * j;
  T* r1 = r0 + ldr;
  r0[0] = a;
  r0[1] = -b;
  r1[0] = b;
  r1[1] = a;
}

template <typename T>
cudaError_t launch_realify(const T* G, int64_t ldg, int64_t M, int64_t n, T* R, int64_t ldr, cudaStream_t st) {
  if (M < 1 || n < 1) return cudaSuccess;
  for (int64_t r0 = 0; r0 < M; r0 += 65535) {
    const int64_t rows = std::min<int64_t>(65535, M - r0);
    dim3 grid((unsigned)cdiv(n, 256), (unsigned)rows);
    realify_kernel<T><<<grid, 256, 0, st>>>(G + 2 * r0 * ldg, ldg, rows, n, R + 2 * r0 * ldr, ldr);
    cudaError_t e = launched();
    if (e) return e;
  }
  return cudaSuccess;
}
template cudaError_t launch_realify<double>(const double*, int64_t, int64_t, int64_t, double*, int64_t, cudaStream_t);
template cudaError_t launch_realify<float>(const float*, int64_t, int64_t, int64_t, float*, int64_t, cudaStream_t);

// D = G widened to FP64 (M x n, row strides ldg and ldd): a thread per entry.
__global__ void widen_kernel(const float* __restrict__ G, int64_t ldg, int64_t M, int64_t n, double* __restrict__ D,
                             int64_t ldd) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = blockIdx.y;
  if (j >= n || i >= M) return;
  D[i * ldd + j] = (double)G[i * ldg + j];
}

cudaError_t launch_widen(const float* G, int64_t ldg, int64_t M, int64_t n, double* D, int64_t ldd, cudaStream_t st) {
  if (M < 1 || n < 1) return cudaSuccess;
  for (int64_t r0 = 0; r0 < M; r0 += 65535) {
    const int64_t rows = std::min<int64_t>(65535, M - r0);
    dim3 grid((unsigned)cdiv(n, 256), (unsigned)rows);
    widen_kernel<<<grid, 256, 0, st>>>(G + r0 * ldg, ldg, rows, n, D + r0 * ldd, ldd);
    cudaError_t e = launched();
    if (e) return e;
  }
  return cudaSuccess;
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

// Omega^T K-major in BF16, the sketch operand of the BF16 mode: each entry is the
// FP64 Gaussian rounded to the nearest FP32, then to the nearest BF16 (ties to even).
__global__ void gaussian_kmajor_bf16_kernel(__nv_bfloat16* Xt, int64_t ldx, int64_t n, int l, int lrows,
                                            uint32_t k0, uint32_t k1, uint32_t pair, uint32_t side,
                                            uint32_t stream) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y;
  if (i >= ldx || j >= lrows) return;
  float v = 0.f;
  if (i < n && j < l) v = (float)gaussian_at<double>(i * (int64_t)l + j, k0, k1, pair, side, stream);
  Xt[(int64_t)j * ldx + i] = __float2bfloat16_rn(v);
}

cudaError_t launch_gaussian_kmajor_bf16(void* Xt, int64_t ldx, int64_t n, int l, int lrows, uint64_t seed,
                                        uint32_t pair, uint32_t side, uint32_t stream, cudaStream_t st) {
  dim3 grid((unsigned)cdiv(ldx, 256), (unsigned)lrows);
  gaussian_kmajor_bf16_kernel<<<grid, 256, 0, st>>>(static_cast<__nv_bfloat16*>(Xt), ldx, n, l, lrows,
                                                    (uint32_t)seed, (uint32_t)(seed >> 32), pair, side, stream);
  return launched();
}

// Qt[j][i] = Y[i][j] (i < M, j < l): a row-major M x l tile into the K-major layout
// of the tensor-core operands, 32 x 32 tiles through shared memory.
template <typename T>
__global__ void transpose_kernel(const T* __restrict__ Y, int64_t ldy, int64_t M, int l, T* __restrict__ Qt,
                                 int64_t ldq) {
  __shared__ T t[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int j0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t i = i0 + r;
    const int j = j0 + threadIdx.x;
    t[r][threadIdx.x] = (i < M && j < l) ? Y[i * ldy + j] : T(0);
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int j = j0 + r;
    const int64_t i = i0 + threadIdx.x;
    if (j < l && i < M) Qt[(int64_t)j * ldq + i] = t[threadIdx.x][r];
  }
}

template <typename T>
cudaError_t launch_transpose(const T* Y, int64_t ldy, int64_t M, int l, T* Qt, int64_t ldq, cudaStream_t st) {
  if (M <= 0 || l <= 0) return cudaSuccess;
  transpose_kernel<T><<<dim3((unsigned)cdiv(M, 32), (unsigned)cdiv(l, 32)), dim3(32, 8), 0, st>>>(Y, ldy, M, l, Qt,
                                                                                               ldq);
  return launched();
}
template cudaError_t launch_transpose<float>(const float*, int64_t, int64_t, int, float*, int64_t, cudaStream_t);
template cudaError_t launch_transpose<double>(const double*, int64_t, int64_t, int, double*, int64_t, cudaStream_t);

// hi = bf16(x) and lo = bf16(x - hi) (x - hi is exact in FP32), both to nearest even, so
// that hi + lo carries x to about 2^-16 of its size.  Eight columns per thread.
__global__ void split_bf16_kernel(const float* __restrict__ src, int64_t lds, int64_t rows, int64_t cols,
                                  __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int64_t ldd,
                                  int vec) {
  const int64_t groups = (cols + 7) / 8;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * groups) return;
  const int64_t r = t / groups, c0 = (t % groups) * 8;
  const float* x = src + r * lds + c0;
  if (vec && c0 + 8 <= cols) {
    const float4 a = *reinterpret_cast<const float4*>(x), b = *reinterpret_cast<const float4*>(x + 4);
    const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    __align__(16) __nv_bfloat16 h[8], w[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      h[e] = __float2bfloat16_rn(v[e]);
      w[e] = __float2bfloat16_rn(v[e] - __bfloat162float(h[e]));
    }
    *reinterpret_cast<uint4*>(hi + r * ldd + c0) = *reinterpret_cast<const uint4*>(h);
    if (lo) *reinterpret_cast<uint4*>(lo + r * ldd + c0) = *reinterpret_cast<const uint4*>(w);
    return;
  }
  for (int e = 0; e < 8 && c0 + e < cols; ++e) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x[e]);
    hi[r * ldd + c0 + e] = h;
    if (lo) lo[r * ldd + c0 + e] = __float2bfloat16_rn(x[e] - __bfloat162float(h));
  }
}

cudaError_t launch_split_bf16(const float* src, int64_t lds, int64_t rows, int64_t cols, void* hi, void* lo,
                              int64_t ldd, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  const int vec = ((uintptr_t)src % 16 == 0) && (lds % 4 == 0) && ((uintptr_t)hi % 16 == 0) &&
                  ((uintptr_t)lo % 16 == 0) && (ldd % 8 == 0);
  const int64_t threads = rows * ((cols + 7) / 8);
  split_bf16_kernel<<<(unsigned)cdiv(threads, 256), 256, 0, st>>>(src, lds, rows, cols,
                                                                  static_cast<__nv_bfloat16*>(hi),
                                                                  static_cast<__nv_bfloat16*>(lo), ldd, vec);
  return launched();
}

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
__device__ __forceinline__ void reduce_splits_body(const TP* __restrict__ part, int splits, int64_t n, int l,
                                                   int64_t lp, T* __restrict__ Z, int64_t ldz, int transpose_out,
                                                   double* sq_part, int bx) {
  int64_t e = (int64_t)bx * blockDim.x + threadIdx.x;
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
    if (threadIdx.x == 0) sq_part[bx] = s;
  }
}

template <typename TP, typename T>
__global__ void reduce_splits_kernel(const TP* __restrict__ part, int splits, int64_t n, int l,
                                     int64_t lp, T* __restrict__ Z, int64_t ldz, int transpose_out,
                                     double* sq_part) {
  reduce_splits_body<TP, T>(part, splits, n, l, lp, Z, ldz, transpose_out, sq_part, (int)blockIdx.x);
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
__device__ __forceinline__ void gram_partial_body(const T* __restrict__ Y, int64_t ldy, int64_t M, int l,
                                                  double* __restrict__ part, int64_t rows_per_chunk, int c, int ti,
                                                  int tj) {
  __shared__ T As[GR_BK][GR_T + 1];
  __shared__ T Bs[GR_BK][GR_T + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t rbeg = (int64_t)c * rows_per_chunk, rend = min(M, rbeg + rows_per_chunk);
  const int i0 = ti * GR_T, j0 = tj * GR_T;
  const bool active = i0 + ty * 4 < l && j0 + tx * 4 < l && (ti != tj || tx >= ty);
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
    // only threads with a stored output (inside l, on or above the diagonal) do the FMAs:
    // for narrow bases most of the 64 x 64 tile is padding
    if (active) {
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

template <typename T>
__global__ __launch_bounds__(256) void gram_partial_kernel(const T* __restrict__ Y, int64_t ldy,
                                                           int64_t M, int l, double* __restrict__ part,
                                                           int64_t rows_per_chunk) {
  if (blockIdx.y > blockIdx.z) return;
  gram_partial_body<T>(Y, ldy, M, l, part, rows_per_chunk, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z);
}

int gram_chunks(int64_t M, int l, int64_t* rows_per_chunk) {
  int64_t t = cdiv(l, GR_T);
  int64_t upper = t * (t + 1) / 2;
  // two CTAs per SM; eight for bases wider than 128 columns, whose CTAs each stream thousands
  // of rows with unhidden load latency at two per SM (0.63 ms, 26% of the FP32 rate, for
  // M = 120000, l = 220)
  int64_t chunks = std::max<int64_t>(1, ((l > 128 ? 8 : 2) * 152) / upper);
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
__device__ __forceinline__ void gram_reduce_body(const double* __restrict__ part, int chunks, int l,
                                                 double* __restrict__ W, int bx) {
  const int64_t wid = ((int64_t)bx * blockDim.x + threadIdx.x) >> 5;
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

__global__ void gram_reduce_kernel(const double* __restrict__ part, int chunks, int l,
                                   double* __restrict__ W) {
  gram_reduce_body(part, chunks, l, W, (int)blockIdx.x);
}

cudaError_t launch_gram_reduce(const double* part, int chunks, int l, double* W, cudaStream_t st) {
  const int64_t threads = (int64_t)l * l * 32;
  gram_reduce_kernel<<<(unsigned)cdiv(threads, 256), 256, 0, st>>>(part, chunks, l, W);
  return launched();
}

// ============================================================================
// Shifted Cholesky with the inverse factor in the same sweep, one CTA of 32
// warps.  Gaussian elimination on the augmented pair [W | I] by symmetric
// pivots turns W into U = D L^T and I into L^{-1} (W = L D L^T, L unit lower),
// so R = D^{1/2} L^T and R^{-1} = L^{-T} D^{-1/2}: no separate triangular
// inverse.  Both halves share one l x lda array M: the upper triangle
// (j >= i) holds the reduced W, the strict lower triangle row i holds the
// off-diagonal part of row i of L^{-1}.  Pivot k updates, for every row
// i > k, the columns c < k (L^{-1} part), c = k (the new multiplier) and
// c >= i (trailing W): one barrier per pivot, rows spread over warps,
// columns over lanes.
// ============================================================================
constexpr int CHOL_THREADS = 1024;

template <typename TC>
__device__ __forceinline__ void chol_shift_body(const double* __restrict__ W, int l, double shift_coef,
                                                double tau_rel, TC* __restrict__ Rinv, DevStatus* st_dev, int stage,
                                                TC* gscr, int use_smem, int ldt = 0) {
  extern __shared__ unsigned char smem_raw[];
  const int lda = l | 1;
  TC* M = use_smem ? reinterpret_cast<TC*>(smem_raw) : gscr;
  __shared__ double s_tr;
  __shared__ int s_bad, s_kept;
  __shared__ TC s_odiag[256], s_scale[256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = CHOL_THREADS / 32;
  if (tid == 0) {
    s_bad = 0;
    s_kept = 0;
  }
  __syncthreads();
  for (int i = warp; i < l; i += NW)
    for (int j = lane; j < l; j += 32) {
      const double v = W[(int64_t)i * l + j];
      if (!isfinite(v)) s_bad = 2;
      M[(int64_t)i * lda + j] = j >= i ? (TC)v : TC(0);
    }
  if (warp == 0) {  // trace in FP64
    double t = 0.0;
    for (int i = lane; i < l; i += 32) t += W[(int64_t)i * l + i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) s_tr = t;
  }
  __syncthreads();
  const double sh = shift_coef * s_tr;
  for (int i = tid; i < l; i += CHOL_THREADS) {
    const TC v = (TC)((double)W[(int64_t)i * l + i] + sh);
    M[(int64_t)i * lda + i] = v;
    s_odiag[i] = v;
  }
  __syncthreads();
  // A pivot at or below the Gram's resolution relative to its own (shifted)
  // diagonal is numerically dependent on the earlier columns.  Dropping it
  // would take its direction out of the span (weak directions of the sketch go
  // with it), so it is clamped to that floor instead; the next CholeskyQR pass
  // re-orthonormalises the column.  The final M[k][k] is the pivot seen at step
  // k, so the same rule is applied again afterwards.
  // effective pivot: d when above tau times the column's own (shifted) diagonal, else that
  // floor (the column keeps its direction in the span; a later pass re-orthonormalises it);
  // 0 (column dropped) only when the floor itself is zero (a zero column)
  auto pivot = [&](int k, TC d) -> TC {
    const TC fl = (TC)tau_rel * s_odiag[k];
    return d > fl ? d : (fl > TC(0) ? fl : TC(0));
  };
  int bad_k = -1;
  if (s_bad == 0) {
    for (int k = 0; k < l; ++k) {
      const TC* rowk = M + (int64_t)k * lda;
      const TC d = rowk[k];
      if (!isfinite(d)) {
        bad_k = k;
        break;
      }
      const TC pv = pivot(k, d);
      if (pv == TC(0)) continue;
      const TC dinv = TC(1) / pv;
      for (int i = k + 1 + warp; i < l; i += NW) {
        const TC f = rowk[i] * dinv;
        TC* ri = M + (int64_t)i * lda;
        for (int c = lane; c < k; c += 32) ri[c] -= f * rowk[c];
        if (lane == 0) ri[k] = -f;
        for (int c = i + lane; c < l; c += 32) ri[c] -= f * rowk[c];
      }
      __syncthreads();
    }
  }
  __syncthreads();
  if (warp == 0 && bad_k < 0 && s_bad == 0) {
    int c = 0;
    for (int i = lane; i < l; i += 32) {
      const TC d = M[(int64_t)i * lda + i];
      const TC pv = pivot(i, d);
      const bool dr = pv == TC(0);
      s_scale[i] = dr ? TC(0) : TC(1) / sqrt(pv);
      c += dr ? 0 : 1;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if (lane == 0) s_kept = c;
  }
  __syncthreads();
  if (bad_k >= 0 || s_bad || s_kept == 0) {
    if (tid == 0) set_status(st_dev, (s_bad == 2 || bad_k >= 0) ? -4 : -5, stage, bad_k);
    return;
  }
  // R^{-1}[c][j] = L^{-1}[j][c] / sqrt(d_j) for c <= j (L^{-1}[j][j] = 1)
  for (int c = warp; c < l; c += NW)
    for (int j = lane; j < l; j += 32) {
      TC v = TC(0);
      if (j == c) v = s_scale[j];
      else if (j > c) v = M[(int64_t)j * lda + c] * s_scale[j];
      if (ldt)
        Rinv[(int64_t)j * ldt + c] = v;  // transposed (K-major operand of Q = Y R^{-1})
      else
        Rinv[(int64_t)c * l + j] = v;
    }
}

template <typename TC>
__global__ __launch_bounds__(CHOL_THREADS) void chol_shift_kernel(const double* __restrict__ W, int l,
                                                                  double shift_coef, double tau_rel,
                                                                  TC* __restrict__ Rinv, DevStatus* st_dev,
                                                                  int stage, TC* gscr, int use_smem, int ldt) {
  chol_shift_body<TC>(W, l, shift_coef, tau_rel, Rinv, st_dev, stage, gscr, use_smem, ldt);
}

// The same elimination for l <= 64 with the augmented rows in registers:
// 8 warps, thread (w, t) holds rows i = w + 8 r (r < 8) and the column slots
// t, t + 32 of W and of L^{-1} (32 values).  Step k publishes row k through a
// double-buffered shared row; every row i > k subtracts (W_ik / W_kk) times it,
// on all columns: entries left of the pivot become (rounding-level) zeros or
// lower-triangle values that are never read.  One barrier per step.
constexpr int CHOL64_THREADS = 256;

template <typename TC>
__device__ __forceinline__ void chol64_body(const double* __restrict__ W, int l, double shift_coef, double tau_rel,
                                            TC* __restrict__ Rinv, DevStatus* st_dev, int stage, int ldt = 0) {
  __shared__ TC s_row[2][128];
  __shared__ TC s_odiag[64], s_scale[64];
  __shared__ double s_tr;
  __shared__ int s_bad, s_kept;
  const int tid = threadIdx.x, w = tid >> 5, t = tid & 31;
  if (tid == 0) {
    s_bad = 0;
    s_kept = 0;
  }
  if (w == 0) {
    double tr = 0.0;
    for (int i = t; i < l; i += 32) tr += W[(int64_t)i * l + i];
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    if (t == 0) s_tr = tr;
  }
  __syncthreads();
  const double sh = shift_coef * s_tr;
  TC a[8][4];
  bool bad = false;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = w + 8 * r;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int j = t + 32 * c;
      double v = (i < l && j < l) ? W[(int64_t)i * l + j] : 0.0;
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
  int bad_k = -1;
  if (s_bad == 0) {
    for (int k = 0; k < l; ++k) {
      TC* row = s_row[k & 1];
      if (w == (k & 7)) {
        switch (k >> 3) {
#define CHOL64_PUB(R) \
  case R:              \
    for (int c = 0; c < 4; ++c) row[t + 32 * c] = a[R][c]; \
    break;
          CHOL64_PUB(0) CHOL64_PUB(1) CHOL64_PUB(2) CHOL64_PUB(3)
          CHOL64_PUB(4) CHOL64_PUB(5) CHOL64_PUB(6) CHOL64_PUB(7)
#undef CHOL64_PUB
        }
      }
      __syncthreads();
      const TC d = row[k];
      if (!isfinite(d)) {
        bad_k = k;
        break;
      }
      const TC pv = pivot(k, d);
      if (pv == TC(0)) continue;
      const TC dinv = TC(1) / pv;
      TC rc[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) rc[c] = row[t + 32 * c];
      // live column slots (uniform): W columns in (k, l), L^{-1} columns in [0, min(k, l - 1)];
      // worth testing only at the FP64 rate
      bool live[4];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        live[c] = sizeof(TC) == 4 || (32 * c < l && 32 * c + 31 > k);
        live[2 + c] = sizeof(TC) == 4 || (32 * c < l && 32 * c <= k);
      }
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
  }
  __syncthreads();
  // the pivots are the final diagonal entries (row k is not touched after step k)
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
    for (int i = t; i < l; i += 32) {
      const TC d = s_row[0][i];
      const TC pv = pivot(i, d);
      const bool dr = pv == TC(0);
      s_scale[i] = dr ? TC(0) : TC(1) / sqrt(pv);
      kept += dr ? 0 : 1;
    }
    for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
    if (t == 0) s_kept = kept;
  }
  __syncthreads();
  if (bad_k >= 0 || s_bad || s_kept == 0) {
    if (tid == 0) set_status(st_dev, (s_bad == 2 || bad_k >= 0) ? -4 : -5, stage, bad_k);
    return;
  }
  // R^{-1}[c][j] = L^{-1}[j][c] / sqrt(d_j) for c <= j, zero below the diagonal
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int j = w + 8 * r;
    if (j >= l) continue;
    const TC sj = s_scale[j];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int cc = t + 32 * c;
      if (cc < l) {
        const TC v = cc <= j ? a[r][2 + c] * sj : TC(0);
        if (ldt)
          Rinv[(int64_t)j * ldt + cc] = v;  // transposed (K-major operand of Q = Y R^{-1})
        else
          Rinv[(int64_t)cc * l + j] = v;
      }
    }
  }
}

template <typename TC>
__global__ __launch_bounds__(CHOL64_THREADS, 1) void chol64_kernel(const double* __restrict__ W, int l,
                                                                double shift_coef, double tau_rel,
                                                                TC* __restrict__ Rinv, DevStatus* st_dev,
                                                                int stage) {
  chol64_body<TC>(W, l, shift_coef, tau_rel, Rinv, st_dev, stage);
}

int64_t chol_scratch_elems(int l) { return (int64_t)l * (l | 1); }

template <typename TC>
cudaError_t launch_chol_shift(const double* W, int l, double shift_coef, double tau_rel, TC* Rinv,
                              TC* scratch, DevStatus* st_dev, int stage, cudaStream_t st, int ldt) {
  if (l < 1 || l > 256) return cudaErrorInvalidValue;
  if (ldt && l <= 64) return cudaErrorInvalidValue;  // the transposed factor is written by the wide kernel only
  if (l <= 64) {
    chol64_kernel<TC><<<1, CHOL64_THREADS, 0, st>>>(W, l, shift_coef, tau_rel, Rinv, st_dev, stage);
    return launched();
  }
  size_t smem = (size_t)chol_scratch_elems(l) * sizeof(TC);
  int use_smem = smem <= 216 * 1024;
  cudaFuncSetAttribute(chol_shift_kernel<TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 216 * 1024);
  chol_shift_kernel<TC><<<1, CHOL_THREADS, use_smem ? smem : 0, st>>>(W, l, shift_coef, tau_rel, Rinv, st_dev,
                                                                      stage, scratch, use_smem, ldt);
  return launched();
}
__global__ __launch_bounds__(CHOL_THREADS) void chol_shift_pair_kernel(CholPairArgs a, int l, DevStatus* st_dev,
                                                                       int use_smem, int ldt) {
  const int s = blockIdx.x;
  chol_shift_body<float>(a.W[s], l, a.shift_coef[s], a.tau_rel[s], a.Rinv[s], st_dev, a.stage[s], a.scratch[s],
                         use_smem, ldt);
}

cudaError_t launch_chol_shift_pair(const CholPairArgs& a, int l, DevStatus* st_dev, cudaStream_t st, int ldt) {
  if (l <= 64 || l > 256) return cudaErrorInvalidValue;
  size_t smem = (size_t)chol_scratch_elems(l) * sizeof(float);
  int use_smem = smem <= 216 * 1024;
  cudaFuncSetAttribute(chol_shift_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 216 * 1024);
  chol_shift_pair_kernel<<<2, CHOL_THREADS, use_smem ? smem : 0, st>>>(a, l, st_dev, use_smem, ldt);
  return launched();
}

template cudaError_t launch_chol_shift<double>(const double*, int, double, double, double*, double*,
                                               DevStatus*, int, cudaStream_t, int);
template cudaError_t launch_chol_shift<float>(const double*, int, double, double, float*, float*,
                                              DevStatus*, int, cudaStream_t, int);

// ============================================================================
// Q = Y R^{-1} over a tile of rows per CTA, register-blocked: 16 x 16 threads,
// thread (ty, tx) computes rows ty + 16 rr (rr < RT) x columns tx CT + cc
// (cc < CT) with lpad = 16 CT >= l.  Optional Gram partial of the produced rows
// (4 x 4 register blocks) and optional transposed store Qt[j * ldq + row].
// ============================================================================
int apply_ct(int l) { return l <= 64 ? 4 : (l <= 128 ? 8 : 16); }
// FP64 tiles are smaller: at the FP64 rate the work of a 128-row tile would leave most SMs idle
int64_t apply_rows_per_cta(int l, int elem_bytes) { return l <= 64 ? (elem_bytes == 8 ? 32 : 128) : 32; }
int apply_ctas(int64_t M, int l, int elem_bytes) { return (int)cdiv(M, apply_rows_per_cta(l, elem_bytes)); }
bool apply_fuses_gram(int l) { return l <= 64; }

// RS: R^{-1} staged in shared memory (else read through L1 from global).
template <typename T, typename TC, int CT, int RT, bool RS>
__device__ __forceinline__ void apply_rinv_body(const T* __restrict__ Y, int64_t ldy, int64_t M, int l,
                                                const TC* __restrict__ Rinv, T* Q, int64_t ldq, int transpose_out,
                                                double* part, int bx) {
  constexpr int LP = 16 * CT;      // padded column count
  constexpr int ROWS = 16 * RT;    // rows per CTA
  constexpr int LS = LP + 1;       // odd stride of the row tiles
  extern __shared__ unsigned char smem_raw[];
  T* Rs = reinterpret_cast<T*>(smem_raw);  // LP x LP (zero padded), when RS
  T* Ys = Rs + (RS ? LP * LP : 0);         // ROWS x LS
  T* Qs = Ys + ROWS * LS;                  // ROWS x LS
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t r0 = (int64_t)bx * ROWS;
  const int rows = (int)(ROWS < M - r0 ? ROWS : M - r0);
  if (RS)
    for (int e = tid; e < LP * LP; e += 256) {
      const int i = e / LP, j = e % LP;
      Rs[e] = (i < l && j < l) ? (T)Rinv[(int64_t)i * l + j] : T(0);
    }
  for (int e = tid; e < ROWS * LP; e += 256) {
    const int r = e / LP, j = e % LP;
    Ys[r * LS + j] = (r < rows && j < l) ? Y[(r0 + r) * ldy + j] : T(0);
  }
  __syncthreads();
  T acc[RT][CT];
#pragma unroll
  for (int a = 0; a < RT; ++a)
#pragma unroll
    for (int b = 0; b < CT; ++b) acc[a][b] = T(0);
  for (int i = 0; i < l; ++i) {
    T av[RT], bv[CT];
#pragma unroll
    for (int rr = 0; rr < RT; ++rr) av[rr] = Ys[(ty + 16 * rr) * LS + i];
#pragma unroll
    for (int cc = 0; cc < CT; ++cc) {
      const int j = tx * CT + cc;
      bv[cc] = RS ? Rs[i * LP + j] : (j < l ? (T)Rinv[(int64_t)i * l + j] : T(0));
    }
#pragma unroll
    for (int rr = 0; rr < RT; ++rr)
#pragma unroll
      for (int cc = 0; cc < CT; ++cc) acc[rr][cc] = fma(av[rr], bv[cc], acc[rr][cc]);
  }
#pragma unroll
  for (int rr = 0; rr < RT; ++rr)
#pragma unroll
    for (int cc = 0; cc < CT; ++cc) Qs[(ty + 16 * rr) * LS + tx * CT + cc] = acc[rr][cc];
  __syncthreads();
  if (transpose_out) {
    for (int e = tid; e < rows * l; e += 256) {
      const int j = e / rows, r = e % rows;
      Q[(int64_t)j * ldq + r0 + r] = Qs[r * LS + j];
    }
  } else {
    for (int e = tid; e < rows * l; e += 256) {
      const int r = e / l, j = e % l;
      Q[(r0 + r) * ldq + j] = Qs[r * LS + j];
    }
  }
  if (part) {
    // Gram of the tile: thread (ty, tx) owns the CT x CT block (ty CT.., tx CT..), upper blocks only
    double* P = part + (int64_t)bx * l * l;
    if (tx >= ty) {
      for (int bi = 0; bi < CT; bi += 4)
        for (int bj = 0; bj < CT; bj += 4) {
          T g[4][4];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) g[a][b] = T(0);
          const int i0 = ty * CT + bi, j0 = tx * CT + bj;
          for (int r = 0; r < rows; ++r) {
            const T* qr = Qs + r * LS;
            T x[4], y[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
              x[a] = qr[i0 + a];
              y[a] = qr[j0 + a];
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int b = 0; b < 4; ++b) g[a][b] = fma(x[a], y[b], g[a][b]);
          }
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              const int i = i0 + a, j = j0 + b;
              if (i < l && j < l && j >= i) P[(int64_t)i * l + j] = (double)g[a][b];
            }
        }
    }
  }
}

template <typename T, typename TC, int CT, int RT, bool RS>
__global__ __launch_bounds__(256) void apply_rinv_kernel(const T* __restrict__ Y, int64_t ldy, int64_t M, int l,
                                                         const TC* __restrict__ Rinv, T* Q, int64_t ldq,
                                                         int transpose_out, double* part) {
  apply_rinv_body<T, TC, CT, RT, RS>(Y, ldy, M, l, Rinv, Q, ldq, transpose_out, part, (int)blockIdx.x);
}

template <typename T, typename TC>
cudaError_t launch_apply_rinv(const T* Y, int64_t ldy, int64_t M, int l, const TC* Rinv, T* Q, int64_t ldq,
                              int transpose_out, double* part, cudaStream_t st) {
  if (l < 1 || l > 256) return cudaErrorInvalidValue;
  const int ct = apply_ct(l);
  const int lp = 16 * ct, rows = (int)apply_rows_per_cta(l, (int)sizeof(T));
  const size_t tiles = 2 * (size_t)rows * (lp + 1) * sizeof(T);
  const bool rs = ct <= 8;  // R^{-1} (lp x lp) staged for l <= 128: <= 128 KB in FP64
  const size_t smem = tiles + (rs ? (size_t)lp * lp * sizeof(T) : 0);
  if (smem > 220 * 1024) return cudaErrorInvalidValue;
  const unsigned blocks = (unsigned)cdiv(M, rows);
#define GSVDR_APPLY(CTV, RTV, RSV)                                                                              \
  do {                                                                                                          \
    cudaFuncSetAttribute(apply_rinv_kernel<T, TC, CTV, RTV, RSV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                         220 * 1024); /* a fixed cap: concurrent launches must not lower it */                  \
    apply_rinv_kernel<T, TC, CTV, RTV, RSV><<<blocks, 256, smem, st>>>(Y, ldy, M, l, Rinv, Q, ldq,            \
                                                                      transpose_out, part);                    \
  } while (0)
  if (ct == 4 && sizeof(T) == 8)
    GSVDR_APPLY(4, 2, true);
  else if (ct == 4)
    GSVDR_APPLY(4, 8, true);
  else if (ct == 8)
    GSVDR_APPLY(8, 2, true);
  else
    GSVDR_APPLY(16, 2, false);
#undef GSVDR_APPLY
  return launched();
}
template cudaError_t launch_apply_rinv<double, double>(const double*, int64_t, int64_t, int, const double*,
                                                       double*, int64_t, int, double*, cudaStream_t);
template cudaError_t launch_apply_rinv<float, float>(const float*, int64_t, int64_t, int, const float*, float*,
                                                     int64_t, int, double*, cudaStream_t);
template cudaError_t launch_apply_rinv<float, double>(const float*, int64_t, int64_t, int, const double*, float*,
                                                      int64_t, int, double*, cudaStream_t);


// ============================================================================
// Batched forms: one launch for many problems (the sides of the pairs of a
// grouped solve).  Argument tables live in device memory, one entry per
// problem (blockIdx.z, or blockIdx.x for one CTA per problem); grids are sized
// for the largest problem and the CTAs past a smaller problem's extent return
// at once (uniformly per CTA, before any barrier).
// ============================================================================
__global__ void gaussian_kmajor_b_kernel(const GaussB* __restrict__ tab) {
  const GaussB a = tab[blockIdx.z];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= a.ldx || j >= a.lrows) return;
  float v = 0.f;
  if (i < a.n && j < a.l)
    v = gaussian_at<float>(i * (int64_t)a.l + j, (uint32_t)a.seed, (uint32_t)(a.seed >> 32), a.pair, a.side,
                           a.stream);
  a.Xt[(int64_t)j * a.ldx + i] = v;
  if (a.lo) a.lo[(int64_t)j * a.ldx + i] = tf32_low_half(v);
}

__global__ void low_half_b_kernel(const LoHalfB* __restrict__ tab) {
  const LoHalfB& a = tab[blockIdx.y];
  if (a.stop && *a.stop) return;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.rows * a.cols) return;
  const int64_t r = e / a.cols, c = e - r * a.cols;
  a.dst[r * a.ld + c] = tf32_low_half(a.src[r * a.ld + c]);
}

cudaError_t launch_low_half_b(const LoHalfB* tab, int nprob, int64_t max_elems, cudaStream_t st) {
  if (nprob <= 0 || max_elems <= 0) return cudaSuccess;
  low_half_b_kernel<<<dim3((unsigned)cdiv(max_elems, 256), (unsigned)nprob), 256, 0, st>>>(tab);
  return launched();
}

// dst (rows x n, row stride ldd) = src (rows x n, contiguous): the re-pitch of a host matrix landed
// in one contiguous copy (a thread per element, reads and writes coalesced along the rows).
__global__ void repitch_kernel(const float* __restrict__ src, int64_t rows, int64_t n, float* __restrict__ dst,
                               int64_t ldd) {
  const int64_t total = rows * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / n, c = e - r * n;
    dst[r * ldd + c] = src[e];
  }
}

cudaError_t launch_repitch(const float* src, int64_t rows, int64_t n, float* dst, int64_t ldd, cudaStream_t st) {
  if (rows < 1 || n < 1) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>(cdiv(rows * n, 256), 152 * 16);
  repitch_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, rows, n, dst, ldd);
  return launched();
}

cudaError_t launch_gaussian_kmajor_b(const GaussB* tab, int nprob, int64_t max_ldx, int max_lrows, cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  gaussian_kmajor_b_kernel<<<dim3((unsigned)cdiv(max_ldx, 256), (unsigned)max_lrows, (unsigned)nprob), 256, 0, st>>>(tab);
  return launched();
}

__global__ void reduce_splits_b_kernel(const ReduceB* __restrict__ tab) {
  const ReduceB& a = tab[blockIdx.z];
  if ((int64_t)blockIdx.x * blockDim.x >= a.n * a.l) return;
  reduce_splits_body<float, float>(a.part, a.splits, a.n, a.l, a.lp, a.Z, a.ldz, a.transpose_out, a.sq_part,
                                   (int)blockIdx.x);
}

cudaError_t launch_reduce_splits_b(const ReduceB* tab, int nprob, int64_t max_nl, cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  reduce_splits_b_kernel<<<dim3((unsigned)cdiv(max_nl, 256), 1, (unsigned)nprob), 256, 0, st>>>(tab);
  return launched();
}



__global__ __launch_bounds__(CHOL64_THREADS, 1) void chol64_b_kernel(const CholB* __restrict__ tab) {
  const CholB& a = tab[blockIdx.x];
  if (a.stop && *a.stop) return;
  chol64_body<float>(a.W, a.l, a.shift_coef, a.tau_rel, a.Rinv, a.st, a.stage, a.ldt);
}

__global__ __launch_bounds__(CHOL_THREADS) void chol_shift_b_kernel(const CholB* __restrict__ tab) {
  const CholB& a = tab[blockIdx.x];
  if (a.stop && *a.stop) return;
  chol_shift_body<float>(a.W, a.l, a.shift_coef, a.tau_rel, a.Rinv, a.st, a.stage, nullptr, 1, a.ldt);
}

cudaError_t launch_chol_b(const CholB* tab, int nprob, int max_l, cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  if (max_l < 1 || max_l > 128) return cudaErrorInvalidValue;
  if (max_l <= 64) {
    chol64_b_kernel<<<nprob, CHOL64_THREADS, 0, st>>>(tab);
    return launched();
  }
  const size_t smem = (size_t)chol_scratch_elems(max_l) * sizeof(float);
  cudaFuncSetAttribute(chol_shift_b_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 216 * 1024);
  chol_shift_b_kernel<<<nprob, CHOL_THREADS, smem, st>>>(tab);
  return launched();
}



// ---------------------------------------------------------------------------
// Batched Gram partials for bases of up to 128 columns (the grouped solve's
// CholeskyQR): one CTA per (chunk of rows, problem) holds the whole upper
// triangle of the chunk's Y^T Y in 8 x 8 register blocks, one block per thread;
// for narrow bases the threads form up to 8 groups that take interleaved rows
// of each 32-row slab, and the groups' sums are added in group order at the end
// (deterministic).  The slabs are double-buffered: the next one is loaded into
// registers while the current one is multiplied.
// ---------------------------------------------------------------------------
constexpr int GB_SLAB = 32, GB_LP = 128, GB_LS = GB_LP + 4;

__global__ __launch_bounds__(256, 2) void gram_blocks_b_kernel(const GramB* __restrict__ tab) {
  const GramB& g = tab[blockIdx.z];
  const int c = blockIdx.x;
  if (c >= g.chunks || (g.stop && *g.stop)) return;
  __shared__ __align__(16) float Ys[2][GB_SLAB * GB_LS];
  const int tid = threadIdx.x, l = g.l;
  const int LB = (l + 7) >> 3, nblk = LB * (LB + 1) / 2;
  const int G = max(1, min(8, 256 / nblk));
  const int grp = tid / nblk, bp = tid - grp * nblk;
  const bool active = grp < G;
  // block pair bp -> (bi, bj), bi <= bj, row by row of the upper triangle
  int bi = 0, rem = bp;
  while (active && rem >= LB - bi) {
    rem -= LB - bi;
    ++bi;
  }
  const int bj = bi + rem;
  const int64_t rbeg = (int64_t)c * g.rpc, rend = min(g.M, rbeg + g.rpc);
  const int nslab = (int)((rend - rbeg + GB_SLAB - 1) / GB_SLAB);
  const int lq = (l + 3) >> 2;  // float4 per row
  // slab loader: element e of the slab (row e / 32, float4 e % 32), four per thread, as
  // asynchronous 16-byte copies that zero-fill past the rows of the chunk and column l
  auto issue = [&](int sidx, int buf) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q, r = e >> 5, c4 = e & 31;
      const int64_t row = rbeg + (int64_t)sidx * GB_SLAB + r;
      const float* src = g.Y;
      int bytes = 0;
      if (row < rend && c4 < lq) {
        src = g.Y + row * g.ldy + 4 * c4;
        bytes = 4 * min(4, l - 4 * c4);
      }
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&Ys[buf][r * GB_LS + 4 * c4]);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
  if (nslab > 0) issue(0, 0);
  for (int si = 0; si < nslab; ++si) {
    const int buf = si & 1;
    if (si + 1 < nslab) {
      issue(si + 1, buf ^ 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    if (active) {
      const float* base = Ys[buf];
      for (int r = grp; r < GB_SLAB; r += G) {
        const float* row = base + r * GB_LS;
        const float4 a0 = *reinterpret_cast<const float4*>(row + 8 * bi);
        const float4 a1 = *reinterpret_cast<const float4*>(row + 8 * bi + 4);
        const float4 b0 = *reinterpret_cast<const float4*>(row + 8 * bj);
        const float4 b1 = *reinterpret_cast<const float4*>(row + 8 * bj + 4);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
      }
    }
    __syncthreads();
  }
  // groups 1..G-1 hand their sums to group 0 through shared memory: the two slab buffers
  // (2 x 32 x 132 floats) take `cap` blocks of 64 values, so as many groups per round
  float* red = &Ys[0][0];
  const int cap = (2 * GB_SLAB * GB_LS) / 64;  // blocks of 64 values that fit
  for (int g0 = 1; g0 < G; g0 += max(1, cap / nblk)) {
    const int g1 = min(G, g0 + max(1, cap / nblk));
    if (active && grp >= g0 && grp < g1) {
      float* dst = red + ((size_t)(grp - g0) * nblk + bp) * 64;
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) dst[a * 8 + b] = acc[a][b];
    }
    __syncthreads();
    if (active && grp == 0)
      for (int gg = g0; gg < g1; ++gg) {
        const float* srcp = red + ((size_t)(gg - g0) * nblk + bp) * 64;
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 8; ++b) acc[a][b] += srcp[a * 8 + b];
      }
    __syncthreads();
  }
  if (active && grp == 0) {
    double* P = g.part + (int64_t)c * l * l;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int i = 8 * bi + a;
      if (i >= l) continue;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int j = 8 * bj + b;
        if (j < l && j >= i) P[(int64_t)i * l + j] = (double)acc[a][b];
      }
    }
  }
}

cudaError_t launch_gram_blocks_b(const GramB* tab, int nprob, int max_chunks, int max_l, cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  if (max_l < 1 || max_l > GB_LP) return cudaErrorInvalidValue;
  gram_blocks_b_kernel<<<dim3((unsigned)max_chunks, 1, (unsigned)nprob), 256, 0, st>>>(tab);
  return launched();
}

// W = sum of the chunk partials in chunk order, a thread per upper entry (coalesced
// across the entries of each partial), mirrored.
__global__ void gram_sum_b_kernel(const GramRedB* __restrict__ tab) {
  const GramRedB& a = tab[blockIdx.z];
  const int64_t ll = (int64_t)a.l * a.l;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ll || (a.stop && *a.stop)) return;
  const int i = (int)(e / a.l), j = (int)(e % a.l);
  if (j < i) return;
  double s = 0.0;
  for (int c = 0; c < a.chunks; ++c) s += a.part[(int64_t)c * ll + e];
  a.W[e] = s;
  a.W[(int64_t)j * a.l + i] = s;
}

cudaError_t launch_gram_sum_b(const GramRedB* tab, int nprob, int max_l, cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  gram_sum_b_kernel<<<dim3((unsigned)cdiv((int64_t)max_l * max_l, 256), 1, (unsigned)nprob), 256, 0, st>>>(tab);
  return launched();
}

}  // namespace gsvdr
