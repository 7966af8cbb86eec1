// Algorithm 1 (BasisExt) for many sides at once: the batched kernels of a grouped adaptive
// solve.  Every side grows its basis Q by blocks of b columns; block i of side s is
//     Y_i = G Omega_i,  Y_i <- Y_i - Q (Q^T Y_i) (twice),  P_i = orth(Y_i),
//     P_i <- orth(P_i - Q (Q^T P_i)),  Q <- [Q, P_i],
// and the side stops once the cumulated residual of Section 2,
//     sqrt(||G||_F^2 - sum_i ||P_i^T G||_F^2) / ||G||_F,
// is at most tol (or its basis reaches its column cap).  The stop test runs here, on the
// device: each side has a stop word (0 while it still adds blocks, then its final column
// count), and every block kernel of a side whose word is set returns at once, so the whole
// sequence of blocks is one static launch sequence (captured into a CUDA graph) with no host
// read between blocks.
//
// The basis is kept K-major (Qt: row a is column a of Q, length M, row stride ldq), the form
// the tensor-core products take; the block Y is row-major (M x bi, ld ldy).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "gsvd_rand.h"
#include "common.cuh"
#include "kernels.h"

namespace gsvdr {

namespace {

constexpr int XG_ROWS = 256;  // rows of one cross-Gram chunk
constexpr int XG_THREADS = 256;

__device__ __forceinline__ bool side_done(const int* stop) { return stop != nullptr && *stop != 0; }

// part[chunk][a][t] = sum over the chunk's rows of Qt[a][row] Y[row][t]  (a < c, t < bi):
// the chunk of Y in shared memory, FP32 FMAs over the chunk, the chunk sum stored in FP64.
__global__ __launch_bounds__(XG_THREADS) void xgram_blocks_b_kernel(const AdaptB* __restrict__ tab) {
  const AdaptB& a = tab[blockIdx.y];
  if (side_done(a.stop) || a.c == 0) return;
  const int64_t r0 = (int64_t)blockIdx.x * XG_ROWS;
  if (r0 >= a.M) return;
  extern __shared__ float ysh[];  // XG_ROWS x bi
  const int rows = (int)min((int64_t)XG_ROWS, a.M - r0), bi = a.bi;
  for (int e = threadIdx.x; e < rows * bi; e += XG_THREADS) {
    const int r = e / bi, t = e % bi;
    ysh[e] = a.Y[(r0 + r) * a.ldy + t];
  }
  __syncthreads();
  double* part = a.xpart + (int64_t)blockIdx.x * a.c * bi;
  for (int o = threadIdx.x; o < a.c * bi; o += XG_THREADS) {
    const int q = o / bi, t = o % bi;
    const float* qr = a.Qt + (int64_t)q * a.ldq + r0;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s = fmaf(qr[r], ysh[r * bi + t], s);
    part[o] = (double)s;
  }
}

// C[a][t] = sum of the chunk partials (FP64, chunk order: deterministic).
__global__ __launch_bounds__(256) void xgram_sum_b_kernel(const AdaptB* __restrict__ tab) {
  const AdaptB& a = tab[blockIdx.y];
  if (side_done(a.stop) || a.c == 0) return;
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= a.c * a.bi) return;
  const int chunks = (int)((a.M + XG_ROWS - 1) / XG_ROWS);
  double s = 0.0;
  for (int k = 0; k < chunks; ++k) s += a.xpart[(int64_t)k * a.c * a.bi + o];
  a.C[o] = s;
}

// Y[row][t] -= sum_a Qt[a][row] C[a][t]: a thread per row, C in shared memory (FP32).
__global__ __launch_bounds__(256) void project_out_b_kernel(const AdaptB* __restrict__ tab) {
  const AdaptB& a = tab[blockIdx.y];
  if (side_done(a.stop) || a.c == 0) return;
  extern __shared__ float csh[];  // c x bi
  const int c = a.c, bi = a.bi;
  for (int e = threadIdx.x; e < c * bi; e += blockDim.x) csh[e] = (float)a.C[e];
  __syncthreads();
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= a.M) return;
  float acc[ADAPT_BMAX];
#pragma unroll
  for (int t = 0; t < ADAPT_BMAX; ++t) acc[t] = 0.f;
  for (int q = 0; q < c; ++q) {
    const float v = a.Qt[(int64_t)q * a.ldq + row];
#pragma unroll
    for (int t = 0; t < ADAPT_BMAX; ++t)
      if (t < bi) acc[t] = fmaf(v, csh[q * bi + t], acc[t]);
  }
  float* y = a.Y + row * a.ldy;
#pragma unroll
  for (int t = 0; t < ADAPT_BMAX; ++t)
    if (t < bi) y[t] -= acc[t];
}

// The stop test of one side after block i: ||G||_F^2 from the first block's partial sums,
// the block's ||P_i^T G||_F^2 added to the running sum, the cumulated relative residual;
// the stop word takes the column count when it is at most tol or the cap is reached.
__global__ void adapt_stop_b_kernel(const AdaptStopB* __restrict__ tab, int nprob) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nprob) return;
  const AdaptStopB& s = tab[j];
  if (*s.stop != 0) return;
  double* st = s.state;  // [0] ||G||^2, [1] running sum, [2] estimate
  if (s.first) {
    double g2 = 0.0;
    for (int k = 0; k < s.ng; ++k) g2 += s.gpart[k];
    st[0] = g2;
    st[1] = 0.0;
  }
  double b2 = 0.0;
  for (int k = 0; k < s.nb; ++k) b2 += s.bpart[k];
  st[1] += b2;
  const double g2 = st[0];
  const double est = g2 > 0.0 ? sqrt(fmax(g2 - st[1], 0.0) / g2) : 0.0;
  st[2] = est;
  *s.resid_out = est;
  if (est <= s.tol || s.last) {
    *s.stop = s.cols;
    if (est > s.tol) set_status(s.st, GSVD_RAND_ERR_TOL_MISS, 90, s.cols);
  }
}

__global__ void adapt_trim_b_kernel(const AdaptTrimB* __restrict__ tab, int mode) {
  const AdaptTrimB& t = tab[blockIdx.y];
  const int ract = min(t.r, *t.stop1 + *t.stop2);
  if (ract >= t.r) return;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (mode == 0) {
    if (e >= (int64_t)t.L * t.r) return;
    const int col = (int)(e % t.r);
    if (col >= ract) t.Zr[e] = 0.0;
  } else {
    const int j = ract + (int)e;
    if (j < t.r) t.C1[(int64_t)j * t.r + j] = -1.0;
  }
}

// Rows [stop, cap) of Qt zeroed (the blocks added after the side stopped never ran, or ran
// before the stop was known): Q^T G then has zero rows there, which leave the GSVs unchanged.
__global__ void adapt_mask_b_kernel(const AdaptMaskB* __restrict__ tab) {
  const AdaptMaskB& m = tab[blockIdx.y];
  const int stop = *m.stop;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t rows = m.cap - stop;
  if (rows <= 0 || e >= rows * m.ldq) return;
  m.Qt[(int64_t)stop * m.ldq + e] = 0.f;
}

// ||P^T G||_F^2 of a block P (bi columns: rows [c, c + bi) of Qt), on the CUDA cores: the
// tensor-core product's long accumulation chains round toward zero (a bias of ~1e-5 relative
// over thousands of rows), which would set a floor near 1e-2 under the cumulated residual.
// Partials: a thread per column j of G, FP32 FMAs over a chunk of EN_ROWS rows (round to
// nearest), part[(chunk n + j) bi + t] = sum over the chunk of P[row][t] G[row][j].
constexpr int EN_ROWS = 2048, EN_COLS = 128, EN_TILE = 64, EN_UNROLL = 8;
__global__ __launch_bounds__(EN_COLS) void energy_part_b_kernel(const AdaptEnergyB* __restrict__ tab) {
  const AdaptEnergyB& a = tab[blockIdx.z];
  if (side_done(a.stop)) return;
  const int64_t r0 = (int64_t)blockIdx.y * EN_ROWS;
  if (r0 >= a.M) return;
  const int64_t j = (int64_t)blockIdx.x * EN_COLS + threadIdx.x;
  __shared__ float psh[EN_TILE][ADAPT_BMAX];
  const int bi = a.bi;
  const int64_t r1 = min(a.M, r0 + EN_ROWS);
  float acc[ADAPT_BMAX];
#pragma unroll
  for (int t = 0; t < ADAPT_BMAX; ++t) acc[t] = 0.f;
  for (int64_t rt = r0; rt < r1; rt += EN_TILE) {
    const int rows = (int)min((int64_t)EN_TILE, r1 - rt);
    __syncthreads();
    for (int e = threadIdx.x; e < rows * bi; e += EN_COLS) {
      const int r = e % rows, t = e / rows;
      psh[r][t] = a.Qt[(int64_t)(a.c + t) * a.ldq + rt + r];
    }
    __syncthreads();
    if ((int64_t)blockIdx.x * EN_COLS >= a.n) continue;
    if (j < a.n) {
      // EN_UNROLL rows of G loaded ahead of their FMAs (memory-level parallelism: one load in
      // flight per warp would leave HBM mostly idle); the sums keep their row order
      const float* gp = a.G + rt * a.ldg + j;
      int r = 0;
      for (; r + EN_UNROLL <= rows; r += EN_UNROLL) {
        float g[EN_UNROLL];
#pragma unroll
        for (int u = 0; u < EN_UNROLL; ++u) g[u] = __ldg(gp + (int64_t)(r + u) * a.ldg);
#pragma unroll
        for (int u = 0; u < EN_UNROLL; ++u)
#pragma unroll
          for (int t = 0; t < ADAPT_BMAX; ++t)
            if (t < bi) acc[t] = fmaf(psh[r + u][t], g[u], acc[t]);
      }
      for (; r < rows; ++r) {
        const float g = gp[(int64_t)r * a.ldg];
#pragma unroll
        for (int t = 0; t < ADAPT_BMAX; ++t)
          if (t < bi) acc[t] = fmaf(psh[r][t], g, acc[t]);
      }
    }
  }
  if (j >= a.n) return;
  float* out = a.part + ((int64_t)blockIdx.y * a.n + j) * bi;
#pragma unroll
  for (int t = 0; t < ADAPT_BMAX; ++t)  // unrolled: acc stays in registers
    if (t < bi) out[t] = acc[t];
}

// epart[b] = sum over entries e in [256 b, 256 b + 256) of (sum over chunks of part)^2, in FP64.
__global__ __launch_bounds__(256) void energy_sum_b_kernel(const AdaptEnergyB* __restrict__ tab) {
  const AdaptEnergyB& a = tab[blockIdx.y];
  if (side_done(a.stop)) return;
  const int64_t nb = a.n * a.bi;
  if ((int64_t)blockIdx.x * 256 >= nb) {  // past the entries: a slot to clear, or nothing
    if (threadIdx.x == 0 && (int64_t)blockIdx.x < a.nb_out) a.epart[blockIdx.x] = 0.0;
    return;
  }
  const int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x;
  double v = 0.0;
  if (e < nb) {
    const int chunks = (int)((a.M + EN_ROWS - 1) / EN_ROWS);
    for (int k = 0; k < chunks; ++k) v += (double)a.part[(int64_t)k * nb + e];
  }
  double sq = v * v;
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  __shared__ double ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += ws[w];
    a.epart[blockIdx.x] = s;
  }
}

}  // namespace

int64_t adapt_energy_part_elems(int64_t M, int64_t n, int bi) {
  return ((M + EN_ROWS - 1) / EN_ROWS) * n * (int64_t)bi;
}

cudaError_t launch_adapt_energy_b(const AdaptEnergyB* tab, int nprob, int64_t max_M, int64_t max_n, int max_bi,
                                  cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  if (max_bi > ADAPT_BMAX) return cudaErrorInvalidValue;
  // (nb_out never exceeds cdiv(max_n ADAPT_BMAX, 256): the grid below covers it when callers
  // pass max_bi = ADAPT_BMAX for tables that clear slots)
  const dim3 g1((unsigned)((max_n + EN_COLS - 1) / EN_COLS), (unsigned)((max_M + EN_ROWS - 1) / EN_ROWS),
                (unsigned)nprob);
  energy_part_b_kernel<<<g1, EN_COLS, 0, st>>>(tab);
  cudaError_t e = launched();
  if (e) return e;
  const dim3 g2((unsigned)((max_n * max_bi + 255) / 256), (unsigned)nprob);
  energy_sum_b_kernel<<<g2, 256, 0, st>>>(tab);
  return launched();
}

cudaError_t launch_adapt_project_b(const AdaptB* tab, int nprob, int64_t max_M, int max_c, int max_bi, cudaStream_t st) {
  if (nprob <= 0 || max_c <= 0) return cudaSuccess;
  if (max_bi > ADAPT_BMAX || max_c > ADAPT_CMAX) return cudaErrorInvalidValue;
  const int chunks = (int)((max_M + XG_ROWS - 1) / XG_ROWS);
  const size_t ysm = (size_t)XG_ROWS * max_bi * sizeof(float);
  xgram_blocks_b_kernel<<<dim3((unsigned)chunks, (unsigned)nprob), XG_THREADS, ysm, st>>>(tab);
  cudaError_t e = launched();
  if (e) return e;
  const int outs = max_c * max_bi;
  xgram_sum_b_kernel<<<dim3((unsigned)((outs + 255) / 256), (unsigned)nprob), 256, 0, st>>>(tab);
  if ((e = launched())) return e;
  const size_t csm = (size_t)max_c * max_bi * sizeof(float);
  project_out_b_kernel<<<dim3((unsigned)((max_M + 255) / 256), (unsigned)nprob), 256, csm, st>>>(tab);
  return launched();
}

int64_t adapt_xpart_elems(int64_t M, int c, int bi) { return ((M + XG_ROWS - 1) / XG_ROWS) * (int64_t)c * bi; }

cudaError_t launch_adapt_stop_b(const AdaptStopB* tab, int nprob, cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  adapt_stop_b_kernel<<<(nprob + 127) / 128, 128, 0, st>>>(tab, nprob);
  return launched();
}

cudaError_t launch_adapt_trim_b(const AdaptTrimB* tab, int nprob, int max_L, int max_r, int mode, cudaStream_t st) {
  if (nprob <= 0 || max_r <= 0) return cudaSuccess;
  const int64_t n = mode == 0 ? (int64_t)max_L * max_r : max_r;
  adapt_trim_b_kernel<<<dim3((unsigned)((n + 255) / 256), (unsigned)nprob), 256, 0, st>>>(tab, mode);
  return launched();
}

cudaError_t launch_adapt_mask_b(const AdaptMaskB* tab, int nprob, int64_t max_elems, cudaStream_t st) {
  if (nprob <= 0 || max_elems <= 0) return cudaSuccess;
  adapt_mask_b_kernel<<<dim3((unsigned)((max_elems + 255) / 256), (unsigned)nprob), 256, 0, st>>>(tab);
  return launched();
}

}  // namespace gsvdr
