// Metrics of Section 1 without any device allocation.
//
// Some callers cannot let a library allocate device memory: their allocator
// owns all of it, or they call from a place where cudaMalloc is not allowed.
// gsvd_rand_metrics stages its inputs and outputs in a context workspace that
// grows by cudaMalloc.  This file gives those callers gsvd_rand_metrics_noalloc:
// the same quantities from a multi-CTA form of the metrics kernel whose
// scratch (staged inputs and outputs, per-block entropy partials, a
// last-block counter) is one fixed array in the module's static device
// memory.  Every GPU that loads the library holds that array until the
// process exits; its size caps the number of pairs.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "gsvd_rand.h"

namespace gsvdr {
namespace {

constexpr int NA_MAX_N = GSVD_RAND_NOALLOC_MAX_N;
constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BLOCKS = 128;
constexpr int NA_MAX_DEVICES = 64;

// Byte offsets of the scratch regions (each a multiple of 256 bytes).
constexpr size_t NA_VEC = (size_t)NA_MAX_N * sizeof(double);
constexpr size_t NA_OFF_A = 0;                          // staged alpha (r <= N doubles)
constexpr size_t NA_OFF_B = NA_OFF_A + NA_VEC;          // staged beta
constexpr size_t NA_OFF_OUT = NA_OFF_B + NA_VEC;        // staged theta, rho, P1, P2 (N each)
constexpr size_t NA_OFF_D = NA_OFF_OUT + 4 * NA_VEC;    // staged D (2 doubles)
constexpr size_t NA_OFF_PART = NA_OFF_D + 256;          // entropy partials, 2 per block
constexpr size_t NA_OFF_CNT = NA_OFF_PART + NA_MAX_BLOCKS * 2 * sizeof(double);  // blocks done
constexpr size_t NA_BYTES = NA_OFF_CNT + 256;
static_assert(NA_VEC % 256 == 0 && NA_OFF_CNT % 256 == 0, "scratch regions must stay 256-byte aligned");

// The scratch itself: about 1.5 MiB of static device memory per GPU.
static __device__ __align__(256) unsigned char g_metrics_scratch[NA_BYTES];


// Pair i of the (padded) list: pad_mode 0 appends (0, 1), pad_mode 1 prepends (1, 0).
__device__ __forceinline__ void padded_pair(const double* alpha, const double* beta, int r, int N, int pad_mode,
                                            int i, double& a, double& b) {
  const int off = pad_mode == 1 ? N - r : 0;
  const int j = i - off;
  if (j >= 0 && j < r) {
    a = alpha[j];
    b = beta[j];
  } else {
    a = pad_mode == 1 ? 1.0 : 0.0;
    b = pad_mode == 1 ? 0.0 : 1.0;
  }
}

// Sum over the block of two values; the result is valid in every thread.
__device__ __forceinline__ void block_sum2(double& x, double& y, double (*red)[NA_THREADS / 32]) {
  const int tid = threadIdx.x;
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_down_sync(0xffffffffu, x, o);
    y += __shfl_down_sync(0xffffffffu, y, o);
  }
  __syncthreads();
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = x;
    red[1][tid >> 5] = y;
  }
  __syncthreads();
  x = 0.0;
  y = 0.0;
  for (int w = 0; w < NA_THREADS / 32; ++w) {
    x += red[0][w];
    y += red[1][w];
  }
}

// Every block forms the totals sum alpha^2, sum beta^2 over all N pairs in one
// fixed order (so all blocks agree bit for bit), writes theta, rho, P1, P2 for
// its own pairs and its share of the entropy sums; the last block to finish
// adds the shares in block order and writes D.  The counter must be zero at
// launch; the last block sets it back to zero.
__global__ __launch_bounds__(NA_THREADS) void metrics_blocks_kernel(
    const double* __restrict__ alpha, const double* __restrict__ beta, int r, int N, int pad_mode,
    double* theta, double* rho, double* P1, double* P2, double* D, double* part, unsigned int* counter) {
  __shared__ double red[2][NA_THREADS / 32];
  __shared__ int s_last;
  const int tid = threadIdx.x;
  const double quarter_pi = 0.78539816339744830962;
  double ta = 0.0, tb = 0.0;
  for (int i = tid; i < N; i += NA_THREADS) {
    double a, b;
    padded_pair(alpha, beta, r, N, pad_mode, i, a, b);
    ta += a * a;
    tb += b * b;
  }
  block_sum2(ta, tb, red);
  double h1 = 0.0, h2 = 0.0;
  for (int i = blockIdx.x * NA_THREADS + tid; i < N; i += gridDim.x * NA_THREADS) {
    double a, b;
    padded_pair(alpha, beta, r, N, pad_mode, i, a, b);
    const double p1 = ta > 0 ? a * a / ta : 0.0, p2 = tb > 0 ? b * b / tb : 0.0;
    if (theta) theta[i] = atan2(a, b) - quarter_pi;
    if (rho) rho[i] = (b == 0.0) ? __longlong_as_double(0x7ff0000000000000ll) : a / b;
    if (P1) P1[i] = p1;
    if (P2) P2[i] = p2;
    if (p1 > 0) h1 += p1 * log(p1);
    if (p2 > 0) h2 += p2 * log(p2);
  }
  block_sum2(h1, h2, red);
  if (tid == 0) {
    part[2 * blockIdx.x] = h1;
    part[2 * blockIdx.x + 1] = h2;
    __threadfence();
    s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last && tid == 0) {
    __threadfence();
    const volatile double* vp = part;
    double s1 = 0.0, s2 = 0.0;
    for (unsigned int blk = 0; blk < gridDim.x; ++blk) {
      s1 += vp[2 * blk];
      s2 += vp[2 * blk + 1];
    }
    const double lg = log((double)N);
    if (D) {
      D[0] = -s1 / lg;
      D[1] = -s2 / lg;
    }
    *counter = 0u;
  }
}

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Address of the scratch array on `device` (current), looked up with
// cudaGetSymbolAddress at every call: the lookup allocates nothing, and a fresh
// lookup stays right after the device's context was torn down and recreated
// (cudaDeviceReset), where the module can load at another address.  The first
// lookup on a device also loads the module there.
int scratch_base(int device, unsigned char** out) {
  (void)device;
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_metrics_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return GSVD_RAND_ERR_CUDA;
  }
  *out = static_cast<unsigned char*>(p);
  return GSVD_RAND_OK;
}

int metrics_noalloc(int device, cudaStream_t st, const double* alpha, const double* beta, int r, int pad_to_n,
                    int pad_mode, double* theta, double* rho, double* P1, double* P2, double* D) {
  if (!alpha || !beta || r < 1 || (pad_mode != 0 && pad_mode != 1)) return GSVD_RAND_ERR_ARG;
  const int N = pad_to_n > r ? pad_to_n : r;
  if (N < 2) return GSVD_RAND_ERR_ARG;
  if (N > NA_MAX_N) return GSVD_RAND_ERR_TOO_LARGE;
  if (device < 0 || device >= NA_MAX_DEVICES) return GSVD_RAND_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device >= ndev) {
    cudaGetLastError();
    return GSVD_RAND_ERR_ARG;
  }
  if (cudaSetDevice(device) != cudaSuccess) return GSVD_RAND_ERR_CUDA;
  unsigned char* base = nullptr;
  int rc = scratch_base(device, &base);
  if (rc) return rc;
  double* a = reinterpret_cast<double*>(base + NA_OFF_A);
  double* b = reinterpret_cast<double*>(base + NA_OFF_B);
  double* part = reinterpret_cast<double*>(base + NA_OFF_PART);
  unsigned int* counter = reinterpret_cast<unsigned int*>(base + NA_OFF_CNT);
  // inputs: used in place on the device, else copied into the scratch
  const double* da = alpha;
  const double* db = beta;
  const size_t in_bytes = (size_t)r * sizeof(double);
  if (!on_device(alpha)) {
    if (cudaMemcpyAsync(a, alpha, in_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return GSVD_RAND_ERR_CUDA;
    da = a;
  }
  if (!on_device(beta)) {
    if (cudaMemcpyAsync(b, beta, in_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return GSVD_RAND_ERR_CUDA;
    db = b;
  }
  // outputs: written in place on the device, else through the scratch
  double* outs[5] = {theta, rho, P1, P2, D};
  double* dst[5];
  bool staged[5];
  for (int i = 0; i < 5; ++i) {
    staged[i] = outs[i] && !on_device(outs[i]);
    double* sp = reinterpret_cast<double*>(base + (i < 4 ? NA_OFF_OUT + i * NA_VEC : NA_OFF_D));
    dst[i] = staged[i] ? sp : outs[i];
  }
  if (cudaMemsetAsync(counter, 0, sizeof(unsigned int), st) != cudaSuccess) return GSVD_RAND_ERR_CUDA;
  const int blocks = (int)std::min<int64_t>(NA_MAX_BLOCKS, cdiv(N, NA_THREADS));
  metrics_blocks_kernel<<<blocks, NA_THREADS, 0, st>>>(da, db, r, N, pad_mode, dst[0], dst[1], dst[2], dst[3],
                                                       dst[4], part, counter);
  if (launched() != cudaSuccess) return GSVD_RAND_ERR_CUDA;
  for (int i = 0; i < 5; ++i) {
    if (!staged[i]) continue;
    const size_t bytes = (i < 4 ? (size_t)N : 2) * sizeof(double);
    if (cudaMemcpyAsync(outs[i], dst[i], bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) return GSVD_RAND_ERR_CUDA;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return GSVD_RAND_ERR_CUDA;
  return GSVD_RAND_OK;
}

}  // namespace
}  // namespace gsvdr

extern "C" int gsvd_rand_metrics_noalloc(int device, void* stream, const double* alpha, const double* beta, int r,
                                         int pad_to_n, int pad_mode, double* theta, double* rho, double* P1,
                                         double* P2, double* D) {
  int prev = -1;
  const bool have_prev = cudaGetDevice(&prev) == cudaSuccess;
  const int rc = gsvdr::metrics_noalloc(device, static_cast<cudaStream_t>(stream), alpha, beta, r, pad_to_n,
                                        pad_mode, theta, rho, P1, P2, D);
  if (have_prev && prev != device) cudaSetDevice(prev);
  return rc;
}
