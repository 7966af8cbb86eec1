// Shared device helpers of the GB300 randomized-GSV library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cmath>

namespace gsvdr {

// Number of kernels this library has launched (all contexts, all threads).
extern std::atomic<uint64_t> g_launch_count;
inline cudaError_t launched(int n = 1) {
  g_launch_count.fetch_add((uint64_t)n, std::memory_order_relaxed);
  return cudaGetLastError();
}

// Device status word: the first failure wins (atomicCAS from 0).
struct DevStatus {
  int code;   // 0 or a GSVD_RAND_ERR_* value
  int where;  // stage id that failed
  int index;  // e.g. the pivot that broke down
  int pad;
};

__device__ __forceinline__ void set_status(DevStatus* st, int code, int where, int index) {
  if (st && atomicCAS(&st->code, 0, code) == 0) {
    st->where = where;
    st->index = index;
  }
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Section 3): written from
// the published definition.  round: (h0,l0) = hi/lo(M0 * c0), (h1,l1) =
// hi/lo(M1 * c2); c <- (h1 ^ c1 ^ k0, l1, h0 ^ c3 ^ k1, l0); the key is bumped
// by the Weyl constants between rounds.
struct Philox4 {
  uint32_t x[4];
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += W0;
      k1 += W1;
    }
    uint32_t h0 = __umulhi(M0, c0), l0 = M0 * c0;
    uint32_t h1 = __umulhi(M1, c2), l1 = M1 * c2;
    uint32_t n0 = h1 ^ c1 ^ k0, n2 = h0 ^ c3 ^ k1;
    c0 = n0;
    c1 = l1;
    c2 = n2;
    c3 = l0;
  }
  Philox4 o;
  o.x[0] = c0;
  o.x[1] = c1;
  o.x[2] = c2;
  o.x[3] = c3;
  return o;
}

// Box-Muller (Box & Muller 1958) of one Philox output in FP64: two 53-bit
// uniforms u1 in (0,1), u2 in [0,1); z0 = r cos(2 pi u2), z1 = r sin(2 pi u2).
__device__ __forceinline__ void box_muller_f64(const Philox4& w, double& z0, double& z1) {
  const double two53i = 1.1102230246251565404236316680908203125e-16;  // 2^-53
  double u1 = ((double)(w.x[0] >> 5) * 67108864.0 + (double)(w.x[1] >> 6) + 0.5) * two53i;
  double u2 = ((double)(w.x[2] >> 5) * 67108864.0 + (double)(w.x[3] >> 6)) * two53i;
  double r = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

// The same transform evaluated in FP32 from the same words (used where Omega
// is rounded to TF32/BF16 anyway).  u1 and u2 are the FP64 uniforms rounded to
// FP32 (relative error 2^-23 at every magnitude), so z agrees with the FP64
// values to about 1e-7 relative.
__device__ __forceinline__ void box_muller_f32(const Philox4& w, float& z0, float& z1) {
  const float s27 = 7.450580596923828125e-09f;   // 2^-27
  const float s53 = 1.1102230246251565e-16f;     // 2^-53
  const float s54 = 5.5511151231257827e-17f;     // 2^-54
  float u1 = fmaf((float)(w.x[0] >> 5), s27, fmaf((float)(w.x[1] >> 6), s53, s54));
  float u2 = fmaf((float)(w.x[2] >> 5), s27, (float)(w.x[3] >> 6) * s53);
  float r = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

template <typename T>
__device__ __forceinline__ bool finite_val(T v) {
  return isfinite(v);
}

__host__ __device__ __forceinline__ int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// x - tf32(x) with tf32(x) the truncation the tensor core applies to an FP32 operand of a
// kind::tf32 MMA (the low 13 mantissa bits cleared): exact, the low half of a 3xTF32 operand.
__device__ __forceinline__ float tf32_low_half(float x) {
  return x - __uint_as_float(__float_as_uint(x) & 0xffffe000u);
}
__host__ __device__ __forceinline__ int64_t round_up(int64_t a, int64_t b) { return cdiv(a, b) * b; }

}  // namespace gsvdr
