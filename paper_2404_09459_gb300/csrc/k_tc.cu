// Tensor-core products of the basis extraction on sm_103a: tcgen05.mma with
// TF32 (kind::tf32) or BF16 (kind::f16) operands and FP32 accumulation in
// tensor memory, operands staged by TMA (cp.async.bulk.tensor, 128-byte
// swizzle) through an mbarrier pipeline.  One stage holds 128 bytes of K per
// operand row: 32 FP32 or 64 BF16 elements.
//
//   GX  : Y (M x l) = G (M x n) X        A = G tile (128 rows, K-major),
//                                        B = X^T tile (K-major), one CTA per 128 rows.
//   GTQ : Z (n x l) = G^T Q, split-K     A = G^T tile (128 columns of G, MN-major),
//                                        B = Q^T tile (K-major), one CTA per
//                                        (128 columns, row chunk); FP32 partials.
//
// Warp roles (6 warps): warp 0 issues TMA, warp 1 owns the tensor memory and
// issues the MMAs (one thread), warps 2-5 drain the accumulator (tcgen05.ld)
// and, on the first sketch pass, fold ||G||_F^2 from the staged tiles.  Every
// mbarrier wait is bounded; a timeout is reported as GSVD_RAND_ERR_TIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "kernels.h"
#include "tc.h"

namespace gsvdr {

// One problem of a grouped product, in device memory (the tensor maps must be
// 64-byte aligned there).
struct TcGroupProb {  // CUtensorMap members carry their own (>= 64-byte) alignment
  CUtensorMap mapA;   // G: row tiles (GX) or unswizzled 32 x 32 boxes (GTQ)
  CUtensorMap mapB;   // K-major B operand: X^T (GX) or Q^T (GTQ)
  CUtensorMap mapBlo; // GX, 3xTF32, has_blo: B - tf32(B), the same geometry as mapB
  float* out;         // Y (GX) or the split partials (GTQ)
  int64_t ldo, out_rows, kdim, rows_per_split, split_stride;
  double* gnorm_part; // GX with the fused norm: 4 partial sums of G^2 per row tile
  int ncols, nmma, tiles_x, transpose_out;  // transpose_out: out[c * ldo + row] (GX)
  const int* stop;    // null, or the stop word of the problem (non-zero: its tiles are filtered out)
  int has_blo, pad_;
};

namespace {

constexpr int TC_BM = 128;       // MMA M (rows of the accumulator / TMEM lanes)
constexpr int TC_BK = 32;        // K depth of one FP32 stage: 32 floats = one 128-byte swizzle row
constexpr int TC_KSTEP_BYTES = 32;  // K of one MMA: 8 TF32 or 16 BF16 elements
constexpr int TC_A_BYTES = TC_BM * TC_BK * 4;  // 16 KB
constexpr uint32_t WAIT_SPINS = 1u << 22;      // bounded waits (try_wait suspends per call)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false if this thread gave up or another role already did.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  for (uint32_t it = 0; it < WAIT_SPINS; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// The same with A read from tensor memory (M rows in lanes, one 32-bit column per K element).
__device__ __forceinline__ void mma_tf32_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Sixteen consecutive 32-bit columns of this thread's lane (warp-wide, its own 32-lane quarter).
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Arrive on `bar` once all previously issued MMAs of this thread have completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading and stride
// byte offsets (all >> 4), descriptor version 1, 128-byte swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor, kind::tf32: D = F32, A = B = TF32, A/B major bits, N >> 3, M >> 4.
__host__ __device__ constexpr uint32_t idesc_tf32(uint32_t m, uint32_t n, uint32_t a_mn, uint32_t b_mn) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (a_mn << 15) | (b_mn << 16) | ((n >> 3) << 17) | ((m >> 4) << 24);
}
// kind::f16 with A = B = BF16 (format 1), D = F32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(uint32_t m, uint32_t n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

struct SqAccF {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float v) {
    float p = v * v;
    float e = fmaf(v, v, -p);
    float t = hi + p;
    float z = t - hi;
    lo += ((hi - (t - z)) + (p - z)) + e;
    hi = t;
  }
  // a short partial sum (of at most 16 squares, summed with plain FMAs: relative error a few
  // units of FP32 rounding, of either sign) added with the same compensation
  __device__ __forceinline__ void add_sum(float p) {
    float t = hi + p;
    float z = t - hi;
    lo += (hi - (t - z)) + (p - z);
    hi = t;
  }
};

}  // namespace

// Byte offsets of the buffers inside one pipeline stage (all 1024-byte aligned):
//   A    TMA target for A: the G tile K-major (GX) or the staged G tile (GTQ)
//   B    TMA target for B (X^T or Q^T tile, K-major)
//   AK   K-major A fed to the MMA (= A in GX, the transposed tile in GTQ)
//   ALO  (3xTF32) A - tf32(A) in the layout of AK
//   BLO  (3xTF32) B - tf32(B); (BF16 split) TMA target for the low half of B
struct StageLayout {
  uint32_t a, b, ak, alo, blo, bytes;
  __host__ __device__ StageLayout(int mode, bool split, int nmma, int eb = 4) {
    const uint32_t nb = ((uint32_t)nmma * 128u + 1023u) & ~1023u;
    a = 0;
    b = TC_A_BYTES;
    uint32_t o = b + nb;
    ak = a;
    if (mode == 1) {
      ak = o;
      o += TC_A_BYTES;
    }
    alo = blo = 0;
    if (split) {
      if (eb == 4) {
        alo = o;
        o += TC_A_BYTES;
      }
      blo = o;
      o += nb;
    }
    bytes = o;
  }
};

__device__ __forceinline__ float tf32_lo(float x) {
  return x - __uint_as_float(__float_as_uint(x) & 0xffffe000u);  // exact; the MMA truncates x to its high part
}

// mode 0 (GX): tile = blockIdx.x (rows m0 = 128 tile), K = n.
// mode 1 (GTQ): tile = blockIdx.x (G columns c0 = 128 tile), split = blockIdx.y (rows).
// EB = 4 (FP32 data, kind::tf32).  SPLIT: 3xTF32, D += A_hi B_hi + A_lo B_hi + A_hi B_lo
// (the tensor core truncates each FP32 operand to TF32, so A_hi is A itself and
// A_lo = A - tf32(A), formed in shared memory).
// EB = 2 (BF16 data, kind::f16).  G is exact in BF16; SPLIT: B comes as two BF16
// halves hi + lo (both loaded by TMA, mapB2 = lo), D += A B_hi + A B_lo.
template <int MODE, bool NORM, bool SPLIT, int EB>
__global__ __launch_bounds__(192) void tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA,
                                                      const __grid_constant__ CUtensorMap mapB,
                                                      const __grid_constant__ CUtensorMap mapB2, float* __restrict__ out,
                                                      int64_t ldo, int64_t out_rows, int ncols, int nmma, int tmem_cols,
                                                      int64_t kdim, int64_t rows_per_split, int64_t split_stride,
                                                      int stages, double* __restrict__ gnorm_part, DevStatus* st_dev) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  constexpr int BKE = 128 / EB;  // K elements of one stage
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const StageLayout L(MODE, SPLIT, nmma, EB);
  const uint32_t b_bytes = (uint32_t)nmma * 128u;
  uint64_t* full = reinterpret_cast<uint64_t*>(base + (size_t)stages * L.bytes);
  uint64_t* empty = full + stages;
  uint64_t* tfull = empty + stages;  // operands prepared by the epilogue warps
  uint64_t* accum = tfull + stages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  // The tensor cores are fed K-major operands only here, so in GTQ the epilogue
  // warps transpose each staged G tile (BKE rows x 128 columns, unswizzled)
  // into the K-major 128-byte-swizzled layout of A (128 rows x 128 bytes).
  constexpr bool TRANSPOSE = MODE == 1;
  constexpr bool PREP = TRANSPOSE || (SPLIT && EB == 4);  // MMA waits for the prepared operands
  constexpr bool EPI_STAGE = PREP || NORM;                // epilogue warps visit every stage
  constexpr bool B2 = SPLIT && EB == 2;                    // second B operand by TMA
  __shared__ int s_abort;
  __shared__ double s_red[4];

  int64_t k_begin, k_end;
  if (MODE == 0) {
    k_begin = 0;
    k_end = kdim;
  } else {
    k_begin = (int64_t)blockIdx.y * rows_per_split;
    k_end = min(kdim, k_begin + rows_per_split);
  }
  const int ktiles = (int)((k_end - k_begin + BKE - 1) / BKE);
  const int tile0 = blockIdx.x * TC_BM;

  if (tid == 0) {
    s_abort = 0;
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], EPI_STAGE ? 5 : 1);
      mbar_init(&tfull[s], 4);
    }
    mbar_init(accum, 1);
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, (uint32_t)tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int* abort_flag = &s_abort;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int issued = 0;
      for (int kt = 0; kt < ktiles; ++kt) {
        const int s = kt % stages;
        const uint32_t ph = (uint32_t)(kt / stages) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag)) break;
        ++issued;
        uint8_t* st = base + (size_t)s * L.bytes;
        mbar_expect_tx(&full[s], (uint32_t)TC_A_BYTES + b_bytes * (B2 ? 2u : 1u));
        const int k0 = (int)(k_begin + (int64_t)kt * BKE);
        if (MODE == 0) {
          tma_load_2d(st + L.a, &mapA, &full[s], k0, tile0);  // G[tile0.., k0..]: 128 rows x 128 bytes
        } else {
          // G[k0.., tile0 + ..]: BKE rows x 128 columns as unswizzled boxes of 128-byte rows
          constexpr int NBOX = 128 / BKE;
#pragma unroll
          for (int q = 0; q < NBOX; ++q)
            tma_load_2d(st + L.a + q * (BKE * 128), &mapA, &full[s], tile0 + BKE * q, k0);
        }
        tma_load_2d(st + L.b, &mapB, &full[s], k0, 0);  // B^T rows 0..nmma-1, K k0..k0+BKE-1
        if (B2) tma_load_2d(st + L.blo, &mapB2, &full[s], k0, 0);
      }
      if (*abort_flag) {
        // drain: wait (bounded) until the copies this thread issued have landed
        for (int kt = max(0, issued - stages); kt < issued; ++kt) {
          volatile int none = 0;
          mbar_wait(&full[kt % stages], (uint32_t)(kt / stages) & 1u, &none);
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = EB == 4 ? idesc_tf32(TC_BM, (uint32_t)nmma, 0u, 0u) : idesc_bf16(TC_BM, (uint32_t)nmma);
      for (int kt = 0; kt < ktiles; ++kt) {
        const int s = kt % stages;
        const uint32_t ph = (uint32_t)(kt / stages) & 1u;
        if (!mbar_wait(PREP ? &tfull[s] : &full[s], ph, abort_flag)) break;
        tc_fence_after();
        const uint32_t st = smem_u32(base + (size_t)s * L.bytes);
#pragma unroll
        for (int ks = 0; ks < 128 / TC_KSTEP_BYTES; ++ks) {
          // K-major operands: 8-row groups 1024 B apart, K step = 32 B inside the swizzle row
          const uint64_t adesc = smem_desc(st + L.ak + ks * TC_KSTEP_BYTES, 16, 1024);
          const uint64_t bdesc = smem_desc(st + L.b + ks * TC_KSTEP_BYTES, 16, 1024);
          const uint32_t acc = (kt > 0 || ks > 0) ? 1u : 0u;
          if (EB == 4) {
            mma_tf32(tmem, adesc, bdesc, idesc, acc);
            if (SPLIT) {
              mma_tf32(tmem, smem_desc(st + L.alo + ks * TC_KSTEP_BYTES, 16, 1024), bdesc, idesc, 1u);
              mma_tf32(tmem, adesc, smem_desc(st + L.blo + ks * TC_KSTEP_BYTES, 16, 1024), idesc, 1u);
            }
          } else {
            mma_f16(tmem, adesc, bdesc, idesc, acc);
            if (SPLIT) mma_f16(tmem, adesc, smem_desc(st + L.blo + ks * TC_KSTEP_BYTES, 16, 1024), idesc, 1u);
          }
        }
        mma_commit(&empty[s]);
      }
      // always: arrives once every MMA issued above has completed (at once if none),
      // so after the epilogue's wait no MMA is in flight when the TMEM is freed
      mma_commit(accum);
    }
  } else {
    // ---------------- epilogue (warps 2-5) ----------------
    const int q = warp & 3;  // TMEM sub-partition of this warp: lanes 32q .. 32q + 31
    const int et = tid - 64;  // 0..127
    SqAccF sq;
    if (EPI_STAGE) {
      for (int kt = 0; kt < ktiles; ++kt) {
        const int s = kt % stages;
        const uint32_t ph = (uint32_t)(kt / stages) & 1u;
        if (!mbar_wait(&full[s], ph, abort_flag)) break;
        uint8_t* st = base + (size_t)s * L.bytes;
        if (TRANSPOSE && EB == 4) {
          // thread c owns row c of the K-major tile: staged value (k, c) sits at
          // (c / 32) * 4 KB + k * 128 B + (c % 32) * 4 B; row c is 128 B whose
          // 16-byte chunk ch lands at chunk ch ^ (c % 8) (128-byte swizzle).
          const int c = et;
          const float* stg = reinterpret_cast<const float*>(st + L.a + (c >> 5) * (TC_BK * 128)) + (c & 31);
          uint8_t* row = st + L.ak + c * 128;
          uint8_t* rlo = st + L.alo + c * 128;
#pragma unroll
          for (int ch = 0; ch < 8; ++ch) {
            float4 v = make_float4(stg[(4 * ch + 0) * 32], stg[(4 * ch + 1) * 32], stg[(4 * ch + 2) * 32],
                                   stg[(4 * ch + 3) * 32]);
            const int off = (ch ^ (c & 7)) << 4;
            *reinterpret_cast<float4*>(row + off) = v;
            if (SPLIT)
              *reinterpret_cast<float4*>(rlo + off) = make_float4(tf32_lo(v.x), tf32_lo(v.y), tf32_lo(v.z), tf32_lo(v.w));
          }
        } else if (TRANSPOSE) {
          // BF16: thread (cp, h) takes columns 2cp, 2cp+1 and K rows 32h .. 32h+31.  The
          // staged 32-bit word (k, cp) holds (k, 2cp) low and (k, 2cp+1) high, at
          // (cp / 32) * 8 KB + k * 128 B + (cp % 32) * 4 B.  Two such words of rows k, k+1
          // give one word of row 2cp and one of row 2cp+1 of the K-major tile.
          const int cp = et & 63, hh = et >> 6;
          const uint32_t* stg = reinterpret_cast<const uint32_t*>(st + L.a + (cp >> 5) * (64 * 128)) + (cp & 31);
          const int r0 = 2 * cp, r1 = 2 * cp + 1;
          uint8_t* row0 = st + L.ak + r0 * 128;
          uint8_t* row1 = st + L.ak + r1 * 128;
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            const int ch = 4 * hh + cc;  // 16-byte chunk: K = 8ch .. 8ch + 7
            uint32_t w[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) w[i] = stg[(8 * ch + i) * 32];
            uint4 a0, a1;
            a0.x = __byte_perm(w[0], w[1], 0x5410);
            a0.y = __byte_perm(w[2], w[3], 0x5410);
            a0.z = __byte_perm(w[4], w[5], 0x5410);
            a0.w = __byte_perm(w[6], w[7], 0x5410);
            a1.x = __byte_perm(w[0], w[1], 0x7632);
            a1.y = __byte_perm(w[2], w[3], 0x7632);
            a1.z = __byte_perm(w[4], w[5], 0x7632);
            a1.w = __byte_perm(w[6], w[7], 0x7632);
            *reinterpret_cast<uint4*>(row0 + ((ch ^ (r0 & 7)) << 4)) = a0;
            *reinterpret_cast<uint4*>(row1 + ((ch ^ (r1 & 7)) << 4)) = a1;
          }
        } else if ((SPLIT && EB == 4) || NORM) {
          // elementwise on the swizzled tile: the layout is preserved
          const float4* a4 = reinterpret_cast<const float4*>(st + L.a);
          float4* lo4 = reinterpret_cast<float4*>(st + L.alo);
          for (int i = et; i < TC_A_BYTES / 16; i += 128) {
            float4 v = a4[i];
            if (EB == 4) {
              if (NORM) {
                sq.add(v.x);
                sq.add(v.y);
                sq.add(v.z);
                sq.add(v.w);
              }
              if (SPLIT) lo4[i] = make_float4(tf32_lo(v.x), tf32_lo(v.y), tf32_lo(v.z), tf32_lo(v.w));
            } else {
              const uint32_t w[4] = {__float_as_uint(v.x), __float_as_uint(v.y), __float_as_uint(v.z),
                                     __float_as_uint(v.w)};
#pragma unroll
              for (int t = 0; t < 4; ++t) {
                sq.add(__uint_as_float(w[t] << 16));
                sq.add(__uint_as_float(w[t] & 0xffff0000u));
              }
            }
          }
        }
        if (SPLIT && EB == 4) {
          const float4* b4 = reinterpret_cast<const float4*>(st + L.b);
          float4* blo4 = reinterpret_cast<float4*>(st + L.blo);
          for (int i = et; i < (int)(b_bytes / 16); i += 128) {
            float4 v = b4[i];
            blo4[i] = make_float4(tf32_lo(v.x), tf32_lo(v.y), tf32_lo(v.z), tf32_lo(v.w));
          }
        }
        // make the generic-proxy writes visible to the tensor cores (async proxy)
        if (PREP) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          if (PREP) mbar_arrive(&tfull[s]);
          mbar_arrive(&empty[s]);
        }
      }
    }
    const bool ok = mbar_wait(accum, 0, abort_flag);
    tc_fence_after();
    if (ok && ktiles > 0) {
      const int row = 32 * q + lane;
      const int64_t grow = (int64_t)tile0 + row;
      float* dst = out + (MODE == 1 ? (int64_t)blockIdx.y * split_stride : 0) + grow * ldo;
      for (int c0 = 0; c0 < nmma; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
        if (grow < out_rows) {
#pragma unroll
          for (int j = 0; j < 16; j += 4) {
            const int c = c0 + j;
            if (c + 3 < ncols) {
              *reinterpret_cast<float4*>(dst + c) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            } else {
              for (int t = 0; t < 4; ++t)
                if (c + t < ncols) dst[c + t] = v[j + t];
            }
          }
        }
      }
    }
    if (NORM) {
      double s = (double)sq.hi + (double)sq.lo;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) s_red[q] = s;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (NORM && tid == 0) gnorm_part[blockIdx.x] = s_red[0] + s_red[1] + s_red[2] + s_red[3];
  if (tid == 0 && s_abort) set_status(st_dev, -7, 200 + MODE, blockIdx.x);
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, (uint32_t)tmem_cols);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

// Looked up once; a function-local static initialised by a call is thread-safe (concurrent
// first calls from the batched workers wait for the one initialisation).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
    return nullptr;
  }();
  return fn;
}

// 2-D tensor map of FP32 (eb = 4) or BF16 (eb = 2) elements, dims {inner, outer}, row
// stride in elements, box {128 bytes of elements, box_outer}, 128 B swizzle (or none).
bool make_map(CUtensorMap* m, const void* ptr, uint64_t inner, uint64_t outer, uint64_t ld, uint32_t box_outer,
              bool swizzle = true, int eb = 4) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {ld * (uint64_t)eb};
  cuuint32_t box[2] = {(cuuint32_t)(128 / eb), box_outer};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, eb == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                  const_cast<void*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int pick_stages(int nmma, int mode, bool split, int eb = 4) {
  const int stage = (int)StageLayout(mode, split, nmma, eb).bytes;
  // two CTAs per SM when the pipeline fits in ~110 KB, else one deeper pipeline
  int s = (110 * 1024 - 2048) / stage;
  if (s < 3) s = std::min(6, (210 * 1024 - 2048) / stage);
  return std::max(2, std::min(s, 8));
}

// The deepest pipeline that still lets `per_sm` CTAs share an SM.
int stages_for(int nmma, int mode, bool split, int per_sm, int eb = 4) {
  const int stage = (int)StageLayout(mode, split, nmma, eb).bytes;
  const int budget = (per_sm >= 2 ? 110 : 210) * 1024 - 2048;
  return std::max(2, std::min(budget / stage, 8));
}

int sm_count() {
  static const int n = []() {
    int dev = 0, c = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        c <= 0) {
      cudaGetLastError();
      c = 152;
    }
    return c;
  }();
  return n;
}

// CTAs of a launch with this dynamic shared memory that fit on one SM (228 KB per SM,
// about 1 KB reserved per CTA).
int ctas_per_sm(size_t smem) { return std::max(1, (int)((228 * 1024) / (smem + 1024))); }

size_t smem_bytes(int nmma, int stages, int mode, bool split, int eb = 4) {
  return 1024 + (size_t)stages * StageLayout(mode, split, nmma, eb).bytes + (3 * (size_t)stages + 1) * 8 + 16;
}

int tmem_cols_for(int nmma) {
  int c = 32;
  while (c < nmma) c <<= 1;
  return c;
}

}  // namespace

bool tc_available(int device) {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, device) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return p.major == 10 && p.minor == 3 && encode_fn() != nullptr;
}

bool tc_shape_ok(const void* G, int64_t ldg, int l, int eb) {
  return ((uintptr_t)G % 16 == 0) && ((ldg * eb) % 16 == 0) && l >= 1 && l <= 256;
}

int tc_gx_ctas(int64_t M) { return (int)cdiv(M, TC_BM); }

template <int MODE, bool NORM, bool SPLIT, int EB = 4>
void launch_tc(dim3 grid, size_t smem, cudaStream_t st, const CUtensorMap& ma, const CUtensorMap& mb, float* out,
               int64_t ldo, int64_t out_rows, int ncols, int nmma, int64_t kdim, int64_t rps, int64_t split_stride,
               int stages, double* gnorm_part, DevStatus* st_dev, const CUtensorMap* mb2 = nullptr) {
  // a fixed cap (pipelines are sized to stay below it): concurrent launches must not lower it
  cudaFuncSetAttribute(tc_gemm_kernel<MODE, NORM, SPLIT, EB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       220 * 1024);
  tc_gemm_kernel<MODE, NORM, SPLIT, EB><<<grid, 192, smem, st>>>(ma, mb, mb2 ? *mb2 : mb, out, ldo, out_rows, ncols,
                                                                 nmma, tmem_cols_for(nmma), kdim, rps, split_stride,
                                                                 stages, gnorm_part, st_dev);
}

cudaError_t tc_gemm_gx(int prec, const float* G, int64_t ldg, int64_t M, int64_t n, const float* Xt, int64_t ldx,
                       int l, float* Y, int64_t ldy, double* gnorm_part, DevStatus* st_dev, cudaStream_t st) {
  const bool split = prec == 3;  // GSVD_RAND_TF32X3
  const int nmma = (int)round_up(l, 16);
  CUtensorMap ma, mb;
  if (!make_map(&ma, G, (uint64_t)n, (uint64_t)M, (uint64_t)ldg, TC_BM)) return cudaErrorInvalidValue;
  if (!make_map(&mb, Xt, (uint64_t)n, (uint64_t)nmma, (uint64_t)ldx, (uint32_t)nmma)) return cudaErrorInvalidValue;
  // one wave: when the row tiles exceed the SMs at full depth, a shallower pipeline lets
  // two CTAs share an SM so that every tile runs at once
  const int64_t tiles = cdiv(M, TC_BM);
  int stages = pick_stages(nmma, 0, split);
  if (tiles > (int64_t)sm_count() * ctas_per_sm(smem_bytes(nmma, stages, 0, split)))
    stages = stages_for(nmma, 0, split, 2);
  const size_t smem = smem_bytes(nmma, stages, 0, split);
  const dim3 grid((unsigned)tiles);
  if (gnorm_part) {
    if (split)
      launch_tc<0, true, true>(grid, smem, st, ma, mb, Y, ldy, M, l, nmma, n, 0, 0, stages, gnorm_part, st_dev);
    else
      launch_tc<0, true, false>(grid, smem, st, ma, mb, Y, ldy, M, l, nmma, n, 0, 0, stages, gnorm_part, st_dev);
  } else {
    if (split)
      launch_tc<0, false, true>(grid, smem, st, ma, mb, Y, ldy, M, l, nmma, n, 0, 0, stages, nullptr, st_dev);
    else
      launch_tc<0, false, false>(grid, smem, st, ma, mb, Y, ldy, M, l, nmma, n, 0, 0, stages, nullptr, st_dev);
  }
  return launched();
}

// Row splits of G^T Q: as many as fill the resident CTA slots in one wave.
int tc_gtq_splits(int64_t M, int64_t n, int prec) {
  const int64_t ctiles = cdiv(n, TC_BM);
  const int nmma = 64;  // slots are sized for the widest basis on the fast path
  const bool split = prec == 3;
  const int per_sm = ctas_per_sm(smem_bytes(nmma, pick_stages(nmma, 1, split), 1, split));
  int64_t s = std::max<int64_t>(1, (int64_t)sm_count() * per_sm / ctiles);
  s = std::min<int64_t>(s, std::max<int64_t>(1, cdiv(M, 4 * TC_BK)));
  return (int)s;
}

int64_t tc_gtq_part_elems(int64_t M, int64_t n, int l) {
  const int s = std::max(std::max(tc_gtq_splits(M, n, 1), tc_gtq_splits(M, n, 3)),
                         std::max(tc_gtq_splits_bf16(M, n, false), tc_gtq_splits_bf16(M, n, true)));
  return (int64_t)s * n * round_up(l, 4);
}

cudaError_t tc_gemm_gtq(int prec, const float* G, int64_t ldg, int64_t M, int64_t n, const float* Qt, int64_t ldq,
                        int l, float* part, int64_t lp, int* splits_out, int64_t max_part_elems, DevStatus* st_dev,
                        cudaStream_t st) {
  const int nmma = (int)round_up(l, 16);
  int splits = tc_gtq_splits(M, n, prec);
  while (splits > 1 && (int64_t)splits * n * lp > max_part_elems) --splits;
  // split boundaries on stage (32-row) boundaries so that no tile crosses into the next split
  const int64_t rps = round_up(cdiv(M, splits), TC_BK);
  splits = (int)cdiv(M, rps);
  *splits_out = splits;
  CUtensorMap ma, mb;
  // G tiles are staged unswizzled (32 rows x 32 columns per box) and transposed in shared memory
  if (!make_map(&ma, G, (uint64_t)n, (uint64_t)M, (uint64_t)ldg, TC_BK, false)) return cudaErrorInvalidValue;
  if (!make_map(&mb, Qt, (uint64_t)M, (uint64_t)nmma, (uint64_t)ldq, (uint32_t)nmma)) return cudaErrorInvalidValue;
  const bool split = prec == 3;  // GSVD_RAND_TF32X3
  const int stages = pick_stages(nmma, 1, split);
  const size_t smem = smem_bytes(nmma, stages, 1, split);
  const dim3 grid((unsigned)cdiv(n, TC_BM), (unsigned)splits);
  if (split)
    launch_tc<1, false, true>(grid, smem, st, ma, mb, part, lp, n, l, nmma, M, rps, n * lp, stages, nullptr, st_dev);
  else
    launch_tc<1, false, false>(grid, smem, st, ma, mb, part, lp, n, l, nmma, M, rps, n * lp, stages, nullptr, st_dev);
  return launched();
}

// ---------------------------------------------------------------------------
// BF16 data (kind::f16).  G is BF16 row-major; the B operands come K-major as
// BF16 hi (+ lo) halves written by split_bf16.
// ---------------------------------------------------------------------------
cudaError_t tc_gemm_gx_bf16(const void* G, int64_t ldg, int64_t M, int64_t n, const void* Xh, const void* Xl,
                            int64_t ldx, int l, float* Y, int64_t ldy, double* gnorm_part, DevStatus* st_dev,
                            cudaStream_t st) {
  const bool split = Xl != nullptr;
  const int nmma = (int)round_up(l, 16);
  CUtensorMap ma, mb, mb2;
  if (!make_map(&ma, G, (uint64_t)n, (uint64_t)M, (uint64_t)ldg, TC_BM, true, 2)) return cudaErrorInvalidValue;
  if (!make_map(&mb, Xh, (uint64_t)n, (uint64_t)nmma, (uint64_t)ldx, (uint32_t)nmma, true, 2))
    return cudaErrorInvalidValue;
  if (split && !make_map(&mb2, Xl, (uint64_t)n, (uint64_t)nmma, (uint64_t)ldx, (uint32_t)nmma, true, 2))
    return cudaErrorInvalidValue;
  const int64_t tiles = cdiv(M, TC_BM);
  int stages = pick_stages(nmma, 0, split, 2);
  if (tiles > (int64_t)sm_count() * ctas_per_sm(smem_bytes(nmma, stages, 0, split, 2)))
    stages = stages_for(nmma, 0, split, 2, 2);
  const size_t smem = smem_bytes(nmma, stages, 0, split, 2);
  const dim3 grid((unsigned)tiles);
  const CUtensorMap* m2 = split ? &mb2 : nullptr;
  if (gnorm_part) {
    if (split)
      launch_tc<0, true, true, 2>(grid, smem, st, ma, mb, Y, ldy, M, l, nmma, n, 0, 0, stages, gnorm_part, st_dev, m2);
    else
      launch_tc<0, true, false, 2>(grid, smem, st, ma, mb, Y, ldy, M, l, nmma, n, 0, 0, stages, gnorm_part, st_dev);
  } else {
    if (split)
      launch_tc<0, false, true, 2>(grid, smem, st, ma, mb, Y, ldy, M, l, nmma, n, 0, 0, stages, nullptr, st_dev, m2);
    else
      launch_tc<0, false, false, 2>(grid, smem, st, ma, mb, Y, ldy, M, l, nmma, n, 0, 0, stages, nullptr, st_dev);
  }
  return launched();
}

int tc_gtq_splits_bf16(int64_t M, int64_t n, bool split) {
  const int64_t ctiles = cdiv(n, TC_BM);
  const int nmma = 64;
  const int per_sm = ctas_per_sm(smem_bytes(nmma, pick_stages(nmma, 1, split, 2), 1, split, 2));
  int64_t s = std::max<int64_t>(1, (int64_t)sm_count() * per_sm / ctiles);
  s = std::min<int64_t>(s, std::max<int64_t>(1, cdiv(M, 2 * 64)));
  return (int)s;
}

cudaError_t tc_gemm_gtq_bf16(const void* G, int64_t ldg, int64_t M, int64_t n, const void* Qh, const void* Ql,
                             int64_t ldq, int l, float* part, int64_t lp, int* splits_out, int64_t max_part_elems,
                             DevStatus* st_dev, cudaStream_t st) {
  const bool split = Ql != nullptr;
  const int nmma = (int)round_up(l, 16);
  int splits = tc_gtq_splits_bf16(M, n, split);
  while (splits > 1 && (int64_t)splits * n * lp > max_part_elems) --splits;
  // split boundaries on stage (64-row) boundaries so that no tile crosses into the next split
  const int64_t rps = round_up(cdiv(M, splits), 64);
  splits = (int)cdiv(M, rps);
  *splits_out = splits;
  CUtensorMap ma, mb, mb2;
  // G tiles are staged unswizzled (64 rows x 64 columns per box) and transposed in shared memory
  if (!make_map(&ma, G, (uint64_t)n, (uint64_t)M, (uint64_t)ldg, 64, false, 2)) return cudaErrorInvalidValue;
  if (!make_map(&mb, Qh, (uint64_t)M, (uint64_t)nmma, (uint64_t)ldq, (uint32_t)nmma, true, 2))
    return cudaErrorInvalidValue;
  if (split && !make_map(&mb2, Ql, (uint64_t)M, (uint64_t)nmma, (uint64_t)ldq, (uint32_t)nmma, true, 2))
    return cudaErrorInvalidValue;
  const int stages = pick_stages(nmma, 1, split, 2);
  const size_t smem = smem_bytes(nmma, stages, 1, split, 2);
  const dim3 grid((unsigned)cdiv(n, TC_BM), (unsigned)splits);
  if (split)
    launch_tc<1, false, true, 2>(grid, smem, st, ma, mb, part, lp, n, l, nmma, M, rps, n * lp, stages, nullptr,
                                 st_dev, &mb2);
  else
    launch_tc<1, false, false, 2>(grid, smem, st, ma, mb, part, lp, n, l, nmma, M, rps, n * lp, stages, nullptr,
                                  st_dev);
  return launched();
}


// ---------------------------------------------------------------------------
// Grouped persistent products: many independent problems (the sides of many
// pairs) in one launch.  The host writes one TcGroupProb per problem (with its
// own tensor maps) and a tile list into device memory; CTA b takes tiles
// b, b + grid, b + 2 grid, ... of the list (sorted longest first), so the
// roles below walk the same sequence and their pipeline counters agree.
//
// Warp roles (14 warps): 0 TMA, 1 MMA (one thread), 2-9 operand preparation,
// 10-13 accumulator drain.  The accumulator is double-buffered in tensor
// memory, so the drain of one tile overlaps the MMAs of the next.
//
// 3xTF32 (SPLIT): the A operand (the G tile, or its transpose for G^T Q) goes
// to the MMA from tensor memory: the preparation warps read it from the staged
// tile and write A and A - tf32(A) into a tensor-memory ring (one 64-column
// stage per pipeline stage, after the two accumulators), so shared memory holds
// only the staged tile, B and B - tf32(B).  Shared-memory traffic per stage is
// then about 2/3 of what A and its low half in shared memory would need, and the
// G^T Q stage no longer holds the transposed copies.
// ---------------------------------------------------------------------------
namespace {

constexpr int TG_PREP_WARPS = 8;                   // operand preparation warps
constexpr int TG_THREADS = 32 * (6 + TG_PREP_WARPS);  // + TMA, MMA and four drain warps
constexpr int TG_TA_STAGE_COLS = 64;              // A-ring stage: 32 columns A, then 32 A_lo

// 3xTF32 tensor-memory plan: one CTA per SM takes all 512 columns (two accumulators in
// [0, 256), a 4-stage A ring in [256, 512)).  Two CTAs per SM take 256 columns each: two
// accumulators and the ring stages that fit after them (3 for bases up to 32 columns, 2 up
// to 64), or, for wider bases, a single accumulator (its drain then overlaps the other CTA's
// work, not the next tile's MMAs) and a 2-stage ring.
struct TaPlan {
  int cols, col0, stages, nacc;
};
__host__ __device__ inline TaPlan ta_plan(int acc_stride, int per_sm) {
  if (per_sm < 2) return TaPlan{512, 256, 2 * acc_stride <= 256 ? 4 : 0, 2};
  int nacc = 2, col0 = 2 * acc_stride;
  if (256 - col0 < 2 * TG_TA_STAGE_COLS) {
    nacc = 1;
    col0 = (acc_stride + TG_TA_STAGE_COLS - 1) / TG_TA_STAGE_COLS * TG_TA_STAGE_COLS;
  }
  const int st = col0 < 256 ? (256 - col0) / TG_TA_STAGE_COLS : 0;
  return TaPlan{256, col0, st, nacc};
}

// Shared-memory stage of the grouped kernel: with SPLIT, the staged A tile (16 KB), B and
// B_lo (each nmma x 128 bytes, 1024-aligned); otherwise the StageLayout of tc_gemm_kernel.
struct GroupLayout {
  uint32_t a, b, blo, ak, alo, bytes;
  __host__ __device__ GroupLayout(int mode, bool split, int nmma) {
    if (split) {
      const uint32_t nb = ((uint32_t)nmma * 128u + 1023u) & ~1023u;
      a = 0;
      ak = 0;
      alo = 0;
      b = TC_A_BYTES;
      blo = b + nb;
      bytes = blo + nb;
    } else {
      const StageLayout L(mode, false, nmma, 4);
      a = L.a;
      b = L.b;
      ak = L.ak;
      alo = L.alo;
      blo = L.blo;
      bytes = L.bytes;
    }
  }
};

template <int MODE, bool NORM, bool SPLIT>
__global__ __launch_bounds__(TG_THREADS, 2) void tc_group_kernel(const TcGroupProb* __restrict__ probs,
                                                              const int2* __restrict__ tiles, int ntiles,
                                                              int nmma_max, int acc_stride, int tmem_cols,
                                                              int ta_col0, int nacc, int stages,
                                                              DevStatus* st_glob, const int* ntiles_dev) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // a filtered launch: the tile list holds the active problems' tiles, their count in memory
  // written before the launch (every role reads the same count, so the pipelines agree)
  if (ntiles_dev) ntiles = *ntiles_dev;
  constexpr int BKE = 32;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const GroupLayout L(MODE, SPLIT, nmma_max);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + (size_t)stages * L.bytes);
  uint64_t* empty = full + stages;
  uint64_t* tfull = empty + stages;   // operands prepared (preparation warps)
  uint64_t* tmfull = tfull + stages;  // [2] accumulator ready (MMA commit)
  uint64_t* tmempty = tmfull + 2;     // [2] accumulator drained (4 drain warps)
  uint64_t* fin = tmempty + 2;        // every MMA of this CTA complete
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  constexpr bool TRANSPOSE = MODE == 1;
  constexpr bool PREP = TRANSPOSE || SPLIT;
  constexpr bool EPI_STAGE = PREP || NORM;
  __shared__ int s_abort;

  if (tid == 0) {
    s_abort = 0;
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      // with PREP the MMA waits for the preparation, so its commit alone releases a stage
      mbar_init(&empty[s], (EPI_STAGE && !PREP) ? 1 + TG_PREP_WARPS : 1);
      mbar_init(&tfull[s], TG_PREP_WARPS);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tmfull[a], 1);
      mbar_init(&tmempty[a], 4);
    }
    mbar_init(fin, 1);
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, (uint32_t)tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int* abort_flag = &s_abort;

  // the k range of a tile
  auto krange = [&](const TcGroupProb& P, int t, int64_t& kb, int64_t& ke, int& t0) {
    if (MODE == 0) {
      kb = 0;
      ke = P.kdim;
      t0 = t * TC_BM;
    } else {
      const int z = t / P.tiles_x;
      t0 = (t - z * P.tiles_x) * TC_BM;
      kb = (int64_t)z * P.rows_per_split;
      ke = min(P.kdim, kb + P.rows_per_split);
    }
  };

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      uint32_t it = 0, issued = 0;
      for (int ti = blockIdx.x; ti < ntiles && !*abort_flag; ti += gridDim.x) {
        const int2 tr = tiles[ti];
        const TcGroupProb& P = probs[tr.x];
        int64_t kb, ke;
        int t0;
        krange(P, tr.y, kb, ke, t0);
        const int kt_n = (int)((ke - kb + BKE - 1) / BKE);
        const uint32_t b_bytes = (uint32_t)P.nmma * 128u;
        for (int kt = 0; kt < kt_n; ++kt, ++it) {
          const int s = (int)(it % (uint32_t)stages);
          const uint32_t ph = (it / (uint32_t)stages) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag)) break;
          ++issued;
          uint8_t* st = base + (size_t)s * L.bytes;
          const bool blo = SPLIT && MODE == 0 && P.has_blo;
          mbar_expect_tx(&full[s], (uint32_t)TC_A_BYTES + b_bytes * (blo ? 2u : 1u));
          const int k0 = (int)(kb + (int64_t)kt * BKE);
          if (MODE == 0) {
            tma_load_2d(st + L.a, &P.mapA, &full[s], k0, t0);
          } else {
#pragma unroll
            for (int q = 0; q < 128 / BKE; ++q) tma_load_2d(st + L.a + q * (BKE * 128), &P.mapA, &full[s], t0 + BKE * q, k0);
          }
          tma_load_2d(st + L.b, &P.mapB, &full[s], k0, 0);
          if (blo) tma_load_2d(st + L.blo, &P.mapBlo, &full[s], k0, 0);
        }
      }
      if (*abort_flag) {
        // wait (bounded) until the copies this thread issued have landed
        const uint32_t first = issued > (uint32_t)stages ? issued - (uint32_t)stages : 0u;
        for (uint32_t j = first; j < issued; ++j) {
          volatile int none = 0;
          mbar_wait(&full[j % (uint32_t)stages], (j / (uint32_t)stages) & 1u, &none);
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      uint32_t it = 0;
      int j = 0;
      for (int ti = blockIdx.x; ti < ntiles && !*abort_flag; ti += gridDim.x, ++j) {
        const int2 tr = tiles[ti];
        const TcGroupProb& P = probs[tr.x];
        int64_t kb, ke;
        int t0;
        krange(P, tr.y, kb, ke, t0);
        const int kt_n = (int)((ke - kb + BKE - 1) / BKE);
        // accumulator acc, its use jj: waits for the drain of its previous use
        const int acc = nacc == 2 ? (j & 1) : 0, jj = nacc == 2 ? (j >> 1) : j;
        if (j >= nacc && !mbar_wait(&tmempty[acc], (uint32_t)(jj + 1) & 1u, abort_flag)) break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(acc * acc_stride);
        const uint32_t idesc = idesc_tf32(TC_BM, (uint32_t)P.nmma, 0u, 0u);
        bool ok = true;
        for (int kt = 0; kt < kt_n; ++kt, ++it) {
          const int s = (int)(it % (uint32_t)stages);
          const uint32_t ph = (it / (uint32_t)stages) & 1u;
          if (!mbar_wait(PREP ? &tfull[s] : &full[s], ph, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_u32(base + (size_t)s * L.bytes);
          const uint32_t ta = tmem + (uint32_t)(ta_col0 + TG_TA_STAGE_COLS * s);  // 0-31 A, 32-63 A_lo
#pragma unroll
          for (int ks = 0; ks < 128 / TC_KSTEP_BYTES; ++ks) {
            const uint64_t bdesc = smem_desc(st + L.b + ks * TC_KSTEP_BYTES, 16, 1024);
            if (SPLIT) {
              const uint32_t ahi = ta + (uint32_t)(8 * ks), alo = ahi + 32u;
              mma_tf32_ta(d, ahi, bdesc, idesc, (kt > 0 || ks > 0) ? 1u : 0u);
              mma_tf32_ta(d, alo, bdesc, idesc, 1u);
              mma_tf32_ta(d, ahi, smem_desc(st + L.blo + ks * TC_KSTEP_BYTES, 16, 1024), idesc, 1u);
            } else {
              const uint64_t adesc = smem_desc(st + L.ak + ks * TC_KSTEP_BYTES, 16, 1024);
              mma_tf32(d, adesc, bdesc, idesc, (kt > 0 || ks > 0) ? 1u : 0u);
            }
          }
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        mma_commit(&tmfull[acc]);
      }
      // arrives once every MMA issued above has completed: none is in flight when the
      // tensor memory is freed
      mma_commit(fin);
      volatile int none = 0;
      mbar_wait(fin, 0, &none);
    }
  } else if (warp < 2 + TG_PREP_WARPS) {
    // ---------------- operand preparation (warps 2 .. 9) ----------------
    if (EPI_STAGE) {
      constexpr int PT = 32 * TG_PREP_WARPS;  // preparation threads
      const int et = tid - 64;                // 0 .. PT - 1
      const int q = warp - 2;                 // partial index of the fused norm
      const int sub = warp & 3;               // tensor-memory lane quarter of this warp
      const int half = (warp - 2) >> 2;       // which 16 of the stage's 32 K columns (SPLIT)
      const int arow = 32 * sub + lane;       // the A row (tensor-memory lane) this thread writes
      uint32_t it = 0;
      for (int ti = blockIdx.x; ti < ntiles && !*abort_flag; ti += gridDim.x) {
        const int2 tr = tiles[ti];
        const TcGroupProb& P = probs[tr.x];
        int64_t kb, ke;
        int t0;
        krange(P, tr.y, kb, ke, t0);
        const int kt_n = (int)((ke - kb + BKE - 1) / BKE);
        const uint32_t b_bytes = (uint32_t)P.nmma * 128u;
        SqAccF sq;
        bool ok = true;
        for (int kt = 0; kt < kt_n; ++kt, ++it) {
          const int s = (int)(it % (uint32_t)stages);
          const uint32_t ph = (it / (uint32_t)stages) & 1u;
          if (!mbar_wait(&full[s], ph, abort_flag)) {
            ok = false;
            break;
          }
          uint8_t* st = base + (size_t)s * L.bytes;
          if (SPLIT) {
            // the A-ring stage was last read by the MMAs whose commit released this stage
            tc_fence_after();
            // this thread's row of A, K columns 16 half .. 16 half + 15, into the A ring
            float v[16], lo[16];
            if (MODE == 0) {
              // staged K-major with the 128-byte swizzle: 16-byte chunk c of row r at c ^ (r & 7)
              const uint8_t* row = st + L.a + arow * 128;
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                const float4 x = *reinterpret_cast<const float4*>(row + (((4 * half + c) ^ (arow & 7)) << 4));
                v[4 * c + 0] = x.x;
                v[4 * c + 1] = x.y;
                v[4 * c + 2] = x.z;
                v[4 * c + 3] = x.w;
              }
            } else {
              // staged G[k][c] (unswizzled 32 x 32 boxes): A row c = column c of G
              const float* stg = reinterpret_cast<const float*>(st + L.a + (arow >> 5) * (TC_BK * 128)) + (arow & 31);
#pragma unroll
              for (int k = 0; k < 16; ++k) v[k] = stg[(16 * half + k) * 32];
            }
            if (NORM) {  // the 16 squares of this thread's row slice, then one compensated add
              float s16 = 0.f;
#pragma unroll
              for (int k = 0; k < 16; ++k) s16 = fmaf(v[k], v[k], s16);
              sq.add_sum(s16);
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) lo[k] = tf32_lo(v[k]);
            const uint32_t ta =
                tmem + ((uint32_t)(32 * sub) << 16) + (uint32_t)(ta_col0 + TG_TA_STAGE_COLS * s + 16 * half);
            tmem_st16(ta, v);
            tmem_st16(ta + 32u, lo);
            // B_lo in shared memory (unless the TMA brought it with B)
            if (!(MODE == 0 && P.has_blo)) {
              const float4* b4 = reinterpret_cast<const float4*>(st + L.b);
              float4* blo4 = reinterpret_cast<float4*>(st + L.blo);
              for (int i = et; i < (int)(b_bytes / 16); i += PT) {
                float4 x = b4[i];
                blo4[i] = make_float4(tf32_lo(x.x), tf32_lo(x.y), tf32_lo(x.z), tf32_lo(x.w));
              }
            }
            tmem_wait_st();
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_fence_before();
          } else if (TRANSPOSE) {
            // row c of the K-major tile (see tc_gemm_kernel), its 16-byte chunks shared by the
            // PT / 128 threads with the same c
            const int c = et & 127, part = et >> 7;
            constexpr int NCH = 8 / (PT / 128);
            const float* stg = reinterpret_cast<const float*>(st + L.a + (c >> 5) * (TC_BK * 128)) + (c & 31);
            uint8_t* row = st + L.ak + c * 128;
#pragma unroll
            for (int ch = part * NCH; ch < (part + 1) * NCH; ++ch) {
              float4 x = make_float4(stg[(4 * ch + 0) * 32], stg[(4 * ch + 1) * 32], stg[(4 * ch + 2) * 32],
                                     stg[(4 * ch + 3) * 32]);
              *reinterpret_cast<float4*>(row + ((ch ^ (c & 7)) << 4)) = x;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          } else if (NORM) {
            const float4* a4 = reinterpret_cast<const float4*>(st + L.a);
            for (int i = et; i < TC_A_BYTES / 16; i += PT) {
              float4 x = a4[i];
              sq.add_sum(fmaf(x.w, x.w, fmaf(x.z, x.z, fmaf(x.y, x.y, x.x * x.x))));
            }
          }
          __syncwarp();
          if (lane == 0) {
            if (PREP) mbar_arrive(&tfull[s]);
            else mbar_arrive(&empty[s]);
          }
        }
        if (!ok) break;
        if (NORM && MODE == 0) {
          // one partial per (row tile, prep warp): summed in order by the residual step
          double x = (double)sq.hi + (double)sq.lo;
          for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
          if (lane == 0 && P.gnorm_part) P.gnorm_part[TG_PREP_WARPS * tr.y + q] = x;
        }
      }
    }
  } else {
    // ---------------- accumulator drain (the last four warps) ----------------
    const int q = warp & 3;  // TMEM sub-partition: lanes 32q .. 32q + 31
    int j = 0;
    for (int ti = blockIdx.x; ti < ntiles && !*abort_flag; ti += gridDim.x, ++j) {
      const int2 tr = tiles[ti];
      const TcGroupProb& P = probs[tr.x];
      int64_t kb, ke;
      int t0;
      krange(P, tr.y, kb, ke, t0);
      const int acc = nacc == 2 ? (j & 1) : 0, jj = nacc == 2 ? (j >> 1) : j;
      if (!mbar_wait(&tmfull[acc], (uint32_t)jj & 1u, abort_flag)) break;
      tc_fence_after();
      const int row = 32 * q + lane;
      const int64_t grow = (int64_t)t0 + row;
      const int z = MODE == 1 ? tr.y / P.tiles_x : 0;
      float* dst = P.out + (int64_t)z * P.split_stride + grow * P.ldo;
      const uint32_t src = tmem + (uint32_t)(acc * acc_stride) + ((uint32_t)(32 * q) << 16);
      for (int c0 = 0; c0 < P.nmma; c0 += 16) {
        float v[16];
        tmem_ld16(src + (uint32_t)c0, v);
        if (MODE == 0 && P.transpose_out) {
          // column-major store: the 32 lanes write 32 consecutive rows of each column
          if (grow < P.out_rows) {
            float* dc = P.out + grow;
#pragma unroll
            for (int jj = 0; jj < 16; ++jj)
              if (c0 + jj < P.ncols) dc[(int64_t)(c0 + jj) * P.ldo] = v[jj];
          }
        } else if (grow < P.out_rows) {
#pragma unroll
          for (int jj = 0; jj < 16; jj += 4) {
            const int c = c0 + jj;
            if (c + 3 < P.ncols) {
              *reinterpret_cast<float4*>(dst + c) = make_float4(v[jj], v[jj + 1], v[jj + 2], v[jj + 3]);
            } else {
              for (int t = 0; t < 4; ++t)
                if (c + t < P.ncols) dst[c + t] = v[jj + t];
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tmempty[acc]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && s_abort) set_status(st_glob, -7, 210 + MODE, blockIdx.x);
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, (uint32_t)tmem_cols);
  }
}

size_t group_smem_bytes(int mode, bool split, int nmma_max, int stages) {
  return 1024 + (size_t)stages * GroupLayout(mode, split, nmma_max).bytes + (3 * (size_t)stages + 5) * 8 + 16;
}

}  // namespace

int tc_group_norm_parts() { return TG_PREP_WARPS; }

int64_t tc_group_tiles(int mode, const TcGroupSpec* specs, int nprob) {
  int64_t t = 0;
  for (int i = 0; i < nprob; ++i) {
    const TcGroupSpec& s = specs[i];
    if (mode == 0)
      t += cdiv(s.M, TC_BM);
    else
      t += cdiv(s.n, TC_BM) * (int64_t)s.splits;
  }
  return t;
}

size_t tc_group_table_bytes(int nprob, int64_t ntiles) {
  return round_up((int64_t)nprob * (int64_t)sizeof(TcGroupProb), 256) + round_up(ntiles * (int64_t)sizeof(int2), 256);
}

bool tc_group_build(int mode, const TcGroupSpec* specs, int nprob, void* host, int* nmma_max) {
  TcGroupProb* P = static_cast<TcGroupProb*>(host);
  int2* T = reinterpret_cast<int2*>(static_cast<unsigned char*>(host) +
                                    round_up((int64_t)nprob * (int64_t)sizeof(TcGroupProb), 256));
  std::vector<std::pair<int64_t, int2>> order;
  int nm = 16;
  for (int i = 0; i < nprob; ++i) {
    const TcGroupSpec& s = specs[i];
    TcGroupProb& p = P[i];
    memset(&p, 0, sizeof(p));
    const int nmma = (int)round_up(s.l, 16);
    if (s.l < 1 || nmma > 256 || !tc_shape_ok(s.G, s.ldg, s.l)) return false;
    nm = std::max(nm, nmma);
    p.out = s.out;
    p.ldo = s.ldo;
    p.ncols = s.l;
    p.nmma = nmma;
    p.gnorm_part = s.gnorm_part;
    p.transpose_out = s.transpose_out;
    p.stop = s.stop;
    if (mode == 0) {
      if (!make_map(&p.mapA, s.G, (uint64_t)s.n, (uint64_t)s.M, (uint64_t)s.ldg, TC_BM)) return false;
      if (!make_map(&p.mapB, s.Bt, (uint64_t)s.n, (uint64_t)nmma, (uint64_t)s.ldb, (uint32_t)nmma)) return false;
      if (s.Bt_lo) {
        if (!make_map(&p.mapBlo, s.Bt_lo, (uint64_t)s.n, (uint64_t)nmma, (uint64_t)s.ldb, (uint32_t)nmma)) return false;
        p.has_blo = 1;
      }
      p.out_rows = s.M;
      p.kdim = s.n;
      p.tiles_x = (int)cdiv(s.M, TC_BM);
      const int64_t kt = cdiv(s.n, TC_BK);
      for (int t = 0; t < p.tiles_x; ++t) order.push_back({kt, make_int2(i, t)});
    } else {
      if (!make_map(&p.mapA, s.G, (uint64_t)s.n, (uint64_t)s.M, (uint64_t)s.ldg, TC_BK, false)) return false;
      if (!make_map(&p.mapB, s.Bt, (uint64_t)s.M, (uint64_t)nmma, (uint64_t)s.ldb, (uint32_t)nmma)) return false;
      if (s.splits < 1 || s.rps % TC_BK != 0 || cdiv(s.M, s.rps) != s.splits) return false;
      p.out_rows = s.n;
      p.kdim = s.M;
      p.rows_per_split = s.rps;
      p.split_stride = s.split_stride;
      p.tiles_x = (int)cdiv(s.n, TC_BM);
      for (int z = 0; z < s.splits; ++z) {
        const int64_t rows = std::min(s.M, (int64_t)(z + 1) * s.rps) - (int64_t)z * s.rps;
        for (int t = 0; t < p.tiles_x; ++t) order.push_back({cdiv(rows, TC_BK), make_int2(i, t + z * p.tiles_x)});
      }
    }
  }
  // longest tiles first: the strided assignment then balances the CTAs
  std::stable_sort(order.begin(), order.end(),
                   [](const std::pair<int64_t, int2>& a, const std::pair<int64_t, int2>& b) { return a.first > b.first; });
  for (size_t t = 0; t < order.size(); ++t) T[t] = order[t].second;
  *nmma_max = nm;
  return true;
}

int tc_group_max_stages(int mode, int prec, int nmma_max, int per_sm) {
  const bool split = prec == 3;
  const int budget = (per_sm >= 2 ? 110 : 214) * 1024 - 2048;
  const int stage = (int)GroupLayout(mode, split, nmma_max).bytes;
  // 3xTF32: each pipeline stage owns a stage of the A ring in tensor memory
  const int cap = split ? ta_plan((int)round_up(nmma_max, 32), per_sm).stages : 8;
  return std::min(budget / stage, cap);
}

namespace {
// Stable compaction of the tile list to the problems whose stop word is zero (one CTA: a
// block-wide scan per 1024 tiles).  out: the kept tiles, then (at out_count) their number.
__global__ __launch_bounds__(1024) void tc_group_filter_kernel(const TcGroupProb* __restrict__ probs,
                                                               const int2* __restrict__ tiles, int ntiles,
                                                               int2* __restrict__ out, int* __restrict__ out_count) {
  __shared__ int s_warp[32];
  __shared__ int s_base;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_base = 0;
  __syncthreads();
  for (int t0 = 0; t0 < ntiles; t0 += 1024) {
    const int t = t0 + tid;
    int2 tr = make_int2(0, 0);
    int keep = 0;
    if (t < ntiles) {
      tr = tiles[t];
      const int* sw = probs[tr.x].stop;
      keep = (sw == nullptr || *sw == 0) ? 1 : 0;
    }
    // inclusive scan of keep over the block
    int v = keep;
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane == 31) s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
      int w = s_warp[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += u;
      }
      s_warp[lane] = w;
    }
    __syncthreads();
    const int before = (warp > 0 ? s_warp[warp - 1] : 0) + v - keep;
    if (keep) out[s_base + before] = tr;
    __syncthreads();
    if (tid == 1023) s_base += s_warp[31];
    __syncthreads();
  }
  if (tid == 0) *out_count = s_base;
}
}  // namespace

size_t tc_group_filter_bytes(int64_t ntiles) { return round_up(ntiles * (int64_t)sizeof(int2), 256) + 256; }

cudaError_t tc_group_filter(const void* dev_table, int nprob, int64_t ntiles, void* dev_filtered, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  const TcGroupProb* probs = static_cast<const TcGroupProb*>(dev_table);
  const int2* tiles = reinterpret_cast<const int2*>(static_cast<const unsigned char*>(dev_table) +
                                                    round_up((int64_t)nprob * (int64_t)sizeof(TcGroupProb), 256));
  int2* out = static_cast<int2*>(dev_filtered);
  int* cnt = reinterpret_cast<int*>(static_cast<unsigned char*>(dev_filtered) +
                                    round_up(ntiles * (int64_t)sizeof(int2), 256));
  tc_group_filter_kernel<<<1, 1024, 0, st>>>(probs, tiles, (int)ntiles, out, cnt);
  return launched();
}

cudaError_t tc_group_launch(int mode, int prec, bool norm, const void* dev_table, int nprob, int64_t ntiles,
                            int nmma_max, int stages, int per_sm, DevStatus* st_dev, cudaStream_t st,
                            const void* dev_filtered) {
  if (ntiles <= 0) return cudaSuccess;
  const bool split = prec == 3;
  const int acc_stride = (int)round_up(nmma_max, 32);
  // 3xTF32: the two accumulators, then the A ring (ta_plan)
  const TaPlan tp = ta_plan(acc_stride, per_sm);
  const int tmem_cols = split ? tp.cols : tmem_cols_for(2 * acc_stride);
  const int ta_col0 = split ? tp.col0 : 0, nacc = split ? tp.nacc : 2;
  if (nacc * acc_stride > (split ? ta_col0 : 512) || (per_sm >= 2 && tmem_cols > 256)) return cudaErrorInvalidValue;
  if (stages < 2 || stages > tc_group_max_stages(mode, prec, nmma_max, per_sm)) return cudaErrorInvalidValue;
  const TcGroupProb* probs = static_cast<const TcGroupProb*>(dev_table);
  const int2* tiles = reinterpret_cast<const int2*>(static_cast<const unsigned char*>(dev_table) +
                                                    round_up((int64_t)nprob * (int64_t)sizeof(TcGroupProb), 256));
  const int* ntiles_dev = nullptr;
  if (dev_filtered) {
    tiles = static_cast<const int2*>(dev_filtered);
    ntiles_dev = reinterpret_cast<const int*>(static_cast<const unsigned char*>(dev_filtered) +
                                              round_up(ntiles * (int64_t)sizeof(int2), 256));
  }
  // the dynamic shared memory also caps the CTAs per SM at per_sm (TMEM columns stay within 512)
  size_t smem = group_smem_bytes(mode, split, nmma_max, stages);
  const size_t floor_smem = per_sm >= 2 ? 80 * 1024 : 120 * 1024;
  smem = std::max(smem, floor_smem);
  const int grid = (int)std::min<int64_t>(ntiles, (int64_t)sm_count() * std::max(1, per_sm));
#define GSVDR_TG(M_, N_, S_)                                                                                  \
  do {                                                                                                       \
    cudaFuncSetAttribute(tc_group_kernel<M_, N_, S_>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024); \
    tc_group_kernel<M_, N_, S_><<<grid, TG_THREADS, smem, st>>>(probs, tiles, (int)ntiles, nmma_max, acc_stride, \
                                                                tmem_cols, ta_col0, nacc, stages, st_dev,    \
                                                                ntiles_dev);                                 \
  } while (0)
  if (mode == 0) {
    if (norm && split) GSVDR_TG(0, true, true);
    else if (norm) GSVDR_TG(0, true, false);
    else if (split) GSVDR_TG(0, false, true);
    else GSVDR_TG(0, false, false);
  } else {
    if (split) GSVDR_TG(1, false, true);
    else GSVDR_TG(1, false, false);
  }
#undef GSVDR_TG
  return launched();
}

}  // namespace gsvdr
