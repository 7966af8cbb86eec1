// The learned (k, q) proposal: probe features of a pair and the 64-128-128-37
// classifier that reads them (training and inference kernels).
//
// Features (per side, from the 64-column probe Y = G Omega_p): log10 of every other
// eigenvalue of Y^T Y (the 1st, 3rd, ..., 63rd largest) over 64 ||G||_F^2, clipped to
// [-12, 1]: 32 per side.  The 64 x 64 eigenvalues come from a Householder
// tridiagonalisation and Sturm bisection in FP64, one CTA per Gram.
//
// Network: x^ = (x - mean) / std; h1 = relu(x^ W1 + b1); h2 = relu(h1 W2 + b2);
// z = h2 W3 + b3 (W row-major in x out).  Loss: softmax cross-entropy of the
// k head (z[0:32]) plus that of the q head (z[32:37]), batch means.  Adam
// (Kingma & Ba 2015) with bias correction.  Every sum runs in a fixed order
// (no atomics), so training is reproducible bit for bit.
#include <cuda_bf16.h>

#include "gsvd_rand.h"
#include "kernels.h"

namespace gsvdr {

namespace {

constexpr int MI = 64, MH = 128, MK = 32, MQ = 5, MO = MK + MQ;
constexpr int O_W1 = 0, O_B1 = O_W1 + MI * MH, O_W2 = O_B1 + MH, O_B2 = O_W2 + MH * MH, O_W3 = O_B2 + MH,
              O_B3 = O_W3 + MH * MO, NPAR = O_B3 + MO;
constexpr float FEAT_LO = -12.f, FEAT_HI = 1.f;

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// ---------------------------------------------------------------- features
// Eigenvalues of the symmetric 64 x 64 Gram W = Y^T Y (row-major, FP64) by one CTA of 64
// threads: Householder tridiagonalisation (Golub & Van Loan, Alg. 8.3.1; thread i owns row i of
// the trailing block), then Sturm-count bisection, thread j finding the j-th smallest eigenvalue.
// W is positive semi-definite, so the bisection runs on a geometric scale between a floor of
// 1e-14 of the Gershgorin bound (below it the feature is clipped anyway) and that bound: 30
// geometric halvings leave a ratio below 1 + 3e-8 between the bracket's ends.
constexpr int PN = GSVD_RAND_MLP_PROBE;  // probe columns (the Gram's order)
static_assert(PN == 64, "one CTA of 64 threads per probe Gram");

__device__ __forceinline__ double block_sum64(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();  // red free (previous readers done)
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  return red[0] + red[1];
}

// Thread j returns the j-th smallest eigenvalue (or a value at or below `floor` when it lies there).
__device__ double eig64_block(double* A, double* vs, double* ws, double* d, double* e2, double* red, double* floor_out) {
  const int i = threadIdx.x;
  for (int k = 0; k < PN - 2; ++k) {
    // reflector of column k below the diagonal: v = x - alpha e_{k+1}, H = I - v v^T / (sg - x0 alpha)
    const double x = i > k ? A[i * PN + k] : 0.0;
    const double sg = block_sum64(x * x, red);
    const double x0 = A[(k + 1) * PN + k];
    const double sig = sqrt(sg);
    const double alpha = x0 >= 0.0 ? -sig : sig;
    const double den = sg - x0 * alpha;
    const bool refl = sig > 0.0 && den > 0.0;
    const double v = (i == k + 1) ? x0 - alpha : x;  // zero at and above row k
    vs[i] = v;
    __syncthreads();
    // p = A v / den (row i), then w = p - (p^T v / (2 den)) v
    double p = 0.0;
    if (refl && i > k)
      for (int j = k + 1; j < PN; ++j) p = fma(A[i * PN + j], vs[j], p);
    p = refl ? p / den : 0.0;
    const double pv = block_sum64(p * v, red);
    const double w = p - (refl ? 0.5 * pv / den : 0.0) * v;
    ws[i] = w;
    __syncthreads();
    if (refl && i > k)  // A <- A - v w^T - w v^T on the trailing block
      for (int j = k + 1; j < PN; ++j) A[i * PN + j] -= v * ws[j] + w * vs[j];
    if (i == 0) {
      d[k] = A[k * PN + k];
      e2[k] = refl ? alpha * alpha : x0 * x0;
    }
    __syncthreads();
  }
  if (i == 0) {
    d[PN - 2] = A[(PN - 2) * PN + PN - 2];
    d[PN - 1] = A[(PN - 1) * PN + PN - 1];
    e2[PN - 2] = A[(PN - 1) * PN + PN - 2] * A[(PN - 1) * PN + PN - 2];
  }
  __syncthreads();
  double hi = 0.0;
  for (int r = 0; r < PN; ++r) {
    const double rad = (r > 0 ? sqrt(e2[r - 1]) : 0.0) + (r < PN - 1 ? sqrt(e2[r]) : 0.0);
    hi = fmax(hi, d[r] + rad);
  }
  const double fl = 1e-14 * hi;
  *floor_out = fl;
  const double pivmin = fmax(1e-300, 1e-30 * hi);
  auto count_below = [&](double xv) {  // eigenvalues of T below xv (Sturm sequence of T - xv I)
    int cnt = 0;
    double q = 1.0;
    for (int r = 0; r < PN; ++r) {
      q = (d[r] - xv) - (r > 0 ? e2[r - 1] / q : 0.0);
      if (fabs(q) < pivmin) q = -pivmin;
      cnt += q < 0.0;
    }
    return cnt;
  };
  if (!(hi > 0.0) || count_below(fl) > i) return 0.0;  // at or below the floor
  double lo = fl, up = hi;
  for (int it = 0; it < 30; ++it) {
    const double mid = sqrt(lo * up);
    if (count_below(mid) > i)
      up = mid;
    else
      lo = mid;
  }
  return sqrt(lo * up);
}

}  // namespace

// One CTA of 64 threads per side: W = Y^T Y (PN x PN, upper triangle valid) and gpart, the
// sketch CTAs' partial sums of G^2 (gcount entries); feats[t] (t = 0 .. 31) = log10 of the
// (2t + 1)-th largest eigenvalue over PN ||G||_F^2, clipped.  The FP64 arithmetic takes a good
// fraction of a millisecond on one SM (FP64 runs at 1/64 of the FP32 rate), so a group's sides
// run as one launch, a CTA each (probe_features_b_kernel).
__device__ void probe_features_body(const double* __restrict__ W, const double* __restrict__ gpart, int gcount,
                                    float* __restrict__ feats) {
  __shared__ double A[PN * PN];
  __shared__ double vs[PN], ws[PN], D[PN], E2[PN], red[2];
  __shared__ double s_g2;
  const int tid = threadIdx.x;
  if (tid < 32) {
    double g = 0.0;
    for (int i = tid; i < gcount; i += 32) g += gpart[i];
    for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
    if (tid == 0) s_g2 = g;
  }
  for (int e = tid; e < PN * PN; e += PN) {
    const int i = e / PN, j = e % PN;
    A[e] = W[(i <= j ? i : j) * PN + (i <= j ? j : i)];  // the Gram sums hold the upper triangle
  }
  __syncthreads();
  double fl;
  const double lam = eig64_block(A, vs, ws, D, E2, red, &fl);
  const int pos = PN - 1 - tid;  // thread j holds the j-th smallest: descending position PN - 1 - j
  if ((pos & 1) == 0) {
    const double den = (double)PN * s_g2;
    const double r = lam > fl && den > 0.0 ? lam / den : 0.0;
    float f = r > 0.0 ? (float)log10(r) : FEAT_LO;
    f = fminf(fmaxf(f, FEAT_LO), FEAT_HI);
    feats[pos >> 1] = f;
  }
}

__global__ __launch_bounds__(PN) void probe_features_kernel(const double* __restrict__ W,
                                                             const double* __restrict__ gpart, int gcount,
                                                             float* __restrict__ feats) {
  probe_features_body(W, gpart, gcount, feats);
}
__global__ __launch_bounds__(PN) void probe_features_b_kernel(const ProbeFeatB* __restrict__ tab) {
  const ProbeFeatB& t = tab[blockIdx.x];
  probe_features_body(t.W, t.gpart, t.gcount, t.feats);
}

cudaError_t launch_probe_features(const double* W, const double* gpart, int gcount, float* feats, cudaStream_t st) {
  probe_features_kernel<<<1, PN, 0, st>>>(W, gpart, gcount, feats);
  return launched();
}
cudaError_t launch_probe_features_b(const ProbeFeatB* tab, int nprob, cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  probe_features_b_kernel<<<nprob, PN, 0, st>>>(tab);
  return launched();
}

// ---------------------------------------------------------------- network
// Dense layer out[b][j] = act(sum_i in[b][i] W[i][j] + bias[j]) for a block of 16
// rows; in is either the raw features (normalised here) or a previous layer.
// rows: optional gather indices into `in` (training minibatches).
template <bool NORM_IN, bool RELU, bool BF16W>
__global__ __launch_bounds__(128) void dense_kernel(const float* __restrict__ in, const int* __restrict__ rows,
                                                    int B, int din, int dout, const float* __restrict__ W,
                                                    const float* __restrict__ bias, const float* __restrict__ norm,
                                                    float* __restrict__ pre, float* __restrict__ out) {
  __shared__ float xs[16][MH + 1];
  const int b0 = blockIdx.x * 16, tid = threadIdx.x;
  for (int e = tid; e < 16 * din; e += 128) {
    const int r = e / din, i = e % din;
    float v = 0.f;
    if (b0 + r < B) {
      const int src = rows ? rows[b0 + r] : b0 + r;
      v = in[(int64_t)src * din + i];
      if (NORM_IN) v = (v - norm[i]) / norm[MI + i];
    }
    xs[r][i] = v;
  }
  __syncthreads();
  for (int j = tid; j < dout; j += 128) {
    float acc[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) acc[r] = 0.f;
    for (int i = 0; i < din; ++i) {
      float w = W[i * dout + j];
      if (BF16W) w = bf16_round(w);
#pragma unroll
      for (int r = 0; r < 16; ++r) acc[r] = fmaf(xs[r][i], w, acc[r]);
    }
    const float bj = bias[j];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      if (b0 + r >= B) break;
      const float a = acc[r] + bj;
      if (pre) pre[(int64_t)(b0 + r) * dout + j] = a;
      out[(int64_t)(b0 + r) * dout + j] = RELU ? fmaxf(a, 0.f) : a;
    }
  }
}

// Softmax cross-entropy of both heads: dz = (softmax - onehot) / B, per-row loss.
__global__ void softmax_ce_kernel(const float* __restrict__ z, const int* __restrict__ yk,
                                  const int* __restrict__ yq, const int* __restrict__ rows, int B,
                                  float* __restrict__ dz, float* __restrict__ row_loss) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const int src = rows ? rows[b] : b;
  const float* zb = z + (int64_t)b * MO;
  float* db = dz + (int64_t)b * MO;
  float loss = 0.f;
  for (int head = 0; head < 2; ++head) {
    const int o = head ? MK : 0, c = head ? MQ : MK, y = head ? yq[src] : yk[src];
    float mx = zb[o];
    for (int j = 1; j < c; ++j) mx = fmaxf(mx, zb[o + j]);
    float s = 0.f;
    for (int j = 0; j < c; ++j) s += expf(zb[o + j] - mx);
    const float ls = logf(s);
    loss += -(zb[o + y] - mx - ls);
    for (int j = 0; j < c; ++j) db[o + j] = (expf(zb[o + j] - mx - ls) - (j == y ? 1.f : 0.f)) / (float)B;
  }
  row_loss[b] = loss;
}

// dW[i][j] = sum_b h[b][i] dz[b][j] and db[j] = sum_b dz[b][j] (thread per (i, j)).
__global__ void dense_wgrad_kernel(const float* __restrict__ h, int B, int din, int dout,
                                   const float* __restrict__ dz, float* __restrict__ dW, float* __restrict__ db) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < din * dout) {
    const int i = e / dout, j = e % dout;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s = fmaf(h[(int64_t)b * din + i], dz[(int64_t)b * dout + j], s);
    dW[e] = s;
  }
  if (e < dout) {
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += dz[(int64_t)b * dout + e];
    db[e] = s;
  }
}

// dh[b][i] = (sum_j dz[b][j] W[i][j]) * (pre[b][i] > 0).
__global__ void dense_xgrad_kernel(const float* __restrict__ dz, int B, int din, int dout,
                                   const float* __restrict__ W, const float* __restrict__ pre,
                                   float* __restrict__ dh) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * din) return;
  const int b = e / din, i = e % din;
  float s = 0.f;
  for (int j = 0; j < dout; ++j) s = fmaf(dz[(int64_t)b * dout + j], W[i * dout + j], s);
  dh[e] = pre[e] > 0.f ? s : 0.f;
}

__global__ void sum_rows_kernel(const float* __restrict__ v, int B, float* __restrict__ out) {
  __shared__ float red[256];
  float s = 0.f;
  for (int i = threadIdx.x; i < B; i += 256) s += v[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] / (float)B;
}

__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ---------------------------------------------------------------- host side

int64_t mlp_param_count() { return NPAR; }
int64_t mlp_scratch_floats(int B) {
  // x^ (B x 64), a1, h1, a2, h2 (B x 128 each), z, dz (B x 37), d2, d1 (B x 128), row loss (B)
  return (int64_t)B * (MI + 4 * MH + 2 * MO + 2 * MH + 1) + 64;
}

namespace {
struct MlpScratch {
  float *x, *a1, *h1, *a2, *h2, *z, *dz, *d2, *d1, *rl;
  MlpScratch(float* s, int B) {
    x = s;
    a1 = x + (int64_t)B * MI;
    h1 = a1 + (int64_t)B * MH;
    a2 = h1 + (int64_t)B * MH;
    h2 = a2 + (int64_t)B * MH;
    z = h2 + (int64_t)B * MH;
    dz = z + (int64_t)B * MO;
    d2 = dz + (int64_t)B * MO;
    d1 = d2 + (int64_t)B * MH;
    rl = d1 + (int64_t)B * MH;
  }
};

__global__ void gather_norm_kernel(const float* __restrict__ X, const int* __restrict__ rows, int B,
                                   const float* __restrict__ norm, float* __restrict__ xh) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * MI) return;
  const int b = e / MI, i = e % MI;
  const int src = rows ? rows[b] : b;
  xh[e] = (X[(int64_t)src * MI + i] - norm[i]) / norm[MI + i];
}

cudaError_t forward_into(const float* P, const float* norm, const float* X, const int* rows, int B, bool bf16,
                         MlpScratch& s, float* logits, cudaStream_t st) {
  const unsigned g16 = (unsigned)cdiv(B, 16);
  if (bf16) {
    dense_kernel<true, true, true><<<g16, 128, 0, st>>>(X, rows, B, MI, MH, P + O_W1, P + O_B1, norm, s.a1, s.h1);
    dense_kernel<false, true, true><<<g16, 128, 0, st>>>(s.h1, nullptr, B, MH, MH, P + O_W2, P + O_B2, nullptr,
                                                          s.a2, s.h2);
    dense_kernel<false, false, true><<<g16, 128, 0, st>>>(s.h2, nullptr, B, MH, MO, P + O_W3, P + O_B3, nullptr,
                                                           nullptr, logits);
  } else {
    dense_kernel<true, true, false><<<g16, 128, 0, st>>>(X, rows, B, MI, MH, P + O_W1, P + O_B1, norm, s.a1, s.h1);
    dense_kernel<false, true, false><<<g16, 128, 0, st>>>(s.h1, nullptr, B, MH, MH, P + O_W2, P + O_B2, nullptr,
                                                           s.a2, s.h2);
    dense_kernel<false, false, false><<<g16, 128, 0, st>>>(s.h2, nullptr, B, MH, MO, P + O_W3, P + O_B3, nullptr,
                                                            nullptr, logits);
  }
  return launched();
}
}  // namespace

cudaError_t mlp_forward(const float* P, const float* norm, const float* X, int B, int bf16, float* logits,
                        float* scratch, cudaStream_t st) {
  MlpScratch s(scratch, B);
  return forward_into(P, norm, X, nullptr, B, bf16 != 0, s, logits, st);
}

cudaError_t mlp_loss_grad(const float* P, const float* norm, const float* X, const int* yk, const int* yq,
                          const int* rows, int B, float* grad, float* loss, float* scratch, cudaStream_t st) {
  MlpScratch s(scratch, B);
  cudaError_t e = forward_into(P, norm, X, rows, B, false, s, s.z, st);
  if (e != cudaSuccess) return e;
  gather_norm_kernel<<<(unsigned)cdiv((int64_t)B * MI, 256), 256, 0, st>>>(X, rows, B, norm, s.x);
  softmax_ce_kernel<<<(unsigned)cdiv(B, 128), 128, 0, st>>>(s.z, yk, yq, rows, B, s.dz, s.rl);
  sum_rows_kernel<<<1, 256, 0, st>>>(s.rl, B, loss);
  dense_wgrad_kernel<<<(unsigned)cdiv(MH * MO, 256), 256, 0, st>>>(s.h2, B, MH, MO, s.dz, grad + O_W3, grad + O_B3);
  dense_xgrad_kernel<<<(unsigned)cdiv((int64_t)B * MH, 256), 256, 0, st>>>(s.dz, B, MH, MO, P + O_W3, s.a2, s.d2);
  dense_wgrad_kernel<<<(unsigned)cdiv(MH * MH, 256), 256, 0, st>>>(s.h1, B, MH, MH, s.d2, grad + O_W2, grad + O_B2);
  dense_xgrad_kernel<<<(unsigned)cdiv((int64_t)B * MH, 256), 256, 0, st>>>(s.d2, B, MH, MH, P + O_W2, s.a1, s.d1);
  dense_wgrad_kernel<<<(unsigned)cdiv(MI * MH, 256), 256, 0, st>>>(s.x, B, MI, MH, s.d1, grad + O_W1, grad + O_B1);
  return launched();
}

cudaError_t mlp_adam(float* P, float* m, float* v, const float* grad, int t, float lr, float b1, float b2, float eps,
                     cudaStream_t st) {
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  adam_kernel<<<(unsigned)cdiv(NPAR, 256), 256, 0, st>>>(P, m, v, grad, NPAR, lr, b1, b2, eps, c1, c2);
  return launched();
}

}  // namespace gsvdr

namespace gsvdr {
namespace {
// The plan of each row of logits (B x (KCLS + QCLS)): kb = the smallest k bucket whose cumulative
// softmax probability reaches `quantile`, q = the most probable q class (first on ties), then
// k = min(KBUCKET (kb + 1), kcap[i], lmax[i] - oversample[i]), at least 1.  A thread per row.
__global__ void mlp_plan_kernel(const float* __restrict__ z, int B, float quantile, const int* __restrict__ kcap,
                                const int* __restrict__ lmax, const int* __restrict__ os, int* __restrict__ plan) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  const float* zi = z + (int64_t)i * (GSVD_RAND_MLP_KCLS + GSVD_RAND_MLP_QCLS);
  double mx = zi[0];
  for (int j = 1; j < GSVD_RAND_MLP_KCLS; ++j) mx = fmax(mx, (double)zi[j]);
  double tot = 0.0;
  for (int j = 0; j < GSVD_RAND_MLP_KCLS; ++j) tot += exp((double)zi[j] - mx);
  int kb = 0;
  double cum = 0.0;
  for (kb = 0; kb < GSVD_RAND_MLP_KCLS - 1; ++kb) {
    cum += exp((double)zi[kb] - mx) / tot;
    if (cum >= (double)quantile) break;
  }
  int q = 0;
  for (int j = 1; j < GSVD_RAND_MLP_QCLS; ++j)
    if (zi[GSVD_RAND_MLP_KCLS + q] < zi[GSVD_RAND_MLP_KCLS + j]) q = j;
  int k = GSVD_RAND_MLP_KBUCKET * (kb + 1);
  if (kcap) k = min(k, kcap[i]);
  if (lmax) k = min(k, lmax[i] - (os ? os[i] : 0));
  plan[3 * i] = max(k, 1);
  plan[3 * i + 1] = q;
  plan[3 * i + 2] = kb;
}
}  // namespace

cudaError_t launch_mlp_plan(const float* logits, int B, float quantile, const int* kcap, const int* lmax,
                            const int* os, int* plan, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  mlp_plan_kernel<<<(B + 127) / 128, 128, 0, st>>>(logits, B, quantile, kcap, lmax, os, plan);
  return launched();
}
}  // namespace gsvdr
