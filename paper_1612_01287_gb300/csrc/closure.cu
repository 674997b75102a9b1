// closure.cu -- learned closure of a low-order velocity set (an addition to
// the paper's method): a per-cell MLP, trained on data the method generates
// with a high-order velocity set, corrects the low-order populations after
// every RK3 step.
//
//  * restriction R: high-order populations -> low-order ones, per radial
//    node, through the Legendre moments m < Q_lo (exact for m <= 2, so the
//    moments of Eq. macro_jk are preserved);
//  * features of cell s, over n_s = sum_v f_{v,s}: the low-order populations
//    of cell s, f_{s+1} - f_s and f_s - f_{s-1}; then log10(tau);
//  * MLP D -> H -> H -> O with SiLU after the hidden layers, BF16 weights
//    (FP32 master copy for Adam), FP32 biases and accumulation, behind a
//    fixed input/output normalisation fitted to the training data;
//  * correction delta = n_s * out_sd * y, minus its component along the collision
//    invariants (1, p, p xi) in the quadrature-weighted sense, so the cell's
//    N^t, T^tt and T^tz are unchanged; the result is scaled down where it
//    would take more than half of a positive population (a positivity
//    limiter that keeps the conservation).
//
// Training: one CTA holds up to 128 samples; each thread runs forward and
// backward for its sample out of shared memory, then the CTA reduces the
// weight gradients over its samples into a per-CTA partial; a second kernel
// sums the partials in a fixed order (deterministic), a third applies Adam.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>

#include "../../include/rslb.h"
#include "host_common.h"

namespace rslb {
namespace {

constexpr int kMaxD = 128;
constexpr int kMaxO = 32;
constexpr int kSmemLimit = 232448;
constexpr float kLimitTheta = 0.5f;  // positivity limiter of the correction

struct MlpShape {
  int D, H, O;
  int oW1, ob1, oW2, ob2, oW3, ob3, P;
};

MlpShape make_shape(int D, int H, int O) {
  MlpShape s;
  s.D = D;
  s.H = H;
  s.O = O;
  s.oW1 = 0;
  s.ob1 = H * D;
  s.oW2 = s.ob1 + H;
  s.ob2 = s.oW2 + H * H;
  s.oW3 = s.ob2 + H;
  s.ob3 = s.oW3 + O * H;
  s.P = s.ob3 + O;
  return s;
}

// Shared-memory weight block: W1T [D][H], W2 [H][H], W3 [O][H] (BF16 values
// widened to FP32), b1 [H], b2 [H], b3 [O], then the fixed normalisation
// mu [D], inv_sd [D], out_sd [O] (the network sees (x - mu) * inv_sd, its
// output is scaled by out_sd).
__host__ __device__ inline int wblock_floats(const MlpShape& s) {
  return s.D * s.H + s.H * s.H + s.O * s.H + 2 * s.H + s.O + 2 * s.D + s.O;
}

__host__ __device__ inline int norm_offset(const MlpShape& s) {
  return s.D * s.H + s.H * s.H + s.O * s.H + 2 * s.H + s.O;
}

__device__ inline void load_weights(const MlpShape& s, const __nv_bfloat16* __restrict__ wb,
                                    const float* __restrict__ theta,
                                    const float* __restrict__ nrm, float* sw) {
  for (int e = threadIdx.x; e < 2 * s.D + s.O; e += blockDim.x) sw[norm_offset(s) + e] = nrm[e];
  float* W1T = sw;
  float* W2 = W1T + s.D * s.H;
  float* W3 = W2 + s.H * s.H;
  float* b1 = W3 + s.O * s.H;
  float* b2 = b1 + s.H;
  float* b3 = b2 + s.H;
  for (int e = threadIdx.x; e < s.H * s.D; e += blockDim.x) {
    const int h = e / s.D, d = e - h * s.D;
    W1T[d * s.H + h] = __bfloat162float(wb[s.oW1 + e]);
  }
  for (int e = threadIdx.x; e < s.H * s.H; e += blockDim.x) W2[e] = __bfloat162float(wb[s.oW2 + e]);
  for (int e = threadIdx.x; e < s.O * s.H; e += blockDim.x) W3[e] = __bfloat162float(wb[s.oW3 + e]);
  for (int e = threadIdx.x; e < s.H; e += blockDim.x) {
    b1[e] = theta[s.ob1 + e];
    b2[e] = theta[s.ob2 + e];
  }
  for (int e = threadIdx.x; e < s.O; e += blockDim.x) b3[e] = theta[s.ob3 + e];
}

__device__ __forceinline__ float silu_f(float a, float* ds) {
  const float sg = 1.f / (1.f + __expf(-a));
  *ds = sg * (1.f + a * (1.f - sg));
  return a * sg;
}

// Forward of one sample.  x(d) supplies input d; h1 and h2 (registers) receive
// the hidden activations; with GRAD, s1[h] = silu'(a1_h) and s2[h] =
// silu'(a2_h) are stored (shared memory); y(o) is handed to put_y.
template <int H, bool GRAD, typename XF, typename YF>
__device__ __forceinline__ void mlp_forward(const MlpShape& s, const float* __restrict__ sw,
                                            XF x, float (&h1)[H], float (&h2)[H], float* s1,
                                            float* s2, YF put_y) {
  const float* W1T = sw;
  const float* W2 = W1T + s.D * H;
  const float* W3 = W2 + H * H;
  const float* b1 = W3 + s.O * H;
  const float* b2 = b1 + H;
  const float* b3 = b2 + H;
#pragma unroll
  for (int h = 0; h < H; ++h) h1[h] = b1[h];
  for (int d = 0; d < s.D; ++d) {
    const float xd = x(d);
    const float4* w = reinterpret_cast<const float4*>(W1T + d * H);
#pragma unroll
    for (int q = 0; q < H / 4; ++q) {
      const float4 wv = w[q];
      h1[4 * q] = fmaf(wv.x, xd, h1[4 * q]);
      h1[4 * q + 1] = fmaf(wv.y, xd, h1[4 * q + 1]);
      h1[4 * q + 2] = fmaf(wv.z, xd, h1[4 * q + 2]);
      h1[4 * q + 3] = fmaf(wv.w, xd, h1[4 * q + 3]);
    }
  }
#pragma unroll
  for (int h = 0; h < H; ++h) {
    float ds;
    h1[h] = silu_f(h1[h], &ds);
    if (GRAD) s1[h] = ds;
  }
#pragma unroll
  for (int h = 0; h < H; ++h) {
    const float4* w = reinterpret_cast<const float4*>(W2 + h * H);
    float acc = b2[h];
#pragma unroll
    for (int q = 0; q < H / 4; ++q) {
      const float4 wv = w[q];
      acc = fmaf(wv.x, h1[4 * q], acc);
      acc = fmaf(wv.y, h1[4 * q + 1], acc);
      acc = fmaf(wv.z, h1[4 * q + 2], acc);
      acc = fmaf(wv.w, h1[4 * q + 3], acc);
    }
    float ds;
    h2[h] = silu_f(acc, &ds);
    if (GRAD) s2[h] = ds;
  }
  for (int o = 0; o < s.O; ++o) {
    const float4* w = reinterpret_cast<const float4*>(W3 + o * H);
    float acc = b3[o];
#pragma unroll
    for (int q = 0; q < H / 4; ++q) {
      const float4 wv = w[q];
      acc = fmaf(wv.x, h2[4 * q], acc);
      acc = fmaf(wv.y, h2[4 * q + 1], acc);
      acc = fmaf(wv.z, h2[4 * q + 2], acc);
      acc = fmaf(wv.w, h2[4 * q + 3], acc);
    }
    put_y(o, acc);
  }
}

// ---------------------------------------------------------------------------
// Training: forward + backward of NS samples per CTA, per-CTA partial gradient
// ---------------------------------------------------------------------------
// Sample row in shared memory (pitch odd): [x (D) | h1 (H) | ga1 (H) | h2 (H) |
// ga2 (H) | gy (O)].
template <int H>
__global__ void __launch_bounds__(128) mlp_train_kernel(MlpShape s, const float* __restrict__ theta,
                                                        const __nv_bfloat16* __restrict__ wb,
                                                        const float* __restrict__ nrm,
                                                        const float* __restrict__ X,
                                                        const float* __restrict__ T,
                                                        const int* __restrict__ perm, int n0,
                                                        int nb, float inv_norm, int pitch,
                                                        float* part, double* lossp) {
  extern __shared__ __align__(16) float smem_f[];
  float* sw = smem_f;
  float* act = sw + ((wblock_floats(s) + 3) & ~3);
  __shared__ double red[128];
  const int NS = blockDim.x;
  const int tid = threadIdx.x;
  const int base = blockIdx.x * NS;
  const int cnt = min(NS, nb - base);
  load_weights(s, wb, theta, nrm, sw);
  __syncthreads();
  const float* mu = sw + norm_offset(s);
  const float* isd = mu + s.D;
  const float* osd = isd + s.D;
  // stage the normalised inputs of the CTA's samples (coalesced)
  for (int e = tid; e < NS * s.D; e += NS) {
    const int r = e / s.D, c = e - r * s.D;
    float v = 0.f;
    if (r < cnt) {
      const int n = n0 + base + r;
      const int src = perm ? perm[n] : n;
      v = (X[(size_t)src * s.D + c] - mu[c]) * isd[c];
    }
    act[r * pitch + c] = v;
  }
  __syncthreads();
  float* row = act + tid * pitch;
  float* rh1 = row + s.D;
  float* rg1 = rh1 + H;
  float* rh2 = rg1 + H;
  float* rg2 = rh2 + H;
  float* rgy = rg2 + H;
  double sq = 0.0;
  if (tid < cnt) {
    const int n = n0 + base + tid;
    const int src = perm ? perm[n] : n;
    const float* t = T + (size_t)src * s.O;
    float h1[H], h2[H];
    // silu'(a1) and silu'(a2) go to the ga1 and ga2 slots, overwritten below
    mlp_forward<H, true>(s, sw, [&](int d) { return row[d]; }, h1, h2, rg1, rg2,
                         [&](int o, float y) {
                           const float r = y - t[o] / osd[o];
                           sq += (double)r * r;
                           rgy[o] = 2.f * r * inv_norm;
                         });
#pragma unroll
    for (int i = 0; i < H; ++i) {
      rh1[i] = h1[i];
      rh2[i] = h2[i];
    }
    // backward through layer 3: gh2 = W3^T gy, ga2 = gh2 * silu'(a2)
    const float* W3 = sw + s.D * H + H * H;
    const float* W2 = sw + s.D * H;
    float g[H];
#pragma unroll
    for (int i = 0; i < H; ++i) g[i] = 0.f;
    for (int o = 0; o < s.O; ++o) {
      const float go = rgy[o];
      const float4* w = reinterpret_cast<const float4*>(W3 + o * H);
#pragma unroll
      for (int q = 0; q < H / 4; ++q) {
        const float4 wv = w[q];
        g[4 * q] = fmaf(wv.x, go, g[4 * q]);
        g[4 * q + 1] = fmaf(wv.y, go, g[4 * q + 1]);
        g[4 * q + 2] = fmaf(wv.z, go, g[4 * q + 2]);
        g[4 * q + 3] = fmaf(wv.w, go, g[4 * q + 3]);
      }
    }
#pragma unroll
    for (int i = 0; i < H; ++i) {
      g[i] *= rg2[i];
      rg2[i] = g[i];
    }
    // layer 2: gh1 = W2^T ga2, ga1 = gh1 * silu'(a1)
#pragma unroll
    for (int i = 0; i < H; ++i) h2[i] = 0.f;  // reused as gh1
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const float gh = g[h];
      const float4* w = reinterpret_cast<const float4*>(W2 + h * H);
#pragma unroll
      for (int q = 0; q < H / 4; ++q) {
        const float4 wv = w[q];
        h2[4 * q] = fmaf(wv.x, gh, h2[4 * q]);
        h2[4 * q + 1] = fmaf(wv.y, gh, h2[4 * q + 1]);
        h2[4 * q + 2] = fmaf(wv.z, gh, h2[4 * q + 2]);
        h2[4 * q + 3] = fmaf(wv.w, gh, h2[4 * q + 3]);
      }
    }
#pragma unroll
    for (int i = 0; i < H; ++i) rg1[i] = h2[i] * rg1[i];
  } else {
    for (int c = s.D; c < s.D + 4 * H + s.O; ++c) row[c] = 0.f;
  }
  red[tid] = sq;
  __syncthreads();
  // weight gradients summed over the CTA's samples
  float* out = part + (size_t)blockIdx.x * s.P;
  for (int e = tid; e < s.P; e += NS) {
    int ca, cb = -1;
    if (e < s.ob1) {
      const int h = e / s.D, d = e - h * s.D;
      ca = s.D + H + h;
      cb = d;
    } else if (e < s.oW2) {
      ca = s.D + H + (e - s.ob1);
    } else if (e < s.ob2) {
      const int k = e - s.oW2, h = k / H, i = k - h * H;
      ca = s.D + 3 * H + h;
      cb = s.D + i;
    } else if (e < s.oW3) {
      ca = s.D + 3 * H + (e - s.ob2);
    } else if (e < s.ob3) {
      const int k = e - s.oW3, o = k / H, i = k - o * H;
      ca = s.D + 4 * H + o;
      cb = s.D + 2 * H + i;
    } else {
      ca = s.D + 4 * H + (e - s.ob3);
    }
    float acc = 0.f;
    if (cb >= 0) {
      for (int n = 0; n < cnt; ++n) acc = fmaf(act[n * pitch + ca], act[n * pitch + cb], acc);
    } else {
      for (int n = 0; n < cnt; ++n) acc += act[n * pitch + ca];
    }
    out[e] = acc;
  }
  if (tid == 0) {
    double t = 0.0;
    for (int i = 0; i < NS; ++i) t += red[i];
    lossp[blockIdx.x] = t;
  }
}

__global__ void mlp_reduce_kernel(const float* __restrict__ part, int nblk, int P, float* grad,
                                  const double* __restrict__ lossp, double loss_scale,
                                  double* loss_acc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < P) {
    float acc = 0.f;
    for (int b = 0; b < nblk; ++b) acc += part[(size_t)b * P + e];
    grad[e] = acc;
  }
  if (e == 0) {
    double t = 0.0;
    for (int b = 0; b < nblk; ++b) t += lossp[b];
    *loss_acc += t * loss_scale;
  }
}

__global__ void mlp_adam_kernel(float* theta, const float* __restrict__ grad, float* m, float* v,
                                int P, float lr, float c1, float c2, MlpShape s,
                                __nv_bfloat16* wb) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= P) return;
  const float g = grad[e];
  const float mm = 0.9f * m[e] + 0.1f * g;
  const float vv = 0.999f * v[e] + 0.001f * g * g;
  m[e] = mm;
  v[e] = vv;
  const float th = theta[e] - lr * (mm * c1) / (sqrtf(vv * c2) + 1e-8f);
  theta[e] = th;
  wb[e] = __float2bfloat16_rn(th);
}

__global__ void mlp_round_kernel(const float* __restrict__ theta, int P, __nv_bfloat16* wb) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < P) wb[e] = __float2bfloat16_rn(theta[e]);
}

// Inference on given inputs: thread per sample, inputs staged through smem.
template <int H>
__global__ void __launch_bounds__(128) mlp_infer_kernel(MlpShape s, const float* __restrict__ theta,
                                                        const __nv_bfloat16* __restrict__ wb,
                                                        const float* __restrict__ nrm,
                                                        const float* __restrict__ X, int n,
                                                        int pitch, float* Y) {
  extern __shared__ __align__(16) float smem_f[];
  float* sw = smem_f;
  float* xs = sw + ((wblock_floats(s) + 3) & ~3);
  const int tid = threadIdx.x, NS = blockDim.x;
  const int base = blockIdx.x * NS;
  const int cnt = min(NS, n - base);
  load_weights(s, wb, theta, nrm, sw);
  __syncthreads();
  const float* mu = sw + norm_offset(s);
  const float* isd = mu + s.D;
  const float* osd = isd + s.D;
  for (int e = tid; e < NS * s.D; e += NS) {
    const int r = e / s.D, c = e - r * s.D;
    xs[r * pitch + c] = r < cnt ? (X[(size_t)(base + r) * s.D + c] - mu[c]) * isd[c] : 0.f;
  }
  __syncthreads();
  if (tid >= cnt) return;
  const float* row = xs + tid * pitch;
  float h1[H], h2[H];
  float* y = Y + (size_t)(base + tid) * s.O;
  mlp_forward<H, false>(s, sw, [&](int d) { return row[d]; }, h1, h2, nullptr, nullptr,
                        [&](int o, float v) { y[o] = v * osd[o]; });
}

// ---------------------------------------------------------------------------
// Closure kernels (FP32 populations, layout [v][ldz])
// ---------------------------------------------------------------------------
struct ClosureConsts {
  float phi[kMaxO][3];  // (1, p_k, p_k xi_j)
  float w[kMaxO];       // w_j w_k
  float ginv[9];        // (Phi^T W Phi)^{-1}
};

__device__ __forceinline__ void project_add(const ClosureConsts& cc, int V, const float* delta,
                                            float* out) {
  float b0 = 0.f, b1 = 0.f, b2 = 0.f;
  for (int v = 0; v < V; ++v) {
    b0 = fmaf(delta[v], cc.phi[v][0], b0);
    b1 = fmaf(delta[v], cc.phi[v][1], b1);
    b2 = fmaf(delta[v], cc.phi[v][2], b2);
  }
  const float c0 = cc.ginv[0] * b0 + cc.ginv[1] * b1 + cc.ginv[2] * b2;
  const float c1 = cc.ginv[3] * b0 + cc.ginv[4] * b1 + cc.ginv[5] * b2;
  const float c2 = cc.ginv[6] * b0 + cc.ginv[7] * b1 + cc.ginv[8] * b2;
  for (int v = 0; v < V; ++v)
    out[v] = delta[v] - cc.w[v] * (c0 * cc.phi[v][0] + c1 * cc.phi[v][1] + c2 * cc.phi[v][2]);
}

// f_out = f_in + projected correction, thread per cell.
template <int H>
__global__ void __launch_bounds__(128) closure_apply_kernel(MlpShape s, const float* __restrict__ theta,
                                                            const __nv_bfloat16* __restrict__ wb,
                                                            const float* __restrict__ nrm,
                                                            const float* __restrict__ fin,
                                                            float* fout, int Z, int ldz,
                                                            float logtau, ClosureConsts cc) {
  extern __shared__ __align__(16) float smem_f[];
  float* sw = smem_f;
  load_weights(s, wb, theta, nrm, sw);
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= Z) return;
  const int V = s.O;
  const int cl = c > 0 ? c - 1 : 0, cr = c < Z - 1 ? c + 1 : Z - 1;
  float n = 0.f;
  for (int v = 0; v < V; ++v) n += fin[(size_t)v * ldz + c];
  const float inv_n = 1.f / n;
  const float* mu = sw + norm_offset(s);
  const float* isd = mu + s.D;
  const float* osd = isd + s.D;
  // features: f_s, f_{s+1} - f_s, f_s - f_{s-1} (over n_s), log10 tau
  auto x = [&](int d) {
    float r;
    if (d >= 3 * V) {
      r = logtau;
    } else {
      const int blk = d / V, v = d - blk * V;
      const float fc = fin[(size_t)v * ldz + c];
      if (blk == 0) r = fc * inv_n;
      else if (blk == 1) r = (fin[(size_t)v * ldz + cr] - fc) * inv_n;
      else r = (fc - fin[(size_t)v * ldz + cl]) * inv_n;
    }
    return (r - mu[d]) * isd[d];
  };
  float h1[H], h2[H];
  float delta[kMaxO], corr[kMaxO];
  mlp_forward<H, false>(s, sw, x, h1, h2, nullptr, nullptr,
                        [&](int o, float y) { delta[o] = n * osd[o] * y; });
  project_add(cc, V, delta, corr);
  // positivity limiter: scale the (conserving) correction so that no
  // positive population loses more than kLimitTheta of itself
  float alpha = 1.f;
  for (int v = 0; v < V; ++v) {
    const float f = fin[(size_t)v * ldz + c];
    if (f > 0.f && corr[v] < 0.f) alpha = fminf(alpha, kLimitTheta * f / -corr[v]);
  }
  for (int v = 0; v < V; ++v)
    fout[(size_t)v * ldz + c] = fin[(size_t)v * ldz + c] + alpha * corr[v];
}

// Restriction, thread per cell: f_lo[k*Ql + i] = sum_j R[i][j] f_hi[k*Qh + j].
__global__ void restrict_kernel(const float* __restrict__ fh, int ldh, int Qh,
                                float* fl, int ldl, int Ql, int QL, const float* __restrict__ Rm,
                                int Z) {
  extern __shared__ float Rs[];
  for (int e = threadIdx.x; e < Ql * Qh; e += blockDim.x) Rs[e] = Rm[e];
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= Z) return;
  for (int k = 0; k < QL; ++k) {
    float acc[kMaxO];
    for (int i = 0; i < Ql; ++i) acc[i] = 0.f;
    for (int j = 0; j < Qh; ++j) {
      const float f = fh[(size_t)(k * Qh + j) * ldh + c];
      for (int i = 0; i < Ql; ++i) acc[i] = fmaf(Rs[i * Qh + j], f, acc[i]);
    }
    for (int i = 0; i < Ql; ++i) fl[(size_t)(k * Ql + i) * ldl + c] = acc[i];
  }
}

// Features of the low-order state (rows of X) and n_s: f_s, f_{s+1} - f_s,
// f_s - f_{s-1}, all over n_s, then log10 tau.
__global__ void features_kernel(const float* __restrict__ f, int Z, int ldz, int V, float logtau,
                                float* X, float* ns) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= Z) return;
  const int cl = c > 0 ? c - 1 : 0, cr = c < Z - 1 ? c + 1 : Z - 1;
  float n = 0.f;
  for (int v = 0; v < V; ++v) n += f[(size_t)v * ldz + c];
  ns[c] = n;
  const float inv = 1.f / n;
  float* row = X + (size_t)c * (3 * V + 1);
  for (int v = 0; v < V; ++v) {
    const float fc = f[(size_t)v * ldz + c];
    row[v] = fc * inv;
    row[V + v] = (f[(size_t)v * ldz + cr] - fc) * inv;
    row[2 * V + v] = (fc - f[(size_t)v * ldz + cl]) * inv;
  }
  row[3 * V] = logtau;
}

// Targets: T[s] = P(f_ref[s] - f_pred[s]) / n_s.
__global__ void target_kernel(const float* __restrict__ fref, const float* __restrict__ fpred,
                              const float* __restrict__ ns, int Z, int ldz, int V,
                              ClosureConsts cc, float* T) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= Z) return;
  float d[kMaxO], p[kMaxO];
  for (int v = 0; v < V; ++v) d[v] = fref[(size_t)v * ldz + c] - fpred[(size_t)v * ldz + c];
  project_add(cc, V, d, p);
  const float inv = 1.f / ns[c];
  for (int v = 0; v < V; ++v) T[(size_t)c * V + v] = p[v] * inv;
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
// Column statistics for the normalisation, one CTA per column (fixed-order
// tree reductions in FP64, two passes for the variance): columns of X give
// mu and 1/sd, columns of T give the root-mean-square (1 for constant or
// zero columns).
__global__ void fit_norm_kernel(const float* __restrict__ X, const float* __restrict__ T, int n,
                                int D, int O, float* nrm) {
  __shared__ double red[256];
  const int col = blockIdx.x, tid = threadIdx.x;
  const bool is_x = col < D;
  const float* src = is_x ? X + col : T + (col - D);
  const int stride = is_x ? D : O;
  auto reduce = [&](double v) {
    red[tid] = v;
    __syncthreads();
    for (int o = 128; o >= 1; o >>= 1) {
      if (tid < o) red[tid] += red[tid + o];
      __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
  };
  double a = 0.0;
  for (int r = tid; r < n; r += 256) a += (double)src[(size_t)r * stride];
  const double mean = reduce(a) / n;
  double b = 0.0;
  for (int r = tid; r < n; r += 256) {
    const double x = (double)src[(size_t)r * stride];
    const double d = is_x ? x - mean : x;
    b += d * d;
  }
  const double sd = sqrt(reduce(b) / n);
  if (tid == 0) {
    if (is_x) {
      nrm[col] = (float)mean;
      nrm[D + col] = sd > 0.0 ? (float)(1.0 / sd) : 1.f;
    } else {
      nrm[2 * D + (col - D)] = sd > 0.0 ? (float)sd : 1.f;
    }
  }
}

uint64_t splitmix(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double unit_normal(uint64_t& st) {
  const double u1 = ((splitmix(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  const double u2 = ((splitmix(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

int closure_consts(int Q, int QL, ClosureConsts* cc) {
  const int V = Q * QL;
  if (V > kMaxO) return RSLB_ERR_UNSUPPORTED;
  std::vector<double> xi(Q), w(Q), xk(QL), wk(QL);
  gauss_legendre_host(Q, xi.data(), w.data());
  gauss_laguerre2_host(QL, xk.data(), wk.data());
  double G[9] = {0};
  std::memset(cc, 0, sizeof(*cc));
  for (int k = 0; k < QL; ++k)
    for (int j = 0; j < Q; ++j) {
      const int v = k * Q + j;
      const double ph[3] = {1.0, xk[k], xk[k] * xi[j]};
      const double wv = w[j] * wk[k];
      for (int a = 0; a < 3; ++a) {
        cc->phi[v][a] = (float)ph[a];
        for (int b = 0; b < 3; ++b) G[3 * a + b] += ph[a] * wv * ph[b];
      }
      cc->w[v] = (float)wv;
    }
  // 3x3 inverse by cofactors
  const double det = G[0] * (G[4] * G[8] - G[5] * G[7]) - G[1] * (G[3] * G[8] - G[5] * G[6]) +
                     G[2] * (G[3] * G[7] - G[4] * G[6]);
  if (!(std::fabs(det) > 0.0)) return RSLB_ERR_ARG;
  const double inv[9] = {(G[4] * G[8] - G[5] * G[7]) / det, (G[2] * G[7] - G[1] * G[8]) / det,
                         (G[1] * G[5] - G[2] * G[4]) / det, (G[5] * G[6] - G[3] * G[8]) / det,
                         (G[0] * G[8] - G[2] * G[6]) / det, (G[2] * G[3] - G[0] * G[5]) / det,
                         (G[3] * G[7] - G[4] * G[6]) / det, (G[1] * G[6] - G[0] * G[7]) / det,
                         (G[0] * G[4] - G[1] * G[3]) / det};
  for (int i = 0; i < 9; ++i) cc->ginv[i] = (float)inv[i];
  return RSLB_OK;
}

}  // namespace
}  // namespace rslb

using namespace rslb;

struct rslb_mlp {
  MlpShape s;
  cudaStream_t stream;
  float* norm;  // mu [D] | inv_sd [D] | out_sd [O]
  float* theta;
  __nv_bfloat16* wb;
  float* grad;
  float* m;
  float* v;
  float* part;
  double* lossp;
  double* loss_acc;
  int* perm;
  int part_blocks;
  int perm_n;
  long long adam_t;
};

namespace {

int mlp_pitch(const MlpShape& s) {
  int p = s.D + 4 * s.H + s.O;
  return (p % 2) ? p : p + 1;
}

int train_ns(const MlpShape& s) {
  for (int ns = 128; ns >= 32; ns /= 2) {
    const size_t b = sizeof(float) * (size_t)(((wblock_floats(s) + 3) & ~3) + ns * mlp_pitch(s));
    if (b <= (size_t)kSmemLimit) return ns;
  }
  return 0;
}

size_t train_smem(const MlpShape& s, int ns) {
  return sizeof(float) * (size_t)(((wblock_floats(s) + 3) & ~3) + ns * mlp_pitch(s));
}

template <typename F>
cudaError_t dispatch_h(int H, F f) {
  switch (H) {
    case 16: return f(std::integral_constant<int, 16>());
    case 32: return f(std::integral_constant<int, 32>());
    case 64: return f(std::integral_constant<int, 64>());
    default: return cudaErrorInvalidValue;
  }
}

void mlp_free(rslb_mlp* m) {
  if (!m) return;
  void* p[] = {m->theta, m->wb, m->grad, m->m, m->v, m->part, m->lossp, m->loss_acc, m->perm,
               m->norm};
  for (void* x : p)
    if (x) cudaFree(x);
  delete m;
}

cudaError_t set_smem_attrs(const MlpShape& s) {
  const int ns = train_ns(s);
  const int tsm = (int)train_smem(s, ns);
  return dispatch_h(s.H, [&](auto Hc) {
    constexpr int H = decltype(Hc)::value;
    cudaError_t e = cudaFuncSetAttribute(mlp_train_kernel<H>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, tsm);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(mlp_infer_kernel<H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kSmemLimit);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(closure_apply_kernel<H>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    return e;
  });
}

// Gradient of the mean-squared loss over samples [n0, n0 + nb) of the
// (permuted) data into m->grad; adds loss * loss_scale to m->loss_acc.
cudaError_t mlp_batch_grad(rslb_mlp* m, const float* X, const float* T, const int* perm, int n0,
                           int nb, double loss_scale) {
  const MlpShape& s = m->s;
  const int ns = train_ns(s);
  const int nblk = (nb + ns - 1) / ns;
  if (nblk > m->part_blocks) {
    if (m->part) cudaFree(m->part);
    if (m->lossp) cudaFree(m->lossp);
    m->part = nullptr;
    m->lossp = nullptr;
    if (cudaMalloc((void**)&m->part, sizeof(float) * (size_t)nblk * s.P) != cudaSuccess ||
        cudaMalloc((void**)&m->lossp, sizeof(double) * nblk) != cudaSuccess)
      return cudaErrorMemoryAllocation;
    m->part_blocks = nblk;
  }
  const float inv_norm = 1.f / ((float)nb * (float)s.O);
  const size_t smem = train_smem(s, ns);
  cudaError_t e = dispatch_h(s.H, [&](auto Hc) {
    constexpr int H = decltype(Hc)::value;
    mlp_train_kernel<H><<<nblk, ns, smem, m->stream>>>(s, m->theta, m->wb, m->norm, X, T, perm,
                                                       n0, nb,
                                                       inv_norm, mlp_pitch(s), m->part, m->lossp);
    return cudaGetLastError();
  });
  if (e != cudaSuccess) return e;
  mlp_reduce_kernel<<<(s.P + 255) / 256, 256, 0, m->stream>>>(m->part, nblk, s.P, m->grad,
                                                               m->lossp, loss_scale, m->loss_acc);
  return cudaGetLastError();
}

}  // namespace

extern "C" int rslb_mlp_create(rslb_mlp** out, int n_in, int n_hidden, int n_out,
                               unsigned long long seed, void* stream) {
  clear_error();
  if (!out) return set_error(RSLB_ERR_ARG, "rslb_mlp_create: NULL output");
  *out = nullptr;
  if (n_in < 1 || n_in > kMaxD || n_out < 1 || n_out > kMaxO ||
      (n_hidden != 16 && n_hidden != 32 && n_hidden != 64))
    return set_error(RSLB_ERR_ARG,
                     "rslb_mlp_create: need 1 <= n_in <= %d, n_hidden in {16, 32, 64}, "
                     "1 <= n_out <= %d",
                     kMaxD, kMaxO);
  rslb_mlp* m = new rslb_mlp();
  std::memset(m, 0, sizeof(*m));
  m->s = make_shape(n_in, n_hidden, n_out);
  m->stream = (cudaStream_t)stream;
  const int P = m->s.P;
  if (train_ns(m->s) == 0) {
    delete m;
    return set_error(RSLB_ERR_UNSUPPORTED, "rslb_mlp_create: network too large for a CTA");
  }
  // initial parameters: weights N(0, 1/fan_in) (output layer scaled by 0.1),
  // biases zero
  std::vector<float> th(P, 0.f);
  uint64_t st = seed ^ 0x243F6A8885A308D3ull;
  const MlpShape& s = m->s;
  for (int e = 0; e < s.H * s.D; ++e) th[s.oW1 + e] = (float)(unit_normal(st) / std::sqrt(s.D));
  for (int e = 0; e < s.H * s.H; ++e) th[s.oW2 + e] = (float)(unit_normal(st) / std::sqrt(s.H));
  for (int e = 0; e < s.O * s.H; ++e)
    th[s.oW3 + e] = (float)(0.1 * unit_normal(st) / std::sqrt(s.H));
  bool ok = cudaMalloc((void**)&m->theta, sizeof(float) * P) == cudaSuccess &&
            cudaMalloc((void**)&m->wb, sizeof(__nv_bfloat16) * P) == cudaSuccess &&
            cudaMalloc((void**)&m->grad, sizeof(float) * P) == cudaSuccess &&
            cudaMalloc((void**)&m->m, sizeof(float) * P) == cudaSuccess &&
            cudaMalloc((void**)&m->v, sizeof(float) * P) == cudaSuccess &&
            cudaMalloc((void**)&m->loss_acc, sizeof(double)) == cudaSuccess &&
            cudaMalloc((void**)&m->norm, sizeof(float) * (2 * s.D + s.O)) == cudaSuccess;
  if (!ok) {
    mlp_free(m);
    return set_error(RSLB_ERR_ALLOC, "rslb_mlp_create: cudaMalloc failed");
  }
  std::vector<float> nrm(2 * s.D + s.O, 1.f);
  for (int d = 0; d < s.D; ++d) nrm[d] = 0.f;  // mu = 0, inv_sd = 1, out_sd = 1
  cudaError_t e = set_smem_attrs(m->s);
  if (e == cudaSuccess)
    e = cudaMemcpy(m->norm, nrm.data(), sizeof(float) * nrm.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(m->theta, th.data(), sizeof(float) * P, cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->m, 0, sizeof(float) * P, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->v, 0, sizeof(float) * P, m->stream);
  if (e == cudaSuccess) {
    mlp_round_kernel<<<(P + 255) / 256, 256, 0, m->stream>>>(m->theta, P, m->wb);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) {
    mlp_free(m);
    return cuda_error(e, "rslb_mlp_create");
  }
  *out = m;
  return RSLB_OK;
}

extern "C" int rslb_mlp_num_params(const rslb_mlp* m) { return m ? m->s.P : 0; }

extern "C" int rslb_mlp_get_params(rslb_mlp* m, float* theta) {
  clear_error();
  if (!m || !theta) return set_error(RSLB_ERR_ARG, "rslb_mlp_get_params: NULL argument");
  cudaError_t e = cudaMemcpyAsync(theta, m->theta, sizeof(float) * m->s.P, cudaMemcpyDeviceToHost,
                                  m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  return e == cudaSuccess ? RSLB_OK : cuda_error(e, "rslb_mlp_get_params");
}

extern "C" int rslb_mlp_set_params(rslb_mlp* m, const float* theta) {
  clear_error();
  if (!m || !theta) return set_error(RSLB_ERR_ARG, "rslb_mlp_set_params: NULL argument");
  const int P = m->s.P;
  cudaError_t e =
      cudaMemcpyAsync(m->theta, theta, sizeof(float) * P, cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) {
    mlp_round_kernel<<<(P + 255) / 256, 256, 0, m->stream>>>(m->theta, P, m->wb);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(m->m, 0, sizeof(float) * P, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->v, 0, sizeof(float) * P, m->stream);
  m->adam_t = 0;
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  return e == cudaSuccess ? RSLB_OK : cuda_error(e, "rslb_mlp_set_params");
}

extern "C" int rslb_mlp_set_normalization(rslb_mlp* m, const float* mu, const float* inv_sd,
                                          const float* out_sd) {
  clear_error();
  if (!m || !mu || !inv_sd || !out_sd)
    return set_error(RSLB_ERR_ARG, "rslb_mlp_set_normalization: NULL argument");
  const MlpShape& s = m->s;
  std::vector<float> h(2 * s.D + s.O);
  std::memcpy(h.data(), mu, sizeof(float) * s.D);
  std::memcpy(h.data() + s.D, inv_sd, sizeof(float) * s.D);
  std::memcpy(h.data() + 2 * s.D, out_sd, sizeof(float) * s.O);
  cudaError_t e = cudaMemcpyAsync(m->norm, h.data(), sizeof(float) * h.size(),
                                  cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  return e == cudaSuccess ? RSLB_OK : cuda_error(e, "rslb_mlp_set_normalization");
}

extern "C" int rslb_mlp_get_normalization(rslb_mlp* m, float* mu, float* inv_sd, float* out_sd) {
  clear_error();
  if (!m || !mu || !inv_sd || !out_sd)
    return set_error(RSLB_ERR_ARG, "rslb_mlp_get_normalization: NULL argument");
  const MlpShape& s = m->s;
  std::vector<float> h(2 * s.D + s.O);
  cudaError_t e = cudaMemcpyAsync(h.data(), m->norm, sizeof(float) * h.size(),
                                  cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_error(e, "rslb_mlp_get_normalization");
  std::memcpy(mu, h.data(), sizeof(float) * s.D);
  std::memcpy(inv_sd, h.data() + s.D, sizeof(float) * s.D);
  std::memcpy(out_sd, h.data() + 2 * s.D, sizeof(float) * s.O);
  return RSLB_OK;
}

extern "C" int rslb_mlp_fit_normalization(rslb_mlp* m, const float* X, const float* T, int n) {
  clear_error();
  if (!m || !X || !T || n < 1)
    return set_error(RSLB_ERR_ARG, "rslb_mlp_fit_normalization: bad arguments");
  const MlpShape& s = m->s;
  fit_norm_kernel<<<s.D + s.O, 256, 0, m->stream>>>(X, T, n, s.D, s.O, m->norm);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  return e == cudaSuccess ? RSLB_OK : cuda_error(e, "rslb_mlp_fit_normalization");
}

extern "C" int rslb_mlp_forward(rslb_mlp* m, const float* X, int n, float* Y) {
  clear_error();
  if (!m || !X || !Y || n < 0) return set_error(RSLB_ERR_ARG, "rslb_mlp_forward: bad arguments");
  if (n == 0) return RSLB_OK;
  const MlpShape& s = m->s;
  const int ns = 128;
  const int pitch = (s.D % 2) ? s.D : s.D + 1;
  const size_t smem = sizeof(float) * (size_t)(((wblock_floats(s) + 3) & ~3) + ns * pitch);
  cudaError_t e = dispatch_h(s.H, [&](auto Hc) {
    constexpr int H = decltype(Hc)::value;
    mlp_infer_kernel<H><<<(n + ns - 1) / ns, ns, smem, m->stream>>>(s, m->theta, m->wb, m->norm,
                                                                    X, n,
                                                                    pitch, Y);
    return cudaGetLastError();
  });
  return e == cudaSuccess ? RSLB_OK : cuda_error(e, "rslb_mlp_forward");
}

extern "C" int rslb_mlp_loss_grad(rslb_mlp* m, const float* X, const float* T, int n,
                                  double* loss, float* grad) {
  clear_error();
  if (!m || !X || !T || n < 1) return set_error(RSLB_ERR_ARG, "rslb_mlp_loss_grad: bad arguments");
  cudaError_t e = cudaMemsetAsync(m->loss_acc, 0, sizeof(double), m->stream);
  if (e == cudaSuccess)
    e = mlp_batch_grad(m, X, T, nullptr, 0, n, 1.0 / ((double)n * m->s.O));
  double L = 0.0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&L, m->loss_acc, sizeof(double), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess && grad)
    e = cudaMemcpyAsync(grad, m->grad, sizeof(float) * m->s.P, cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_error(e, "rslb_mlp_loss_grad");
  if (loss) *loss = L;
  return RSLB_OK;
}

extern "C" int rslb_mlp_train(rslb_mlp* m, const float* X, const float* T, int n, int epochs,
                              int batch, double lr, unsigned long long seed, double* epoch_loss) {
  clear_error();
  if (!m || !X || !T || n < 1 || epochs < 0 || batch < 1 || !(lr > 0.0))
    return set_error(RSLB_ERR_ARG, "rslb_mlp_train: bad arguments");
  if (n > m->perm_n) {
    if (m->perm) cudaFree(m->perm);
    m->perm = nullptr;
    if (cudaMalloc((void**)&m->perm, sizeof(int) * (size_t)n) != cudaSuccess)
      return set_error(RSLB_ERR_ALLOC, "rslb_mlp_train: cudaMalloc failed");
    m->perm_n = n;
  }
  std::vector<int> perm(n);
  uint64_t st = seed ^ 0x13198A2E03707344ull;
  cudaError_t e = cudaSuccess;
  const int P = m->s.P;
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int i = n - 1; i > 0; --i) std::swap(perm[i], perm[splitmix(st) % (uint64_t)(i + 1)]);
    e = cudaMemcpyAsync(m->perm, perm.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice,
                        m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->loss_acc, 0, sizeof(double), m->stream);
    for (int n0 = 0; n0 < n && e == cudaSuccess; n0 += batch) {
      const int nb = std::min(batch, n - n0);
      e = mlp_batch_grad(m, X, T, m->perm, n0, nb, 1.0 / ((double)n * m->s.O));
      if (e != cudaSuccess) break;
      m->adam_t += 1;
      const double c1 = 1.0 / (1.0 - std::pow(0.9, (double)m->adam_t));
      const double c2 = 1.0 / (1.0 - std::pow(0.999, (double)m->adam_t));
      mlp_adam_kernel<<<(P + 255) / 256, 256, 0, m->stream>>>(m->theta, m->grad, m->m, m->v, P,
                                                              (float)lr, (float)c1, (float)c2,
                                                              m->s, m->wb);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess && epoch_loss) {
      // the stream-ordered copy lands before the host buffer is read at the sync below
      e = cudaMemcpyAsync(epoch_loss + ep, m->loss_acc, sizeof(double), cudaMemcpyDeviceToHost,
                          m->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  return e == cudaSuccess ? RSLB_OK : cuda_error(e, "rslb_mlp_train");
}

extern "C" void rslb_mlp_destroy(rslb_mlp* m) {
  if (!m) return;
  cudaStreamSynchronize(m->stream);
  mlp_free(m);
}

// ---------------------------------------------------------------------------
// closure entry points
// ---------------------------------------------------------------------------
namespace {

int check_pair(rslb_handle* hi, rslb_handle* lo, SodView* vh, SodView* vl, const char* what) {
  if (sod_view(hi, vh) || sod_view(lo, vl)) return set_error(RSLB_ERR_ARG, "%s: NULL handle", what);
  if (vh->fp64 || vl->fp64) return set_error(RSLB_ERR_UNSUPPORTED, "%s: needs RSLB_F32 handles", what);
  if (vh->Z != vl->Z || vh->Q_L != vl->Q_L || vh->Q_xi < vl->Q_xi || vl->V > kMaxO)
    return set_error(RSLB_ERR_ARG,
                     "%s: handles need equal Z and Q_L, Q_xi(hi) >= Q_xi(lo), Q_L*Q_xi(lo) <= %d",
                     what, kMaxO);
  return RSLB_OK;
}

// R[i][j] = w_i sum_{m < Ql} (2m+1)/2 P_m(xi^lo_i) P_m(xi^hi_j), FP64 -> FP32.
cudaError_t upload_restriction(int Qh, int Ql, float** dev, cudaStream_t st) {
  std::vector<double> xh(Qh), wh(Qh), xl(Ql), wl(Ql);
  gauss_legendre_host(Qh, xh.data(), wh.data());
  gauss_legendre_host(Ql, xl.data(), wl.data());
  std::vector<float> R((size_t)Ql * Qh);
  for (int i = 0; i < Ql; ++i)
    for (int j = 0; j < Qh; ++j) {
      double acc = 0.0;
      for (int mm = 0; mm < Ql; ++mm)
        acc += 0.5 * (2.0 * mm + 1.0) * legendre_p(mm, xl[i]) * legendre_p(mm, xh[j]);
      R[(size_t)i * Qh + j] = (float)(wl[i] * acc);
    }
  cudaError_t e = cudaMalloc((void**)dev, sizeof(float) * R.size());
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(*dev, R.data(), sizeof(float) * R.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

cudaError_t launch_restrict(const SodView& vh, const SodView& vl, const float* R, float* dst,
                            cudaStream_t st) {
  const int T = 128;
  restrict_kernel<<<(vh.Z + T - 1) / T, T, sizeof(float) * vl.Q_xi * vh.Q_xi, st>>>(
      (const float*)vh.F0, vh.ldz, vh.Q_xi, dst, vl.ldz, vl.Q_xi, vl.Q_L, R, vh.Z);
  return cudaGetLastError();
}

}  // namespace

extern "C" int rslb_restrict(rslb_handle* hi, rslb_handle* lo) {
  clear_error();
  SodView vh, vl;
  int rc = check_pair(hi, lo, &vh, &vl, "rslb_restrict");
  if (rc) return rc;
  float* R = nullptr;
  cudaError_t e = cudaStreamSynchronize(vh.stream);
  if (e == cudaSuccess) e = upload_restriction(vh.Q_xi, vl.Q_xi, &R, vl.stream);
  if (e == cudaSuccess) e = launch_restrict(vh, vl, R, (float*)vl.F0, vl.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(vl.stream);
  if (R) cudaFree(R);
  return e == cudaSuccess ? RSLB_OK : cuda_error(e, "rslb_restrict");
}

extern "C" int rslb_closure_sample(rslb_handle* hi, rslb_handle* lo, double tau, float* X,
                                   float* T) {
  clear_error();
  SodView vh, vl;
  int rc = check_pair(hi, lo, &vh, &vl, "rslb_closure_sample");
  if (rc) return rc;
  if (!X || !T || !(tau > 0.0)) return set_error(RSLB_ERR_ARG, "rslb_closure_sample: bad arguments");
  ClosureConsts cc;
  rc = closure_consts(vl.Q_xi, vl.Q_L, &cc);
  if (rc) return set_error(rc, "rslb_closure_sample: low-order set too large");
  float *R = nullptr, *ns = nullptr, *ref = nullptr;
  cudaStream_t st = vl.stream;
  cudaError_t e = cudaStreamSynchronize(vh.stream);
  if (e == cudaSuccess) e = upload_restriction(vh.Q_xi, vl.Q_xi, &R, st);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ns, sizeof(float) * vl.Z);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ref, sizeof(float) * (size_t)vl.V * vl.ldz);
  const int TB = 128, G = (vl.Z + TB - 1) / TB;
  if (e == cudaSuccess) e = launch_restrict(vh, vl, R, (float*)vl.F0, st);
  if (e == cudaSuccess) {
    features_kernel<<<G, TB, 0, st>>>((const float*)vl.F0, vl.Z, vl.ldz, vl.V,
                                      (float)std::log10(tau), X, ns);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && (rc = rslb_step(lo, 1)) != RSLB_OK) e = cudaErrorUnknown;
  if (e == cudaSuccess && (rc = rslb_step(hi, 1)) != RSLB_OK) e = cudaErrorUnknown;
  if (e == cudaSuccess) e = cudaStreamSynchronize(vh.stream);
  if (e == cudaSuccess) e = launch_restrict(vh, vl, R, ref, st);
  if (e == cudaSuccess) {
    target_kernel<<<G, TB, 0, st>>>(ref, (const float*)vl.F0, ns, vl.Z, vl.ldz, vl.V, cc, T);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (R) cudaFree(R);
  if (ns) cudaFree(ns);
  if (ref) cudaFree(ref);
  if (rc) return rc;
  return e == cudaSuccess ? RSLB_OK : cuda_error(e, "rslb_closure_sample");
}

extern "C" int rslb_closure_step(rslb_handle* lo, rslb_mlp* m, double tau, int nsteps) {
  clear_error();
  SodView vl;
  if (sod_view(lo, &vl) || !m || nsteps < 0 || !(tau > 0.0))
    return set_error(RSLB_ERR_ARG, "rslb_closure_step: bad arguments");
  if (vl.fp64) return set_error(RSLB_ERR_UNSUPPORTED, "rslb_closure_step: needs an RSLB_F32 handle");
  if (m->s.O != vl.V || m->s.D != 3 * vl.V + 1)
    return set_error(RSLB_ERR_ARG, "rslb_closure_step: network shape (%d -> %d) does not match "
                     "3V+1 -> V for V = %d", m->s.D, m->s.O, vl.V);
  ClosureConsts cc;
  int rc = closure_consts(vl.Q_xi, vl.Q_L, &cc);
  if (rc) return set_error(rc, "rslb_closure_step: low-order set too large");
  const MlpShape& s = m->s;
  const size_t smem = sizeof(float) * (size_t)((wblock_floats(s) + 3) & ~3);
  const int TB = 128, G = (vl.Z + TB - 1) / TB;
  const float lt = (float)std::log10(tau);
  for (int n = 0; n < nsteps; ++n) {
    rc = rslb_step(lo, 1);
    if (rc) return rc;
    cudaError_t e = dispatch_h(s.H, [&](auto Hc) {
      constexpr int H = decltype(Hc)::value;
      closure_apply_kernel<H><<<G, TB, smem, vl.stream>>>(s, m->theta, m->wb, m->norm,
                                                          (const float*)vl.F0, (float*)vl.F1,
                                                          vl.Z, vl.ldz, lt, cc);
      return cudaGetLastError();
    });
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(vl.F0, vl.F1, sizeof(float) * (size_t)vl.V * vl.ldz,
                          cudaMemcpyDeviceToDevice, vl.stream);
    if (e != cudaSuccess) return cuda_error(e, "rslb_closure_step");
  }
  return RSLB_OK;
}
