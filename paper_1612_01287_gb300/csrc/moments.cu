// moments.cu -- output moments of the shock-tube populations (sm_103a).
//
// Per cell: the first and second moments (Eq. macro_jk), Landau matching
// (Sec. II E, Eqs. E_landau-pi_val) in FP64 and the 14 fields of rslb.h.
// Five sums are formed directly, each with a non-negative weight, as the
// factored Landau form needs them:
//   N+- = sum f (1 +- xi),  A+- = sum f p (1 +- xi)^2,  D = sum f p (1 - xi^2);
// the conserved currents follow exactly:
//   N^t = (N+ + N-)/2,  N^z = (N+ - N-)/2,  T^tz = (A+ - A-)/4,
//   T^tt = (A+ + A-)/4 + D/2,  T^zz = (A+ + A-)/4 - D/2.
//
// Layout: a block covers kMomCells32 (FP32) or kMomCells64 (FP64) cells; its
// warps 2c and 2c+1 read the c-th of kMomChunks velocity chunks, so every
// load is a coalesced piece of a row of the [V][ldz] population array.  The
// chunk partials meet in shared memory and one thread per cell finishes the
// cell in FP64.
//
// FP32 populations: the FP64 weight w is split as w_hi + w_lo (two FP32
// numbers, host-made table); f w_hi is formed exactly as a product plus its
// fma remainder, and the sum is kept as a double-float: the hi parts are
// added with an error-free TwoSum (Knuth), the remainders, f w_lo and the
// TwoSum errors in a plain FP32 sum of the low part.  Two neighbouring cells
// share a thread in packed FP32x2 arithmetic.  GB300's FP64 pipe is a small
// fraction of its FP32 rate, so FP64 is used only for the per-cell finish.
// FP64 populations: plain FP64 products and sums, one cell per thread.
#include "rslb_device.cuh"
#include "sod.cuh"

namespace rslb {

namespace {

constexpr int kMomChunks = 4;                 // velocity chunks per block
constexpr int kMomThreads = 64 * kMomChunks;  // two warps per chunk

__device__ __forceinline__ float2 mom_add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b with one rounding
__device__ __forceinline__ float2 mom_sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}

// (H, L) += x * (wh + wl) for two cells; H + L is a double-float.
__device__ __forceinline__ void mom_acc2(float2& H, float2& L, float2 x, float wh, float wl) {
  const float2 WH = make_float2(wh, wh), WL = make_float2(wl, wl);
  const float2 ph = __fmul2_rn(x, WH);
  float2 pl = __ffma2_rn(x, WH, make_float2(-ph.x, -ph.y));  // exact: x wh = ph + pl
  pl = __ffma2_rn(x, WL, pl);
  const float2 s = mom_add2(H, ph);  // TwoSum(H, ph) = s + e exactly
  const float2 bp = mom_sub2(s, H);
  const float2 e = mom_add2(mom_sub2(H, mom_sub2(s, bp)), mom_sub2(ph, bp));
  H = s;
  L = mom_add2(L, mom_add2(e, pl));
}

// Per-cell finish: Landau matching and the 14 output fields (rslb.h order).
__device__ __forceinline__ void mom_finish(const double* S, int s, int Z, double* out, int* err) {
  const double Np = S[0], Nm = S[1], Ap = S[2], Am = S[3], D = S[4];
  const LandauOut L = landau_factored(Np, Nm, Ap, Am, D);
  if (!L.ok && atomicCAS(err, 0, 6) == 0) err[1] = s;
  const double Nt = 0.5 * (Np + Nm), Nz = 0.5 * (Np - Nm);
  const double tr = 0.25 * (Ap + Am);
  const size_t z = (size_t)Z;
  out[0 * z + s] = L.n;
  out[1 * z + s] = L.E;
  out[2 * z + s] = L.E / 3.0;
  out[3 * z + s] = L.T;
  out[4 * z + s] = L.beta;
  out[5 * z + s] = L.gamma;
  out[6 * z + s] = L.n / (L.T * L.T * L.T);
  out[7 * z + s] = -4.0 * L.T * (Nz - L.n * L.beta * L.gamma);
  out[8 * z + s] = 2.0 * L.E / 3.0 - D;
  out[9 * z + s] = Nt;
  out[10 * z + s] = Nz;
  out[11 * z + s] = tr + 0.5 * D;
  out[12 * z + s] = 0.25 * (Ap - Am);
  out[13 * z + s] = tr - 0.5 * D;
}

// FP32 populations.  w: per velocity three float4 =
// {hi0 hi1 hi2 hi3} {hi4 lo0 lo1 lo2} {lo3 lo4 0 0}.
constexpr int kMomCells32 = 128;  // 64 threads x 2 cells per chunk

__global__ void __launch_bounds__(kMomThreads)
sod_moments32_kernel(int Z, int ldz, int V, const float4* __restrict__ w,
                     const float* __restrict__ f, double* out, int* err) {
  __shared__ float2 part[kMomChunks][5][2][kMomCells32 / 2];  // [chunk][sum][hi/lo][pair]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int chunk = warp >> 1;
  const int pr = (warp & 1) * 32 + lane;             // pair within the block
  const int c0 = blockIdx.x * kMomCells32 + 2 * pr;  // first cell of the pair
  const bool active = c0 < ldz;                      // ldz is even: the pair fits
  const int vb = (chunk * V) / kMomChunks, ve = ((chunk + 1) * V) / kMomChunks;
  float2 H[5], L[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    H[q] = make_float2(0.f, 0.f);
    L[q] = make_float2(0.f, 0.f);
  }
  const float* fp = f + c0;
  int v = vb;
  for (; v + 4 <= ve; v += 4) {
    float2 x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      x[u] = active ? __ldg(reinterpret_cast<const float2*>(fp + (size_t)(v + u) * ldz))
                    : make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float4 a = __ldg(w + 3 * (v + u)), b = __ldg(w + 3 * (v + u) + 1),
                   c = __ldg(w + 3 * (v + u) + 2);
      mom_acc2(H[0], L[0], x[u], a.x, b.y);
      mom_acc2(H[1], L[1], x[u], a.y, b.z);
      mom_acc2(H[2], L[2], x[u], a.z, b.w);
      mom_acc2(H[3], L[3], x[u], a.w, c.x);
      mom_acc2(H[4], L[4], x[u], b.x, c.y);
    }
  }
  for (; v < ve; ++v) {
    const float2 x = active ? __ldg(reinterpret_cast<const float2*>(fp + (size_t)v * ldz))
                            : make_float2(0.f, 0.f);
    const float4 a = __ldg(w + 3 * v), b = __ldg(w + 3 * v + 1), c = __ldg(w + 3 * v + 2);
    mom_acc2(H[0], L[0], x, a.x, b.y);
    mom_acc2(H[1], L[1], x, a.y, b.z);
    mom_acc2(H[2], L[2], x, a.z, b.w);
    mom_acc2(H[3], L[3], x, a.w, c.x);
    mom_acc2(H[4], L[4], x, b.x, c.y);
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    part[chunk][q][0][pr] = H[q];
    part[chunk][q][1][pr] = L[q];
  }
  __syncthreads();
  if (threadIdx.x >= kMomCells32) return;
  const int cl = threadIdx.x, s = blockIdx.x * kMomCells32 + cl;
  if (s >= Z) return;
  const int p = cl >> 1, odd = cl & 1;
  double S[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < kMomChunks; ++k) {
      const float2 h = part[k][q][0][p], l = part[k][q][1][p];
      acc += odd ? ((double)h.y + (double)l.y) : ((double)h.x + (double)l.x);
    }
    S[q] = acc;
  }
  mom_finish(S, s, Z, out, err);
}

// FP64 populations.  w: per velocity three double2 = {w0 w1} {w2 w3} {w4 0}.
constexpr int kMomCells64 = 64;  // 64 threads x 1 cell per chunk

__global__ void __launch_bounds__(kMomThreads)
sod_moments64_kernel(int Z, int ldz, int V, const double2* __restrict__ w,
                     const double* __restrict__ f, double* out, int* err) {
  __shared__ double part[kMomChunks][5][kMomCells64];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int chunk = warp >> 1;
  const int cl = (warp & 1) * 32 + lane;
  const int s0 = blockIdx.x * kMomCells64 + cl;
  const bool active = s0 < ldz;
  const int vb = (chunk * V) / kMomChunks, ve = ((chunk + 1) * V) / kMomChunks;
  double S[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const double* fp = f + s0;
  int v = vb;
  for (; v + 4 <= ve; v += 4) {
    double x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = active ? __ldg(fp + (size_t)(v + u) * ldz) : 0.0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const double2 a = __ldg(w + 3 * (v + u)), b = __ldg(w + 3 * (v + u) + 1),
                    c = __ldg(w + 3 * (v + u) + 2);
      S[0] = fma(x[u], a.x, S[0]);
      S[1] = fma(x[u], a.y, S[1]);
      S[2] = fma(x[u], b.x, S[2]);
      S[3] = fma(x[u], b.y, S[3]);
      S[4] = fma(x[u], c.x, S[4]);
    }
  }
  for (; v < ve; ++v) {
    const double x = active ? __ldg(fp + (size_t)v * ldz) : 0.0;
    const double2 a = __ldg(w + 3 * v), b = __ldg(w + 3 * v + 1), c = __ldg(w + 3 * v + 2);
    S[0] = fma(x, a.x, S[0]);
    S[1] = fma(x, a.y, S[1]);
    S[2] = fma(x, b.x, S[2]);
    S[3] = fma(x, b.y, S[3]);
    S[4] = fma(x, c.x, S[4]);
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) part[chunk][q][cl] = S[q];
  __syncthreads();
  if (threadIdx.x >= kMomCells64) return;
  const int s = blockIdx.x * kMomCells64 + threadIdx.x;
  if (s >= Z) return;
  double T[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < kMomChunks; ++k) acc += part[k][q][threadIdx.x];
    T[q] = acc;
  }
  mom_finish(T, s, Z, out, err);
}

}  // namespace

size_t sod_moment_weights(bool fp64, int V, const double* xi, const double* p, void* out) {
  const size_t bytes = fp64 ? sizeof(double) * 6 * (size_t)V : sizeof(float) * 12 * (size_t)V;
  if (!out) return bytes;
  for (int v = 0; v < V; ++v) {
    const double x = xi[v], pv = p[v];
    const double wq[5] = {1.0 + x, 1.0 - x, pv * (1.0 + x) * (1.0 + x), pv * (1.0 - x) * (1.0 - x),
                          pv * (1.0 - x) * (1.0 + x)};
    if (fp64) {
      double* o = static_cast<double*>(out) + 6 * (size_t)v;
      for (int q = 0; q < 5; ++q) o[q] = wq[q];
      o[5] = 0.0;
    } else {
      float hi[5], lo[5];
      for (int q = 0; q < 5; ++q) {
        hi[q] = (float)wq[q];
        lo[q] = (float)(wq[q] - (double)hi[q]);
      }
      float* o = static_cast<float*>(out) + 12 * (size_t)v;
      const float row[12] = {hi[0], hi[1], hi[2], hi[3], hi[4], lo[0],
                             lo[1], lo[2], lo[3], lo[4], 0.f,   0.f};
      for (int i = 0; i < 12; ++i) o[i] = row[i];
    }
  }
  return bytes;
}

template <>
cudaError_t sod_moments_launch<float>(const SodGeom& g, const void* w, const float* f,
                                      double* out, int* err, cudaStream_t st) {
  if (g.Z <= 0) return cudaSuccess;
  sod_moments32_kernel<<<(g.Z + kMomCells32 - 1) / kMomCells32, kMomThreads, 0, st>>>(
      g.Z, g.ldz, g.V, static_cast<const float4*>(w), f, out, err);
  return cudaGetLastError();
}

template <>
cudaError_t sod_moments_launch<double>(const SodGeom& g, const void* w, const double* f,
                                       double* out, int* err, cudaStream_t st) {
  if (g.Z <= 0) return cudaSuccess;
  sod_moments64_kernel<<<(g.Z + kMomCells64 - 1) / kMomCells64, kMomThreads, 0, st>>>(
      g.Z, g.ldz, g.V, static_cast<const double2*>(w), f, out, err);
  return cudaGetLastError();
}

}  // namespace rslb
