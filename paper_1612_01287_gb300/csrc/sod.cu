// sod.cu -- fused RK-stage kernel of the R-SLB Sod shock tube (sm_103a).
//
// One CTA owns a tile of B consecutive cells and all V velocities.  A stage
// (Eq. rk3) is one launch:
//   1. the tile plus a 3-cell halo on each side is staged in shared memory
//      (velocity-major rows, boundary cells mapped by the boundary condition);
//   2. moments: each lane owns velocity rows, accumulates the five sums of the
//      factored Landau form (Kahan-compensated in FP32), and a warp-shuffle
//      tree reduces them across the velocity set;
//   3. per cell: Landau matching in FP64 (Sec. II E), relaxation time, and the
//      f^eq expansion coefficients (Sec. III D) by a Gauss-Legendre rule spread
//      over all threads of the CTA and reduced by shuffles;
//   4. per (velocity, cell): WENO5 flux difference (Sec. III F) along the row
//      with a sliding register window, f^eq from the per-cell coefficients,
//      Anderson-Witting relaxation (Eq. L_Sod) and the RK combination;
//   5. coalesced store of the tile interior (plus the f_n term of stages 2, 3).
#include "rslb_device.cuh"
#include "sod.cuh"

namespace rslb {

constexpr int kThreads = 256;
constexpr int kMaxQL = 8;

template <typename T, int B>
struct SodTile {
  // row pitch of the staged tile: B + 6 cells, made odd so that lanes that
  // own consecutive rows hit distinct shared-memory banks
  static constexpr int W = B + 6;
  static constexpr int P = (W % 2 == 0) ? W + 1 : W;
  __host__ __device__ static size_t tile_bytes(int V) { return sizeof(T) * (size_t)V * P; }
  __host__ __device__ static size_t extra_bytes() {
    return sizeof(double) * (5 * B + 8 * B) + sizeof(T) * (kMaxQL * kMaxM * B + 2 * B);
  }
  __host__ __device__ static size_t smem_bytes(int V) {
    size_t t = (tile_bytes(V) + 15) & ~size_t(15);
    return t + extra_bytes();
  }
};

__device__ __forceinline__ void report_error(int* err, int code, int cell) {
  if (atomicCAS(err, 0, code) == 0) err[1] = cell;
}

// Kahan-compensated accumulation (FP32) / plain accumulation (FP64).
template <typename T> struct Acc;
template <> struct Acc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
template <> struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  return x;
}

template <typename T>
__device__ __forceinline__ T load_cell(const T* __restrict__ fin, const SodGeom& g,
                                       const SodTables<T>& tb, int v, int s) {
  if (s >= 0 && s < g.Z) return fin[(size_t)v * g.ldz + s];
  if (g.bc == kBcPeriodic) {
    int sp = s % g.Z;
    if (sp < 0) sp += g.Z;
    return fin[(size_t)v * g.ldz + sp];
  }
  if (g.bc == kBcOutflow) return fin[(size_t)v * g.ldz + (s < 0 ? 0 : g.Z - 1)];
  return s < 0 ? tb.ghostL[v] : tb.ghostR[v];
}

// Phase 4 for one work unit: velocity row v, local cells [i0, i0 + SL).
// If out != nullptr the results are kept in registers (segmented rows share
// halo cells, so they may only be written back after a barrier); otherwise
// they are written in place, which is safe because a row is owned by exactly
// one thread and the window has already consumed the overwritten cell.
template <typename T, int B, int SL>
__device__ __forceinline__ void sweep_row(T* __restrict__ row, int v, int i0, const SodGeom& g,
                                          const SodTables<T>& tb, const T* __restrict__ coef,
                                          const T* __restrict__ gco, T* out) {
  const T xi = tb.xi[v];
  const int k = tb.kidx[v];
  T wp[kMaxM];
#pragma unroll
  for (int m = 0; m < kMaxM; ++m) wp[m] = (m < g.nm) ? tb.wp[m * g.V + v] : T(0);
  const bool pos = xi > T(0);
  const T inv_dz = T(g.inv_dz), dt = T(g.dt);
  const T* ck = coef + (size_t)k * kMaxM * B;
  // window J[0..6] = J at local cells i-3 .. i+3 (tile element e = cell + 3)
  T J0 = xi * row[i0 + 0], J1 = xi * row[i0 + 1], J2 = xi * row[i0 + 2];
  T J3 = xi * row[i0 + 3], J4 = xi * row[i0 + 4], J5 = xi * row[i0 + 5];
  T J6 = xi * row[i0 + 6];
  // left face of cell i0
  T Fl = weno5_face<T>(pos ? J0 : J5, pos ? J1 : J4, pos ? J2 : J3, pos ? J3 : J2,
                       pos ? J4 : J1);
#pragma unroll
  for (int ii = 0; ii < SL; ++ii) {
    const int i = i0 + ii;
    const T Fr = weno5_face<T>(pos ? J1 : J6, pos ? J2 : J5, pos ? J3 : J4, pos ? J4 : J3,
                               pos ? J5 : J2);
    const T f = row[i + 3];
    T feq = T(0);
#pragma unroll
    for (int m = 0; m < kMaxM; ++m)
      if (m < g.nm) feq += ck[m * B + i] * wp[m];
    const T coll = (gco[i] - gco[B + i] * xi) * (f - feq);
    const T L = -(Fr - Fl) * inv_dz - coll;
    const T r = f + dt * L;
    if (out) out[ii] = r; else row[i + 3] = r;
    Fl = Fr;
    if (ii + 1 < SL) {
      J0 = J1; J1 = J2; J2 = J3; J3 = J4; J4 = J5; J5 = J6;
      J6 = xi * row[i + 7];
    }
  }
}

template <typename T, int B>
__global__ void __launch_bounds__(kThreads)
sod_stage_kernel(const T* __restrict__ fin, const T* __restrict__ fn, T* fout, int stage,
                 int* err, SodGeom g, SodTables<T> tb, int nseg) {
  using Tile = SodTile<T, B>;
  constexpr int W = Tile::W, P = Tile::P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);
  double* msum = reinterpret_cast<double*>(smem_raw + ((Tile::tile_bytes(g.V) + 15) & ~size_t(15)));
  double* cell = msum + 5 * B;
  T* coef = reinterpret_cast<T*>(cell + 8 * B);
  T* gco = coef + kMaxQL * kMaxM * B;

  const int s0 = blockIdx.x * B;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int V = g.V;

  // ---- 1. stage tile + halo ----
  for (int idx = tid; idx < V * W; idx += kThreads) {
    const int v = idx / W, e = idx - v * W;
    tile[v * P + e] = load_cell<T>(fin, g, tb, v, s0 - 3 + e);
  }
  __syncthreads();

  const bool collide = g.tau_mode != kTauNone;
  if (collide) {
    // ---- 2. moments: lanes own rows, warps own cells ----
    constexpr int CPW = B / (kThreads / 32);
    Acc<T> acc[CPW][5];
    for (int v = lane; v < V; v += 32) {
      T w[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) w[q] = tb.mw[q * V + v];
      const T* row = tile + v * P + 3 + warp * CPW;
#pragma unroll
      for (int c = 0; c < CPW; ++c) {
        const T x = row[c];
#pragma unroll
        for (int q = 0; q < 5; ++q) acc[c][q].add(x * w[q]);
      }
    }
#pragma unroll
    for (int c = 0; c < CPW; ++c)
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const double s = warp_sum(acc[c][q].value());
        if (lane == 0) msum[q * B + warp * CPW + c] = s;
      }
    __syncthreads();

    // ---- 3a. Landau matching and relaxation time, one thread per cell ----
    if (tid < B) {
      const int c = tid;
      LandauOut Lo = landau_factored(msum[c], msum[B + c], msum[2 * B + c], msum[3 * B + c],
                                     msum[4 * B + c]);
      double g0 = 0.0, g1 = 0.0;
      if (!Lo.ok) {
        if (s0 + c < g.Z) report_error(err, 6, s0 + c);
        Lo.n = 1.0; Lo.T = 1.0; Lo.beta = 0.0; Lo.gamma = 1.0; Lo.u = 0.0;
      } else {
        double tau = g.tau;
        if (g.tau_mode == kTauEtas)
          tau = g.tau_AW0 / Lo.T *
                (1.0 - 0.25 * log(Lo.n / (Lo.T * Lo.T * Lo.T) * g.lambda_ref));
        g0 = Lo.gamma / tau;
        g1 = Lo.gamma * Lo.beta / tau;
      }
      const double A = asinh(Lo.u);
      const double sh = sinh(0.5 * A);
      cell[0 * B + c] = Lo.n;
      cell[1 * B + c] = Lo.T;
      cell[2 * B + c] = Lo.u;
      cell[3 * B + c] = A;
      cell[4 * B + c] = (Lo.u > 0.0) ? A / Lo.u : 1.0;
      cell[5 * B + c] = 2.0 * sh * sh;
      cell[6 * B + c] = (Lo.beta < 0.0) ? -1.0 : 1.0;
      cell[7 * B + c] = Lo.ok ? 1.0 : 0.0;
      gco[c] = T(g0);
      gco[B + c] = T(g1);
    }
    __syncthreads();

    // ---- 3b. f^eq coefficients: G threads per cell share the nodes ----
    {
      constexpr int G = kThreads / B;
      const int c = tid / G, q = tid - c * G;
      const double ud = cell[2 * B + c];
      const T A = T(cell[3 * B + c]), sh2 = T(cell[5 * B + c]);
      const T uinv = (ud > 0.0) ? T(1.0 / ud) : T(0);
      const bool at_rest = !(ud > 0.0);
      T J3[kMaxM], J4[kMaxM];
#pragma unroll
      for (int m = 0; m < kMaxM; ++m) { J3[m] = T(0); J4[m] = T(0); }
      for (int i = q; i < kAeqNodes; i += G)
        aeq_node<T>(T(tb.gl_t[i]), T(tb.gl_w[i]), A, sh2, uinv, at_rest, g.nm, J3, J4);
#pragma unroll
      for (int off = G / 2; off >= 1; off >>= 1)
#pragma unroll
        for (int m = 0; m < kMaxM; ++m)
          if (m < g.nm) {
            J3[m] += __shfl_xor_sync(0xffffffffu, J3[m], off);
            J4[m] += __shfl_xor_sync(0xffffffffu, J4[m], off);
          }
      if (q == 0) {
        // c''_{k,m} = sgn^m (2m+1)/2 (n r/4) [J3_m + (3 - x_k)(J3_m - theta J4_m)]
        const double ok = cell[7 * B + c];
        const T fac = T(ok * cell[0 * B + c] * cell[4 * B + c] * 0.25);
        const T theta = T(cell[1 * B + c]);
        const T sgn = T(cell[6 * B + c]);
        T sm = fac;
#pragma unroll
        for (int m = 0; m < kMaxM; ++m) {
          if (m < g.nm) {
            const T h = sm * T(0.5 * (2 * m + 1));
            const T d = J3[m] - theta * J4[m];
            for (int k = 0; k < g.QL; ++k)
              coef[(k * kMaxM + m) * B + c] = h * (J3[m] + tb.L1k[k] * d);
            sm *= sgn;
          }
        }
      }
    }
    __syncthreads();
  } else {
    if (tid < B) { gco[tid] = T(0); gco[B + tid] = T(0); }
    for (int i = tid; i < kMaxQL * kMaxM * B; i += kThreads) coef[i] = T(0);
    __syncthreads();
  }

  // ---- 4. WENO5 + relaxation + RK update, row sweeps ----
  if (nseg == 1) {
    for (int v = tid; v < V; v += kThreads)
      sweep_row<T, B, B>(tile + v * P, v, 0, g, tb, coef, gco, nullptr);
  } else if (nseg == 2) {
    T out[B / 2];
    const int v = tid % V, seg = tid / V;
    const bool active = tid < 2 * V;
    if (active) sweep_row<T, B, B / 2>(tile + v * P, v, seg * (B / 2), g, tb, coef, gco, out);
    __syncthreads();
    if (active)
#pragma unroll
      for (int ii = 0; ii < B / 2; ++ii) tile[v * P + 3 + seg * (B / 2) + ii] = out[ii];
  } else if (nseg == 4) {
    T out[B / 4];
    const int v = tid % V, seg = tid / V;
    const bool active = tid < 4 * V;
    if (active) sweep_row<T, B, B / 4>(tile + v * P, v, seg * (B / 4), g, tb, coef, gco, out);
    __syncthreads();
    if (active)
#pragma unroll
      for (int ii = 0; ii < B / 4; ++ii) tile[v * P + 3 + seg * (B / 4) + ii] = out[ii];
  } else {
    T out[B / 8];
    const int v = tid % V, seg = tid / V;
    const bool active = tid < 8 * V;
    if (active) sweep_row<T, B, B / 8>(tile + v * P, v, seg * (B / 8), g, tb, coef, gco, out);
    __syncthreads();
    if (active)
#pragma unroll
      for (int ii = 0; ii < B / 8; ++ii) tile[v * P + 3 + seg * (B / 8) + ii] = out[ii];
  }
  __syncthreads();

  // ---- 5. coalesced store ----
  const T a = (stage == 1) ? T(0.75) : T(1.0 / 3.0);
  const T b = (stage == 1) ? T(0.25) : T(2.0 / 3.0);
  for (int idx = tid; idx < V * B; idx += kThreads) {
    const int v = idx / B, i = idx - v * B;
    const int s = s0 + i;
    if (s < g.Z) {
      const size_t o = (size_t)v * g.ldz + s;
      T r = tile[v * P + 3 + i];
      if (stage != 0) r = a * fn[o] + b * r;
      fout[o] = r;
    }
  }
}

SodLaunch sod_pick_launch(bool fp64, int V, int QL, int max_smem) {
  SodLaunch L{0, 0};
  if (QL > kMaxQL || V < 1) return L;
  const size_t half = (size_t)max_smem / 2 - 1024;
  if (!fp64) {
    if (SodTile<float, 32>::smem_bytes(V) <= half) return {32, SodTile<float, 32>::smem_bytes(V)};
    if (SodTile<float, 16>::smem_bytes(V) <= (size_t)max_smem)
      return {16, SodTile<float, 16>::smem_bytes(V)};
    if (SodTile<float, 8>::smem_bytes(V) <= (size_t)max_smem)
      return {8, SodTile<float, 8>::smem_bytes(V)};
  } else {
    if (SodTile<double, 16>::smem_bytes(V) <= half) return {16, SodTile<double, 16>::smem_bytes(V)};
    if (SodTile<double, 8>::smem_bytes(V) <= (size_t)max_smem)
      return {8, SodTile<double, 8>::smem_bytes(V)};
  }
  return L;
}

static int pick_nseg(int V, int B) {
  int nseg = 1;
  while (nseg < 8 && B / (2 * nseg) >= 2 && V * 2 * nseg <= kThreads) nseg *= 2;
  return nseg;
}

template <typename T, int B>
static cudaError_t launch_b(const SodLaunch& L, const SodGeom& g, const SodTables<T>& tb,
                            const T* fin, const T* fn, T* fout, int stage, int* err,
                            cudaStream_t st) {
  static bool attr_set = false;  // per device this is cheap to repeat; keep it simple
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(sod_stage_kernel<T, B>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int grid = (g.Z + B - 1) / B;
  sod_stage_kernel<T, B><<<grid, kThreads, L.smem, st>>>(fin, fn, fout, stage, err, g, tb,
                                                         pick_nseg(g.V, B));
  return cudaGetLastError();
}

template <typename T>
cudaError_t sod_stage_launch(const SodLaunch& L, const SodGeom& g, const SodTables<T>& tb,
                             const T* fin, const T* fn, T* fout, int stage, int* err,
                             cudaStream_t st) {
  switch (L.B) {
    case 32: return launch_b<T, 32>(L, g, tb, fin, fn, fout, stage, err, st);
    case 16: return launch_b<T, 16>(L, g, tb, fin, fn, fout, stage, err, st);
    case 8: return launch_b<T, 8>(L, g, tb, fin, fn, fout, stage, err, st);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t sod_stage_launch<float>(const SodLaunch&, const SodGeom&,
                                             const SodTables<float>&, const float*, const float*,
                                             float*, int, int*, cudaStream_t);
template cudaError_t sod_stage_launch<double>(const SodLaunch&, const SodGeom&,
                                              const SodTables<double>&, const double*,
                                              const double*, double*, int, int*, cudaStream_t);

// ---------------------------------------------------------------------------
// Initialisation: per-cell FP64 coefficients, then populations.
// ---------------------------------------------------------------------------
__global__ void sod_init_coef_kernel(SodGeom g, SodTablesF64 tb, const double* __restrict__ n,
                                     const double* __restrict__ Tt,
                                     const double* __restrict__ beta, double* coef, int* err) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.Z) return;
  const double nn = n[s], TT = Tt[s], bb = beta[s];
  if (!(nn > 0.0) || !(TT > 0.0) || !(fabs(bb) < 1.0)) {
    report_error(err, 6, s);
    for (int i = 0; i < kMaxQL * kMaxM; ++i) coef[(size_t)s * kMaxQL * kMaxM + i] = 0.0;
    return;
  }
  const double gam = 1.0 / sqrt((1.0 - bb) * (1.0 + bb));
  const double u = gam * fabs(bb);
  const double A = asinh(u);
  const double sh = sinh(0.5 * A);
  const double sh2 = 2.0 * sh * sh;
  const double uinv = u > 0.0 ? 1.0 / u : 0.0;
  double J3[kMaxM], J4[kMaxM];
  for (int m = 0; m < kMaxM; ++m) { J3[m] = 0.0; J4[m] = 0.0; }
  for (int i = 0; i < kAeqNodes; ++i)
    aeq_node<double>(tb.gl_t[i], tb.gl_w[i], A, sh2, uinv, !(u > 0.0), g.nm, J3, J4);
  const double r = u > 0.0 ? A / u : 1.0;
  double sm = nn * r * 0.25;
  const double sgn = bb < 0.0 ? -1.0 : 1.0;
  for (int m = 0; m < g.nm; ++m) {
    const double h = sm * 0.5 * (2 * m + 1);
    const double d = J3[m] - TT * J4[m];
    for (int k = 0; k < g.QL; ++k)
      coef[(size_t)s * kMaxQL * kMaxM + k * kMaxM + m] = h * (J3[m] + tb.L1k[k] * d);
    sm *= sgn;
  }
}

template <typename T>
__global__ void sod_init_pop_kernel(SodGeom g, SodTablesF64 tb, const double* __restrict__ coef,
                                    T* f) {
  const size_t total = (size_t)g.V * g.Z;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int v = (int)(idx / g.Z), s = (int)(idx - (size_t)v * g.Z);
    const int k = tb.kidx[v];
    const double* c = coef + (size_t)s * kMaxQL * kMaxM + k * kMaxM;
    double acc = 0.0;
    for (int m = 0; m < g.nm; ++m) acc += c[m] * tb.wp[m * g.V + v];
    f[(size_t)v * g.ldz + s] = T(acc);
  }
}

template <typename T>
cudaError_t sod_init_launch(const SodGeom& g, const SodTablesF64& tb, const double* n,
                            const double* Tt, const double* beta, double* coef_scratch, T* f,
                            int* err, cudaStream_t st) {
  sod_init_coef_kernel<<<(g.Z + 127) / 128, 128, 0, st>>>(g, tb, n, Tt, beta, coef_scratch, err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sod_init_pop_kernel<T><<<1024, 256, 0, st>>>(g, tb, coef_scratch, f);
  return cudaGetLastError();
}

template cudaError_t sod_init_launch<float>(const SodGeom&, const SodTablesF64&, const double*,
                                            const double*, const double*, double*, float*, int*,
                                            cudaStream_t);
template cudaError_t sod_init_launch<double>(const SodGeom&, const SodTablesF64&, const double*,
                                             const double*, const double*, double*, double*,
                                             int*, cudaStream_t);

// ---------------------------------------------------------------------------
// Output moments: one warp per cell, FP64 sums.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void sod_moments_kernel(SodGeom g, SodTablesF64 tb, const T* __restrict__ f,
                                   double* out, int* err) {
  const int warps = blockDim.x >> 5;
  const int s = blockIdx.x * warps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= g.Z) return;
  double S[10];
  for (int q = 0; q < 10; ++q) S[q] = 0.0;
  for (int v = lane; v < g.V; v += 32) {
    const double x = (double)f[(size_t)v * g.ldz + s];
    const double xi = tb.xi[v], p = tb.p[v];
    S[0] += x;
    S[1] += x * xi;
    S[2] += x * p;
    S[3] += x * p * xi;
    S[4] += x * p * xi * xi;
    S[5] += x * (1.0 + xi);
    S[6] += x * (1.0 - xi);
    S[7] += x * p * (1.0 + xi) * (1.0 + xi);
    S[8] += x * p * (1.0 - xi) * (1.0 - xi);
    S[9] += x * p * (1.0 - xi) * (1.0 + xi);
  }
  for (int q = 0; q < 10; ++q) S[q] = warp_sum(S[q]);
  if (lane != 0) return;
  const LandauOut L = landau_factored(S[5], S[6], S[7], S[8], S[9]);
  if (!L.ok) report_error(err, 6, s);
  const size_t Z = g.Z;
  out[0 * Z + s] = L.n;
  out[1 * Z + s] = L.E;
  out[2 * Z + s] = L.E / 3.0;
  out[3 * Z + s] = L.T;
  out[4 * Z + s] = L.beta;
  out[5 * Z + s] = L.gamma;
  out[6 * Z + s] = L.n / (L.T * L.T * L.T);
  out[7 * Z + s] = -4.0 * L.T * (S[1] - L.n * L.beta * L.gamma);
  out[8 * Z + s] = 2.0 * L.E / 3.0 - S[9];
  for (int q = 0; q < 5; ++q) out[(9 + q) * Z + s] = S[q];
}

template <typename T>
cudaError_t sod_moments_launch(const SodGeom& g, const SodTablesF64& tb, const T* f,
                               double* out, int* err, cudaStream_t st) {
  sod_moments_kernel<T><<<(g.Z + 7) / 8, 256, 0, st>>>(g, tb, f, out, err);
  return cudaGetLastError();
}

template cudaError_t sod_moments_launch<float>(const SodGeom&, const SodTablesF64&, const float*,
                                               double*, int*, cudaStream_t);
template cudaError_t sod_moments_launch<double>(const SodGeom&, const SodTablesF64&,
                                                const double*, double*, int*, cudaStream_t);

}  // namespace rslb
