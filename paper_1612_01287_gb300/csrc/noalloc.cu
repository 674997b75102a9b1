// noalloc.cu -- rslb_sod_step_noalloc: the shock-tube step without any device
// allocation.
//
// The RK stage buffers, velocity tables and error word live in one static
// __device__ array of fixed size.  Each GPU that loads the library holds it
// until the process exits.  Host code never uses the array's name as an
// address: the device address is taken once per device with
// cudaGetSymbolAddress and cached.
#include <cmath>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/rslb.h"
#include "host_common.h"
#include "rslb_device.cuh"
#include "sod.cuh"

namespace rslb {

constexpr size_t kNoAllocScratchBytes = size_t(RSLB_NOALLOC_SCRATCH_BYTES);
constexpr int kNoAllocMaxV = RSLB_NOALLOC_MAX_VELOCITIES;
constexpr int kNoAllocMaxQL = 8;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[kNoAllocMaxDevices];

// Device address of the scratch array on the current device (set up on the
// first call per device).
static int noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "rslb_sod_step_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return set_error(RSLB_ERR_UNSUPPORTED, "rslb_sod_step_noalloc: device index %d too large",
                     dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    // the large-shared-memory opt-in of the stage kernels holds per device:
    // make it on this device before its first launch here
    e = sod_set_attributes();
    if (e != cudaSuccess)
      return cuda_error(e, "rslb_sod_step_noalloc: shared-memory opt-in of the stage kernels");
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return cuda_error(e, "rslb_sod_step_noalloc: cudaGetSymbolAddress of the scratch array");
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return RSLB_OK;
}

// Velocity tables of the Sod kernels, built on the device from the quadrature
// nodes (the same tables rslb_init uploads; here nothing is allocated).
template <typename T>
__global__ void noalloc_tables_kernel(int Qx, int QL, int nm, const double* __restrict__ q,
                                      T* mw, T* xi, T* wp, int* kidx, int* rowv, T* L1k,
                                      double* dxi, double* dp, double* dwp, double* dL1k) {
  // q = [xi(Qx) | w_xi(Qx) | x_k(QL) | w_k(QL)]
  const int V = Qx * QL;
  const double* xj = q;
  const double* wj = q + Qx;
  const double* xk = q + 2 * Qx;
  const double* wk = q + 2 * Qx + QL;
  const int half = Qx / 2;  // nodes with xi < 0 (symmetric rule)
  const int nneg = QL * half;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
    const int k = v / Qx, j = v - k * Qx;
    const double x = xj[j], p = xk[k];
    mw[0 * V + v] = T(1.0 + x);
    mw[1 * V + v] = T(1.0 - x);
    mw[2 * V + v] = T(p * (1.0 + x) * (1.0 + x));
    mw[3 * V + v] = T(p * (1.0 - x) * (1.0 - x));
    mw[4 * V + v] = T(p * (1.0 - x) * (1.0 + x));
    xi[v] = T(x);
    kidx[v] = k;
    dxi[v] = x;
    dp[v] = p;
    double p0 = 1.0, p1 = x;
    for (int m = 0; m < kMaxM; ++m) {
      const double pm = (m == 0) ? 1.0 : p1;
      const double val = (m < nm) ? wj[j] * wk[k] * pm : 0.0;
      wp[m * V + v] = T(val);
      dwp[m * V + v] = val;
      if (m >= 1) {
        const double p2 = ((2.0 * m + 1.0) * x * p1 - m * p0) / (m + 1.0);
        p0 = p1;
        p1 = p2;
      }
    }
    // row order: negative xi first, ascending v within each group
    int r;
    if (j < half) r = k * half + j;
    else r = nneg + k * (Qx - half) + (j - half);
    rowv[r] = v;
    if (v < QL) {
      L1k[v] = T(3.0 - xk[v]);
      dL1k[v] = 3.0 - xk[v];
    }
  }
}

template <typename T>
static int noalloc_run(const rslb_config& c, void* f, int nsteps, cudaStream_t st) {
  const int Qx = c.Q_xi, QL = c.Q_L, V = Qx * QL, nm = c.N_Omega + 1;
  const int ldz = (c.Z + 31) / 32 * 32;
  const size_t es = sizeof(T);
  // scratch layout (256-byte aligned blocks)
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  };
  const size_t oF0 = take(es * (size_t)V * ldz), oF1 = take(es * (size_t)V * ldz),
               oF2 = take(es * (size_t)V * ldz);
  const size_t omw = take(es * 5 * V), oxi = take(es * V), owp = take(es * kMaxM * V),
               oL1 = take(es * kNoAllocMaxQL), ogL = take(es * V), ogR = take(es * V),
               okidx = take(sizeof(int) * V), orow = take(sizeof(int) * V),
               oglt = take(sizeof(double) * kAeqTable), oglw = take(sizeof(double) * kAeqTable),
               odxi = take(sizeof(double) * V), odp = take(sizeof(double) * V),
               odwp = take(sizeof(double) * kMaxM * V), odL1 = take(sizeof(double) * kNoAllocMaxQL),
               oq = take(sizeof(double) * (2 * Qx + 2 * QL)), odg = take(sizeof(double) * 6),
               ogc = take(sizeof(double) * 2 * 8 * kMaxM), ogp = take(es * 2 * (size_t)V),
               oerr = take(sizeof(int) * 2);
  if (off > kNoAllocScratchBytes)
    return set_error(RSLB_ERR_UNSUPPORTED,
                     "rslb_sod_step_noalloc: this problem needs %zu bytes of scratch; the static "
                     "scratch array holds %zu (reduce Z or the velocity count)",
                     off, kNoAllocScratchBytes);

  // quadrature on the host (stack arrays; V <= kNoAllocMaxV was checked)
  double q[2 * kNoAllocMaxV + 2 * kNoAllocMaxQL];
  double glt[kAeqTable], glw[kAeqTable];
  gauss_legendre_host(Qx, q, q + Qx);
  gauss_laguerre2_host(QL, q + 2 * Qx, q + 2 * Qx + QL);
  gauss_legendre_host(kAeqNodes, glt, glw);
  gauss_legendre_host(kAeqNodesF32, glt + kAeqNodes, glw + kAeqNodes);
  const double dz = (c.z_max - c.z_min) / c.Z;
  double ximax = 0.0;
  for (int j = 0; j < Qx; ++j) ximax = std::fmax(ximax, std::fabs(q[j]));
  if (ximax * c.dt / dz >= 1.0)
    return set_error(RSLB_ERR_CFL, "rslb_sod_step_noalloc: CFL = %g >= 1", ximax * c.dt / dz);
  if (c.tau_mode == RSLB_TAU_CONST && c.dt >= c.tau)
    return set_error(RSLB_ERR_STIFF, "rslb_sod_step_noalloc: dt >= tau");

  // the tile shape, checked before any device work
  int dev = 0, max_smem = 0;
  cudaError_t qe = cudaGetDevice(&dev);
  if (qe == cudaSuccess)
    qe = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (qe != cudaSuccess) return cuda_error(qe, "rslb_sod_step_noalloc: device query");
  const SodLaunch L = sod_pick_launch(sizeof(T) == 8, V, QL, nm, max_smem);
  if (L.B == 0)
    return set_error(RSLB_ERR_UNSUPPORTED, "rslb_sod_step_noalloc: V = %d does not fit a tile", V);

  void* base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc) return rc;
  unsigned char* S = static_cast<unsigned char*>(base);
  T* F0 = (T*)(S + oF0);
  T* F1 = (T*)(S + oF1);
  T* F2 = (T*)(S + oF2);
  int* err = (int*)(S + oerr);

  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
    return e == cudaSuccess;
  };
  ok(cudaMemcpyAsync(S + oq, q, sizeof(double) * (2 * Qx + 2 * QL), cudaMemcpyHostToDevice, st));
  ok(cudaMemcpyAsync(S + oglt, glt, sizeof(glt), cudaMemcpyHostToDevice, st));
  ok(cudaMemcpyAsync(S + oglw, glw, sizeof(glw), cudaMemcpyHostToDevice, st));
  ok(cudaMemsetAsync(err, 0, 2 * sizeof(int), st));
  // tables must be in place before the pageable copies above are reused
  if (ok(cudaSuccess)) {
    noalloc_tables_kernel<T><<<(V + 255) / 256, 256, 0, st>>>(
        Qx, QL, nm, (const double*)(S + oq), (T*)(S + omw), (T*)(S + oxi), (T*)(S + owp),
        (int*)(S + okidx), (int*)(S + orow), (T*)(S + oL1), (double*)(S + odxi),
        (double*)(S + odp), (double*)(S + odwp), (double*)(S + odL1));
    ok(cudaGetLastError());
  }
  SodGeom g;
  g.Z = c.Z;
  g.ldz = ldz;
  g.V = V;
  g.Qx = Qx;
  g.QL = QL;
  g.nm = nm;
  g.bc = c.bc;
  g.tau_mode = c.tau_mode;
  g.inv_dz = 1.0 / dz;
  g.dt = c.dt;
  g.tau = c.tau;
  g.tau_AW0 = c.tau_AW0;
  g.lambda_ref = c.lambda_ref;
  SodTablesF64 t64;
  t64.xi = (const double*)(S + odxi);
  t64.p = (const double*)(S + odp);
  t64.wp = (const double*)(S + odwp);
  t64.kidx = (const int*)(S + okidx);
  t64.L1k = (const double*)(S + odL1);
  t64.gl_t = (const double*)(S + oglt);
  t64.gl_w = (const double*)(S + oglw);
  if (c.bc == RSLB_BC_FIXED_EQ) {
    const double hs[6] = {c.nL, c.nR, c.TL, c.TR, c.betaL, c.betaR};
    ok(cudaMemcpyAsync(S + odg, hs, sizeof(hs), cudaMemcpyHostToDevice, st));
    SodGeom g2 = g;
    g2.Z = 2;
    g2.ldz = 2;
    const double* dg = (const double*)(S + odg);
    if (ok(cudaSuccess))
      ok(sod_init_launch<T>(g2, t64, dg, dg + 2, dg + 4, (double*)(S + ogc), (T*)(S + ogp), err,
                            st));
    ok(cudaMemcpy2DAsync(S + ogL, es, S + ogp, 2 * es, es, V, cudaMemcpyDeviceToDevice, st));
    ok(cudaMemcpy2DAsync(S + ogR, es, S + ogp + es, 2 * es, es, V, cudaMemcpyDeviceToDevice, st));
  } else {
    ok(cudaMemsetAsync(S + ogL, 0, es * V, st));
    ok(cudaMemsetAsync(S + ogR, 0, es * V, st));
  }
  SodTables<T> tb;
  tb.mw = (const T*)(S + omw);
  tb.xi = (const T*)(S + oxi);
  tb.wp = (const T*)(S + owp);
  tb.kidx = (const int*)(S + okidx);
  tb.L1k = (const T*)(S + oL1);
  tb.ghostL = (const T*)(S + ogL);
  tb.ghostR = (const T*)(S + ogR);
  tb.gl_t = (const double*)(S + oglt);
  tb.gl_w = (const double*)(S + oglw);
  const int nneg = QL * (Qx / 2);

  // caller's populations (pitch Z) into the padded stage buffer
  ok(cudaMemcpy2DAsync(F0, es * ldz, f, es * c.Z, es * c.Z, V, cudaMemcpyDeviceToDevice, st));
  for (int n = 0; n < nsteps && e == cudaSuccess; ++n) {
    ok(sod_stage_launch<T>(L, g, tb, (const int*)(S + orow), nneg, F0, F0, F1, 0, err, st));
    ok(sod_stage_launch<T>(L, g, tb, (const int*)(S + orow), nneg, F1, F0, F2, 1, err, st));
    ok(sod_stage_launch<T>(L, g, tb, (const int*)(S + orow), nneg, F2, F0, F0, 2, err, st));
  }
  ok(cudaMemcpy2DAsync(f, es * c.Z, F0, es * ldz, es * c.Z, V, cudaMemcpyDeviceToDevice, st));
  int herr[2] = {0, 0};
  ok(cudaMemcpyAsync(herr, err, sizeof(herr), cudaMemcpyDeviceToHost, st));
  ok(cudaStreamSynchronize(st));
  if (e != cudaSuccess) return cuda_error(e, "rslb_sod_step_noalloc");
  if (herr[0] != 0)
    return set_error(RSLB_ERR_NONPHYSICAL,
                     "rslb_sod_step_noalloc: non-physical state in cell %d", herr[1]);
  return RSLB_OK;
}

}  // namespace rslb

using namespace rslb;

extern "C" int rslb_sod_step_noalloc(const rslb_config* cfg, void* f, int nsteps, void* stream) {
  clear_error();
  if (!cfg || !f || nsteps < 0)
    return set_error(RSLB_ERR_ARG, "rslb_sod_step_noalloc: NULL argument or nsteps < 0");
  const rslb_config& c = *cfg;
  if (c.Z < 1 || !(c.z_max > c.z_min) || c.Q_xi < 1 || c.Q_L < 1 || c.Q_L > kNoAllocMaxQL ||
      c.N_Omega < 0 || c.N_Omega > kMaxM - 1 || c.N_Omega >= c.Q_xi ||
      (c.precision != RSLB_F32 && c.precision != RSLB_F64) || c.bc < 0 || c.bc > 2 ||
      c.tau_mode < 0 || c.tau_mode > 2 || !(c.dt > 0.0) || !std::isfinite(c.dt) ||
      (c.tau_mode == RSLB_TAU_CONST && !(c.tau > 0.0)) ||
      (c.tau_mode == RSLB_TAU_ETAS && !(c.tau_AW0 > 0.0 && c.lambda_ref > 0.0)) ||
      (c.bc == RSLB_BC_PERIODIC && c.Z < 6))
    return set_error(RSLB_ERR_ARG, "rslb_sod_step_noalloc: invalid configuration");
  if ((long long)c.Q_xi * c.Q_L > kNoAllocMaxV)
    return set_error(RSLB_ERR_UNSUPPORTED,
                     "rslb_sod_step_noalloc: Q_xi*Q_L = %d exceeds the limit of %d velocities",
                     c.Q_xi * c.Q_L, kNoAllocMaxV);
  cudaStream_t st = (cudaStream_t)stream;
  return c.precision == RSLB_F64 ? noalloc_run<double>(c, f, nsteps, st)
                                 : noalloc_run<float>(c, f, nsteps, st);
}
