// host.cu -- C ABI of the R-SLB library (include/rslb.h): argument checks,
// FP64 quadrature generation, velocity tables, device buffers and launches.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/rslb.h"
#include "host_common.h"
#include "rslb_device.cuh"
#include "sod.cuh"

namespace rslb {

static thread_local char g_err[512] = "";

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

void clear_error() { g_err[0] = '\0'; }
const char* last_error() { return g_err; }

int cuda_error(cudaError_t e, const char* what) {
  return set_error(RSLB_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// Gauss-Legendre (Sec. III C): Newton on P_Q from Tricomi's initial guess,
// weights 2/((1 - x^2) P'_Q(x)^2), which equals the printed
// 2(1 - x^2)/[(Q+1) P_{Q+1}(x)]^2 at the roots and is better conditioned.
// ---------------------------------------------------------------------------
static void legendre_pq(int Q, double x, double* pq, double* pqm1) {
  double a = 1.0, b = x;  // P_0, P_1
  if (Q == 0) { *pq = 1.0; *pqm1 = 0.0; return; }
  for (int n = 2; n <= Q; ++n) {
    const double c = ((2 * n - 1) * x * b - (n - 1) * a) / n;
    a = b;
    b = c;
  }
  *pq = b;
  *pqm1 = a;
}

int gauss_legendre_host(int Q, double* x, double* w) {
  if (Q < 1) return RSLB_ERR_ARG;
  const double pi = 3.14159265358979323846;
  const int half = Q / 2;
  for (int i = 1; i <= half; ++i) {
    const double th = pi * (4.0 * i - 1.0) / (4.0 * Q + 2.0);
    double z = (1.0 - (Q - 1.0) / (8.0 * Q * Q * Q)) * std::cos(th);
    for (int it = 0; it < 100; ++it) {
      double pq, pm;
      legendre_pq(Q, z, &pq, &pm);
      const double dp = Q * (pm - z * pq) / ((1.0 - z) * (1.0 + z));
      const double step = pq / dp;
      z -= step;
      if (std::fabs(step) < 1e-15) {
        legendre_pq(Q, z, &pq, &pm);
        z -= pq / (Q * (pm - z * pq) / ((1.0 - z) * (1.0 + z)));
        break;
      }
    }
    double pq, pm;
    legendre_pq(Q, z, &pq, &pm);
    const double dp = Q * (pm - z * pq) / ((1.0 - z) * (1.0 + z));
    const double wi = 2.0 / ((1.0 - z) * (1.0 + z) * dp * dp);
    x[Q - i] = z;
    x[i - 1] = -z;
    w[Q - i] = wi;
    w[i - 1] = wi;
  }
  if (Q & 1) {
    double pq, pm;
    legendre_pq(Q, 0.0, &pq, &pm);
    const double dp = Q * pm;  // P'_Q(0) = Q P_{Q-1}(0)
    x[half] = 0.0;
    w[half] = 2.0 / (dp * dp);
  }
  return RSLB_OK;
}

// ---------------------------------------------------------------------------
// Gauss-Laguerre for the weight e^{-x} x^2 (Sec. III B): eigenvalues of the
// symmetric Jacobi matrix of the L^{(2)} recurrence (diagonal 2i+3,
// off-diagonal sqrt(i(i+2))) by cyclic Jacobi rotations, polished by Newton;
// weights (Q+1)(Q+2)/(x L'_Q(x)^2), equal to the printed
// x(Q+2)/((Q+1)[L_{Q+1}(x)]^2) at the roots.
// ---------------------------------------------------------------------------
static void laguerre2_ql(int Q, double x, double* lq, double* lqm1) {
  double a = 1.0, b = 3.0 - x;  // L_0, L_1 for alpha = 2
  if (Q == 0) { *lq = 1.0; *lqm1 = 0.0; return; }
  for (int n = 1; n < Q; ++n) {
    const double c = ((2.0 * n + 3.0 - x) * b - (n + 2.0) * a) / (n + 1.0);
    a = b;
    b = c;
  }
  *lq = b;
  *lqm1 = a;
}

int gauss_laguerre2_host(int Q, double* x, double* w) {
  if (Q < 1 || Q > 12) return RSLB_ERR_ARG;
  double M[12][12];
  for (int i = 0; i < Q; ++i)
    for (int j = 0; j < Q; ++j) M[i][j] = 0.0;
  for (int i = 0; i < Q; ++i) M[i][i] = 2.0 * i + 3.0;
  for (int i = 1; i < Q; ++i) M[i][i - 1] = M[i - 1][i] = std::sqrt(i * (i + 2.0));
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < Q; ++p)
      for (int q = p + 1; q < Q; ++q) off += M[p][q] * M[p][q];
    if (off < 1e-30) break;
    for (int p = 0; p < Q; ++p)
      for (int q = p + 1; q < Q; ++q) {
        if (std::fabs(M[p][q]) < 1e-300) continue;
        const double th = 0.5 * (M[q][q] - M[p][p]) / M[p][q];
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < Q; ++k) {
          const double mkp = M[k][p], mkq = M[k][q];
          M[k][p] = c * mkp - s * mkq;
          M[k][q] = s * mkp + c * mkq;
        }
        for (int k = 0; k < Q; ++k) {
          const double mpk = M[p][k], mqk = M[q][k];
          M[p][k] = c * mpk - s * mqk;
          M[q][k] = s * mpk + c * mqk;
        }
      }
  }
  for (int i = 0; i < Q; ++i) x[i] = M[i][i];
  // sort ascending
  for (int i = 1; i < Q; ++i)
    for (int j = i; j > 0 && x[j] < x[j - 1]; --j) std::swap(x[j], x[j - 1]);
  for (int i = 0; i < Q; ++i) {
    double z = x[i];
    for (int it = 0; it < 4; ++it) {
      double lq, lm;
      laguerre2_ql(Q, z, &lq, &lm);
      const double d = (Q * lq - (Q + 2.0) * lm) / z;
      z -= lq / d;
    }
    double lq, lm;
    laguerre2_ql(Q, z, &lq, &lm);
    const double d = (Q * lq - (Q + 2.0) * lm) / z;
    x[i] = z;
    w[i] = (Q + 1.0) * (Q + 2.0) / (z * d * d);
  }
  return RSLB_OK;
}

double legendre_p(int m, double x) {
  double pq, pm;
  legendre_pq(m, x, &pq, &pm);
  return pq;
}

}  // namespace rslb

using namespace rslb;

extern "C" const char* rslb_last_error(void) { return rslb::last_error(); }

extern "C" int rslb_quadrature(int Q_xi, int Q_L, double* xi, double* w_xi, double* xk,
                               double* w_L) {
  clear_error();
  if (xi || w_xi) {
    if (!xi || !w_xi || Q_xi < 1 || Q_xi > 4096)
      return set_error(RSLB_ERR_ARG, "rslb_quadrature: need 1 <= Q_xi <= 4096 and both arrays");
    gauss_legendre_host(Q_xi, xi, w_xi);
  }
  if (xk || w_L) {
    if (!xk || !w_L || Q_L < 1 || Q_L > 12)
      return set_error(RSLB_ERR_ARG, "rslb_quadrature: need 1 <= Q_L <= 12 and both arrays");
    gauss_laguerre2_host(Q_L, xk, w_L);
  }
  return RSLB_OK;
}

// ---------------------------------------------------------------------------
// Sod handle
// ---------------------------------------------------------------------------
struct rslb_handle {
  rslb_config cfg;
  int V, ldz, nm;
  bool fp64;
  cudaStream_t stream;
  SodGeom geom;
  SodLaunch launch;
  void* F[3];
  // tables in working precision
  void* t_mw;
  void* t_xi;
  void* t_wp;
  void* t_L1k;
  void* t_gL;
  void* t_gR;
  int* t_kidx;
  int* t_rowv;
  int nneg;
  double* t_gl_t;
  double* t_gl_w;
  // FP64 tables
  double* d_xi;
  double* d_p;
  double* d_wp;
  double* d_L1k;
  void* d_mom;  // output-moment weights (sod_moment_weights)
  int* d_err;
  double* d_fields;
  double t;
  long long steps;
  // CUDA graph of kGraphSteps steps (3 stage launches each), captured on the
  // handle's stream the first time rslb_step is asked for that many steps
  cudaGraphExec_t graph;
  bool graph_failed;
};

static constexpr int kGraphSteps = 8;

namespace {

template <typename T>
SodTables<T> tables_of(const rslb_handle* h) {
  SodTables<T> tb;
  tb.mw = (const T*)h->t_mw;
  tb.xi = (const T*)h->t_xi;
  tb.wp = (const T*)h->t_wp;
  tb.kidx = h->t_kidx;
  tb.L1k = (const T*)h->t_L1k;
  tb.ghostL = (const T*)h->t_gL;
  tb.ghostR = (const T*)h->t_gR;
  tb.gl_t = h->t_gl_t;
  tb.gl_w = h->t_gl_w;
  return tb;
}

SodTablesF64 tables64_of(const rslb_handle* h) {
  SodTablesF64 tb;
  tb.xi = h->d_xi;
  tb.p = h->d_p;
  tb.wp = h->d_wp;
  tb.kidx = h->t_kidx;
  tb.L1k = h->d_L1k;
  tb.gl_t = h->t_gl_t;
  tb.gl_w = h->t_gl_w;
  return tb;
}

void free_handle(rslb_handle* h) {
  if (!h) return;
  if (h->graph) cudaGraphExecDestroy(h->graph);
  void* ptrs[] = {h->F[0], h->F[1], h->F[2], h->t_mw, h->t_xi, h->t_wp, h->t_L1k, h->t_gL,
                  h->t_gR, h->t_kidx, h->t_rowv, h->t_gl_t, h->t_gl_w, h->d_xi, h->d_p, h->d_wp,
                  h->d_L1k, h->d_mom, h->d_err, h->d_fields};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete h;
}

int check_device_error(rslb_handle* h) {
  int herr[2] = {0, 0};
  cudaError_t e = cudaMemcpyAsync(herr, h->d_err, sizeof(herr), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_error(e, "synchronising the stream");
  if (herr[0] != 0) {
    cudaMemsetAsync(h->d_err, 0, 2 * sizeof(int), h->stream);
    cudaStreamSynchronize(h->stream);
    if (herr[0] == RSLB_ERR_TIMEOUT)
      return set_error(RSLB_ERR_TIMEOUT, "a bounded wait in a stage kernel ran out (tile at cell %d)",
                       herr[1]);
    return set_error(RSLB_ERR_NONPHYSICAL,
                     "non-physical state (n, E <= 0, |beta| >= 1 or non-finite) in cell %d",
                     herr[1]);
  }
  return RSLB_OK;
}

template <typename T>
int upload(void** dst, const std::vector<double>& src) {
  std::vector<T> tmp(src.begin(), src.end());
  if (cudaMalloc(dst, sizeof(T) * tmp.size() + 16) != cudaSuccess)
    return set_error(RSLB_ERR_ALLOC, "cudaMalloc of a table failed");
  if (cudaMemcpy(*dst, tmp.data(), sizeof(T) * tmp.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return set_error(RSLB_ERR_CUDA, "copying a table to the device failed");
  return RSLB_OK;
}

int upload_int(int** dst, const std::vector<int>& src) {
  if (cudaMalloc((void**)dst, sizeof(int) * src.size() + 16) != cudaSuccess)
    return set_error(RSLB_ERR_ALLOC, "cudaMalloc of a table failed");
  if (cudaMemcpy(*dst, src.data(), sizeof(int) * src.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return set_error(RSLB_ERR_CUDA, "copying a table to the device failed");
  return RSLB_OK;
}

}  // namespace

extern "C" int rslb_init(rslb_handle** out, const rslb_config* cfg, void* stream) {
  clear_error();
  if (!out || !cfg) return set_error(RSLB_ERR_ARG, "rslb_init: NULL argument");
  *out = nullptr;
  const rslb_config& c = *cfg;
  if (c.Z < 1 || !(c.z_max > c.z_min) || c.Q_xi < 1 || c.Q_xi > 2048 || c.Q_L < 1 ||
      c.Q_L > 8 || c.N_Omega < 0 || c.N_Omega > kMaxM - 1 || c.N_Omega >= c.Q_xi ||
      (c.precision != RSLB_F32 && c.precision != RSLB_F64) || c.bc < 0 || c.bc > 2 ||
      c.tau_mode < 0 || c.tau_mode > 2 || !(c.dt > 0.0) || !std::isfinite(c.dt))
    return set_error(RSLB_ERR_ARG,
                     "rslb_init: invalid configuration (need Z >= 1, z_max > z_min, "
                     "1 <= Q_xi <= 2048, 1 <= Q_L <= 8, 0 <= N_Omega < min(Q_xi, 13), "
                     "known precision/bc/tau_mode, dt > 0)");
  if (c.tau_mode == RSLB_TAU_CONST && !(c.tau > 0.0))
    return set_error(RSLB_ERR_ARG, "rslb_init: tau must be > 0");
  if (c.tau_mode == RSLB_TAU_ETAS && !(c.tau_AW0 > 0.0 && c.lambda_ref > 0.0))
    return set_error(RSLB_ERR_ARG, "rslb_init: tau_AW0 and lambda_ref must be > 0");
  if (c.bc == RSLB_BC_PERIODIC && c.Z < 6)
    return set_error(RSLB_ERR_ARG, "rslb_init: periodic domains need Z >= 6");
  const int Qx = c.Q_xi, QL = c.Q_L, V = Qx * QL, nm = c.N_Omega + 1;
  // the kernels index a population buffer [V][ldz] with 32-bit offsets in places
  if ((long long)V * (((long long)c.Z + 31) / 32 * 32) >= (1LL << 31))
    return set_error(RSLB_ERR_UNSUPPORTED,
                     "rslb_init: V x Z = %d x %d populations per buffer (limit 2^31)", V, c.Z);
  std::vector<double> xj(Qx), wj(Qx), xk(QL), wk(QL), glt(kAeqTable), glw(kAeqTable);
  gauss_legendre_host(Qx, xj.data(), wj.data());
  gauss_laguerre2_host(QL, xk.data(), wk.data());
  gauss_legendre_host(kAeqNodes, glt.data(), glw.data());
  gauss_legendre_host(kAeqNodesF32, glt.data() + kAeqNodes, glw.data() + kAeqNodes);
  const double dz = (c.z_max - c.z_min) / c.Z;
  double ximax = 0.0;
  for (double v : xj) ximax = std::fmax(ximax, std::fabs(v));
  if (ximax * c.dt / dz >= 1.0)
    return set_error(RSLB_ERR_CFL, "rslb_init: CFL = max|xi| dt/dz = %g >= 1", ximax * c.dt / dz);
  if (c.tau_mode == RSLB_TAU_CONST && c.dt >= c.tau)
    return set_error(RSLB_ERR_STIFF, "rslb_init: dt = %g >= tau = %g (explicit RK3 is stiff)",
                     c.dt, c.tau);

  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return cuda_error(ce, "cudaGetDevice");
  int max_smem = 0;
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  ce = sod_set_attributes();
  if (ce != cudaSuccess) return cuda_error(ce, "rslb_init: kernel attributes");
  const bool fp64 = c.precision == RSLB_F64;
  SodLaunch L = sod_pick_launch(fp64, V, QL, nm, max_smem);
  if (c.tile_cells != 0) {
    // explicit tile width (tuning): must be one the kernels are built for
    const bool okB = fp64 ? (c.tile_cells == 16 || c.tile_cells == 8)
                          : (c.tile_cells == kSod32Cells || c.tile_cells == 128 || c.tile_cells == 64 ||
                             c.tile_cells == 32 || c.tile_cells == 16);
    if (!okB)
      return set_error(RSLB_ERR_ARG, "rslb_init: tile_cells must be 0 or one of %s",
                       fp64 ? "16, 8" : "the packed width, 128, 64, 32, 16");
    if (c.tile_cells == kSod32Cells && (V < 128 || nm > 8))
      return set_error(RSLB_ERR_ARG,
                       "rslb_init: the packed tile width needs V >= 128 and N_Omega <= 7");
    L.B = c.tile_cells;
  }
  if (L.B == 0)
    return set_error(RSLB_ERR_UNSUPPORTED, "rslb_init: V = %d velocities do not fit one tile", V);
  if (c.packed_form < RSLB_PACKED_AUTO || c.packed_form > RSLB_PACKED_PERSISTENT)
    return set_error(RSLB_ERR_ARG, "rslb_init: unknown packed_form %d", c.packed_form);
  if (L.B == kSod32Cells && c.packed_form == RSLB_PACKED_PERSISTENT) {
    // the persistent pipelined form on request (the population buffers are
    // cudaMalloc'd, so 16-byte aligned for its bulk-tensor copies); measured
    // slower than two CTAs per SM of the per-tile form, so not the default
    SodGeom gq;
    std::memset(&gq, 0, sizeof(gq));
    gq.Z = c.Z;
    gq.ldz = (c.Z + 31) / 32 * 32;
    gq.V = V;
    gq.QL = QL;
    gq.nm = nm;
    int nsm = 0;
    ce = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (ce != cudaSuccess) return cuda_error(ce, "rslb_init: SM count");
    if (!sod32p_fits(gq, max_smem))
      return set_error(RSLB_ERR_ARG,
                       "rslb_init: the persistent packed kernel does not fit (V = %d, Z = %d)", V,
                       c.Z);
    L.form = 1;
    L.nsm = nsm;
  } else if (c.packed_form == RSLB_PACKED_PERSISTENT) {
    return set_error(RSLB_ERR_ARG, "rslb_init: packed_form needs the packed FP32 kernel");
  }

  rslb_handle* h = new rslb_handle();
  std::memset((void*)h, 0, sizeof(*h));
  h->cfg = c;
  h->cfg.n0 = h->cfg.T0 = h->cfg.beta0 = nullptr;
  h->V = V;
  h->nm = nm;
  h->fp64 = fp64;
  h->stream = (cudaStream_t)stream;
  h->ldz = (c.Z + 31) / 32 * 32;
  h->launch = L;
  SodGeom& g = h->geom;
  g.Z = c.Z;
  g.ldz = h->ldz;
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

  // velocity tables (FP64 on the host)
  std::vector<double> mw(5 * (size_t)V), xiv(V), pv(V), wp(kMaxM * (size_t)V, 0.0), L1k(QL);
  std::vector<int> kidx(V);
  for (int k = 0; k < QL; ++k) {
    L1k[k] = 3.0 - xk[k];
    for (int j = 0; j < Qx; ++j) {
      const int v = k * Qx + j;
      const double x = xj[j], p = xk[k];
      mw[0 * V + v] = 1.0 + x;
      mw[1 * V + v] = 1.0 - x;
      mw[2 * V + v] = p * (1.0 + x) * (1.0 + x);
      mw[3 * V + v] = p * (1.0 - x) * (1.0 - x);
      mw[4 * V + v] = p * (1.0 - x) * (1.0 + x);
      xiv[v] = x;
      pv[v] = p;
      kidx[v] = k;
      for (int m = 0; m < nm; ++m) wp[(size_t)m * V + v] = wj[j] * wk[k] * legendre_p(m, x);
    }
  }
  // rows ordered negative-xi first (ascending v within each group)
  std::vector<int> rowv;
  rowv.reserve(V);
  for (int v = 0; v < V; ++v)
    if (xiv[v] < 0.0) rowv.push_back(v);
  h->nneg = (int)rowv.size();
  for (int v = 0; v < V; ++v)
    if (!(xiv[v] < 0.0)) rowv.push_back(v);
  std::vector<double> zeros(V, 0.0);
  int rc = RSLB_OK;
  auto up = [&](void** dst, const std::vector<double>& src) {
    return fp64 ? upload<double>(dst, src) : upload<float>(dst, src);
  };
  if (!rc) rc = up(&h->t_mw, mw);
  if (!rc) rc = up(&h->t_xi, xiv);
  if (!rc) rc = up(&h->t_wp, wp);
  if (!rc) rc = up(&h->t_L1k, L1k);
  if (!rc) rc = up(&h->t_gL, zeros);
  if (!rc) rc = up(&h->t_gR, zeros);
  if (!rc) rc = upload_int(&h->t_kidx, kidx);
  if (!rc) rc = upload_int(&h->t_rowv, rowv);
  if (!rc) rc = upload<double>((void**)&h->t_gl_t, glt);
  if (!rc) rc = upload<double>((void**)&h->t_gl_w, glw);
  if (!rc) rc = upload<double>((void**)&h->d_xi, xiv);
  if (!rc) rc = upload<double>((void**)&h->d_p, pv);
  if (!rc) rc = upload<double>((void**)&h->d_wp, wp);
  if (!rc) rc = upload<double>((void**)&h->d_L1k, L1k);
  if (!rc) {
    std::vector<unsigned char> mom(sod_moment_weights(fp64, V, xiv.data(), pv.data(), nullptr));
    sod_moment_weights(fp64, V, xiv.data(), pv.data(), mom.data());
    if (cudaMalloc(&h->d_mom, mom.size()) != cudaSuccess)
      rc = set_error(RSLB_ERR_ALLOC, "cudaMalloc of a table failed");
    else if (cudaMemcpy(h->d_mom, mom.data(), mom.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      rc = set_error(RSLB_ERR_CUDA, "copying a table to the device failed");
  }
  const size_t es = fp64 ? sizeof(double) : sizeof(float);
  const size_t fbytes = es * (size_t)V * h->ldz;
  for (int i = 0; i < 3 && !rc; ++i) {
    if (cudaMalloc(&h->F[i], fbytes) != cudaSuccess)
      rc = set_error(RSLB_ERR_ALLOC, "rslb_init: cannot allocate %zu bytes of populations", fbytes);
    else
      cudaMemsetAsync(h->F[i], 0, fbytes, h->stream);
  }
  if (!rc && cudaMalloc((void**)&h->d_err, 2 * sizeof(int)) != cudaSuccess)
    rc = set_error(RSLB_ERR_ALLOC, "rslb_init: cudaMalloc failed");
  if (!rc && cudaMalloc((void**)&h->d_fields, sizeof(double) * RSLB_NFIELDS * (size_t)c.Z) !=
                 cudaSuccess)
    rc = set_error(RSLB_ERR_ALLOC, "rslb_init: cudaMalloc failed");
  if (rc) {
    free_handle(h);
    return rc;
  }
  cudaMemsetAsync(h->d_err, 0, 2 * sizeof(int), h->stream);

  // FIXED_EQ ghost populations: the truncated f^eq of the left/right states,
  // built by the same initialisation kernels on a two-cell geometry
  if (c.bc == RSLB_BC_FIXED_EQ) {
    double* dg = nullptr;
    double* gcoef = nullptr;
    void* gpop = nullptr;
    const double hs[6] = {c.nL, c.nR, c.TL, c.TR, c.betaL, c.betaR};
    cudaError_t ge = cudaMalloc((void**)&dg, sizeof(hs));
    if (ge == cudaSuccess) ge = cudaMalloc((void**)&gcoef, sizeof(double) * 2 * 8 * kMaxM);
    if (ge == cudaSuccess) ge = cudaMalloc(&gpop, es * 2 * (size_t)V);
    if (ge == cudaSuccess) ge = cudaMemcpy(dg, hs, sizeof(hs), cudaMemcpyHostToDevice);
    SodGeom g2 = g;
    g2.Z = 2;
    g2.ldz = 2;
    if (ge == cudaSuccess)
      ge = fp64 ? sod_init_launch<double>(g2, tables64_of(h), dg, dg + 2, dg + 4, gcoef,
                                          (double*)gpop, h->d_err, h->stream)
                : sod_init_launch<float>(g2, tables64_of(h), dg, dg + 2, dg + 4, gcoef,
                                         (float*)gpop, h->d_err, h->stream);
    if (ge == cudaSuccess)
      ge = cudaMemcpy2DAsync(h->t_gL, es, gpop, 2 * es, es, V, cudaMemcpyDeviceToDevice, h->stream);
    if (ge == cudaSuccess)
      ge = cudaMemcpy2DAsync(h->t_gR, es, (char*)gpop + es, 2 * es, es, V,
                             cudaMemcpyDeviceToDevice, h->stream);
    if (ge == cudaSuccess) ge = cudaStreamSynchronize(h->stream);
    if (dg) cudaFree(dg);
    if (gcoef) cudaFree(gcoef);
    if (gpop) cudaFree(gpop);
    if (ge != cudaSuccess) {
      free_handle(h);
      return cuda_error(ge, "rslb_init: ghost equilibria");
    }
    if (check_device_error(h) != RSLB_OK) {
      free_handle(h);
      return set_error(RSLB_ERR_NONPHYSICAL, "rslb_init: a boundary state is not physical");
    }
  }

  // initial fields per cell
  std::vector<double> n0(c.Z), T0(c.Z), b0(c.Z);
  const bool given = c.n0 && c.T0 && c.beta0;
  for (int s = 0; s < c.Z; ++s) {
    if (given) {
      n0[s] = c.n0[s];
      T0[s] = c.T0[s];
      b0[s] = c.beta0[s];
    } else {
      const double z = c.z_min + (s + 0.5) * dz;
      const bool left = z < 0.0;
      n0[s] = left ? c.nL : c.nR;
      T0[s] = left ? c.TL : c.TR;
      b0[s] = left ? c.betaL : c.betaR;
    }
  }
  double *dn = nullptr, *coef = nullptr;
  if (cudaMalloc((void**)&dn, sizeof(double) * 3 * (size_t)c.Z) != cudaSuccess ||
      cudaMalloc((void**)&coef, sizeof(double) * (size_t)c.Z * 8 * kMaxM) != cudaSuccess) {
    if (dn) cudaFree(dn);
    free_handle(h);
    return set_error(RSLB_ERR_ALLOC, "rslb_init: cannot allocate initialisation scratch");
  }
  cudaMemcpy(dn, n0.data(), sizeof(double) * c.Z, cudaMemcpyHostToDevice);
  cudaMemcpy(dn + c.Z, T0.data(), sizeof(double) * c.Z, cudaMemcpyHostToDevice);
  cudaMemcpy(dn + 2 * (size_t)c.Z, b0.data(), sizeof(double) * c.Z, cudaMemcpyHostToDevice);
  cudaError_t e;
  if (fp64)
    e = sod_init_launch<double>(g, tables64_of(h), dn, dn + c.Z, dn + 2 * c.Z, coef,
                                (double*)h->F[0], h->d_err, h->stream);
  else
    e = sod_init_launch<float>(g, tables64_of(h), dn, dn + c.Z, dn + 2 * c.Z, coef,
                               (float*)h->F[0], h->d_err, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(dn);
  cudaFree(coef);
  if (e != cudaSuccess) {
    free_handle(h);
    return cuda_error(e, "rslb_init: initialisation kernels");
  }
  rc = check_device_error(h);
  if (rc) {
    free_handle(h);
    return set_error(RSLB_ERR_NONPHYSICAL, "rslb_init: an initial state is not physical");
  }
  *out = h;
  return RSLB_OK;
}

template <typename T>
static cudaError_t enqueue_steps(rslb_handle* h, int nsteps) {
  const SodTables<T> tb = tables_of<T>(h);
  T* F0 = (T*)h->F[0];
  T* F1 = (T*)h->F[1];
  T* F2 = (T*)h->F[2];
  for (int n = 0; n < nsteps; ++n) {
    cudaError_t e;
    e = sod_stage_launch<T>(h->launch, h->geom, tb, h->t_rowv, h->nneg, F0, F0, F1, 0, h->d_err,
                            h->stream);
    if (e != cudaSuccess) return e;
    e = sod_stage_launch<T>(h->launch, h->geom, tb, h->t_rowv, h->nneg, F1, F0, F2, 1, h->d_err,
                            h->stream);
    if (e != cudaSuccess) return e;
    e = sod_stage_launch<T>(h->launch, h->geom, tb, h->t_rowv, h->nneg, F2, F0, F0, 2, h->d_err,
                            h->stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Capture kGraphSteps steps into an executable graph (non-default streams only:
// the legacy default stream cannot be captured).
static cudaError_t build_graph(rslb_handle* h) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t le =
      h->fp64 ? enqueue_steps<double>(h, kGraphSteps) : enqueue_steps<float>(h, kGraphSteps);
  e = cudaStreamEndCapture(h->stream, &g);
  if (le != cudaSuccess) e = le;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  return e;
}

extern "C" int rslb_step(rslb_handle* h, int nsteps) {
  clear_error();
  if (!h || nsteps < 0) return set_error(RSLB_ERR_ARG, "rslb_step: bad handle or nsteps");
  cudaError_t e = cudaSuccess;
  int rest = nsteps;
  if (h->stream != nullptr && nsteps >= kGraphSteps && !h->graph_failed) {
    if (!h->graph) {
      e = build_graph(h);
      if (e != cudaSuccess) {
        // fall back to plain launches (e.g. the caller's stream is being captured)
        h->graph = nullptr;
        h->graph_failed = true;
        cudaGetLastError();
        e = cudaSuccess;
      }
    }
    while (h->graph && rest >= kGraphSteps && e == cudaSuccess) {
      e = cudaGraphLaunch(h->graph, h->stream);
      rest -= kGraphSteps;
    }
  }
  if (e == cudaSuccess && rest > 0)
    e = h->fp64 ? enqueue_steps<double>(h, rest) : enqueue_steps<float>(h, rest);
  if (e != cudaSuccess) return cuda_error(e, "rslb_step: launch");
  h->steps += nsteps;
  h->t = h->steps * h->cfg.dt;
  return RSLB_OK;
}

extern "C" int rslb_sync(rslb_handle* h) {
  clear_error();
  if (!h) return set_error(RSLB_ERR_ARG, "rslb_sync: NULL handle");
  return check_device_error(h);
}

extern "C" int rslb_moments(rslb_handle* h, double* out, int out_on_device) {
  clear_error();
  if (!h || !out) return set_error(RSLB_ERR_ARG, "rslb_moments: NULL argument");
  cudaError_t e = h->fp64 ? sod_moments_launch<double>(h->geom, h->d_mom,
                                                       (const double*)h->F[0], h->d_fields,
                                                       h->d_err, h->stream)
                          : sod_moments_launch<float>(h->geom, h->d_mom,
                                                      (const float*)h->F[0], h->d_fields,
                                                      h->d_err, h->stream);
  if (e != cudaSuccess) return cuda_error(e, "rslb_moments: launch");
  const size_t bytes = sizeof(double) * RSLB_NFIELDS * (size_t)h->cfg.Z;
  e = cudaMemcpyAsync(out, h->d_fields, bytes,
                      out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                      h->stream);
  if (e != cudaSuccess) return cuda_error(e, "rslb_moments: copy");
  return check_device_error(h);
}

extern "C" int rslb_get_state(rslb_handle* h, void* f, int on_device) {
  clear_error();
  if (!h || !f) return set_error(RSLB_ERR_ARG, "rslb_get_state: NULL argument");
  const size_t es = h->fp64 ? sizeof(double) : sizeof(float);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  // one linear copy when the rows are not padded
  cudaError_t e = h->ldz == h->cfg.Z
                      ? cudaMemcpyAsync(f, h->F[0], es * (size_t)h->cfg.Z * h->V, kind, h->stream)
                      : cudaMemcpy2DAsync(f, es * h->cfg.Z, h->F[0], es * h->ldz, es * h->cfg.Z,
                                          h->V, kind, h->stream);
  if (e != cudaSuccess) return cuda_error(e, "rslb_get_state: copy");
  return check_device_error(h);
}

extern "C" int rslb_set_state(rslb_handle* h, const void* f, int on_device) {
  clear_error();
  if (!h || !f) return set_error(RSLB_ERR_ARG, "rslb_set_state: NULL argument");
  const size_t es = h->fp64 ? sizeof(double) : sizeof(float);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e = h->ldz == h->cfg.Z
                      ? cudaMemcpyAsync(h->F[0], f, es * (size_t)h->cfg.Z * h->V, kind, h->stream)
                      : cudaMemcpy2DAsync(h->F[0], es * h->ldz, f, es * h->cfg.Z, es * h->cfg.Z,
                                          h->V, kind, h->stream);
  if (e != cudaSuccess) return cuda_error(e, "rslb_set_state: copy");
  return RSLB_OK;
}

namespace rslb {
int sod_view(rslb_handle* h, SodView* v) {
  if (!h || !v) return RSLB_ERR_ARG;
  v->Z = h->cfg.Z;
  v->ldz = h->ldz;
  v->V = h->V;
  v->Q_xi = h->cfg.Q_xi;
  v->Q_L = h->cfg.Q_L;
  v->fp64 = h->fp64;
  v->stream = h->stream;
  v->F0 = h->F[0];
  v->F1 = h->F[1];
  v->dt = h->cfg.dt;
  return RSLB_OK;
}
}  // namespace rslb

extern "C" int rslb_launch_info(const rslb_handle* h, int* tile_cells, int* threads) {
  clear_error();
  if (!h) return set_error(RSLB_ERR_ARG, "rslb_launch_info: NULL handle");
  if (tile_cells) *tile_cells = h->launch.B;
  if (threads)
    *threads = h->launch.B == kSod32Cells ? (h->launch.form == 1 ? sod32p_threads() : kSod32Threads)
                                          : 320;
  return RSLB_OK;
}

extern "C" int rslb_time(const rslb_handle* h, double* t, long long* steps) {
  clear_error();
  if (!h) return set_error(RSLB_ERR_ARG, "rslb_time: NULL handle");
  if (t) *t = h->t;
  if (steps) *steps = h->steps;
  return RSLB_OK;
}

extern "C" void rslb_destroy(rslb_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  free_handle(h);
}

// ---------------------------------------------------------------------------
// Batches of shock tubes
// ---------------------------------------------------------------------------
struct SodClass {
  int V, nm, B, ctas_per_sm;
  size_t smem;
  void* runs_dev;  // SodRunDesc<T>[nr]
  SodTask* tasks_dev;
  int ntasks;
  void* maps_dev;  // packed FP32 kernel: 4 tensor maps per run, or NULL
};

struct rslb_sod_batch {
  int nruns;
  bool fp64;
  cudaStream_t stream;
  std::vector<rslb_handle*> h;       // per run, caller order
  std::vector<long long> nsteps;     // per run
  std::vector<SodClass> cls;
  long long* step_dev;
  int* err;
  long long steps_done, max_steps;
  double total_cv;
  int nsm;
  cudaGraphExec_t graph;
  bool graph_failed;
};

namespace {

__global__ void batch_step_increment(long long* step) { *step += 1; }

void batch_free(rslb_sod_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (auto& c : b->cls) {
    if (c.runs_dev) cudaFree(c.runs_dev);
    if (c.maps_dev) cudaFree(c.maps_dev);
    if (c.tasks_dev) cudaFree(c.tasks_dev);
  }
  if (b->step_dev) cudaFree(b->step_dev);
  if (b->err) cudaFree(b->err);
  for (rslb_handle* x : b->h) free_handle(x);
  delete b;
}

template <typename T>
cudaError_t batch_enqueue(rslb_sod_batch* b, int nsteps) {
  for (int n = 0; n < nsteps; ++n) {
    for (int stage = 0; stage < 3; ++stage)
      for (const SodClass& c : b->cls) {
        cudaError_t e = sod_batch_stage_launch<T>(
            c.B, c.smem, c.ctas_per_sm * b->nsm, (const SodRunDesc<T>*)c.runs_dev, c.tasks_dev,
            c.ntasks, b->step_dev, stage, b->err, c.V, b->stream,
            c.B == kSod32Cells ? c.maps_dev : nullptr);
        if (e != cudaSuccess) return e;
      }
    batch_step_increment<<<1, 1, 0, b->stream>>>(b->step_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Tuning results of this process: (device, FP64, V, Q_L, N_Omega + 1) ->
// (tile cells, CTAs per SM).
struct TuneKey {
  int dev, fp64, V, QL, nm;
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, fp64, V, QL, nm) < std::tie(o.dev, o.fp64, o.V, o.QL, o.nm);
  }
};
std::map<TuneKey, std::pair<int, int>> g_tune;
std::mutex g_tune_mu;

template <typename T>
int batch_build_classes(rslb_sod_batch* b, int autotune) {
  // runs grouped by (V, nm); each group's runs sorted by decreasing step count
  std::vector<int> order(b->nruns);
  for (int r = 0; r < b->nruns; ++r) order[r] = r;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    if (b->h[x]->V != b->h[y]->V) return b->h[x]->V < b->h[y]->V;
    if (b->h[x]->nm != b->h[y]->nm) return b->h[x]->nm < b->h[y]->nm;
    return b->nsteps[x] > b->nsteps[y];
  });
  int dev = 0, max_smem = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  const int QL = b->h[0]->cfg.Q_L;
  for (size_t i = 0; i < order.size();) {
    const int V = b->h[order[i]]->V, nm = b->h[order[i]]->nm;
    size_t j = i;
    while (j < order.size() && b->h[order[j]]->V == V && b->h[order[j]]->nm == nm) ++j;
    SodClass c{};
    c.V = V;
    c.nm = nm;
    const SodLaunch L = sod_pick_launch(b->fp64, V, QL, nm, max_smem);
    if (L.B == 0)
      return set_error(RSLB_ERR_UNSUPPORTED, "rslb_sod_batch_init: V = %d does not fit a tile", V);
    c.B = L.B;
    std::vector<SodRunDesc<T>> rd;
    std::vector<SodTask> tasks;
    for (size_t q = i; q < j; ++q) {
      rslb_handle* hh = b->h[order[q]];
      SodRunDesc<T> d;
      d.g = hh->geom;
      d.tb = tables_of<T>(hh);
      d.rowv = hh->t_rowv;
      d.nneg = hh->nneg;
      d.F0 = (T*)hh->F[0];
      d.F1 = (T*)hh->F[1];
      d.F2 = (T*)hh->F[2];
      d.nsteps = b->nsteps[order[q]];
      rd.push_back(d);
    }
    c.smem = 0;
    // tensor maps of every run for the packed FP32 kernel's bulk-tensor staging
    if constexpr (sizeof(T) == 4) {
      const size_t mb = sod32_map_bytes();
      std::vector<unsigned char> maps(4 * mb * rd.size());
      bool ok = true;
      for (size_t q = 0; q < rd.size() && ok; ++q)
        ok = sod32_make_maps(maps.data() + 4 * mb * q, (const float*)rd[q].F0,
                             (const float*)rd[q].F1, (const float*)rd[q].F2, rd[q].g.Z,
                             rd[q].g.ldz, V);
      if (ok && cudaMalloc(&c.maps_dev, maps.size()) == cudaSuccess)
        cudaMemcpy(c.maps_dev, maps.data(), maps.size(), cudaMemcpyHostToDevice);
    }
    auto make_tasks = [&](int B) {
      tasks.clear();
      for (size_t q = i; q < j; ++q) {
        const int Z = b->h[order[q]]->cfg.Z;
        for (int s0 = 0; s0 < Z; s0 += B) tasks.push_back(SodTask{(int)(q - i), s0});
      }
    };
    if (cudaMalloc(&c.runs_dev, sizeof(SodRunDesc<T>) * rd.size()) != cudaSuccess)
      return set_error(RSLB_ERR_ALLOC, "rslb_sod_batch_init: cudaMalloc failed");
    cudaMemcpy(c.runs_dev, rd.data(), sizeof(SodRunDesc<T>) * rd.size(), cudaMemcpyHostToDevice);
    // candidate tile kernels for this V (the automatic choice first); a
    // choice already timed in this process for the same device, precision
    // and velocity set is reused
    const TuneKey key{dev, b->fp64 ? 1 : 0, V, QL, nm};
    int cachedB = 0, cachedK = 0;
    if (autotune) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find(key);
      if (it != g_tune.end()) {
        cachedB = it->second.first;
        cachedK = it->second.second;
      }
    }
    std::vector<int> cands = {cachedB ? cachedB : c.B};
    if (autotune && !cachedB) {
      const int alt[] = {kSod32Cells, 128, 64, 32, 16, 8};
      for (int B : alt)
        if (B != c.B && sod_stage_smem_bytes(b->fp64, B, V, QL, nm) > 0 &&
            sod_stage_smem_bytes(b->fp64, B, V, QL, nm) <= (size_t)max_smem &&
            !(B == kSod32Cells && (V < 128 || nm > 8)))
          cands.push_back(B);
    }
    float best = 1e30f;
    int bestB = c.B, bestK = 1;
    for (int B : cands) {
      make_tasks(B);
      SodTask* td = nullptr;
      if (cudaMalloc((void**)&td, sizeof(SodTask) * tasks.size()) != cudaSuccess)
        return set_error(RSLB_ERR_ALLOC, "rslb_sod_batch_init: cudaMalloc failed");
      cudaMemcpy(td, tasks.data(), sizeof(SodTask) * tasks.size(), cudaMemcpyHostToDevice);
      const size_t smem = sod_stage_smem_bytes(b->fp64, B, V, QL, nm);
      const int maxk = (smem * 2 + 4096 <= (size_t)max_smem + 1024) ? 2 : 1;
      const bool timing = autotune && !cachedB;
      for (int k = 1; k <= (timing ? maxk : 1); ++k) {
        float ms = 0.f;
        if (timing) {
          cudaEvent_t e0, e1;
          cudaEventCreate(&e0);
          cudaEventCreate(&e1);
          // stage 0 reads F0 and writes F1 only: safe to repeat
          sod_batch_stage_launch<T>(B, smem, k * b->nsm, (const SodRunDesc<T>*)c.runs_dev, td,
                                    (int)tasks.size(), b->step_dev, 0, b->err, V, b->stream,
                                    B == kSod32Cells ? c.maps_dev : nullptr);
          cudaEventRecord(e0, b->stream);
          for (int rep = 0; rep < 3; ++rep)
            sod_batch_stage_launch<T>(B, smem, k * b->nsm, (const SodRunDesc<T>*)c.runs_dev, td,
                                      (int)tasks.size(), b->step_dev, 0, b->err, V, b->stream,
                                      B == kSod32Cells ? c.maps_dev : nullptr);
          cudaEventRecord(e1, b->stream);
          cudaEventSynchronize(e1);
          cudaEventElapsedTime(&ms, e0, e1);
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
        }
        if (!timing || ms < best) {
          best = ms;
          bestB = B;
          bestK = cachedB ? cachedK : k;
        }
      }
      cudaFree(td);
    }
    if (autotune && !cachedB) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune[key] = {bestB, bestK};
    }
    c.B = bestB;
    c.ctas_per_sm = bestK;
    c.smem = sod_stage_smem_bytes(b->fp64, bestB, V, QL, nm);
    make_tasks(bestB);
    c.ntasks = (int)tasks.size();
    if (cudaMalloc((void**)&c.tasks_dev, sizeof(SodTask) * tasks.size()) != cudaSuccess)
      return set_error(RSLB_ERR_ALLOC, "rslb_sod_batch_init: cudaMalloc failed");
    cudaMemcpy(c.tasks_dev, tasks.data(), sizeof(SodTask) * tasks.size(), cudaMemcpyHostToDevice);
    b->cls.push_back(c);
    i = j;
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_error(e, "rslb_sod_batch_init: tuning");
  // tuning launches changed only F1; clear the error word they may have set
  cudaMemset(b->err, 0, 2 * sizeof(int));
  return RSLB_OK;
}

}  // namespace

extern "C" int rslb_sod_batch_init(rslb_sod_batch** out, const rslb_sod_run* runs, int nruns,
                                   const rslb_sod_batch_opts* o, void* stream) {
  clear_error();
  if (!out || !runs || !o || nruns < 1)
    return set_error(RSLB_ERR_ARG, "rslb_sod_batch_init: NULL argument or nruns < 1");
  *out = nullptr;
  if (o->Q_L < 1 || o->Q_L > 8 || (o->precision != RSLB_F32 && o->precision != RSLB_F64) ||
      (o->bc != RSLB_BC_FIXED_EQ && o->bc != RSLB_BC_OUTFLOW) || !(o->z_max > o->z_min) ||
      !(o->cfl > 0.0 && o->cfl < 1.0) || !(o->dt_over_tau > 0.0 && o->dt_over_tau < 1.0))
    return set_error(RSLB_ERR_ARG, "rslb_sod_batch_init: invalid options");
  rslb_sod_batch* b = new rslb_sod_batch();
  b->nruns = nruns;
  b->fp64 = o->precision == RSLB_F64;
  b->stream = (cudaStream_t)stream;
  b->step_dev = nullptr;
  b->err = nullptr;
  b->steps_done = 0;
  b->max_steps = 0;
  b->total_cv = 0.0;
  b->graph = nullptr;
  b->graph_failed = false;
  int rc = RSLB_OK;
  for (int r = 0; r < nruns && !rc; ++r) {
    const rslb_sod_run& R = runs[r];
    const bool tconst = R.tau_mode == RSLB_TAU_CONST;
    if (R.Z < 1 || R.Q_xi < 2 || !(R.t_end > 0.0) || R.tau_mode < RSLB_TAU_CONST ||
        R.tau_mode > RSLB_TAU_NONE || (tconst && !(R.tau > 0.0)) ||
        (R.tau_mode == RSLB_TAU_ETAS && !(R.tau_AW0 > 0.0 && R.lambda_ref > 0.0)) ||
        !(R.dt >= 0.0) || (!tconst && !(R.dt > 0.0)) || R.N_Omega < -1) {
      rc = set_error(RSLB_ERR_ARG, "rslb_sod_batch_init: run %d: invalid parameters", r);
      break;
    }
    long long ns;
    double dt;
    if (R.dt > 0.0) {
      ns = std::max(1LL, (long long)std::llround(R.t_end / R.dt));
      dt = R.dt;
    } else {
      std::vector<double> xi(R.Q_xi), w(R.Q_xi);
      gauss_legendre_host(R.Q_xi, xi.data(), w.data());
      const double dz = (o->z_max - o->z_min) / R.Z;
      const double dtmax =
          std::fmin(o->cfl * dz / std::fabs(xi[R.Q_xi - 1]), o->dt_over_tau * R.tau);
      ns = (long long)std::ceil(R.t_end / dtmax - 1e-12);
      dt = R.t_end / (double)ns;
    }
    rslb_config c{};
    c.Z = R.Z;
    c.z_min = o->z_min;
    c.z_max = o->z_max;
    c.Q_xi = R.Q_xi;
    c.Q_L = o->Q_L;
    c.N_Omega = R.N_Omega >= 0 ? R.N_Omega
                               : (o->N_Omega >= 0 ? o->N_Omega : std::min(R.Q_xi - 1, 5));
    c.precision = o->precision;
    c.bc = o->bc;
    c.tau_mode = R.tau_mode;
    c.tau = R.tau;
    c.tau_AW0 = R.tau_AW0;
    c.lambda_ref = R.tau_mode == RSLB_TAU_ETAS ? R.lambda_ref : 1.0;
    c.dt = dt;
    c.nL = R.nL;
    c.TL = R.TL;
    c.nR = R.nR;
    c.TR = R.TR;
    rslb_handle* hh = nullptr;
    rc = rslb_init(&hh, &c, stream);
    if (rc) {
      set_error(rc, "rslb_sod_batch_init: run %d: %s", r, rslb::last_error());
      break;
    }
    b->h.push_back(hh);
    b->nsteps.push_back(ns);
    b->max_steps = std::max(b->max_steps, ns);
    b->total_cv += (double)ns * R.Z * (double)hh->V;
  }
  if (!rc && cudaMalloc((void**)&b->step_dev, sizeof(long long)) != cudaSuccess)
    rc = set_error(RSLB_ERR_ALLOC, "rslb_sod_batch_init: cudaMalloc failed");
  if (!rc && cudaMalloc((void**)&b->err, 2 * sizeof(int)) != cudaSuccess)
    rc = set_error(RSLB_ERR_ALLOC, "rslb_sod_batch_init: cudaMalloc failed");
  if (!rc) {
    cudaMemset(b->step_dev, 0, sizeof(long long));
    cudaMemset(b->err, 0, 2 * sizeof(int));
    rc = b->fp64 ? batch_build_classes<double>(b, o->autotune)
                 : batch_build_classes<float>(b, o->autotune);
  }
  if (rc) {
    batch_free(b);
    return rc;
  }
  *out = b;
  return RSLB_OK;
}

extern "C" int rslb_sod_batch_step(rslb_sod_batch* b, int nsteps) {
  clear_error();
  if (!b || nsteps < 0) return set_error(RSLB_ERR_ARG, "rslb_sod_batch_step: bad arguments");
  cudaError_t e = cudaSuccess;
  int rest = nsteps;
  if (b->stream != nullptr && nsteps >= kGraphSteps && !b->graph_failed) {
    if (!b->graph) {
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
      cudaError_t le = cudaSuccess;
      if (e == cudaSuccess) {
        le = b->fp64 ? batch_enqueue<double>(b, kGraphSteps) : batch_enqueue<float>(b, kGraphSteps);
        e = cudaStreamEndCapture(b->stream, &g);
      }
      if (le != cudaSuccess) e = le;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        b->graph = nullptr;
        b->graph_failed = true;
        cudaGetLastError();
        e = cudaSuccess;
      }
    }
    while (b->graph && rest >= kGraphSteps && e == cudaSuccess) {
      e = cudaGraphLaunch(b->graph, b->stream);
      rest -= kGraphSteps;
    }
  }
  if (e == cudaSuccess && rest > 0)
    e = b->fp64 ? batch_enqueue<double>(b, rest) : batch_enqueue<float>(b, rest);
  if (e != cudaSuccess) return cuda_error(e, "rslb_sod_batch_step");
  b->steps_done += nsteps;
  return RSLB_OK;
}

extern "C" int rslb_sod_batch_info(const rslb_sod_batch* b, long long* max_steps,
                                   long long* steps_done, double* total_cv_updates) {
  clear_error();
  if (!b) return set_error(RSLB_ERR_ARG, "rslb_sod_batch_info: NULL batch");
  if (max_steps) *max_steps = b->max_steps;
  if (steps_done) *steps_done = b->steps_done;
  if (total_cv_updates) *total_cv_updates = b->total_cv;
  return RSLB_OK;
}

extern "C" int rslb_sod_batch_run_info(const rslb_sod_batch* b, int run, long long* nsteps,
                                       double* dt) {
  clear_error();
  if (!b || run < 0 || run >= b->nruns)
    return set_error(RSLB_ERR_ARG, "rslb_sod_batch_run_info: bad run");
  if (nsteps) *nsteps = b->nsteps[run];
  if (dt) *dt = b->h[run]->cfg.dt;
  return RSLB_OK;
}

extern "C" int rslb_sod_batch_tuning(const rslb_sod_batch* b, int g, int* V, int* tile_cells,
                                     int* ctas_per_sm) {
  clear_error();
  if (!b || g < 0 || g >= (int)b->cls.size())
    return set_error(RSLB_ERR_ARG, "rslb_sod_batch_tuning: bad group");
  if (V) *V = b->cls[g].V;
  if (tile_cells) *tile_cells = b->cls[g].B;
  if (ctas_per_sm) *ctas_per_sm = b->cls[g].ctas_per_sm;
  return RSLB_OK;
}

extern "C" int rslb_sod_batch_moments(rslb_sod_batch* b, int run, double* out) {
  clear_error();
  if (!b || run < 0 || run >= b->nruns || !out)
    return set_error(RSLB_ERR_ARG, "rslb_sod_batch_moments: bad arguments");
  int herr[2] = {0, 0};
  cudaMemcpyAsync(herr, b->err, sizeof(herr), cudaMemcpyDeviceToHost, b->stream);
  cudaStreamSynchronize(b->stream);
  if (herr[0])
    return set_error(RSLB_ERR_NONPHYSICAL, "rslb_sod_batch: non-physical state (cell %d of a run)",
                     herr[1]);
  return rslb_moments(b->h[run], out, 0);
}

extern "C" void rslb_sod_batch_destroy(rslb_sod_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  batch_free(b);
}
