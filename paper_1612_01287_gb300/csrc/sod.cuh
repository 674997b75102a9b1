// sod.cuh -- host-visible declarations of the Sod shock-tube kernels.
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "../../include/rslb.h"

namespace rslb {

enum { kBcFixedEq = 0, kBcOutflow = 1, kBcPeriodic = 2 };
enum { kTauConst = 0, kTauEtas = 1, kTauNone = 2 };

struct SodGeom {
  int Z;     // interior cells
  int ldz;   // row pitch (elements) of a population buffer, >= Z
  int V;     // velocities Q_xi * Q_L
  int Qx, QL;
  int nm;    // N_Omega + 1
  int bc, tau_mode;
  double inv_dz, dt, tau, tau_AW0, lambda_ref;
};

// Per-velocity tables in the working precision (device pointers).
template <typename T>
struct SodTables {
  const T* mw;      // [5][V]: 1+xi, 1-xi, p(1+xi)^2, p(1-xi)^2, p(1-xi^2)
  const T* xi;      // [V]
  const T* wp;      // [kMaxM][V]: w_j w_k P_m(xi_j)
  const int* kidx;  // [V]
  const T* L1k;     // [QL]: L_1^{(2)}(x_k) = 3 - x_k
  const T* ghostL;  // [V] fixed-equilibrium ghost populations
  const T* ghostR;  // [V]
  const double* gl_t;  // [kAeqNodes] Gauss-Legendre nodes on [-1, 1]
  const double* gl_w;  // [kAeqNodes]
};

// One run of a batch (batched stage kernels): geometry, tables and the three
// population buffers; nsteps is the run's total step count.
template <typename T>
struct SodRunDesc {
  SodGeom g;
  SodTables<T> tb;
  const int* rowv;
  int nneg;
  T* F0;
  T* F1;
  T* F2;
  long long nsteps;
};

// One CTA task of a batched stage: a tile starting at cell s0 of run `run`.
// Task lists are ordered by decreasing run step count, so the tasks still to
// do at step n form a prefix.
struct SodTask {
  int run;
  int s0;
};

// FP64 tables used by the initialisation and moment kernels.
struct SodTablesF64 {
  const double* xi;   // [V]
  const double* p;    // [V] p_k of row v
  const double* wp;   // [kMaxM][V]
  const int* kidx;    // [V]
  const double* L1k;  // [QL]
  const double* gl_t;
  const double* gl_w;
};

// Tile shape chosen for a given precision and velocity count.
struct SodLaunch {
  int B;        // cells per CTA
  size_t smem;  // dynamic shared memory bytes
  int form;     // packed FP32 kernel: 0 = one CTA per tile, 1 = persistent pipelined
  int nsm;      // SMs of the device (persistent grid)
};

// Opt the stage kernels into large dynamic shared memory (call at set-up,
// outside stream capture).
cudaError_t sod_set_attributes();
// Packed FP32x2 stage kernel (sod32.cu): tile width and threads per CTA
// (8 threads per cell in the f^eq coefficient phase, a warp per 4 cells in
// the moments).
constexpr int kSod32Cells = RSLB_PACKED_TILE_CELLS;
constexpr int kSod32Threads = 8 * kSod32Cells;

// Tensor maps for batched packed-kernel launches (bytes per map; four maps
// per run: F0, F1, F2 with 36-cell boxes, F0 with tile-wide boxes).
size_t sod32_map_bytes();
bool sod32_make_maps(void* out4, const float* F0, const float* F1, const float* F2, int Z,
                     int ldz, int V);

cudaError_t sod32_set_attributes();

// Pick the tile width for V velocities; returns B = 0 if V does not fit.
SodLaunch sod_pick_launch(bool fp64, int V, int QL, int nm, int max_smem);

// Enqueue one RK stage (stage = 0, 1, 2): fout = stage update of fin (and fn).
// rowv: velocity rows ordered with negative xi first (nneg of them), so that
// the upwind direction is uniform within a warp.
template <typename T>
cudaError_t sod_stage_launch(const SodLaunch& L, const SodGeom& g, const SodTables<T>& tb,
                             const int* rowv, int nneg, const T* fin, const T* fn, T* fout,
                             int stage, int* err, cudaStream_t st);

// FP32 stage kernel with packed FP32x2 arithmetic (sod32.cu): 28-cell tiles,
// N_Omega <= 7.  Shared-memory bytes for V velocities and Q_L radial nodes.
size_t sod32_smem_bytes(int V, int QL);
cudaError_t sod32_stage_launch(const SodGeom& g, const SodTables<float>& tb, const int* rowv,
                               int nneg, const float* fin, const float* fn, float* fout, int stage,
                               int* err, cudaStream_t st);

// Persistent pipelined form of the packed FP32x2 kernel (sod32p.cu): one CTA
// per SM, two tile buffers, warp-specialised producer / cell / sweep groups.
size_t sod32p_smem_bytes(int V, int QL);
int sod32p_threads();
cudaError_t sod32p_set_attributes();
bool sod32p_fits(const SodGeom& g, int max_smem);
cudaError_t sod32p_stage_launch(const SodGeom& g, const SodTables<float>& tb, const int* rowv,
                                int nneg, const float* fin, const float* fn, float* fout,
                                int stage, int* err, int num_sms, cudaStream_t st);

// Batched stage launches: a persistent grid of `grid` CTAs walks the task list
// (tile width B as chosen by sod_pick_launch / the tuner for this class).
template <typename T>
cudaError_t sod_batch_stage_launch(int B, size_t smem, int grid, const SodRunDesc<T>* runs,
                                   const SodTask* tasks, int ntasks, const long long* step,
                                   int stage, int* err, int V, cudaStream_t st,
                                   const void* maps = nullptr);
size_t sod_stage_smem_bytes(bool fp64, int B, int V, int QL, int nm);

// Per-cell coefficients c''_{k,m} (FP64) of f^eq for given (n, T, beta) per
// cell, then populations f[v*ldz + s] = sum_m c''_{k(v),m}(s) wp_m(v).
template <typename T>
cudaError_t sod_init_launch(const SodGeom& g, const SodTablesF64& tb, const double* n,
                            const double* Tt, const double* beta, double* coef_scratch, T* f,
                            int* err, cudaStream_t st);

// 14 FP64 fields per cell (rslb.h order), out[field*Z + s] (moments.cu).
// w: per-velocity weight table of sod_moment_weights.
template <typename T>
cudaError_t sod_moments_launch(const SodGeom& g, const void* w, const T* f, double* out,
                               int* err, cudaStream_t st);

// Host: the moment weight table, for velocity v w_q = (1+xi), (1-xi),
// p(1+xi)^2, p(1-xi)^2, p(1-xi^2): FP32 populations get 12 floats per
// velocity {hi0..hi3}{hi4 lo0 lo1 lo2}{lo3 lo4 0 0} with w = hi + lo; FP64
// populations get 6 doubles {w0..w4 0}.  With out == NULL only the byte
// size is returned.
size_t sod_moment_weights(bool fp64, int V, const double* xi, const double* p, void* out);

}  // namespace rslb
