// sod32p.cu -- persistent, warp-specialised form of the packed FP32x2 shock-tube
// stage kernel.
//
// One CTA per SM walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ... of
// the domain with two tile buffers in shared memory, so that the per-cell
// work of one tile overlaps the per-velocity work of the previous one:
//   cell warps (4)    ghost cells of boundary tiles, moments, FP64 Landau
//                     matching and f^eq coefficients of tile t+1 (one warp
//                     per SM sub-partition, so the FP64 work of a tile is
//                     spread over all four);
//   sweep warps (12)  WENO5 sweep, relaxation, RK update and store of tile t,
//                     then the bulk-tensor copy (cp.async.bulk.tensor) of
//                     tile t+2 into the buffer just stored, and an L2
//                     prefetch of its f_n.
// Sixteen warps of 128 registers fill the register file (16 K registers per
// sub-partition).  The groups hand buffers to each other through mbarriers:
// full[b] (copy landed) and ready[b] (coefficients written).  The arithmetic
// is the phase code of sod32_core.cuh, the same as the one-CTA-per-tile
// kernel, so both give bitwise identical results.
//
// Every wait is bounded (clock64 budget, ~2 s); a group whose wait runs out
// records an error code, raises a CTA-wide abort flag so that the other group
// stops waiting too, and leaves its loop; the thread that issues the copies
// then waits (bounded) for the ones in flight before the CTA exits.
#include <cuda.h>

#include <cstring>

#include "sod32_core.cuh"

namespace rslb {
namespace {

using namespace p32;

constexpr int kCellWarps = 4;    // one per SM sub-partition
constexpr int kSweepWarps = 12;  // 600 rows in two rounds of 384
constexpr int kCellT = 32 * kCellWarps;    // 128
constexpr int kSweepT = 32 * kSweepWarps;  // 384
constexpr int kThreads = kCellT + kSweepT;
constexpr int kCellGroups = kB2 / 4;  // moments: 4 cells per warp pass
constexpr int kStoreInflight = 12;    // f_n loads in flight per sweep thread in the store
constexpr long long kWaitCycles = 4000000000ll;  // ~2 s at the maximum SM clock
constexpr uint32_t kSuspendNs = 1000;
constexpr int kBarCell = 1, kBarSweep = 2;  // named barriers (0 is __syncthreads)

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase of the given parity; false if the budget ran
// out or another group raised the abort flag.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          volatile int* abort_flag) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

__device__ __forceinline__ void named_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Barrier among the n threads of named barrier id that returns whether any
// of them passed pred != 0 (a group-uniform decision).
__device__ __forceinline__ bool named_sync_or(int id, int n, int pred) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n"
      " bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"(pred), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

struct Smem {
  float* tile[2];
  float* coef[2];
  float* gco[2];
  float* mws;
  float* cst;
  RowTables rt;
  double* msum;
  float* cellf;
  uint64_t* full;
  uint64_t* ready;
  int* abort_flag;
};

__host__ __device__ __forceinline__ size_t al128(size_t x) { return (x + 127) & ~size_t(127); }

__host__ __device__ __forceinline__ size_t tile_bytes(int V) {
  int nb = 0;
  const int r = tma_box_rows(V, &nb);
  return al128(sizeof(float) * (size_t)nb * r * kP);
}

__host__ __device__ __forceinline__ size_t coef_bytes(int QL) {
  return al128(sizeof(float) * (size_t)QL * kH * kMP * 2);
}

__host__ __device__ __forceinline__ size_t rowtab_bytes(int V) {
  return 3 * al128(sizeof(int) * (size_t)V) + al128(sizeof(float) * kMP * (size_t)V);
}

__host__ __device__ __forceinline__ size_t smem_total(int V, int QL) {
  return 2 * tile_bytes(V) + 2 * coef_bytes(QL) + 2 * al128(sizeof(float) * kH * 4) +
         al128(sizeof(float) * 5 * (size_t)V) + al128(sizeof(float) * kConsts) +
         rowtab_bytes(V) + al128(sizeof(double) * 5 * kB2) + al128(sizeof(float) * 8 * kB2) +
         128 + 128;
}

__device__ __forceinline__ Smem carve(unsigned char* base, int V, int QL) {
  Smem m;
  size_t o = 0;
  for (int b = 0; b < 2; ++b) {
    m.tile[b] = reinterpret_cast<float*>(base + o);
    o += tile_bytes(V);
  }
  for (int b = 0; b < 2; ++b) {
    m.coef[b] = reinterpret_cast<float*>(base + o);
    o += coef_bytes(QL);
  }
  for (int b = 0; b < 2; ++b) {
    m.gco[b] = reinterpret_cast<float*>(base + o);
    o += al128(sizeof(float) * kH * 4);
  }
  m.mws = reinterpret_cast<float*>(base + o);
  o += al128(sizeof(float) * 5 * (size_t)V);
  m.cst = reinterpret_cast<float*>(base + o);
  o += al128(sizeof(float) * kConsts);
  m.rt.v = reinterpret_cast<int*>(base + o);
  o += al128(sizeof(int) * (size_t)V);
  m.rt.xi = reinterpret_cast<float*>(base + o);
  o += al128(sizeof(float) * (size_t)V);
  m.rt.k = reinterpret_cast<int*>(base + o);
  o += al128(sizeof(int) * (size_t)V);
  m.rt.wp = reinterpret_cast<float*>(base + o);
  o += al128(sizeof(float) * kMP * (size_t)V);
  m.msum = reinterpret_cast<double*>(base + o);
  o += al128(sizeof(double) * 5 * kB2);
  m.cellf = reinterpret_cast<float*>(base + o);
  o += al128(sizeof(float) * 8 * kB2);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + o);
  m.full = bars;
  m.ready = bars + 2;
  m.abort_flag = reinterpret_cast<int*>(bars + 4);
  return m;
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 1)
sod32p_stage_kernel(const float* __restrict__ fin, const float* __restrict__ fn, float* fout,
                    int stage, int* err, SodGeom g, SodTables<float> tb,
                    const int* __restrict__ rowv, int nneg,
                    const __grid_constant__ CUtensorMap tmap,
                    const __grid_constant__ CUtensorMap fnmap, int box_rows, int nbox,
                    int ntiles) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const int V = g.V;
  const Smem S = carve(base, V, g.QL);
  volatile int* abort_flag = S.abort_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  const uint32_t box_bytes = (uint32_t)(box_rows * kP * sizeof(float));
  // the bulk copy of tile t (local index i) into buffer i & 1, completing on
  // full[i & 1], and an L2 prefetch of its f_n for the store's RK combination
  auto issue = [&](int i) {
    const int t = blockIdx.x + i * gridDim.x;
    const int b = i & 1;
    const int s0 = t * kB2;
    fence_proxy_async();
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                     smem_u32(&S.full[b])),
                 "r"(box_bytes * (uint32_t)nbox)
                 : "memory");
    for (int q = 0; q < nbox; ++q)
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
          " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(S.tile[b] + (size_t)q * box_rows * kP)),
          "l"(&tmap), "r"(s0 - 4), "r"(q * box_rows), "r"(smem_u32(&S.full[b]))
          : "memory");
    if (stage != 0)
      for (int q = 0; q < nbox; ++q)
        asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                         &fnmap),
                     "r"(s0), "r"(q * box_rows)
                     : "memory");
  };
  const int ntile_cta = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&S.full[b], 1);
      mbar_init(&S.ready[b], kCellT);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // the first two tiles; the issuing thread of the sweep group keeps count
  const int issuer = kCellT;  // sweep thread 0
  int issued = 0;
  if (tid == issuer)
    for (; issued < 2 && issued < ntile_cta; ++issued) issue(issued);
  for (int e = tid; e < 5 * V; e += kThreads) S.mws[e] = tb.mw[e];
  load_consts(S.cst, tb, g.QL, tid, kThreads);
  load_row_tables(S.rt, g, tb, rowv, tid, kThreads);
  __syncthreads();

  const bool collide = g.tau_mode != kTauNone;

  if (tid < kCellT) {
    // ---------------------------------------------------------- cell warps
    for (int i = 0; i < ntile_cta; ++i) {
      const int b = i & 1;
      const int s0 = (blockIdx.x + i * gridDim.x) * kB2;
      const bool ok = mbar_wait(&S.full[b], (uint32_t)(i >> 1) & 1u, abort_flag);
      if (named_sync_or(kBarCell, kCellT, !ok)) {
        if (tid == 0) {
          if (!*abort_flag) report_err(err, kErrWait, s0);
          *abort_flag = 1;
        }
        break;
      }
      float* tile = S.tile[b];
      if (s0 - 4 < 0 || s0 + kB2 + 4 > g.Z) {
        fix_ghosts(tile, fin, g, tb, s0, tid, kCellT);
        named_sync(kBarCell, kCellT);
      }
      if (collide) {
        for (int grp = warp; grp < kCellGroups; grp += kCellWarps)
          moments(tile, S.mws, S.msum, V, grp, lane);
        named_sync(kBarCell, kCellT);
        // Landau matching: the cells spread over the warps, so that the FP64
        // work of the tile is shared by all four SM sub-partitions
        {
          const int c = warp + kCellWarps * lane;
          if (lane < (kB2 + kCellWarps - 1) / kCellWarps && c < kB2)
            landau_cell(S.msum, S.cellf, S.gco[b], g, s0, c, err);
        }
        named_sync(kBarCell, kCellT);
        for (int q = tid; q < kCellThreads; q += kCellT) coefs(S.cellf, S.coef[b], g, S.cst, q);
      } else {
        for (int e = tid; e < g.QL * kH * kMP * 2; e += kCellT) S.coef[b][e] = 0.f;
        for (int e = tid; e < kH * 4; e += kCellT) S.gco[b][e] = 0.f;
      }
      mbar_arrive(&S.ready[b]);
    }
    return;
  }

  // ------------------------------------------------------------ sweep warps
  const int st = tid - kCellT;
  for (int i = 0; i < ntile_cta; ++i) {
    const int b = i & 1;
    const int s0 = (blockIdx.x + i * gridDim.x) * kB2;
    const uint32_t par = (uint32_t)(i >> 1) & 1u;
    const bool ok = mbar_wait(&S.full[b], par, abort_flag) &&
                    mbar_wait(&S.ready[b], par, abort_flag);
    if (named_sync_or(kBarSweep, kSweepT, !ok)) {
      if (st == 0) {
        if (!*abort_flag) report_err(err, kErrWait, s0);
        *abort_flag = 1;
      }
      break;
    }
    float* tile = S.tile[b];
    sweep_rows_tab(tile, S.coef[b], S.gco[b], g, S.rt, nneg, st, kSweepT);
    named_sync(kBarSweep, kSweepT);
    store<kStoreInflight>(tile, fn, fout, g, stage, s0, st, kSweepT);
    // every sweep thread is done with this buffer before the next copy
    // (async proxy) overwrites it
    fence_proxy_async();
    named_sync(kBarSweep, kSweepT);
    if (tid == issuer && issued < ntile_cta) issue(issued++);
  }
  if (tid == issuer) {
    // no copy may still be writing shared memory when the CTA exits: wait
    // (bounded) for the last copy issued into each buffer
    for (int i = issued - 2; i < issued; ++i) {
      if (i < 0) continue;
      const long long t0 = clock64();
      while (!mbar_try(&S.full[i & 1], (uint32_t)(i >> 1) & 1u))
        if (clock64() - t0 > kWaitCycles) break;
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
size_t sod32p_smem_bytes(int V, int QL) { return smem_total(V, QL) + 128; }

int sod32p_threads() { return kThreads; }

cudaError_t sod32p_set_attributes() {
  return cudaFuncSetAttribute(sod32p_stage_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              232448);
}

bool sod32p_fits(const SodGeom& g, int max_smem) {
  return g.V >= 128 && g.nm <= kMP && g.Z >= kB2 + 8 && (g.ldz % 4) == 0 &&
         sod32p_smem_bytes(g.V, g.QL) <= (size_t)max_smem;
}

cudaError_t sod32p_stage_launch(const SodGeom& g, const SodTables<float>& tb, const int* rowv,
                                int nneg, const float* fin, const float* fn, float* fout,
                                int stage, int* err, int num_sms, cudaStream_t st) {
  int nbox = 0;
  const int br = tma_box_rows(g.V, &nbox);
  CUtensorMap m, mn;
  std::memset(&m, 0, sizeof(m));
  std::memset(&mn, 0, sizeof(mn));
  if ((reinterpret_cast<uintptr_t>(fin) % 16) != 0 || (reinterpret_cast<uintptr_t>(fn) % 16) != 0 ||
      !sod32_make_map(&m, fin, g.Z, g.ldz, g.V, kC, br) ||
      !sod32_make_map(&mn, fn, g.Z, g.ldz, g.V, kB2, br))
    return cudaErrorInvalidValue;
  const int ntiles = (g.Z + kB2 - 1) / kB2;
  const int grid = ntiles < num_sms ? ntiles : num_sms;
  sod32p_stage_kernel<<<grid, kThreads, sod32p_smem_bytes(g.V, g.QL), st>>>(
      fin, fn, fout, stage, err, g, tb, rowv, nneg, m, mn, br, nbox, ntiles);
  return cudaGetLastError();
}

}  // namespace rslb
