// sod32.cu -- FP32 RK-stage kernel of the Sod shock tube using the packed
// FP32x2 instructions of sm_100+ (FFMA2 / FADD2 / FMUL2), one CTA per tile.
//
// The tile shape and the phases (moments, FP64 Landau matching, f^eq
// coefficients, WENO5 sweep, store) are in sod32_core.cuh.  Here a CTA of
// 8 kB2 threads runs the phases of one tile one after another, separated by
// CTA barriers.  Interior tiles are brought in by tensor-memory-access bulk
// copies (cp.async.bulk.tensor, one box per block of rows, completion on an
// mbarrier), boundary tiles by plain loads.  The batched kernel walks the
// tile list of many runs with the same code.
#include <cuda.h>

#include <cstring>
#include <mutex>

#include "sod32_core.cuh"

namespace rslb {
namespace {

using namespace p32;
constexpr int kNT = kSod32Threads;  // a warp per 4 cells in the moments, 8 threads per cell
                                    // in the f^eq coefficients
static_assert(kNT == kCellThreads, "one thread per coefficient slot");
constexpr int kMinCtas = kB2 <= 20 ? 3 : 2;  // CTAs per SM the registers are sized for

}  // namespace

// Shared memory: tile [rows][kP] floats (rows = V rounded up to whole TMA
// boxes), then partial moments, cell scalars, coefficients
// [QL][kH][kMP][2] floats, gco [kH][4] floats, an mbarrier, the five
// moment weights of every velocity [5][V] and the coefficient constants.
static size_t tile_rows(int V) {
  int nb = 0;
  const int r = tma_box_rows(V, &nb);
  return (size_t)nb * r;
}

size_t sod32_smem_bytes(int V, int QL) {
  auto al = [](size_t x) { return (x + 127) & ~size_t(127); };
  return al(sizeof(float) * tile_rows(V) * kP) + al(sizeof(double) * 5 * kB2) +
         al(sizeof(double) * 8 * kB2) + al(sizeof(float) * (size_t)QL * kH * kMP * 2) +
         al(sizeof(float) * kH * 4) + 128 + al(sizeof(float) * 5 * (size_t)V) +
         al(sizeof(float) * kConsts) + 128;
}

// One stage of one tile starting at cell s0 (the whole CTA).
__device__ __forceinline__ void sod32_tile(const float* __restrict__ fin,
                                           const float* __restrict__ fn, float* fout, int stage,
                                           int* err, const SodGeom& g, const SodTables<float>& tb,
                                           const int* __restrict__ rowv, int nneg, int s0,
                                           const CUtensorMap* tmap, const CUtensorMap* fnmap,
                                           int box_rows, int nbox, int& bar_uses) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  auto al = [](size_t x) { return (x + 127) & ~size_t(127); };
  const int V = g.V;
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  float* tile = reinterpret_cast<float*>(base);
  const size_t tile_bytes = al(sizeof(float) * (size_t)nbox * box_rows * kP);
  double* msum = reinterpret_cast<double*>(base + tile_bytes);
  double* cell = msum + 5 * kB2;
  float* coef = reinterpret_cast<float*>(
      base + tile_bytes + al(sizeof(double) * 5 * kB2) + al(sizeof(double) * 8 * kB2));
  float* gco = coef + (size_t)g.QL * kH * kMP * 2;  // [kH][g0x g0y g1x g1y]
  uint64_t* bar = reinterpret_cast<uint64_t*>(
      reinterpret_cast<unsigned char*>(gco) + al(sizeof(float) * kH * 4));
  float* mws = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(bar) + 128);
  float* cst = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(mws) +
                                        al(sizeof(float) * 5 * (size_t)V));
  auto copy_weights = [&]() {
    for (int e = threadIdx.x; e < 5 * V; e += kNT) mws[e] = tb.mw[e];
    load_consts(cst, tb, g.QL, threadIdx.x, kNT);
  };

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // ---- 1. stage rows: cell s0-4+p goes to position p (0 <= p < kC) ----
  const bool interior = (s0 - 4 >= 0) && (s0 + kB2 + 4 <= g.Z);
  if (interior && tmap) {
    // one thread issues the box copies; everyone waits on the mbarrier (set
    // up at the CTA's first bulk-copied tile, one phase per tile after that)
    const uint32_t phase = (uint32_t)(bar_uses & 1);
    if (tid == 0) {
      if (bar_uses == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      const uint32_t bytes = (uint32_t)(nbox * box_rows * kP * sizeof(float));
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                   "r"(bytes)
                   : "memory");
      for (int b = 0; b < nbox; ++b)
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(tile + (size_t)b * box_rows * kP)),
            "l"(tmap), "r"(s0 - 4), "r"(b * box_rows), "r"(smem_u32(bar))
            : "memory");
      // f_n of the tile is read only by the final RK combination: start
      // bringing it into L2 now
      if (fnmap && stage != 0)
        for (int b = 0; b < nbox; ++b)
          asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                           fnmap),
                       "r"(s0), "r"(b * box_rows)
                       : "memory");
    }
    __syncthreads();  // the barrier is initialised before anyone polls it
    copy_weights();   // while the boxes are in flight
    uint32_t ok = 0;
    for (int it = 0; it < (1 << 22) && !ok; ++it) {
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
          " selp.u32 %0, 1, 0, p;\n}"
          : "=r"(ok)
          : "r"(smem_u32(bar)), "r"(phase)
          : "memory");
      if (!ok && it > 32) __nanosleep(32);
    }
    if (!ok && tid == 0) report_err(err, kErrWait, s0);
    ++bar_uses;
  } else if (interior) {
    stage_interior_vec(tile, fin, g, s0, tid, kNT);
  } else {
    stage_plain(tile, fin, g, tb, s0, tid, kNT);
  }
  if (!(interior && tmap)) copy_weights();
  __syncthreads();

  const bool collide = g.tau_mode != kTauNone;
  if (collide) {
    // ---- 2. moments: warp w owns cells 4w .. 4w+3 of the tile ----
    moments(tile, mws, msum, V, warp, lane);
    __syncthreads();
    // ---- 3a. Landau matching (FP64) and relaxation time, one thread per cell ----
    float* cellf = reinterpret_cast<float*>(cell);  // [8][kB2]
    if (tid < kB2) landau_cell(msum, cellf, gco, g, s0, tid, err);
    __syncthreads();
    // ---- 3b. f^eq coefficients: 8 threads per cell share the 16 nodes ----
    coefs(cellf, coef, g, cst, tid);
    __syncthreads();
  } else {
    for (int i = tid; i < g.QL * kH * kMP * 2 + kH * 4; i += kNT) coef[i] = 0.f;
    __syncthreads();
  }

  // ---- 4. row sweeps (negative-xi rows first: warp-uniform direction) ----
  sweep_rows(tile, coef, gco, g, tb, rowv, nneg, tid, kNT);
  __syncthreads();

  // ---- 5. store: cell c of the tile is position 4 + c ----
  store(tile, fn, fout, g, stage, s0, tid, kNT);
}

__global__ void __launch_bounds__(kNT, kMinCtas)
sod32_stage_kernel(const float* __restrict__ fin, const float* __restrict__ fn, float* fout,
                   int stage, int* err, SodGeom g, SodTables<float> tb, const int* __restrict__ rowv,
                   int nneg, const __grid_constant__ CUtensorMap tmap,
                   const __grid_constant__ CUtensorMap fnmap, int use_tma, int box_rows,
                   int nbox) {
  int bar_uses = 0;
  sod32_tile(fin, fn, fout, stage, err, g, tb, rowv, nneg, blockIdx.x * kB2,
             use_tma ? &tmap : nullptr, use_tma ? &fnmap : nullptr, box_rows, nbox, bar_uses);
}

// Batched: a persistent grid walks the task list of all runs of one class.
// maps (optional): per run, the tensor maps of F0, F1, F2 (36-cell boxes) and
// of F0 with tile-wide boxes for the f_n prefetch; without them the tiles
// are staged by plain loads.
__global__ void __launch_bounds__(kNT, kMinCtas)
sod32_batch_kernel(const SodRunDesc<float>* __restrict__ runs, const SodTask* __restrict__ tasks,
                   int ntasks, const long long* __restrict__ step, int stage, int* err,
                   const CUtensorMap* __restrict__ maps) {
  const long long n = *step;
  int bar_uses = 0;
  for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const SodTask tk = tasks[t];
    const SodRunDesc<float>& R = runs[tk.run];
    if (n >= R.nsteps) break;  // tasks are ordered by decreasing step count
    const float* fin = stage == 0 ? R.F0 : (stage == 1 ? R.F1 : R.F2);
    float* fout = stage == 0 ? R.F1 : (stage == 1 ? R.F2 : R.F0);
    int nbox = 0;
    const int br = tma_box_rows(R.g.V, &nbox);
    const CUtensorMap* tm = maps ? maps + (size_t)tk.run * 4 + stage : nullptr;
    const CUtensorMap* fm = maps ? maps + (size_t)tk.run * 4 + 3 : nullptr;
    sod32_tile(fin, R.F0, fout, stage, err, R.g, R.tb, R.rowv, R.nneg, tk.s0, tm, fm, br, nbox,
               bar_uses);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

}  // namespace

bool sod32_make_map(CUtensorMap* m, const float* f, int Z, int ldz, int V, int box_cells,
                    int box_rows) {
  EncodeTiled enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)Z, (cuuint64_t)V};
  const cuuint64_t strides[1] = {(cuuint64_t)ldz * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)box_cells, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(f), dims, strides, box,
             es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t sod32_batch_launch(size_t smem, int grid, const SodRunDesc<float>* runs,
                               const SodTask* tasks, int ntasks, const long long* step, int stage,
                               int* err, const void* maps, cudaStream_t st) {
  sod32_batch_kernel<<<grid, kNT, smem, st>>>(runs, tasks, ntasks, step, stage, err,
                                              static_cast<const CUtensorMap*>(maps));
  return cudaGetLastError();
}

size_t sod32_map_bytes() { return sizeof(CUtensorMap); }

// The four tensor maps of one run (see sod32_batch_kernel); false if the
// encoder is not available or a map cannot be built.
bool sod32_make_maps(void* out4, const float* F0, const float* F1, const float* F2, int Z,
                     int ldz, int V) {
  if (Z < kB2 + 8 || (ldz % 4) != 0) return false;
  int nbox = 0;
  const int br = tma_box_rows(V, &nbox);
  CUtensorMap* m = static_cast<CUtensorMap*>(out4);
  return sod32_make_map(&m[0], F0, Z, ldz, V, kC, br) && sod32_make_map(&m[1], F1, Z, ldz, V, kC, br) &&
         sod32_make_map(&m[2], F2, Z, ldz, V, kC, br) && sod32_make_map(&m[3], F0, Z, ldz, V, kB2, br);
}

cudaError_t sod32_set_attributes() {
  cudaError_t e = cudaFuncSetAttribute(sod32_batch_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(sod32_stage_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              232448);
}

cudaError_t sod32_stage_launch(const SodGeom& g, const SodTables<float>& tb, const int* rowv,
                               int nneg, const float* fin, const float* fn, float* fout, int stage,
                               int* err, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = sod32_set_attributes();
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  int nbox = 0;
  const int br = tma_box_rows(g.V, &nbox);
  CUtensorMap m, mn;
  std::memset(&m, 0, sizeof(m));
  std::memset(&mn, 0, sizeof(mn));
  // TMA needs 16-byte aligned bases and row stride (cudaMalloc'd buffers,
  // ldz a multiple of 32) and at least one whole interior tile
  const bool tma = g.Z >= kB2 + 8 && (reinterpret_cast<uintptr_t>(fin) % 16) == 0 &&
                   (reinterpret_cast<uintptr_t>(fn) % 16) == 0 && (g.ldz % 4) == 0 &&
                   sod32_make_map(&m, fin, g.Z, g.ldz, g.V, kC, br) &&
                   sod32_make_map(&mn, fn, g.Z, g.ldz, g.V, kB2, br);
  const int grid = (g.Z + kB2 - 1) / kB2;
  sod32_stage_kernel<<<grid, kNT, sod32_smem_bytes(g.V, g.QL), st>>>(
      fin, fn, fout, stage, err, g, tb, rowv, nneg, m, mn, tma ? 1 : 0, br, nbox);
  return cudaGetLastError();
}

}  // namespace rslb
