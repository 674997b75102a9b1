// bjorken_tc.cu -- the Bjorken K^P contraction on the 5th-generation tensor
// cores (tcgen05, kind::tf32, FP32 accumulators in tensor memory).
//
// One RK stage (Eq. rk3 with L_Bjorken, Eq. L_Bjorken) of a block of runs
// that share Q_xi is split over the M-tiles of K^P: the CTA of M-tile mt
// computes, for rows j in [128 mt, 128 mt + 128) and every column c = (run, k)
// of the block,
//     D[j][c] = sum_j' K^P[j][j'] f_c[j']                          (Eq. K_leg_disc)
// as an M = 128, N = nc, K = 8 MMA chain.  FP32 operands are split
// x = hi + lo with hi = tf32(x) (round to nearest) and lo = x - hi (exact),
// and D = Khi fhi + Khi flo + Klo fhi ("3xTF32"): the dropped Klo flo term
// and the TF32 truncation of the lo parts leave ~2^-20 relative error per
// product, FP32-level for this contraction.
//
// Data movement: K^P is stored once per distinct Q, already split: for every
// 128-row x 32-column tile the image holds the hi part and then the lo part,
// each in the 128-byte-swizzled K-major order the MMA descriptors expect; the
// two are brought in by bulk copies (cp.async.bulk, completion on one
// mbarrier) and used as they land.  The state f of the block is read from
// HBM/L2 per 32-row K-block, split and stored swizzled by the threads.  Two
// pipeline stages: the bulk copies of K-block it+1 and the thread work of
// K-block it+1 overlap the MMAs of it.
// The epilogue reads its row of D from TMEM (tcgen05.ld), adds the K^L and
// -f/tau terms and the Anderson-Witting collision with the equilibrium of
// the stage state, applies the RK combination and writes f and the run's
// moment partials (N, E) for the next stage.
//
// Every mbarrier wait is bounded; on time-out the CTA records an error,
// waits (bounded) for what it issued, frees its tensor memory and returns.
#include <cstdint>

#include "../../include/rslb.h"
#include "bjorken.cuh"

namespace rslb {
namespace {

constexpr int kTcThreads = 160;  // 4 worker warps + 1 issuer warp
constexpr int kTcWorkers = 128;
constexpr uint32_t kATile = 128 * 128;  // bytes: 128 rows x 32 FP32
constexpr int kSpinLimit = 150000;       // try_wait rounds of at most kSuspendNs: ~0.3 s
constexpr uint32_t kSuspendNs = 2000;
constexpr int kErrTimeout = RSLB_ERR_TIMEOUT;
constexpr int kTcMaxRowsPerWarp = kTcMaxCols / 4;  // state rows per warp in a K-block

__device__ __forceinline__ uint32_t su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)),
               "r"(bytes)
               : "memory");
}

// One potentially blocking test: the thread is suspended until the phase
// completes or about kSuspendNs have passed, so a waiting warp does not take
// issue slots from the others.
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase of the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (int i = 0; i < kSpinLimit; ++i)
    if (mbar_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// 128B-swizzled K-major smem descriptor (tile base 1024-byte aligned; the
// start address may be advanced by 32 B per K step inside the swizzle atom).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for this layout): 16 B
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}

// Instruction descriptor: D FP32, A and B TF32, both K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          su32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Byte offset of element (row, col), col < 32, in a 128B-swizzled K-major
// FP32 tile: 16-byte chunk index XOR (row mod 8).
__host__ __device__ __forceinline__ uint32_t swz(int row, int col) {
  return (uint32_t)(row * 128 + ((((col >> 2) ^ row) & 7) << 4) + ((col & 3) << 2));
}

__device__ __forceinline__ void tc_report(int* err, int code, int run) {
  if (atomicCAS(err, 0, code) == 0) err[1] = run;
}

// ---------------------------------------------------------------------------
// The stage kernel
// ---------------------------------------------------------------------------
template <int QL>
__global__ void __launch_bounds__(kTcThreads, 2) bj_tc_stage_kernel(BjTcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  const BjTcBlock blk = a.blocks[blockIdx.x];
  const int Q = blk.Q, R = blk.R, NC = blk.nc, mt = blk.mt;
  const int qh = blk.qh, hp = blk.h;  // rows of E and of O
  const int ncv = R * QL;
  const int nkbE = (qh + 31) / 32;
  const int rowsE = min(128, qh - 128 * mt);
  const int rowsO = max(0, min(128, hp - 128 * mt));
  const int nkbOf = (hp + 31) / 32;         // K-blocks of the O image
  const int nkbO = rowsO > 0 ? nkbOf : 0;   // K-blocks of O this M-tile computes
  const int nkb = nkbE + nkbO;
  // iteration order: even and odd K-blocks of the same 32 rows j' alternate
  // (E kb, O kb, E kb+1, ...) while both exist, then the remaining even ones,
  // so the workers load each pair f_j', f_{Q-1-j'} once for both parts
  auto kb_of = [&](int it) { return it < 2 * nkbO ? it >> 1 : it - nkbO; };
  auto odd_of = [&](int it) { return it < 2 * nkbO && (it & 1); };
  const uint32_t dodd = (uint32_t)blk.tmem_cols / 2;  // column of the O accumulator
  const uint32_t btile = (uint32_t)NC * 128u;
  const uint32_t sstride = 2 * kATile + 2 * btile;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  auto Ahi = [&](int s) { return base + s * sstride; };
  auto Alo = [&](int s) { return base + s * sstride + kATile; };
  auto Bhi = [&](int s) { return base + s * sstride + 2 * kATile; };
  auto Blo = [&](int s) { return base + s * sstride + 2 * kATile + btile; };
  unsigned char* tail = base + 2 * sstride;
  uint64_t* full = reinterpret_cast<uint64_t*>(tail);  // [2] K^P tile landed
  uint64_t* ready = full + 2;                          // [2] workers filled the stage
  uint64_t* done = ready + 2;                          // [2] MMAs of the stage finished
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 2);
  float* rs = reinterpret_cast<float*>(tail + 64);  // rate[R] | neq4[R] | omt[R]
  float* mp = rs + 3 * R;                           // [4 warps][R][2]

  // zero the rows of the A buffers that the copies of the shorter image (O,
  // rowsO <= rowsE) do not fill; rows past rowsE stay zero, rows in
  // [rowsO, rowsE) only reach rows of the O accumulator that are not read
  {
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int s = 0; s < 2; ++s)
      for (int hh = 0; hh < 2; ++hh) {
        float4* z = reinterpret_cast<float4*>(base + s * sstride + hh * kATile);
        for (int i = rowsO * 8 + tid; i < (int)(kATile / 16); i += kTcThreads) z[i] = zero;
      }
  }
  if (tid == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&ready[0], kTcWorkers);
    mbar_init(&ready[1], kTcWorkers);
    mbar_init(&done[0], 1);
    mbar_init(&done[1], 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_slot)),
                 "r"(blk.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // E tile (mt, kb): hi at AsrcE + kb * rowsE * 64, lo rowsE * 32 floats after
  // it; O tiles likewise from AsrcO
  const float* AsrcE = a.kimg + blk.img + (size_t)mt * 128 * nkbE * 64;
  const float* AsrcO = a.kimg + blk.imgO + (size_t)mt * 128 * nkbOf * 64;
  auto copy_a = [&](int s, int it) {
    const bool ev = !odd_of(it);
    const int rows = ev ? rowsE : rowsO;
    const float* src = (ev ? AsrcE : AsrcO) + (size_t)kb_of(it) * rows * 64;
    const uint32_t abytes = (uint32_t)rows * 128u;
    mbar_expect_tx(&full[s], 2 * abytes);
    bulk_g2s(Ahi(s), src, abytes, &full[s]);
    bulk_g2s(Alo(s), src + (size_t)rows * 32, abytes, &full[s]);
  };
  const uint32_t idesc = idesc_tf32(NC);
  // The issuer (lane 0 of warp 4) keeps the bulk copies two K-blocks ahead
  // and issues the MMAs; issued-but-unconfirmed work is tracked for the
  // abort path.
  const bool issuer = tid == kTcWorkers;
  int last_copy = -1, last_commit = -1;
  if (issuer) {
    for (int it = 0; it < 2 && it < nkb; ++it) {
      copy_a(it, it);
      last_copy = it;
    }
    // the block's state (its runs are contiguous) is read by the K-loop
    // (both halves of every column) and by the epilogue: bring f^(i) and f_n
    // into L2 at once (the 16-byte-aligned interior of each region)
    const size_t nst = (size_t)ncv * Q;
    const float* regs[2] = {a.Fin + blk.soff, a.Fn + blk.soff};
    for (int q = 0; q < (a.stage > 0 ? 2 : 1); ++q) {
      const uintptr_t b0 = reinterpret_cast<uintptr_t>(regs[q]);
      const uintptr_t e0 = reinterpret_cast<uintptr_t>(regs[q] + nst);
      const uintptr_t b1 = (b0 + 15) & ~uintptr_t(15), e1 = e0 & ~uintptr_t(15);
      if (e1 > b1)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(b1),
                     "r"((uint32_t)(e1 - b1))
                     : "memory");
    }
  }

  // per-run equilibrium of the stage state from the moment partials, by the
  // issuer's 31 idle lanes while the workers start on the K-loop (the
  // epilogue reads it after the CTA barrier that ends the loop)
  const bool rk = a.stage >= 0;
  if (rk && warp == 4 && lane > 0) {
    for (int r = lane - 1; r < R; r += 31) {
      const int gr = blk.first + r;
      double N = 0.0, E = 0.0;
      for (int m = 0; m < blk.nmt; ++m) {
        N += a.mp_in[((size_t)gr * 4 + m) * 2];
        E += a.mp_in[((size_t)gr * 4 + m) * 2 + 1];
      }
      double rate = 0.0, neq4 = 0.0, omt = 0.0;
      const double P = E / 3.0;
      const double t0 = a.tau_aw0[gr];
      const bool coll = t0 > 0.0 && isfinite(t0);
      if (!(P > 0.0) || !isfinite(P) || (a.gas[gr] == RSLB_GAS_IDEAL && !(N > 0.0))) {
        if (mt == 0) tc_report(a.err, RSLB_ERR_NONPHYSICAL, gr);
      } else if (coll) {
        double T_, n_eq, tau_aw;
        if (a.gas[gr] == RSLB_GAS_PARTON) {
          T_ = sqrt(sqrt(P));
          n_eq = P / T_;
          tau_aw = t0 / T_;
        } else {
          T_ = P / N;
          n_eq = N;
          tau_aw = t0 / T_ * (1.0 - 0.25 * log(N / (T_ * T_ * T_)));
        }
        rate = 1.0 / tau_aw;
        neq4 = 0.25 * n_eq;
        omt = 1.0 - T_;
      }
      rs[r] = float(rate);
      rs[R + r] = float(neq4);
      rs[2 * R + r] = float(omt);
    }
  }

  // what the epilogue needs from global memory, loaded before the K-loop so
  // the latency is not paid after it.  Worker thread i (row i of E and O)
  // writes rows j1 = i and, if i < h, j2 = Q - 1 - i of K^P f.
  const int i = 128 * mt + 32 * (warp & 3) + lane;
  const bool okE = i < qh, okO = i < hp;
  const int j1 = i, j2 = Q - 1 - i;
  float xi2a = 0.f, wja = 0.f, xi2b = 0.f, wjb = 0.f;
  float KL[QL * QL], xk[QL], wk[QL], l1[QL];
  if (warp < 4) {
    if (okE) {
      const double x = a.npool[blk.xoff + j1];
      xi2a = float(x * x);
      wja = float(a.npool[blk.xoff + Q + j1]);
    }
    if (okO) {
      const double x = a.npool[blk.xoff + j2];
      xi2b = float(x * x);
      wjb = float(a.npool[blk.xoff + Q + j2]);
    }
#pragma unroll
    for (int k = 0; k < QL; ++k) {
      xk[k] = float(a.xk[k]);
      wk[k] = float(a.wk[k]);
      l1[k] = float(3.0 - a.xk[k]);
#pragma unroll
      for (int q = 0; q < QL; ++q) KL[k * QL + q] = float(a.KL[k * QL + q]);
    }
  }

  // ---- main loop over K-blocks of 32 rows j' (E and O alternating) ----
  // Workers (warps 0-3): store the even (s) or odd (d) parts of the state
  // rows of K-block it (the pair loaded into registers earlier) split into
  // hi/lo, load the next pair after its last use and arrive on ready[s].  Issuer: wait full[s] (the
  // image tiles) and ready[s], issue the 12 MMAs into the E or O
  // accumulator, commit to done[s]; once they are done, refill stage s with
  // the tiles of it+2.  No CTA-wide barrier inside the loop.
  const float* Fblk = a.Fin + blk.soff;
  int lost = 0;
  if (issuer) {
    for (int it = 0; it < nkb; ++it) {
      const int s = it & 1;
      const uint32_t par = (uint32_t)(it >> 1) & 1u;
      if (!mbar_wait(&full[s], par) || !mbar_wait(&ready[s], par)) {
        lost = 1;
        break;
      }
      tc_fence_after();
      const uint32_t dacc = odd_of(it) ? tmem + dodd : tmem;
      const int k0 = kb_of(it);
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const uint64_t ah = sdesc(su32(Ahi(s)) + 32u * ks), al = sdesc(su32(Alo(s)) + 32u * ks);
        const uint64_t bh = sdesc(su32(Bhi(s)) + 32u * ks), bl = sdesc(su32(Blo(s)) + 32u * ks);
        mma_tf32(dacc, ah, bh, idesc, (k0 > 0 || ks > 0) ? 1u : 0u);
        mma_tf32(dacc, ah, bl, idesc, 1u);
        mma_tf32(dacc, al, bh, idesc, 1u);
      }
      mma_commit(&done[s]);
      last_commit = it;
      if (it + 2 < nkb) {
        if (!mbar_wait(&done[s], par)) {
          lost = 1;
          break;
        }
        copy_a(s, it + 2);
        last_copy = it + 2;
      }
    }
  } else if (warp < 4) {
    // fa, fb: f_j' and f_{Q-1-j'} of the current K-block pair; after the even
    // part s is stored, fa holds the odd part d until its iteration
    float fa[kTcMaxRowsPerWarp], fb[kTcMaxRowsPerWarp];
    auto load_pair = [&](int kb) {
      const int jj = kb * 32 + lane;
#pragma unroll
      for (int u = 0; u < kTcMaxRowsPerWarp; ++u) {
        const int c = warp + 4 * u;
        const float* col = Fblk + (size_t)c * Q;
        fa[u] = (c < ncv && jj < qh) ? col[jj] : 0.f;
        fb[u] = (c < ncv && jj < hp) ? col[Q - 1 - jj] : 0.f;
      }
    };
    auto store_b = [&](int s, const float* v) {
#pragma unroll
      for (int u = 0; u < kTcMaxRowsPerWarp; ++u) {
        const int c = warp + 4 * u;
        if (c < NC) {
          const float hi = tf32_rn(v[u]);
          const uint32_t o = swz(c, lane);
          *reinterpret_cast<float*>(Bhi(s) + o) = hi;
          *reinterpret_cast<float*>(Blo(s) + o) = v[u] - hi;
        }
      }
    };
    load_pair(0);
    for (int it = 0; it < nkb; ++it) {
      const int s = it & 1;
      // stage s was last read by the MMAs of it-2
      if (it >= 2 && !mbar_wait(&done[s], (uint32_t)((it - 2) >> 1) & 1u)) {
        lost = 1;
        break;
      }
      const int kb = kb_of(it);
      const bool has_odd = kb < nkbO;
      if (!odd_of(it)) {
        // even part s_j' = f_j' + f_{Q-1-j'} (the middle row of odd Q alone)
        const int jj = kb * 32 + lane;
#pragma unroll
        for (int u = 0; u < kTcMaxRowsPerWarp; ++u) {
          const float f1 = fa[u], f2 = fb[u];
          fb[u] = jj < hp ? f1 + f2 : f1;
          fa[u] = f1 - f2;  // odd part d_j' (zero past h: f2 = 0 there, unused)
        }
        store_b(s, fb);
        if (!has_odd && it + 1 < nkb) load_pair(kb_of(it + 1));
      } else {
        store_b(s, fa);
        if (it + 1 < nkb) load_pair(kb_of(it + 1));
      }
      fence_proxy_async();
      if (!a.withhold_ready) mbar_arrive(&ready[s]);
    }
    // the last commit completes after all earlier MMAs
    if (!lost && !mbar_wait(&done[(nkb - 1) & 1], (uint32_t)((nkb - 1) >> 1) & 1u)) lost = 1;
  }
  // all MMAs done (commits complete in issue order); the outcome is made
  // uniform across the CTA before anyone branches on it
  if (__syncthreads_or(lost)) {
    if (tid == 0) tc_report(a.err, kErrTimeout, blk.first);
    // bounded wait for what the issuer issued, then release tensor memory
    if (issuer) {
      if (last_commit >= 0) mbar_wait(&done[last_commit & 1], (uint32_t)(last_commit >> 1) & 1u);
      // up to two copies may still be in flight
      for (int c = last_copy > last_commit + 1 ? last_copy - 1 : last_commit + 1; c <= last_copy;
           ++c)
        mbar_wait(&full[c & 1], (uint32_t)(c >> 1) & 1u);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
      tc_fence_after();
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"(blk.tmem_cols)
                   : "memory");
    }
    return;
  }
  tc_fence_after();

  // ---- epilogue (worker warps): rows j1 = i and j2 = Q-1-i per thread ----
  // (K f)_{j1} = (Y_E + Y_O)/2, (K f)_{j2} = (Y_E - Y_O)/2 (Y_O = 0 past h)
  if (warp < 4) {
    const double tau_s =
        a.step ? a.tau0 + ((double)*a.step + (a.stage == 1 ? 1.0 : (a.stage == 2 ? 0.5 : 0.0))) *
                              a.dtau
               : a.tau;
    const float itau = float(1.0 / tau_s), dt = float(a.dtau);
    const float ca = a.stage == 1 ? 0.75f : 1.f / 3.f, cb = a.stage == 1 ? 0.25f : 2.f / 3.f;
    const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
    const float* Fin = a.Fin + blk.soff;
    const float* Fn = a.Fn + blk.soff;
    float* Fout = a.Fout + blk.soff;
    constexpr int RG = 4;  // runs per TMEM read
    for (int rb = 0; rb < R; rb += RG) {
      const int c0 = rb * QL;
      uint32_t de[RG * QL], dd[RG * QL];
#pragma unroll
      for (int p = 0; p < QL; ++p)
        if (c0 + RG * p < NC) {
          tmem_ld4(trow + (uint32_t)(c0 + RG * p), de + RG * p);
          tmem_ld4(trow + dodd + (uint32_t)(c0 + RG * p), dd + RG * p);
        }
      tmem_wait_ld();
      // four runs at a time: all their loads of f^(i) and f_n (both rows) are
      // issued before any of their stores (the output may alias f_n)
#pragma unroll
      for (int g = 0; g < RG; g += 4) {
        float fk[2][4][QL], fnv[2][4][QL];
#pragma unroll
        for (int w2 = 0; w2 < 2; ++w2) {
          const bool ok = w2 == 0 ? okE : okO;
          const int jr = w2 == 0 ? j1 : j2;
#pragma unroll
          for (int ii = 0; ii < 4; ++ii) {
            const int r = rb + g + ii;
#pragma unroll
            for (int k = 0; k < QL; ++k) {
              const size_t o = (size_t)(r * QL + k) * Q + jr;
              const bool okr = r < R && ok;
              fk[w2][ii][k] = okr ? Fin[o] : 0.f;
              fnv[w2][ii][k] = (okr && rk && a.stage != 0) ? Fn[o] : 0.f;
            }
          }
        }
        float mv[8];  // (N, E) partials of the four runs
#pragma unroll
        for (int ii = 0; ii < 4; ++ii) {
          const int cidx = g + ii, r = rb + cidx;
          float on = 0.f, oe = 0.f;
#pragma unroll
          for (int w2 = 0; w2 < 2; ++w2) {
            const bool ok = w2 == 0 ? okE : okO;
            const int jr = w2 == 0 ? j1 : j2;
            const float xi2 = w2 == 0 ? xi2a : xi2b, wj = w2 == 0 ? wja : wjb;
            if (r < R && ok) {
#pragma unroll
              for (int k = 0; k < QL; ++k) {
                const float ye = __uint_as_float(de[cidx * QL + k]);
                const float yo = okO ? __uint_as_float(dd[cidx * QL + k]) : 0.f;
                const float kpf = 0.5f * (w2 == 0 ? ye + yo : ye - yo);
                const size_t o = (size_t)(r * QL + k) * Q + jr;
                if (!rk) {
                  a.dout[blk.soff + o] = kpf;
                } else {
                  const float rate = rs[r], neq4 = rs[R + r], omt = rs[2 * R + r];
                  float klf = 0.f;
#pragma unroll
                  for (int q = 0; q < QL; ++q) klf += KL[k * QL + q] * fk[w2][ii][q];
                  const float feq = neq4 * (wj * wk[k]) * (1.f + l1[k] * omt);
                  const float L = (-fk[w2][ii][k] + xi2 * klf + kpf) * itau -
                                  (fk[w2][ii][k] - feq) * rate;
                  const float v = fk[w2][ii][k] + dt * L;
                  float out = v;
                  if (a.stage == 1) out = ca * fnv[w2][ii][k] + cb * v;
                  else if (a.stage == 2) out = fnv[w2][ii][k] * ca + cb * v;
                  Fout[o] = out;
                  on += out;
                  oe += xk[k] * out;
                }
              }
            }
          }
          mv[2 * ii] = on;
          mv[2 * ii + 1] = oe;
        }
        if (rk) {
          // warp sums of the eight values by a transposing reduction: lanes
          // with the level's bit set keep the upper half of their values and
          // trade the lower half with the partner lane (9 shuffles, not 40)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const bool up = lane & 16;
            const float send = up ? mv[q] : mv[q + 4], keep = up ? mv[q + 4] : mv[q];
            mv[q] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
          }
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const bool up = lane & 8;
            const float send = up ? mv[q] : mv[q + 2], keep = up ? mv[q + 2] : mv[q];
            mv[q] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
          }
          {
            const bool up = lane & 4;
            const float send = up ? mv[0] : mv[1], keep = up ? mv[1] : mv[0];
            mv[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
          }
          mv[0] += __shfl_xor_sync(0xffffffffu, mv[0], 2);
          mv[0] += __shfl_xor_sync(0xffffffffu, mv[0], 1);
          // lane 4 m (m < 8) holds value m = 2 (run) + (0: N, 1: E)
          const int m = lane >> 2, r = rb + g + (m >> 1);
          if ((lane & 3) == 0 && r < R) mp[(warp * R + r) * 2 + (m & 1)] = mv[0];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (rk) {
    for (int r = tid; r < R; r += kTcThreads) {
      double N = 0.0, E = 0.0;
      for (int w = 0; w < 4; ++w) {
        N += (double)mp[(w * R + r) * 2];
        E += (double)mp[(w * R + r) * 2 + 1];
      }
      const int gr = blk.first + r;
      a.mp_out[((size_t)gr * 4 + mt) * 2] = N;
      a.mp_out[((size_t)gr * 4 + mt) * 2 + 1] = E;
    }
  }
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(blk.tmem_cols)
                 : "memory");
  }
}

// Images of one Q, split for 3xTF32: the even matrix E (qh x qh) at img and
// the odd matrix O (h x h) after it (see BjTcBlock).  Tile (mt, kb) of an
// n x n matrix = rows i in M-tile mt (rows(mt) of them) x columns
// 32 kb .. 32 kb + 31; its hi part tf32(X) (round to nearest) is stored
// swizzled at (mt * 128 * nkb + kb * rows(mt)) * 64 floats and its lo part
// X - hi (exact in FP32) rows(mt) * 32 floats after it.  Columns past n stay
// zero (the buffer is cleared first).  Entries from FP64 K^P (Eq. K_leg_disc).
__global__ void bj_tc_image_kernel(int Q, const double* __restrict__ xw,
                                   const double* __restrict__ kc, float* img) {
  const int h = Q / 2, qh = Q - h;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= qh * qh + h * h) return;
  const bool odd = idx >= qh * qh;
  const int n = odd ? h : qh;
  const int e = odd ? idx - qh * qh : idx;
  const int i = e / n, jp = e - i * n;
  const double k1 = kp_entry(Q, xw, kc, i, jp), k2 = kp_entry(Q, xw, kc, i, Q - 1 - jp);
  const float x = float(odd ? k1 - k2 : k1 + k2);
  const int nkb = (n + 31) / 32;
  const int mt = i >> 7, row = i & 127, kb = jp >> 5, col = jp & 31;
  const int rows = min(128, n - 128 * mt);
  float* tile = img + (odd ? bj_tc_image_floats(qh) : 0) + ((size_t)mt * 128 * nkb +
                                                            (size_t)kb * rows) * 64;
  const float hi = tf32_rn(x);
  tile[swz(row, col) >> 2] = hi;
  tile[(size_t)rows * 32 + (swz(row, col) >> 2)] = x - hi;
}

// Moments (N, E) of each run into partial slot 0 (slots 1-3 cleared).
__global__ void bj_tc_moments_kernel(int nruns, int QL, const int* __restrict__ rq,
                                     const long long* __restrict__ roff,
                                     const double* __restrict__ xk, const float* __restrict__ f,
                                     double* mp) {
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= nruns) return;
  const int Q = rq[r];
  double N = 0.0, E = 0.0;
  for (int v = lane; v < Q * QL; v += 32) {
    const double fv = (double)f[roff[r] + v];
    N += fv;
    E += fv * xk[v / Q];
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    N += __shfl_xor_sync(0xffffffffu, N, o);
    E += __shfl_xor_sync(0xffffffffu, E, o);
  }
  if (lane < 8) mp[(size_t)r * 8 + lane] = lane == 0 ? N : (lane == 1 ? E : 0.0);
}

}  // namespace

size_t bj_tc_smem_bytes(int nc, int R) {
  return 1024 + 2 * (2 * (size_t)kATile + 2 * (size_t)nc * 128) + 64 + sizeof(float) * 11 * (size_t)R;
}

cudaError_t bj_tc_set_attributes() {
  const void* fns[] = {(const void*)bj_tc_stage_kernel<1>, (const void*)bj_tc_stage_kernel<2>,
                       (const void*)bj_tc_stage_kernel<3>, (const void*)bj_tc_stage_kernel<4>};
  for (const void* f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

__global__ void bj_step_count_kernel(long long* step) { *step += 1; }

cudaError_t bj_step_count_launch(long long* step, cudaStream_t st) {
  bj_step_count_kernel<<<1, 1, 0, st>>>(step);
  return cudaGetLastError();
}

cudaError_t bj_tc_stage_launch(const BjTcArgs& a, int nblocks, size_t smem, cudaStream_t st) {
  switch (a.QL) {
    case 1: bj_tc_stage_kernel<1><<<nblocks, kTcThreads, smem, st>>>(a); break;
    case 2: bj_tc_stage_kernel<2><<<nblocks, kTcThreads, smem, st>>>(a); break;
    case 3: bj_tc_stage_kernel<3><<<nblocks, kTcThreads, smem, st>>>(a); break;
    case 4: bj_tc_stage_kernel<4><<<nblocks, kTcThreads, smem, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t bj_tc_image_launch(int Q, const double* xw, const double* kc, float* img,
                               cudaStream_t st) {
  const int n = (Q - Q / 2) * (Q - Q / 2) + (Q / 2) * (Q / 2);
  bj_tc_image_kernel<<<(n + 255) / 256, 256, 0, st>>>(Q, xw, kc, img);
  return cudaGetLastError();
}

cudaError_t bj_tc_moments_launch(int nruns, int QL, const int* rq, const long long* roff,
                                 const double* xk, const float* state, double* mp,
                                 cudaStream_t st) {
  bj_tc_moments_kernel<<<(nruns + 7) / 8, 256, 0, st>>>(nruns, QL, rq, roff, xk, state, mp);
  return cudaGetLastError();
}

}  // namespace rslb
