// sod.cu -- fused RK-stage kernel of the R-SLB Sod shock tube (sm_103a).
//
// One CTA owns a tile of B consecutive cells (128, 64, 32 or 16 for FP32, 16
// or 8 for FP64) and all V velocities.  A stage (Eq. rk3) is one launch:
//   1. the tile plus a 4-cell halo on each side is staged in shared memory
//      with 16-byte cp.async copies (velocity-major rows; boundary tiles map
//      out-of-domain cells through the boundary condition);
//   2. moments: the five sums of the factored Landau form.  Up to 128
//      velocities one lane per (cell, sum) adds every row itself (blocks of
//      four rows, Kahan-compensated in FP32); above that each warp owns a
//      16-byte column chunk of cells, its lanes own velocity rows, and an
//      error-free FP32 transposing warp reduction (FP64 shuffles for FP64
//      populations) combines the lanes;
//   3. per cell: Landau matching in FP64 (Sec. II E), the relaxation time, and
//      the f^eq expansion coefficients (Sec. III D) by a Gauss-Legendre rule
//      spread over the CTA and reduced by shuffles;
//   4. per (velocity, cell): the WENO5 flux difference (Sec. III F) along the
//      row, written in terms of first and second differences of J = xi f so
//      that a sliding window shares them between neighbouring faces; f^eq
//      from the per-cell coefficients; Anderson-Witting relaxation
//      (Eq. L_Sod); the RK combination.  Rows are visited negative-xi first so
//      that the upwind direction is uniform within a warp; with few
//      velocities each row is split into segments of B/2 .. B/8 cells so that
//      enough threads have work;
//   5. vectorised, coalesced store of the tile interior (with the f_n term of
//      stages 2 and 3).
// Shared-memory rows have a pitch whose 16-byte count is odd, so the 16-byte
// accesses of eight consecutive rows fall in distinct bank groups.
#include "rslb_device.cuh"
#include "sod.cuh"

namespace rslb {

constexpr int kMaxQL = 8;
constexpr int kHalo = 4;
constexpr int kMaxMP = 16;  // kMaxM rounded up to a whole number of 16-byte vectors
// Up to this many velocities each moment is summed by one lane over all rows;
// above it the lanes of a warp take rows and a warp reduction follows.
constexpr int kSerialMomentRows = 128;

template <typename T> struct V16;
template <> struct V16<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <> struct V16<double> {
  using type = double2;
  static constexpr int n = 2;
};

template <typename T>
__host__ __device__ constexpr int tile_pitch(int W) {
  // smallest P >= W with P a multiple of the 16-byte vector and P/vector odd
  constexpr int n = V16<T>::n;
  int p = (W + n - 1) / n;
  if (p % 2 == 0) ++p;
  return p * n;
}

template <typename T>
__host__ __device__ inline int coef_pitch(int nm) {
  constexpr int n = V16<T>::n;
  return (nm + n - 1) / n * n;
}

// Shared-memory carve-up of one CTA (all offsets 16-byte aligned).
template <typename T>
struct SodSmem {
  size_t tile, outb, msum, cell, coef, gco, total;
  __host__ __device__ SodSmem(int V, int B, int QL, int nm, bool seg) {
    auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
    const int P = tile_pitch<T>(B + 2 * kHalo);
    tile = 0;
    outb = al(sizeof(T) * (size_t)V * P);
    msum = outb + (seg ? al(sizeof(T) * (size_t)V * B) : 0);
    cell = msum + al(sizeof(double) * 5 * B);
    coef = cell + al(sizeof(double) * 8 * B);
    gco = coef + al(sizeof(T) * (size_t)QL * B * coef_pitch<T>(nm));
    total = gco + al(sizeof(T) * 2 * B);
  }
};

__device__ __forceinline__ void report_error(int* err, int code, int cell) {
  if (atomicCAS(err, 0, code) == 0) err[1] = cell;
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  return x;
}

__device__ __forceinline__ float fast_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double fast_rcp(double x) { return 1.0 / x; }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::);
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

// ---------------------------------------------------------------------------
// WENO5 face correction in difference form.
// For the upwind-ordered values (a, b, c, d, e) of Sec. III F with first
// differences D0 = b-a, D1 = c-b, D2 = d-c, D3 = e-d and second differences
// S1 = a-2b+c, S2 = b-2c+d, S3 = c-2d+e (K_q = 13/12 S_q^2):
//   sigma_1 = K_1 + (3 D1 - D0)^2/4, sigma_2 = K_2 + (D1 + D2)^2/4,
//   sigma_3 = K_3 + (D3 - 3 D2)^2/4,
//   F^q = c + g_q/6 with g_1 = 5 D1 - 2 D0, g_2 = D1 + 2 D2, g_3 = 4 D2 - D3,
// so F = c + (omega . g)/6.  With omega_q ~ delta_q / sigma_q^2 multiplied
// through by prod_p (sigma_p/sigma_max)^2, the limiting rules (i)-(iii) of
// the paper all reduce to "correction = 0" when every product vanishes (the
// g_q of the vanishing stencils are exactly zero there), and rule (iii) is
// the natural limit of the formula.  Returns (omega . g) (without the 1/6).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T weno_corr(T D0, T D1, T D2, T D3, T K1, T K2, T K3) {
  const T e1 = T(3) * D1 - D0, e2 = D1 + D2, e3 = D3 - T(3) * D2;
  const T s1 = K1 + T(0.25) * e1 * e1;
  const T s2 = K2 + T(0.25) * e2 * e2;
  const T s3 = K3 + T(0.25) * e3 * e3;
  const T g1 = T(5) * D1 - T(2) * D0, g2 = D1 + T(2) * D2, g3 = T(4) * D2 - D3;
  // A denominator below the smallest normal number counts as zero: the FP32
  // reciprocal flushes subnormal inputs, and a vanishing denominator means
  // the correction vanishes (limit rules).
  // The indicators are scaled by the power of two at or below their maximum
  // (the weights are homogeneous in sigma; the scaling only keeps the fourth
  // powers in range), formed from the exponent bits with an AND and a
  // subtract; a zero or subnormal maximum gives the largest such power, which
  // keeps zero indicators zero and brings subnormal ones into range.
  const T tiny = Prec<T>::tiny();
  const T smax = fmax(s1, fmax(s2, s3));
  T inv;
  if constexpr (sizeof(T) == 4)
    inv = __int_as_float(0x7F000000 - (__float_as_int(smax) & 0x7F800000));
  else
    inv = __longlong_as_double(0x7FE0000000000000LL -
                               (__double_as_longlong(smax) & 0x7FF0000000000000LL));
  const T r1 = s1 * inv, r2 = s2 * inv, r3 = s3 * inv;
  const T t1 = r1 * r1, t2 = r2 * r2, t3 = r3 * r3;
  const T n1 = T(0.1) * (t2 * t3), n2 = T(0.6) * (t1 * t3), n3 = T(0.3) * (t1 * t2);
  const T den = n1 + n2 + n3;
  const T num = n1 * g1 + n2 * g2 + n3 * g3;
  return den > tiny ? num * fast_rcp(den) : T(0);
}

// 16-byte chunk of a shared-memory row as scalars.
template <typename T>
__device__ __forceinline__ void ld_chunk(const T* p, T* out) {
  using VT = typename V16<T>::type;
  const VT v = *reinterpret_cast<const VT*>(p);
  if constexpr (V16<T>::n == 4) {
    out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
  } else {
    out[0] = v.x; out[1] = v.y;
  }
}
template <typename T>
__device__ __forceinline__ void st_chunk(T* p, const T* in) {
  using VT = typename V16<T>::type;
  VT v;
  if constexpr (V16<T>::n == 4) {
    v.x = in[0]; v.y = in[1]; v.z = in[2]; v.w = in[3];
  } else {
    v.x = in[0]; v.y = in[1];
  }
  *reinterpret_cast<VT*>(p) = v;
}

// ---------------------------------------------------------------------------
// Phase 4: sweep one row segment [i0, i0+SL) (local cells; tile element
// e = cell + kHalo) in chunks of VN cells with a sliding window of J = xi f
// over cells [i-4, i+VN+4) of the current chunk start i.  POS: xi > 0.
// Positive: face s+1/2 uses J_{s-2..s+2} with centre J_s:
//   (D0..D3) = Delta_{s-2..s+1}, (K1, K2, K3) = K_{s-1}, K_s, K_{s+1}.
// Negative: the mirror (J_{s+3}, ..., J_{s-1}) with centre J_{s+1}:
//   (D0..D3) = -Delta_{s+2}, -Delta_{s+1}, -Delta_s, -Delta_{s-1},
//   (K1, K2, K3) = K_{s+2}, K_{s+1}, K_s.
// (Delta_s = J_{s+1} - J_s, K_s = 13/12 (J_{s-1} - 2 J_s + J_{s+1})^2.)
// The flux difference of cell i is then
//   POS: F_{i+1/2} - F_{i-1/2} = Delta_{i-1} + (C_{i+1/2} - C_{i-1/2})/6,
//   NEG: F_{i+1/2} - F_{i-1/2} = Delta_i     + (C_{i+1/2} - C_{i-1/2})/6.
// With the loop fully unrolled, differences shared between neighbouring
// faces are computed once (common subexpressions across iterations).
// ---------------------------------------------------------------------------
template <typename T, bool POS>
__device__ __forceinline__ T face_corr(const T* J, int wc) {
  // J: window values, wc: window index of the face's left cell
  const T k13 = T(13) / T(12);
  auto D = [&](int c) { return J[c + 1] - J[c]; };
  auto K = [&](int c) {
    const T s2 = (J[c + 1] - J[c]) - (J[c] - J[c - 1]);
    return k13 * s2 * s2;
  };
  if constexpr (POS)
    return weno_corr<T>(D(wc - 2), D(wc - 1), D(wc), D(wc + 1), K(wc - 1), K(wc), K(wc + 1));
  else
    return weno_corr<T>(-D(wc + 2), -D(wc + 1), -D(wc), -D(wc - 1), K(wc + 2), K(wc + 1),
                        K(wc));
}

template <typename T, bool POS, int SL>
__device__ __forceinline__ void sweep_segment(const T* row, T* orow, int i0, T xi,
                                              const T* __restrict__ wp, int nm, int MP,
                                              const T* __restrict__ ck,
                                              const T* __restrict__ gco, T inv_dz, T dt) {
  constexpr int VN = V16<T>::n;
  constexpr int NW = VN + 2 * kHalo;  // window cells [i-4, i+VN+4)
  const T sixth = T(1) / T(6);
  T R[NW];  // f at cells i-4+c
  T J[NW];  // J = xi f at the same cells
#pragma unroll
  for (int c = 0; c < NW; c += VN) ld_chunk<T>(row + i0 + c, R + c);
#pragma unroll
  for (int c = 0; c < NW; ++c) J[c] = xi * R[c];
  // correction at the left face of cell i0 (window cell of its left cell: 3)
  T Cl = face_corr<T, POS>(J, kHalo - 1);
#pragma unroll
  for (int t = 0; t < SL / VN; ++t) {
    const int i = i0 + t * VN;
    T out[VN];
#pragma unroll
    for (int c = 0; c < VN; ++c) {
      const int wc = kHalo + c;  // window index of cell i + c
      const T Cr = face_corr<T, POS>(J, wc);
      const T dF = (POS ? (J[wc] - J[wc - 1]) : (J[wc + 1] - J[wc])) + (Cr - Cl) * sixth;
      Cl = Cr;
      const T* cc = ck + (size_t)(i + c) * MP;
      T feq = T(0);
#pragma unroll
      for (int m0 = 0; m0 < kMaxMP; m0 += VN) {
        if (m0 < nm) {
          T cv[VN];
          ld_chunk<T>(cc + m0, cv);
#pragma unroll
          for (int q = 0; q < VN; ++q) feq += cv[q] * wp[m0 + q];
        }
      }
      const T f = R[kHalo + c];
      const T coll = (gco[2 * (i + c)] - gco[2 * (i + c) + 1] * xi) * (f - feq);
      const T L = -dF * inv_dz - coll;
      out[c] = f + dt * L;
    }
    if (t + 1 < SL / VN) {
      // slide the window by one chunk: load the chunk at cells i+VN+4 ..
#pragma unroll
      for (int c = 0; c < NW - VN; ++c) {
        J[c] = J[c + VN];
        R[c] = R[c + VN];
      }
      ld_chunk<T>(row + i + NW, R + NW - VN);  // tile element of cell i+VN+4 is i + NW
#pragma unroll
      for (int c = 0; c < VN; ++c) J[NW - VN + c] = xi * R[NW - VN + c];
    }
    st_chunk<T>(orow + kHalo + i, out);
  }
}

template <typename T, int B, int NT>
__device__ __forceinline__ void sod_tile(const T* __restrict__ fin, const T* __restrict__ fn,
                                         T* fout, int stage, int* err, const SodGeom& g,
                                         const SodTables<T>& tb, const int* __restrict__ rowv,
                                         int nneg, int nseg, int s0) {
  constexpr int VN = V16<T>::n;
  constexpr int W = B + 2 * kHalo;
  constexpr int P = tile_pitch<T>(W);
  constexpr int CH = B / VN;  // 16-byte chunks of interior cells
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int V = g.V;
  const SodSmem<T> lay(V, B, g.QL, g.nm, nseg > 1);
  T* tile = reinterpret_cast<T*>(smem_raw + lay.tile);
  T* outb = (nseg > 1) ? reinterpret_cast<T*>(smem_raw + lay.outb) : nullptr;
  double* msum = reinterpret_cast<double*>(smem_raw + lay.msum);
  // per-cell results of the Landau phase for the coefficient phase, [8][B]
  // values of the kernel's type (the FP32 kernel takes its coefficient
  // arithmetic in FP32)
  T* cellT = reinterpret_cast<T*>(smem_raw + lay.cell);
  T* coef = reinterpret_cast<T*>(smem_raw + lay.coef);
  T* gco = reinterpret_cast<T*>(smem_raw + lay.gco);
  const int MP = coef_pitch<T>(g.nm);

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;

  // ---- 1. stage tile + halo ----
  const bool interior = (s0 - kHalo >= 0) && (s0 + B + kHalo <= g.Z);
  if (interior) {
    constexpr int CPR = W / VN;  // chunks per row
    for (int idx = tid; idx < V * CPR; idx += NT) {
      const int v = idx / CPR, c = idx - v * CPR;
      cp_async16(tile + v * P + c * VN, fin + (size_t)v * g.ldz + (s0 - kHalo) + c * VN);
    }
    cp_async_wait_all();
  } else {
    for (int idx = tid; idx < V * W; idx += NT) {
      const int v = idx / W, e = idx - v * W;
      tile[v * P + e] = load_cell<T>(fin, g, tb, v, s0 - kHalo + e);
    }
  }
  __syncthreads();

  const bool collide = g.tau_mode != kTauNone;
  if (collide) {
    // ---- 2. moments ----
    if (V <= kSerialMomentRows) {
      // few velocities: lane 5c + q sums moment q of cell c of the warp's
      // 16-byte chunk over every row by itself (blocks of four rows, then
      // compensated), so no cross-lane reduction is needed
      const int c = lane / 5, q = lane - 5 * (lane / 5);
      for (int ch = warp; ch < CH; ch += NT / 32) {
        if (lane >= VN * 5) break;
        const T* col = tile + kHalo + ch * VN + c;
        const T* wq = tb.mw + (size_t)q * V;
        Acc<T> acc;
        int v = 0;
        for (; v + 4 <= V; v += 4) {
          T blk = col[v * P] * wq[v];
          blk += col[(v + 1) * P] * wq[v + 1];
          blk += col[(v + 2) * P] * wq[v + 2];
          blk += col[(v + 3) * P] * wq[v + 3];
          acc.add(blk);
        }
        T blk = T(0);
        for (; v < V; ++v) blk += col[v * P] * wq[v];
        acc.add(blk);
        msum[q * B + ch * VN + c] = acc.value();
      }
    } else {
      // warp = 16-byte chunk of cells (warps loop over the chunks), lanes = rows
      for (int ch = warp; ch < CH; ch += NT / 32) {
      Acc<T> acc[VN][5];
      for (int v0 = lane; v0 < V; v0 += 128) {
        T blk[VN][5];
#pragma unroll
        for (int c = 0; c < VN; ++c)
#pragma unroll
          for (int q = 0; q < 5; ++q) blk[c][q] = T(0);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int v = v0 + 32 * u;
          if (v < V) {
            T x[VN];
            ld_chunk<T>(tile + v * P + kHalo + ch * VN, x);
            T w[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) w[q] = tb.mw[q * V + v];
#pragma unroll
            for (int c = 0; c < VN; ++c)
#pragma unroll
              for (int q = 0; q < 5; ++q) blk[c][q] += x[c] * w[q];
          }
        }
#pragma unroll
        for (int c = 0; c < VN; ++c)
#pragma unroll
          for (int q = 0; q < 5; ++q) acc[c][q].add(blk[c][q]);
      }
      if constexpr (sizeof(T) == 4) {
        // FP32 transposing reduction of the compensated pairs (sum, -c):
        // lane l ends with value l; only hi + lo is formed in FP64
        static_assert(VN * 5 <= 32, "moment values per warp");
        float h[32], lo[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          h[i] = 0.f;
          lo[i] = 0.f;
        }
#pragma unroll
        for (int c = 0; c < VN; ++c)
#pragma unroll
          for (int q = 0; q < 5; ++q) {
            h[c * 5 + q] = acc[c][q].s;
            lo[c * 5 + q] = -acc[c][q].c;
          }
        tr_level<16>(h, lo, lane);
        tr_level<8>(h, lo, lane);
        tr_level<4>(h, lo, lane);
        tr_level<2>(h, lo, lane);
        tr_level<1>(h, lo, lane);
        if (lane < VN * 5) {
          const int c = lane / 5, q = lane - 5 * (lane / 5);
          msum[q * B + ch * VN + c] = (double)h[0] + (double)lo[0];
        }
      } else {
#pragma unroll
        for (int c = 0; c < VN; ++c)
#pragma unroll
          for (int q = 0; q < 5; ++q) {
            const double s = warp_sum(acc[c][q].value());
            if (lane == 0) msum[q * B + ch * VN + c] = s;
          }
      }
      }
    }
    __syncthreads();

    // ---- 3a. Landau matching and relaxation time, one thread per cell ----
    if (tid < B) {
      const int c = tid;
      LandauOut Lo = landau_factored(msum[c], msum[B + c], msum[2 * B + c], msum[3 * B + c],
                                     msum[4 * B + c]);
      T g0 = T(0), g1 = T(0);
      if (!Lo.ok) {
        if (s0 + c < g.Z) report_error(err, 6, s0 + c);
        Lo.n = 1.0; Lo.T = 1.0; Lo.beta = 0.0; Lo.gamma = 1.0; Lo.u = 0.0;
      } else if (g.tau_mode == kTauEtas) {
        const double tau = g.tau_AW0 / Lo.T *
                           (1.0 - 0.25 * log(Lo.n / (Lo.T * Lo.T * Lo.T) * g.lambda_ref));
        g0 = T(Lo.gamma / tau);
        g1 = T(Lo.gamma * Lo.beta / tau);
      } else if constexpr (sizeof(T) == 4) {
        const float itau = 1.f / float(g.tau);
        g0 = float(Lo.gamma) * itau;
        g1 = float(Lo.gamma * Lo.beta) * itau;
      } else {
        g0 = Lo.gamma / g.tau;
        g1 = Lo.gamma * Lo.beta / g.tau;
      }
      if constexpr (sizeof(T) == 4) {
        // FP32 from here on: the coefficients are computed in FP32
        const float u = float(Lo.u);
        const float A = asinhf(u);
        cellT[0 * B + c] = float(Lo.n);
        cellT[1 * B + c] = float(Lo.T);
        cellT[2 * B + c] = u;
        cellT[3 * B + c] = A;
        cellT[4 * B + c] = (u > 0.f) ? A / u : 1.f;
        cellT[5 * B + c] = u * u / (float(Lo.gamma) + 1.f);  // 2 sinh^2(A/2) = gamma - 1
      } else {
        const double A = asinh(Lo.u);
        const double sh = sinh(0.5 * A);
        cellT[0 * B + c] = Lo.n;
        cellT[1 * B + c] = Lo.T;
        cellT[2 * B + c] = Lo.u;
        cellT[3 * B + c] = A;
        cellT[4 * B + c] = (Lo.u > 0.0) ? A / Lo.u : 1.0;
        cellT[5 * B + c] = 2.0 * sh * sh;
      }
      cellT[6 * B + c] = (Lo.beta < 0.0) ? T(-1) : T(1);
      cellT[7 * B + c] = Lo.ok ? T(1) : T(0);
      gco[2 * c] = g0;
      gco[2 * c + 1] = g1;
    }
    __syncthreads();

    // ---- 3b. f^eq coefficients: G threads per cell share the nodes ----
    {
      constexpr int G = (256 / B) < 32 ? (256 / B) : 32;
      const int c = tid / G, q = tid - c * G;
      if (c < B) {
        const T ud = cellT[2 * B + c];
        const T A = cellT[3 * B + c], sh2 = cellT[5 * B + c];
        const T uinv = (ud > T(0)) ? T(1) / ud : T(0);
        const bool at_rest = !(ud > T(0));
        T J3[kMaxM], J4[kMaxM];
#pragma unroll
        for (int m = 0; m < kMaxM; ++m) { J3[m] = T(0); J4[m] = T(0); }
        // FP32 with N_Omega <= 7: the 16-node rule (stored after the 32-node one)
        const bool short_rule = sizeof(T) == 4 && g.nm <= 8;
        const int nn = short_rule ? kAeqNodesF32 : kAeqNodes, n0 = short_rule ? kAeqNodes : 0;
        for (int i = q; i < nn; i += G)
          aeq_node<T>(T(tb.gl_t[n0 + i]), T(tb.gl_w[n0 + i]), A, sh2, uinv, at_rest, g.nm, J3, J4);
#pragma unroll
        for (int off = G / 2; off >= 1; off >>= 1)
#pragma unroll
          for (int m = 0; m < kMaxM; ++m)
            if (m < g.nm) {
              J3[m] += __shfl_xor_sync(0xffffffffu, J3[m], off, G);
              J4[m] += __shfl_xor_sync(0xffffffffu, J4[m], off, G);
            }
        if (q == 0) {
          // c''_{k,m} = sgn^m (2m+1)/2 (n r/4) [J3_m + (3 - x_k)(J3_m - theta J4_m)]
          const T fac = cellT[7 * B + c] * cellT[0 * B + c] * cellT[4 * B + c] * T(0.25);
          const T theta = cellT[1 * B + c];
          const T sgn = cellT[6 * B + c];
          T sm = fac;
#pragma unroll
          for (int m = 0; m < kMaxM; ++m) {
            if (m < g.nm) {
              const T h = sm * T(0.5 * (2 * m + 1));
              const T d = J3[m] - theta * J4[m];
              for (int k = 0; k < g.QL; ++k)
                coef[((size_t)k * B + c) * MP + m] = h * (J3[m] + tb.L1k[k] * d);
              sm *= sgn;
            }
          }
          for (int m = g.nm; m < MP; ++m)
            for (int k = 0; k < g.QL; ++k) coef[((size_t)k * B + c) * MP + m] = T(0);
        }
      }
    }
    __syncthreads();
  } else {
    for (int i = tid; i < 2 * B; i += NT) gco[i] = T(0);
    for (int i = tid; i < g.QL * B * MP; i += NT) coef[i] = T(0);
    __syncthreads();
  }

  // ---- 4. WENO5 + relaxation + RK update, row sweeps ----
  const T inv_dz = T(g.inv_dz), dt = T(g.dt);
  const int SLr = B / nseg;
  for (int u = tid; u < V * nseg; u += NT) {
    const int ir = u % V, seg = u / V;
    const int v = rowv[ir];
    const bool pos = ir >= nneg;
    const T xi = tb.xi[v];
    const int k = tb.kidx[v];
    T wp[kMaxMP];
#pragma unroll
    for (int m = 0; m < kMaxMP; ++m) wp[m] = (m < g.nm) ? tb.wp[m * V + v] : T(0);
    const T* row = tile + v * P;
    T* orow = (nseg > 1) ? (outb + v * B - kHalo) : (tile + v * P);
    const T* ck = coef + (size_t)k * B * MP;
    const int i0 = seg * SLr;
    // the segment length is one of B, B/2, B/4, B/8 (>= one 16-byte chunk)
    if (SLr == B) {
      if (pos) sweep_segment<T, true, B>(row, orow, i0, xi, wp, g.nm, MP, ck, gco, inv_dz, dt);
      else sweep_segment<T, false, B>(row, orow, i0, xi, wp, g.nm, MP, ck, gco, inv_dz, dt);
    } else if (SLr == B / 2) {
      if (pos) sweep_segment<T, true, B / 2>(row, orow, i0, xi, wp, g.nm, MP, ck, gco, inv_dz, dt);
      else sweep_segment<T, false, B / 2>(row, orow, i0, xi, wp, g.nm, MP, ck, gco, inv_dz, dt);
    } else if constexpr (B / 4 >= VN) {
      if (SLr == B / 4) {
        if (pos) sweep_segment<T, true, B / 4>(row, orow, i0, xi, wp, g.nm, MP, ck, gco, inv_dz, dt);
        else sweep_segment<T, false, B / 4>(row, orow, i0, xi, wp, g.nm, MP, ck, gco, inv_dz, dt);
      } else if constexpr (B / 8 >= VN) {
        if (pos) sweep_segment<T, true, B / 8>(row, orow, i0, xi, wp, g.nm, MP, ck, gco, inv_dz, dt);
        else sweep_segment<T, false, B / 8>(row, orow, i0, xi, wp, g.nm, MP, ck, gco, inv_dz, dt);
      }
    }
  }
  __syncthreads();

  // ---- 5. coalesced store of the interior ----
  const T a = (stage == 1) ? T(0.75) : T(1.0 / 3.0);
  const T b = (stage == 1) ? T(0.25) : T(2.0 / 3.0);
  const T* res = (nseg > 1) ? outb : tile + kHalo;
  const int rp = (nseg > 1) ? B : P;
  if (s0 + B <= g.Z) {
    for (int idx = tid; idx < V * CH; idx += NT) {
      const int v = idx / CH, c = idx - v * CH;
      const size_t o = (size_t)v * g.ldz + s0 + c * VN;
      T r[VN];
      ld_chunk<T>(res + v * rp + c * VN, r);
      if (stage != 0) {
        T fo[VN];
        ld_chunk<T>(fn + o, fo);
#pragma unroll
        for (int q = 0; q < VN; ++q) r[q] = a * fo[q] + b * r[q];
      }
      st_chunk<T>(fout + o, r);
    }
  } else {
    for (int idx = tid; idx < V * B; idx += NT) {
      const int v = idx / B, i = idx - v * B;
      const int s = s0 + i;
      if (s < g.Z) {
        const size_t o = (size_t)v * g.ldz + s;
        T r = res[v * rp + i];
        if (stage != 0) r = a * fn[o] + b * r;
        fout[o] = r;
      }
    }
  }
}

template <typename T, int B, int NT>
__global__ void __launch_bounds__(NT, 2)
sod_stage_kernel(const T* __restrict__ fin, const T* __restrict__ fn, T* fout, int stage,
                 int* err, SodGeom g, SodTables<T> tb, const int* __restrict__ rowv, int nneg,
                 int nseg) {
  sod_tile<T, B, NT>(fin, fn, fout, stage, err, g, tb, rowv, nneg, nseg, blockIdx.x * B);
}

template <typename T, int B, int NT>
__global__ void __launch_bounds__(NT, 2)
sod_batch_kernel(const SodRunDesc<T>* __restrict__ runs, const SodTask* __restrict__ tasks,
                 int ntasks, const long long* __restrict__ step, int stage, int* err, int nseg) {
  const long long n = *step;
  for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const SodTask tk = tasks[t];
    const SodRunDesc<T> R = runs[tk.run];
    if (n >= R.nsteps) break;  // tasks are ordered by decreasing step count
    const T* fin = stage == 0 ? R.F0 : (stage == 1 ? R.F1 : R.F2);
    T* fout = stage == 0 ? R.F1 : (stage == 1 ? R.F2 : R.F0);
    sod_tile<T, B, NT>(fin, R.F0, fout, stage, err, R.g, R.tb, R.rowv, R.nneg, nseg, tk.s0);
    __syncthreads();
  }
}

template <typename T, int B, int NT>
static size_t smem_for(int V, int QL, int nm, int nseg) {
  return SodSmem<T>(V, B, QL, nm, nseg > 1).total;
}

static int pick_nseg(int V, int B, int NT, int VN) {
  int nseg = 1;
  while (nseg < 8 && B / (2 * nseg) >= VN && V * 2 * nseg <= NT) nseg *= 2;
  return nseg;
}

// Opt every stage kernel into the large dynamic shared-memory carve-out
// (done once at set-up, outside any stream capture).
cudaError_t sod_set_attributes() {
  const void* fns[] = {(const void*)sod_stage_kernel<float, 128, 320>,
                       (const void*)sod_stage_kernel<float, 64, 320>,
                       (const void*)sod_stage_kernel<float, 32, 320>,
                       (const void*)sod_stage_kernel<float, 16, 320>,
                       (const void*)sod_stage_kernel<double, 16, 320>,
                       (const void*)sod_stage_kernel<double, 8, 320>,
                       (const void*)sod_batch_kernel<float, 128, 320>,
                       (const void*)sod_batch_kernel<float, 64, 320>,
                       (const void*)sod_batch_kernel<float, 32, 320>,
                       (const void*)sod_batch_kernel<float, 16, 320>,
                       (const void*)sod_batch_kernel<double, 16, 320>,
                       (const void*)sod_batch_kernel<double, 8, 320>};
  for (const void* f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = sod32_set_attributes();
  if (e != cudaSuccess) return e;
  return sod32p_set_attributes();
}

SodLaunch sod_pick_launch(bool fp64, int V, int QL, int nm, int max_smem) {
  SodLaunch L{0, 0};
  if (QL > kMaxQL || V < 1 || nm < 1 || nm > kMaxM) return L;
  const size_t half = (size_t)max_smem / 2 - 2048;
  if (!fp64) {
    // packed FP32x2 kernel: whole rows per thread, so it needs enough rows to
    // fill a CTA, N_Omega <= 7, and two CTAs per SM
    if (V >= 128 && nm <= 8 && sod32_smem_bytes(V, QL) <= half) return {kSod32Cells, 0};
    // few velocities: wide tiles share each tile's fixed costs among more
    // cells and give the row segments more cells (65536 cells, V = 24: 0.15 ms
    // per step with 128-cell tiles, 0.18 with 64, 0.26 with 32)
    if (V < 48 && smem_for<float, 128, 320>(V, QL, nm, pick_nseg(V, 128, 320, 4)) <= half)
      return {128, 0};
    if (V < 128 && smem_for<float, 64, 320>(V, QL, nm, pick_nseg(V, 64, 320, 4)) <= half)
      return {64, 0};
    const int n32 = pick_nseg(V, 32, 320, 4), n16 = pick_nseg(V, 16, 320, 4);
    if (smem_for<float, 32, 320>(V, QL, nm, n32) <= half) return {32, 0};
    if (smem_for<float, 16, 320>(V, QL, nm, n16) <= half) return {16, 0};
    if (smem_for<float, 16, 320>(V, QL, nm, n16) <= (size_t)max_smem) return {16, 0};
  } else {
    const int n16 = pick_nseg(V, 16, 320, 2), n8 = pick_nseg(V, 8, 320, 2);
    if (smem_for<double, 16, 320>(V, QL, nm, n16) <= half) return {16, 0};
    if (smem_for<double, 8, 320>(V, QL, nm, n8) <= half) return {8, 0};
    if (smem_for<double, 8, 320>(V, QL, nm, n8) <= (size_t)max_smem) return {8, 0};
  }
  return L;
}

template <typename T, int B>
static cudaError_t launch_b(const SodGeom& g, const SodTables<T>& tb, const int* rowv, int nneg,
                            const T* fin, const T* fn, T* fout, int stage, int* err,
                            cudaStream_t st) {
  constexpr int NT = 320;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(sod_stage_kernel<T, B, NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int nseg = pick_nseg(g.V, B, NT, V16<T>::n);
  const size_t smem = smem_for<T, B, NT>(g.V, g.QL, g.nm, nseg);
  const int grid = (g.Z + B - 1) / B;
  sod_stage_kernel<T, B, NT><<<grid, NT, smem, st>>>(fin, fn, fout, stage, err, g, tb, rowv,
                                                     nneg, nseg);
  return cudaGetLastError();
}

template <typename T>
cudaError_t sod_stage_launch(const SodLaunch& L, const SodGeom& g, const SodTables<T>& tb,
                             const int* rowv, int nneg, const T* fin, const T* fn, T* fout,
                             int stage, int* err, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (L.B == kSod32Cells && L.form == 1)
      return sod32p_stage_launch(g, tb, rowv, nneg, fin, fn, fout, stage, err, L.nsm, st);
    if (L.B == kSod32Cells) return sod32_stage_launch(g, tb, rowv, nneg, fin, fn, fout, stage, err, st);
  }
  switch (L.B) {
    case 128:
      if constexpr (sizeof(T) == 4) return launch_b<T, 128>(g, tb, rowv, nneg, fin, fn, fout, stage, err, st);
      break;
    case 64:
      if constexpr (sizeof(T) == 4) return launch_b<T, 64>(g, tb, rowv, nneg, fin, fn, fout, stage, err, st);
      break;
    case 32:
      if constexpr (sizeof(T) == 4) return launch_b<T, 32>(g, tb, rowv, nneg, fin, fn, fout, stage, err, st);
      break;
    case 16: return launch_b<T, 16>(g, tb, rowv, nneg, fin, fn, fout, stage, err, st);
    case 8:
      if constexpr (sizeof(T) == 8) return launch_b<T, 8>(g, tb, rowv, nneg, fin, fn, fout, stage, err, st);
      break;
    default: break;
  }
  return cudaErrorInvalidValue;
}

template cudaError_t sod_stage_launch<float>(const SodLaunch&, const SodGeom&,
                                             const SodTables<float>&, const int*, int,
                                             const float*, const float*, float*, int, int*,
                                             cudaStream_t);
template cudaError_t sod_stage_launch<double>(const SodLaunch&, const SodGeom&,
                                              const SodTables<double>&, const int*, int,
                                              const double*, const double*, double*, int, int*,
                                              cudaStream_t);

size_t sod_stage_smem_bytes(bool fp64, int B, int V, int QL, int nm) {
  if (!fp64) {
    if (B == kSod32Cells) return sod32_smem_bytes(V, QL);
    if (B == 128) return smem_for<float, 128, 320>(V, QL, nm, pick_nseg(V, 128, 320, 4));
    if (B == 64) return smem_for<float, 64, 320>(V, QL, nm, pick_nseg(V, 64, 320, 4));
    if (B == 32) return smem_for<float, 32, 320>(V, QL, nm, pick_nseg(V, 32, 320, 4));
    if (B == 16) return smem_for<float, 16, 320>(V, QL, nm, pick_nseg(V, 16, 320, 4));
  } else {
    if (B == 16) return smem_for<double, 16, 320>(V, QL, nm, pick_nseg(V, 16, 320, 2));
    if (B == 8) return smem_for<double, 8, 320>(V, QL, nm, pick_nseg(V, 8, 320, 2));
  }
  return 0;
}

cudaError_t sod32_batch_launch(size_t smem, int grid, const SodRunDesc<float>* runs,
                               const SodTask* tasks, int ntasks, const long long* step, int stage,
                               int* err, const void* maps, cudaStream_t st);

// Batched stages: all runs of a class share V (so nseg and the tile width).
template <typename T>
cudaError_t sod_batch_stage_launch(int B, size_t smem, int grid, const SodRunDesc<T>* runs,
                                   const SodTask* tasks, int ntasks, const long long* step,
                                   int stage, int* err, int V, cudaStream_t st,
                                   const void* maps) {
  if (ntasks == 0) return cudaSuccess;
  if constexpr (sizeof(T) == 4) {
    if (B == kSod32Cells)
      return sod32_batch_launch(smem, grid, runs, tasks, ntasks, step, stage, err, maps, st);
    if (B == 128) {
      sod_batch_kernel<T, 128, 320><<<grid, 320, smem, st>>>(runs, tasks, ntasks, step, stage, err,
                                                            pick_nseg(V, 128, 320, 4));
      return cudaGetLastError();
    }
    if (B == 64) {
      sod_batch_kernel<T, 64, 320><<<grid, 320, smem, st>>>(runs, tasks, ntasks, step, stage, err,
                                                           pick_nseg(V, 64, 320, 4));
      return cudaGetLastError();
    }
    if (B == 32) {
      sod_batch_kernel<T, 32, 320><<<grid, 320, smem, st>>>(runs, tasks, ntasks, step, stage, err,
                                                           pick_nseg(V, 32, 320, 4));
      return cudaGetLastError();
    }
    if (B == 16) {
      sod_batch_kernel<T, 16, 320><<<grid, 320, smem, st>>>(runs, tasks, ntasks, step, stage, err,
                                                           pick_nseg(V, 16, 320, 4));
      return cudaGetLastError();
    }
  } else {
    if (B == 16) {
      sod_batch_kernel<T, 16, 320><<<grid, 320, smem, st>>>(runs, tasks, ntasks, step, stage, err,
                                                           pick_nseg(V, 16, 320, 2));
      return cudaGetLastError();
    }
    if (B == 8) {
      sod_batch_kernel<T, 8, 320><<<grid, 320, smem, st>>>(runs, tasks, ntasks, step, stage, err,
                                                          pick_nseg(V, 8, 320, 2));
      return cudaGetLastError();
    }
  }
  return cudaErrorInvalidValue;
}

template cudaError_t sod_batch_stage_launch<float>(int, size_t, int, const SodRunDesc<float>*,
                                                   const SodTask*, int, const long long*, int,
                                                   int*, int, cudaStream_t, const void*);
template cudaError_t sod_batch_stage_launch<double>(int, size_t, int, const SodRunDesc<double>*,
                                                    const SodTask*, int, const long long*, int,
                                                    int*, int, cudaStream_t, const void*);

// ---------------------------------------------------------------------------
// Initialisation: per-cell FP64 coefficients, then populations.
// ---------------------------------------------------------------------------
__global__ void sod_init_coef_kernel(SodGeom g, SodTablesF64 tb, const double* __restrict__ n,
                                     const double* __restrict__ Tt,
                                     const double* __restrict__ beta, double* coef, int* err) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.Z) return;
  const double nn = n[s], TT = Tt[s], bb = beta[s];
  double* cs = coef + (size_t)s * kMaxQL * kMaxM;
  if (!(nn > 0.0) || !(TT > 0.0) || !(fabs(bb) < 1.0)) {
    report_error(err, 6, s);
    for (int i = 0; i < kMaxQL * kMaxM; ++i) cs[i] = 0.0;
    return;
  }
  const double gam = 1.0 / sqrt((1.0 - bb) * (1.0 + bb));
  const double u = gam * fabs(bb);
  const double A = asinh(u);
  const double sh = sinh(0.5 * A);
  const double sh2 = 2.0 * sh * sh;
  const double uinv = u > 0.0 ? 1.0 / u : 0.0;
  double J3[kMaxM], J4[kMaxM];
#pragma unroll
  for (int m = 0; m < kMaxM; ++m) { J3[m] = 0.0; J4[m] = 0.0; }
  for (int i = 0; i < kAeqNodes; ++i)
    aeq_node<double>(tb.gl_t[i], tb.gl_w[i], A, sh2, uinv, !(u > 0.0), g.nm, J3, J4);
  const double r = u > 0.0 ? A / u : 1.0;
  double sm = nn * r * 0.25;
  const double sgn = bb < 0.0 ? -1.0 : 1.0;
#pragma unroll
  for (int m = 0; m < kMaxM; ++m) {
    if (m < g.nm) {
      const double h = sm * 0.5 * (2 * m + 1);
      const double d = J3[m] - TT * J4[m];
      for (int k = 0; k < g.QL; ++k) cs[k * kMaxM + m] = h * (J3[m] + tb.L1k[k] * d);
      sm *= sgn;
    }
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

}  // namespace rslb
