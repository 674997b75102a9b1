// sod32_core.cuh -- the phases of the packed FP32x2 shock-tube stage, shared by
// the one-CTA-per-tile kernel (sod32.cu) and the persistent pipelined kernel
// (sod32p.cu), so that both perform exactly the same arithmetic.
//
// A tile is kB2 = RSLB_PACKED_TILE_CELLS output cells, split into two halves of
// kH; a thread walks a velocity row and advances both halves in lock-step, the
// left half in the x lane and the right half in the y lane of float2 values,
// so every arithmetic instruction of the sweep does two cells.  Shared memory
// holds the kB2 + 8 cells s0-4 .. s0+kB2+3 of every velocity row densely
// (the row pitch is an odd number of 16-byte units, so 16-byte accesses of 8
// consecutive rows hit distinct banks); "slot" s of the sweep is the pair
// (position s, position s + kH).
//
// Phases of one RK stage of one tile (Sec. III F, Eq. rk3):
//   moments    Kahan-compensated FP32 sums of N+-, A+-, D (Eq. macro_jk in the
//              factored form) with an error-free FP32 warp reduction;
//   landau     FP64 Landau matching (Eqs. E_landau, u_landau) and tau;
//   coefs      f^eq coefficients (Eq. feq_trunc via Eq. aeq_aux, 16-node rule);
//   sweep      WENO5 flux difference (Eqs. flux_weno, weno5_omega), f^eq at
//              the nodes (Eq. fjk), relaxation (Eq. L_Sod), stage update;
//   store      RK combination with f_n and the write of the tile.
#pragma once

#include <cuda.h>

#include <cstdint>

#include "rslb_device.cuh"
#include "sod.cuh"

namespace rslb {
namespace p32 {

constexpr int kB2 = kSod32Cells;  // output cells per tile
constexpr int kH = kB2 / 2;        // cells per half
constexpr int kC = kB2 + 8;        // cells staged per row (4-cell halo per side)
constexpr int kP = kC;             // floats per row (an odd number of 16-byte units)
constexpr int kCellThreads = 8 * kB2;  // moments: a warp per 4 cells; coefficients: 8 per cell
static_assert(kB2 % 4 == 0 && kH % 2 == 0 && (kC / 4) % 2 == 1, "packed tile shape");
constexpr int kMP = 8;        // coefficient pitch (m) for N_Omega <= 7
constexpr int kInflight = 8;  // 16-byte global loads in flight per thread (staging, store)
constexpr int kErrWait = RSLB_ERR_TIMEOUT;  // error code: a bounded wait ran out

__device__ __forceinline__ float2 splat(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b with one rounding
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, splat(-1.f), a); }

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void report_err(int* err, int code, int cell) {
  if (atomicCAS(err, 0, code) == 0) err[1] = cell;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Rows of one bulk-tensor box (<= 256 rows, a multiple of 8 so that a box of
// kC floats per row is a multiple of 128 bytes) and the number of boxes.
__host__ __device__ __forceinline__ int tma_box_rows(int V, int* nbox) {
  const int nb = (V + 255) / 256;
  int r = (V + nb - 1) / nb;
  r = (r + 7) / 8 * 8;
  *nbox = nb;
  return r;
}

// WENO5 correction (omega . g) of sod.cu::weno_corr for two faces at once,
// with delta_q folded into g_q: n_q = prod_{p != q} t_p.
__device__ __forceinline__ float2 weno_corr2(float2 D0, float2 D1, float2 D2, float2 D3,
                                             float2 K1, float2 K2, float2 K3) {
  const float tiny = 1.17549435e-38f;
  const float2 e1 = fma2(splat(-3.f), D1, D0);  // -(3 D1 - D0); squared below
  const float2 e2 = add2(D1, D2);
  const float2 e3 = fma2(splat(-3.f), D2, D3);
  const float2 s1 = fma2(mul2(splat(0.25f), e1), e1, K1);
  const float2 s2 = fma2(mul2(splat(0.25f), e2), e2, K2);
  const float2 s3 = fma2(mul2(splat(0.25f), e3), e3, K3);
  // delta_q g_q: 0.1 (5 D1 - 2 D0), 0.6 (D1 + 2 D2), 0.3 (4 D2 - D3)
  const float2 h1 = fma2(splat(0.5f), D1, mul2(splat(-0.2f), D0));
  const float2 h2 = fma2(splat(1.2f), D2, mul2(splat(0.6f), D1));
  const float2 h3 = fma2(splat(1.2f), D2, mul2(splat(-0.3f), D3));
  // scale the smoothness indicators by the power of two at or below their
  // maximum (the weights are homogeneous in sigma; this only keeps the
  // fourth powers inside the FP32 range): integer exponent arithmetic
  // instead of a reciprocal
  const float mx = fmaxf(s1.x, fmaxf(s2.x, s3.x));
  const float my = fmaxf(s1.y, fmaxf(s2.y, s3.y));
  // 2^(127 - e) for the biased exponent e of m: an AND and a subtract; a
  // zero or subnormal m gives 2^127, which keeps zero sigmas zero and brings
  // subnormal ones into range
  auto inv_pow2 = [&](float m) {
    return __int_as_float(0x7F000000 - (__float_as_int(m) & 0x7F800000));
  };
  const float2 inv = make_float2(inv_pow2(mx), inv_pow2(my));
  const float2 r1 = mul2(s1, inv), r2 = mul2(s2, inv), r3 = mul2(s3, inv);
  const float2 t1 = mul2(r1, r1), t2 = mul2(r2, r2), t3 = mul2(r3, r3);
  const float2 p23 = mul2(t2, t3), p13 = mul2(t1, t3), p12 = mul2(t1, t2);
  const float2 den = fma2(splat(0.1f), p23, fma2(splat(0.6f), p13, mul2(splat(0.3f), p12)));
  const float2 num = fma2(p23, h1, fma2(p13, h2, mul2(p12, h3)));
  return make_float2(den.x > tiny ? num.x * rcp_approx(den.x) : 0.f,
                     den.y > tiny ? num.y * rcp_approx(den.y) : 0.f);
}

__device__ __forceinline__ void ld2slots(const float* p, float2* out) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  out[0] = make_float2(v.x, v.y);
  out[1] = make_float2(v.z, v.w);
}

// Slots s, s+1 (s even) of a dense row: x from positions s, s+1, y from
// positions s+kH, s+kH+1.
__device__ __forceinline__ void ld_slot_pair(const float* row, int s, float2* out) {
  const float2 a = *reinterpret_cast<const float2*>(row + s);
  const float2 b = *reinterpret_cast<const float2*>(row + s + kH);
  out[0] = make_float2(a.x, b.x);
  out[1] = make_float2(a.y, b.y);
}

// Sweep a whole row (both halves): slots 4 .. kH+3 are the outputs; window of
// 10 slots [i-4, i+6) around the current two-slot chunk i, with the first
// differences D[c] = J[c+1] - J[c] and the smoothness terms
// K[c] = 13/12 (D[c] - D[c-1])^2 slid along with it (two new of each per
// chunk).  For xi < 0 the stencil is mirrored; weno_corr2 is odd in its D
// arguments, so the mirrored correction is taken as -weno_corr2 of the
// un-negated differences.  Results go back into the row in place: the
// left-half outputs (positions 4 .. kH+3) and the right-half outputs of slots
// >= 8 (positions >= kH+8) are never read again by the sweep; the right-half
// outputs of slots 4..7 (positions kH+4 .. kH+7) are held until the left half
// has read those positions (its last four slots).
template <bool POS>
__device__ __forceinline__ void sweep_row2(float* row, float xi, const float2* wp2, int nm,
                                           const float* __restrict__ ck,
                                           const float* __restrict__ gco, float inv_dz,
                                           float dt) {
  constexpr int NW = 10;
  const float2 xi2 = splat(xi);
  const float2 sixth = splat(1.f / 6.f);
  const float2 k13 = splat(13.f / 12.f);
  float2 R[NW], J[NW], Dw[NW - 1], Kw[NW - 1];
  float2 held[2];
#pragma unroll
  for (int c = 0; c < NW; c += 2) ld_slot_pair(row, c, R + c);
#pragma unroll
  for (int c = 0; c < NW; ++c) J[c] = mul2(xi2, R[c]);
#pragma unroll
  for (int c = 0; c < NW - 1; ++c) Dw[c] = sub2(J[c + 1], J[c]);
  Kw[0] = splat(0.f);
#pragma unroll
  for (int c = 1; c < NW - 1; ++c) {
    const float2 d2 = sub2(Dw[c], Dw[c - 1]);
    Kw[c] = mul2(mul2(k13, d2), d2);
  }
  auto face = [&](int wc) {
    if constexpr (POS)
      return weno_corr2(Dw[wc - 2], Dw[wc - 1], Dw[wc], Dw[wc + 1], Kw[wc - 1], Kw[wc],
                        Kw[wc + 1]);
    else
      return weno_corr2(Dw[wc + 2], Dw[wc + 1], Dw[wc], Dw[wc - 1], Kw[wc + 2], Kw[wc + 1],
                        Kw[wc]);
  };
  float2 Cl = face(3);
#pragma unroll
  for (int t = 0; t < kH / 2; ++t) {
    const int i = 4 + 2 * t;  // slot of the first cell of this chunk
    float2 out[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int wc = 4 + c;
      const float2 Cr = face(wc);
      const float2 dF = POS ? fma2(sub2(Cr, Cl), sixth, Dw[wc - 1])
                            : fma2(sub2(Cl, Cr), sixth, Dw[wc]);
      Cl = Cr;
      // f^eq for the two cells of this slot: coefficients (x cell, y cell) per m
      const float* cc = ck + (size_t)(i + c - 4) * (2 * kMP);
      float2 feq = splat(0.f);
#pragma unroll
      for (int m0 = 0; m0 < kMP; m0 += 2) {
        if (m0 < nm) {
          float2 cv[2];
          ld2slots(cc + 2 * m0, cv);
          feq = fma2(cv[0], wp2[m0], feq);
          feq = fma2(cv[1], wp2[m0 + 1], feq);
        }
      }
      const float4 g = *reinterpret_cast<const float4*>(gco + 4 * (i + c - 4));
      const float2 g0 = make_float2(g.x, g.y), g1 = make_float2(g.z, g.w);
      const float2 f = R[wc];
      const float2 rate = fma2(splat(-xi), g1, g0);  // g0 - g1 xi
      const float2 coll = mul2(rate, sub2(f, feq));
      const float2 L = fma2(splat(-inv_dz), dF, mul2(splat(-1.f), coll));
      out[c] = fma2(splat(dt), L, f);
    }
    if (t + 1 < kH / 2) {
#pragma unroll
      for (int c = 0; c < NW - 2; ++c) {
        J[c] = J[c + 2];
        R[c] = R[c + 2];
      }
#pragma unroll
      for (int c = 0; c < NW - 3; ++c) {
        Dw[c] = Dw[c + 2];
        Kw[c] = Kw[c + 2];
      }
      ld_slot_pair(row, i + 6, R + NW - 2);  // slots i+6, i+7
      J[NW - 2] = mul2(xi2, R[NW - 2]);
      J[NW - 1] = mul2(xi2, R[NW - 1]);
#pragma unroll
      for (int c = NW - 3; c < NW - 1; ++c) {
        Dw[c] = sub2(J[c + 1], J[c]);
        const float2 d2 = sub2(Dw[c], Dw[c - 1]);
        Kw[c] = mul2(mul2(k13, d2), d2);
      }
    }
    *reinterpret_cast<float2*>(row + i) = make_float2(out[0].x, out[1].x);
    if (t < 2) {
      held[t] = make_float2(out[0].y, out[1].y);
    } else {
      *reinterpret_cast<float2*>(row + i + kH) = make_float2(out[0].y, out[1].y);
    }
    if (t == kH / 2 - 2) {  // the last two slots have just been read
      *reinterpret_cast<float2*>(row + 4 + kH) = held[0];
      *reinterpret_cast<float2*>(row + 6 + kH) = held[1];
    }
  }
}

// Value of ghost cell sc (outside [0, Z)) of velocity row v under the
// boundary rule (Sec. IV A: fixed equilibria; outflow copies; periodic).
__device__ __forceinline__ float ghost_value(const float* __restrict__ fin, const SodGeom& g,
                                             const SodTables<float>& tb, int v, int sc) {
  if (g.bc == kBcPeriodic) {
    int sp = sc % g.Z;
    if (sp < 0) sp += g.Z;
    return fin[(size_t)v * g.ldz + sp];
  }
  if (g.bc == kBcOutflow) return fin[(size_t)v * g.ldz + (sc < 0 ? 0 : g.Z - 1)];
  return sc < 0 ? tb.ghostL[v] : tb.ghostR[v];
}

// Staging by plain loads, any tile: cell s0-4+p goes to position p
// (0 <= p < kC), ghost cells by the boundary rule.  Threads t of nt.
__device__ __forceinline__ void stage_plain(float* tile, const float* __restrict__ fin,
                                            const SodGeom& g, const SodTables<float>& tb, int s0,
                                            int t, int nt) {
  const int V = g.V;
  for (int idx = t; idx < V * kC; idx += nt) {
    const int v = idx / kC, c = idx - v * kC;
    const int sc = s0 - 4 + c;
    tile[v * kP + c] = (sc >= 0 && sc < g.Z) ? fin[(size_t)v * g.ldz + sc]
                                             : ghost_value(fin, g, tb, v, sc);
  }
}

// Staging of an interior tile by plain 16-byte loads, eight in flight per thread.
__device__ __forceinline__ void stage_interior_vec(float* tile, const float* __restrict__ fin,
                                                   const SodGeom& g, int s0, int t, int nt) {
  const int V = g.V;
  const float* src = fin + s0 - 4;
  for (int base_i = t; base_i < V * (kC / 4); base_i += kInflight * nt) {
    float4 x[kInflight];
#pragma unroll
    for (int u = 0; u < kInflight; ++u) {
      const int idx = base_i + u * nt;
      if (idx < V * (kC / 4)) {
        const int v = idx / (kC / 4), q = idx - v * (kC / 4);
        x[u] = __ldg(reinterpret_cast<const float4*>(src + (size_t)v * g.ldz + 4 * q));
      }
    }
#pragma unroll
    for (int u = 0; u < kInflight; ++u) {
      const int idx = base_i + u * nt;
      if (idx < V * (kC / 4)) {
        const int v = idx / (kC / 4), q = idx - v * (kC / 4);
        *reinterpret_cast<float4*>(tile + v * kP + 4 * q) = x[u];
      }
    }
  }
}

// After a bulk-tensor copy of a boundary tile (out-of-range cells read as
// zero): overwrite the positions whose cells lie outside [0, Z) with their
// ghost values.  Only the leftmost tile has such cells on the left (p < 4)
// and only tiles reaching past Z on the right.  Threads t of nt.
__device__ __forceinline__ void fix_ghosts(float* tile, const float* __restrict__ fin,
                                           const SodGeom& g, const SodTables<float>& tb, int s0,
                                           int t, int nt) {
  const int V = g.V;
  const int nl = s0 - 4 < 0 ? 4 - s0 : 0;                        // leading positions
  const int first_r = g.Z - (s0 - 4);                             // first position >= Z
  const int nr = first_r < kC ? kC - (first_r < 0 ? 0 : first_r) : 0;
  const int per = nl + nr;
  if (per == 0) return;
  for (int idx = t; idx < V * per; idx += nt) {
    const int v = idx / per, q = idx - v * per;
    const int p = q < nl ? q : kC - nr + (q - nl);
    tile[v * kP + p] = ghost_value(fin, g, tb, v, s0 - 4 + p);
  }
}

// Moments of the kB2 cells of a staged tile: warp w (0 <= w < kB2/4) owns
// cells 4w .. 4w+3, its lanes take rows; blocks of four rows,
// Kahan-compensated across blocks.  msum[q*kB2 + c] = sum_v f w_q (FP64 from
// the compensated FP32 hi + lo).  mws: the five moment weights [5][V].
__device__ __forceinline__ void moments(const float* tile, const float* mws, double* msum, int V,
                                        int warp, int lane) {
  // cells (0, 1) and (2, 3) of the warp's four are the two lanes of packed
  // FP32x2 values (adjacent in the 16-byte loads): same roundings as the
  // scalar fma / Kahan steps, half the instructions
  float2 s2[2][5], c2[2][5];
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int q = 0; q < 5; ++q) { s2[p][q] = splat(0.f); c2[p][q] = splat(0.f); }
  for (int v0 = lane; v0 < V; v0 += 128) {
    float2 b2[2][5];
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < 5; ++q) b2[p][q] = splat(0.f);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int v = v0 + 32 * u;
      if (v < V) {
        const float4 x = *reinterpret_cast<const float4*>(tile + v * kP + 4 + 4 * warp);
        const float2 X0 = make_float2(x.x, x.y), X1 = make_float2(x.z, x.w);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          const float2 W = splat(mws[q * V + v]);
          b2[0][q] = fma2(X0, W, b2[0][q]);
          b2[1][q] = fma2(X1, W, b2[1][q]);
        }
      }
    }
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const float2 y = sub2(b2[p][q], c2[p][q]);
        const float2 t = add2(s2[p][q], y);
        c2[p][q] = sub2(sub2(t, s2[p][q]), y);
        s2[p][q] = t;
      }
  }
  float s[4][5], cpen[4][5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    s[0][q] = s2[0][q].x; s[1][q] = s2[0][q].y; s[2][q] = s2[1][q].x; s[3][q] = s2[1][q].y;
    cpen[0][q] = c2[0][q].x; cpen[1][q] = c2[0][q].y;
    cpen[2][q] = c2[1][q].x; cpen[3][q] = c2[1][q].y;
  }
  // FP32 transposing reduction of the 20 (sum, -compensation) pairs; only
  // the final hi + lo of each is formed in FP64
  float h[32], lo[32];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      h[c * 5 + q] = s[c][q];
      lo[c * 5 + q] = -cpen[c][q];
    }
#pragma unroll
  for (int i = 20; i < 32; ++i) {
    h[i] = 0.f;
    lo[i] = 0.f;
  }
  tr_level<16>(h, lo, lane);
  tr_level<8>(h, lo, lane);
  tr_level<4>(h, lo, lane);
  tr_level<2>(h, lo, lane);
  tr_level<1>(h, lo, lane);
  if (lane < 20) {
    const int c = lane / 5, q = lane - 5 * (lane / 5);
    msum[q * kB2 + 4 * warp + c] = (double)h[0] + (double)lo[0];
  }
}

// Landau matching (FP64) and relaxation time of cell c (0 <= c < kB2) of the
// tile at s0; what the f^eq coefficients need goes to cellf [8][kB2] in FP32,
// the collision rates gamma/tau and gamma beta/tau to gco [kH][g0x g0y g1x g1y].
__device__ __forceinline__ void landau_cell(const double* msum, float* cellf, float* gco,
                                            const SodGeom& g, int s0, int c, int* err) {
  LandauOut Lo = landau_factored(msum[c], msum[kB2 + c], msum[2 * kB2 + c], msum[3 * kB2 + c],
                                 msum[4 * kB2 + c]);
  float g0 = 0.f, g1 = 0.f;
  if (!Lo.ok) {
    if (s0 + c < g.Z) report_err(err, 6, s0 + c);
    Lo.n = 1.0; Lo.T = 1.0; Lo.beta = 0.0; Lo.gamma = 1.0; Lo.u = 0.0;
  } else if (g.tau_mode == kTauEtas) {
    const double tau = g.tau_AW0 / Lo.T *
                       (1.0 - 0.25 * log(Lo.n / (Lo.T * Lo.T * Lo.T) * g.lambda_ref));
    g0 = float(Lo.gamma / tau);
    g1 = float(Lo.gamma * Lo.beta / tau);
  } else {
    const float itau = 1.f / float(g.tau);
    g0 = float(Lo.gamma) * itau;
    g1 = float(Lo.gamma * Lo.beta) * itau;
  }
  const float u = float(Lo.u);
  const float A = asinhf(u);
  cellf[0 * kB2 + c] = float(Lo.n);
  cellf[1 * kB2 + c] = float(Lo.T);
  cellf[2 * kB2 + c] = u;
  cellf[3 * kB2 + c] = A;
  cellf[4 * kB2 + c] = (u > 0.f) ? A / u : 1.f;
  cellf[5 * kB2 + c] = u * u / (float(Lo.gamma) + 1.f);  // 2 sinh^2(A/2) = gamma - 1
  cellf[6 * kB2 + c] = (Lo.beta < 0.0) ? -1.f : 1.f;
  cellf[7 * kB2 + c] = Lo.ok ? 1.f : 0.f;
  // gco[i][g0x g0y g1x g1y], cell c = half h, index i
  const int h = c / kH, i = c - h * kH;
  gco[4 * i + h] = g0;
  gco[4 * i + 2 + h] = g1;
}

// FP32 constants of the coefficient phase, copied into shared memory by
// load_consts: cst[0..15] the nodes and cst[16..31] the weights of the 16-node
// Gauss-Legendre rule of the a_{l,m} integrals, cst[32 + k] = L_1^{(2)}(x_k).
constexpr int kConsts = 32 + 8;

__device__ __forceinline__ void load_consts(float* cst, const SodTables<float>& tb, int QL, int t,
                                            int nt) {
  for (int e = t; e < 32 + QL; e += nt)
    cst[e] = e < 16 ? float(tb.gl_t[kAeqNodes + e])
                    : (e < 32 ? float(tb.gl_w[kAeqNodes + e - 16]) : tb.L1k[e - 32]);
}

// f^eq coefficients of the tile: thread t (0 <= t < 8 kB2), 8 threads per cell
// share the 16 nodes of the a_{l,m} rule; after an xor butterfly every thread
// of a cell holds all the integrals, and thread q writes the coefficients of
// order m = q for every radial node; coef [QL][kH][kMP][2 halves].
__device__ __forceinline__ void coefs(const float* cellf, float* coef, const SodGeom& g,
                                      const float* cst, int t) {
  static_assert(kMP == 8, "one thread per order m");
  const int c = t >> 3, q = t & 7;  // 8 threads per cell
  const float ud = cellf[2 * kB2 + c];
  const float A = cellf[3 * kB2 + c], sh2 = cellf[5 * kB2 + c];
  const float uinv = (ud > 0.f) ? 1.f / ud : 0.f;
  const bool at_rest = !(ud > 0.f);
  float J3[kMaxM], J4[kMaxM];
#pragma unroll
  for (int m = 0; m < kMaxM; ++m) { J3[m] = 0.f; J4[m] = 0.f; }
#pragma unroll
  for (int i = 0; i < kAeqNodesF32 / 8; ++i)  // the 16-node rule (N_Omega <= 7 here)
    aeq_node<float>(cst[q + 8 * i], cst[16 + q + 8 * i], A, sh2, uinv, at_rest, g.nm, J3, J4);
#pragma unroll
  for (int o = 4; o >= 1; o >>= 1)
#pragma unroll
    for (int m = 0; m < kMaxM; ++m)
      if (m < g.nm) {
        J3[m] += __shfl_xor_sync(0xffffffffu, J3[m], o);
        J4[m] += __shfl_xor_sync(0xffffffffu, J4[m], o);
      }
  const int m = q;
  float j3 = 0.f, j4 = 0.f;
#pragma unroll
  for (int mm = 0; mm < kMP; ++mm)
    if (mm == m) {
      j3 = J3[mm];
      j4 = J4[mm];
    }
  const float fac = cellf[7 * kB2 + c] * cellf[0 * kB2 + c] * cellf[4 * kB2 + c] * 0.25f;
  const float theta = cellf[1 * kB2 + c];
  const float sgn = cellf[6 * kB2 + c];
  const int h = c / kH, i = c - h * kH;
  const float sm = ((m & 1) && sgn < 0.f) ? -fac : fac;  // fac sgn^m (sgn = +-1)
  const float hh = sm * (float(m) + 0.5f);                // (2m + 1)/2, exact
  const float d = j3 - theta * j4;
  for (int k = 0; k < g.QL; ++k)
    coef[(((size_t)k * kH + i) * kMP + m) * 2 + h] =
        m < g.nm ? hh * (j3 + cst[32 + k] * d) : 0.f;
}

// Row sweeps: rows ir = first, first + stride, ... (negative-xi rows first,
// so the upwind direction is uniform within a warp).
__device__ __forceinline__ void sweep_rows(float* tile, const float* coef, const float* gco,
                                           const SodGeom& g, const SodTables<float>& tb,
                                           const int* __restrict__ rowv, int nneg, int first,
                                           int stride) {
  const float inv_dz = float(g.inv_dz), dt = float(g.dt);
  const int V = g.V;
  for (int ir = first; ir < V; ir += stride) {
    const int v = rowv[ir];
    const float xi = tb.xi[v];
    const int k = tb.kidx[v];
    float2 wp2[kMP];
#pragma unroll
    for (int m = 0; m < kMP; ++m) wp2[m] = splat((m < g.nm) ? tb.wp[m * V + v] : 0.f);
    const float* ck = coef + (size_t)k * kH * kMP * 2;
    if (ir >= nneg) sweep_row2<true>(tile + v * kP, xi, wp2, g.nm, ck, gco, inv_dz, dt);
    else sweep_row2<false>(tile + v * kP, xi, wp2, g.nm, ck, gco, inv_dz, dt);
  }
}

// Per-row tables of the sweep in row order (shared memory): velocity index,
// xi, radial index and w_j w_k P_m(xi_j) [kMP][V]; the same values as the
// tables sweep_rows reads from global memory.
struct RowTables {
  int* v;
  float* xi;
  int* k;
  float* wp;
};

__device__ __forceinline__ void load_row_tables(const RowTables& rt, const SodGeom& g,
                                                const SodTables<float>& tb,
                                                const int* __restrict__ rowv, int t, int nt) {
  const int V = g.V;
  for (int ir = t; ir < V; ir += nt) {
    const int v = rowv[ir];
    rt.v[ir] = v;
    rt.xi[ir] = tb.xi[v];
    rt.k[ir] = tb.kidx[v];
#pragma unroll
    for (int m = 0; m < kMP; ++m) rt.wp[m * V + ir] = (m < g.nm) ? tb.wp[m * V + v] : 0.f;
  }
}

__device__ __forceinline__ void sweep_rows_tab(float* tile, const float* coef, const float* gco,
                                               const SodGeom& g, const RowTables& rt, int nneg,
                                               int first, int stride) {
  const float inv_dz = float(g.inv_dz), dt = float(g.dt);
  const int V = g.V;
  for (int ir = first; ir < V; ir += stride) {
    const int v = rt.v[ir];
    const float xi = rt.xi[ir];
    const int k = rt.k[ir];
    float2 wp2[kMP];
#pragma unroll
    for (int m = 0; m < kMP; ++m) wp2[m] = splat(rt.wp[m * V + ir]);
    const float* ck = coef + (size_t)k * kH * kMP * 2;
    if (ir >= nneg) sweep_row2<true>(tile + v * kP, xi, wp2, g.nm, ck, gco, inv_dz, dt);
    else sweep_row2<false>(tile + v * kP, xi, wp2, g.nm, ck, gco, inv_dz, dt);
  }
}

// Store: cell c of the tile is position 4 + c; stages 2 and 3 combine with
// f_n (Eq. rk3: 3/4 f_n + 1/4 f, then 1/3 f_n + 2/3 f).  Threads t of nt.
template <int INFL = kInflight>
__device__ __forceinline__ void store(const float* tile, const float* __restrict__ fn, float* fout,
                                      const SodGeom& g, int stage, int s0, int t, int nt) {
  const int V = g.V;
  const float a = (stage == 1) ? 0.75f : 1.f / 3.f;
  const float b = (stage == 1) ? 0.25f : 2.f / 3.f;
  if (s0 + kB2 <= g.Z) {
    // full tile: kB2/4 chunks of 4 cells per row, 16-byte accesses, INFL loads
    // of f_n in flight per thread
    for (int base_i = t; base_i < V * (kB2 / 4); base_i += INFL * nt) {
      float4 fo[INFL];
#pragma unroll
      for (int u = 0; u < INFL; ++u) {
        const int idx = base_i + u * nt;
        if (stage != 0 && idx < V * (kB2 / 4)) {
          const int v = idx / (kB2 / 4), q = idx - v * (kB2 / 4);
          fo[u] = __ldg(reinterpret_cast<const float4*>(fn + (size_t)v * g.ldz + s0 + 4 * q));
        }
      }
#pragma unroll
      for (int u = 0; u < INFL; ++u) {
        const int idx = base_i + u * nt;
        if (idx < V * (kB2 / 4)) {
          const int v = idx / (kB2 / 4), q = idx - v * (kB2 / 4);
          float4 r = *reinterpret_cast<const float4*>(tile + v * kP + 4 + 4 * q);
          if (stage != 0) {
            r.x = a * fo[u].x + b * r.x;
            r.y = a * fo[u].y + b * r.y;
            r.z = a * fo[u].z + b * r.z;
            r.w = a * fo[u].w + b * r.w;
          }
          *reinterpret_cast<float4*>(fout + (size_t)v * g.ldz + s0 + 4 * q) = r;
        }
      }
    }
  } else {
    for (int idx = t; idx < V * kB2; idx += nt) {
      const int v = idx / kB2, c = idx - v * kB2;
      const int sc = s0 + c;
      if (sc < g.Z) {
        const size_t o = (size_t)v * g.ldz + sc;
        float r = tile[v * kP + 4 + c];
        if (stage != 0) r = a * fn[o] + b * r;
        fout[o] = r;
      }
    }
  }
}

}  // namespace p32

// Host: tensor map of one FP32 population buffer [V][Z] with row stride ldz,
// boxes of box_cells cells x box_rows rows, zero fill outside (sod32.cu).
bool sod32_make_map(CUtensorMap* m, const float* f, int Z, int ldz, int V, int box_cells,
                    int box_rows);

}  // namespace rslb
