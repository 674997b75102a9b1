// sod32.cu -- FP32 RK-stage kernel of the Sod shock tube using the packed
// FP32x2 instructions of sm_100+ (FFMA2 / FADD2 / FMUL2).
//
// A CTA owns 28 output cells, split into two halves of 14; one thread walks a
// velocity row and advances both halves in lock-step, the left half in the x
// lane and the right half in the y lane of float2 values, so every arithmetic
// instruction of the sweep does two cells.  Shared-memory rows are stored as
// 22 float2 "slots": slot s holds (cell s0-4+s, cell s0+10+s), i.e. each half
// with its own 4-cell halo on each side.  The rest of the stage -- moments
// (Kahan-compensated FP32, FP64 combination), FP64 Landau matching, the f^eq
// coefficients, WENO5 in difference form, relaxation, RK update -- follows
// the scalar kernel of sod.cu.
#include "rslb_device.cuh"
#include "sod.cuh"

namespace rslb {
namespace {

constexpr int kH = 14;          // cells per half
constexpr int kB2 = 2 * kH;     // output cells per CTA
constexpr int kS = kH + 8;      // float2 slots per row (4-cell halo per side)
constexpr int kP = 2 * kS;      // floats per row: 44 = 11 x 16 B (odd count)
constexpr int kNT = 224;        // 7 warps: one per two-slot chunk in the moments
constexpr int kMP = 8;          // coefficient pitch (m) for N_Omega <= 7

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

__device__ __forceinline__ double warp_sum_d(double x) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  return x;
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
  const float mx = fmaxf(s1.x, fmaxf(s2.x, s3.x));
  const float my = fmaxf(s1.y, fmaxf(s2.y, s3.y));
  const float2 inv = make_float2(mx > tiny ? rcp_approx(mx) : 0.f, my > tiny ? rcp_approx(my) : 0.f);
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

template <bool POS>
__device__ __forceinline__ float2 face_corr2(const float2* J, int wc) {
  const float2 k13 = splat(13.f / 12.f);
  auto D = [&](int c) { return sub2(J[c + 1], J[c]); };
  auto K = [&](int c) {
    const float2 s2 = sub2(sub2(J[c + 1], J[c]), sub2(J[c], J[c - 1]));
    return mul2(mul2(k13, s2), s2);
  };
  if constexpr (POS)
    return weno_corr2(D(wc - 2), D(wc - 1), D(wc), D(wc + 1), K(wc - 1), K(wc), K(wc + 1));
  else
    return weno_corr2(sub2(splat(0.f), D(wc + 2)), sub2(splat(0.f), D(wc + 1)),
                      sub2(splat(0.f), D(wc)), sub2(splat(0.f), D(wc - 1)), K(wc + 2),
                      K(wc + 1), K(wc));
}

// Sweep a whole row (both halves): slots 4..17 are the outputs; window of
// 10 slots [i-4, i+6) around the current two-slot chunk i.
template <bool POS>
__device__ __forceinline__ void sweep_row2(float* row, float xi, const float2* wp2, int nm,
                                           const float* __restrict__ ck,
                                           const float* __restrict__ gco, float inv_dz,
                                           float dt) {
  constexpr int NW = 10;
  const float2 xi2 = splat(xi);
  const float2 sixth = splat(1.f / 6.f);
  float2 R[NW], J[NW];
#pragma unroll
  for (int c = 0; c < NW; c += 2) ld2slots(row + 2 * c, R + c);
#pragma unroll
  for (int c = 0; c < NW; ++c) J[c] = mul2(xi2, R[c]);
  float2 Cl = face_corr2<POS>(J, 3);
#pragma unroll
  for (int t = 0; t < kH / 2; ++t) {
    const int i = 4 + 2 * t;  // slot of the first cell of this chunk
    float2 out[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int wc = 4 + c;
      const float2 Cr = face_corr2<POS>(J, wc);
      const float2 dJ = POS ? sub2(J[wc], J[wc - 1]) : sub2(J[wc + 1], J[wc]);
      const float2 dF = fma2(sub2(Cr, Cl), sixth, dJ);
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
      ld2slots(row + 2 * (i + 6), R + NW - 2);  // slots i+6, i+7
      J[NW - 2] = mul2(xi2, R[NW - 2]);
      J[NW - 1] = mul2(xi2, R[NW - 1]);
    }
    *reinterpret_cast<float4*>(row + 2 * i) = make_float4(out[0].x, out[0].y, out[1].x, out[1].y);
  }
}

}  // namespace

// Shared memory: tile [V][kP] floats, then partial moments, cell scalars,
// coefficients [QL][kH][kMP][2] floats and gco [kH][4] floats.
size_t sod32_smem_bytes(int V, int QL) {
  auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
  return al(sizeof(float) * (size_t)V * kP) + al(sizeof(double) * 5 * kB2) +
         al(sizeof(double) * 8 * kB2) + al(sizeof(float) * (size_t)QL * kH * kMP * 2) +
         al(sizeof(float) * kH * 4);
}

// One stage of one tile starting at cell s0 (the whole CTA).
__device__ __forceinline__ void sod32_tile(const float* __restrict__ fin,
                                           const float* __restrict__ fn, float* fout, int stage,
                                           int* err, const SodGeom& g, const SodTables<float>& tb,
                                           const int* __restrict__ rowv, int nneg, int s0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
  const int V = g.V;
  float* tile = reinterpret_cast<float*>(smem_raw);
  double* msum = reinterpret_cast<double*>(smem_raw + al(sizeof(float) * (size_t)V * kP));
  double* cell = msum + 5 * kB2;
  float* coef = reinterpret_cast<float*>(cell + 8 * kB2);  // [QL][kH][kMP][2]
  float* gco = coef + (size_t)g.QL * kH * kMP * 2;         // [kH][g0x g0y g1x g1y]

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // ---- 1. stage rows: cell c (relative to s0-4, 0 <= c < 36) goes to slot c
  //         (x, left half) if c < 22 and to slot c-14 (y, right half) if c >= 14 ----
  const bool interior = (s0 - 4 >= 0) && (s0 + kB2 + 4 <= g.Z);
  if (interior) {
    // four 16-byte loads in flight per thread before any shared-memory store
    const float* src = fin + s0 - 4;
    for (int base = tid; base < V * 9; base += 4 * kNT) {
      float4 x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int idx = base + u * kNT;
        if (idx < V * 9) {
          const int v = idx / 9, q = idx - v * 9;
          x[u] = __ldg(reinterpret_cast<const float4*>(src + (size_t)v * g.ldz + 4 * q));
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int idx = base + u * kNT;
        if (idx < V * 9) {
          const int v = idx / 9, q = idx - v * 9;
          float* row = tile + v * kP;
          const float e[4] = {x[u].x, x[u].y, x[u].z, x[u].w};
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            const int c = 4 * q + w;
            if (c < kS) row[2 * c] = e[w];
            if (c >= kH) row[2 * (c - kH) + 1] = e[w];
          }
        }
      }
    }
  } else {
    for (int idx = tid; idx < V * 36; idx += kNT) {
      const int v = idx / 36, c = idx - v * 36;
      const int s = s0 - 4 + c;
      float val;
      if (s >= 0 && s < g.Z) val = fin[(size_t)v * g.ldz + s];
      else if (g.bc == kBcPeriodic) {
        int sp = s % g.Z;
        if (sp < 0) sp += g.Z;
        val = fin[(size_t)v * g.ldz + sp];
      } else if (g.bc == kBcOutflow) val = fin[(size_t)v * g.ldz + (s < 0 ? 0 : g.Z - 1)];
      else val = s < 0 ? tb.ghostL[v] : tb.ghostR[v];
      float* row = tile + v * kP;
      if (c < kS) row[2 * c] = val;
      if (c >= kH) row[2 * (c - kH) + 1] = val;
    }
  }
  __syncthreads();

  const bool collide = g.tau_mode != kTauNone;
  if (collide) {
    // ---- 2. moments: warp w owns slots 4+2w, 5+2w (4 cells), lanes own rows;
    //         blocks of four rows, Kahan-compensated across blocks ----
    {
      float s[4][5], cpen[4][5];
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int q = 0; q < 5; ++q) { s[c][q] = 0.f; cpen[c][q] = 0.f; }
      for (int v0 = lane; v0 < V; v0 += 128) {
        float blk[4][5];
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int q = 0; q < 5; ++q) blk[c][q] = 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int v = v0 + 32 * u;
          if (v < V) {
            const float4 x = *reinterpret_cast<const float4*>(tile + v * kP + 2 * (4 + 2 * warp));
            const float e[4] = {x.x, x.y, x.z, x.w};
            float w[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) w[q] = tb.mw[q * V + v];
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
              for (int q = 0; q < 5; ++q) blk[c][q] = fmaf(e[c], w[q], blk[c][q]);
          }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int q = 0; q < 5; ++q) {
            const float y = blk[c][q] - cpen[c][q];
            const float t = s[c][q] + y;
            cpen[c][q] = (t - s[c][q]) - y;
            s[c][q] = t;
          }
      }
      // element e of the float4 is: slot 4+2w (x, y), slot 5+2w (x, y)
      // x = left half cell 2w + {0,1}, y = right half cell 14 + 2w + {0,1}
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int cellidx = (c & 1) ? kH + 2 * warp + (c >> 1) : 2 * warp + (c >> 1);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          const double sum = warp_sum_d((double)s[c][q] - (double)cpen[c][q]);
          if (lane == 0) msum[q * kB2 + cellidx] = sum;
        }
      }
    }
    __syncthreads();

    // ---- 3a. Landau matching (FP64) and relaxation time, one thread per cell ----
    if (tid < kB2) {
      const int c = tid;
      LandauOut Lo = landau_factored(msum[c], msum[kB2 + c], msum[2 * kB2 + c],
                                     msum[3 * kB2 + c], msum[4 * kB2 + c]);
      double g0 = 0.0, g1 = 0.0;
      if (!Lo.ok) {
        if (s0 + c < g.Z) report_err(err, 6, s0 + c);
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
      cell[0 * kB2 + c] = Lo.n;
      cell[1 * kB2 + c] = Lo.T;
      cell[2 * kB2 + c] = Lo.u;
      cell[3 * kB2 + c] = A;
      cell[4 * kB2 + c] = (Lo.u > 0.0) ? A / Lo.u : 1.0;
      cell[5 * kB2 + c] = 2.0 * sh * sh;
      cell[6 * kB2 + c] = (Lo.beta < 0.0) ? -1.0 : 1.0;
      cell[7 * kB2 + c] = Lo.ok ? 1.0 : 0.0;
      // gco[i][g0x g0y g1x g1y], cell c = half h, index i
      const int h = c / kH, i = c - h * kH;
      gco[4 * i + h] = float(g0);
      gco[4 * i + 2 + h] = float(g1);
    }
    __syncthreads();

    // ---- 3b. f^eq coefficients: 8 threads per cell share the 32 nodes ----
    {
      const int c = tid >> 3, q = tid & 7;  // 28 cells x 8 = 224 threads
      const double ud = cell[2 * kB2 + c];
      const float A = float(cell[3 * kB2 + c]), sh2 = float(cell[5 * kB2 + c]);
      const float uinv = (ud > 0.0) ? float(1.0 / ud) : 0.f;
      const bool at_rest = !(ud > 0.0);
      float J3[kMaxM], J4[kMaxM];
#pragma unroll
      for (int m = 0; m < kMaxM; ++m) { J3[m] = 0.f; J4[m] = 0.f; }
#pragma unroll
      for (int i = 0; i < kAeqNodes / 8; ++i)
        aeq_node<float>(float(tb.gl_t[q + 8 * i]), float(tb.gl_w[q + 8 * i]), A, sh2, uinv,
                        at_rest, g.nm, J3, J4);
#pragma unroll
      for (int o = 4; o >= 1; o >>= 1)
#pragma unroll
        for (int m = 0; m < kMaxM; ++m)
          if (m < g.nm) {
            J3[m] += __shfl_xor_sync(0xffffffffu, J3[m], o);
            J4[m] += __shfl_xor_sync(0xffffffffu, J4[m], o);
          }
      if (q == 0) {
        const float fac = float(cell[7 * kB2 + c] * cell[0 * kB2 + c] * cell[4 * kB2 + c] * 0.25);
        const float theta = float(cell[1 * kB2 + c]);
        const float sgn = float(cell[6 * kB2 + c]);
        const int h = c / kH, i = c - h * kH;
        float sm = fac;
#pragma unroll
        for (int m = 0; m < kMP; ++m) {
          if (m < g.nm) {
            const float hh = sm * float(0.5 * (2 * m + 1));
            const float d = J3[m] - theta * J4[m];
            for (int k = 0; k < g.QL; ++k)
              coef[(((size_t)k * kH + i) * kMP + m) * 2 + h] = hh * (J3[m] + tb.L1k[k] * d);
            sm *= sgn;
          } else {
            for (int k = 0; k < g.QL; ++k) coef[(((size_t)k * kH + i) * kMP + m) * 2 + h] = 0.f;
          }
        }
      }
    }
    __syncthreads();
  } else {
    for (int i = tid; i < g.QL * kH * kMP * 2 + kH * 4; i += kNT) coef[i] = 0.f;
    __syncthreads();
  }

  // ---- 4. row sweeps (negative-xi rows first: warp-uniform direction) ----
  const float inv_dz = float(g.inv_dz), dt = float(g.dt);
  for (int ir = tid; ir < V; ir += kNT) {
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
  __syncthreads();

  // ---- 5. store: cell c of the tile = slot 4 + (c mod 14), half c / 14 ----
  const float a = (stage == 1) ? 0.75f : 1.f / 3.f;
  const float b = (stage == 1) ? 0.25f : 2.f / 3.f;
  if (s0 + kB2 <= g.Z) {
    // full tile: 7 chunks of 4 cells per row, 16-byte global accesses, four
    // loads of f_n in flight per thread
    for (int base = tid; base < V * 7; base += 4 * kNT) {
      float4 fo[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int idx = base + u * kNT;
        if (stage != 0 && idx < V * 7) {
          const int v = idx / 7, q = idx - v * 7;
          fo[u] = __ldg(reinterpret_cast<const float4*>(fn + (size_t)v * g.ldz + s0 + 4 * q));
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int idx = base + u * kNT;
        if (idx < V * 7) {
          const int v = idx / 7, q = idx - v * 7;
          const float* row = tile + v * kP;
          float r[4];
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            const int c = 4 * q + w;
            const int h = c >= kH, i = c - h * kH;
            r[w] = row[2 * (4 + i) + h];
          }
          if (stage != 0) {
            r[0] = a * fo[u].x + b * r[0];
            r[1] = a * fo[u].y + b * r[1];
            r[2] = a * fo[u].z + b * r[2];
            r[3] = a * fo[u].w + b * r[3];
          }
          *reinterpret_cast<float4*>(fout + (size_t)v * g.ldz + s0 + 4 * q) =
              make_float4(r[0], r[1], r[2], r[3]);
        }
      }
    }
  } else {
    for (int idx = tid; idx < V * kB2; idx += kNT) {
      const int v = idx / kB2, c = idx - v * kB2;
      const int s = s0 + c;
      if (s < g.Z) {
        const int h = c / kH, i = c - h * kH;
        const size_t o = (size_t)v * g.ldz + s;
        float r = tile[v * kP + 2 * (4 + i) + h];
        if (stage != 0) r = a * fn[o] + b * r;
        fout[o] = r;
      }
    }
  }
}

__global__ void __launch_bounds__(kNT, 2)
sod32_stage_kernel(const float* __restrict__ fin, const float* __restrict__ fn, float* fout,
                   int stage, int* err, SodGeom g, SodTables<float> tb, const int* __restrict__ rowv,
                   int nneg) {
  sod32_tile(fin, fn, fout, stage, err, g, tb, rowv, nneg, blockIdx.x * kB2);
}

// Batched: a persistent grid walks the task list of all runs of one class.
__global__ void __launch_bounds__(kNT, 2)
sod32_batch_kernel(const SodRunDesc<float>* __restrict__ runs, const SodTask* __restrict__ tasks,
                   int ntasks, const long long* __restrict__ step, int stage, int* err) {
  const long long n = *step;
  for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const SodTask tk = tasks[t];
    const SodRunDesc<float> R = runs[tk.run];
    if (n >= R.nsteps) break;  // tasks are ordered by decreasing step count
    const float* fin = stage == 0 ? R.F0 : (stage == 1 ? R.F1 : R.F2);
    float* fout = stage == 0 ? R.F1 : (stage == 1 ? R.F2 : R.F0);
    sod32_tile(fin, R.F0, fout, stage, err, R.g, R.tb, R.rowv, R.nneg, tk.s0);
    __syncthreads();
  }
}

cudaError_t sod32_batch_launch(size_t smem, int grid, const SodRunDesc<float>* runs,
                               const SodTask* tasks, int ntasks, const long long* step, int stage,
                               int* err, cudaStream_t st) {
  sod32_batch_kernel<<<grid, kNT, smem, st>>>(runs, tasks, ntasks, step, stage, err);
  return cudaGetLastError();
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
    cudaError_t e = cudaFuncSetAttribute(sod32_stage_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int grid = (g.Z + kB2 - 1) / kB2;
  sod32_stage_kernel<<<grid, kNT, sod32_smem_bytes(g.V, g.QL), st>>>(fin, fn, fout, stage, err, g,
                                                                      tb, rowv, nneg);
  return cudaGetLastError();
}

}  // namespace rslb
