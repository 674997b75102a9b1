// rslb_device.cuh -- device building blocks of the R-SLB step (sm_103a).
//
// Landau matching, the WENO5 face flux and the f^eq expansion coefficients,
// templated on the working precision.  Used by the Sod and Bjorken kernels.
#pragma once

#include <cfloat>
#include <cstdint>
#include <cuda_runtime.h>

namespace rslb {

constexpr int kMaxM = 13;    // N_Omega <= 12
constexpr int kAeqNodes = 32;  // Gauss-Legendre nodes for the a_{l,m} integrals
// The FP32 stage kernels use a 16-node rule for N_Omega <= 7: for m <= 7 it
// agrees with the exact a_{l,m} to 2e-14 of a_{l,0} up to u = 20 and to 5e-13
// at u = 50, far inside FP32.  The node table holds the 32-node rule and then
// the 16-node one.
constexpr int kAeqNodesF32 = 16;
constexpr int kAeqTable = kAeqNodes + kAeqNodesF32;

template <typename T> struct Prec;
template <> struct Prec<float> {
  static __device__ __forceinline__ float tiny() { return FLT_MIN; }
  static __device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
};
template <> struct Prec<double> {
  static __device__ __forceinline__ double tiny() { return DBL_MIN; }
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
};

__device__ __forceinline__ float dev_exp(float x) { return expf(x); }
__device__ __forceinline__ double dev_exp(double x) { return exp(x); }
__device__ __forceinline__ float dev_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double dev_expm1(double x) { return expm1(x); }

// ---------------------------------------------------------------------------
// WENO5 face flux (Sec. III F, Eqs. flux_weno, weno5_omega).
// (a, b, c, d, e) are the five J = xi f values ordered upwind to downwind
// around the face: (J_{s-2}, J_{s-1}, J_s, J_{s+1}, J_{s+2}) for xi > 0 and
// the mirror (J_{s+3}, J_{s+2}, J_{s+1}, J_s, J_{s-1}) for xi < 0.
// No epsilon: the limiting rules (i)-(iii) decide the weights when smoothness
// indicators vanish.  The weights are scale-invariant, so sigma_q is divided
// by max_q sigma_q first; a ratio whose square is below the smallest normal
// number of T counts as a vanishing sigma_q.  Branch-free, one reciprocal
// for the scale and one for the normalisation.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T weno5_face(T a, T b, T c, T d, T e) {
  const T c6 = T(1) / T(6);
  const T F1 = (T(2) * a - T(7) * b + T(11) * c) * c6;
  const T F2 = (-b + T(5) * c + T(2) * d) * c6;
  const T F3 = (T(2) * c + T(5) * d - e) * c6;
  const T k13 = T(13) / T(12);
  const T d1 = a - T(2) * b + c, e1 = a - T(4) * b + T(3) * c;
  const T d2 = b - T(2) * c + d, e2 = b - d;
  const T d3 = c - T(2) * d + e, e3 = T(3) * c - T(4) * d + e;
  const T s1 = k13 * d1 * d1 + T(0.25) * e1 * e1;
  const T s2 = k13 * d2 * d2 + T(0.25) * e2 * e2;
  const T s3 = k13 * d3 * d3 + T(0.25) * e3 * e3;
  const T D1 = T(0.1), D2 = T(0.6), D3 = T(0.3);
  const bool alleq = (s1 == s2) && (s2 == s3);
  const T smax = fmax(s1, fmax(s2, s3));
  const T inv = alleq ? T(0) : Prec<T>::rcp(smax);
  const T r1 = s1 * inv, r2 = s2 * inv, r3 = s3 * inv;
  const T t1 = r1 * r1, t2 = r2 * r2, t3 = r3 * r3;
  const T tiny = Prec<T>::tiny();
  const bool z1 = t1 < tiny, z2 = t2 < tiny, z3 = t3 < tiny;
  const int nz = int(z1) + int(z2) + int(z3);
  // general case: omega_q ~ delta_q / sigma_q^2, multiplied through by the
  // product of all three t's
  const T n1 = D1 * t2 * t3, n2 = D2 * t1 * t3, n3 = D3 * t1 * t2;
  const T dz = (z1 ? D1 : T(0)) + (z2 ? D2 : T(0)) + (z3 ? D3 : T(0));
  const T den = (nz == 0) ? (n1 + n2 + n3) : ((nz == 1) ? T(1) : dz);
  const T rden = Prec<T>::rcp(den);
  T w1, w2, w3;
  if (nz == 0) {
    w1 = n1 * rden; w2 = n2 * rden; w3 = n3 * rden;
  } else if (nz == 1) {  // rule (iii)
    w1 = z1 ? T(1) : T(0); w2 = z2 ? T(1) : T(0); w3 = z3 ? T(1) : T(0);
  } else {  // rule (ii): the vanishing ones share delta_q / sum
    w1 = z1 ? D1 * rden : T(0); w2 = z2 ? D2 * rden : T(0); w3 = z3 ? D3 * rden : T(0);
  }
  if (alleq) { w1 = D1; w2 = D2; w3 = D3; }  // rule (i)
  return w1 * F1 + w2 * F2 + w3 * F3;
}

// ---------------------------------------------------------------------------
// Landau frame of the 1-D stress tensor (Sec. II E, Eqs. E_landau, u_landau),
// in FP64, from the five direct sums
//   Np = sum f(1+xi), Nm = sum f(1-xi), Ap = sum f p (1+xi)^2,
//   Am = sum f p (1-xi)^2, D = sum f p (1-xi^2).
// With a = sqrt(Ap), b = sqrt(Am) the discriminant of Eq. E_landau is
// (T^tt+T^zz)^2 - 4(T^tz)^2 = Ap*Am, so
//   E = (D + a b)/2,  beta = (a - b)/(a + b),  gamma = (a + b)/(2 sqrt(ab)),
//   n = gamma (N^t - beta N^z) = (b Np + a Nm)/(2 sqrt(ab)),
// which is algebraically identical to the printed formulas and has no
// cancellation as |beta| -> 1 when f >= 0.
// ---------------------------------------------------------------------------
struct LandauOut {
  double n, E, T, beta, gamma, u;  // u = gamma |beta|
  bool ok;
};

__device__ __forceinline__ LandauOut landau_factored(double Np, double Nm, double Ap,
                                                     double Am, double D) {
  LandauOut o;
  const double a = sqrt(Ap), b = sqrt(Am);
  const double ab = a * b, apb = a + b;
  const double sab = sqrt(ab);
  const double X = b * Np + a * Nm;
  // one FP64 division (slow on this part) gives 1/(2 sqrt(ab)), 1/(a+b) and
  // 1/X: r = 1/(sqrt(ab) (a+b) X)
  const double r = 1.0 / (sab * apb * X);
  const double h = 0.5 * apb * X * r;  // 1/(2 sqrt(ab))
  o.E = 0.5 * (D + ab);
  o.beta = (a - b) * sab * X * r;      // (a - b)/(a + b)
  o.gamma = apb * h;
  o.u = fabs(a - b) * h;
  o.n = X * h;
  o.T = (2.0 / 3.0) * o.E * ab * apb * r;  // E/(3n) = 2 E sqrt(ab)/(3X)
  o.ok = (Ap > 0.0) && (Am > 0.0) && (o.E > 0.0) && (o.n > 0.0) && isfinite(o.E) &&
         isfinite(o.n) && isfinite(o.beta) && (fabs(o.beta) < 1.0);
  return o;
}

// ---------------------------------------------------------------------------
// f^eq expansion coefficients (Sec. III D, Eq. aeq_aux).  With u0 = cosh A,
// u = sinh A and the exact substitution u0 - u c = e^{-s}, s = A t:
//   a_{l,m} = n (l+1)(l+2)/(8 pi) (A/u) int_{-1}^{1} dt e^{2s}
//             (1 - theta e^{s})^l P_m(c(s)),
//   c(s) = (2 sinh^2(A/2) - expm1(-s))/u   (c = t when u = 0).
// The integrand is a short sum of exponentials; kAeqNodes Gauss-Legendre
// nodes give round-off accuracy for |beta| up to ~0.95.  This helper adds the
// contribution of one node to J3_m = int e^{2s} P_m, J4_m = int e^{3s} P_m,
// so that a_{0,m} = n (A/u) J3_m/(4 pi) and
// a_{1,m} = 3 n (A/u) (J3_m - theta J4_m)/(4 pi).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void aeq_node(T t, T wt, T A, T sh2, T uinv, bool at_rest, int nm,
                                         T* J3, T* J4) {
  const T s = A * t;
  const T c = at_rest ? t : (sh2 - dev_expm1(-s)) * uinv;
  const T e1 = dev_exp(s);
  const T e2 = e1 * e1;
  const T w3 = wt * e2, w4 = w3 * e1;
  T p0 = T(1), p1 = c;
  J3[0] += w3;
  J4[0] += w4;
#pragma unroll
  for (int m = 1; m < kMaxM; ++m) {
    if (m < nm) {
      J3[m] += w3 * p1;
      J4[m] += w4 * p1;
      const T p2 = (T(2 * m + 1) * c * p1 - T(m) * p0) * T(1.0 / (m + 1));
      p0 = p1;
      p1 = p2;
    }
  }
}

// One level of a transposing warp reduction of 32 compensated (hi, lo)
// values per lane: lanes with bit OFF set keep the upper half of their
// values, exchange the other half with lane ^ OFF and add with an
// error-free TwoSum, so after the levels 16, 8, 4, 2, 1 lane l holds the
// warp total of value l in h[0] + lo[0].
template <int OFF>
__device__ __forceinline__ void tr_level(float (&h)[32], float (&lo)[32], int lane) {
  const bool up = (lane & OFF) != 0;
#pragma unroll
  for (int i = 0; i < OFF; ++i) {
    const float sh = up ? h[i] : h[i + OFF];
    const float sl = up ? lo[i] : lo[i + OFF];
    const float kh = up ? h[i + OFF] : h[i];
    const float kl = up ? lo[i + OFF] : lo[i];
    const float rh = __shfl_xor_sync(0xffffffffu, sh, OFF);
    const float rl = __shfl_xor_sync(0xffffffffu, sl, OFF);
    const float t = kh + rh;
    const float bp = t - kh;
    const float e = (kh - (t - bp)) + (rh - bp);
    h[i] = t;
    lo[i] = (kl + rl) + e;
  }
}

}  // namespace rslb
