// bjorken.cuh -- pieces shared by the SIMT and tensor-core Bjorken kernels.
#pragma once
#include <cuda_runtime.h>

namespace rslb {

// One entry of K^P (Eq. K_leg_disc), FP64:
//   K^P_{j,j'} = w_j sum_{m=1}^{Q-3} m(m+1)(m+2)/(2(2m+3)) P_m(xi_j) P_{m+2}(xi_j')
//              - w_j sum_{m=1}^{Q-1} m(m+1)/2 P_m(xi_j) [ (2m+1) P_m(xi_j') /
//                ((2m-1)(2m+3)) + (m-1)/(2m-1) P_{m-2}(xi_j') ]
// xw = [xi_0 .. xi_{Q-1} | w_0 .. w_{Q-1}].  P_m(xi_j) advances by the
// Bonnet recurrence; the xi_j' values are carried as a window
// P_{m-2} .. P_{m+2}.  kc holds, per m, the m-dependent factors of both sums
// and of both recurrences (kp_coefficients), so the loop has no divisions.
constexpr int kKpCoef = 8;

// Host: kc[m * kKpCoef + i] for m = 0 .. qmax - 1.
inline void kp_coefficients(int qmax, double* kc) {
  for (int m = 0; m < qmax; ++m) {
    const double d = m;
    double* c = kc + (size_t)m * kKpCoef;
    c[0] = d * (d + 1.0) * (d + 2.0) / (2.0 * (2.0 * d + 3.0));
    c[1] = m >= 1 ? 0.5 * d * (d + 1.0) * (2.0 * d + 1.0) / ((2.0 * d - 1.0) * (2.0 * d + 3.0))
                  : 0.0;
    c[2] = m >= 1 ? 0.5 * d * (d + 1.0) * (d - 1.0) / (2.0 * d - 1.0) : 0.0;
    c[3] = (2.0 * d + 1.0) / (d + 1.0);  // P_{m+1} = c3 x P_m - c4 P_{m-1}
    c[4] = d / (d + 1.0);
    c[5] = (2.0 * d + 5.0) / (d + 3.0);  // P_{m+3} = c5 y P_{m+2} - c6 P_{m+1}
    c[6] = (d + 2.0) / (d + 3.0);
    c[7] = 0.0;
  }
}

__device__ inline double kp_entry(int Q, const double* __restrict__ xw,
                                  const double* __restrict__ kc, int j, int jp) {
  const double x = xw[j], y = xw[jp], w = xw[Q + j];
  double px = x, pxm1 = 1.0;  // P_1(x), P_0(x)
  double ym2 = 0.0, ym1 = 1.0, y0 = y;
  double yp1 = 0.5 * (3.0 * y * y - 1.0);
  double yp2 = (5.0 * y * yp1 - 2.0 * y0) / 3.0;
  double s1 = 0.0, s2 = 0.0;
  for (int m = 1; m <= Q - 1; ++m) {
    const double* c = kc + (size_t)m * kKpCoef;
    const double2 c01 = *reinterpret_cast<const double2*>(c);
    const double2 c23 = *reinterpret_cast<const double2*>(c + 2);
    const double2 c45 = *reinterpret_cast<const double2*>(c + 4);
    const double c6 = c[6];
    if (m <= Q - 3) s1 += c01.x * px * yp2;
    s2 += px * (c01.y * y0 + c23.x * ym2);
    const double pxn = c23.y * x * px - c45.x * pxm1;
    pxm1 = px;
    px = pxn;
    const double yn = c45.y * y * yp2 - c6 * yp1;
    ym2 = ym1;
    ym1 = y0;
    y0 = yp1;
    yp1 = yp2;
    yp2 = yn;
  }
  return w * (s1 - s2);
}

// K^P is centrosymmetric, K^P_{Q-1-j, Q-1-j'} = K^P_{j j'} (the nodes are
// symmetric and P_m(-x) = (-1)^m P_m(x); every term pairs P_m with P_m or
// P_{m+-2}).  With h = floor(Q/2) mirror pairs and qh = ceil(Q/2), the even
// and odd parts of a column f,
//   s_j = f_j + f_{Q-1-j} (j < h),  s_h = f_h for odd Q  (j < qh),
//   d_j = f_j - f_{Q-1-j}                                (j < h),
// give K^P f through two half-size products:
//   (K f)_j + (K f)_{Q-1-j} = sum_j' E_{j j'} s_j',  E_{j j'} = K_{j j'} + K_{j, Q-1-j'},
//   (K f)_j - (K f)_{Q-1-j} = sum_j' O_{j j'} d_j',  O_{j j'} = K_{j j'} - K_{j, Q-1-j'},
// for j < h (E also for the middle row j = h of odd Q, where it gives twice
// (K f)_h).  E is qh x qh, O is h x h: half the flops and half the image.
//
// Work unit of the tensor-core stage kernel: the runs [first, first + R)
// (sorted order, all with Q_xi = Q, states contiguous from soff) and the
// M-tile mt (rows i = 128 mt .. 128 mt + 127 of E and O).
struct BjTcBlock {
  int Q, first, R, mt;
  int nmt;         // M-tiles: ceil(qh / 128)
  int nc;          // MMA N: R * Q_L rounded up to a multiple of 16
  int tmem_cols;   // TMEM columns allocated: two accumulators (E, O) of a
                   // power of two >= max(nc, 32) columns each
  int qh, h;       // rows of E (ceil(Q/2)) and of O (floor(Q/2))
  int pad;
  long long soff;  // state offset (floats) of run `first`
  long long img;   // offset (floats) of the E image of this Q
  long long imgO;  // offset (floats) of the O image of this Q
  long long xoff;  // offset of [xi | w] of this Q in the node pool
};

// Floats of the split, swizzled image of an n x n matrix (n rows of
// ceil(n/32) tiles of 32 columns, hi and lo parts).
__host__ __device__ inline long long bj_tc_image_floats(int n) { return (long long)n * ((n + 31) / 32) * 64; }

struct BjTcArgs {
  const BjTcBlock* blocks;
  const float* kimg;      // K^P images (FP32, tiles pre-swizzled)
  const double* npool;    // [xi | w] per distinct Q
  const double* tau_aw0;  // per run (sorted); <= 0 or inf: collisionless
  const int* gas;         // per run (sorted)
  const double* xk;
  const double* wk;
  const double* KL;       // [QL][QL]
  int QL;
  int stage;              // 0, 1, 2 (Eq. rk3); -1: write K^P f to dout only
  const float* Fin;       // state the stage differentiates
  const float* Fn;        // f at the start of the step
  float* Fout;
  const double* mp_in;    // moments (N, E) of Fin: [run][4][2] partial sums over M-tiles
  double* mp_out;         // moments of Fout
  float* dout;            // stage -1 only
  double tau, dtau;       // stage time and step
  const long long* step;  // if set: the stage time is tau0 + (*step + c_stage) dtau, with
  double tau0;            // c = 0, 1, 1/2 (Tab. II), read on the device (graph replays)
  int* err;
  int withhold_ready;     // failure-handling self-test: the workers never
                          // signal that their operand tiles are ready
};

// Largest MMA N (state columns per block) of the tensor-core stage kernel.
constexpr int kTcMaxCols = 80;

cudaError_t bj_tc_set_attributes();
size_t bj_tc_smem_bytes(int nc, int R);
cudaError_t bj_tc_stage_launch(const BjTcArgs& a, int nblocks, size_t smem, cudaStream_t st);
cudaError_t bj_step_count_launch(long long* step, cudaStream_t st);
cudaError_t bj_tc_image_launch(int Q, const double* xw, const double* kc, float* img,
                               cudaStream_t st);
cudaError_t bj_tc_moments_launch(int nruns, int QL, const int* rq, const long long* roff,
                                 const double* xk, const float* state, double* mp,
                                 cudaStream_t st);

}  // namespace rslb
