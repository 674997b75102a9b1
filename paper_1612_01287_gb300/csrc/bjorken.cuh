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
// P_{m-2} .. P_{m+2}.
__device__ inline double kp_entry(int Q, const double* __restrict__ xw, int j, int jp) {
  const double x = xw[j], y = xw[jp], w = xw[Q + j];
  double px = x, pxm1 = 1.0;  // P_1(x), P_0(x)
  double ym2 = 0.0, ym1 = 1.0, y0 = y;
  double yp1 = 0.5 * (3.0 * y * y - 1.0);
  double yp2 = (5.0 * y * yp1 - 2.0 * y0) / 3.0;
  double s1 = 0.0, s2 = 0.0;
  for (int m = 1; m <= Q - 1; ++m) {
    const double dm = m;
    if (m <= Q - 3) s1 += dm * (dm + 1.0) * (dm + 2.0) / (2.0 * (2.0 * dm + 3.0)) * px * yp2;
    s2 += 0.5 * dm * (dm + 1.0) * px *
          ((2.0 * dm + 1.0) / ((2.0 * dm - 1.0) * (2.0 * dm + 3.0)) * y0 +
           (dm - 1.0) / (2.0 * dm - 1.0) * ym2);
    const double pxn = ((2.0 * dm + 1.0) * x * px - dm * pxm1) / (dm + 1.0);
    pxm1 = px;
    px = pxn;
    const double yn = ((2.0 * dm + 5.0) * y * yp2 - (dm + 2.0) * yp1) / (dm + 3.0);
    ym2 = ym1;
    ym1 = y0;
    y0 = yp1;
    yp1 = yp2;
    yp2 = yn;
  }
  return w * (s1 - s2);
}

// Work unit of the tensor-core stage kernel: the runs [first, first + R)
// (sorted order, all with Q_xi = Q, states contiguous from soff) and the
// M-tile mt (rows j = 128 mt .. 128 mt + 127 of K^P).
struct BjTcBlock {
  int Q, first, R, mt;
  int nmt;         // M-tiles of Q: ceil(Q / 128)
  int nc;          // MMA N: R * Q_L rounded up to a multiple of 16
  int tmem_cols;   // TMEM columns allocated (power of two >= max(nc, 32))
  int pad;
  long long soff;  // state offset (floats) of run `first`
  long long img;   // offset (floats) of the K^P image of this Q
  long long xoff;  // offset of [xi | w] of this Q in the node pool
};

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
  int* err;
};

// Largest MMA N (state columns per block) of the tensor-core stage kernel.
constexpr int kTcMaxCols = 80;

cudaError_t bj_tc_set_attributes();
size_t bj_tc_smem_bytes(int nc, int R);
cudaError_t bj_tc_stage_launch(const BjTcArgs& a, int nblocks, size_t smem, cudaStream_t st);
cudaError_t bj_tc_image_launch(int Q, const double* xw, float* img, cudaStream_t st);
cudaError_t bj_tc_moments_launch(int nruns, int QL, const int* rq, const long long* roff,
                                 const double* xk, const float* state, double* mp,
                                 cudaStream_t st);

}  // namespace rslb
