// peaks.cu -- measurement support: the FP64 fused multiply-add rate of the
// device, against which the FP64 shock-tube path is placed on its roofline.
#include <cuda_runtime.h>

#include "../../include/rslb.h"
#include "host_common.h"

namespace rslb {
namespace {

constexpr int kChains = 8;  // independent FMA chains per thread

// Every thread runs kChains dependent chains of DFMAs; the result is written
// out only if it is non-finite (it never is), so nothing is optimised away.
__global__ void fp64_fma_kernel(int iters, double seed, double* sink) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = seed + 1e-3 * (threadIdx.x + c);
  const double a = 0.999999, b = 1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (!isfinite(s)) sink[0] = s;
}

}  // namespace
}  // namespace rslb

using namespace rslb;

extern "C" int rslb_measure_fp64_fma(int reps, double* fma_per_s, void* stream) {
  clear_error();
  if (reps < 1 || !fma_per_s) return set_error(RSLB_ERR_ARG, "rslb_measure_fp64_fma: bad arguments");
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_error(e, "rslb_measure_fp64_fma: device query");
  cudaStream_t st = (cudaStream_t)stream;
  const int threads = 256, blocks = 8 * nsm, iters = 4096;
  cudaEvent_t a = nullptr, b = nullptr;
  e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  fp64_fma_kernel<<<blocks, threads, 0, st>>>(iters, 1.0, nullptr);  // warm-up
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventRecord(a, st);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    fp64_fma_kernel<<<blocks, threads, 0, st>>>(iters, 1.0 + r, nullptr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_error(e, "rslb_measure_fp64_fma");
  *fma_per_s = (double)reps * blocks * threads * iters * kChains / (ms * 1e-3);
  return RSLB_OK;
}
