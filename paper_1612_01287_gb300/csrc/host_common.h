// host_common.h -- host helpers shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include "../../include/rslb.h"

namespace rslb {

int set_error(int code, const char* fmt, ...);
void clear_error();
const char* last_error();
int cuda_error(cudaError_t e, const char* what);

int gauss_legendre_host(int Q, double* x, double* w);
int gauss_laguerre2_host(int Q, double* x, double* w);
double legendre_p(int m, double x);

// Internal view of a shock-tube handle for the other translation units.
struct SodView {
  int Z, ldz, V, Q_xi, Q_L;
  bool fp64;
  cudaStream_t stream;
  void* F0;
  void* F1;
  double dt;
};
int sod_view(rslb_handle* h, SodView* v);

}  // namespace rslb
