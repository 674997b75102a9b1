// host_common.h -- host helpers shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>

namespace rslb {

int set_error(int code, const char* fmt, ...);
void clear_error();
const char* last_error();
int cuda_error(cudaError_t e, const char* what);

int gauss_legendre_host(int Q, double* x, double* w);
int gauss_laguerre2_host(int Q, double* x, double* w);
double legendre_p(int m, double x);

}  // namespace rslb
