// expcheck.cu -- diagnostic entry point for the FP64 exp of the rate
// evaluation: evaluates the kernels' exp (Tang's table-driven method,
// expf64.cuh) and CUDA's library exp on the same arguments, so that a test
// can hold the former to its error bound.
#include <cuda_runtime.h>

#include "expf64.cuh"
#include "../../include/netburn.h"

namespace {

__global__ void k_exp_eval(const double* x, double* y_tang, double* y_lib, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  y_tang[i] = nb::exp_tang(x[i]);
  if (y_lib) y_lib[i] = exp(x[i]);
}

}  // namespace

extern "C" int nb_exp_eval(const double* x, double* y_tang, double* y_lib, int64_t n,
                           void* stream) {
  if (n < 0 || (n > 0 && (!x || !y_tang))) return NB_E_ARG;
  if (n == 0) return NB_OK;
  const int tpb = 256;
  k_exp_eval<<<(unsigned)((n + tpb - 1) / tpb), tpb, 0, (cudaStream_t)stream>>>(x, y_tang, y_lib, n);
  return cudaGetLastError() == cudaSuccess ? NB_OK : NB_E_CUDA;
}
