// recip_check.cu -- the integrator's Newton-Raphson reciprocals (recip1 for
// the error weights, recip2 for the LU pivots) evaluated on the GPU for the
// tests, which compare them with the correctly rounded 1/a.  Test
// infrastructure, built by the tests into its own small library.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../paper_2312_02836_gb300/csrc/device.cuh"

namespace {

__global__ void k_recip(const double* a, double* r1, double* r2, double* rd, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  r1[i] = nb::recip1(a[i]);
  r2[i] = nb::recip2(a[i]);
  rd[i] = 1.0 / a[i];
}

}  // namespace

// a [n] host input; r1, r2, rd [n] host outputs (recip1, recip2 and CUDA's
// 1/a).  Returns 0, -1 for a bad argument, -4 for a CUDA error.  Synchronous.
extern "C" int recip_eval(const double* a, long long n, double* r1, double* r2, double* rd) {
  if (!a || !r1 || !r2 || !rd || n <= 0) return -1;
  double* d = nullptr;
  const size_t b = (size_t)n * sizeof(double);
  if (cudaMalloc(&d, 4 * b) != cudaSuccess) return -4;
  int rc = 0;
  if (cudaMemcpy(d, a, b, cudaMemcpyHostToDevice) != cudaSuccess) rc = -4;
  if (!rc) {
    k_recip<<<(unsigned)((n + 255) / 256), 256>>>(d, d + n, d + 2 * n, d + 3 * n, n);
    if (cudaDeviceSynchronize() != cudaSuccess) rc = -4;
  }
  if (!rc && (cudaMemcpy(r1, d + n, b, cudaMemcpyDeviceToHost) != cudaSuccess ||
              cudaMemcpy(r2, d + 2 * n, b, cudaMemcpyDeviceToHost) != cudaSuccess ||
              cudaMemcpy(rd, d + 3 * n, b, cudaMemcpyDeviceToHost) != cudaSuccess))
    rc = -4;
  cudaFree(d);
  return rc;
}
