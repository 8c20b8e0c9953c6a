// fp64_probe.cu -- FP64 pipe microbenchmark: the measured denominator of the
// burn's roofline.  Measurement infrastructure, built by the tests into its
// own small library; the burn library does not contain it.
//
// Every thread runs 8 independent DFMA chains; lanes >= active_lanes leave at
// once, so the run also shows whether idle lanes of a warp free FP64 issue
// slots (on GB300 they do not: the per-warp cost is the same).
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__global__ void __launch_bounds__(256) k_probe_dfma(double* out, int iters, int active,
                                                    double a, double b) {
  const int lane = threadIdx.x & 31;
  if (lane >= active) return;
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

}  // namespace

// Useful FP64 rate in TFLOP/s (an FMA counted as 2) of blocks_per_sm x SMs
// blocks of 256 threads with active_lanes working lanes per warp.  Returns 0,
// -1 for a bad argument, -4 for a CUDA error.  Synchronous.
extern "C" int fp64_probe(int32_t active_lanes, int32_t iters, int32_t blocks_per_sm,
                          double* tflops_useful, double* ms_out) {
  if (active_lanes < 1 || active_lanes > 32 || iters < 1 || blocks_per_sm < 1 ||
      blocks_per_sm > 8 || !tflops_useful)
    return -1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return -4;
  const int threads = 256;
  const int blocks = sms * blocks_per_sm;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) return -4;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_probe_dfma<<<blocks, threads>>>(out, 64, active_lanes, 0.999, 1e-3);
  cudaEventRecord(e0);
  k_probe_dfma<<<blocks, threads>>>(out, iters, active_lanes, 0.999, 1e-3);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return -4;
  const double lane_fma = (double)blocks * threads / 32 * active_lanes * iters * 8;
  *tflops_useful = 2.0 * lane_fma / (ms * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
  return 0;
}
