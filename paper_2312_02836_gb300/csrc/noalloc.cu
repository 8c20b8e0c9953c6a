// noalloc.cu -- a burn entry point that performs no device allocation.
//
// nb_burn_batch allocates (and grows) a device workspace on first use.  Some
// callers cannot allow that at burn time: a solver whose memory is fully
// reserved up front by its own pool, a time step that runs while another
// library holds the allocator, or code that must not trigger the implicit
// synchronisation a cudaMalloc/cudaFree can bring.  nb_burn_batch_noalloc
// runs the same persistent lane-per-zone integration, but its work queue
// counter and per-lane workspace live in one fixed array compiled into this
// library, so the call itself never asks the driver for memory.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds NB_NOALLOC_SCRATCH_BYTES of it until the process exits, and
// all calls share it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "blob.h"
#include "device.cuh"
#include "host.h"
#include "../../include/netburn.h"

using namespace nb;

namespace {

constexpr size_t kCounterBytes = 256;  // queue counter, padded to 256 bytes

// Shared scratch: [queue counter | per-lane workspace].
static __device__ __align__(256) unsigned char g_noalloc_scratch[NB_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device (host code cannot use the
// symbol's name as a device pointer).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return NB_E_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return NB_E_CUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return NB_OK;
}

// The persistent claim loop of the burn with the workspace in global memory,
// taking the counter and workspace from the fixed scratch.
__global__ void __launch_bounds__(128, 2) k_burn_noalloc(BurnParams P) {
  extern __shared__ __align__(16) unsigned char sm[];
  const unsigned char* blob = P.blob;
  if (P.blob_in_smem) {
    const int4* src = reinterpret_cast<const int4*>(P.blob);
    int4* dst = reinterpret_cast<int4*>(sm);
    for (int i = threadIdx.x; i < P.blob_bytes / 16; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    blob = sm;
  }
  const Net t = make_net(blob);
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  WS w = make_ws(t, P.ws + warp * (long long)t.lane_doubles * WS_LANES + lane);
  burn_claim_loop(t, w, P);
}

}  // namespace

extern "C" int nb_burn_batch_noalloc(nb_net net, int64_t Z, const double* Y0,
                                     const double* T9_0, const double* rho, double t_end,
                                     double rtol, double atol, const double* ln_mult,
                                     int32_t ln_mult_per_zone, double* Y, double* T9,
                                     double* E, int32_t* counters, int32_t* status,
                                     const nb_options* opt, void* stream) {
  if (!net) return NB_E_ARG;
  if (Z < 0 || !(rtol > 0.0) || !(atol > 0.0) || !(t_end >= 0.0) || !std::isfinite(t_end))
    return NB_E_ARG;
  if (Z == 0) return NB_OK;
  if (!Y0 || !T9_0 || !rho || !Y || !T9 || !status) return NB_E_ARG;
  nb_options o;
  nb_default_options(&o);
  if (opt) o = *opt;
  if (o.max_attempts <= 0 || !(o.time_budget_s >= 0.0)) return NB_E_ARG;
  const int tpb = o.threads_per_block > 0 ? o.threads_per_block : 128;
  if (tpb % 32 != 0 || tpb > 128) return NB_E_ARG;

  // How many lanes fit: every lane needs lane_doubles of workspace.
  const size_t lane_bytes = (size_t)net->h.lane_doubles * sizeof(double);
  const size_t lanes_fit = (NB_NOALLOC_SCRATCH_BYTES - kCounterBytes) / lane_bytes;
  const long long blocks_fit = (long long)(lanes_fit / (size_t)tpb);
  if (blocks_fit < 1) return NB_E_TOO_LARGE;   // one block's workspace exceeds the scratch

  int dev = 0;
  CK(cudaGetDevice(&dev));
  void* scratch = nullptr;
  int rc = scratch_address(dev, &scratch);
  if (rc) return rc;

  const size_t blob_b = (size_t)net->h.bytes;
  int in_smem = o.blob_in_shared;
  if (in_smem < 0) in_smem = blob_b <= 96 * 1024 ? 1 : 0;
  const size_t dyn = in_smem ? blob_b : 0;
  if (dyn > net->smem_optin) return NB_E_TOO_LARGE;
  if (dyn > 48 * 1024)
    CK(cudaFuncSetAttribute(k_burn_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  int occ = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_burn_noalloc, tpb, dyn));
  if (occ < 1) return NB_E_TOO_LARGE;
  int bps = o.blocks_per_sm > 0 ? o.blocks_per_sm : 1;
  bps = std::max(1, std::min(bps, occ));
  long long blocks = (long long)bps * net->sm_count;
  blocks = std::min(blocks, blocks_fit);
  blocks = std::min(blocks, (long long)((Z + tpb - 1) / tpb));

  BurnParams P;
  std::memset(&P, 0, sizeof(P));
  P.blob = net->d_blob;
  P.blob_bytes = net->h.bytes;
  P.blob_in_smem = in_smem;
  P.Z = Z; P.Y0 = Y0; P.T9_0 = T9_0; P.rho = rho;
  P.t_end = t_end; P.rtol = rtol; P.atol = atol;
  P.lnm = ln_mult; P.lnm_per_zone = ln_mult_per_zone ? 1 : 0;
  P.Y = Y; P.T9 = T9; P.E = E; P.counters = counters; P.status = status;
  P.max_attempts = o.max_attempts;
  // the per-zone options of nb_burn_batch: read-only inputs of the claim
  // loop, so they need no scratch
  P.budget_ns = o.time_budget_s > 0.0 ? (unsigned long long)(o.time_budget_s * 1e9) + 1ull : 0ull;
  P.t_end_zone = o.t_end_zone;
  P.zeta_zone = o.zeta_zone;
  P.queue = reinterpret_cast<unsigned long long*>(scratch);
  P.ws = reinterpret_cast<double*>(static_cast<unsigned char*>(scratch) + kCounterBytes);
  cudaStream_t st = (cudaStream_t)stream;
  // the queue counter must start at zero; the workspace needs no clearing
  CK(cudaMemsetAsync(P.queue, 0, sizeof(unsigned long long), st));
  k_burn_noalloc<<<(unsigned)blocks, tpb, dyn, st>>>(P);
  CK(cudaGetLastError());
  return NB_OK;
}
