// host.h -- host-side objects behind the C ABI handles (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "blob.h"
#include "device.cuh"
#include "../../include/netburn.h"

struct nb_net_s {
  nb::BlobHeader h;
  std::vector<uint8_t> blob;
  unsigned char* d_blob = nullptr;
  int device = 0;
  int sm_count = 0;
  size_t smem_optin = 0;
  double* ws = nullptr;
  size_t ws_bytes = 0;
  unsigned long long* queue = nullptr;
  // staging for the host-pointer entry point
  unsigned char* stage = nullptr;
  size_t stage_bytes = 0;
  double* ws_adj = nullptr;   // adjoint per-lane workspace
  size_t ws_adj_bytes = 0;
  unsigned char* sched = nullptr;   // claim-order keys, indices, sort scratch
  size_t sched_bytes = 0;
  unsigned char* sched_adj = nullptr;   // the adjoint's claim order and sort scratch
  size_t sched_adj_bytes = 0;
  // network-specialised kernels by storage variant (1..3): 0 not built,
  // 1 loaded, -1 failed (log kept)
  struct Spec {
    int state = 0;
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
    std::string log;
  } spec[4];
  int last_spec = 0;   // variant the last burn ran (0 generic)
  std::mutex mu;
};

struct nb_tape_s {
  nb_net net;
  long long Z;
  int cap;
  nb::TapeDev dev{};
  long long recZ = 0;       // zones of the recorded burn
  double* lnm = nullptr;   // copy of the multipliers of the recorded burn
  int lnm_per_zone = 0;
  int has_lnm = 0;
  double t_end = 0, rtol = 0, atol = 0;
  int recorded = 0;
  // arithmetic of the recording burn: NB_KERNEL_PERSISTENT for the
  // one-zone-per-lane kernels (which share their bits), NB_KERNEL_COOP for
  // one zone per warp; a checkpointed block is recomputed in the same one
  int family = 0;
  unsigned magic = 0x7a9e5eedu;
};

// device buffers of a tape (each may be null)
inline void tape_release(nb_tape_s* tp) {
  cudaFree(tp->dev.sched); cudaFree(tp->dev.ord); cudaFree(tp->dev.states);
  cudaFree(tp->dev.steps); cudaFree(tp->dev.zstat); cudaFree(tp->dev.rho);
  cudaFree(tp->dev.T9f); cudaFree(tp->dev.scr); cudaFree(tp->lnm);
}

#define CK(call)                                                   \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return NB_E_CUDA;                       \
  } while (0)


namespace nb {
// (Re)allocate a device buffer of at least `need` bytes.
inline int ensure(void** p, size_t* have, size_t need) {
  if (*have >= need && *p) return NB_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  if (cudaMalloc(p, need) != cudaSuccess) {
    *p = nullptr;
    return NB_E_NOMEM;
  }
  *have = need;
  return NB_OK;
}
}  // namespace nb
