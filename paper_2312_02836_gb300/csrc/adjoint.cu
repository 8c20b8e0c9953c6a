// adjoint.cu -- discrete adjoint of a recorded burn.
//
// The rate sensitivity the paper explores by re-running the detonation with
// changed networks (arXiv:2312.02836 Sec. 1 and Sec. 3) is computed here as
// the exact gradient of the discrete map the forward burn applied, with the
// step schedule (t_n, h_n, k_n) frozen and every Newton solution treated as
// exact.  Forward step s solves
//     G_s = alpha_0 x_s + sum_{j=1..k} alpha_j x_{s-j} - h f(x_s; p) = 0,
//     E_s = (h edot(x_s; p) - sum_j alpha_j E_{s-j}) / alpha_0,
// so, walking s = S..1 with cotangents lam_s (of x_s) and e_s (of E_s):
//     lam_s += e_s h / alpha_0 * d edot / dx,   e_{s-j} -= e_s alpha_j / alpha_0
//     (alpha_0 I - h J(x_s))^T mu = lam_s
//     lam_{s-j} -= alpha_j mu
//     dL/dp_r += R_r(x_s) (h c_r^T mu + e_s h / alpha_0 Q_r)
// (plus mu_T Q_r / c_v in c_r^T mu under self-heating, and the temperature
// derivative through g_r = d ln lambda_r / dT9 when T9 is a parameter).
// The tape keeps states only at checkpoints: the reverse sweep takes the steps
// in blocks of the tape's stride, last block first, recomputes each block's
// states forward from its checkpointed history window with the forward's
// own step computation (attempt_solve, so the same bits), then reverses it.
// One lane per zone, K cotangent sets share each LU factorisation.
#include <cuda_runtime.h>
#include <cub/device/device_radix_sort.cuh>

#include <algorithm>
#include <cstring>

#include "blob.h"
#include "adjoint.cuh"
#include "device.cuh"
#include "host.h"
#include "../../include/netburn.h"

using namespace nb;

namespace {

__global__ void __launch_bounds__(128) k_adjoint(AdjParams A) {
  extern __shared__ __align__(16) unsigned char sm[];
  const unsigned char* blob = A.blob;
  if (A.blob_in_smem) {
    const int4* src = reinterpret_cast<const int4*>(A.blob);
    int4* dst = reinterpret_cast<int4*>(sm);
    for (int i = threadIdx.x; i < A.blob_bytes / 16; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    blob = sm;
  }
  const Net t = make_net(blob);
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  double* lane_base = A.ws + warp * A.lane_doubles * WS_LANES + lane;
  const WS w = make_ws(t, lane_base);
  const AWS a = make_aws(A, lane_base);
  AdjZone Zs;
  Zs.z = -1;
  Zs.s = -1;
  Zs.rs = 1;
  Zs.re = 0;
  Zs.lo = 1;
  Zs.fail = false;
  bool active = false, retired = false, fresh = false;
  for (;;) {
    const unsigned need = __ballot_sync(0xffffffffu, !active && !retired);
    if (need) {
      const int leader = __ffs(need) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(A.queue, (unsigned long long)__popc(need));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (!active && !retired) {
        const unsigned long long z = base + __popc(need & ((1u << lane) - 1u));
        if (z < (unsigned long long)A.Z) {
          Zs.z = A.order ? (long long)A.order[z] : (long long)z;
          active = true;
          fresh = true;
        } else {
          retired = true;
        }
      }
    }
    if (__all_sync(0xffffffffu, retired)) break;
    if (active) {
      bool done;
      if (fresh) {
        done = adj_init(t, Zs, w, a, A);
        fresh = false;
      } else if (Zs.rs <= Zs.re) {
        done = adj_replay(t, Zs, w, a, A);
      } else {
        done = adj_step(t, Zs, w, a, A);
      }
      if (done) {
        adj_finish(t, Zs, a, A);
        active = false;
      }
    }
  }
}

__global__ void k_zone_index(int32_t* idx, long long Z) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < Z) idx[i] = (int32_t)i;
}

}  // namespace

extern "C" int nb_burn_adjoint(nb_net net, void* tape, int32_t K, const double* gY,
                               const double* gE, const double* gT9, double* d_ln_mult,
                               double* dY0, double* dT0, void* stream) {
  if (!net || !tape || K < 1 || K > 64 || !gY || !d_ln_mult) return NB_E_ARG;
  nb_tape_s* tp = (nb_tape_s*)tape;
  if (tp->magic != 0x7a9e5eedu || tp->net != net || !tp->recorded) return NB_E_TAPE;
  const BlobHeader& h = net->h;
  const long long Z = tp->recZ;
  if (Z == 0) return NB_OK;
  AdjParams A;
  std::memset(&A, 0, sizeof(A));
  A.blob = net->d_blob;
  A.blob_bytes = h.bytes;
  A.Z = Z;
  A.K = K;
  A.tape = tp->dev;
  A.rtol = tp->rtol;
  A.atol = tp->atol;
  A.lnm = tp->has_lnm ? tp->lnm : nullptr;
  A.lnm_per_zone = tp->lnm_per_zone;
  A.gY = gY; A.gE = gE; A.gT9 = gT9;
  A.dl = d_ln_mult; A.dY0 = dY0; A.dT0 = dT0;
  const int n = h.n;
  long long off = h.lane_doubles;
  A.o_lam = (int)off; off += (long long)HMAX * K * n;
  A.o_ee = (int)off; off += (long long)HMAX * K;
  A.o_gr = (int)off; off += (long long)K * h.R;
  A.o_gt = (int)off; off += K;
  A.o_mu = (int)off; off += n;
  A.o_de = (int)off; off += n;
  A.o_seg = (int)off; off += (long long)tp->dev.stride * n;
  A.lane_doubles = off;
  // one zone per lane; smaller blocks when there are few zones per SM
  const long long per_sm = (Z + net->sm_count - 1) / net->sm_count;
  const int tpb = per_sm >= 128 ? 128 : (int)std::max(32LL, per_sm / 32 * 32);
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(net->mu);
  const size_t smem = (size_t)h.bytes;
  const int in_smem = smem <= 96 * 1024 ? 1 : 0;
  const size_t dyn = in_smem ? smem : 0;
  if (dyn > 48 * 1024)
    CK(cudaFuncSetAttribute(k_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  int occ = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_adjoint, tpb, dyn));
  long long blocks = (long long)std::max(1, std::min(occ, 2)) * net->sm_count;
  const long long needed = (Z + tpb - 1) / tpb;
  if (blocks > needed) blocks = needed;
  const size_t need = (size_t)blocks * tpb * A.lane_doubles * sizeof(double);
  int rc = nb::ensure((void**)&net->ws_adj, &net->ws_adj_bytes, need);
  if (rc) return rc;
  A.ws = net->ws_adj;
  A.queue = net->queue + 1;   // a second counter in the same allocation
  A.blob_in_smem = in_smem;
  // Claim order: the tape holds every zone's step count, the exact length of
  // its reverse sweep, so zones are claimed longest first and the last lanes
  // to finish run short zones (one lane per zone otherwise waits on the
  // longest zone).
  if (Z > 1 && Z <= 0x7fffffffLL) {
    size_t temp = 0;
    CK(cub::DeviceRadixSort::SortPairsDescending(nullptr, temp, (const int32_t*)nullptr,
                                                 (int32_t*)nullptr, (const int32_t*)nullptr,
                                                 (int32_t*)nullptr, (int)Z, 0, 32, st));
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t ib = al((size_t)Z * 4);
    rc = nb::ensure((void**)&net->sched_adj, &net->sched_adj_bytes, 3 * ib + al(temp));
    if (rc) return rc;
    int32_t* k_out = (int32_t*)net->sched_adj;
    int32_t* i_in = (int32_t*)(net->sched_adj + ib);
    int32_t* i_out = (int32_t*)(net->sched_adj + 2 * ib);
    k_zone_index<<<(unsigned)((Z + 255) / 256), 256, 0, st>>>(i_in, Z);
    CK(cudaGetLastError());
    CK(cub::DeviceRadixSort::SortPairsDescending(net->sched_adj + 3 * ib, temp, tp->dev.steps,
                                                 k_out, i_in, i_out, (int)Z, 0, 32, st));
    A.order = i_out;
  }
  CK(cudaMemsetAsync(A.queue, 0, sizeof(unsigned long long), st));
  k_adjoint<<<(unsigned)blocks, tpb, dyn, st>>>(A);
  CK(cudaGetLastError());
  return NB_OK;
}
