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
// One lane per zone (k_adjoint), or one warp per zone for large networks
// (k_adjoint_coop: the same per-zone code with the network spread over the
// warp, coop.cuh); K cotangent sets share each LU factorisation.
#include <cuda_runtime.h>
#include <cub/device/device_radix_sort.cuh>

#include <algorithm>
#include <cstring>

#include "blob.h"
#include "adjoint.cuh"
#include "coop.cuh"
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

// One warp per zone.  With A.blob_in_smem > 1 the warp's Newton-loop arrays
// and its adjoint arrays sit in shared memory after the (optional) blob
// copy: [forward hot | adjoint] per warp, adj_doubles of adjoint arrays.
struct CoopAdj {
  int smem;           // arrays in shared memory
  int adj_doubles;    // adjoint arrays per zone
};

__global__ void __launch_bounds__(256, 1) k_adjoint_coop(AdjParams A, CoopAdj C) {
  extern __shared__ __align__(16) unsigned char sm[];
  const unsigned char* blob = A.blob;
  if (A.blob_in_smem) {
    const int4* src = reinterpret_cast<const int4*>(A.blob);
    int4* dst = reinterpret_cast<int4*>(sm);
    for (int i = threadIdx.x; i < A.blob_bytes / 16; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    blob = sm;
  }
  const WNet t = make_wnet<32>(blob, threadIdx.x & 31);
  const int wib = threadIdx.x >> 5;
  const long long warp = (long long)blockIdx.x * (blockDim.x >> 5) + wib;
  const long long fwd = t.g.lane_doubles;
  CWS w;
  AWST<CV> a;
  if (C.smem) {
    double* hot = reinterpret_cast<double*>(sm + (A.blob_in_smem ? A.blob_bytes : 0)) +
                  (size_t)wib * (t.g.hot_doubles + C.adj_doubles);
    w = make_cws(t.g, hot, A.ws + warp * (fwd - t.g.hot_doubles));
    a = make_aws_at<CV>(A, hot + t.g.hot_doubles - fwd, 1);
  } else {
    double* base = A.ws + warp * A.lane_doubles;
    w = make_cws(t.g, base, base + t.g.hot_doubles);
    a = make_aws_at<CV>(A, base, 1);
  }
  for (;;) {
    unsigned long long c = 0;
    if (t.lane == 0) c = atomicAdd(A.queue, 1ull);
    c = __shfl_sync(kFullMask, c, 0);
    if (c >= (unsigned long long)A.Z) break;
    AdjZone Zs;
    Zs.z = A.order ? (long long)A.order[c] : (long long)c;
    Zs.rs = 1;
    Zs.re = 0;
    Zs.lo = 1;
    bool done = adj_init(t, Zs, w, a, A);
    while (!done) done = Zs.rs <= Zs.re ? adj_replay(t, Zs, w, a, A) : adj_step(t, Zs, w, a, A);
    adj_finish(t, Zs, a, A);
    __syncwarp();
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
  return nb_burn_adjoint_ex(net, tape, K, gY, gE, gT9, d_ln_mult, dY0, dT0, nullptr, stream);
}

extern "C" int nb_burn_adjoint_ex(nb_net net, void* tape, int32_t K, const double* gY,
                                  const double* gE, const double* gT9, double* d_ln_mult,
                                  double* dY0, double* dT0, const nb_options* opt,
                                  void* stream) {
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
  nb_options o;
  nb_default_options(&o);
  if (opt) o = *opt;
  // the kernel: as asked; else, when blocks are recomputed (stride > 1), the
  // arithmetic of the recording burn, so that the recomputed states are the
  // forward's bits; else one warp per zone from 24 state entries on
  int kernel = o.kernel;
  const bool recompute = tp->dev.stride > 1;
  const bool family_ok = tp->family == NB_KERNEL_COOP || tp->family == NB_KERNEL_PERSISTENT;
  if (!opt || kernel == NB_KERNEL_AUTO) {
    if (recompute && !family_ok) return NB_E_TAPE;   // recorded by teams of warps
    kernel = recompute ? tp->family : (n >= 24 ? NB_KERNEL_COOP : NB_KERNEL_PERSISTENT);
  }
  if (kernel != NB_KERNEL_COOP && kernel != NB_KERNEL_PERSISTENT) return NB_E_ARG;
  if (recompute && kernel != tp->family) return NB_E_TAPE;
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(net->mu);
  const size_t blob_b = (size_t)h.bytes;
  int tpb, in_smem;
  size_t dyn;
  long long blocks;
  CoopAdj C{0, (int)(A.lane_doubles - h.lane_doubles)};
  size_t per_unit;   // global workspace per lane (lane kernel) or warp (coop)
  if (kernel == NB_KERNEL_COOP) {
    // per warp in shared memory: the forward hot arrays and the adjoint's
    const size_t warp_b = ((size_t)h.hot_doubles + C.adj_doubles) * sizeof(double);
    int wpb = o.threads_per_block > 0 ? o.threads_per_block / 32 : 0;
    if (o.threads_per_block % 32 != 0 || wpb > 8) return NB_E_ARG;
    in_smem = 0;
    C.smem = o.ws_in_shared != 0 && warp_b <= net->smem_optin;
    if (wpb == 0) {
      wpb = 4;
      if (C.smem) while (wpb > 1 && (size_t)wpb * warp_b > net->smem_optin) --wpb;
    }
    if (o.blob_in_shared != 0 && blob_b <= 96 * 1024 &&
        blob_b + (C.smem ? wpb * warp_b : 0) <= net->smem_optin)
      in_smem = 1;
    dyn = (in_smem ? blob_b : 0) + (C.smem ? wpb * warp_b : 0);
    if (dyn > net->smem_optin) return NB_E_TOO_LARGE;
    tpb = wpb * 32;
    CK(cudaFuncSetAttribute(k_adjoint_coop, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)dyn));
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_adjoint_coop, tpb, dyn));
    if (occ < 1) return NB_E_TOO_LARGE;
    const int bps = std::max(1, std::min(o.blocks_per_sm > 0 ? o.blocks_per_sm : occ, occ));
    blocks = (long long)bps * net->sm_count;
    const long long needed = (Z + wpb - 1) / wpb;
    if (blocks > needed) blocks = needed;
    per_unit = (C.smem ? (size_t)(h.lane_doubles - h.hot_doubles) : (size_t)A.lane_doubles) * 8;
    const size_t need = (size_t)blocks * wpb * per_unit;
    int rc = nb::ensure((void**)&net->ws_adj, &net->ws_adj_bytes, std::max<size_t>(need, 256));
    if (rc) return rc;
  } else {
    // one zone per lane; smaller blocks when there are few zones per SM
    const long long per_sm = (Z + net->sm_count - 1) / net->sm_count;
    tpb = o.threads_per_block > 0 ? o.threads_per_block
                                  : (per_sm >= 128 ? 128 : (int)std::max(32LL, per_sm / 32 * 32));
    if (tpb % 32 != 0 || tpb > 128) return NB_E_ARG;
    in_smem = blob_b <= 96 * 1024 ? 1 : 0;
    dyn = in_smem ? blob_b : 0;
    if (dyn > 48 * 1024)
      CK(cudaFuncSetAttribute(k_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_adjoint, tpb, dyn));
    blocks = (long long)std::max(1, std::min(o.blocks_per_sm > 0 ? o.blocks_per_sm : 2, occ)) *
             net->sm_count;
    const long long needed = (Z + tpb - 1) / tpb;
    if (blocks > needed) blocks = needed;
    per_unit = (size_t)A.lane_doubles * sizeof(double);
    int rc = nb::ensure((void**)&net->ws_adj, &net->ws_adj_bytes, (size_t)blocks * tpb * per_unit);
    if (rc) return rc;
  }
  int rc = NB_OK;
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
  if (kernel == NB_KERNEL_COOP)
    k_adjoint_coop<<<(unsigned)blocks, tpb, dyn, st>>>(A, C);
  else
    k_adjoint<<<(unsigned)blocks, tpb, dyn, st>>>(A);
  CK(cudaGetLastError());
  return NB_OK;
}
