// multi.cu -- several networks burned in one launch.
//
// The paper's study burns the same hydro zones with different networks
// (aprox13-like, subch_simple, He-C-Fe; arXiv:2312.02836 Sec. 3 and 4) to see
// which nuclear physics matters.  nb_burn_multi takes up to
// NB_MULTI_MAX_SETS (network, zones) sets and runs them in one persistent
// launch: all lanes of the GPU claim from one device queue that spans every
// set's zones, so a set of few expensive zones and a set of many cheap ones
// keep the same warps busy.  Each lane reads the compiled network of the
// zone it claimed (from global memory, through L1) and runs the generic
// integrator, so every zone gives the same bits as a single-network burn.
#include <cuda_runtime.h>
#include <cub/device/device_segmented_radix_sort.cuh>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "blob.h"
#include "device.cuh"
#include "host.h"
#include "../../include/netburn.h"

using namespace nb;

namespace {

struct MultiParams {
  int n;                                  // sets, in claim order
  long long off[NB_MULTI_MAX_SETS + 1];   // first claim index of each set
  BurnParams p[NB_MULTI_MAX_SETS];
  double* ws;                             // per-lane workspace, max lane_doubles
  int lane_doubles;
  unsigned long long* queue;
  unsigned long long budget_ns;
  const int32_t* order;                   // claim position -> claim index, or null
};
// passed by value as the kernel's parameter block (the classic 4 KB limit)
static_assert(sizeof(MultiParams) <= 4000, "MultiParams exceeds the kernel parameter space");

__global__ void __launch_bounds__(128, 1) k_burn_multi(const __grid_constant__ MultiParams M) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  double* lane_base = M.ws + warp * (long long)M.lane_doubles * WS_LANES + lane;
  const long long total = M.off[M.n];
  Zone s;
  s.z = -1;
  int m = 0;
  bool active = false, retired = false, fresh = false;
  const unsigned long long t_start = M.budget_ns ? gpu_ns() : 0ull;
  for (;;) {
    const unsigned need = __ballot_sync(0xffffffffu, !active && !retired);
    if (need) {
      const int leader = __ffs(need) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(M.queue, (unsigned long long)__popc(need));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (!active && !retired) {
        const unsigned long long c = base + __popc(need & ((1u << lane) - 1u));
        if (c < (unsigned long long)total) {
          // the order keeps every position within its own set's range
          const long long ci = M.order ? (long long)M.order[c] : (long long)c;
          m = 0;
          while (m + 1 < M.n && ci >= M.off[m + 1]) ++m;
          s.z = ci - M.off[m];
          active = true;
          fresh = true;
        } else {
          retired = true;
        }
      }
    }
    if (__all_sync(0xffffffffu, retired)) break;
    if (active) {
      const BurnParams& P = M.p[m];
      const Net t = make_net(P.blob);
      WS w = make_ws(t, lane_base);
      const bool expired = M.budget_ns && gpu_ns() - t_start > M.budget_ns;
      bool done;
      if (expired && fresh) {
        zone_timeout_unstarted(t, s.z, P);
        fresh = false;
        active = false;
        continue;
      }
      if (expired) {
        s.status = NB_Z_TIMEOUT;
        done = true;
      } else if (fresh) {
        done = zone_init(t, s, w, P);
        fresh = false;
      } else {
        done = zone_attempt(t, s, w, P);
      }
      if (done) {
        zone_finish(t, s, w, P);
        active = false;
      }
    }
  }
}

// Scheduling pre-pass: every zone's starting step h0 (the integrator's own
// start-up) as the key of its claim index; zones that finish in start-up go
// last.  Sorted within each set, the keys give each set's zones longest
// first, so a warp's lanes get zones of alike length.
__global__ void __launch_bounds__(128, 1) k_multi_estimate(const __grid_constant__ MultiParams M,
                                                          double* key, int32_t* idx) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  double* lane_base = M.ws + warp * (long long)M.lane_doubles * WS_LANES + lane;
  const long long total = M.off[M.n];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += stride) {
    int m = 0;
    while (m + 1 < M.n && c >= M.off[m + 1]) ++m;
    const BurnParams& P = M.p[m];
    const Net t = make_net(P.blob);
    WS w = make_ws(t, lane_base);
    Zone s;
    s.z = c - M.off[m];
    const bool done = zone_init(t, s, w, P);
    key[c] = done ? 1e300 : s.h;
    idx[c] = (int32_t)c;
  }
}

// a cost proxy per zone of a network: sets with larger networks are claimed
// first, so their long zones start early
long long set_cost(const nb_net net) {
  const BlobHeader& h = net->h;
  return (long long)h.nnz * 4 + (long long)h.nd + (long long)h.R * 8;
}

}  // namespace

extern "C" int nb_burn_multi(int32_t n_sets, const nb_burn_set* sets, double t_end,
                             double rtol, double atol, const nb_options* opt, void* stream) {
  if (n_sets < 1 || n_sets > NB_MULTI_MAX_SETS || !sets) return NB_E_ARG;
  if (!(rtol > 0.0) || !(atol > 0.0) || !(t_end >= 0.0) || !std::isfinite(t_end)) return NB_E_ARG;
  nb_options o;
  nb_default_options(&o);
  if (opt) o = *opt;
  if (o.max_attempts <= 0 || !(o.time_budget_s >= 0.0)) return NB_E_ARG;
  const int tpb = o.threads_per_block > 0 ? o.threads_per_block : 128;
  if (tpb % 32 != 0 || tpb > 128) return NB_E_ARG;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  long long total = 0;
  int lane_doubles = 1;
  for (int i = 0; i < n_sets; ++i) {
    const nb_burn_set& b = sets[i];
    if (!b.net || b.Z < 0 || b.net->device != dev) return NB_E_ARG;
    if (b.Z > 0 && (!b.Y0 || !b.T9_0 || !b.rho || !b.Y || !b.T9 || !b.status)) return NB_E_ARG;
    total += b.Z;
    lane_doubles = std::max(lane_doubles, (int)b.net->h.lane_doubles);
  }
  if (total == 0) return NB_OK;
  // claim order: larger networks first
  std::vector<int> ord(n_sets);
  for (int i = 0; i < n_sets; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
    return set_cost(sets[a].net) > set_cost(sets[b].net);
  });
  MultiParams M;
  std::memset(&M, 0, sizeof(M));
  M.n = n_sets;
  M.lane_doubles = lane_doubles;
  M.budget_ns = o.time_budget_s > 0.0 ? (unsigned long long)(o.time_budget_s * 1e9) + 1ull : 0ull;
  long long off = 0;
  for (int k = 0; k < n_sets; ++k) {
    const nb_burn_set& b = sets[ord[k]];
    BurnParams& P = M.p[k];
    M.off[k] = off;
    off += b.Z;
    P.blob = b.net->d_blob;
    P.blob_bytes = b.net->h.bytes;
    P.Z = b.Z;
    P.Y0 = b.Y0; P.T9_0 = b.T9_0; P.rho = b.rho;
    P.t_end = t_end; P.rtol = rtol; P.atol = atol;
    P.lnm = b.ln_mult; P.lnm_per_zone = b.ln_mult_per_zone ? 1 : 0;
    P.Y = b.Y; P.T9 = b.T9; P.E = b.E; P.counters = b.counters; P.status = b.status;
    P.max_attempts = o.max_attempts;
    P.t_end_zone = b.t_end_zone;
    P.zeta_zone = b.zeta_zone;
  }
  M.off[n_sets] = off;
  // the first set's network lends its workspace and queue counter
  nb_net host = sets[0].net;
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(host->mu);
  int occ = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_burn_multi, tpb, 0));
  if (occ < 1) return NB_E_TOO_LARGE;
  const int bps = std::max(1, std::min(o.blocks_per_sm > 0 ? o.blocks_per_sm : 1, occ));
  long long blocks = (long long)bps * host->sm_count;
  blocks = std::min(blocks, (total + tpb - 1) / tpb);
  const size_t need = (size_t)blocks * tpb * lane_doubles * sizeof(double);
  int rc = nb::ensure((void**)&host->ws, &host->ws_bytes, need);
  if (rc) return rc;
  M.ws = host->ws;
  M.queue = host->queue;
  M.order = nullptr;
  if (o.schedule == 1 && total > 1 && total <= 0x7fffffffLL) {
    // longest first within each set (segments at the sets' claim offsets)
    int seg[NB_MULTI_MAX_SETS + 1];
    for (int k = 0; k <= n_sets; ++k) seg[k] = (int)M.off[k];
    size_t temp = 0;
    CK(cub::DeviceSegmentedRadixSort::SortPairs(
        nullptr, temp, (const double*)nullptr, (double*)nullptr, (const int32_t*)nullptr,
        (int32_t*)nullptr, (int)total, n_sets, seg, seg + 1, 0, 64, st));
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t kb = al((size_t)total * 8), ib = al((size_t)total * 4);
    const size_t sb = al(sizeof(seg));
    rc = nb::ensure((void**)&host->sched, &host->sched_bytes, 2 * kb + 2 * ib + sb + al(temp));
    if (rc) return rc;
    unsigned char* base = host->sched;
    double* k_in = (double*)base;
    double* k_out = (double*)(base + kb);
    int32_t* i_in = (int32_t*)(base + 2 * kb);
    int32_t* i_out = (int32_t*)(base + 2 * kb + ib);
    int* d_seg = (int*)(base + 2 * kb + 2 * ib);
    void* tmp = base + 2 * kb + 2 * ib + sb;
    CK(cudaMemcpyAsync(d_seg, seg, sizeof(seg), cudaMemcpyHostToDevice, st));
    k_multi_estimate<<<(unsigned)blocks, tpb, 0, st>>>(M, k_in, i_in);
    CK(cudaGetLastError());
    CK(cub::DeviceSegmentedRadixSort::SortPairs(tmp, temp, k_in, k_out, i_in, i_out, (int)total,
                                                n_sets, d_seg, d_seg + 1, 0, 64, st));
    M.order = i_out;
  }
  CK(cudaMemsetAsync(host->queue, 0, sizeof(unsigned long long), st));
  k_burn_multi<<<(unsigned)blocks, tpb, 0, st>>>(M);
  CK(cudaGetLastError());
  return NB_OK;
}
