// burn.cu -- kernels and C ABI of the batched reaction-network burn.
//
// Three launch shapes run the same per-zone integrator (integrator.cuh):
//  * persistent: a grid sized to the GPU (blocks_per_sm x SMs); every lane
//    claims zones from a device work queue and claims the next one as soon as
//    its zone finishes, so zones needing 10 or 10^4 steps share warps without
//    idling the FP64 pipe;
//  * cooperative: persistent too, but one warp per zone (coop.cuh), its
//    Newton-loop arrays in shared memory: for large networks;
//  * plain: one thread per zone, one launch over all zones (the comparison
//    launch).
#include <cuda_runtime.h>
#include <cub/device/device_radix_sort.cuh>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "blob.h"
#include "codegen.h"
#include "coop.cuh"
#include "device.cuh"
#include "../../include/netburn.h"

namespace nb {
int build_blob(const nb_topology* T, const double* coeffs,
               std::vector<uint8_t>* out, BlobHeader* hdr_out);
}

using namespace nb;

// ------------------------------------------------------------------ kernels

// Work arrays of a lane: the first P.smem_warps warps of every block keep
// their Newton-loop ("hot") arrays in shared memory after the (optional) blob
// copy and only their history in global memory; the other warps keep
// everything in the global workspace.  Per block the global workspace holds
// smem_warps x cold + (warps - smem_warps) x lane_doubles doubles per lane.
__global__ void __launch_bounds__(256, 1) k_burn_persistent(BurnParams P) {
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
  const int wib = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const long long cold = t.lane_doubles - t.hot_doubles;
  const long long block_doubles =
      ((long long)P.smem_warps * cold + (long long)(wpb - P.smem_warps) * t.lane_doubles) * WS_LANES;
  double* gbase = P.ws + (long long)blockIdx.x * block_doubles;
  WS w;
  if (wib < P.smem_warps) {
    double* hot = reinterpret_cast<double*>(sm + (P.blob_in_smem ? P.blob_bytes : 0)) +
                  (size_t)wib * t.hot_doubles * WS_LANES + lane;
    w = make_ws_split(t, hot, gbase + (long long)wib * cold * WS_LANES + lane);
  } else {
    w = make_ws(t, gbase + (long long)P.smem_warps * cold * WS_LANES +
                       (long long)(wib - P.smem_warps) * t.lane_doubles * WS_LANES + lane);
  }
  burn_claim_loop(t, w, P);
}

// One zone per team of W threads: a warp (W = 32, every warp of the block
// its own team), or the whole block (W = 64 or 128).  With P.smem_warps > 0
// every team keeps the Newton-loop part of its arrays in shared memory after
// the (optional) blob copy and only the history in the global workspace;
// otherwise everything is in the global workspace, lane_doubles per team.
// A team larger than a warp has its sums' partials and its broadcast slot
// after its arrays in shared memory.
// MINB 1: blocks of up to 8 warps, registers as the code wants (about 250);
// MINB 3: blocks of up to 4 warps, three per SM, registers capped at 168
// (some spilled to L1), for networks whose shared-memory arrays let three
// blocks share an SM.
template <int MINB, int W>
__global__ void __launch_bounds__(W > 32 ? W : (MINB == 1 ? 256 : 128), MINB)
    k_burn_coop(BurnParams P) {
  extern __shared__ __align__(16) unsigned char sm[];
  const unsigned char* blob = P.blob;
  if (P.blob_in_smem) {
    const int4* src = reinterpret_cast<const int4*>(P.blob);
    int4* dst = reinterpret_cast<int4*>(sm);
    for (int i = threadIdx.x; i < P.blob_bytes / 16; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    blob = sm;
  }
  double* smd = reinterpret_cast<double*>(sm + (P.blob_in_smem ? P.blob_bytes : 0));
  const int tib = threadIdx.x / W;
  const long long team = (long long)blockIdx.x * (blockDim.x / W) + tib;
  const BlobHeader* bh = reinterpret_cast<const BlobHeader*>(blob);
  double* red = nullptr;
  if constexpr (W > 32) red = smd + (P.smem_warps > 0 ? bh->hot_doubles : 0);
  const WNetT<W> t = make_wnet<W>(blob, threadIdx.x % W, red);
  double *hot, *cold;
  if (P.smem_warps > 0) {
    hot = smd + (size_t)tib * t.g.hot_doubles;
    cold = P.ws + team * (long long)(t.g.lane_doubles - t.g.hot_doubles);
  } else {
    hot = P.ws + team * (long long)t.g.lane_doubles;
    cold = hot + t.g.hot_doubles;
  }
  CWS w = make_cws(t.g, hot, cold);
  coop_claim_loop(t, w, P);
}

// Scheduling pre-pass: each zone's starting step h0 (the integrator's own
// start-up, nothing recorded) as its sort key; zones that finish in start-up
// go last.
__global__ void __launch_bounds__(128, 2) k_burn_estimate(BurnParams P, double* key,
                                                           int32_t* idx) {
  const Net t = make_net(P.blob);
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const WS w = make_ws(t, P.ws + warp * (long long)t.lane_doubles * WS_LANES + lane);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x; z < P.Z; z += stride) {
    Zone s;
    s.z = z;
    const bool done = zone_init(t, s, w, P);
    key[z] = done ? 1e300 : s.h;
    idx[z] = (int32_t)z;
  }
}

// Predicted cost of every zone, (1 + ln(t_end / h0))^2 from the starting step
// h0 of the integrator's start-up (0 for zones that finish in start-up): on
// the 48-species network it follows the step attempts with correlation 0.96.
__global__ void __launch_bounds__(128, 2) k_zone_cost(BurnParams P, double* cost) {
  const Net t = make_net(P.blob);
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const WS w = make_ws(t, P.ws + warp * (long long)t.lane_doubles * WS_LANES + lane);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x; z < P.Z; z += stride) {
    Zone s;
    s.z = z;
    const bool done = zone_init(t, s, w, P);
    const double e = done ? -1.0 : log(s.tend / s.h);
    cost[z] = done ? 0.0 : (1.0 + fmax(e, 0.0)) * (1.0 + fmax(e, 0.0));
  }
}

__global__ void __launch_bounds__(128, 2) k_burn_plain(BurnParams P) {
  const Net t = make_net(P.blob);
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= P.Z) return;
  const int lane = threadIdx.x & 31;
  double* lane_base = P.ws + (gid >> 5) * (long long)t.lane_doubles * WS_LANES + lane;
  const WS w = make_ws(t, lane_base);
  Zone s;
  s.z = gid;
  const unsigned long long t_start = P.budget_ns ? gpu_ns() : 0ull;
  if (P.budget_ns && gpu_ns() - t_start > P.budget_ns) {
    zone_timeout_unstarted(t, gid, P);
    return;
  }
  bool done = zone_init(t, s, w, P);
  while (!done) {
    if (P.budget_ns && gpu_ns() - t_start > P.budget_ns) {
      s.status = NB_Z_TIMEOUT;
      break;
    }
    done = zone_attempt(t, s, w, P);
  }
  zone_finish(t, s, w, P);
}

// ------------------------------------------------------------------ host side

#include "host.h"

extern "C" {

void nb_default_options(nb_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->max_attempts = 500000;
  o->kernel = NB_KERNEL_PERSISTENT;
  o->threads_per_block = 0;
  o->blocks_per_sm = 0;
  o->blob_in_shared = -1;
  o->schedule = 1;
}

const char* nb_strerror(int code) {
  switch (code) {
    case NB_OK: return "ok";
    case NB_E_ARG: return "bad argument";
    case NB_E_TOPOLOGY: return "bad topology (species index out of range or empty reaction)";
    case NB_E_TOO_LARGE: return "network exceeds the compiled limits";
    case NB_E_CUDA: return "CUDA runtime error";
    case NB_E_NOMEM: return "allocation failed";
    case NB_E_TAPE: return "tape missing, too small or from another network";
    case NB_E_COMPILE: return "network-specialised kernel could not be generated, compiled or loaded";
    default: return "unknown error";
  }
}

int nb_net_load(const nb_topology* T, const double* coeffs, nb_net* out) {
  if (!T || !out || (T->n_reactions > 0 && (!coeffs || !T->reactants || !T->products)))
    return NB_E_ARG;
  *out = nullptr;
  const int N = T->n_species, R = T->n_reactions;
  if (N < 1 || R < 0) return NB_E_ARG;
  if (T->self_heating && !T->Q) return NB_E_ARG;
  for (int r = 0; r < R; ++r) {
    int nre = 0;
    for (int s = 0; s < 3; ++s) {
      const int a = T->reactants[3 * r + s], b = T->products[3 * r + s];
      if (a < -1 || a >= N || b < -1 || b >= N) return NB_E_TOPOLOGY;
      nre += a >= 0;
    }
    if (nre == 0) return NB_E_TOPOLOGY;
    for (int j = 0; j < 7; ++j)
      if (!std::isfinite(coeffs[7 * r + j])) return NB_E_ARG;
    if (T->Q && !std::isfinite(T->Q[r])) return NB_E_ARG;
    if (T->scale && !std::isfinite(T->scale[r])) return NB_E_ARG;
  }
  nb_net net = new (std::nothrow) nb_net_s();
  if (!net) return NB_E_NOMEM;
  int rc = build_blob(T, coeffs, &net->blob, &net->h);
  if (rc != NB_OK) { delete net; return rc; }
  if (cudaGetDevice(&net->device) != cudaSuccess) { delete net; return NB_E_CUDA; }
  cudaDeviceGetAttribute(&net->sm_count, cudaDevAttrMultiProcessorCount, net->device);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, net->device);
  net->smem_optin = (size_t)optin;
  if (cudaMalloc(&net->d_blob, net->blob.size()) != cudaSuccess ||
      cudaMemcpy(net->d_blob, net->blob.data(), net->blob.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMalloc(&net->queue, 256) != cudaSuccess) {
    if (net->d_blob) cudaFree(net->d_blob);
    if (net->queue) cudaFree(net->queue);
    delete net;
    return NB_E_CUDA;
  }
  *out = net;
  return NB_OK;
}

int nb_net_free(nb_net net) {
  if (!net) return NB_E_ARG;
  cudaFree(net->d_blob);
  cudaFree(net->queue);
  if (net->ws) cudaFree(net->ws);
  if (net->stage) cudaFree(net->stage);
  if (net->ws_adj) cudaFree(net->ws_adj);
  if (net->sched) cudaFree(net->sched);
  if (net->sched_adj) cudaFree(net->sched_adj);
  for (auto& sp : net->spec)
    if (sp.lib) cudaLibraryUnload(sp.lib);
  delete net;
  return NB_OK;
}

int nb_net_get_info(nb_net net, nb_net_info* o) {
  if (!net || !o) return NB_E_ARG;
  const BlobHeader& h = net->h;
  std::memset(o, 0, sizeof(*o));
  o->n_state = h.n;
  o->n_reactions = h.R;
  o->nnz_jacobian = h.nnz_jac;
  o->nnz_lu = h.nnz;
  o->n_dterms = h.nd;
  o->lane_doubles = h.lane_doubles;
  o->blob_bytes = h.bytes;
  o->has_energy = h.has_E;
  o->flops_rate_eval = h.fl_teval;
  o->flops_rate_deriv = h.fl_teval_g;
  o->flops_terms = h.fl_terms;
  o->flops_tsolve = h.fl_tsolve;
  o->flops_rhs = h.fl_rhs;
  o->flops_jacobian = h.fl_jac;
  o->flops_lu = h.fl_lu;
  o->flops_solve = h.fl_solve;
  o->flops_edot = h.fl_edot;
  o->exp_per_rate_eval = h.n_exp_per_teval;
  o->specialize_auto = specialize_auto_ok(h) ? 1 : 0;
  o->last_specialized = net->last_spec;
  return NB_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ specialised kernel

// The specialised kernel of `variant` (1..3) for this network, generated,
// compiled and loaded on first use.  Caller holds net->mu.
static int spec_get(nb_net net, int variant, const void** fn) {
  nb_net_s::Spec& sp = net->spec[variant];
  if (sp.state == 0) {
    std::vector<char> cubin;
    const std::string src = specialized_source(net->blob, variant);
    int rc = compile_specialized(src, &cubin, &sp.log, false);
    if (rc == NB_OK &&
        (cudaLibraryLoadData(&sp.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) !=
             cudaSuccess ||
         cudaLibraryGetKernel(&sp.kern, sp.lib, "nb_spec_burn") != cudaSuccess)) {
      cudaGetLastError();
      if (sp.lib) cudaLibraryUnload(sp.lib);
      sp.lib = nullptr;
      sp.kern = nullptr;
      sp.log += "\nloading the compiled kernel failed";
      rc = NB_E_COMPILE;
    }
    sp.state = rc == NB_OK ? 1 : -1;
  }
  if (sp.state != 1) return NB_E_COMPILE;
  *fn = reinterpret_cast<const void*>(sp.kern);
  return NB_OK;
}

static void copy_log(const std::string& s, char* log, int64_t cap) {
  if (!log || cap <= 0) return;
  const size_t n = std::min<size_t>(s.size(), (size_t)cap - 1);
  std::memcpy(log, s.data(), n);
  log[n] = '\0';
}

extern "C" int nb_net_specialize(nb_net net, int32_t variant, char* log, int64_t log_bytes) {
  if (!net || variant < 0 || variant > 3) return NB_E_ARG;
  std::lock_guard<std::mutex> lk(net->mu);
  const int v = resolve_variant(net->h, variant);
  const void* fn = nullptr;
  const int rc = spec_get(net, v, &fn);
  copy_log(net->spec[v].log, log, log_bytes);
  return rc;
}

// build the blob of a topology on the host (the checks of nb_net_load)
static int host_blob(const nb_topology* T, const double* coeffs, std::vector<uint8_t>* blob) {
  if (!T || (T->n_reactions > 0 && (!coeffs || !T->reactants || !T->products))) return NB_E_ARG;
  if (T->n_species < 1 || T->n_reactions < 0 || (T->self_heating && !T->Q)) return NB_E_ARG;
  BlobHeader h;
  return build_blob(T, coeffs, blob, &h);
}

extern "C" int nb_specialize_source(const nb_topology* T, const double* coeffs,
                                    int32_t variant, char* buf, int64_t cap, int64_t* len) {
  if (!len || variant < 0 || variant > 3) return NB_E_ARG;
  std::vector<uint8_t> blob;
  int rc = host_blob(T, coeffs, &blob);
  if (rc) return rc;
  const std::string src = specialized_source(blob, variant);
  *len = (int64_t)src.size();
  if (!buf || cap < (int64_t)src.size() + 1) return NB_E_ARG;
  std::memcpy(buf, src.c_str(), src.size() + 1);
  return NB_OK;
}

extern "C" int nb_specialize_compile(const nb_topology* T, const double* coeffs,
                                     int32_t variant, char* log, int64_t log_bytes) {
  if (variant < 0 || variant > 3) return NB_E_ARG;
  std::vector<uint8_t> blob;
  int rc = host_blob(T, coeffs, &blob);
  if (rc) return rc;
  std::string lg;
  std::vector<char> cubin;
  rc = compile_specialized(specialized_source(blob, variant), &cubin, &lg, true);
  copy_log(lg, log, log_bytes);
  return rc;
}

// Longest-first claim order: h0 of every zone (pre-pass over the workspace
// lanes already allocated), then a radix sort of (h0, zone).  Sets P.order.
static int schedule_longest_first(nb_net net, BurnParams& P, long long lanes,
                                  cudaStream_t st) {
  const long long Z = P.Z;
  if (Z > 0x7fffffffLL) return NB_E_TOO_LARGE;
  size_t temp = 0;
  CK(cub::DeviceRadixSort::SortPairs(nullptr, temp, (const double*)nullptr, (double*)nullptr,
                                     (const int32_t*)nullptr, (int32_t*)nullptr, (int)Z, 0,
                                     64, st));
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t kb = al((size_t)Z * 8), ib = al((size_t)Z * 4);
  const size_t need = 2 * kb + 2 * ib + al(temp);
  int rc = nb::ensure((void**)&net->sched, &net->sched_bytes, need);
  if (rc) return rc;
  unsigned char* base = net->sched;
  double* k_in = (double*)base;
  double* k_out = (double*)(base + kb);
  int32_t* i_in = (int32_t*)(base + 2 * kb);
  int32_t* i_out = (int32_t*)(base + 2 * kb + ib);
  void* tmp = base + 2 * kb + 2 * ib;
  BurnParams E = P;
  E.use_tape = 0;
  const long long fit = (long long)(net->ws_bytes / ((size_t)net->h.lane_doubles * sizeof(double)));
  const long long eblocks = std::max(1LL, std::min(lanes, fit) / 128);
  k_burn_estimate<<<(unsigned)eblocks, 128, 0, st>>>(E, k_in, i_in);
  CK(cudaGetLastError());
  CK(cub::DeviceRadixSort::SortPairs(tmp, temp, k_in, k_out, i_in, i_out, (int)Z, 0, 64, st));
  P.order = i_out;
  return NB_OK;
}

// The cooperative launch: one warp per zone.  threads_per_block (default:
// the warps whose Newton-loop arrays fit in shared memory, at most 4 of
// them) and blocks_per_sm set the zones in flight; ws_in_shared 0 keeps all
// arrays in global memory, otherwise (default) in shared memory when they
// fit; blob_in_shared as for the persistent kernel.
static int launch_coop(nb_net net, BurnParams& P, const nb_options& o, cudaStream_t st) {
  const size_t blob_b = (size_t)net->h.bytes;
  const size_t hot_team = (size_t)net->h.hot_doubles * sizeof(double);
  const size_t team_doubles = (size_t)net->h.lane_doubles;
  const int wpz = o.warps_per_zone <= 1 ? 1 : o.warps_per_zone;
  if (o.warps_per_zone < 0 || (wpz != 1 && wpz != 2 && wpz != 4)) return NB_E_ARG;
  const size_t scratch = (size_t)team_scratch_doubles(32 * wpz) * sizeof(double);
  const bool hot_smem = o.ws_in_shared != 0 && hot_team + scratch <= net->smem_optin;
  int in_smem = o.blob_in_shared;
  if (in_smem < 0)
    in_smem = blob_b <= 96 * 1024 &&
              blob_b + (hot_smem ? hot_team : 0) + scratch <= net->smem_optin;
  const size_t fixed = (in_smem ? blob_b : 0) + scratch;
  // teams per block; three blocks of at most four warps per SM when asked for
  int tpb_teams;
  const bool dense =
      wpz == 1 && o.blocks_per_sm >= 3 && o.threads_per_block > 0 && o.threads_per_block <= 128;
  const void* kern = wpz == 4 ? (const void*)k_burn_coop<1, 128>
                   : wpz == 2 ? (const void*)k_burn_coop<1, 64>
                   : dense    ? (const void*)k_burn_coop<3, 32>
                              : (const void*)k_burn_coop<1, 32>;
  if (wpz > 1) {
    tpb_teams = 1;
  } else if (o.threads_per_block > 0) {
    if (o.threads_per_block % 32 != 0 || o.threads_per_block > 256) return NB_E_ARG;
    tpb_teams = o.threads_per_block / 32;
  } else {
    tpb_teams = 4;
    if (hot_smem)
      while (tpb_teams > 1 && fixed + (size_t)tpb_teams * hot_team > net->smem_optin) --tpb_teams;
  }
  const int threads = wpz > 1 ? 32 * wpz : 32 * tpb_teams;
  const size_t dyn = fixed + (hot_smem ? (size_t)tpb_teams * hot_team : 0);
  if (dyn > net->smem_optin) return NB_E_TOO_LARGE;
  CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  int occ = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, dyn));
  if (occ < 1) return NB_E_TOO_LARGE;
  const int bps = std::max(1, std::min(o.blocks_per_sm > 0 ? o.blocks_per_sm : occ, occ));
  long long blocks = (long long)bps * net->sm_count;
  const long long needed = (P.Z + tpb_teams - 1) / tpb_teams;
  if (blocks > needed) blocks = needed;
  const size_t per_team = (hot_smem ? team_doubles - net->h.hot_doubles : team_doubles) * 8;
  size_t need = std::max<size_t>((size_t)blocks * tpb_teams * per_team, 256);
  const size_t lane_bytes = team_doubles * sizeof(double);
  if (o.schedule == 1) need = std::max(need, (size_t)128 * lane_bytes);  // pre-pass lanes
  int rc = nb::ensure((void**)&net->ws, &net->ws_bytes, need);
  if (rc) return rc;
  P.ws = net->ws;
  P.queue = net->queue;
  P.blob_in_smem = in_smem;
  P.smem_warps = hot_smem ? tpb_teams : 0;
  P.order = nullptr;
  if (o.schedule == 1 && P.Z > 1) {
    rc = schedule_longest_first(net, P, 128, st);
    if (rc) return rc;
  }
  CK(cudaMemsetAsync(net->queue, 0, sizeof(unsigned long long), st));
  if (wpz == 4)
    k_burn_coop<1, 128><<<(unsigned)blocks, threads, dyn, st>>>(P);
  else if (wpz == 2)
    k_burn_coop<1, 64><<<(unsigned)blocks, threads, dyn, st>>>(P);
  else if (dense)
    k_burn_coop<3, 32><<<(unsigned)blocks, threads, dyn, st>>>(P);
  else
    k_burn_coop<1, 32><<<(unsigned)blocks, threads, dyn, st>>>(P);
  CK(cudaGetLastError());
  return NB_OK;
}

// Launch one burn (device pointers).  Caller holds net->mu.
static int launch_burn(nb_net net, BurnParams& P, const nb_options& o,
                       cudaStream_t st) {
  net->last_spec = 0;
  if (o.kernel != NB_KERNEL_PERSISTENT && o.kernel != NB_KERNEL_PLAIN &&
      o.kernel != NB_KERNEL_COOP)
    return NB_E_ARG;
  int tpb = o.threads_per_block > 0 ? o.threads_per_block : 128;
  if (o.threads_per_block <= 0 && o.kernel != NB_KERNEL_PLAIN) {
    // few zones: smaller blocks, so that every SM gets some
    const long long per_sm = (P.Z + net->sm_count - 1) / net->sm_count;
    if (per_sm < 128) tpb = (int)std::max(32LL, per_sm / 32 * 32);
  }
  if (tpb % 32 != 0 || tpb > 256 || (o.kernel == NB_KERNEL_PLAIN && tpb > 128)) return NB_E_ARG;
  const size_t lane_bytes = (size_t)net->h.lane_doubles * sizeof(double);
  P.blob = net->d_blob;
  P.blob_bytes = net->h.bytes;
  if (o.kernel == NB_KERNEL_COOP) return launch_coop(net, P, o, st);
  if (o.kernel == NB_KERNEL_PLAIN) {
    const long long blocks = (P.Z + tpb - 1) / tpb;
    const size_t need = (size_t)blocks * tpb * lane_bytes;
    int rc = nb::ensure((void**)&net->ws, &net->ws_bytes, need);
    if (rc) return rc;
    P.ws = net->ws;
    P.blob_in_smem = 0;
    k_burn_plain<<<(unsigned)blocks, tpb, 0, st>>>(P);
    CK(cudaGetLastError());
    return NB_OK;
  }
  // the specialised kernel: o.specialize > 0 asks for it, 0 takes it when
  // the network qualifies and it builds
  const void* spec_fn = nullptr;
  int spec_variant = 0;
  if (o.specialize > 3 || o.specialize < -1) return NB_E_ARG;
  if (o.kernel == NB_KERNEL_PERSISTENT && o.ws_in_shared <= 0 && o.specialize >= 0) {
    if (o.specialize > 0) {
      int rc = spec_get(net, o.specialize, &spec_fn);
      if (rc) return rc;
      spec_variant = o.specialize;
    } else if (specialize_auto_ok(net->h)) {
      spec_variant = resolve_variant(net->h, 0);
      if (spec_get(net, spec_variant, &spec_fn) != NB_OK) {
        spec_fn = nullptr;
        spec_variant = 0;
      }
    }
  }
  if (spec_fn) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, spec_fn, tpb, 0) != cudaSuccess) {
      cudaGetLastError();
      occ = 1;
    }
    if (occ < 1) return NB_E_TOO_LARGE;
    int bps = o.blocks_per_sm > 0 ? std::min(o.blocks_per_sm, occ) : 1;
    long long blocks = (long long)bps * net->sm_count;
    const long long needed_blocks = (P.Z + tpb - 1) / tpb;
    if (blocks > needed_blocks) blocks = needed_blocks;
    size_t need = std::max<size_t>((size_t)blocks * tpb * lane_bytes, 256);
    if (o.schedule == 1) need = std::max(need, (size_t)128 * lane_bytes);  // pre-pass lanes
    int rc = nb::ensure((void**)&net->ws, &net->ws_bytes, need);
    if (rc) return rc;
    P.ws = net->ws;
    P.queue = net->queue;
    P.blob_in_smem = 0;
    P.smem_warps = 0;
    P.order = nullptr;
    if (o.schedule == 1 && P.Z > 1) {
      rc = schedule_longest_first(net, P, blocks * (long long)tpb, st);
      if (rc) return rc;
    }
    CK(cudaMemsetAsync(net->queue, 0, sizeof(unsigned long long), st));
    void* args[] = {&P};
    CK(cudaLaunchKernel(spec_fn, dim3((unsigned)blocks), dim3(tpb), args, 0, st));
    net->last_spec = spec_variant;
    return NB_OK;
  }
  const size_t blob_b = (size_t)net->h.bytes;
  const size_t hot_warp = (size_t)net->h.hot_doubles * WS_LANES * sizeof(double);
  const int wpb = tpb / 32;
  // ws_in_shared: -1 none by default, >= 1 that many warps of each block
  // keep their Newton-loop arrays in shared memory
  const int smem_warps = o.ws_in_shared > 0 ? std::min(o.ws_in_shared, wpb) : 0;
  int in_smem = o.blob_in_shared;
  if (in_smem < 0) in_smem = blob_b <= 96 * 1024 && blob_b + smem_warps * hot_warp <= net->smem_optin;
  size_t dyn = (in_smem ? blob_b : 0) + (size_t)smem_warps * hot_warp;
  if (dyn > net->smem_optin) return NB_E_TOO_LARGE;
  if (dyn > 48 * 1024)
    CK(cudaFuncSetAttribute(k_burn_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  int bps = o.blocks_per_sm;
  int occ = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_burn_persistent, tpb, dyn));
  if (occ < 1) return NB_E_TOO_LARGE;
  if (bps <= 0) bps = 1;
  bps = std::max(1, std::min(bps, occ));
  long long blocks = (long long)bps * net->sm_count;
  const long long needed_blocks = (P.Z + tpb - 1) / tpb;
  if (blocks > needed_blocks) blocks = needed_blocks;
  const size_t cold_bytes = lane_bytes - (size_t)net->h.hot_doubles * sizeof(double);
  const size_t per_block = (size_t)32 * (smem_warps * cold_bytes + (wpb - smem_warps) * lane_bytes);
  size_t need = std::max<size_t>((size_t)blocks * per_block, 256);
  if (o.schedule == 1) need = std::max(need, (size_t)128 * lane_bytes);  // pre-pass lanes
  int rc = nb::ensure((void**)&net->ws, &net->ws_bytes, need);
  if (rc) return rc;
  P.ws = net->ws;
  P.queue = net->queue;
  P.blob_in_smem = in_smem;
  P.smem_warps = smem_warps;
  P.order = nullptr;
  if (o.schedule == 1 && P.Z > 1) {
    rc = schedule_longest_first(net, P, blocks * (long long)tpb, st);
    if (rc) return rc;
  }
  CK(cudaMemsetAsync(net->queue, 0, sizeof(unsigned long long), st));
  k_burn_persistent<<<(unsigned)blocks, tpb, dyn, st>>>(P);
  CK(cudaGetLastError());
  return NB_OK;
}

extern "C" int nb_zone_costs(nb_net net, int64_t Z, const double* Y0, const double* T9_0,
                             const double* rho, double t_end, double rtol, double atol,
                             const nb_options* opt, double* cost, void* stream) {
  if (!net || Z < 0 || !(rtol > 0.0) || !(atol > 0.0) || !(t_end >= 0.0) ||
      !std::isfinite(t_end))
    return NB_E_ARG;
  if (Z == 0) return NB_OK;
  if (!Y0 || !T9_0 || !rho || !cost) return NB_E_ARG;
  nb_options o;
  nb_default_options(&o);
  if (opt) o = *opt;
  BurnParams P;
  std::memset(&P, 0, sizeof(P));
  P.Z = Z; P.Y0 = Y0; P.T9_0 = T9_0; P.rho = rho;
  P.t_end = t_end; P.rtol = rtol; P.atol = atol;
  P.t_end_zone = o.t_end_zone;
  P.zeta_zone = o.zeta_zone;
  P.blob = net->d_blob;
  P.blob_bytes = net->h.bytes;
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(net->mu);
  const size_t lane_bytes = (size_t)net->h.lane_doubles * sizeof(double);
  const long long lanes = std::min<long long>((long long)net->sm_count * 256, (Z + 31) / 32 * 32);
  int rc = nb::ensure((void**)&net->ws, &net->ws_bytes, (size_t)lanes * lane_bytes);
  if (rc) return rc;
  P.ws = net->ws;
  k_zone_cost<<<(unsigned)((lanes + 127) / 128), 128, 0, st>>>(P, cost);
  CK(cudaGetLastError());
  return NB_OK;
}

static int check_burn_args(long long Z, double t_end, double rtol, double atol) {
  if (Z < 0) return NB_E_ARG;
  if (!(rtol > 0.0) || !(atol > 0.0) || !(t_end >= 0.0) || !std::isfinite(t_end))
    return NB_E_ARG;
  return NB_OK;
}

extern "C" int nb_burn_batch(nb_net net, int64_t Z, const double* Y0, const double* T9_0,
                             const double* rho, double t_end, double rtol, double atol,
                             const double* ln_mult, int32_t ln_mult_per_zone, double* Y,
                             double* T9, double* E, int32_t* counters, int32_t* status,
                             const nb_options* opt, void* tape, void* stream) {
  if (!net) return NB_E_ARG;
  int rc = check_burn_args(Z, t_end, rtol, atol);
  if (rc) return rc;
  if (Z == 0) return NB_OK;
  if (!Y0 || !T9_0 || !rho || !Y || !T9 || !status) return NB_E_ARG;
  nb_options o;
  nb_default_options(&o);
  if (opt) o = *opt;
  if (o.max_attempts <= 0) return NB_E_ARG;
  BurnParams P;
  std::memset(&P, 0, sizeof(P));
  P.Z = Z; P.Y0 = Y0; P.T9_0 = T9_0; P.rho = rho;
  P.t_end = t_end; P.rtol = rtol; P.atol = atol;
  P.lnm = ln_mult; P.lnm_per_zone = ln_mult_per_zone ? 1 : 0;
  P.Y = Y; P.T9 = T9; P.E = E; P.counters = counters; P.status = status;
  P.max_attempts = o.max_attempts;
  if (!(o.time_budget_s >= 0.0)) return NB_E_ARG;
  P.budget_ns = o.time_budget_s > 0.0 ? (unsigned long long)(o.time_budget_s * 1e9) + 1ull : 0ull;
  P.t_end_zone = o.t_end_zone;
  P.zeta_zone = o.zeta_zone;
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(net->mu);
  nb_tape_s* tp = (nb_tape_s*)tape;
  if (tp) {
    if (tp->magic != 0x7a9e5eedu || tp->net != net || tp->Z < Z) return NB_E_TAPE;
    P.use_tape = 1;
    P.tape = tp->dev;
    tp->recorded = 0;
    if (ln_mult) {
      const size_t cnt = (size_t)(P.lnm_per_zone ? Z : 1) * net->h.R;
      CK(cudaMemcpyAsync(tp->lnm, ln_mult, cnt * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
  }
  rc = launch_burn(net, P, o, st);
  if (rc || !tp) return rc;
  tp->recZ = Z;
  tp->recorded = 1;
  // teams of several warps per zone sum in another order than one warp: a
  // family of their own, which no adjoint kernel recomputes
  tp->family = o.kernel != NB_KERNEL_COOP ? NB_KERNEL_PERSISTENT
               : o.warps_per_zone > 1    ? NB_KERNEL_COOP + 8 * o.warps_per_zone
                                         : NB_KERNEL_COOP;
  tp->t_end = t_end; tp->rtol = rtol; tp->atol = atol;
  tp->has_lnm = ln_mult != nullptr;
  tp->lnm_per_zone = P.lnm_per_zone;
  return NB_OK;
}

extern "C" int nb_burn_batch_host(nb_net net, int64_t Z, const double* Y0,
                                  const double* T9_0, const double* rho, double t_end,
                                  double rtol, double atol, const double* ln_mult,
                                  int32_t ln_mult_per_zone, double* Y, double* T9,
                                  double* E, int32_t* counters, int32_t* status,
                                  const nb_options* opt, void* stream) {
  if (!net) return NB_E_ARG;
  int rc = check_burn_args(Z, t_end, rtol, atol);
  if (rc) return rc;
  if (Z == 0) return NB_OK;
  if (!Y0 || !T9_0 || !rho || !Y || !T9 || !status) return NB_E_ARG;
  nb_options o;
  nb_default_options(&o);
  if (opt) o = *opt;
  if (o.max_attempts <= 0) return NB_E_ARG;
  const int N = net->h.N, R = net->h.R;
  const size_t zN = (size_t)Z * N * 8, z8 = (size_t)Z * 8, z4 = (size_t)Z * 4;
  const size_t nl = ln_mult ? (size_t)(ln_mult_per_zone ? Z : 1) * R * 8 : 0;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t off_Y0 = 0, off_T0 = off_Y0 + al(zN), off_rho = off_T0 + al(z8),
               off_l = off_rho + al(z8), off_Y = off_l + al(nl), off_T = off_Y + al(zN),
               off_E = off_T + al(z8), off_c = off_E + al(z8),
               off_s = off_c + al(z4 * NCOUNT), total = off_s + al(z4);
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(net->mu);
  rc = nb::ensure((void**)&net->stage, &net->stage_bytes, total);
  if (rc) return rc;
  unsigned char* b = net->stage;
  CK(cudaMemcpyAsync(b + off_Y0, Y0, zN, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(b + off_T0, T9_0, z8, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(b + off_rho, rho, z8, cudaMemcpyHostToDevice, st));
  if (nl) CK(cudaMemcpyAsync(b + off_l, ln_mult, nl, cudaMemcpyHostToDevice, st));
  BurnParams P;
  std::memset(&P, 0, sizeof(P));
  P.Z = Z;
  P.Y0 = (const double*)(b + off_Y0);
  P.T9_0 = (const double*)(b + off_T0);
  P.rho = (const double*)(b + off_rho);
  P.t_end = t_end; P.rtol = rtol; P.atol = atol;
  P.lnm = nl ? (const double*)(b + off_l) : nullptr;
  P.lnm_per_zone = ln_mult_per_zone ? 1 : 0;
  P.Y = (double*)(b + off_Y);
  P.T9 = (double*)(b + off_T);
  P.E = (double*)(b + off_E);
  P.counters = (int32_t*)(b + off_c);
  P.status = (int32_t*)(b + off_s);
  P.max_attempts = o.max_attempts;
  if (!(o.time_budget_s >= 0.0)) return NB_E_ARG;
  P.budget_ns = o.time_budget_s > 0.0 ? (unsigned long long)(o.time_budget_s * 1e9) + 1ull : 0ull;
  P.t_end_zone = o.t_end_zone;
  P.zeta_zone = o.zeta_zone;
  rc = launch_burn(net, P, o, st);
  if (rc) return rc;
  CK(cudaMemcpyAsync(Y, b + off_Y, zN, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(T9, b + off_T, z8, cudaMemcpyDeviceToHost, st));
  if (E) CK(cudaMemcpyAsync(E, b + off_E, z8, cudaMemcpyDeviceToHost, st));
  if (counters) CK(cudaMemcpyAsync(counters, b + off_c, z4 * NCOUNT, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(status, b + off_s, z4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return NB_OK;
}

// ------------------------------------------------------------------ tape

extern "C" int nb_tape_alloc(nb_net net, int64_t Z, int32_t max_steps, int32_t ckpt_stride,
                             void** tape) {
  if (!net || !tape || Z <= 0 || max_steps < 1 || max_steps > 0x3ffffffe || ckpt_stride < 0)
    return NB_E_ARG;
  *tape = nullptr;
  nb_tape_s* tp = new (std::nothrow) nb_tape_s();
  if (!tp) return NB_E_NOMEM;
  tp->net = net;
  tp->Z = Z;
  tp->cap = max_steps + 1;
  tp->dev.stride = ckpt_stride > 0 ? ckpt_stride : NB_TAPE_DEFAULT_STRIDE;
  const int m = std::min(tp->dev.stride, HMAX);
  const long long blocks = (max_steps + tp->dev.stride - 1) / tp->dev.stride;
  if (1 + blocks * m > 0x7fffffffLL) { delete tp; return NB_E_ARG; }
  tp->dev.scap = (int32_t)(1 + blocks * m);
  const int n = net->h.n;
  const size_t sched = (size_t)Z * tp->cap * 2 * sizeof(double);
  const size_t ord = (size_t)Z * tp->cap;
  const size_t states = (size_t)Z * tp->dev.scap * (n + 1) * sizeof(double);
  bool ok = cudaMalloc(&tp->dev.sched, sched) == cudaSuccess &&
            cudaMalloc(&tp->dev.ord, ord) == cudaSuccess &&
            cudaMalloc(&tp->dev.states, states) == cudaSuccess &&
            cudaMalloc(&tp->dev.steps, (size_t)Z * 4) == cudaSuccess &&
            cudaMalloc(&tp->dev.zstat, (size_t)Z * 4) == cudaSuccess &&
            cudaMalloc(&tp->dev.rho, (size_t)Z * 8) == cudaSuccess &&
            cudaMalloc(&tp->dev.T9f, (size_t)Z * 8) == cudaSuccess &&
            cudaMalloc(&tp->dev.scr, (size_t)Z * 8) == cudaSuccess &&
            cudaMalloc(&tp->lnm, (size_t)Z * std::max(net->h.R, 1) * 8) == cudaSuccess;
  tp->dev.cap = tp->cap;
  if (!ok) {
    cudaGetLastError();
    tape_release(tp);
    delete tp;
    return NB_E_NOMEM;
  }
  *tape = tp;
  return NB_OK;
}

extern "C" int nb_tape_free(void* tape) {
  nb_tape_s* tp = (nb_tape_s*)tape;
  if (!tp || tp->magic != 0x7a9e5eedu) return NB_E_ARG;
  tape_release(tp);
  tp->magic = 0;
  delete tp;
  return NB_OK;
}

extern "C" int nb_tape_steps(void* tape, const int32_t** steps) {
  nb_tape_s* tp = (nb_tape_s*)tape;
  if (!tp || tp->magic != 0x7a9e5eedu || !steps) return NB_E_ARG;
  *steps = tp->dev.steps;
  return NB_OK;
}

extern "C" int nb_tape_read(void* tape, int64_t z, int32_t cap, double* t, double* h,
                            int32_t* order, double* x, double* E, int32_t* count) {
  nb_tape_s* tp = (nb_tape_s*)tape;
  if (!tp || tp->magic != 0x7a9e5eedu || !count || cap < 0) return NB_E_ARG;
  if (!tp->recorded) return NB_E_TAPE;
  if (z < 0 || z >= tp->recZ) return NB_E_ARG;
  const int n = tp->net->h.n;
  std::lock_guard<std::mutex> lk(tp->net->mu);
  CK(cudaDeviceSynchronize());
  int32_t cnt = 0;
  CK(cudaMemcpy(&cnt, tp->dev.steps + z, 4, cudaMemcpyDeviceToHost));
  *count = cnt;
  if (cnt > cap) return NB_E_ARG;
  if (cnt == 0) return NB_OK;
  std::vector<double> sched((size_t)cnt * 2);
  std::vector<int8_t> ord(cnt);
  CK(cudaMemcpy(sched.data(), tp->dev.sched + (size_t)z * tp->cap * 2, sched.size() * 8,
                cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(ord.data(), tp->dev.ord + (size_t)z * tp->cap, cnt, cudaMemcpyDeviceToHost));
  int kept = 0;   // state slots in use: they increase with the record index
  for (int q = 0; q < cnt; ++q) kept = std::max(kept, tape_state_slot(q, tp->dev.stride) + 1);
  std::vector<double> st((size_t)kept * (n + 1));
  if (kept)
    CK(cudaMemcpy(st.data(), tp->dev.states + (size_t)z * tp->dev.scap * (n + 1),
                  st.size() * 8, cudaMemcpyDeviceToHost));
  for (int q = 0; q < cnt; ++q) {
    if (t) t[q] = sched[2 * q];
    if (h) h[q] = sched[2 * q + 1];
    if (order) order[q] = ord[q];
    const int slot = tape_state_slot(q, tp->dev.stride);
    for (int i = 0; i < n; ++i)
      if (x) x[(size_t)q * n + i] = slot >= 0 ? st[(size_t)slot * (n + 1) + i] : NAN;
    if (E) E[q] = slot >= 0 ? st[(size_t)slot * (n + 1) + n] : NAN;
  }
  return NB_OK;
}
