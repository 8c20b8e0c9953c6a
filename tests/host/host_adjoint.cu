// host_adjoint.cu -- the library's forward burn with a tape and its
// checkpointed reverse sweep (device.cuh, integrator.cuh, adjoint.cuh: the
// generic network) compiled for the host, one zone after another.  Test
// infrastructure: lets the CPU suite check the adjoint's recomputation of
// checkpointed blocks and its gradients against the oracle without a GPU.
#define NB_HD __host__ __device__
#include <cstring>
#include <vector>

#include "../../paper_2312_02836_gb300/csrc/adjoint.cuh"

namespace nb {
int build_blob(const nb_topology*, const double*, std::vector<uint8_t>*, BlobHeader*);
}
using namespace nb;

// Forward burn of Z zones with a tape of cap records and checkpoint stride
// `stride` (host arrays sched [Z, cap, 2], ord [Z, cap], states [Z, scap,
// n+1] with scap = 1 + ceil((cap-1)/stride) min(stride, 7), steps [Z]), then
// the reverse sweep with K cotangent sets (gY [K, Z, N], gE, gT9 [K, Z] or
// null) into dl [K, Z, R], dY0 [K, Z, N], dT0 [K, Z].  -1 if scap differs.
extern "C" int host_adjoint(const nb_topology* T, const double* coeffs, long long Z,
                            const double* Y0, const double* T9_0, const double* rho,
                            const double* zeta, double t_end, double rtol, double atol,
                            int cap, int stride, int scap, int K, const double* gY,
                            const double* gE,
                            const double* gT9, double* Y, double* T9, double* E, int* cnt,
                            int* status, double* sched, signed char* ord, double* states,
                            int* steps, double* dl, double* dY0, double* dT0) {
  std::vector<uint8_t> blob;
  BlobHeader h;
  int rc = build_blob(T, coeffs, &blob, &h);
  if (rc) return rc;
  const Net t = make_net(blob.data());
  const int n = t.n;
  std::vector<int> zstat(Z);
  std::vector<double> trho(Z), tT9(Z), tscr(Z);
  TapeDev tp;
  tp.sched = sched; tp.ord = (int8_t*)ord; tp.states = states; tp.steps = steps;
  tp.zstat = zstat.data(); tp.rho = trho.data(); tp.T9f = tT9.data(); tp.scr = tscr.data();
  tp.cap = cap;
  tp.stride = stride;
  const int m = stride < HMAX ? stride : HMAX;
  tp.scap = 1 + (cap - 1 + stride - 1) / stride * m;
  if (tp.scap != scap) return -1;

  // forward
  std::vector<double> ws((size_t)h.lane_doubles * WS_LANES, 0.0);
  WS w = make_ws(t, ws.data());
  BurnParams P;
  std::memset(&P, 0, sizeof(P));
  P.Z = Z; P.Y0 = Y0; P.T9_0 = T9_0; P.rho = rho; P.zeta_zone = zeta;
  P.t_end = t_end; P.rtol = rtol; P.atol = atol;
  P.Y = Y; P.T9 = T9; P.E = E; P.counters = cnt; P.status = status;
  P.max_attempts = 500000;
  P.use_tape = 1;
  P.tape = tp;
  for (long long z = 0; z < Z; ++z) {
    Zone s;
    s.z = z;
    bool done = zone_init(t, s, w, P);
    while (!done) done = zone_attempt(t, s, w, P);
    zone_finish(t, s, w, P);
  }

  // reverse sweep
  AdjParams A;
  std::memset(&A, 0, sizeof(A));
  A.Z = Z; A.K = K; A.tape = tp; A.rtol = rtol; A.atol = atol;
  A.gY = gY; A.gE = gE; A.gT9 = gT9; A.dl = dl; A.dY0 = dY0; A.dT0 = dT0;
  long long off = h.lane_doubles;
  A.o_lam = (int)off; off += (long long)HMAX * K * n;
  A.o_ee = (int)off; off += (long long)HMAX * K;
  A.o_gr = (int)off; off += (long long)K * h.R;
  A.o_gt = (int)off; off += K;
  A.o_mu = (int)off; off += n;
  A.o_de = (int)off; off += n;
  A.o_seg = (int)off; off += (long long)stride * n;
  A.lane_doubles = off;
  std::vector<double> aws((size_t)off * WS_LANES, 0.0);
  const WS wa = make_ws(t, aws.data());
  const AWS a = make_aws(A, aws.data());
  for (long long z = 0; z < Z; ++z) {
    AdjZone Zs;
    Zs.z = z;
    Zs.rs = 1; Zs.re = 0; Zs.lo = 1;
    bool done = adj_init(t, Zs, wa, a, A);
    while (!done) done = Zs.rs <= Zs.re ? adj_replay(t, Zs, wa, a, A) : adj_step(t, Zs, wa, a, A);
    adj_finish(t, Zs, a, A);
  }
  return 0;
}
