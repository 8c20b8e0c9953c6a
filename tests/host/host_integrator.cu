// host_integrator.cu -- the library's per-zone integrator (device.cuh and
// integrator.cuh, the generic network) compiled for the host, one zone after
// another.  Test infrastructure: lets the CPU suite check the device code's
// integrator logic against the oracle without a GPU.  The host's libm rounds
// differently from the device's, so results agree to the parity bar, not
// bit for bit.
#define NB_HD __host__ __device__
#include <cstring>
#include <vector>

#include "../../paper_2312_02836_gb300/csrc/device.cuh"

namespace nb {
int build_blob(const nb_topology*, const double*, std::vector<uint8_t>*, BlobHeader*);
}
using namespace nb;

extern "C" int host_burn(const nb_topology* T, const double* coeffs, long long Z,
                         const double* Y0, const double* T9_0, const double* rho,
                         const double* zeta, double t_end, double rtol, double atol,
                         double* Y, double* T9, double* E, int* cnt, int* status) {
  std::vector<uint8_t> blob;
  BlobHeader h;
  int rc = build_blob(T, coeffs, &blob, &h);
  if (rc) return rc;
  const Net t = make_net(blob.data());
  std::vector<double> ws((size_t)h.lane_doubles * WS_LANES, 0.0);
  WS w = make_ws(t, ws.data());
  BurnParams P;
  std::memset(&P, 0, sizeof(P));
  P.Z = Z; P.Y0 = Y0; P.T9_0 = T9_0; P.rho = rho; P.zeta_zone = zeta;
  P.t_end = t_end; P.rtol = rtol; P.atol = atol;
  P.Y = Y; P.T9 = T9; P.E = E; P.counters = cnt; P.status = status;
  P.max_attempts = 500000;
  for (long long z = 0; z < Z; ++z) {
    Zone s;
    s.z = z;
    bool done = zone_init(t, s, w, P);
    while (!done) done = zone_attempt(t, s, w, P);
    zone_finish(t, s, w, P);
  }
  return 0;
}
