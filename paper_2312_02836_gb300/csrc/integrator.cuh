// integrator.cuh -- the per-zone BDF/Newton integrator, independent of how
// the network is evaluated.
//
// Every function here is a template over two types:
//   NT  the network: sizes n (state), N (species), R (reactions), flags sh
//       (self-heating), hasE (energy), inv_n = 1/n;
//   WT  one lane's work arrays x, xp, psi, d, f, iw, tmp, f0 (length n),
//       k, g, rr (length R), lu (LU slots) and the history xh [HMAX*n],
//       eh [HMAX], th [HMAX]; each is indexable with operator[].
// and calls the network-specific operations by unqualified name, so that the
// overloads for NT are found at instantiation:
//   eval_rates(t, s, w, p, T9, with_g)  k_r (and g_r = d ln lambda_r/dT9),
//                                     p = t_powers(T9, with_g)
//   save_ref_rates(t, w)              kp_r = k_r (the reference rates)
//   tab_zone(t, s, x0)                the zone's density cell of the rate
//                                     tables, from its initial composition
//   eval_rates_near(t, s, w, T9, ref, T9ref)  k_r from kp_r (rate_near)
//   eval_terms(t, w, v)               rr_r = k_r prod Y of the reactants
//   eval_f(t, w, v, out)              out = f(v) from rr
//   eval_edot(t, w)                   sum_r Q_r rr_r
//   assemble_M(t, w, v, alpha0, h)    lu = alpha0 I - h J(v)
//   factor_M(t, w)                    static-pivot LU of lu in place
//   solve_M(t, w, v)                  v <- M^-1 v with the factored lu
// Three network types exist: the generic one (device.cuh) walks a compiled
// network held in memory; the specialised one is generated per network as
// straight-line code with every index a constant and compiled at run time.
// Both run one zone per lane and perform the same floating-point operations
// in the same order, so they give the same bits.  The cooperative one
// (coop.cuh) runs one zone per team of W threads, a warp or a block of two
// or four warps: its vector loops are spread over the team (vbeg/vstep),
// its sums are team reductions (vsum) and its phases are separated by the
// team's barriers (vsync); every thread holds the same copy of the zone's
// scalars, so control flow stays uniform.  For the one-zone-per-lane types
// these helpers reduce to the plain loops and do nothing.
//
// This header is also compiled by the run-time compiler, so it includes no
// system header.
#pragma once
#include "blob.h"
#include "expf64.cuh"
#include "../../include/netburn.h"

#ifndef NB_HD
#define NB_HD __device__
#endif

// Loops over the state vector are unrolled in the specialised kernel (their
// trip counts are constants there, and unrolling keeps the work arrays in
// registers); the generic kernel leaves them as loops.
#ifdef NB_SPECIALIZED
#define NB_UNROLL _Pragma("unroll")
#else
#define NB_UNROLL
#endif

namespace nb {

// Network types that spread one zone over the lanes of a warp specialise this
template <class NT>
struct is_coop {
  static constexpr bool value = false;
};

// first index and stride of this thread's share of a vector loop
template <class NT>
NB_HD __forceinline__ constexpr int vbeg(const NT& t) {
  if constexpr (is_coop<NT>::value) return t.lane; else return 0;
}
template <class NT>
NB_HD __forceinline__ constexpr int vstep(const NT&) {
  if constexpr (is_coop<NT>::value) return NT::width; else return 1;
}
// sum over the zone's threads of their partial sums (the same bits in all)
template <class NT>
NB_HD __forceinline__ double vsum(const NT& t, double x) {
  if constexpr (is_coop<NT>::value) return t.sum(x); else return x;
}
template <class NT>
NB_HD __forceinline__ bool vall(const NT& t, bool b) {
  if constexpr (is_coop<NT>::value) return t.all(b); else return b;
}
// make the zone's vector writes visible to all its threads
template <class NT>
NB_HD __forceinline__ void vsync(const NT& t) {
  if constexpr (is_coop<NT>::value) t.sync();
}
// the one thread that writes the zone's scalar outputs
template <class NT>
NB_HD __forceinline__ bool vlead(const NT& t) {
  if constexpr (is_coop<NT>::value) return t.lane == 0; else return true;
}

// lane-strided view of one per-lane array
struct LV {
  double* p;
  NB_HD __forceinline__ double& operator[](int i) const {
    return p[i * WS_LANES];
  }
};

// Tape written by a burn that will be differentiated: the schedule of every
// accepted step, and the states only at checkpoints.  Record s = 0 is the
// initial point, record s >= 1 accepted step s.  A state is kept for s = 0
// and for the last min(stride, HMAX) steps of every block of `stride` steps,
// which is the history window the reverse sweep restarts a segment from
// (tape_state_slot); stride 1 keeps every state.
struct TapeDev {
  double* sched;     // [Z, cap, 2]: t_s, h_s (the step size the forward used)
  int8_t* ord;       // [Z, cap] BDF order of step s (0 for s = 0)
  double* states;    // [Z, scap, n + 1]: x_s, E_s of the kept records
  int32_t* steps;    // [Z] records written (accepted steps + 1)
  int32_t* zstat;    // [Z] status the zone finished with
  double* rho;       // [Z]
  double* T9f;       // [Z] fixed temperature (or initial T9)
  double* scr;       // [Z] screening factor sqrt(rho zeta) 10^-4.5 of the zone
  int32_t cap, scap, stride;
};

// slot of record s's state on the tape, or -1 when it is not kept (host
// code reads tapes too)
__host__ __device__ __forceinline__ int tape_state_slot(int s, int stride) {
  if (s == 0) return 0;
  const int m = stride < HMAX ? stride : HMAX;
  const int b = (s - 1) / stride, p = (s - 1) - b * stride;
  return p >= stride - m ? 1 + b * m + (p - (stride - m)) : -1;
}

struct BurnParams {
  const unsigned char* blob;
  int blob_bytes, blob_in_smem;
  long long Z;
  const double *Y0, *T9_0, *rho;
  double t_end, rtol, atol;
  const double* lnm;
  int lnm_per_zone;
  double *Y, *T9, *E;
  int32_t *counters, *status;
  int max_attempts;
  double* ws;                 // per-lane workspace, lane_doubles * 32 per warp
  unsigned long long* queue;  // zone counter of the persistent kernel
  TapeDev tape;
  int use_tape;
  int smem_warps;             // warps per block with hot arrays in shared memory
  unsigned long long budget_ns;  // watchdog budget per block, 0 = none
  const int32_t* order;       // claim order (zone index per claim), or null
  const double* t_end_zone;   // [Z] per-zone end time (operator split), or null
  const double* zeta_zone;    // [Z] plasma parameter for screening, or null
};

// Register state of the zone a lane is integrating.
struct Zone {
  long long z;
  double t, h, E, T9f, rho, rho2, tend;
  double scr;                 // sqrt(rho zeta) 10^-4.5: H_r = s_r scr T9^(-3/2)
  int tab_i;                  // density cell of the rate tables (log10 rho Ye)
  double tab_u;               // and the weight within it
  const double* lnm;
  int k, nh, hh, nconsec, nfail, status;
  int c_acc, c_rej_err, c_rej_newton, c_newton, c_jac, c_rhs, c_teval, c_edot, c_ordsum;
};

NB_HD __forceinline__ int hslot(const Zone& s, int j) {
  int v = s.hh + j;
  return v >= HMAX ? v - HMAX : v;
}

// Finite and nonzero, decided on the exponent bits with integer ops (FP64
// compares would occupy the FP64 pipe).
NB_HD __forceinline__ long long dbits(double v) {
#ifdef __CUDA_ARCH__
  return __double_as_longlong(v);
#else
  long long b;
  memcpy(&b, &v, sizeof(b));
  return b;
#endif
}
NB_HD __forceinline__ bool finite_nonzero(double v) {
  const long long b = dbits(v) & 0x7fffffffffffffffLL;
  return b != 0 && b < 0x7ff0000000000000LL;
}
NB_HD __forceinline__ bool finite_bits(double v) {
  return (dbits(v) & 0x7fffffffffffffffLL) < 0x7ff0000000000000LL;
}

// Pivot guard of the static-pivot LU: pivot u_kk, finite and nonzero, has
// not lost more than 40 bits to cancellation against the diagonal a_kk of M
// before elimination (|u_kk| >= 2^-40 |a_kk|, on the exponents).  A static
// pivot order cannot swap rows, so a pivot eaten by cancellation rejects the
// attempt; the step then shrinks, and M = alpha0 I - h J tends to alpha0 I,
// whose static pivots are safe.
NB_HD __forceinline__ bool pivot_kept(double u, double a) {
  const long long eu = (dbits(u) >> 52) & 0x7ff, ea = (dbits(a) >> 52) & 0x7ff;
  return finite_nonzero(u) && eu + 40 >= ea;
}

// Reciprocals by Newton-Raphson iteration, y <- y + y (1 - a y), which
// squares the relative error of y, from the approximate reciprocal
// instruction (rcp.approx.ftz.f64) as the seed: two FMAs a step instead of a
// full division.  Arguments whose exponent is 0 or >= 2^1021 (0, subnormal,
// huge, inf, NaN) take the division.
NB_HD __forceinline__ bool recip_plain(double a) {
  const long long e = (dbits(a) >> 52) & 0x7ff;
  return e == 0 || e >= 0x7fd;
}
// One step: about 2^-40 relative (the seed has about 20 good bits).  For
// the error weights 1/(atol + rtol |x|), which only scale the norms the step
// control compares with 1e-3 and 1.
NB_HD __forceinline__ double recip1(double a) {
#ifdef __CUDA_ARCH__
  if (recip_plain(a)) return 1.0 / a;
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(a));
  return fma(y, fma(-a, y, 1.0), y);
#else
  return 1.0 / a;
#endif
}
// Two steps: about 2^-80 before rounding, so within an ulp of 1/a (correctly
// rounded on every one of 250,000 test inputs).  For the LU pivots.
NB_HD __forceinline__ double recip2(double a) {
#ifdef __CUDA_ARCH__
  if (recip_plain(a)) return 1.0 / a;
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(a));
  y = fma(y, fma(-a, y, 1.0), y);
  return fma(y, fma(-a, y, 1.0), y);
#else
  return 1.0 / a;
#endif
}

// ---------------------------------------------------------------- model
// pieces both network types share, so that their arithmetic is one text

// Powers of T9 in the rate fit (and their T9-derivative factors)
struct TPow {
  double t13, iT, t23, it13, T53, lnT, d1, d2, d3, d5;
  double hz, hzd;   // screening: scr T9^(-3/2) and its T9-derivative factor
};

// scr: the zone's screening factor (0 without screening)
NB_HD __forceinline__ TPow t_powers(double T9, bool with_g, double scr) {
  TPow p;
  p.t13 = cbrt(T9);
  p.iT = 1.0 / T9;
  p.t23 = p.t13 * p.t13;
  p.it13 = p.t23 * p.iT;          // T9^(-1/3) without a second division
  p.T53 = T9 * p.t23;
  p.lnT = log(T9);
  p.d1 = p.d2 = p.d3 = p.d5 = 0.0;
  if (with_g) {
    p.d1 = -p.iT * p.iT;
    p.d2 = (-1.0 / 3.0) * p.iT * p.it13;
    p.d3 = (1.0 / 3.0) * p.it13 * p.it13;
    p.d5 = (5.0 / 3.0) * p.t23;
  }
  // weak screening H_r = s_r sqrt(rho zeta) T6^(-3/2) = s_r hz, T6 = 1e3 T9;
  // dH_r/dT9 = -1.5 H_r / T9 = s_r hzd
  p.hz = p.hzd = 0.0;
  if (scr != 0.0) {
    p.hz = scr * (p.iT * sqrt(p.iT));
    if (with_g) p.hzd = -1.5 * p.hz * p.iT;
  }
  return p;
}

// exponent a0 + a1/T9 + a2 T9^-1/3 + a3 T9^1/3 + a4 T9 + a5 T9^5/3 + a6 ln T9
// as two independent partial sums
NB_HD __forceinline__ double rate_exponent(double a0, double a1, double a2, double a3,
                                           double a4, double a5, double a6,
                                           const TPow& p, double T9) {
  double e1 = fma(a1, p.iT, a0);
  double e2 = a4 * T9;
  e1 = fma(a2, p.it13, e1);
  e2 = fma(a5, p.T53, e2);
  e1 = fma(a3, p.t13, e1);
  e2 = fma(a6, p.lnT, e2);
  return e1 + e2;
}

// d ln lambda / dT9 of the same fit
NB_HD __forceinline__ double rate_dlog(double a1, double a2, double a3, double a4,
                                       double a5, double a6, const TPow& p) {
  double g1 = fma(a1, p.d1, a4);
  double g2 = a5 * p.d5;
  g1 = fma(a2, p.d2, g1);
  g2 = fma(a6, p.iT, g2);
  g1 = fma(a3, p.d3, g1);
  return g1 + g2;
}

// Tabulated rates: ln lambda bilinear in (log10 rho Ye, T9) on a rectilinear
// grid, clamped to its edges.  The density cell is the zone's (Ye from its
// initial composition, held over the burn); the temperature cell is found
// once per rate evaluation.

// cell c and weight w in [0, 1] of v on increasing nodes x[0..m), clamped
NB_HD __forceinline__ void grid_cell(const double* x, int m, double v, int& c, double& w) {
  if (!(v > x[0])) { c = 0; w = 0.0; return; }
  if (v >= x[m - 1]) { c = m - 2; w = 1.0; return; }
  int i = 0;
  while (v > x[i + 1]) ++i;       // stops at i <= m - 2, since v < x[m-1]
  c = i;
  w = (v - x[i]) / (x[i + 1] - x[i]);
}

struct TCell {
  int j;             // temperature cell
  double v, dt;      // weight within it, its width
  bool inside;       // strictly inside the grid (else the T9 slope is 0)
};

NB_HD __forceinline__ TCell t_cell(const double* t9, int nt, double T9) {
  TCell c;
  grid_cell(t9, nt, T9, c.j, c.v);
  c.dt = t9[c.j + 1] - t9[c.j];
  c.inside = T9 > t9[0] && T9 < t9[nt - 1];
  return c;
}

// the zone's density cell from Ye = sum Z_i Y_i (accumulated by the caller)
NB_HD __forceinline__ void density_cell(const double* dens, int nd, double rho, double ye,
                                        Zone& s) {
  grid_cell(dens, nd, log10(rho * ye), s.tab_i, s.tab_u);
}

// ln lambda of one table L [nd, nt] and its T9-derivative
NB_HD __forceinline__ double table_lnl(const double* L, int nt, const Zone& s, const TCell& c,
                                       double* dl) {
  const int a = s.tab_i * nt + c.j, b = a + nt;
  const double u = s.tab_u;
  const double at_j = (1.0 - u) * L[a] + u * L[b];
  const double at_j1 = (1.0 - u) * L[a + 1] + u * L[b + 1];
  *dl = c.inside ? (at_j1 - at_j) / c.dt : 0.0;
  return (1.0 - c.v) * at_j + c.v * at_j1;
}

// Effective (alpha,p)(p,gamma) rate from the exponents of its four channels
// (the multiplier already added to the direct and (a,p) ones):
// lambda = l_ag + l_ap frac, frac = l_pg / (l_pg + l_pa), here written
// 1 / (1 + exp(e_pa - e_pg)) so that it stays defined when both proton
// channels underflow.
struct APRate {
  double lam, l_ag, via_p, frac;
};

NB_HD __forceinline__ APRate ap_rate(double e_ag, double e_ap, double e_pg, double e_pa) {
  APRate a;
  a.l_ag = exp_tang(e_ag);
  a.frac = 1.0 / (1.0 + exp_tang(e_pa - e_pg));
  a.via_p = exp_tang(e_ap) * a.frac;
  a.lam = a.l_ag + a.via_p;
  return a;
}

// d ln lambda / dT9 from the channels' g = d ln lambda_c / dT9, with
// d frac / dT9 = frac (1 - frac) (g_pg - g_pa)
NB_HD __forceinline__ double ap_dlog(const APRate& a, double g_ag, double g_ap, double g_pg,
                                     double g_pa) {
  if (!finite_nonzero(a.lam)) return g_ag;
  return (a.l_ag * g_ag + a.via_p * (g_ap + (1.0 - a.frac) * (g_pg - g_pa))) / a.lam;
}

// Rates near a reference temperature.  Within one step attempt T9 moves
// only slightly from the predictor's value T9ref, where every k_r was
// evaluated in full.  Then k_r(T9) = k_r(T9ref) exp(de_r) with
// de_r = e_r(T9) - e_r(T9ref) = sum_{i>=1} a_i (phi_i(T9) - phi_i(T9ref));
// the constant part of the exponent (a0, the multiplier) and the factors
// rho^(n_r-1) scale_r cancel.  For |de| <= 2^-10, exp(de) - 1 comes from its
// Taylor polynomial of degree 4 (truncation x^5/120 < 2^-56 relative), and
// k = kref + kref (exp(de) - 1).  The exponent's absolute rounding error is
// the same as when it is formed whole, so the rates are as accurate as the
// full evaluation's.  A larger de takes the full evaluation.
struct DPhi {
  double d1, d2, d3, d4, d5, d6, d7;   // d7: change of the screening term hz
};

NB_HD __forceinline__ DPhi delta_phi(const TPow& p, const TPow& r, double T9, double T9r) {
  DPhi d;
  d.d1 = p.iT - r.iT;
  d.d2 = p.it13 - r.it13;
  d.d3 = p.t13 - r.t13;
  d.d4 = T9 - T9r;
  d.d5 = p.T53 - r.T53;
  d.d6 = p.lnT - r.lnT;
  d.d7 = p.hz - r.hz;
  return d;
}

// The same differences from the relative change x = (T9 - T9r)/T9r when
// |x| <= 2^-14, the case of every Newton iteration of an attempt: the
// binomial and logarithm series of (1+x)^a - 1 and ln(1+x) to x^4, whose
// first omitted term is below 2^-55 of the kept ones (more accurate than the
// difference of the two rounded powers), with no cbrt, log or division.
// False, and d untouched, for a larger change.
NB_HD __forceinline__ double binom4(double x, double c1, double c2, double c3, double c4) {
  return x * fma(x, fma(x, fma(x, c4, c3), c2), c1);
}
NB_HD __forceinline__ bool delta_phi_series(const TPow& r, double T9, double T9r, DPhi& d) {
  const double dT = T9 - T9r;
  const double x = dT * r.iT;
  if ((dbits(x) & 0x7fffffffffffffffLL) > 0x3f10000000000000LL) return false;
  d.d1 = r.iT * binom4(x, -1.0, 1.0, -1.0, 1.0);
  d.d2 = r.it13 * binom4(x, -1.0 / 3.0, 2.0 / 9.0, -14.0 / 81.0, 35.0 / 243.0);
  d.d3 = r.t13 * binom4(x, 1.0 / 3.0, -1.0 / 9.0, 5.0 / 81.0, -10.0 / 243.0);
  d.d4 = dT;
  d.d5 = r.T53 * binom4(x, 5.0 / 3.0, 5.0 / 9.0, -5.0 / 81.0, 5.0 / 243.0);
  d.d6 = binom4(x, 1.0, -0.5, 1.0 / 3.0, -0.25);
  d.d7 = r.hz * binom4(x, -1.5, 15.0 / 8.0, -35.0 / 16.0, 315.0 / 128.0);
  return true;
}

NB_HD __forceinline__ double rate_delta(double a1, double a2, double a3, double a4,
                                        double a5, double a6, const DPhi& d) {
  double e1 = a1 * d.d1;
  double e2 = a4 * d.d4;
  e1 = fma(a2, d.d2, e1);
  e2 = fma(a5, d.d5, e2);
  e1 = fma(a3, d.d3, e1);
  e2 = fma(a6, d.d6, e2);
  return e1 + e2;
}

// |de| <= 2^-10 (and finite), decided on the bits
NB_HD __forceinline__ bool small_delta(double de) {
  return (dbits(de) & 0x7fffffffffffffffLL) <= 0x3f50000000000000LL;
}

NB_HD __forceinline__ double rate_near(double kref, double de) {
  double q = fma(de, 1.0 / 24.0, 1.0 / 6.0);
  q = fma(q, de, 0.5);
  q = fma(q, de, 1.0);
  return fma(kref, q * de, kref);
}

// c_v = 1.5 sum_i Y_i + 1e-3 T9^3 (two interleaved partial sums)
template <class NT, class V>
NB_HD __forceinline__ double heat_capacity(const NT& t, const V& v) {
  if constexpr (is_coop<NT>::value) {
    double sy = 0.0;
    for (int i = vbeg(t); i < t.N; i += vstep(t)) sy += v[i];
    sy = vsum(t, sy);
    const double T9 = v[t.N];
    return 1.5 * sy + 1e-3 * T9 * T9 * T9;
  }
  double s0 = 0.0, s1 = 0.0;
  int i = 0;
  NB_UNROLL
  for (; i + 1 < t.N; i += 2) {
    s0 += v[i];
    s1 += v[i + 1];
  }
  if (i < t.N) s0 += v[i];
  const double T9 = v[t.N];
  return 1.5 * (s0 + s1) + 1e-3 * T9 * T9 * T9;
}

// Rows of the T9 equation in M: with S_j = sum_r Q_r dR_r/dx_j,
// dfT/dY_j = S_j a1 + b1, dfT/dT9 = S_T a1 + b2
struct TRow {
  double a1, b1, b2;
};

NB_HD __forceinline__ TRow t_row(double ed, double cv, double T9) {
  TRow r;
  const double icv = recip2(cv);
  const double fT = ed * icv;
  r.a1 = icv;
  r.b1 = -fT * 1.5 * icv;
  r.b2 = -fT * (3e-3 * T9 * T9) * icv;
  return r;
}

// ---------------------------------------------------------------- integrator

// ||v||^2 = mean (v_i * iw_i)^2, two interleaved partial sums (the tests
// compare squares, which spares a square root per norm)
template <class NT, class WT, class V>
NB_HD __forceinline__ double wnorm2(const NT& t, const WT& w, const V& v) {
  if constexpr (is_coop<NT>::value) {
    double sq = 0.0;
    for (int i = vbeg(t); i < t.n; i += vstep(t)) {
      const double q = v[i] * w.iw[i];
      sq = fma(q, q, sq);
    }
    return vsum(t, sq) * t.inv_n;
  }
  double s0 = 0.0, s1 = 0.0;
  int i = 0;
  NB_UNROLL
  for (; i + 1 < t.n; i += 2) {
    const double q0 = v[i] * w.iw[i], q1 = v[i + 1] * w.iw[i + 1];
    s0 = fma(q0, q0, s0);
    s1 = fma(q1, q1, s1);
  }
  if (i < t.n) {
    const double q = v[i] * w.iw[i];
    s0 = fma(q, q, s0);
  }
  return (s0 + s1) * t.inv_n;
}

// out_i = sum_{j<cnt} c_j xh[base_j + i], summed in increasing j.  Loops over
// the history points run to the lane's own count (a warp runs as many
// iterations as its highest-order lane), not to the maximum order with the
// extra terms predicated off.  The specialised build accumulates in registers
// over that loop; the generic one loops over i outside.  Same operations in
// the same order either way.
template <class NT, class WT, class V>
NB_HD __forceinline__ void hist_combine(const NT& t, const WT& w, int cnt, const double* c,
                                        const int* base, V&& out) {
#ifdef NB_SPECIALIZED
  double acc[NT::n];
  NB_UNROLL
  for (int i = 0; i < NT::n; ++i) acc[i] = 0.0;
#pragma unroll 1
  for (int j = 0; j < cnt; ++j) {
    const double cj = c[j];
    const int b = base[j];
    NB_UNROLL
    for (int i = 0; i < NT::n; ++i) acc[i] = fma(cj, w.xh[b + i], acc[i]);
  }
  NB_UNROLL
  for (int i = 0; i < NT::n; ++i) out[i] = acc[i];
#else
  for (int i = vbeg(t); i < t.n; i += vstep(t)) {
    double acc = 0.0;
    for (int j = 0; j < cnt; ++j) acc = fma(c[j], w.xh[base[j] + i], acc);
    out[i] = acc;
  }
#endif
}

// Lagrange weights at time tt of the q+1 newest history points starting at
// history index j0 (0 = newest): lw[j] = prod_{m!=j} (tt - t_m)/(t_j - t_m)
template <class WT>
NB_HD __forceinline__ void lagrange_weights(const Zone& s, const WT& w, int j0,
                                            int q, double tt, double* lw) {
  double tp[KMAX + 2], e[KMAX + 2];
#pragma unroll 1
  for (int j = 0; j <= q; ++j) {
    tp[j] = w.th[hslot(s, j0 + j)];
    e[j] = tt - tp[j];
  }
#pragma unroll 1
  for (int j = 0; j <= q; ++j) {
    double num = 1.0, den = 1.0;
#pragma unroll 1
    for (int m = 0; m <= q; ++m) {
      if (m != j) {
        num *= e[m];
        den *= tp[j] - tp[m];
      }
    }
    lw[j] = num / den;
  }
}

// out = value at tt of the degree-q polynomial through history j0..j0+q
template <class NT, class WT, class V>
NB_HD __forceinline__ void extrapolate(const NT& t, const Zone& s, const WT& w, int j0,
                                       int q, double tt, V&& out) {
  double lw[KMAX + 2];
  lagrange_weights(s, w, j0, q, tt, lw);
  int base[KMAX + 2];
#pragma unroll 1
  for (int j = 0; j <= q; ++j) base[j] = hslot(s, j0 + j) * t.n;
  hist_combine(t, w, q + 1, lw, base, out);
}

// 0.9 E^(-1/(q+1)) from E^2, as 0.9 exp(-ln(E^2) / (2(q+1))): the factor only
// sets the next step size, so the few-ulp exp/log route replaces the library
// pow (which computes in extended precision, several times the FP64 work)
NB_HD __forceinline__ double err_factor(double E2, int q) {
  return 0.9 * exp_tang(log(E2) * (-0.5 / (q + 1)));
}

NB_HD __forceinline__ double step_factor(double E2, int q) {
  if (!(E2 > 0.0)) return 5.0;
  return err_factor(E2, q);
}

// E_q^2 after acceptance: newest point vs extrapolation through the q+1 older
template <class NT, class WT>
NB_HD __forceinline__ double order_estimate(const NT& t, const Zone& s, WT& w, int q,
                                            double h) {
  extrapolate(t, s, w, 1, q, w.th[hslot(s, 0)], w.tmp);
  const double c = h / (w.th[hslot(s, 0)] - w.th[hslot(s, q + 1)]);
  const int b0 = hslot(s, 0) * t.n;
  double acc = 0.0;
  NB_UNROLL
  for (int i = vbeg(t); i < t.n; i += vstep(t)) {
    const double v = c * (w.xh[b0 + i] - w.tmp[i]) * w.iw[i];
    acc = fma(v, v, acc);
  }
  return vsum(t, acc) * t.inv_n;   // E_q^2
}

// Record an accepted point (time, step, order; state and energy when the
// record is a kept one); false when the zone's tape is full.
template <class NT, class V>
NB_HD __forceinline__ bool tape_record(const NT& t, const BurnParams& P, const Zone& s,
                                       const V& x, double h, int ord) {
  if (!P.use_tape) return true;
  int32_t* cnt = P.tape.steps + s.z;
  const int idx = *cnt;
  vsync(t);   // every thread has read the count before it moves on
  if (idx >= P.tape.cap) return false;
  const unsigned long long r = (unsigned long long)s.z * P.tape.cap + idx;
  const int slot = tape_state_slot(idx, P.tape.stride);
  if (slot >= 0) {
    double* rec = P.tape.states + ((unsigned long long)s.z * P.tape.scap + slot) * (t.n + 1);
    NB_UNROLL
    for (int i = vbeg(t); i < t.n; i += vstep(t)) rec[i] = x[i];
    if (vlead(t)) rec[t.n] = s.E;
  }
  if (vlead(t)) {
    P.tape.sched[2 * r] = s.t;
    P.tape.sched[2 * r + 1] = h;
    P.tape.ord[r] = (int8_t)ord;
    *cnt = idx + 1;
  }
  return true;
}

// alpha_j = h l_j'(tau_0), Lagrange basis on tau_0..tau_kk (unused j -> 0)
NB_HD __forceinline__ void bdf_alpha(int kk, const double* tau, double h, double* alpha) {
  double acc = 0.0;
#pragma unroll 1
  for (int m = 1; m <= kk; ++m) acc += 1.0 / (tau[0] - tau[m]);
  alpha[0] = h * acc;
#pragma unroll 1
  for (int j = 1; j <= kk; ++j) {
    double num = 1.0, den = 1.0;
#pragma unroll 1
    for (int m = 0; m <= kk; ++m) {
      if (m != j) {
        if (m != 0) num *= tau[0] - tau[m];
        den *= tau[j] - tau[m];
      }
    }
    alpha[j] = h * num / den;
  }
#pragma unroll
  for (int j = 1; j <= KMAX; ++j)
    if (j > kk) alpha[j] = 0.0;
}

// ---------------------------------------------------------------- zone start

// Load zone s.z, evaluate f(x0) and the starting step.  Returns true when the
// zone is already finished (bad input or t_end == 0).
template <class NT, class WT>
NB_HD __forceinline__ bool zone_init(const NT& t, Zone& s, WT& w, const BurnParams& P) {
  const long long z = s.z;
  const int n = t.n, N = t.N;
  s.t = 0.0; s.E = 0.0; s.k = 1; s.nh = 1; s.hh = 0; s.nconsec = 0; s.nfail = 0;
  s.status = NB_Z_OK;
  s.c_acc = s.c_rej_err = s.c_rej_newton = s.c_newton = 0;
  s.c_jac = s.c_rhs = s.c_teval = s.c_edot = s.c_ordsum = 0;
  s.T9f = P.T9_0[z];
  s.rho = P.rho[z];
  s.rho2 = s.rho * s.rho;
  const double zeta = P.zeta_zone ? P.zeta_zone[z] : 0.0;
  s.scr = zeta > 0.0 ? sqrt(s.rho * zeta) * 3.1622776601683794e-05 : 0.0;   // 10^-4.5
  s.lnm = P.lnm ? (P.lnm_per_zone ? P.lnm + (unsigned long long)z * t.R : P.lnm) : nullptr;
  s.tend = P.t_end_zone ? P.t_end_zone[z] : P.t_end;
  auto& x0 = w.xh;  // history slot 0
  bool fin = finite_bits(s.T9f) && s.T9f > 0.0 && finite_bits(s.rho) &&
             finite_bits(s.tend) && s.tend >= 0.0 && finite_bits(zeta) && zeta >= 0.0;
  NB_UNROLL
  for (int i = vbeg(t); i < N; i += vstep(t)) {
    const double y = P.Y0[(unsigned long long)z * N + i];
    x0[i] = y;
    fin = fin && finite_bits(y);
  }
  if (t.sh && vlead(t)) x0[N] = s.T9f;
  vsync(t);
  tab_zone(t, s, x0);
  w.th[0] = 0.0;
  w.eh[0] = 0.0;
  if (P.use_tape) {
    P.tape.steps[z] = 0;
    P.tape.rho[z] = s.rho;
    P.tape.T9f[z] = s.T9f;
    P.tape.scr[z] = s.scr;
    tape_record(t, P, s, x0, 0.0, 0);
  }
  eval_rates(t, s, w, t_powers(s.T9f, false, s.scr), s.T9f, false);
  s.c_teval++;
  eval_terms(t, w, x0);
  eval_f(t, w, x0, w.f0);
  s.c_rhs++;
  NB_UNROLL
  for (int r = vbeg(t); r < t.R; r += vstep(t)) fin = fin && finite_bits(w.k[r]);
  NB_UNROLL
  for (int i = vbeg(t); i < n; i += vstep(t)) fin = fin && finite_bits(w.f0[i]);
  fin = vall(t, fin);
  if (!fin) { s.status = NB_Z_NONFINITE; return true; }
  if (!(s.tend > 0.0)) return true;
  // starting step: Hairer-Norsett-Wanner I, Sec. II.4, p = 1
  double s0 = 0.0, s1 = 0.0;
  NB_UNROLL
  for (int i = vbeg(t); i < n; i += vstep(t)) {
    const double iw = recip1(P.atol + P.rtol * fabs(x0[i]));
    w.iw[i] = iw;
    const double a = x0[i] * iw, b = w.f0[i] * iw;
    s0 = fma(a, a, s0);
    s1 = fma(b, b, s1);
  }
  s0 = vsum(t, s0);
  s1 = vsum(t, s1);
  const double d0 = sqrt(s0 / n), d1 = sqrt(s1 / n);
  double hp = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
  if (hp > s.tend) hp = s.tend;
  NB_UNROLL
  for (int i = vbeg(t); i < n; i += vstep(t)) w.x[i] = fma(hp, w.f0[i], x0[i]);
  vsync(t);
  if (t.sh) {
    const double T9 = w.x[N];
    eval_rates(t, s, w, t_powers(T9, false, s.scr), T9, false);
    s.c_teval++;
  }
  eval_terms(t, w, w.x);
  eval_f(t, w, w.x, w.f);
  s.c_rhs++;
  double s2 = 0.0;
  const double ihp = 1.0 / hp;
  NB_UNROLL
  for (int i = vbeg(t); i < n; i += vstep(t)) {
    const double q = (w.f[i] - w.f0[i]) * ihp * w.iw[i];
    s2 = fma(q, q, s2);
  }
  s2 = vsum(t, s2);
  const double d2 = sqrt(s2 / n);
  const double dm = fmax(d1, d2);
  const double h1 = dm <= 1e-15 ? fmax(1e-6, hp * 1e-3) : sqrt(0.01 / dm);
  double h = fmin(100.0 * hp, h1);
  if (h > s.tend) h = s.tend;
  if (!(h >= 1e-30 * s.tend)) h = 1e-30 * s.tend;
  s.h = h;
  return false;
}

// ---------------------------------------------------------------- one attempt

// The computation of one step attempt from t_n = s.t to t_new with step h at
// order kk: BDF coefficients, history sum, weights from x_n, predictor,
// Jacobian and LU at the predictor, modified Newton.  Leaves the solution in
// w.x and the predictor in w.xp, alpha_0..alpha_kk in alpha and, with
// self-heating, the reference temperature of the rates in Tref (powers
// pref); returns true when Newton converged.  The forward burn and the
// adjoint's recomputation of checkpointed segments both run it, so that they
// produce the same bits.
template <class NT, class WT>
NB_HD __forceinline__ bool attempt_solve(const NT& t, Zone& s, WT& w, double atol, double rtol,
                                         double h, double t_new, int kk, double* alpha,
                                         TPow& pref, double& Tref, bool& lu_ok) {
  const int n = t.n, N = t.N;
  vsync(t);   // the history written by the last accepted step
  // alpha_j = h l_j'(t_new) over t_new, t_n, .., t_{n+1-kk}
  double tau[KMAX + 1];
  tau[0] = t_new;
#pragma unroll 1
  for (int j = 1; j <= kk; ++j) tau[j] = w.th[hslot(s, j - 1)];
  bdf_alpha(kk, tau, h, alpha);
  // psi = sum_{j>=1} alpha_j x_{n+1-j}; weights from x_n
  {
    int base[KMAX];
#pragma unroll 1
    for (int j = 0; j < kk; ++j) base[j] = hslot(s, j) * n;
    hist_combine(t, w, kk, alpha + 1, base, w.psi);
    const int b0 = hslot(s, 0) * n;
    NB_UNROLL
    for (int i = vbeg(t); i < n; i += vstep(t))
      w.iw[i] = recip1(atol + rtol * fabs(w.xh[b0 + i]));
  }
  // predictor
  if (s.nh >= kk + 1) extrapolate(t, s, w, 0, kk, t_new, w.xp);
  else if (s.nh >= 2) extrapolate(t, s, w, 0, s.nh - 1, t_new, w.xp);
  else {
    const int b0 = hslot(s, 0) * n;
    NB_UNROLL
    for (int i = vbeg(t); i < n; i += vstep(t)) w.xp[i] = fma(h, w.f0[i], w.xh[b0 + i]);
  }
  NB_UNROLL
  for (int i = vbeg(t); i < n; i += vstep(t)) w.x[i] = w.xp[i];
  vsync(t);
  // Jacobian at the predictor, M, LU; with self-heating the predictor's
  // temperature is the attempt's reference for the rates
  Tref = 0.0;
  if (t.sh) {
    Tref = w.x[N];
    pref = t_powers(Tref, true, s.scr);
    eval_rates(t, s, w, pref, Tref, true);
    save_ref_rates(t, w);
    s.c_teval++;
  }
  eval_terms(t, w, w.x);
  assemble_M(t, w, w.x, alpha[0], h);
  s.c_jac++;
  bool ok = factor_M(t, w);
  lu_ok = ok;
  // modified Newton
  bool converged = false;
  double nrm_prev = 0.0;
  for (int m = 0; ok && m < 4; ++m) {
    if (m > 0) {
      if (t.sh) { eval_rates_near(t, s, w, w.x[N], pref, Tref); s.c_teval++; }
      eval_terms(t, w, w.x);
    }
    eval_f(t, w, w.x, w.f);
    s.c_rhs++;
    NB_UNROLL
    for (int i = vbeg(t); i < n; i += vstep(t))
      w.d[i] = -(fma(alpha[0], w.x[i], w.psi[i]) - h * w.f[i]);
    solve_M(t, w, w.d);
    NB_UNROLL
    for (int i = vbeg(t); i < n; i += vstep(t)) w.x[i] += w.d[i];
    vsync(t);
    s.c_newton++;
    const double nrm2 = wnorm2(t, w, w.d);
    if (!finite_bits(nrm2)) { ok = false; break; }
    if (nrm2 <= 1e-6) { converged = true; break; }          // ||d|| <= 1e-3
    if (m > 0) {
      if (nrm2 > 0.81 * nrm_prev) { ok = false; break; }     // theta > 0.9
      const double theta = sqrt(nrm2 / nrm_prev);
      if (theta / (1.0 - theta) * sqrt(nrm2) <= 1e-3) { converged = true; break; }
    }
    nrm_prev = nrm2;
  }
  return converged;
}

// One step attempt.  Returns true when the zone is finished.
template <class NT, class WT>
NB_HD __forceinline__ bool zone_attempt(const NT& t, Zone& s, WT& w, const BurnParams& P) {
  const int n = t.n, N = t.N;
  if (s.c_acc + s.c_rej_err + s.c_rej_newton >= P.max_attempts) {
    s.status = NB_Z_MAX_STEPS;
    return true;
  }
  double h = s.h;
  if (h < 1e-30 * s.tend || h < 1e-14 * s.t) {
    s.status = NB_Z_DT_UNDERFLOW;
    return true;
  }
  double t_new;
  if (s.t + h >= s.tend) { h = s.tend - s.t; t_new = s.tend; }
  else t_new = s.t + h;
  const int kk = s.k < s.nh ? s.k : s.nh;
  double alpha[KMAX + 1];
  TPow pref;
  double Tref;
  bool lu_ok;
  const bool converged =
      attempt_solve(t, s, w, P.atol, P.rtol, h, t_new, kk, alpha, pref, Tref, lu_ok);
  if (!converged) {
    s.c_rej_newton++;
    if (++s.nfail >= 10) { s.status = lu_ok ? NB_Z_NEWTON_FAIL : NB_Z_SINGULAR; return true; }
    s.h = h * 0.25;
    return false;
  }
  s.nfail = 0;
  // local error estimate
  const double c = s.nh >= kk + 1 ? h / (t_new - w.th[hslot(s, kk)]) : 0.5;
  double err2;   // err^2
  {
    double acc = 0.0;
    NB_UNROLL
    for (int i = vbeg(t); i < n; i += vstep(t)) {
      const double v = c * (w.x[i] - w.xp[i]) * w.iw[i];
      acc = fma(v, v, acc);
    }
    err2 = vsum(t, acc) * t.inv_n;
  }
  if (!(err2 <= 1.0)) {
    s.c_rej_err++;
    const double fac = finite_bits(err2) ? err_factor(err2, kk) : 0.2;
    s.h = h * (fac > 0.2 ? fac : 0.2);
    return false;
  }
  // accept
  double E_new = 0.0;
  if (t.hasE) {
    if (t.sh) { eval_rates_near(t, s, w, w.x[N], pref, Tref); s.c_teval++; }
    eval_terms(t, w, w.x);
    const double ed = eval_edot(t, w);
    s.c_edot++;
    double acc = 0.0;
#pragma unroll 1
    for (int j = 1; j <= kk; ++j) acc = fma(alpha[j], w.eh[hslot(s, j - 1)], acc);
    E_new = (h * ed - acc) / alpha[0];
  }
  // push the new point into the history ring
  s.hh = s.hh == 0 ? HMAX - 1 : s.hh - 1;
  vsync(t);   // every thread has read the ring's old scalars
  {
    const int b0 = s.hh * n;
    NB_UNROLL
    for (int i = vbeg(t); i < n; i += vstep(t)) w.xh[b0 + i] = w.x[i];
    if (vlead(t)) {
      w.th[s.hh] = t_new;
      w.eh[s.hh] = E_new;
    }
  }
  vsync(t);
  if (s.nh < HMAX) s.nh++;
  s.t = t_new;
  s.E = E_new;
  s.c_acc++;
  s.c_ordsum += kk;
  if (!tape_record(t, P, s, w.x, h, kk)) { s.status = NB_Z_TAPE_FULL; return true; }
  if (s.t >= s.tend) { s.h = h; return true; }
  // next step size and order
  s.nconsec++;
  double factor;
  if (s.nconsec >= s.k + 1) {
    const int k = s.k;
    int best_q = k;
    // E_k is the step's own error estimate: the same extrapolation through
    // the same points at the same time, so the same bits
    double best = step_factor(err2, k);
    if (k > 1) {
      const double fq = step_factor(order_estimate(t, s, w, k - 1, h), k - 1);
      if (fq > best) { best = fq; best_q = k - 1; }
    }
    if (k < KMAX && s.nh >= k + 3) {
      const double fq = step_factor(order_estimate(t, s, w, k + 1, h), k + 1);
      if (fq > best) { best = fq; best_q = k + 1; }
    }
    if (best_q != k) { s.k = best_q; s.nconsec = 0; }
    factor = best;
  } else {
    factor = step_factor(err2, kk);
  }
  if (factor < 0.2) factor = 0.2;
  if (factor > 5.0) factor = 5.0;
  if (factor >= 1.0 && factor < 1.2) factor = 1.0;
  s.h = h * factor;
  return false;
}

// Recompute accepted step (h, t_new, order kk) of a recorded burn from the
// history held in w and push its solution (the adjoint's recomputation of a
// checkpointed segment; energies are not recomputed).  The forward burn's
// attempt converged on the same inputs, so this one does too; false if not.
template <class NT, class WT>
NB_HD __forceinline__ bool replay_step(const NT& t, Zone& s, WT& w, double atol, double rtol,
                                       double h, double t_new, int kk) {
  double alpha[KMAX + 1];
  TPow pref;
  double Tref;
  bool lu_ok;
  if (!attempt_solve(t, s, w, atol, rtol, h, t_new, kk, alpha, pref, Tref, lu_ok)) return false;
  s.hh = s.hh == 0 ? HMAX - 1 : s.hh - 1;
  vsync(t);
  const int b0 = s.hh * t.n;
  NB_UNROLL
  for (int i = vbeg(t); i < t.n; i += vstep(t)) w.xh[b0 + i] = w.x[i];
  if (vlead(t)) {
    w.th[s.hh] = t_new;
    w.eh[s.hh] = 0.0;
  }
  vsync(t);
  if (s.nh < HMAX) s.nh++;
  s.t = t_new;
  return true;
}

// GPU global timer (ns)
NB_HD __forceinline__ unsigned long long gpu_ns() {
#ifdef __CUDA_ARCH__
  unsigned long long v;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
  return v;
#else
  return 0ull;
#endif
}

// A zone claimed after the watchdog budget ran out: outputs are its inputs.
template <class NT>
NB_HD __forceinline__ void zone_timeout_unstarted(const NT& t, long long z,
                                                  const BurnParams& P) {
  for (int i = vbeg(t); i < t.N; i += vstep(t))
    P.Y[(unsigned long long)z * t.N + i] = P.Y0[(unsigned long long)z * t.N + i];
  if (!vlead(t)) return;
  P.T9[z] = P.T9_0[z];
  if (P.E) P.E[z] = 0.0;
  P.status[z] = NB_Z_TIMEOUT;
  if (P.use_tape) { P.tape.zstat[z] = NB_Z_TIMEOUT; P.tape.steps[z] = 0; }
  if (P.counters)
    for (int c = 0; c < NCOUNT; ++c) P.counters[(unsigned long long)z * NCOUNT + c] = 0;
}

// write a finished zone
template <class NT, class WT>
NB_HD __forceinline__ void zone_finish(const NT& t, const Zone& s, const WT& w,
                                       const BurnParams& P) {
  const long long z = s.z;
  const int b0 = hslot(s, 0) * t.n;
  vsync(t);
  NB_UNROLL
  for (int i = vbeg(t); i < t.N; i += vstep(t)) P.Y[(unsigned long long)z * t.N + i] = w.xh[b0 + i];
  if (!vlead(t)) return;
  P.T9[z] = t.sh ? w.xh[b0 + t.N] : s.T9f;
  if (P.E) P.E[z] = w.eh[s.hh];
  P.status[z] = s.status;
  if (P.use_tape) P.tape.zstat[z] = s.status;
  if (P.counters) {
    int32_t* c = P.counters + (unsigned long long)z * NCOUNT;
    c[C_ACC] = s.c_acc; c[C_REJ_ERR] = s.c_rej_err; c[C_REJ_NEWTON] = s.c_rej_newton;
    c[C_NEWTON_IT] = s.c_newton; c[C_JAC] = s.c_jac; c[C_RHS] = s.c_rhs;
    c[C_TEVAL] = s.c_teval; c[C_EDOT] = s.c_edot; c[C_ORDSUM] = s.c_ordsum;
  }
}

// The persistent lane-per-zone loop: every lane claims zones from the device
// queue (one atomic per warp for all lanes that need a zone), initialises,
// attempts steps and writes each zone back, and claims the next one as soon
// as its zone is done.  A lane whose block ran past the watchdog budget ends
// its zone with NB_Z_TIMEOUT (and every zone it claims afterwards).
template <class NT, class WT>
__device__ __forceinline__ void burn_claim_loop(const NT& t, WT& w, const BurnParams& P) {
  const int lane = threadIdx.x & 31;
  Zone s;
  s.z = -1;
  bool active = false, retired = false, fresh = false;
  const unsigned long long t_start = P.budget_ns ? gpu_ns() : 0ull;
  for (;;) {
    const unsigned need = __ballot_sync(0xffffffffu, !active && !retired);
    if (need) {
      const int leader = __ffs(need) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(P.queue, (unsigned long long)__popc(need));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (!active && !retired) {
        const unsigned long long z = base + __popc(need & ((1u << lane) - 1u));
        if (z < (unsigned long long)P.Z) {
          s.z = P.order ? (long long)P.order[z] : (long long)z;
          active = true;
          fresh = true;
        } else {
          retired = true;
        }
      }
    }
    if (__all_sync(0xffffffffu, retired)) break;
    if (active) {
      const bool expired = P.budget_ns && gpu_ns() - t_start > P.budget_ns;
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

}  // namespace nb
