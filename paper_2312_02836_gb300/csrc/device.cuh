// device.cuh -- per-zone integrator device code shared by the persistent
// lane-per-zone kernel and the plain one-thread-per-zone kernel.
//
// Mapping: one zone per lane.  On this GPU an FP64 warp instruction costs the
// FP64 pipe the same time whether 1 or 32 lanes are active, so the zone is not
// spread over lanes: every lane runs its own zone and every FP64 instruction
// does 32 zones' work.  All lanes walk the same compiled network programs, so
// program reads are shared-memory broadcasts.  Per-zone vectors live in a
// per-lane workspace interleaved by lane (element e of a lane at
// base[e * 32]), so a warp's access to "element e" is one coalesced 256-byte
// transaction.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "blob.h"
#include "expf64.cuh"
#include "../../include/netburn.h"

#ifndef NB_HD
#define NB_HD __device__
#endif

namespace nb {

// lane-strided view of one per-lane array
struct LV {
  double* p;
  NB_HD __forceinline__ double& operator[](int i) const {
    return p[i * WS_LANES];
  }
};

struct Net {
  int n, N, R, sh, hasE, nnz, nd;
  double inv_n;
  const double *coef, *Q, *scale, *rhs_c, *dt_m, *js_c, *rg_c;
  const int32_t *nrho, *nreac, *rhs_ptr, *js_ptr, *diag_orig, *rg_ptr;
  const int16_t *reac, *rhs_r, *dt_r, *dt_o, *dt_j, *js_src, *lslot, *uslot, *dslot;
  const int16_t *fw_s, *fw_c, *bw_s, *bw_c, *tfw_s, *tfw_c, *tbw_s, *tbw_c, *rg_i;
  const uint8_t* js_flag;
  const Pivot* piv;
  const TriRow *fw, *bw, *tfw, *tbw;
  int w_x, w_xp, w_psi, w_d, w_f, w_iw, w_tmp, w_f0, w_xh, w_eh, w_th, w_k,
      w_g, w_rr, w_dt, w_lu, lane_doubles, hot_doubles;
};

template <class T>
NB_HD __forceinline__ const T* at(const unsigned char* b, int off) {
  return reinterpret_cast<const T*>(b + off);
}

NB_HD inline Net make_net(const unsigned char* b) {
  const BlobHeader* h = reinterpret_cast<const BlobHeader*>(b);
  Net t;
  t.n = h->n; t.N = h->N; t.R = h->R; t.sh = h->self_heating; t.hasE = h->has_E;
  t.nnz = h->nnz; t.nd = h->nd;
  t.inv_n = 1.0 / h->n;
  t.coef = at<double>(b, h->o_coef); t.Q = at<double>(b, h->o_Q);
  t.scale = at<double>(b, h->o_scale); t.rhs_c = at<double>(b, h->o_rhs_c);
  t.dt_m = at<double>(b, h->o_dt_m); t.js_c = at<double>(b, h->o_js_c);
  t.rg_c = at<double>(b, h->o_rg_c);
  t.nrho = at<int32_t>(b, h->o_nrho); t.nreac = at<int32_t>(b, h->o_nreac);
  t.rhs_ptr = at<int32_t>(b, h->o_rhs_ptr); t.js_ptr = at<int32_t>(b, h->o_js_ptr);
  t.diag_orig = at<int32_t>(b, h->o_diag_orig); t.rg_ptr = at<int32_t>(b, h->o_rg_ptr);
  t.reac = at<int16_t>(b, h->o_reac); t.rhs_r = at<int16_t>(b, h->o_rhs_r);
  t.dt_r = at<int16_t>(b, h->o_dt_r); t.dt_o = at<int16_t>(b, h->o_dt_o);
  t.dt_j = at<int16_t>(b, h->o_dt_j);
  t.js_src = at<int16_t>(b, h->o_js_src); t.lslot = at<int16_t>(b, h->o_lslot);
  t.uslot = at<int16_t>(b, h->o_uslot); t.dslot = at<int16_t>(b, h->o_dslot);
  t.fw_s = at<int16_t>(b, h->o_fw_s); t.fw_c = at<int16_t>(b, h->o_fw_c);
  t.bw_s = at<int16_t>(b, h->o_bw_s); t.bw_c = at<int16_t>(b, h->o_bw_c);
  t.tfw_s = at<int16_t>(b, h->o_tfw_s); t.tfw_c = at<int16_t>(b, h->o_tfw_c);
  t.tbw_s = at<int16_t>(b, h->o_tbw_s); t.tbw_c = at<int16_t>(b, h->o_tbw_c);
  t.rg_i = at<int16_t>(b, h->o_rg_i);
  t.js_flag = at<uint8_t>(b, h->o_js_flag);
  t.piv = at<Pivot>(b, h->o_piv);
  t.fw = at<TriRow>(b, h->o_fw); t.bw = at<TriRow>(b, h->o_bw);
  t.tfw = at<TriRow>(b, h->o_tfw); t.tbw = at<TriRow>(b, h->o_tbw);
  t.w_x = h->w_x; t.w_xp = h->w_xp; t.w_psi = h->w_psi; t.w_d = h->w_d;
  t.w_f = h->w_f; t.w_iw = h->w_iw; t.w_tmp = h->w_tmp; t.w_f0 = h->w_f0;
  t.w_xh = h->w_xh; t.w_eh = h->w_eh; t.w_th = h->w_th; t.w_k = h->w_k;
  t.w_g = h->w_g; t.w_rr = h->w_rr; t.w_dt = h->w_dt; t.w_lu = h->w_lu;
  t.lane_doubles = h->lane_doubles;
  t.hot_doubles = h->hot_doubles;
  return t;
}

// Views of one lane's workspace.  The arrays before hot_doubles may live in
// shared memory (hot_base) while the rest stay in global memory (cold_base,
// offsets relative to hot_doubles).
struct WS {
  LV x, xp, psi, d, f, iw, tmp, f0, xh, eh, th, k, g, rr, dt, lu;
};

NB_HD __forceinline__ WS make_ws_split(const Net& t, double* hot_base, double* cold_base) {
  WS w;
  w.x.p = hot_base + t.w_x * WS_LANES;
  w.xp.p = hot_base + t.w_xp * WS_LANES;
  w.psi.p = hot_base + t.w_psi * WS_LANES;
  w.d.p = hot_base + t.w_d * WS_LANES;
  w.f.p = hot_base + t.w_f * WS_LANES;
  w.iw.p = hot_base + t.w_iw * WS_LANES;
  w.k.p = hot_base + t.w_k * WS_LANES;
  w.g.p = hot_base + t.w_g * WS_LANES;
  w.rr.p = hot_base + t.w_rr * WS_LANES;
  w.dt.p = hot_base + t.w_dt * WS_LANES;
  w.lu.p = hot_base + t.w_lu * WS_LANES;
  w.tmp.p = cold_base + (t.w_tmp - t.hot_doubles) * WS_LANES;
  w.f0.p = cold_base + (t.w_f0 - t.hot_doubles) * WS_LANES;
  w.xh.p = cold_base + (t.w_xh - t.hot_doubles) * WS_LANES;
  w.eh.p = cold_base + (t.w_eh - t.hot_doubles) * WS_LANES;
  w.th.p = cold_base + (t.w_th - t.hot_doubles) * WS_LANES;
  return w;
}

NB_HD __forceinline__ WS make_ws(const Net& t, double* lane_base) {
  WS w;
  w.x.p = lane_base + t.w_x * WS_LANES;
  w.xp.p = lane_base + t.w_xp * WS_LANES;
  w.psi.p = lane_base + t.w_psi * WS_LANES;
  w.d.p = lane_base + t.w_d * WS_LANES;
  w.f.p = lane_base + t.w_f * WS_LANES;
  w.iw.p = lane_base + t.w_iw * WS_LANES;
  w.tmp.p = lane_base + t.w_tmp * WS_LANES;
  w.f0.p = lane_base + t.w_f0 * WS_LANES;
  w.xh.p = lane_base + t.w_xh * WS_LANES;
  w.eh.p = lane_base + t.w_eh * WS_LANES;
  w.th.p = lane_base + t.w_th * WS_LANES;
  w.k.p = lane_base + t.w_k * WS_LANES;
  w.g.p = lane_base + t.w_g * WS_LANES;
  w.rr.p = lane_base + t.w_rr * WS_LANES;
  w.dt.p = lane_base + t.w_dt * WS_LANES;
  w.lu.p = lane_base + t.w_lu * WS_LANES;
  return w;
}

// Tape written by a burn that will be differentiated.
struct TapeDev {
  double* rec;       // [Z, cap, n + 3]: t, h, x[0..n), E
  int8_t* ord;       // [Z, cap] BDF order of the step (0 for the start point)
  int32_t* steps;    // [Z] records written
  int32_t* zstat;    // [Z] status the zone finished with
  double* rho;       // [Z]
  double* T9f;       // [Z] fixed temperature (or initial T9)
  int32_t cap;
};

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
};

// Register state of the zone a lane is integrating.
struct Zone {
  long long z;
  double t, h, E, T9f, rho, rho2, tend;
  const double* lnm;
  int k, nh, hh, nconsec, nfail, status;
  int c_acc, c_rej_err, c_rej_newton, c_newton, c_jac, c_rhs, c_teval, c_edot;
};

NB_HD __forceinline__ int hslot(const Zone& s, int j) {
  int v = s.hh + j;
  return v >= HMAX ? v - HMAX : v;
}

// ---------------------------------------------------------------- model

// k_r (and g_r = d ln lambda_r / dT9 when with_g) for temperature T9
NB_HD inline void eval_rates(const Net& t, const Zone& s, const WS& w,
                                  double T9, bool with_g) {
  const double t13 = cbrt(T9);
  const double iT = 1.0 / T9;
  const double t23 = t13 * t13;
  const double it13 = t23 * iT;          // T9^(-1/3) without a second division
  const double T53 = T9 * t23;
  const double lnT = log(T9);
  double d1 = 0.0, d2 = 0.0, d3 = 0.0, d5 = 0.0;
  if (with_g) {
    d1 = -iT * iT;
    d2 = (-1.0 / 3.0) * iT * it13;
    d3 = (1.0 / 3.0) * it13 * it13;
    d5 = (5.0 / 3.0) * t23;
  }
  // one warp per scheduler leaves FP64 latency exposed: two reactions per
  // iteration and two partial sums per exponent give independent chains
#pragma unroll 2
  for (int r = 0; r < t.R; ++r) {
    const double* a = t.coef + 7 * r;
    double e1 = fma(a[1], iT, a[0]);
    double e2 = a[4] * T9;
    e1 = fma(a[2], it13, e1);
    e2 = fma(a[5], T53, e2);
    e1 = fma(a[3], t13, e1);
    e2 = fma(a[6], lnT, e2);
    double e = e1 + e2;
    if (s.lnm) e += s.lnm[r];
    const int nr = t.nrho[r];
    const double rp = nr == 0 ? 1.0 : (nr == 1 ? s.rho : s.rho2);
    w.k[r] = exp_tang(e) * (rp * t.scale[r]);
    if (with_g) {
      double g1 = fma(a[1], d1, a[4]);
      double g2 = a[5] * d5;
      g1 = fma(a[2], d2, g1);
      g2 = fma(a[6], iT, g2);
      g1 = fma(a[3], d3, g1);
      w.g[r] = g1 + g2;
    }
  }
}

// R_r = k_r prod Y over reactant occurrences, for state v
NB_HD inline void eval_terms(const Net& t, const WS& w, const LV& v) {
#pragma unroll 4
  for (int r = 0; r < t.R; ++r) {
    const int16_t* ra = t.reac + 3 * r;
    const int m = t.nreac[r];
    double q = w.k[r];
    q *= v[ra[0]];
    if (m > 1) q *= v[ra[1]];
    if (m > 2) q *= v[ra[2]];
    w.rr[r] = q;
  }
}

NB_HD __forceinline__ double heat_capacity(const Net& t, const LV& v) {
  double s0 = 0.0, s1 = 0.0;
  int i = 0;
  for (; i + 1 < t.N; i += 2) {
    s0 += v[i];
    s1 += v[i + 1];
  }
  if (i < t.N) s0 += v[i];
  const double T9 = v[t.N];
  return 1.5 * (s0 + s1) + 1e-3 * T9 * T9 * T9;
}

NB_HD __forceinline__ double eval_edot(const Net& t, const WS& w) {
  double e0 = 0.0, e1 = 0.0;
  int r = 0;
  for (; r + 1 < t.R; r += 2) {
    e0 = fma(t.Q[r], w.rr[r], e0);
    e1 = fma(t.Q[r + 1], w.rr[r + 1], e1);
  }
  if (r < t.R) e0 = fma(t.Q[r], w.rr[r], e0);
  return e0 + e1;
}

// sum_e c[e] * v[idx[e]] over [beg, end), two interleaved partial sums
template <class TI>
NB_HD __forceinline__ double gather2(const double* c, const TI* idx, int beg, int end,
                                     const LV& v) {
  double a0 = 0.0, a1 = 0.0;
  int e = beg;
  for (; e + 1 < end; e += 2) {
    a0 = fma(c[e], v[idx[e]], a0);
    a1 = fma(c[e + 1], v[idx[e + 1]], a1);
  }
  if (e < end) a0 = fma(c[e], v[idx[e]], a0);
  return a0 + a1;
}

// out = f(v) given w.rr for v
NB_HD inline void eval_f(const Net& t, const WS& w, const LV& v, const LV& out) {
#pragma unroll 2
  for (int i = 0; i < t.N; ++i)
    out[i] = gather2(t.rhs_c, t.rhs_r, t.rhs_ptr[i], t.rhs_ptr[i + 1], w.rr);
  if (t.sh) out[t.N] = eval_edot(t, w) / heat_capacity(t, v);
}

// M = alpha0 I - h J(v) into w.lu (needs w.k, w.g (self-heating), w.rr at v)
NB_HD inline void assemble_M(const Net& t, const WS& w, const LV& v,
                                  double alpha0, double h) {
#pragma unroll 4
  for (int d = 0; d < t.nd; ++d) {
    const int16_t o0 = t.dt_o[2 * d], o1 = t.dt_o[2 * d + 1];
    double q = w.k[t.dt_r[d]] * t.dt_m[d];
    if (o0 >= 0) q *= v[o0];
    if (o1 >= 0) q *= v[o1];
    w.dt[d] = q;
  }
  double a1 = 0.0, b1 = 0.0, b2 = 0.0;
  if (t.sh) {
    for (int r = 0; r < t.R; ++r) w.dt[t.nd + r] = w.rr[r] * w.g[r];
    const double ed = eval_edot(t, w);
    const double cv = heat_capacity(t, v);
    const double icv = 1.0 / cv;
    const double fT = ed / cv;
    const double T9 = v[t.N];
    a1 = icv;
    b1 = -fT * 1.5 * icv;
    b2 = -fT * (3e-3 * T9 * T9) * icv;
  }
  const double mh = -h;
#pragma unroll 2
  for (int s = 0; s < t.nnz; ++s) {
    double acc = gather2(t.js_c, t.js_src, t.js_ptr[s], t.js_ptr[s + 1], w.dt);
    const uint8_t fl = t.js_flag[s];
    if (fl & SLOT_TROW) acc = fma(acc, a1, b1);
    else if (fl & SLOT_TT) acc = fma(acc, a1, b2);
    double m = mh * acc;
    if (fl & SLOT_DIAG) m += alpha0;
    w.lu[s] = m;
  }
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

// static-pivot LU in place; the diagonal keeps 1/pivot.  false if singular.
NB_HD inline bool factor_M(const Net& t, const WS& w) {
  bool ok = true;
  for (int k = 0; k < t.n; ++k) {
    const Pivot p = t.piv[k];
    const double pv = w.lu[p.dslot];
    ok = ok && finite_nonzero(pv);
    const double inv = 1.0 / pv;
    w.lu[p.dslot] = inv;
    const int nu = p.uend - p.ubeg;
    int dpos = p.dbeg;
    for (int li = p.lbeg; li < p.lend; ++li) {
      const int ls = t.lslot[li];
      const double l = w.lu[ls] * inv;
      w.lu[ls] = l;
      const double ml = -l;
#pragma unroll 4
      for (int u = 0; u < nu; ++u, ++dpos) {
        const int ds = t.dslot[dpos];
        w.lu[ds] = fma(ml, w.lu[t.uslot[p.ubeg + u]], w.lu[ds]);
      }
    }
  }
  return ok;
}

// one triangular gather program applied in place to v
NB_HD __forceinline__ void tri_solve(const TriRow* rows, const int16_t* es,
                                          const int16_t* ec, int n, const LV& lu,
                                          const LV& v) {
  for (int q = 0; q < n; ++q) {
    const TriRow r = rows[q];
    double a0 = v[r.tgt], a1 = 0.0;
    int e = r.beg;
    for (; e + 1 < r.end; e += 2) {
      a0 = fma(-lu[es[e]], v[ec[e]], a0);
      a1 = fma(-lu[es[e + 1]], v[ec[e + 1]], a1);
    }
    if (e < r.end) a0 = fma(-lu[es[e]], v[ec[e]], a0);
    double acc = a0 + a1;
    if (r.dslot >= 0) acc *= lu[r.dslot];
    v[r.tgt] = acc;
  }
}

// ||v||^2 = mean (v_i * iw_i)^2, two interleaved partial sums (the tests
// compare squares, which spares a square root per norm)
NB_HD __forceinline__ double wnorm2(const Net& t, const WS& w, const LV& v) {
  double s0 = 0.0, s1 = 0.0;
  int i = 0;
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

// Lagrange weights at time tt of the q+1 newest history points starting at
// history index j0 (0 = newest)
NB_HD __forceinline__ void lagrange_weights(const Zone& s, const WS& w, int j0,
                                                 int q, double tt, double* lw) {
  double tp[KMAX + 2];
#pragma unroll
  for (int j = 0; j < KMAX + 2; ++j) tp[j] = (j <= q) ? w.th[hslot(s, j0 + j)] : 0.0;
#pragma unroll
  for (int j = 0; j < KMAX + 2; ++j) {
    double num = 1.0, den = 1.0;
#pragma unroll
    for (int m = 0; m < KMAX + 2; ++m) {
      if (m != j && m <= q && j <= q) {
        num *= tt - tp[m];
        den *= tp[j] - tp[m];
      }
    }
    lw[j] = (j <= q) ? num / den : 0.0;
  }
}

// out = value at tt of the degree-q polynomial through history j0..j0+q
NB_HD inline void extrapolate(const Net& t, const Zone& s, const WS& w, int j0,
                                   int q, double tt, const LV& out) {
  double lw[KMAX + 2];
  lagrange_weights(s, w, j0, q, tt, lw);
  int base[KMAX + 2];
#pragma unroll
  for (int j = 0; j < KMAX + 2; ++j) base[j] = hslot(s, j0 + j) * t.n;
  for (int i = 0; i < t.n; ++i) {
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < KMAX + 2; ++j)
      if (j <= q) acc = fma(lw[j], w.xh[base[j] + i], acc);
    out[i] = acc;
  }
}

// 0.9 E^(-1/(q+1)) from E^2
NB_HD __forceinline__ double step_factor(double E2, int q) {
  if (!(E2 > 0.0)) return 5.0;
  return 0.9 * pow(E2, -0.5 / (q + 1));
}

// E_q^2 after acceptance: newest point vs extrapolation through the q+1 older
NB_HD inline double order_estimate(const Net& t, const Zone& s, const WS& w,
                                        int q, double h) {
  extrapolate(t, s, w, 1, q, w.th[hslot(s, 0)], w.tmp);
  const double c = h / (w.th[hslot(s, 0)] - w.th[hslot(s, q + 1)]);
  const int b0 = hslot(s, 0) * t.n;
  double acc = 0.0;
  for (int i = 0; i < t.n; ++i) {
    const double v = c * (w.xh[b0 + i] - w.tmp[i]) * w.iw[i];
    acc = fma(v, v, acc);
  }
  return acc * t.inv_n;   // E_q^2
}

// Record an accepted point (time, step, state, energy, order); false when
// the zone's tape is full.
NB_HD __forceinline__ bool tape_record(const Net& t, const BurnParams& P,
                                       const Zone& s, const LV& x, double h, int ord) {
  if (!P.use_tape) return true;
  int32_t* cnt = P.tape.steps + s.z;
  const int idx = *cnt;
  if (idx >= P.tape.cap) return false;
  double* rec = P.tape.rec + ((size_t)s.z * P.tape.cap + idx) * (t.n + 3);
  rec[0] = s.t;
  rec[1] = h;
  for (int i = 0; i < t.n; ++i) rec[2 + i] = x[i];
  rec[2 + t.n] = s.E;
  P.tape.ord[(size_t)s.z * P.tape.cap + idx] = (int8_t)ord;
  *cnt = idx + 1;
  return true;
}

// alpha_j = h l_j'(tau_0), Lagrange basis on tau_0..tau_kk (unused j -> 0)
NB_HD __forceinline__ void bdf_alpha(int kk, const double* tau, double h, double* alpha) {
  double acc = 0.0;
#pragma unroll
  for (int m = 1; m <= KMAX; ++m)
    if (m <= kk) acc += 1.0 / (tau[0] - tau[m]);
  alpha[0] = h * acc;
#pragma unroll
  for (int j = 1; j <= KMAX; ++j) {
    double num = 1.0, den = 1.0;
#pragma unroll
    for (int m = 0; m <= KMAX; ++m) {
      if (m != j && m <= kk && j <= kk) {
        if (m != 0) num *= tau[0] - tau[m];
        den *= tau[j] - tau[m];
      }
    }
    alpha[j] = (j <= kk) ? h * num / den : 0.0;
  }
}

// ---------------------------------------------------------------- zone start

// Load zone s.z, evaluate f(x0) and the starting step.  Returns true when the
// zone is already finished (bad input or t_end == 0).
NB_HD inline bool zone_init(const Net& t, Zone& s, const WS& w, const BurnParams& P) {
  const long long z = s.z;
  const int n = t.n, N = t.N;
  s.t = 0.0; s.E = 0.0; s.k = 1; s.nh = 1; s.hh = 0; s.nconsec = 0; s.nfail = 0;
  s.status = NB_Z_OK;
  s.c_acc = s.c_rej_err = s.c_rej_newton = s.c_newton = 0;
  s.c_jac = s.c_rhs = s.c_teval = s.c_edot = 0;
  s.T9f = P.T9_0[z];
  s.rho = P.rho[z];
  s.rho2 = s.rho * s.rho;
  s.lnm = P.lnm ? (P.lnm_per_zone ? P.lnm + (size_t)z * t.R : P.lnm) : nullptr;
  s.tend = P.t_end_zone ? P.t_end_zone[z] : P.t_end;
  const LV x0{w.xh.p};  // history slot 0
  bool fin = isfinite(s.T9f) && s.T9f > 0.0 && isfinite(s.rho) && finite_bits(s.tend) &&
             s.tend >= 0.0;
  for (int i = 0; i < N; ++i) {
    const double y = P.Y0[(size_t)z * N + i];
    x0[i] = y;
    fin = fin && isfinite(y);
  }
  if (t.sh) x0[N] = s.T9f;
  w.th[0] = 0.0;
  w.eh[0] = 0.0;
  if (P.use_tape) {
    P.tape.steps[z] = 0;
    P.tape.rho[z] = s.rho;
    P.tape.T9f[z] = s.T9f;
    tape_record(t, P, s, x0, 0.0, 0);
  }
  eval_rates(t, s, w, s.T9f, false);
  s.c_teval++;
  eval_terms(t, w, x0);
  eval_f(t, w, x0, w.f0);
  s.c_rhs++;
  for (int r = 0; r < t.R; ++r) fin = fin && finite_bits(w.k[r]);
  for (int i = 0; i < n; ++i) fin = fin && finite_bits(w.f0[i]);
  if (!fin) { s.status = NB_Z_NONFINITE; return true; }
  if (!(s.tend > 0.0)) return true;
  // starting step: Hairer-Norsett-Wanner I, Sec. II.4, p = 1
  double s0 = 0.0, s1 = 0.0;
  for (int i = 0; i < n; ++i) {
    const double iw = 1.0 / (P.atol + P.rtol * fabs(x0[i]));
    w.iw[i] = iw;
    const double a = x0[i] * iw, b = w.f0[i] * iw;
    s0 = fma(a, a, s0);
    s1 = fma(b, b, s1);
  }
  const double d0 = sqrt(s0 / n), d1 = sqrt(s1 / n);
  double hp = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
  if (hp > s.tend) hp = s.tend;
  for (int i = 0; i < n; ++i) w.x[i] = fma(hp, w.f0[i], x0[i]);
  if (t.sh) { eval_rates(t, s, w, w.x[N], false); s.c_teval++; }
  eval_terms(t, w, w.x);
  eval_f(t, w, w.x, w.f);
  s.c_rhs++;
  double s2 = 0.0;
  const double ihp = 1.0 / hp;
  for (int i = 0; i < n; ++i) {
    const double q = (w.f[i] - w.f0[i]) * ihp * w.iw[i];
    s2 = fma(q, q, s2);
  }
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

// One step attempt.  Returns true when the zone is finished.
NB_HD inline bool zone_attempt(const Net& t, Zone& s, const WS& w,
                                    const BurnParams& P) {
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

  // alpha_j = h l_j'(t_new) over t_new, t_n, .., t_{n+1-kk}
  double tau[KMAX + 1];
  tau[0] = t_new;
#pragma unroll
  for (int j = 1; j <= KMAX; ++j) tau[j] = (j <= kk) ? w.th[hslot(s, j - 1)] : 0.0;
  double alpha[KMAX + 1];
  bdf_alpha(kk, tau, h, alpha);
  // psi = sum_{j>=1} alpha_j x_{n+1-j}; weights from x_n
  {
    int base[KMAX];
#pragma unroll
    for (int j = 0; j < KMAX; ++j) base[j] = hslot(s, j) * n;
    for (int i = 0; i < n; ++i) {
      double acc = 0.0;
#pragma unroll
      for (int j = 1; j <= KMAX; ++j)
        if (j <= kk) acc = fma(alpha[j], w.xh[base[j - 1] + i], acc);
      w.psi[i] = acc;
      w.iw[i] = 1.0 / (P.atol + P.rtol * fabs(w.xh[base[0] + i]));
    }
  }
  // predictor
  if (s.nh >= kk + 1) extrapolate(t, s, w, 0, kk, t_new, w.xp);
  else if (s.nh >= 2) extrapolate(t, s, w, 0, s.nh - 1, t_new, w.xp);
  else {
    const int b0 = hslot(s, 0) * n;
    for (int i = 0; i < n; ++i) w.xp[i] = fma(h, w.f0[i], w.xh[b0 + i]);
  }
  for (int i = 0; i < n; ++i) w.x[i] = w.xp[i];
  // Jacobian at the predictor, M, LU
  if (t.sh) { eval_rates(t, s, w, w.x[N], true); s.c_teval++; }
  eval_terms(t, w, w.x);
  assemble_M(t, w, w.x, alpha[0], h);
  s.c_jac++;
  bool ok = factor_M(t, w);
  // modified Newton
  bool converged = false;
  double nrm_prev = 0.0;
  for (int m = 0; ok && m < 4; ++m) {
    if (m > 0) {
      if (t.sh) { eval_rates(t, s, w, w.x[N], false); s.c_teval++; }
      eval_terms(t, w, w.x);
    }
    eval_f(t, w, w.x, w.f);
    s.c_rhs++;
    for (int i = 0; i < n; ++i)
      w.d[i] = -(fma(alpha[0], w.x[i], w.psi[i]) - h * w.f[i]);
    tri_solve(t.fw, t.fw_s, t.fw_c, n, w.lu, w.d);
    tri_solve(t.bw, t.bw_s, t.bw_c, n, w.lu, w.d);
    for (int i = 0; i < n; ++i) w.x[i] += w.d[i];
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
  if (!converged) {
    s.c_rej_newton++;
    if (++s.nfail >= 10) { s.status = NB_Z_NEWTON_FAIL; return true; }
    s.h = h * 0.25;
    return false;
  }
  s.nfail = 0;
  // local error estimate
  const double c = s.nh >= kk + 1 ? h / (t_new - w.th[hslot(s, kk)]) : 0.5;
  double err2;   // err^2
  {
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
      const double v = c * (w.x[i] - w.xp[i]) * w.iw[i];
      acc = fma(v, v, acc);
    }
    err2 = acc * t.inv_n;
  }
  if (!(err2 <= 1.0)) {
    s.c_rej_err++;
    const double fac = finite_bits(err2) ? 0.9 * pow(err2, -0.5 / (kk + 1)) : 0.2;
    s.h = h * (fac > 0.2 ? fac : 0.2);
    return false;
  }
  // accept
  double E_new = 0.0;
  if (t.hasE) {
    if (t.sh) { eval_rates(t, s, w, w.x[N], false); s.c_teval++; }
    eval_terms(t, w, w.x);
    const double ed = eval_edot(t, w);
    s.c_edot++;
    double acc = 0.0;
#pragma unroll
    for (int j = 1; j <= KMAX; ++j)
      if (j <= kk) acc = fma(alpha[j], w.eh[hslot(s, j - 1)], acc);
    E_new = (h * ed - acc) / alpha[0];
  }
  // push the new point into the history ring
  s.hh = s.hh == 0 ? HMAX - 1 : s.hh - 1;
  {
    const int b0 = s.hh * n;
    for (int i = 0; i < n; ++i) w.xh[b0 + i] = w.x[i];
    w.th[s.hh] = t_new;
    w.eh[s.hh] = E_new;
  }
  if (s.nh < HMAX) s.nh++;
  s.t = t_new;
  s.E = E_new;
  s.c_acc++;
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
NB_HD inline void zone_timeout_unstarted(const Net& t, long long z, const BurnParams& P) {
  for (int i = 0; i < t.N; ++i) P.Y[(size_t)z * t.N + i] = P.Y0[(size_t)z * t.N + i];
  P.T9[z] = P.T9_0[z];
  if (P.E) P.E[z] = 0.0;
  P.status[z] = NB_Z_TIMEOUT;
  if (P.use_tape) { P.tape.zstat[z] = NB_Z_TIMEOUT; P.tape.steps[z] = 0; }
  if (P.counters)
    for (int c = 0; c < NCOUNT; ++c) P.counters[(size_t)z * NCOUNT + c] = 0;
}

// write a finished zone
NB_HD inline void zone_finish(const Net& t, const Zone& s, const WS& w,
                                   const BurnParams& P) {
  const long long z = s.z;
  const int b0 = hslot(s, 0) * t.n;
  for (int i = 0; i < t.N; ++i) P.Y[(size_t)z * t.N + i] = w.xh[b0 + i];
  P.T9[z] = t.sh ? w.xh[b0 + t.N] : s.T9f;
  if (P.E) P.E[z] = w.eh[s.hh];
  P.status[z] = s.status;
  if (P.use_tape) P.tape.zstat[z] = s.status;
  if (P.counters) {
    int32_t* c = P.counters + (size_t)z * NCOUNT;
    c[C_ACC] = s.c_acc; c[C_REJ_ERR] = s.c_rej_err; c[C_REJ_NEWTON] = s.c_rej_newton;
    c[C_NEWTON_IT] = s.c_newton; c[C_JAC] = s.c_jac; c[C_RHS] = s.c_rhs;
    c[C_TEVAL] = s.c_teval; c[C_EDOT] = s.c_edot;
  }
}

}  // namespace nb
