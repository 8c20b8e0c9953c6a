// device.cuh -- the generic network evaluation of the per-zone integrator,
// shared by the persistent lane-per-zone kernel, the plain one-thread-per-zone
// kernel and the adjoint.
//
// Mapping: one zone per lane.  On this GPU an FP64 warp instruction costs the
// FP64 pipe the same time whether 1 or 32 lanes are active, so the zone is not
// spread over lanes: every lane runs its own zone and every FP64 instruction
// does 32 zones' work.  All lanes walk the same compiled network programs, so
// program reads are shared-memory broadcasts.  Per-zone vectors live in a
// per-lane workspace interleaved by lane (element e of a lane at
// base[e * 32]), so a warp's access to "element e" is one coalesced 256-byte
// transaction.
//
// The integrator itself (integrator.cuh) is generic over the network type;
// this file supplies the network type that reads a compiled network ("blob")
// from memory.  The specialised kernel generated per network at run time
// supplies another with the same arithmetic.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "blob.h"
#include "expf64.cuh"
#include "integrator.cuh"
#include "../../include/netburn.h"

namespace nb {

struct Net {
  int n, N, R, sh, hasE, nnz, nd;
  double inv_n;
  const double *coef, *Q, *scale, *rhs_c, *dt_m, *js_c, *rg_c, *apc;
  const double* scr;   // weak-screening strengths s_r, null without screening
  const int32_t* tab_of;   // table of reaction r (-1 fit), null without tables
  const double *tab_dens, *tab_t9, *tab_lnl, *charge;
  int tab_nd, tab_nt;
  const int32_t *nrho, *nreac, *rhs_ptr, *js_ptr, *diag_orig, *rg_ptr, *ap;
  const int16_t *reac, *rhs_r, *dt_r, *dt_o, *dt_j, *js_src, *lslot, *uslot, *dslot;
  const int16_t *fw_s, *fw_c, *bw_s, *bw_c, *tfw_s, *tfw_c, *tbw_s, *tbw_c, *rg_i;
  const uint8_t* js_flag;
  const Pivot* piv;
  const TriRow *fw, *bw, *tfw, *tbw;
  int w_x, w_xp, w_psi, w_d, w_f, w_iw, w_tmp, w_f0, w_xh, w_eh, w_th, w_k,
      w_g, w_rr, w_kp, w_dt, w_lu, lane_doubles, hot_doubles;
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
  t.apc = at<double>(b, h->o_apc); t.ap = at<int32_t>(b, h->o_ap);
  t.scr = h->has_scr ? at<double>(b, h->o_scr) : nullptr;
  t.tab_of = h->n_tab > 0 ? at<int32_t>(b, h->o_tab_of) : nullptr;
  t.tab_dens = at<double>(b, h->o_tab_dens); t.tab_t9 = at<double>(b, h->o_tab_t9);
  t.tab_lnl = at<double>(b, h->o_tab_lnl); t.charge = at<double>(b, h->o_charge);
  t.tab_nd = h->tab_nd; t.tab_nt = h->tab_nt;
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
  t.w_g = h->w_g; t.w_rr = h->w_rr; t.w_kp = h->w_kp; t.w_dt = h->w_dt; t.w_lu = h->w_lu;
  t.lane_doubles = h->lane_doubles;
  t.hot_doubles = h->hot_doubles;
  return t;
}

// Views of one lane's workspace.  The arrays before hot_doubles may live in
// shared memory (hot_base) while the rest stay in global memory (cold_base,
// offsets relative to hot_doubles).
struct WS {
  LV x, xp, psi, d, f, iw, tmp, f0, xh, eh, th, k, g, rr, kp, dt, lu;
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
  // g and kp sit with the cold part at fixed temperature
  w.g.p = t.w_g < t.hot_doubles ? hot_base + t.w_g * WS_LANES
                                : cold_base + (t.w_g - t.hot_doubles) * WS_LANES;
  w.rr.p = hot_base + t.w_rr * WS_LANES;
  w.kp.p = t.w_kp < t.hot_doubles ? hot_base + t.w_kp * WS_LANES
                                  : cold_base + (t.w_kp - t.hot_doubles) * WS_LANES;
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
  w.kp.p = lane_base + t.w_kp * WS_LANES;
  w.dt.p = lane_base + t.w_dt * WS_LANES;
  w.lu.p = lane_base + t.w_lu * WS_LANES;
  return w;
}

// ---------------------------------------------------------------- model

// k_r of reaction r (and g_r = d ln lambda_r / dT9 when g) at T9 with powers p
// (tc: the temperature cell of the rate tables at T9)
NB_HD __forceinline__ double rate_full(const Net& t, const Zone& s, int r, const TPow& p,
                                       double T9, const TCell& tc, double* g) {
  const double* a = t.coef + 7 * r;
  const int tb = t.tab_of ? t.tab_of[r] : -1;
  double dl = 0.0;
  double e = tb >= 0 ? table_lnl(t.tab_lnl + (size_t)tb * t.tab_nd * t.tab_nt, t.tab_nt, s,
                                 tc, &dl)
                     : rate_exponent(a[0], a[1], a[2], a[3], a[4], a[5], a[6], p, T9);
  if (s.lnm) e += s.lnm[r];
  const double sr = t.scr ? t.scr[r] : 0.0;
  if (t.scr) e = fma(sr, p.hz, e);
  const int nr = t.nrho[r];
  const double rp = nr == 0 ? 1.0 : (nr == 1 ? s.rho : s.rho2);
  const int api = t.ap[r];
  if (api < 0) {
    if (g) {
      *g = tb >= 0 ? dl : rate_dlog(a[1], a[2], a[3], a[4], a[5], a[6], p);
      if (t.scr) *g = fma(sr, p.hzd, *g);
    }
    return exp_tang(e) * (rp * t.scale[r]);
  }
  const double* b = t.apc + 21 * api;
  double eap = rate_exponent(b[0], b[1], b[2], b[3], b[4], b[5], b[6], p, T9);
  if (s.lnm) eap += s.lnm[r];
  if (t.scr) eap = fma(sr, p.hz, eap);
  const double epg = rate_exponent(b[7], b[8], b[9], b[10], b[11], b[12], b[13], p, T9);
  const double epa = rate_exponent(b[14], b[15], b[16], b[17], b[18], b[19], b[20], p, T9);
  const APRate q = ap_rate(e, eap, epg, epa);
  if (g) {
    double gag = rate_dlog(a[1], a[2], a[3], a[4], a[5], a[6], p);
    double gap = rate_dlog(b[1], b[2], b[3], b[4], b[5], b[6], p);
    if (t.scr) {
      gag = fma(sr, p.hzd, gag);
      gap = fma(sr, p.hzd, gap);
    }
    *g = ap_dlog(q, gag, gap,
                 rate_dlog(b[8], b[9], b[10], b[11], b[12], b[13], p),
                 rate_dlog(b[15], b[16], b[17], b[18], b[19], b[20], p));
  }
  return q.lam * (rp * t.scale[r]);
}

// k_r (and g_r = d ln lambda_r / dT9 when with_g) for temperature T9, whose
// powers p = t_powers(T9, with_g) the caller supplies
NB_HD inline void eval_rates(const Net& t, const Zone& s, const WS& w, const TPow& p,
                             double T9, bool with_g) {
  // one warp per scheduler leaves FP64 latency exposed: two reactions per
  // iteration and two partial sums per exponent give independent chains
  const TCell tc = t.tab_of ? t_cell(t.tab_t9, t.tab_nt, T9) : TCell{0, 0.0, 1.0, false};
#pragma unroll 2
  for (int r = 0; r < t.R; ++r) {
    double g;
    w.k[r] = rate_full(t, s, r, p, T9, tc, with_g ? &g : nullptr);
    if (with_g) w.g[r] = g;
  }
}

// k_r at T9 from the rates kept at the attempt's reference temperature
// (rate_near); the reference's own k_r are saved by save_ref_rates.
// Effective (alpha,p)(p,gamma) rates always take the full evaluation.
NB_HD inline void eval_rates_near(const Net& t, const Zone& s, const WS& w, double T9,
                                  const TPow& ref, double T9ref) {
  // the changes of the powers by their series when T9 is close to the
  // reference; the powers themselves only when a rate needs them
  DPhi d;
  TPow p;
  bool have_p = !delta_phi_series(ref, T9, T9ref, d);
  if (have_p) {
    p = t_powers(T9, false, s.scr);
    d = delta_phi(p, ref, T9, T9ref);
  }
  const TCell tc = t.tab_of ? t_cell(t.tab_t9, t.tab_nt, T9) : TCell{0, 0.0, 1.0, false};
#pragma unroll 2
  for (int r = 0; r < t.R; ++r) {
    const double* a = t.coef + 7 * r;
    double de = rate_delta(a[1], a[2], a[3], a[4], a[5], a[6], d);
    if (t.scr) de = fma(t.scr[r], d.d7, de);
    // tabulated and effective rates always take the full evaluation
    if (t.ap[r] < 0 && !(t.tab_of && t.tab_of[r] >= 0) && small_delta(de)) {
      w.k[r] = rate_near(w.kp[r], de);
    } else {
      if (!have_p) {
        p = t_powers(T9, false, s.scr);
        have_p = true;
      }
      w.k[r] = rate_full(t, s, r, p, T9, tc, nullptr);
    }
  }
}

// the zone's density cell of the rate tables: Ye = sum Z_i Y_i of x0
template <class V>
NB_HD __forceinline__ void tab_zone(const Net& t, Zone& s, const V& x0) {
  s.tab_i = 0;
  s.tab_u = 0.0;
  if (!t.tab_of) return;
  double ye = 0.0;
  for (int i = 0; i < t.N; ++i) ye = fma(t.charge[i], x0[i], ye);
  density_cell(t.tab_dens, t.tab_nd, s.rho, ye, s);
}

NB_HD __forceinline__ void save_ref_rates(const Net& t, const WS& w) {
  for (int r = 0; r < t.R; ++r) w.kp[r] = w.k[r];
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
  TRow tr{0.0, 0.0, 0.0};
  if (t.sh) {
    for (int r = 0; r < t.R; ++r) w.dt[t.nd + r] = w.rr[r] * w.g[r];
    tr = t_row(eval_edot(t, w), heat_capacity(t, v), v[t.N]);
  }
  const double mh = -h;
#pragma unroll 2
  for (int s = 0; s < t.nnz; ++s) {
    double acc = gather2(t.js_c, t.js_src, t.js_ptr[s], t.js_ptr[s + 1], w.dt);
    const uint8_t fl = t.js_flag[s];
    if (fl & SLOT_TROW) acc = fma(acc, tr.a1, tr.b1);
    else if (fl & SLOT_TT) acc = fma(acc, tr.a1, tr.b2);
    double m = mh * acc;
    if (fl & SLOT_DIAG) m += alpha0;
    w.lu[s] = m;
  }
}

// static-pivot LU in place; the diagonal keeps 1/pivot.  false if a pivot is
// zero, not finite or eaten by cancellation (pivot_kept; the diagonal of M
// before elimination is kept in w.tmp, free during an attempt)
NB_HD inline bool factor_M(const Net& t, const WS& w) {
  for (int k = 0; k < t.n; ++k) w.tmp[k] = w.lu[t.piv[k].dslot];
  bool ok = true;
  for (int k = 0; k < t.n; ++k) {
    const Pivot p = t.piv[k];
    const double pv = w.lu[p.dslot];
    ok = ok && pivot_kept(pv, w.tmp[k]);
    const double inv = recip2(pv);
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

// v <- M^-1 v: forward then back substitution with the factored w.lu
NB_HD __forceinline__ void solve_M(const Net& t, const WS& w, const LV& v) {
  tri_solve(t.fw, t.fw_s, t.fw_c, t.n, w.lu, v);
  tri_solve(t.bw, t.bw_s, t.bw_c, t.n, w.lu, v);
}

}  // namespace nb
