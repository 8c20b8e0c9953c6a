// adjoint.cuh -- the per-zone steps of the discrete adjoint's reverse sweep
// (the kernel and the entry point are in adjoint.cu).  Written for the
// device; the tests also compile it for the host.
#pragma once
#include "device.cuh"

namespace nb {

NB_HD __forceinline__ double quiet_nan() {
#ifdef __CUDA_ARCH__
  return __longlong_as_double(0x7ff8000000000000LL);
#else
  const long long b = 0x7ff8000000000000LL;
  double v;
  memcpy(&v, &b, sizeof v);
  return v;
#endif
}

struct AdjParams {
  const unsigned char* blob;
  int blob_bytes, blob_in_smem;
  long long Z;
  int K;
  TapeDev tape;
  double rtol, atol;       // of the recorded burn (its Newton weights)
  const double* lnm;
  int lnm_per_zone;
  const double *gY, *gE, *gT9;
  double *dl, *dY0, *dT0;
  double* ws;
  long long lane_doubles;  // adjoint workspace per lane
  int o_lam, o_ee, o_gr, o_gt, o_mu, o_de, o_seg;
  unsigned long long* queue;
  const int32_t* order;    // claim order (zone per claim), longest first, or null
};

// Reverse-sweep state of one zone.  The steps are taken in blocks of the
// tape's stride C, last block first: steps lo..re of the current block are
// recomputed forward (rs is the next one) from the checkpointed history
// window at record lo - 1, their states kept in the segment buffer, and
// then reversed from s down to lo.
struct AdjZone {
  long long z;
  int s;        // next step to reverse
  int lo, rs, re;
  bool fail;    // a recomputed step did not converge
  Zone fz;      // forward context: rates, density, screening, history ring
};

NB_HD __forceinline__ int ring(int s) { return s % HMAX; }

NB_HD __forceinline__ const double* sched_ptr(const AdjParams& A, long long z, int q) {
  return A.tape.sched + ((size_t)z * A.tape.cap + q) * 2;
}

// state and energy of kept record q
NB_HD __forceinline__ const double* state_ptr(int n, const AdjParams& A, long long z, int q) {
  return A.tape.states + ((size_t)z * A.tape.scap + tape_state_slot(q, A.tape.stride)) * (n + 1);
}

// The adjoint's own arrays of one zone, views of type V (lane-strided for
// one zone per lane, contiguous for one zone per warp)
template <class V>
struct AWST {
  V lam, ee, gr, gt, mu, de, seg;
};
using AWS = AWST<LV>;

template <class V>
NB_HD __forceinline__ AWST<V> make_aws_at(const AdjParams& A, double* base, int stride) {
  AWST<V> a;
  a.lam.p = base + (size_t)A.o_lam * stride;
  a.ee.p = base + (size_t)A.o_ee * stride;
  a.gr.p = base + (size_t)A.o_gr * stride;
  a.gt.p = base + (size_t)A.o_gt * stride;
  a.mu.p = base + (size_t)A.o_mu * stride;
  a.de.p = base + (size_t)A.o_de * stride;
  a.seg.p = base + (size_t)A.o_seg * stride;
  return a;
}

NB_HD __forceinline__ AWS make_aws(const AdjParams& A, double* lane_base) {
  return make_aws_at<LV>(A, lane_base, WS_LANES);
}

// the compiled network of either network type
NB_HD __forceinline__ const Net& net_of(const Net& t) { return t; }
template <class NT>
NB_HD __forceinline__ const Net& net_of(const NT& t) { return t.g; }

// Set up the recomputation of the block holding step s_hi: load its history
// window (records q0, q0-1, .. with q0 = the block's start) from the tape
// into the forward history ring, as the forward burn held it before step
// q0 + 1.
template <class NT, class WT>
NB_HD inline void seg_start(const NT& t, AdjZone& Zs, WT& w, const AdjParams& A, int s_hi) {
  const int C = A.tape.stride;
  const int q0 = (s_hi - 1) / C * C;
  if (C == 1) {   // every state is on the tape: nothing to recompute
    Zs.lo = s_hi;
    Zs.rs = s_hi + 1;
    Zs.re = s_hi;
    return;
  }
  Zone& s = Zs.fz;
  const int nh = q0 + 1 < HMAX ? q0 + 1 : HMAX;
  vsync(t);
  for (int i = 0; i < nh; ++i) {
    const double* st = state_ptr(t.n, A, Zs.z, q0 - i);
    for (int e = vbeg(t); e < t.n; e += vstep(t)) w.xh[i * t.n + e] = st[e];
    if (vlead(t)) {
      w.eh[i] = st[t.n];
      w.th[i] = sched_ptr(A, Zs.z, q0 - i)[0];
    }
  }
  vsync(t);
  s.hh = 0;
  s.nh = nh;
  s.t = w.th[0];
  if (q0 == 0) {
    // f(x0) for the first step's predictor, as the forward start-up forms it
    if (t.sh) eval_rates(t, s, w, t_powers(s.T9f, false, s.scr), s.T9f, false);
    eval_terms(t, w, w.xh);
    eval_f(t, w, w.xh, w.f0);
  }
  Zs.lo = q0 + 1;
  Zs.rs = q0 + 1;
  Zs.re = s_hi;
}

// returns true when the zone needs no reverse steps
template <class NT, class WT, class AT>
NB_HD inline bool adj_init(const NT& t, AdjZone& Zs, WT& w, const AT& a, const AdjParams& A) {
  const long long z = Zs.z;
  const int n = t.n, N = t.N, K = A.K;
  const int st = A.tape.zstat[z];
  const int S = A.tape.steps[z] - 1;
  vsync(t);
  for (int e = vbeg(t); e < HMAX * K * n; e += vstep(t)) a.lam[e] = 0.0;
  for (int e = vbeg(t); e < HMAX * K; e += vstep(t)) a.ee[e] = 0.0;
  for (int e = vbeg(t); e < K * t.R; e += vstep(t)) a.gr[e] = 0.0;
  for (int q = vbeg(t); q < K; q += vstep(t)) a.gt[q] = 0.0;
  Zs.fail = false;
  Zs.s = (st == NB_Z_OK && S >= 0) ? S : -1;
  vsync(t);
  if (Zs.s < 0) return true;
  const int sl = ring(S);
  for (int q = 0; q < K; ++q) {
    const size_t qz = (size_t)q * A.Z + z;
    for (int i = vbeg(t); i < N; i += vstep(t)) a.lam[(sl * K + q) * n + i] = A.gY[qz * N + i];
    if (vlead(t)) {
      if (t.sh) a.lam[(sl * K + q) * n + N] = A.gT9 ? A.gT9[qz] : 0.0;
      a.ee[sl * K + q] = A.gE ? A.gE[qz] : 0.0;
    }
  }
  vsync(t);
  Zone& s = Zs.fz;
  s.z = z;
  s.rho = A.tape.rho[z];
  s.rho2 = s.rho * s.rho;
  s.T9f = A.tape.T9f[z];
  s.scr = A.tape.scr[z];
  s.E = 0.0;
  s.k = 1;
  s.c_acc = s.c_rej_err = s.c_rej_newton = s.c_newton = 0;
  s.c_jac = s.c_rhs = s.c_teval = s.c_edot = s.c_ordsum = 0;
  tab_zone(t, s, state_ptr(n, A, z, 0));   // the recorded initial state
  s.lnm = A.lnm ? (A.lnm_per_zone ? A.lnm + (size_t)z * t.R : A.lnm) : nullptr;
  // fixed temperature: the rates of the whole burn (with their T9 slopes)
  if (!t.sh) eval_rates(t, s, w, t_powers(s.T9f, true, s.scr), s.T9f, true);
  if (S == 0) return true;
  seg_start(t, Zs, w, A, S);
  return false;
}

// Recompute the next step of the current block; false when the zone is done.
template <class NT, class WT, class AT>
NB_HD inline bool adj_replay(const NT& t, AdjZone& Zs, WT& w, const AT& a, const AdjParams& A) {
  const int q = Zs.rs;
  const double* sc = sched_ptr(A, Zs.z, q);
  const int kk = A.tape.ord[(size_t)Zs.z * A.tape.cap + q];
  if (!replay_step(t, Zs.fz, w, A.atol, A.rtol, sc[1], sc[0], kk)) {
    Zs.fail = true;
    return true;
  }
  const int b0 = Zs.fz.hh * t.n;
  const int o = (q - Zs.lo) * t.n;
  for (int e = vbeg(t); e < t.n; e += vstep(t)) a.seg[o + e] = w.xh[b0 + e];
  Zs.rs = q + 1;
  return false;
}

// d edot / dx into a.de (needs w.dt at x): per species, its derivative terms
// in increasing order (the order a scatter over the terms adds them in)
template <class NT, class WT, class AT>
NB_HD __forceinline__ void edot_gradient(const NT& t, const WT& w, const AT& a) {
  const Net& g = net_of(t);
  if constexpr (is_coop<NT>::value) {
    for (int j = vbeg(t); j < t.N; j += vstep(t)) {
      double acc = 0.0;
      for (int e = t.dej_ptr[j]; e < t.dej_ptr[j + 1]; ++e) {
        const int d = t.dej_d[e];
        acc += g.Q[g.dt_r[d]] * w.dt[d];
      }
      a.de[j] = acc;
    }
    if (t.sh) {
      double acc = 0.0;
      for (int r = vbeg(t); r < t.R; r += vstep(t)) acc = fma(g.Q[r], w.dt[g.nd + r], acc);
      acc = vsum(t, acc);
      if (vlead(t)) a.de[t.N] = acc;
    }
  } else {
    for (int i = 0; i < t.n; ++i) a.de[i] = 0.0;
    for (int d = 0; d < g.nd; ++d) a.de[g.dt_j[d]] += g.Q[g.dt_r[d]] * w.dt[d];
    if (t.sh) {
      double acc = 0.0;
      for (int r = 0; r < t.R; ++r) acc = fma(g.Q[r], w.dt[g.nd + r], acc);
      a.de[t.N] = acc;
    }
  }
  vsync(t);
}

// v <- M^-T v with the factored LU of either network type
NB_HD __forceinline__ void solve_MT_of(const Net& t, const LV& lu, const LV& v) {
  tri_solve(t.tfw, t.tfw_s, t.tfw_c, t.n, lu, v);
  tri_solve(t.tbw, t.tbw_s, t.tbw_c, t.n, lu, v);
}
template <class NT, class LUV, class V>
NB_HD __forceinline__ void solve_MT_of(const NT& t, const LUV& lu, const V& v) {
  solve_MT(t, lu, v);
}

// reverse one step; returns true when the zone is done
template <class NT, class WT, class AT>
NB_HD inline bool adj_step(const NT& t, AdjZone& Zs, WT& w, const AT& a, const AdjParams& A) {
  const Net& g = net_of(t);
  const long long z = Zs.z;
  const int n = t.n, N = t.N, K = A.K, s = Zs.s;
  const double* ss = sched_ptr(A, z, s);
  const int kk = A.tape.ord[(size_t)z * A.tape.cap + s];
  const double h = ss[1];
  double tau[KMAX + 1];
  tau[0] = ss[0];
#pragma unroll
  for (int j = 1; j <= KMAX; ++j) tau[j] = (j <= kk) ? sched_ptr(A, z, s - j)[0] : 0.0;
  double alpha[KMAX + 1];
  bdf_alpha(kk, tau, h, alpha);
  const int o = (s - Zs.lo) * n;
  vsync(t);
  if (A.tape.stride == 1) {
    const double* xs = state_ptr(n, A, z, s);
    for (int i = vbeg(t); i < n; i += vstep(t)) w.x[i] = xs[i];
  } else {
    for (int i = vbeg(t); i < n; i += vstep(t)) w.x[i] = a.seg[o + i];
  }
  vsync(t);
  if (t.sh) eval_rates(t, Zs.fz, w, t_powers(w.x[N], true, Zs.fz.scr), w.x[N], true);
  eval_terms(t, w, w.x);
  assemble_M(t, w, w.x, alpha[0], h);
  factor_M(t, w);
  double icv = 0.0;
  if (t.sh) icv = 1.0 / heat_capacity(t, w.x);
  if (t.hasE) edot_gradient(t, w, a);
  const double ia0 = 1.0 / alpha[0];
  const int sl = ring(s);
  int sj[KMAX + 1];
#pragma unroll
  for (int j = 1; j <= KMAX; ++j) sj[j] = ring(s + HMAX - j);
  for (int q = 0; q < K; ++q) {
    const int lo = (sl * K + q) * n;
    const double es = a.ee[sl * K + q];
    const double ce = es * h * ia0;
    for (int i = vbeg(t); i < n; i += vstep(t)) {
      double v = a.lam[lo + i];
      if (t.hasE) v = fma(ce, a.de[i], v);
      a.mu[i] = v;
      a.lam[lo + i] = 0.0;
    }
    vsync(t);
    if (vlead(t)) a.ee[sl * K + q] = 0.0;
    solve_MT_of(t, w.lu, a.mu);
    vsync(t);
#pragma unroll
    for (int j = 1; j <= KMAX; ++j) {
      if (j > kk) continue;
      const int lj = (sj[j] * K + q) * n;
      const double ma = -alpha[j];
      for (int i = vbeg(t); i < n; i += vstep(t)) a.lam[lj + i] = fma(ma, a.mu[i], a.lam[lj + i]);
      if (t.hasE && vlead(t)) a.ee[sj[j] * K + q] = fma(-es * ia0, alpha[j], a.ee[sj[j] * K + q]);
    }
    const double muT = t.sh ? a.mu[N] * icv : 0.0;
    double gt = 0.0;
    for (int r = vbeg(t); r < t.R; r += vstep(t)) {
      double acc = 0.0;
      for (int e = g.rg_ptr[r]; e < g.rg_ptr[r + 1]; ++e)
        acc = fma(g.rg_c[e], a.mu[g.rg_i[e]], acc);
      const double Qr = g.Q[r];
      acc = fma(muT, Qr, acc);
      const double v = w.rr[r] * fma(h, acc, ce * Qr);
      a.gr[q * t.R + r] += v;
      if (!t.sh) gt = fma(v, w.g[r], gt);
    }
    gt = vsum(t, gt);
    if (vlead(t)) a.gt[q] += gt;
    vsync(t);
  }
  Zs.s = s - 1;
  if (Zs.s == 0) return true;
  if (Zs.s < Zs.lo) seg_start(t, Zs, w, A, Zs.s);
  return false;
}

template <class NT, class AT>
NB_HD inline void adj_finish(const NT& t, const AdjZone& Zs, const AT& a, const AdjParams& A) {
  const long long z = Zs.z;
  const int n = t.n, N = t.N, K = A.K;
  const bool ok = Zs.s == 0 && !Zs.fail;
  // a failed recomputation is reported as NaN; a zone the forward burn did
  // not finish gets zero gradients
  const double bad = Zs.fail ? quiet_nan() : 0.0;
  const int s0 = ring(0);
  vsync(t);
  for (int q = 0; q < K; ++q) {
    const size_t qz = (size_t)q * A.Z + z;
    for (int r = vbeg(t); r < t.R; r += vstep(t)) A.dl[qz * t.R + r] = ok ? a.gr[q * t.R + r] : bad;
    if (A.dY0)
      for (int i = vbeg(t); i < N; i += vstep(t))
        A.dY0[qz * N + i] = ok ? a.lam[(s0 * K + q) * n + i] : bad;
    if (A.dT0 && vlead(t)) A.dT0[qz] = ok ? (t.sh ? a.lam[(s0 * K + q) * n + N] : a.gt[q]) : bad;
  }
}

}  // namespace nb
