// coop.cuh -- one zone per warp (or per block of two or four warps, see
// WNetT): the network evaluation of the integrator (integrator.cuh) spread
// over the team's threads, for large networks.
//
// On this GPU an FP64 warp instruction costs the FP64 pipe the same time
// whatever its active lanes, so one lane per zone keeps the pipe busiest
// while a zone's work is small.  A 48- or 128-species network is not small:
// its LU alone holds 1,300 or 8,900 slots and its per-lane work arrays (26
// or 119 KB) overflow the L2 once the GPU's lanes are all in flight, so the
// lane-per-zone kernel waits on memory.  Here a warp integrates one zone:
//  * its Newton-loop arrays (LU slots, rates, terms, derivatives, state
//    vectors) sit in shared memory, contiguous per warp; the BDF history in
//    global memory;
//  * loops over reactions, derivative terms, Jacobian slots and species are
//    spread over the lanes;
//  * the LU keeps the static pivot order: per pivot the lanes scale the L
//    column, then update the |L| x |U| pairs of the trailing matrix, which
//    are independent (93 % and 99 % of the lanes busy on the 48- and
//    128-species networks); each slot sees the lane kernel's operations in
//    the same order, so the factors are the lane kernel's bits;
//  * the triangular solves go column by column (a pivot's L column, or U's
//    column, updated by the lanes), sums are warp reductions: those round
//    differently from the lane kernel's row-wise gathers.
// Every lane holds the zone's scalars (time, step, order, counters) and
// computes them identically, so branches are uniform across the warp.
#pragma once
#include "device.cuh"
#include "integrator.cuh"

namespace nb {

constexpr unsigned kFullMask = 0xffffffffu;

// The compiled network seen by one of the W threads that own a zone: a warp
// (W = 32), or a block of two or four warps (W = 64, 128) for networks whose
// per-pivot work fills more lanes than a warp has.  A team larger than a
// warp is one whole block, so its barrier is the block's.
template <int W>
struct WNetT {
  static constexpr int width = W;
  Net g;
  int n, N, R, sh, hasE;
  double inv_n;
  int lane;   // 0 .. W-1
  const int16_t *perm, *ltgt, *ucol_s, *ucol_t, *utgt, *lrow_s, *lrow_t, *dej_d;
  const int32_t *ucol_ptr, *lrow_ptr, *dej_ptr;
  // W > 32: two alternating rows of W/32 partial sums and a broadcast slot
  // in shared memory
  double* red;
  mutable int ph;
  // sum over the team, the same bits in every thread: an xor butterfly in
  // each warp (it adds the same two operands in both lanes of each pair),
  // then the warps' sums added in warp order
  __device__ __forceinline__ double sum(double x) const {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) x += __shfl_xor_sync(kFullMask, x, m);
    if constexpr (W > 32) {
      double* row = red + ph * (W / 32);
      ph ^= 1;
      if ((lane & 31) == 0) row[lane >> 5] = x;
      __syncthreads();
      x = row[0];
#pragma unroll
      for (int q = 1; q < W / 32; ++q) x += row[q];
    }
    return x;
  }
  __device__ __forceinline__ bool all(bool b) const {
    if constexpr (W > 32) return __syncthreads_and(b) != 0;
    else return __all_sync(kFullMask, b);
  }
  __device__ __forceinline__ void sync() const {
    if constexpr (W > 32) __syncthreads();
    else __syncwarp();
  }
  // thread 0's value in every thread of the team
  __device__ __forceinline__ unsigned long long bcast(unsigned long long v) const {
    if constexpr (W > 32) {
      unsigned long long* slot = reinterpret_cast<unsigned long long*>(red + 2 * (W / 32));
      __syncthreads();
      if (lane == 0) *slot = v;
      __syncthreads();
      return *slot;
    } else {
      return __shfl_sync(kFullMask, v, 0);
    }
  }
};
using WNet = WNetT<32>;

// shared-memory doubles a team of W threads needs for its sums and broadcasts
constexpr int team_scratch_doubles(int W) { return W > 32 ? 2 * (W / 32) + 1 : 0; }

template <int W>
struct is_coop<WNetT<W>> {
  static constexpr bool value = true;
};

template <int W>
__device__ __forceinline__ WNetT<W> make_wnet(const unsigned char* blob, int lane,
                                              double* red = nullptr) {
  WNetT<W> t;
  t.g = make_net(blob);
  t.n = t.g.n; t.N = t.g.N; t.R = t.g.R; t.sh = t.g.sh; t.hasE = t.g.hasE;
  t.inv_n = t.g.inv_n;
  t.lane = lane;
  t.red = red;
  t.ph = 0;
  const BlobHeader* h = reinterpret_cast<const BlobHeader*>(blob);
  t.perm = at<int16_t>(blob, h->o_perm);
  t.ltgt = at<int16_t>(blob, h->o_ltgt);
  t.ucol_ptr = at<int32_t>(blob, h->o_ucol_ptr);
  t.ucol_s = at<int16_t>(blob, h->o_ucol_s);
  t.ucol_t = at<int16_t>(blob, h->o_ucol_t);
  t.utgt = at<int16_t>(blob, h->o_utgt);
  t.lrow_ptr = at<int32_t>(blob, h->o_lrow_ptr);
  t.lrow_s = at<int16_t>(blob, h->o_lrow_s);
  t.lrow_t = at<int16_t>(blob, h->o_lrow_t);
  t.dej_ptr = at<int32_t>(blob, h->o_dej_ptr);
  t.dej_d = at<int16_t>(blob, h->o_dej_d);
  return t;
}

// contiguous view of one of the warp's arrays
struct CV {
  double* p;
  __device__ __forceinline__ double& operator[](int i) const { return p[i]; }
};

struct CWS {
  CV x, xp, psi, d, f, iw, tmp, f0, xh, eh, th, k, g, rr, kp, dt, lu;
};

// The warp's arrays: the Newton-loop ("hot") part of the compiled layout at
// hot, the history and start-up part at cold (offsets past hot_doubles).
__device__ __forceinline__ CWS make_cws(const Net& t, double* hot, double* cold) {
  CWS w;
  w.x.p = hot + t.w_x; w.xp.p = hot + t.w_xp; w.psi.p = hot + t.w_psi;
  w.d.p = hot + t.w_d; w.f.p = hot + t.w_f; w.iw.p = hot + t.w_iw;
  w.k.p = hot + t.w_k; w.rr.p = hot + t.w_rr;
  w.dt.p = hot + t.w_dt; w.lu.p = hot + t.w_lu;
  // g and kp sit with the cold part at fixed temperature
  w.g.p = t.w_g < t.hot_doubles ? hot + t.w_g : cold + (t.w_g - t.hot_doubles);
  w.kp.p = t.w_kp < t.hot_doubles ? hot + t.w_kp : cold + (t.w_kp - t.hot_doubles);
  w.tmp.p = cold + (t.w_tmp - t.hot_doubles);
  w.f0.p = cold + (t.w_f0 - t.hot_doubles);
  w.xh.p = cold + (t.w_xh - t.hot_doubles);
  w.eh.p = cold + (t.w_eh - t.hot_doubles);
  w.th.p = cold + (t.w_th - t.hot_doubles);
  return w;
}

// ---------------------------------------------------------------- model

template <int W>
__device__ __forceinline__ void eval_rates(const WNetT<W>& t, const Zone& s, const CWS& w,
                                           const TPow& p, double T9, bool with_g) {
  t.sync();
  const Net& g = t.g;
  const TCell tc = g.tab_of ? t_cell(g.tab_t9, g.tab_nt, T9) : TCell{0, 0.0, 1.0, false};
  for (int r = t.lane; r < t.R; r += W) {
    double gr;
    w.k[r] = rate_full(g, s, r, p, T9, tc, with_g ? &gr : nullptr);
    if (with_g) w.g[r] = gr;
  }
  t.sync();
}

template <int W>
__device__ __forceinline__ void save_ref_rates(const WNetT<W>& t, const CWS& w) {
  for (int r = t.lane; r < t.R; r += W) w.kp[r] = w.k[r];
  t.sync();
}

template <int W>
__device__ __forceinline__ void eval_rates_near(const WNetT<W>& t, const Zone& s, const CWS& w,
                                                double T9, const TPow& ref, double T9ref) {
  t.sync();
  const Net& g = t.g;
  DPhi d;
  TPow p;
  bool have_p = !delta_phi_series(ref, T9, T9ref, d);
  if (have_p) {
    p = t_powers(T9, false, s.scr);
    d = delta_phi(p, ref, T9, T9ref);
  }
  const TCell tc = g.tab_of ? t_cell(g.tab_t9, g.tab_nt, T9) : TCell{0, 0.0, 1.0, false};
  for (int r = t.lane; r < t.R; r += W) {
    const double* a = g.coef + 7 * r;
    double de = rate_delta(a[1], a[2], a[3], a[4], a[5], a[6], d);
    if (g.scr) de = fma(g.scr[r], d.d7, de);
    if (g.ap[r] < 0 && !(g.tab_of && g.tab_of[r] >= 0) && small_delta(de)) {
      w.k[r] = rate_near(w.kp[r], de);
    } else {
      if (!have_p) {
        p = t_powers(T9, false, s.scr);
        have_p = true;
      }
      w.k[r] = rate_full(g, s, r, p, T9, tc, nullptr);
    }
  }
  t.sync();
}

// the zone's density cell of the rate tables (every lane, the same sum)
template <int W, class V>
__device__ __forceinline__ void tab_zone(const WNetT<W>& t, Zone& s, const V& x0) {
  t.sync();
  tab_zone(t.g, s, x0);
}

template <int W>
__device__ __forceinline__ void eval_terms(const WNetT<W>& t, const CWS& w, const CV& v) {
  t.sync();
  const Net& g = t.g;
  for (int r = t.lane; r < t.R; r += W) {
    const int16_t* ra = g.reac + 3 * r;
    const int m = g.nreac[r];
    double q = w.k[r];
    q *= v[ra[0]];
    if (m > 1) q *= v[ra[1]];
    if (m > 2) q *= v[ra[2]];
    w.rr[r] = q;
  }
  t.sync();
}

// sum_r Q_r rr_r, the same value in every lane
template <int W>
__device__ __forceinline__ double eval_edot(const WNetT<W>& t, const CWS& w) {
  double e = 0.0;
  for (int r = t.lane; r < t.R; r += W) e = fma(t.g.Q[r], w.rr[r], e);
  return t.sum(e);
}

// sum_e c[e] v[idx[e]] over [beg, end)
template <class TI, class V>
__device__ __forceinline__ double gather(const double* c, const TI* idx, int beg, int end,
                                         const V& v) {
  double a0 = 0.0, a1 = 0.0;
  int e = beg;
  for (; e + 1 < end; e += 2) {
    a0 = fma(c[e], v[idx[e]], a0);
    a1 = fma(c[e + 1], v[idx[e + 1]], a1);
  }
  if (e < end) a0 = fma(c[e], v[idx[e]], a0);
  return a0 + a1;
}

template <int W>
__device__ __forceinline__ void eval_f(const WNetT<W>& t, const CWS& w, const CV& v, const CV& out) {
  t.sync();
  const Net& g = t.g;
  for (int i = t.lane; i < t.N; i += W)
    out[i] = gather(g.rhs_c, g.rhs_r, g.rhs_ptr[i], g.rhs_ptr[i + 1], w.rr);
  if (t.sh) {
    const double fT = eval_edot(t, w) / heat_capacity(t, v);
    if (t.lane == 0) out[t.N] = fT;
  }
  t.sync();
}

// M = alpha0 I - h J(v) into w.lu (needs w.k, w.g (self-heating), w.rr at v)
template <int W>
__device__ __forceinline__ void assemble_M(const WNetT<W>& t, const CWS& w, const CV& v,
                                           double alpha0, double h) {
  t.sync();
  const Net& g = t.g;
  for (int d = t.lane; d < g.nd; d += W) {
    const int16_t o0 = g.dt_o[2 * d], o1 = g.dt_o[2 * d + 1];
    double q = w.k[g.dt_r[d]] * g.dt_m[d];
    if (o0 >= 0) q *= v[o0];
    if (o1 >= 0) q *= v[o1];
    w.dt[d] = q;
  }
  TRow tr{0.0, 0.0, 0.0};
  if (t.sh) {
    for (int r = t.lane; r < t.R; r += W) w.dt[g.nd + r] = w.rr[r] * w.g[r];
    tr = t_row(eval_edot(t, w), heat_capacity(t, v), v[t.N]);
  }
  t.sync();
  const double mh = -h;
  for (int s = t.lane; s < g.nnz; s += W) {
    double acc = gather(g.js_c, g.js_src, g.js_ptr[s], g.js_ptr[s + 1], w.dt);
    const uint8_t fl = g.js_flag[s];
    if (fl & SLOT_TROW) acc = fma(acc, tr.a1, tr.b1);
    else if (fl & SLOT_TT) acc = fma(acc, tr.a1, tr.b2);
    double m = mh * acc;
    if (fl & SLOT_DIAG) m += alpha0;
    w.lu[s] = m;
  }
  t.sync();
}

// Static-pivot LU in place, the diagonal keeping 1/pivot; the lane
// kernel's operations slot by slot.  false if a pivot is zero, not finite
// or eaten by cancellation (pivot_kept).
template <int W>
__device__ __forceinline__ bool factor_M(const WNetT<W>& t, const CWS& w) {
  t.sync();
  const Net& g = t.g;
  for (int k = t.lane; k < t.n; k += W) w.tmp[k] = w.lu[g.piv[k].dslot];
  t.sync();
  bool ok = true;
  for (int k = 0; k < t.n; ++k) {
    const Pivot p = g.piv[k];
    const double pv = w.lu[p.dslot];
    ok = ok && pivot_kept(pv, w.tmp[k]);
    const double inv = recip2(pv);
    const int nl = p.lend - p.lbeg, nu = p.uend - p.ubeg;
    for (int li = p.lbeg + t.lane; li < p.lend; li += W) {
      const int ls = g.lslot[li];
      w.lu[ls] = w.lu[ls] * inv;
    }
    t.sync();
    if (t.lane == 0) w.lu[p.dslot] = inv;
    const int np = nl * nu;
    if (np > 0) {
      // pair e = li * nu + u, walked in steps of W without a division per pair
      const int qW = W / nu, rW = W - qW * nu;
      int li = t.lane / nu, u = t.lane - li * nu;
      for (int e = t.lane; e < np; e += W) {
        const int ds = g.dslot[p.dbeg + e];
        const double l = w.lu[g.lslot[p.lbeg + li]];
        w.lu[ds] = fma(-l, w.lu[g.uslot[p.ubeg + u]], w.lu[ds]);
        li += qW;
        u += rW;
        if (u >= nu) { u -= nu; ++li; }
      }
    }
    t.sync();
  }
  return ok;
}

// v <- M^-1 v with the factored w.lu: L column by column, then U column by
// column from the last
template <int W>
__device__ __forceinline__ void solve_M(const WNetT<W>& t, const CWS& w, const CV& v) {
  t.sync();
  const Net& g = t.g;
  for (int k = 0; k < t.n; ++k) {
    const Pivot p = g.piv[k];
    const double vk = v[t.perm[k]];
    for (int li = p.lbeg + t.lane; li < p.lend; li += W) {
      const int r = t.ltgt[li];
      v[r] = fma(-w.lu[g.lslot[li]], vk, v[r]);
    }
    t.sync();
  }
  for (int k = t.n - 1; k >= 0; --k) {
    const int pk = t.perm[k];
    const double xk = v[pk] * w.lu[g.piv[k].dslot];
    for (int e = t.ucol_ptr[k] + t.lane; e < t.ucol_ptr[k + 1]; e += W) {
      const int r = t.ucol_t[e];
      v[r] = fma(-w.lu[t.ucol_s[e]], xk, v[r]);
    }
    t.sync();
    // every thread has read v[pk]; no later column reads or updates it
    // (their targets lie above them in the pivot order)
    if (t.lane == 0) v[pk] = xk;
  }
  t.sync();
}

// v <- M^-T v with the factored w.lu (the adjoint): U^T column by column
// (pivot rows of U), then L^T column by column from the last (rows of L)
template <int W, class V>
__device__ __forceinline__ void solve_MT(const WNetT<W>& t, const CV& lu, const V& v) {
  t.sync();
  const Net& g = t.g;
  for (int k = 0; k < t.n; ++k) {
    const Pivot p = g.piv[k];
    const int pk = t.perm[k];
    const double xk = v[pk] * lu[p.dslot];
    for (int u = p.ubeg + t.lane; u < p.uend; u += W) {
      const int r = t.utgt[u];
      v[r] = fma(-lu[g.uslot[u]], xk, v[r]);
    }
    t.sync();
    // every thread has read v[pk]; no later row reads or updates it (their
    // targets lie below them in the pivot order)
    if (t.lane == 0) v[pk] = xk;
  }
  t.sync();
  for (int k = t.n - 1; k >= 0; --k) {
    const double xk = v[t.perm[k]];
    for (int e = t.lrow_ptr[k] + t.lane; e < t.lrow_ptr[k + 1]; e += W) {
      const int r = t.lrow_t[e];
      v[r] = fma(-lu[t.lrow_s[e]], xk, v[r]);
    }
    t.sync();
  }
}

// ---------------------------------------------------------------- claim loop

// One zone per warp: lane 0 claims zones from the device queue and every
// lane of the warp integrates it.  The watchdog reads lane 0's clock, so the
// warp decides as one.
template <int W, class WT>
__device__ __forceinline__ void coop_claim_loop(const WNetT<W>& t, WT& w, const BurnParams& P) {
  unsigned long long t_start = 0ull;
  if (P.budget_ns) t_start = t.bcast(t.lane == 0 ? gpu_ns() : 0ull);
  auto expired = [&]() {
    if (!P.budget_ns) return false;
    const unsigned long long now = t.bcast(t.lane == 0 ? gpu_ns() : 0ull);
    return now - t_start > P.budget_ns;
  };
  for (;;) {
    unsigned long long c = 0;
    if (t.lane == 0) c = atomicAdd(P.queue, 1ull);
    c = t.bcast(c);
    if (c >= (unsigned long long)P.Z) break;
    Zone s;
    s.z = P.order ? (long long)P.order[c] : (long long)c;
    if (expired()) {
      zone_timeout_unstarted(t, s.z, P);
      continue;
    }
    bool done = zone_init(t, s, w, P);
    while (!done) {
      if (expired()) {
        s.status = NB_Z_TIMEOUT;
        break;
      }
      done = zone_attempt(t, s, w, P);
    }
    zone_finish(t, s, w, P);
    t.sync();
  }
}

}  // namespace nb
