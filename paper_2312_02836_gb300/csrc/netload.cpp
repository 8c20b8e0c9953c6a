// netload.cpp -- host-side compilation of a reaction network into the blob
// the kernels walk (see blob.h).
//
// The paper's pynucastro writes a network-specific RHS and analytic Jacobian
// as C++ source (arXiv:2312.02836 Sec. 2, "write_network").  Here the same
// information is compiled at load time into data instead of code: gather
// lists for the right-hand side and for every Jacobian entry, a minimum-degree
// elimination order, the symbolic LU fill of alpha0 I - h J under static
// diagonal pivots, and gather programs for the triangular solves (and their
// transposes for the adjoint).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "blob.h"
#include "../../include/netburn.h"

namespace nb {

namespace {

struct Builder {
  std::vector<uint8_t> buf;
  int32_t add(const void* p, size_t bytes) {
    size_t off = (buf.size() + 15) & ~size_t(15);
    buf.resize(off + ((bytes + 15) & ~size_t(15)), 0);
    if (bytes) std::memcpy(buf.data() + off, p, bytes);
    return (int32_t)off;
  }
  template <class T>
  int32_t add(const std::vector<T>& v) {
    return add(v.data(), v.size() * sizeof(T));
  }
};

}  // namespace

// Minimum-degree order on the symmetrised pattern (ties: lowest index).
static std::vector<int> min_degree_order(int n, const std::vector<std::vector<char>>& P) {
  std::vector<std::vector<char>> G(n, std::vector<char>(n, 0));
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (i != j && (P[i][j] || P[j][i])) G[i][j] = 1;
  std::vector<char> done(n, 0);
  std::vector<int> order;
  for (int step = 0; step < n; ++step) {
    int best = -1, bestdeg = 1 << 30;
    for (int v = 0; v < n; ++v) {
      if (done[v]) continue;
      int d = 0;
      for (int u = 0; u < n; ++u) d += (!done[u] && G[v][u]);
      if (d < bestdeg) { bestdeg = d; best = v; }
    }
    order.push_back(best);
    done[best] = 1;
    std::vector<int> nb_;
    for (int u = 0; u < n; ++u)
      if (!done[u] && G[best][u]) nb_.push_back(u);
    for (int a : nb_)
      for (int b : nb_)
        if (a != b) G[a][b] = 1;
  }
  return order;
}

int build_blob(const nb_topology* T, const double* coeffs,
               std::vector<uint8_t>* out, BlobHeader* hdr_out) {
  const int N = T->n_species, R = T->n_reactions;
  const int sh = T->self_heating ? 1 : 0;
  const int n = N + sh;
  const int hasE = T->Q != nullptr;
  if (n > 4096 || R > 32767) return NB_E_TOO_LARGE;

  // reactant occurrences (compacted) and stoichiometry
  std::vector<int16_t> reac(3 * R, -1);
  std::vector<int32_t> nreac(R), nrho(R);
  std::vector<std::map<int, double>> stoich(R);  // species -> c_ir
  for (int r = 0; r < R; ++r) {
    int m = 0;
    for (int s = 0; s < 3; ++s) {
      int j = T->reactants[3 * r + s];
      if (j < 0) continue;
      reac[3 * r + m++] = (int16_t)j;
      stoich[r][j] -= 1.0;
    }
    for (int s = 0; s < 3; ++s) {
      int j = T->products[3 * r + s];
      if (j >= 0) stoich[r][j] += 1.0;
    }
    nreac[r] = m;
    nrho[r] = m - 1;
    for (auto it = stoich[r].begin(); it != stoich[r].end();)
      it = it->second == 0.0 ? stoich[r].erase(it) : std::next(it);
  }

  // RHS gather: f_i = sum_r c_ir R_r, in reaction order
  std::vector<int32_t> rhs_ptr(N + 1, 0);
  std::vector<int16_t> rhs_r;
  std::vector<double> rhs_c;
  for (int i = 0; i < N; ++i) {
    for (int r = 0; r < R; ++r) {
      auto it = stoich[r].find(i);
      if (it != stoich[r].end()) {
        rhs_r.push_back((int16_t)r);
        rhs_c.push_back(it->second);
      }
    }
    rhs_ptr[i + 1] = (int32_t)rhs_r.size();
  }

  // derivative terms dR_r/dY_j = k_r m_j prod(remaining occurrences)
  std::vector<int16_t> dt_r, dt_o, dt_j;
  std::vector<double> dt_m;
  std::vector<std::vector<int>> dterms_of_r(R);
  for (int r = 0; r < R; ++r) {
    std::vector<int> seen;
    for (int s = 0; s < nreac[r]; ++s) {
      int j = reac[3 * r + s];
      if (std::find(seen.begin(), seen.end(), j) != seen.end()) continue;
      seen.push_back(j);
      int m = 0;
      for (int q = 0; q < nreac[r]; ++q) m += reac[3 * r + q] == j;
      int16_t o[2] = {-1, -1};
      int no = 0, skipped = 0;
      for (int q = 0; q < nreac[r]; ++q) {
        int l = reac[3 * r + q];
        if (l == j && !skipped) { skipped = 1; continue; }
        o[no++] = (int16_t)l;
      }
      dterms_of_r[r].push_back((int)dt_r.size());
      dt_r.push_back((int16_t)r);
      dt_o.push_back(o[0]);
      dt_o.push_back(o[1]);
      dt_m.push_back((double)m);
      dt_j.push_back((int16_t)j);
    }
  }
  const int nd = (int)dt_r.size();
  if (nd + R > 32767) return NB_E_TOO_LARGE;

  // structural pattern of M = alpha0 I - h J (original indices)
  std::vector<std::vector<char>> P(n, std::vector<char>(n, 0));
  for (int i = 0; i < n; ++i) P[i][i] = 1;
  for (int r = 0; r < R; ++r)
    for (auto& kv : stoich[r])
      for (int d : dterms_of_r[r]) P[kv.first][dt_j[d]] = 1;
  if (sh) {
    for (int r = 0; r < R; ++r)
      for (auto& kv : stoich[r]) P[kv.first][N] = 1;   // T column
    for (int j = 0; j <= N; ++j) P[N][j] = 1;          // T row (c_v term)
  }
  int nnz_jac = 0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) nnz_jac += P[i][j];

  // elimination order and fill (position space)
  std::vector<int> perm = min_degree_order(n, P);  // position -> original
  std::vector<int> pos(n);
  for (int k = 0; k < n; ++k) pos[perm[k]] = k;
  std::vector<std::vector<char>> F(n, std::vector<char>(n, 0));
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (P[i][j]) F[pos[i]][pos[j]] = 1;
  for (int k = 0; k < n; ++k)
    for (int i = k + 1; i < n; ++i)
      if (F[i][k])
        for (int j = k + 1; j < n; ++j)
          if (F[k][j]) F[i][j] = 1;
  std::vector<std::vector<int>> slot(n, std::vector<int>(n, -1));
  int nnz = 0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (F[i][j]) slot[i][j] = nnz++;
  // the pre-ordered LU may fill M's pattern to at most 4 times its nonzeros
  if (nnz > 32767 || nnz > 4 * nnz_jac) return NB_E_TOO_LARGE;

  // Jacobian gather per slot; sources: dterm d (index d) or R_r g_r (nd + r)
  std::vector<int32_t> js_ptr(nnz + 1, 0);
  std::vector<int16_t> js_src;
  std::vector<double> js_c;
  std::vector<uint8_t> js_flag(nnz, 0);
  {
    int s = 0;
    for (int pi = 0; pi < n; ++pi)
      for (int pj = 0; pj < n; ++pj) {
        if (!F[pi][pj]) continue;
        int i = perm[pi], j = perm[pj];
        uint8_t fl = (i == j) ? SLOT_DIAG : 0;
        if (i < N && j < N) {
          for (int r = 0; r < R; ++r) {
            auto it = stoich[r].find(i);
            if (it == stoich[r].end()) continue;
            for (int d : dterms_of_r[r])
              if (dt_j[d] == j) { js_src.push_back((int16_t)d); js_c.push_back(it->second); }
          }
        } else if (i < N && j == N) {
          for (int r = 0; r < R; ++r) {
            auto it = stoich[r].find(i);
            if (it != stoich[r].end()) { js_src.push_back((int16_t)(nd + r)); js_c.push_back(it->second); }
          }
        } else if (i == N && j < N) {
          fl |= SLOT_TROW;
          for (int r = 0; r < R; ++r)
            for (int d : dterms_of_r[r])
              if (dt_j[d] == j) { js_src.push_back((int16_t)d); js_c.push_back(T->Q[r]); }
        } else {  // (T, T)
          fl |= SLOT_TT;
          for (int r = 0; r < R; ++r) { js_src.push_back((int16_t)(nd + r)); js_c.push_back(T->Q[r]); }
        }
        js_flag[s] = fl;
        js_ptr[++s] = (int32_t)js_src.size();
      }
  }

  // LU program
  std::vector<Pivot> piv(n);
  std::vector<int16_t> lslot, uslot, dslot;
  for (int k = 0; k < n; ++k) {
    Pivot p;
    p.dslot = slot[k][k];
    p.lbeg = (int32_t)lslot.size();
    std::vector<int> L, U;
    for (int i = k + 1; i < n; ++i) if (F[i][k]) L.push_back(i);
    for (int j = k + 1; j < n; ++j) if (F[k][j]) U.push_back(j);
    for (int i : L) lslot.push_back((int16_t)slot[i][k]);
    p.lend = (int32_t)lslot.size();
    p.ubeg = (int32_t)uslot.size();
    for (int j : U) uslot.push_back((int16_t)slot[k][j]);
    p.uend = (int32_t)uslot.size();
    p.dbeg = (int32_t)dslot.size();
    for (int i : L)
      for (int j : U) dslot.push_back((int16_t)slot[i][j]);
    piv[k] = p;
  }

  // triangular gather programs (vectors stay in original index order)
  auto tri = [&](bool forward, bool transposed, bool unit, std::vector<TriRow>* rows,
                 std::vector<int16_t>* es, std::vector<int16_t>* ec) {
    for (int step = 0; step < n; ++step) {
      int k = forward ? step : n - 1 - step;
      TriRow tr;
      tr.tgt = perm[k];
      tr.beg = (int32_t)es->size();
      for (int j = 0; j < n; ++j) {
        bool use = forward ? j < k : j > k;
        if (!use) continue;
        int a = transposed ? j : k, b = transposed ? k : j;  // entry (a, b)
        if (!F[a][b]) continue;
        es->push_back((int16_t)slot[a][b]);
        ec->push_back((int16_t)perm[j]);
      }
      tr.end = (int32_t)es->size();
      tr.dslot = unit ? -1 : slot[k][k];
      rows->push_back(tr);
    }
  };
  std::vector<TriRow> fw, bw, tfw, tbw;
  std::vector<int16_t> fw_s, fw_c, bw_s, bw_c, tfw_s, tfw_c, tbw_s, tbw_c;
  tri(true, false, true, &fw, &fw_s, &fw_c);      // L y = b
  tri(false, false, false, &bw, &bw_s, &bw_c);    // U z = y
  tri(true, true, false, &tfw, &tfw_s, &tfw_c);   // U^T v = w
  tri(false, true, true, &tbw, &tbw_s, &tbw_c);   // L^T u = v
  std::vector<int32_t> diag_orig(n);
  for (int i = 0; i < n; ++i) diag_orig[i] = slot[pos[i]][pos[i]];
  // column-oriented solves: rows of the L entries, and U by columns
  std::vector<int16_t> perm16(n), ltgt, ucol_s, ucol_t;
  std::vector<int32_t> ucol_ptr(n + 1, 0);
  for (int k = 0; k < n; ++k) perm16[k] = (int16_t)perm[k];
  for (int k = 0; k < n; ++k)
    for (int i = k + 1; i < n; ++i)
      if (F[i][k]) ltgt.push_back((int16_t)perm[i]);
  for (int k = 0; k < n; ++k) {
    for (int i = 0; i < k; ++i)
      if (F[i][k]) { ucol_s.push_back((int16_t)slot[i][k]); ucol_t.push_back((int16_t)perm[i]); }
    ucol_ptr[k + 1] = (int32_t)ucol_s.size();
  }
  // transposed solves: the columns of the U entries (pivot rows), L by rows
  std::vector<int16_t> utgt, lrow_s, lrow_t;
  std::vector<int32_t> lrow_ptr(n + 1, 0);
  for (int k = 0; k < n; ++k)
    for (int j = k + 1; j < n; ++j)
      if (F[k][j]) utgt.push_back((int16_t)perm[j]);
  for (int k = 0; k < n; ++k) {
    for (int i = 0; i < k; ++i)
      if (F[k][i]) { lrow_s.push_back((int16_t)slot[k][i]); lrow_t.push_back((int16_t)perm[i]); }
    lrow_ptr[k + 1] = (int32_t)lrow_s.size();
  }

  // adjoint: species entries of each rate, d f_i / d p_r = c_ir R_r
  std::vector<int32_t> rg_ptr(R + 1, 0);
  std::vector<int16_t> rg_i;
  std::vector<double> rg_c;
  for (int r = 0; r < R; ++r) {
    for (auto& kv : stoich[r]) { rg_i.push_back((int16_t)kv.first); rg_c.push_back(kv.second); }
    rg_ptr[r + 1] = (int32_t)rg_i.size();
  }

  std::vector<double> coef(coeffs, coeffs + 7 * (size_t)R);
  // effective (alpha,p)(p,gamma) rates: their three extra fits, one row each
  std::vector<int32_t> ap(R, -1);
  std::vector<double> apc;
  if (T->ap_pg) {
    if (!T->ap_coeffs) return NB_E_ARG;
    for (int r = 0; r < R; ++r) {
      if (T->ap_pg[r] == 0) continue;
      if (T->ap_pg[r] != 1) return NB_E_ARG;
      const double* b = T->ap_coeffs + 21 * (size_t)r;
      for (int j = 0; j < 21; ++j)
        if (!std::isfinite(b[j])) return NB_E_ARG;
      ap[r] = (int32_t)(apc.size() / 21);
      apc.insert(apc.end(), b, b + 21);
    }
  }
  const int n_ap = (int)(apc.size() / 21);
  // tabulated rates: validate and copy the grid, the tables and the charges
  std::vector<int32_t> tab_of(R > 0 ? R : 1, -1);
  std::vector<double> tab_dens(1, 0.0), tab_t9(1, 0.0), tab_lnl(1, 0.0), charge(1, 0.0);
  int n_tab = 0, n_tabr = 0;
  if (T->tab_of) {
    const int nd = T->tab_nd, nt = T->tab_nt;
    if (nd < 2 || nt < 2 || nd > 4096 || nt > 4096 || !T->tab_dens || !T->tab_t9 ||
        !T->tab_lnl || !T->charge)
      return NB_E_ARG;
    for (int r = 0; r < R; ++r) {
      const int tb = T->tab_of[r];
      if (tb < -1) return NB_E_ARG;
      if (tb >= 0 && T->ap_pg && T->ap_pg[r]) return NB_E_ARG;   // tabulated or effective
      n_tab = std::max(n_tab, tb + 1);
      n_tabr += tb >= 0;
      tab_of[r] = tb;
    }
    tab_dens.assign(T->tab_dens, T->tab_dens + nd);
    tab_t9.assign(T->tab_t9, T->tab_t9 + nt);
    for (int a = 0; a + 1 < nd; ++a)
      if (!(tab_dens[a + 1] > tab_dens[a])) return NB_E_ARG;
    for (int a = 0; a + 1 < nt; ++a)
      if (!(tab_t9[a + 1] > tab_t9[a])) return NB_E_ARG;
    for (double v : tab_dens) if (!std::isfinite(v)) return NB_E_ARG;
    for (double v : tab_t9) if (!std::isfinite(v)) return NB_E_ARG;
    tab_lnl.assign(T->tab_lnl, T->tab_lnl + (size_t)std::max(n_tab, 1) * nd * nt);
    if (n_tab == 0) tab_lnl.assign(1, 0.0);
    for (double v : tab_lnl) if (!std::isfinite(v)) return NB_E_ARG;
    charge.assign(T->charge, T->charge + N);
    for (double v : charge) if (!std::isfinite(v)) return NB_E_ARG;
  }
  std::vector<double> scr(R > 0 ? R : 1, 0.0);
  if (T->screen)
    for (int r = 0; r < R; ++r) {
      if (!std::isfinite(T->screen[r]) || T->screen[r] < 0.0) return NB_E_ARG;
      scr[r] = T->screen[r];
    }
  if (apc.empty()) apc.push_back(0.0);
  std::vector<double> Q(R, 0.0), scale(R, 1.0);
  for (int r = 0; r < R; ++r) {
    if (T->Q) Q[r] = T->Q[r];
    if (T->scale) scale[r] = T->scale[r];
  }

  BlobHeader h;
  std::memset(&h, 0, sizeof(h));
  Builder B;
  B.add(&h, sizeof(h));  // placeholder
  h.n = n; h.N = N; h.R = R; h.self_heating = sh; h.has_E = hasE;
  h.nnz = nnz; h.nd = nd; h.nnz_jac = nnz_jac;
  h.o_coef = B.add(coef);
  h.o_ap = B.add(ap);
  h.o_apc = B.add(apc);
  h.n_ap = n_ap;
  h.o_scr = B.add(scr);
  h.has_scr = T->screen ? 1 : 0;
  h.n_tab = n_tab;
  h.tab_nd = T->tab_of ? T->tab_nd : 0;
  h.tab_nt = T->tab_of ? T->tab_nt : 0;
  h.o_tab_of = B.add(tab_of);
  h.o_tab_dens = B.add(tab_dens);
  h.o_tab_t9 = B.add(tab_t9);
  h.o_tab_lnl = B.add(tab_lnl);
  h.o_charge = B.add(charge);
  h.o_Q = B.add(Q);
  h.o_scale = B.add(scale);
  h.o_nrho = B.add(nrho);
  h.o_reac = B.add(reac);
  h.o_nreac = B.add(nreac);
  h.o_rhs_ptr = B.add(rhs_ptr);
  h.o_rhs_r = B.add(rhs_r);
  h.o_rhs_c = B.add(rhs_c);
  h.o_dt_r = B.add(dt_r);
  h.o_dt_o = B.add(dt_o);
  h.o_dt_m = B.add(dt_m);
  h.o_dt_j = B.add(dt_j);
  h.o_js_ptr = B.add(js_ptr);
  h.o_js_src = B.add(js_src);
  h.o_js_c = B.add(js_c);
  h.o_js_flag = B.add(js_flag);
  h.o_piv = B.add(piv);
  h.o_lslot = B.add(lslot);
  h.o_uslot = B.add(uslot);
  h.o_dslot = B.add(dslot);
  h.o_fw = B.add(fw); h.o_bw = B.add(bw); h.o_tfw = B.add(tfw); h.o_tbw = B.add(tbw);
  h.o_fw_s = B.add(fw_s); h.o_fw_c = B.add(fw_c);
  h.o_bw_s = B.add(bw_s); h.o_bw_c = B.add(bw_c);
  h.o_tfw_s = B.add(tfw_s); h.o_tfw_c = B.add(tfw_c);
  h.o_tbw_s = B.add(tbw_s); h.o_tbw_c = B.add(tbw_c);
  h.o_diag_orig = B.add(diag_orig);
  h.o_rg_ptr = B.add(rg_ptr);
  h.o_rg_i = B.add(rg_i);
  h.o_rg_c = B.add(rg_c);
  h.o_perm = B.add(perm16);
  h.o_ltgt = B.add(ltgt);
  h.o_ucol_ptr = B.add(ucol_ptr);
  h.o_ucol_s = B.add(ucol_s);
  h.o_ucol_t = B.add(ucol_t);
  h.n_ucol = (int32_t)ucol_s.size();
  h.o_utgt = B.add(utgt);
  h.o_lrow_ptr = B.add(lrow_ptr);
  h.o_lrow_s = B.add(lrow_s);
  h.o_lrow_t = B.add(lrow_t);
  h.n_lrow = (int32_t)lrow_s.size();
  {
    // derivative terms by the species they are taken by (state index j < N)
    std::vector<int32_t> dej_ptr(n + 1, 0);
    std::vector<int16_t> dej_d;
    for (int j = 0; j < n; ++j) {
      for (int d = 0; d < nd; ++d)
        if (dt_j[d] == j) dej_d.push_back((int16_t)d);
      dej_ptr[j + 1] = (int32_t)dej_d.size();
    }
    h.o_dej_ptr = B.add(dej_ptr);
    h.o_dej_d = B.add(dej_d);
  }
  h.nL = (int32_t)lslot.size(); h.nU = (int32_t)uslot.size(); h.nD = (int32_t)dslot.size();
  h.n_rhs = (int32_t)rhs_r.size(); h.n_js = (int32_t)js_src.size();
  h.n_fw = (int32_t)fw_s.size(); h.n_bw = (int32_t)bw_s.size();
  h.n_tfw = (int32_t)tfw_s.size(); h.n_tbw = (int32_t)tbw_s.size();
  h.n_rg = (int32_t)rg_i.size();
  B.buf.resize((B.buf.size() + 15) & ~size_t(15), 0);
  h.bytes = (int32_t)B.buf.size();

  // per-lane workspace layout (doubles)
  int w = 0;
  auto take = [&](int cnt) { int o = w; w += cnt; return o; };
  // arrays touched inside every Newton iteration first ("hot": they may be
  // placed in shared memory), then the history and start-up arrays
  h.w_x = take(n); h.w_xp = take(n); h.w_psi = take(n); h.w_d = take(n);
  h.w_f = take(n); h.w_iw = take(n);
  // the T9 slopes g_r, the reference rates kp_r and the terms R_r g_r are
  // Newton-loop arrays only with self-heating; at fixed temperature g_r is
  // the adjoint's (the T9 gradient of the rates) and sits with the cold part
  h.w_k = take(R);
  if (sh) h.w_g = take(R);
  h.w_rr = take(R);
  if (sh) h.w_kp = take(R);
  h.w_dt = take(nd + (sh ? R : 0));   // [dterms | R_r g_r]
  h.w_lu = take(nnz);
  h.hot_doubles = w;
  if (!sh) { h.w_g = take(R); h.w_kp = take(R); }
  h.w_tmp = take(n); h.w_f0 = take(n);
  h.w_xh = take(HMAX * n); h.w_eh = take(HMAX); h.w_th = take(HMAX);
  h.lane_doubles = w;

  // algorithmic FP64 operation counts per event (an FMA counts 2 flops;
  // exp, log, cbrt, pow, sqrt and divisions are counted apart as special
  // functions, not as flops)
  int64_t terms = 0, jac = 0, lu = 0;
  for (int r = 0; r < R; ++r) terms += nreac[r];
  for (int d = 0; d < nd; ++d) jac += 1 + (dt_o[2 * d] >= 0) + (dt_o[2 * d + 1] >= 0);
  jac += 2 * (int64_t)js_src.size() + nnz + n;
  if (sh) jac += 3 * (int64_t)R + (N + 5) + 5 + 2 * (int64_t)(N + 1);
  for (int k = 0; k < n; ++k) {
    int64_t nl = piv[k].lend - piv[k].lbeg, nu = piv[k].uend - piv[k].ubeg;
    lu += nl + 2 * nl * nu;
  }
  // powers of T9, 7-term exponents, k_r; an effective rate adds three
  // exponents and their combination
  h.fl_teval = 2 + 14 * (int64_t)(R - n_tabr) + 10 * (int64_t)n_tabr + 45 * (int64_t)n_ap +
               (T->screen ? 3 + 2 * (int64_t)(R + n_ap) : 0);
  h.fl_teval_g = 6 + 10 * (int64_t)R + 38 * (int64_t)n_ap;  // d ln lambda / dT9
  h.fl_terms = terms;                        // R_r = k_r prod Y
  h.fl_rhs = 2 * (int64_t)rhs_r.size() + (sh ? 2 * (int64_t)R + N + 5 : 0);
  h.fl_jac = jac;
  h.fl_lu = lu;
  h.fl_solve = 2 * (int64_t)(fw_s.size() + bw_s.size()) + n;
  h.fl_edot = 2 * (int64_t)R;
  h.fl_tsolve = 2 * (int64_t)(tfw_s.size() + tbw_s.size()) + n;
  h.n_exp_per_teval = R + 2 * n_ap;

  std::memcpy(B.buf.data(), &h, sizeof(h));
  *out = std::move(B.buf);
  *hdr_out = h;
  return NB_OK;
}

}  // namespace nb
