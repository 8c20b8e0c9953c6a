// codegen.cpp -- the network-specialised burn kernel: CUDA source generated
// from a compiled network, compiled at run time for sm_103a and loaded.
//
// The paper's pynucastro writes every network as its own C++ code, with the
// rates, the right-hand side and the analytic Jacobian spelled out term by
// term (arXiv:2312.02836 Sec. 2).  The generic kernel instead walks the
// network's gather programs from memory: every term costs index loads and
// address arithmetic besides its FP64 operation, and all of them sit on one
// warp's dependency chain.  Here the same programs are printed as straight
// -line code: every coefficient is a literal and every array index a
// constant, so the per-lane work arrays can live in registers and the
// compiler can interleave independent FP64 chains.  The code performs the
// generic kernel's floating-point operations in the same order (same
// association, same explicit FMAs; both are compiled without implicit
// contraction), so the two kernels give the same bits.
//
// Storage variants for one lane's work arrays (history and f0 always stay in
// the global workspace, as do k and g of a fixed-temperature network, which
// live for the whole zone):
//   1  every Newton-loop array in registers (x, d, f, psi, iw, xp, tmp, lu)
//   2  as 1 with the LU slots in the workspace
//   3  only x, d, f in registers
// Arrays the compiler cannot keep in registers spill to local memory.
#include <dlfcn.h>
#include <nvrtc.h>

#include <cinttypes>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "blob.h"
#include "codegen.h"
#include "nb_embedded.h"   // the integrator headers as text (written by the build)
#include "../../include/netburn.h"

namespace nb {

namespace {

template <class T>
const T* arr(const std::vector<uint8_t>& blob, int off) {
  return reinterpret_cast<const T*>(blob.data() + off);
}

std::string lit(double v) {
  char b[64];
  std::snprintf(b, sizeof b, "%a", v);
  return v < 0 || std::signbit(v) ? "(" + std::string(b) + ")" : std::string(b);
}

struct Out {
  std::string s;
  void operator()(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    s += buf;
  }
  void raw(const std::string& t) { s += t; }
};

// pairs of a two-partial-sum gather over [beg, end): entries beg, beg+2, ..
// go to a0 and beg+1, beg+3, .. to a1, except an odd last entry, which goes
// to a0 (the order of the generic gather)
template <class F>
void emit_pairs(Out& o, int beg, int end, F term) {
  int e = beg;
  for (; e + 1 < end; e += 2) {
    o("    a0 = %s;\n", term(e, "a0").c_str());
    o("    a1 = %s;\n", term(e + 1, "a1").c_str());
  }
  if (e < end) o("    a0 = %s;\n", term(e, "a0").c_str());
}

}  // namespace

int resolve_variant(const BlobHeader& h, int variant) {
  if (variant >= 1 && variant <= 3) return variant;
  const int vec = 7 * h.n;
  if (vec + h.nnz <= 160) return 1;
  if (vec <= 160) return 2;
  return 3;
}

bool specialize_auto_ok(const BlobHeader& h) {
  // straight-line size: RHS + Jacobian gathers, LU updates, solves
  const long long stmts = (long long)h.n_rhs + h.n_js + h.nD + h.n_fw + h.n_bw + h.nd +
                          2LL * h.R;
  return stmts <= 6000;
}

std::string specialized_source(const std::vector<uint8_t>& blob, int variant) {
  const BlobHeader& h = *reinterpret_cast<const BlobHeader*>(blob.data());
  variant = resolve_variant(h, variant);
  const int n = h.n, N = h.N, R = h.R, nnz = h.nnz, nd = h.nd;
  const bool sh = h.self_heating != 0;
  const double* coef = arr<double>(blob, h.o_coef);
  const double* Q = arr<double>(blob, h.o_Q);
  const double* scale = arr<double>(blob, h.o_scale);
  const int32_t* nrho = arr<int32_t>(blob, h.o_nrho);
  const int16_t* reac = arr<int16_t>(blob, h.o_reac);
  const int32_t* nreac = arr<int32_t>(blob, h.o_nreac);
  const int32_t* rhs_ptr = arr<int32_t>(blob, h.o_rhs_ptr);
  const int16_t* rhs_r = arr<int16_t>(blob, h.o_rhs_r);
  const double* rhs_c = arr<double>(blob, h.o_rhs_c);
  const int16_t* dt_r = arr<int16_t>(blob, h.o_dt_r);
  const int16_t* dt_o = arr<int16_t>(blob, h.o_dt_o);
  const double* dt_m = arr<double>(blob, h.o_dt_m);
  const int32_t* js_ptr = arr<int32_t>(blob, h.o_js_ptr);
  const int16_t* js_src = arr<int16_t>(blob, h.o_js_src);
  const double* js_c = arr<double>(blob, h.o_js_c);
  const uint8_t* js_flag = arr<uint8_t>(blob, h.o_js_flag);
  const Pivot* piv = arr<Pivot>(blob, h.o_piv);
  const int16_t* lslot = arr<int16_t>(blob, h.o_lslot);
  const int16_t* uslot = arr<int16_t>(blob, h.o_uslot);
  const int16_t* dslot = arr<int16_t>(blob, h.o_dslot);
  const TriRow* fw = arr<TriRow>(blob, h.o_fw);
  const TriRow* bw = arr<TriRow>(blob, h.o_bw);
  const int16_t* fw_s = arr<int16_t>(blob, h.o_fw_s);
  const int16_t* fw_c = arr<int16_t>(blob, h.o_fw_c);
  const int16_t* bw_s = arr<int16_t>(blob, h.o_bw_s);
  const int16_t* bw_c = arr<int16_t>(blob, h.o_bw_c);

  Out o;
  o("// network-specialised burn kernel: N = %d species, R = %d reactions, "
    "n = %d, LU slots %d, storage variant %d\n", N, R, n, nnz, variant);
  o.raw(
      "typedef signed char int8_t;\ntypedef short int16_t;\ntypedef int int32_t;\n"
      "typedef long long int64_t;\ntypedef unsigned char uint8_t;\n"
      "typedef unsigned int uint32_t;\ntypedef unsigned long long uint64_t;\n"
      "#include \"expf64.cuh\"\n#include \"integrator.cuh\"\n\nnamespace nb {\n\n");
  o("struct GNet {\n  static constexpr int n = %d, N = %d, R = %d, sh = %d, hasE = %d;\n"
    "  static constexpr double inv_n = 1.0 / %d;\n};\n\n",
    n, N, R, sh ? 1 : 0, h.has_E ? 1 : 0, n);
  const int Rd = R > 0 ? R : 1;
  const bool lu_reg = variant == 1, vec_reg = variant <= 2;
  const bool k_reg = sh;   // fixed-T rates live for the whole zone
  o("struct GWS {\n  double x[%d], d[%d], f[%d], rr[%d];\n", n, n, n, Rd);
  if (vec_reg) o("  double psi[%d], iw[%d], xp[%d], tmp[%d];\n", n, n, n, n);
  else o("  LV psi, iw, xp, tmp;\n");
  if (lu_reg) o("  double lu[%d];\n", nnz);
  else o("  LV lu;\n");
  if (k_reg) o("  double k[%d], g[%d], kp[%d];\n", Rd, Rd, Rd);
  else o("  LV k;\n");
  o("  LV f0, xh, eh, th;\n};\n\n");

  // ---- rate tables (grid, ln lambda at the nodes, charges) as literal arrays
  const bool has_tab = h.n_tab > 0;
  const int32_t* tab_of = arr<int32_t>(blob, h.o_tab_of);
  auto lit_array = [&](const char* name, const double* v, size_t cnt) {
    o("__device__ const double %s[%zu] = {", name, cnt);
    for (size_t i = 0; i < cnt; ++i) o("%s%s", i ? ", " : "", lit(v[i]).c_str());
    o("};\n");
  };
  if (has_tab) {
    lit_array("NB_TAB_T9", arr<double>(blob, h.o_tab_t9), (size_t)h.tab_nt);
    lit_array("NB_TAB_DENS", arr<double>(blob, h.o_tab_dens), (size_t)h.tab_nd);
    lit_array("NB_TAB_L", arr<double>(blob, h.o_tab_lnl),
              (size_t)h.n_tab * h.tab_nd * h.tab_nt);
    o("\n");
  }
  o("template <class V>\nNB_HD __forceinline__ void tab_zone(const GNet&, Zone& s, const V& x0) {\n"
    "  s.tab_i = 0;\n  s.tab_u = 0.0;\n");
  if (has_tab) {
    const double* charge = arr<double>(blob, h.o_charge);
    o("  double ye = 0.0;\n");
    for (int i = 0; i < N; ++i) o("  ye = fma(%s, x0[%d], ye);\n", lit(charge[i]).c_str(), i);
    o("  density_cell(NB_TAB_DENS, %d, s.rho, ye, s);\n", h.tab_nd);
  }
  o("}\n\n");

  // ---- rates
  const int32_t* ap = arr<int32_t>(blob, h.o_ap);
  const double* apc = arr<double>(blob, h.o_apc);
  auto fit7 = [&](const double* a, int from) {
    std::string t;
    for (int j = from; j < 7; ++j) t += (j > from ? ", " : "") + lit(a[j]);
    return t;
  };
  // the full evaluation of k_r (and g_r when `g`), in the generic kernel's
  // order (rate_full)
  const bool has_scr = h.has_scr != 0;
  const double* scr = arr<double>(blob, h.o_scr);
  // screening of the exponent and of d ln k / dT9 (as rate_full does)
  auto scr_e = [&](int r) { return "fma(" + lit(scr[r]) + ", p.hz, "; };
  auto dlog = [&](int r, const double* c) {
    const std::string d = "rate_dlog(" + fit7(c, 1) + ", p)";
    return has_scr ? "fma(" + lit(scr[r]) + ", p.hzd, " + d + ")" : d;
  };
  auto emit_full = [&](int r, const char* ind, bool g) {
    const double* a = coef + 7 * r;
    const char* rp = nrho[r] == 0 ? "1.0" : (nrho[r] == 1 ? "s.rho" : "s.rho2");
    const int tb = has_tab ? tab_of[r] : -1;
    if (tb >= 0)
      o("%se = table_lnl(NB_TAB_L + %lld, %d, s, tc, &dl);\n", ind,
        (long long)tb * h.tab_nd * h.tab_nt, h.tab_nt);
    else
      o("%se = rate_exponent(%s, p, T9);\n", ind, fit7(a, 0).c_str());
    o("%sif (lnm) e += lnm[%d];\n", ind, r);
    if (has_scr) o("%se = %se);\n", ind, scr_e(r).c_str());
    if (ap[r] < 0) {
      o("%sw.k[%d] = exp_tang(e) * (%s * %s);\n", ind, r, rp, lit(scale[r]).c_str());
      if (g) {
        const std::string gd = tb >= 0 ? (has_scr ? "fma(" + lit(scr[r]) + ", p.hzd, dl)" : "dl")
                                       : dlog(r, a);
        o("%sif (with_g) w.g[%d] = %s;\n", ind, r, gd.c_str());
      }
      return;
    }
    const double* b = apc + 21 * ap[r];
    o("%s{\n%s  double eap = rate_exponent(%s, p, T9);\n", ind, ind, fit7(b, 0).c_str());
    o("%s  if (lnm) eap += lnm[%d];\n", ind, r);
    if (has_scr) o("%s  eap = %seap);\n", ind, scr_e(r).c_str());
    o("%s  const double epg = rate_exponent(%s, p, T9);\n", ind, fit7(b + 7, 0).c_str());
    o("%s  const double epa = rate_exponent(%s, p, T9);\n", ind, fit7(b + 14, 0).c_str());
    o("%s  const APRate q = ap_rate(e, eap, epg, epa);\n", ind);
    if (g)
      o("%s  if (with_g)\n%s    w.g[%d] = ap_dlog(q, %s, %s,\n"
        "%s                     rate_dlog(%s, p), rate_dlog(%s, p));\n",
        ind, ind, r, dlog(r, a).c_str(), dlog(r, b).c_str(), ind, fit7(b + 7, 1).c_str(),
        fit7(b + 14, 1).c_str());
    o("%s  w.k[%d] = q.lam * (%s * %s);\n%s}\n", ind, r, rp, lit(scale[r]).c_str(), ind);
  };
  o("NB_HD __forceinline__ void eval_rates(const GNet&, const Zone& s, GWS& w, const TPow& p,"
    " double T9, bool with_g) {\n  const double* lnm = s.lnm;\n  double e;\n");
  if (has_tab) o("  const TCell tc = t_cell(NB_TAB_T9, %d, T9);\n  double dl;\n", h.tab_nt);
  for (int r = 0; r < R; ++r) emit_full(r, "  ", sh);
  o("}\n\n");

  // ---- rates near the attempt's reference temperature (self-heating);
  // effective (alpha,p)(p,gamma) rates always take the full evaluation
  o("NB_HD __forceinline__ void save_ref_rates(const GNet&, GWS& w) {\n");
  if (sh)
    for (int r = 0; r < R; ++r) o("  w.kp[%d] = w.k[%d];\n", r, r);
  o("}\n\n");
  o("NB_HD __forceinline__ void eval_rates_near(const GNet&, const Zone& s, GWS& w, double T9,"
    " const TPow& ref, double T9ref) {\n");
  if (sh) {
    o("  DPhi d;\n  TPow p;\n  bool have_p = !delta_phi_series(ref, T9, T9ref, d);\n"
      "  if (have_p) {\n    p = t_powers(T9, false, s.scr);\n    d = delta_phi(p, ref, T9, T9ref);\n  }\n"
      "  const double* lnm = s.lnm;\n  double de, e;\n");
    if (has_tab) o("  const TCell tc = t_cell(NB_TAB_T9, %d, T9);\n  double dl;\n", h.tab_nt);
    // hot part: the small-delta updates, straight-line; a reaction whose
    // delta is large is marked and evaluated in full in the cold part
    // below, so the rarely run full evaluations do not sit between the hot
    // instructions
    o("  unsigned long long full = 0ull;\n");
    int nbit = 0;
    std::vector<int> marked;
    for (int r = 0; r < R; ++r) {
      if (ap[r] >= 0 || (has_tab && tab_of[r] >= 0)) continue;
      o("  de = rate_delta(%s, d);\n", fit7(coef + 7 * r, 1).c_str());
      if (has_scr) o("  de = fma(%s, d.d7, de);\n", lit(scr[r]).c_str());
      if (nbit < 64) {
        o("  if (small_delta(de)) w.k[%d] = rate_near(w.kp[%d], de);\n"
          "  else full |= 1ull << %d;\n", r, r, nbit);
        marked.push_back(r);
        ++nbit;
      } else {
        o("  if (small_delta(de)) {\n    w.k[%d] = rate_near(w.kp[%d], de);\n  } else {\n", r, r);
        o("    if (!have_p) {\n      p = t_powers(T9, false, s.scr);\n      have_p = true;\n    }\n");
        emit_full(r, "    ", false);
        o("  }\n");
      }
    }
    bool always = false;
    for (int r = 0; r < R; ++r) always = always || ap[r] >= 0 || (has_tab && tab_of[r] >= 0);
    if (always) o("  if (!have_p) {\n    p = t_powers(T9, false, s.scr);\n    have_p = true;\n  }\n");
    for (int r = 0; r < R; ++r)
      if (ap[r] >= 0 || (has_tab && tab_of[r] >= 0)) emit_full(r, "  ", false);
    if (!marked.empty()) {
      o("  if (full) {\n");
      o("    if (!have_p) p = t_powers(T9, false, s.scr);\n");
      for (size_t b = 0; b < marked.size(); ++b) {
        o("    if (full & (1ull << %zu)) {\n", b);
        emit_full(marked[b], "      ", false);
        o("    }\n");
      }
      o("  }\n");
    }
  }
  o("}\n\n");

  // ---- terms
  o("template <class V>\nNB_HD __forceinline__ void eval_terms(const GNet&, GWS& w, const V& v) {\n");
  for (int r = 0; r < R; ++r) {
    o("  w.rr[%d] = w.k[%d]", r, r);
    for (int m = 0; m < nreac[r]; ++m) o(" * v[%d]", reac[3 * r + m]);
    o(";\n");
  }
  o("}\n\n");

  // ---- edot
  o("NB_HD __forceinline__ double eval_edot(const GNet&, GWS& w) {\n"
    "  double a0 = 0.0, a1 = 0.0;\n");
  emit_pairs(o, 0, R, [&](int r, const char* acc) {
    return "fma(" + lit(Q[r]) + ", w.rr[" + std::to_string(r) + "], " + acc + ")";
  });
  o("  return a0 + a1;\n}\n\n");

  // ---- f
  o("template <class V, class O>\nNB_HD __forceinline__ void eval_f(const GNet& t, GWS& w,"
    " const V& v, O&& out) {\n");
  for (int i = 0; i < N; ++i) {
    o("  {\n    double a0 = 0.0, a1 = 0.0;\n");
    emit_pairs(o, rhs_ptr[i], rhs_ptr[i + 1], [&](int e, const char* acc) {
      return "fma(" + lit(rhs_c[e]) + ", w.rr[" + std::to_string(rhs_r[e]) + "], " + acc + ")";
    });
    o("    out[%d] = a0 + a1;\n  }\n", i);
  }
  if (sh) o("  out[%d] = eval_edot(t, w) / heat_capacity(t, v);\n", N);
  o("}\n\n");

  // ---- M = alpha0 I - h J
  const int ndt = nd + (sh ? R : 0);
  o("template <class V>\nNB_HD __forceinline__ void assemble_M(const GNet& t, GWS& w,"
    " const V& v, double alpha0, double h) {\n  double dt[%d];\n", ndt > 0 ? ndt : 1);
  for (int d = 0; d < nd; ++d) {
    o("  dt[%d] = w.k[%d] * %s", d, dt_r[d], lit(dt_m[d]).c_str());
    if (dt_o[2 * d] >= 0) o(" * v[%d]", dt_o[2 * d]);
    if (dt_o[2 * d + 1] >= 0) o(" * v[%d]", dt_o[2 * d + 1]);
    o(";\n");
  }
  if (sh) {
    for (int r = 0; r < R; ++r) o("  dt[%d] = w.rr[%d] * w.g[%d];\n", nd + r, r, r);
    o("  const TRow tr = t_row(eval_edot(t, w), heat_capacity(t, v), v[%d]);\n", N);
  }
  o("  const double mh = -h;\n");
  for (int s = 0; s < nnz; ++s) {
    o("  {\n    double a0 = 0.0, a1 = 0.0;\n");
    emit_pairs(o, js_ptr[s], js_ptr[s + 1], [&](int e, const char* acc) {
      return "fma(" + lit(js_c[e]) + ", dt[" + std::to_string(js_src[e]) + "], " + acc + ")";
    });
    o("    double acc = a0 + a1;\n");
    const uint8_t fl = js_flag[s];
    if (fl & SLOT_TROW) o("    acc = fma(acc, tr.a1, tr.b1);\n");
    else if (fl & SLOT_TT) o("    acc = fma(acc, tr.a1, tr.b2);\n");
    o("    double m = mh * acc;\n");
    if (fl & SLOT_DIAG) o("    m += alpha0;\n");
    o("    w.lu[%d] = m;\n  }\n", s);
  }
  o("}\n\n");

  // ---- LU
  o("NB_HD __forceinline__ bool factor_M(const GNet&, GWS& w) {\n  bool ok = true;\n");
  // the diagonal of M before elimination, for the pivot guard
  for (int k = 0; k < n; ++k) o("  const double a%d = w.lu[%d];\n", k, piv[k].dslot);
  for (int k = 0; k < n; ++k) {
    const Pivot& p = piv[k];
    o("  {\n    const double pv = w.lu[%d];\n    ok = ok && pivot_kept(pv, a%d);\n"
      "    const double inv = recip2(pv);\n    w.lu[%d] = inv;\n", p.dslot, k, p.dslot);
    const int nu = p.uend - p.ubeg;
    int dpos = p.dbeg;
    for (int li = p.lbeg; li < p.lend; ++li) {
      const int ls = lslot[li];
      o("    {\n      const double l = w.lu[%d] * inv;\n      w.lu[%d] = l;\n"
        "      const double ml = -l;\n", ls, ls);
      for (int u = 0; u < nu; ++u, ++dpos) {
        const int ds = dslot[dpos];
        o("      w.lu[%d] = fma(ml, w.lu[%d], w.lu[%d]);\n", ds, uslot[p.ubeg + u], ds);
      }
      o("    }\n");
    }
    o("  }\n");
  }
  o("  return ok;\n}\n\n");

  // ---- solves
  o("template <class V>\nNB_HD __forceinline__ void solve_M(const GNet&, GWS& w, V&& v) {\n");
  auto tri = [&](const TriRow* rows, const int16_t* es, const int16_t* ec) {
    for (int q = 0; q < n; ++q) {
      const TriRow& r = rows[q];
      o("  {\n    double a0 = v[%d], a1 = 0.0;\n", r.tgt);
      emit_pairs(o, r.beg, r.end, [&](int e, const char* acc) {
        return "fma(-w.lu[" + std::to_string(es[e]) + "], v[" + std::to_string(ec[e]) + "], " +
               acc + ")";
      });
      o("    double acc = a0 + a1;\n");
      if (r.dslot >= 0) o("    acc *= w.lu[%d];\n", r.dslot);
      o("    v[%d] = acc;\n  }\n", r.tgt);
    }
  };
  tri(fw, fw_s, fw_c);
  tri(bw, bw_s, bw_c);
  o("}\n\n}  // namespace nb\n\n");

  // ---- kernel
  o("extern \"C\" __global__ void __launch_bounds__(256, 1) nb_spec_burn(nb::BurnParams P) {\n"
    "  using namespace nb;\n  GNet t;\n  const int lane = threadIdx.x & 31;\n"
    "  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;\n"
    "  double* base = P.ws + warp * (long long)%d * WS_LANES + lane;\n  GWS w;\n",
    h.lane_doubles);
  auto lv = [&](const char* name, int off) {
    o("  w.%s.p = base + %d * WS_LANES;\n", name, off);
  };
  if (!vec_reg) { lv("psi", h.w_psi); lv("iw", h.w_iw); lv("xp", h.w_xp); lv("tmp", h.w_tmp); }
  if (!lu_reg) lv("lu", h.w_lu);
  if (!k_reg) lv("k", h.w_k);
  lv("f0", h.w_f0); lv("xh", h.w_xh); lv("eh", h.w_eh); lv("th", h.w_th);
  o("  burn_claim_loop(t, w, P);\n}\n");
  return o.s;
}

// ------------------------------------------------------------------ NVRTC

namespace {

struct Nvrtc {
  bool ok = false;
  std::string why;
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) log = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) cubin = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
};

Nvrtc load_nvrtc() {
  Nvrtc api;
  std::vector<std::string> names = {"libnvrtc.so.13", "libnvrtc.so"};
  if (const char* home = std::getenv("CUDA_HOME")) {
    names.push_back(std::string(home) + "/lib64/libnvrtc.so.13");
    names.push_back(std::string(home) + "/lib64/libnvrtc.so");
  }
  names.push_back("/usr/local/cuda/lib64/libnvrtc.so.13");
  names.push_back("/usr/local/cuda/lib64/libnvrtc.so");
  void* h = nullptr;
  for (const auto& nm : names)
    if ((h = dlopen(nm.c_str(), RTLD_NOW | RTLD_LOCAL))) break;
  if (!h) { api.why = "libnvrtc not found"; return api; }
  bool good = true;
  auto sym = [&](auto& fn, const char* name) {
    fn = reinterpret_cast<std::remove_reference_t<decltype(fn)>>(dlsym(h, name));
    good = good && fn != nullptr;
  };
  sym(api.create, "nvrtcCreateProgram");
  sym(api.compile, "nvrtcCompileProgram");
  sym(api.log_size, "nvrtcGetProgramLogSize");
  sym(api.log, "nvrtcGetProgramLog");
  sym(api.cubin_size, "nvrtcGetCUBINSize");
  sym(api.cubin, "nvrtcGetCUBIN");
  sym(api.destroy, "nvrtcDestroyProgram");
  api.ok = good;
  if (!good) api.why = "libnvrtc lacks a needed entry point";
  return api;
}

const Nvrtc& nvrtc() {
  static const Nvrtc api = load_nvrtc();
  return api;
}

}  // namespace

int compile_specialized(const std::string& src, std::vector<char>* cubin, std::string* log,
                        bool verbose) {
  const Nvrtc& api = nvrtc();
  if (!api.ok) {
    if (log) *log = api.why;
    return NB_E_COMPILE;
  }
  nvrtcProgram prog;
  if (api.create(&prog, src.c_str(), "nb_spec.cu", kEmbedCount, kEmbedSources, kEmbedNames) !=
      NVRTC_SUCCESS) {
    if (log) *log = "nvrtcCreateProgram failed";
    return NB_E_COMPILE;
  }
  std::vector<const char*> opts = {"--gpu-architecture=sm_103a", "-std=c++17", "--fmad=false",
                                   "-DNB_SPECIALIZED=1"};
  if (verbose) opts.push_back("--ptxas-options=-v");
  const nvrtcResult rc = api.compile(prog, (int)opts.size(), opts.data());
  size_t ls = 0;
  api.log_size(prog, &ls);
  if (log) {
    log->assign(ls, '\0');
    if (ls) api.log(prog, &(*log)[0]);
    while (!log->empty() && log->back() == '\0') log->pop_back();
  }
  int out = NB_OK;
  if (rc != NVRTC_SUCCESS) {
    out = NB_E_COMPILE;
  } else if (cubin) {
    size_t cs = 0;
    api.cubin_size(prog, &cs);
    cubin->assign(cs, 0);
    if (cs == 0 || api.cubin(prog, cubin->data()) != NVRTC_SUCCESS) out = NB_E_COMPILE;
  }
  api.destroy(&prog);
  return out;
}

}  // namespace nb
