// blob.h -- layout of the compiled network ("blob") shared by the host-side
// symbolic analysis (netload.cpp) and the kernels (burn.cu).
//
// A network is compiled once into one contiguous, 16-byte aligned byte
// buffer: a header followed by index/coefficient arrays.  Kernels copy it
// into shared memory (or read it through L1) and walk its gather programs;
// nothing in it depends on the zone.
#pragma once
#ifndef __CUDACC_RTC__  // the run-time compiler has no system headers
#include <stdint.h>
#endif

namespace nb {

constexpr int HMAX = 7;       // accepted points kept per zone
constexpr int KMAX = 5;       // highest BDF order
constexpr int NCOUNT = 9;     // per-zone event counters
constexpr int WS_LANES = 32;  // per-lane workspace is interleaved by warp lane

enum Counter { C_ACC = 0, C_REJ_ERR, C_REJ_NEWTON, C_NEWTON_IT, C_JAC, C_RHS,
               C_TEVAL, C_EDOT, C_ORDSUM };

// Jacobian slot flags
enum : uint8_t { SLOT_DIAG = 1, SLOT_TROW = 2, SLOT_TT = 4 };

// One row of a triangular gather program: v[tgt] = (v[tgt] - sum_e a[slot_e]
// v[col_e]) * (dslot >= 0 ? a[dslot] : 1)
struct TriRow {
  int32_t tgt, beg, end, dslot;
};

// One pivot of the static-pivot LU: a[d] <- 1/a[d]; a[L] *= a[d];
// a[D(i,j)] -= a[L_i] a[U_j]
struct Pivot {
  int32_t dslot, lbeg, lend, ubeg, uend, dbeg;
};

struct BlobHeader {
  int32_t n, N, R, self_heating, has_E;
  int32_t nnz;        // slots of the filled LU pattern
  int32_t nd;         // derivative terms dR_r/dY_j
  int32_t nnz_jac;    // structural nonzeros of M before fill
  int32_t lane_doubles;  // per-lane workspace, in doubles
  int32_t bytes;      // total blob bytes (multiple of 16)
  // offsets (bytes from blob start)
  int32_t o_coef;     // double [R*7]
  int32_t o_Q;        // double [R] (zeros when !has_E)
  int32_t o_scale;    // double [R]
  int32_t o_nrho;     // int32 [R]  n_r - 1
  int32_t o_reac;     // int16 [R*3] reactant occurrences, -1 padded
  int32_t o_nreac;    // int32 [R]
  int32_t o_rhs_ptr;  // int32 [N+1]
  int32_t o_rhs_r;    // int16 [rhs entries]
  int32_t o_rhs_c;    // double [rhs entries]
  int32_t o_dt_r;     // int16 [nd]
  int32_t o_dt_o;     // int16 [nd*2] remaining reactant occurrences, -1 = none
  int32_t o_dt_m;     // double [nd] multiplicity
  int32_t o_dt_j;     // int16 [nd] species the derivative is taken by
  int32_t o_js_ptr;   // int32 [nnz+1] Jacobian gather per slot
  int32_t o_js_src;   // int16 [js entries] index into [dterms | R_r g_r]
  int32_t o_js_c;     // double [js entries]
  int32_t o_js_flag;  // uint8 [nnz]
  int32_t o_piv;      // Pivot [n]
  int32_t o_lslot;    // int16 [nL]
  int32_t o_uslot;    // int16 [nU]
  int32_t o_dslot;    // int16 [nD]
  int32_t o_fw, o_bw, o_tfw, o_tbw;       // TriRow [n] each
  int32_t o_fw_s, o_fw_c, o_bw_s, o_bw_c; // int16 entries (slot, col)
  int32_t o_tfw_s, o_tfw_c, o_tbw_s, o_tbw_c;
  int32_t o_diag_orig;  // int32 [n] slot of the diagonal, by original index
  int32_t o_rg_ptr;   // int32 [R+1] adjoint: species entries of rate r
  int32_t o_rg_i;     // int16 [...]  species index i
  int32_t o_rg_c;     // double [...] c_ir
  int32_t nL, nU, nD, n_rhs, n_js, n_fw, n_bw, n_tfw, n_tbw, n_rg;
  // per-lane workspace offsets, in doubles (element e of array A of a lane
  // lives at ws_base[(A + e) * WS_LANES])
  int32_t w_x, w_xp, w_psi, w_d, w_f, w_iw, w_tmp, w_f0, w_xh, w_eh, w_th,
      w_k, w_g, w_rr, w_dt, w_lu;
  // algorithmic FP64 operation counts per event (an FMA counts 2)
  int64_t fl_teval, fl_teval_g, fl_terms, fl_rhs, fl_jac, fl_lu, fl_solve,
      fl_edot, fl_tsolve;
  int32_t n_exp_per_teval;
  int32_t hot_doubles;  // leading part of the per-lane layout kept hot
  int32_t w_kp;         // k_r at the step's reference temperature (self-heating)
  int32_t o_ap;         // int32 [R] row of the effective-rate fits, -1 = plain
  int32_t o_apc;        // double [n_ap * 21] (a,p), (p,g), (p,a) fits
  int32_t n_ap;         // effective (alpha,p)(p,gamma) rates
  int32_t o_scr;        // double [R] weak-screening strengths s_r
  int32_t has_scr;      // 1 when the network is screened
  int32_t n_tab;        // tables of tabulated rates (0: none)
  int32_t tab_nd, tab_nt;  // their grid: density and temperature nodes
  int32_t o_tab_of;     // int32 [R] table of reaction r, -1 = fit
  int32_t o_tab_dens;   // double [tab_nd] log10(rho Ye) nodes
  int32_t o_tab_t9;     // double [tab_nt] T9 nodes
  int32_t o_tab_lnl;    // double [n_tab * tab_nd * tab_nt] ln lambda at the nodes
  int32_t o_charge;     // double [N] species charges
  // column-oriented triangular solves (one zone spread over a warp)
  int32_t o_perm;       // int16 [n] original index of position k
  int32_t o_ltgt;       // int16 [nL] original row index of each L entry (lslot order)
  int32_t o_ucol_ptr;   // int32 [n+1] entries of U column k (rows above k)
  int32_t o_ucol_s;     // int16 [...] their slots
  int32_t o_ucol_t;     // int16 [...] their original row indices
  int32_t n_ucol;
  // transposed solves of the adjoint, column by column
  int32_t o_utgt;       // int16 [nU] original column index of each U entry (uslot order)
  int32_t o_lrow_ptr;   // int32 [n+1] entries of L row k (columns left of k)
  int32_t o_lrow_s;     // int16 [...] their slots
  int32_t o_lrow_t;     // int16 [...] their original column indices
  int32_t o_dej_ptr;    // int32 [n+1] derivative terms taken by species j
  int32_t o_dej_d;      // int16 [nd] those terms, in increasing order
  int32_t n_lrow, pad3_;
};

}  // namespace nb
