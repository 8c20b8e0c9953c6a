/*
 * oracle.c -- plain, slow, FP64 CPU reference for the batched stiff
 * reaction-network burn and its rate sensitivities.
 *
 * TEST INFRASTRUCTURE ONLY.  It is called by the tests, by the smoke check
 * and by the benchmark's CPU-baseline leg, never by the library.  It shares
 * no code, header, table or constant generator with the CUDA path.
 *
 * What it computes (the method of arXiv:2312.02836, Sec. 2-3: a generated
 * network right-hand side and analytic Jacobian integrated per zone by a
 * stiff BDF/Newton integrator, with an optional self-heating temperature
 * equation):
 *
 *   rate        lambda_r(T9) = exp(a0 + a1/T9 + a2 T9^(-1/3) + a3 T9^(1/3)
 *                                  + a4 T9 + a5 T9^(5/3) + a6 ln T9)
 *               (the 7-parameter ReacLib fit the paper's networks use, Sec. 2)
 *   term        R_r = s_r e^(p_r) rho^(n_r - 1) lambda_r(T9) prod_j Y_j
 *   RHS         dY_i/dt = sum_r c_ir R_r,  c_ir = #(i in products) - #(i in reactants)
 *   energy      edot = sum_r Q_r R_r,  dE/dt = edot
 *   heating     dT9/dt = edot / c_v,  c_v = 1.5 sum_i Y_i + 1e-3 T9^3
 *   screening   weak screening (Salpeter 1954): R_r is multiplied by exp(H_r),
 *               H_r = s_r sqrt(rho zeta) T6^(-3/2), T6 = 1e3 T9, where
 *               s_r = 0.188 sum Z_a Z_b over the reactants' successive pairs
 *               (given per reaction) and zeta the zone's plasma parameter
 *               sum (Z_i^2 + Z_i) Y_i, an input of the zone held over its burn
 *   tabulated   a reaction given as a table (TabularRate, Sec. 2: weak rates
 *               tabulated in (rho Ye, T)) takes ln lambda by bilinear
 *               interpolation in (log10(rho Ye), T9) on a rectilinear grid,
 *               clamped to the grid's edges; Ye = sum Z_i Y_i of the zone's
 *               initial composition, held over the burn
 *   effective   a reaction flagged as the (alpha,p)(p,gamma) approximation of
 *               Sec. 2 (A(a,p)X(p,g)B merged into one A(a,g)B rate, valid
 *               when proton capture on X is fast, so that the proton flow
 *               through X is in equilibrium) uses
 *               lambda = lambda_ag + lambda_ap lambda_pg / (lambda_pg + lambda_pa):
 *               X in steady state, d(Y_X Y_p)/dt = 0, splits the flow from
 *               A(a,p)X between X(p,g)B and the return X(p,a)A.  Each of the
 *               four lambdas is a 7-parameter fit; the paper states the
 *               approximation in words only, this is its first-principles form
 *
 * The integrator is variable-step, variable-order (1..5) BDF in Lagrange
 * (variable-coefficient) form with a modified Newton iteration, as in the
 * VODE family the paper's Microphysics uses (Sec. 2).  The paper prints no
 * integrator details; the rules below are this project's reading, and the
 * CUDA path follows the same rules:
 *
 *   weights   w_i = atol + rtol |x_i(t_n)|,  ||v|| = sqrt(mean_i (v_i / w_i)^2)
 *   h0        Hairer-Norsett-Wanner, Solving ODEs I, Sec. II.4 starting-step
 *             algorithm with p = 1, then h0 <- min(h0, t_end), >= 1e-30 t_end;
 *             a step below 1e-30 t_end or 1e-14 t ends the zone (DT_UNDERFLOW)
 *   step k    alpha_j = h l_j'(t_{n+1}) over nodes t_{n+1}, t_n, .., t_{n+1-k};
 *             solve G(x) = sum_j alpha_j x_{n+1-j} - h f(x) = 0
 *   predictor degree-k extrapolation through x_n .. x_{n-k}; the very first
 *             step (one point) uses x_n + h f(x_n)
 *   Newton    J at the predictor, M = alpha_0 I - h J factored once per
 *             attempt (dense LU, partial pivoting); <= 4 iterations; converged
 *             when ||d|| <= 1e-3, or theta/(1-theta) ||d|| <= 1e-3 with
 *             theta = ||d_m|| / ||d_{m-1}||; theta > 0.9 diverges.  Failure:
 *             h <- h/4.
 *   error     err = || h/(t_{n+1} - t_{n-k}) (x_{n+1} - x_pred) ||  (1/2 on
 *             the first step); accept iff err <= 1, else
 *             h <- h max(0.2, 0.9 err^(-1/(k+1)))
 *   order     after k+1 accepted steps at order k, E_q for q = k-1, k, k+1
 *             (the same estimate with the degree-q extrapolation through the
 *             q+1 newest old points), factor_q = 0.9 E_q^(-1/(q+1)); the
 *             largest factor wins (ties keep k, then k-1)
 *   step size factor clamped to [0.2, 5], kept at 1 when in [1, 1.2);
 *             the step that would pass t_end lands on it exactly
 *   E         after convergence E_{n+1} = (h edot(x_{n+1}) - sum_{j>=1}
 *             alpha_j E_{n+1-j}) / alpha_0; E is not in the error norm.
 *
 * Sensitivities: the forward sensitivity of the same discrete map under a
 * frozen schedule (t_n, k_n), with the exact Jacobian at the converged
 * x_{n+1}:  (alpha_0 I - h J(x_{n+1})) s_{n+1} = -sum_{j>=1} alpha_j s_{n+1-j}
 * + h df/dtheta.
 *
 * Rounding variants (ora_options.variant, 0 = the oracle as described):
 * equally valid orderings of the same arithmetic, for measuring how far
 * rounding alone moves a burn.  Bit 1 takes every sum over reactions, over
 * species and over the seven fit terms in decreasing index order; bit 2
 * factors the index-reversed Newton matrix (partial pivoting kept); bit 4
 * moves every exp, log and cbrt result by one ulp, up or down by the last
 * bit of the argument (another libm of the same accuracy); bit 8 computes the
 * step-size factor 0.9 E^(-1/(q+1)) as 0.9 exp(-ln(E)/(q+1)); bit 16 factors
 * the Newton matrix with its indices in a fixed pseudo-random order (another
 * elimination order; partial pivoting kept).  They change no
 * rule of the method, only the order and the last bits of its floating-point
 * operations.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared oracle.c -lm -lpthread
 * (no FMA contraction, so x86-64 and aarch64 hosts give the same bits).
 */
#define _GNU_SOURCE
#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define HMAX 7      /* accepted points kept: the newest and six older ones */
#define KMAX 5      /* highest BDF order */

enum { ST_OK = 0, ST_MAX_STEPS = 1, ST_DT_UNDERFLOW = 2, ST_NEWTON_FAIL = 3,
       ST_NONFINITE = 5, ST_SINGULAR = 7 };

/* per-zone event counters */
enum { C_ACC = 0, C_REJ_ERR, C_REJ_NEWTON, C_NEWTON_IT, C_JAC, C_RHS, C_TEVAL,
       C_EDOT, C_ORDSUM, C_COUNT };   /* C_ORDSUM: sum of the accepted steps' orders */

typedef struct {
    int32_t N, R, self_heating;
    const int16_t* reactants;   /* [R*3], -1 padded */
    const int16_t* products;    /* [R*3], -1 padded */
    const double* Q;            /* [R] or NULL */
    const double* scale;        /* [R] or NULL (1) */
    const double* coeffs;       /* [R*7] */
    const int8_t* ap_pg;        /* [R] or NULL: 1 = (alpha,p)(p,gamma) effective */
    const double* ap_coeffs;    /* [R*21] fits of (a,p), (p,g), (p,a), or NULL */
    const double* screen;       /* [R] weak-screening strengths s_r, or NULL */
    const int32_t* tab_of;      /* [R] table of reaction r (-1: fit), or NULL */
    int32_t tab_nd, tab_nt;     /* grid: density and temperature nodes */
    const double* tab_dens;     /* [tab_nd] log10(rho Ye) nodes, increasing */
    const double* tab_t9;       /* [tab_nt] T9 nodes, increasing */
    const double* tab_lnl;      /* [n_tab * tab_nd * tab_nt] ln lambda at the nodes */
    const double* charge;       /* [N] species charges Z_i (for Ye), or NULL */
} ora_network;

typedef struct {
    double rtol, atol, t_end;
    int32_t max_attempts;       /* accepted + rejected attempts */
    double newton_tol;          /* 1e-3 */
    int32_t newton_maxit;       /* 4 */
    double fixed_h;             /* > 0: constant step, no error test */
    int32_t fixed_order;        /* > 0: order never changes from this value */
    int32_t max_order;          /* KMAX unless smaller */
    int32_t variant;            /* rounding variant bits (header), 0 = none */
} ora_options;

enum { VAR_SUM_REVERSE = 1, VAR_LU_REVERSE = 2, VAR_ULP = 4, VAR_STEP_EXP = 8,
       VAR_LU_PERMUTE = 16 };

/* the rounding variant of the zone this thread is burning (0 outside a burn) */
static _Thread_local int g_variant = 0;

/* q-th index of a sum over [0, m): increasing, or decreasing under the
   reversed-sum variant */
static int sum_index(int q, int m) {
    return (g_variant & VAR_SUM_REVERSE) ? m - 1 - q : q;
}

/* a transcendental result y = fn(x), moved by one ulp under the ulp variant:
   up when the last bit of x is set, else down */
static double ulp_variant(double y, double x) {
    if (!(g_variant & VAR_ULP) || !isfinite(y) || y == 0.0) return y;
    uint64_t b;
    memcpy(&b, &x, sizeof b);
    return nextafter(y, (b & 1u) ? INFINITY : -INFINITY);
}

static double v_exp(double x) { return ulp_variant(exp(x), x); }
static double v_log(double x) { return ulp_variant(log(x), x); }
static double v_cbrt(double x) { return ulp_variant(cbrt(x), x); }

/* ------------------------------------------------------------------ */
/* model                                                               */
/* ------------------------------------------------------------------ */

static int n_reactants(const ora_network* net, int r) {
    int n = 0;
    for (int s = 0; s < 3; ++s) n += net->reactants[3 * r + s] >= 0;
    return n;
}

/* stoichiometric coefficient c_ir */
static double stoich(const ora_network* net, int i, int r) {
    double c = 0.0;
    for (int s = 0; s < 3; ++s) {
        if (net->products[3 * r + s] == i) c += 1.0;
        if (net->reactants[3 * r + s] == i) c -= 1.0;
    }
    return c;
}

/* k_r = s_r e^(p_r) rho^(n_r-1) lambda_r(T9) and g_r = d ln lambda_r / dT9 */
/* cell c and weight w in [0, 1] of value v on increasing nodes x[0..m), clamped */
static void grid_cell(const double* x, int m, double v, int* c, double* w) {
    if (v <= x[0]) { *c = 0; *w = 0.0; return; }
    if (v >= x[m - 1]) { *c = m - 2; *w = 1.0; return; }
    int i = 0;
    while (v > x[i + 1]) ++i;
    *c = i;
    *w = (v - x[i]) / (x[i + 1] - x[i]);
}

/* ln lambda of table tb at (log10(rho Ye), T9) by bilinear interpolation, and
   its T9-derivative (0 outside the temperature range) */
static double table_lnl(const ora_network* net, int tb, double lrye, double T9, double* dl) {
    int i, j;
    double u, v;
    grid_cell(net->tab_dens, net->tab_nd, lrye, &i, &u);
    grid_cell(net->tab_t9, net->tab_nt, T9, &j, &v);
    const double* L = net->tab_lnl + (size_t)tb * net->tab_nd * net->tab_nt;
    const int nt = net->tab_nt;
    double l00 = L[i * nt + j], l01 = L[i * nt + j + 1];
    double l10 = L[(i + 1) * nt + j], l11 = L[(i + 1) * nt + j + 1];
    double at_j = (1 - u) * l00 + u * l10;      /* along density, at T node j */
    double at_j1 = (1 - u) * l01 + u * l11;     /* and at node j+1 */
    int inside = T9 > net->tab_t9[0] && T9 < net->tab_t9[nt - 1];
    *dl = inside ? (at_j1 - at_j) / (net->tab_t9[j + 1] - net->tab_t9[j]) : 0.0;
    return (1 - v) * at_j + v * at_j1;
}

void ora_rate_factors(const ora_network* net, double T9, double rho, double zeta,
                      double ye, const double* ln_mult, double* k, double* g) {
    double t13 = v_cbrt(T9);
    double phi[7] = {1.0, 1.0 / T9, 1.0 / t13, t13, T9, T9 * t13 * t13, v_log(T9)};
    double dphi[7] = {0.0,
                      -1.0 / (T9 * T9),
                      -1.0 / (3.0 * T9 * t13),
                      1.0 / (3.0 * t13 * t13),
                      1.0,
                      5.0 / 3.0 * t13 * t13,
                      1.0 / T9};
    for (int r = 0; r < net->R; ++r) {
        const double* a = net->coeffs + 7 * r;
        double e = 0.0, de = 0.0;
        for (int q = 0; q < 7; ++q) {
            int j = sum_index(q, 7);
            e += a[j] * phi[j];
            de += a[j] * dphi[j];
        }
        double s = net->scale ? net->scale[r] : 1.0;
        double p = ln_mult ? ln_mult[r] : 0.0;
        double rp = 1.0;
        for (int m = 1; m < n_reactants(net, r); ++m) rp *= rho;
        if (net->tab_of && net->tab_of[r] >= 0) {
            /* a tabulated rate replaces the fit's exponent */
            double dl;
            e = table_lnl(net, net->tab_of[r], log10(rho * ye), T9, &dl);
            de = dl;
        }
        /* screening: H_r = s_r sqrt(rho zeta) T6^(-3/2), dH/dT9 = -1.5 H / T9 */
        double H = 0.0;
        if (net->screen && zeta > 0.0)
            H = net->screen[r] * sqrt(rho * zeta) * pow(1e3 * T9, -1.5);
        e += H;
        de += -1.5 * H / T9;
        double lam = v_exp(e);
        if (net->ap_pg && net->ap_pg[r]) {
            /* lambda = lambda_ag + lambda_ap lambda_pg / (lambda_pg + lambda_pa) */
            double ec[3], dec[3];
            for (int c = 0; c < 3; ++c) {
                const double* b = net->ap_coeffs + 21 * r + 7 * c;
                ec[c] = 0.0;
                dec[c] = 0.0;
                for (int q = 0; q < 7; ++q) {
                    int j = sum_index(q, 7);
                    ec[c] += b[j] * phi[j];
                    dec[c] += b[j] * dphi[j];
                }
            }
            /* the alpha capture screens the (a,p) channel as it does the direct one */
            ec[0] += H;
            dec[0] += -1.5 * H / T9;
            double l_ag = lam, l_ap = v_exp(ec[0]), l_pg = v_exp(ec[1]), l_pa = v_exp(ec[2]);
            double frac = l_pg / (l_pg + l_pa);
            double via_p = l_ap * frac;
            lam = l_ag + via_p;
            /* d ln lambda / dT9: d frac/dT9 = frac (1 - frac) (g_pg - g_pa) */
            de = (l_ag * de + via_p * (dec[0] + (1.0 - frac) * (dec[1] - dec[2]))) / lam;
        }
        k[r] = s * v_exp(p) * rp * lam;
        if (g) g[r] = de;
    }
}

/* species with c_ir != 0 of every reaction (increasing species index), so
   the sums over r below visit only the reactions that touch a species */
typedef struct {
    int cnt;
    int sp[6];
    double c[6];
} rxn_species;

static rxn_species* species_lists(const ora_network* net) {
    rxn_species* L = calloc((size_t)net->R + 1, sizeof(rxn_species));
    for (int r = 0; r < net->R; ++r)
        for (int i = 0; i < net->N; ++i) {
            double c = stoich(net, i, r);
            if (c != 0.0) {
                L[r].sp[L[r].cnt] = i;
                L[r].c[L[r].cnt] = c;
                L[r].cnt++;
            }
        }
    return L;
}

/* R_r = k_r prod over reactant occurrences of Y */
static void reaction_terms(const ora_network* net, const double* x,
                           const double* k, double* Rr) {
    for (int r = 0; r < net->R; ++r) {
        double v = k[r];
        for (int s = 0; s < 3; ++s) {
            int j = net->reactants[3 * r + s];
            if (j >= 0) v *= x[j];
        }
        Rr[r] = v;
    }
}

static double heat_capacity(const ora_network* net, const double* x) {
    double sy = 0.0;
    for (int q = 0; q < net->N; ++q) sy += x[sum_index(q, net->N)];
    double T9 = x[net->N];
    return 1.5 * sy + 1e-3 * T9 * T9 * T9;
}

/* f (n entries) and edot at state x, given k_r for the state's T9.
   f_i = sum_r c_ir R_r, accumulated over r in increasing order. */
static void rhs_given_k(const ora_network* net, const rxn_species* L,
                        const double* x, const double* k,
                        double* f, double* edot, double* Rr) {
    int N = net->N, R = net->R;
    reaction_terms(net, x, k, Rr);
    for (int i = 0; i < N; ++i) f[i] = 0.0;
    for (int qr = 0; qr < R; ++qr) {
        int r = sum_index(qr, R);
        for (int q = 0; q < L[r].cnt; ++q) f[L[r].sp[q]] += L[r].c[q] * Rr[r];
    }
    double ed = 0.0;
    if (net->Q)
        for (int qr = 0; qr < R; ++qr) ed += net->Q[sum_index(qr, R)] * Rr[sum_index(qr, R)];
    if (edot) *edot = ed;
    if (net->self_heating) f[N] = ed / heat_capacity(net, x);
}

/* dR_r/dY_j: product over the reactant occurrences with one j removed,
   times the multiplicity of j */
static double dterm_dY(const ora_network* net, const double* x, const double* k,
                       int r, int j) {
    int m = 0;
    for (int s = 0; s < 3; ++s) m += net->reactants[3 * r + s] == j;
    if (m == 0) return 0.0;
    double v = k[r] * (double)m;
    int skipped = 0;
    for (int s = 0; s < 3; ++s) {
        int l = net->reactants[3 * r + s];
        if (l < 0) continue;
        if (l == j && !skipped) { skipped = 1; continue; }
        v *= x[l];
    }
    return v;
}

/* distinct reactant species of reaction r; returns their count */
static int distinct_reactants(const ora_network* net, int r, int* out) {
    int m = 0;
    for (int s = 0; s < 3; ++s) {
        int j = net->reactants[3 * r + s];
        if (j < 0) continue;
        int seen = 0;
        for (int q = 0; q < m; ++q) seen |= out[q] == j;
        if (!seen) out[m++] = j;
    }
    return m;
}

/* dense Jacobian J[i*n + j] = d f_i / d x_j at x (k, g for the state's T9):
   J_ij = sum_r c_ir dR_r/dY_j, accumulated over r in increasing order */
static void jacobian_given_k(const ora_network* net, const rxn_species* L,
                             const double* x, const double* k, const double* g,
                             double* J, double* Rr) {
    int N = net->N, R = net->R, n = N + (net->self_heating ? 1 : 0);
    memset(J, 0, sizeof(double) * n * n);
    for (int qr = 0; qr < R; ++qr) {
        int r = sum_index(qr, R);
        int js[3];
        int m = distinct_reactants(net, r, js);
        for (int a = 0; a < m; ++a) {
            double d = dterm_dY(net, x, k, r, js[a]);
            for (int q = 0; q < L[r].cnt; ++q)
                J[L[r].sp[q] * n + js[a]] += L[r].c[q] * d;
        }
    }
    if (!net->self_heating) return;
    reaction_terms(net, x, k, Rr);
    double cv = heat_capacity(net, x);
    double ed = 0.0, dedT = 0.0;
    for (int qr = 0; qr < R; ++qr) {
        int r = sum_index(qr, R);
        ed += net->Q[r] * Rr[r];
        dedT += net->Q[r] * Rr[r] * g[r];
    }
    double fT = ed / cv;
    for (int qr = 0; qr < R; ++qr) {
        int r = sum_index(qr, R);
        for (int q = 0; q < L[r].cnt; ++q)
            J[L[r].sp[q] * n + N] += L[r].c[q] * Rr[r] * g[r];
    }
    /* T row: d edot / dY_j, accumulated over r in increasing order */
    for (int qr = 0; qr < R; ++qr) {
        int r = sum_index(qr, R);
        int js[3];
        int m = distinct_reactants(net, r, js);
        for (int a = 0; a < m; ++a)
            J[N * n + js[a]] += net->Q[r] * dterm_dY(net, x, k, r, js[a]);
    }
    for (int j = 0; j < N; ++j) J[N * n + j] = J[N * n + j] / cv - fT * 1.5 / cv;
    double T9 = x[N];
    J[N * n + N] = dedT / cv - fT * (3e-3 * T9 * T9) / cv;
}

static int state_dim(const ora_network* net) { return net->N + (net->self_heating ? 1 : 0); }

/* Public single-state evaluations (used by the tests).  T9 is the fixed
   temperature when the network has no self-heating; otherwise x[N] is used. */
void ora_rhs(const ora_network* net, const double* x, double T9, double rho, double zeta,
             double ye, const double* ln_mult, double* f, double* edot) {
    double* k = malloc(sizeof(double) * (net->R + 1));
    double* Rr = malloc(sizeof(double) * (net->R + 1));
    rxn_species* L = species_lists(net);
    ora_rate_factors(net, net->self_heating ? x[net->N] : T9, rho, zeta, ye, ln_mult, k, NULL);
    rhs_given_k(net, L, x, k, f, edot, Rr);
    free(L);
    free(k);
    free(Rr);
}

void ora_jacobian(const ora_network* net, const double* x, double T9, double rho,
                  double zeta, double ye, const double* ln_mult, double* J) {
    double* k = malloc(sizeof(double) * (net->R + 1));
    double* g = malloc(sizeof(double) * (net->R + 1));
    double* Rr = malloc(sizeof(double) * (net->R + 1));
    rxn_species* L = species_lists(net);
    ora_rate_factors(net, net->self_heating ? x[net->N] : T9, rho, zeta, ye, ln_mult, k, g);
    jacobian_given_k(net, L, x, k, g, J, Rr);
    free(L);
    free(k);
    free(g);
    free(Rr);
}

/* ------------------------------------------------------------------ */
/* dense linear algebra (textbook LU with partial pivoting)            */
/* ------------------------------------------------------------------ */

/* reverse the index order of an n x n matrix in place: A[i][j] <->
   A[n-1-i][n-1-j] (the reversed-LU variant factors this matrix) */
static void reverse_matrix(double* A, int n) {
    for (int e = 0; e < n * n / 2; ++e) {
        double t = A[e]; A[e] = A[n * n - 1 - e]; A[n * n - 1 - e] = t;
    }
}

static void reverse_vector(double* b, int n) {
    for (int i = 0; i < n / 2; ++i) {
        double t = b[i]; b[i] = b[n - 1 - i]; b[n - 1 - i] = t;
    }
}

/* the fixed pseudo-random order of the permuted-LU variant: position i holds
   index perm_index(i, n) (multiplication by an odd constant modulo n, a
   bijection for n not sharing its factors) */
static int perm_mult(int n) {
    int m = 7919 % n;
    for (;; ++m) {
        int a = m, b = n;
        while (b) { int t = a % b; a = b; b = t; }
        if (a == 1 && m > 1) return m;
        if (m > 4 * n + 8) return 1;
    }
}

static void permute_matrix(double* A, int n, int inverse) {
    int m = perm_mult(n);
    double* B = malloc(sizeof(double) * n * n);
    memcpy(B, A, sizeof(double) * n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            int pi = (int)((long)i * m % n), pj = (int)((long)j * m % n);
            if (inverse) A[pi * n + pj] = B[i * n + j];
            else A[i * n + j] = B[pi * n + pj];
        }
    free(B);
}

static void permute_vector(double* b, int n, int inverse) {
    int m = perm_mult(n);
    double* c = malloc(sizeof(double) * n);
    memcpy(c, b, sizeof(double) * n);
    for (int i = 0; i < n; ++i) {
        int pi = (int)((long)i * m % n);
        if (inverse) b[pi] = c[i];
        else b[i] = c[pi];
    }
    free(c);
}

/* factor A (n x n, row-major) in place; returns 0 or -1 if singular */
static int lu_factor(double* A, int* piv, int n) {
    if (g_variant & VAR_LU_PERMUTE) permute_matrix(A, n, 0);
    if (g_variant & VAR_LU_REVERSE) reverse_matrix(A, n);
    for (int c = 0; c < n; ++c) {
        int p = c;
        double best = fabs(A[c * n + c]);
        for (int i = c + 1; i < n; ++i)
            if (fabs(A[i * n + c]) > best) { best = fabs(A[i * n + c]); p = i; }
        piv[c] = p;
        if (!(best > 0.0) || !isfinite(best)) return -1;
        if (p != c)
            for (int j = 0; j < n; ++j) {
                double t = A[c * n + j]; A[c * n + j] = A[p * n + j]; A[p * n + j] = t;
            }
        for (int i = c + 1; i < n; ++i) {
            double l = A[i * n + c] / A[c * n + c];
            A[i * n + c] = l;
            for (int j = c + 1; j < n; ++j) A[i * n + j] -= l * A[c * n + j];
        }
    }
    return 0;
}

static void lu_solve(const double* A, const int* piv, int n, double* b) {
    if (g_variant & VAR_LU_PERMUTE) permute_vector(b, n, 0);
    if (g_variant & VAR_LU_REVERSE) reverse_vector(b, n);
    for (int c = 0; c < n; ++c) {
        int p = piv[c];
        if (p != c) { double t = b[c]; b[c] = b[p]; b[p] = t; }
    }
    for (int i = 1; i < n; ++i) {
        double s = b[i];
        for (int j = 0; j < i; ++j) s -= A[i * n + j] * b[j];
        b[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * b[j];
        b[i] = s / A[i * n + i];
    }
    if (g_variant & VAR_LU_REVERSE) reverse_vector(b, n);
    if (g_variant & VAR_LU_PERMUTE) permute_vector(b, n, 1);
}

/* ------------------------------------------------------------------ */
/* BDF pieces                                                          */
/* ------------------------------------------------------------------ */

/* alpha_j = h * l_j'(tau_0), Lagrange basis on tau_0 = t_new, tau_j = t_old[j-1] */
void ora_bdf_alpha(int k, double t_new, const double* t_old, double h, double* alpha) {
    double tau[KMAX + 1];
    tau[0] = t_new;
    for (int j = 1; j <= k; ++j) tau[j] = t_old[j - 1];
    double s = 0.0;
    for (int m = 1; m <= k; ++m) s += 1.0 / (tau[0] - tau[m]);
    alpha[0] = h * s;
    for (int j = 1; j <= k; ++j) {
        double num = 1.0, den = 1.0;
        for (int m = 0; m <= k; ++m) {
            if (m == j) continue;
            if (m != 0) num *= tau[0] - tau[m];
            den *= tau[j] - tau[m];
        }
        alpha[j] = h * num / den;
    }
}

/* value at t of the degree-q polynomial through (t_pts[j], x_pts[j]), j=0..q */
void ora_extrapolate(int q, int n, const double* t_pts, const double* x_pts,
                     double t, double* out) {
    for (int i = 0; i < n; ++i) out[i] = 0.0;
    for (int j = 0; j <= q; ++j) {
        double lj = 1.0;
        for (int m = 0; m <= q; ++m)
            if (m != j) lj *= (t - t_pts[m]) / (t_pts[j] - t_pts[m]);
        for (int i = 0; i < n; ++i) out[i] += lj * x_pts[j * n + i];
    }
}

static double wnorm(int n, const double* v, const double* w) {
    double s = 0.0;
    for (int qi = 0; qi < n; ++qi) {
        int i = sum_index(qi, n);
        double q = v[i] / w[i];
        s += q * q;
    }
    return sqrt(s / n);
}

static int all_finite(int n, const double* v) {
    for (int i = 0; i < n; ++i) if (!isfinite(v[i])) return 0;
    return 1;
}

/* ------------------------------------------------------------------ */
/* one zone                                                            */
/* ------------------------------------------------------------------ */

typedef struct {
    /* optional record of the accepted schedule: entry 0 is the initial
       point (k = 0), entry s >= 1 the s-th accepted step */
    int32_t cap;
    double* t;      /* [cap] */
    int32_t* k;     /* [cap] */
    double* x;      /* [cap * n] */
    double* E;      /* [cap] */
    int32_t count;
    double* hnext;  /* [cap] or NULL: the step size the controller chose after
                       accepted step s (the next attempt's h before it is cut
                       to land on t_end) */
} ora_tape;

typedef struct {
    rxn_species* L;
    double* k; double* g; double* Rr;
    double* J; double* M; int* piv;
    double* f; double* x; double* xp; double* psi; double* d; double* G;
    double* w; double* x1; double* f1; double* tmp;
    double* xh;     /* [HMAX * n] newest first */
    double th[HMAX];
    double Eh[HMAX];
} work_t;

static work_t* work_alloc(const ora_network* net) {
    int n = net->N + (net->self_heating ? 1 : 0), R = net->R;
    work_t* W = calloc(1, sizeof(work_t));
    W->L = species_lists(net);
    W->k = malloc(sizeof(double) * (R + 1));
    W->g = malloc(sizeof(double) * (R + 1));
    W->Rr = malloc(sizeof(double) * (R + 1));
    W->J = malloc(sizeof(double) * n * n);
    W->M = malloc(sizeof(double) * n * n);
    W->piv = malloc(sizeof(int) * n);
    double** vecs[] = {&W->f, &W->x, &W->xp, &W->psi, &W->d, &W->G, &W->w,
                       &W->x1, &W->f1, &W->tmp};
    for (size_t i = 0; i < sizeof(vecs) / sizeof(vecs[0]); ++i)
        *vecs[i] = malloc(sizeof(double) * n);
    W->xh = malloc(sizeof(double) * HMAX * n);
    return W;
}

static void work_free(work_t* W) {
    free(W->L);
    free(W->k); free(W->g); free(W->Rr); free(W->J); free(W->M); free(W->piv);
    free(W->f); free(W->x); free(W->xp); free(W->psi); free(W->d); free(W->G);
    free(W->w); free(W->x1); free(W->f1); free(W->tmp); free(W->xh);
    free(W);
}

typedef struct {
    const ora_network* net;
    double rho, T9_fixed;
    const double* ln_mult;
    int32_t* cnt;
    double zeta, ye;
} zone_ctx;

/* Ye = sum Z_i Y_i of a composition (1 without charges) */
static double electron_fraction(const ora_network* net, const double* Y) {
    if (!net->charge) return 1.0;
    double ye = 0.0;
    for (int i = 0; i < net->N; ++i) ye += net->charge[i] * Y[i];
    return ye;
}

/* rate factors for state x (fixed temperature or x[N]) */
static void rates_for(zone_ctx* z, const double* x, work_t* W, int with_g) {
    const ora_network* net = z->net;
    double T9 = net->self_heating ? x[net->N] : z->T9_fixed;
    ora_rate_factors(net, T9, z->rho, z->zeta, z->ye, z->ln_mult, W->k, with_g ? W->g : NULL);
    z->cnt[C_TEVAL]++;
}

static void push_history(work_t* W, int n, int* nh, double t, const double* x, double E) {
    int m = *nh < HMAX ? *nh : HMAX - 1;
    for (int j = m; j >= 1; --j) {
        W->th[j] = W->th[j - 1];
        W->Eh[j] = W->Eh[j - 1];
        memcpy(W->xh + j * n, W->xh + (j - 1) * n, sizeof(double) * n);
    }
    W->th[0] = t;
    W->Eh[0] = E;
    memcpy(W->xh, x, sizeof(double) * n);
    if (*nh < HMAX) (*nh)++;
}

/* 0.9 E^(-1/(q+1)) */
static double err_power(double E, int q) {
    if (g_variant & VAR_STEP_EXP) return 0.9 * exp(-log(E) / (q + 1));
    return 0.9 * pow(E, -1.0 / (q + 1));
}

static double step_factor(double E, int q) {
    if (!(E > 0.0)) return 5.0;
    return err_power(E, q);
}

/* E_q after an accepted step: the newest point is W->xh[0] (time th[0]),
   the q+1 older points are xh[1..q+1] */
static double order_estimate(int q, int n, work_t* W, double h) {
    ora_extrapolate(q, n, W->th + 1, W->xh + n, W->th[0], W->tmp);
    for (int i = 0; i < n; ++i) W->tmp[i] = W->xh[i] - W->tmp[i];
    double c = h / (W->th[0] - W->th[q + 1]);
    for (int i = 0; i < n; ++i) W->tmp[i] *= c;
    return wnorm(n, W->tmp, W->w);
}

static int burn_zone(const ora_network* net, const ora_options* opt,
                     const double* Y0, double T9_0, double rho, double zeta,
                     const double* ln_mult, double* Y_out, double* T9_out,
                     double* E_out, int32_t* cnt, ora_tape* tape, work_t* W) {
    const int N = net->N, n = state_dim(net);
    const int has_E = net->Q != NULL;
    const double t_end = opt->t_end, rtol = opt->rtol, atol = opt->atol;
    const int kmax = opt->max_order > 0 && opt->max_order < KMAX ? opt->max_order : KMAX;
    g_variant = opt->variant;
    zone_ctx z = {net, rho, T9_0, ln_mult, cnt, zeta, electron_fraction(net, Y0)};
    double* f0 = malloc(sizeof(double) * n);   /* f(x_0), for the first predictor */
    memset(cnt, 0, sizeof(int32_t) * C_COUNT);

    double* x0 = W->x1;            /* reuse: initial state */
    for (int i = 0; i < N; ++i) x0[i] = Y0[i];
    if (net->self_heating) x0[N] = T9_0;
    int status = ST_OK;
    double t = 0.0, E = 0.0;
    int nh = 0;
    push_history(W, n, &nh, t, x0, E);
    if (tape) {
        tape->count = 0;
        if (tape->cap > 0) {
            tape->t[0] = 0.0; tape->k[0] = 0; tape->E[0] = 0.0;
            memcpy(tape->x, x0, sizeof(double) * n);
            tape->count = 1;
        }
    }

    /* rates, f(x0); with a fixed temperature these rates serve the whole burn */
    rates_for(&z, W->xh, W, 0);
    double ed0;
    rhs_given_k(net, W->L, W->xh, W->k, W->f, &ed0, W->Rr);
    cnt[C_RHS]++;
    int finite0 = all_finite(n, W->xh) && all_finite(n, W->f) && T9_0 > 0.0;
    for (int r = 0; r < net->R && finite0; ++r) finite0 = isfinite(W->k[r]);
    if (!finite0 || !(t_end > 0.0)) {
        status = finite0 ? ST_OK : ST_NONFINITE;
        goto done;
    }
    memcpy(f0, W->f, sizeof(double) * n);

    for (int i = 0; i < n; ++i) W->w[i] = atol + rtol * fabs(W->xh[i]);
    double h;
    if (opt->fixed_h > 0.0) {
        h = opt->fixed_h;
    } else {
        /* starting step, Hairer-Norsett-Wanner I, Sec. II.4, p = 1 */
        double d0 = wnorm(n, W->xh, W->w), d1 = wnorm(n, f0, W->w);
        double hp = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
        if (hp > t_end) hp = t_end;
        for (int i = 0; i < n; ++i) W->x[i] = W->xh[i] + hp * f0[i];
        if (net->self_heating) rates_for(&z, W->x, W, 0);
        rhs_given_k(net, W->L, W->x, W->k, W->f1, NULL, W->Rr);
        cnt[C_RHS]++;
        for (int i = 0; i < n; ++i) W->tmp[i] = (W->f1[i] - f0[i]) / hp;
        double d2 = wnorm(n, W->tmp, W->w);
        double dm = d1 > d2 ? d1 : d2;
        double h1 = dm <= 1e-15 ? fmax(1e-6, hp * 1e-3) : sqrt(0.01 / dm);
        h = fmin(100.0 * hp, h1);
        if (h > t_end) h = t_end;
        if (!(h >= 1e-30 * t_end)) h = 1e-30 * t_end;
    }

    int k = opt->fixed_order > 0 ? opt->fixed_order : 1;
    if (k > kmax) k = kmax;
    int nconsec = 0, newton_fails = 0;
    const double hmin = 1e-30 * t_end;

    while (t < t_end) {
        if (cnt[C_ACC] + cnt[C_REJ_ERR] + cnt[C_REJ_NEWTON] >= opt->max_attempts) {
            status = ST_MAX_STEPS; break;
        }
        if (h < hmin || h < 1e-14 * t) { status = ST_DT_UNDERFLOW; break; }
        double t_new;
        if (t + h >= t_end) { h = t_end - t; t_new = t_end; } else t_new = t + h;
        int kk = k < nh ? k : nh;             /* fixed-order ramp-up */
        double alpha[KMAX + 1];
        ora_bdf_alpha(kk, t_new, W->th, h, alpha);
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int j = 1; j <= kk; ++j) s += alpha[j] * W->xh[(j - 1) * n + i];
            W->psi[i] = s;
        }
        for (int i = 0; i < n; ++i) W->w[i] = atol + rtol * fabs(W->xh[i]);
        /* predictor (fewer than kk+1 points happens on the first step only,
           or while a fixed order ramps up) */
        if (nh >= kk + 1)
            ora_extrapolate(kk, n, W->th, W->xh, t_new, W->xp);
        else if (nh >= 2)
            ora_extrapolate(nh - 1, n, W->th, W->xh, t_new, W->xp);
        else
            for (int i = 0; i < n; ++i) W->xp[i] = W->xh[i] + h * f0[i];
        /* Jacobian + f at the predictor, LU of M */
        memcpy(W->x, W->xp, sizeof(double) * n);
        if (net->self_heating) rates_for(&z, W->x, W, 1);
        jacobian_given_k(net, W->L, W->x, W->k, W->g, W->J, W->Rr);
        cnt[C_JAC]++;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                W->M[i * n + j] = (i == j ? alpha[0] : 0.0) - h * W->J[i * n + j];
        const int lu_ok = lu_factor(W->M, W->piv, n) == 0;
        int ok = lu_ok;
        double nrm_prev = 0.0;
        int converged = 0;
        for (int m = 0; ok && m < opt->newton_maxit; ++m) {
            if (m > 0 && net->self_heating) rates_for(&z, W->x, W, 0);
            rhs_given_k(net, W->L, W->x, W->k, W->f, NULL, W->Rr);
            cnt[C_RHS]++;
            for (int i = 0; i < n; ++i)
                W->G[i] = alpha[0] * W->x[i] + W->psi[i] - h * W->f[i];
            for (int i = 0; i < n; ++i) W->d[i] = -W->G[i];
            lu_solve(W->M, W->piv, n, W->d);
            for (int i = 0; i < n; ++i) W->x[i] += W->d[i];
            cnt[C_NEWTON_IT]++;
            double nrm = wnorm(n, W->d, W->w);
            if (!isfinite(nrm)) { ok = 0; break; }
            if (nrm <= opt->newton_tol) { converged = 1; break; }
            if (m > 0) {
                double theta = nrm / nrm_prev;
                if (theta > 0.9) { ok = 0; break; }
                if (theta / (1.0 - theta) * nrm <= opt->newton_tol) { converged = 1; break; }
            }
            nrm_prev = nrm;
        }
        if (!converged) {
            cnt[C_REJ_NEWTON]++;
            /* ten in a row: SINGULAR when the last one's LU broke down */
            if (++newton_fails >= 10) { status = lu_ok ? ST_NEWTON_FAIL : ST_SINGULAR; break; }
            h *= 0.25;
            continue;
        }
        newton_fails = 0;
        /* local error estimate */
        double c = nh >= kk + 1 ? h / (t_new - W->th[kk]) : 0.5;
        for (int i = 0; i < n; ++i) W->tmp[i] = c * (W->x[i] - W->xp[i]);
        double err = wnorm(n, W->tmp, W->w);
        if (opt->fixed_h <= 0.0 && !(err <= 1.0)) {
            cnt[C_REJ_ERR]++;
            double fac = isfinite(err) ? err_power(err, kk) : 0.2;
            h *= fac > 0.2 ? fac : 0.2;
            continue;
        }
        /* accept */
        double E_new = 0.0;
        if (has_E) {
            double ed;
            if (net->self_heating) rates_for(&z, W->x, W, 0);
            reaction_terms(net, W->x, W->k, W->Rr);
            ed = 0.0;
            for (int r = 0; r < net->R; ++r) ed += net->Q[r] * W->Rr[r];
            cnt[C_EDOT]++;
            double s = 0.0;
            for (int j = 1; j <= kk; ++j) s += alpha[j] * W->Eh[j - 1];
            E_new = (h * ed - s) / alpha[0];
        }
        push_history(W, n, &nh, t_new, W->x, E_new);
        t = t_new;
        E = E_new;
        cnt[C_ACC]++;
        cnt[C_ORDSUM] += kk;
        if (tape && tape->count < tape->cap) {
            int s = tape->count++;
            tape->t[s] = t; tape->k[s] = kk; tape->E[s] = E;
            memcpy(tape->x + (size_t)s * n, W->x, sizeof(double) * n);
        }
        if (opt->fixed_h > 0.0) {
            h = opt->fixed_h;
            if (tape && tape->hnext && tape->count <= tape->cap) tape->hnext[tape->count - 1] = h;
            continue;
        }
        /* step size and order for the next step */
        nconsec++;
        double factor;
        if (opt->fixed_order <= 0 && nconsec >= k + 1) {
            int best_q = k;
            double best = step_factor(order_estimate(k, n, W, h), k);
            if (k > 1) {
                double fq = step_factor(order_estimate(k - 1, n, W, h), k - 1);
                if (fq > best) { best = fq; best_q = k - 1; }
            }
            if (k < kmax && nh >= k + 3) {
                double fq = step_factor(order_estimate(k + 1, n, W, h), k + 1);
                if (fq > best) { best = fq; best_q = k + 1; }
            }
            if (best_q != k) { k = best_q; nconsec = 0; }
            factor = best;
        } else {
            factor = step_factor(err, kk);
        }
        if (factor < 0.2) factor = 0.2;
        if (factor > 5.0) factor = 5.0;
        if (factor >= 1.0 && factor < 1.2) factor = 1.0;
        h *= factor;
        if (tape && tape->hnext && tape->count >= 1 && tape->count <= tape->cap)
            tape->hnext[tape->count - 1] = h;
    }
done:
    free(f0);
    for (int i = 0; i < N; ++i) Y_out[i] = W->xh[i];
    if (T9_out) *T9_out = net->self_heating ? W->xh[N] : T9_0;
    if (E_out) *E_out = W->Eh[0];
    g_variant = 0;
    return status;
}

/* ------------------------------------------------------------------ */
/* batch over zones with a thread pool                                 */
/* ------------------------------------------------------------------ */

typedef struct {
    const ora_network* net;
    const ora_options* opt;
    int64_t Z;
    const double* t_end_z;      /* per-zone end times or NULL */
    const double *Y0, *T9, *rho, *ln_mult, *zeta;
    int per_zone_mult;
    double *Y, *T9_out, *E;
    int32_t *cnt, *status;
    atomic_long next;
} batch_t;

static void* batch_worker(void* arg) {
    batch_t* B = arg;
    const ora_network* net = B->net;
    work_t* W = work_alloc(net);
    for (;;) {
        long z = atomic_fetch_add(&B->next, 1);
        if (z >= B->Z) break;
        const double* lm = B->ln_mult
            ? (B->per_zone_mult ? B->ln_mult + (size_t)z * net->R : B->ln_mult) : NULL;
        ora_options oz = *B->opt;
        if (B->t_end_z) oz.t_end = B->t_end_z[z];
        if (!(oz.t_end >= 0.0) || !isfinite(oz.t_end)) {
            /* a zone without a valid end time keeps its inputs */
            memcpy(B->Y + (size_t)z * net->N, B->Y0 + (size_t)z * net->N, sizeof(double) * net->N);
            if (B->T9_out) B->T9_out[z] = B->T9[z];
            if (B->E) B->E[z] = 0.0;
            memset(B->cnt + (size_t)z * C_COUNT, 0, sizeof(int32_t) * C_COUNT);
            B->status[z] = ST_NONFINITE;
            continue;
        }
        B->status[z] = burn_zone(net, &oz, B->Y0 + (size_t)z * net->N, B->T9[z],
                                 B->rho[z], B->zeta ? B->zeta[z] : 0.0, lm,
                                 B->Y + (size_t)z * net->N,
                                 B->T9_out ? B->T9_out + z : NULL,
                                 B->E ? B->E + z : NULL,
                                 B->cnt + (size_t)z * C_COUNT, NULL, W);
    }
    work_free(W);
    return NULL;
}

/* Burn Z zones.  Y0 [Z*N], T9 [Z], rho [Z]; ln_mult [R] shared or [Z*R];
   outputs Y [Z*N], T9_out [Z], E [Z] (may be NULL), cnt [Z*8], status [Z].
   nthreads <= 0 means one thread per online core.  t_end_z: per-zone end
   times (each zone burns for its own step) or NULL for opt->t_end.  zeta:
   per-zone plasma parameters for screening, or NULL (no screening).
   Returns the threads used. */
int ora_burn_batch(const ora_network* net, const ora_options* opt, int64_t Z,
                   const double* Y0, const double* T9, const double* rho,
                   const double* ln_mult, int per_zone_mult, double* Y,
                   double* T9_out, double* E, int32_t* cnt, int32_t* status,
                   int nthreads, const double* t_end_z, const double* zeta) {
    if (nthreads <= 0) {
        long c = sysconf(_SC_NPROCESSORS_ONLN);
        nthreads = c > 0 ? (int)c : 1;
    }
    if (nthreads > Z) nthreads = Z > 0 ? (int)Z : 1;
    batch_t B;
    B.net = net; B.opt = opt; B.Z = Z; B.t_end_z = t_end_z; B.Y0 = Y0; B.T9 = T9; B.rho = rho;
    B.ln_mult = ln_mult; B.per_zone_mult = per_zone_mult; B.Y = Y; B.zeta = zeta;
    B.T9_out = T9_out; B.E = E; B.cnt = cnt; B.status = status;
    atomic_init(&B.next, 0);
    pthread_t* th = malloc(sizeof(pthread_t) * nthreads);
    for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, batch_worker, &B);
    for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
    free(th);
    return nthreads;
}

/* One zone with its accepted schedule recorded (t, k, x, E per point). */
int ora_burn_tape(const ora_network* net, const ora_options* opt,
                  const double* Y0, double T9_0, double rho, double zeta,
                  const double* ln_mult, double* Y, double* T9_out, double* E,
                  int32_t* cnt, int32_t cap, double* tape_t, int32_t* tape_k,
                  double* tape_x, double* tape_E, int32_t* tape_count,
                  double* tape_hnext) {
    work_t* W = work_alloc(net);
    ora_tape tp = {cap, tape_t, tape_k, tape_x, tape_E, 0, tape_hnext};
    int st = burn_zone(net, opt, Y0, T9_0, rho, zeta, ln_mult, Y, T9_out, E, cnt, &tp, W);
    *tape_count = tp.count;
    work_free(W);
    return st;
}

/* ------------------------------------------------------------------ */
/* frozen-schedule replay and forward sensitivity                      */
/* ------------------------------------------------------------------ */

/* Re-take the steps t[1..S] with orders k[1..S] from (Y0, T9_0) with full
   Newton (fresh Jacobian every iteration) until ||d|| <= tol, plus one more
   iteration.  Output the
   final state x_S [n] and E_S.  Returns 0, or -1 if a step did not converge. */
int ora_replay(const ora_network* net, const ora_options* opt, const double* Y0,
               double T9_0, double rho, double zeta, const double* ln_mult, int32_t S,
               const double* tape_t, const int32_t* tape_k, double tol,
               int32_t maxit, double* x_out, double* E_out) {
    const int N = net->N, n = state_dim(net);
    work_t* W = work_alloc(net);
    int32_t cnt[C_COUNT] = {0};
    zone_ctx z = {net, rho, T9_0, ln_mult, cnt, zeta, electron_fraction(net, Y0)};
    int nh = 0, rc = 0;
    for (int i = 0; i < N; ++i) W->x1[i] = Y0[i];
    if (net->self_heating) W->x1[N] = T9_0;
    push_history(W, n, &nh, tape_t[0], W->x1, 0.0);
    rates_for(&z, W->xh, W, 1);
    double* f0 = malloc(sizeof(double) * n);
    rhs_given_k(net, W->L, W->xh, W->k, f0, NULL, W->Rr);
    for (int s = 1; s <= S && rc == 0; ++s) {
        int kk = tape_k[s];
        double t_new = tape_t[s], h = t_new - W->th[0];
        double alpha[KMAX + 1];
        ora_bdf_alpha(kk, t_new, W->th, h, alpha);
        for (int i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int j = 1; j <= kk; ++j) acc += alpha[j] * W->xh[(j - 1) * n + i];
            W->psi[i] = acc;
            W->w[i] = opt->atol + opt->rtol * fabs(W->xh[i]);
        }
        if (nh >= kk + 1) ora_extrapolate(kk, n, W->th, W->xh, t_new, W->x);
        else for (int i = 0; i < n; ++i) W->x[i] = W->xh[i] + h * f0[i];
        int conv = 0, polish = 0;
        for (int m = 0; m < maxit; ++m) {
            rates_for(&z, W->x, W, 1);
            jacobian_given_k(net, W->L, W->x, W->k, W->g, W->J, W->Rr);
            rhs_given_k(net, W->L, W->x, W->k, W->f, NULL, W->Rr);
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j)
                    W->M[i * n + j] = (i == j ? alpha[0] : 0.0) - h * W->J[i * n + j];
            if (lu_factor(W->M, W->piv, n) != 0) break;
            for (int i = 0; i < n; ++i)
                W->d[i] = -(alpha[0] * W->x[i] + W->psi[i] - h * W->f[i]);
            lu_solve(W->M, W->piv, n, W->d);
            for (int i = 0; i < n; ++i) W->x[i] += W->d[i];
            /* once within tol, one more (quadratically convergent) iteration */
            if (polish) { conv = 1; break; }
            if (wnorm(n, W->d, W->w) <= tol) polish = 1;
        }
        if (!conv) { rc = -1; break; }
        double E_new = 0.0;
        if (net->Q) {
            rates_for(&z, W->x, W, 0);
            reaction_terms(net, W->x, W->k, W->Rr);
            double ed = 0.0;
            for (int r = 0; r < net->R; ++r) ed += net->Q[r] * W->Rr[r];
            double acc = 0.0;
            for (int j = 1; j <= kk; ++j) acc += alpha[j] * W->Eh[j - 1];
            E_new = (h * ed - acc) / alpha[0];
        }
        push_history(W, n, &nh, t_new, W->x, E_new);
    }
    memcpy(x_out, W->xh, sizeof(double) * n);
    if (E_out) *E_out = W->Eh[0];
    free(f0);
    work_free(W);
    return rc;
}

/* Forward sensitivity of the final state and energy along a recorded
   schedule.  Parameters theta, in this order: the R ln-multipliers, the n
   initial-state entries, and (fixed temperature only) T9.  Outputs
   dx [n * P] (row i, column theta) and dE [P], P = R + n + (1 - self_heating).
   tape_h [S+1] or NULL: the step sizes the recorded burn used (else
   t_s - t_{s-1}, which can differ from them in the last bit).  variant:
   rounding variant bits, as in ora_options. */
int ora_forward_sensitivity(const ora_network* net, double T9_fixed, double rho,
                            double zeta, const double* ln_mult, int32_t S, const double* tape_t,
                            const int32_t* tape_k, const double* tape_x, const double* tape_h,
                            int32_t variant, double* dx_out, double* dE_out) {
    g_variant = variant;
    const int N = net->N, R = net->R, n = state_dim(net);
    const int P = R + n + (net->self_heating ? 0 : 1);
    work_t* W = work_alloc(net);
    int32_t cnt[C_COUNT] = {0};
    zone_ctx z = {net, rho, T9_fixed, ln_mult, cnt, zeta, electron_fraction(net, tape_x)};
    /* history of sensitivity matrices, newest first */
    double* Sh = calloc((size_t)HMAX * n * P, sizeof(double));
    double* SEh = calloc((size_t)HMAX * P, sizeof(double));
    double* rhs = malloc(sizeof(double) * (size_t)n * P);
    double* col = malloc(sizeof(double) * n);
    double* dedx = malloc(sizeof(double) * n);
    double th[HMAX];
    int nh = 1, rc = 0;
    th[0] = tape_t[0];
    for (int i = 0; i < n; ++i) Sh[(size_t)i * P + R + i] = 1.0;  /* ds/dx0 = I */
    for (int s = 1; s <= S; ++s) {
        int kk = tape_k[s];
        double t_new = tape_t[s], h = tape_h ? tape_h[s] : t_new - th[0];
        double alpha[KMAX + 1];
        ora_bdf_alpha(kk, t_new, th, h, alpha);
        const double* x = tape_x + (size_t)s * n;
        rates_for(&z, x, W, 1);
        jacobian_given_k(net, W->L, x, W->k, W->g, W->J, W->Rr);
        reaction_terms(net, x, W->k, W->Rr);
        double cv = net->self_heating ? heat_capacity(net, x) : 1.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                W->M[i * n + j] = (i == j ? alpha[0] : 0.0) - h * W->J[i * n + j];
        if (lu_factor(W->M, W->piv, n) != 0) { rc = -1; break; }
        /* right-hand sides: -sum_j alpha_j S_{n+1-j} + h df/dtheta */
        for (int i = 0; i < n; ++i)
            for (int p = 0; p < P; ++p) {
                double acc = 0.0;
                for (int j = 1; j <= kk; ++j)
                    acc += alpha[j] * Sh[((size_t)(j - 1) * n + i) * P + p];
                rhs[(size_t)i * P + p] = -acc;
            }
        for (int r = 0; r < R; ++r) {
            for (int i = 0; i < N; ++i)
                rhs[(size_t)i * P + r] += h * stoich(net, i, r) * W->Rr[r];
            if (net->self_heating)
                rhs[(size_t)N * P + r] += h * net->Q[r] * W->Rr[r] / cv;
        }
        if (!net->self_heating) {   /* T9 as a parameter */
            for (int i = 0; i < N; ++i) {
                double acc = 0.0;
                for (int r = 0; r < R; ++r) acc += stoich(net, i, r) * W->Rr[r] * W->g[r];
                rhs[(size_t)i * P + (P - 1)] += h * acc;
            }
        }
        /* solve column by column */
        double* Snew = malloc(sizeof(double) * (size_t)n * P);
        for (int p = 0; p < P; ++p) {
            for (int i = 0; i < n; ++i) col[i] = rhs[(size_t)i * P + p];
            lu_solve(W->M, W->piv, n, col);
            for (int i = 0; i < n; ++i) Snew[(size_t)i * P + p] = col[i];
        }
        /* energy sensitivity */
        double* SEnew = malloc(sizeof(double) * P);
        if (net->Q) {
            for (int j = 0; j < N; ++j) {
                double acc = 0.0;
                for (int r = 0; r < R; ++r) acc += net->Q[r] * dterm_dY(net, x, W->k, r, j);
                dedx[j] = acc;
            }
            if (net->self_heating) {
                double acc = 0.0;
                for (int r = 0; r < R; ++r) acc += net->Q[r] * W->Rr[r] * W->g[r];
                dedx[N] = acc;
            }
            for (int p = 0; p < P; ++p) {
                double acc = 0.0;
                for (int i = 0; i < n; ++i) acc += dedx[i] * Snew[(size_t)i * P + p];
                double dp = 0.0;
                if (p < R) dp = net->Q[p] * W->Rr[p];
                else if (p == P - 1 && !net->self_heating) {
                    for (int r = 0; r < R; ++r) dp += net->Q[r] * W->Rr[r] * W->g[r];
                }
                double hist = 0.0;
                for (int j = 1; j <= kk; ++j) hist += alpha[j] * SEh[(size_t)(j - 1) * P + p];
                SEnew[p] = (h * (acc + dp) - hist) / alpha[0];
            }
        } else {
            for (int p = 0; p < P; ++p) SEnew[p] = 0.0;
        }
        /* push */
        int m = nh < HMAX ? nh : HMAX - 1;
        for (int j = m; j >= 1; --j) {
            th[j] = th[j - 1];
            memcpy(Sh + (size_t)j * n * P, Sh + (size_t)(j - 1) * n * P, sizeof(double) * n * P);
            memcpy(SEh + (size_t)j * P, SEh + (size_t)(j - 1) * P, sizeof(double) * P);
        }
        th[0] = t_new;
        memcpy(Sh, Snew, sizeof(double) * n * P);
        memcpy(SEh, SEnew, sizeof(double) * P);
        if (nh < HMAX) nh++;
        free(Snew);
        free(SEnew);
    }
    memcpy(dx_out, Sh, sizeof(double) * n * P);
    memcpy(dE_out, SEh, sizeof(double) * P);
    g_variant = 0;
    free(Sh); free(SEh); free(rhs); free(col); free(dedx);
    work_free(W);
    return rc;
}

int ora_counter_count(void) { return C_COUNT; }
int ora_history_max(void) { return HMAX; }
