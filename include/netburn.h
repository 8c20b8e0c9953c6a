/*
 * netburn.h -- C ABI of the GB300 batched reaction-network burner.
 *
 * The operation: arXiv:2312.02836 (Chen, Johnson, Katz, Smith Clark, Boyd,
 * Zingale, "A Framework for Exploring Nuclear Physics Sensitivity in
 * Numerical Simulations") generates a reaction network's right-hand side and
 * analytic Jacobian (Sec. 2) and integrates it per zone with a stiff
 * implicit integrator, optionally with self-heating (Sec. 2, Microphysics;
 * Sec. 3, every zone of the Castro detonation).  This library does that
 * per-zone burn for many zones at once on one GPU, and the sensitivity of
 * the result to every rate (the quantity the paper's Sec. 1 and Sec. 3 study
 * by re-running with changed networks).
 *
 * Model per zone (state x = [Y_0..Y_{N-1}] plus T9 when self-heating):
 *   lambda_r(T9) = exp(a0 + a1/T9 + a2 T9^(-1/3) + a3 T9^(1/3) + a4 T9
 *                      + a5 T9^(5/3) + a6 ln T9)      (ReacLib fit, Sec. 2)
 *   R_r   = scale_r exp(p_r) rho^(n_r-1) lambda_r(T9) prod_j Y_j
 *   dY_i/dt = sum_r c_ir R_r,   c_ir = #i in products - #i in reactants
 *   edot  = sum_r Q_r R_r,  dE/dt = edot,  dT9/dt = edot / c_v,
 *   c_v   = 1.5 sum_i Y_i + 1e-3 T9^3
 * Integrator: variable-step, variable-order (1..5) BDF in Lagrange form with
 * a modified Newton iteration (the VODE family named in Sec. 2), with the
 * step, order and Newton rules listed in this project's design notes.
 *
 * Conventions for every entry point:
 *  - Return value: NB_OK (0) or a negative NB_E* code; nb_strerror() names it.
 *    Argument checks happen before any GPU work; on error nothing is written.
 *  - Device pointers are owned by the caller and must stay valid until the
 *    work queued on `stream` has finished.  Work is asynchronous on `stream`
 *    (a cudaStream_t passed as void*; NULL = the legacy default stream)
 *    unless the function says otherwise.
 *  - Arrays are dense, row-major, FP64 unless stated: [Z, N] means zone-major.
 *  - Per-zone outcomes are in status[] (NB_Z_*), never an error code.
 *  - An nb_net is not safe for concurrent burns from several host threads:
 *    its device workspace is shared.
 */
#ifndef NETBURN_H
#define NETBURN_H

#ifndef __CUDACC_RTC__ /* also read by the library's run-time compiled kernels */
#include <stddef.h>
#include <stdint.h>
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* call-level error codes */
#define NB_OK 0
#define NB_E_ARG -1          /* bad argument (null pointer, size, tolerance) */
#define NB_E_TOPOLOGY -2     /* species index out of range, empty reaction */
#define NB_E_TOO_LARGE -3    /* network exceeds the compiled limits */
#define NB_E_CUDA -4         /* a CUDA runtime call failed */
#define NB_E_NOMEM -5        /* host or device allocation failed */
#define NB_E_TAPE -6         /* tape missing, too small or from another net */
#define NB_E_COMPILE -7      /* the network-specialised kernel could not be
                                generated, compiled or loaded */

/* per-zone status */
#define NB_Z_OK 0
#define NB_Z_MAX_STEPS 1     /* more than max_attempts step attempts */
#define NB_Z_DT_UNDERFLOW 2  /* step below 1e-30 t_end or 1e-14 t */
#define NB_Z_NEWTON_FAIL 3   /* 10 consecutive Newton failures */
#define NB_Z_TAPE_FULL 4     /* adjoint tape capacity exceeded */
#define NB_Z_NONFINITE 5     /* non-finite input, rate or first derivative */
#define NB_Z_TIMEOUT 6       /* the call's time budget ran out before the zone
                                finished (outputs: the state reached) */
#define NB_Z_SINGULAR 7      /* 10 consecutive failed attempts, the last of them
                                because the LU of alpha0 I - h J broke down: a
                                zero or non-finite pivot, or a static pivot
                                that lost more than 40 bits to cancellation */

/* per-zone counters, counters[z * NB_NCOUNT + c] */
#define NB_NCOUNT 9
#define NB_C_ACCEPTED 0
#define NB_C_REJ_ERROR 1
#define NB_C_REJ_NEWTON 2
#define NB_C_NEWTON_ITERS 3
#define NB_C_JACOBIANS 4     /* = LU factorizations */
#define NB_C_RHS 5
#define NB_C_RATE_EVALS 6    /* evaluations of all lambda_r(T9) */
#define NB_C_EDOT 7          /* energy-only evaluations for E */
#define NB_C_ORDER_SUM 8     /* sum of the BDF orders of the accepted steps: with
                                the counts above, a fingerprint of the path the
                                step and order control took */

#ifndef __CUDACC_RTC__ /* the run-time compiled kernels need only the codes above */
typedef struct nb_net_s* nb_net;

/* Network topology (host pointers, copied by nb_net_load). */
typedef struct {
  int32_t n_species;        /* N >= 1 */
  int32_t n_reactions;      /* R >= 0 */
  const int16_t* reactants; /* [R, 3] species indices, -1 padded; >= 1 each */
  const int16_t* products;  /* [R, 3] species indices, -1 padded */
  const double* Q;          /* [R] energy per reaction, or NULL (no E) */
  const double* scale;      /* [R] constant factor scale_r, or NULL (= 1) */
  int32_t self_heating;     /* 1: T9 is integrated (requires Q) */
  /* (alpha,p)(p,gamma) effective rates (Sec. 2: A(a,p)X(p,g)B taken as one
   * A(a,g)B rate when proton capture on X is fast and the proton flow
   * through X is in equilibrium).  ap_pg [R] or NULL: 1 marks reaction r as
   * effective, 0 a plain fit.  ap_coeffs [R, 3, 7] (required with ap_pg):
   * the fits of the (a,p), (p,g) and (p,a) channels; coeffs[r] is then the
   * direct (a,g) channel.  X in steady state gives
   *   lambda_r = lambda_ag + lambda_ap lambda_pg / (lambda_pg + lambda_pa),
   * and the multiplier p_r scales the whole effective rate. */
  const int8_t* ap_pg;
  const double* ap_coeffs;
  /* Weak screening (Salpeter 1954): R_r is multiplied by exp(H_r),
   * H_r = s_r sqrt(rho zeta) T6^(-3/2), T6 = 1e3 T9.  screen [R] or NULL (no
   * screening): s_r = 0.188 sum Z_a Z_b over the reactants' successive
   * pairs.  zeta, the plasma parameter sum (Z_i^2 + Z_i) Y_i, is a per-zone
   * input (nb_options.zeta_zone) held over the burn. */
  const double* screen;
  /* Tabulated rates (Sec. 2: TabularRate, weak rates tabulated in
   * (rho Ye, T)).  tab_of [R] or NULL: the table of reaction r, -1 = its
   * fit; tables 0..n_tab-1 share one grid of tab_nd density nodes tab_dens
   * [tab_nd] (log10(rho Ye), increasing) and tab_nt temperature nodes tab_t9
   * [tab_nt] (T9, increasing), and hold ln lambda at the nodes in tab_lnl
   * [n_tab, tab_nd, tab_nt].  ln lambda is bilinear in (log10 rho Ye, T9)
   * between nodes and clamped to the grid's edges.  charge [N] (required
   * with tables): Z_i; Ye = sum Z_i Y_i of the zone's initial composition,
   * held over the burn.  A reaction is tabulated or effective, not both. */
  const int32_t* tab_of;
  int32_t tab_nd, tab_nt;
  const double* tab_dens;
  const double* tab_t9;
  const double* tab_lnl;
  const double* charge;
} nb_topology;

typedef struct {
  int32_t n_state;          /* N + self_heating */
  int32_t n_reactions;
  int32_t nnz_jacobian;     /* structural nonzeros of alpha0 I - h J */
  int32_t nnz_lu;           /* after the fill of the pre-ordered LU */
  int32_t n_dterms;         /* distinct (reaction, reactant) derivatives */
  int32_t lane_doubles;     /* device workspace per zone in flight */
  int32_t blob_bytes;       /* compiled network size (shared memory) */
  int32_t has_energy;
  /* algorithmic FP64 operations per event, an FMA counted as 2; exp, log,
   * cbrt, pow, sqrt and divisions are special functions, not flops */
  int64_t flops_rate_eval;  /* all k_r at one T9 (NB_C_RATE_EVALS) */
  int64_t flops_rate_deriv; /* extra for d ln lambda_r/dT9 (self-heating Jacobian) */
  int64_t flops_terms;      /* R_r = k_r prod Y (per RHS and per E evaluation) */
  int64_t flops_rhs;        /* f from R_r (NB_C_RHS) */
  int64_t flops_jacobian;   /* derivative terms + assembly of M (NB_C_JACOBIANS) */
  int64_t flops_lu;         /* static-pivot factorisation (NB_C_JACOBIANS) */
  int64_t flops_solve;      /* forward + back substitution (NB_C_NEWTON_ITERS) */
  int64_t flops_edot;       /* edot from R_r (NB_C_EDOT) */
  int64_t flops_tsolve;     /* transposed solves of the adjoint, per cotangent */
  int32_t exp_per_rate_eval;
  int32_t specialize_auto;  /* 1: burns with options.specialize = 0 use the
                               network-specialised kernel (when it builds) */
  int32_t last_specialized; /* storage variant of the specialised kernel the
                               last burn ran, 0 = a generic kernel */
  int32_t reserved;
} nb_net_info;

typedef struct {
  int32_t max_attempts;     /* step attempts per zone (default 500000) */
  int32_t kernel;           /* NB_KERNEL_* */
  int32_t threads_per_block;/* 0 = 128; a multiple of 32, at most 256
                               (128 for the plain kernel) */
  int32_t blocks_per_sm;    /* 0 = library choice (persistent kernel); the
                               warp kernel (NB_KERNEL_COOP) with >= 3 and
                               threads_per_block <= 128 runs its variant
                               built for three blocks per SM (registers
                               capped at 168) */
  int32_t blob_in_shared;   /* -1 auto, 0 global (L1), 1 shared memory */
  int32_t ws_in_shared;     /* persistent kernel: the first ws_in_shared warps
                               of each block keep their Newton-loop arrays in
                               shared memory (history stays in global
                               memory); <= 0: all work arrays in the global
                               workspace (the default) */
  int32_t schedule;         /* persistent kernel claim order: 0 zone index
                               order; 1 longest first (default): a pre-pass
                               computes every zone's starting step h0 (the
                               integrator's own start-up) and zones are
                               claimed in increasing h0, which tracks their
                               step count, so the last zones claimed are
                               short and a warp's lanes get alike zones */
  int32_t specialize;       /* persistent kernel, generic or specialised:
                               0 (default) automatic: the kernel generated
                               for this network (see nb_net_specialize) when
                               the network is small enough for it and it
                               builds, else the generic kernel; -1 always the
                               generic kernel; 1..3 the specialised kernel
                               with that storage variant (NB_E_COMPILE when it
                               cannot be built).  Ignored with ws_in_shared
                               > 0 and by nb_burn_batch_noalloc (always the
                               generic kernel). */
  const double* t_end_zone; /* [Z] device array of per-zone end times, or NULL
                               (every zone burns to t_end): operator-split use,
                               each zone burning for its own hydro step.
                               A negative or non-finite entry gives that zone
                               NB_Z_NONFINITE.  Every burn entry point (a
                               device pointer in nb_burn_batch_host too). */
  double time_budget_s;     /* > 0: device watchdog.  Every lane reads the GPU
                               timer between step attempts; once the budget,
                               counted from the start of its block, has run
                               out it ends its zone with NB_Z_TIMEOUT and
                               ends every zone it claims after that the same
                               way, so the call always finishes.  0: none. */
  const double* zeta_zone;  /* [Z] device array of per-zone plasma parameters
                               for screening, or NULL (no screening).  A
                               negative or non-finite entry gives that zone
                               NB_Z_NONFINITE. */
  int32_t warps_per_zone;   /* NB_KERNEL_COOP: 0 or 1, one warp per zone;
                               2 or 4, a block of that many warps integrates
                               one zone (one zone per block, its arrays in
                               shared memory once, the LU pairs, reactions
                               and slots spread over 64 or 128 threads):
                               for networks whose per-zone arrays let few
                               warps share an SM.  threads_per_block is then
                               ignored.  Other values: NB_E_ARG. */
} nb_options;

#define NB_KERNEL_AUTO (-1)     /* adjoint only: the choice made for opt NULL */
#define NB_KERNEL_PERSISTENT 0  /* lane-per-zone, device work queue */
#define NB_KERNEL_PLAIN 1       /* one thread per zone, no queue */
#define NB_KERNEL_COOP 2        /* warp-per-zone, device work queue: the
                                   zone's Newton-loop arrays in shared memory
                                   and its vector, Jacobian and LU work spread
                                   over the warp's lanes (large networks).
                                   threads_per_block: warps per block x 32
                                   (default: as many as fit, at most 4);
                                   ws_in_shared 0: arrays in global memory */

/* Compile a network: validate the topology, build the Jacobian sparsity
 * pattern, choose a minimum-degree elimination order, compute the LU fill
 * and the gather programs, and upload them to the current device.
 * coeffs: [R, 7] host array of (a0..a6).  *out receives a handle to free
 * with nb_net_free.  NB_E_TOO_LARGE when the state exceeds 4096 entries,
 * the reactions 32767, or the pre-ordered LU fills the pattern of
 * alpha0 I - h J to more than 4 times its nonzeros (nb_net_info reports
 * both counts).  Synchronous. */
int nb_net_load(const nb_topology* topo, const double* coeffs, nb_net* out);
int nb_net_free(nb_net net);
int nb_net_get_info(nb_net net, nb_net_info* out);

/* Fill *opt with the defaults. */
void nb_default_options(nb_options* opt);

/* Burn Z zones from t = 0 to t_end.
 *  Y0 [Z, N], T9_0 [Z], rho [Z]       device inputs
 *  ln_mult   NULL, [R] (per_zone = 0) or [Z, R] (per_zone = 1): p_r above
 *  Y [Z, N], T9 [Z]                   device outputs (may alias Y0, T9_0)
 *  E [Z]                              device output or NULL (0 without Q)
 *  counters [Z, NB_NCOUNT] int32, status [Z] int32  device outputs
 *  rtol > 0, atol > 0, t_end >= 0.  opt may be NULL (defaults).
 *  tape: NULL, or a tape from nb_tape_alloc to record the accepted
 *  schedule for nb_burn_adjoint.  Z = 0 is a no-op. */
int nb_burn_batch(nb_net net, int64_t Z, const double* Y0, const double* T9_0,
                  const double* rho, double t_end, double rtol, double atol,
                  const double* ln_mult, int32_t ln_mult_per_zone, double* Y,
                  double* T9, double* E, int32_t* counters, int32_t* status,
                  const nb_options* opt, void* tape, void* stream);

/* Predicted cost of burning each zone, for splitting zones across GPUs
 * with balanced work (the paper's zones sit on a hydro grid, where burn
 * cost follows the local temperature and density, so equal zone counts
 * need not be equal work).  cost [Z] device output: (1 + ln(t_end/h0))^2,
 * h0 the starting step of the integrator's own start-up (0 for a zone that
 * finishes in start-up).  Arguments as for nb_burn_batch; from opt:
 * t_end_zone and zeta_zone.  Asynchronous on stream. */
int nb_zone_costs(nb_net net, int64_t Z, const double* Y0, const double* T9_0,
                  const double* rho, double t_end, double rtol, double atol,
                  const nb_options* opt, double* cost, void* stream);

/* Same burn from HOST arrays (pageable or pinned): copies the inputs to
 * library-owned device buffers, burns, copies the outputs back and waits
 * for the stream.  Synchronous.  E, counters may be NULL. */
int nb_burn_batch_host(nb_net net, int64_t Z, const double* Y0,
                       const double* T9_0, const double* rho, double t_end,
                       double rtol, double atol, const double* ln_mult,
                       int32_t ln_mult_per_zone, double* Y, double* T9,
                       double* E, int32_t* counters, int32_t* status,
                       const nb_options* opt, void* stream);

/* Adjoint tape (Sec. 1 and 3: the rate sensitivity of a burn), in device
 * memory owned by the tape.  Per zone it holds, for up to max_steps
 * accepted steps, the schedule of every step (time t_s, step size h_s, BDF
 * order), and states x_s, E_s only at checkpoints: the initial state and
 * the last min(ckpt_stride, 7) states of every block of ckpt_stride steps,
 * the BDF history window from which nb_burn_adjoint recomputes each block's
 * states, bit for bit, in its reverse sweep.  Memory per zone is about
 * 17 (max_steps + 1) + 8 (n + 1) (1 + 7 max_steps / ckpt_stride) bytes
 * (n = N + self_heating).  ckpt_stride: 1 keeps every state (no
 * recomputation); 0 takes NB_TAPE_DEFAULT_STRIDE.  Synchronous. */
#define NB_TAPE_DEFAULT_STRIDE 16
int nb_tape_alloc(nb_net net, int64_t Z, int32_t max_steps, int32_t ckpt_stride,
                  void** tape);
int nb_tape_free(void* tape);
/* Device pointer to the record counts [Z] int32 (accepted steps + 1) of the
 * last burn recorded on the tape. */
int nb_tape_steps(void* tape, const int32_t** steps);
/* Copy zone z's record of the last burn on the tape to HOST arrays: per
 * record s = 0 .. count-1 (s = 0 the initial point, s >= 1 accepted step s)
 * t [cap], h [cap] (the step size that step used; 0 for s = 0), order [cap]
 * (its BDF order; 0 for s = 0), x [cap, n] and E [cap] (the state and energy
 * after it where the tape keeps them, NaN elsewhere; every record with
 * ckpt_stride 1).  Any array may be NULL.  *count receives the record
 * count; NB_E_ARG (arrays untouched) when it exceeds cap, NB_E_TAPE when
 * the tape holds no burn.  Waits for the device (cudaDeviceSynchronize). */
int nb_tape_read(void* tape, int64_t z, int32_t cap, double* t, double* h,
                 int32_t* order, double* x, double* E, int32_t* count);

/* Discrete adjoint of a recorded burn (same net, same ln_mult, same
 * inputs).  K cotangent sets per zone:
 *  gY [K, Z, N], gE [K, Z] or NULL, gT9 [K, Z] or NULL   device inputs
 *  d_ln_mult [K, Z, R]   device output: d(sum of cotangent . outputs)/dp_r
 *  dY0 [K, Z, N] or NULL, dT0 [K, Z] or NULL  device outputs
 * The schedule (step times and orders) is held fixed and the Newton
 * solutions are treated as exact: this is the exact gradient of the
 * discrete map the forward burn computed.  The reverse sweep takes the
 * blocks of ckpt_stride steps last to first, recomputes each block's states
 * from its checkpoint with the forward's own step computation (same bits),
 * then reverses the block.  Zones whose forward status was not NB_Z_OK get
 * zero gradients; a zone whose recomputation failed to converge (which the
 * forward's convergence on the same inputs excludes) gets NaN. */
int nb_burn_adjoint(nb_net net, void* tape, int32_t K, const double* gY,
                    const double* gE, const double* gT9, double* d_ln_mult,
                    double* dY0, double* dT0, void* stream);
/* nb_burn_adjoint with launch options (opt NULL, or opt->kernel
 * NB_KERNEL_AUTO: as nb_burn_adjoint, which on a tape with checkpoint stride
 * above 1 recomputes in the arithmetic of the burn that recorded it (one
 * lane per zone after NB_KERNEL_PERSISTENT or NB_KERNEL_PLAIN, one warp per
 * zone after NB_KERNEL_COOP), and at stride 1 runs one warp per zone for
 * networks of 24 or more state entries and one lane per zone below).  From
 * opt: kernel (NB_KERNEL_PERSISTENT one lane per zone, NB_KERNEL_COOP one
 * warp per zone; at stride above 1 it must be the recording burn's family,
 * else NB_E_TAPE, because the other family's arithmetic would recompute
 * states that differ from the recorded burn's in the last bits; a tape
 * recorded with warps_per_zone > 1 is read only at stride 1),
 * threads_per_block (lane kernel at
 * most 128; warp kernel: warps per block x 32, at most 256, default as many
 * as fit in shared memory up to 4), blocks_per_sm, ws_in_shared (0: the
 * warp kernel keeps its arrays in global memory) and blob_in_shared (0: the
 * warp kernel reads the network from global memory).  Every kernel and
 * launch shape gives the same gradients up to the rounding of the
 * transposed solves and sums. */
int nb_burn_adjoint_ex(nb_net net, void* tape, int32_t K, const double* gY,
                       const double* gE, const double* gT9, double* d_ln_mult,
                       double* dY0, double* dT0, const nb_options* opt, void* stream);

/* Burn without any device allocation.  The paper has no counterpart: this is
 * for callers that may not allocate device memory while they run the burn
 * (a solver whose memory is reserved up front by its own pool, a time step
 * run while another library owns the allocator, code that cannot afford the
 * implicit synchronisation of cudaMalloc/cudaFree).  Same arguments and
 * results as nb_burn_batch (same per-zone integration, bit for bit), without
 * a tape; the caller passes every input and output.
 *  - Scratch: the work-queue counter and the per-zone workspace live in one
 *    array of NB_NOALLOC_SCRATCH_BYTES compiled into the library, which every
 *    GPU that loads the library keeps until the process exits.  The number
 *    of zones in flight is capped so that their workspace fits; any Z works.
 *    NB_E_TOO_LARGE when not even one block of threads_per_block zones fits
 *    (a network whose per-zone workspace exceeds the array).
 *  - Options: those of nb_burn_batch (per-zone end times, plasma
 *    parameters, watchdog, launch shape), except that threads_per_block is
 *    at most 128 (NB_E_ARG beyond) and specialize and ws_in_shared are
 *    ignored: this entry point always runs the generic kernel, so its bits
 *    are those nb_burn_batch gives with specialize = -1.
 *  - Set-up: the first call on each device looks up the array's device
 *    address (cudaGetSymbolAddress) with that device current and keeps it
 *    for the life of the process; make that first call before any stream
 *    capture on the device.  A cudaDeviceReset discards the array and makes
 *    the kept address stale: do not use this entry point after a reset.
 *  - All calls share the one array: calls that can overlap on the GPU (on
 *    different streams, or from several host threads) race and corrupt each
 *    other's results.  Serialise them.  Each call zeroes the counter itself;
 *    the workspace needs no clearing (every zone initialises its own). */
#define NB_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
int nb_burn_batch_noalloc(nb_net net, int64_t Z, const double* Y0,
                          const double* T9_0, const double* rho, double t_end,
                          double rtol, double atol, const double* ln_mult,
                          int32_t ln_mult_per_zone, double* Y, double* T9,
                          double* E, int32_t* counters, int32_t* status,
                          const nb_options* opt, void* stream);

/* Several networks in one launch.  The paper's study burns the same hydro
 * zones with different networks to see which nuclear physics matters
 * (Sec. 3, 4).  nb_burn_multi burns up to NB_MULTI_MAX_SETS sets, each a
 * network with its own zones and arrays (as for nb_burn_batch, device
 * pointers, [Z, N] with that network's N), in one persistent launch whose
 * device queue spans all of them: a few expensive zones of a large network
 * and many cheap zones of a small one share the GPU's lanes.  Sets of larger
 * networks are claimed first, and within a set (schedule 1, the default)
 * the zones longest first by their starting step, as nb_burn_batch orders
 * them.  Every zone follows the generic kernel, bit for bit the result
 * nb_burn_batch gives it.  t_end, rtol and atol are common; t_end_zone (per
 * set, may be NULL) overrides t_end per zone.  From opt: max_attempts,
 * threads_per_block (<= 128), blocks_per_sm, schedule and time_budget_s; no
 * tape, no specialised kernel.  All networks must live on the current
 * device.  The first set's network lends its device workspace and its
 * scheduling buffers: do not burn with it concurrently.  Asynchronous on
 * stream. */
#define NB_MULTI_MAX_SETS 12
typedef struct {
  nb_net net;
  int64_t Z;
  const double* Y0;         /* [Z, N] */
  const double* T9_0;       /* [Z] */
  const double* rho;        /* [Z] */
  const double* ln_mult;    /* NULL, [R] or [Z, R] */
  int32_t ln_mult_per_zone;
  const double* t_end_zone; /* [Z] or NULL */
  const double* zeta_zone;  /* [Z] plasma parameters (screening) or NULL */
  double* Y;                /* [Z, N] out */
  double* T9;               /* [Z] out */
  double* E;                /* [Z] out or NULL */
  int32_t* counters;        /* [Z, NB_NCOUNT] out or NULL */
  int32_t* status;          /* [Z] out */
} nb_burn_set;
int nb_burn_multi(int32_t n_sets, const nb_burn_set* sets, double t_end, double rtol,
                  double atol, const nb_options* opt, void* stream);
/* Network-specialised kernel.  The paper's pynucastro writes each network
 * as its own code, every rate, RHS term and Jacobian entry spelled out
 * (Sec. 2).  The generic kernel instead walks the compiled network from
 * memory.  nb_net_specialize prints the network as straight-line CUDA (every
 * coefficient a literal, every index a constant), compiles it for sm_103a
 * with the CUDA run-time compiler (libnvrtc, loaded on first use) and loads
 * it; burns then use it as options.specialize says.  It performs the
 * generic kernel's floating-point operations in the same order, so both give
 * the same bits.
 *  variant  0: chosen from the network's sizes; 1: all Newton-loop arrays of
 *           a zone in registers; 2: as 1 with the LU in the workspace;
 *           3: only x, d, f in registers.
 *  log      NULL or a host buffer of log_bytes for the compiler's log
 *           (NUL-terminated, truncated to fit).
 * Synchronous; compiling takes seconds.  NB_E_COMPILE on failure.  A kernel
 * built once is kept with the network. */
int nb_net_specialize(nb_net net, int32_t variant, char* log, int64_t log_bytes);
/* The specialised kernel's source for a topology, without any GPU: host
 * buffer buf of cap bytes (NUL-terminated when it fits); *len = source
 * length in bytes (without the NUL).  NB_E_ARG when cap is too small (buf
 * untouched, *len set). */
int nb_specialize_source(const nb_topology* topo, const double* coeffs,
                         int32_t variant, char* buf, int64_t cap, int64_t* len);
/* Generate and compile the specialised kernel for a topology without any GPU
 * (a build check): NB_OK or NB_E_COMPILE; log as for nb_net_specialize,
 * including the register and spill report of the sm_103a assembler. */
int nb_specialize_compile(const nb_topology* topo, const double* coeffs,
                          int32_t variant, char* log, int64_t log_bytes);
/* The FP64 exp the rate evaluation uses (Tang's table-driven method, see
 * the kernels' expf64.cuh), and optionally the CUDA library exp, on a device
 * array x [n]: y_tang [n] (and y_lib [n] unless NULL).  A diagnostic for
 * its error bound; the paper has no counterpart.  Asynchronous on stream. */
int nb_exp_eval(const double* x, double* y_tang, double* y_lib, int64_t n,
                void* stream);

const char* nb_strerror(int code);

#endif /* __CUDACC_RTC__ */
#ifdef __cplusplus
}
#endif
#endif /* NETBURN_H */
