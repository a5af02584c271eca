/*
 * at_dns.h -- C ABI of the GB300 (sm_103a) library for one explicit time step
 * of the compressible Navier-Stokes equations with Asynchrony-Tolerant (AT)
 * finite differences at the faces of virtual processing elements (PEs).
 *
 * Method: Kumari & Donzis, "Direct numerical simulations of turbulent flows
 * using high-order asynchrony-tolerant schemes: accuracy and performance",
 * arXiv 2003.10561.
 *   - equations: Sec. 2, Eqs. (cont), (mome), (ie) (solved here in total-energy
 *     form E = rho e + rho|u|^2/2, divergence form for the inviscid flux);
 *   - 4th-order central stencils inside a PE and AT stencils at PE faces:
 *     Sec. 2.1, Eq. (at) and Table B (Appendix B), T_l = 3 time levels; or
 *     the 6th-order rows of Table B (T_l = 4) with 6th-order stencils inside
 *     (the sixth-order comparison of Sec. 4.1.2);
 *   - mixed derivatives by the three-step rule of Sec. 2.1;
 *   - second-order Adams-Bashforth with a fixed dt: Sec. 2.2, Eq. (time_ab);
 *   - PE decomposition, control parameters c_r and L, storage of L + T_l
 *     levels: Sec. 3, Eqs. (NT)-(NB), Sec. 3.1;
 *   - delays: synchronous, periodic (Communication-Avoiding, Algorithm 2) or
 *     random (Synchronization-Avoiding, Algorithm 1), the random ones drawn
 *     from Philox4x32-10 instead of a network;
 *   - large-scale solenoidal forcing on |kappa| <= kappa_f: Sec. 4.2.
 *
 * Units: rho_0 = T_0 = c_0 = 1, so p = rho T / gamma, c^2 = T and
 * c_p = 1/(gamma-1).  Viscosity mu = mu0 T^visc_exp (power law, default) or
 * Sutherland's law mu0 T^(3/2) (1 + S) / (T + S); conductivity
 * k = mu c_p / Pr.  The box is (2 pi)^3, dx_d = 2 pi / n[d].
 *
 * Field layout (every state array crossing this ABI): FP64, structure of
 * arrays [5][n[2]][n[1]][n[0]] -- variable (rho, rho u, rho v, rho w, E)
 * (with energy_form = AT_DNS_ENERGY_INTERNAL the fifth variable is rho e),
 * then z, y, x with x fastest -- i.e. 5 * n0 * n1 * n2 doubles.
 *
 * Ownership: the library owns every device allocation it makes (released by
 * at_dns_destroy), unless the configuration hands it a device pool: then all
 * of the handle's device memory is carved from that region, which the caller
 * owns and must keep alive until at_dns_destroy.  Caller buffers are read or
 * written only during the call;
 * `where` says whether a pointer is host (AT_DNS_HOST, any pageable or pinned
 * memory) or device (AT_DNS_DEVICE, memory of the handle's device).
 *
 * Errors: every int-returning call returns AT_DNS_OK (0) or a negative
 * AT_DNS_E_* code and never throws; at_dns_last_error() gives a text.
 * Calls on one handle are ordered on its stream and are not thread-safe.
 */
#ifndef AT_DNS_H
#define AT_DNS_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define AT_DNS_OK              0
#define AT_DNS_E_INVALID_ARG  -1   /* bad pointer, size, mode or configuration */
#define AT_DNS_E_OOM          -2   /* a device allocation failed */
#define AT_DNS_E_CUDA         -3   /* a CUDA runtime call failed */
#define AT_DNS_E_UNSTABLE     -4   /* NaN/Inf, rho <= 0 or p <= 0 seen in a step */
#define AT_DNS_E_UNSUPPORTED  -5   /* a combination the library does not run */
#define AT_DNS_E_STATE        -6   /* no state has been set yet */
#define AT_DNS_E_TOO_LARGE    -7   /* problem above a fixed size limit (at_dns_rhs_noalloc) */
#define AT_DNS_E_TIMEOUT      -8   /* a bounded wait inside a kernel gave up (persistent batch step) */
#define AT_DNS_E_BOUNDS       -9   /* bounds-checked builds only (compiled with -DAT_DNS_CHECKS): an
                                      index check in a kernel failed; the access was redirected to
                                      index 0 of its buffer, so results of the call are not valid */

/* delay modes (Sec. 3.1) */
#define AT_DNS_SYNC      0   /* k = 0 on every face: standard scheme */
#define AT_DNS_PERIODIC  1   /* CAA: k = (n - n0) mod c_r (Algorithm 2) */
#define AT_DNS_RANDOM    2   /* SAA: k iid uniform on {0..L} (Algorithm 1) */
#define AT_DNS_FIXED     3   /* k = L on every face after the start-up: the worst case
                                of the stability analysis (Sec. 3.2) */
#define AT_DNS_ORDERED   4   /* SAA with ordered arrivals: a PE's messages arrive in order
                                (Algorithm 1 tests its receives each step), so the newest
                                level received ages by at most one step per step:
                                k_n = min(d_n, k_{n-1} + 1) over the AT_DNS_RANDOM draws d,
                                k = 0 through the start-up; a pure function of
                                (seed, n, PE, face) via the last L + 1 draws */

/* precision forms */
#define AT_DNS_P64  0        /* FP64 storage and arithmetic */
#define AT_DNS_P32  1        /* FP32 state, stencils, update and ring; FP64 reductions */
#define AT_DNS_P32C 2        /* as P32, but the state is carried as FP32 hi + lo words and
                                updated by TwoSum (compensated, ~48-bit accumulation) */

/* energy forms (Sec. 2) */
#define AT_DNS_ENERGY_TOTAL     0   /* fifth variable E = rho e + rho|u|^2/2, divergence form */
#define AT_DNS_ENERGY_INTERNAL  1   /* fifth variable rho e, Eq. (ie): source -p theta + sigma S + conduction */

/* viscosity laws (Sec. 2) */
#define AT_DNS_VISC_POWER       0   /* mu0 T^visc_exp */
#define AT_DNS_VISC_SUTHERLAND  1   /* mu0 T^(3/2) (1 + S) / (T + S), S = sutherland_s */

/* time integrators (Sec. 2.2) */
#define AT_DNS_AB2  0   /* second-order Adams-Bashforth, Eq. (time_ab): the paper's integrator for AT */
#define AT_DNS_RK3  1   /* low-storage three-stage RK3 (Williamson 1980), synchronous steps only */

/* pointer locations */
#define AT_DNS_HOST    0
#define AT_DNS_DEVICE  1

typedef struct at_dns at_dns_t;   /* opaque handle; owned by the library */

typedef struct {
  int32_t  n[3];         /* grid points in x, y, z (each >= order + 1)                  */
  int32_t  pes[3];       /* virtual PEs per direction; n[d] % pes[d] == 0 and, when
                            pes[d] > 1, n[d]/pes[d] >= order + 1.  pes[d] == 1: no
                            faces in d                                                  */
  double   gamma;        /* ratio of specific heats (1.4)                               */
  double   prandtl;      /* Prandtl number (0.7)                                        */
  double   mu0;          /* viscosity at T = 1                                          */
  double   visc_exp;     /* power-law exponent omega (0.76)                             */
  double   dt;           /* fixed time step; <= 0: set from cfl when a state is set     */
  double   cfl;          /* convective CFL used when dt <= 0                            */
  int32_t  max_delay;    /* L >= 0: largest delay; the ring holds L + T_l levels        */
  int32_t  comm_period;  /* c_r >= 1 for AT_DNS_PERIODIC; needs c_r - 1 <= L            */
  uint64_t seed;         /* key of the random delay stream                              */
  int32_t  forcing;      /* 0: decaying; 1: OU solenoidal forcing on |kappa| <= kf      */
  double   kf;           /* forcing shell radius kappa_f (<= 4)                         */
  double   f_amp;        /* OU amplitude sigma of each forcing coefficient              */
  double   f_tcorr;      /* OU correlation time T_f                                     */
  uint64_t f_seed;       /* key of the forcing noise stream                             */
  int32_t  precision;    /* AT_DNS_P64, AT_DNS_P32 or AT_DNS_P32C                       */
  int32_t  stats_every;  /* 1: reduce statistics in every step; 0: only on request      */
  void*    stream;       /* cudaStream_t to run on; NULL = the legacy default stream    */
  int32_t  kernel_path;  /* AT_DNS_PATH_AUTO, _MULTIPASS, _FUSED or _PAIRED              */
  int32_t  order;        /* spatial order: 4 (Table B (1,4)/(2,4), T_l = 3, default) or
                            6 (Table B (1,6)/(2,6), T_l = 4; multi-pass path only)      */
  int32_t  energy_form;  /* AT_DNS_ENERGY_TOTAL (default) or AT_DNS_ENERGY_INTERNAL     */
  int32_t  visc_law;     /* AT_DNS_VISC_POWER (default) or AT_DNS_VISC_SUTHERLAND        */
  double   sutherland_s; /* S, Sutherland temperature / reference temperature (0.368:
                            110.4 K over 300 K; the paper gives no constants)           */
  int32_t  integrator;   /* AT_DNS_AB2 (default) or AT_DNS_RK3 (AT_DNS_SYNC steps only:
                            the stages of an RK step would need a synchronisation each) */
  void*    pool;         /* NULL, or device memory (256-byte aligned) the handle carves all
                            of its buffers from -- e.g. a framework tensor; OOM if too small.
                            Each handle (and each batch member) needs its own region. */
  size_t   pool_bytes;   /* size of the pool                                            */
  int32_t  extrapolate_state;
                         /* what Table B's weights extrapolate at a delayed stencil point
                            (Sec. 2.1, Eq. (at)): 0 (default) each differentiated
                            quantity -- flux, velocity, temperature -- at the levels
                            n-k-l; 1 the state U, the quantities then evaluated once from
                            sum_l w_l(k) U^{n-k-l}.  The two agree without delays and for
                            quantities linear in U                                      */
} at_dns_config_t;

/* kernel paths (same results up to rounding): the multi-pass path stores
 * derived fields and gradients between kernels; the fused path does one pass
 * over U per step on PE-aligned tiles (needs the per-direction PE extent, or
 * the grid extent where a direction has one PE, to be a multiple of 8 and the
 * tile to hold a multiple of 32 points; 4th order only).  AUTO takes the path
 * that is faster on GB300 at the benchmark workload: for P32 / P32C the paired
 * fused kernel where its tiles fit, else the fused one where it applies;
 * multi-pass otherwise. */
#define AT_DNS_PATH_AUTO       0
#define AT_DNS_PATH_MULTIPASS  1
#define AT_DNS_PATH_FUSED      2
/* the fused pass with two x-adjacent points per thread carried through packed
 * FP32 (f32x2) arithmetic: P32 / P32C only, tiles 32x8, 32x16, 16x16, 16x8
 * (PE extents multiples of 16 in x and 8 in y) */
#define AT_DNS_PATH_PAIRED     3

typedef struct {
  int64_t step;          /* n of the state the statistics describe                      */
  double  time, dt;
  double  mass;          /* <rho>                                                       */
  double  mom[3];        /* <rho u_i>                                                   */
  double  energy;        /* <E>                                                         */
  double  tke;           /* K = <rho u_i u_i / 2>                                       */
  double  dissipation;   /* <sigma_ij S_ij>                                             */
  double  grad_m2, grad_m3, grad_m4;  /* <(du_i/dx_i)^k>, averaged over i = 1..3         */
  double  skewness, flatness;         /* m3 / m2^1.5, m4 / m2^2                          */
  double  enstrophy;     /* <omega_i omega_i>                                           */
  double  pressure_dilatation;        /* <p theta>                                      */
  double  forcing_power; /* <rho f_i u_i>                                               */
  double  urms;          /* sqrt(<u_i u_i>/3)                                           */
  double  mach_t;        /* sqrt(<u_i u_i>) / <c>                                       */
  double  max_wave_speed;/* max over points and d of |u_d| + c                          */
  double  min_rho, min_p;
  int32_t unstable;      /* nonzero: a NaN/Inf, rho <= 0 or p <= 0 was seen             */
} at_dns_stats_t;

typedef struct {
  int64_t step;          /* current level n                                             */
  double  time, dt;
  int32_t n_levels;      /* L + T_l time levels in the ring                             */
  double  boundary_fraction;  /* N_B / N_T per PE, Eqs. (NT)-(NB)                       */
  size_t  device_bytes;  /* device memory held by the handle                            */
  int32_t kernels_per_step;   /* kernel launches of one at_dns_step step                */
  int32_t kernel_path;   /* path in use: AT_DNS_PATH_MULTIPASS, _FUSED or _PAIRED       */
  int32_t tile[3];       /* fused path: TX, TY, planes per CTA (0 on the multi-pass path)*/
  int32_t order;         /* spatial order of the scheme (4 or 6)                        */
} at_dns_info_t;

/* Fill *cfg with defaults: 32^3, one PE, gamma 1.4, Pr 0.7, omega 0.76,
 * mu0 0.01, cfl 0.5 (dt from it), L = 2, c_r = 3, no forcing, P64, stats every
 * step, default stream.  Returns AT_DNS_E_INVALID_ARG if cfg is NULL. */
int at_dns_config_default(at_dns_config_t* cfg);

/* Validate *cfg, allocate device state (double-buffered U, AB2 history,
 * slab ring of L + T_l levels, ghost and derivative work arrays) on the current
 * device and return a handle in *out.  Errors: INVALID_ARG (see the field
 * rules above), OOM, CUDA.  Sec. 3: PE geometry and L + T_l levels. */
int at_dns_create(const at_dns_config_t* cfg, at_dns_t** out);

/* Set U^0 = u (5*N^3 FP64, layout above), step n = 0, t = 0, fill every ring
 * level with U^0 (the synchronous start-up of Algorithms 1 and 2), forget the
 * AB2 history (the next step is forward Euler) and, if cfg.dt <= 0, set
 * dt = cfl / max_{x,d}((|u_d| + c)/dx_d) (Sec. 2.2, fixed dt).
 * Errors: INVALID_ARG (NULL, bad where), CUDA. */
int at_dns_set_state(at_dns_t* h, const double* u, int where);

/* Set a state with an explicit past: levels holds nlevels consecutive fields
 * U^step, U^(step-1), ..., each 5*N^3 FP64 (1 <= nlevels <= L + T_l; missing
 * older levels repeat the oldest one given).  The step counter becomes `step`
 * (>= 0), so the delay map of that step applies to the next rhs/step; the
 * forcing coefficients are advanced to `step`; the AB2 history is forgotten.
 * dt is not recomputed if already set.  Errors: INVALID_ARG, CUDA. */
int at_dns_set_history(at_dns_t* h, const double* levels, int32_t nlevels,
                       int64_t step, int where);

/* Copy U^n out (5*N^3 FP64).  Errors: INVALID_ARG, STATE, CUDA. */
int at_dns_get_state(at_dns_t* h, double* u_out, int where);

/* Evaluate R(U^n), the right-hand side of the conserved variables at the
 * current level with this step's delay map (mode = AT_DNS_*) and forcing,
 * into rhs_out (5*N^3 FP64).  Does not advance time.  Also refreshes the
 * statistics record.  Errors: INVALID_ARG, STATE, CUDA. */
int at_dns_rhs(at_dns_t* h, int32_t delay_mode, double* rhs_out, int where);

/* Advance nsteps AB2 steps (Eq. (time_ab)): for each step n, build the delay
 * map, assemble AT ghost values from the ring, evaluate R(U^n), update
 * U^{n+1} = U^n + dt(3/2 R^n - 1/2 R^{n-1}) (forward Euler on the first step
 * after a state is set), store U^{n+1}'s PE-boundary slabs in the ring and
 * advance the forcing.  With integrator AT_DNS_RK3 a step is the three stages
 * dU = A_s dU + dt R(U), U = U + B_s dU, A = (0, -5/9, -153/128),
 * B = (1/3, 15/16, 8/15), with the forcing of step n in every stage and the
 * statistics of U^n; only AT_DNS_SYNC is accepted.  Asynchronous on the
 * handle's stream except that the health word is read back once at the end.
 * Errors: INVALID_ARG, STATE, CUDA, UNSUPPORTED (RK3 with delays), UNSTABLE
 * (NaN/Inf, rho <= 0 or p <= 0 in any evaluated state; the state is left as
 * computed). */
int at_dns_step(at_dns_t* h, int32_t nsteps, int32_t delay_mode);

/* Statistics of the state at which the last RHS was evaluated (a step or
 * at_dns_rhs).  If none was evaluated since the state was set, one RHS
 * evaluation in synchronous mode is made first (time does not advance).
 * Blocks until the record is on the host.  Errors: INVALID_ARG, STATE, CUDA. */
int at_dns_stats(at_dns_t* h, at_dns_stats_t* out);

/* Delay map of step `step` for delay mode `mode`: out[p*6 + f] for PE
 * p = (pz*Py + py)*Px + px and face f = x-, x+, y-, y+, z-, z+ (host buffer of
 * Px*Py*Pz*6 bytes), computed by the same device code the step uses.
 * Sec. 3.1 / Algorithms 1-2: zero for step < L + T_l; periodic
 * (step - L - T_l) mod c_r; random floor(w0 (L+1) / 2^32) with w0 the first
 * word of Philox4x32-10(counter = (step, p, f, 0x4154), key = (seed lo, seed hi)).
 * Errors: INVALID_ARG, CUDA. */
int at_dns_get_delay_map(at_dns_t* h, int64_t step, int32_t mode, uint8_t* out);

/* Handle facts (step, time, dt, levels, N_B fraction, memory, launches). */
int at_dns_get_info(at_dns_t* h, at_dns_info_t* out);

/* Per-kernel device time, gathered with CUDA events recorded on the handle's
 * stream around every launch while profiling is on. */
typedef struct {
  char    name[24];      /* kernel family: "delay_map", "prim", "ghost", "grad",
                            "force_lines", "main", "stats_final", "force_advance"   */
  int64_t launches;
  double  total_ms;
} at_dns_kernel_time_t;

/* enable = 1: clear the records and start recording an event pair around each
 * launch of at_dns_step / at_dns_rhs; enable = 0: stop.  Errors: INVALID_ARG. */
int at_dns_profile(at_dns_t* h, int32_t enable);

/* Wait for the recorded launches, and write up to `max` kernel families with
 * their launch counts and summed event times into out; *count = families.
 * Errors: INVALID_ARG, CUDA. */
int at_dns_kernel_times(at_dns_t* h, at_dns_kernel_time_t* out, int32_t max, int32_t* count);

/* Autotuner: for the current state, time `trials` right-hand-side
 * evaluations (no state change) of every kernel path that applies -- the
 * multi-pass path and each compiled fused tile shape (32x8, 16x16, 16x8, 8x32,
 * 8x16, 8x8, and 32x16 for P32 / P32C; 4th order only) with whole-PE, half and
 * quarter z chunks -- and
 * keep the fastest
 * (at_dns_get_info reports it).  *best_ms (may be NULL) receives its time per
 * evaluation.  Candidates that cannot get their work arrays are skipped.
 * Errors: INVALID_ARG, STATE, CUDA. */
int at_dns_tune(at_dns_t* h, int32_t delay_mode, int32_t trials, double* best_ms);

/* Select the kernel path explicitly: AT_DNS_PATH_MULTIPASS (tile ignored) or
 * AT_DNS_PATH_FUSED / AT_DNS_PATH_PAIRED with tile = {TX, TY, ZC}, one of the candidates that
 * at_dns_tune times for this handle (a compiled tile shape whose TX and TY
 * divide the PE extents, ZC planes per CTA dividing the PE extent in z).
 * Captured step graphs are dropped; the state is kept.
 * Errors: INVALID_ARG (NULL), UNSUPPORTED (not a candidate), OOM. */
int at_dns_set_kernel_path(at_dns_t* h, int32_t path, const int32_t tile[3]);

/* ---- checkpoints ----------------------------------------------------------
 * The run state of a handle in one self-describing buffer: U^n (and its low
 * words in P32C), R^{n-1}, the FP64 slab ring of the last L + T_l levels, the
 * forcing coefficients, the last statistics record, the step counter, the
 * time step and the start-up (forward Euler) flag, after a header that
 * records the configuration.  The delay map and the forcing noise are pure
 * functions of (seed, step, PE, face) and (f_seed, step, mode), so a handle
 * of the same configuration that loads the buffer continues the saved run
 * bit for bit (the paper's checkpoints serve averaging, Sec. 4).  The layout
 * is this library's own (not a portable file format); sections start at
 * 256-byte offsets. */

/* *bytes receives the size of a checkpoint of h.  Errors: INVALID_ARG. */
int at_dns_checkpoint_size(const at_dns_t* h, int64_t* bytes);

/* Write the run state into buf (where = AT_DNS_HOST or AT_DNS_DEVICE, at least
 * at_dns_checkpoint_size bytes; caller-owned).  Blocks until written.
 * Errors: INVALID_ARG, STATE (no state set), CUDA. */
int at_dns_checkpoint_save(at_dns_t* h, void* buf, int where);

/* Restore the run state from buf into h, whose configuration must equal the
 * saved one (grid, PEs, precision, order, forms, delays, seeds, physical and
 * forcing constants; INVALID_ARG names the first field that differs); the
 * saved time step replaces h's.  The next step continues the saved run.
 * Errors: INVALID_ARG, CUDA. */
int at_dns_checkpoint_load(at_dns_t* h, const void* buf, int where);

/* Block until all work queued on the handle's stream has finished. */
int at_dns_synchronize(at_dns_t* h);

/* ---- batched ensembles --------------------------------------------------
 * Independent members (own grid, PEs, physics, precision, delays) advance
 * together.  Each batch step is one launch of a captured graph holding one
 * step of every member on its own branch (each member on its own kernels and
 * tuned path, bit-identical to the member stepped alone).  Members are
 * ordinary handles (set their state, read them back through
 * at_dns_batch_member); each runs on a stream the batch owns, and a batch
 * step is ordered after earlier work on those streams.
 *
 * Opt-in (at_dns_batch_persistent): when the batch has at most 64 members,
 * every member runs an FP32 form (P32 / P32C), the 4th-order scheme, AB2 and
 * no forcing, and the members' PE extents (grid extents where a direction
 * has one PE) fit one paired tile shape (16x16, or 32x8), a batch step can
 * instead be ONE persistent cooperative kernel launch over work items dealt
 * round-robin to the CTAs: the members' ghost assembly in chunks, then their
 * tiles of the paired fused kernel (each member's description in constant
 * memory), each tile waiting (bounded) for its own member's ghost items
 * only; the CTA that finishes a member's last tile sums its statistics and
 * advances its step.  Each member then takes the arithmetic of the paired
 * kernel with the batch's tile, and agrees with the member stepped alone to
 * about one FP32 rounding of the right-hand side (the same operations,
 * compiled into another kernel: P32C states within the low words).  Constant
 * memory holds one batch's descriptions at a time: stepping another batch
 * re-uploads them, ordered after the earlier batch's last persistent launch.
 * The graph form is the default because it is the faster of the two on
 * GB300: inside one kernel, the tile body reads its coefficients through a
 * table instead of as kernel parameters, and the ghost assembly runs at the
 * tile's occupancy. */
typedef struct at_dns_batch at_dns_batch_t;

/* Create `count` members from cfgs[0..count-1] (their `stream` fields are
 * ignored); `stream` is the cudaStream_t the batch steps run on (NULL: a
 * stream owned by the batch).  Errors: INVALID_ARG, OOM, CUDA. */
int at_dns_batch_create(const at_dns_config_t* cfgs, int32_t count, void* stream, at_dns_batch_t** out);

/* Handle of member i (owned by the batch; do not destroy it). */
int at_dns_batch_member(at_dns_batch_t* b, int32_t i, at_dns_t** out);

/* Advance every member nsteps AB2 steps with delay mode `delay_mode`; blocks
 * until done.  Errors: INVALID_ARG, STATE (a member without state), CUDA,
 * UNSTABLE (a member saw NaN/Inf, rho <= 0 or p <= 0), TIMEOUT (a bounded
 * wait of the persistent step for a member's ghost items gave up; the
 * members' states are then not valid). */
int at_dns_batch_step(at_dns_batch_t* b, int32_t nsteps, int32_t delay_mode);

/* Allow (enable > 0) or forbid (enable == 0, the default) the persistent
 * single-launch step for eligible batches; enable < 0 changes nothing.
 * *persistent (may be NULL) receives 1 if the next at_dns_batch_step runs as
 * one persistent launch per step, 0 if as a graph launch.
 * Errors: INVALID_ARG. */
int at_dns_batch_persistent(at_dns_batch_t* b, int32_t enable, int32_t* persistent);

/* Self-test of the persistent step's bounded wait: one GPU thread waits for
 * a device counter that nothing advances, giving up after at most
 * 2^log2_polls polls about 64 ns apart (log2_polls in [0, 26]); *gave_up
 * receives 1 when the wait returned unsatisfied (the expected result) and
 * the context stays usable.  Errors: INVALID_ARG, CUDA. */
int at_dns_wait_selftest(int32_t log2_polls, int32_t* gave_up);

/* Autotune the batch's graph step as a whole: each member is first tuned
 * alone (at_dns_tune); then the batch step is timed (trials steps after one
 * untimed step) with the members on their paths before the call, on their
 * own picks, and on every tile shape some member supports applied to each
 * member that has it (its largest z chunk), and the fastest of these
 * configurations is kept: members share the GPU in the graph, so the fastest
 * path of a member alone is not always the fastest inside the batch.  The
 * members' run states are saved in device checkpoints before the timed steps
 * and restored after them, so the call leaves every state as it was; without
 * device memory for the checkpoints the members keep their own picks.
 * Errors: INVALID_ARG, STATE, CUDA. */
int at_dns_batch_tune(at_dns_batch_t* b, int32_t delay_mode, int32_t trials);

/* Text of the last batch error (NULL batch: last failed batch create). */
const char* at_dns_batch_last_error(const at_dns_batch_t* b);

/* Destroy the members, their streams and the batch. */
void at_dns_batch_destroy(at_dns_batch_t* b);

/* Largest n[0]*n[1]*n[2] accepted by at_dns_rhs_noalloc (64^3). */
#define AT_DNS_NOALLOC_MAX_POINTS 262144

/* Right-hand side R(U) without any device allocation.  The paper has no
 * counterpart: this serves callers that cannot call cudaMalloc (code running
 * while another component owns all device memory, code inside a region that
 * must not allocate or synchronise, plugins in processes that forbid new
 * allocations after start-up).
 *
 * Computes, in FP64 on the current device, the right-hand side that
 * at_dns_rhs gives for a single PE (periodic box, no PE faces, hence no
 * delays) of a handle with order 4, the total-energy form, the power-law
 * viscosity mu0 T^visc_exp and no forcing: the call always uses the
 * 4th-order central stencils, whatever scheme other handles use.  The
 * physics parameters are given here (all finite): u_dev is the state and
 * rhs_dev receives R, both device pointers to 5*n0*n1*n2 doubles in the
 * layout above; stream is a cudaStream_t (NULL = legacy default stream).
 * The work is queued on that stream and the call returns without waiting.
 *
 * Work arrays come from one file-scope device array of fixed size (about
 * 59 MB, held by every GPU that loads the library until the process exits);
 * no allocation is made.  Its device address is looked up, with the
 * caller's device current, on every call; the first call on a device also
 * loads the library's device code there, so make that first call before any
 * stream capture.  All
 * calls on a device share that array and it keeps the last call's contents:
 * calls whose work can overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.
 * Errors: INVALID_ARG (NULL pointer, n[d] < 5, gamma <= 1, prandtl <= 0,
 * mu0 < 0, or a non-finite gamma, prandtl, mu0 or visc_exp),
 * TOO_LARGE (n0*n1*n2 > AT_DNS_NOALLOC_MAX_POINTS), CUDA. */
int at_dns_rhs_noalloc(const int32_t n[3], double gamma, double prandtl, double mu0, double visc_exp,
                       const double* u_dev, double* rhs_dev, void* stream);

/* Text of the last error on this handle ("" if none); a NULL handle gives the
 * last error of a failed at_dns_create on this thread.  Valid until the next
 * call on the handle. */
const char* at_dns_last_error(const at_dns_t* h);

/* Release every device allocation of the handle.  NULL is ignored. */
void at_dns_destroy(at_dns_t* h);

#ifdef __cplusplus
}
#endif
#endif /* AT_DNS_H */
