/*
 * hgks.h -- C ABI of a GB300 (sm_103a) implementation of one time step of the
 * high-order gas-kinetic scheme (HGKS) of Cao, Pan & Xu, "High-order
 * gas-kinetic scheme with parallel computation for direct numerical
 * simulation of turbulent flows" (arXiv:2005.08736).
 *
 * The problem is stated as in the paper:
 *   - gas: specific-heat ratio gamma and internal degrees of freedom
 *     N = (5 - 3 gamma)/(gamma - 1) (Sec. 2.1, after Eq. (2)); Prandtl number
 *     (Sec. 3.1); gas constant R = 1, so p = rho T;
 *   - viscosity: constant (Sec. 3.1, 3.3) or mu = mu_ref (T/T_ref)^visc_exp
 *     (Sec. 3.4);
 *   - an orthogonal Cartesian grid, uniform or with the tanh stretching of
 *     Sec. 3.3 in y; boundaries periodic, or isothermal no-slip walls at both
 *     ends of y (Sec. 3.3); optional streamwise body force f_x (Sec. 3.3);
 *   - reconstruction: WENO5 with linear weights, WENO-JS or WENO-Z
 *     (Sec. 2.1, Remark 1); flux: the simplified smooth BGK flux or the full
 *     second-order flux of Eq. (5); collision time tau = mu/p plus, for the
 *     full flux, C |p_l - p_r|/(p_l + p_r) dt (Sec. 3 opening);
 *   - time stepping: the two-stage fourth-order scheme of Eq. (6) with the
 *     linear flux fit of Eq. (7); dt = cfl * min over cells and directions of
 *     width / (|u_d| + c).
 *
 * Conventions for every call:
 *   - Field arrays crossing the ABI are FP64, laid out [5][nz][ny][nx]
 *     (x fastest).  Primitive arrays hold (rho, u, v, w, p); conservative
 *     arrays hold (rho, rho u, rho v, rho w, rho E).
 *   - Pointers passed in are borrowed for the duration of the call only.
 *     "is_host" selects host (pageable or pinned) or device memory.
 *   - All GPU work runs on the CUDA stream given to hgks_create.  A call
 *     returns after enqueuing its work unless it reads results back to the
 *     host or is asked to synchronise.
 *   - Every function returns an hgks_status; HGKS_OK is 0.  No error is
 *     reported by any other route; hgks_last_error gives a message.
 */
#ifndef HGKS_H
#define HGKS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HGKS_OK = 0,
  HGKS_E_INVAL = 1,        /* invalid argument or configuration */
  HGKS_E_NOMEM = 2,        /* device allocation failed */
  HGKS_E_CUDA = 3,         /* a CUDA call failed */
  HGKS_E_NONPHYSICAL = 4,  /* rho <= 0, p <= 0 or NaN in the state after a step */
  HGKS_E_TIMEOUT = 5,      /* reserved: a bounded device wait expired */
  HGKS_E_UNSUPPORTED = 6   /* a valid request the library does not implement */
} hgks_status;

typedef enum { HGKS_BC_PERIODIC = 0, HGKS_BC_WALL_ISOTHERMAL = 1 } hgks_bc;
typedef enum { HGKS_RECON_LINEAR = 0, HGKS_RECON_WENO_JS = 1, HGKS_RECON_WENO_Z = 2 } hgks_recon;
typedef enum { HGKS_FLUX_SMOOTH = 0, HGKS_FLUX_FULL = 1 } hgks_flux;
typedef enum { HGKS_VISC_CONST = 0, HGKS_VISC_POWER = 1 } hgks_visc;
typedef enum { HGKS_FP64 = 0, HGKS_FP32 = 1 } hgks_prec;
/* Streamwise body force of Sec. 3.3: the constant force_x, or the force that
 * keeps the volume integral of rho U at mass_flux times the box volume
 * (f_x = (that target - int (rho U)~^{n+1}) / (dt/2 int (rho^n + rho~^{n+1})),
 * with ~ the state after the two S2O4 stages). */
typedef enum { HGKS_FORCE_CONSTANT = 0, HGKS_FORCE_MASS_FLUX = 1 } hgks_force;

typedef struct {
  int nx, ny, nz;                  /* interior cells; 6 .. 65529 on every axis */
  double x0, lx, y0, ly, z0, lz;   /* origin and extent of the box */
  int y_stretch;                   /* 0 uniform y; 1 tanh mapping of Sec. 3.3 (ly = 2, else E_INVAL) */
  double stretch_b;                /* b_g of the mapping */
  int bc_y;                        /* hgks_bc for both y ends; x and z are periodic */
  double gamma, prandtl;           /* gamma > 1; Pr > 0 */
  int visc;                        /* hgks_visc */
  double mu_ref, T_ref, visc_exp;  /* mu = mu_ref (T/T_ref)^visc_exp, or mu_ref */
  double T_wall, force_x;          /* wall temperature; streamwise body force */
  int recon, flux;                 /* hgks_recon, hgks_flux */
  double tau_num_C;                /* C of the numerical collision time (full flux) */
  double cfl;                      /* > 0 */
  int prec;                        /* hgks_prec: arithmetic and storage type */
  double rho_ref, p_ref;           /* reference state at rest; the state is stored as its
                                      deviation from it (must be > 0) */
  int force_mode;                  /* hgks_force (force_x is ignored in mode 1) */
  double mass_flux;                /* HGKS_FORCE_MASS_FLUX: target volume average of rho U */
  int recon_vars;                  /* 0 conservative variables; 1 characteristic variables
                                      (Sec. 2.1, Remark 1) for the WENO modes: each
                                      reconstruction serving a face point projects onto the
                                      eigenvectors of the Euler Jacobian along the face normal
                                      at the mean of the two cells beside it (no effect with
                                      linear weights) */
} hgks_config;

typedef struct hgks_ctx hgks_ctx;  /* opaque; owns every device buffer it uses */

/* Fill *cfg with the Taylor-Green settings of Sec. 3.1 on an n^3 grid
 * (gamma 1.4, Pr 0.72, mu = 1/1600, Ma 0.1, periodic [0, 2 pi]^3, linear
 * weights and smooth flux, CFL 0.5, FP32).  Never fails for n >= 6. */
hgks_status hgks_default_config(hgks_config* cfg, int n);

/* Validate cfg, allocate the context's device buffers and bind it to the
 * CUDA stream `stream` (a cudaStream_t).  NULL gives the context a
 * non-blocking stream of its own (the legacy default stream cannot be
 * captured into a CUDA graph); work on it is then ordered with the caller's
 * streams only through the synchronising calls.  On success *out owns the context.  E_INVAL for a bad config
 * (n < 6, gamma <= 1, Pr <= 0, cfl <= 0, reference <= 0, unknown enum),
 * E_NOMEM when a device allocation fails, E_CUDA for other CUDA errors. */
hgks_status hgks_create(const hgks_config* cfg, void* stream, hgks_ctx** out);

/* Release every resource of ctx (synchronises its stream first).  NULL is OK. */
hgks_status hgks_destroy(hgks_ctx* ctx);

/* Set the state from primitive cell values (rho, u, v, w, p), FP64
 * [5][nz][ny][nx]; resets t and the step count to 0. */
hgks_status hgks_init_state(hgks_ctx* ctx, const double* prim, int is_host);

/* Same from conservative cell averages. */
hgks_status hgks_init_conservative(hgks_ctx* ctx, const double* cons, int is_host);

/* Copy the conservative state (FP64 [5][nz][ny][nx]) out; synchronises when
 * is_host != 0. */
hgks_status hgks_get_state(hgks_ctx* ctx, double* cons_out, int is_host);

/* Set the simulated time and the step counter (both reset to 0 by
 * hgks_init_state / hgks_init_conservative): with hgks_get_state and
 * hgks_init_conservative this checkpoints and resumes a run.  step >= 0
 * (else E_INVAL).  Enqueued on the context's stream. */
hgks_status hgks_set_time(hgks_ctx* ctx, double t, long long step);

/* Advance nsteps S2O4 steps (Eq. (6)).  dt > 0 fixes the step; dt <= 0 takes
 * the CFL step each time (computed on the device).  One step is captured as
 * a CUDA graph on first use and replayed.  With sync != 0 the call waits,
 * checks the state and writes the time reached to *t_out (may be NULL).
 * With sync == 0 it returns after enqueuing.
 * Non-physical states (rho <= 0, p <= 0 or NaN in some cell): each step
 * checks its input state on the device first; once one is non-physical,
 * that step and every later one write nothing (no host round trip per
 * step).  The next synchronising call (this one with sync != 0, or a later
 * hgks_step(ctx, 0, dt, 1, ...)) then returns E_NONPHYSICAL with the state,
 * time and step count left at the last good step -- the step before the
 * first non-physical state (or the state the caller set, if that was
 * non-physical) -- and clears the flag, so that stepping may resume (e.g.
 * with a smaller fixed dt). */
hgks_status hgks_step(hgks_ctx* ctx, int nsteps, double dt, int sync, double* t_out);

typedef struct {
  double t, dt;          /* time reached and last step */
  double mass, mom[3], energy;  /* totals sum Q |Omega_c| */
  double Ek;             /* (1/(rho_ref |Omega|)) sum rho |U|^2/2 |Omega_c| (Sec. 3.1) */
  double rho_min, p_min;
  long long step;
  double force_x;        /* streamwise force of the last step (Sec. 3.3) */
} hgks_diag;

/* FP64 reductions of the current state (synchronises). */
hgks_status hgks_diagnostics(hgks_ctx* ctx, hgks_diag* out);

/* Turbulence statistics of the current state (Sec. 3.1 and Sec. 3.4).  <f>
 * is the volume average over the domain, rho0 = rho_ref, U the velocity,
 * G_ij = dU_i/dx_j by the sixth-order central difference, theta = tr G,
 * omega = curl U, S^d the deviatoric part of (G + G^T)/2, mu the local
 * viscosity mu(T) of the configured law and mu_b = 2N/(3(N+3)) mu its bulk
 * part (N internal degrees of freedom). */
typedef struct {
  double t;          /* time of the state */
  double Ek;         /* <rho |U|^2/2> / rho0 */
  double K;          /* <rho |U|^2/2> */
  double zeta;       /* <rho |omega|^2/2> / rho0 (enstrophy) */
  double eps1;       /* 2 <mu S^d:S^d> / rho0 */
  double eps2;       /* <mu_b theta^2> / rho0 */
  double eps3;       /* -<p theta> / rho0 */
  double rho_mean, rho_rms;  /* <rho>, sqrt(<(rho - <rho>)^2>) */
  double u_rms;      /* sqrt(<|U|^2> / 3) */
  double Su, Fu;     /* means over the axes i with <(d_i U_i)^2> > 0 of
                        <(d_i U_i)^3>/<(d_i U_i)^2>^1.5 and <(d_i U_i)^4>/<(d_i U_i)^2>^2 */
  double eps_s;      /* <mu |omega|^2> (solenoidal dissipation) */
  double eps_d;      /* 4/3 <mu theta^2> (dilatational dissipation) */
  double p_theta;    /* <p theta> (pressure dilatation) */
  double theta_rms, omega_rms;  /* sqrt(<theta^2>), sqrt(<|omega|^2>) */
  double du2[3], du3[3], du4[3];  /* <(d_i U_i)^k>, k = 2, 3, 4 */
  double eps_zeta;   /* 2 mu_ref zeta / rho0 (Sec. 3.1, the incompressible-limit dissipation
                        rate; mu_ref is the configured viscosity, the paper's constant mu) */
} hgks_turbulence;

/* Fill *out from the current state: one statistics kernel and one final
 * reduction on the context's stream, then a synchronise.  Needs a periodic,
 * uniform grid (E_UNSUPPORTED for walls or a stretched y).  Allocates its
 * FP64 partial-sum buffers on the first call. */
hgks_status hgks_turbulence_stats(hgks_ctx* ctx, hgks_turbulence* out);

/* Statistics history (Sec. 3.1: the time histories of E_k, eps(E_k),
 * eps(zeta), eps1..eps3 and the numerical dissipation eps_num).
 * hgks_history_start records the current state at once and then makes every
 * step whose step count is a multiple of `every` (> 0) append a record of its
 * new state, inside the captured step on the device (the statistics kernels
 * of hgks_turbulence_stats, gated on the step count; no host round trip),
 * until `capacity` (> 0) records are stored; later records are dropped.  It
 * clears the records of an earlier start.  Steps with a non-physical state
 * record nothing.  Needs a periodic, uniform grid (E_UNSUPPORTED otherwise).
 * Allocates its device buffers on the first call (and when capacity grows).
 * hgks_history_stop ends the recording (the records stay readable). */
hgks_status hgks_history_start(hgks_ctx* ctx, int every, int capacity);
hgks_status hgks_history_stop(hgks_ctx* ctx);

/* One record of the statistics history. */
typedef struct {
  hgks_turbulence s;  /* statistics of the recorded state; s.t its time */
  long long step;     /* step count of the recorded state */
  double eps_Ek;      /* eps(E_k) = -dE_k/dt (Sec. 3.1), by second-order differences of the
                         recorded E_k over the recorded times (non-uniform spacing allowed):
                         central inside, one-sided three-point at both ends; with two
                         records the one difference; NaN for a single record */
  double eps_num;     /* the numerical dissipation eps(E_k) - (eps1 + eps2 + eps3) (Sec. 3.1) */
} hgks_history_rec;

/* Copy the first min(count, capacity) records (HOST array out, may be NULL
 * if capacity is 0) and write the number recorded to *count.  The
 * differences are taken over all records stored.  Synchronises. */
hgks_status hgks_history_read(hgks_ctx* ctx, hgks_history_rec* out, int capacity, int* count);

/* Mean-flow statistics of the wall-bounded channel (Sec. 3.3), from the
 * current state, instantaneous (time averaging is the caller's): plane
 * averages over x and z of each y row, and from them
 *   tau_w = mu(T_wall) d<U>/dn at each wall (the paper's tau_wall =
 *     dU/dy|wall with the viscosity its dimensions need), d<U>/dn from the
 *     quadratic with <U> = 0 at the wall whose averages over the two
 *     wall-adjacent cells equal theirs;
 *   u_tau = sqrt(tau_w / rho_w), Re_tau = rho_w u_tau H / mu_w with H = ly/2
 *     and rho_w the mean of the two wall-adjacent rows' <rho>;
 *   U_b = (1/ly) int <U> dy, rho_b likewise, U_c = <U> at the mid-plane (the
 *     cubic through the averages of the four cells nearest to it),
 *     nu = mu_w / rho_b, Re_c = U_c H / nu, Re_b = U_b 2H / nu,
 *     C_f = tau_w / (rho_b U_b^2 / 2).
 * profiles (HOST, may be NULL): [14][ny], per y row j: rows 0-7 the plane
 * means of rho, rho U, U, V, W, U V, U U and T = p / rho; then
 *   8  y_j, the cell centre;
 *   9  y+ = rho_w u_tau d_j / mu_w, d_j the distance to the nearer wall;
 *   10 U+ = <U> / u_tau;
 *   11 <u'v'>+ = (<U V> - <U><V>) / u_tau^2;
 *   12 dU+/dY+ = mu_w d<U>/dy / (rho_w u_tau^2), d<U>/dy by the second-order
 *      difference of the row means on the non-uniform centres (one-sided in
 *      the first and last rows);
 *   13 the total-stress residual of the statistically stationary channel,
 *      dU+/dY+ - <u'v'>+ - (1 - Y+/Re_tau) (Sec. 3.3: the total stress is
 *      linear in y; Y+ = y+ here).
 * Needs bc_y = HGKS_BC_WALL_ISOTHERMAL (else E_UNSUPPORTED).  Allocates a
 * small device buffer on the first call; synchronises.  The host part is
 * hgks_channel_compose. */
typedef struct {
  double t;                       /* time of the state */
  double tau_w, tau_w_lower, tau_w_upper;
  double rho_w, mu_w, u_tau, Re_tau;
  double U_b, U_c, rho_b, Re_b, Re_c, C_f;
} hgks_channel;
hgks_status hgks_channel_stats(hgks_ctx* ctx, double* profiles, hgks_channel* out);

/* The host part of hgks_channel_stats: from the plane means `means` (HOST,
 * [8][ny], rows as rows 0-7 of the profiles above) of a channel configured by
 * cfg, the statistics *out (t = 0) and, if profiles is not NULL, the
 * [14][ny] profiles.  No device work; E_INVAL for a bad cfg, E_UNSUPPORTED
 * without walls in y. */
hgks_status hgks_channel_compose(const hgks_config* cfg, const double* means, double* profiles,
                                 hgks_channel* out);

/* Cell widths of axis 0, 1 or 2 (x, y, z) of the grid cfg describes: the
 * uniform extent / n, or the tanh mapping of Sec. 3.3 in y
 * (y_j = y0 + ly/2 (1 + tanh(b (eta_j / (1.5 pi) - 1)) / tanh b),
 * eta_j = 3 pi j / ny).  out (HOST): n doubles.  No device work. */
hgks_status hgks_cell_widths(const hgks_config* cfg, int axis, double* out);

/* Kinetic energy functional of Sec. 3.1 of an FP64 conservative array cons
 * (DEVICE, [5][nz][ny][nx], e.g. a state read with hgks_get_state):
 *   *ek_out = (1 / (rho_ref |Omega|)) sum_c |rho U|^2 / (2 rho) |Omega_c|,
 * an FP64 sum over the cells with the context's cell volumes, in a fixed
 * order (deterministic).  If grad (DEVICE, same layout, may not alias cons)
 * is not NULL it receives dE_k/dQ per cell: -|U|^2/2, U, V, W, 0 times
 * |Omega_c| / (rho_ref |Omega|) -- the seed of an adjoint (hgks_adjoint_step)
 * for a final kinetic-energy functional.  Enqueued on the context's stream;
 * synchronises to return *ek_out.  Allocates a small device buffer on the
 * first call. */
hgks_status hgks_kinetic_energy(hgks_ctx* ctx, const double* cons, double* grad, double* ek_out);

/* Ensembles (no counterpart in the paper): a batch of independent contexts,
 * e.g. instances of uneven sizes, advanced together.  hgks_ensemble_create
 * takes n distinct contexts on the same device, each on its own stream (the
 * handle borrows them; they must outlive it).  hgks_ensemble_step captures,
 * on first use (and again when dt or the members' buffer assignment
 * changes), ONE CUDA graph holding one S2O4 step of every member, and
 * launches it nsteps times on the first member's stream (which first waits
 * for the work already enqueued on the other members' streams; they wait for
 * the batch afterwards).  Two forms of the graph:
 *   - batched (the default when the members share precision, reconstruction
 *     and its variables, flux and sweep tile variant, and have no mass-flux
 *     force and no statistics history): ONE kernel launch per phase of the
 *     step (CFL reduction, dt, the ghost fills, the transposed copy, the three
 *     sweeps and the update of each stage, time) for all members, driven by
 *     an instance table of up to 32 members per launch (kernel parameter):
 *     each block finds its instance and its local block and runs that
 *     instance's part of the phase; ragged grids are fine, no block waits on
 *     another;
 *   - graph branches (any members): every member's own launches as a parallel
 *     branch forked from and joined into the first member's stream.
 * dt > 0 fixes every member's step; dt <= 0 takes each member's own CFL step.
 * With sync != 0 it waits and checks each member as hgks_step does (a member
 * with a non-physical state is left at its last good step).
 * hgks_ensemble_set_batched(ens, 0 or 1) selects the form (E_UNSUPPORTED if
 * the members cannot share batched launches). */
typedef struct hgks_ensemble hgks_ensemble;
hgks_status hgks_ensemble_create(hgks_ctx** ctxs, int n, hgks_ensemble** out);
hgks_status hgks_ensemble_step(hgks_ensemble* ens, int nsteps, double dt, int sync);
hgks_status hgks_ensemble_set_batched(hgks_ensemble* ens, int batched);
hgks_status hgks_ensemble_destroy(hgks_ensemble* ens);
const char* hgks_ensemble_last_error(const hgks_ensemble* ens);

/* Adjoint of one S2O4 step (no counterpart in the paper): with the context's
 * state at Q^n (set it with hgks_init_conservative, e.g. from a checkpoint)
 * and dt the forward step's dt (frozen, > 0), write
 *   adj_out = (dQ^{n+1}/dQ^n)^T adj_in,
 * the vector-Jacobian product of the step map Q^n -> Q^{n+1} of Eq. (6) in
 * the context's scheme and precision.  adj_in, adj_out: DEVICE FP64 arrays
 * [5][nz][ny][nx] of cotangents of the conservative variables (may not
 * alias).  The state is left unchanged.  Conventions where the scheme is not
 * differentiable: d|x|/dx = sign(x), sign(0) = 0.  Periodic boundaries and no
 * body force only (else E_UNSUPPORTED).  Allocates its work buffers on the
 * first call.  Enqueued on the context's stream; does not synchronise. */
hgks_status hgks_adjoint_step(hgks_ctx* ctx, double dt, const double* adj_in, double* adj_out);

/* Tile autotuner (no counterpart in the paper): time the launch shapes of
 * the sweep kernel on the context's current state -- the tile variants
 * available for its configuration (four for linear weights + smooth flux in
 * FP32, one otherwise) times the number of face layers each CTA marches
 * through -- with CUDA events on the context's stream, and keep the fastest
 * for later steps.  The state is unchanged (ghost layers and face-flux
 * buffers are scratch).  Writes the choice and the time of one stage's three
 * sweeps (ms) if the pointers are non-NULL.  Synchronises. */
hgks_status hgks_autotune(hgks_ctx* ctx, int* variant_out, int* chunk_out, double* ms_out);

/* Set the sweep launch shape directly (a cached autotuner result): variant
 * in [0, number of variants), chunk >= 0 face layers per CTA (0 automatic). */
hgks_status hgks_set_sweep_shape(hgks_ctx* ctx, int variant, int chunk);

/* Profiling aid (not on the hot path): advance ONE step without the graph,
 * with CUDA events around every kernel launch on the context's stream, and
 * write the summed device time in milliseconds of each kernel class to
 * ms_out[0..nclass-1] (nclass >= 6): 0 CFL reduction and dt, 1 ghost-cell
 * fills, 2 face fields (3 directions x 2 stages), 3 Gauss-point flux of
 * stage 1 (3 launches), 4 Gauss-point flux of stage 2 (3 launches),
 * 5 update (2 launches).  dt as in hgks_step.  Synchronises. */
hgks_status hgks_profile_step(hgks_ctx* ctx, double dt, double* ms_out, int nclass);

/* Advance nsteps S2O4 steps of the conservative state cons_inout (DEVICE
 * pointer, FP64 [5][nz][ny][nx]) in place, without allocating any device
 * memory.  This is for callers that cannot call cudaMalloc (a host framework
 * that owns all device allocations, a context whose memory footprint must
 * not grow, a path that must not synchronise the device as an allocation
 * may).  No counterpart in the paper: it is the step of hgks_step with its
 * working buffers in one scratch array of fixed size (about 16 MiB) that is
 * part of the library image; every GPU that loads the library holds it until
 * the process exits.  Limits: at most 32 cells on every axis and the
 * constant body force only (larger grids and force_mode 1 return
 * E_UNSUPPORTED); cfg must be valid (else E_INVAL).  dt > 0 fixes the
 * step, dt <= 0 takes the CFL step.  Work is enqueued on `stream` (a
 * cudaStream_t; NULL is the legacy default stream) and the call returns
 * without waiting; no non-physical-state check is made.  The first call on a
 * device looks up the scratch array's device address with that device
 * current; make it before any stream capture.  All calls share the one array:
 * calls whose work overlaps on the GPU (other streams, other threads) race
 * and corrupt each other.  Calls no cudaMalloc, cudaFree or other allocating
 * routine. */
hgks_status hgks_step_noalloc(const hgks_config* cfg, double* cons_inout, int nsteps, double dt,
                              void* stream);

/* Measured arithmetic peaks of the current device (no counterpart in the
 * paper; the denominators of the kernels' ALU rooflines): tflops_out[0] FP32
 * FMA throughput, [1] the same with packed FP32 pairs (one instruction, two
 * FMAs on a float2), [2] FP64 FMA throughput, in TFLOP/s (an FMA counts as
 * two flops).  Each is the best of two timed launches of independent FMA
 * chains over 8 CTAs of 256 threads per SM, after one warm-up launch, on
 * `stream` (a cudaStream_t; NULL the legacy default stream); about 0.1 s in
 * all.  Allocates and frees a small output buffer; synchronises. */
hgks_status hgks_measure_fp_peaks(void* stream, double* tflops_out);

/* Algorithmic operation count of one face of the sweep kernel (no
 * counterpart in the paper; the numerator of the sweep's ALU roofline).  The
 * closed forms the kernel evaluates -- WENO5 end values, normal slopes and
 * the compatibility state of Sec. 2.1 and Remark 1 at one face point, the
 * tangential pass along t1 at one point, and the tangential pass along t2
 * with the flux of Eq. (5) (smooth or full) at the four Gauss points of one
 * face -- are run on the HOST with a counting number type, once each, i.e.
 * without the recomputation of a tile's halo.  Stage 1 or 2 (stage 2 needs
 * dF only, Eq. (6)).  out (host, 21 doubles): for each part p = 0 (face
 * fields, per point), 1 (t1 pass, per point), 2 (t2 pass and flux, per face)
 * the counts out[7p + 0..6] of additions (and subtractions), multiplications,
 * divisions, square roots, exponentials, error functions and powers.  An FMA
 * counts as one addition and one multiplication; operations on per-run
 * constants only are not counted.  Conservative-variable reconstruction only
 * (E_UNSUPPORTED for recon_vars = 1 with WENO).  No device work. */
hgks_status hgks_count_flops(const hgks_config* cfg, int stage, double* out);

/* Message of the last failed call on ctx ("" if none); valid until the next
 * call on ctx.  ctx may be NULL for errors of hgks_create. */
const char* hgks_last_error(const hgks_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* HGKS_H */
