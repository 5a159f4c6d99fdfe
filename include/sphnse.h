/*
 * sphnse.h -- C ABI of libsphnse: the pseudospectral quadrature method for the
 * incompressible Navier-Stokes equations on the rotating unit sphere
 * (Ganesh, Le Gia & Sloan), evaluated on one NVIDIA GB300 (sm_103a).
 *
 * Problem (Sec. 2, Eq. (NSE_sphere)):  u_t + grad_u u - nu Delta u
 *   + omega x u + grad p / rho = f,  div u = 0,  omega = 2 Omega cos(theta) xhat.
 * Unknowns (Eq. (app_soln_rep)): u_N = sum_{L=1..N} sum_{|m|<=L} alpha_{L,m} Z_{L,m},
 *   Z_{L,m} = lambda_L^{-1/2} Curl Y_{L,m}, lambda_L = L(L+1) (Eq. (stok_eig)).
 * ODE system (Eq. (ode)): d alpha/dt = F(t, alpha),
 *   F_{L,m} = fhat_{L,m} - nu lambda_L alpha_{L,m}
 *             - ((zeta + 2 Omega cos theta) xhat x u, Z_{L,m})_M
 *   with the discrete inner product of Eq. (disc_ip) on the Gauss-rectangle
 *   rule Q_M of Eq. (quadrule): nlat = M/2 Gauss-Legendre latitudes x
 *   nlon = M equispaced longitudes.  The vorticity/Coriolis product is the
 *   non-gradient part of the nonlinear term (Eq. (short_nonlin1)) plus the
 *   Coriolis operator (Eq. (C)).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Packed coefficient vector: complex128 stored as interleaved (re, im)
 *   doubles, m-major: index(m, L) = off[m] + L - max(m, 1) for m = 0..N and
 *   L = max(m, 1)..N, off[0] = 0, off[m+1] = off[m] + N - max(m, 1) + 1;
 *   n_coeff = (N+1)(N+2)/2 - 1 complex entries.  Only m >= 0 is stored;
 *   alpha_{L,-m} = (-1)^m conj(alpha_{L,m}) and alpha_{L,0} is real.
 * Y_{L,m} = Pt_L^m(cos theta) e^{i m phi} with the orthonormal associated
 *   Legendre functions including the Condon-Shortley phase (Eq. (sph_har)).
 * Grid arrays: row-major [nlat][nlon] doubles, latitude rows ordered north to
 *   south (theta ascending), longitude phi_q = 2 pi q / nlon, q = 0..nlon-1.
 * Memory: every pointer argument marked (device) is device memory owned by
 *   the caller; the plan owns its tables and workspaces.  Calls are ordered
 *   on the plan's stream (sphnse_set_stream) and do not synchronise the host,
 *   except where a host output is documented (step info, norms).
 * Errors: 0 on success, a negative SPHNSE_E_* code otherwise; inputs are not
 *   modified on error.  Calls on one plan are not thread-safe.
 */
#ifndef SPHNSE_H
#define SPHNSE_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define SPHNSE_OK                  0
#define SPHNSE_E_ARG              -1  /* bad argument: L < 1, nlon not even, nlat != nlon/2, nu < 0, NULL */
#define SPHNSE_E_INEXACT          -2  /* nlon < 3L + 2: Q_M not exact on the Galerkin integrals (Eq. (M_choice)) */
#define SPHNSE_E_NOMEM            -3  /* device or host allocation failed */
#define SPHNSE_E_CUDA             -4  /* a CUDA runtime call failed */
#define SPHNSE_E_NONFINITE        -5  /* a non-finite value appeared in the state or an input */
#define SPHNSE_E_STEP_TOO_SMALL   -6  /* the adaptive step fell below 16 eps |t| */
#define SPHNSE_E_TIMEOUT          -7  /* a bounded device wait ran out */
#define SPHNSE_E_UNSUPPORTED      -8  /* nlon not 2^a 3^b or above 1536, or a precision not built */
#define SPHNSE_E_TOO_LARGE        -9  /* size beyond a fixed capacity: the scratch of an allocation-free
                                         entry point, the steps a tape was created for */

/* ---- plan parameters (sphnse_plan_set / sphnse_plan_get) ---------------- */
#define SPHNSE_KEY_PRECISION       1  /* SPHNSE_FP64 | SPHNSE_FP32 | SPHNSE_BF16X3 (default FP64) */
#define SPHNSE_KEY_NU              2  /* viscosity nu >= 0 */
#define SPHNSE_KEY_OMEGA           3  /* rotation rate Omega */
#define SPHNSE_KEY_RTOL            4  /* relative tolerance of sphnse_step (default 1e-6) */
#define SPHNSE_KEY_ATOL            5  /* absolute tolerance of sphnse_step (default 1e-12) */
#define SPHNSE_KEY_MAX_ORDER       6  /* highest NDF order, 1..5 (default 5) */
#define SPHNSE_KEY_NEWTON_MAX_ITER 7  /* simplified-Newton iteration cap (default 4) */
#define SPHNSE_KEY_H_MAX           8  /* largest step size (default 1) */
#define SPHNSE_KEY_BDF             9  /* 1: kappa = 0 (BDF), 0: NDF (default) */
#define SPHNSE_KEY_CORIOLIS_SPLIT 10  /* 1: apply the Coriolis term as the diagonal
                                         (C Z_{L,m}, Z_{L,m}) = -2 i Omega m / lambda_L
                                         (Sec. 3, Eq. (Coriolis_ZLm)) in the finish
                                         step and drop 2 Omega cos(theta) from the
                                         grid product; 0: in the product (default).
                                         Same F up to rounding; forward RHS only (the
                                         adjoint always carries it in the product) */
#define SPHNSE_KEY_TIMING_PERIOD  11  /* stage timing records every period-th launch of a
                                         timed stage (default 1) */
#define SPHNSE_KEY_AUTOTUNE       12  /* ensemble: 1 (default) times the candidate shapes of
                                        * the tensor-core synthesis per truncation (instances per
                                        * group, pipeline stages, CTAs per cluster) when BF16X3
                                        * is selected and keeps the fastest (sphnse_ensemble_bucket);
                                        * 0 takes the widest instance groups; set it first */
#define SPHNSE_KEY_RING_THREADS   13  /* four-step FFT ring kernel (nlon = 24 M2): threads per
                                         CTA of 128 / M2 latitude rings.  128: one thread per
                                         column carries both packed spectra; 256 (M2 >= 16):
                                         a thread per column and spectrum, for grids of less
                                         than four CTAs per SM; 0 (default) chooses by the
                                         grid.  The results are identical */
#define SPHNSE_KEY_SYN_CLUSTER    14  /* ensemble, with SPHNSE_KEY_AUTOTUNE 0: CTAs per cluster of
                                         the batched tensor-core synthesis (1 default, 2, 4); the
                                         CTAs of a cluster take consecutive instance groups and
                                         share every table tile by TMA multicast.  Set it first */
#define SPHNSE_KEY_N_COEFF       100  /* read-only: n_coeff */
#define SPHNSE_KEY_L             101  /* read-only: truncation degree */
#define SPHNSE_KEY_NLAT          102  /* read-only */
#define SPHNSE_KEY_NLON          103  /* read-only */
#define SPHNSE_KEY_TABLE_BYTES   104  /* read-only: device bytes of Legendre tables held */
#define SPHNSE_KEY_ROUNDS        105  /* read-only (ensemble): graph launches (rounds) of the
                                         last sphnse_ensemble_advance / _step call */
#define SPHNSE_KEY_SYN_ENTRIES   106  /* read-only: table entries Pt_K^m(x_p) one tensor-core
                                         synthesis reads (tiles of negligible entries
                                         excluded; 0 before the BF16X3 tables exist) */
#define SPHNSE_KEY_ANA_ENTRIES   107  /* read-only: the same for the tensor-core analysis */
#define SPHNSE_KEY_BUCKETS       108  /* read-only (ensemble): truncation buckets */

#define SPHNSE_FP64    0  /* FP64 tables and arithmetic throughout */
#define SPHNSE_FP32    1  /* FP32 tables, contractions, FFTs; FP64 state and update */
#define SPHNSE_BF16X3  2  /* BF16 hi+lo split Legendre contractions on tcgen05 tensor
                             cores with FP32 accumulation; FP32 FFTs; FP64 state */

#define SPHNSE_MAXK 5     /* highest NDF order */

typedef struct sphnse_plan sphnse_plan;


/* Create a plan for truncation L on the nlat x nlon Gauss-rectangle grid.
 * Computes in FP64 on the host the Gauss-Legendre nodes/weights and the
 * orthonormal associated Legendre tables (Sec. 3 Eq. (quadrule); Sec. 4.2),
 * and uploads them to the current CUDA device.  Requires nlon even,
 * nlat == nlon/2, nlon >= 3L+2 (Eq. (M_choice)), nlon = 2^a 3^b <= 1536.
 * Returns NULL on error; sphnse_last_error() then gives the code. */
sphnse_plan* sphnse_plan_create(int L, int nlat, int nlon, double nu, double Omega);

/* Status of the last sphnse_plan_create on this thread. */
int sphnse_last_error(void);

/* Short text for a status code (static storage). */
const char* sphnse_error_string(int code);

/* Release the plan and its device memory (waits for its stream). NULL is ignored. */
void sphnse_plan_destroy(sphnse_plan* plan);

/* Set / read a plan parameter (SPHNSE_KEY_*).  Setting the precision builds
 * the tables that precision needs (host FP64 master copy converted once). */
int sphnse_plan_set(sphnse_plan* plan, int key, double value);
int sphnse_plan_get(const sphnse_plan* plan, int key, double* value);

/* Order all later work of the plan on this cudaStream_t (NULL: legacy default stream). */
int sphnse_set_stream(sphnse_plan* plan, void* stream);

/* Wait for the plan's stream.  Returns SPHNSE_E_TIMEOUT if a kernel of the
 * plan gave up a bounded wait since the last call (the status is cleared),
 * SPHNSE_E_CUDA on a CUDA error. */
int sphnse_sync(sphnse_plan* plan);

/* Gauss-rectangle nodes: theta, cos(theta), sin(theta) and Gauss weights w_p
 * (host arrays of nlat doubles each; any may be NULL).  Sec. 3, Eq. (quadrule). */
int sphnse_grid_nodes(const sphnse_plan* plan, double* theta, double* x, double* sin_theta, double* w);

/* ---- the right-hand side (the hot path) --------------------------------- */

/* F = dalpha/dt of Eq. (ode) (Eqs. (app1_weak_form), (short_nonlin1), (C),
 * (Coriolis_ZLm), Sec. 4.2):  dalpha_dt = forcing - nu lambda alpha
 *   - ((zeta + 2 Omega cos theta) xhat x u, Z_{L,m})_M.
 * alpha, forcing, dalpha_dt: (device) packed complex128, n_coeff entries;
 * forcing may be NULL (zero).  t is accepted for the autonomous interface
 * (the forcing is the caller's value at t).  alpha and dalpha_dt must not
 * overlap.  Runs entirely on the device: coefficient prep, per-order Legendre
 * synthesis, per-latitude inverse FFT + pointwise product + forward FFT,
 * per-order Legendre analysis, recombination and diagonal update. */
int sphnse_rhs(sphnse_plan* plan, double t, const double* alpha, const double* forcing,
               double* dalpha_dt);

/* F(t, alpha) of Eq. (ode) from HOST arrays, pipelined across calls.  Each
 * call copies alpha_h (and forcing_h, nullable) into one of two plan-owned
 * device staging slots on an upload stream, evaluates F on the plan's
 * stream, and returns without waiting for F (*ticket, nullable, numbers the
 * call from 0).  F reaches out_h in one of two ways:
 * - out_h page-locked and mapped, BF16X3 plan on the fused tensor-core RHS:
 *   the call waits for its upload before queueing the RHS, and the analysis
 *   writes F into out_h itself (the plan's stream then holds only the RHS
 *   kernels, so consecutive calls overlap);
 * - otherwise a copy on a download stream; call k + 1's upload overlaps call
 *   k's RHS and call k's download overlaps call k + 1's RHS.
 * The host arrays (n_coeff complex128 each; page-locked for the transfers
 * to overlap) must stay valid, and alpha_h / forcing_h unmodified, until
 * sphnse_host_wait(plan, ticket) has returned; out_h is valid from then on. */
int sphnse_rhs_host(sphnse_plan* plan, double t, const double* alpha_h, const double* forcing_h,
                    double* out_h, long long* ticket);

/* Block until call `ticket` of sphnse_rhs_host has delivered F to the host
 * (E_ARG for a ticket not yet issued; E_TIMEOUT if a direct-output call has
 * not reported completion within 30 s). */
int sphnse_host_wait(sphnse_plan* plan, long long ticket);

/* Grid values of zeta = xhat.Curl_n u (Eq. (vort_app)), u_theta and u_phi
 * for the field with coefficients alpha (Eq. (app_soln_rep)).
 * alpha: (device) packed; zeta, u_theta, u_phi: (device) [nlat][nlon] doubles,
 * any may be NULL. */
int sphnse_grid_fields(sphnse_plan* plan, const double* alpha, double* zeta,
                       double* u_theta, double* u_phi);

/* Discrete projection of a tangential grid field onto Z_{L,m}
 * (Eq. (disc_vec_orth_proj)): out_{L,m} = (v, Z_{L,m})_M.
 * v_theta, v_phi: (device) [nlat][nlon]; out: (device) packed. */
int sphnse_project(sphnse_plan* plan, const double* v_theta, const double* v_phi, double* out);

/* ---- diagnostics (Sec. 6.2) --------------------------------------------- */

/* Energy spectrum E(L) = sum_{|m| <= L} |alpha_{L,m}|^2, Eq. (energy), for
 * L = 0..N (E(0) = 0; an order m > 0 counts twice, for m and -m).
 * alpha: (device) packed; E: (device) N + 1 doubles.  Deterministic: a fixed
 * summation order per degree. */
int sphnse_energy_spectrum(sphnse_plan* plan, const double* alpha, double* E);

/* The field alpha_in of truncation N_in in the packed layout of the plan's
 * truncation N: modes with L <= min(N_in, N, L_max) copied, all others zero
 * (L_max < 0: no extra cut).  With L_max = N1 this is the projection P_{N1}
 * of Eq. (eq: cut_app_soln).  alpha_in, alpha_out: (device), not
 * overlapping. */
int sphnse_resize(sphnse_plan* plan, int N_in, const double* alpha_in, int L_max, double* alpha_out);

/* Approximate inertial manifold of Eq. (eq:p-p) on a plan of truncation
 * N2 = N > N1: phi = (nu A + C)^{-1} (P_{N2} - P_{N1}) [f - B(u1, u1)] with
 * u1 = P_{N1} alpha, i.e. the RHS of Eq. (ode) at u1 divided by
 * nu lambda_L - 2 i Omega m / lambda_L for N1 < L <= N2, and 0 for L <= N1.
 * alpha, forcing (nullable), phi: (device) packed, degree N2.  Uses the
 * plan's step workspace as scratch (do not call it inside a step).
 * E_ARG unless 1 <= N1 < N and nu > 0. */
int sphnse_inertial_manifold(sphnse_plan* plan, int N1, const double* alpha, const double* forcing,
                             double* phi);

/* ---- adaptive NDF time step (Sec. 4.2, Eq. (ode_disc)) ------------------ */

typedef struct {
    double* alpha;  /* (device) packed alpha_n, n_coeff complex; updated in place */
    double* dif;    /* (device) (SPHNSE_MAXK + 2) x n_coeff complex backward differences */
    double t;       /* current time t_n */
    double h;       /* step size the next attempt starts from */
    double t_end;   /* steps never pass t_end (use +inf for none) */
    int    order;   /* current order k, 1..5 */
    /* controller memory, set by sphnse_state_init; not for the caller */
    int    nconhk;
    int    havrate;
    int    miter_k;
    double h_dif;
    double rate;
    double miter_h;
} sphnse_state;

typedef struct {
    double t;           /* time reached */
    double h;           /* step size taken */
    double err;         /* local error estimate of the accepted step (weighted max-norm) */
    int    order;       /* order of the accepted step */
    int    newton_iters;/* Newton iterations over all attempts */
    int    rejections;  /* rejected attempts before acceptance */
    int    rhs_evals;   /* F evaluations over all attempts */
    int    next_order;  /* order chosen for the next step */
    double next_h;      /* step size chosen for the next step */
    double h_dif_before;/* step size the differences were expressed in before this step */
} sphnse_step_info;

/* Initialise an NDF state at (t0, alpha already in st->alpha): first
 * difference D_0 = h0 F(t0, alpha0), order 1.  h0 <= 0 chooses
 * h0 = min(h_max, sqrt(rtol) / (1.25 ||F / wt||_inf)).  forcing: (device) or NULL. */
int sphnse_state_init(sphnse_plan* plan, sphnse_state* st, double t0, double h0,
                      const double* forcing);

/* One accepted step of the variable-order NDF integrator: predictor,
 * simplified Newton on c F(alpha0 + d) - psi - d = 0 with the diagonal
 * iteration matrix I - c J_d, J_d = -nu lambda + 2 i Omega m / lambda,
 * local error estimate, step rejection and order/step selection (the
 * MATLAB ODE-suite scheme the paper follows).  forcing: (device) steady over
 * the step, or NULL.  Fills *info (host).  The attempts, their Newton
 * iterations and the controller run as one CUDA-graph launch whose loop
 * conditions are set on the device (one host synchronisation per call);
 * with stage timing enabled the host drives the attempts instead. */
int sphnse_step(sphnse_plan* plan, sphnse_state* st, const double* forcing,
                sphnse_step_info* info);

/* nsteps >= 0 accepted steps of sphnse_step in one call and one graph
 * launch (no host synchronisation between steps); info: host array of
 * nsteps entries or NULL.  On an error the state holds the steps accepted
 * before it, and info their entries. */
int sphnse_advance(sphnse_plan* plan, sphnse_state* st, const double* forcing, int nsteps,
                   sphnse_step_info* info);

/* One step with the step size h and order k fixed by the caller (frozen
 * controller) and the corrector iterated until the Newton update is below
 * 1e-15 in the weighted norm (at most newton_max iterations).  This is the
 * map the adjoint differentiates. */
int sphnse_replay_step(sphnse_plan* plan, sphnse_state* st, const double* forcing,
                       double h, int k, int newton_max, sphnse_step_info* info);

/* ---- adjoint (discretise-then-differentiate, frozen controller) --------- */

/* out = J(alpha)^T w, J = dF/dalpha as a real-linear map of the packed real
 * components.  alpha, w, out: (device) packed; out must not alias w.
 * If nu_bar is not NULL, *nu_bar += <w, dF/dnu> = -<w, lambda alpha> (host). */
int sphnse_rhs_adjoint(sphnse_plan* plan, const double* alpha, const double* w,
                       double* out, double* nu_bar);

/* Reverse of one sphnse_replay_step(h, k) taken from a state whose
 * differences were expressed in step size h_dif_before, with alpha_next the
 * state it produced.  abar (device, packed) and dbar (device,
 * (SPHNSE_MAXK+2) x n_coeff complex) hold the adjoints of (alpha, dif) after
 * the step on entry and before it on return; *nu_bar (host) is accumulated.
 * The transposed corrector system (I - c J^T) mu = dbar_d is solved by
 * fixed-point iteration preconditioned with (I - c J_d)^{-T}.  The caller
 * keeps the forward states; sphnse_adjoint_step does this through a tape. */
int sphnse_adjoint_step_explicit(sphnse_plan* plan, double h, int k, double h_dif_before,
                                 const double* alpha_next, double* abar, double* dbar,
                                 double* nu_bar);

/* Reverse of sphnse_state_init: with D_0 = h0 F(alpha0), adds
 * h0 J(alpha0)^T dbar_0 to abar and h0 <dbar_0, dF/dnu> to *nu_bar. */
int sphnse_adjoint_init(sphnse_plan* plan, double h0, const double* alpha0,
                        double* abar, const double* dbar, double* nu_bar);

/* ---- checkpointed trajectory tape (the map the adjoint differentiates) --- */

/* A tape records the replay of a step schedule [(h_n, k_n)] from alpha0
 * (frozen controller, each corrector iterated to convergence: the map of
 * sphnse_replay_step, Sec. 4.2 Eq. (ode_disc)) and drives the reverse sweep.
 * It keeps every C-th state (alpha, differences, controller scalars) in
 * device memory it owns, and during the reverse sweep replays one segment of
 * C steps from its checkpoint to get the states the reverse steps need:
 * about (1 + ceil(max_steps / C)) (SPHNSE_MAXK + 3) + C + SPHNSE_MAXK + 2
 * packed vectors of device memory, and one extra forward pass of work. */
typedef struct sphnse_tape sphnse_tape;

/* Allocate a tape on the plan's device for up to max_steps steps with a
 * checkpoint every checkpoint_every steps; *tape = NULL on error (E_ARG,
 * E_NOMEM).  The tape refers to the plan, which must outlive it. */
int sphnse_tape_create(sphnse_plan* plan, int max_steps, int checkpoint_every, sphnse_tape** tape);
/* Release the tape (waits for the plan's stream).  NULL is ignored. */
void sphnse_tape_destroy(sphnse_tape* tape);

/* Start a trajectory at (t0, alpha0) as sphnse_state_init does (h0 <= 0:
 * automatic initial step).  alpha0 (device, packed) is copied; forcing
 * (device or NULL) is steady over the trajectory and must stay valid and
 * unmodified until the reverse sweep ends.  The tape records the plan's nu,
 * Omega, precision and BDF switch: later recording and reverse calls return
 * E_ARG if any of them has changed.  Clears any earlier trajectory. */
int sphnse_tape_begin(sphnse_tape* tape, const double* alpha0, double t0, double h0,
                      const double* forcing);

/* Append one step of size h and order k (sphnse_replay_step with newton_max
 * corrector iterations at most); info (host, nullable) as sphnse_replay_step.
 * E_TOO_LARGE beyond max_steps. */
int sphnse_tape_record(sphnse_tape* tape, double h, int k, int newton_max, sphnse_step_info* info);

/* Steps recorded, the time reached and the initial step size h0 (host
 * outputs, any may be NULL). */
int sphnse_tape_info(const sphnse_tape* tape, int* nsteps, double* t, double* h0);

/* Copy the state after the last recorded step into alpha_out (device, packed). */
int sphnse_tape_state(const sphnse_tape* tape, double* alpha_out);

/* Reverse of recorded step step_index (discretise-then-differentiate).
 * lambda (device, packed, in/out): on entry the adjoint of the state after
 * the step (for step_index = nsteps - 1, dJ/dalpha(t_n) of the objective),
 * on return the adjoint of the state before it.  *dJ_dnu (host, nullable)
 * is accumulated with the step's contribution to dJ/dnu.  The tape holds the
 * adjoint of the difference array between calls, which is why it is not
 * const.  A sweep starts at step_index = nsteps - 1 (which clears that
 * adjoint) and must name nsteps - 2, ..., 0 in turn (E_ARG otherwise); the
 * call for step 0 also applies the reverse of sphnse_state_init, so lambda
 * then holds dJ/dalpha0.  The first call inside a checkpoint segment replays
 * the segment forward. */
int sphnse_adjoint_step(sphnse_plan* plan, sphnse_tape* tape, int step_index, double* lambda,
                        double* dJ_dnu);

/* The whole reverse sweep: sphnse_adjoint_step for nsteps - 1 down to 0. */
int sphnse_adjoint_run(sphnse_plan* plan, sphnse_tape* tape, double* lambda, double* dJ_dnu);

/* Final-time objective of a latitude band and a coefficient misfit:
 * J = 1/2 sum over nodes with colatitude in [theta_lo, theta_hi] of
 *     (2 pi / M) w_p |u|^2  +  sum_{all L,m} |alpha - target|^2,
 * and its gradient with respect to the packed real components of alpha.
 * alpha, target, grad: (device) packed; *J (host). */
int sphnse_objective(sphnse_plan* plan, const double* alpha, const double* target,
                     double theta_lo, double theta_hi, double* J, double* grad);

/* ---- batched ensemble ----------------------------------------------------- */

typedef struct sphnse_ensemble sphnse_ensemble;

/* n independent problems with truncations L[i] and viscosities nu[i] (host
 * arrays), common Omega, each on its Gauss-rectangle grid with nlon the
 * smallest even 2^a 3^b >= 3 L + 2 (nlat = nlon / 2).  Instances of equal L
 * share one set of Legendre tables and run every RHS stage as one launch over
 * all of them; FP32 contractions, FP64 state.  Supported L: those whose
 * northern node count nlat/2 is a multiple of 4 and >= 32 (e.g. 63, 127, 255).
 * The ensemble owns its state vectors (see sphnse_ensemble_instance).
 * Returns NULL on error. */
sphnse_ensemble* sphnse_ensemble_create(int n, const int* L, const double* nu, double Omega);
/* (FP32 contractions by default; SPHNSE_KEY_PRECISION selects BF16X3.) */
void sphnse_ensemble_destroy(sphnse_ensemble* ens);

/* SPHNSE_KEY_RTOL, _ATOL, _MAX_ORDER, _NEWTON_MAX_ITER, _H_MAX and
 * _PRECISION (SPHNSE_FP32, default, or SPHNSE_BF16X3: instances of one
 * truncation then share every table tile on the tensor cores). */
int sphnse_ensemble_set(sphnse_ensemble* ens, int key, double value);
/* Read SPHNSE_KEY_RTOL, _ATOL, _MAX_ORDER, _NEWTON_MAX_ITER, _H_MAX,
 * _PRECISION or _ROUNDS into *value. */
int sphnse_ensemble_get(sphnse_ensemble* ens, int key, double* value);
int sphnse_ensemble_set_stream(sphnse_ensemble* ens, void* stream);

/* Device pointers (owned by the ensemble) of instance i's packed state alpha
 * and of its last RHS F (complex128, n_coeff entries); any output may be NULL. */
int sphnse_ensemble_instance(sphnse_ensemble* ens, int i, double** alpha, double** F, int* n_coeff);

/* Bucket b (0 .. SPHNSE_KEY_BUCKETS - 1; instances of one truncation share its
 * Legendre tables): its truncation L, instance count, and on the BF16X3
 * tensor-core path the shape of its synthesis (instances per group, pipeline
 * stages, CTAs per cluster that share every table tile by TMA multicast) and
 * that synthesis' duration in microseconds as timed by the autotuner (0 when
 * not tuned; group = stages = cluster = 0 off the tensor-core path).  Any
 * output may be NULL. */
int sphnse_ensemble_bucket(sphnse_ensemble* ens, int b, int* L, int* count, int* group, int* stages, int* cluster,
                           double* syn_us);

/* F_i = F(alpha_i) for every instance (Eq. (ode)), as one CUDA-graph launch. */
int sphnse_ensemble_rhs(sphnse_ensemble* ens);

/* Initialise every instance's NDF state at t0 from its current alpha
 * (automatic initial step per instance, as sphnse_state_init). */
int sphnse_ensemble_init(sphnse_ensemble* ens, double t0);

/* One accepted step of every instance, each with its own adaptive step size
 * and order (the controller of sphnse_step); info: host array of n entries
 * or NULL.  Same as sphnse_ensemble_advance(ens, 1, info). */
int sphnse_ensemble_step(sphnse_ensemble* ens, sphnse_step_info* info);

/* nsteps >= 0 accepted steps of every instance, each at its own pace: the
 * instances advance in rounds (accept, rescale and predictor where due, one
 * batched RHS of all instances, one Newton update, then the per-instance
 * controllers on the device), all rounds in one CUDA-graph launch with a
 * device-side loop condition, so an instance never waits for another's
 * rejected attempts or Newton iterations and the host waits once per call.  Each instance follows exactly the
 * step/order sequence sphnse_step gives it alone.  info (host, n entries or
 * NULL): the last step's t, h, err, order, next_order, next_h, h_dif_before,
 * with newton_iters, rhs_evals and rejections summed over the call.
 * SPHNSE_E_ARG before sphnse_ensemble_init. */
int sphnse_ensemble_advance(sphnse_ensemble* ens, int nsteps, sphnse_step_info* info);

/* ---- stage timing ------------------------------------------------------- */

#define SPHNSE_STAGE_PREP       0  /* coefficient sets for synthesis */
#define SPHNSE_STAGE_SYNTHESIS  1  /* per-order Legendre synthesis */
#define SPHNSE_STAGE_RING       2  /* per-latitude FFTs and pointwise product */
#define SPHNSE_STAGE_ANALYSIS   3  /* per-order Legendre analysis */
#define SPHNSE_STAGE_FINISH     4  /* recombination and diagonal update */
#define SPHNSE_STAGE_STEP       5  /* NDF vector kernels (predictor, Newton update, accept) */
#define SPHNSE_STAGE_TRANSPOSE  6  /* order-major <-> latitude-major transposes */
#define SPHNSE_NSTAGES          7

#define SPHNSE_STAGE_ALL        (-1)

/* enable = bit mask of stages (bit s = stage s; SPHNSE_STAGE_ALL for every
 * stage): record a CUDA event pair on the plan's stream around every later
 * kernel launch of an enabled stage; enable == 0: stop and keep totals.
 * Enabling clears the totals.  Every event pair costs stream time (the kernel
 * after it cannot start before the pair's kernel completes), so a throughput
 * measurement should enable only the stage it reports, and may time only
 * every period-th launch of it (SPHNSE_KEY_TIMING_PERIOD). */
int sphnse_stage_timing(sphnse_plan* plan, int enable);

/* Synchronise the plan's stream, fold the recorded events into totals and
 * return per stage the summed device milliseconds and the number of
 * launches (host arrays of SPHNSE_NSTAGES entries; either may be NULL). */
int sphnse_stage_times(sphnse_plan* plan, double* ms, long* launches);

/* ---- allocation-free entry point ---------------------------------------- */

/* The paper has no counterpart: this is a service for callers that cannot
 * call cudaMalloc -- a caller whose device memory is entirely owned by a
 * framework's caching allocator (where a raw cudaMalloc can fail or
 * fragment the pool), or a latency-critical loop that cannot afford the
 * device synchronisation and the milliseconds of an allocation -- and that
 * may hold no plan, since creating one allocates.
 *
 * Writes *out = <w, dF/dnu> = -sum_{packed (L,m)} L(L+1) (Re alpha Re w +
 * Im alpha Im w), the value sphnse_rhs_adjoint adds to its nu_bar, for
 * packed complex128 vectors alpha, w of truncation L (n = (L+1)(L+2)/2 - 1
 * entries).  alpha, w, out: device pointers owned by the caller (out: one
 * double); stream: cudaStream_t or NULL.  Stream-ordered, no host sync.
 * Allocates nothing: block partial sums go to a file-scope device array of
 * SPHNSE_NOALLOC_MAX_BLOCKS doubles (32 KB per device that loads the
 * library, held until the process exits).  Sizes with n > 2048 *
 * SPHNSE_NOALLOC_MAX_BLOCKS (L above about 4090) return SPHNSE_E_TOO_LARGE.
 * The first call on a device looks up the array's device address with that
 * device current (a one-time set-up; a lookup that fails returns
 * SPHNSE_E_CUDA and is tried again by the next call); make that first call
 * before any stream capture.  All calls share the array and each call
 * overwrites the slots it reads; calls that overlap on the GPU race on it. */
#define SPHNSE_NOALLOC_MAX_BLOCKS 4096
int sphnse_nu_sensitivity_noalloc(int L, const double* alpha, const double* w, double* out, void* stream);

/* ---- host-only helpers (no CUDA call; usable without a GPU) ------------- */

/* Gauss-Legendre nodes and weights of the n-point rule the plan uses
 * (Sec. 3, Eq. (quadrule)), nodes north to south: theta, cos(theta),
 * sin(theta), w (host arrays of n doubles). */
int sphnse_host_gauss_nodes(int n, double* theta, double* x, double* sin_theta, double* w);

/* Orthonormal associated Legendre functions Pt_K^m(x_p), K = m..Kmax, at np
 * nodes (Eq. (sph_har), Condon-Shortley phase): out[(K - m) * np + p] (host).
 * sin_theta[p] = sqrt(1 - x[p]^2) supplied by the caller. */
int sphnse_host_legendre(int Kmax, int m, int np, const double* x, const double* sin_theta,
                         double* out);

#ifdef __cplusplus
}
#endif
#endif /* SPHNSE_H */
