/*
 * rlb.h -- C ABI of the GB300 relativistic lattice Boltzmann step with a
 * quasiparticle (non-ideal) equation of state, after Romatschke,
 * "Relativistic (Lattice) Boltzmann Equation with Non-Ideal Equation of
 * State", arXiv:1108.5561.
 *
 * The library advances the on-shell distribution f(tau, x, y; v) of one
 * uncharged quasiparticle species with medium-dependent mass M in the Milne
 * metric ds^2 = dtau^2 - dx^2 - dy^2 - tau^2 dY^2 (Sec. 3.3, Eq. Bmilne),
 * boost invariant (no Y dependence), on a periodic transverse grid.  Momenta
 * are the nodes of the Sec. 4.3 lattice, p~ = M v with
 * v = sinh(xi) (sin th cos ph, sin th sin ph, cos th); one time step is the
 * predictor-corrector of Sec. 4.4 applied to (f, ln M).
 *
 * Units: T, M in GeV; tau, dtau, dx in fm (fm/c); energy densities returned in
 * GeV/fm^3.
 *
 * Conventions
 *   - Every function returns rlb_status; nothing throws or exits across the ABI.
 *     On failure a message is kept in the context (rlb_last_error).
 *   - Device memory is owned by the caller: the library states how many bytes
 *     it needs (rlb_workspace_size) and borrows the caller's buffers
 *     (rlb_bind_buffers).  Host-side tables are owned by the context.
 *   - Work is enqueued on the caller's cudaStream_t (passed as void*; NULL is
 *     the legacy default stream).  Launch errors are returned at once; numeric
 *     failures found on the device (no timelike Landau eigenvector, temperature
 *     inversion outside the EOS table, non-finite values) set a device error
 *     word that rlb_check, rlb_moments and rlb_sync_error report as
 *     RLB_ERR_NUMERIC.  Bits: 1 Landau, 2 EOS inversion, 4 non-finite, 8 index
 *     check, 16 a bounded device wait expired (reported as RLB_ERR_TIMEOUT).  The library built with checks (RLB_CHECKS; the Python front end
 *     loads it when RLB_CHECKED=1) also range-checks every site index and grid
 *     coordinate the kernels derive (bit 8, the access then goes to site 0)
 *     and the finiteness of every stored population (bit 4).
 *   - A context is not thread safe; use one per host thread.
 *
 * State layout (the bound state buffer; offsets from rlb_state_offsets):
 *   f[site][node] in the storage precision, site = y*nx + x,
 *   node = (l*n_theta + j)*n_xi + k   (k radial xi_k, j polar th_j, l azimuth ph_l),
 *   then lnM[site] as double (ln of the dynamical mass M, GeV).
 */
#ifndef RLB_H
#define RLB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rlb_ctx rlb_ctx;

typedef enum {
  RLB_OK = 0,
  RLB_ERR_ARG = -1,     /* invalid argument or size                        */
  RLB_ERR_CUDA = -2,    /* a CUDA runtime call or launch failed            */
  RLB_ERR_NUMERIC = -3, /* device error word set (see above)              */
  RLB_ERR_TIMEOUT = -4, /* a bounded device wait expired                  */
  RLB_ERR_STATE = -5,   /* call out of order (e.g. step before init_grid) */
  RLB_ERR_NOMEM = -6    /* host allocation failed                         */
} rlb_status;

typedef enum { RLB_F64 = 0, RLB_F32 = 1, RLB_BF16 = 2 } rlb_prec;
typedef enum { RLB_EOS_CROSSOVER = 0, RLB_EOS_CONST_MASS = 1, RLB_EOS_CONFORMAL = 2 } rlb_eos_kind;
typedef enum { RLB_RADIAL_PAPER = 0, RLB_RADIAL_LAGUERRE = 1 } rlb_radial_family;
typedef enum { RLB_MINKOWSKI = 0, RLB_MILNE = 1 } rlb_metric;

/* Equation of state (Sec. 3.1).  kind CROSSOVER: entropy density
 * s(T) = T^3 [a (1 + tanh((T - Tc)/w))/2 + b]; the quasiparticle mass M(T)
 * solves Z M^3 K_3(M/T)/(2 pi^2) = s(T) and the bag function B(T) solves
 * dB/dT = -Z M^2 T K_1(M/T) dM/dT /(2 pi^2) with B(0) = 0.  CONST_MASS: ideal
 * Boltzmann gas of mass m0 (B = 0).  CONFORMAL: M = B = 0.
 * Z is the number of degrees of freedom (Sec. 3.1: pi^4/180 (4(Nc^2-1)+7 Nc Nf)).
 * The library tabulates the EOS on [T_min, T_max] (GeV, uniform in ln T,
 * table_points nodes; 0 selects 65536). */
typedef struct {
  int kind;
  int table_points;
  double a, b, Tc, w;
  double m0;
  double Z;
  double T_min, T_max;
} rlb_eos_params;

/* Grid, momentum lattice and physics of one run.
 *   nx, ny, dx            periodic transverse grid, spacing in fm
 *   metric                RLB_MILNE (expansion term S1/tau) or RLB_MINKOWSKI
 *   n_xi, n_theta,        lattice of Sec. 4.3: n_xi radial roots, n_theta
 *   n_phi_half              Gauss-Legendre polar nodes, 2 n_phi_half azimuths.
 *                         Supported (n_xi, n_theta, 2 n_phi_half): (8, 8, 12),
 *                         (16, 8, 16), (5, 5, 2), (6, 4, 6), (8, 8, 2).
 *   family, z0, T0        radial rule: PAPER (weight e^{-z0 cosh xi} sinh^2 xi,
 *                         z0 = M0/T0 of Eq. fansatz) or LAGUERRE (massless limit,
 *                         |p~| = T0 x, weight x e^{-x}; needs the conformal EOS)
 *   prec                  population storage: F64 (all arithmetic FP64), F32 or
 *                         BF16 (FP32 arithmetic, FP32 Landau matching and EOS
 *                         inversion)
 *   eta_over_s            shear viscosity to entropy ratio; tau_R follows from
 *                         the Chapman-Enskog relation of Sec. 4.1; INFINITY
 *                         switches collisions off
 *   tau0, dtau            initial proper time and time step (fm/c) */
typedef struct {
  int nx, ny;
  int metric;
  int n_xi, n_theta, n_phi_half;
  int family;
  int prec;
  double dx;
  double z0, T0;
  double eta_over_s;
  double tau0, dtau;
} rlb_grid_params;

/* Create a context bound to CUDA device `cuda_device` (the device is made
 * current for every later call on this context). */
rlb_status rlb_create(rlb_ctx** out, int cuda_device);
void rlb_destroy(rlb_ctx* ctx);
/* Message of the last failed call; owned by ctx, valid until the next call. */
const char* rlb_last_error(const rlb_ctx* ctx);

/* Build the host EOS table (Sec. 3.1).  Must precede rlb_bind_buffers. */
rlb_status rlb_init_eos(rlb_ctx* ctx, const rlb_eos_params* eos);

/* Bytes of device memory a run with grid parameters `g` needs: `state` holds
 * the populations and ln M (layout above); `scratch` holds the predictor
 * state, per-site temperatures, the error word and the EOS table.  Pure
 * function of g and of the EOS table size; may be called before
 * rlb_init_eos (then 65536 table points are assumed).  With g == NULL: the
 * sizes for the grid or batch configured in ctx. */
rlb_status rlb_workspace_size(const rlb_ctx* ctx, const rlb_grid_params* g, size_t* state_bytes,
                              size_t* scratch_bytes);

/* Configure the grid and momentum lattice (host work only). */
rlb_status rlb_configure(rlb_ctx* ctx, const rlb_grid_params* g);

/* One event of a batch: its own periodic nx x ny grid and eta/s. */
typedef struct {
  int nx, ny;
  double eta_over_s;
} rlb_event_desc;

/* Configure a batch of independent events instead of one grid: every event
 * evolves with the scheme of the paper (Sec. 4.4) on its own periodic grid,
 * with its own eta/s; all events share the lattice, precision, dx, tau0, dtau,
 * metric and EOS of `base` (its nx, ny and eta_over_s are ignored).  Sites are
 * stored event after event, row-major inside an event, so the state layout is
 * that of one grid of sum(nx * ny) sites; each rlb_step advances all events
 * with one launch per kernel.  Size the buffers with rlb_workspace_size(ctx,
 * NULL, ...).  Limits: nx <= 65535, fewer than 2^31 sites in total. */
rlb_status rlb_configure_batch(rlb_ctx* ctx, const rlb_grid_params* base, int n_events,
                               const rlb_event_desc* events);

/* Borrow caller-owned device buffers of at least the rlb_workspace_size bytes,
 * 256-byte aligned; the library never frees them.  Uploads the EOS table and
 * the lattice line table and clears the error word on `stream`; the first
 * bind of a context also measures the mean relative error of the device's
 * hardware 2^x over the exponents of f_eq (one small kernel; the FP32 stage
 * kernels divide it out of Z) and synchronises `stream`. */
rlb_status rlb_bind_buffers(rlb_ctx* ctx, void* state, void* scratch, void* stream);

/* Initial condition: local equilibrium at rest with energy density eps0[site]
 * (GeV/fm^3, FP64, nx*ny values on the host or, if eps0_on_device, on the
 * device).  Solves eps_EOS(T) = eps0 for T, sets M = M(T) and
 * f = Z exp(-E/T) at every node, and tau = tau0.  The host array is copied
 * before return; a device array must stay valid until `stream` reaches it. */
rlb_status rlb_init_grid(rlb_ctx* ctx, const double* eps0, int eps0_on_device, void* stream);

/* Initial state of a batch: eps0_concat holds the energy densities of all
 * events' sites in storage order (event after event, row-major); otherwise as
 * rlb_init_grid. */
rlb_status rlb_init_batch(rlb_ctx* ctx, const double* eps0_concat, int eps0_on_device, void* stream);

/* Advance by `nsteps` predictor-corrector steps of dtau (Sec. 4.4).  Each step
 * launches, for the predictor and again for the corrector, a per-site
 * matching kernel (Landau matching and EOS inversion, FP64) and the fused
 * stream-collide kernel.  Asynchronous on `stream`. */
rlb_status rlb_step(rlb_ctx* ctx, int nsteps, void* stream);

/* Step variant for callers that cannot allocate device memory.
 *
 * Some callers may not call cudaMalloc or hand the library scratch of their
 * own: code hosted inside a framework whose allocator owns all device memory,
 * latency-critical loops that cannot absorb the implicit synchronisation of an
 * allocation, or deployments that forbid allocating after start-up.  This
 * entry point advances `nsteps` predictor-corrector steps exactly as rlb_step
 * does, in place on the caller's state buffer (layout of rlb_state_offsets,
 * 256-byte aligned; it needs rlb_init_eos and rlb_configure but no bound
 * buffers), and keeps every intermediate array in one file-scope device array
 * of 24 MiB declared by the library.  It calls no allocating routine: no
 * cudaMalloc, no cudaFree, no library allocator.
 *   - The first call on a device looks up the device address of that array
 *     (cudaGetSymbolAddress) with the context's device current, and the first
 *     call of a context that has no bound buffers measures the mean error of
 *     the device's 2^x approximation (one small kernel using 8 bytes of the
 *     array, and a synchronisation); make these first calls before any stream
 *     capture begins.
 *   - Grids whose scratch would exceed 24 MiB are rejected with RLB_ERR_ARG
 *     (about 4,700 sites with FP32 populations on the 8x8x12 lattice, 2,500 with
 *     FP64).
 *   - Every call in the process shares the array, which keeps whatever the last
 *     call left in it: each call re-uploads the EOS tables, clears the error
 *     word and the Newton starting temperatures, and recomputes the moments of
 *     its input.  Calls whose GPU work overlaps (other streams, threads or
 *     contexts on the same device) race on the array; the caller serialises
 *     them.
 *   - The call synchronises `stream` before returning and reports a numeric
 *     failure recorded during it as RLB_ERR_NUMERIC.
 * The paper has no counterpart of this entry point: it concerns memory
 * management only. */
rlb_status rlb_step_static_scratch(rlb_ctx* ctx, void* state, int nsteps, void* stream);

/* Checkpoint and restart (blobs in host or device memory).  A state blob holds a header (grid, lattice and
 * precision it belongs to, and tau), the populations f, ln M, the per-site
 * Newton starting temperatures and the stored moments of f, so that a run
 * restarted from a blob continues bit for bit like the uninterrupted run (same
 * library build, same GPU).  rlb_state_blob_size gives the bytes (configured
 * context).  rlb_save_state copies the current state into `host_buf` (host
 * or device memory of at least that size; a host buffer is complete when the
 * call returns (it synchronises `stream`), a device buffer once `stream`
 * reaches the copies: the call enqueues them and returns); rlb_load_state
 * checks the header against the configured grid (RLB_ERR_ARG on a mismatch or
 * a short buffer, the message says which) and replaces the state, tau
 * included (it reads the header on the host and synchronises `stream`); eta/s,
 * dtau and the EOS are taken from the context, not from the blob.
 * rlb_load_state_async replaces the state from a device blob that
 * rlb_save_state of this context wrote, without reading its header back: the
 * caller passes the tau rlb_get_tau reported when the blob was saved, and the
 * copies are only enqueued on `stream` (RLB_ERR_ARG for a host pointer or a
 * short buffer).  The paper's scheme needs exactly this state to continue
 * (Sec. 4.4: f, M and T at tau). */
rlb_status rlb_state_blob_size(const rlb_ctx* ctx, size_t* bytes);
rlb_status rlb_save_state(rlb_ctx* ctx, void* host_buf, size_t bytes, void* stream);
rlb_status rlb_load_state(rlb_ctx* ctx, const void* host_buf, size_t bytes, void* stream);
rlb_status rlb_load_state_async(rlb_ctx* ctx, const void* dev_buf, size_t bytes, double tau, void* stream);

/* Launch tuning.  rlb_step records one time step (match, predictor stage,
 * match, corrector stage) as a CUDA graph on the context's own stream the first
 * time it runs and replays it for every step; the caller's stream is ordered
 * before and after the replays with events, so the call stays asynchronous on
 * `stream`.  The launch parameters are the same for every step because the
 * proper time lives in a device clock.  A step that follows rlb_moments
 * starts from the matching rlb_moments made and replays a second graph without
 * the first matching.  rlb_set_graphs(ctx, 0) switches back to plain launches
 * (per-kernel timing does so by itself).  The graphs are recaptured after
 * rlb_bind_buffers, rlb_autotune or rlb_set_stage_variant.
 *
 * rlb_autotune times every compiled variant of the stage kernel for the
 * configured lattice and precision (packed FP32 kernel with one site per CTA,
 * with and without its register cap; generic kernel; packed kernel with two
 * sites per CTA, with and without its cap; for the 8 x 8 x 12 lattice the
 * mirror-paired kernel, variant 5, the default there: one thread holds the
 * polar lines theta and pi - theta; with FP32 storage also variant 6, the
 * mirror-paired kernel reading its own and its upwind neighbours' lines from
 * shared memory filled by bulk asynchronous copies (one grid with an even nx;
 * elsewhere variant 6 runs variant 5); one variant for lattices only the
 * generic kernel takes) on three predictor launches over the current state,
 * and keeps the fastest for later steps.  The state (f, ln M, tau) is
 * unchanged.  Outputs: the chosen variant, optionally the milliseconds per
 * launch of each variant (variant_ms holds at least RLB_MAX_STAGE_VARIANTS
 * doubles; -1 for a variant that would run another variant's kernel on this
 * configuration, which is never chosen) and their number.  Synchronises
 * `stream`.  Implementation choices, not part of the paper's scheme. */
#define RLB_MAX_STAGE_VARIANTS 8
rlb_status rlb_autotune(rlb_ctx* ctx, void* stream, int* chosen, double* variant_ms, int* n_variants);
/* rlb_set_stage_variant picks a stage-kernel variant by number (the order of
 * rlb_autotune's list) for later steps; variant < 0 only reports their number
 * in n_variants (optional).  RLB_ERR_ARG for a number outside the list; every
 * variant computes the same result.  Needs rlb_configure (or rlb_init_grid). */
rlb_status rlb_set_stage_variant(rlb_ctx* ctx, int variant, int* n_variants);
rlb_status rlb_set_graphs(rlb_ctx* ctx, int enable);

/* Adjoint of the time evolution (discrete adjoint of the predictor-corrector of
 * Sec. 4.4 with the 2+1D terms, for every storage precision; per-node work in
 * FP64 (default) or FP32 arithmetic, per-site matching adjoint in FP64).
 * The objective is the final-state elliptic flow v2_pt of rlb_observables; the
 * gradients are with respect to the initial energy density (projected on a
 * caller basis, e.g. the hotspot Gaussians) and to eta/s.  The paper has no
 * adjoint; this is the sensitivity of its scheme.
 *
 *   rlb_adjoint_set_arithmetic
 *       RLB_F64 (default) or RLB_F32: the arithmetic and storage of the
 *       per-node adjoints (the stage adjoints: forward recompute, transposed
 *       operators and stencil).  A change unbinds the workspace (its layout
 *       changes); call before rlb_adjoint_workspace_size.  RLB_ERR_ARG for
 *       another value.
 *   rlb_adjoint_workspace_size / rlb_adjoint_bind
 *       Device workspace (caller-owned, 256-byte aligned): the adjoints of f
 *       and ln M and per-stage intermediates (about 3 x 8 bytes x populations
 *       in FP64, 3 x 4 in FP32).
 *   rlb_adjoint_seed_v2
 *       v2_pt of the current state (written to *v2) and the adjoint buffers set
 *       to d v2_pt / d(f, ln M) of that state; the eta/s accumulator is cleared.
 *   rlb_adjoint_seed
 *       A general objective J: the adjoint buffers set to fbar = dJ/df (sites x
 *       nodes FP64, the state's layout) and lbar = dJ/d ln M (sites FP64) of the
 *       current state, host or device memory (any pointer CUDA's unified
 *       addressing knows); the eta/s accumulator is cleared.  Synchronises.
 *   rlb_adjoint_step
 *       The adjoint buffers hold the adjoints of the output of one time step;
 *       the context state (f, ln M, tau: e.g. restored with rlb_load_state) is
 *       that step's input.  Replaces them by the adjoints of the step's input
 *       and adds the step's contribution to d v2/d(eta/s).  The step's
 *       predictor output is recomputed with the forward kernels, bit for bit as
 *       in the forward run; the matchings are recomputed in FP64 for the FP64
 *       adjoint arithmetic, and taken as the forward step makes them (FP32
 *       moment partials, the same Newton starts) by the FP32 adjoint of the
 *       FP32/BF16 storage paths.
 *   rlb_adjoint_ic
 *       After the last rlb_adjoint_step (the adjoint buffers hold the adjoints
 *       of the initial state rlb_init_grid made from eps0, device FP64,
 *       GeV/fm^3): grad[i] = sum_x basis[i][x] d v2/d eps0(x) for the n_basis
 *       rows of `basis` (device FP64, n_basis x sites, n_basis <= sites), then
 *       grad[n_basis] = d v2/d(eta/s).  `grad` is host memory; synchronises.
 *   rlb_adjoint_step_from
 *       The same reversed step with its input state read in place from a
 *       device blob that rlb_save_state of this context wrote (`bytes` its
 *       size, `tau` the rlb_get_tau value it was saved at; the header is not
 *       read back): no copy into the context.  The context's state and tau
 *       are unchanged; its Newton starting temperatures become the blob's.
 * Checkpointing (which states to keep and recompute) is the caller's choice;
 * the Python module adjoint.py keeps one every k steps. */
rlb_status rlb_adjoint_set_arithmetic(rlb_ctx* ctx, int prec);
rlb_status rlb_adjoint_workspace_size(rlb_ctx* ctx, size_t* bytes);
rlb_status rlb_adjoint_bind(rlb_ctx* ctx, void* workspace);
rlb_status rlb_adjoint_seed_v2(rlb_ctx* ctx, double* v2, void* stream);
rlb_status rlb_adjoint_seed(rlb_ctx* ctx, const double* fbar, const double* lbar, void* stream);
rlb_status rlb_adjoint_step(rlb_ctx* ctx, void* stream);
rlb_status rlb_adjoint_step_from(rlb_ctx* ctx, const void* state_blob, size_t bytes, double tau, void* stream);
rlb_status rlb_adjoint_ic(rlb_ctx* ctx, const double* eps0, const double* basis, int n_basis, double* grad,
                          void* stream);

/* Current proper time (host bookkeeping, fm/c). */
rlb_status rlb_get_tau(const rlb_ctx* ctx, double* tau);

/* Per-site observables of the current state, 8 doubles per site:
 *   eps [GeV/fm^3] (Landau energy density incl. B), T [GeV], u^tau, u^x, u^y,
 *   M [GeV] (dynamical mass), P_L [GeV/fm^3] (tau^2 T^{YY}), M(T) [GeV].
 * `out` is host memory (synchronises `stream`) or device memory
 * (out_on_device != 0, asynchronous).  The call runs the matching of the
 * current state (Landau condition and EOS inversion, Sec. 4.4); the next
 * rlb_step starts from it instead of repeating it, so stepping with per-step
 * observables costs no extra matching and gives the same states bit for bit. */
rlb_status rlb_moments(rlb_ctx* ctx, double* out, int out_on_device, void* stream);
/* The same observables into page-locked host memory without waiting for them:
 * the matching runs on `stream` into one of two device staging slots (sites x 8
 * doubles each, allocated by the context at its first call and freed by
 * rlb_destroy), and the download runs on a copy stream of the context, so
 * that the next rlb_step on `stream` overlaps it.  `host_out` (caller-owned)
 * must stay allocated and untouched until rlb_moments_wait returns (it waits
 * for every download enqueued so far and reports the device error word like
 * rlb_check); a slot's next use waits for its previous download.  RLB_ERR_ARG
 * for pageable host memory. */
rlb_status rlb_moments_async(rlb_ctx* ctx, double* host_out, void* stream);
rlb_status rlb_moments_wait(rlb_ctx* ctx);

/* Grid observables of the current state (two host doubles; synchronises
 * `stream`):
 *   eps_p = sum_x (T^xx - T^yy) / sum_x (T^xx + T^yy)  (momentum anisotropy,
 *           T^{mu nu} = T_kin^{mu nu} + B(T) g^{mu nu}, lab-frame components),
 *   v2_pt = sum_{x,n} W_n p_perp,n cos(2 phi_n) f_n / sum_{x,n} W_n p_perp,n f_n
 *           (elliptic flow weighted by transverse momentum, W_n = M^2 w_n/(2 pi^2),
 *           p_perp,n = M sinh(xi_k) sin(theta_j)).
 * Built on the moments of Eq. emtnew and the weights of Sec. 4.3; the paper
 * itself defines no observables (these are the usual heavy-ion ones).  The
 * matching needed for B(T) runs on the stored moments; a numeric failure there
 * returns RLB_ERR_NUMERIC.  Sums over sites run in a fixed order in FP64. */
rlb_status rlb_observables(rlb_ctx* ctx, double* eps_p, double* v2_pt, void* stream);

/* Per-kernel device timing.  While enabled, every launch made by this
 * context is bracketed by CUDA events on its stream; rlb_get_timing waits for
 * the pending events and returns the accumulated milliseconds and launch
 * counts of the fused stream-collide kernel (two per step) and of the per-site
 * matching kernel (two per step).  Enabling resets the counters. */
rlb_status rlb_set_timing(rlb_ctx* ctx, int enable);
rlb_status rlb_get_timing(rlb_ctx* ctx, double* stage_ms, long* stage_launches, double* match_ms,
                          long* match_launches);

/* Arithmetic-pipe peaks of device `cuda_device`, measured (not nominal), for
 * the ALU rooflines of the stage kernels: tflops[0] FP32 fused multiply-add,
 * tflops[1] packed FP32 pairs (FFMA2), tflops[2] FP64 fused multiply-add, in
 * TFLOP/s (2 flops per multiply-add).  Independent multiply-add chains in 8
 * CTAs of 256 threads per SM, one warm-up and one timed launch of about 20 ms
 * each, CUDA events; at whatever SM clock the device runs.  A measurement
 * helper with no counterpart in the paper.  Synchronises the device's work it
 * launches; no context needed. */
rlb_status rlb_alu_peaks(int cuda_device, double* tflops);

/* The bounded wait of the halo-staged stage kernel (stage variant 6) on its
 * own: one CTA sets up the mbarrier its staging completes on, expecting 16
 * bytes, issues the 16-byte bulk copy of a device value 1.25 only when
 * `deliver` is nonzero, and waits at most limit_ms (0 < limit_ms <= 2000).
 * *expired = 1 when the wait ran out (the stage kernel then sets device error
 * bit 16 and rlb_check returns RLB_ERR_TIMEOUT), 0 when the copy arrived;
 * *value (optional) = the copied value.  A test helper with no counterpart in
 * the paper: it shows on a GPU that the wait ends and the context stays
 * usable, without a fault.  Synchronous; no context needed. */
rlb_status rlb_wait_selftest(int cuda_device, int deliver, double limit_ms, int* expired, float* value);

/* Synchronise `stream` and report the device error word (RLB_ERR_NUMERIC if set). */
rlb_status rlb_check(rlb_ctx* ctx, void* stream);

/* Byte offsets of f and lnM inside the state buffer, and the storage size of
 * one population in bytes. */
rlb_status rlb_state_offsets(const rlb_ctx* ctx, size_t* f_offset, size_t* lnM_offset,
                             size_t* pop_bytes);

/* Host copies of the momentum lattice (for checks): radial c = cosh xi_k
 * (or x_k), s = sinh xi_k (or x_k), w^xi_k; polar mu_j = cos th_j, w^th_j;
 * azimuth cos ph_l, sin ph_l.  Arrays of n_xi, n_theta and 2 n_phi_half. */
rlb_status rlb_lattice(const rlb_ctx* ctx, double* c, double* s, double* wxi, double* mu,
                       double* wth, double* cph, double* sph);

/* Host copies of the nodal operator matrices (row-major [out][in]) of
 * Sec. 4.4: Dr, the Galerkin representation of v.d/dv on the radial nodes
 * (n_xi^2; the radial part of S1 and S2), and Dth, the Galerkin representation
 * of (mu - mu^3) d/dmu on the polar nodes (n_theta^2; the polar part of S1). */
rlb_status rlb_operators(const rlb_ctx* ctx, double* Dr, double* Dth);

#ifdef __cplusplus
}
#endif
#endif /* RLB_H */
