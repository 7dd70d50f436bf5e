/*
 * pnp.h — C ABI of the GB300 NS-PNP fractional-step library (libpnp.so).
 *
 * The library advances the coupled Navier-Stokes / Poisson-Nernst-Planck
 * equations of arXiv:1701.02005 (Eqs. (1)-(4), Numerical methods) for plane
 * Couette flow of a dilute binary univalent electrolyte: walls at y = -1, +1
 * moving at -Uw, +Uw and held at potentials -V, +V; periodic x and z.
 * Quantities are nondimensional with h (half gap), U (wall speed), h/U,
 * c0 (bulk concentration), V_T (thermal voltage) and rho_w U^2 (pressure).
 *
 * Ownership: the caller allocates ONE device workspace (size from
 * pnp_workspace_bytes) and keeps it alive until pnp_destroy; the context only
 * borrows it.  Host memory of the context is freed by pnp_destroy.
 * Streams: every kernel and copy is issued on the stream given to
 * pnp_init_grid (a cudaStream_t passed as void*; NULL = legacy default
 * stream, in which case steps are launched without CUDA graphs).
 * Errors: every entry point returns PNP_OK (0) or a negative pnp_status
 * code; nothing throws across the ABI.  There is no CPU fallback: without a
 * CUDA device every call that launches work returns PNP_ERR_CUDA.
 * Layout: all fields are [y][z][x] with x fastest.  Cell-centred fields have
 * (Ny-1)*Nz*Nx entries; v lives on the y faces and has Ny*Nz*Nx entries
 * whose first and last planes (the walls) are zero.  Ny counts y face nodes.
 */
#ifndef PNP_H
#define PNP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pnp_ctx pnp_ctx;

/* Status codes. */
enum {
  PNP_OK = 0,
  PNP_ERR_ARG = -1,          /* null pointer, bad enum, non-finite parameter      */
  PNP_ERR_GRID = -2,         /* Nx, Nz not powers of two in [4, 4096], Ny < 3     */
  PNP_ERR_WORKSPACE = -3,    /* workspace too small or misaligned (256 B)         */
  PNP_ERR_CUDA = -4,         /* a CUDA runtime call failed (no device, launch)    */
  PNP_ERR_STATE = -5,        /* parameters or state not set yet                   */
  PNP_ERR_NONFINITE = -6,    /* device check: NaN/Inf in a prognostic field       */
  PNP_ERR_NEGATIVE_C = -7,   /* device check: a concentration went negative       */
  PNP_ERR_UNSUPPORTED = -8,  /* option not available for this precision          */
  PNP_ERR_TOO_LARGE = -9,    /* grid exceeds the static scratch of pnp_poisson_noalloc */
  PNP_ERR_TIMEOUT = -10,     /* device check: an asynchronous copy did not complete in time */
  PNP_ERR_CFL = -11,         /* device check: advective CFL number of the last dt above its limit */
  PNP_ERR_DPHI = -12         /* device check: potential step between neighbouring cells above its limit */
};

/* Arithmetic precision of a context. */
enum {
  PNP_FP64 = 0,   /* every field, stencil, FFT and solve in FP64                  */
  PNP_MIXED = 1   /* FP32: u, v, w, p and every stencil (advection, viscous and
                     Coulomb terms, ion fluxes of the fluctuations about the
                     plane-mean reference profiles); FP64-level: the ion state
                     (FP64 reference profile + double-float fluctuation), the
                     reference double-layer terms (FP64 per plane), the global
                     sums (double-float per thread, FP64 across threads).  The
                     solves depend on the policy (pnp_set_policy): by default
                     the spectral y-solves of both Poisson problems in double-
                     float, the (0,0) potential mode and the reference ion CN
                     in FP64, the transforms and the velocity and ion-
                     fluctuation CN solves in FP32; PNP_POLICY_FP64_SOLVES moves
                     every transform and tridiagonal solve to FP64 arithmetic */
};

/* Solve precision of a PNP_MIXED context (see above). */
enum {
  PNP_POLICY_DEFAULT = 0,      /* FP32 transforms and CN, double-float spectral solves */
  PNP_POLICY_FP64_SOLVES = 1   /* FP64 transforms, spectral and CN solves                 */
};

/* Fields for pnp_set_state / pnp_get_state / pnp_mean_profile. */
enum {
  PNP_U = 0, PNP_V = 1, PNP_W = 2, PNP_P = 3,
  PNP_CP = 4, PNP_CM = 5, PNP_PHI = 6,       /* PHI is the total potential V y + phi */
  PNP_HU = 7, PNP_HV = 8, PNP_HW = 9,        /* explicit terms of the last substage  */
  PNP_HCP = 10, PNP_HCM = 11,
  PNP_NFIELDS = 12
};
/* The next step's first RK3 substage has zeta = 0 and never reads H, so after
 * pnp_step in PNP_MIXED the H fields hold the second substage's explicit terms
 * (the third substage's are not written); PNP_FP64 keeps the third's. Either
 * way the continuation of the run is the same. pnp_eval_explicit always
 * stores them. */

/* Initial conditions for pnp_init_state. */
enum {
  PNP_IC_LAMINAR = 0,  /* u = Uw y, uniform ions c+ = c- = 1                        */
  PNP_IC_PB = 1        /* u = Uw y, superposed Gouy-Chapman double layers           */
};

/* Boundary condition of pnp_poisson. */
enum { PNP_NEUMANN = 0, PNP_DIRICHLET = 1 };

/* Diagnostics (Numerical methods: tau_w, c_f, Re_tau; Fig. 1: wall flux). */
typedef struct pnp_diag {
  double tau_bot;     /* (1/Re) d<u>/dy at y = -1 (plane average)                 */
  double tau_top;     /* (1/Re) d<u>/dy at y = +1                                 */
  double cf;          /* 2 tau_w / Uw^2, tau_w the mean of the two walls          */
  double re_tau;      /* Re sqrt(tau_w)                                           */
  double n_plus;      /* sum c+ dV                                                */
  double n_minus;     /* sum c- dV                                                */
  double net_charge;  /* n_plus - n_minus                                         */
  double wall_flux;   /* |flux_plus| + |flux_minus| (zero by design, Fig. 1)     */
  double max_div;     /* max |div u| over the cells                               */
  double ke;          /* kinetic energy 1/2 sum |u|^2 dV                          */
  double time;        /* simulated time                                           */
  long long nstep;    /* completed steps                                          */
  int status;         /* device error word (PNP_OK or a PNP_ERR_* code)           */
  int precision;
  double cfl;         /* dt max(|u|/dx + |v|/dy + |w|/dz), cell-centred velocities,
                         dt the last step's size (0 before the first step)       */
  double max_dphi;    /* max |Phi difference| between neighbouring cells (x, z,
                         interior y faces), in units of V_T                      */
  double flux_plus;   /* net c+ flux out through the two wall faces implied by the
                         stored explicit terms: -sum H_c+ dV (the discrete
                         divergence theorem; the implicit y-diffusion has no wall
                         coupling), per unit time                                */
  double flux_minus;  /* the same for c-                                         */
  double dt_cfl;      /* dt at which the advective CFL number reaches 1          */
  double dt_migration;/* dt at which the ion drift D |grad Phi| crosses one cell
                         (the explicit migration term's CFL number reaches 1)    */
  double dt_dielectric; /* 1 / max D (c+ + c-) / (2 lam^2): the time scale of
                         dielectric (charge) relaxation, explicit in the scheme  */
} pnp_diag;

/* Bytes of device workspace needed for an Nx x Ny x Nz grid (Ny = face nodes). */
int pnp_workspace_bytes(int nx, int ny, int nz, int precision, size_t* out_bytes);

/* Create a context on the grid of Fig. 1: Nx, Nz powers of two (periodic,
 * lengths Lx, Lz), Ny y-face nodes with tanh stretching yf_j =
 * tanh(g (2j/(Ny-1) - 1)) / tanh(g) (g = stretch; 0 = uniform).  The
 * workspace (device, >= pnp_workspace_bytes, 256-byte aligned) is borrowed. */
int pnp_init_grid(pnp_ctx** out, int nx, int ny, int nz, double Lx, double Lz,
                  double stretch, int precision, void* device_workspace,
                  size_t workspace_bytes, void* cuda_stream);

/* Replace the y faces by Ny host values; y_faces[0] and y_faces[Ny-1] are
 * forced to -1 and +1.  Invalidates the state. */
int pnp_set_yfaces(pnp_ctx* ctx, const double* y_faces_host, int ny);

/* Control parameters (Numerical methods): Re = rho_w U h / eta, debye_len =
 * lambda_D / h, Sc = eta / (rho_w D), wall_potential = V / V_T (the paper's
 * V-hat is 2 V), beta = eps V_T^2 / (eta D) (typically 0.5).  Restores the
 * uniform walls -V, +V.  With a state present (parameters changed mid-run) the
 * potential of the present ions is solved again under the new parameters
 * (synchronises). */
int pnp_set_params(pnp_ctx* ctx, double Re, double debye_len, double Sc,
                   double wall_potential, double beta);

/* Wall potentials that vary along the walls (the paper's walls may carry any
 * potential; Eq. (4) with Dirichlet data): bottom, top = Nz*Nx host values
 * ([z][x], one per wall face below / above a cell column), in units of V_T.
 * Phi = Phi_0 + phi with Phi_0 = (1 - y)/2 bottom + (1 + y)/2 top the linear
 * lift (on which the finite-volume y-operator is exact) and phi = 0 on the
 * walls solving L phi = -(c+ - c-) / (2 lam^2) - (d_xx + d_zz) Phi_0.  The
 * context solves the charge-free part of the wall variations once here (one
 * FP64 Dirichlet solve) and adds it in every potential solve; the plane means
 * act as the uniform walls (V = (mean top - mean bottom) / 2 plus a constant).
 * If a state is loaded its potential is re-solved under the new walls at once.
 * Call again between steps for a time-varying potential; both NULL restore the
 * uniform walls of pnp_set_params (which also resets them).  Synchronises. */
int pnp_set_wall_potential(pnp_ctx* ctx, const double* bottom_host, const double* top_host);

/* Wall speed in units of U (default 1; 0 gives the quiescent validation run). */
int pnp_set_wall_velocity(pnp_ctx* ctx, double Uw);

/* Initial state on the device: Couette profile plus SplitMix64 noise of
 * amplitude noise_amp damped by (1 - y^2) and projected to zero divergence;
 * ions by ic_kind; Phi from Eq. (4); p = 0 and stored explicit terms zero. */
int pnp_init_state(pnp_ctx* ctx, int ic_kind, uint64_t seed, double noise_amp);

/* Copy one field in or out as FP64 values in the layout above (converted on
 * the device in mixed precision).  on_device != 0: src/dst is a device
 * pointer; otherwise host memory (pinned for asynchrony; get_state to host
 * synchronises the stream). */
int pnp_set_state(pnp_ctx* ctx, int field, const void* src, int on_device);
int pnp_get_state(pnp_ctx* ctx, int field, void* dst, int on_device);

/* Number of FP64 values of a field (cells or v faces). */
int pnp_field_size(pnp_ctx* ctx, int field, size_t* out_count);

/* Advance nsteps full RK3 steps of size dt (three substages each: explicit
 * terms, y-implicit Crank-Nicolson solves, pressure projection, potential
 * solve).  Asynchronous on the context's stream; on a non-default stream the
 * step is captured once per dt into a CUDA graph and replayed. */
int pnp_step(pnp_ctx* ctx, int nsteps, double dt);

/* Deterministic reductions of the current state (fixed order; FP64 block
 * sums); synchronises the stream.  PNP_MIXED after a step reads the FP32
 * fields and the double-float ion state directly: per-thread sums in
 * double-float (squares exact, weights dy, h and the divergence coefficients
 * as double-float pairs), no FP64 copy of the state; the ion numbers and
 * energies agree with their FP64 evaluation to ~1e-13 relative. */
int pnp_diagnostics(pnp_ctx* ctx, pnp_diag* out);

/* The same diagnostics in two halves, so that a caller can read them every
 * step without stalling the GPU.  pnp_diagnostics_post queues the reductions
 * of the current state on the context's stream and a copy of their raw sums
 * into raw_host (PNP_DIAG_RAW_BYTES bytes, caller-owned; pinned host memory
 * keeps the copy asynchronous), and returns without waiting; the record also
 * keeps the host-side values of that moment (time, step count, dt, reference
 * sums).  Once the stream has passed the post (an event recorded after it, or
 * a synchronisation), pnp_diagnostics_read turns the record into a pnp_diag
 * (host work only) and returns its status.  raw_host must not be reused
 * before then.  pnp_diagnostics is post + synchronise + read. */
#define PNP_DIAG_RAW_BYTES 256
int pnp_diagnostics_post(pnp_ctx* ctx, void* raw_host);
int pnp_diagnostics_read(const pnp_ctx* ctx, const void* raw_host, pnp_diag* out);

/* Adaptive time step (the explicit parts of the scheme -- advection,
 * migration and with it the dielectric relaxation -- bound dt; Numerical
 * methods, the stiffness of the double layer): advances nsteps steps; before
 * every block of check_every steps (>= 1) it reads the state's limits (as
 * pnp_diagnostics, synchronising) and takes dt = min(dt_max, cfl dt_cfl,
 * cfl dt_migration, 4 cfl dt_dielectric), rounded down to the ladder
 * dt_max 2^(-k/8) so that a run revisits few distinct dt values (each new dt
 * recomputes the CN factors and recaptures the step's graph); dt grows by at
 * most one rung per check.  dts_out (host, optional, nsteps values) receives
 * the dt of every step.  0 < cfl <= 1.  Stops with the device status if a
 * check reports one (PNP_ERR_NONFINITE, ...). */
int pnp_step_adaptive(pnp_ctx* ctx, int nsteps, double dt_max, double cfl, int check_every, double* dts_out);

/* Time-integration scheme of the viscous and diffusive terms (Numerical
 * methods: the AFiD fractional step).  PNP_SCHEME_CN: Crank-Nicolson in y
 * (the wall-normal Thomas solves), x/z terms explicit in the RK3 right-hand
 * side.  PNP_SCHEME_AF: Crank-Nicolson in all three directions, approximately
 * factorised, (I - s L_x)(I - s L_z)(I - s L_y) dq = r with r holding the
 * explicit half of the full Laplacian: periodic (cyclic) tridiagonal solves in
 * x and z, which lift the x/z viscous and diffusive stability limits.
 * Migration and advection stay explicit.  The cyclic systems have constant
 * coefficients, so their inverses are circulant: where the inverse's kernel
 * falls below the arithmetic's rounding within eight taps, both directions run
 * as one pass of truncated convolutions (the same result to rounding), else as
 * cyclic Thomas sweeps.  With the fused CN elimination (pnp_set_fusion) the x/z
 * solves act on the stencil's forward-elimination values, which they commute
 * with. */
enum { PNP_SCHEME_CN = 0, PNP_SCHEME_AF = 1 };
int pnp_set_scheme(pnp_ctx* ctx, int scheme);

/* PNP_MIXED with the default policy: fuse the forward elimination of the
 * wall-normal CN solves into the explicit-term stencil (on != 0, the default).
 * The stencil, which marches y in chunks, stores each chunk's forward-
 * elimination values started from zero instead of the right-hand sides; the CN
 * kernel recovers every line's true values from the chunk-end values and
 * per-row products of the factors, then back-substitutes: the right-hand sides
 * never make an HBM round trip.  Off: the right-hand sides are stored and the
 * CN kernels eliminate both ways (the shared-memory CN tiles, launch code 32,
 * always take that path). */
int pnp_set_fusion(pnp_ctx* ctx, int on);

/* Select the solve precision of a PNP_MIXED context (PNP_POLICY_*): the
 * stencils, storage and sums are the same under both; PNP_POLICY_FP64_SOLVES
 * runs the wall-normal CN solves of u, v, w and of the ion fluctuations, both
 * Poisson problems' x/z transforms and their spectral y-solves in FP64
 * arithmetic (FP64 forward values, one rounding to the state's storage), as a
 * plain reading of "FP64 for the tridiagonal and Poisson solves" asks.
 * PNP_ERR_UNSUPPORTED for a non-default policy on a PNP_FP64 context. */
int pnp_set_policy(pnp_ctx* ctx, int policy);

/* Stability limits of the diagnostics' device checks: PNP_ERR_CFL when dt max(|u|/dx + |v|/dy + |w|/dz) of the
 * last step exceeds cfl_max (default sqrt(3), the imaginary-axis stability
 * bound of the three-stage RK3 for centred advection), PNP_ERR_DPHI when the
 * potential changes by more than dphi_max between neighbouring cells (default
 * 2: beyond it the discrete Boltzmann ratio (2 - dPhi) / (2 + dPhi) of the
 * arithmetic face means turns negative and the migration flux can drive a
 * concentration below zero).  Both are reported by pnp_diagnostics / pnp_status
 * after NaN/Inf and negative-concentration checks; the step is not stopped. */
int pnp_set_limits(pnp_ctx* ctx, double cfl_max, double dphi_max);

/* Time statistics (Results: the mean profiles in wall units, the RMS ion and
 * potential fluctuations, the friction coefficient c_f): pnp_stats_sample adds
 * the plane means of q and q^2 of the current state for q = u, v, w, c+, c-,
 * Phi to FP64 accumulators (asynchronous; call it every few steps);
 * pnp_stats_get returns, per y-plane, the time-and-plane mean <q>(y) and the
 * RMS fluctuation sqrt(<q^2> - <q>^2) in mean_out / rms_out (host, 6 x Ny
 * values: [u, v, w, c+, c-, Phi][Ny], cell quantities in the first Ny-1, v on
 * all Ny faces), the time-averaged c_f = (tau_bot + tau_top) / Uw^2 of the
 * mean profile, and the number of samples (synchronises).  pnp_stats_reset
 * zeroes them. */
int pnp_stats_reset(pnp_ctx* ctx);
int pnp_stats_sample(pnp_ctx* ctx);
int pnp_stats_get(pnp_ctx* ctx, double* mean_out, double* rms_out, double* cf_mean, long long* nsamples);

/* Plane average <q>(y) of a field into host memory (Ny-1 values, Ny for v). */
int pnp_mean_profile(pnp_ctx* ctx, int field, double* out_host);

/* Separable Poisson solve on the context's grid (Numerical methods, potential
 * paragraph): (d_xx + d_zz + L_y) x = rhs with modified wavenumbers, real FFT
 * in x and z and one Thomas solve in y per wavenumber.  PNP_NEUMANN: zero wall
 * flux, mode (0,0) pinned to zero in its bottom cell; PNP_DIRICHLET: x = 0 on
 * the wall faces.  rhs and x are device FP64 arrays of (Ny-1)*Nz*Nx values and
 * may alias.  Uses the context's scratch; asynchronous. */
int pnp_poisson(pnp_ctx* ctx, int bc, const double* rhs_dev, double* x_dev);

/* No counterpart in the paper: a convenience for callers that cannot allocate
 * device memory (a plug-in inside a framework that owns every allocation, or a
 * latency-critical path where cudaMalloc may synchronise or fail).  Performs the
 * same separable Poisson solve as pnp_poisson, but needs no context and
 * allocates nothing: its scratch is one static device array of about 48 MB
 * (held by every GPU that loads the library until the process exits), which
 * serves grids with (Ny-1) * Nz * pitch <= 2^20 spectral points (pitch = Nx/2+1
 * rounded up to a multiple of 8), Nx, Nz <= 4096 and Ny <= 2049; larger grids
 * return PNP_ERR_TOO_LARGE.  y_faces_host: Ny increasing host values (the first
 * and last are taken as -1 and +1), read before the call returns: they travel
 * to the GPU as a kernel argument, which also builds the grid constants in the
 * scratch, in stream order; rhs_dev, x_dev: device FP64 arrays of
 * (Ny-1)*Nz*Nx values in the [y][z][x] layout (they may alias); cuda_stream:
 * the stream to run on (NULL = legacy default stream).  The first call on a
 * device looks up the device address of the scratch (cudaGetSymbolAddress);
 * make that first call before any stream capture.  All calls share the one
 * scratch, which keeps the last call's contents: calls queued on one stream
 * run one after the other, but calls that overlap on the GPU (different
 * streams, or different host threads) race and corrupt each other's results;
 * serialise them.  Asynchronous; returns PNP_OK or an error. */
int pnp_poisson_noalloc(int nx, int ny, int nz, double Lx, double Lz, const double* y_faces_host, int bc,
                        const double* rhs_dev, double* x_dev, void* cuda_stream);

/* Overwrite the stored explicit terms H (fields PNP_HU..PNP_HCM) with those of
 * the current state (advection, x/z diffusion, Coulomb force, migration). */
int pnp_eval_explicit(pnp_ctx* ctx);

/* Device error word of the last diagnostics, or PNP_ERR_TIMEOUT when a bounded
 * copy wait of a kernel ran out (sticky, takes precedence); synchronises. */
int pnp_status(pnp_ctx* ctx);

/* Zero the device error words (synchronises). */
int pnp_clear_status(pnp_ctx* ctx);

/* Failure-path self-test (no counterpart in the paper): one block waits, with
 * the same bounded mbarrier wait the TMA stencil uses, on a barrier that no
 * copy completes; after limit_s seconds (0 < limit_s <= 10) the wait gives up
 * and records PNP_ERR_TIMEOUT.  Faults and hangs nothing; returns pnp_status
 * (PNP_ERR_TIMEOUT on a working GPU).  Clear with pnp_clear_status. */
int pnp_selftest_wait_timeout(pnp_ctx* ctx, double limit_s);

/* Measured FP64 FMA throughput of this device in FLOP/s (bounded microbenchmark
 * on the context's stream): the ALU ceiling of the FP64 kernels. */
int pnp_fp64_peak(pnp_ctx* ctx, double* flops_out);

/* Autotuner (no counterpart in the paper; launch-shape selection for GB300):
 * times candidate launch codes of the stencil (FP64: block x-extent 16/32/64/128
 * of 128 threads; mixed: 16 one-cell tiles, 32 / 64 packed two-cell tiles
 * 32 / 64 cells wide, 128 TMA rows), the
 * wall-normal CN sweeps (32 = mixed
 * shared-memory line tiles, else 64/128/256 threads per block), the spectral
 * y-solves (16 = mixed shared-memory tiles, else 32/64/128 threads) and the
 * z-transform (8..64 threads per column; mixed: 64 = stage-by-stage kernel,
 * else register FFT) on this context's grid with CUDA events and keeps the
 * fastest; then re-checks each choice, one code at a time, on the time of
 * whole steps of size dt (pnp_step from a Poisson-Boltzmann initial state),
 * since launch shapes interact inside a step.  cfg_out[4] receives the choice
 * (same order as pnp_set_launch_config), ms_out[4] (optional) the best time of
 * each site alone.  It runs on the workspace and overwrites the state: call it
 * after pnp_set_params and before pnp_init_state / pnp_set_state.
 * Synchronises the stream. */
int pnp_autotune(pnp_ctx* ctx, double dt, int* cfg_out, double* ms_out);
/* Set / read the launch shapes {stencil block x, CN block, spectral block,
 * z-transform threads per column} (e.g. from a cache of autotuner results). */
int pnp_set_launch_config(pnp_ctx* ctx, const int* cfg);
int pnp_get_launch_config(pnp_ctx* ctx, int* cfg);

/* Ensemble of independent cases (no counterpart in the paper: the data-parallel
 * axis of a parameter sweep, e.g. over wall potential and Debye length on
 * uneven grids).  Each case is a distinct context with its own workspace,
 * parameters and state.  pnp_ensemble_step advances every case by nsteps
 * steps of its own dt[i] with ONE CUDA graph launch per step on `stream` (a
 * non-default stream): the graph forks each case onto a private branch stream
 * of the ensemble so that the cases' kernels overlap.  Work issued afterwards
 * on a case's own stream is ordered after the ensemble's steps.  Each case's
 * arithmetic is exactly that of pnp_step on the case alone (bitwise equal).
 * The ensemble borrows the contexts; destroy it before them. */
typedef struct pnp_ensemble pnp_ensemble;
int pnp_ensemble_create(pnp_ensemble** out, pnp_ctx* const* cases, int ncases, void* cuda_stream);
int pnp_ensemble_step(pnp_ensemble* ens, int nsteps, const double* dt);
void pnp_ensemble_destroy(pnp_ensemble* ens);

/* ---- Learned electric-double-layer wall model (no counterpart in the paper) ----
 * A coarse y-grid cannot resolve the Debye layer; a small network maps
 * near-wall columns of the coarse state to wall slip velocities (and reports
 * the potential offset and ion fluxes next to the wall).  Coarse grid: every
 * ry-th y-face of a fine grid, Nx_c = Nx_f / rx, Nz_c = Nz_f / rz.  Rows are
 * wall columns [wall][z][x] (bottom first), in the wall frame: the top wall
 * is mapped onto the bottom by (x, y) -> (-x, -y) with c+ <-> c-, Phi -> -Phi;
 * streamwise velocities are relative to the wall.
 * Features (5 * ncells per row): [u_rel | w | c_counter | c_co | phi] for the
 * ncells cells nearest the wall, phi = Phi - V y.
 * Outputs / labels (5 per row): 0 / 1 the filtered fine wall shear rates
 * d(u_rel)/dy and dw/dy, 2 phi of the first coarse cell, 3 / 4 total counter-
 * / co-ion flux away from the wall through the first interior coarse face.
 * Network: 40 -> 128 -> 128 -> 128 -> 128 -> 5, erf-GELU on hidden layers; every
 * GEMM (forward, data gradient, weight gradient) on the tensor cores with BF16
 * operands (weights, activations, output gradients) and FP32 accumulation;
 * FP32 master weights, Adam; loss = mean squared error of normalised outputs. */
typedef struct pnp_mlp pnp_mlp;
int pnp_mlp_param_count(size_t* out_count);
/* Device workspace for a network that processes up to max_batch rows. */
int pnp_mlp_workspace_bytes(int max_batch, size_t* out_bytes);
/* Weights U(-a, a), a = sqrt(6 / fan_in), from SplitMix64(seed); biases 0. */
int pnp_mlp_create(pnp_mlp** out, int max_batch, void* device_workspace, size_t bytes, void* cuda_stream,
                   uint64_t seed);
int pnp_mlp_get_params(pnp_mlp* mlp, float* host_params, size_t count);
/* Replace the FP32 master parameters (layer by layer: W [out][in] then b [out])
 * and reset the Adam moments. */
int pnp_mlp_set_params(pnp_mlp* mlp, const float* host_params, size_t count);
/* Input x_n = (x - in_shift) * in_scale (40 each), output y = y_n / out_scale +
 * out_shift (5 each); host arrays. */
int pnp_mlp_set_normalization(pnp_mlp* mlp, const float* in_shift, const float* in_scale, const float* out_shift,
                              const float* out_scale);
/* Residual output: output out_col becomes the network's value plus the raw
 * input column in_col, y_o = n_o / out_scale_o + out_shift_o + x_i, so that the
 * network learns y_o - x_i (the output normalisation of column o then applies to
 * that difference, and the training loss compares the network with t_o - x_i).
 * out_col < 0 removes it (the default).  PNP_ERR_ARG for out_col >= 5, in_col >=
 * 40, or in_col < 0 with out_col >= 0.  Host state only; takes effect from the
 * next call. */
int pnp_mlp_set_skip(pnp_mlp* mlp, int out_col, int in_col);
/* Y[B][5] = network(X[B][40]); device arrays; asynchronous.  Normalised
 * outputs are clipped to +-6 (six standard deviations of the training labels
 * when the normalisation is set from them). */
int pnp_mlp_forward(pnp_mlp* mlp, const float* X_dev, int B, float* Y_dev);
/* Gradient of the loss against targets T[B][5] w.r.t. the parameters (host
 * copy, optional) and the loss (host, optional); synchronises. */
int pnp_mlp_gradient(pnp_mlp* mlp, const float* X_dev, const float* T_dev, int B, float* grad_host, float* loss_host);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at learning rate lr. */
int pnp_mlp_train_step(pnp_mlp* mlp, const float* X_dev, const float* T_dev, int B, float lr, float* loss_host);
/* Device status of the network's kernels: PNP_OK, or PNP_ERR_TIMEOUT when a
 * bounded wait for the tensor cores ran out (sticky); synchronises. */
int pnp_mlp_status(pnp_mlp* mlp);
void pnp_mlp_destroy(pnp_mlp* mlp);

/* Feature rows of a context's state: X[2 Nz Nx][5 ncells] (ncells <= 8).  With
 * the wall model's potential offsets in place (pnp_set_wallmodel_edl), the
 * potential column leaves out their charge-free lift: it is the potential the
 * present ions give between the uniform walls -V, +V, the same quantity the
 * network sees when it is trained on uncoupled runs. */
int pnp_wall_features(pnp_ctx* ctx, int ncells, float* X_dev);
/* Coarse state := volume-weighted restriction of the fine state (u, v, w, p,
 * c+-, Phi); the coarse stored explicit terms are zeroed. */
int pnp_restrict_state(pnp_ctx* fine, pnp_ctx* coarse);
/* Labels T[2 Nz_c Nx_c][5] of the coarse wall columns from the fine state. */
int pnp_wall_labels(pnp_ctx* fine, pnp_ctx* coarse, float* T_dev);
/* Wall slip velocities that impose the wall shear rates predicted in Y[2 Nz
 * Nx][5] (columns 0 and 1): s = q_0 - h_0 g with q_0 the first-cell value in
 * the feature rows X (ncells per field, as from pnp_wall_features) and h_0 the
 * wall-to-centre distance; a non-finite slip or one above ten wall speeds
 * falls back to no slip.  Y = NULL restores the uniform wall speeds.
 * pnp_diagnostics then reports the wall shear against the plane-mean wall
 * velocity. */
int pnp_set_wall_slip(pnp_ctx* ctx, const float* X_dev, int ncells, const float* Y_dev);
/* The same wall values as a prescribed wall stress: the explicit terms see the
 * wall flux nu g the slip implies, and the wall-normal implicit solves of u
 * and w drop their wall coupling (zero-flux rows), so the near-wall cells are
 * not pulled towards the slip value within a step. */
int pnp_set_wall_stress(pnp_ctx* ctx, const float* X_dev, int ncells, const float* Y_dev);
/* How pnp_step_wallmodel couples the network to the solver: mode 0 = wall slip
 * (pnp_set_wall_slip), 1 = wall stress (pnp_set_wall_stress), 2 = wall stress
 * from the plane means of the predicted rates (one rate per wall), 3 = no wall
 * shear from the network (the solver's no-slip walls; for coarse grids that
 * still resolve the viscous sublayer, with the double-layer coupling of
 * pnp_set_wallmodel_edl); relax in (0, 1]:
 * the wall-shear rates used each step move that fraction of the way from the
 * previous step's to the new prediction (1 = no relaxation). */
int pnp_set_wallmodel_coupling(pnp_ctx* ctx, int mode, double relax);
/* Double-layer coupling of pnp_step_wallmodel, beside the wall shear (the
 * network's columns 2-4; no counterpart in the paper, which resolves the layer).
 * potential_gain in [0, 1]: before each step the wall potentials move by
 * potential_gain (phi_pred - phi_1) per wall column, phi_1 the first cell's
 * potential perturbation Phi - V y_c and phi_pred the one the network predicts
 * from features that leave the offsets' own lift out (so that a fixed point
 * exists: the prediction does not move with the offsets), as offsets
 * on top of the uniform walls -V, +V (within +-max(1, |V|)), and the potential
 * of the present ions is solved again under them.  flux_gain in [0, 1]: after
 * each step, ions move across the first interior face of each wall column so
 * that the face's total flux F = v c_f - D (dc/dy + s c_f dPhi/dy) moves that
 * fraction of the way to the predicted one over dt; conservative per column, a
 * cell gives at most half its ions.  0 switches a part off; potential_gain 0
 * also removes the offsets (the uniform walls return and the potential is
 * solved again).  PNP_ERR_UNSUPPORTED from a coupled step when a wall-potential
 * map of pnp_set_wall_potential is set. */
int pnp_set_wallmodel_edl(pnp_ctx* ctx, double potential_gain, double flux_gain);
/* One potential-offset update from device feature rows X [2 Nz Nx][5 ncells]
 * (as pnp_wall_features gives them: without the offsets' lift, which the update
 * adds back to compare the prediction with the first cell's present potential)
 * and outputs Y [2 Nz Nx][5] (the step pnp_step_wallmodel takes before each
 * step; needs potential_gain > 0).  Stream-ordered on the context's stream. */
int pnp_set_wall_edl(pnp_ctx* ctx, const float* X_dev, int ncells, const float* Y_dev);
/* One ion-flux transfer over dt from device outputs Y [2 Nz Nx][5] (the step
 * pnp_step_wallmodel takes after each step; needs flux_gain > 0 and Nyc >= 4,
 * so that the two walls' cell pairs are disjoint; PNP_ERR_ARG otherwise). */
int pnp_correct_wall_flux(pnp_ctx* ctx, const float* Y_dev, double dt);
/* nsteps steps of the coarse solver with the wall model: before each step,
 * features (8 cells) -> network -> (relaxed) wall rates -> wall slip or stress
 * [-> wall-potential offsets]; after it [-> ion-flux transfer]. */
int pnp_step_wallmodel(pnp_ctx* ctx, pnp_mlp* mlp, int nsteps, double dt);

/* Launch sites timed by pnp_profile, in launch order within a substage. */
enum {
  PNP_SITE_RHS = 0,         /* explicit terms + CN right-hand sides            */
  PNP_SITE_CN = 1,          /* wall-normal CN Thomas solves                    */
  PNP_SITE_P_FFTX = 2,      /* divergence + forward real x-FFT                 */
  PNP_SITE_P_FFTZ = 3,      /* forward z-FFT                                   */
  PNP_SITE_P_THOMAS = 4,    /* spectral Thomas, Neumann                        */
  PNP_SITE_P_IFFTZ = 5,     /* inverse z-FFT                                   */
  PNP_SITE_P_IFFTX = 6,     /* inverse real x-FFT -> Phi_p                     */
  PNP_SITE_PROJECT = 7,     /* projection + pressure update                    */
  PNP_SITE_E_FFTX = 8,      /* charge + forward real x-FFT                     */
  PNP_SITE_E_FFTZ = 9,
  PNP_SITE_E_THOMAS = 10,   /* spectral Thomas, Dirichlet                      */
  PNP_SITE_E_IFFTZ = 11,
  PNP_SITE_E_IFFTX = 12,    /* inverse real x-FFT -> Phi = V y + phi           */
  PNP_PROFILE_SITES = 13
};

/* Advance nsteps steps without a CUDA graph, timing every launch site with
 * CUDA events on the context's stream.  ms_out[site] receives the summed
 * milliseconds over all 3*nsteps substages (nsites >= PNP_PROFILE_SITES);
 * *launches_per_step the number of kernels one step launches, counted from a
 * capture of the step's CUDA graph (-1 when the context has no stream). */
int pnp_profile(pnp_ctx* ctx, int nsteps, double dt, double* ms_out, int nsites, int* launches_per_step);

/* Trace of one step (no counterpart in the paper; a tracing aid): runs one
 * full RK3 step of size dt in the step's own concurrent schedule (two
 * streams), with a timing event after every launch site on the stream that
 * ran it: launched eagerly (in_graph = 0), or captured with the events as
 * event-record nodes into one CUDA graph and launched once (in_graph != 0;
 * needs a context stream), which times the step as pnp_step runs it.  For each event i < *n_out (at most cap; about 15 per
 * substage): site_out[i] = its PNP_SITE_* (-1: the start of a substage),
 * stream_out[i] = 0 for the context's stream, 1 for the auxiliary stream,
 * t_ms_out[i] = milliseconds since the first event.  The wall-normal CN solve
 * appears twice per mixed substage (ions on the auxiliary stream, velocities
 * on the main one).  Advances the state by one step; synchronises. */
int pnp_timeline(pnp_ctx* ctx, double dt, int in_graph, int cap, int* site_out, int* stream_out,
                 double* t_ms_out, int* n_out);

const char* pnp_error_string(int code);

void pnp_destroy(pnp_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* PNP_H */
