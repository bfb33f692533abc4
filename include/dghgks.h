/*
 * dghgks.h -- C ABI of the DG-HGKS per-stage residual on one NVIDIA B300.
 *
 * The method is the discontinuous-Galerkin high-order gas-kinetic scheme of
 * arXiv:2202.13821 for the 3D Euler and Navier-Stokes equations:
 *   - Sec. 2, Eq. (flux): second-order gas-kinetic interface flux from the
 *     BGK integral solution, with collision time tau = mu/p (Sec. 3 Remark 1);
 *   - Sec. 3, Eq. (flux-2): simplified interior flux f = g0(1 - tau(a.u+A) + At);
 *   - Sec. 3, Eqs. (expansion), (operator), (surface), (volume): P_k Legendre
 *     modal DG residual R(Q_h), diagonal mass matrix, L = M^-1 R;
 *   - Sec. 3, Eq. (expansion-1): F and d_t F from the time integrals of the
 *     flux over [0, dt] and [0, dt/2];
 *   - Sec. 3, Eq. (two-stage): the two-stage fourth-order (S2O4) step.
 *
 * Conventions shared by every call
 *   State layout: Q[var][mode][z][y][x], float64, contiguous, on the device
 *   unless the name ends in _host.  var = (rho, rho U, rho V, rho W, rho E)
 *   with rho E = p/(gamma-1) + rho|U|^2/2.  Modes of P_k by total degree,
 *   pure powers first: (000) (100)(010)(001) (200)(020)(002)(110)(101)(011).
 *   Mode n of a cell is the coefficient of P_nx(xi) P_ny(eta) P_nz(zeta) with
 *   xi = 2 (x - x_i) / dx.  N_m = (k+1)(k+2)(k+3)/6 modes.
 *   Ownership: the caller owns every state/output buffer.  The library owns
 *   its scratch (stage buffers, face moments, reduction partials), allocated
 *   in dghgks_init and freed in dghgks_destroy.
 *   Streams: `stream` is a cudaStream_t passed as void* (NULL = default
 *   stream).  Calls enqueue work and return without synchronising, except
 *   those documented as synchronising.
 *   Errors: 0 on success, negative otherwise; dghgks_last_error() gives text.
 *     DGHGKS_EARG    (-1) bad argument (NULL pointer, size, dt <= 0)
 *     DGHGKS_EUNSUP  (-2) unsupported order / Gauss count / boundary
 *     DGHGKS_ECUDA   (-3) CUDA error
 *     DGHGKS_EPHYS   (-4) non-physical state met (rho <= 0 or p <= 0); the
 *                         kernels set a device flag, read by dghgks_status()
 *                         and by the synchronising calls; no trap
 *     DGHGKS_ENOMEM  (-5) device allocation failed
 */
#ifndef DGHGKS_H
#define DGHGKS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DGHGKS_OK 0
#define DGHGKS_EARG (-1)
#define DGHGKS_EUNSUP (-2)
#define DGHGKS_ECUDA (-3)
#define DGHGKS_EPHYS (-4)
#define DGHGKS_ENOMEM (-5)
#define DGHGKS_ESCRATCH (-6) /* problem too large for dghgks_residual_static's fixed scratch */

#define DGHGKS_FP64 0       /* flux and quadrature arithmetic in FP64 */
/* FP32-mixed: flux, quadrature, projection sums, the face-moment assembly,
 * M^-1 and the stage increments in FP32; the stored state, its update and
 * the reductions in FP64 */
#define DGHGKS_FP32_MIXED 1
/* FP32 flux, quadrature, projection sums and their assembly with the face
 * moments (as DGHGKS_FP32_MIXED; the cell averages' face terms summed exactly,
 * so that the conserved totals hold to FP64 rounding); M^-1 and the S2O4 stage
 * combination (Q*, the stage increment, the state update) in FP64, with the
 * stage increment stored in FP64 and Q* stored rounded to FP32 (its only
 * reader is the FP32 flux arithmetic of stage 2) */
#define DGHGKS_FP32_STAGE64 2

typedef struct dghgks_ctx dghgks_ctx;

/* Cartesian hexahedral mesh K_ijk = [x_{i-1/2}, x_{i+1/2}] x ... (Sec. 3).
 * nx, ny, nz >= 1 cells; only periodic boundaries are supported
 * (periodic[d] must be 1).
 * nodes[d] == NULL: uniform cells of width (hi[d] - lo[d]) / n_d along axis d.
 * nodes[d] != NULL: host array of the n_d + 1 strictly increasing node
 * coordinates x_{1/2} .. x_{n_d+1/2} of axis d (a rectilinear, non-uniform
 * mesh such as the mapped grid x = xi + 0.05 sin(pi xi) of Sec. 5.1);
 * lo[d] and hi[d] are then ignored.  dghgks_init copies the nodes (the
 * caller keeps ownership); non-increasing or non-finite nodes give
 * DGHGKS_EARG.  Fields must be zero-initialised (NULL nodes) by callers that
 * want the uniform mesh. */
typedef struct {
  int nx, ny, nz;
  double lo[3], hi[3];
  int periodic[3];
  const double* nodes[3];
} dghgks_mesh;

/* n_q: Gauss points per direction (faces n_q^2, cells n_q^3); 0 = order+1.
 * precision: DGHGKS_FP64, DGHGKS_FP32_MIXED or DGHGKS_FP32_STAGE64.
 * tau_eps: tau = mu/p + tau_eps*dt (0 = the paper's tau = mu/p). */
typedef struct {
  int n_q;
  int precision;
  double tau_eps;
} dghgks_opts;

/* Create a solver for P_order elements (order 1 with n_q = 2; order 2 with
 * n_q = 2 or 3; order 3 with n_q = 3 or 4) on `mesh`, for a gas with ratio of specific heats gamma, viscosity
 * mu >= 0 and Prandtl number Pr > 0 (Pr = 1 is the BGK value used by the
 * paper; Pr != 1 adds (1/Pr - 1) times the heat flux of the same distribution
 * to the energy flux F at t_n, not to its time derivative F_t, which the
 * paper does not define).  opts may be NULL
 * (n_q = order+1, FP64, tau_eps = 0).  Uses the current CUDA device.
 * Allocates the scratch: 2 stage buffers with the state's values in the flux
 * precision (Q* and the stage increment; the increment in FP64 with
 * DGHGKS_FP32_STAGE64), on FP32 contexts also the FP32 state copy, plus the
 * face moments (3 * 10 * (k+1)(k+2)/2 values per cell in the flux precision). */
int dghgks_init(const dghgks_mesh* mesh, int order, double gamma, double mu, double Pr, const dghgks_opts* opts,
                dghgks_ctx** out);

/* Destroy a context and free its scratch.  NULL is ignored. */
void dghgks_destroy(dghgks_ctx* ctx);

/* Text of the last error of this context (or of a failed init if ctx is NULL). */
const char* dghgks_last_error(const dghgks_ctx* ctx);

/* Number of modal coefficients per cell and variable, N_m. */
int dghgks_n_modes(const dghgks_ctx* ctx);

/* Change the viscosity mu (>= 0) used by later calls. */
int dghgks_set_mu(dghgks_ctx* ctx, double mu);

/* One residual evaluation (Sec. 3, Eqs. operator/surface/volume with the
 * fluxes of Eqs. flux and flux-2 fitted over [0, dt] and [0, dt/2]):
 *   L = M^-1 R(Q), Lt = M^-1 R_t(Q).
 * Q, L, Lt: device, state layout; L and Lt must not alias Q.  Asynchronous. */
int dghgks_residual(dghgks_ctx* ctx, const double* Q, double dt, double* L, double* Lt, void* stream);

/* One S2O4 step (Sec. 3, Eq. two-stage), in place on the device state Q:
 *   Q* = Q + dt/2 L(Q) + dt^2/8 L_t(Q)
 *   Q <- Q + dt L(Q) + dt^2/6 (L_t(Q) + 2 L_t(Q*)).
 * On an FP32 context (DGHGKS_FP32_MIXED or DGHGKS_FP32_STAGE64) the stage-1
 * kernels read Q rounded to FP32 (one extra elementwise launch rounds it into
 * a library buffer).
 * Asynchronous; consecutive calls on one context must share a stream. */
int dghgks_step(dghgks_ctx* ctx, double* Q, double dt, void* stream);

/* nsteps S2O4 steps in place on the device state Q, replaying CUDA graphs
 * of one step (8 kernel launches) on `stream`.  The graphs are captured on a
 * private stream at the first call and re-captured when Q, dt or the
 * viscosity (dghgks_set_mu) changes (the executable graph is updated in
 * place when possible).  On an FP32 context the stage-1 kernels read the
 * state rounded to FP32 in a library buffer: the first step of a call rounds Q
 * into it, and every step's state update writes it for the next step (a
 * second graph); Q may therefore change between calls but not during one.
 * Results are identical to nsteps calls of dghgks_step.  Asynchronous.  Must not be
 * called while `stream` itself is being captured.  With profiling on
 * (dghgks_profile) the same launches are enqueued directly, each recorded,
 * instead of replaying the graphs. */
int dghgks_steps(dghgks_ctx* ctx, double* Q, double dt, int nsteps, void* stream);

/* nsteps S2O4 steps on a HOST state (pinned or pageable): copies Q_host to
 * the device, steps (with the FP32 state copy between steps, as
 * dghgks_steps), and copies the result back; if ek_host is not NULL it
 * receives E_k (as dghgks_kinetic_energy with rho0) after every step (host
 * memory, nsteps doubles).  The E_k of step n runs on a second, library-owned
 * stream beside step n+1, whose state update waits for it; results are
 * bitwise those of dghgks_step + dghgks_kinetic_energy.  Synchronises.
 * Allocates one device state buffer (and the second stream) on first use. */
int dghgks_run_host(dghgks_ctx* ctx, double* Q_host, double dt, int nsteps, double rho0, double* ek_host,
                    void* stream);

/* Conserved totals sum_cells |K| Q_(var, mode 0), var = 0..4, in FP64
 * (|K| per cell on a rectilinear mesh).
 * Synchronises; out is host memory (5 doubles). */
int dghgks_totals(dghgks_ctx* ctx, const double* Q, double* out, void* stream);

/* Volume-averaged kinetic energy E_k = 1/(rho0 |Omega|) int rho|U|^2/2
 * (Sec. 5.3), by the n_q^3 cell Gauss rule, in FP64 (point values by sum
 * factorisation; 1/rho from an FP32 estimate and two Newton steps, exact to
 * FP64 rounding).  Synchronises; Ek is host memory. */
int dghgks_kinetic_energy(dghgks_ctx* ctx, const double* Q, double rho0, double* Ek, void* stream);

/* Enstrophy-based dissipation rate (Sec. 5.3):
 *   eps(zeta) = 2 mu / (rho0 |Omega|) int rho |omega|^2 / 2,  omega = curl U,
 * with the context's mu, by the n_q^3 cell Gauss rule, in FP64.
 * Synchronises; eps is host memory. */
int dghgks_enstrophy_dissipation(dghgks_ctx* ctx, const double* Q, double rho0, double* eps, void* stream);

/* L2 norm over the domain of the difference of two modal states, variable
 * var, in FP64 (orthogonal basis: sum_cells sum_n M_nn (A_n - B_n)^2).
 * Synchronises; out is host memory. */
int dghgks_l2_diff(dghgks_ctx* ctx, const double* A, const double* B, int var, double* out, void* stream);

/* Synchronise `stream` and report the device error flag: DGHGKS_EPHYS if a
 * non-physical state was met since the last check (the flag is then
 * cleared), DGHGKS_ECUDA on a CUDA error or if a cell kernel gave up a
 * shared-memory barrier wait (bounded at 2 s; its results are then invalid),
 * else 0. */
int dghgks_status(dghgks_ctx* ctx, void* stream);

/* ---- adjoint (reverse mode, FP64 contexts only; the paper has none) ----
 * The vector-Jacobian products below are exact to rounding: the point-flux
 * Jacobian transposes are a hand-written reverse mode of the flux code (one
 * backward sweep per Gauss point), the projection and trace operators are
 * transposed exactly.  Uniform and rectilinear meshes.  They allocate
 * adjoint scratch on first use (face cotangents 3 x 2 x 5 N_m doubles per
 * cell, a state-sized buffer, per-CTA partials).  Every order and Gauss
 * count of dghgks_init; FP32 contexts return DGHGKS_EUNSUP. */

/* (lamQ, dmu) = (dL/dQ, dL/dmu)^T lamL + (dL_t/dQ, dL_t/dmu)^T lamLt at Q for
 * the residual of dghgks_residual with the same dt.  lamQ (device, state
 * layout) is overwritten; the viscosity cotangent is ADDED to the device
 * scalar *dmu.  Asynchronous. */
int dghgks_residual_vjp(dghgks_ctx* ctx, const double* Q, double dt, const double* lamL, const double* lamLt,
                        double* lamQ, double* dmu, void* stream);

/* Adjoint of one S2O4 step (Eq. two-stage) from the checkpoint Q^n:
 * lam_n = (dQ^{n+1}/dQ^n)^T lam_next, and (dQ^{n+1}/dmu)^T lam_next is ADDED to
 * the device scalar *dJ_dmu.  Q* is recomputed from Q^n (one forward stage);
 * then the stage-2 VJP at Q* with cotangent (0, dt^2/3 lam) gives lam*, and
 * the stage-1 VJP at Q^n with (dt lam + dt/2 lam*, dt^2/6 lam + dt^2/8 lam*)
 * gives the rest: lam_n = lam + lam* + VJP.  lam_n may alias lam_next.
 * Asynchronous. */
int dghgks_adjoint_step(dghgks_ctx* ctx, const double* Qn, const double* lam_next, double dt, double* lam_n,
                        double* dJ_dmu, void* stream);

/* Gradient of dghgks_kinetic_energy with respect to Q (device, state layout,
 * overwritten).  Works on any context (FP64 arithmetic).  Asynchronous. */
int dghgks_kinetic_energy_vjp(dghgks_ctx* ctx, const double* Q, double rho0, double* dEk_dQ, void* stream);

/* Per-kernel timing with CUDA events recorded on the launching stream around
 * every launch of this context.  enable = 1 starts (and clears) the record,
 * 0 stops it.  Kernel kinds: 0..2 face flux for normals x, y, z; 3 cell
 * kernel of a residual; 4 cell kernel of stage 1; 5 cell kernel of stage 2;
 * 6 reductions.  dghgks_profile_read synchronises and returns, per kind,
 * the summed milliseconds and the number of launches (arrays of length
 * DGHGKS_NKINDS, host memory).  At most 65536 launches are recorded. */
#define DGHGKS_NKINDS 7
int dghgks_profile(dghgks_ctx* ctx, int enable);
int dghgks_profile_read(dghgks_ctx* ctx, double* ms, int64_t* launches);

/* Kernel launches made by this context since creation (all entry points). */
int64_t dghgks_launch_count(const dghgks_ctx* ctx);

/* One residual evaluation (as dghgks_residual) that allocates no memory and
 * needs no context.  The paper has no counterpart: this is an interface for
 * callers that cannot call cudaMalloc/cudaFree when they need a residual --
 * code running inside another framework's memory plan (a caching allocator
 * that owns the free device memory, a budget fixed at start-up), real-time or
 * embedded loops that forbid allocation after initialisation, and code that
 * must not trigger the device-wide synchronisation of cudaFree.
 * Arguments are those of dghgks_init plus those of dghgks_residual; the caller
 * passes Q, L, Lt (device, state layout, distinct buffers).  Supported: uniform
 * periodic meshes (nodes all NULL), order 1 with n_q = 2 and order 2 with
 * n_q = 2 or 3, precision DGHGKS_FP64 or DGHGKS_FP32_MIXED.  A rectilinear mesh
 * (any nodes[d] != NULL), order 3 or another n_q return DGHGKS_EUNSUP, and
 * DGHGKS_FP32_STAGE64 returns DGHGKS_EARG, all before any GPU work.
 * Scratch: the face moments live in one file-scope __device__ array of
 * DGHGKS_STATIC_SCRATCH_BYTES (16 MiB), which every GPU that loads the library
 * holds until the process exits; problems needing more
 * (bytes = 30 * (k+1)(k+2)/2 * cells * (8 for FP64, 4 for FP32-mixed); e.g.
 * P2 FP64 up to 11650 cells) are rejected with DGHGKS_ESCRATCH before any GPU
 * work.  The first call on each device (with that device current) looks up
 * the array's device address and sets kernel attributes; make that first call
 * before any stream capture.  All calls share the array and a device flag,
 * which keep the last call's contents (the flag is cleared at each call), so
 * calls that overlap on the GPU -- concurrent streams, host threads or devices
 * sharing nothing else -- race: serialise them.  Synchronises `stream`;
 * returns 0, DGHGKS_EARG, DGHGKS_EUNSUP, DGHGKS_ESCRATCH, DGHGKS_ECUDA, or
 * DGHGKS_EPHYS if a non-physical state was met (no error text is kept). */
#define DGHGKS_STATIC_SCRATCH_BYTES (16u << 20)
int dghgks_residual_static(const dghgks_mesh* mesh, int order, double gamma, double mu, double Pr,
                           const dghgks_opts* opts, const double* Q, double dt, double* L, double* Lt, void* stream);

/* Measured arithmetic throughput of the current GPU, for the roofline of the
 * (ALU-bound) residual kernels; the paper has no counterpart.  out[0..6]
 * (host memory, n_out >= DGHGKS_NRATES): FP32 FMA FLOP/s (2 FLOP per FFMA),
 * FP64 FMA FLOP/s, then operations/s of the FP32 flux's approximate division,
 * reciprocal square root and exponential and of erfcf (each loop iteration is
 * the operation plus one FP32 add), and the SM count.  Each rate is the best
 * of three launches of about 10-20 ms filling every SM.  Allocates and frees
 * a small device buffer; synchronises the device; returns 0, DGHGKS_EARG,
 * DGHGKS_ENOMEM or DGHGKS_ECUDA. */
#define DGHGKS_NRATES 7
int dghgks_pipe_rates(double* out, int n_out);

/* Gauss-Legendre rule used on the device: nodes x[n] ascending on [-1,1],
 * weights w[n] normalised to sum 1 (n = 1..5).  Host-only, no GPU needed. */
int dghgks_gauss_rule(int n, double* x, double* w);

#ifdef __cplusplus
}
#endif

#endif /* DGHGKS_H */
