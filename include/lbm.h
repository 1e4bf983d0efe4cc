/*
 * lbm.h -- C ABI of the GB300 library for the ternary "2f1s" phase-field
 * lattice Boltzmann method of Zhan, Chai and Shi, "A ternary phase-field model
 * for two-phase flows in complex geometries" (arXiv 2311.05091).
 *
 * Model.  Phase 0 is a frozen, diffuse solid (indicator phi0), phase 1 the
 * droplet / driving fluid (phi1, the only evolved order parameter), phase 2
 * the other fluid, phi2 = 1 - phi0 - phi1 (Sec. 2.2, Remarks 1-3).  Each time
 * step (Sec. 2 and Sec. 3):
 *   1. phi1 = sum_i f_i over the Cahn-Hilliard (CH) populations;
 *   2. isotropic central stencils give grad / Laplacian of phi0, phi1;
 *   3. chemical potentials mu_p = df_b/dphi_p - (3D/4) gamma_p lap phi_p and
 *      mubar_1 = gamma_T/3 sum_{q != 1} (mu_1 - mu_q)/gamma_q (Sec. 2.1);
 *   4. grad mubar_1, degenerate mobility, mass flux S, surface-tension force
 *      F_s = sum mu_p grad phi_p, correction force F_c = div(S u - u S)/2,
 *      body force, solid penalisation force (Sec. 2.3, Sec. 3);
 *   5. Hermite-moment collision of the CH populations f (Sec. 3, Sec. 4 intro);
 *   6. Hermite-moment collision of the Navier-Stokes (NS) populations g with
 *      the pressure formulation and second-order force moment M^2F;
 *   7. streaming with half-way bounce-back on non-periodic axes.
 * The spreading coefficients follow Young's law with s01 = k s12 and the
 * closure k(theta, kappa) of Eq. kk (Sec. 2.2).
 *
 * Lattice units: dx = dt = c = 1, cs^2 = d0 (scale factor).
 *
 * Layout.  Every field is float32, structure of arrays, x fastest:
 *   scalar field   [b][z][y][x]            (b = instance of a batch)
 *   vector field   [b][a][z][y][x]         (a = x, y[, z] component)
 *   populations    [b][i][z][y][x]         (i = lattice direction)
 * 2D lattices have nz = 1.  D2Q9 directions follow the paper's printed M0:
 *   0 (0,0) 1 (1,0) 2 (0,1) 3 (-1,0) 4 (0,-1) 5 (1,1) 6 (-1,1) 7 (-1,-1) 8 (1,-1).
 * D3Q19 directions: 0 rest; 1..6 (+x,-x,+y,-y,+z,-z); 7..18 edges
 *   (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1) (1,0,-1) (-1,0,1)
 *   (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1).
 * D3Q15 directions (the paper's printed M0): 0 rest; 1..6 as D3Q19; 7..14
 *   corners (1,1,1) (-1,1,1) (1,-1,1) (-1,-1,1) (1,1,-1) (-1,1,-1) (1,-1,-1)
 *   (-1,-1,-1).  Both 3D lattices use the D3Q19 isotropic stencil for
 *   gradients and Laplacians; a D3Q19 / D3Q15 step is two launches (moment
 *   pass, fused kernel).
 *
 * Ownership.  A context owns all of its device memory (allocated in
 * lbm_create*, freed in lbm_destroy).  Host pointers passed in are read or
 * written during the call only and never kept.  Device pointers passed to
 * the *_device calls must stay valid until the work enqueued by that call
 * has completed on the context's stream.
 *
 * Streams.  Every device operation is enqueued on the context's stream
 * (lbm_set_stream; by default a stream the context creates).  Calls that
 * return host data synchronise that stream.
 *
 * Errors.  Every call returns an lbm_status and never aborts the process.
 * Invalid arguments give LBM_EINVAL and leave the context unchanged.  A
 * failed CUDA call gives LBM_ECUDA; the context is then marked failed and
 * every later call except lbm_destroy and lbm_last_error returns LBM_ESTATE.
 * Asynchronous failures and divergence (NaN or |u| > 0.5 found by the step
 * that closes each lbm_step call) surface at the next synchronising call
 * (lbm_sync, lbm_get_*, lbm_observables) as LBM_ECUDA / LBM_EDIVERGED; a
 * bounded device wait for an asynchronous tile load that gave up surfaces
 * there as LBM_ETIMEOUT (the step it belonged to is incomplete).
 */
#ifndef LBM_H_
#define LBM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = -1,      /* invalid argument                                  */
  LBM_ENOMEM = -2,      /* device or host allocation failed                  */
  LBM_ECUDA = -3,       /* a CUDA runtime call failed                        */
  LBM_EDIVERGED = -4,   /* NaN or |u| > 0.5 detected                          */
  LBM_ETIMEOUT = -5,    /* a bounded device wait gave up                     */
  LBM_ESTATE = -6,      /* context not initialised, or failed earlier        */
  LBM_EUNSUPPORTED = -7 /* lattice / option not built                        */
} lbm_status;

typedef enum {
  LBM_D2Q9 = 0,   /* 2D, Appendix A weights and matrices                     */
  LBM_D3Q19 = 1,  /* 3D, weights from the same moment conditions (d0 < 1/2)  */
  LBM_D3Q15 = 2   /* 3D, Appendix A weights and matrices (d0 < 1/2)          */
} lbm_lattice;

/* Periodicity bit mask; a clear bit means half-way bounce-back walls (no-flux
 * for phi1, no-slip for u) half a spacing outside the first and last node. */
enum { LBM_PERIODIC_X = 1, LBM_PERIODIC_Y = 2, LBM_PERIODIC_Z = 4 };

/* Physical and numerical parameters of one instance (lattice units). */
typedef struct {
  double W;             /* interface thickness D (Sec. 2.1), > 0                     */
  double M_deg;         /* degenerate mobility coefficient (Sec. 2.2), >= 0         */
  double M_cst;         /* constant mobility part, >= 0, M_cst + M_deg > 0          */
  double theta_deg;     /* contact angle of fluid 1 on the solid, in (0, 180)       */
  double kappa;         /* minimum dimensionless solid curvature (Eq. kk), > -1      */
  double sigma;         /* fluid-fluid tension sigma_12, > 0                        */
  double rho[3];        /* densities of solid, fluid 1, fluid 2, > 0                */
  double mu[3];         /* dynamic viscosities of solid, fluid 1, fluid 2, > 0      */
  double d0;            /* scale factor cs^2 = d0: (0,1) for D2Q9, (0,1/2) in 3D    */
  double eta_hat;       /* CH parameter eta_1 = eta_hat / gamma_1, > 0 (0.1)        */
  double s_free_ch;     /* CH rates s0, s2a, s2b, s3, s4, in (0,2) (1)              */
  double s_free_ns;     /* NS rates s1, s3, in (0,2) (1)                            */
  double body_force[3]; /* body-force density b; F_b = (1 - phi0) b                 */
} lbm_params;

/* Diagnostics of one instance, computed from the fields of the last step
 * (time t-1 after t steps): sums in float64 (Sec. 4.2-4.3 diagnostics). */
typedef struct {
  double mass1;      /* sum of phi1                                          */
  double mass0;      /* sum of phi0                                          */
  double umax;       /* max |u|                                              */
  double p_in;       /* mean pressure where phi1 >= 0.99                      */
  double p_out;      /* mean pressure where phi2 >= 0.99                      */
  double dp;         /* p_in - p_out (Laplace pressure)                      */
  int64_t n_in;      /* nodes in the p_in set                                 */
  int64_t n_out;     /* nodes in the p_out set                                */
  int64_t step;      /* completed steps                                       */
} lbm_obs;

/* Fill *p with the defaults: W 4, M_deg 0.1, M_cst 0, theta 90, kappa 0,
 * sigma 0.01, rho 1, mu 0.01, d0 0.5 (Appendix A), eta_hat 0.1, free rates 1,
 * no body force.  Returns LBM_EINVAL if p is NULL. */
int lbm_default_params(lbm_params* p);

/* What the library derives from one parameter set, in float64 before the
 * kernels round it to float32 (the paper has no counterpart: a diagnostic of
 * the host derivation of Sec. 2.2, Sec. 3 and Appendix A). */
typedef struct {
  double k;          /* wetting closure k(theta, kappa) of Eq. kk                 */
  double gamma[3];   /* spreading coefficients gamma_0 (solid), gamma_1, gamma_2  */
  double gamma_T;    /* 3 / (1/gamma_0 + 1/gamma_1 + 1/gamma_2)                    */
  double eta;        /* eta_1 = eta_hat / gamma_1                                  */
  double s1_ch;      /* CH first-moment rate 1 / (1/2 + M / (gamma_1 eta_1 cs2))  */
  double cs2;        /* squared sound speed: d0 rounded to float32, as the kernels */
  double w[3];       /* weights: rest, axis, and diagonal (D2Q9), edge (D3Q19) or
                        corner (D3Q15), all from cs2                               */
  double visc[2];    /* kinematic viscosity nu = (1/s - 1/2) visc[i], s = s2a (i = 0)
                        or s2b (i = 1) of the NS collision                        */
  double p_f, p_w;   /* pressure formula prefactor cs2 / (1 - w0) and w0 / (1 - cs2) */
  double p_K;        /* K of the pressure formula                                 */
  double p_h[3];     /* H = K (p_h[0] / s0 - p_h[1] / s2a + p_h[2])               */
} lbm_derived;

/* Fill *out with the constants a context created with `params` on `lattice`
 * would use.  Host only (no context, no device call).  LBM_EINVAL, with the
 * reason in lbm_last_error(NULL), for a NULL pointer, an unknown lattice or
 * parameters lbm_create would reject. */
int lbm_derive(lbm_lattice lattice, const lbm_params* params, lbm_derived* out);

/* Create a context for one lattice of nx * ny * nz nodes (nz = 1 for D2Q9).
 * Derives k, gamma_p, gamma_T, eta_1 and the CH rate s1 from *p (Sec. 2.2,
 * Sec. 3) on the host in float64 and allocates the device state.  Axes
 * without their LBM_PERIODIC_* bit need at least 2 nodes.  On success *out
 * holds the context; the state is not initialised until lbm_set_phase. */
int lbm_create(lbm_lattice lattice, int nx, int ny, int nz, int periodic_mask,
               const lbm_params* p, lbm_ctx** out);

/* Same, for nbatch independent instances of the same size advanced together
 * by one launch per step; params points to nbatch parameter sets. */
int lbm_create_batch(lbm_lattice lattice, int nx, int ny, int nz, int periodic_mask,
                     int nbatch, const lbm_params* params, lbm_ctx** out);

/* Storage options of lbm_create_ex. */
enum {
  /* NS populations g stored in HBM as IEEE FP16 holding g * 2^12 (the rest
   * population already shifted by rho_0), arithmetic in float32; the CH
   * populations stay float32, so the conserved phase field keeps float32
   * rounding.  Every lattice, nx % 8 == 0 (LBM_EINVAL otherwise).  Relative
   * storage error 2^-11 per value per step; no pattern of the paper, a
   * bandwidth option: bytes per lattice update 188 -> 152 (D2Q9),
   * 364 -> 288 (D3Q19), 300 -> 240 (D3Q15). */
  LBM_STORE_G_F16 = 1
};

/* lbm_create_batch with storage options (0 or LBM_STORE_G_F16). */
int lbm_create_ex(lbm_lattice lattice, int nx, int ny, int nz, int periodic_mask,
                  int nbatch, const lbm_params* params, int flags, lbm_ctx** out);

/* Device-memory callbacks for lbm_create_alloc: alloc returns a device
 * pointer to `bytes` bytes usable on `stream` (NULL on failure, which the
 * creating call reports as LBM_ENOMEM); free takes back a pointer alloc
 * returned, with its size and the context's stream.  `user` is passed
 * through.  Both are called from the thread that makes the library call. */
typedef void* (*lbm_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*lbm_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

/* lbm_create_ex whose device buffers come from the caller's allocator (for
 * example a framework's caching allocator, so that the simulation's memory is
 * accounted and reused with the caller's) and whose work runs on the caller's
 * stream (cudaStream_t; NULL: the library creates its own, as lbm_create).
 * alloc and free: both or neither (neither: cudaMalloc / cudaFree).  Every
 * device allocation of the context goes through alloc (populations, history,
 * fields, scratch of the diagnostics, the autotuner's save area, the inlet
 * profile); before handing memory back through free the library waits for
 * the context's stream, so the caller may reuse it on any stream at once. */
int lbm_create_alloc(lbm_lattice lattice, int nx, int ny, int nz, int periodic_mask, int nbatch,
                     const lbm_params* params, int flags, void* stream, lbm_alloc_fn alloc, lbm_free_fn free_fn,
                     void* user, lbm_ctx** out);

/* ninst independent D2Q9 instances of different sizes nx[k] x ny[k] (same
 * periodicity), advanced together by one persistent launch per step that
 * walks a work list of (instance, 128-column tile, row strip) items; no
 * pattern of the paper, a throughput form for many small geometries.
 * Layout: instance k occupies a contiguous block of each buffer starting at
 * node offset off_k = sum_{j<k} nx_j ny_j (lbm_get_instance_shape); fields
 * passed to lbm_set_solid / lbm_set_phase / lbm_get_fields are the
 * instances' blocks back to back (u: [k][a][y][x]).  Every other call works
 * as for a batch, with instance-local shapes; lbm_get_shape reports nx = ny
 * = 0.  Each instance's result is bitwise that of a single-instance context.
 * D2Q9 only (LBM_EUNSUPPORTED otherwise); flags as lbm_create_ex. */
int lbm_create_multi(lbm_lattice lattice, int ninst, const int* nx, const int* ny,
                     int periodic_mask, const lbm_params* params, int flags, lbm_ctx** out);

/* Shape and node offset of one instance (any context). */
int lbm_get_instance_shape(const lbm_ctx* ctx, int instance, int* nx, int* ny, int64_t* offset);

/* Launch autotuner: chooses the row strip (of every size class of a
 * multi-size context, or the context's single strip) among 4, 8, 12, 16, 18,
 * 20, 24, 32, 48, 64 by timing `trial` steps per candidate, two
 * coordinate-descent passes.  The
 * evolving state is saved before and restored after (bitwise), so the call can
 * come at any point after lbm_set_phase.  strips_out (nbatch ints, may be
 * NULL) receives the chosen strip of each instance. */
int lbm_tune(lbm_ctx* ctx, int trial, int* strips_out);

/* Free all device memory of the context.  Safe on NULL. */
void lbm_destroy(lbm_ctx* ctx);

/* Enqueue all later work on `stream` (a cudaStream_t, may be NULL for the
 * legacy default stream, which disables CUDA-graph replay).  The caller keeps
 * ownership of the stream and must keep it alive while the context uses it. */
int lbm_set_stream(lbm_ctx* ctx, void* stream);

/* Launch tuning; results do not depend on it (bitwise).  strip >= 1: rows
 * (D2Q9) or z planes (D3Q19) swept by one CTA of the step kernel; by default
 * 16 rows or 32 planes, or, when that gives fewer CTAs than two waves on the
 * device, the shorter strip a wave model picks.  depth in
 * 1..3 (0 keeps the current value): D2Q9, rows of asynchronous
 * global-to-shared copies each CTA keeps in flight (default 1); D3Q19, 1
 * selects the generic fused kernel (synchronous halo loads), 2 or 3 the
 * pipelined one (TMA tile loads of the owned columns, asynchronous halo
 * copies one plane ahead; default 2), which needs nx % 4 == 0 and otherwise
 * falls back to the generic kernel. */
int lbm_set_launch(lbm_ctx* ctx, int strip, int depth);

/* Poll limit of the bounded device waits (the paper has no counterpart; a
 * failure-detection service).  The pipelined 3D kernel waits on an mbarrier
 * for the TMA tile load of each z plane; after `polls` unsuccessful polls
 * it stops the step, drains the load still in flight (at the default
 * limit), and sets a flag that the next synchronising call reports as
 * LBM_ETIMEOUT; the context stays usable and its state must be set again
 * (lbm_set_phase or lbm_set_state) before it is trusted.  polls < 0
 * restores the default (2^22); polls = 0 makes every such wait give up at
 * once, which is how tests inject the failure without faulting the GPU.
 * Synchronises the context's stream; applies to later steps. */
int lbm_set_wait_limit(lbm_ctx* ctx, int polls);

/* Kernel timing.  While enabled, every time step is bracketed by CUDA
 * events recorded on the context's stream, with one more between the D3Q19
 * moment pass and the fused kernel (CUDA-graph replay is off meanwhile).
 * lbm_kernel_time synchronises, returns the summed device duration (ms) and
 * the number of steps timed since the last read, and starts a new count.
 * Outputs may be NULL. */
int lbm_set_profiling(lbm_ctx* ctx, int enable);
int lbm_kernel_time(lbm_ctx* ctx, double* total_ms, int64_t* launches);

/* Same timing split per kernel: part_ms[0] the D3Q19 moment pass (0 for
 * D2Q9), part_ms[1] the fused step kernel, summed over the *steps timed
 * steps; also starts a new count.  part_ms points to 2 doubles or is NULL. */
int lbm_kernel_time_split(lbm_ctx* ctx, double* part_ms, int64_t* steps);

/* Copy the solid indicator phi0 (host, nbatch*nz*ny*nx floats) to the device. */
int lbm_set_solid(lbm_ctx* ctx, const float* phi0_host);
int lbm_set_solid_device(lbm_ctx* ctx, const float* phi0_dev);

/* Copy the initial phi1 (host, same size), then initialise every node at
 * equilibrium: f = f^eq(phi1, mubar_1(phi1), u = 0), g = g^eq(p = 0, u = 0),
 * history (phi1, u = 0, S = 0); resets the step count.  Requires lbm_set_solid. */
int lbm_set_phase(lbm_ctx* ctx, const float* phi1_host);
int lbm_set_phase_device(lbm_ctx* ctx, const float* phi1_dev);

/* Velocity inlet at the first x column and pressure outlet at the last one,
 * by the non-equilibrium extrapolation the paper names for velocity and
 * pressure boundaries (Sec. 4 intro, the scheme of Guo, Zheng and Shi).
 * After every step the populations f and g of a boundary node become those
 * of its neighbouring column plus the difference of the equilibria at the
 * boundary state and at the neighbour's state.  Neighbour state: phi1 = sum
 * f, u = sum c g / rho, p from the local part of the pressure formula
 * (p = cs2/(1 - w0) (sum_{i != 0} g_i - w0 rho |u|^2 / (1 - cs2))).
 * mode bit 0: inlet at x = 0 with velocity u_in ([d][nz][ny] floats, host,
 * copied; |u| < 0.5) and phase field phi_in (phi_in < 0: taken from the
 * neighbour); bit 1: outlet at x = nx - 1 with pressure p_out, velocity and
 * phase field taken from the neighbour.  mode 0 turns both off (the columns
 * are half-way bounce-back walls again).  Needs a non-periodic x axis and
 * nx >= 4; every instance of a batch shares the settings; not for
 * lbm_create_multi contexts (LBM_EUNSUPPORTED). */
int lbm_set_inout(lbm_ctx* ctx, int mode, const float* u_in, double phi_in, double p_out);

/* Enqueue n >= 0 coupled time steps (D2Q9: one fused kernel per step;
 * D3Q19: a moment pass, phi1 = sum f and j = sum c f, then one fused kernel;
 * replayed from a captured CUDA graph where the stream allows).  Returns once
 * the work is enqueued.  The last step also writes the pressure field and
 * checks for divergence. */
int lbm_step(lbm_ctx* ctx, int n);

/* Wait for the context's stream; report deferred errors. */
int lbm_sync(lbm_ctx* ctx);

/* Macroscopic fields of the last step (time t-1): phi1 (scalar), u (vector,
 * d components), p (scalar); host buffers, any may be NULL.  Synchronous. */
int lbm_get_fields(lbm_ctx* ctx, float* phi1, float* u, float* p);

/* Current populations f (CH) and g (NS), host buffers of nbatch*Q*nodes
 * floats.  The rest population g_0 is stored minus the constant rho_0 of the
 * pressure equilibrium (lambda_0, Sec. 3), which the dynamics do not depend
 * on.  With LBM_STORE_G_F16, g is converted back to float32 (unscaled).
 * Either pointer may be NULL.  Synchronous. */
int lbm_get_populations(lbm_ctx* ctx, float* f, float* g);

/* Checkpoint: the whole evolving state (populations, history, step count) as
 * a byte image: a 64-byte header (uint32 magic "LBM1", int32 lattice, nx, ny,
 * nz, nbatch, q, d, int64 step, int64 nodes, int32 g storage (0 float32, 1
 * FP16 scaled by 2^12), 12 bytes padding) followed by float32 f [b][i][nodes],
 * g [b][i][nodes] in its storage type (g_0 minus rho_0) and the float32
 * history [b][k][nodes] with k = phi1, u (d components), S (d components) of
 * the last step.  With buf == NULL, *bytes receives the size.  lbm_set_state restores
 * an image taken from a context of the same shape; a run continued after
 * restore is bitwise identical. */
int lbm_get_state(lbm_ctx* ctx, void* buf, size_t* bytes);
int lbm_set_state(lbm_ctx* ctx, const void* buf, size_t bytes);

/* Reductions of instance `instance` (float64 accumulation, deterministic
 * two-pass tree over warp-shuffle partials).  Synchronous. */
int lbm_observables(lbm_ctx* ctx, int instance, lbm_obs* out);

/* Allocation-free diagnostics, for callers that cannot allocate device memory
 * when they need these numbers: a solver embedded in an application that owns
 * all device memory through its own pool, a latency-bound loop in which
 * cudaMalloc would synchronise the device, or a caller out of memory budget.
 * The paper has no counterpart; this is a service of the library.
 *
 * Same sums as lbm_observables, computed from caller-owned device buffers of
 * one instance: phi0, phi1, p (n floats each), u (d planes of n floats, d in
 * 1..3).  out: device buffer of 8 doubles receiving sum phi1, sum phi0,
 * max |u|, sum p over phi1 >= 0.99, that node count, sum p over phi2 >= 0.99,
 * that node count, number of non-finite nodes.  The work is enqueued on
 * `stream` (a cudaStream_t, NULL for the legacy stream); read `out` after
 * synchronising it.  No device memory is allocated or freed: the partial sums
 * live in a fixed 1 MiB array inside the library (one record per 1024 nodes),
 * resident on every device that loads the library until exit, so n is at most
 * 16,777,216; larger n, n < 1, NULL buffers or a bad d give LBM_EINVAL before
 * any launch.  The first call on each device looks the array's device address
 * up (cudaGetSymbolAddress); make it before capturing a stream.  Every call
 * shares the array and it keeps the previous call's contents (nothing needs
 * clearing: each call overwrites the records it reads); calls whose kernels
 * overlap on the GPU race on it.  The buffers and the stream must belong to
 * the calling thread's current device, whose array the call uses; devices of
 * ordinal 64 and above are not served (LBM_ECUDA).  The looked-up address is
 * kept for the life of the process, so do not call this on a device after
 * cudaDeviceReset.  LBM_ECUDA if the look-up or a launch fails, or if the
 * device already holds an error from earlier work when the call starts (that
 * error is left in place for cudaGetLastError). */
int lbm_observables_noalloc(const float* phi0, const float* phi1, const float* u, int d, const float* p,
                            long long n, double* out, void* stream);

/* Pore-space phase fluxes for the relative permeability (Sec. 4.6, Eq. eq-Kp):
 * over the nodes with phi0 <= 1/2 of instance `instance`, q1 = sum phi1 u_a,
 * q2 = sum phi2 u_a (phi2 = 1 - phi0 - phi1), q = sum u_a for the velocity
 * component a = axis, n_pore the node count and s1, s2 the saturations
 * sum phi_p / sum (phi1 + phi2).  The relative permeability of fluid p is
 * K_p = q_p (two-phase run) / q (single-phase run of fluid p in the same
 * medium under the same driving).  Synchronous, float64 sums in a fixed
 * order; uses the fields of the last step (as lbm_get_fields). */
typedef struct {
  double q1, q2, q;
  double s1, s2;
  int64_t n_pore;
} lbm_flux;
int lbm_phase_flux(lbm_ctx* ctx, int instance, int axis, lbm_flux* out);

/* Contact angle of instance `instance` from the droplet height on the
 * vertical grid column x = column (2D).  mode 0: flat bottom wall, H measured
 * from the phi0 = 1/2 level on that column, R0 = sqrt(2 A / pi) from the area
 * A = sum phi1, theta solves H/R0 = (1 - cos t) sqrt((pi/2)/(t - sin t cos t))
 * (Sec. 4.2).  mode 1: disk of radius disk_radius centred at (column, y_c):
 * H_max above the centre and the drop area solve the two-circle relation of
 * Sec. 4.3.  Outputs may be NULL.  Synchronous. */
int lbm_contact_angle(lbm_ctx* ctx, int instance, int mode, int column, double y_c,
                      double disk_radius, double* theta_deg, double* height);

/* Sizes. */
int lbm_get_shape(const lbm_ctx* ctx, int* nx, int* ny, int* nz, int* nbatch, int* q);

/* Message for a status code (static string). */
const char* lbm_strerror(int status);

/* Text of the last error raised on this context (static per context). */
const char* lbm_last_error(const lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H_ */
