/*
 * fdtd.h -- C ABI of libfdtd: leapfrog FDTD on the staggered Yee grid with the
 * extended, coefficient-parameterised curl-E stencil of Blinne et al.,
 * "A Systematic Approach to Numerical Dispersion in Maxwell Solvers"
 * (arXiv:1710.06829), its adjoint, and the paper's dispersion norm.
 *
 * Units: c = 1, mu0 = eps0 = 1.
 *
 * Grid and staggering (App. A, update equations).  Field arrays are dense
 * [nz][ny][nx] (x fastest).  Integer index (i,j,k) of each component denotes
 *     E_x (i+1/2, j, k)    B_x (i, j+1/2, k+1/2)
 *     E_y (i, j+1/2, k)    B_y (i+1/2, j, k+1/2)
 *     E_z (i, j, k+1/2)    B_z (i+1/2, j+1/2, k)
 * All axes are periodic.  A field array set is always ordered
 * {E_x, E_y, E_z, B_x, B_y, B_z}.
 *
 * Coefficients (Sec. 2, Eq. D*): beta[i][j] is beta_ij (taps of D*_i displaced
 * along axis j; the diagonal is ignored), delta[i] is delta_i.  alpha_i is
 * never passed: it is eliminated with Eq. (alpha),
 *     alpha_i = 1 - 2 sum_{j != i} beta_ij - 3 delta_i.
 * With dims < 3 every coefficient that refers to an absent axis is ignored.
 *
 * Memory: the library owns the simulation state (two padded copies of the six
 * fields, ping-ponged by the fused step kernel), the adjoint state, the
 * recorded E history and the checkpoint slots, all in device memory it
 * allocates with cudaMalloc.  Caller buffers are only read or written during
 * the call that receives them (asynchronously on the handle's stream).
 *
 * Errors: every entry point returns an int status (FDTD_OK = 0, negative on
 * failure) and sets a thread-local message readable with fdtd_last_error().
 * Argument and stability errors are detected synchronously; CUDA errors are
 * reported by the call that observes them.
 */
#ifndef FDTD_H
#define FDTD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define FDTD_OK          0
#define FDTD_EINVAL     -1   /* bad argument, shape or layout */
#define FDTD_EUNSTABLE  -2   /* coefficients/dt violate Eq. (constraints) */
#define FDTD_ECUDA      -3   /* a CUDA runtime or driver call failed */
#define FDTD_ENOMEM     -4   /* device allocation failed */
#define FDTD_ENONFINITE -5   /* a non-finite value was found */
#define FDTD_ESTATE     -6   /* call not valid in the handle's current state */
#define FDTD_ETIMEOUT   -7   /* a bounded wait inside a kernel expired (reported by fdtd_sync) */

/* dtypes */
#define FDTD_F32 0
#define FDTD_F64 1

/* where caller buffers live */
#define FDTD_MEM_DEVICE 0
#define FDTD_MEM_HOST   1

/* sources */
#define FDTD_SRC_NONE  0
#define FDTD_SRC_BUNCH 1
#define FDTD_SRC_DENSE 2

/* dispersion-norm weights (Sec. 4 and Eq. norm_x_axis) */
#define FDTD_W_UNIFORM 0   /* w = 1 */
#define FDTD_W_CONE_X  1   /* w = 1 inside a cone of half-angle `param` (rad) about +x, else 0 */
#define FDTD_W_GAUSS_Y 2   /* w = exp(-(k_y dy / param)^2) */

typedef struct fdtd_handle fdtd_handle;

typedef struct {
    int32_t dims;          /* 1, 2 or 3: axes that carry wave propagation */
    int32_t nx, ny, nz;    /* cells; nx % 4 == 0; dims 2 needs nz == 1 (unless batched),
                              dims 1 needs ny == nz == 1 */
    int32_t dtype;         /* FDTD_F32 or FDTD_F64: precision of fields and stepping */
    int32_t absorb_cells;  /* width L of absorbing sponge layers on +-y and +-z (0 = none) */
    double  absorb_sigma;  /* sponge strength: fields scaled by 1 - sigma (d/L)^3, d = 1..L */
    int32_t batched;       /* dims == 2 only: 1 = the nz planes are nz independent 2D problems
                              (no coupling along z; sponge on +-y only; no bunch source) */
} fdtd_grid;

typedef struct {
    double beta[3][3];
    double delta[3];
} fdtd_coeffs;

/* Current J^{n+1/2} in Ampere's law (App. A update equations).
 * FDTD_SRC_BUNCH: a rigid Gaussian charge moving along +x (stand-in for a PIC beam); its
 *   J_x^{n+1/2} is evaluated inside the E update from the cell-integrated Gaussian so that
 *   the discrete continuity equation of App. A holds exactly.  Uses q .. sigma_perp.
 * FDTD_SRC_DENSE: a current given on the grid: J[a] is a device array, dense [nz][ny][nx], of
 *   the handle's dtype holding J_a at the E_a positions (NULL = 0), borrowed for the call and
 *   applied in every step of it (one call per step for a current that changes in time).  The
 *   step forms E^{n+1} without the current and subtracts dt J (times the sponge factor) from
 *   it, which Ampere's law's linearity in J makes the same update. */
typedef struct {
    int32_t kind;          /* FDTD_SRC_NONE, FDTD_SRC_BUNCH or FDTD_SRC_DENSE */
    double q, v;           /* bunch: charge, speed (units of c) */
    double x0, y0, z0;     /* bunch: centre at absolute step 0 (length units) */
    double sigma_par, sigma_perp;
    const void* J[3];      /* dense: J_x, J_y, J_z (device) */
} fdtd_source;

/* Probe: squared misfit of one E component on the plane i = x_index against a
 * target, summed over all probed steps (the propagation loss of the
 * differentiable path). */
typedef struct {
    int32_t component;     /* 0, 1, 2 -> E_x, E_y, E_z */
    int32_t x_index;       /* plane i = x_index */
    const void* target;    /* device, grid dtype, [target_steps][nz][ny]; row s-1 is the target
                              at absolute step s (after s leapfrog steps) */
    int64_t target_steps;
} fdtd_probe;

/* ---- handle ------------------------------------------------------------- */

/* Create a simulation.  dx[3] > 0; dt > 0.  Validates Eq. (constraints):
 * returns FDTD_EUNSTABLE if dt^2 max_k S(k) > 1 or min_k S(k) < 0.
 * `stream` is a cudaStream_t (NULL = legacy default stream).  The initial
 * state is all zero.  The handle is returned in *out. */
int fdtd_create(const fdtd_grid* grid, const double dx[3], double dt, const fdtd_coeffs* coeffs,
                void* stream, fdtd_handle** out);

/* Replace coefficients and dt (re-validated as in fdtd_create). */
int fdtd_set_coeffs(fdtd_handle* h, double dt, const fdtd_coeffs* coeffs);

/* Copy the six fields in (set) or out (get).  fields[c] points to nx*ny*nz
 * elements of the grid dtype in `mem` (FDTD_MEM_DEVICE or FDTD_MEM_HOST).
 * For set_state a NULL entry means zero.  Host buffers may be pageable; the
 * call returns after the host copy has completed.  set_state also resets the
 * step counter to `step0`. */
int fdtd_set_state(fdtd_handle* h, void* const fields[6], int32_t mem, int64_t step0);
int fdtd_get_state(fdtd_handle* h, void* const fields[6], int32_t mem);

/* Absolute step counter (number of leapfrog steps taken since set_state's step0). */
int fdtd_get_step(fdtd_handle* h, int64_t* step);

/* Advance n >= 0 leapfrog steps (App. A update equations):
 *   B^{n+1/2} = B^{n-1/2} - dt D* x E^n            (extended stencil, Eq. D*)
 *   E^{n+1}   = E^n + dt (D x B^{n+1/2} - J^{n+1/2}) (Yee stencil)
 * `src` may be NULL (no current).  If `probe` is non-NULL, after every step s
 * the probe misfit sum_{j,k} (E_c^s[x_index, j, k] - T^s[j,k])^2 is added in
 * FP64 to *loss_dev (one device double).  If `record` is non-zero, E^n before
 * each step and E after the last one are stored in the handle's history
 * (n + 1 snapshots, replacing any earlier history) for fdtd_step_adjoint.
 * The step kernels check every E value they write: a non-finite value (the fields
 * blew up, or the state or the current held an infinity or NaN; a non-finite B
 * reaches E in the same step) makes the next fdtd_sync return FDTD_ENONFINITE. */
int fdtd_step(fdtd_handle* h, int32_t n, const fdtd_source* src, const fdtd_probe* probe,
              double* loss_dev, int32_t record);

/* Checkpoint slots: op 0 = save the current state (fields + step counter) to
 * `slot`, op 1 = restore it.  Slots are allocated on first save. */
int fdtd_checkpoint(fdtd_handle* h, int32_t slot, int32_t op);

/* Adjoint state lambda = (lambda_E, lambda_B), same layout as the fields.
 * set with NULL entries = zero. */
int fdtd_set_adjoint(fdtd_handle* h, void* const fields[6], int32_t mem);
int fdtd_get_adjoint(fdtd_handle* h, void* const fields[6], int32_t mem);

/* Run n reverse steps of the transposed leapfrog map over the recorded
 * history (which must hold >= n steps; the last n recorded steps are used,
 * newest first).  Before reversing the step that produced E^s, the probe
 * source 2 (E_c^s - T^s) is added to lambda_E on the probe plane (if probe is
 * non-NULL).  Adds dt * sum_cells lambda_B^{s+1/2} . (dF/dtheta) E^s to
 * grad_dev (12 device doubles: beta[3][3] row-major, then delta[3]; the
 * diagonal entries stay unchanged), where F E = -D* x E.  The sponge is
 * applied as its own transpose.  On return the history is consumed.
 * FP32 handles whose grid the TMA tiles fit (nx a multiple of 64, ny of 8) run one kernel
 * per reverse step, out of place: the library then holds two adjoint sets (12 padded arrays,
 * allocated with the first adjoint call) and alternates between them; fdtd_get_adjoint always
 * reads the current one.  Setting FDTD_ADJOINT_SPLIT=1 in the environment before
 * fdtd_create selects the two-kernel in-place step instead (same lambda bitwise). */
int fdtd_step_adjoint(fdtd_handle* h, int32_t n, const fdtd_probe* probe, double* grad_dev);

/* Diagnostics on the current state, FP64 accumulation, result in device memory
 * (asynchronous on the handle's stream):
 *   FDTD_DIAG_ENERGY:    params = {x_lo, x_len, margin}; out_dev[0] = (1/2) sum (E^2 + B^2) dV
 *                        over cells with i in the periodic window [x_lo, x_lo + x_len) and
 *                        margin <= j < ny - margin (and margin <= k < nz - margin when z is a
 *                        spatial axis) -- field energy, e.g. the radiation behind a moving
 *                        bunch (Sec. 6).
 *   FDTD_DIAG_PLANEWAVE: params = {component 0..5, k_x, k_y, k_z}; out_dev[0..1] = Re, Im of
 *                        sum_cells F exp(-i k . r) with r the component's staggered position
 *                        (App. A); its phase advance per step measures the scheme's omega(k)
 *                        of Eq. (dispersion_relation), Sec. 3.
 *   FDTD_DIAG_MOMENTS:   params = {axis 0..2}; out_dev[0..2] = (W, C, S) = sum over the six
 *                        components and all cells of (1/2) F^2 dV (1, cos th, sin th), with
 *                        th = 2 pi (index_a + o) / n_a and o = 1/2 for components staggered
 *                        along the axis (App. A).  atan2(S, C) n_a dx_a / (2 pi) is the
 *                        periodic (circular-mean) energy centroid of a wave packet; its
 *                        speed is the packet's group velocity (Sec. 5).               */
#define FDTD_DIAG_ENERGY    0
#define FDTD_DIAG_PLANEWAVE 1
#define FDTD_DIAG_MOMENTS   2
int fdtd_diagnostic(fdtd_handle* h, int32_t kind, const double* params, double* out_dev);

/* Divergences of the current state, FP64, dense [nz][ny][nx] into out_dev (device):
 *   FDTD_DIV_STAR_B: D* . B with the extended stencil (Eq. divstarb), conserved by the
 *                    scheme for any coefficients (Sec. 2.1);
 *   FDTD_DIV_YEE_B:  Yee D . B, conserved only under Eq. (beta) (Sec. 2.2);
 *   FDTD_DIV_E:      Yee D . E at the nodes (Eq. divE; equals rho_E of App. A).        */
#define FDTD_DIV_STAR_B 0
#define FDTD_DIV_YEE_B  1
#define FDTD_DIV_E      2
int fdtd_divergence(fdtd_handle* h, int32_t which, double* out_dev);

/* ---- macro-particles (PIC coupling) -------------------------------------
 *
 * The paper keeps Yee's stencil in Ampere's law so that a charge-conserving current
 * weighting makes the discrete continuity equation D_t rho + D . J = 0 hold (App. A,
 * numerical continuity equation, after Esirkepov); Gauss's law D . E = rho (Eq. divE)
 * is then kept from step to step.  Its particle runs (Sec. 6) use relativistic electron
 * bunches.  The library's particle coupling (the shape and the pusher are readings; the
 * paper names neither):
 *   shape     first order: node i of axis a carries max(0, 1 - |x_a / dx_a - i|);
 *   rho       at the nodes (i, j, k), sum_p q S_i S_j S_k / (dx dy dz);
 *   gather    every field component from its own staggered positions (table above)
 *             with the same shape; B^n = (B^{n-1/2} + B^{n+1/2}) / 2;
 *   push      Boris's relativistic scheme in u = gamma v (c = 1);
 *   current   Esirkepov's decomposition of the shape change, J_a at the E_a positions.
 *
 * A species: n macro-particles of charge q and charge-to-mass ratio q_over_m.  x[a] and
 * u[a] (a = x, y, z) are device arrays of n values in the handle's dtype (float for
 * FDTD_F32, double for FDTD_F64), structure of arrays, borrowed for the call and updated
 * in place: positions in the units of dx (any finite value; they are wrapped into
 * [0, n_a dx_a) by the step), u = gamma v.  A particle whose position or momentum is not
 * finite is left unchanged, deposits nothing, and makes the next fdtd_sync return
 * FDTD_ENONFINITE. */
typedef struct {
    void* x[3];
    void* u[3];
    int64_t n;
    double q;
    double q_over_m;
} fdtd_species;

/* Advance n >= 0 PIC cycles of the current state and the nspecies species:
 *   B^{n+1/2} = B^{n-1/2} - dt D* x E^n                        (extended stencil, Eq. D*)
 *   per particle: gather E^n, B^n at x^n; Boris u^{n-1/2} -> u^{n+1/2};
 *                 x^{n+1} = x^n + dt u^{n+1/2} / gamma^{n+1/2}; Esirkepov J^{n+1/2}
 *   E^{n+1}   = E^n + dt (D x B^{n+1/2} - J^{n+1/2})           (Yee stencil)
 * The grid must be 3D (dims = 3) and not batched: FDTD_EINVAL otherwise.  With an absorbing
 * layer the sponge factor multiplies B after the Faraday half and E after the Ampere half,
 * as in fdtd_step (Gauss's law then holds outside the layer only); particles inside it are
 * pushed as anywhere else.  Ampere's law is linear in J: the step forms E^{n+1} without the
 * current and the particles add -dt J^{n+1/2} into it with floating-point reductions (summed
 * over a warp first when its 32 particles share their cells), so the summation order, and
 * the last bits of E, may differ between runs.
 * The recorded history of fdtd_step is dropped (a PIC cycle has no adjoint here). */
int fdtd_pic_step(fdtd_handle* h, int32_t n, const fdtd_species* species, int32_t nspecies);

/* Add the charge density of the species at the nodes (first-order shape) to rho_dev:
 * dense [nz][ny][nx] device array of the handle's dtype (the caller zeroes it).  With
 * fdtd_divergence(FDTD_DIV_E) this checks Gauss's law D . E = rho (Eq. divE). */
int fdtd_deposit_rho(fdtd_handle* h, const fdtd_species* species, int32_t nspecies,
                     void* rho_dev);

/* Failure-path self-test (no counterpart in the paper): launches, on the handle's stream, one
 * thread that polls an mbarrier phase nothing will complete, with the same bounded-wait helper
 * the TMA step kernels use, limited to `tries` polls (1 .. 2^20).  When the polls run out it
 * raises the handle's error flag as an expired wait in a step kernel does, so the next
 * fdtd_sync returns FDTD_ETIMEOUT (and clears the flag).  Nothing faults, traps or hangs; the
 * handle stays usable.  Returns FDTD_EINVAL for tries outside the range. */
int fdtd_selftest_wait_expiry(fdtd_handle* h, int32_t tries);

/* Temporal blocking of the FP32 fused step (the multi-step blocking named as the next
 * throughput lever for a memory-bound stencil; the paper itself describes no kernel).  With
 * T = 2, fdtd_step advances pairs of leapfrog steps (App. A update equations, unchanged
 * arithmetic: the fields are bitwise equal to T = 1) slab by slab along z: step n+1 of slab
 * s+1, then step n+2 of slab s, so that the intermediate state (E^{n+1}, B^{n+1/2}) is read
 * back from L2 while it is still resident, and the intermediate planes no later launch needs
 * are dropped from L2 without being written to DRAM.  slab_planes (>= 3; 0 = 32) sets the slab
 * length.  Applies to FP32 grids on the fused path (nx % 64 == 0, ny % 8 == 0) with at least
 * two slabs, and to fdtd_step calls without a source, probe or history; other calls, and an
 * odd last step, run one launch per step.  T = 1 (the default) restores one launch per step.
 * Returns FDTD_EINVAL for other T or slab_planes in 1 .. 2. */
int fdtd_set_temporal_blocking(fdtd_handle* h, int32_t T, int32_t slab_planes);

/* Block until all work on the handle's stream has finished; reports any
 * asynchronous CUDA error, FDTD_ETIMEOUT when a bounded wait inside a kernel
 * expired since the last call, and FDTD_ENONFINITE when a step wrote a
 * non-finite field value or met a non-finite particle since the last call.  The
 * flags are cleared once reported. */
int fdtd_sync(fdtd_handle* h);

void fdtd_destroy(fdtd_handle* h);

/* ---- dispersion analysis (no handle) ------------------------------------ */

/* Eq. (norm) by the midpoint rule on an N[0] x N[1] (x N[2]) grid over the
 * positive octant 0 < k_i < pi/dx_i (axes beyond dims are absent), with
 * omega(k) from Eq. (dispersion_relation), and its exact gradient.
 * out (host, 14 doubles): [0] norm, [1..9] d/d beta (3x3 row-major, diagonal
 * 0), [10..12] d/d delta, [13] d/d dt.  Accumulation is FP64 on the GPU;
 * per-point arithmetic is FP64.  Runs on `stream` and synchronises it. */
int disp_norm_eval(const fdtd_coeffs* coeffs, double dt, const double dx[3], int32_t dims,
                   const int32_t N[3], int32_t weight, double weight_param, double* out,
                   void* stream);

/* Group-velocity norm: the conclusions (Sec. 7) propose minimising the numerical group velocity
 * error but give no formula; this library's reading uses the grid, weights and quadrature of
 * Eq. (norm) with |d omega/dk| - c in place of omega - c|k|:
 *     f_g = prod(dx) sum_points w (|grad_k omega| - 1)^2 prod(pi / (N_i dx_i)),
 * grad_k omega = omega'(S) grad_k S from Eq. (dispersion_relation) (c = 1).
 * Arguments, weights, limits, errors and synchronisation as disp_norm_eval; out (host, 14
 * doubles) in the same layout: [0] f_g, [1..9] d/d beta, [10..12] d/d delta, [13] d/d dt.
 * Allocates its scratch on `stream` (stream-ordered) and frees it before returning. */
int disp_group_norm_eval(const fdtd_coeffs* coeffs, double dt, const double dx[3], int32_t dims,
                         const int32_t N[3], int32_t weight, double weight_param, double* out,
                         void* stream);

/* omega(k) of Eq. (dispersion_relation), omega = (2/dt) asin(dt sqrt(sum_i s_i^2 A_i)), at n
 * wave vectors (k_dev: device, n x 3 doubles, row-major; axes beyond dims ignored) into
 * omega_dev (device, n doubles).  FP64.  Validates Eq. (constraints) like disp_norm_eval.
 * Phase velocity is omega/|k| (Sec. 5); asynchronous on `stream`. */
int disp_omega_eval(const fdtd_coeffs* coeffs, double dt, const double dx[3], int32_t dims,
                    const double* k_dev, int32_t n, double* omega_dev, void* stream);

/* disp_norm_eval without any device allocation.  The paper has no counterpart:
 * this is a library service for callers that may not allocate device memory
 * when they need the norm (for instance while another stream of the device is
 * being captured into a CUDA graph, or under a host that owns every byte of the
 * GPU through its own pool).  Same arguments, results and synchronisation as
 * disp_norm_eval; the kernels work in a scratch area the library declares
 * statically on each device (512 KiB, kept until the process exits).
 * Limit: N[i] <= 4096 on every used axis, else FDTD_EINVAL (use disp_norm_eval).
 * The first call on a device (with that device current) looks the area's
 * address up; make it before any stream capture.  The address is looked up again
 * after the device's context changes (for instance after cudaDeviceReset), which
 * makes that call a set-up call too.  All calls share the one area, so calls that
 * overlap on the GPU (different streams, no ordering) race; calls ordered on one
 * stream are safe.  The area needs no clearing: every entry is written before it
 * is read within a call. */
int disp_norm_eval_noalloc(const fdtd_coeffs* coeffs, double dt, const double dx[3],
                           int32_t dims, const int32_t N[3], int32_t weight, double weight_param,
                           double* out, void* stream);

/* One step of the constrained coefficient minimisation (Sec. 4; projected gradient descent
 * in FP64 on the GPU instead of SLSQP).  The n <= 16 free parameters theta map linearly
 * onto the 13 scheme parameters c = (beta 3x3 row-major, delta 3, dt) as c = c0 + T^T theta
 * (T: n x 13 row-major, host; the tying of Sec. 4, e.g. beta_xy = beta_yx).  With grad13 the
 * gradient of the objective in c (the layout of disp_norm_eval's out[1..13]):
 *     theta' = clip(theta - eta T grad13, lo, hi),   c' = c0 + T^T theta'.
 * theta, grad13, T, c0, lo, hi are host arrays; out_dev is a caller-owned device buffer of
 * n + 13 doubles receiving (theta', c').  Asynchronous on `stream`.  Eq. (constraints) is not
 * checked here: the caller validates c' (fdtd_dt_max or disp_norm_eval) and backtracks. */
int fdtd_coeff_update(int32_t n, const double* theta, const double* grad13, const double* T,
                      const double* c0, double eta, const double* lo, const double* hi,
                      double* out_dev, void* stream);

/* Exact extremes of S(k) = sum_i s_i^2 A_i over the Brillouin box (host, FP64)
 * and dt_max = 1/sqrt(max S), the CFL limit of Eq. (constraints). */
int fdtd_dt_max(const fdtd_coeffs* coeffs, const double dx[3], int32_t dims, double* dt_max,
                double* s_min, double* s_max);

/* Thread-local description of the last error (never NULL). */
const char* fdtd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FDTD_H */
