/*
 * ibfsa.h -- C ABI of the GB300 (sm_103a) stage right-hand side of the immersed-boundary
 * WENO/TENO method for fluid-structure-acoustics interaction of Wang, Tian & Lai
 * (arXiv:1905.00182, Sec. 2).
 *
 * What one call computes (Sec. 2):
 *   compressible Navier-Stokes, Eq. 2-5, on a Cartesian grid with cell-centred nodes
 *   x_i = lo + (i + 1/2) h, h = (hi - lo)/n, or stretched per direction (ibfsa_set_mesh);
 *   Q = [rho, rho u, rho v, (rho w), E];
 *   convective fluxes split by a global Lax-Friedrichs splitting f+- = (F +- alpha_d Q)/2 with
 *   alpha_d = max(|u_d| + c) of the stage input, reconstructed component-wise (or, as an
 *   option, characteristic-wise) at every face by fifth-order WENO5-JS or TENO5 (text after
 *   Eq. 5), differenced conservatively;
 *   viscous fluxes [0, tau_{.d}, b_d] (Eq. 5, no heat flux) by fourth-order central
 *   differences (gradients, then divergence), scaled by 1/Re;
 *   penalty immersed boundary: U_ib = sum_j u_j delta_h(X - x_j) h^d (Eq. 8),
 *   F = alpha_pen xi + beta_pen (U_ib - U) with xi = int (U_ib - U) dt (Eq. 7),
 *   f = -sum_k F_k delta_h(X_k - x) dS_k (Eq. 9), delta_h from Peskin's four-point
 *   lambda (Eq. 10-11); the fluid source is S = [0, f, f.u];
 *   third-order TVD (SSP) Runge-Kutta of Shu & Osher on Q and xi (text after Eq. 5).
 *
 * Conventions shared by every entry point:
 *  - Return value: IBFSA_OK (0) or a negative IBFSA_ERR_* code; ibfsa_last_error() gives a
 *    thread-local message for the last failure.
 *  - Memory: the library allocates NO device memory.  The caller allocates one workspace of
 *    ibfsa_workspace_bytes() bytes (256-byte aligned) and owns it; all grid state lives there.
 *    Array arguments may be device pointers or host pointers (copies use cudaMemcpyDefault);
 *    host memory should be pinned for asynchronous copies.
 *  - Streams: every launch and copy goes to the stream given at ibfsa_create_grid (a
 *    cudaStream_t passed as void*, NULL = legacy default stream).  Calls are asynchronous
 *    unless stated; only calls returning values to the host synchronise that stream.
 *  - Layouts: state arrays are structure-of-arrays [nv][nz][ny][nx], x fastest, FP64, with
 *    nv = dim + 2 and nz = 1 in 2D.  Marker and probe arrays are [dim][n] (coordinates of point
 *    k at k, n + k, 2n + k).
 *  - Errors found on the device (a marker whose four-point support leaves the interior) set
 *    bits of a device status word, read by ibfsa_get_status(); kernels never trap.
 */
#ifndef IBFSA_H
#define IBFSA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  IBFSA_OK = 0,
  IBFSA_ERR_ARG = -1,         /* invalid argument (NULL, size, descriptor field) */
  IBFSA_ERR_CUDA = -2,        /* a CUDA runtime call failed */
  IBFSA_ERR_NONFINITE = -3,   /* state holds NaN/Inf (reported by ibfsa_get_status) */
  IBFSA_ERR_BOUNDS = -4,      /* marker/probe support outside the interior */
  IBFSA_ERR_UNSUPPORTED = -5, /* descriptor asks for a variant the library does not provide */
  IBFSA_ERR_WORKSPACE = -6    /* workspace too small or misaligned */
};

/* convective schemes (text after Eq. 5); IBFSA_MLP_TENO5 = the learned-weight variant: TENO5
 * decides where the flow is smooth, and there the weights come from the network attached with
 * ibfsa_set_mlp (FP32 perturbation arithmetic only) */
enum { IBFSA_WENO5JS = 0, IBFSA_TENO5 = 1, IBFSA_MLP_TENO5 = 2 };
/* arithmetic of the stage kernels: FP64 throughout, or the perturbation form -- the stencil
 * arithmetic (split fluxes, reconstruction, viscous terms, right-hand side) in FP32 on
 * q' = Q - qinf and on primitive perturbations, expanded so that no O(1) free-stream terms
 * cancel, while the RK state, its combination, the IB markers and the probes stay FP64 */
enum { IBFSA_FP64 = 0, IBFSA_FP32_PERTURB = 1 };
/* boundary rules per face of the box: ghost cells copy the nearest interior cell, hold the
 * free stream, or wrap around; or the characteristic non-reflecting condition (Sec. 2, after
 * Thompson): ghosts copy the boundary cell, and at the boundary cell the convective term normal
 * to the face is replaced by the characteristic form of the Euler equations along the normal --
 * wave amplitudes L1 = (u - c)(p_x - rho c u_x), L2 = u (c^2 rho_x - p_x), L_t = u (u_t)_x,
 * L5 = (u + c)(p_x + rho c u_x) from fourth-order one-sided derivatives of the primitives into
 * the domain, those whose speed points into the domain set to zero, mapped back to the
 * conservative variables (needs n >= 5 along that direction) */
enum { IBFSA_BC_ZERO_GRAD = 0, IBFSA_BC_FREESTREAM = 1, IBFSA_BC_PERIODIC = 2,
       IBFSA_BC_CHARACTERISTIC = 3 };
/* status bits of ibfsa_get_status: a marker or probe support left the grid; a non-finite
 * value entered the state; a kernel gave up waiting for its tensor copies (iteration limit), so
 * the results of that call are invalid */
enum { IBFSA_STATUS_BOUNDS = 1, IBFSA_STATUS_NONFINITE = 2, IBFSA_STATUS_TIMEOUT = 4 };

typedef struct ibfsa_grid ibfsa_grid; /* opaque; created and destroyed by the library */

typedef struct {
  int dim;                 /* 2 or 3 */
  int n[3];                /* interior cells per direction; n[2] = 1 in 2D */
  double lo[3], hi[3];     /* domain box */
  double gamma;            /* ratio of specific heats (ideal gas) */
  double Re;               /* Reynolds number of Eq. 2; Re <= 0 drops the viscous terms */
  double qinf[5];          /* free-stream conservative state (first nv entries used) */
  int scheme;              /* IBFSA_WENO5JS | IBFSA_TENO5 | IBFSA_MLP_TENO5 */
  int precision;           /* IBFSA_FP64 | IBFSA_FP32_PERTURB */
  int strict_fp;           /* 1: every FP64 operation rounded separately (no fused
                              multiply-add), divisions kept as divisions, spreading summed
                              cell by cell in marker order -- the result is reproducible bit
                              for bit by a sequential FP64 evaluation of the same formulas in
                              the same order.  0: fused multiply-add and reciprocals allowed,
                              spreading by atomics, TENO5's linear weights taken wherever its
                              sufficient all-kept test (tau5 <= 4 min beta, evaluated in FP32
                              on the stencil's FP64 differences) passes -- the weights TENO5
                              gives there (faster; rounding differs). */
  int bc[3][2];            /* IBFSA_BC_* for the low/high face of each direction; periodic
                              needs both faces periodic and n >= 4 */
  int sponge_cells;        /* width S of an absorbing layer (0 = none): L -= sigma (Q - qinf)
                              with sigma = sponge_sigma ((S - m)/S)^3, m = cells to the wall */
  double sponge_sigma;
  double alpha_pen;        /* alpha of Eq. 7 */
  double beta_pen;         /* beta of Eq. 7 */
  int max_markers;         /* capacity for Lagrangian markers */
  int max_probes;          /* capacity for probe points */
  int charwise;            /* 0: each split-flux component reconstructed on its own (the
                              paper is silent; the default); 1: characteristic-wise -- the
                              split fluxes of each stencil projected on the left eigenvectors
                              of the Euler flux Jacobian along the face normal at the Roe
                              average of the face's two cells, reconstructed per field and
                              projected back.  In the FP32 perturbation form the split-flux
                              perturbations are projected, on eigenvectors built in FP32 from
                              the face's full primitive state.  Not with IBFSA_MLP_TENO5
                              (IBFSA_ERR_UNSUPPORTED). */
} ibfsa_grid_desc;

/* Bytes of device workspace a grid with this descriptor needs (for the caller to allocate). */
int ibfsa_workspace_bytes(const ibfsa_grid_desc *desc, size_t *bytes);

/* Create a grid on the current CUDA device.  d_workspace: device memory of at least
 * ibfsa_workspace_bytes() bytes, 256-byte aligned, owned by the caller and kept alive until
 * ibfsa_destroy_grid.  cuda_stream: cudaStream_t for all work of this grid.  The state is
 * undefined until ibfsa_set_state; the marker count is 0 until ibfsa_set_markers. */
int ibfsa_create_grid(const ibfsa_grid_desc *desc, void *d_workspace, size_t workspace_bytes,
                      void *cuda_stream, ibfsa_grid **out);

/* Release the host-side grid object (the workspace stays the caller's). */
int ibfsa_destroy_grid(ibfsa_grid *g);

/* Copy the interior state Q [nv][nz][ny][nx] (device or host pointer) in, or out.
 * ibfsa_get_state synchronises the grid's stream when Q is host memory. */
int ibfsa_set_state(ibfsa_grid *g, const double *Q);
int ibfsa_get_state(ibfsa_grid *g, double *Q);

/* Lagrangian markers of the immersed boundary (Eq. 7-9): positions X [dim][n], velocities U
 * [dim][n] (held for the whole step) and quadrature weights dS [n] (arc length in 2D, area in
 * 3D).  reset_integral = 1 zeroes xi = int (U_ib - U) dt; 0 keeps it (same markers, moved).
 * Every marker's support must lie two cells inside the interior; violations set
 * IBFSA_STATUS_BOUNDS (checked on the device, read with ibfsa_get_status). */
int ibfsa_set_markers(ibfsa_grid *g, int n, const double *X, const double *U, const double *dS,
                      int reset_integral);

/* Penalty force F_k of Eq. 7 at the last evaluated stage, [dim][n] (device or host). */
int ibfsa_get_marker_forces(ibfsa_grid *g, double *F);

/* xi = int (U_ib - U) dt per marker, [dim][n], in or out (device or host). */
int ibfsa_get_penalty_integral(ibfsa_grid *g, double *xi);
int ibfsa_set_penalty_integral(ibfsa_grid *g, const double *xi);

/* Right-hand side dQ/dt = L(Q) + S at the current state (Eq. 2 with the IB source of Eq. 9),
 * written to L [nv][nz][ny][nx] (device pointer).  Also leaves the marker forces of Eq. 7. */
int ibfsa_rhs(ibfsa_grid *g, double *L);

/* Advance the state and xi by nsteps third-order SSP Runge-Kutta steps of size dt:
 *   Q1 = Qn + dt L(Qn);  Q2 = 3/4 Qn + 1/4 (Q1 + dt L(Q1));  Qn+1 = 1/3 Qn + 2/3 (Q2 + dt L(Q2)),
 * each stage evaluated as a Qn + b (Qs + dt L(Qs)).  Markers stay fixed during the call; the
 * stages see the source at t, t + dt, t + dt/2 and the grid's clock advances by dt per step.
 * dt must be finite and positive, nsteps >= 0 (IBFSA_ERR_ARG otherwise). */
int ibfsa_rk3_step(ibfsa_grid *g, double dt, int nsteps);

/* Periodic Gaussian pressure source of Sec. 3.6 (Eq. 16), A_p = amp exp(-b ln2 |x - xc|^2)
 * cos(omega t), entering the energy equation as A_p / (gamma - 1) (a source in the pressure
 * equation; no mass or momentum source).  xc: [dim] host array.  amp = 0 removes it.  Length
 * and time in the grid's units (for the paper's values A = 0.01, B = 16, omega = 2 pi in units
 * of the sphere radius R and R/c: amp = -0.01, b = 16/R^2, omega = 2 pi c/R).  Evaluated at the
 * stage times t, t + dt, t + dt/2 of each step on the grid's clock. */
int ibfsa_set_source(ibfsa_grid *g, double amp, double b, double omega, const double *xc);
/* Non-uniform (stretched) mesh along direction a (Sec. 2: a uniform box around the body,
 * stretched away from it; Sec. 3.2: a sinusoidal transition between the two spacings), given as
 * a mapping x(xi) of a computational coordinate xi with unit spacing per cell: x_nodes[i + 4] is
 * the coordinate of node i and dxdxi[i + 4] the metric dx/dxi there, for i = -4 .. n[a] + 3
 * (n[a] + 8 entries each, ghost nodes included; host or device memory).  Every difference along
 * a -- the convective flux difference and both fourth-order viscous differences -- is taken in
 * xi and divided by dx/dxi at the node where it is taken; the pressure source is evaluated at the
 * node coordinates; markers and probes must keep their four-point support (and one node beyond
 * each side) where dx/dxi is constant (relative 1e-12), the delta then taking that spacing (else
 * IBFSA_STATUS_BOUNDS); the sponge width stays in cells; a time step must respect the smallest
 * spacing.  Nodes must be finite and strictly increasing, the metric positive
 * (IBFSA_ERR_ARG otherwise); a periodic direction cannot be stretched (IBFSA_ERR_UNSUPPORTED).
 * Both pointers NULL: back to the uniform spacing (hi - lo)/n.  The arrays are copied into the
 * grid's workspace; synchronises the grid's stream. */
int ibfsa_set_mesh(ibfsa_grid *g, int a, const double *x_nodes, const double *dxdxi);

/* The grid's clock: ibfsa_rk3_step and ibfsa_fsi_step advance it by dt per step; ibfsa_rhs
 * evaluates the source at it.  Starts at 0. */
int ibfsa_set_time(ibfsa_grid *g, double t);
int ibfsa_get_time(ibfsa_grid *g, double *host_t);

/* Split speeds alpha_d = max over the interior of |u_d| + c of the current state, d < dim,
 * to the host (synchronises), for dt = CFL / sum_d (alpha_d / h_d). */
int ibfsa_max_wavespeed(ibfsa_grid *g, double *host_alpha);

/* Pressure fluctuation dp = sum_j p_j prod_d lambda((x_p - x_j)/h_d) - p_inf (the fluctuation
 * of Sec. 3.1 sampled with the same four-point kernel as Eq. 8) at np points xp [dim][np]
 * (device or host) into out [np] (device or host; synchronises when out is host memory). */
int ibfsa_probe(ibfsa_grid *g, int np, const double *xp, double *out);

/* Time statistics of probe signals (Sec. 3.2): the fluctuating pressure about its time mean,
 * dp~ = dp - mean_t(dp), and the root mean square of dp~ that Sec. 3.3 and 4 plot on rings of
 * probes.  ibfsa_probe_accumulate samples dp at np points exactly as ibfsa_probe does (out, device
 * or host, may be NULL) and folds the samples into acc, caller-owned device memory of 3*np
 * doubles laid out [count | mean | M2] (Welford's running update, accurate when the mean
 * dominates the fluctuation), zero-filled by the caller before the first sample.
 * ibfsa_probe_stats writes, per probe, the time mean of dp and the RMS of dp~ (population form,
 * sqrt(M2 / count); both 0 for a probe without samples) to mean and rms [np], device memory.
 * FP64, each operation rounded on its own; stream-ordered on the grid's stream.  Host pointers
 * for acc, mean or rms: IBFSA_ERR_ARG. */
int ibfsa_probe_accumulate(ibfsa_grid *g, int np, const double *xp, double *out, double *acc);
int ibfsa_probe_stats(ibfsa_grid *g, int np, const double *acc, double *mean, double *rms);

/* Force on the body and power delivered to it, from the penalty forces of the last evaluated
 * stage (Eq. 7): host_force[d] = sum_k F_k,d dS_k (d < dim), *host_power = sum_k (F_k . U_k) dS_k
 * (may be NULL).  The force the body exerts on the fluid is the opposite (Eq. 9); the drag,
 * lift and power coefficients of Sec. 4 are these divided by 0.5 rho U^2 L (and U).  FP64,
 * summed in a fixed order; synchronises the stream. */
int ibfsa_body_force(ibfsa_grid *g, double *host_force, double *host_power);

/* Device status bits (IBFSA_STATUS_*) accumulated since the last call; clears them.
 * Synchronises the grid's stream. */
int ibfsa_get_status(ibfsa_grid *g, int *host_flags);

/* Self-test of the kernels' bounded waits (not part of the method; the paper has no
 * counterpart): one thread block waits on a shared-memory barrier that no tensor copy will
 * complete, gives up after the poll limit the convective kernels use, and reports
 * IBFSA_STATUS_TIMEOUT in the grid's status word (read and cleared by ibfsa_get_status) through
 * the same code path -- no fault, no trap, nothing left in flight; the grid stays usable.
 * Asynchronous on the grid's stream. */
int ibfsa_selftest_wait(ibfsa_grid *g);

/* Instrumentation (not part of the method): launch counts per kernel class are always kept;
 * with profiling enabled every launch is bracketed by CUDA events on the grid's stream.
 * Classes, in order: 0 pad (ghosts, primitives, split speeds), 1 IB interpolation and penalty
 * force, 2-4 convective x/y/z, 5 viscous fluxes, 6 viscous divergence, 7 IB spreading,
 * 8 finish (sponge, source, RK combination), 9 probes, 10 plate (markers from the plate, stage
 * force averaging, structure step; ibfsa_fsi_step).  ibfsa_profile_read synchronises the
 * stream, copies up to nclass entries (milliseconds summed over timed launches, launches,
 * timed launches; any pointer may be NULL) and resets the counters. */
int ibfsa_profile_enable(ibfsa_grid *g, int enable);
int ibfsa_profile_read(ibfsa_grid *g, int nclass, double *host_ms, long long *host_launches,
                       long long *host_timed);

/* ---- Learned reconstruction weights (the learned-weight variant of the fifth-order
 * reconstruction of Sec. 2, text after Eq. 5) ------------------------------------------------
 * A network maps the normalised five-point stencil x = (v - v_2)/amp, amp = max_j |v_j - v_2|,
 * of one split-flux component to the three weights of the third-order candidates:
 * 5 -> 32 -> 32 -> 32 (gelu, tanh form) -> 3 -> softmax; face = v_2 + amp sum_k w_k qhat_k.
 * Parameters: one float vector of IBFSA_MLP_NPARAM = 2403 entries [W1 (32x5, row = output
 * unit), b1, W2 (32x32), b2, W3 (32x32), b3, W4 (3x32), b4].  Inference and training run on the
 * tensor cores with every parameter and activation rounded to bfloat16 and FP32 accumulation.
 * A training state (ibfsa_mlp_state_bytes() bytes of caller-allocated device memory, 16-byte
 * aligned) holds FP32 master parameters, Adam moments, the last gradient and loss, and the
 * packed bfloat16 image the kernels read.  Stencils are float [n][5] (upwind-ordered: the
 * reconstruction is at the face between entries 2 and 3), targets float [n] (the face value),
 * device memory.  Loss = mean over the batch of (sum_k w_k qhat_k - (target - v_2)/amp)^2;
 * stencils with amp = 0 contribute nothing. */
#define IBFSA_MLP_NPARAM 2403
size_t ibfsa_mlp_state_bytes(void);
/* Set the master parameters (params: 2403 floats, device or host) and zero the Adam moments. */
int ibfsa_mlp_init(void *d_state, const float *params, void *cuda_stream);
/* One Adam step (lr > 0; beta 0.9 / 0.999, eps 1e-8, step = 1, 2, ...) on the gradient of the
 * batch; with lr = 0 only the gradient and the loss are computed (parameters unchanged). */
int ibfsa_mlp_train_step(void *d_state, int n, const float *d_stencils, const float *d_targets,
                         float lr, int step, void *cuda_stream);
/* Copy master parameters, last gradient and last loss out (any pointer may be NULL; host or
 * device memory); synchronises the stream. */
int ibfsa_mlp_read(const void *d_state, float *params, float *grad, float *loss,
                   void *cuda_stream);
/* Inference on n stencils: face values [n], weights [n][3] and, with targets, the mean loss
 * (each output may be NULL; device memory). */
int ibfsa_mlp_eval(const void *d_state, int n, const float *d_stencils, const float *d_targets,
                   float *d_face, float *d_omega, float *d_loss, void *cuda_stream);

/* Attach the learned weights of a training state to a grid (IBFSA_MLP_TENO5): a
 * reconstruction uses the network when TENO5 keeps all three stencils and the stencil's
 * amplitude max_j |v_j - v_2| exceeds 1e-9 (split-flux perturbation units); otherwise TENO5's
 * weights.  The image is copied (asynchronously), the state may be freed afterwards. */
int ibfsa_set_mlp(ibfsa_grid *g, const void *d_state);
/* Reconstructions that used the network and all reconstructions evaluated since the last call
 * (host array of two counts; synchronises). */
int ibfsa_mlp_stats(ibfsa_grid *g, unsigned long long *host_counts);
/* Training stencils from the grid's current state (FP32 perturbation grids): random faces,
 * directions, components and split-flux signs; kept when the learned form would use the
 * network there (TENO5 keeps all three stencils, amplitude above the floor).  Writes up to n_max
 * stencils [n][5] (upwind-ordered) and targets [n]: the face value of the ninth-order
 * upwind-biased reconstruction of the same split flux from the 9 cells on its upwind side
 * (exact for polynomials of degree 8), and the number of stencils accepted (device int; the
 * first min(count, n_max) were written).  attempts: candidate faces drawn per thread. */
int ibfsa_mlp_sample(ibfsa_grid *g, int n_max, unsigned long long seed, int attempts,
                     float *d_stencils, float *d_targets, int *d_count);

/* ---- Flexible plate and two-way coupling (Sec. 2, Eq. 1; Sec. 4.1, Eq. 17) ----------------
 * A plate immersed in a 2D fluid, governed by Eq. 1 and discretised in the absolute nodal
 * coordinate formulation named by the paper: n_el equal elements of length l = L / n_el; node j
 * carries e_j = [x, y, x_s, y_s] (position and slope); inside an element r(s) is the cubic
 * Hermite interpolation of the two nodes.  Eq. 1 is taken as the Euler-Lagrange equation of the
 * kinetic energy 1/2 int rho_s |r_t|^2 ds and the elastic energy
 * 1/2 int [K_S (|r_s| - 1)^2 + K_B |r_ss|^2] ds: consistent mass matrix, constant bending matrix,
 * stretching force by five-point Gauss-Legendre quadrature.  Time: the implicit midpoint rule
 *   e_{n+1} = e_n + dt (v_n + v_{n+1}) / 2,  M (v_{n+1} - v_n) = dt [Q_f - Q_int((e_n + e_{n+1})/2)],
 * solved by Newton's method (block cyclic reduction over the 4 x 4 node blocks) in one thread
 * block, in FP64 with every operation rounded separately except explicit fused multiply-adds
 * (deterministic: the same inputs give the same bits on every run).
 * Load: the penalty force F_k of Eq. 7 (force of the fluid on the structure, per unit length) at
 * markers s_k = (k + 1/2) L / n_markers, dS_k = L / n_markers: Q_f = sum_k S(s_k)^T F_k dS_k in
 * marker order.  Clamp (IBFSA_PLATE_CLAMPED): node 0 at x0 + (A0/2) cos(2 pi f t)[cos b, sin b]
 * with its slope along [cos(theta0 + a), sin(theta0 + a)], a = (alpha_m/2) sin(2 pi f t + phi)
 * (Eq. 17); the slope's length stays free.  Layouts: e, v [4 (n_el + 1)] node-major; marker
 * arrays [2][n_markers].  Memory: one caller-owned workspace of ibfsa_plate_workspace_bytes(),
 * 256-byte aligned; the library allocates nothing.  Work goes to the stream given at creation;
 * Newton failures (iteration limit, zero or non-finite pivot, non-finite increment) set
 * IBFSA_STATUS_NOCONV, read with ibfsa_plate_get_status. */
enum { IBFSA_PLATE_FREE = 0, IBFSA_PLATE_CLAMPED = 1 };
enum { IBFSA_STATUS_NOCONV = 8 };
#define IBFSA_PLATE_MAX_EL 128
typedef struct ibfsa_plate ibfsa_plate; /* opaque; created and destroyed by the library */
typedef struct {
  int n_el;              /* elements, 1..IBFSA_PLATE_MAX_EL */
  int n_markers;         /* Lagrangian markers along the plate, >= 1 */
  double length;         /* L */
  double rho_s;          /* mass per unit length (Eq. 1) */
  double K_S, K_B;       /* stretching and bending rigidity (Eq. 1) */
  int clamp;             /* IBFSA_PLATE_FREE | IBFSA_PLATE_CLAMPED */
  double x0[2];          /* clamp mean position */
  double theta0;         /* chord direction of the clamp at a = 0 */
  double A0, freq, beta, alpha_m, phi;  /* clamp motion, Eq. 17 */
  int newton_max;        /* Newton iteration limit (>= 1) */
  double newton_tol;     /* converged when max |Newton increment| <= newton_tol * L */
} ibfsa_plate_desc;

int ibfsa_plate_workspace_bytes(const ibfsa_plate_desc *desc, size_t *bytes);
/* Create a plate on the current device; the state is undefined until ibfsa_plate_set_state. */
int ibfsa_plate_create(const ibfsa_plate_desc *desc, void *d_workspace, size_t workspace_bytes,
                       void *cuda_stream, ibfsa_plate **out);
int ibfsa_plate_destroy(ibfsa_plate *p);
/* Nodal coordinates e and rates v (device or host) and the time t of the clamp motion. */
int ibfsa_plate_set_state(ibfsa_plate *p, const double *e, const double *v, double t);
/* Copy e, v out (device or host; either may be NULL) and the time to *host_t (may be NULL);
 * synchronises when an output is host memory. */
int ibfsa_plate_get_state(ibfsa_plate *p, double *e, double *v, double *host_t);
/* One step of size dt > 0 under marker forces F [2][n_markers] (device or host; NULL = none),
 * held over the step; the clamp is taken to t + dt. */
int ibfsa_plate_step(ibfsa_plate *p, double dt, const double *F);
/* Marker positions X, velocities U [2][n_markers] and weights dS [n_markers] of the current
 * state (device or host; synchronises when an output is host memory). */
int ibfsa_plate_markers(ibfsa_plate *p, double *X, double *U, double *dS);
/* Status bits (IBFSA_STATUS_NOCONV) and the largest Newton iteration count since the last
 * call (either pointer may be NULL); clears both; synchronises. */
int ibfsa_plate_get_status(ibfsa_plate *p, int *host_flags, int *host_max_iters);

/* Force of the fluid on the plate and the power it delivers, over the last step (ibfsa_plate_step
 * or ibfsa_fsi_step): host_force[a] = sum_k F_k,a dS_k and *host_power = sum_k (F_k . U_k) dS_k
 * (may be NULL), with F the step's load and U the marker velocities held during the step, FP64
 * summed in marker order; synchronises.  The thrust, lift and power coefficients of Sec. 4.1
 * (Eq. 19) are -host_force[0], host_force[1] and -*host_power times 2 / (rho U^2 L) (power:
 * 2 / (rho U^3 L)) for a stream along +x. */
int ibfsa_plate_force(ibfsa_plate *p, double *host_force, double *host_power);

/* nsteps coupled steps of plate and fluid (2D grid with max_markers >= n_markers; the grid's
 * stream must be the plate's): the grid's markers take the plate's positions, velocities and
 * weights at the step start and keep them for the three SSP-RK3 stages (ibfsa_rk3_step); the
 * plate then steps under Fbar = F1/6 + F2/6 + 2 F3/3 of the stages' penalty forces -- the
 * weights the Runge-Kutta update gives the stages -- so the impulse the fluid receives through
 * Eq. 9 is exactly the opposite of the plate's.  The penalty integral xi carries over between
 * calls (zero it when the coupling starts, e.g. ibfsa_set_markers(..., 1)).  Asynchronous. */
int ibfsa_fsi_step(ibfsa_grid *g, ibfsa_plate *p, double dt, int nsteps);

/* Allocation-free right-hand side.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory -- plug-ins whose host application owns the whole
 * device-memory budget, latency-critical loops that must not pay the implicit device-wide
 * synchronisation of cudaMalloc/cudaFree, and foreign-language front ends that can only pass
 * pointers they were given.  It computes what ibfsa_rhs computes for a grid with this
 * descriptor, state Q [nv][nz][ny][nx], n_markers markers (X, U [dim][n_markers], dS
 * [n_markers], xi [dim][n_markers]) into L [nv][nz][ny][nx], and the marker penalty forces (as
 * ibfsa_rhs computes them) into F [dim][n_markers] when F is not NULL; all pointers are device
 * memory owned by the caller.  status (device int, may be NULL) receives the IBFSA_STATUS_*
 * bits of this call.
 * The descriptor must ask for IBFSA_FP64 arithmetic (strict or fast).
 * No grid object and no workspace: its scratch (padded state, primitives, viscous fluxes, split
 * speeds) lives in one static device array of IBFSA_NOALLOC_SCRATCH_BYTES that every GPU loading
 * this library holds until the process exits.  Grids whose scratch would exceed it are
 * rejected with IBFSA_ERR_WORKSPACE (about 50^3 cells in 3D with viscosity, 550^2 in 2D).
 * It calls no cudaMalloc, cudaFree or other allocating routine.  The first call on a device
 * looks up the device address of that array (cudaGetSymbolAddress, with the device current)
 * and caches it for that device's current context; make that first call before any stream
 * capture.  After a device reset (cudaDeviceReset) the new context's first call looks the
 * address up again, and the same rule applies to it.  Every call shares the array
 * and it keeps the previous call's contents (what must start at zero is cleared by each call);
 * calls whose work overlaps on the GPU -- different streams, or different host threads -- race
 * on it and must be serialised by the caller.  Asynchronous on cuda_stream. */
#define IBFSA_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int ibfsa_rhs_noalloc(const ibfsa_grid_desc *desc, const double *Q, int n_markers,
                      const double *X, const double *U, const double *dS, const double *xi,
                      double *L, double *F, int *status, void *cuda_stream);

/* Message of the last failing call on this thread. */
const char *ibfsa_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* IBFSA_H */
