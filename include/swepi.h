/*
 * swepi.h -- C ABI of libswepi.so: the GB300 (sm_103a) hot path of the
 * high-order shallow-water method of Gaudreault, Charron, Dallerit and Tokman
 * (arXiv 2101.05617): complex-step Jacobian-vector products of the direct-flux-
 * reconstruction (DFR) right-hand side on the rotated cubed sphere, taken at
 * every Krylov iteration of the phi-function solver inside every multistep
 * exponential propagation iterative (EPI) step.
 *
 * Conventions shared by every call
 * --------------------------------
 * State layout ("canonical"): FP64, contiguous, index
 *     [var][panel][e2][e1][k2][k1]
 * var 0 = sqrt(g) H, var i = sqrt(g) H u^i (i = 1, 2): the tensor density q^mu
 * of App. D (Eq. 136) in the angular cubed-sphere coordinates x^i in
 * [-pi/4, pi/4] of Eq. (1)-(2); panel 0..5, elements e1, e2 in 0..n_e-1,
 * Gauss-Legendre points k1, k2 in 0..p (N_s = p + 1 per direction, Sec. 3.1).
 * n = 3 * 6 * n_e^2 * N_s^2 unknowns.
 *
 * Memory: every vector argument named *_dev is a device pointer owned by the
 * caller (e.g. a torch tensor), 8-byte aligned, at least n doubles; the library
 * never frees caller memory.  Host pointers are named *_host.  The library owns
 * its workspace (metric tables, Krylov basis, Hessenberg matrix, EPI history),
 * allocated in sw_init / on first use and released by sw_free.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Calls enqueue their kernels on it and return; results are valid
 * after the stream is synchronised.  Calls that return statistics (kiops,
 * epi) synchronise the stream internally because the adaptive controller reads
 * small device scalars between Krylov batches.
 *
 * Errors: every int-returning call returns SW_OK (0) or a negative status;
 * no exception crosses the ABI; sw_status_str() names the status.  A context
 * is used by one host thread at a time, with the device it was created on
 * current: a call that takes a context and launches work returns SW_EINVAL,
 * before any launch, when another device is current.
 */
#ifndef SWEPI_H
#define SWEPI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SW_OK 0
#define SW_EINVAL (-1)      /* bad argument: size, pointer, order, option */
#define SW_ENOMEM (-2)      /* device or host allocation failed */
#define SW_ECUDA (-3)       /* a CUDA runtime call or kernel launch failed */
#define SW_EKRYLOV (-4)     /* phi-function solver hit its substep/rejection cap */
#define SW_ETIMEOUT (-5)    /* a bounded device-side wait gave up */
#define SW_ENONFINITE (-6)  /* NaN/Inf met where a finite value is required */
#define SW_ESCRATCH (-7)    /* grid too large for the fixed scratch of sw_jvp_static_scratch */

typedef struct sw_ctx* sw_ctx_t;

/* Physical constants and grid rotation (App. B: panel 0 centred at longitude
 * lambda0, latitude phi0, rotated by alpha0; the other five panels follow the
 * cube, Eq. 81-95).  precision: 0 = FP64 throughout (the split FP64 JVP of
 * sw_set_jvp_mode 1); 1 = the complex64-bulk form from the start (the Krylov
 * JVPs' imaginary half in FP32, everything else FP64: sw_set_jvp_mode 2); other
 * values are rejected.  sw_set_jvp_mode may change the form later. */
typedef struct {
  double radius;   /* a, m */
  double gravity;  /* g_r, m s^-2 (Eq. 51) */
  double omega;    /* Omega, s^-1 */
  double lambda0, phi0, alpha0;
  int precision;
} sw_params;

/* Options of the adaptive Krylov phi-function solver (Eq. 29).  tol is relative
 * to the 2-norm of the initial augmented vector; m_* bound the Krylov size;
 * iop is the incomplete-orthogonalisation window (2 and 3 run fused into the
 * JVP epilogue and two vector passes, wider windows with separate dot and axpy
 * launches); tau_init <= 0 means "start with the whole interval". */
typedef struct {
  double tol;
  int m_init, m_min, m_max, iop;
  double tau_init;
} sw_kiops_opts;

typedef struct {
  int substeps, rejects, krylov_iters, m_final;
  double tau_final, err_last;
} sw_kiops_stats;

/* Build the grid of 6 x n_e x n_e elements of degree p (N_s = p + 1 points per
 * direction, Sec. 3.1-3.2): panel frames, Gauss-Legendre points, DFR matrices
 * (Eq. 8, 13), metric and Christoffel tables at nodes (Eq. 67-80) and at
 * interface points, the panel connectivity with the App. C transforms.
 * 1 <= n_e <= 1024, 1 <= p <= 7.  Selects the current CUDA device for the
 * context.  *out receives the context (NULL on failure). */
int sw_init(int n_e, int p, const sw_params* params, sw_ctx_t* out);

/* Release the context and all library-owned device memory. NULL is a no-op. */
void sw_free(sw_ctx_t ctx);

/* n (number of unknowns), nodes per variable, and grid sizes. */
long long sw_num_unknowns(sw_ctx_t ctx);
int sw_grid_info(sw_ctx_t ctx, int* n_e, int* p, double* dx);

/* Unit position vectors of the nodes, host array [3][nodes] in canonical node
 * order (used to evaluate initial fields). */
int sw_node_xyz(sw_ctx_t ctx, double* xyz_host);

/* State from fields at the nodes (host arrays, canonical node order):
 * free-surface height h, bottom height hB, Cartesian wind V[3][nodes] (m/s).
 * Writes q_host[3][nodes] with q^0 = sqrt(g)(h - hB), q^i = q^0 u^i,
 * u^i = h^{ij} (V . d r / d x^j), and stores hB in the context as by
 * sw_set_bottom. */
int sw_state_from_fields(sw_ctx_t ctx, const double* h_host, const double* hB_host,
                         const double* V_host, double* q_host);

/* Bottom height h_B at the nodes (nodes = n/3 doubles, canonical node order):
 * the topography source of Eq. (2) uses its element-local collocation
 * gradient.  sw_set_bottom takes a DEVICE pointer (on the context's device;
 * anything else is SW_EINVAL), copies it to the host and builds the
 * topography coefficients there, as sw_set_bottom_host does from a host array.
 * Both are initialisation calls: they synchronise the device, and the next
 * RHS/JVP/EPI call uses the new bottom. */
int sw_set_bottom(sw_ctx_t ctx, const double* hB_dev);
int sw_set_bottom_host(sw_ctx_t ctx, const double* hB_host);

/* F(q): the DFR right-hand side of Eq. (1)-(2) (Sec. 3, Eq. 14 per direction,
 * AUSM interface flux of App. D).  q_dev, F_dev: n doubles, may not alias. */
int sw_rhs(sw_ctx_t ctx, const double* q_dev, double* F_dev, void* stream);

/* Complex-step Jacobian-vector product, Eq. (28): Jv = Im F(q + i eps v) / eps.
 * The kernels carry the imaginary parts to first order (they drop the
 * O(eps^2) cross terms), so the result is the Jacobian-vector product J(q) v
 * itself, the eps -> 0 limit of the quotient; it equals the quotient of Eq.
 * (28) to FP64 rounding whenever eps max|v^mu| / |q^mu| is below ~1e-8 (true
 * for eps = 1e-30 and for the paper's eps ~ 1.5e-8 with v scaled like q).
 * eps > 0 and finite, else SW_EINVAL.  Jv_dev may not alias q_dev or v_dev. */
int sw_jvp(sw_ctx_t ctx, const double* q_dev, const double* v_dev, double eps,
           double* Jv_dev, void* stream);

/* The same product as sw_jvp for callers that may not allocate device memory
 * while running (an application whose memory manager owns the device memory
 * and forbids other libraries from calling cudaMalloc, a plug-in host without
 * allocation rights, a loop that cannot take cudaMalloc's implicit
 * synchronisation).  The paper has no counterpart: this is a deployment
 * variant.  It allocates nothing; its interface-flux scratch is a fixed
 * 16 MiB device array inside the library (held by every GPU that loads the
 * library until exit), so it serves grids with 6 n_e^2 * 12 * (p+1) <= 2^21
 * (e.g. n_e = 60, p = 5) and returns SW_ESCRATCH for larger ones.  The first
 * call on a device looks up the array's device address (once per device, with
 * that device current); make that first call before any stream capture.  The
 * address stays cached for the process's primary context: do not use this
 * call across a cudaDeviceReset.  With a device current other than the
 * context's it returns SW_EINVAL before any launch.  All calls share the
 * array: calls that overlap on the GPU race.  Arguments and results as
 * sw_jvp. */
int sw_jvp_static_scratch(sw_ctx_t ctx, const double* q_dev, const double* v_dev, double eps,
                          double* Jv_dev, void* stream);

/* Diagnostics of Sec. 5 (synchronises): out[0..3] = the Gauss-Legendre
 * integrals (Eq. 42, without the common element Jacobian) of mass H, total
 * energy (H g_ij u^i u^j + g_r((H + h_B)^2 - h_B^2))/2 and potential enstrophy
 * (zeta + f)^2/(2H) -- the invariants whose normalised drift Eq. (44) monitors
 * -- and max |zeta|, with zeta the relative vorticity of Eq. (43) (element-local
 * collocation derivative of u_j = g_jk u^k) and f of Eq. (46).  zeta_dev (n/3
 * doubles, may be NULL) receives zeta at the nodes. */
int sw_diagnostics(sw_ctx_t ctx, const double* q_dev, double* out_host, double* zeta_dev, void* stream);

/* Error norms of Eq. (39)-(41) of H = q^0/sqrt(g) against the H of q_ref:
 * out[0] = L1, out[1] = L2, out[2] = Linf (synchronises). */
int sw_error_norms(sw_ctx_t ctx, const double* q_dev, const double* q_ref_dev, double* out_host, void* stream);

/* Split evaluation of the complex-step product (Eq. 28) for many v at one q:
 * sw_linearize evaluates the real half of F(q + i eps v) -- every quantity that
 * depends on q alone -- and stores the coefficients of the imaginary half
 * (library-owned, allocated on first use); sw_jvp_linearized then returns
 * Im F(q + i eps v)/eps for the last linearised q by propagating imaginary
 * parts only.  Equal to sw_jvp up to rounding.  Jv_dev may not alias v_dev. */
int sw_linearize(sw_ctx_t ctx, const double* q_dev, void* stream);
int sw_jvp_linearized(sw_ctx_t ctx, const double* v_dev, double* Jv_dev, void* stream);

/* How sw_kiops_phi, sw_epi_step and sw_jvp_linearized evaluate their JVPs:
 * 0 = sw_jvp per Krylov vector; 1 = sw_linearize once per linearisation point
 * then the imaginary half per vector in FP64 (default); 2 = the complex64-bulk
 * form: as 1 but the imaginary half of the Krylov JVPs runs in FP32
 * (coefficient tables rounded from the FP64 linearisation, FP32 accumulation),
 * while the Krylov basis, the orthogonalisation dot products, the small
 * exponential, the error estimate and the EPI remainder products (a small
 * difference of large terms, Eq. 33) stay FP64.  Changing the mode invalidates the last
 * linearisation. */
int sw_set_jvp_mode(sw_ctx_t ctx, int mode);

/* Where the phi-function solver's adaptive controller runs (Eq. 29 and the
 * KIOPS reading: accept/reject, the next substep tau and Krylov size m):
 * 0 = on the host (default), which reads a few device scalars after each
 * substep attempt; 1 = on the device: the whole call is one CUDA graph whose
 * conditional loops (attempts, Krylov iterations, squarings of the small
 * exponential) are steered by device kernels running the same controller, and
 * the host synchronises once, when the call returns.  The device controller
 * applies to the split JVP (modes 1 and 2) with windows 2 and 3 and the plain
 * rule while profiling is off; other calls use the host controller.  It caps a
 * call at 2000 substep attempts (SW_EKRYLOV).  The graph is built on the first
 * call and again when the window, the number of phi-vectors, the form or the
 * Krylov workspace changes. */
int sw_set_kiops_driver(sw_ctx_t ctx, int driver);

/* The two vector passes of the fused incomplete orthogonalisation (the
 * modified Gram-Schmidt updates with ||z||, then the scaling with the next
 * window dot; the KIOPS reading of Eq. 29's Krylov projection) in one launch:
 * enable = 1 (default) runs them as one cooperative launch whose CTAs wait on
 * one another for ||z|| (a bounded wait: SW_ETIMEOUT past about a second),
 * where the GPU holds the whole grid at once; 0 = two launches.  The results
 * are the same bit for bit.  Applies to the host controller; the device
 * controller's graph keeps two launches.  *active_out (may be NULL) = 1 when
 * the next phi-function call will fuse them. */
int sw_set_orth_fused(sw_ctx_t ctx, int enable, int* active_out);

/* w = sum_{k=0}^{nb-1} tau_out^k phi_k(tau_out dt J(q_lin)) b_k (Eq. 29), J by
 * the complex-step product above.  b_dev_host: host array of nb device
 * pointers (1 <= nb <= 8); a NULL entry means a zero vector.  w_dev: n
 * doubles, may alias none of the inputs.  opts NULL = defaults (tol 1e-10,
 * m 10/10/128, iop 2).  st may be NULL.  Synchronises `stream`. */
int sw_kiops_phi(sw_ctx_t ctx, const double* q_lin_dev, double dt, double tau_out, int nb,
                 const double* const* b_dev_host, const sw_kiops_opts* opts, double* w_dev,
                 sw_kiops_stats* st, void* stream);

/* One multistep EPI step of order 2..6 (Eq. 25, 30, 34-38) advancing q_dev in
 * place by dt.  The context keeps the history (q_{n-i}, F(q_{n-i})); while it
 * holds fewer than P entries the step is taken by 8 EPI2 substeps of dt/8
 * (Sec. 4 start-up).  The KIOPS size warm-starts from the previous call.
 * st (may be NULL) accumulates the step's KIOPS statistics.  Synchronises.
 * Errors: SW_EINVAL (order, dt, pointers, options), SW_ENONFINITE (a non-finite
 * phi-vector or error estimate), SW_EKRYLOV (substep or rejection cap),
 * SW_ENOMEM / SW_ECUDA.  After an error q_dev and the history may hold part of
 * the step (the start-up substeps advance q_dev one by one): restart from a
 * saved state after sw_epi_reset. */
int sw_epi_step(sw_ctx_t ctx, int order, double dt, double* q_dev, const sw_kiops_opts* opts,
                sw_kiops_stats* st, void* stream);

/* sw_epi_step on a state held in HOST memory: q_host (n doubles, caller-owned,
 * pinned or pageable) is copied to a library-owned device buffer (allocated on
 * first use), advanced by one step exactly as sw_epi_step does, and copied back
 * on `stream`; returns after the copy back.  On an error status q_host is left
 * unchanged.  Same history, statistics and errors as sw_epi_step. */
int sw_epi_step_host(sw_ctx_t ctx, int order, double dt, double* q_host, const sw_kiops_opts* opts,
                     sw_kiops_stats* st, void* stream);

/* Seed history entry i (1 = most recent) with (q_{n-i}, F(q_{n-i})) device
 * vectors (copied); F_dev NULL computes it.  i <= 4.  The multistep schemes of
 * Eq. (34)-(38) read the remainders R(q_{n-i}) of Eq. (33) at the previous
 * states; Sec. 4 (the paragraph after Eq. 38) leaves open how the starting
 * values are obtained and computes them with EPI2 at a smaller step, which
 * sw_epi_step does while the history is short.  This call supplies them
 * instead (e.g. from a finer reference run, for order tests). */
int sw_epi_set_history(sw_ctx_t ctx, int i, const double* q_dev, const double* F_dev, void* stream);

/* Forget the EPI history (the previous states of Eq. 33-38) and the KIOPS
 * warm start, so that the next sw_epi_step starts again with the EPI2 start-up
 * of Sec. 4 (the paragraph after Eq. 38). */
int sw_epi_reset(sw_ctx_t ctx);

/* Checkpoint and resume of the multistep state.  Besides q itself, the next
 * sw_epi_step reads the history pairs (q_{n-i}, F(q_{n-i})) of Eq. 33-38 (Sec.
 * 4: the previous steps' states and right-hand sides that the remainders
 * R(q_{n-i}) need), the KIOPS warm start (the previous phi-function call's
 * final Krylov size) and the previous call's features of the learned Krylov
 * controller.  A context restored from a checkpoint and given the saved q, the
 * same options, JVP mode and controller continues bit for bit as the saved one
 * would have.
 *
 * sw_epi_checkpoint_size: *bytes = the size of the checkpoint of the current
 * state (a header of 144 bytes plus 2 n doubles per history entry; n = 3 nodes).
 * Host only.
 *
 * sw_epi_checkpoint_save: writes it to buf_host (caller-owned host memory,
 * pageable or pinned, at least that many bytes): the header (format tag, grid,
 * rotation and constants, counts, warm start, controller features, an FNV-1a
 * checksum of the payload), then the entries from the most recent back, each
 * q then F, FP64 in the canonical layout.  Copies on `stream` and waits for it.
 *
 * sw_epi_checkpoint_load: replaces the context's multistep state by the one in
 * buf_host (`bytes` must be its exact size).  SW_EINVAL, before any CUDA call,
 * for a buffer that is not a checkpoint of this grid (format tag, n_e, p,
 * rotation, constants, size) or whose checksum fails.  After a CUDA failure
 * the context holds no history, as after sw_epi_reset.  Copies on `stream` and
 * waits for it. */
int sw_epi_checkpoint_size(sw_ctx_t ctx, size_t* bytes);
int sw_epi_checkpoint_save(sw_ctx_t ctx, void* buf_host, size_t bytes, void* stream);
int sw_epi_checkpoint_load(sw_ctx_t ctx, const void* buf_host, size_t bytes, void* stream);

/* The EPI coefficient matrix of order 3..6 as sw_epi_step uses it (Eq. 30,
 * 36-38; alpha_{m,i} of Eq. 35): *M rows (phi_1 .. phi_M) by *P columns
 * (R(q_{n-1}) .. R(q_{n-P})), row-major into A_host (at least 16 doubles).
 * Host only: no CUDA call, no context. */
int sw_epi_coefficients(int order, int* M, int* P, double* A_host);

/* The DFR operators of degree p (N_s = p + 1, Sec. 3.1) exactly as sw_init
 * builds them: Gauss-Legendre points xi_host[N_s] (ascending) and weights
 * w_host[N_s] on [-1, 1]; D_ext_host[N_s][N_s + 2] (row-major), the derivative
 * at xi_k of the Lagrange basis on the extended nodes {-1, xi_1 .. xi_Ns, +1}
 * (Eq. 13); l_minus_host, l_plus_host [N_s], the Lagrange basis of xi at -1 and
 * +1 (the trace rows of Eq. 8).  Any pointer may be NULL.  0 <= p <= 7.  Host
 * only: no CUDA call, no context. */
int sw_dfr_operators(int p, double* xi_host, double* w_host, double* D_ext_host, double* l_minus_host,
                     double* l_plus_host);

/* The node coefficients sw_init tabulates, at any points (X, Y) = (tan x^1,
 * tan x^2) of one panel (0..5) of the grid rotated by params: out_host[k * npts
 * + i] for k = 0..12 = g_r h^11/(2 sqrt g), g_r h^12/(2 sqrt g), g_r h^22/(2
 * sqrt g) (App. D pressure term; Eq. 67-70), -2 Gamma^1_{01}, -2 Gamma^1_{02},
 * -2 Gamma^2_{01}, -2 Gamma^2_{02} (Eq. 71-74, the panel frame giving the
 * Coriolis bracket), Gamma^1_11, 2 Gamma^1_12, 2 Gamma^2_12, Gamma^2_22 (Eq.
 * 75-80), and two topography entries (zero here: they depend on the bottom).
 * Host only: no CUDA call, no context. */
int sw_node_coefficients(const sw_params* params, int panel, int npts, const double* X_host,
                         const double* Y_host, double* out_host);

/* Interface k (0..11) of the cube as the library connects it: panels pa, pb,
 * their edges (0 = x^1 = -pi/4, 1 = x^1 = +pi/4, 2 = x^2 = -pi/4, 3 = x^2 =
 * +pi/4), rev = 1 when the along-edge coordinates run opposite, and T_host (2x2
 * row-major) = the App. C transform (Eq. 100-135) taking contravariant
 * components on panel pb to panel pa at the point with along-edge coordinate t
 * on panel pa.  Any output may be NULL.  Host only. */
int sw_interface_transform(int k, double t, int* pa, int* ea, int* pb, int* eb, int* rev, double* T_host);

/* ---- Learned Krylov control (the adaptive rule stays in charge) ----------
 * A 16 -> 64 -> 64 -> 2 perceptron with GELU hidden layers, BF16 weights and
 * FP32 accumulation predicts, per phi-function call, the initial substep
 * log(tau/tau_out) and Krylov size m/m_max from 16 per-call features (log10 of
 * max ||b_k||_1 and of the initial augmented norm; the previous call's first
 * accepted tau, its m, final m, substeps, rejections and Krylov iterations;
 * log10 of its last four h_{j+1,j}; EPI order and start-up flag; log10 dt; p).
 * Trained on log(tau_star/tau_out) and m_1/m_max of plain-rule calls (see
 * sw_kiops_log).  The error estimate still accepts or rejects every substep; without a network
 * (or on a non-finite prediction) the plain rule applies (tau = tau_out, m =
 * previous final m).  Training runs on the GPU (mean squared error on
 * standardised data, Adam on FP32 master weights, BF16 copies).
 * params: SW_MLP_PARAMS floats, W1[64][16] b1[64] W2[64][64] b2[64] W3[2][64]
 * b3[2]; norm: SW_MLP_NORM floats, input mean[16], input std[16], output
 * mean[2], output std[2].  X: n x 16 raw features, T/Y: n x 2 raw outputs
 * (device, row-major).  No paper counterpart beyond the KIOPS step choice. */
#define SW_MLP_PARAMS 5378
#define SW_MLP_NORM 36
#define SW_KIOPS_LOG_FIELDS 23
typedef struct sw_mlp* sw_mlp_t;
int sw_mlp_create(sw_mlp_t* out);
void sw_mlp_free(sw_mlp_t mlp);
int sw_mlp_set_params(sw_mlp_t mlp, const float* params_host, const float* norm_host);
int sw_mlp_get_params(sw_mlp_t mlp, float* params_host, float* bf16_params_host);
int sw_mlp_forward(sw_mlp_t mlp, const float* X_dev, int n, float* Y_dev, void* stream);
/* gradient of the loss at the current weights (no update); synchronises */
int sw_mlp_gradient(sw_mlp_t mlp, const float* X_dev, const float* T_dev, int n, float* grad_host,
                    float* loss_host, void* stream);
/* `steps` full-batch Adam steps; loss_host (may be NULL) receives each step's loss */
int sw_mlp_train(sw_mlp_t mlp, const float* X_dev, const float* T_dev, int n, int steps, float lr,
                 float* loss_host, void* stream);
/* use `mlp` (not owned; NULL = plain rule) for the context's phi-function calls */
int sw_set_controller(sw_ctx_t ctx, sw_mlp_t mlp);
/* per-call log of the phi-function solver: SW_KIOPS_LOG_FIELDS floats per call
 * (16 features, log(tau_1/tau_out) of the first accepted substep, its m/m_max,
 * Krylov iterations, rejections, substeps, m_final/m_max, log(tau_star/tau_out) with
 * tau_star = tau_1 (0.8/omega_1)^(1/order) the largest first substep the error
 * model admits); copies up to max_records, returns the number held */
int sw_kiops_log(sw_ctx_t ctx, float* out_host, int max_records);
int sw_kiops_log_clear(sw_ctx_t ctx);

/* ---- Batched ensemble -------------------------------------------------------
 * Many independent members (each an sw_ctx_t of its own grid: n_e, p in 3..5,
 * rotation, bottom) advanced together by sw_epi_step's method.  Per member the
 * sequence of operations, the adaptive rule and the statistics are those of
 * sw_epi_step (FP64 split JVP, iop 2, plain rule); results agree with
 * per-member sw_epi_step runs up to the order of floating-point sums.  Each
 * Krylov iteration of all members that are building a basis is one launch of
 * a persistent kernel captured once in a CUDA graph; the small exponentials of
 * all members that finished a basis are batched, and one read-back serves all
 * members waiting for a decision (Sec. 4's KIOPS per member).  The members'
 * contexts stay owned by the caller and must outlive the ensemble; the
 * ensemble uses their workspace and EPI history (sw_epi_reset still applies).
 * Every call synchronises `stream` before returning.
 *
 * Tiles (per member) and threads per CTA (per ensemble) shape the batched
 * kernel: interface points per face task, element tiles per volume task (a
 * tile = threads per CTA / (p+1)^2 elements, one thread per solution point)
 * and vector entries per orthogonalisation task.  sw_ens_tune searches them
 * per (n_e, p) class and threads per CTA in {128, 256, 512} by timing `iters`
 * batched iterations at the members' states q_dev (it overwrites the members'
 * Krylov workspace, not q).  sw_ens_set_policy: while the members that iterate
 * hold at least theta (0..1, default 0.5) of the unfinished members' nodes, the
 * driver keeps iterating and defers the members that wait for a decision.
 * q_dev_host / stats: host arrays of `members` entries (device state vectors;
 * per-member statistics accumulated over the run, may be NULL). */
typedef struct sw_ens* sw_ens_t;
typedef struct {
  int face_pts;   /* interface points per face task */
  int vol_tiles;  /* element tiles per volume task */
  int vec_len;    /* vector entries per update / scale task */
} sw_ens_tiles;
typedef struct {
  long long ticks;         /* batched Krylov iterations (graph replays) in the last run */
  long long reads;         /* host read-backs in the last run */
  long long expm_batches;  /* batched exponentials in the last run */
  long long launches;      /* kernel launches of the last run (graph replays count one) */
  double iter_ms;          /* device time of the batched iterations (while sw_ens_profile is on) */
  int block;               /* threads per CTA of the batched iteration kernel */
  int ctas;                /* its persistent grid */
} sw_ens_stats;
int sw_ens_create(int members, const sw_ctx_t* ctxs_host, sw_ens_t* out);
int sw_ens_free(sw_ens_t ens);
int sw_ens_set_block(sw_ens_t ens, int block);
int sw_ens_set_tiles(sw_ens_t ens, int member, const sw_ens_tiles* tiles);
int sw_ens_get_tiles(sw_ens_t ens, int member, sw_ens_tiles* tiles);
int sw_ens_set_policy(sw_ens_t ens, double theta);
int sw_ens_tune(sw_ens_t ens, double* const* q_dev_host, int iters, int* block, void* stream);
/* `steps` EPI steps of every member: orders (2..6) and dts per member. */
int sw_ens_epi_run(sw_ens_t ens, int steps, const int* orders_host, const double* dts_host,
                   double* const* q_dev_host, const sw_kiops_opts* opts, sw_kiops_stats* stats_host,
                   void* stream);
int sw_ens_stats_read(sw_ens_t ens, sw_ens_stats* out);
/* Failure-path test hook (no paper counterpart).  The batched kernel's tasks
 * wait, bounded, for their member's previous phase; every such wait ends by
 * construction, and the bound only turns a broken invariant into SW_ETIMEOUT
 * instead of a hang.  This call sets that bound to limit_s seconds (0 = the
 * default 2 s, at most 2) and adds `extra` (0 or 1) to every wait target: with
 * extra = 1 no wait can be satisfied, so the next sw_ens_epi_run / sw_ens_tune
 * launch completes after one bound and the call returns SW_ETIMEOUT (the
 * members' states are then meaningless: restore them and sw_epi_reset the
 * members).  It synchronises the device and clears an earlier give-up;
 * sw_ens_set_wait_test(e, 0, 0) restores normal operation. */
int sw_ens_set_wait_test(sw_ens_t ens, double limit_s, int extra);
/* bracket every batched iteration with CUDA events on the run's stream */
int sw_ens_profile(sw_ens_t ens, int enable);

/* Number of kernels the library launched since the context was created. */
long long sw_kernel_launches(sw_ctx_t ctx);

/* Kernel timing (tracing aid; the paper has no counterpart).  While enabled,
 * the library brackets its face-flux, volume and small-exponential kernels with
 * CUDA events recorded on the launch stream; sw_profile_read() waits for the
 * pending events and returns per-family launch counts and summed device
 * milliseconds since the last sw_profile(ctx, 1).  kind: 0 = face flux (JVP),
 * 1 = volume (JVP), 2 = face flux (RHS), 3 = volume (RHS), 4 = exponential,
 * 5 = linearisation of the split JVP, 6 = the two vector passes of the fused
 * orthogonalisation (update + norm, scale + dot). */
#define SW_PROF_KINDS 7
typedef struct {
  long long count[SW_PROF_KINDS];
  double ms[SW_PROF_KINDS];
} sw_profile_stats;
int sw_profile(sw_ctx_t ctx, int enable);
/* time only the kinds whose bit (1 << kind) is set in mask (0 = off); resets the counts */
int sw_profile_kinds(sw_ctx_t ctx, unsigned mask);
/* bracket only every `every`-th launch (every >= 1; 1 = all, the default) of
 * each timed JVP or RHS kernel family (kinds 0-3), so that a timed run is
 * perturbed less: an event pair between two kernels keeps the second from
 * starting under the first's tail (programmatic dependent launch).  Counts
 * then report the bracketed launches.  Resets the counts. */
int sw_profile_every(sw_ctx_t ctx, int every);
int sw_profile_read(sw_ctx_t ctx, sw_profile_stats* out);

/* Bounds-checked builds (a debugging aid with no paper counterpart; the
 * library built with -DSW_CHECK, libswepi_check.so).  There the kernels that
 * index through the grid tables or issue bulk copies from computed ranges test
 * those indices first: an interface line's element and edge numbers (every
 * face kernel), a staged tile's copy ranges and alignment (the complex64-bulk
 * volume kernel), a batched task's member, range and basis index (the
 * ensemble kernel).  A failed test records a code (1 interface line, 2 tile
 * copy, 3 ensemble task) and the access it guards is skipped, so the kernel
 * neither traps nor reads or writes out of range; the results of that launch
 * are then not valid.  Returns the first code recorded since the last call (0
 * none) and clears the record, or SW_ECUDA when it cannot be read; *checked
 * (may be NULL) = 1 in a checked build, else 0.  In the default build the
 * tests compile to nothing, it returns 0 and makes no CUDA call. */
int sw_check_status(int* checked);
/* Checked builds only (SW_EINVAL otherwise): what = 1 moves the first
 * interface line's owner element one grid past the last element in the
 * context's device table, so that the next face kernel's check fires (the
 * test of the checks); what = 0 moves it back. */
int sw_check_inject(sw_ctx_t ctx, int what);

/* Measured FP64 fused-multiply-add throughput of the current device in
 * TFLOP/s (2 flops per FMA), from a register-resident FMA-chain kernel: the
 * ALU roofline of the FP64 path (the paper has no counterpart). */
int sw_fp64_fma_peak(double* tflops);

/* Human-readable name of a status code (static storage). */
const char* sw_status_str(int status);

#ifdef __cplusplus
}
#endif

#endif /* SWEPI_H */
