// Internal declarations of libswepi: the context, device tables and kernel
// launchers shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <vector>

#include "../../include/swepi.h"

namespace swepi {

// Named range for tracing tools (NVTX): EPI steps, phi-function calls and
// their substep attempts show up on a profiler's timeline; without a tool
// attached the push and pop return at once.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

constexpr int MAX_NS = 8;   // p <= 7
constexpr int MAX_NB = 8;   // phi_0 .. phi_7
constexpr int MAX_HIST = 4; // EPI6 uses q_{n-1..n-4}
constexpr int KIOPS_LOG_FIELDS = 23;   // 16 features + 7 outcomes per KIOPS call
constexpr size_t KIOPS_LOG_MAX = 200000;

// Per-node coefficient arrays (structure of arrays, `nodes` doubles each).
enum NodeCoef {
  NC_C11 = 0, NC_C12, NC_C22,        // g_r h^ij / (2 sqrt g): pressure part of sqrt(g) T^ij
  NC_K11, NC_K12, NC_K21, NC_K22,    // -2 Gamma^i_{j0} (Coriolis, Eq. 71-74)
  NC_G1A, NC_G1B, NC_G2A, NC_G2B,    // Gamma^1_11, 2 Gamma^1_12, 2 Gamma^2_12, Gamma^2_22 (Eq. 75-80)
  NC_B1, NC_B2,                      // -g_r h^ij d h_B / dx^j (topography)
  NC_COUNT
};

// Per-interface-point coefficients (structure of arrays over face points), in
// the coordinates of the face's owner side.
enum FaceCoef {
  FC_AD = 0,        // g_r h^dd / sqrt g   (a^d = sqrt(FC_AD * q^0), App. E)
  FC_P1, FC_P2,     // g_r h^{i d} / (2 sqrt g)   (pressure component, App. D)
  FC_T00, FC_T01, FC_T10, FC_T11,  // neighbour -> owner contravariant transform (App. C)
  FC_M00, FC_M01, FC_M10, FC_M11,  // sigma * (owner -> neighbour transform), applied to the flux
  FC_SIG,           // sigma = +-1: sign of the normal flux on the neighbour side
  FC_COUNT
};

// Per-node coefficients of the imaginary half of the complex-step JVP at a
// linearisation point (dfr_split.cu).
enum LinNode {
  LN_U1 = 0, LN_U2,
  LN_A11, LN_A12, LN_A22,           // Im sqrt(g)T^ij coefficient of Im q^0
  LN_S11, LN_S12, LN_S10,           // Im S^1 = s11 Im q^1 + s12 Im q^2 + s10 Im q^0
  LN_S21, LN_S22, LN_S20,
  LN_COUNT
};

// One face line = the N_s points shared by two element edges.
struct FaceLine {
  int owner, owner_edge;   // element index, edge 0=W 1=E 2=S 3=N
  int nbr, nbr_edge;
  int reversed;            // neighbour point index = N_s-1-i
  int dir;                 // owner normal direction (1 or 2)
  int owner_is_left;       // owner edge is E or N
  int pad;
};

// Small DFR constants passed by value to the kernels.
struct DfrConst {
  double D[MAX_NS][MAX_NS + 2];   // l~'_n(xi_k), Eq. (12)-(13)
  double Dg[MAX_NS][MAX_NS];      // l'_l(xi_k) on the solution points (collocation derivative)
  double lm[MAX_NS], lp[MAX_NS];  // l_k(-1), l_k(+1), Eq. (8)
  float lm32[MAX_NS], lp32[MAX_NS];  // the same rounded to FP32 (complex64-bulk form)
  double two_over_dx;             // Eq. (6)
  double gravity;
};

struct Mlp;   // learned Krylov control network (mlp.cu)

struct Ctx {
  int device = 0;
  int ne = 0, ns = 0;
  double dx = 0;
  long long nelem = 0, nodes = 0, n = 0;
  int nlines = 0;
  long long nfacepts = 0;
  sw_params prm{};
  double frame[6][3][3]{};        // per panel: centre, e1, e2
  std::vector<double> xi, wq;     // Gauss-Legendre points and weights
  std::vector<double> Dg;         // collocation derivative on the points [ns][ns]
  DfrConst dc{};
  std::vector<double> node_coef_h;  // [NC_COUNT][nodes]
  // device tables
  double* d_node_coef = nullptr;
  double* d_face_coef = nullptr;
  FaceLine* d_lines = nullptr;
  double* d_fb = nullptr;         // face flux buffer [nelem][4][3][ns]
  // Krylov workspace
  int vcap = 0;                   // rows of V allocated (m_max + 1)
  long long ldv = 0;              // leading dimension of V (>= n + MAX_NB)
  double* d_V = nullptr;
  double* d_X = nullptr;          // current augmented vector [ldv]
  int ldh = 0;                    // leading dimension of H and F (m_max + 2)
  double* d_H = nullptr;
  double* d_F = nullptr;
  double* d_expm_ws = nullptr;    // expm workspace
  double* d_partials = nullptr;   // reduction partials
  double* d_vpart = nullptr;      // partials of the epilogue dot products (2 per volume block)
  double* d_cdot = nullptr;       // V_j . V_{j-1} per basis index
  double* d_cdot2 = nullptr;      // V_j . V_{j-2} per basis index (window of three)
  double* d_scal = nullptr;       // device scalars (see kiops.cu)
  int* d_flags = nullptr;         // happy flag, happy size
  double* h_pinned = nullptr;     // pinned read-back area
  const double** d_bptr = nullptr;
  // EPI state
  double* d_Fn = nullptr;
  double* d_tmp = nullptr;
  double* d_tmp2 = nullptr;
  double* d_qhost = nullptr;     // device copy of the state of sw_epi_step_host
  double* d_R[MAX_HIST] = {};
  double* d_b[MAX_NB] = {};
  double* d_hq[MAX_HIST] = {};    // history ring: q_{n-i}
  double* d_hF[MAX_HIST] = {};
  int hist_count = 0;
  int hist_head = 0;              // slot of the most recent entry
  int m_warm = 0;                 // KIOPS warm start (0 = none)
  long long launches = 0;
  // split JVP (dfr_split.cu): coefficients of the imaginary half at the last linearisation point
  int jvp_mode = 1;                 // 0 = plain complex-step evaluation per JVP, 1 = split, 2 = split FP32 bulk
  bool linearized = false;
  double* d_lin_node = nullptr;     // [LN_COUNT][nodes]
  double* d_lin_face = nullptr;     // [18][nfacepts]
  float* d_lin_node32 = nullptr;    // FP32 copies (complex64-bulk form)
  float* d_lin_face32 = nullptr;    // [23][nfacepts]: the 18 flux-map rows, then M00, M01, M10, M11, sigma
  float* d_V32 = nullptr;           // FP32 copy of the Krylov basis [vcap][ldv] (complex64-bulk form)
  int v32_cap = 0;                  // rows allocated in d_V32
  float* d_b32 = nullptr;           // FP32 copies of nu * b_l of the current phi-function call [MAX_NB][n]
  int b32_cap = 0;                  // vectors allocated in d_b32
  // device-driven phi-function solver (kiops_graph.cu)
  int kiops_driver = 0;           // 0: controller on the host (kiops.cu), 1: on the device, one CUDA graph per call
  int orth_fused = 0;             // the GPU holds the fused orthogonalisation grid: 0 unknown, 1 yes, -1 no
  int orth_fuse_enable = 1;       // both orthogonalisation passes in one cooperative launch where it can
  void* kg = nullptr;             // its graph, state and staging (owned, kiops_graph.cu)
  // KIOPS call log and learned control
  Mlp* controller = nullptr;      // not owned
  int epi_order = 0;              // EPI order of the current call (0: direct sw_kiops_phi)
  int epi_stage = 0;              // 1 during EPI2 start-up substeps
  std::vector<float> kiops_log;   // KIOPS_LOG_FIELDS floats per call
  float prev_call[8] = {};        // log10 tau_1, m_1/m_max, m_final/m_max, substeps, rejects, krylov/m_max, valid
  float prev_h[4] = {};           // log10 of the last four h_{j+1,j} of the previous call
  // diagnostics (diag.cu)
  double* d_diag_tab = nullptr;    // sqrt g, w_m w_n, g_ij, f, h_B per node
  double* d_diag_part = nullptr;
  double* d_diag_out = nullptr;
  void* d_diag_flags = nullptr;
  std::vector<double> hB_h;        // nodal bottom (host copy)
  // event profiling (sw_profile)
  unsigned prof = 0;               // bit k: time kernels of kind k (ProfKind)
  struct ProfRec { int kind; cudaEvent_t a, b; };
  std::vector<ProfRec> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  int prof_every = 1;               // bracket every prof_every-th launch of a JVP/RHS family (sw_profile_every)
  long long prof_seen[SW_PROF_KINDS] = {};
  long long prof_count[SW_PROF_KINDS] = {};
  double prof_ms[SW_PROF_KINDS] = {};
};

// learned Krylov control (mlp.cu)
int mlp_nparam();
int mlp_nnorm();
int mlp_create(Mlp** out);
void mlp_destroy(Mlp* m);
int mlp_set(Mlp* m, const float* params, const float* norm);
int mlp_get(Mlp* m, float* params, float* bf16_as_float);
int mlp_forward(Mlp* m, const float* X, int n, float* Y, cudaStream_t s);
int mlp_step(Mlp* m, const float* X, const float* T, int n, bool adam, float lr, float* loss_host, cudaStream_t s);
int mlp_grad_host(Mlp* m, float* grad_host);
int mlp_predict_host(Mlp* m, const float* feat, float* out2, cudaStream_t s);

// event profiling helpers (capi.cu)
cudaEvent_t prof_event(Ctx& c);
void prof_record(Ctx& c, int kind, cudaEvent_t a, cudaEvent_t b);
void prof_drain(Ctx& c);
enum ProfKind {
  PK_FACE_JVP = 0, PK_VOL_JVP = 1, PK_FACE_RHS = 2, PK_VOL_RHS = 3, PK_EXPM = 4, PK_LIN = 5, PK_ORTH = 6
};
inline bool prof_on(const Ctx& c, int kind) { return (c.prof >> kind) & 1u; }
// whether this launch of a JVP or RHS kernel family is bracketed: every
// prof_every-th launch of the family while it is timed (an event pair between
// two kernels keeps the second from overlapping the first's tail, so a timed
// run that brackets fewer launches is closer to an untimed one)
inline bool prof_take(Ctx& c, int kind) {
  if (!prof_on(c, kind)) return false;
  return (c.prof_seen[kind]++ % c.prof_every) == 0;
}

// ---- multistep EPI driver pieces (capi.cu), shared with the ensemble driver
constexpr int EPI_STARTUP_SUBSTEPS = 8;   // EPI2 substeps of a start-up step (Sec. 4)
struct Coefs {                            // Eq. 34-38: b_m = sum_i a[m][i] dt R(q_{n-1-i})
  int M, P;
  double a[4][4];
};
const Coefs* coefs_for(int order);        // orders 3..6, else null
sw_kiops_opts default_opts();
int ensure_epi(Ctx& c);
int hist_slot(const Ctx& c, int i);       // slot of history entry i (1 = most recent)
int push_history(Ctx& c, const double* q, const double* F, cudaStream_t s);
void add_stats(sw_kiops_stats* acc, const sw_kiops_stats& s);

// ---- geometry / tables (geom.cpp)
int build_tables(Ctx& c);
void node_unit_xyz(const Ctx& c, double* xyz);
int bottom_coefficients(Ctx& c, const double* hB);
int fields_to_state(const Ctx& c, const double* h, const double* hB, const double* V, double* q);
void diag_tables_host(const Ctx& c, double* tab);

// ---- diagnostics (diag.cu)
int ensure_diag(Ctx& c);
int refresh_diag_bottom(Ctx& c, const double* hB);
int launch_diagnostics(Ctx& c, const double* q, const double* qref, double* zeta, double* out_host, cudaStream_t s);

// ---- DFR kernels (dfr.cu)
struct AugEpilogue {
  // out = scale * result + nu * sum_l tail_in[l] * b[l]   (b[l] may be null)
  double scale = 1.0;
  double nu = 0.0;
  int p = 0;
  const double* b[MAX_NB] = {};
  // complex64-bulk form: FP32 copies of nu * b[l] (same l); the FP32 volume
  // kernels add the b-column terms in FP32 from these (the FP64 b[l] are then
  // not read by them)
  const float* b32[MAX_NB] = {};
  // complex64-bulk form: FP32 copy of the product's input vector v (first n
  // entries; rounded to nearest), read by the FP32 kernels instead of v
  const float* v32 = nullptr;
  const double* tail_in = nullptr;  // p doubles (device)
  double* tail_out = nullptr;       // p doubles (device): (tail_in[1..p-1], 0)
  const int* skip = nullptr;        // if non-null and *skip != 0 the kernels return
  // incomplete orthogonalisation fused into the epilogue (window of two or
  // three): with dotB set, the modified Gram-Schmidt coefficients of z against
  // V_C = V_{j-2}, V_A = V_{j-1}, V_B = V_j (oldest first) are formed from the
  // dots z . V over the augmented length n + p and the stored V . V products:
  //   h0 = V_C . z,  h1 = V_A . z - h0 (V_A . V_C),
  //   h2 = V_B . z - h0 (V_B . V_C) - h1 (V_B . V_A)
  // (block partials, last block finalises); absent vectors drop their terms
  const double* dotA = nullptr;     // V_{j-1} (null for the first basis vector)
  const double* dotB = nullptr;     // V_j
  const double* dotC = nullptr;     // V_{j-2} (window of three, j >= 2)
  const double* cprev = nullptr;    // V_j . V_{j-1}
  const double* cprevC = nullptr;   // V_j . V_{j-2}
  const double* cprevAC = nullptr;  // V_{j-1} . V_{j-2}
  double* h0_out = nullptr;
  double* h1_out = nullptr;
  double* h2_out = nullptr;
  // with cdot_out set, V_j . V_{j-1} (and, window of three, V_j . V_{j-2}) are
  // formed here from the window vectors and written there, instead of being
  // read from cprev / cprevC (complex64-bulk form: the scale pass then forms
  // no dots)
  double* cdot_out = nullptr;
  double* cdot2_out = nullptr;
  double* dpart = nullptr;          // 5 doubles per block
  unsigned int* dticket = nullptr;
  long long n = 0;
};
int launch_rhs(Ctx& c, const double* q, double* F, cudaStream_t s);
int launch_jvp(Ctx& c, const double* q, const double* v, double eps, double* out,
               const AugEpilogue& ep, cudaStream_t s);
// split JVP: evaluate the real half at q, then imaginary halves for any v
int launch_linearize(Ctx& c, const double* q, cudaStream_t s);
// fp32: the imaginary half in FP32 (complex64-bulk form; needs a mode-2 linearisation)
int launch_jvp_lin(Ctx& c, const double* v, double* out, const AugEpilogue& ep, cudaStream_t s, bool fp32);
// the FP32 tangent volume kernel with bulk-copy staging of each element tile
// (dfr_tile.cu): SW_OK when launched, 1 when the grid or a pointer does not
// meet its 16-byte alignment (the caller then launches volume_tangent_kernel);
// a tile wait that gave up sets d_flags[3]
template <int NS>
int launch_volume_tile_f32(Ctx& c, const double* v, double* out, const AugEpilogue& ep, cudaStream_t s);
// the JVP with a caller-supplied interface-flux buffer (nelem * 12 * ns doubles)
int launch_jvp_fb(Ctx& c, const double* q, const double* v, double eps, double* out, double* fb,
                  cudaStream_t s);

// ---- Krylov kernels (krylov.cu)
constexpr int RED_BLOCKS = 608;   // 4 x 152 SMs
int launch_dot(Ctx& c, const double* x, const double* y, long long n, double* dst, const int* skip,
               cudaStream_t s);
int launch_norm2(Ctx& c, const double* x, long long n, double* dst, double tol, int* happy,
                 int happy_value, const int* skip, cudaStream_t s);
int launch_norm1(Ctx& c, const double* x, long long n, double* dst, cudaStream_t s);
int launch_axpy_dev(Ctx& c, double* y, const double* x, const double* alpha, long long n,
                    const int* skip, cudaStream_t s);
int launch_scale_inv(Ctx& c, double* y, const double* x, const double* s_dev, long long n,
                     const int* skip, cudaStream_t s);
// small exponential: prep builds A = t [[H_j, e_1], [0, 0]] and its 1-norm
// (device scalars), eval evaluates exp(A) into F once the host knows N and the norm
int launch_expm_prep(Ctx& c, int j, double tau, double tau_happy, cudaStream_t s);
int launch_expm_eval(Ctx& c, int N, double norm1, int* squarings, cudaStream_t s);
int launch_combine(Ctx& c, int j, long long n, cudaStream_t s);
// dst = (float)(scale * src), n entries (the complex64-bulk form's b-column copies)
int launch_to_float_scaled(Ctx& c, const double* src, float* dst, long long n, double scale, cudaStream_t s);
// fused incomplete orthogonalisation (window two or three) after an epilogue
// with dots: z -= h0 V_C + h1 V_A + h2 V_B and ||z|| -> *hsub (happy flag below
// tol), then V_next = z / *hsub, V_next . V_B -> *c_out and, with V_A given,
// V_next . V_A -> *c2_out
int launch_update_norm(Ctx& c, double* z, const double* VA, const double* VB, const double* h1, const double* h2,
                       long long N, double* hsub, double tol, int happy_value, cudaStream_t s,
                       const double* VC = nullptr, const double* h0 = nullptr);
int launch_scale_dot(Ctx& c, double* z, const double* VB, const double* hsub, long long N, double* c_out,
                     cudaStream_t s, const double* VA = nullptr, double* c2_out = nullptr, float* z32 = nullptr);
// dst = src rounded to FP32 (n entries)
int launch_to_float(Ctx& c, const double* src, float* dst, long long n, cudaStream_t s);
// both orthogonalisation passes (launch_update_norm, then launch_scale_dot with
// c_out, VA2, c2_out, z32) in one cooperative launch, where the GPU holds its
// whole grid at once (orth_fused_available); a wait past its bound sets d_flags[3]
int orth_fused_available(Ctx& c);
// the complex64-bulk form's window dots as a pass of their own (its FP32
// volume kernel forms none): the five sums over the augmented vectors, the
// modified Gram-Schmidt coefficients into the H entries, V_j . V_{j-1} and
// V_j . V_{j-2} into cdot_out, cdot2_out (orth_dots_dev)
int launch_orth_dots(Ctx& c, const double* z, const double* VB, const double* VA, const double* VC, long long N,
                     double* h0_out, double* h1_out, double* h2_out, double* cdot_out, double* cdot2_out,
                     const double* cprevAC, cudaStream_t s);
// that pass, the update pass and the scale pass (no dots, the FP32 copy z32)
// in one cooperative launch, where orth_fused_available
int launch_orth3_fused(Ctx& c, double* z, const double* VA, const double* VB, const double* VC, long long N,
                       double tol, int happy_value, double* h0p, double* h1p, double* h2p, double* hsub,
                       double* cdot_out, double* cdot2_out, const double* cprevAC, float* z32, cudaStream_t s);
int launch_orth_fused(Ctx& c, double* z, const double* VA, const double* VB, const double* h1, const double* h2,
                      long long N, double* hsub, double tol, int happy_value, const double* VC, const double* h0,
                      double* c_out, const double* VA2, double* c2_out, float* z32, cudaStream_t s);
double fp64_fma_peak_tflops();
int launch_set_tail(Ctx& c, double* x, long long n, int p, const double* vals, cudaStream_t s);
int launch_lincomb(Ctx& c, double* out, long long n, int k, const double* const* xs,
                   const double* coef, cudaStream_t s);

// ---- drivers
// use_lin: JVPs by the split path (launch_linearize must have been called at q_lin)
int kiops_run(Ctx& c, const double* q_lin, double dt, double tau_out, int nb, const double* const* b,
              const sw_kiops_opts& o, double* w, sw_kiops_stats* st, cudaStream_t s, bool use_lin);
int ensure_krylov(Ctx& c, int m_max);
// the device-driven solver (kiops_graph.cu): used by kiops_run when selected and
// applicable (split JVP, window 2 or 3, plain rule, profiling off)
bool kiops_graph_applies(const Ctx& c, const sw_kiops_opts& o, bool use_lin);
int kiops_run_graph(Ctx& c, double dt, double tau_out, int nb, const double* const* b, const sw_kiops_opts& o,
                    double* w, sw_kiops_stats* st, cudaStream_t s);
void kiops_graph_free(Ctx& c);

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? SW_OK : SW_ECUDA; }

// Programmatic dependent launch for the kernels of one Krylov iteration (face
// and volume tangent kernels, the two orthogonalisation passes): a kernel
// launched by launch_pdl can be scheduled while its predecessor on the stream
// is still running, so the launch latency between consecutive kernels is
// hidden.  Each such kernel calls pdl_wait() before its first global memory
// access of any kind (which returns once the predecessor has completed and its
// writes are visible) and pdl_trigger() to let its own successor be scheduled.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}
#endif

}  // namespace swepi

// the public context handle is the internal context
struct sw_ctx : public swepi::Ctx {};
