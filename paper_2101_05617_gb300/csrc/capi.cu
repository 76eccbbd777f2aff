// C ABI of libswepi (declared in include/swepi.h): argument checking, context
// life cycle and the multistep EPI driver (Eq. 25, 30, 34-38).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <stdexcept>
#include <vector>

#include "check.cuh"
#include "swepi_internal.h"

using namespace swepi;

namespace {
cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// The context's tables and workspace live on the device sw_init ran on; a call
// made with another device current would launch there on foreign pointers, so
// it is refused before any launch.
int check_device(const Ctx& c) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return SW_ECUDA;
  return dev == c.device ? SW_OK : SW_EINVAL;
}
}  // namespace

namespace swepi {

// EPI coefficient matrices: rows phi_1..phi_M, columns q_{n-1}..q_{n-P}
// (Eq. 30 for order 3, Eq. 36-38 for orders 4-6).
namespace {
const Coefs kEpi3 = {2, 1, {{0.0}, {2.0 / 3.0}}};
const Coefs kEpi4 = {3, 2, {{0.0, 0.0}, {-3.0 / 10.0, 3.0 / 40.0}, {32.0 / 5.0, -11.0 / 10.0}}};
const Coefs kEpi5 = {4, 3,
                     {{0.0, 0.0, 0.0}, {-4.0 / 5.0, 2.0 / 5.0, -4.0 / 45.0}, {12.0, -9.0 / 2.0, 8.0 / 9.0},
                      {3.0, 0.0, -1.0 / 3.0}}};
const Coefs kEpi6 = {4, 4,
                     {{0.0, 0.0, 0.0, 0.0},
                      {-49.0 / 60.0, 351.0 / 560.0, -359.0 / 1260.0, 367.0 / 6720.0},
                      {92.0 / 7.0, -99.0 / 14.0, 176.0 / 63.0, -1.0 / 2.0},
                      {485.0 / 21.0, -151.0 / 14.0, 23.0 / 9.0, -31.0 / 168.0}}};
}  // namespace

const Coefs* coefs_for(int order) {
  switch (order) {
    case 3: return &kEpi3;
    case 4: return &kEpi4;
    case 5: return &kEpi5;
    case 6: return &kEpi6;
    default: return nullptr;
  }
}
sw_kiops_opts default_opts() {
  sw_kiops_opts o;
  o.tol = 1e-10;
  o.m_init = 10;
  o.m_min = 10;
  o.m_max = 128;
  o.iop = 2;
  o.tau_init = 0.0;
  return o;
}

static int alloc_vec(double*& p, long long n) {
  if (p) return SW_OK;
  return cudaMalloc(&p, sizeof(double) * n) == cudaSuccess ? SW_OK : SW_ENOMEM;
}

int ensure_epi(Ctx& c) {
  int rc;
  if ((rc = alloc_vec(c.d_Fn, c.n)) || (rc = alloc_vec(c.d_tmp, c.n)) || (rc = alloc_vec(c.d_tmp2, c.n))) return rc;
  for (int i = 0; i < MAX_HIST; ++i)
    if ((rc = alloc_vec(c.d_R[i], c.n)) || (rc = alloc_vec(c.d_hq[i], c.n)) || (rc = alloc_vec(c.d_hF[i], c.n)))
      return rc;
  for (int i = 0; i < 4; ++i)
    if ((rc = alloc_vec(c.d_b[i], c.n))) return rc;
  return SW_OK;
}

// history entry i (1 = most recent) lives in slot (head - (i - 1)) mod MAX_HIST
int hist_slot(const Ctx& c, int i) { return ((c.hist_head - (i - 1)) % MAX_HIST + MAX_HIST) % MAX_HIST; }

int push_history(Ctx& c, const double* q, const double* F, cudaStream_t s) {
  c.hist_head = (c.hist_head + 1) % MAX_HIST;
  int slot = c.hist_head;
  if (cudaMemcpyAsync(c.d_hq[slot], q, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(c.d_hF[slot], F, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return SW_ECUDA;
  if (c.hist_count < MAX_HIST) c.hist_count++;
  return SW_OK;
}

void add_stats(sw_kiops_stats* acc, const sw_kiops_stats& s) {
  if (!acc) return;
  acc->substeps += s.substeps;
  acc->rejects += s.rejects;
  acc->krylov_iters += s.krylov_iters;
  acc->m_final = s.m_final;
  acc->tau_final = s.tau_final;
  acc->err_last = s.err_last;
}

}  // namespace swepi

namespace {
constexpr double kEpsJvp = 1e-30;

// KIOPS call of the EPI driver; in split mode the caller has linearised at q
int phi_call(Ctx& c, const double* q, double dt, int nb, const double* const* b, const sw_kiops_opts& o0, double* w,
             sw_kiops_stats* acc, cudaStream_t s) {
  sw_kiops_opts o = o0;
  if (c.m_warm > 0) o.m_init = c.m_warm;
  sw_kiops_stats st{};
  int rc = kiops_run(c, q, dt, 1.0, nb, b, o, w, &st, s, c.jvp_mode >= 1);
  if (rc) return rc;
  c.m_warm = st.m_final;
  add_stats(acc, st);
  return SW_OK;
}

// one exponential-Euler step (Eq. 25) of size h on q in place; F = F(q) given
int epi2_inplace(Ctx& c, double* q, const double* F, double h, const sw_kiops_opts& o, sw_kiops_stats* acc,
                 cudaStream_t s) {
  int rc;
  const double* xs[1] = {F};
  double cf[1] = {h};
  if ((rc = launch_lincomb(c, c.d_b[0], c.n, 1, xs, cf, s))) return rc;
  if (c.jvp_mode >= 1 && (rc = launch_linearize(c, q, s))) return rc;
  const double* b[2] = {nullptr, c.d_b[0]};
  if ((rc = phi_call(c, q, h, 2, b, o, c.d_tmp, acc, s))) return rc;
  const double* ys[2] = {q, c.d_tmp};
  double one[2] = {1.0, 1.0};
  return launch_lincomb(c, q, c.n, 2, ys, one, s);
}

}  // namespace

namespace swepi {
cudaEvent_t prof_event(Ctx& c) {
  if (c.prof_pool.empty()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  cudaEvent_t e = c.prof_pool.back();
  c.prof_pool.pop_back();
  return e;
}
void prof_record(Ctx& c, int kind, cudaEvent_t a, cudaEvent_t b) {
  c.prof_pending.push_back({kind, a, b});
  if (c.prof_pending.size() > 30000) prof_drain(c);
}
void prof_drain(Ctx& c) {
  std::vector<cudaEvent_t> seen;
  for (const Ctx::ProfRec& r : c.prof_pending) {
    if (cudaEventSynchronize(r.b) == cudaSuccess) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
        c.prof_count[r.kind]++;
        c.prof_ms[r.kind] += ms;
      }
    }
    seen.push_back(r.a);
    seen.push_back(r.b);
  }
  c.prof_pending.clear();
  // events are shared between consecutive records: return each once
  std::sort(seen.begin(), seen.end());
  seen.erase(std::unique(seen.begin(), seen.end()), seen.end());
  for (cudaEvent_t e : seen) c.prof_pool.push_back(e);
}
}  // namespace swepi

extern "C" {

int sw_profile(sw_ctx_t c, int enable) {
  if (!c) return SW_EINVAL;
  prof_drain(*c);
  c->prof = enable ? (1u << SW_PROF_KINDS) - 1u : 0u;
  for (int k = 0; k < SW_PROF_KINDS; ++k) {
    c->prof_count[k] = 0;
    c->prof_ms[k] = 0.0;
  }
  return SW_OK;
}

int sw_profile_kinds(sw_ctx_t c, unsigned mask) {
  if (!c || (mask >> SW_PROF_KINDS)) return SW_EINVAL;
  prof_drain(*c);
  c->prof = mask;
  for (int k = 0; k < SW_PROF_KINDS; ++k) {
    c->prof_count[k] = 0;
    c->prof_ms[k] = 0.0;
  }
  return SW_OK;
}

int sw_profile_every(sw_ctx_t c, int every) {
  if (!c || every < 1) return SW_EINVAL;
  prof_drain(*c);
  c->prof_every = every;
  for (int k = 0; k < SW_PROF_KINDS; ++k) {
    c->prof_seen[k] = 0;
    c->prof_count[k] = 0;
    c->prof_ms[k] = 0.0;
  }
  return SW_OK;
}

int sw_profile_read(sw_ctx_t c, sw_profile_stats* out) {
  if (!c || !out) return SW_EINVAL;
  prof_drain(*c);
  for (int k = 0; k < SW_PROF_KINDS; ++k) {
    out->count[k] = c->prof_count[k];
    out->ms[k] = c->prof_ms[k];
  }
  return SW_OK;
}

int sw_check_status(int* checked) {
  if (checked) *checked = kChecked ? 1 : 0;
  const unsigned w[4] = {check_word_dfr(), check_word_split(), check_word_tile(), check_word_ensemble()};
  int first = 0;
  for (unsigned v : w) {
    if (v == ~0u) return SW_ECUDA;
    if (!first && v) first = (int)v;
  }
  return first;
}

int sw_check_inject(sw_ctx_t c, int what) {
  if (!c || !kChecked || what < 0 || what > 1) return SW_EINVAL;
  if (int rc = check_device(*c)) return rc;
  FaceLine L;
  if (cudaMemcpy(&L, c->d_lines, sizeof(L), cudaMemcpyDeviceToHost) != cudaSuccess) return SW_ECUDA;
  // 1: the first interface line's owner moved past the last element; 0: moved back
  if (what == 1 && L.owner < c->nelem) L.owner += (int)c->nelem;
  if (what == 0 && L.owner >= c->nelem) L.owner -= (int)c->nelem;
  return cudaMemcpy(c->d_lines, &L, sizeof(L), cudaMemcpyHostToDevice) == cudaSuccess ? SW_OK : SW_ECUDA;
}

int sw_fp64_fma_peak(double* tflops) {
  if (!tflops) return SW_EINVAL;
  double t = fp64_fma_peak_tflops();
  if (!(t > 0)) return SW_ECUDA;
  *tflops = t;
  return SW_OK;
}


const char* sw_status_str(int status) {
  switch (status) {
    case SW_OK: return "ok";
    case SW_EINVAL: return "invalid argument";
    case SW_ENOMEM: return "out of memory";
    case SW_ECUDA: return "CUDA error";
    case SW_EKRYLOV: return "Krylov solver substep or rejection limit reached";
    case SW_ETIMEOUT: return "bounded device wait timed out";
    case SW_ENONFINITE: return "non-finite value";
    case SW_ESCRATCH: return "grid larger than the fixed scratch of sw_jvp_static_scratch";
    default: return "unknown status";
  }
}

int sw_init(int n_e, int p, const sw_params* prm, sw_ctx_t* out) {
  if (!out) return SW_EINVAL;
  *out = nullptr;
  if (!prm || n_e < 1 || n_e > 1024 || p < 0 || p > MAX_NS - 1 || prm->precision < 0 || prm->precision > 1 ||
      !(prm->radius > 0) ||
      !(prm->gravity > 0) || !std::isfinite(prm->omega))
    return SW_EINVAL;
  sw_ctx* c = new (std::nothrow) sw_ctx();
  if (!c) return SW_ENOMEM;
  cudaGetDevice(&c->device);
  c->ne = n_e;
  c->ns = p + 1;
  c->prm = *prm;
  // precision 1: the complex64-bulk form from the start (as sw_set_jvp_mode 2)
  c->jvp_mode = prm->precision == 1 ? 2 : 1;
  // the host tables of a very large grid can exceed host memory: no exception
  // may cross the C ABI
  int rc;
  try {
    rc = build_tables(*c);
  } catch (const std::bad_alloc&) {
    rc = SW_ENOMEM;
  } catch (const std::length_error&) {
    rc = SW_ENOMEM;
  } catch (...) {
    rc = SW_EINVAL;
  }
  if (rc) {
    sw_free(c);
    return rc;
  }
  *out = c;
  return SW_OK;
}

void sw_free(sw_ctx_t c) {
  if (!c) return;
  kiops_graph_free(*c);
  double* ptrs[] = {c->d_node_coef, c->d_face_coef, c->d_fb, c->d_V, c->d_X, c->d_H, c->d_F, c->d_expm_ws,
                    c->d_partials, c->d_scal, c->d_Fn, c->d_tmp, c->d_tmp2, c->d_lin_node, c->d_lin_face,
                    c->d_vpart, c->d_cdot, c->d_cdot2, c->d_diag_tab, c->d_diag_part, c->d_diag_out, c->d_qhost};
  if (c->d_diag_flags) cudaFree(c->d_diag_flags);
  if (c->d_lin_node32) cudaFree(c->d_lin_node32);
  if (c->d_lin_face32) cudaFree(c->d_lin_face32);
  if (c->d_b32) cudaFree(c->d_b32);
  if (c->d_V32) cudaFree(c->d_V32);
  for (double* p : ptrs)
    if (p) cudaFree(p);
  for (int i = 0; i < MAX_HIST; ++i) {
    if (c->d_R[i]) cudaFree(c->d_R[i]);
    if (c->d_hq[i]) cudaFree(c->d_hq[i]);
    if (c->d_hF[i]) cudaFree(c->d_hF[i]);
  }
  for (int i = 0; i < 4; ++i)
    if (c->d_b[i]) cudaFree(c->d_b[i]);
  if (c->d_lines) cudaFree(c->d_lines);
  if (c->d_flags) cudaFree(c->d_flags);
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  prof_drain(*c);
  for (cudaEvent_t e : c->prof_pool) cudaEventDestroy(e);
  delete c;
}

long long sw_num_unknowns(sw_ctx_t c) { return c ? c->n : -1; }

int sw_grid_info(sw_ctx_t c, int* n_e, int* p, double* dx) {
  if (!c) return SW_EINVAL;
  if (n_e) *n_e = c->ne;
  if (p) *p = c->ns - 1;
  if (dx) *dx = c->dx;
  return SW_OK;
}

int sw_node_xyz(sw_ctx_t c, double* xyz) {
  if (!c || !xyz) return SW_EINVAL;
  node_unit_xyz(*c, xyz);
  return SW_OK;
}

int sw_set_bottom_host(sw_ctx_t c, const double* hB) {
  if (!c || !hB) return SW_EINVAL;
  int rc = bottom_coefficients(*c, hB);
  return rc ? rc : refresh_diag_bottom(*c, hB);
}

int sw_set_bottom(sw_ctx_t c, const double* hB_dev) {
  if (!c || !hB_dev) return SW_EINVAL;
  int rc = check_device(*c);
  if (rc) return rc;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, hB_dev) != cudaSuccess) {
    cudaGetLastError();
    return SW_EINVAL;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return SW_EINVAL;
  if (at.type == cudaMemoryTypeDevice && at.device != c->device) return SW_EINVAL;
  // the topography coefficients are built by the same host routine as
  // sw_set_bottom_host from a host copy of h_B (an initialisation call)
  std::vector<double> h;
  try {
    h.resize((size_t)c->nodes);
  } catch (const std::bad_alloc&) {
    return SW_ENOMEM;
  }
  if (cudaMemcpy(h.data(), hB_dev, sizeof(double) * c->nodes, cudaMemcpyDeviceToHost) != cudaSuccess) return SW_ECUDA;
  return sw_set_bottom_host(c, h.data());
}

int sw_diagnostics(sw_ctx_t c, const double* q, double* out, double* zeta, void* stream) {
  if (!c || !q || !out) return SW_EINVAL;
  double r[6];
  int rc = check_device(*c);
  if (rc) return rc;
  rc = launch_diagnostics(*c, q, nullptr, zeta, r, as_stream(stream));
  if (rc) return rc;
  for (int k = 0; k < 4; ++k) out[k] = r[k];
  return SW_OK;
}

int sw_error_norms(sw_ctx_t c, const double* q, const double* q_ref, double* out, void* stream) {
  if (!c || !q || !q_ref || !out) return SW_EINVAL;
  double r[6];
  int rc = check_device(*c);
  if (rc) return rc;
  rc = launch_diagnostics(*c, q, q_ref, nullptr, r, as_stream(stream));
  if (rc) return rc;
  if (!(r[2] != 0) || !(r[3] > 0) || !(r[5] > 0)) return SW_ENONFINITE;
  out[0] = r[0] / r[2];
  out[1] = std::sqrt(r[1] / r[3]);
  out[2] = r[4] / r[5];
  return SW_OK;
}

int sw_state_from_fields(sw_ctx_t c, const double* h, const double* hB, const double* V, double* q) {
  if (!c || !h || !hB || !V || !q) return SW_EINVAL;
  int rc = bottom_coefficients(*c, hB);
  if (rc) return rc;
  if ((rc = refresh_diag_bottom(*c, hB))) return rc;
  return fields_to_state(*c, h, hB, V, q);
}

int sw_rhs(sw_ctx_t c, const double* q, double* F, void* stream) {
  if (!c || !q || !F || q == F) return SW_EINVAL;
  if (int rc = check_device(*c)) return rc;
  return launch_rhs(*c, q, F, as_stream(stream));
}

int sw_jvp(sw_ctx_t c, const double* q, const double* v, double eps, double* Jv, void* stream) {
  if (!c || !q || !v || !Jv || Jv == q || Jv == v || !(eps > 0) || !std::isfinite(eps)) return SW_EINVAL;
  if (int rc = check_device(*c)) return rc;
  AugEpilogue ep;
  return launch_jvp(*c, q, v, eps, Jv, ep, as_stream(stream));
}

int sw_kiops_phi(sw_ctx_t c, const double* q_lin, double dt, double tau_out, int nb, const double* const* b,
                 const sw_kiops_opts* opts, double* w, sw_kiops_stats* st, void* stream) {
  if (!c || !q_lin || !w || !b || nb < 1 || nb > MAX_NB || !std::isfinite(dt) || !(tau_out > 0)) return SW_EINVAL;
  for (int k = 0; k < nb; ++k)
    if (b[k] == w) return SW_EINVAL;
  if (w == q_lin) return SW_EINVAL;
  int rc = check_device(*c);
  if (rc) return rc;
  sw_kiops_opts o = opts ? *opts : default_opts();
  cudaStream_t s = as_stream(stream);
  c->epi_order = 0;
  c->epi_stage = 0;
  if (c->jvp_mode >= 1 && (rc = launch_linearize(*c, q_lin, s))) return rc;
  rc = kiops_run(*c, q_lin, dt, tau_out, nb, b, o, w, st, s, c->jvp_mode >= 1);
  return rc;
}

int sw_epi_reset(sw_ctx_t c) {
  if (!c) return SW_EINVAL;
  c->hist_count = 0;
  c->hist_head = 0;
  c->m_warm = 0;
  return SW_OK;
}

int sw_epi_set_history(sw_ctx_t c, int i, const double* q, const double* F, void* stream) {
  if (!c || !q || i < 1 || i > MAX_HIST) return SW_EINVAL;
  cudaStream_t s = as_stream(stream);
  int rc = check_device(*c);
  if (rc) return rc;
  rc = ensure_epi(*c);
  if (rc) return rc;
  // seeding addresses entries relative to head = 0: entry i lives in slot (0 - (i-1)) mod MAX_HIST
  c->hist_head = 0;
  int slot = hist_slot(*c, i);
  if (cudaMemcpyAsync(c->d_hq[slot], q, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return SW_ECUDA;
  if (F) {
    if (cudaMemcpyAsync(c->d_hF[slot], F, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return SW_ECUDA;
  } else if ((rc = launch_rhs(*c, c->d_hq[slot], c->d_hF[slot], s))) {
    return rc;
  }
  if (c->hist_count < i) c->hist_count = i;
  return SW_OK;
}

// ---- checkpoint of the multistep state (the history pairs of Eq. 33-38, the
// KIOPS warm start, the learned controller's previous-call features)
namespace {
constexpr char kCkMagic[8] = {'S', 'W', 'E', 'P', 'I', 'C', 'K', '1'};

struct CkHeader {
  char magic[8];
  int32_t version, ne, p, count;
  int64_t n;
  double geom[6];          // radius, gravity, omega, lambda0, phi0, alpha0
  int32_t m_warm, pad;
  float prev_call[8];
  float prev_h[4];
  uint64_t checksum;       // FNV-1a 64 over the payload that follows the header
};
static_assert(sizeof(CkHeader) == 144, "the header size the C ABI states; payload doubles stay aligned");

uint64_t fnv1a(const unsigned char* p, size_t len, uint64_t h) {
  for (size_t i = 0; i < len; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}
constexpr uint64_t kFnvBasis = 14695981039346656037ull;

size_t ck_bytes(const Ctx& c, int count) { return sizeof(CkHeader) + sizeof(double) * 2 * (size_t)c.n * count; }

void ck_geom(const Ctx& c, double g[6]) {
  g[0] = c.prm.radius;
  g[1] = c.prm.gravity;
  g[2] = c.prm.omega;
  g[3] = c.prm.lambda0;
  g[4] = c.prm.phi0;
  g[5] = c.prm.alpha0;
}
}  // namespace

int sw_epi_checkpoint_size(sw_ctx_t c, size_t* bytes) {
  if (!c || !bytes) return SW_EINVAL;
  *bytes = ck_bytes(*c, c->hist_count);
  return SW_OK;
}

int sw_epi_checkpoint_save(sw_ctx_t c, void* buf, size_t bytes, void* stream) {
  if (!c || !buf) return SW_EINVAL;
  if (bytes < ck_bytes(*c, c->hist_count)) return SW_EINVAL;
  if (int rc = check_device(*c)) return rc;
  cudaStream_t s = as_stream(stream);
  CkHeader hd{};
  std::memcpy(hd.magic, kCkMagic, sizeof(kCkMagic));
  hd.version = 1;
  hd.ne = c->ne;
  hd.p = c->ns - 1;
  hd.count = c->hist_count;
  hd.n = c->n;
  ck_geom(*c, hd.geom);
  hd.m_warm = c->m_warm;
  std::memcpy(hd.prev_call, c->prev_call, sizeof(hd.prev_call));
  std::memcpy(hd.prev_h, c->prev_h, sizeof(hd.prev_h));
  unsigned char* out = static_cast<unsigned char*>(buf);
  double* pay = reinterpret_cast<double*>(out + sizeof(CkHeader));
  const size_t vb = sizeof(double) * c->n;
  // entry i (1 = most recent): q_{n-i} then F(q_{n-i})
  for (int i = 1; i <= c->hist_count; ++i) {
    const int slot = hist_slot(*c, i);
    if (cudaMemcpyAsync(pay + (size_t)(2 * (i - 1)) * c->n, c->d_hq[slot], vb, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(pay + (size_t)(2 * (i - 1) + 1) * c->n, c->d_hF[slot], vb, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess)
      return SW_ECUDA;
  }
  if (int rc = cuda_status(cudaStreamSynchronize(s))) return rc;
  hd.checksum = fnv1a(reinterpret_cast<const unsigned char*>(pay), 2 * vb * c->hist_count, kFnvBasis);
  std::memcpy(out, &hd, sizeof(hd));
  return SW_OK;
}

int sw_epi_checkpoint_load(sw_ctx_t c, const void* buf, size_t bytes, void* stream) {
  if (!c || !buf || bytes < sizeof(CkHeader)) return SW_EINVAL;
  CkHeader hd;
  std::memcpy(&hd, buf, sizeof(hd));
  double g[6];
  ck_geom(*c, g);
  if (std::memcmp(hd.magic, kCkMagic, sizeof(kCkMagic)) != 0 || hd.version != 1 || hd.ne != c->ne ||
      hd.p != c->ns - 1 || hd.n != c->n || hd.count < 0 || hd.count > MAX_HIST ||
      std::memcmp(hd.geom, g, sizeof(g)) != 0 || bytes != ck_bytes(*c, hd.count) || hd.m_warm < 0)
    return SW_EINVAL;
  const unsigned char* in = static_cast<const unsigned char*>(buf);
  const double* pay = reinterpret_cast<const double*>(in + sizeof(CkHeader));
  const size_t vb = sizeof(double) * c->n;
  if (fnv1a(reinterpret_cast<const unsigned char*>(pay), 2 * vb * hd.count, kFnvBasis) != hd.checksum)
    return SW_EINVAL;
  if (int rc = check_device(*c)) return rc;
  if (int rc = ensure_epi(*c)) return rc;
  cudaStream_t s = as_stream(stream);
  // until every copy has landed the context holds no history: a failure here
  // leaves it as after sw_epi_reset
  c->hist_count = 0;
  c->hist_head = 0;
  c->m_warm = 0;
  for (int i = 1; i <= hd.count; ++i) {
    const int slot = hist_slot(*c, i);
    if (cudaMemcpyAsync(c->d_hq[slot], pay + (size_t)(2 * (i - 1)) * c->n, vb, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(c->d_hF[slot], pay + (size_t)(2 * (i - 1) + 1) * c->n, vb, cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
      return SW_ECUDA;
  }
  if (int rc = cuda_status(cudaStreamSynchronize(s))) return rc;
  c->hist_count = hd.count;
  c->m_warm = hd.m_warm;
  std::memcpy(c->prev_call, hd.prev_call, sizeof(hd.prev_call));
  std::memcpy(c->prev_h, hd.prev_h, sizeof(hd.prev_h));
  return SW_OK;
}

int sw_epi_step(sw_ctx_t c, int order, double dt, double* q, const sw_kiops_opts* opts, sw_kiops_stats* st,
                void* stream) {
  if (!c || !q || order < 2 || order > 6 || !std::isfinite(dt) || !(dt > 0)) return SW_EINVAL;
  if (int rc = check_device(*c)) return rc;
  TraceRange trace("EPI step");
  cudaStream_t s = as_stream(stream);
  sw_kiops_opts o = opts ? *opts : default_opts();
  int rc = ensure_epi(*c);
  if (rc) return rc;
  if (st) std::memset(st, 0, sizeof(*st));
  const long long n = c->n;
  c->epi_order = order;
  c->epi_stage = 0;
  if ((rc = launch_rhs(*c, q, c->d_Fn, s))) return rc;
  if (order == 2) {
    rc = epi2_inplace(*c, q, c->d_Fn, dt, o, st, s);
    if (rc) return rc;
    return cuda_status(cudaStreamSynchronize(s));
  }
  const Coefs* A = coefs_for(order);
  const int P = A->P, M = A->M;
  if (c->hist_count < P) {
    // start-up: EPI2 with N_sub smaller steps (Sec. 4)
    if ((rc = push_history(*c, q, c->d_Fn, s))) return rc;
    const double h = dt / EPI_STARTUP_SUBSTEPS;
    c->epi_stage = 1;
    for (int k = 0; k < EPI_STARTUP_SUBSTEPS; ++k) {
      if (k > 0 && (rc = launch_rhs(*c, q, c->d_Fn, s))) return rc;
      if ((rc = epi2_inplace(*c, q, c->d_Fn, h, o, st, s))) return rc;
    }
    c->epi_stage = 0;
    return cuda_status(cudaStreamSynchronize(s));
  }
  // remainders R(q_{n-i}) = F(q_{n-i}) - F_n - J_n (q_{n-i} - q_n)  (Eq. 33)
  const bool split = c->jvp_mode >= 1;
  if (split && (rc = launch_linearize(*c, q, s))) return rc;
  for (int i = 1; i <= P; ++i) {
    int slot = hist_slot(*c, i);
    const double* d1[2] = {c->d_hq[slot], q};
    double c1[2] = {1.0, -1.0};
    if ((rc = launch_lincomb(*c, c->d_tmp, n, 2, d1, c1, s))) return rc;
    AugEpilogue ep;
    // the remainder is a small difference of large terms: its JVP stays FP64 in every mode
    rc = split ? launch_jvp_lin(*c, c->d_tmp, c->d_tmp2, ep, s, false)
               : launch_jvp(*c, q, c->d_tmp, kEpsJvp, c->d_tmp2, ep, s);
    if (rc) return rc;
    const double* d2[3] = {c->d_hF[slot], c->d_Fn, c->d_tmp2};
    double c2[3] = {1.0, -1.0, -1.0};
    if ((rc = launch_lincomb(*c, c->d_R[i - 1], n, 3, d2, c2, s))) return rc;
  }
  // b_1 = dt F_n + v_1, b_m = v_m with v_m = sum_i alpha_{m,i} dt R_i  (Eq. 34-35)
  for (int m = 0; m < M; ++m) {
    const double* xs[MAX_HIST + 1];
    double cf[MAX_HIST + 1];
    int k = 0;
    if (m == 0) { xs[k] = c->d_Fn; cf[k] = dt; ++k; }
    for (int i = 0; i < P; ++i) { xs[k] = c->d_R[i]; cf[k] = A->a[m][i] * dt; ++k; }
    if ((rc = launch_lincomb(*c, c->d_b[m], n, k, xs, cf, s))) return rc;
  }
  const double* b[MAX_NB] = {nullptr};
  for (int m = 0; m < M; ++m) b[m + 1] = c->d_b[m];
  if ((rc = phi_call(*c, q, dt, M + 1, b, o, c->d_tmp, st, s))) return rc;
  if ((rc = push_history(*c, q, c->d_Fn, s))) return rc;
  const double* ys[2] = {q, c->d_tmp};
  double one[2] = {1.0, 1.0};
  if ((rc = launch_lincomb(*c, q, n, 2, ys, one, s))) return rc;
  return cuda_status(cudaStreamSynchronize(s));
}

int sw_epi_step_host(sw_ctx_t c, int order, double dt, double* q_host, const sw_kiops_opts* opts,
                     sw_kiops_stats* st, void* stream) {
  if (!c || !q_host) return SW_EINVAL;
  cudaStream_t s = as_stream(stream);
  int rc = alloc_vec(c->d_qhost, c->n);
  if (rc) return rc;
  if (cudaMemcpyAsync(c->d_qhost, q_host, sizeof(double) * c->n, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return SW_ECUDA;
  if ((rc = sw_epi_step(c, order, dt, c->d_qhost, opts, st, stream))) return rc;
  if (cudaMemcpyAsync(q_host, c->d_qhost, sizeof(double) * c->n, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return SW_ECUDA;
  return cuda_status(cudaStreamSynchronize(s));
}

int sw_epi_coefficients(int order, int* M, int* P, double* A) {
  const Coefs* cf = coefs_for(order);
  if (!cf || !M || !P || !A) return SW_EINVAL;
  *M = cf->M;
  *P = cf->P;
  for (int m = 0; m < cf->M; ++m)
    for (int i = 0; i < cf->P; ++i) A[m * cf->P + i] = cf->a[m][i];
  return SW_OK;
}

long long sw_kernel_launches(sw_ctx_t c) { return c ? c->launches : -1; }

// sw_mlp_t is an opaque handle to a swepi::Mlp
static Mlp* as_mlp(sw_mlp_t m) { return reinterpret_cast<Mlp*>(m); }

int sw_mlp_create(sw_mlp_t* out) {
  if (!out) return SW_EINVAL;
  *out = nullptr;
  Mlp* m = nullptr;
  int rc = mlp_create(&m);
  if (rc) return rc;
  *out = reinterpret_cast<sw_mlp_t>(m);
  return SW_OK;
}

void sw_mlp_free(sw_mlp_t m) { mlp_destroy(as_mlp(m)); }

int sw_mlp_set_params(sw_mlp_t m, const float* params, const float* norm) {
  if (!m) return SW_EINVAL;
  return mlp_set(as_mlp(m), params, norm);
}

int sw_mlp_get_params(sw_mlp_t m, float* params, float* bf16_params) {
  if (!m) return SW_EINVAL;
  return mlp_get(as_mlp(m), params, bf16_params);
}

int sw_mlp_forward(sw_mlp_t m, const float* X, int n, float* Y, void* stream) {
  if (!m || !X || !Y || n < 1 || n > (1 << 30)) return SW_EINVAL;
  return mlp_forward(as_mlp(m), X, n, Y, as_stream(stream));
}

int sw_mlp_gradient(sw_mlp_t m, const float* X, const float* T, int n, float* grad, float* loss, void* stream) {
  if (!m || !X || !T || !grad || n < 1) return SW_EINVAL;
  cudaStream_t s = as_stream(stream);
  float l = 0.f;
  int rc = mlp_step(as_mlp(m), X, T, n, false, 0.f, &l, s);
  if (rc) return rc;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SW_ECUDA;
  if (loss) *loss = l;
  return mlp_grad_host(as_mlp(m), grad);
}

int sw_mlp_train(sw_mlp_t m, const float* X, const float* T, int n, int steps, float lr, float* loss, void* stream) {
  if (!m || !X || !T || n < 1 || steps < 0 || !(lr > 0)) return SW_EINVAL;
  cudaStream_t s = as_stream(stream);
  for (int k = 0; k < steps; ++k) {
    float l = 0.f;
    int rc = mlp_step(as_mlp(m), X, T, n, true, lr, loss ? &l : nullptr, s);
    if (rc) return rc;
    if (loss) {
      if (cudaStreamSynchronize(s) != cudaSuccess) return SW_ECUDA;
      loss[k] = l;
    }
  }
  return cuda_status(cudaStreamSynchronize(s));
}

int sw_set_controller(sw_ctx_t c, sw_mlp_t m) {
  if (!c) return SW_EINVAL;
  c->controller = as_mlp(m);
  return SW_OK;
}

int sw_kiops_log(sw_ctx_t c, float* out, int max_records) {
  if (!c || max_records < 0 || (max_records > 0 && !out)) return SW_EINVAL;
  const int have = (int)(c->kiops_log.size() / KIOPS_LOG_FIELDS);
  const int k = have < max_records ? have : max_records;
  if (k > 0) std::memcpy(out, c->kiops_log.data(), sizeof(float) * KIOPS_LOG_FIELDS * k);
  return have;
}

int sw_kiops_log_clear(sw_ctx_t c) {
  if (!c) return SW_EINVAL;
  c->kiops_log.clear();
  return SW_OK;
}

int sw_set_kiops_driver(sw_ctx_t c, int driver) {
  if (!c || driver < 0 || driver > 1) return SW_EINVAL;
  c->kiops_driver = driver;
  return SW_OK;
}

int sw_set_orth_fused(sw_ctx_t c, int enable, int* active_out) {
  if (!c || enable < 0 || enable > 1) return SW_EINVAL;
  if (int rc = check_device(*c)) return rc;
  c->orth_fuse_enable = enable;
  if (active_out) *active_out = (enable && swepi::orth_fused_available(*c)) ? 1 : 0;
  return SW_OK;
}

int sw_set_jvp_mode(sw_ctx_t c, int mode) {
  if (!c || mode < 0 || mode > 2) return SW_EINVAL;
  if (mode != c->jvp_mode) c->linearized = false;
  c->jvp_mode = mode;
  return SW_OK;
}

int sw_linearize(sw_ctx_t c, const double* q, void* stream) {
  if (!c || !q) return SW_EINVAL;
  if (int rc = check_device(*c)) return rc;
  return launch_linearize(*c, q, as_stream(stream));
}

int sw_jvp_linearized(sw_ctx_t c, const double* v, double* Jv, void* stream) {
  if (!c || !v || !Jv || v == Jv) return SW_EINVAL;
  if (!c->linearized) return SW_EINVAL;
  if (int rc = check_device(*c)) return rc;
  AugEpilogue ep;
  return launch_jvp_lin(*c, v, Jv, ep, as_stream(stream), c->jvp_mode == 2);
}

}  // extern "C"
