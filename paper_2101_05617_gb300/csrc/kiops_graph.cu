// Device-driven phi-function solver (Eq. 29): the same computation and the same
// controller as kiops_run (kiops.cu), with every decision taken on the device.
//
// One CUDA graph per context (rebuilt when the window, the number of
// phi-vectors, the form or the workspace changes) holds the whole call:
//
//   setup (nu, mu, the tail of X, beta_0 = ||X||, the controller's start)
//   WHILE not done:                                  -- substep attempts
//     start of a basis when j = 0 (beta, V_0, clear H and the flags)
//     WHILE it < m and no happy breakdown:           -- Krylov iterations
//       face and volume kernels of the JVP (augmented operator, window dots),
//       update-and-norm pass, scale-and-dot pass, it += 1
//     the exponential: A = tau [[H, e_1], [0, 0]], 8 products,
//       WHILE q < s: squaring q                      -- squarings
//     decision (KiopsController::decide and finish in one device thread),
//     the tail of X after an accepted substep, the combination of the basis
//
// The loop conditions are set with cudaGraphSetConditional by the kernels that
// know them.  Every loop is bounded on the device: at most m_max iterations
// per basis, kDevMaxSquarings squarings, kDevMaxAttempts attempts per call
// (then SW_EKRYLOV), so a graph launch always ends.  The host uploads the
// call's constants, launches the graph, copies the result and reads the
// controller state back once, at the end of the call.  Kernel-level event
// timing (sw_profile) needs the host driver: with profiling on, calls take
// kiops_run; so do calls with the learned controller or with windows other
// than 2 and 3.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "kiops_dev.h"
#include "krylov_device.cuh"
#include "swepi_internal.h"

namespace swepi {

namespace {

constexpr int kRedThreads = kPassThreads;   // threads of the reduction launches (as krylov.cu)

struct KGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  KDev* d_kd = nullptr;
  KDev* h_kd = nullptr;   // pinned staging of the call's state
  // configuration the graph was built for
  int p = -1, iop = -1, fp32 = -1, mmax = -1;
  const double* V = nullptr;
  const float* V32 = nullptr;
  const float* b32 = nullptr;
};

int grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)std::max(1LL, std::min(b, 4LL * 152 * 4));
}

// ---------------------------------------------------------------- kernels
__global__ void kg_setup_kernel(KDev* kd, KFix f) {
  double normb = 0.0;
  for (int k = 1; k <= kd->p; ++k) normb = kc_max(normb, f.scal[S_NORMB + k]);
  kd->normb = normb;
  kd->err = kc_finite(normb) ? 0 : SW_ENONFINITE;
  kd->attempts = 0;
  kd->accept = 0;
  double nu = 1.0, mu = 1.0;
  if (normb > 0 && kc_finite(normb)) {
    const int ex = (int)::ceil(::log2(normb));
    nu = ::ldexp(1.0, -ex);
    mu = ::ldexp(1.0, ex);
  }
  kd->nu = nu;
  kd->mu = mu;
  for (int l = 0; l < kd->p; ++l) f.X[f.n + l] = (l == kd->p - 1) ? mu : 0.0;
}

// complex64-bulk form: FP32 copies of nu * b_l
__global__ void kg_b32_kernel(const KDev* __restrict__ kd, KFix f) {
  if (kd->err) return;
  const double nu = kd->nu;
  for (int l = 0; l < kd->p && l < MAX_NB; ++l) {
    const double* src = kd->b[l];
    float* dst = const_cast<float*>(kd->b32[l]);
    if (!src || !dst) continue;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < f.n; i += (long long)gridDim.x * blockDim.x)
      dst[i] = (float)(nu * src[i]);
  }
}

__global__ void kg_start_kernel(KDev* kd, KFix f, cudaGraphConditionalHandle ho) {
  const double beta0 = f.scal[S_BETA0];
  kd->beta0 = beta0;
  if (!kd->err && !kc_finite(beta0)) kd->err = SW_ENONFINITE;
  sw_kiops_opts o{};
  o.tol = kd->tol;
  o.m_init = kd->m0;
  o.m_min = kd->m_min;
  o.m_max = kd->m_max;
  o.iop = 2;
  kd->K = KiopsController{};
  kd->K.start(kd->tau_end, kd->tol, beta0, o, kd->tau0, kd->m0);
  cudaGraphSetConditional(ho, (kd->err || kd->K.done()) ? 0u : 1u);
}

__global__ void kg_prep_kernel(KDev* kd, cudaGraphConditionalHandle hi) {
  if (!kd->err && ++kd->attempts > kDevMaxAttempts) kd->err = SW_EKRYLOV;
  kd->it = kd->K.j;
  kd->m_cur = kd->K.m;
  kd->skip0 = (kd->err || kd->K.j != 0) ? 1 : 0;
  cudaGraphSetConditional(hi, (!kd->err && kd->it < kd->m_cur) ? 1u : 0u);
}

// start of a basis (j = 0): H and the happy flag cleared
__global__ void kg_clear_kernel(const KDev* __restrict__ kd, KFix f) {
  if (kd->skip0) return;
  const long long total = (long long)f.ldh * f.ldh;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
    f.H[i] = 0.0;
  if (blockIdx.x == 0 && threadIdx.x < 2) f.flags[threadIdx.x] = 0;
}

__global__ void to_float_skip_kernel(const double* __restrict__ src, float* __restrict__ dst, long long n,
                                     const int* skip) {
  if (*skip) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = f64_to_f32_bits(src[i]);
}

// the complex64-bulk form's dot pass (orth_dots_dev), as the host driver runs it
template <bool W3>
__global__ void __launch_bounds__(kRedThreads) kg_dots_kernel(const KDev* __restrict__ kd, KFix f) {
  const int it = kd->it;
  const double* Vi = f.V + (long long)it * f.ldv;
  const double* Vn = Vi + f.ldv;
  const double* VA = (it >= 1) ? Vi - f.ldv : nullptr;
  const double* VC = (W3 && it >= 2) ? Vi - 2 * f.ldv : nullptr;
  double* hA = (it >= 1) ? f.H + (long long)(it - 1) * f.ldh + it : nullptr;
  double* hB = f.H + (long long)it * f.ldh + it;
  double* hC = (W3 && it >= 2) ? f.H + (long long)(it - 2) * f.ldh + it : nullptr;
  orth_dots_dev(Vn, Vi, VA, VC, f.N, f.partials, reinterpret_cast<unsigned int*>(f.flags + 8), f.flags, hC, hA, hB,
                VA ? f.cdot + it : nullptr, VC ? f.cdot2 + it : nullptr, VC ? f.cdot + it - 1 : nullptr);
}

template <bool W3>
__global__ void __launch_bounds__(kRedThreads) kg_update_kernel(const KDev* __restrict__ kd, KFix f) {
  const int it = kd->it;
  double* Vi = f.V + (long long)it * f.ldv;
  double* Vn = Vi + f.ldv;
  const double* VA = (it >= 1) ? Vi - f.ldv : nullptr;
  const double* VC = (W3 && it >= 2) ? Vi - 2 * f.ldv : nullptr;
  const double* hA = (it >= 1) ? f.H + (long long)(it - 1) * f.ldh + it : nullptr;
  const double* hB = f.H + (long long)it * f.ldh + it;
  const double* hC = (W3 && it >= 2) ? f.H + (long long)(it - 2) * f.ldh + it : nullptr;
  double* hs = f.H + (long long)(it + 1) * f.ldh + it;
  update_norm_dev(Vn, VA, Vi, hA, hB, f.N, f.partials, reinterpret_cast<unsigned int*>(f.flags + 8), hs, kd->tol,
                  f.flags, it + 1, VC, hC);
}

template <bool W3>
__global__ void __launch_bounds__(kRedThreads) kg_scale_kernel(const KDev* __restrict__ kd, KFix f) {
  const int it = kd->it;
  double* Vi = f.V + (long long)it * f.ldv;
  double* Vn = Vi + f.ldv;
  const double* hs = f.H + (long long)(it + 1) * f.ldh + it;
  const double* Vprev = (W3 && it >= 1) ? Vi - f.ldv : nullptr;
  float* z32 = f.V32 ? f.V32 + (long long)(it + 1) * f.ldv : nullptr;
  // complex64-bulk form (FP32 basis copy): the next volume kernel forms the V . V dots
  scale_dot_dev(Vn, Vi, hs, f.N, f.partials, reinterpret_cast<unsigned int*>(f.flags + 8),
                f.V32 ? nullptr : f.cdot + it + 1, f.flags, Vprev, f.cdot2 + it + 1, z32);
}

__global__ void kg_advance_kernel(KDev* kd, KFix f, cudaGraphConditionalHandle hi) {
  const int it = kd->it + 1;
  kd->it = it;
  const bool go = it < kd->m_cur && f.flags[0] == 0 && it < MAX_EXPM - 1;
  cudaGraphSetConditional(hi, go ? 1u : 0u);
}

__global__ void kg_expm_prep_kernel(KDev* kd, KFix f, cudaGraphConditionalHandle hq) {
  if (kd->err) {
    if (threadIdx.x == 0) {
      kd->N = 0;
      kd->sq = 0;
      kd->sq_i = 0;
      cudaGraphSetConditional(hq, 0u);
    }
    return;
  }
  expm_prep_body(f.H, f.ldh, kd->m_cur, kd->K.tau, kd->K.tau_end - kd->K.tau_now, f.flags, f.ws, f.scal + S_STAT);
  if (threadIdx.x == 0) {
    const int N = (int)f.scal[S_STAT + 1] + 1;
    const double nrm = f.scal[S_STAT + 5];
    int sq = kc_finite(nrm) ? expm_squarings(nrm) : -1;
    if (N < 2 || N > MAX_EXPM || sq < 0 || sq > kDevMaxSquarings) {
      kd->err = SW_ENONFINITE;
      kd->N = 0;
      sq = 0;
    } else {
      kd->N = N;
    }
    kd->sq = sq;
    kd->sq_i = 0;
    cudaGraphSetConditional(hq, (kd->N >= 2 && sq > 0) ? 1u : 0u);
  }
}

__global__ void __launch_bounds__(64) kg_expm_gemm_kernel(const KDev* __restrict__ kd, KFix f, ExpmProduct pr,
                                                          int scaling) {
  const int N = kd->N;
  const int r = blockIdx.y * 8 + threadIdx.y, c = blockIdx.x * 8 + threadIdx.x;
  if (N < 2 || r >= N || c >= N) return;
  MatEpi e = pr.e;
  if (scaling) e.alpha = ::ldexp(1.0, -kd->sq);
  expm_gemm_entry(f.ws, N, pr.c, pr.a, pr.b, e, r, c);
}

__global__ void __launch_bounds__(64) kg_expm_square_kernel(const KDev* __restrict__ kd, KFix f) {
  const int N = kd->N, q = kd->sq_i;
  const int r = blockIdx.y * 8 + threadIdx.y, c = blockIdx.x * 8 + threadIdx.x;
  if (N < 2 || q >= kd->sq || r >= N || c >= N) return;
  const MatEpi none{0, 0, 0, 0, -1, -1, -1, 1.0};
  const int src = expm_square_src(q);
  expm_gemm_entry(f.ws, N, expm_square_dst(q), src, src, none, r, c);
}

__global__ void kg_sq_advance_kernel(KDev* kd, cudaGraphConditionalHandle hq) {
  const int q = kd->sq_i + 1;
  kd->sq_i = q;
  cudaGraphSetConditional(hq, (q < kd->sq && q < kDevMaxSquarings) ? 1u : 0u);
}

__global__ void kg_expm_finish_kernel(const KDev* __restrict__ kd, KFix f) {
  const int N = kd->N;
  if (N < 2) return;
  const long long NN = (long long)N * N;
  const double* P = f.ws + expm_result_slot(kd->sq) * NN;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < NN; i += (long long)gridDim.x * blockDim.x)
    expm_finish_entry(P, N, f.F, f.ldh, f.scal + S_STAT, i);
}

// the controller's decision on the finished attempt (one thread)
__global__ void kg_decide_kernel(KDev* kd, KFix f, cudaGraphConditionalHandle ho) {
  kd->accept = 0;
  if (!kd->err) {
    const bool happy = f.flags[0] != 0;
    const int jn = happy ? f.flags[1] : kd->m_cur;
    int rc = kd->K.decide(happy, jn, f.scal[S_BETA], f.scal[S_STAT + 4], f.scal[S_STAT + 0]);
    if (rc) {
      kd->err = rc;
    } else {
      kd->accept = kd->K.accept ? 1 : 0;
      rc = kd->K.finish(kMaxSubsteps, kMaxRejects);
      if (rc) {
        kd->err = rc;
      } else if (kd->accept) {
        double tv[MAX_NB];
        kd->K.tail(kd->p, kd->mu, tv);
        for (int l = 0; l < kd->p; ++l) f.X[f.n + l] = tv[l];
      }
    }
  }
  cudaGraphSetConditional(ho, (!kd->err && !kd->K.done()) ? 1u : 0u);
}

// X = beta sum_{k < j} F[k][0] V_k (first n entries) after an accepted substep
__global__ void kg_combine_kernel(const KDev* __restrict__ kd, KFix f) {
  if (kd->err || !kd->accept) return;
  const int j = kd->K.j_used;
  __shared__ double coef[MAX_EXPM];
  for (int k = threadIdx.x; k < j; k += blockDim.x) coef[k] = f.F[(long long)k * f.ldh];
  __syncthreads();
  const double beta = f.scal[S_BETA];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < f.n; i += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < j; ++k) s = fma(coef[k], f.V[k * f.ldv + i], s);
    f.X[i] = beta * s;
  }
}

// ---------------------------------------------------------------- graph assembly
template <typename Fn>
int capture_into(cudaGraph_t gr, std::vector<cudaGraphNode_t>& deps, cudaStream_t cs, Fn fn) {
  if (cudaStreamBeginCaptureToGraph(cs, gr, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                                    cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return SW_ECUDA;
  const int rc = fn(cs);
  cudaStreamCaptureStatus status;
  const cudaGraphNode_t* d = nullptr;
  size_t nd = 0;
  const cudaError_t e1 = cudaStreamGetCaptureInfo(cs, &status, nullptr, nullptr, &d, nullptr, &nd);
  std::vector<cudaGraphNode_t> sink;
  if (e1 == cudaSuccess && d) sink.assign(d, d + nd);
  cudaGraph_t out = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(cs, &out);
  if (rc) return rc;
  if (e1 != cudaSuccess || e2 != cudaSuccess || status != cudaStreamCaptureStatusActive) return SW_ECUDA;
  deps.swap(sink);
  return SW_OK;
}

int add_while(cudaGraph_t gr, std::vector<cudaGraphNode_t>& deps, cudaGraphConditionalHandle h, cudaGraph_t* body) {
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  if (cudaGraphAddNode(&node, gr, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &np) != cudaSuccess)
    return SW_ECUDA;
  *body = np.conditional.phGraph_out[0];
  deps.assign(1, node);
  return SW_OK;
}

void release(KGraph& G) {
  if (G.exec) cudaGraphExecDestroy(G.exec);
  if (G.graph) cudaGraphDestroy(G.graph);
  G.exec = nullptr;
  G.graph = nullptr;
}

KFix make_fix(const Ctx& c, int p, bool fp32) {
  KFix f{};
  f.V = c.d_V;
  f.V32 = fp32 ? c.d_V32 : nullptr;
  f.b32 = fp32 ? c.d_b32 : nullptr;
  f.ldv = c.ldv;
  f.n = c.n;
  f.N = c.n + p;
  f.H = c.d_H;
  f.ldh = c.ldh;
  f.F = c.d_F;
  f.X = c.d_X;
  f.flags = c.d_flags;
  f.scal = c.d_scal;
  f.cdot = c.d_cdot;
  f.cdot2 = c.d_cdot2;
  f.vpart = c.d_vpart;
  f.partials = c.d_partials;
  f.ws = c.d_expm_ws;
  return f;
}

int build(Ctx& c, KGraph& G, int p, int iop, bool fp32, int mmax) {
  release(G);
  const KFix f = make_fix(c, p, fp32);
  const bool w3 = iop == 3;
  KDev* kd = G.d_kd;
  const long long n = c.n, N = c.n + p;
  cudaGraph_t g = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return SW_ECUDA;
  G.graph = g;
  cudaGraphConditionalHandle ho, hi, hq;
  if (cudaGraphConditionalHandleCreate(&ho, g, 0, cudaGraphCondAssignDefault) != cudaSuccess) return SW_ECUDA;
  std::vector<cudaGraphNode_t> top;
  int rc = capture_into(g, top, G.cap, [&](cudaStream_t s) {
    kg_setup_kernel<<<1, 1, 0, s>>>(kd, f);
    if (int r = launch_norm2(c, c.d_X, N, c.d_scal + S_BETA0, 0.0, nullptr, 0, nullptr, s)) return r;
    if (fp32) kg_b32_kernel<<<grid_for(n), 256, 0, s>>>(kd, f);
    kg_start_kernel<<<1, 1, 0, s>>>(kd, f, ho);
    return cuda_status(cudaGetLastError());
  });
  if (rc) return rc;
  cudaGraph_t attempt = nullptr, iter = nullptr, squares = nullptr;
  if ((rc = add_while(g, top, ho, &attempt))) return rc;
  if (cudaGraphConditionalHandleCreate(&hi, attempt, 0, cudaGraphCondAssignDefault) != cudaSuccess ||
      cudaGraphConditionalHandleCreate(&hq, attempt, 0, cudaGraphCondAssignDefault) != cudaSuccess)
    return SW_ECUDA;
  std::vector<cudaGraphNode_t> a;
  rc = capture_into(attempt, a, G.cap, [&](cudaStream_t s) {
    kg_prep_kernel<<<1, 1, 0, s>>>(kd, hi);
    if (int r = launch_norm2(c, c.d_X, N, c.d_scal + S_BETA, 0.0, nullptr, 0, &kd->skip0, s)) return r;
    if (int r = launch_scale_inv(c, c.d_V, c.d_X, c.d_scal + S_BETA, N, &kd->skip0, s)) return r;
    if (fp32) to_float_skip_kernel<<<grid_for(N), 256, 0, s>>>(c.d_V, c.d_V32, N, &kd->skip0);
    kg_clear_kernel<<<32, 256, 0, s>>>(kd, f);
    return cuda_status(cudaGetLastError());
  });
  if (rc) return rc;
  if ((rc = add_while(attempt, a, hi, &iter))) return rc;
  std::vector<cudaGraphNode_t> it;
  rc = capture_into(iter, it, G.cap, [&](cudaStream_t s) {
    if (int r = capture_iter_jvp(c, kd, f, fp32, w3, p, s)) return r;
    if (fp32) {   // complex64-bulk form: the dots in a pass of their own
      if (w3)
        kg_dots_kernel<true><<<RED_BLOCKS, kRedThreads, 0, s>>>(kd, f);
      else
        kg_dots_kernel<false><<<RED_BLOCKS, kRedThreads, 0, s>>>(kd, f);
    }
    if (w3) {
      kg_update_kernel<true><<<RED_BLOCKS, kRedThreads, 0, s>>>(kd, f);
      kg_scale_kernel<true><<<RED_BLOCKS, kRedThreads, 0, s>>>(kd, f);
    } else {
      kg_update_kernel<false><<<RED_BLOCKS, kRedThreads, 0, s>>>(kd, f);
      kg_scale_kernel<false><<<RED_BLOCKS, kRedThreads, 0, s>>>(kd, f);
    }
    kg_advance_kernel<<<1, 1, 0, s>>>(kd, f, hi);
    return cuda_status(cudaGetLastError());
  });
  if (rc) return rc;
  const int NE = mmax + 2;
  const dim3 eb(8, 8), eg((NE + 7) / 8, (NE + 7) / 8);
  ExpmProduct pr[8];
  expm_products(0, pr);   // the scaling 2^-s of the first product is applied on the device
  rc = capture_into(attempt, a, G.cap, [&](cudaStream_t s) {
    kg_expm_prep_kernel<<<1, 256, 0, s>>>(kd, f, hq);
    for (int k = 0; k < 8; ++k) kg_expm_gemm_kernel<<<eg, eb, 0, s>>>(kd, f, pr[k], k == 0 ? 1 : 0);
    return cuda_status(cudaGetLastError());
  });
  if (rc) return rc;
  if ((rc = add_while(attempt, a, hq, &squares))) return rc;
  std::vector<cudaGraphNode_t> sqd;
  rc = capture_into(squares, sqd, G.cap, [&](cudaStream_t s) {
    kg_expm_square_kernel<<<eg, eb, 0, s>>>(kd, f);
    kg_sq_advance_kernel<<<1, 1, 0, s>>>(kd, hq);
    return cuda_status(cudaGetLastError());
  });
  if (rc) return rc;
  rc = capture_into(attempt, a, G.cap, [&](cudaStream_t s) {
    kg_expm_finish_kernel<<<(NE * NE + 255) / 256, 256, 0, s>>>(kd, f);
    kg_decide_kernel<<<1, 1, 0, s>>>(kd, f, ho);
    kg_combine_kernel<<<grid_for(n), 256, 0, s>>>(kd, f);
    return cuda_status(cudaGetLastError());
  });
  if (rc) return rc;
  if (cudaGraphInstantiate(&G.exec, g, 0) != cudaSuccess) {
    G.exec = nullptr;
    return SW_ECUDA;
  }
  G.p = p;
  G.iop = iop;
  G.fp32 = fp32 ? 1 : 0;
  G.mmax = mmax;
  G.V = c.d_V;
  G.V32 = fp32 ? c.d_V32 : nullptr;
  G.b32 = fp32 ? c.d_b32 : nullptr;
  return SW_OK;
}

KGraph* graph_of(Ctx& c) {
  if (c.kg) return static_cast<KGraph*>(c.kg);
  KGraph* G = new (std::nothrow) KGraph();
  if (!G) return nullptr;
  if (cudaStreamCreateWithFlags(&G->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&G->d_kd, sizeof(KDev)) != cudaSuccess || cudaMallocHost(&G->h_kd, sizeof(KDev)) != cudaSuccess) {
    if (G->cap) cudaStreamDestroy(G->cap);
    if (G->d_kd) cudaFree(G->d_kd);
    delete G;
    return nullptr;
  }
  c.kg = G;
  return G;
}

}  // namespace

bool kiops_graph_applies(const Ctx& c, const sw_kiops_opts& o, bool use_lin) {
  return c.kiops_driver == 1 && use_lin && (o.iop == 2 || o.iop == 3) && !c.controller && c.prof == 0;
}

void kiops_graph_free(Ctx& c) {
  if (!c.kg) return;
  KGraph* G = static_cast<KGraph*>(c.kg);
  release(*G);
  if (G->cap) cudaStreamDestroy(G->cap);
  if (G->d_kd) cudaFree(G->d_kd);
  if (G->h_kd) cudaFreeHost(G->h_kd);
  delete G;
  c.kg = nullptr;
}

int kiops_run_graph(Ctx& c, double dt, double tau_out, int nb, const double* const* b, const sw_kiops_opts& o,
                    double* w, sw_kiops_stats* st, cudaStream_t s) {
  TraceRange trace("phi-function call (device-driven)");
  int rc = ensure_krylov(c, o.m_max);
  if (rc) return rc;
  const long long n = c.n;
  int p = nb - 1;
  const double* bk[MAX_NB + 1] = {};
  for (int k = 0; k < nb; ++k) bk[k] = b[k];
  if (p == 0) {
    p = 1;
    bk[1] = nullptr;
  }
  const long long N = n + p;
  const bool fp32 = c.jvp_mode == 2;
  if (fp32) {   // the FP32 basis copy and b-column copies (as kiops_run)
    if (c.v32_cap < c.vcap) {
      if (c.d_V32) cudaFree(c.d_V32);
      c.d_V32 = nullptr;
      c.v32_cap = 0;
      if (cudaMalloc(&c.d_V32, sizeof(float) * (size_t)c.vcap * c.ldv) != cudaSuccess) return SW_ENOMEM;
      c.v32_cap = c.vcap;
    }
    if (c.b32_cap < p) {
      if (c.d_b32) cudaFree(c.d_b32);
      c.d_b32 = nullptr;
      c.b32_cap = 0;
      if (cudaMalloc(&c.d_b32, sizeof(float) * (size_t)p * n) != cudaSuccess) return SW_ENOMEM;
      c.b32_cap = p;
    }
  }
  KGraph* G = graph_of(c);
  if (!G) return SW_ENOMEM;
  // the 1-norms of b_1..b_p and X = [b_0; 0] (the tail is set on the device)
  for (int k = 1; k <= p; ++k) {
    if (bk[k]) {
      if ((rc = launch_norm1(c, bk[k], n, c.d_scal + S_NORMB + k, s))) return rc;
    } else if (cudaMemsetAsync(c.d_scal + S_NORMB + k, 0, sizeof(double), s) != cudaSuccess) {
      return SW_ECUDA;
    }
  }
  if (bk[0]) {
    if (cudaMemcpyAsync(c.d_X, bk[0], sizeof(double) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return SW_ECUDA;
  } else if (cudaMemsetAsync(c.d_X, 0, sizeof(double) * n, s) != cudaSuccess) {
    return SW_ECUDA;
  }
  if (cudaMemsetAsync(c.d_flags + 3, 0, sizeof(int), s) != cudaSuccess) return SW_ECUDA;
  if (!G->exec || G->p != p || G->iop != o.iop || G->fp32 != (fp32 ? 1 : 0) || G->mmax != o.m_max ||
      G->V != c.d_V || G->V32 != (fp32 ? c.d_V32 : nullptr) || G->b32 != (fp32 ? c.d_b32 : nullptr)) {
    const unsigned prof = c.prof;
    c.prof = 0;   // no event records inside the graph
    rc = fp32 ? prepare_volume_tile_dev(c) : SW_OK;
    if (rc == SW_OK) rc = prepare_volume_dev(c, fp32);
    if (rc == SW_OK) {   // the device attribute query of the persistent grid, before capture too
      int sms = 0;
      rc = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device) == cudaSuccess ? SW_OK : SW_ECUDA;
    }
    if (rc == SW_OK) rc = build(c, *G, p, o.iop, fp32, o.m_max);
    c.prof = prof;
    if (rc) {
      release(*G);
      return rc;
    }
  }
  KDev& hk = *G->h_kd;
  hk = KDev{};
  hk.dt = dt;
  hk.tau_end = tau_out;
  hk.tol = o.tol;
  hk.tau0 = (o.tau_init > 0) ? std::min(o.tau_init, tau_out) : tau_out;
  hk.m0 = std::min(std::max(o.m_init, o.m_min), o.m_max);
  hk.m_min = o.m_min;
  hk.m_max = o.m_max;
  hk.p = p;
  for (int l = 0; l < p; ++l) {
    hk.b[l] = bk[p - l];
    hk.b32[l] = (fp32 && bk[p - l]) ? c.d_b32 + (long long)l * n : nullptr;
  }
  if (cudaMemcpyAsync(G->d_kd, G->h_kd, sizeof(KDev), cudaMemcpyHostToDevice, s) != cudaSuccess) return SW_ECUDA;
  if (cudaGraphLaunch(G->exec, s) != cudaSuccess) return SW_ECUDA;
  c.launches++;
  if (cudaMemcpyAsync(w, c.d_X, sizeof(double) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(G->h_kd, G->d_kd, sizeof(KDev), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(c.h_pinned + 32, c.d_flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return SW_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SW_ECUDA;
  if (reinterpret_cast<const int*>(c.h_pinned + 32)[3] != 0) return SW_ETIMEOUT;
  if (hk.err) return hk.err;
  float feat[16];
  kiops_features(c, hk.normb, hk.beta0, dt, p, feat);
  kiops_finish_call(c, hk.K, feat, o, st);
  return SW_OK;
}

}  // namespace swepi
