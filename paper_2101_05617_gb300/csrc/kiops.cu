// Adaptive Krylov phi-function solver (Eq. 29) with incomplete
// orthogonalisation and substepping, and the multistep EPI driver (Eq. 25, 30,
// 34-38).  Host control code: every vector operation is a kernel of this
// library; the host only reads a handful of device scalars once per substep
// attempt to take the accept/reject and step-size decisions.
//
// Controller reading (the paper defers the algorithm to its reference [10]):
//  * augmentation with nu = 2^-ceil(log2 max_k ||b_k||_1), mu = 1/nu: the
//    operator [x; y] -> [dt J x + nu (y_1 b_p + .. + y_p b_1); (y_2, .., y_p, 0)]
//    and the start vector [b_0; 0, .., 0, mu];
//  * each substep builds a fresh basis from the current augmented vector; the
//    new vector is orthogonalised against the last `iop` basis vectors
//    (modified Gram-Schmidt, oldest first; windows of two and three fused into
//    the JVP epilogue and two vector passes); ||z|| < tol is a happy breakdown,
//    after which the projection is exact and the rest of the interval is taken;
//  * err = beta h_{j+1,j} |F[j-1, j]| with F = exp(tau [[H_j, e_1], [0, 0]])
//    (device exponential, krylov.cu; the host reads the order and 1-norm of
//    the matrix to choose the number of squarings),
//    omega = (tau_end / tau) err / (tol beta_0), beta_0 = ||[b_0; mu e_p]||;
//  * accept when omega <= 1.2; new tau from the order estimate (j/4, or
//    measured from two tries at equal m), new m from the growth estimate (2, or
//    measured from two tries at equal tau), safety factor 0.8, tau in
//    [tau/5, 5 tau], m in [max(m_min, floor(3m/4)), min(m_max, ceil(4m/3))];
//    change whichever of tau or m costs fewer projected products, tau on ties
//    or when j == m_max.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "kiops_ctl.h"
#include "swepi_internal.h"

namespace swepi {

namespace {
constexpr double kEpsJvp = 1e-30;

int read_back(Ctx& c, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(c.h_pinned, c.d_scal, sizeof(double) * 32, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return SW_ECUDA;
  e = cudaMemcpyAsync(c.h_pinned + 32, c.d_flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return SW_ECUDA;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return SW_ECUDA;
  if (c.prof) prof_drain(c);
  return SW_OK;
}
const int* pinned_flags(const Ctx& c) { return reinterpret_cast<const int*>(c.h_pinned + 32); }
// flags[3]: a bounded wait of a staged volume kernel gave up (dfr_tile.cu)
bool wait_gave_up(const Ctx& c) { return pinned_flags(c)[3] != 0; }

void free_ptr(double*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}
}  // namespace

int ensure_krylov(Ctx& c, int m_max) {
  if (c.vcap >= m_max + 1 && c.d_V) return SW_OK;
  free_ptr(c.d_V);
  free_ptr(c.d_X);
  free_ptr(c.d_H);
  free_ptr(c.d_F);
  free_ptr(c.d_expm_ws);
  c.ldv = ((c.n + MAX_NB + 31) / 32) * 32;
  c.vcap = m_max + 1;
  c.ldh = m_max + 2;
  if (cudaMalloc(&c.d_V, sizeof(double) * c.ldv * c.vcap) != cudaSuccess) return SW_ENOMEM;
  if (cudaMalloc(&c.d_X, sizeof(double) * c.ldv) != cudaSuccess) return SW_ENOMEM;
  if (cudaMalloc(&c.d_H, sizeof(double) * c.ldh * c.ldh) != cudaSuccess) return SW_ENOMEM;
  if (cudaMalloc(&c.d_F, sizeof(double) * c.ldh * c.ldh) != cudaSuccess) return SW_ENOMEM;
  if (cudaMalloc(&c.d_expm_ws, sizeof(double) * 8 * 160 * 160) != cudaSuccess) return SW_ENOMEM;
  if (!c.d_partials && cudaMalloc(&c.d_partials, sizeof(double) * 5 * RED_BLOCKS) != cudaSuccess) return SW_ENOMEM;
  if (!c.d_vpart && cudaMalloc(&c.d_vpart, sizeof(double) * 5 * (c.nelem + 1)) != cudaSuccess) return SW_ENOMEM;
  free_ptr(c.d_cdot);
  if (cudaMalloc(&c.d_cdot, sizeof(double) * c.ldh) != cudaSuccess) return SW_ENOMEM;
  free_ptr(c.d_cdot2);
  if (cudaMalloc(&c.d_cdot2, sizeof(double) * c.ldh) != cudaSuccess) return SW_ENOMEM;
  if (!c.d_scal && cudaMalloc(&c.d_scal, sizeof(double) * 64) != cudaSuccess) return SW_ENOMEM;
  if (!c.d_flags) {
    if (cudaMalloc(&c.d_flags, sizeof(int) * 16) != cudaSuccess) return SW_ENOMEM;
    if (cudaMemset(c.d_flags, 0, sizeof(int) * 16) != cudaSuccess) return SW_ECUDA;
  }
  if (!c.h_pinned && cudaMallocHost(&c.h_pinned, sizeof(double) * 64) != cudaSuccess) return SW_ENOMEM;
  if (cudaMemset(c.d_V, 0, sizeof(double) * c.ldv * c.vcap) != cudaSuccess) return SW_ECUDA;
  return SW_OK;
}

int kiops_run(Ctx& c, const double* q_lin, double dt, double tau_out, int nb, const double* const* b,
              const sw_kiops_opts& o, double* w, sw_kiops_stats* st, cudaStream_t s, bool use_lin) {
  if (nb < 1 || nb > MAX_NB || !(tau_out > 0) || o.m_min < 1 || o.m_max < o.m_min || o.m_max > 150 || o.iop < 1 ||
      !(o.tol > 0))
    return SW_EINVAL;
  if (kiops_graph_applies(c, o, use_lin)) return kiops_run_graph(c, dt, tau_out, nb, b, o, w, st, s);
  TraceRange trace("phi-function call");
  int rc = ensure_krylov(c, o.m_max);
  if (rc) return rc;
  const long long n = c.n;
  int p = nb - 1;
  const double* bk[MAX_NB + 1] = {};
  for (int k = 0; k < nb; ++k) bk[k] = b[k];
  if (p == 0) { p = 1; bk[1] = nullptr; }
  const long long N = n + p;

  // scaling of the augmented operator
  for (int k = 1; k <= p; ++k) {
    if (bk[k]) {
      if ((rc = launch_norm1(c, bk[k], n, c.d_scal + S_NORMB + k, s))) return rc;
    } else if (cudaMemsetAsync(c.d_scal + S_NORMB + k, 0, sizeof(double), s) != cudaSuccess) {
      return SW_ECUDA;
    }
  }
  if (cudaMemsetAsync(c.d_flags + 3, 0, sizeof(int), s) != cudaSuccess) return SW_ECUDA;
  // the pass and epilogue tickets, in case a wait that gave up left them mid-count
  if (cudaMemsetAsync(c.d_flags + 8, 0, sizeof(int) * 2, s) != cudaSuccess) return SW_ECUDA;
  // X = [b_0; 0 .. 0 mu]
  if (bk[0]) {
    if (cudaMemcpyAsync(c.d_X, bk[0], sizeof(double) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return SW_ECUDA;
  } else if (cudaMemsetAsync(c.d_X, 0, sizeof(double) * n, s) != cudaSuccess) {
    return SW_ECUDA;
  }
  if ((rc = read_back(c, s))) return rc;
  double normb = 0.0;
  for (int k = 1; k <= p; ++k) normb = std::max(normb, c.h_pinned[S_NORMB + k]);
  if (!std::isfinite(normb)) return SW_ENONFINITE;
  double nu = 1.0, mu = 1.0;
  if (normb > 0) {
    int ex = (int)std::ceil(std::log2(normb));
    nu = std::ldexp(1.0, -ex);
    mu = std::ldexp(1.0, ex);
  }
  double tail[MAX_NB] = {};
  tail[p - 1] = mu;
  if ((rc = launch_set_tail(c, c.d_X, n, p, tail, s))) return rc;
  if ((rc = launch_norm2(c, c.d_X, N, c.d_scal + S_BETA0, 0.0, nullptr, 0, nullptr, s))) return rc;
  if ((rc = read_back(c, s))) return rc;
  const double beta0 = c.h_pinned[S_BETA0];
  if (!std::isfinite(beta0)) return SW_ENONFINITE;

  AugEpilogue ep;
  ep.scale = dt;
  ep.nu = nu;
  ep.p = p;
  for (int l = 0; l < p; ++l) ep.b[l] = bk[p - l];
  ep.skip = c.d_flags;
  if (use_lin && c.jvp_mode == 2) {
    // complex64-bulk form: the operator's b-column terms in FP32, from nu * b_l
    // rounded once per call (the FP32 volume kernels read these instead)
    if (c.b32_cap < p) {
      if (c.d_b32) cudaFree(c.d_b32);
      c.d_b32 = nullptr;
      c.b32_cap = 0;
      if (cudaMalloc(&c.d_b32, sizeof(float) * (size_t)p * n) != cudaSuccess) return SW_ENOMEM;
      c.b32_cap = p;
    }
    for (int l = 0; l < p; ++l) {
      if (!ep.b[l]) continue;
      float* dst = c.d_b32 + (long long)l * n;
      if ((rc = launch_to_float_scaled(c, ep.b[l], dst, n, nu, s))) return rc;
      ep.b32[l] = dst;
    }
  }

  const double tau_end = tau_out;
  double tau = (o.tau_init > 0) ? std::min(o.tau_init, tau_end) : tau_end;
  int m = std::min(std::max(o.m_init, o.m_min), o.m_max);

  // per-call features (learned control input and log record)
  float feat[16];
  kiops_features(c, normb, beta0, dt, p, feat);
  if (c.controller) {
    // learned initial (tau, m); the omega test below still accepts or rejects
    // every substep, and a non-finite prediction leaves the plain rule
    float pred[2];
    if ((rc = mlp_predict_host(c.controller, feat, pred, s))) return rc;
    if (std::isfinite(pred[0]) && std::isfinite(pred[1])) {
      double lt = std::min(0.0, std::max(std::log(1e-3), (double)pred[0]));
      tau = tau_end * std::exp(lt);
      m = std::min(o.m_max, std::max(o.m_min, (int)std::lround(pred[1] * o.m_max)));
    }
  }
  KiopsController K;
  K.start(tau_end, o.tol, beta0, o, tau, m);
  double* V = c.d_V;
  const long long ldv = c.ldv;
  // complex64-bulk form with a fused window: an FP32 copy of the basis, written
  // by the scale pass with each new vector, feeds the FP32 kernels
  const bool use32 = use_lin && c.jvp_mode == 2 && (o.iop == 2 || o.iop == 3);
  const bool fused = c.orth_fuse_enable && orth_fused_available(c);
  if (use32 && c.v32_cap < c.vcap) {
    if (c.d_V32) cudaFree(c.d_V32);
    c.d_V32 = nullptr;
    c.v32_cap = 0;
    if (cudaMalloc(&c.d_V32, sizeof(float) * (size_t)c.vcap * ldv) != cudaSuccess) return SW_ENOMEM;
    c.v32_cap = c.vcap;
  }

  while (!K.done()) {
    TraceRange attempt("substep attempt");
    const int j = K.j, m_cur = K.m;
    if (j == 0) {
      if ((rc = launch_norm2(c, c.d_X, N, c.d_scal + S_BETA, 0.0, nullptr, 0, nullptr, s))) return rc;
      if ((rc = launch_scale_inv(c, V, c.d_X, c.d_scal + S_BETA, N, nullptr, s))) return rc;
      if (use32 && (rc = launch_to_float(c, V, c.d_V32, N, s))) return rc;
      if (cudaMemsetAsync(c.d_flags, 0, sizeof(int) * 2, s) != cudaSuccess) return SW_ECUDA;
      if (cudaMemsetAsync(c.d_H, 0, sizeof(double) * c.ldh * c.ldh, s) != cudaSuccess) return SW_ECUDA;
    }
    for (int it = j; it < m_cur; ++it) {
      double* Vi = V + it * ldv;
      double* Vn = V + (it + 1) * ldv;
      ep.tail_in = Vi + n;
      ep.tail_out = Vn + n;
      if (o.iop == 2 || o.iop == 3) {
        // orthogonalisation fused into the JVP epilogue (dots) and two passes
        double* hB = c.d_H + (long long)it * c.ldh + it;
        double* hA = (it >= 1) ? c.d_H + (long long)(it - 1) * c.ldh + it : nullptr;
        double* hC = (o.iop == 3 && it >= 2) ? c.d_H + (long long)(it - 2) * c.ldh + it : nullptr;
        // the window: V_{j-1}, V_j, V_{j-2}
        const double* wA = (it >= 1) ? V + (it - 1) * ldv : nullptr;
        const double* wC = hC ? V + (it - 2) * ldv : nullptr;
        // complex64-bulk form: the FP32 volume kernel forms no dots; a pass of
        // their own (orth_dots_dev) takes them and the V . V products
        ep.dotA = use32 ? nullptr : wA;
        ep.dotB = use32 ? nullptr : Vi;
        ep.dotC = use32 ? nullptr : wC;
        ep.cprev = c.d_cdot + it;
        ep.cprevC = c.d_cdot2 + it;
        ep.cprevAC = (it >= 1) ? c.d_cdot + it - 1 : nullptr;
        ep.h0_out = hC;
        ep.h1_out = hA;
        ep.h2_out = hB;
        ep.dpart = c.d_vpart;
        ep.dticket = (unsigned int*)(c.d_flags + 9);
        ep.n = n;
        ep.v32 = use32 ? c.d_V32 + it * ldv : nullptr;
        ep.cdot_out = ep.cdot2_out = nullptr;
        rc = use_lin ? launch_jvp_lin(c, Vi, Vn, ep, s, c.jvp_mode == 2) : launch_jvp(c, q_lin, Vi, kEpsJvp, Vn, ep, s);
        if (rc) return rc;
        double* hs = c.d_H + (long long)(it + 1) * c.ldh + it;
        if (use32) {
          double* cd = wA ? c.d_cdot + it : nullptr;
          double* cd2 = wC ? c.d_cdot2 + it : nullptr;
          const double* cpac = wC ? c.d_cdot + it - 1 : nullptr;
          float* z32 = c.d_V32 + (it + 1) * ldv;
          if (fused) {
            rc = launch_orth3_fused(c, Vn, wA, Vi, wC, N, o.tol, it + 1, hC, hA, hB, hs, cd, cd2, cpac, z32, s);
          } else if (!(rc = launch_orth_dots(c, Vn, Vi, wA, wC, N, hC, hA, hB, cd, cd2, cpac, s)) &&
                     !(rc = launch_update_norm(c, Vn, wA, Vi, hA, hB, N, hs, o.tol, it + 1, s, wC, hC))) {
            rc = launch_scale_dot(c, Vn, Vi, hs, N, nullptr, s, nullptr, nullptr, z32);
          }
          if (rc) return rc;
          continue;
        }
        // V_{j+1} . V_{j-1} is needed by the window of three two iterations later
        const double* Vprev = (o.iop == 3 && it >= 1) ? V + (it - 1) * ldv : nullptr;
        double* cn = c.d_cdot + it + 1;
        if (fused) {
          rc = launch_orth_fused(c, Vn, wA, Vi, hA, hB, N, hs, o.tol, it + 1, wC, hC, cn, Vprev,
                                 c.d_cdot2 + it + 1, nullptr, s);
        } else if (!(rc = launch_update_norm(c, Vn, wA, Vi, hA, hB, N, hs, o.tol, it + 1, s, wC, hC))) {
          rc = launch_scale_dot(c, Vn, Vi, hs, N, cn, s, Vprev, c.d_cdot2 + it + 1, nullptr);
        }
        if (rc) return rc;
        continue;
      }
      ep.dotA = ep.dotB = ep.dotC = nullptr;
      ep.v32 = nullptr;
      ep.cdot_out = ep.cdot2_out = nullptr;
      rc = use_lin ? launch_jvp_lin(c, Vi, Vn, ep, s, c.jvp_mode == 2) : launch_jvp(c, q_lin, Vi, kEpsJvp, Vn, ep, s);
      if (rc) return rc;
      for (int i = std::max(0, it - o.iop + 1); i <= it; ++i) {
        double* h = c.d_H + (long long)i * c.ldh + it;
        if ((rc = launch_dot(c, V + i * ldv, Vn, N, h, c.d_flags, s))) return rc;
        if ((rc = launch_axpy_dev(c, Vn, V + i * ldv, h, N, c.d_flags, s))) return rc;
      }
      double* hs = c.d_H + (long long)(it + 1) * c.ldh + it;
      if ((rc = launch_norm2(c, Vn, N, hs, o.tol, c.d_flags, it + 1, c.d_flags, s))) return rc;
      if ((rc = launch_scale_inv(c, Vn, Vn, hs, N, c.d_flags, s))) return rc;
    }
    if ((rc = launch_expm_prep(c, m_cur, K.tau, tau_end - K.tau_now, s))) return rc;
    if ((rc = read_back(c, s))) return rc;
    {
      const int Ne = (int)c.h_pinned[S_STAT + 1] + 1;
      if ((rc = launch_expm_eval(c, Ne, c.h_pinned[S_STAT + 5], nullptr, s))) return rc;
    }
    if ((rc = read_back(c, s))) return rc;
    if (wait_gave_up(c)) return SW_ETIMEOUT;
    const int* fl = pinned_flags(c);
    const bool happy = fl[0] != 0;
    if ((rc = K.decide(happy, happy ? fl[1] : m_cur, c.h_pinned[S_BETA], c.h_pinned[S_STAT + 4],
                       c.h_pinned[S_STAT + 0])))
      return rc;
    if (K.accept) {
      if ((rc = launch_combine(c, K.j_used, n, s))) return rc;
    }
    if ((rc = K.finish(kMaxSubsteps, kMaxRejects))) return rc;
    if (K.accept) {
      double tv[MAX_NB];
      K.tail(p, mu, tv);
      if ((rc = launch_set_tail(c, c.d_X, n, p, tv, s))) return rc;
    }
  }
  if (cudaMemcpyAsync(w, c.d_X, sizeof(double) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return SW_ECUDA;
  kiops_finish_call(c, K, feat, o, st);
  return cuda_status(cudaGetLastError());
}

}  // namespace swepi
