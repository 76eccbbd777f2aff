// Host-side controller of the adaptive phi-function solver (one instance per
// solve): substep size tau and Krylov size m, accept/reject from the error
// estimate, and the bookkeeping of one call.  Shared by the single-grid driver
// (kiops.cu) and the ensemble driver (ensemble.cu); the reading it implements
// is written out at the top of kiops.cu.
#pragma once

#include <algorithm>
#include <cmath>

#include "swepi_internal.h"

#ifdef __CUDACC__
#define SW_HD __host__ __device__
#else
#define SW_HD
#endif

namespace swepi {

// plain helpers usable on the host (the glibc functions) and on the device;
// min and max take the same branches as std::min and std::max (NaN included)
SW_HD inline double kc_min(double a, double b) { return (b < a) ? b : a; }
SW_HD inline double kc_max(double a, double b) { return (a < b) ? b : a; }
SW_HD inline int kc_mini(int a, int b) { return (b < a) ? b : a; }
SW_HD inline int kc_maxi(int a, int b) { return (a < b) ? b : a; }
SW_HD inline bool kc_finite(double x) { return x - x == 0.0; }   // false for NaN and +-inf

constexpr int kMaxSubsteps = 100000;   // per call: beyond this the solver gives up (SW_EKRYLOV)
constexpr int kMaxRejects = 100000;
// device scalar slots of a context (Ctx::d_scal): beta of the current substep,
// beta_0, the exponential's statistics (S_STAT + 0..5, see krylov_device.cuh)
// and the 1-norms of b_1..b_p
constexpr int S_BETA = 0, S_BETA0 = 1, S_STAT = 8, S_NORMB = 16;

struct KiopsController {
  static constexpr double kDelta = 1.2;   // acceptance threshold on omega
  static constexpr double kGamma = 0.8;   // safety factor of the step proposals

  // configuration
  double tau_end = 1.0, tol = 1e-10, beta0 = 1.0;
  int m_min = 10, m_max = 128;
  // state of the solve
  double tau_now = 0.0, tau = 1.0;
  int m = 10, j = 0;
  bool have_prev = false;
  int prev_m = 0;
  double prev_tau = 0.0, prev_omega = 0.0;
  double last_omega = 0.0, last_order = 1.0, last_err = 0.0;
  int krylov = 0, substeps = 0, rejects = 0;
  double tau_first = -1.0, tau_star = -1.0;
  int m_first = 0;
  double hist_h[4] = {0, 0, 0, 0};
  int nh = 0;
  // outcome of the last attempt
  bool accept = false, happy = false;
  int m_new = 0, j_used = 0;
  double tau_new = 0.0;

  SW_HD void start(double tau_out, double tol_, double beta0_, const sw_kiops_opts& o, double tau0, int m0) {
    tau_end = tau_out;
    tol = tol_;
    beta0 = beta0_;
    m_min = o.m_min;
    m_max = o.m_max;
    tau = tau0;
    m = m0;
  }

  SW_HD bool done() const { return tau_now >= tau_end; }

  // Decide after an attempt with Krylov size jnew (happy breakdown or m).
  // beta: norm of the substep's start vector; hsub = h_{j+1,j}; Fjj = F[j-1][j].
  SW_HD int decide(bool happy_, int jnew, double beta, double hsub, double Fjj) {
    happy = happy_;
    krylov += jnew - j;
    j = jnew;
    double err = 0.0;
    if (happy) {
      tau = tau_end - tau_now;
      accept = true;
      m_new = m;
      tau_new = tau;
    } else {
      hist_h[nh % 4] = hsub;
      ++nh;
      err = beta * hsub * ::fabs(Fjj);
      const double omega = (tau_end / tau) * err / (tol * beta0);
      if (!kc_finite(omega)) return SW_ENONFINITE;
      accept = omega <= kDelta;
      last_omega = omega;
      const double order = (have_prev && prev_m == m && prev_tau != tau)
                               ? kc_max(1.0, ::log(omega / prev_omega) / ::log(tau / prev_tau))
                               : j / 4.0;
      last_order = order;
      const double kappa = (have_prev && prev_tau == tau && prev_m != m)
                               ? kc_max(1.1, ::pow(omega / prev_omega, 1.0 / (prev_m - m)))
                               : 2.0;
      const double remaining = accept ? tau_end - (tau_now + tau) : tau_end - tau_now;
      const double tau_same = kc_min(remaining, tau);
      double tau_opt = (omega > 0) ? tau * ::pow(kGamma / omega, 1.0 / order) : 5 * tau;
      tau_opt = kc_min(remaining, kc_max(tau / 5, kc_min(5 * tau, tau_opt)));
      int m_opt = (omega > 0) ? (int)::ceil(j + ::log(omega / kGamma) / ::log(kappa)) : m_min;
      m_opt = kc_maxi(m_min, kc_mini(m_max, kc_maxi((int)::floor(3.0 * m / 4.0),
                                                    kc_mini(m_opt, (int)::ceil(4.0 * m / 3.0)))));
      if (j == m_max) {
        m_new = m;
        tau_new = tau_opt;
      } else {
        const double cost_tau = tau_opt > 0 ? m * ::ceil(remaining / tau_opt) : 0.0;
        const double cost_m = tau_same > 0 ? m_opt * ::ceil(remaining / tau_same) : 0.0;
        if (cost_tau <= cost_m) {
          m_new = m;
          tau_new = tau_opt;
        } else {
          m_new = m_opt;
          tau_new = tau_same;
        }
      }
      if (!accept) {
        have_prev = true;
        prev_m = m;
        prev_tau = tau;
        prev_omega = omega;
      }
    }
    last_err = err;
    j_used = j;
    if (accept && tau_first < 0) {
      tau_first = tau;
      m_first = j;
      // largest first substep the error model admits: omega ~ tau^order
      tau_star = (happy || last_omega <= 0) ? tau_end : tau * ::pow(kGamma / last_omega, 1.0 / last_order);
      tau_star = kc_min(tau_end, kc_max(tau, tau_star));
    }
    return SW_OK;
  }

  // After the caller has combined the basis (on acceptance): advance the state.
  // Returns the new tau_now.  Limits on substeps / rejections -> SW_EKRYLOV.
  SW_HD int finish(int max_substeps, int max_rejects) {
    if (accept) {
      tau_now += tau;
      ++substeps;
      j = 0;
      have_prev = false;
      if (substeps > max_substeps) return SW_EKRYLOV;
    } else {
      ++rejects;
      if (rejects > max_rejects) return SW_EKRYLOV;
      if (m_new < j) j = m_new;
    }
    m = m_new;
    if (tau_now < tau_end) tau = (tau_new > 0) ? kc_min(tau_new, tau_end - tau_now) : tau_end - tau_now;
    return SW_OK;
  }

  // tail of the augmented vector after acceptance: mu (tau_now^{p-1}/(p-1)!, ..., tau_now, 1)
  SW_HD void tail(int p, double mu, double* out) const {
    for (int l = 0; l < p; ++l) {
      const int k = p - 1 - l;
      double f = 1.0;
      for (int t = 2; t <= k; ++t) f *= t;
      out[l] = mu * ::pow(tau_now, k) / f;
    }
  }
};

// per-call features (learned control input and log record): log10 of the
// largest 1-norm of b_1..b_p and of beta_0, the previous call's outcome, the
// last four h_{j+1,j} of the previous call, EPI order and stage, log10 dt, p
inline void kiops_features(const Ctx& c, double normb, double beta0, double dt, int p, float feat[16]) {
  feat[0] = (float)std::log10(std::max(normb, 1e-300));
  feat[1] = (float)std::log10(std::max(beta0, 1e-300));
  for (int k = 0; k < 6; ++k) feat[2 + k] = c.prev_call[k];
  for (int k = 0; k < 4; ++k) feat[8 + k] = c.prev_h[k];
  feat[12] = (float)c.epi_order;
  feat[13] = (float)c.epi_stage;
  feat[14] = (float)((dt > 0) ? std::log10(dt) : 0.0);
  feat[15] = (float)p;
}

// log record of a finished call (features, then log(tau_1/tau_end), m_1/m_max,
// Krylov iterations, rejections, substeps, m_final/m_max, log(tau_star/tau_end)
// with tau_star the largest first substep the error model admits), the
// previous-call features of the next one, and the call's statistics
inline void kiops_finish_call(Ctx& c, const KiopsController& K, const float feat[16], const sw_kiops_opts& o,
                              sw_kiops_stats* st) {
  const double tau_end = K.tau_end;
  float rec[KIOPS_LOG_FIELDS];
  for (int k = 0; k < 16; ++k) rec[k] = feat[k];
  rec[16] = (float)std::log(K.tau_first / tau_end);
  rec[17] = (float)K.m_first / o.m_max;
  rec[18] = (float)K.krylov;
  rec[19] = (float)K.rejects;
  rec[20] = (float)K.substeps;
  rec[21] = (float)K.m / o.m_max;
  rec[22] = (float)std::log(K.tau_star / tau_end);
  if (c.kiops_log.size() + KIOPS_LOG_FIELDS <= KIOPS_LOG_MAX * KIOPS_LOG_FIELDS)
    c.kiops_log.insert(c.kiops_log.end(), rec, rec + KIOPS_LOG_FIELDS);
  c.prev_call[0] = (float)std::log10(K.tau_first / tau_end);
  c.prev_call[1] = rec[17];
  c.prev_call[2] = rec[21];
  c.prev_call[3] = (float)K.substeps;
  c.prev_call[4] = (float)K.rejects;
  c.prev_call[5] = (float)K.krylov / o.m_max;
  for (int k = 0; k < 4; ++k) {
    double hv = (K.nh > k) ? K.hist_h[(K.nh - 1 - k) % 4] : 0.0;
    c.prev_h[k] = (hv > 0) ? (float)std::log10(hv) : 0.0f;
  }
  if (st) {
    st->substeps = K.substeps;
    st->rejects = K.rejects;
    st->krylov_iters = K.krylov;
    st->m_final = K.m;
    st->tau_final = K.tau;
    st->err_last = K.last_err;
  }
}

}  // namespace swepi
