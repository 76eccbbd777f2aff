// Replays a sequence of phi-solver attempts through the library's host-side
// controller (KiopsController) and prints every decision, so that a CPU test
// can compare the controller with the oracle's decisions on the same inputs.
//
// stdin:  tau_end tol beta0 m_min m_max tau0 m0
//         then one line per attempt: happy j beta h_{j+1,j} F[j-1][j]
// stdout: per attempt: m tau accept m_new tau_new omega tau_now_after
//         last line:   krylov substeps rejects m_final status
#include <cstdio>

#include "../paper_2101_05617_gb300/csrc/kiops_ctl.h"

int main() {
  double tau_end, tol, beta0, tau0;
  int m_min, m_max, m0;
  if (std::scanf("%lf %lf %lf %d %d %lf %d", &tau_end, &tol, &beta0, &m_min, &m_max, &tau0, &m0) != 7) return 2;
  sw_kiops_opts o{};
  o.tol = tol;
  o.m_min = m_min;
  o.m_max = m_max;
  o.m_init = m0;
  o.iop = 2;
  swepi::KiopsController K;
  K.start(tau_end, tol, beta0, o, tau0, m0);
  int happy, j;
  double beta, hsub, fjj;
  int status = 0;
  while (!K.done() && std::scanf("%d %d %lf %lf %lf", &happy, &j, &beta, &hsub, &fjj) == 5) {
    const int m_before = K.m;
    const double tau_before = K.tau;
    status = K.decide(happy != 0, j, beta, hsub, fjj);
    if (status) break;
    const int accept = K.accept ? 1 : 0;
    const int m_new = K.m_new;
    const double tau_new = K.tau_new, omega = K.happy ? 0.0 : K.last_omega;
    status = K.finish(swepi::kMaxSubsteps, swepi::kMaxRejects);
    std::printf("%d %.17g %d %d %.17g %.17g %.17g\n", m_before, tau_before, accept, m_new, tau_new, omega,
                K.tau_now);
    if (status) break;
  }
  std::printf("%d %d %d %d %d\n", K.krylov, K.substeps, K.rejects, K.m, status);
  return 0;
}
