"""phi-function linear combinations w = sum_k tau^k phi_k(tau A) b_k (Eq. 29)
by an adaptive Krylov projection with incomplete orthogonalisation and
substepping (the KIOPS scheme the paper relies on, Sec. 4).  Plain numpy FP64;
the small exponential uses scipy.linalg.expm as a library primitive.

Test infrastructure only (see ``oracle/__init__.py``).

The paper defers the algorithm to its reference [10], which is not available
here; the steps below are this project's written reading, shared as a
specification by the CUDA driver:

 1. Augmentation: with nu = 2^-ceil(log2 max_k ||b_k||_1) (k >= 1) and
    mu = 1/nu, the operator A~[x; y] = [A x + nu (y_1 b_p + ... + y_p b_1);
    (y_2, ..., y_p, 0)] and start vector [b_0; 0, .., 0, mu] give
    exp(tau A~)[b_0; mu e_p] = [w(tau); mu (tau^{p-1}/(p-1)!, .., tau, 1)].
 2. Each substep starts a new basis from the current augmented vector
    (beta = its 2-norm) and runs Arnoldi; the new vector is orthogonalised
    against the last `iop` basis vectors only (modified Gram-Schmidt, oldest
    first).  ||z|| < tol is a happy breakdown.
 3. After j vectors: F = expm(tau [[H_j, e_1], [0, 0]]); the error estimate is
    err = beta h_{j+1,j} |F[j-1, j]|, and omega = (tau_end/tau) err / (tol beta_0)
    with beta_0 the 2-norm of the initial augmented vector (relative tolerance).
 4. Accept if omega <= 1.2.  New step proposals: order q = j/4 unless the
    previous try was rejected at the same m with another tau (then
    q = max(1, log(omega/omega_old)/log(tau/tau_old))); kappa = 2 unless the
    previous try was rejected at the same tau with another m (then
    kappa = max(1.1, (omega/omega_old)^(1/(m_old - m)))).
    tau_opt = tau (0.8/omega)^(1/q) clamped to [tau/5, 5 tau] and to the
    remaining interval; m_opt = ceil(j + log(omega/0.8)/log kappa) clamped to
    [max(m_min, floor(3m/4)), min(m_max, ceil(4m/3))].
    With `remaining` the time left after this try (from the substep start if
    rejected, from its end if accepted) and tau_same = min(tau, remaining):
    change tau (keep m) if m ceil(remaining/tau_opt) <= m_opt
    ceil(remaining/tau_same) or if j == m_max, else change m (keep tau_same).
 5. On acceptance: w = beta V_j F[0:j, 0] (first n entries), tau_now += tau,
    tail = mu (tau_now^{p-1}/(p-1)!, ..., tau_now, 1).  On a happy breakdown
    the projection is exact: tau is set to the remaining interval and the
    substep is accepted.
 6. A rejection that keeps m reuses the basis; one that grows m continues
    Arnoldi from the existing vectors; one that shrinks m truncates the basis.
"""
import math

import numpy as np
import scipy.linalg

DELTA = 1.2
GAMMA = 0.8


class KiopsError(RuntimeError):
    pass


def kiops(tau_out, matvec, b, tol=1e-10, m_init=10, m_min=10, m_max=128, iop=2,
          tau_init=None, max_substeps=10000, max_rejects=10000, trace=None):
    """Return (w, stats) with w = sum_k tau_out^k phi_k(tau_out A) b_k (Eq. 29; the
    steps listed in the module docstring).

    matvec(x) returns A x for a length-n vector x; b is a list [b_0, .., b_p]
    (p >= 0; p == 0 is padded with a zero b_1).  `trace`, if a list, receives one
    dict per substep attempt (for comparing decision sequences)."""
    b = [np.asarray(x, dtype=float) for x in b]
    if len(b) == 1:
        b.append(np.zeros_like(b[0]))
    n = b[0].size
    p = len(b) - 1
    norm_b = max(np.sum(np.abs(x)) for x in b[1:])
    if norm_b > 0:
        ex = math.ceil(math.log2(norm_b))
        nu, mu = 2.0 ** (-ex), 2.0 ** ex
    else:
        nu, mu = 1.0, 1.0

    def aug_matvec(x):
        z = np.empty(n + p)
        top = matvec(x[:n])
        for l in range(p):                     # y_{l+1} multiplies b_{p-l}
            top = top + nu * x[n + l] * b[p - l]
        z[:n] = top
        z[n:n + p - 1] = x[n + 1:n + p]
        z[n + p - 1] = 0.0
        return z

    x = np.zeros(n + p)
    x[:n] = b[0]
    x[n + p - 1] = mu
    beta0 = np.linalg.norm(x)
    tau_end = float(tau_out)
    tau_now = 0.0
    tau = tau_end if tau_init is None or tau_init <= 0 else min(float(tau_init), tau_end)
    m = int(min(max(m_init, m_min), m_max))
    V = np.zeros((m_max + 1, n + p))
    H = np.zeros((m_max + 1, m_max + 1))
    j = 0
    beta = 0.0
    omega = None
    prev = None                 # (m, tau, omega) of the previous rejected try
    krylov = substeps = rejects = 0
    last_err = 0.0
    while tau_now < tau_end:
        if j == 0:
            beta = np.linalg.norm(x)
            V[0] = x / beta
            H[:] = 0.0
        happy = False
        while j < m:
            z = aug_matvec(V[j])
            krylov += 1
            for i in range(max(0, j - iop + 1), j + 1):
                H[i, j] = np.dot(V[i], z)
                z = z - H[i, j] * V[i]
            s = np.linalg.norm(z)
            if s < tol:
                happy = True
                j += 1
                break
            H[j + 1, j] = s
            V[j + 1] = z / s
            j += 1
        if happy:
            tau = tau_end - tau_now
        Ht = np.zeros((j + 1, j + 1))
        Ht[:j, :j] = H[:j, :j]
        Ht[0, j] = 1.0
        F = scipy.linalg.expm(tau * Ht)
        if happy:
            omega = 0.0
            accept = True
            m_new, tau_new = m, tau
            err = 0.0
        else:
            err = beta * H[j, j - 1] * abs(F[j - 1, j])
            omega = (tau_end / tau) * err / (tol * beta0)
            if not math.isfinite(omega):
                raise KiopsError("non-finite error estimate")
            accept = omega <= DELTA
            if prev is not None and prev[0] == m and prev[1] != tau:
                order = max(1.0, math.log(omega / prev[2]) / math.log(tau / prev[1]))
            else:
                order = j / 4.0
            if prev is not None and prev[1] == tau and prev[0] != m:
                kappa = max(1.1, (omega / prev[2]) ** (1.0 / (prev[0] - m)))
            else:
                kappa = 2.0
            remaining = tau_end - tau_now if not accept else tau_end - (tau_now + tau)
            tau_same = min(remaining, tau)
            if omega > 0:
                tau_opt = tau * (GAMMA / omega) ** (1.0 / order)
            else:
                tau_opt = 5 * tau
            tau_opt = min(remaining, max(tau / 5, min(5 * tau, tau_opt)))
            if omega > 0:
                m_opt = math.ceil(j + math.log(omega / GAMMA) / math.log(kappa))
            else:
                m_opt = m_min
            m_opt = max(m_min, min(m_max, max(math.floor(3 * m / 4), min(m_opt, math.ceil(4 * m / 3)))))
            if j == m_max:
                m_new, tau_new = m, tau_opt
            else:
                cost_tau = m * math.ceil(remaining / tau_opt) if tau_opt > 0 else 0
                cost_m = m_opt * math.ceil(remaining / tau_same) if tau_same > 0 else 0
                if cost_tau <= cost_m:
                    m_new, tau_new = m, tau_opt
                else:
                    m_new, tau_new = m_opt, tau_same
        last_err = err
        if trace is not None:
            trace.append(dict(j=j, m=m, tau=tau, omega=omega, accept=accept, happy=happy,
                              m_new=m_new, tau_new=tau_new, beta=beta,
                              hsub=0.0 if happy else H[j, j - 1], Fjj=0.0 if happy else F[j - 1, j]))
        if accept:
            w = beta * (V[:j, :n].T @ F[:j, 0])
            tau_now += tau
            x = np.zeros(n + p)
            x[:n] = w
            for l in range(p):
                k = p - 1 - l                       # tail entry l holds tau_now^k / k!
                x[n + l] = mu * tau_now ** k / math.factorial(k)
            substeps += 1
            j = 0
            prev = None
            if substeps > max_substeps:
                raise KiopsError("substep limit")
        else:
            rejects += 1
            prev = (m, tau, omega)
            if rejects > max_rejects:
                raise KiopsError("rejection limit")
            if m_new < j:
                j = m_new                           # truncate the basis
        m = int(m_new)
        if tau_now < tau_end:
            tau = min(tau_new, tau_end - tau_now) if tau_new > 0 else tau_end - tau_now
    stats = dict(substeps=substeps, rejects=rejects, krylov_iters=krylov, m_final=m,
                 tau_final=tau, err_last=last_err)
    return x[:n].copy(), stats
