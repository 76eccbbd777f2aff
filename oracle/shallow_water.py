"""Semi-discrete DFR right-hand side of the covariant shallow-water equations
(paper Eq. 1-2, Sec. 3, App. C-E) in complex FP64, and the complex-step JVP
(Eq. 28).  Plain numpy, vectorised only over elements and points.

Test infrastructure only (see ``oracle/__init__.py``).

State layout: q[var, panel, e2, e1, k2, k1] with var 0 = sqrt(g) H,
var i = sqrt(g) H u^i (the tensor density q^mu of App. D), x^i angular
cubed-sphere coordinates in [-pi/4, pi/4], H = h - h_B.

Readings of passages the paper leaves open:
  * metric at interface points: evaluated analytically at the point;
  * each interface flux is computed once, in the coordinates of the side with
    the lower panel index (within a panel: the lower element), and handed to
    the other side through the App. C contravariant transform;
  * AUSM split functions (App. D cites them without printing them): basic
    AUSM, M+- = +-(M+-1)^2/4 and P+- = P (M+-1)^2 (2-+M)/4 for |M| <= 1,
    M+- = (M +- |M|)/2 and P+- = P (1 +- sign M)/2 otherwise;  '+' is the
    side with the lower coordinate;
  * complex arguments: max/min/|.|/sign and the |M| <= 1 test act on the real
    part (a tie Re = 0 takes the '<= 0' branch), sqrt is the principal root;
  * the term sqrt(g) Gamma^i_jk g_r h^jk H^2 / 2 of Eq. (2) is dropped: the
    contraction h^jk Gamma^i_jk vanishes on the cubed sphere (App. B);
  * the bottom gradient dh_B/dx^j is the element-local collocation derivative
    of the nodal h_B.
"""
import numpy as np

from . import geometry as geo
from . import dfr

EDGES = ('W', 'E', 'S', 'N')


class Grid:
    """6 x n_e x n_e elements of N_s x N_s Gauss-Legendre points (Sec. 3.2)."""

    def __init__(self, ne, ns, rotation=(0.0, 0.0, 0.0), radius=geo.RADIUS,
                 gravity=geo.GRAVITY, omega=geo.OMEGA):
        self.ne, self.ns = ne, ns
        self.a, self.gr, self.omega = radius, gravity, omega
        self.rotation = tuple(float(r) for r in rotation)
        self.dx = (np.pi / 2) / ne
        self.xi, self.w = dfr.gauss_legendre(ns)
        self.D = dfr.flux_derivative_matrix(ns)
        self.lm, self.lp = dfr.trace_rows(ns)
        self.Dg = dfr.collocation_derivative_matrix(ns)
        self.angles = geo.panel_angles(*self.rotation)
        self.frames = [geo.panel_frame(*ang) for ang in self.angles]

        # 1-D coordinate of (element, point) along an axis: [ne, ns]
        self.x_line = (-np.pi / 4 + (np.arange(ne)[:, None] + 0.5) * self.dx
                       + self.xi[None, :] * self.dx / 2)
        shp = (6, ne, ne, ns, ns)
        self.x1 = np.broadcast_to(self.x_line[None, None, :, None, :], shp).copy()
        self.x2 = np.broadcast_to(self.x_line[None, :, None, :, None], shp).copy()
        X, Y = np.tan(self.x1), np.tan(self.x2)
        self.m = geo.metric(X, Y, self.a)
        self.gam_t = [[np.empty(shp) for _ in range(2)] for _ in range(2)]
        for p in range(6):
            _, php, alp = self.angles[p]
            G = geo.christoffel_time(X[p], Y[p], php, alp, self.omega)
            for i in range(2):
                for j in range(2):
                    self.gam_t[i][j][p] = G[i][j]
        self.gam_s = geo.christoffel_space(X, Y)
        self.set_bottom(np.zeros(shp))

    # ------------------------------------------------------------------ nodes
    @property
    def n_unknowns(self):
        return 3 * 6 * self.ne ** 2 * self.ns ** 2

    def node_xyz(self):
        """Unit position vectors of all nodes (App. B): [3, 6, ne, ne, ns, ns]."""
        out = np.empty((3,) + self.x1.shape)
        for p in range(6):
            out[:, p] = geo.unit_position(self.x1[p], self.x2[p], self.frames[p])
        return out

    def set_bottom(self, hB):
        """Nodal h_B and its element-local collocation gradient (the bottom term of Eq. 2; reading in the
        module docstring)."""
        self.hB = np.asarray(hB, dtype=float).reshape(self.x1.shape)
        s = 2.0 / self.dx
        self.dhB1 = s * np.einsum('kl,pefjl->pefjk', self.Dg, self.hB)    # d/dx^1 along k1
        self.dhB2 = s * np.einsum('kl,pefli->pefki', self.Dg, self.hB)    # d/dx^2 along k2

    def quad_weights(self):
        """w_m w_n sqrt(g) of Eq. (42), per node."""
        return self.w[None, None, None, :, None] * self.w[None, None, None, None, :] * self.m['sqrtg']

    # --------------------------------------------------------------- faces
    def face_metric_x1(self, i_face):
        """Metric (Eq. 67-70, evaluated at the point) on the x^1 = const line i_face (0..ne) at all (e2, k2) points."""
        x1 = -np.pi / 4 + i_face * self.dx
        X = np.tan(np.full(self.x_line.shape, x1))
        Y = np.tan(self.x_line)
        return geo.metric(X, Y, self.a)

    def face_metric_x2(self, i_face):
        """Metric (Eq. 67-70, evaluated at the point) on the x^2 = const line i_face (0..ne)."""
        x2 = -np.pi / 4 + i_face * self.dx
        X = np.tan(self.x_line)
        Y = np.tan(np.full(self.x_line.shape, x2))
        return geo.metric(X, Y, self.a)


# ---------------------------------------------------------------- helpers
def _gt0(z):
    return np.real(z) > 0


def _max0(z):
    return np.where(_gt0(z), z, 0)


def _min0(z):
    return np.where(_gt0(z), 0, z)


def _sign(z):
    return np.where(_gt0(z), 1.0, -1.0)


def split_mach(M):
    """(M+, M-) of basic AUSM (reading of App. D, Eq. 138)."""
    inside = np.abs(np.real(M)) <= 1
    mp = np.where(inside, 0.25 * (M + 1) ** 2, 0.5 * (M + M * _sign(M)))
    mm = np.where(inside, -0.25 * (M - 1) ** 2, 0.5 * (M - M * _sign(M)))
    return mp, mm


def split_pressure(M):
    """(P+/P, P-/P) of basic AUSM (reading of App. D, Eq. 139)."""
    inside = np.abs(np.real(M)) <= 1
    bp = np.where(inside, 0.25 * (M + 1) ** 2 * (2 - M), 0.5 * (1 + _sign(M)))
    bm = np.where(inside, 0.25 * (M - 1) ** 2 * (2 + M), 0.5 * (1 - _sign(M)))
    return bp, bm


def ausm_flux(qL, qR, d, sqrtg, hdd, h1d, h2d, gr):
    """AUSM interface flux sqrt(g) T^{mu d} (App. D, Eq. 137-143).

    qL, qR: sequences of the three components q^0, q^1, q^2 on the lower ('+')
    and upper ('-') side, in the same coordinates; d in {1, 2} the normal
    direction; metric values at the interface point.
    """
    def side(q):
        H = q[0] / sqrtg
        a = np.sqrt(hdd * gr * H + 0j)          # a^d (App. E)
        M = (q[d] / q[0]) / a                    # Froude number u^d / a^d
        A = [a * q[0], a * q[1], a * q[2]]       # A^{mu d} = q^mu sqrt(g) H a / q^0
        Pc = gr * q[0] ** 2 / (2 * sqrtg)
        P = [0 * q[0], Pc * h1d, Pc * h2d]       # P^{mu d} = g_r h^{mu d} (q^0)^2 / (2 sqrt g)
        return M, A, P

    ML, AL, PL = side(qL)
    MR, AR, PR = side(qR)
    mpL, _ = split_mach(ML)
    _, mmR = split_mach(MR)
    bpL, _ = split_pressure(ML)
    _, bmR = split_pressure(MR)
    Mh = mpL + mmR                               # Eq. (138), second splitting Eq. (140)
    return [_max0(Mh) * AL[mu] + bpL * PL[mu] + _min0(Mh) * AR[mu] + bmR * PR[mu]
            for mu in range(3)]                  # Eq. (141)-(143)


def _edge_get(arr, edge, p, ne, ns):
    """Values on a panel edge ordered by increasing along-edge coordinate:
    arr is the W/E trace array [.., 6, ne, ne, ns] (for 'W'/'E') or the S/N one."""
    if edge == 'E':
        v = arr[:, p, :, ne - 1, :]      # [3, e2, k2]
    elif edge == 'W':
        v = arr[:, p, :, 0, :]
    elif edge == 'N':
        v = arr[:, p, ne - 1, :, :]      # [3, e1, k1]
    else:
        v = arr[:, p, 0, :, :]
    return v.reshape(v.shape[0], ne * ns)


def _edge_set(arr, edge, p, ne, ns, val):
    val = val.reshape(val.shape[0], ne, ns)
    if edge == 'E':
        arr[:, p, :, ne - 1, :] = val
    elif edge == 'W':
        arr[:, p, :, 0, :] = val
    elif edge == 'N':
        arr[:, p, ne - 1, :, :] = val
    else:
        arr[:, p, 0, :, :] = val


def rhs(grid, q):
    """F(q): the semi-discrete right-hand side (Eq. 14 in 2-D, Sec. 3.2) of
    Eq. (1)-(2) in quasi-flux form.  q may be real or complex."""
    g = grid
    ne, ns, gr = g.ne, g.ns, g.gr
    q = np.asarray(q).reshape((3, 6, ne, ne, ns, ns))
    q = q.astype(np.complex128)
    m = g.m
    q0, q1, q2 = q[0], q[1], q[2]

    # interior fluxes sqrt(g) T^{mu j} at the solution points (Eq. 136)
    pre = gr * q0 ** 2 / (2 * m['sqrtg'])
    hij = [[m['h11'], m['h12']], [m['h12'], m['h22']]]
    qv = [q0, q1, q2]
    F = [[None, None] for _ in range(3)]
    for j in range(2):
        F[0][j] = qv[j + 1]
        for i in range(2):
            F[i + 1][j] = qv[i + 1] * qv[j + 1] / q0 + pre * hij[i][j]

    # sources: right-hand side of Eq. (2) divided into q variables
    S = [np.zeros_like(q0), None, None]
    dhB = [g.dhB1, g.dhB2]
    for i in range(2):
        s = np.zeros_like(q0)
        for j in range(2):
            s = s - 2 * g.gam_t[i][j] * qv[j + 1]                       # -2 sqrt(g) Gamma^i_j0 H u^j
            for k in range(2):
                s = s - g.gam_s[i][j][k] * qv[j + 1] * qv[k + 1] / q0   # -sqrt(g) Gamma^i_jk H u^j u^k
            s = s - gr * q0 * hij[i][j] * dhB[j]                       # -sqrt(g) H g_r h^ij dh_B/dx^j
        S[i + 1] = s

    # traces at the element ends (Eq. 7 at xi = -1, +1)
    tW = np.einsum('k,vpefjk->vpefj', g.lm, q)
    tE = np.einsum('k,vpefjk->vpefj', g.lp, q)
    tS = np.einsum('k,vpefkj->vpefj', g.lm, q)
    tN = np.einsum('k,vpefkj->vpefj', g.lp, q)

    FW = np.zeros_like(tW)
    FE = np.zeros_like(tW)
    FS = np.zeros_like(tW)
    FN = np.zeros_like(tW)

    # interior faces inside each panel: the lower element is the '+' side
    for i in range(1, ne):
        mf = g.face_metric_x1(i)          # [e2, k2]
        fl = ausm_flux(tE[:, :, :, i - 1], tW[:, :, :, i], 1, mf['sqrtg'], mf['h11'], mf['h11'], mf['h12'], gr)
        for mu in range(3):
            FE[mu, :, :, i - 1] = fl[mu]
            FW[mu, :, :, i] = fl[mu]
        mf = g.face_metric_x2(i)          # [e1, k1]
        fl = ausm_flux(tN[:, :, i - 1], tS[:, :, i], 2, mf['sqrtg'], mf['h22'], mf['h12'], mf['h22'], gr)
        for mu in range(3):
            FN[mu, :, i - 1] = fl[mu]
            FS[mu, :, i] = fl[mu]

    # panel interfaces (App. C)
    t_line = g.x_line.reshape(-1)
    arrays = {'W': (tW, FW), 'E': (tE, FE), 'S': (tS, FS), 'N': (tN, FN)}
    for (pa, ea, pb, eb, rev) in geo.INTERFACES:
        qa = _edge_get(arrays[ea][0], ea, pa, ne, ns)
        qb = _edge_get(arrays[eb][0], eb, pb, ne, ns)
        x1b, x2b = geo.edge_coords(eb, t_line)
        Jab = geo.contravariant_jacobian(x1b, x2b, g.frames[pb], g.frames[pa], g.a)   # d x_(a) / d x_(b)
        if rev:
            qb = qb[:, ::-1]
            Jab = Jab[:, :, ::-1]
        qb_a = [qb[0], Jab[0, 0] * qb[1] + Jab[0, 1] * qb[2], Jab[1, 0] * qb[1] + Jab[1, 1] * qb[2]]
        x1a, x2a = geo.edge_coords(ea, t_line)
        mf = geo.metric(np.tan(x1a), np.tan(x2a), g.a)
        da = 1 if ea in ('E', 'W') else 2
        hdd = mf['h11'] if da == 1 else mf['h22']
        h1d = mf['h11'] if da == 1 else mf['h12']
        h2d = mf['h12'] if da == 1 else mf['h22']
        own = [qa[0], qa[1], qa[2]]
        if ea in ('E', 'N'):
            fl = ausm_flux(own, qb_a, da, mf['sqrtg'], hdd, h1d, h2d, gr)
        else:
            fl = ausm_flux(qb_a, own, da, mf['sqrtg'], hdd, h1d, h2d, gr)
        _edge_set(arrays[ea][1], ea, pa, ne, ns, np.array(fl))
        # hand the flux to panel b: F^{mu d_b}_(b) = sigma dx^mu_(b)/dx^alpha_(a) F^{alpha d_a}_(a)
        Jba = geo.contravariant_jacobian(x1a, x2a, g.frames[pa], g.frames[pb], g.a)  # d x_(b) / d x_(a)
        db = 1 if eb in ('E', 'W') else 2
        sigma = np.sign(Jba[db - 1, da - 1])
        fb = [sigma * fl[0],
              sigma * (Jba[0, 0] * fl[1] + Jba[0, 1] * fl[2]),
              sigma * (Jba[1, 0] * fl[1] + Jba[1, 1] * fl[2])]
        fb = np.array(fb)
        if rev:
            fb = fb[:, ::-1]
        _edge_set(arrays[eb][1], eb, pb, ne, ns, fb)

    # DFR derivative sweeps (Eq. 11-14): extended flux [F(-1), f_1..f_Ns, F(+1)]
    D = g.D
    out = np.empty_like(q)
    for mu in range(3):
        ext1 = np.concatenate([FW[mu][..., None], F[mu][0], FE[mu][..., None]], axis=-1)   # [.., k2, n]
        d1 = np.einsum('kn,pefjn->pefjk', D, ext1)
        ext2 = np.concatenate([FS[mu][..., None, :], F[mu][1], FN[mu][..., None, :]], axis=-2)  # [.., n, k1]
        d2 = np.einsum('kn,pefnj->pefkj', D, ext2)
        out[mu] = -(2.0 / g.dx) * (d1 + d2) + S[mu]
    return out


def rhs_real(grid, q):
    """F(q) of Eq. (1)-(2) (Sec. 3) for a real state (the real part of the complex evaluation)."""
    return np.real(rhs(grid, q))


def jvp(grid, q, v, eps=1e-30):
    """Complex-step Jacobian-vector product, Eq. (28): Im F(q + i eps v) / eps."""
    q = np.asarray(q, dtype=float).reshape((3, 6, grid.ne, grid.ne, grid.ns, grid.ns))
    v = np.asarray(v, dtype=float).reshape(q.shape)
    return np.imag(rhs(grid, q + 1j * eps * v)) / eps


def mass_integral(grid, q):
    """Eq. (42) with Psi = H: sum of H sqrt(g) w_m w_n = sum of q^0 w_m w_n."""
    q = np.asarray(q).reshape((3, 6, grid.ne, grid.ne, grid.ns, grid.ns))
    w2 = grid.w[:, None] * grid.w[None, :]
    return np.sum(q[0] * w2)
