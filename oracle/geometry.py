"""Rotated cubed-sphere geometry (paper App. B and App. C), plain numpy FP64.

Test infrastructure only (see ``oracle/__init__.py``).

Coordinates: each panel p has angular coordinates x^1, x^2 in [-pi/4, pi/4],
X = tan x^1, Y = tan x^2, delta^2 = 1 + X^2 + Y^2 (App. B).
"""
import numpy as np

RADIUS = 6.37122e6       # a
GRAVITY = 9.80616        # g_r (Eq. 51)
OMEGA = 7.292e-5         # Omega


def panel_angles(lam0, phi0, alpha0):
    """(lambda_p, phi_p, alpha_p) of the six panels from panel 0's rotation.

    Eq. (81)-(95), reading every tan^{-1}(num/den) as atan2(num, den) (the
    paper requires the branch that puts the angle in the right quadrant, after
    Eq. 95), and the special case
    phi_0 = alpha_0 = 0 given there.
    """
    cl, sl = np.cos(lam0), np.sin(lam0)
    cp, sp = np.cos(phi0), np.sin(phi0)
    ca, sa = np.cos(alpha0), np.sin(alpha0)
    ang = [(lam0, phi0, alpha0)]
    # Eq. (81)-(83)
    ang.append((np.arctan2(cl * ca + sl * sp * sa, cl * sp * sa - sl * ca),
                -np.arcsin(cp * sa),
                np.arctan2(sp, cp * ca)))
    # Eq. (84)-(86)
    ang.append((lam0 + np.pi, -phi0, -alpha0))
    # Eq. (87)-(89)
    ang.append((-np.arctan2(cl * ca + sl * sp * sa, sl * ca - cl * sp * sa),
                np.arcsin(cp * sa),
                -np.arctan2(sp, cp * ca)))
    if phi0 == 0.0 and alpha0 == 0.0:
        # special case stated after Eq. (95)
        ang.append((0.0, np.pi / 2, -lam0))
        ang.append((0.0, -np.pi / 2, lam0))
    else:
        # Eq. (90)-(92)
        ang.append((np.arctan2(cl * sa - sl * sp * ca, -cl * sp * ca - sl * sa),
                    np.arcsin(cp * ca),
                    np.arctan2(cp * sa, -sp)))
        # Eq. (93)-(95)
        ang.append((np.arctan2(sl * sp * ca - cl * sa, cl * sp * ca + sl * sa),
                    -np.arcsin(cp * ca),
                    np.arctan2(cp * sa, sp)))
    return ang


def panel_frame(lam_p, phi_p, alpha_p):
    """Centre c and axis vectors e1, e2 with X = r.e1/r.c, Y = r.e2/r.c.

    Obtained by writing the numerator and denominator of Eq. (59)-(60) as dot
    products of the unit position r = (cos phi cos lam, cos phi sin lam, sin phi)
    (after multiplying both by cos phi).
    """
    c = np.array([np.cos(phi_p) * np.cos(lam_p), np.cos(phi_p) * np.sin(lam_p), np.sin(phi_p)])
    e_lam = np.array([-np.sin(lam_p), np.cos(lam_p), 0.0])
    e_phi = np.array([-np.sin(phi_p) * np.cos(lam_p), -np.sin(phi_p) * np.sin(lam_p), np.cos(phi_p)])
    e1 = np.cos(alpha_p) * e_lam - np.sin(alpha_p) * e_phi
    e2 = np.sin(alpha_p) * e_lam + np.cos(alpha_p) * e_phi
    return c, e1, e2


def xy_from_lonlat(lam, phi, lam_p, phi_p, alpha_p):
    """Eq. (59)-(60) literally: (X, Y) of geographic (lam, phi) on panel p."""
    d = lam - lam_p
    den = np.cos(phi_p) * np.cos(d) + np.tan(phi) * np.sin(phi_p)
    X = (np.sin(d) * np.cos(alpha_p) + np.sin(phi_p) * np.cos(d) * np.sin(alpha_p)
         - np.tan(phi) * np.cos(phi_p) * np.sin(alpha_p)) / den
    Y = (np.sin(d) * np.sin(alpha_p) - np.sin(phi_p) * np.cos(d) * np.cos(alpha_p)
         + np.tan(phi) * np.cos(phi_p) * np.cos(alpha_p)) / den
    return X, Y


def unit_position(x1, x2, frame):
    """Unit vector of the point (x1, x2) of a panel with frame (c, e1, e2)
    (Eq. 59-60 inverted: X = tan x^1, Y = tan x^2 along e1, e2 from the centre c)."""
    c, e1, e2 = frame
    X, Y = np.tan(x1), np.tan(x2)
    delta = np.sqrt(1 + X * X + Y * Y)
    r = (c[:, None] + e1[:, None] * np.ravel(X)[None] + e2[:, None] * np.ravel(Y)[None]) / np.ravel(delta)[None]
    return r.reshape((3,) + np.shape(X))


def tangent_vectors(x1, x2, frame, a=RADIUS):
    """Covariant basis d(a r)/dx^1, d(a r)/dx^2 (3-vectors; App. B, whose dot products are Eq. 64-66) by differentiating
    a (c + X e1 + Y e2)/delta with X = tan x^1, Y = tan x^2."""
    c, e1, e2 = frame
    X, Y = np.tan(x1), np.tan(x2)
    d2 = 1 + X * X + Y * Y
    d = np.sqrt(d2)
    P = c[:, None] + e1[:, None] * np.ravel(X)[None] + e2[:, None] * np.ravel(Y)[None]
    Xf, Yf, df = np.ravel(X), np.ravel(Y), np.ravel(d)
    dX = 1 + Xf * Xf
    dY = 1 + Yf * Yf
    t1 = a * (e1[:, None] * dX / df - P * Xf * dX / df ** 3)
    t2 = a * (e2[:, None] * dY / df - P * Yf * dY / df ** 3)
    shape = (3,) + np.shape(X)
    return t1.reshape(shape), t2.reshape(shape)


def metric(X, Y, a=RADIUS):
    """sqrt(g) (Eq. 70), h^{ij} (Eq. 67-69) and g_ij (Eq. 64-66)."""
    d2 = 1 + X * X + Y * Y
    sqrtg = a * a * (1 + X * X) * (1 + Y * Y) / d2 ** 1.5
    h11 = d2 / (a * a * (1 + X * X))
    h12 = X * Y * d2 / (a * a * (1 + X * X) * (1 + Y * Y))
    h22 = d2 / (a * a * (1 + Y * Y))
    g11 = a * a / d2 ** 2 * (1 + X * X) ** 2 * (1 + Y * Y)
    g12 = -a * a / d2 ** 2 * X * Y * (1 + X * X) * (1 + Y * Y)
    g22 = a * a / d2 ** 2 * (1 + X * X) * (1 + Y * Y) ** 2
    return dict(sqrtg=sqrtg, h11=h11, h12=h12, h22=h22, g11=g11, g12=g12, g22=g22)


def coriolis_bracket(X, Y, phi_p, alpha_p):
    """sin phi_p - X cos phi_p sin alpha_p + Y cos phi_p cos alpha_p (Eq. 71-74, 46)."""
    return np.sin(phi_p) - X * np.cos(phi_p) * np.sin(alpha_p) + Y * np.cos(phi_p) * np.cos(alpha_p)


def christoffel_time(X, Y, phi_p, alpha_p, omega=OMEGA):
    """Gamma^i_{0j} = Gamma^i_{j0}, Eq. (71)-(74): returns G[i][j] (0-based i,j)."""
    d2 = 1 + X * X + Y * Y
    s = coriolis_bracket(X, Y, phi_p, alpha_p)
    return [[omega * X * Y / d2 * s, -omega * (1 + Y * Y) / d2 * s],
            [omega * (1 + X * X) / d2 * s, -omega * X * Y / d2 * s]]


def christoffel_space(X, Y):
    """Gamma^i_{jk}, Eq. (75)-(80): returns G[i][j][k] (0-based)."""
    d2 = 1 + X * X + Y * Y
    z = np.zeros_like(X)
    G1 = [[2 * X * Y * Y / d2, -Y * (1 + Y * Y) / d2], [-Y * (1 + Y * Y) / d2, z]]
    G2 = [[z, -X * (1 + X * X) / d2], [-X * (1 + X * X) / d2, 2 * X * X * Y / d2]]
    return [G1, G2]


def spacetime_metric_g0(X, Y, phi_p, alpha_p, a=RADIUS, omega=OMEGA):
    """g_00, g_01, g_02 of Eq. (61)-(63) (used only by tests that re-derive Eq. 71-74)."""
    d2 = 1 + X * X + Y * Y
    s = coriolis_bracket(X, Y, phi_p, alpha_p)
    g00 = 1 + a * a / d2 * omega ** 2 * (d2 - s * s)
    g01 = a * a / d2 * omega * (1 + X * X) * (np.cos(phi_p) * np.cos(alpha_p) - Y * np.sin(phi_p))
    g02 = a * a / d2 * omega * (1 + Y * Y) * (np.cos(phi_p) * np.sin(alpha_p) + X * np.sin(phi_p))
    return g00, g01, g02


# ----------------------------------------------------------------------------
# Panel connectivity.  Edges: 'E' x^1 = +pi/4, 'W' x^1 = -pi/4, 'N' x^2 = +pi/4,
# 'S' x^2 = -pi/4.  The along-edge coordinate is x^2 on E/W edges and x^1 on
# N/S edges.  The table is what the frames of Eq. (81)-(95) imply (App. C lists
# the same twelve interfaces); tests check that paired edge points coincide in
# 3-D.  Each entry: (panel_a, edge_a, panel_b, edge_b, reversed).
# ----------------------------------------------------------------------------
INTERFACES = [
    (0, 'E', 1, 'W', False), (1, 'E', 2, 'W', False), (2, 'E', 3, 'W', False), (0, 'W', 3, 'E', False),
    (0, 'N', 4, 'S', False), (1, 'N', 4, 'E', False), (2, 'N', 4, 'N', True), (3, 'N', 4, 'W', True),
    (0, 'S', 5, 'N', False), (1, 'S', 5, 'E', True), (2, 'S', 5, 'S', True), (3, 'S', 5, 'W', False),
]


def edge_coords(edge, t):
    """(x^1, x^2) of the points with along-edge coordinate t on an edge (App. C)."""
    q = np.pi / 4
    t = np.asarray(t, dtype=float)
    if edge == 'E':
        return np.full_like(t, q), t
    if edge == 'W':
        return np.full_like(t, -q), t
    if edge == 'N':
        return t, np.full_like(t, q)
    return t, np.full_like(t, -q)


def contravariant_jacobian(x1, x2, frame_from, frame_to, a=RADIUS):
    """d x^i_(to) / d x^j_(from) at points given in 'from' coordinates (the
    contravariant transforms that App. C prints as Eq. 100-135).

    Plain definition: a contravariant vector A^j_(from) is the 3-vector
    V = A^j t_j(from); its components on panel 'to' are e^i_(to) . V with the
    dual basis e^i = h^{ik} t_k of panel 'to' evaluated at the same point.
    """
    r = unit_position(x1, x2, frame_from)
    c, e1, e2 = frame_to
    rc = np.einsum('k...,k->...', r, c)
    Xt = np.einsum('k...,k->...', r, e1) / rc
    Yt = np.einsum('k...,k->...', r, e2) / rc
    x1t, x2t = np.arctan(Xt), np.arctan(Yt)
    tf1, tf2 = tangent_vectors(x1, x2, frame_from, a)
    tt1, tt2 = tangent_vectors(x1t, x2t, frame_to, a)
    m = metric(Xt, Yt, a)
    d1 = m['h11'] * tt1 + m['h12'] * tt2
    d2 = m['h12'] * tt1 + m['h22'] * tt2
    J = np.empty((2, 2) + np.shape(x1))
    for i, di in enumerate((d1, d2)):
        for j, tj in enumerate((tf1, tf2)):
            J[i, j] = np.einsum('k...,k...->...', di, tj)
    return J
