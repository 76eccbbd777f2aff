"""Seeded synthetic inputs for the shallow-water workloads.

This module holds no arithmetic of the numerical method: it only draws random
numbers and evaluates smooth fields (real spherical-harmonic sums) at Cartesian
unit vectors supplied by the caller.  Both the CUDA path and the CPU oracle
evaluate the fields at their own node positions and convert them to the state
with their own geometry.

Field recipe (stand-in for the Williamson-style test cases, whose definitions
are not reproduced here): free-surface height h = h_mean + h' with h' a sum of
real orthonormal spherical harmonics of degree 1..L with N(0, 1) coefficients,
scaled so that max |h'| over a 1 deg x 1 deg longitude-latitude sample equals
the stated amplitude; wind V = g / (2 Omega a) r x grad h' (geostrophic with a
constant Coriolis parameter 2 Omega); optional non-divergent perturbation
r x grad chi scaled to a stated peak speed; optional bottom h_B of the same form.
Grid rotation angles lambda_0 in U[-pi, pi), phi_0 in U[-pi/3, pi/3],
alpha_0 in U[-pi, pi).
"""
from dataclasses import dataclass, field

import numpy as np

RADIUS = 6.37122e6
GRAVITY = 9.80616
OMEGA = 7.292e-5


@dataclass
class Workload:
    name: str
    ne: int
    ns: int
    order: int
    dt: float
    steps: int
    tol: float
    h_degree: int
    h_amp: float
    h_mean: float = 8000.0
    wind_pert: float = 0.0       # peak m/s of the non-divergent perturbation
    pert_degree: int = 8
    bottom_amp: float = 0.0
    bottom_degree: int = 8
    eps: float = 1e-30

    @property
    def p(self):
        return self.ns - 1

    @property
    def n_unknowns(self):
        return 3 * 6 * self.ne ** 2 * self.ns ** 2


WORKLOADS = {
    "small_ne4_p3": Workload("small_ne4_p3", 4, 4, 4, 900.0, 10, 1e-12, 4, 100.0),
    "ne30_p5": Workload("ne30_p5", 30, 6, 5, 1800.0, 48, 1e-10, 16, 200.0, wind_pert=2.0),
    "ne90_p6": Workload("ne90_p6", 90, 7, 6, 1200.0, 36, 1e-10, 32, 300.0,
                        bottom_amp=1500.0, bottom_degree=8),
    "ne60_p5": Workload("ne60_p5", 60, 6, 5, 1800.0, 48, 1e-10, 4, 100.0),
}


def real_sph_harm(L, xyz):
    """All real orthonormal spherical harmonics of degree 0..L at unit vectors
    xyz[3, N]; returns dict {(l, m): values} with m in -l..l (m < 0: sin)."""
    x, y, z = (np.asarray(c, dtype=float) for c in xyz)
    ct = np.clip(z, -1.0, 1.0)
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    lon = np.arctan2(y, x)
    out = {}
    pmm = np.full_like(ct, np.sqrt(1.0 / (4 * np.pi)))
    for m in range(L + 1):
        if m > 0:
            pmm = pmm * np.sqrt((2 * m + 1) / (2.0 * m)) * st
        cols = {m: pmm}
        if m + 1 <= L:
            cols[m + 1] = np.sqrt(2 * m + 3.0) * ct * pmm
        for l in range(m + 2, L + 1):
            a = np.sqrt((4.0 * l * l - 1) / (l * l - m * m))
            b = np.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1) ** 2 - 1))
            cols[l] = a * (ct * cols[l - 1] - b * cols[l - 2])
        for l, plm in cols.items():
            if m == 0:
                out[(l, 0)] = plm
            else:
                out[(l, m)] = np.sqrt(2.0) * plm * np.cos(m * lon)
                out[(l, -m)] = np.sqrt(2.0) * plm * np.sin(m * lon)
    return out


_SUM_CHUNK = 1 << 15   # points per chunk of a harmonic sum (its work arrays stay in cache)


class HarmonicField:
    """Seeded sum of real spherical harmonics of degree 1..L, unit peak."""

    def __init__(self, rng, L):
        self.L = L
        self.coef = {(l, m): rng.standard_normal() for l in range(1, L + 1) for m in range(-l, l + 1)}
        self.scale = 1.0
        peak = np.max(np.abs(self.raw(_latlon_sample())))
        self.scale = 1.0 / peak

    def raw(self, xyz):
        # the harmonics of real_sph_harm, accumulated degree by degree over
        # cache-sized chunks of points instead of stored (equal to rounding)
        r = np.asarray(xyz, dtype=float)
        flat = r.reshape(3, -1)
        n = flat.shape[1]
        if n <= _SUM_CHUNK:
            return _sph_sum(self.L, self.coef, flat).reshape(r.shape[1:])
        parts = [_sph_sum(self.L, self.coef, flat[:, i:i + _SUM_CHUNK]) for i in range(0, n, _SUM_CHUNK)]
        return np.concatenate(parts).reshape(r.shape[1:])

    def __call__(self, xyz):
        return self.scale * self.raw(xyz)

    def grad(self, xyz, delta=1e-5):
        """Surface gradient on the unit sphere (3-vectors) by central
        differences along two great circles through each point."""
        r = np.asarray(xyz, dtype=float)
        t1, t2 = _tangent_frame(r)
        g = np.zeros_like(r)
        for t in (t1, t2):
            fp = self(np.cos(delta) * r + np.sin(delta) * t)
            fm = self(np.cos(delta) * r - np.sin(delta) * t)
            g = g + t * ((fp - fm) / (2 * delta))[None]
        return g


def _tangent_frame(r):
    ref = np.where(np.abs(r[2:3]) < 0.9, np.array([0.0, 0.0, 1.0])[:, None] + 0 * r[0:1],
                   np.array([1.0, 0.0, 0.0])[:, None] + 0 * r[0:1])
    t1 = np.cross(ref, r, axis=0)
    t1 = t1 / np.linalg.norm(t1, axis=0)
    t2 = np.cross(r, t1, axis=0)
    return t1, t2


def _latlon_sample():
    lat = np.deg2rad(np.arange(-90.0, 90.0 + 1e-9, 1.0))
    lon = np.deg2rad(np.arange(-180.0, 180.0, 1.0))
    LA, LO = np.meshgrid(lat, lon, indexing="ij")
    return np.stack([np.cos(LA) * np.cos(LO), np.cos(LA) * np.sin(LO), np.sin(LA)]).reshape(3, -1)


@dataclass
class Fields:
    workload: Workload
    seed: int
    rotation: tuple
    h_pert: HarmonicField
    chi: object = None
    bottom: object = None
    chi_scale: float = 0.0

    def evaluate(self, xyz):
        """(h, h_B, V[3]) at unit vectors xyz[3, ...]."""
        wl = self.workload
        shp = np.shape(xyz)[1:]
        r = np.asarray(xyz, dtype=float).reshape(3, -1)
        h = wl.h_mean + wl.h_amp * self.h_pert(r)
        gh = wl.h_amp * self.h_pert.grad(r)
        V = GRAVITY / (2 * OMEGA * RADIUS) * np.cross(r, gh, axis=0)
        if self.chi is not None:
            V = V + self.chi_scale * np.cross(r, self.chi.grad(r), axis=0)
        hB = np.zeros(r.shape[1])
        if self.bottom is not None:
            hB = wl.bottom_amp * self.bottom(r)
        return h.reshape(shp), hB.reshape(shp), V.reshape((3,) + shp)


def make_fields(workload, seed):
    """Draw the rotation and the harmonic coefficients of a workload."""
    if isinstance(workload, str):
        workload = WORKLOADS[workload]
    rng = np.random.Generator(np.random.PCG64(seed))
    rotation = (rng.uniform(-np.pi, np.pi), rng.uniform(-np.pi / 3, np.pi / 3), rng.uniform(-np.pi, np.pi))
    hp = HarmonicField(rng, workload.h_degree)
    f = Fields(workload, seed, rotation, hp)
    if workload.wind_pert > 0:
        f.chi = HarmonicField(rng, workload.pert_degree)
        s = _latlon_sample()
        speed = np.linalg.norm(np.cross(s, f.chi.grad(s), axis=0), axis=0)
        f.chi_scale = workload.wind_pert / np.max(speed)
    if workload.bottom_amp > 0:
        f.bottom = HarmonicField(rng, workload.bottom_degree)
    return f


# ---------------------------------------------------------------- ensemble
# Members on uneven grids: every (n_e, p) class of ENSEMBLE_NE x ENSEMBLE_P
# appears equally often, in a seeded order; each member draws its own grid
# rotation, EPI order (4 or 5) and a degree <= 12 harmonic perturbation of 50 m
# peak on top of the ensemble's shared degree <= 4, 100 m base field; the wind
# is geostrophic for the member's total height anomaly.
ENSEMBLE_NE = (8, 16, 24, 32)
ENSEMBLE_P = (3, 4, 5)
ENSEMBLE_BASE = (4, 100.0)      # degree, peak (m)
ENSEMBLE_PERT = (12, 50.0)


@dataclass
class EnsembleMember:
    index: int
    ne: int
    p: int
    order: int
    dt: float
    seed: int

    @property
    def ns(self):
        return self.p + 1

    @property
    def nodes(self):
        return 6 * self.ne ** 2 * self.ns ** 2


def ensemble_members(count=96, seed=0, ne_choices=ENSEMBLE_NE, p_choices=ENSEMBLE_P, orders=(4, 5), dt=900.0):
    """The seeded member list (grid class, EPI order, member seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    classes = [(ne, p) for ne in ne_choices for p in p_choices]
    reps = -(-count // len(classes))
    pool = [classes[i % len(classes)] for i in range(reps * len(classes))]
    perm = rng.permutation(len(pool))[:count]
    out = []
    for i, k in enumerate(perm):
        ne, p = pool[k]
        order = int(orders[rng.integers(len(orders))])
        out.append(EnsembleMember(i, ne, p, order, dt, int(rng.integers(1 << 31))))
    return out


def _sph_sum(L, coef, xyz):
    """sum over (l, m) of coef[(l, m)] Y_lm at unit vectors xyz[3, N] (same
    harmonics and normalisation as real_sph_harm, accumulated degree by degree
    instead of stored)."""
    x, y, z = (np.asarray(c, dtype=float) for c in xyz)
    ct = np.clip(z, -1.0, 1.0)
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    lon = np.arctan2(y, x)
    s = np.zeros_like(ct)
    pmm = np.full_like(ct, np.sqrt(1.0 / (4 * np.pi)))
    for m in range(L + 1):
        if m > 0:
            pmm = pmm * np.sqrt((2 * m + 1) / (2.0 * m)) * st
        acc_c = coef.get((m, m), 0.0) * pmm
        acc_s = coef.get((m, -m), 0.0) * pmm if m > 0 else None
        p2, p1 = None, pmm
        for l in range(m + 1, L + 1):
            if l == m + 1:
                pl = np.sqrt(2 * m + 3.0) * ct * pmm
            else:
                a = np.sqrt((4.0 * l * l - 1) / (l * l - m * m))
                b = np.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1) ** 2 - 1))
                pl = a * (ct * p1 - b * p2)
            acc_c = acc_c + coef.get((l, m), 0.0) * pl
            if m > 0:
                acc_s = acc_s + coef.get((l, -m), 0.0) * pl
            p2, p1 = p1, pl
        if m == 0:
            s = s + acc_c
        else:
            s = s + np.sqrt(2.0) * (acc_c * np.cos(m * lon) + acc_s * np.sin(m * lon))
    return s


class _SumField:
    """A fixed harmonic sum (coefficients already scaled) and its surface gradient."""

    def __init__(self, L, coef):
        self.L, self.coef = L, coef

    def __call__(self, xyz):
        return _sph_sum(self.L, self.coef, np.asarray(xyz, dtype=float))

    grad = HarmonicField.grad


@dataclass
class EnsembleFields:
    member: EnsembleMember
    rotation: tuple
    anomaly: _SumField
    h_mean: float = 8000.0

    def evaluate(self, xyz):
        """(h, h_B, V[3]) at unit vectors xyz[3, ...] (flat bottom)."""
        shp = np.shape(xyz)[1:]
        r = np.asarray(xyz, dtype=float).reshape(3, -1)
        h = self.h_mean + self.anomaly(r)
        V = GRAVITY / (2 * OMEGA * RADIUS) * np.cross(r, self.anomaly.grad(r), axis=0)
        return h.reshape(shp), np.zeros(r.shape[1]).reshape(shp), V.reshape((3,) + shp)


def _draw_rotation(rng):
    return (rng.uniform(-np.pi, np.pi), rng.uniform(-np.pi / 3, np.pi / 3), rng.uniform(-np.pi, np.pi))


def ensemble_rotation(member):
    """The member's grid rotation (the first draws of its generator)."""
    return _draw_rotation(np.random.Generator(np.random.PCG64(member.seed)))


def ensemble_fields(member, ensemble_seed=0):
    """Fields of one ensemble member: shared base plus the member's perturbation."""
    sample = _latlon_sample()

    def unit_peak(rng, L):
        # the draws of HarmonicField, normalised to unit peak on the same sample
        c = {(l, m): rng.standard_normal() for l in range(1, L + 1) for m in range(-l, l + 1)}
        return c, 1.0 / np.max(np.abs(_sph_sum(L, c, sample)))

    base, sb = unit_peak(np.random.Generator(np.random.PCG64(ensemble_seed)), ENSEMBLE_BASE[0])
    rng = np.random.Generator(np.random.PCG64(member.seed))
    rotation = _draw_rotation(rng)
    pert, sp = unit_peak(rng, ENSEMBLE_PERT[0])
    coef = {}
    for c, amp in ((base, ENSEMBLE_BASE[1] * sb), (pert, ENSEMBLE_PERT[1] * sp)):
        for k, v in c.items():
            coef[k] = coef.get(k, 0.0) + amp * v
    return EnsembleFields(member, rotation, _SumField(ENSEMBLE_PERT[0], coef))


def _member_fields_job(args):
    member, xyz, ensemble_seed = args
    return ensemble_fields(member, ensemble_seed).evaluate(xyz)


def ensemble_member_fields(members, xyz_list, ensemble_seed=0, workers=None):
    """(h, h_B, V) of every member at its node positions xyz_list[i] (3 x nodes).
    workers > 1 evaluates them in a pool of fresh ('spawn') processes, which is
    safe after the parent has initialised CUDA."""
    jobs = [(m, x, ensemble_seed) for m, x in zip(members, xyz_list)]
    if not workers or workers <= 1 or len(jobs) <= 1:
        return [_member_fields_job(j) for j in jobs]
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(workers, len(jobs))) as pool:
        return pool.map(_member_fields_job, jobs, chunksize=1)


def random_perturbation(n, seed, scale=1.0):
    """A seeded N(0, scale^2) vector (Krylov-like direction for JVP checks)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return scale * rng.standard_normal(n)
