"""Seeded inputs (host only): the ensemble's member list and member fields,
and the workload fields.  Both are evaluated by an accumulating
spherical-harmonic sum; it must equal the sum over the stored harmonics."""
import numpy as np

from paper_2101_05617_gb300 import synth


def _unit_vectors(n, seed):
    x = np.random.default_rng(seed).standard_normal((3, n))
    return x / np.linalg.norm(x, axis=0)


def test_accumulated_harmonic_sum_equals_stored_harmonics():
    xyz = _unit_vectors(3000, 1)
    for L, seed in ((4, 3), (12, 5)):
        rng = np.random.Generator(np.random.PCG64(seed))
        coef = {(l, m): rng.standard_normal() for l in range(1, L + 1) for m in range(-l, l + 1)}
        Y = synth.real_sph_harm(L, xyz)
        ref = sum(c * Y[k] for k, c in coef.items())
        np.testing.assert_allclose(synth._sph_sum(L, coef, xyz), ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))


def test_workload_field_is_the_stored_harmonic_sum_over_chunks():
    """The workload fields (HarmonicField) accumulate their sum over chunks of
    points: over several chunks and a ragged tail, and for an input of more than
    one dimension, the result equals the sum over the stored harmonics."""
    n = 2 * synth._SUM_CHUNK + 1234
    xyz = _unit_vectors(n, 7)
    f = synth.HarmonicField(np.random.Generator(np.random.PCG64(11)), 16)
    Y = synth.real_sph_harm(16, xyz)
    ref = f.scale * sum(c * Y[k] for k, c in f.coef.items())
    got = f(xyz)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.max(np.abs(ref)))
    assert f(xyz.reshape(3, 2, -1)).shape == (2, n // 2) and np.array_equal(f(xyz.reshape(3, 2, -1)).ravel(), got)


def test_member_list_is_balanced_and_seeded():
    a = synth.ensemble_members(96, seed=0)
    b = synth.ensemble_members(96, seed=0)
    c = synth.ensemble_members(96, seed=1)
    assert a == b and a != c
    classes = {}
    for m in a:
        classes[(m.ne, m.p)] = classes.get((m.ne, m.p), 0) + 1
        assert m.order in (4, 5) and m.dt == 900.0
    assert sorted(classes) == sorted((ne, p) for ne in synth.ENSEMBLE_NE for p in synth.ENSEMBLE_P)
    assert set(classes.values()) == {8}
    assert sum(m.nodes for m in a) == 8 * sum(6 * ne * ne * (p + 1) ** 2 for ne in synth.ENSEMBLE_NE
                                              for p in synth.ENSEMBLE_P)
    assert len({m.seed for m in a}) == 96


def test_member_fields():
    m = synth.ensemble_members(96, seed=0)[7]
    f = synth.ensemble_fields(m)
    assert f.rotation == synth.ensemble_rotation(m)
    xyz = _unit_vectors(4000, 2)
    h, hB, V = f.evaluate(xyz)
    # base (100 m peak) + perturbation (50 m peak) around 8 km, flat bottom
    assert np.all(np.abs(h - 8000.0) <= 150.0 + 1e-9) and np.max(np.abs(h - 8000.0)) > 20.0
    assert np.all(hB == 0.0)
    # the wind is tangent to the sphere and geostrophic for the anomaly
    assert np.max(np.abs(np.sum(V * xyz, axis=0))) < 1e-9 * np.max(np.abs(V))
    assert 0.1 < np.max(np.linalg.norm(V, axis=0)) < 50.0
    # two members differ; the same member is reproduced
    f2 = synth.ensemble_fields(synth.ensemble_members(96, seed=0)[8])
    assert not np.allclose(f2.evaluate(xyz)[0], h)
    assert np.array_equal(synth.ensemble_fields(m).evaluate(xyz)[0], h)
