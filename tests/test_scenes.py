"""The synthetic inputs follow their stated recipe (CPU).

The paper has no dataset; every benchmark and test input comes from the
seeded generators in scenes.py.  These checks pin what the inputs are said
to be: node counts, grid spacing, per-body mass, rigid velocity fields with
matching affine matrices, unit or zero normals, friction tables, and
reproducibility from the seed.
"""
import numpy as np
import pytest

from paper_2108_02259_gb300 import scenes


def _rigid_per_body(s, tol=1e-12):
    """Per body: C is one skew matrix, and v is the rigid field it implies."""
    for b in range(s.n_bodies):
        sel = s.body == b
        C = s.C[sel]
        assert np.abs(C - C[0]).max() <= tol
        assert np.abs(C[0] + C[0].T).max() <= tol  # skew: a rotation rate
        x, v = s.x[sel], s.v[sel]
        # v(x) - v(x0) = C (x - x0) for every node of the body
        dv = (v - v[0]) - (x - x[0]) @ C[0].T
        assert np.abs(dv).max() <= 1e-9 * max(1.0, np.abs(v).max())


def _normals_unit_or_zero(s):
    n2 = np.sum(s.nrm * s.nrm, axis=1)
    assert np.all((n2 == 0) | (np.abs(n2 - 1) < 1e-9))


def test_two_cubes_recipe():
    s = scenes.two_cubes(mu=0.3, n_iter=10)
    assert s.n == 1024 and s.n_bodies == 2 and s.h == 1 / 32 and s.mu == 0.3 and s.n_iter == 10
    assert np.allclose(s.m, 1 / 512)
    for b, (cx, vx) in enumerate(((0.35, 1.0), (0.65, -1.0))):
        sel = s.body == b
        assert np.allclose(s.x[sel].mean(axis=0), [cx, 0.5, 0.5])
        assert np.allclose(s.v[sel], [vx, 0, 0]) and not s.C[sel].any()
    spacing = np.diff(np.unique(np.round(s.x[s.body == 0][:, 0], 12)))
    assert np.allclose(spacing, 1 / 32)
    _normals_unit_or_zero(s)


def test_four_bodies_recipe_and_seed():
    s = scenes.four_bodies()
    assert s.n == 200_000 and s.n_bodies == 4 and s.h == 1 / 256 and s.mu == 0.3 and s.n_iter == 8
    for b in range(4):
        sel = s.body == b
        assert sel.sum() == 50_000
        assert abs(s.m[sel].sum() - 1.0) <= 1e-12
    _rigid_per_body(s)
    _normals_unit_or_zero(s)
    # |v0| <= 2 and |omega| <= 5: the rotation rate of each body
    for b in range(4):
        C = s.C[s.body == b][0]
        w = np.array([C[2, 1], C[0, 2], C[1, 0]])
        assert np.linalg.norm(w) <= 5
    t = scenes.four_bodies()
    assert np.array_equal(s.x, t.x) and np.array_equal(s.v, t.v)  # the seed fixes everything


@pytest.mark.parametrize("per_body", [20_000])
def test_eight_bodies_recipe(per_body):
    """The 4 M-node scene at a reduced node count per body (same recipe)."""
    s = scenes.eight_bodies(per_body=per_body)
    assert s.n == 8 * per_body and s.n_bodies == 8 and s.h == 1 / 512 and s.n_iter == 8
    for b in range(8):
        sel = s.body == b
        assert sel.sum() == per_body
        assert abs(s.m[sel].sum() - 1.0) <= 1e-12
        lm = np.log(s.m[sel] * per_body)
        assert 0.25 < lm.std() < 0.35  # lognormal, sigma 0.3
    mp = s.mu_pair
    assert mp.shape == (8, 8) and np.array_equal(mp, mp.T) and mp.min() >= 0.1 and mp.max() <= 0.5
    _rigid_per_body(s)
    _normals_unit_or_zero(s)


def test_batched_scene_recipe():
    sc = scenes.batch_of_scenes(64)
    assert len(sc) == 64
    sizes = np.array([s.n for s in sc])
    assert sizes.min() >= 1_000 * 0.9 and sizes.max() <= 200_000 * 1.1
    assert {s.h for s in sc} <= {1 / 64, 1 / 128, 1 / 256}
    assert all(2 <= s.n_bodies <= 6 and s.n_iter == 8 for s in sc)
