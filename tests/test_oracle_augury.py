"""Pins of the oracle's augury dynamics (Sec. 2.2: eq. apic_accel integrated
with eq. Newmark, read as velocity Verlet; linear-spring foreground).

Closed forms where the contact operator is the identity (particles that
share no grid node, affine fields): an isolated spring pair follows the
discrete Verlet solution exactly; free fall and rigid translation are exact.
With contact: net momentum is kept, mirror symmetry is kept, and two elastic
cubes rebound (the rebound's size is not pinned: the paper reports the
method as dissipative without a number for this case)."""
import numpy as np
import pytest

import oracle
from paper_2108_02259_gb300 import scenes


def _run(e, n_steps, **kw):
    s = e.scene
    return oracle.augury_steps(s.x, s.v, s.C, s.m, s.body, e.springs, e.rest, e.stiffness, e.tri, s.h, s.mu,
                               s.n_iter, e.dt, e.tau, n_steps, **kw)


def test_isolated_spring_pair_follows_discrete_verlet():
    """u'' = -(2k/m) u for the stretch u of a spring between two equal masses;
    velocity Verlet from rest gives u_n = u_0 cos(n theta) exactly, with
    cos(theta) = 1 - omega^2 dt^2 / 2.  The particles are 10 cells apart, so
    the transfers reproduce each one's own (affine) field and A_hat = 0."""
    h, L0, u0, m, k, dt = 0.1, 1.0, 0.05, 0.5, 40.0, 0.01
    x = np.array([[0.33, 0.41, 0.52], [0.33 + L0 + u0, 0.41, 0.52]])
    w2 = 2.0 * k / m
    theta = np.arccos(1.0 - 0.5 * w2 * dt * dt)
    xs, vs = x, np.zeros((2, 3))
    av = aC = Cm = None
    for n in range(1, 61):
        xs, vs, Cm, av, aC, _ = oracle.augury_steps(xs, vs, np.zeros((2, 9)) if Cm is None else Cm, [m, m], [0, 1],
                                                    [[0, 1]], [L0], [k], np.zeros((0, 3), np.int32), h, 0.3, 3,
                                                    dt, dt, 1, av=av, aC=aC, n_bodies=2, init=(n == 1))
        u = xs[1, 0] - xs[0, 0] - L0
        assert abs(u - u0 * np.cos(n * theta)) < 1e-12, n
        assert abs(xs[0, 0] + xs[1, 0] - (x[0, 0] + x[1, 0])) < 1e-13  # centre of mass at rest
    assert np.abs(Cm).max() < 1e-9


def test_free_fall_is_exact():
    g = np.array([0.0, -9.81, 2.0])
    x0, v0, dt, n = np.array([[0.2, 0.7, 0.4]]), np.array([[1.5, 0.5, -0.25]]), 1e-3, 80
    x, v, _, _, _, en = oracle.augury_steps(x0, v0, np.zeros((1, 9)), [2.0], [0], np.zeros((0, 2), np.int32), [],
                                            [], np.zeros((0, 3), np.int32), 0.05, 0.3, 2, dt, dt, n, gravity=g)
    t = n * dt
    assert np.abs(x - (x0 + v0 * t + 0.5 * g * t * t)).max() < 1e-13
    assert np.abs(v - (v0 + g * t)).max() < 1e-12


def test_rigid_translation_is_exact():
    e = scenes.elastic_pair(n_side=5)
    s = e.scene
    one = s.body == 0
    x0 = s.x[one]
    idx = np.flatnonzero(one)
    remap = -np.ones(len(s.x), np.int64)
    remap[idx] = np.arange(len(idx))
    keep = one[e.springs].all(1)
    tri = remap[e.tri[one[e.tri].all(1)]]
    v = np.tile([0.7, -0.2, 0.4], (len(x0), 1))
    x, vo, Co, _, _, en = oracle.augury_steps(x0, v, np.zeros((len(x0), 9)), s.m[one], np.zeros(len(x0), np.int32),
                                              remap[e.springs[keep]], e.rest[keep], e.stiffness[keep], tri, s.h, 0.3,
                                              4, e.dt, e.tau, 40)
    assert np.abs(x - (x0 + 40 * e.dt * v)).max() < 1e-13
    assert np.abs(vo - v).max() < 1e-12
    assert np.abs(Co).max() < 1e-9
    assert en["springs"] < 1e-20


def test_momentum_kept_through_frictional_contact():
    e = scenes.elastic_pair(tilt=0.3, mu=0.3)
    s = e.scene
    x, v, Cm, _, _, _ = _run(e, 150)
    scale = np.sum(s.m * np.linalg.norm(s.v, axis=1))
    assert np.abs((s.m[:, None] * v).sum(0)).max() < 1e-13 * scale


def test_mirror_symmetry_through_contact():
    e = scenes.elastic_pair(mu=0.3)
    s = e.scene
    nb = s.n // 2
    x, v, Cm, _, _, _ = _run(e, 150)
    xb = x[nb:] * np.array([-1.0, 1.0, 1.0]) + np.array([1.0, 0.0, 0.0])  # mirror about x = 0.5
    assert np.abs(xb - x[:nb]).max() < 1e-12
    assert np.abs(v[nb:] * np.array([-1.0, 1.0, 1.0]) - v[:nb]).max() < 1e-10
    assert v[:nb, 0].mean() < 0.9  # they did interact


def test_elastic_cubes_rebound():
    e = scenes.elastic_pair()
    s = e.scene
    nb = s.n // 2
    x, v, Cm, _, _, en = _run(e, 720)
    assert v[:nb, 0].mean() < -0.3 and v[nb:, 0].mean() > 0.3  # centre-of-mass velocities reversed
    assert x[nb:, 0].min() - x[:nb, 0].max() > 2.0 * s.h  # separated
    e0 = 0.5 * np.sum(s.m * np.sum(s.v ** 2, axis=1))
    assert 0.2 * e0 < en["kinetic"] + en["springs"] < e0  # dissipative, but a rebound


def test_fixed_nodes_stay():
    e = scenes.elastic_pair(n_side=5)
    s = e.scene
    fixed = (s.body == 0).astype(np.uint8)  # hold the first cube in place
    x, v, Cm, av, _, _ = _run(e, 200, fixed=fixed)
    f = fixed.astype(bool)
    assert np.all(x[f] == s.x[f]) and np.all(v[f] == 0.0) and np.all(av[f] == 0.0)
    assert v[~f, 0].mean() > 0.0  # the free cube bounced off the held one


def test_bad_spring_index_rejected():
    e = scenes.elastic_pair(n_side=3)
    s = e.scene
    bad = e.springs.copy()
    bad[0, 1] = s.n
    with pytest.raises(ValueError):
        oracle.augury_steps(s.x, s.v, s.C, s.m, s.body, bad, e.rest, e.stiffness, e.tri, s.h, 0.0, 2, e.dt, e.tau, 1)
