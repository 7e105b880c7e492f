"""apic_augury_steps (Sec. 2.2 augury dynamics) against the FP64 oracle.

FP64: the whole run matches the oracle (positions within 1e-11 of the body
size, velocities within 1e-9 of max|v| after 40 steps through frictional
contact).  FP32: one step from the same state within the contact step's FP32
tolerances (v 1e-5 of max|v|; the acceleration scaled by tau likewise); a
long FP32 run keeps momentum and rebounds like the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2108_02259_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2108_02259_gb300 import apic, build

    build.build()
    c = apic.Context(0)
    yield apic, c, torch
    c.close()


def _state(torch, e, dt=np.float64, x=None, v=None, Cm=None, av=None, aC=None):
    s = e.scene
    n = s.n
    td = torch.float64 if dt == np.float64 else torch.float32

    def d(a, ty):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=ty, device="cuda")

    return dict(x=d(s.x if x is None else x, torch.float64), v=d(s.v if v is None else v, td),
                Cm=d(np.zeros((n, 9)) if Cm is None else np.reshape(Cm, (n, 9)), td),
                av=d(np.zeros((n, 3)) if av is None else av, td),
                aC=d(np.zeros((n, 9)) if aC is None else np.reshape(aC, (n, 9)), td),
                m=d(s.m, td), body=d(s.body, torch.int32), springs=d(e.springs, torch.int32),
                rest=d(e.rest, torch.float64), stiffness=d(e.stiffness, torch.float64), tri=d(e.tri, torch.int32))


def _gpu(apic, ctx, e, st, n_steps, init, **kw):
    s = e.scene
    return apic.augury_steps(ctx, st["x"], st["v"], st["Cm"], st["av"], st["aC"], st["m"], st["body"], st["springs"],
                             st["rest"], st["stiffness"], st["tri"], s.h, s.mu, s.n_iter, e.dt, e.tau, n_steps,
                             n_bodies=s.n_bodies, init=init, **kw)


def _host(st):
    return {k: t.cpu().double().numpy() for k, t in st.items()}


def test_fp64_run_matches_oracle(env):
    apic, ctx, torch = env
    e = scenes.elastic_pair(tilt=0.3, mu=0.3)
    s = e.scene
    st = _state(torch, e)
    stats = _gpu(apic, ctx, e, st, 40, True, stats=True)
    x, v, Cm, av, aC, en = oracle.augury_steps(s.x, s.v, s.C, s.m, s.body, e.springs, e.rest, e.stiffness, e.tri,
                                               s.h, s.mu, s.n_iter, e.dt, e.tau, 40)
    g = _host(st)
    size = np.ptp(s.x, axis=0).max()
    vs = np.abs(s.v).max()
    assert np.abs(g["x"] - x).max() <= 1e-11 * size
    assert np.abs(g["v"] - v).max() <= 1e-9 * vs
    assert np.abs(g["Cm"] - Cm.reshape(-1, 9)).max() <= 1e-9 * vs / s.h
    assert np.abs(g["av"] - av).max() * e.tau <= 1e-9 * vs
    assert abs(stats["kinetic"] - en["kinetic"]) <= 1e-9 * en["kinetic"]
    assert abs(stats["springs"] - en["springs"]) <= 1e-8 * max(en["springs"], 1e-30)
    assert np.abs(stats["P"]).max() <= 1e-12 * np.sum(s.m * np.abs(s.v[:, 0]))


def test_fp32_step_matches_oracle_from_the_same_state(env):
    apic, ctx, torch = env
    e = scenes.elastic_pair(tilt=0.2, mu=0.3)
    s = e.scene
    # bring the oracle into contact, then take one more step on both sides
    x, v, Cm, av, aC, _ = oracle.augury_steps(s.x, s.v, s.C, s.m, s.body, e.springs, e.rest, e.stiffness, e.tri,
                                              s.h, s.mu, s.n_iter, e.dt, e.tau, 60)
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)  # noqa: E731
    x1, v1, C1, av1, aC1, _ = oracle.augury_steps(x, f32(v), f32(Cm), f32(s.m), s.body, e.springs, e.rest, e.stiffness,
                                                  e.tri, s.h, s.mu, s.n_iter, e.dt, e.tau, 1, av=f32(av), aC=f32(aC),
                                                  init=False)
    st = _state(torch, e, np.float32, x=x, v=v, Cm=Cm, av=av, aC=aC)
    _gpu(apic, ctx, e, st, 1, False)
    g = _host(st)
    vs = np.abs(v).max()
    cs = max(np.linalg.norm(C1.reshape(-1, 9), axis=1).max(), 1e-30)
    assert np.abs(g["x"] - x1).max() <= 1e-5 * vs * e.dt + 1e-12
    assert np.abs(g["v"] - v1).max() <= 1e-5 * vs
    assert np.abs(g["Cm"] - C1.reshape(-1, 9)).max() <= 1e-4 * cs
    assert np.abs(g["av"] - av1).max() * e.tau <= 2e-5 * vs


def test_fp32_run_rebounds_and_keeps_momentum(env):
    apic, ctx, torch = env
    e = scenes.elastic_pair()
    s = e.scene
    nb = s.n // 2
    st = _state(torch, e, np.float32)
    stats = _gpu(apic, ctx, e, st, 720, True, stats=True)
    g = _host(st)
    assert g["v"][:nb, 0].mean() < -0.3 and g["v"][nb:, 0].mean() > 0.3
    assert g["x"][nb:, 0].min() - g["x"][:nb, 0].max() > 2.0 * s.h
    assert np.abs(stats["P"]).max() <= 1e-4 * np.sum(s.m * np.abs(s.v[:, 0]))
    _, vo, _, _, _, en = oracle.augury_steps(s.x, s.v, s.C, s.m, s.body, e.springs, e.rest, e.stiffness, e.tri, s.h,
                                             s.mu, s.n_iter, e.dt, e.tau, 720)
    assert abs(g["v"][:nb, 0].mean() - vo[:nb, 0].mean()) < 0.02  # the same rebound as the FP64 oracle


def test_isolated_spring_pair_closed_form(env):
    apic, ctx, torch = env
    h, L0, u0, m, k, dt = 0.1, 1.0, 0.05, 0.5, 40.0, 0.01
    d = lambda a, ty=torch.float64: torch.as_tensor(np.asarray(a), dtype=ty, device="cuda")  # noqa: E731
    x = d([[0.33, 0.41, 0.52], [0.33 + L0 + u0, 0.41, 0.52]])
    v, Cm, av, aC = d(np.zeros((2, 3))), d(np.zeros((2, 9))), d(np.zeros((2, 3))), d(np.zeros((2, 9)))
    theta = np.arccos(1.0 - 0.5 * (2.0 * k / m) * dt * dt)
    args = (d([m, m]), d([0, 1], torch.int32), d([[0, 1]], torch.int32), d([L0]), d([k]),
            d(np.zeros((0, 3)), torch.int32), h, 0.3, 3, dt, dt)
    apic.augury_steps(ctx, x, v, Cm, av, aC, *args, 60, n_bodies=2, init=True)
    u = float(x[1, 0] - x[0, 0]) - L0
    assert abs(u - u0 * np.cos(60 * theta)) < 1e-12


def test_fixed_nodes_and_bad_spring(env):
    apic, ctx, torch = env
    e = scenes.elastic_pair(n_side=5)
    s = e.scene
    st = _state(torch, e, np.float32)
    fixed = torch.as_tensor((s.body == 0).astype(np.uint8), device="cuda")
    _gpu(apic, ctx, e, st, 200, True, fixed=fixed)
    g = _host(st)
    f = s.body == 0
    assert np.all(g["x"][f] == s.x[f]) and np.all(g["v"][f] == 0) and np.all(g["av"][f] == 0)
    assert g["v"][~f, 0].mean() > 0.0
    bad = e.springs.copy()
    bad[3, 0] = s.n
    st = _state(torch, e, np.float32)
    st["springs"] = torch.as_tensor(bad, device="cuda")
    with pytest.raises(apic.ApicError) as ex:
        _gpu(apic, ctx, e, st, 1, True)
    assert ex.value.code == apic.APIC_ERR_INVALID_ARG
