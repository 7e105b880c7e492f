"""apic_contact_step_static: the contact step for callers that cannot allocate
device memory (a host whose own pool owns the GPU's memory, or a real-time
loop that cannot afford cudaMalloc's implicit device synchronisation).

It must give the same results as apic_contact_step and as the FP64 oracle,
on consecutive calls that share the library's static scratch array (scalar
friction and a per-pair friction table, FP32 and FP64), and refuse scenes
too large for that array.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
import parity_log
from paper_2108_02259_gb300 import scenes

pytestmark = pytest.mark.gpu

TOL_V, TOL_C = 1e-5, 1e-4  # the FP32 tolerances of the parity tests


@pytest.fixture(scope="module")
def lib():
    from paper_2108_02259_gb300 import apic, build

    build.build()
    return apic


def _tensors(s, dtype):
    import torch

    f = s.astype(dtype)
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    dev = torch.device("cuda:0")

    def t(a, d):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=d).to(dev)

    return (t(f.x, torch.float64), t(f.v, tdt), t(f.C, tdt), t(f.m, tdt), t(f.nrm, tdt), t(f.body, torch.int32))


def _compare(s, a, b, label="", tol=(TOL_V, TOL_C)):
    v_ref, C_ref = a
    v, Cm = b
    vs = np.abs(s.v).max()
    cs = max(np.linalg.norm(s.C.reshape(-1, 9), axis=1).max(), np.linalg.norm(C_ref.reshape(-1, 9), axis=1).max())
    if cs == 0:
        cs = 2 * vs / s.h
    ev, ec = np.abs(v - v_ref).max() / vs, np.abs(Cm - C_ref).max() / cs
    if label:
        parity_log.record(label, s.n, {"v": ev, "C": ec}, {"v": tol[0], "C": tol[1]})
    assert ev <= tol[0], (label, ev)
    assert ec <= tol[1], (label, ec)


def test_static_matches_allocating_step_on_consecutive_calls(lib):
    import torch

    apic = lib
    cases = [(scenes.four_bodies(scale=0.05), np.float32), (scenes.two_cubes(mu=0.3, n_iter=10), np.float32),
             (scenes.random_cloud(4000, n_bodies=3, seed=5, h=0.1, n_iter=3), np.float64)]
    with apic.Context(0) as ctx:
        for s, dt in cases:
            X, V, Cc, M, NR, B = _tensors(s, dt)
            ref = apic.contact_step(ctx, X, V, Cc, M, NR, B, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies, stats=True)
            got = apic.contact_step_static(X, V, Cc, M, NR, B, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies, stats=True)
            torch.cuda.synchronize()
            a = (ref.v.cpu().double().numpy(), ref.C.cpu().double().numpy())
            b = (got.v.cpu().double().numpy(), got.C.cpu().double().numpy())
            _compare(s, a, b)
            # and the FP64 oracle, so that a fault shared by both GPU entry points is caught
            rv, rC, _ = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, s.mu, s.n_iter,
                                            n_bodies=s.n_bodies)
            tol = (TOL_V, TOL_C) if dt == np.float32 else (1e-11, 1e-11)
            _compare(s, (rv, rC), b, f"no-allocation entry point vs oracle, {np.dtype(dt).name}", tol)
            assert got.stats["multibody_nodes"] == ref.stats["multibody_nodes"]
            assert got.stats["work_items"] == ref.stats["work_items"]
            sP = float(np.sum(s.m * np.linalg.norm(s.v, axis=1)))
            assert np.abs(got.stats["P_out"] - got.stats["P_in"]).max() <= 1e-6 * sP


def test_static_refuses_scene_beyond_its_array(lib):
    apic = lib
    s = scenes.four_bodies()  # 200,000 particles: more scratch than the static array holds
    X, V, Cc, M, NR, B = _tensors(s, np.float32)
    with pytest.raises(apic.ApicError) as e:
        apic.contact_step_static(X, V, Cc, M, NR, B, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies)
    assert e.value.code == apic.APIC_ERR_INVALID_ARG
    assert "static scratch" in str(e.value)
    # and a small scene still works afterwards
    s2 = scenes.two_cubes(mu=0.3, n_iter=2)
    X, V, Cc, M, NR, B = _tensors(s2, np.float32)
    r = apic.contact_step_static(X, V, Cc, M, NR, B, s2.h, s2.mu, s2.n_iter, n_bodies=s2.n_bodies)
    assert np.isfinite(r.v.cpu().numpy()).all()


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_static_per_pair_friction_matches_oracle(lib, dt):
    """The per-pair friction route of the no-allocation entry point: the
    table is staged from host memory into the static array, and the per-body
    node masses and particle friction come from it.  Two calls in a row (the
    second with negated velocities) against the oracle and the allocating
    step."""
    import torch

    apic = lib
    s = scenes.random_cloud(3000, n_bodies=4, seed=21, h=0.08, n_iter=3)
    rng = np.random.default_rng(22)
    a = rng.uniform(0.05, 0.6, (4, 4))
    mp = (a + a.T) / 2
    tol = (TOL_V, TOL_C) if dt == np.float32 else (1e-11, 1e-11)
    with apic.Context(0) as ctx:
        for sign in (1.0, -1.0):
            sc = scenes.Scene(s.x, sign * s.v, sign * s.C, s.m, s.nrm, s.body, s.n_bodies, s.h, s.mu, s.n_iter)
            X, V, Cc, M, NR, B = _tensors(sc, dt)
            got = apic.contact_step_static(X, V, Cc, M, NR, B, sc.h, sc.mu, sc.n_iter, n_bodies=4, mu_pair=mp)
            ref = apic.contact_step(ctx, X, V, Cc, M, NR, B, sc.h, sc.mu, sc.n_iter, n_bodies=4, mu_pair=mp)
            torch.cuda.synchronize()
            b = (got.v.cpu().double().numpy(), got.C.cpu().double().numpy())
            rv, rC, _ = oracle.contact_step(sc.x, sc.v, sc.C, sc.m, sc.nrm, sc.body, sc.h, sc.mu, sc.n_iter,
                                            n_bodies=4, mu_pair=mp)
            _compare(sc, (rv, rC), b, f"no-allocation entry point, per-pair mu, {np.dtype(dt).name}, sign {sign}",
                     tol)
            _compare(sc, (ref.v.cpu().double().numpy(), ref.C.cpu().double().numpy()), b, "", tol)
