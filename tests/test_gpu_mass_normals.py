"""Normals from each body's grid mass on the GPU (apic_mass_normals and the
APIC_MASS_NORMALS flag of the contact step) against the FP64 oracle.

Where a particle's ratio |grad rho| h / rho lies within 1e-4 (relative) of
the threshold, FP32 and FP64 may take the surface decision differently; such
a particle's GPU normal must then be 0 or the oracle's direction.  Every
other particle is compared element by element: within 1e-5 (FP32) or 1e-11
(FP64).  The contact step with device-computed normals is compared with the
oracle's step fed the same normals (so both take the same decisions).
"""
import numpy as np
import pytest

import oracle
import parity_log
from paper_2108_02259_gb300 import scenes

pytestmark = pytest.mark.gpu

TOL_V, TOL_C = 1e-5, 1e-4
THR = 0.5


@pytest.fixture(scope="module")
def ctx():
    from paper_2108_02259_gb300 import apic, build

    build.build()
    c = apic.Context(0)
    yield c
    c.close()


def _t(a, dt):
    import torch

    return torch.as_tensor(np.ascontiguousarray(a), device="cuda:0", dtype=dt)


def _lattice_box():
    n, h = 20, 0.1
    I, J, K = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    x = np.stack([I.ravel(), J.ravel(), K.ravel()], 1) * (h / 2) + np.array([0.013, -0.021, 0.007])
    z = np.zeros((len(x), 3))
    return scenes.Scene(x, z, np.zeros((len(x), 3, 3)), np.full(len(x), 1.0 / len(x)), z, np.zeros(len(x), np.int32),
                        1, h, 0.3, 2)


def _cases():
    rng = np.random.default_rng(41)
    return [("lattice box", _lattice_box()),
            ("four bodies small", scenes.four_bodies(scale=0.05)),
            ("random cloud, 5 bodies", scenes.random_cloud(4000, n_bodies=5, seed=42, h=0.08, n_iter=2,
                                                            origin=(-1.2, 0.4, 2.0))),
            ("multi-body scene", scenes.multi_body_scene(rng, 30000, 4, 1 / 128, n_iter=3))]


def _compare_normals(label, s, got, tol):
    ref, ratio = oracle.mass_normals(s.x, s.m, s.body, s.h, n_bodies=s.n_bodies, threshold=THR)
    dir0, _ = oracle.mass_normals(s.x, s.m, s.body, s.h, n_bodies=s.n_bodies, threshold=0.0)
    near = np.abs(ratio - THR) <= 1e-4 * THR
    clear = ~near
    err = np.abs(got[clear] - ref[clear]).max() if clear.any() else 0.0
    parity_log.record(f"mass normals, {label}", s.n, {"n": err}, {"n": tol})
    assert err <= tol, (label, err)
    for g, d in zip(got[near], dir0[near]):  # either side of the threshold, but a valid normal
        assert np.abs(g).max() == 0.0 or np.abs(g - d).max() <= tol
    # a reasonable share of the particles is on the surface, and only there
    on = np.linalg.norm(got, axis=1) > 0
    assert 0 < on.sum() < s.n


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_mass_normals_match_oracle(ctx, dt):
    import torch

    from paper_2108_02259_gb300 import apic

    tdt = torch.float32 if dt == np.float32 else torch.float64
    tol = 1e-5 if dt == np.float32 else 1e-11
    for label, s in _cases():
        out = apic.mass_normals(ctx, _t(s.x, torch.float64), _t(s.m, tdt), _t(s.body, torch.int32), s.h,
                                n_bodies=s.n_bodies)
        torch.cuda.synchronize()
        _compare_normals(f"{label} {np.dtype(dt).name}", s, out.cpu().double().numpy(), tol)


def test_mass_normals_deterministic_mode_is_reproducible(ctx):
    import torch

    from paper_2108_02259_gb300 import apic

    s = _cases()[2][1]
    args = (_t(s.x, torch.float64), _t(s.m, torch.float32), _t(s.body, torch.int32), s.h)
    a = apic.mass_normals(ctx, *args, n_bodies=s.n_bodies, deterministic=True).clone()
    b = apic.mass_normals(ctx, *args, n_bodies=s.n_bodies, deterministic=True).clone()
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    _compare_normals("deterministic", s, a.cpu().double().numpy(), 1e-5)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_contact_step_with_device_normals(ctx, dt):
    """APIC_MASS_NORMALS (nrm omitted): the step uses the normals that
    apic_mass_normals gives, so it matches the oracle's step fed those
    normals, and the same call with those normals passed explicitly."""
    import torch

    from paper_2108_02259_gb300 import apic

    tdt = torch.float32 if dt == np.float32 else torch.float64
    tol = (TOL_V, TOL_C) if dt == np.float32 else (1e-11, 1e-11)
    for label, s in _cases()[1:]:
        f = s.astype(dt)
        X, V, Cc, M, B = (_t(f.x, torch.float64), _t(f.v, tdt), _t(f.C, tdt), _t(f.m, tdt), _t(f.body, torch.int32))
        nrm = apic.mass_normals(ctx, X, M, B, s.h, n_bodies=s.n_bodies)
        r = apic.contact_step(ctx, X, V, Cc, M, None, B, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies, stats=True)
        r2 = apic.contact_step(ctx, X, V, Cc, M, nrm, B, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies)
        torch.cuda.synchronize()
        n64 = nrm.cpu().double().numpy()
        rv, rC, _ = oracle.contact_step(s.x, s.v, s.C, s.m, n64, s.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies)
        v, Cm = r.v.cpu().double().numpy(), r.C.cpu().double().numpy()
        vs = np.abs(s.v).max()
        cs = max(np.linalg.norm(s.C.reshape(-1, 9), axis=1).max(), np.linalg.norm(rC.reshape(-1, 9), axis=1).max())
        ev, ec = np.abs(v - rv).max() / vs, np.abs(Cm - rC).max() / cs
        parity_log.record(f"step with mass normals, {label} {np.dtype(dt).name}", s.n, {"v": ev, "C": ec},
                          {"v": tol[0], "C": tol[1]})
        assert ev <= tol[0] and ec <= tol[1], (label, ev, ec)
        assert np.abs(r2.v.cpu().double().numpy() - v).max() <= 2 * tol[0] * vs
        sP = np.sum(s.m * np.linalg.norm(s.v, axis=1))
        assert np.abs(r.stats["P_out"] - r.stats["P_in"]).max() <= 1e-6 * sP


def test_batched_and_host_calls_with_device_normals(ctx):
    """The flag in a batched call (device arrays) and on the host-pointer
    path: each scene as its single-scene device call."""
    import torch

    from paper_2108_02259_gb300 import apic

    sc = [c[1] for c in _cases()[1:]]
    bs, single = [], []
    for s in sc:
        f = s.astype(np.float32)
        X, V, Cc, M, B = (_t(f.x, torch.float64), _t(f.v, torch.float32), _t(f.C, torch.float32),
                          _t(f.m, torch.float32), _t(f.body, torch.int32))
        bs.append(apic.BatchScene(X, V, Cc, M, None, B, s.h, s.mu, n_bodies=s.n_bodies))
        single.append(apic.contact_step(ctx, X, V, Cc, M, None, B, s.h, s.mu, 3, n_bodies=s.n_bodies))
    apic.contact_step_batched(ctx, bs, 3, flags=apic.APIC_MASS_NORMALS)
    torch.cuda.synchronize()
    for s, b, r in zip(sc, bs, single):
        vs = np.abs(s.v).max()
        assert torch.abs(b.v_out - r.v).max().item() <= 2e-6 * vs
        f = s.astype(np.float32)
        h = apic.contact_step(ctx, f.x, f.v, f.C, f.m, None, f.body, s.h, s.mu, 3, n_bodies=s.n_bodies)
        assert np.abs(h.v - r.v.cpu().numpy()).max() <= 2e-6 * vs
