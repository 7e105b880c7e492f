"""apic_contact_step_static: the contact step for callers that cannot allocate
device memory (a host whose own pool owns the GPU's memory, or a real-time
loop that cannot afford cudaMalloc's implicit device synchronisation).

It must give the same results as apic_contact_step, on consecutive calls
that share the library's static scratch array, and refuse scenes too large
for that array.  This file is collected last on purpose.
"""
import numpy as np
import pytest

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


def _compare(s, a, b):
    v_ref, C_ref = a
    v, Cm = b
    vs = np.abs(s.v).max()
    cs = max(np.linalg.norm(s.C.reshape(-1, 9), axis=1).max(), np.linalg.norm(C_ref.reshape(-1, 9), axis=1).max())
    if cs == 0:
        cs = 2 * vs / s.h
    assert np.abs(v - v_ref).max() <= TOL_V * vs
    assert np.abs(Cm - C_ref).max() <= TOL_C * cs


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
