"""apic_node_normals (Sec. 2.3 node normals) against the FP64 oracle, and a
contact step fed with device-built normals.

FP32 output is rounded from FP64 sums: within 1e-6 of the oracle per
component (the rounding is 6e-8; atomics change the summation order only).
FP64 output within 1e-13.
"""
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


def _meshes():
    rng = np.random.default_rng(11)
    x, t = scenes.icosphere(4)
    yield "icosphere4", x * rng.uniform(0.5, 2.0, (1, 3)) + 5.0, t
    yield "cube", *scenes.cube_surface_mesh(3.0)
    x, t = scenes.box_lattice_surface(50, 40, 25, spacing=1 / 512)  # a four-body box, interior nodes too
    yield "box_lattice", x, t
    # ragged: many meshes, nodes on no face, shuffled ids
    xs, ts, off = [], [], 0
    for lv in (0, 1, 2):
        x, t = scenes.icosphere(lv, radius=1.0 + lv)
        xs.append(x + rng.normal(size=3) * 10)
        ts.append(t + off)
        off += len(x)
    xs.append(rng.normal(size=(37, 3)))
    x = np.vstack(xs)
    t = np.vstack(ts)
    perm = rng.permutation(len(x))
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(x))
    yield "ragged", x[perm], inv[t].astype(np.int32)


@pytest.mark.parametrize("fp64", [False, True])
def test_normals_match_oracle(env, fp64):
    apic, ctx, torch = env
    for name, x, t in _meshes():
        ref = oracle.node_normals(x, t)
        got = apic.node_normals(ctx, torch.as_tensor(x, device="cuda"), torch.as_tensor(t, device="cuda"),
                                fp64=fp64)
        torch.cuda.synchronize()
        err = np.abs(got.cpu().double().numpy() - ref).max()
        assert err <= (1e-13 if fp64 else 1e-6), f"{name}: {err}"
        zero = np.linalg.norm(ref, axis=1) == 0
        assert np.all(got.cpu().numpy()[zero] == 0), name


def test_normals_host_path_empty_and_bad_index(env):
    apic, ctx, torch = env
    x, t = scenes.cube_surface_mesh()
    got = apic.node_normals(ctx, x, t)  # numpy: host pointers
    assert np.abs(got - oracle.node_normals(x, t)).max() <= 1e-6
    assert np.all(apic.node_normals(ctx, x, np.zeros((0, 3), np.int32)) == 0)
    with pytest.raises(apic.ApicError) as e:
        apic.node_normals(ctx, x, np.vstack([t, [[0, 1, len(x)]]]))
    assert e.value.code == apic.APIC_ERR_INVALID_ARG
    # the context still works
    got = apic.node_normals(ctx, torch.as_tensor(x, device="cuda"), torch.as_tensor(t, device="cuda"))
    assert np.abs(got.cpu().numpy() - oracle.node_normals(x, t)).max() <= 1e-6


def test_contact_step_with_device_normals(env):
    """Two lattice boxes approaching head on; normals built on the device from
    their boundary triangles give the same step as the oracle's normals."""
    apic, ctx, torch = env
    h = 1 / 32
    xa, ta = scenes.box_lattice_surface(8, 8, 8, spacing=h / 2, origin=(0.3, 0.4, 0.4))
    xb, tb = scenes.box_lattice_surface(8, 8, 8, spacing=h / 2, origin=(0.3 + 7 * h / 2 + 0.6 * h, 0.4, 0.4))
    x = np.vstack([xa, xb])
    tri = np.vstack([ta, tb + len(xa)]).astype(np.int32)
    n = len(x)
    body = np.repeat([0, 1], len(xa)).astype(np.int32)
    v = np.zeros((n, 3))
    v[body == 0, 0], v[body == 1, 0] = 1.0, -1.0
    Cm = np.zeros((n, 9))
    m = np.full(n, 1.0 / len(xa))
    nrm_ref = oracle.node_normals(x, tri)
    ref = oracle.contact_step(x, v, Cm, m, nrm_ref, body, h, 0.3, 6, n_bodies=2)
    dev = lambda a, d: torch.as_tensor(np.ascontiguousarray(a), dtype=d, device="cuda")  # noqa: E731
    X = dev(x, torch.float64)
    nrm = apic.node_normals(ctx, X, dev(tri, torch.int32))
    r = apic.contact_step(ctx, X, dev(v, torch.float32), dev(Cm, torch.float32), dev(m, torch.float32), nrm,
                          dev(body, torch.int32), h, 0.3, 6, n_bodies=2)
    torch.cuda.synchronize()
    vs = np.abs(v).max()
    cs = np.linalg.norm(ref[1].reshape(-1, 9), axis=1).max()  # input C = 0
    assert cs > 0
    assert np.abs(r.v.cpu().double().numpy() - ref[0].reshape(-1, 3)).max() <= 1e-5 * vs
    assert np.abs(r.C.cpu().double().numpy().reshape(-1, 9) - ref[1].reshape(-1, 9)).max() <= 1e-4 * cs
    assert np.abs(r.v.cpu().double().numpy() - v).max() > 1e-3  # the bodies did interact
