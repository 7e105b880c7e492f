"""Partitions of one scene (APIC_PARTITIONED).

Each partition of the particles keeps its own sparse grid; after every
particle-to-grid transfer the nodes of grid blocks active in several
partitions are summed across them (the exchange a spatial decomposition of
one scene over devices needs once per transfer pair, Sec. 2.3 series), so
every partition normalises and interpolates the whole scene's grid.  The
outputs must therefore equal the FP64 oracle's on the whole scene, whatever
the split: spatial halves, a random three-way split, with a body-pair
friction table, in FP32 and FP64, on direct launches and graph replays.
"""
import numpy as np
import pytest

import oracle
import parity_log
from paper_2108_02259_gb300 import scenes

pytestmark = pytest.mark.gpu

TOL_V, TOL_C = 1e-5, 1e-4
TOL64 = 1e-11


@pytest.fixture(scope="module")
def ctx():
    from paper_2108_02259_gb300 import apic, build

    build.build()
    c = apic.Context(0)
    yield c
    c.close()


def _run_parts(ctx, s, parts, dt=np.float32, mu_pair=None, flags=None):
    """Step scene s as the partitions `parts` (index arrays into its
    particles) in one batched call; returns (v, C) in the scene's order."""
    import torch

    from paper_2108_02259_gb300 import apic

    f = s.astype(dt)
    tdt = torch.float32 if dt == np.float32 else torch.float64
    d = torch.device("cuda:0")

    def t(a, ty):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=ty, device=d)

    batch = [apic.BatchScene(t(f.x[ix], torch.float64), t(f.v[ix], tdt), t(f.C[ix], tdt), t(f.m[ix], tdt),
                             t(f.nrm[ix], tdt), t(f.body[ix], torch.int32), s.h, s.mu, n_bodies=s.n_bodies,
                             mu_pair=mu_pair) for ix in parts]
    fl = apic.APIC_PARTITIONED | (apic.APIC_FP64 if dt == np.float64 else 0) if flags is None else flags
    apic.contact_step_batched(ctx, batch, s.n_iter, flags=fl)
    torch.cuda.synchronize()
    v = np.zeros((s.n, 3))
    C = np.zeros((s.n, 9))
    for ix, b in zip(parts, batch):
        v[ix] = b.v_out.cpu().double().numpy().reshape(-1, 3)
        C[ix] = b.C_out.cpu().double().numpy().reshape(-1, 9)
    return v, C


def _compare(s, v, C, ref, tol_v, tol_c, label):
    rv, rC = ref[0], ref[1].reshape(-1, 9)
    vs = np.abs(s.v).max()
    cs = max(np.linalg.norm(s.C.reshape(-1, 9), axis=1).max(), np.linalg.norm(rC, axis=1).max())
    cs = cs if cs > 0 else 2 * vs / s.h
    ev, ec = np.abs(v - rv).max() / vs, np.abs(C - rC).max() / cs
    parity_log.record(f"partitioned {label}", s.n, {"v": ev, "C": ec}, {"v": tol_v, "C": tol_c})
    assert ev <= tol_v and ec <= tol_c, (label, ev, ec)


def _halves(s, axis=0):
    xm = np.median(s.x[:, axis])
    return [np.flatnonzero(s.x[:, axis] < xm), np.flatnonzero(s.x[:, axis] >= xm)]


def test_spatial_halves_match_the_whole_scene(ctx):
    """Two halves along x of the 4-body scene: the bodies are cut, and the
    blocks along the cut are active in both partitions."""
    s = scenes.four_bodies(scale=0.1, n_iter=4)
    ref = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies)
    v, C = _run_parts(ctx, s, _halves(s))
    _compare(s, v, C, ref, TOL_V, TOL_C, "x halves fp32")


def test_random_three_way_split_with_friction_table(ctx):
    """Any split of the particles is a valid partition (grid sums are
    additive): a random one shares nearly every block, and a per-pair
    friction table needs the per-body masses summed too."""
    s = scenes.random_cloud(6000, n_bodies=4, seed=23, h=0.05, n_iter=3)
    rng = np.random.default_rng(9)
    a = rng.uniform(0.1, 0.5, (4, 4))
    mu_pair = (a + a.T) / 2
    lab = rng.integers(0, 3, s.n)
    parts = [np.flatnonzero(lab == k) for k in range(3)]
    ref = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies,
                              mu_pair=mu_pair)
    v, C = _run_parts(ctx, s, parts, mu_pair=mu_pair)
    _compare(s, v, C, ref, TOL_V, TOL_C, "random 3-way split, mu table")


def test_fp64_partitions_match_the_oracle(ctx):
    """The two cubes cut across both bodies (halves along y), in FP64."""
    s = scenes.two_cubes(mu=0.3, n_iter=5)
    ref = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies)
    v, C = _run_parts(ctx, s, _halves(s, axis=1), dt=np.float64)
    _compare(s, v, C, ref, TOL64, TOL64, "y halves fp64")


def test_repeated_partitioned_calls_replay_the_exchange(ctx):
    """Direct launches, then the captured series (with the exchange
    kernels), then replays: the same results every time."""
    s = scenes.four_bodies(scale=0.05, n_iter=3)
    ref = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies)
    parts = _halves(s, axis=2)
    for k in range(4):
        v, C = _run_parts(ctx, s, parts)
        _compare(s, v, C, ref, TOL_V, TOL_C, f"z halves, call {k}")


def test_partitions_must_describe_one_scene(ctx):
    import torch

    from paper_2108_02259_gb300 import apic

    s = scenes.four_bodies(scale=0.05, n_iter=3)
    f = s.astype(np.float32)
    d = torch.device("cuda:0")

    def t(a, ty):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=ty, device=d)

    def part(ix, h):
        return apic.BatchScene(t(f.x[ix], torch.float64), t(f.v[ix], torch.float32), t(f.C[ix], torch.float32),
                               t(f.m[ix], torch.float32), t(f.nrm[ix], torch.float32), t(f.body[ix], torch.int32), h,
                               s.mu, n_bodies=s.n_bodies)

    a, b = _halves(s)
    with pytest.raises(apic.ApicError):
        apic.contact_step_batched(ctx, [part(a, s.h), part(b, s.h * 2)], 3, flags=apic.APIC_PARTITIONED)
    with pytest.raises(apic.ApicError):
        apic.contact_step_batched(ctx, [part(a, s.h), part(b, s.h)], 3,
                                  flags=apic.APIC_PARTITIONED | apic.APIC_DETERMINISTIC)


def test_mass_normals_and_host_arrays_across_the_cut(ctx):
    """With APIC_MASS_NORMALS the normals come from each body's grid mass,
    so the per-body masses of the blocks along the cut must be summed across
    the partitions; with host arrays every partition is staged on its own.
    The partitioned call must give what one call on the whole scene gives."""
    from paper_2108_02259_gb300 import apic

    s = scenes.four_bodies(scale=0.1, n_iter=3)
    f = s.astype(np.float32)
    whole = apic.contact_step(ctx, f.x, f.v, f.C, f.m, None, f.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies,
                              flags=apic.APIC_MASS_NORMALS)
    parts = _halves(s)
    batch = [apic.BatchScene(np.ascontiguousarray(f.x[ix]), np.ascontiguousarray(f.v[ix]),
                             np.ascontiguousarray(f.C[ix]), np.ascontiguousarray(f.m[ix]), None,
                             np.ascontiguousarray(f.body[ix]), s.h, s.mu, n_bodies=s.n_bodies) for ix in parts]
    apic.contact_step_batched(ctx, batch, s.n_iter, flags=apic.APIC_PARTITIONED | apic.APIC_MASS_NORMALS)
    v = np.zeros((s.n, 3))
    C = np.zeros((s.n, 9))
    for ix, b in zip(parts, batch):
        v[ix] = b.v_out.reshape(-1, 3)
        C[ix] = b.C_out.reshape(-1, 9)
    wv, wC = np.asarray(whole.v, np.float64).reshape(-1, 3), np.asarray(whole.C, np.float64).reshape(-1, 9)
    vs = np.abs(s.v).max()
    cs = max(np.linalg.norm(wC, axis=1).max(), 2 * vs / s.h)
    ev, ec = np.abs(v - wv).max() / vs, np.abs(C - wC).max() / cs
    parity_log.record("partitioned, mass normals, host arrays vs one call", s.n, {"v": ev, "C": ec},
                      {"v": TOL_V, "C": TOL_C})
    assert ev <= TOL_V and ec <= TOL_C, (ev, ec)
