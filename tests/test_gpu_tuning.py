"""Kernel variants, the per-size-class autotuner and CUDA-graph replay.

None of these may change what a step computes: every variant must match the
FP64 oracle at the FP32 tolerances, a graph replay must give what direct
launches give on the same inputs (and pick up new input values and new
output buffers between replays), and tuning must settle on one variant.
"""
import numpy as np
import pytest

import oracle
import parity_log
from paper_2108_02259_gb300 import scenes

pytestmark = pytest.mark.gpu

TOL_V, TOL_C = 1e-5, 1e-4


@pytest.fixture(scope="module")
def apic():
    import torch  # noqa: F401

    from paper_2108_02259_gb300 import apic as a, build

    build.build()
    return a


def _dev(s, dt=np.float32):
    import torch

    f = s.astype(dt)
    tdt = torch.float32 if dt == np.float32 else torch.float64
    d = torch.device("cuda:0")

    def t(a, ty):
        return torch.as_tensor(np.ascontiguousarray(a), device=d, dtype=ty)

    return t(f.x, torch.float64), t(f.v, tdt), t(f.C, tdt), t(f.m, tdt), t(f.nrm, tdt), t(f.body, torch.int32)


def _scales(s, rC):
    vs = np.abs(s.v).max()
    cs = max(np.linalg.norm(s.C.reshape(-1, 9), axis=1).max(), np.linalg.norm(rC.reshape(-1, 9), axis=1).max())
    return vs, (cs if cs > 0 else 2 * vs / s.h)


def _close(s, v, Cm, rv, rC, label):
    vs, cs = _scales(s, rC)
    ev = np.abs(v - rv).max() / vs
    ec = np.abs(Cm - rC).max() / cs
    parity_log.record(f"tuning {label}", s.n, {"v": ev, "C": ec}, {"v": TOL_V, "C": TOL_C})
    assert ev <= TOL_V and ec <= TOL_C, f"{label}: v err {ev:.3g}, C err {ec:.3g}"


def test_variants_are_described(apic):
    names = apic.variants()
    assert len(names) == apic.load().apic_variant_count() >= 2
    assert all("CTAs/SM" in n for n in names)
    assert apic.load().apic_variant_name(len(names)) == b""


@pytest.mark.parametrize("case", ["four_bodies", "mu_pair"])
def test_every_variant_matches_oracle(apic, case):
    import torch

    if case == "four_bodies":
        s, mu_pair = scenes.four_bodies(scale=0.1), None
    else:
        s = scenes.random_cloud(6000, n_bodies=4, seed=17, h=0.05, n_iter=4)
        rng = np.random.default_rng(3)
        a = rng.uniform(0.1, 0.5, (4, 4))
        mu_pair = (a + a.T) / 2
    ref = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies,
                              mu_pair=mu_pair)
    with apic.Context(0) as ctx:
        for var in range(len(apic.variants())):
            ctx.set_variant(var)
            assert ctx.variant(s.x.shape[0]) == (var, True)
            X, V, Cc, M, NR, B = _dev(s)
            r = apic.contact_step(ctx, X, V, Cc, M, NR, B, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies, mu_pair=mu_pair)
            torch.cuda.synchronize()
            _close(s, r.v.cpu().double().numpy(), r.C.cpu().double().numpy(), ref[0], ref[1], f"variant {var}")
        with pytest.raises(apic.ApicError):
            ctx.set_variant(len(apic.variants()))


def test_persistent_grid_walks_several_items_per_cta(apic):
    """The persistent variant launches only as many CTAs as fit on the device
    at once; the 200,000-particle scene has about 2,000 work items, more than
    the 152 x 9 resident CTAs, so CTAs run several items one after another and
    reuse their shared tiles."""
    import torch

    names = apic.variants()
    var = next(i for i, nm in enumerate(names) if "persistent" in nm)
    s = scenes.four_bodies()
    ref = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies)
    with apic.Context(0) as ctx:
        ctx.set_variant(var)
        X, V, Cc, M, NR, B = _dev(s)
        for rep in range(3):  # direct launches, then the captured graph, then a replay
            r = apic.contact_step(ctx, X, V, Cc, M, NR, B, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies)
            torch.cuda.synchronize()
            _close(s, r.v.cpu().double().numpy(), r.C.cpu().double().numpy(), ref[0], ref[1],
                   f"persistent variant, call {rep}")


def test_graph_replay_matches_direct_launches(apic):
    """Same sizes and buffers on consecutive calls: the second call captures
    the passes, later ones replay them.  Each call gets new velocities and
    (every other call) new output tensors; a scene of another size in the
    middle forces a fresh capture."""
    import torch

    s = scenes.four_bodies(scale=0.1)
    other = scenes.two_cubes(mu=0.3, n_iter=s.n_iter)
    X, V, Cc, M, NR, B = _dev(s)
    X2, V2, C2, M2, N2, B2 = _dev(other)
    with apic.Context(0) as g, apic.Context(0) as d:
        d.set_graphs(False)
        for c in (g, d):
            c.set_variant(0)
        outs = [(torch.empty_like(V), torch.empty_like(Cc)) for _ in range(2)]
        for k in range(6):
            Vk = V * (1.0 + 0.25 * k)
            if k == 3:
                for c in (g, d):
                    apic.contact_step(c, X2, V2, C2, M2, N2, B2, other.h, other.mu, other.n_iter, n_bodies=2)
            vo, Co = outs[k % 2]
            rg = apic.contact_step(g, X, Vk, Cc, M, NR, B, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies,
                                   v_out=vo, C_out=Co)
            rd = apic.contact_step(d, X, Vk, Cc, M, NR, B, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies)
            torch.cuda.synchronize()
            sk = scenes.Scene(**{**s.__dict__, "v": s.v * (1.0 + 0.25 * k)})
            _close(sk, rg.v.cpu().double().numpy(), rg.C.cpu().double().numpy(), rd.v.cpu().double().numpy(),
                   rd.C.cpu().double().numpy(), f"call {k}")
        assert float(rg.v.abs().max()) > 0
        # graphs ran on g (sizing and series, replayed), none on d; both
        # contexts count the same kernel launches
        pg, pd = g.profile(), d.profile()
        assert pg["graph_launches"] >= 4
        assert pd["graph_launches"] == 0
        assert pg["kernel_launches"] == pd["kernel_launches"]
        assert pg["sort_launches"] == pd["sort_launches"]


def test_autotune_settles_and_keeps_parity(apic):
    import torch

    s = scenes.four_bodies(scale=0.25)
    n = s.x.shape[0]
    X, V, Cc, M, NR, B = _dev(s)
    with apic.Context(0) as ctx:
        assert ctx.variant(n) == (0, False)
        sc = [apic.BatchScene(X, V, Cc, M, NR, B, s.h, s.mu, n_bodies=s.n_bodies)]
        chosen = ctx.autotune(sc, s.n_iter)
        assert 0 <= chosen < len(apic.variants())
        assert ctx.variant(n) == (chosen, True)
        # another size class is still undecided
        assert ctx.variant(n * 8)[1] is False
        ref = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies)
        for _ in range(3):  # direct, captured, replayed
            r = apic.contact_step(ctx, X, V, Cc, M, NR, B, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies)
            torch.cuda.synchronize()
            _close(s, r.v.cpu().double().numpy(), r.C.cpu().double().numpy(), ref[0], ref[1], "tuned")
        ctx.set_variant(1)
        with pytest.raises(apic.ApicError):
            ctx.autotune(sc, s.n_iter)


@pytest.mark.parametrize("case", ["four_bodies", "mu_pair", "single_pass"])
def test_dependent_launch_keeps_parity(apic, case):
    """Programmatic dependent launch lets each pass start its prologue while
    the grid before it finishes; the passes must still see the finished node
    velocities and D.  Direct launches and graph replays, overlap on and off,
    all match the oracle (the mu pass and the single N = 0 pass included)."""
    import torch

    mu_pair = None
    if case == "four_bodies":
        s = scenes.four_bodies(scale=0.1)
    elif case == "mu_pair":
        s = scenes.random_cloud(6000, n_bodies=4, seed=23, h=0.05, n_iter=3)
        rng = np.random.default_rng(5)
        a = rng.uniform(0.1, 0.5, (4, 4))
        mu_pair = (a + a.T) / 2
    else:
        s = scenes.random_cloud(5000, n_bodies=3, seed=29, h=0.05, n_iter=0)
    ref = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies,
                              mu_pair=mu_pair)
    X, V, Cc, M, NR, B = _dev(s)
    for on in (True, False):
        with apic.Context(0) as ctx:
            ctx.set_variant(len(apic.variants()) - 1)
            ctx.set_overlap(on)
            for k in range(4):  # direct, direct, captured, replayed
                r = apic.contact_step(ctx, X, V, Cc, M, NR, B, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies,
                                      mu_pair=mu_pair)
                torch.cuda.synchronize()
                _close(s, r.v.cpu().double().numpy(), r.C.cpu().double().numpy(), ref[0], ref[1],
                       f"overlap {on}, call {k}")
            assert ctx.profile()["graph_launches"] >= 2


def test_tuning_table_round_trip(apic, tmp_path):
    """The autotuner's decision exported, saved to a file keyed by the GPU
    model, and loaded into a fresh context: the size class is decided there
    without timing, and its steps still match the oracle."""
    import json

    import torch

    s = scenes.four_bodies(scale=0.25)
    n = s.x.shape[0]
    X, V, Cc, M, NR, B = _dev(s)
    path = str(tmp_path / "tuning.json")
    with apic.Context(0) as a:
        sc = [apic.BatchScene(X, V, Cc, M, NR, B, s.h, s.mu, n_bodies=s.n_bodies)]
        chosen = a.autotune(sc, s.n_iter)
        assert a.tuning() == {n.bit_length(): chosen}
        a.save_tuning(path)
    ref = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies)
    with apic.Context(0) as b:
        assert b.variant(n) == (0, False)
        assert b.load_tuning(path)
        assert b.variant(n) == (chosen, True)
        r = apic.contact_step(b, X, V, Cc, M, NR, B, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies)
        torch.cuda.synchronize()
        _close(s, r.v.cpu().double().numpy(), r.C.cpu().double().numpy(), ref[0], ref[1], "loaded tuning")
        for bad in ({5: len(apic.variants())}, {63: 0}, {-1: 0}):
            with pytest.raises(apic.ApicError):
                b.set_tuning(bad)
        assert b.tuning() == {n.bit_length(): chosen}  # nothing set by the refused calls
    doc = json.load(open(path))
    doc["gpu"] = "another GPU"
    json.dump(doc, open(path, "w"))
    with apic.Context(0) as c:
        assert not c.load_tuning(path)
        assert c.variant(n) == (0, False)
