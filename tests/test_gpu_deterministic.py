"""APIC_DETERMINISTIC: bitwise-reproducible contact steps.

In this mode node sums are added as 64-bit fixed-point integers, so their
order no longer matters.  The tests check what that promises: the same bits
from run to run, with graphs and dependent launch on or off, alone or in any
batch, through the context and the no-allocation entry points; parity with
the FP64 oracle at the FP32 tolerances; and the error path (non-finite input)
that leaves the caller's outputs untouched and the context usable.
"""
import numpy as np
import pytest

import discontinuity
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


def _dev(s):
    import torch

    f = s.astype(np.float32)
    d = torch.device("cuda:0")

    def t(a, ty):
        return torch.as_tensor(np.ascontiguousarray(a), device=d, dtype=ty)

    return (t(f.x, torch.float64), t(f.v, torch.float32), t(f.C, torch.float32), t(f.m, torch.float32),
            t(f.nrm, torch.float32), t(f.body, torch.int32))


def _close(s, v, Cm, rv, rC, label, env=None):
    """env: the oracle's envelope at the step of the Sec. 2.3 rule
    (tests/discontinuity.py); errors are then measured beyond it."""
    vs = np.abs(s.v).max()
    cs = max(np.linalg.norm(s.C.reshape(-1, 9), axis=1).max(), np.linalg.norm(rC.reshape(-1, 9), axis=1).max())
    cs = cs if cs > 0 else 2 * vs / s.h
    if env is None:
        ev = np.abs(v - rv).max() / vs
        ec = np.abs(Cm - rC).max() / cs
    else:
        ev = discontinuity.excess(v, rv, env[0], vs)
        ec = discontinuity.excess(Cm.reshape(rC.shape), rC, env[1], cs)
    parity_log.record(f"deterministic {label}", s.n, {"v": ev, "C": ec}, {"v": TOL_V, "C": TOL_C})
    assert ev <= TOL_V and ec <= TOL_C, f"{label}: v err {ev:.3g}, C err {ec:.3g}"


def _mu_scene():
    s = scenes.random_cloud(6000, n_bodies=4, seed=31, h=0.05, n_iter=3)
    rng = np.random.default_rng(9)
    a = rng.uniform(0.1, 0.5, (4, 4))
    return s, (a + a.T) / 2


def _step(apic, ctx, s, dev, flags, mu_pair=None):
    import torch

    X, V, Cc, M, NR, B = dev
    r = apic.contact_step(ctx, X, V, Cc, M, NR, B, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies, mu_pair=mu_pair,
                          flags=flags)
    torch.cuda.synchronize()
    return r.v.clone(), r.C.clone()


@pytest.mark.parametrize("case", ["four_bodies", "mu_pair", "pic", "sep23", "single_pass"])
def test_repeatable_bits_and_oracle_parity(apic, case):
    import torch

    det = apic.APIC_DETERMINISTIC
    mu_pair, extra = None, 0
    if case == "mu_pair":
        s, mu_pair = _mu_scene()
    elif case == "single_pass":
        s = scenes.random_cloud(5000, n_bodies=3, seed=37, h=0.05, n_iter=0)
    else:
        s = scenes.four_bodies(scale=0.1)
        extra = {"four_bodies": 0, "pic": apic.APIC_VARIANT_PIC, "sep23": apic.APIC_VARIANT_SEP23}[case]
    oflags = (oracle.FLAG_PIC if extra & apic.APIC_VARIANT_PIC else 0) | (
        oracle.FLAG_SEP23 if extra & apic.APIC_VARIANT_SEP23 else 0)
    ref = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies,
                              mu_pair=mu_pair, flags=oflags)
    dev = _dev(s)
    runs = []
    with apic.Context(0) as ctx:
        for _ in range(4):  # direct, direct, captured, replayed
            runs.append(_step(apic, ctx, s, dev, det | extra, mu_pair))
    with apic.Context(0) as ctx:  # a fresh context, no graphs, strict launch order
        ctx.set_graphs(False)
        ctx.set_overlap(False)
        runs.append(_step(apic, ctx, s, dev, det | extra, mu_pair))
    for k, (v, Cm) in enumerate(runs[1:], 1):
        assert torch.equal(v, runs[0][0]) and torch.equal(Cm, runs[0][1]), f"run {k} differs from run 0"
    v, Cm = runs[0]
    env = None
    if case == "sep23":  # a step at dn = 0: measured beyond the oracle's own envelope there
        _, _, ev, eC = discontinuity.envelope(
            lambda vv, CC: oracle.contact_step(s.x, vv, CC, s.m, s.nrm, s.body, s.h, s.mu, s.n_iter,
                                               n_bodies=s.n_bodies, flags=oflags)[:2], s.v, s.C)
        env = (ev, eC)
    _close(s, v.cpu().double().numpy(), Cm.cpu().double().numpy(), ref[0], ref[1], case, env)


def test_same_bits_alone_and_in_any_batch(apic):
    """Scales are per scene and items never mix scenes, so a scene's result
    does not depend on what else is in the batch."""
    import torch

    det = apic.APIC_DETERMINISTIC
    parts = [scenes.four_bodies(scale=0.05), scenes.random_cloud(7000, n_bodies=3, seed=41, h=0.04, n_iter=8),
             scenes.two_cubes(mu=0.3, n_iter=8)]
    devs = [_dev(s) for s in parts]
    with apic.Context(0) as ctx:
        alone = [_step(apic, ctx, s, d, det) for s, d in zip(parts, devs)]
        for order in ([0, 1, 2], [2, 0, 1], [1, 2]):
            bs = [apic.BatchScene(*devs[i], parts[i].h, parts[i].mu, n_bodies=parts[i].n_bodies) for i in order]
            apic.contact_step_batched(ctx, bs, 8, flags=det)
            torch.cuda.synchronize()
            for i, b in zip(order, bs):
                assert torch.equal(b.v_out, alone[i][0]) and torch.equal(b.C_out, alone[i][1]), (
                    f"scene {i} in batch {order}")


def test_static_entry_point_gives_the_same_bits(apic):
    import torch

    det = apic.APIC_DETERMINISTIC
    s = scenes.four_bodies(scale=0.05)
    X, V, Cc, M, NR, B = _dev(s)
    with apic.Context(0) as ctx:
        v0, C0 = _step(apic, ctx, s, (X, V, Cc, M, NR, B), det)
    r = apic.contact_step_static(X, V, Cc, M, NR, B, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies, flags=det)
    torch.cuda.synchronize()
    assert torch.equal(r.v, v0) and torch.equal(r.C, C0)


def test_rejected_with_fp64(apic):
    import torch

    s = scenes.two_cubes(mu=0.3, n_iter=2)
    f = s.astype(np.float64)
    d = torch.device("cuda:0")
    t = [torch.as_tensor(np.ascontiguousarray(a), device=d) for a in (f.x, f.v, f.C, f.m, f.nrm)]
    body = torch.as_tensor(f.body, device=d, dtype=torch.int32)
    with apic.Context(0) as ctx, pytest.raises(apic.ApicError, match="FP32 path"):
        apic.contact_step(ctx, *t, body, s.h, s.mu, s.n_iter, n_bodies=2, flags=apic.APIC_DETERMINISTIC)


@pytest.mark.parametrize("n_iter", [0, 3])
def test_non_finite_input_fails_and_leaves_outputs(apic, n_iter):
    """A NaN velocity makes its scene's term bound non-finite: both attempts
    record it, the call fails, the outputs keep what they held, and the
    context steps the next (finite) scene normally."""
    import torch

    det = apic.APIC_DETERMINISTIC
    s = scenes.random_cloud(3000, n_bodies=2, seed=43, h=0.05, n_iter=n_iter)
    X, V, Cc, M, NR, B = _dev(s)
    Vbad = V.clone()
    Vbad[17, 1] = float("nan")
    vo = torch.full_like(V, 7.0)
    Co = torch.full_like(Cc, 7.0)
    with apic.Context(0) as ctx:
        with pytest.raises(apic.ApicError, match="fixed-point range"):
            apic.contact_step(ctx, X, Vbad, Cc, M, NR, B, s.h, s.mu, s.n_iter, n_bodies=2, flags=det, v_out=vo,
                              C_out=Co)
        torch.cuda.synchronize()
        assert bool((vo == 7.0).all()) and bool((Co == 7.0).all())
        ref = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, s.mu, s.n_iter, n_bodies=2)
        v, Cm = _step(apic, ctx, s, (X, V, Cc, M, NR, B), det)
        _close(s, v.cpu().double().numpy(), Cm.cpu().double().numpy(), ref[0], ref[1], "after the failure")
