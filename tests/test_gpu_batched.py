"""apic_contact_step_batched: several independent scenes in one call must give,
scene by scene, what the oracle gives for each scene alone."""
import numpy as np
import pytest

import oracle
import parity_log
from paper_2108_02259_gb300 import scenes

pytestmark = pytest.mark.gpu

TOL_V, TOL_C, TOL_MOM = 1e-5, 1e-4, 1e-6


@pytest.fixture(scope="module")
def ctx():
    from paper_2108_02259_gb300 import apic, build

    build.build()
    c = apic.Context(0)
    yield c
    c.close()


def _dev(s, dt):
    import torch

    f = s.astype(dt)
    tdt = torch.float32 if dt == np.float32 else torch.float64
    dev = torch.device("cuda:0")

    def t(a, d):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=d).to(dev)

    return t(f.x, torch.float64), t(f.v, tdt), t(f.C, tdt), t(f.m, tdt), t(f.nrm, tdt), t(f.body, torch.int32)


def _check(s, v, Cm, st, mu_pair=None, tol_v=TOL_V, tol_c=TOL_C, label=""):
    rv, rC, rst = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies,
                                      mu_pair=mu_pair)
    vs = np.abs(s.v).max()
    cs = max(np.linalg.norm(s.C.reshape(-1, 9), axis=1).max(), np.linalg.norm(rC.reshape(-1, 9), axis=1).max())
    cs = cs if cs > 0 else 2 * vs / s.h
    ev, ec = np.abs(v - rv).max() / vs, np.abs(Cm - rC).max() / cs
    parity_log.record(f"batched {label}", s.n, {"v": ev, "C": ec}, {"v": tol_v, "C": tol_c})
    assert ev <= tol_v and ec <= tol_c, (label, ev, ec)
    if st is not None:
        sP = np.sum(s.m * np.linalg.norm(s.v, axis=1))
        assert np.abs(st["P_out"] - st["P_in"]).max() <= TOL_MOM * sP
        assert st["multibody_nodes"] == rst["multibody_nodes"]


def _mixed_batch():
    rng = np.random.default_rng(123)
    sc = [scenes.multi_body_scene(rng, 1500, 2, 1 / 64, n_iter=3),
          scenes.two_cubes(mu=0.0, n_iter=3),
          scenes.multi_body_scene(rng, 4000, 5, 1 / 128, mu=0.5, n_iter=3),
          scenes.random_cloud(800, n_bodies=3, seed=4, h=0.1, n_iter=3, origin=(-2.0, 1.0, 0.5)),
          scenes.multi_body_scene(rng, 2500, 3, 1 / 256, mu=0.1, n_iter=3)]
    # same location for two scenes: scenes are independent even when they overlap in space
    sc.append(scenes.Scene(sc[0].x.copy(), -sc[0].v, -sc[0].C, sc[0].m, sc[0].nrm, sc[0].body, sc[0].n_bodies, sc[0].h,
                           0.3, 3))
    return sc


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_batched_matches_oracle_per_scene(ctx, dt):
    import torch

    from paper_2108_02259_gb300 import apic

    sc = _mixed_batch()
    mp = np.array([[0.2, 0.4, 0.3], [0.4, 0.1, 0.25], [0.3, 0.25, 0.5]])
    bs = []
    for i, s in enumerate(sc):
        X, V, C, M, N, B = _dev(s, dt)
        bs.append(apic.BatchScene(X, V, C, M, N, B, s.h, s.mu, n_bodies=s.n_bodies,
                                  mu_pair=mp if i == 4 else None))
    stats = apic.contact_step_batched(ctx, bs, n_iter=3, stats=True)
    torch.cuda.synchronize()
    tol = (TOL_V, TOL_C) if dt == np.float32 else (1e-11, 1e-11)
    for i, (s, b) in enumerate(zip(sc, bs)):
        _check(s, b.v_out.cpu().double().numpy(), b.C_out.cpu().double().numpy(), stats[i],
               mu_pair=mp if i == 4 else None, tol_v=tol[0], tol_c=tol[1], label=f"scene {i} {dt.__name__}")


def test_batched_equals_single_scene_calls(ctx):
    import torch

    from paper_2108_02259_gb300 import apic

    sc = _mixed_batch()
    bs, single = [], []
    for s in sc:
        X, V, C, M, N, B = _dev(s, np.float32)
        bs.append(apic.BatchScene(X, V, C, M, N, B, s.h, s.mu, n_bodies=s.n_bodies))
        r = apic.contact_step(ctx, X, V, C, M, N, B, s.h, s.mu, 3, n_bodies=s.n_bodies)
        single.append((r.v, r.C))
    apic.contact_step_batched(ctx, bs, n_iter=3)
    torch.cuda.synchronize()
    for s, b, (v1, C1) in zip(sc, bs, single):
        vs = np.abs(s.v).max()
        assert torch.abs(b.v_out - v1).max().item() <= 2e-6 * vs
        assert torch.abs(b.C_out - C1).max().item() <= 2e-5 * max(np.abs(s.C).max(), 2 * vs / s.h)


def test_batched_host_pointers_and_empty_scene(ctx):
    from paper_2108_02259_gb300 import apic

    sc = _mixed_batch()[:3]
    empty = scenes.Scene(sc[0].x[:0], sc[0].v[:0], sc[0].C[:0], sc[0].m[:0], sc[0].nrm[:0], sc[0].body[:0], 1,
                         0.05, 0.3, 3)
    sc.insert(1, empty)
    bs = []
    for s in sc:
        f = s.astype(np.float32)
        bs.append(apic.BatchScene(f.x, f.v, f.C, f.m, f.nrm, f.body, s.h, s.mu, n_bodies=s.n_bodies))
    stats = apic.contact_step_batched(ctx, bs, n_iter=3, stats=True)
    assert stats[1]["work_items"] == 0
    for i, (s, b) in enumerate(zip(sc, bs)):
        if s.n:
            _check(s, b.v_out.astype(np.float64), b.C_out.astype(np.float64), stats[i], tol_v=TOL_V,
                   label=f"host scene {i}")


def test_batched_rejects_mixed_flags(ctx):
    from paper_2108_02259_gb300 import apic

    sc = _mixed_batch()[:2]
    bs = []
    for s in sc:
        X, V, C, M, N, B = _dev(s, np.float32)
        bs.append(apic.BatchScene(X, V, C, M, N, B, s.h, s.mu, n_bodies=s.n_bodies))
    lib = apic.load()
    import ctypes

    arr = (apic.StepArgs * 2)()
    for i, b in enumerate(bs):
        arr[i] = apic.StepArgs(int(b.x.shape[0]), b.n_bodies, 3 + i, b.body.data_ptr(), b.x.data_ptr(),
                               b.v.data_ptr(), b.C.data_ptr(), b.m.data_ptr(), b.nrm.data_ptr(), b.v_out.data_ptr(),
                               b.C_out.data_ptr(), b.h, b.mu, None, 0)
    rc = lib.apic_contact_step_batched(ctx.handle, arr, 2, None, None)
    assert rc == apic.APIC_ERR_INVALID_ARG
    assert b"n_iter" in lib.apic_last_error()


def test_batched_calls_with_changing_membership_and_inputs(ctx):
    """Consecutive batched calls whose membership changes (all scenes, a
    subset, all again ...) and whose velocities change every call: each
    scene's result matches the oracle for that call's inputs, through graph
    captures, replays and re-captures."""
    import torch

    from paper_2108_02259_gb300 import apic

    sc = _mixed_batch()
    dev = [_dev(s, np.float32) for s in sc]
    plan = [range(6), range(6), [0, 2, 4], [0, 2, 4], [0, 2, 4], range(6), range(6), range(6)]
    for k, members in enumerate(plan):
        scale = 1.0 + 0.1 * k
        bs, used = [], []
        for i in members:
            X, V, Cc, M, NR, B = dev[i]
            s = sc[i]
            bs.append(apic.BatchScene(X, V * scale, Cc * scale, M, NR, B, s.h, s.mu, n_bodies=s.n_bodies))
            used.append(scenes.Scene(**{**s.__dict__, "v": s.v * scale, "C": s.C * scale}))
        apic.contact_step_batched(ctx, bs, 3)
        torch.cuda.synchronize()
        for s, b in zip(used, bs):
            _check(s, b.v_out.cpu().double().numpy(), b.C_out.cpu().double().numpy().reshape(-1, 3, 3), None,
                   label=f"call {k}")
    assert ctx.profile()["graph_launches"] > 0


def test_page_locked_host_arrays(ctx):
    """Host-pointer calls whose arrays are page-locked take the one-kernel
    staging path (inputs and results); some views start off 16-byte
    boundaries.  Results must match the oracle and the pageable path."""
    import torch

    from paper_2108_02259_gb300 import apic

    def pinned(a, dt, offset_rows=0):
        a = np.ascontiguousarray(a, dt)
        t = torch.empty((a.shape[0] + offset_rows,) + a.shape[1:], dtype=getattr(torch, np.dtype(dt).name)).pin_memory()
        v = t.numpy()[offset_rows:]  # a view starting offset_rows rows in
        v[...] = a
        return v

    sc = _mixed_batch()
    pin_scenes, page_scenes = [], []
    for k, s in enumerate(sc):
        f = s.astype(np.float32)
        off = k % 2  # every other scene's arrays start one row in
        pin_scenes.append(apic.BatchScene(pinned(f.x, np.float64, off), pinned(f.v, np.float32, off),
                                          pinned(f.C, np.float32, off), pinned(f.m, np.float32, off),
                                          pinned(f.nrm, np.float32, off), pinned(f.body, np.int32, off), s.h, s.mu,
                                          n_bodies=s.n_bodies, v_out=pinned(np.zeros_like(f.v), np.float32, off),
                                          C_out=pinned(np.zeros_like(f.C), np.float32, off)))
        page_scenes.append(apic.BatchScene(f.x, f.v, f.C, f.m, f.nrm, f.body, s.h, s.mu, n_bodies=s.n_bodies))
    for _ in range(2):  # direct launches, then graph replay of the sizing sequence
        apic.contact_step_batched(ctx, pin_scenes, 3)
        apic.contact_step_batched(ctx, page_scenes, 3)
        for s, a, b in zip(sc, pin_scenes, page_scenes):
            _check(s, a.v_out.astype(np.float64), a.C_out.astype(np.float64).reshape(-1, 3, 3), None, label="pinned")
            vs = np.abs(s.v).max()
            assert np.abs(a.v_out - b.v_out).max() <= 2 * TOL_V * vs
    # single scene, pinned
    s = sc[2]
    f = s.astype(np.float32)
    vo, Co = pinned(np.zeros_like(f.v), np.float32, 1), pinned(np.zeros_like(f.C), np.float32, 1)
    r = apic.contact_step(ctx, pinned(f.x, np.float64), pinned(f.v, np.float32, 1), pinned(f.C, np.float32),
                          pinned(f.m, np.float32, 1), pinned(f.nrm, np.float32), pinned(f.body, np.int32, 1), s.h, s.mu,
                          3, n_bodies=s.n_bodies, v_out=vo, C_out=Co)
    _check(s, r.v.astype(np.float64), r.C.astype(np.float64).reshape(-1, 3, 3), None, label="pinned single")


def test_page_locked_repeat_calls_pick_up_new_inputs(ctx):
    """With page-locked arrays, v and C are staged on a side stream while the
    sizing sequence runs, and their sorted planes are gathered at the start
    of the passes.  Repeated calls (direct, captured, replayed) must each see
    the velocities written into the same host buffers just before the call."""
    import torch

    from paper_2108_02259_gb300 import apic

    def pinned(a, dt):
        a = np.ascontiguousarray(a, dt)
        t = torch.empty(a.shape, dtype=getattr(torch, np.dtype(dt).name)).pin_memory()
        v = t.numpy()
        v[...] = a
        return v

    s = scenes.four_bodies(scale=0.05, n_iter=3)
    f = s.astype(np.float32)
    X, V, Cc, M, NR, B = (pinned(f.x, np.float64), pinned(f.v, np.float32), pinned(f.C, np.float32),
                          pinned(f.m, np.float32), pinned(f.nrm, np.float32), pinned(f.body, np.int32))
    vo, Co = pinned(np.zeros_like(f.v), np.float32), pinned(np.zeros_like(f.C), np.float32)
    for k in range(4):
        scale = 1.0 + 0.5 * k
        V[...] = f.v * scale
        Cc[...] = f.C * scale
        # the normals cross in a copy of their own, waited for inside the
        # captured series: every other call takes them away (all interior)
        nrm = s.nrm if k % 2 == 0 else np.zeros_like(s.nrm)
        NR[...] = nrm
        apic.contact_step(ctx, X, V, Cc, M, NR, B, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies, v_out=vo, C_out=Co)
        sk = scenes.Scene(**{**s.__dict__, "v": s.v * scale, "C": s.C * scale, "nrm": nrm})
        _check(sk, vo.astype(np.float64), Co.astype(np.float64).reshape(-1, 3, 3), None, label=f"call {k}")


def test_page_locked_arrays_of_many_chunks(ctx):
    """The copy beside the sizing sequence splits the arrays into 64 KB
    chunks over a bounded grid, so each CTA walks several chunks across
    array boundaries.  A 200,000-particle scene (about 180 chunks of
    normals, v and C) with arrays starting off 16-byte boundaries must give
    what the device-pointer call gives."""
    import torch

    from paper_2108_02259_gb300 import apic

    def pinned(a, dt, offset_rows):
        a = np.ascontiguousarray(a, dt)
        t = torch.empty((a.shape[0] + offset_rows,) + a.shape[1:], dtype=getattr(torch, np.dtype(dt).name)).pin_memory()
        v = t.numpy()[offset_rows:]
        v[...] = a
        return v

    s = scenes.four_bodies(n_iter=3)
    f = s.astype(np.float32)
    d = torch.device("cuda:0")

    def dev(a, dt):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=d)

    ref = apic.contact_step(ctx, dev(f.x, torch.float64), dev(f.v, torch.float32), dev(f.C, torch.float32),
                            dev(f.m, torch.float32), dev(f.nrm, torch.float32), dev(f.body, torch.int32), s.h, s.mu,
                            s.n_iter, n_bodies=s.n_bodies)
    rv, rC = ref.v.cpu().numpy().astype(np.float64), ref.C.cpu().numpy().astype(np.float64)
    vs = np.abs(s.v).max()
    cs = max(np.linalg.norm(rC.reshape(-1, 9), axis=1).max(), 2 * vs / s.h)
    for off in (0, 1):
        vo, Co = pinned(np.zeros_like(f.v), np.float32, off), pinned(np.zeros_like(f.C), np.float32, off)
        for _ in range(3):  # direct launches, capture, replay
            apic.contact_step(ctx, pinned(f.x, np.float64, off), pinned(f.v, np.float32, off),
                              pinned(f.C, np.float32, off), pinned(f.m, np.float32, off),
                              pinned(f.nrm, np.float32, off), pinned(f.body, np.int32, off), s.h, s.mu, s.n_iter,
                              n_bodies=s.n_bodies, v_out=vo, C_out=Co)
            ev = np.abs(vo - rv).max() / vs
            ec = np.abs(Co.reshape(-1, 9) - rC.reshape(-1, 9)).max() / cs
            parity_log.record(f"pinned, many chunks, offset {off} vs device call", s.n, {"v": ev, "C": ec},
                              {"v": TOL_V, "C": TOL_C})
            assert ev <= TOL_V and ec <= TOL_C, (off, ev, ec)


def test_failed_batch_leaves_every_scene_untouched(ctx):
    """A batched call refused for one scene's data (here APIC_CHECK finds a
    NaN velocity) writes no scene's outputs, so a caller can step the valid
    scenes again on their own."""
    import torch

    from paper_2108_02259_gb300 import apic

    d = torch.device("cuda:0")
    sc = _mixed_batch()[:3]
    bs = []
    for k, s in enumerate(sc):
        f = s.astype(np.float32)
        t = [torch.as_tensor(np.ascontiguousarray(a), device=d) for a in (f.x, f.v, f.C, f.m, f.nrm)]
        t[0] = t[0].double()
        if k == 1:
            t[1][4, 0] = float("nan")
        body = torch.as_tensor(f.body, device=d, dtype=torch.int32)
        bs.append(apic.BatchScene(*t, body, s.h, s.mu, n_bodies=s.n_bodies, v_out=torch.full_like(t[1], 7.0),
                                  C_out=torch.full_like(t[2], 7.0)))
    for flags, msg in ((apic.APIC_CHECK, "not finite"), (apic.APIC_CHECK | apic.APIC_DETERMINISTIC, "not finite"),
                       (apic.APIC_DETERMINISTIC, "fixed-point range")):  # the last: refused after the passes ran
        with pytest.raises(apic.ApicError, match=msg):
            apic.contact_step_batched(ctx, bs, 3, flags=flags)
        torch.cuda.synchronize()
        assert all(bool((b.v_out == 7.0).all()) and bool((b.C_out == 7.0).all()) for b in bs)


def test_batched64_full_size_matches_oracle_per_scene(ctx):
    """The benchmarked batch (64 scenes, 2,080,567 nodes, 1k-200k per scene,
    2-6 bodies, h in {1/64, 1/128, 1/256}, N = 8) in one batched call: every
    particle of every scene against the oracle run on that scene alone (in
    parallel threads; the oracle holds no global state)."""
    from concurrent.futures import ThreadPoolExecutor

    import torch

    from paper_2108_02259_gb300 import apic

    sc = scenes.batch_of_scenes(64, seed=scenes.SEED_BASE + 4)
    bs = []
    for s in sc:
        X, V, C, M, N, B = _dev(s, np.float32)
        bs.append(apic.BatchScene(X, V, C, M, N, B, s.h, s.mu, n_bodies=s.n_bodies))
    stats = apic.contact_step_batched(ctx, bs, n_iter=sc[0].n_iter, stats=True)
    torch.cuda.synchronize()
    got = [(b.v_out.cpu().double().numpy(), b.C_out.cpu().double().numpy()) for b in bs]

    def ref(s):
        return oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies)

    with ThreadPoolExecutor(min(16, len(sc))) as ex:
        refs = list(ex.map(ref, sc))
    for i, (s, (v, Cm), (rv, rC, rst)) in enumerate(zip(sc, got, refs)):
        vs = np.abs(s.v).max()
        cs = max(np.linalg.norm(s.C.reshape(-1, 9), axis=1).max(), np.linalg.norm(rC.reshape(-1, 9), axis=1).max())
        ev, ec = np.abs(v - rv).max() / vs, np.abs(Cm - rC).max() / cs
        parity_log.record(f"batched64 scene {i} (h=1/{round(1 / s.h)}, {s.n_bodies} bodies)", s.n,
                          {"v": ev, "C": ec}, {"v": TOL_V, "C": TOL_C})
        assert ev <= TOL_V and ec <= TOL_C, (i, ev, ec)
        sP = np.sum(s.m * np.linalg.norm(s.v, axis=1))
        assert np.abs(stats[i]["P_out"] - stats[i]["P_in"]).max() <= TOL_MOM * sP
        assert stats[i]["multibody_nodes"] == rst["multibody_nodes"], i


def test_growing_scene_table_keeps_the_copy_table():
    """A context that stages page-locked arrays (its pinned copy table), then
    grows its pinned scene table for a larger batch, then stages page-locked
    arrays again: results match the oracle each time, and destroying the
    context leaves no pending CUDA error for the next call."""
    import torch

    from paper_2108_02259_gb300 import apic

    def pinned(a, dt):
        a = np.ascontiguousarray(a, dt)
        t = torch.empty(a.shape, dtype=getattr(torch, np.dtype(dt).name)).pin_memory()
        v = t.numpy()
        v[...] = a
        return v

    small = _mixed_batch()[:3]
    large = _mixed_batch() + _mixed_batch()[:4]

    def pinned_scenes(sc):
        out = []
        for s in sc:
            f = s.astype(np.float32)
            out.append(apic.BatchScene(pinned(f.x, np.float64), pinned(f.v, np.float32), pinned(f.C, np.float32),
                                       pinned(f.m, np.float32), pinned(f.nrm, np.float32), pinned(f.body, np.int32),
                                       s.h, s.mu, n_bodies=s.n_bodies, v_out=pinned(np.zeros_like(f.v), np.float32),
                                       C_out=pinned(np.zeros_like(f.C), np.float32)))
        return out

    with apic.Context(0) as c:
        for sc in (small, large, small):
            bs = pinned_scenes(sc)
            apic.contact_step_batched(c, bs, 3)
            for i, (s, b) in enumerate(zip(sc, bs)):
                _check(s, b.v_out.astype(np.float64), b.C_out.astype(np.float64).reshape(-1, 3, 3), None,
                       label=f"pinned after growth, {len(sc)} scenes, scene {i}")
    with apic.Context(0) as c:  # a fresh context's first launch sees no stale error
        s = small[0]
        f = s.astype(np.float32)
        r = apic.contact_step(c, f.x, f.v, f.C, f.m, f.nrm, f.body, s.h, s.mu, 3, n_bodies=s.n_bodies)
        _check(s, r.v.astype(np.float64), r.C.astype(np.float64).reshape(-1, 3, 3), None, label="after destroy")


def test_non_finite_velocity_stays_in_its_scene(ctx):
    """Without APIC_CHECK a NaN velocity is not refused: as with floating-point
    sums it reaches the outputs of its own scene (the transfer kernel's
    fixed-point node sums turn a non-finite term bound into NaN node sums),
    and an independent scene of the same batch keeps its oracle result."""
    import torch

    from paper_2108_02259_gb300 import apic

    rng = np.random.default_rng(5)
    bad = scenes.multi_body_scene(rng, 3000, 3, 1 / 64, n_iter=3)
    good = scenes.multi_body_scene(rng, 2000, 2, 1 / 128, mu=0.2, n_iter=3)
    d = torch.device("cuda:0")

    def dev(a, dt):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=d)

    batch = []
    for k, s in enumerate((bad, good)):
        f = s.astype(np.float32)
        v = f.v.copy()
        if k == 0:
            v[1234, 1] = np.nan
        batch.append(apic.BatchScene(dev(f.x, torch.float64), dev(v, torch.float32), dev(f.C, torch.float32),
                                     dev(f.m, torch.float32), dev(f.nrm, torch.float32), dev(f.body, torch.int32),
                                     s.h, s.mu, n_bodies=s.n_bodies))
    apic.contact_step_batched(ctx, batch, 3)
    torch.cuda.synchronize()
    vb = batch[0].v_out.cpu().numpy()
    assert np.isnan(vb[1234]).any()
    _check(good, batch[1].v_out.cpu().double().numpy(), batch[1].C_out.cpu().double().numpy().reshape(-1, 3, 3),
           None, label="finite scene beside a NaN one")
