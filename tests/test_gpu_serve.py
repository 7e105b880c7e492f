"""The serving loop: resident simulations stepped by batching workers.

Each served result must equal what the oracle gives for that simulation
stepped alone, and a simulation must give the same result alone and in a mix
of concurrent simulations (within the FP32 tolerance)."""
import threading
import time

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
    from paper_2108_02259_gb300 import apic, build

    build.build()
    return apic


def _sims(k, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(k):
        h = [1 / 64, 1 / 128][i % 2]
        out.append(scenes.multi_body_scene(rng, int(rng.integers(800, 4000)), int(rng.integers(2, 5)), h,
                                           mu=float(rng.uniform(0, 0.5)), n_iter=3))
    return out


def _oracle_steps(s, steps, dt):
    x, v, Cm = s.x.copy(), s.v.copy(), s.C.copy()
    for _ in range(steps):
        v, Cm, _ = oracle.contact_step(x, v, Cm, s.m, s.nrm, s.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies)
        x = x + dt * v
    return x, v, Cm


def _err(s, got, ref):
    vs = np.abs(s.v).max()
    cs = max(np.abs(ref[2]).max(), np.abs(s.C).max(), 2 * vs / s.h)
    return np.abs(got[1] - ref[1]).max() / vs, np.abs(got[2] - ref[2]).max() / cs, np.abs(got[0] - ref[0]).max()


def test_served_steps_match_oracle(apic):
    sims = _sims(5)
    with apic.Server(0, n_workers=2, max_batch_scenes=8) as srv:
        handles = []
        for s in sims:
            f = s.astype(np.float32)
            handles.append(srv.open_sim(f.x, f.v, f.C, f.m, f.nrm, f.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies))
        steps = 3
        dts = [0.1 * s.h / np.abs(s.v).max() for s in sims]
        tickets = []
        for _ in range(steps):
            for hdl, dt in zip(handles, dts):
                tickets.append(hdl.submit(dt))
        for t in tickets:
            assert srv.wait(t, 60.0) >= 0.0
        st = srv.stats()
        assert st["completed"] == steps * len(sims) and st["failed"] == 0
        assert st["latency_p99_ms"] >= st["latency_p50_ms"] > 0
        for s, hdl, dt in zip(sims, handles, dts):
            got = hdl.read()
            ev, ec, ex = _err(s, got, _oracle_steps(s, steps, dt))
            xtol = steps * dt * TOL_V * np.abs(s.v).max()
            parity_log.record(f"served, {steps} steps", s.n, {"v": ev, "C": ec, "x": ex / xtol},
                              {"v": TOL_V, "C": TOL_C, "x": 1.0})
            # x moves by dt * v_hat each step: its error is bounded by the v error times steps * dt
            assert ev <= TOL_V and ec <= TOL_C and ex <= xtol
            hdl.close()


@pytest.mark.parametrize("det", [False, True])
def test_same_result_alone_and_in_the_mix(apic, det):
    """A simulation stepped alone and stepped while many others are submitted
    concurrently (so its requests share batches and overlap with other
    batches on the GPU) reaches the same state: within the FP32 tolerance,
    and bit for bit when every simulation runs with APIC_DETERMINISTIC."""
    target = _sims(1, seed=7)[0]
    others = _sims(12, seed=8)
    steps = 4
    dt = 0.1 * target.h / np.abs(target.v).max()
    flags = apic.APIC_DETERMINISTIC if det else 0

    def run(with_mix):
        with apic.Server(0, n_workers=3, max_batch_scenes=16) as srv:
            f = target.astype(np.float32)
            a = srv.open_sim(f.x, f.v, f.C, f.m, f.nrm, f.body, target.h, target.mu, target.n_iter,
                             n_bodies=target.n_bodies, flags=flags)
            mix = []
            if with_mix:
                for s in others:
                    g = s.astype(np.float32)
                    mix.append(srv.open_sim(g.x, g.v, g.C, g.m, g.nrm, g.body, s.h, s.mu, s.n_iter,
                                            n_bodies=s.n_bodies, flags=flags))
            stop = threading.Event()

            def churn():
                while not stop.is_set():
                    ts = [m.submit(0.0) for m in mix]
                    for t in ts:
                        srv.wait(t, 60.0)

            th = threading.Thread(target=churn) if with_mix else None
            if th:
                th.start()
            for _ in range(steps):
                srv.wait(a.submit(dt), 60.0)
                time.sleep(0.002)
            stop.set()
            if th:
                th.join()
            out = a.read()
            batches = srv.stats()["mean_batch_scenes"]
            return out, batches

    alone, _ = run(False)
    mixed, mean_batch = run(True)
    assert mean_batch > 1.0  # the target really shared batches
    ev, ec, ex = _err(target, mixed, alone)
    parity_log.record(f"served alone vs in the mix (det={det}, mean batch {mean_batch:.2f})", target.n,
                      {"v": ev, "C": ec}, {"v": TOL_V, "C": TOL_C})
    assert ev <= TOL_V and ec <= TOL_C and ex <= steps * dt * TOL_V * np.abs(target.v).max()
    if det:
        assert all(np.array_equal(p, q) for p, q in zip(mixed, alone))


def test_admission_by_budget(apic):
    s = _sims(1, seed=3)[0]
    f = s.astype(np.float32)
    # resident state is 92 B per particle (FP32); admission also reserves
    # 640 B per particle of step scratch for the simulation being admitted:
    # two fit in 2*92n + 640n, a third needs 3*92n + 640n.
    budget = s.n * (2 * 92 + 640) + s.n * 46
    with apic.Server(0, hbm_budget_bytes=budget, n_workers=1) as srv:
        a = srv.open_sim(f.x, f.v, f.C, f.m, f.nrm, f.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies)
        b = srv.open_sim(f.x, f.v, f.C, f.m, f.nrm, f.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies)
        with pytest.raises(apic.ApicError) as e:
            srv.open_sim(f.x, f.v, f.C, f.m, f.nrm, f.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies)
        assert e.value.code == apic.APIC_ERR_ADMISSION
        b.close()
        c = srv.open_sim(f.x, f.v, f.C, f.m, f.nrm, f.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies)
        srv.wait(c.submit(0.0), 60.0)
        srv.wait(a.submit(0.0), 60.0)
        assert srv.stats()["open_sims"] == 2


def test_wait_timeout_and_poll(apic):
    s = scenes.four_bodies(scale=0.3)
    f = s.astype(np.float32)
    with apic.Server(0, n_workers=1) as srv:
        a = srv.open_sim(f.x, f.v, f.C, f.m, f.nrm, f.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies)
        ts = [a.submit(0.0) for _ in range(20)]
        with pytest.raises(apic.ApicError) as e:
            srv.wait(ts[-1], 1e-6)
        assert e.value.code == apic.APIC_ERR_TIMEOUT
        srv.wait(ts[-1], 120.0)
        done, lat = srv.poll(ts[0])
        assert done and lat > 0
        # a reported ticket is forgotten
        for t in (ts[0], ts[-1]):
            with pytest.raises(apic.ApicError) as e:
                srv.poll(t)
            assert e.value.code == apic.APIC_ERR_INVALID_ARG
        # the others are still known until their simulation closes
        assert srv.poll(ts[5])[0]
        assert srv.wait(ts[6], 1.0) > 0
        a.close()
        with pytest.raises(apic.ApicError):
            srv.poll(ts[7])


def test_mixed_precisions_variants_and_iterations(apic):
    """One server, simulations that must never share a batch (FP64 and FP32,
    PIC, the Sec. 2.3 rule, different N) and one with a body-pair friction
    table, submitted interleaved: each matches the oracle stepped alone."""
    rng = np.random.default_rng(7)
    PIC, SEP23 = apic.APIC_VARIANT_PIC, apic.APIC_VARIANT_SEP23
    cases = []
    for k, (dt, flags, n_iter) in enumerate([(np.float64, 0, 3), (np.float32, 0, 3), (np.float32, PIC, 3),
                                             (np.float32, SEP23, 2), (np.float32, 0, 5), (np.float64, PIC, 1)]):
        s = scenes.multi_body_scene(rng, int(rng.integers(800, 2500)), 3, 1 / 64, mu=0.3, n_iter=n_iter)
        mp = None
        if k == 4:
            a = rng.uniform(0.1, 0.5, (3, 3))
            mp = (a + a.T) / 2
        cases.append((s, dt, flags, mp))
    with apic.Server(0, n_workers=2, max_batch_scenes=8) as srv:
        hs = []
        for s, dt, flags, mp in cases:
            f = s.astype(dt)
            hs.append(srv.open_sim(f.x, f.v, f.C, f.m, f.nrm, f.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies,
                                   mu_pair=mp, flags=flags))
        tickets = [h.submit(0.0) for _ in range(2) for h in hs]
        for t in tickets:
            srv.wait(t, 60.0)
        assert srv.stats()["failed"] == 0
        oflag = {0: 0, PIC: oracle.FLAG_PIC, SEP23: oracle.FLAG_SEP23}
        for (s, dt, flags, mp), h in zip(cases, hs):
            def two_steps(v, Cm, s=s, mp=mp, flags=flags):
                for _ in range(2):
                    v, Cm, _ = oracle.contact_step(s.x, v, Cm, s.m, s.nrm, s.body, s.h, s.mu, s.n_iter,
                                                   n_bodies=s.n_bodies, mu_pair=mp, flags=oflag[flags])
                return v, Cm

            if flags == SEP23:
                # a step at dn = 0 (tests/discontinuity.py): beyond the oracle's own envelope
                v, Cm, env_v, env_C = discontinuity.envelope(two_steps, s.v, s.C)
            else:
                v, Cm = two_steps(s.v.copy(), s.C.copy())
                env_v, env_C = np.zeros_like(v), np.zeros_like(Cm)
            x, gv, gC = h.read()
            vs = np.abs(s.v).max()
            cs = max(np.abs(Cm).max(), np.abs(s.C).max(), 2 * vs / s.h)
            tol = (1e-11, 1e-11) if dt == np.float64 else (TOL_V, TOL_C)
            ev = discontinuity.excess(gv, v, env_v, vs)
            ec = discontinuity.excess(gC.reshape(-1, 9), Cm.reshape(-1, 9), env_C.reshape(-1, 9), cs)
            parity_log.record(f"served mixed kinds {np.dtype(dt).name} flags={flags} N={s.n_iter}", s.n,
                              {"v": ev, "C": ec}, {"v": tol[0], "C": tol[1]})
            assert ev <= tol[0], (dt, flags, s.n_iter)
            assert ec <= tol[1], (dt, flags, s.n_iter)
            assert np.all(x == s.x)  # dt_advect = 0
            h.close()


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_checkpoint_and_resume(apic, dt):
    """A simulation exported after two steps, closed, and imported again
    continues like one that was never interrupted; broken checkpoints are
    refused."""
    rng = np.random.default_rng(11)
    s = scenes.multi_body_scene(rng, 2000, 3, 1 / 64, mu=0.3, n_iter=3)
    a = rng.uniform(0.1, 0.5, (3, 3))
    mp = (a + a.T) / 2
    f = s.astype(dt)
    step_dt = 0.1 * s.h / np.abs(s.v).max()
    with apic.Server(0, n_workers=1) as srv:
        ref = srv.open_sim(f.x, f.v, f.C, f.m, f.nrm, f.body, s.h, s.mu, s.n_iter, n_bodies=3, mu_pair=mp)
        sim = srv.open_sim(f.x, f.v, f.C, f.m, f.nrm, f.body, s.h, s.mu, s.n_iter, n_bodies=3, mu_pair=mp)
        for t in [ref.submit(step_dt) for _ in range(4)] + [sim.submit(step_dt) for _ in range(2)]:
            srv.wait(t, 60.0)
        ck = sim.export()
        x2, v2, C2 = sim.read()
        sim.close()
        back = srv.import_sim(ck)
        assert back.n == s.n and back.dtype == dt
        x3, v3, C3 = back.read()
        assert np.array_equal(x2, x3) and np.array_equal(v2, v3) and np.array_equal(C2, C3)
        for t in [back.submit(step_dt) for _ in range(2)]:
            srv.wait(t, 60.0)
        xr, vr, Cr = ref.read()
        xb, vb, Cb = back.read()
        vs = np.abs(s.v).max()
        tol = 1e-12 if dt == np.float64 else TOL_V
        assert np.abs(vb - vr).max() <= tol * vs
        assert np.abs(xb - xr).max() <= 4 * step_dt * tol * vs + 1e-15
        for bad in (ck[:-1], b"NOTACKPT" + ck[8:], ck[:20]):
            with pytest.raises(apic.ApicError) as e:
                srv.import_sim(bad)
            assert e.value.code == apic.APIC_ERR_INVALID_ARG
        ref.close()
        back.close()


@pytest.mark.parametrize("det", [False, True])
def test_invalid_request_fails_alone(apic, det):
    """One simulation with a NaN velocity among valid ones (all with
    APIC_CHECK, so they may share a batch): its request fails with the
    validation message, the batch is stepped again scene by scene, and every
    other request completes and matches the oracle."""
    flags = apic.APIC_CHECK | (apic.APIC_DETERMINISTIC if det else 0)
    sims = _sims(6, seed=21)
    bad = 2
    with apic.Server(0, n_workers=1, max_batch_scenes=16) as srv:
        # a larger request (other flags, so a batch of its own) keeps the one
        # worker busy while the six queue up and are then taken together
        big = scenes.four_bodies(scale=0.5)
        g = big.astype(np.float32)
        blocker = srv.open_sim(g.x, g.v, g.C, g.m, g.nrm, g.body, big.h, big.mu, big.n_iter,
                               n_bodies=big.n_bodies)
        t_block = blocker.submit(0.0)
        hs = []
        for k, s in enumerate(sims):
            f = s.astype(np.float32)
            v = f.v.copy()
            if k == bad:
                v[3, 1] = np.nan
            hs.append(srv.open_sim(f.x, v, f.C, f.m, f.nrm, f.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies,
                                   flags=flags))
        tickets = [h.submit(0.0) for h in hs]
        for k, t in enumerate(tickets):
            if k == bad:
                with pytest.raises(apic.ApicError, match="not finite"):
                    srv.wait(t, 60.0)
            else:
                srv.wait(t, 60.0)
        srv.wait(t_block, 60.0)
        st = srv.stats()
        assert st["failed"] == 1 and st["completed"] == len(sims)
        print(f"[serve] invalid request (det={det}): mean batch {st['mean_batch_scenes']:.2f}")
        for k, (s, h) in enumerate(zip(sims, hs)):
            x, v, Cm = h.read()
            if k == bad:
                assert np.isnan(v[3, 1])  # left as it was
                continue
            ref = _oracle_steps(s, 1, 0.0)
            ev, ec, ex = _err(s, (x, v, Cm), ref)
            assert ev <= TOL_V and ec <= TOL_C and ex == 0.0, (k, ev, ec)
