"""Server groups (apic_group_*): simulations spread over the members by HBM
budget, stepped by each member's own workers, with results equal to the
oracle's, and admission refused when no member has room.  The members here
are two independent servers on one GPU (a run of this suite has one); their
work never waits on one another."""
import numpy as np
import pytest

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


def _sims(k, seed):
    rng = np.random.default_rng(seed)
    return [scenes.multi_body_scene(rng, int(rng.integers(1000, 6000)), int(rng.integers(2, 5)),
                                    [1 / 64, 1 / 128][i % 2], mu=float(rng.uniform(0, 0.5)), n_iter=3)
            for i in range(k)]


def test_group_places_by_budget_and_steps_like_the_oracle(apic):
    sims = _sims(8, 21)
    with apic.Group([0, 0], hbm_budget_per_device=1 << 30, n_workers=2, max_batch_scenes=8) as g:
        hs = []
        for s in sims:
            f = s.astype(np.float32)
            hs.append(g.open_sim(f.x, f.v, f.C, f.m, f.nrm, f.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies))
        members = [h.member for h in hs]
        assert set(members) == {0, 1}  # both members got simulations
        # the members' resident bytes differ by at most the largest simulation's admission size
        res = [0, 0]
        for s, k in zip(sims, members):
            res[k] += s.n
        assert abs(res[0] - res[1]) <= max(s.n for s in sims)
        tickets = [(h, h.submit(0.0)) for _ in range(2) for h in hs]
        for h, t in tickets:
            assert h.wait(t, 60.0) >= 0.0
        st = g.stats()
        assert st["completed"] == 16 and st["failed"] == 0 and st["open_sims"] == 8
        assert st["latency_p99_ms"] >= st["latency_p50_ms"] > 0
        for s, h in zip(sims, hs):
            v, Cm = s.v.copy(), s.C.copy()
            for _ in range(2):
                v, Cm, _ = oracle.contact_step(s.x, v, Cm, s.m, s.nrm, s.body, s.h, s.mu, s.n_iter,
                                               n_bodies=s.n_bodies)
            x, gv, gC = h.read()
            vs = np.abs(s.v).max()
            cs = max(np.abs(Cm).max(), np.abs(s.C).max(), 2 * vs / s.h)
            ev, ec = np.abs(gv - v).max() / vs, np.abs(gC.reshape(-1, 9) - Cm.reshape(-1, 9)).max() / cs
            parity_log.record(f"group member {h.member}, 2 steps", s.n, {"v": ev, "C": ec},
                              {"v": TOL_V, "C": TOL_C})
            assert ev <= TOL_V and ec <= TOL_C
            h.close()


def test_group_refuses_when_no_member_has_room(apic):
    big = _sims(1, 5)[0]
    f = big.astype(np.float32)
    with apic.Group([0, 0], hbm_budget_per_device=1 << 20, n_workers=1) as g:  # 1 MiB each
        with pytest.raises(apic.ApicError) as e:
            g.open_sim(f.x, f.v, f.C, f.m, f.nrm, f.body, big.h, big.mu, big.n_iter, n_bodies=big.n_bodies)
        assert e.value.code == apic.APIC_ERR_ADMISSION
