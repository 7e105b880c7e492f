"""Sec. 3.1 gap analysis, reproduced from the oracle's own 1-D transfers.

Two equal particles at -x and +x in one linear-hat cell [-1, 1] approach at
unit speed.  With A_hat = (H - I) V / tau (eq. apic_accel) the augury
dynamics is x' = v, (v, B)' = (H - I)(v, B) / tau, with H the oracle's 1-D
APIC transfers (PIC: B = 0 throughout).  The paper states: PIC particles may
come to rest at any gap, APIC particles only once co-located (for B != 0),
and at high tau v0 / L contact is lost.  The curves of its figures are not
printed as numbers, so the thresholds below are this reproduction's."""
import numpy as np

import oracle


def _rhs(y, tau, apic):
    p, v, b = y
    x = np.array([p, -p])
    V = np.array([v, -v])
    B = np.full(2, b if apic else 0.0)  # B is even under the mirror
    vo, Bo = oracle.apic1d_linear(x, V, B, np.ones(2), 2.0, -1.0)  # nodes at -1, 1 (spacing 2)
    return np.array([v, (vo[0] - v) / tau, (Bo[0] - b) / tau if apic else 0.0])


def _run(tau, apic, T=20.0, dt=5e-3, p0=-0.9):
    y = np.array([p0, 1.0, 0.0])
    traj = [y]
    for _ in range(int(round(T / dt))):
        k1 = _rhs(y, tau, apic)
        k2 = _rhs(y + 0.5 * dt * k1, tau, apic)
        k3 = _rhs(y + 0.5 * dt * k2, tau, apic)
        k4 = _rhs(y + dt * k3, tau, apic)
        y = y + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        traj.append(y)
    return np.array(traj)


def test_pic_stops_at_a_gap_apic_only_at_contact():
    pic = _run(0.3, apic=False)
    apic = _run(0.3, apic=True)
    # PIC: at rest, still apart
    assert abs(pic[-1, 1]) < 1e-10 and abs(pic[-1, 0]) > 0.2
    # APIC: at rest only once co-located, B nonzero on the way
    assert abs(apic[-1, 0]) < 1e-4 and abs(apic[-1, 1]) < 1e-4
    assert np.abs(apic[:, 2]).max() > 0.1
    assert np.all(apic[:, 0] <= 1e-4)  # never passed through each other


def test_fixed_points():
    """PIC: v = 0 is at rest for any x.  APIC with B != 0: v = 0 is at rest
    only at x = 0 (v' = -x B / tau there, with the R13 sign)."""
    for p in (-0.8, -0.5, -0.2):
        assert abs(_rhs(np.array([p, 0.0, 0.0]), 1.0, apic=False)[1]) < 1e-15
        d = _rhs(np.array([p, 0.0, 0.7]), 1.0, apic=True)
        assert abs(d[1]) > 1e-3
    d = _rhs(np.array([0.0, 0.0, 0.7]), 1.0, apic=True)
    assert abs(d[1]) < 1e-15 and abs(d[2]) < 1e-15


def test_contact_lost_at_high_tau():
    """tau v0 / L = 3: the correction is too slow and the particles pass
    through each other and leave the cell."""
    for apic in (False, True):
        tr = _run(3.0, apic=apic, T=20.0, dt=1e-2)
        assert tr[-1, 0] > 1.0
