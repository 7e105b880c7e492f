"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it pins.  Together they are chosen so that a
plausible mistake anywhere in the oracle (a dropped affine term, a wrong
sign in the cone, a transposed C, a wrong weight, a mis-indexed node) fails
at least one of them; ``test_planted_mistakes`` checks that claim by
planting such mistakes in a copy of the oracle source.
"""
from fractions import Fraction
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2108_02259_gb300 import scenes

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append([float(Fraction(tok)) for tok in line.split()])
    return np.array(out)


def _scale_P(m, v):
    return float(np.sum(m * np.linalg.norm(v, axis=1)))


def _scale_L(x, m, v, Cm, h):
    return float(np.sum(m * (np.linalg.norm(x, axis=1) * np.linalg.norm(v, axis=1)
                             + h * h * np.linalg.norm(Cm.reshape(-1, 9), axis=1))))


# ---------------------------------------------------------------- App. B ----

def test_weights_golden():
    """App. B weights at hand-evaluated points (exact rationals)."""
    for row in _rows("bspline_weights.txt"):
        il, N = oracle.weights(row[0])
        assert il == np.floor(row[0])
        np.testing.assert_allclose(N, row[1:], rtol=0, atol=1e-15)


def test_weights_pou_completeness_D():
    """eq. pou, eq. linearCompleteness and D_p = (h^2/2) I (App. A, App. B)."""
    rng = np.random.default_rng(1)
    for xi in np.concatenate([rng.uniform(-50, 50, 200), [0.0, 1.0, -1.0, 7.0 - 1e-12]]):
        il, N = oracle.weights(xi)
        nodes = il - 1 + np.arange(4)
        assert abs(N.sum() - 1.0) < 1e-14
        assert abs((N * nodes).sum() - xi) < 1e-12 * max(1, abs(xi))
        d = nodes - xi
        assert abs((N * d * d).sum() - 0.5) < 1e-12
        assert np.all(N >= 0)
    # 3-D D_p from the oracle's own stencil sum, at positive and negative x
    h = 0.37
    x = rng.uniform(-3, 3, (50, 3))
    D = oracle.D_tensor(x, h)
    np.testing.assert_allclose(D, np.broadcast_to(0.5 * h * h * np.eye(3), D.shape), atol=1e-14)


def test_printed_one_eighth_is_garbled():
    """With the printed 1/8 on the middle functions the partition of unity
    (eq. pou), which App. A requires, fails: (6 - b)/8 at t = 0 is 0.625."""
    t = 0.0
    a, b, c = (1 - t) ** 2, (1 + t) * (1 - t) + (2 - t) * t, t * t
    assert abs(a / 4 + (a + b) / 8 + (b + c) / 8 + c / 4 - 1.0) > 0.3
    _, N = oracle.weights(t)
    assert abs(N.sum() - 1) < 1e-15


def test_weights_continuous_across_cells():
    """The basis is C^1: cell i at t -> 1 and cell i+1 at t = 0 agree."""
    il0, N0 = oracle.weights(5.0 - 1e-13)
    il1, N1 = oracle.weights(5.0)
    # node sets {3,4,5,6} and {4,5,6,7}
    w0 = dict(zip(range(il0 - 1, il0 + 3), N0))
    w1 = dict(zip(range(il1 - 1, il1 + 3), N1))
    for k in set(w0) | set(w1):
        assert abs(w0.get(k, 0.0) - w1.get(k, 0.0)) < 1e-12


# ------------------------------------------------- affine reproduction ----

@pytest.mark.parametrize("seed", [0, 1])
def test_affine_reproduction_H(seed):
    """App. A: an affine field v = v0 + L x, B = L D (C = L) is reproduced by H."""
    s = scenes.random_cloud(300, n_bodies=3, seed=seed, h=0.13, affine=True, spread=1.0, origin=(-0.4, 0.2, -1.1))
    vo, Co = oracle.apply_H(s.x, s.v, s.C, s.m, s.h)
    sc = np.abs(s.v).max()
    assert np.abs(vo - s.v).max() < 1e-13 * sc * 10
    assert np.abs(Co - s.C).max() < 1e-12 * np.abs(s.C).max() * 10


@pytest.mark.parametrize("n_iter,mu", [(0, 0.3), (4, 0.3), (3, 0.0), (2, 5.0)])
def test_affine_reproduction_full_step(n_iter, mu):
    """App. A + Sec. 2.3: with an affine input, Delta_0 = 0, so every W_n is 0
    and the whole series returns its input, for several bodies sharing it."""
    s = scenes.random_cloud(200, n_bodies=4, seed=7, h=0.2, affine=True, mu=mu, n_iter=n_iter)
    vo, Co, st = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, mu, n_iter)
    assert np.abs(vo - s.v).max() < 1e-12 * np.abs(s.v).max()
    assert np.abs(Co - s.C).max() < 1e-11 * np.abs(s.C).max()


def test_single_rigid_body_returns_input():
    """A single body in rigid motion (no contact) is returned unchanged."""
    s = scenes.four_bodies(scale=0.004)
    keep = s.body == 1
    vo, Co, st = oracle.contact_step(s.x[keep], s.v[keep], s.C[keep], s.m[keep], s.nrm[keep],
                                     np.zeros(keep.sum(), np.int32), s.h, 0.3, 8)
    assert np.abs(vo - s.v[keep]).max() < 1e-12 * np.abs(s.v[keep]).max()
    assert np.abs(Co - s.C[keep]).max() < 1e-11 * np.abs(s.C[keep]).max()
    assert st["multibody_nodes"] == 0


# ------------------------------------------------------------- momentum ----

def test_p2g_conserves_momentum():
    """Sec. 2.1.2 (Jiang et al. 2017): P2G preserves linear momentum and the
    APIC angular momentum sum m [x x v + eps:B], for any state."""
    s = scenes.random_cloud(250, n_bodies=2, seed=3, h=0.11, origin=(-0.3, -0.2, 0.4))
    ijk, mi, pi = oracle.p2g_grid(s.x, s.v, s.C, s.m, s.h)
    xi = ijk * s.h
    P, L = oracle.momentum(s.x, s.v, s.C, s.m, s.h)
    sP, sL = _scale_P(s.m, s.v), _scale_L(s.x, s.m, s.v, s.C, s.h)
    assert np.abs(pi.sum(0) - P).max() < 1e-13 * sP
    assert np.abs(np.cross(xi, pi).sum(0) - L).max() < 1e-13 * sL
    assert abs(mi.sum() - s.m.sum()) < 1e-13 * s.m.sum()


def test_g2p_conserves_momentum():
    """G2P from any grid velocity field preserves sum m_i v_i and
    sum x_i x m_i v_i (Jiang et al. 2017, cited in Sec. 2.1.2)."""
    s = scenes.random_cloud(250, n_bodies=2, seed=4, h=0.11)
    ijk, mi, _ = oracle.p2g_grid(s.x, s.v, s.C, s.m, s.h)
    rng = np.random.default_rng(5)
    vg = rng.standard_normal((ijk.shape[0], 3))
    vo, Co = oracle.g2p_from_grid(s.x, s.h, ijk, vg)
    P, L = oracle.momentum(s.x, vo, Co, s.m, s.h)
    Pg = (mi[:, None] * vg).sum(0)
    Lg = np.cross(ijk * s.h, mi[:, None] * vg).sum(0)
    assert np.abs(P - Pg).max() < 1e-12 * np.abs(mi[:, None] * vg).sum()
    assert np.abs(L - Lg).max() < 1e-12 * np.abs(np.cross(ijk * s.h, mi[:, None] * vg)).sum()


@pytest.mark.parametrize("n_iter,mu,flags", [(0, 0.3, 0), (3, 0.3, 0), (5, 0.0, 0), (2, 1.0, oracle.FLAG_SEP23)])
def test_series_conserves_momentum(n_iter, mu, flags):
    """Sec. 2.3: every G W_n has zero net linear and angular momentum, so the
    series keeps the momentum of V for any W_n (relative drift <= 1e-12)."""
    s = scenes.random_cloud(300, n_bodies=3, seed=11, h=0.15, origin=(0.5, -2.0, 0.1))
    vo, Co, st = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, mu, n_iter, flags=flags)
    sP, sL = _scale_P(s.m, s.v), _scale_L(s.x, s.m, s.v, s.C, s.h)
    assert np.abs(st["P_out"] - st["P_in"]).max() <= 1e-12 * sP
    assert np.abs(st["L_out"] - st["L_in"]).max() <= 1e-12 * sL
    # and the change is not trivially zero
    assert np.abs(vo - s.v).max() > 1e-3


def test_pic_keeps_linear_not_angular():
    """Sec. 2.1.1: PIC transfers keep linear momentum; angular momentum is not
    guaranteed (it changes for a generic state)."""
    s = scenes.random_cloud(200, n_bodies=2, seed=12, h=0.15)
    Cz = np.zeros_like(s.C)
    vo, Co = oracle.apply_H(s.x, s.v, Cz, s.m, s.h, flags=oracle.FLAG_PIC)
    P0, L0 = oracle.momentum(s.x, s.v, Cz, s.m, s.h)
    P1, L1 = oracle.momentum(s.x, vo, Co, s.m, s.h)
    assert np.abs(P1 - P0).max() < 1e-12 * _scale_P(s.m, s.v)
    assert np.abs(L1 - L0).max() > 1e-6 * _scale_L(s.x, s.m, s.v, Cz, s.h)


# ---------------------------------------------- operator structure ----

def _inner(s, D, v1, C1, v2, C2):
    # <V, V'> = sum m (v . v' + tr(C D C'^T))
    t = np.einsum("pab,pbc,pac->p", C1, D, C2)
    return float(np.sum(s.m * (np.einsum("pa,pa->p", v1, v2) + t)))


def test_H_self_adjoint_psd_contraction():
    """Derived from eq. particleToGrid / gridToParticle: <HV, V'> = sum_i
    p_i . p'_i / m_i, so H is self-adjoint and 0 <= <HV, V> <= <V, V> in the
    mass inner product (APIC never adds generalized kinetic energy)."""
    s = scenes.random_cloud(120, n_bodies=2, seed=21, h=0.2)
    D = oracle.D_tensor(s.x, s.h)
    rng = np.random.default_rng(22)
    v2, C2 = rng.standard_normal(s.v.shape), rng.standard_normal(s.C.shape) / s.h
    Hv1, HC1 = oracle.apply_H(s.x, s.v, s.C, s.m, s.h)
    Hv2, HC2 = oracle.apply_H(s.x, v2, C2, s.m, s.h)
    a = _inner(s, D, Hv1, HC1, v2, C2)
    b = _inner(s, D, s.v, s.C, Hv2, HC2)
    assert abs(a - b) < 1e-12 * (abs(a) + abs(b))
    e0 = _inner(s, D, s.v, s.C, s.v, s.C)
    e1 = _inner(s, D, Hv1, HC1, s.v, s.C)
    assert 0.0 <= e1 <= e0
    # H is a projection-like contraction: H(HV) energy <= HV energy
    e2 = _inner(s, D, Hv1, HC1, Hv1, HC1)
    assert e2 <= e0 * (1 + 1e-14)


def test_quasi_null_space():
    """Sec. 2.3: two co-located equal-mass particles with opposite velocities
    (C = 0) cancel on the grid, H V has zero velocity, so G W = -W on v."""
    x = np.array([[0.31, 0.47, 0.52], [0.31, 0.47, 0.52]])
    v = np.array([[1.0, -2.0, 0.5], [-1.0, 2.0, -0.5]])
    Cm = np.zeros((2, 3, 3))
    m = np.array([2.0, 2.0])
    vo, Co = oracle.apply_H(x, v, Cm, m, 0.1)
    assert np.abs(vo).max() < 1e-15
    assert np.abs(Co).max() < 1e-13
    G_v = vo - v
    np.testing.assert_allclose(G_v, -v, atol=1e-15)


def _dense_H_numpy(x, m, h):
    """Brute force from the definitions, written independently of the
    oracle's hash-map grid: enumerate all nodes, build the dense weight matrix
    Nm[p, i] and offsets, and apply eq. particleToGrid / gridToParticle as
    dense matrix algebra to each unit vector of R^{12P}."""
    P = x.shape[0]

    def w1(xi):
        i = np.floor(xi)
        t = xi - i
        return i, np.array([(1 - t) ** 2 / 4, (2 - t * t) / 4, (1 + 2 * t - t * t) / 4, t * t / 4])

    nodes = {}
    W = []
    for p in range(P):
        ws = [w1(x[p, d] / h) for d in range(3)]
        row = {}
        for kz in range(4):
            for ky in range(4):
                for kx in range(4):
                    key = (int(ws[0][0]) - 1 + kx, int(ws[1][0]) - 1 + ky, int(ws[2][0]) - 1 + kz)
                    nodes.setdefault(key, len(nodes))
                    row[nodes[key]] = ws[0][1][kx] * ws[1][1][ky] * ws[2][1][kz]
        W.append(row)
    G = len(nodes)
    Nm = np.zeros((P, G))
    for p in range(P):
        for i, w in W[p].items():
            Nm[p, i] = w
    X = np.zeros((G, 3))
    for k, i in nodes.items():
        X[i] = np.array(k) * h
    R = X[None, :, :] - x[:, None, :]  # x_i - x_p
    mi = Nm.T @ m
    D = np.einsum("pi,pia,pib->pab", Nm, R, R)
    Dinv = np.linalg.inv(D)
    H = np.zeros((12 * P, 12 * P))
    for col in range(12 * P):
        e = np.zeros(12 * P)
        e[col] = 1.0
        v = e[: 3 * P].reshape(P, 3)
        Cm = e[3 * P:].reshape(P, 3, 3)
        mom = np.einsum("pi,p,pia->ia", Nm, m, v[:, None, :] + np.einsum("pab,pib->pia", Cm, R))
        vg = np.where(mi[:, None] > 0, mom / np.where(mi[:, None] > 0, mi[:, None], 1), 0)
        vo = Nm @ vg
        B = np.einsum("pi,ia,pib->pab", Nm, vg, R)
        Co = np.einsum("pab,pbc->pac", B, Dinv)
        H[:, col] = np.concatenate([vo.ravel(), Co.ravel()])
    return H, D


def test_dense_brute_force():
    """Brute force on tiny inputs (P <= 5): the oracle's H equals an
    independent dense-matrix construction, column by column; the dense H is
    self-adjoint in the mass inner product with spectrum in [0, 1]."""
    rng = np.random.default_rng(31)
    P, h = 5, 0.25
    x = rng.uniform(-0.3, 0.3, (P, 3))
    m = rng.uniform(0.5, 2.0, P)
    Hd, D = _dense_H_numpy(x, m, h)
    Ho = np.zeros_like(Hd)
    for col in range(12 * P):
        e = np.zeros(12 * P)
        e[col] = 1.0
        vo, Co = oracle.apply_H(x, e[: 3 * P].reshape(P, 3), e[3 * P:].reshape(P, 3, 3), m, h)
        Ho[:, col] = np.concatenate([vo.ravel(), Co.ravel()])
    assert np.abs(Ho - Hd).max() < 1e-12 * max(1.0, np.abs(Hd).max())
    # mass matrix of the inner product <V,V'> = sum m (v.v' + tr(C D C'^T))
    M = np.zeros((12 * P, 12 * P))
    for p in range(P):
        M[3 * p:3 * p + 3, 3 * p:3 * p + 3] = m[p] * np.eye(3)
        for a in range(3):
            base = 3 * P + 9 * p + 3 * a
            M[base:base + 3, base:base + 3] = m[p] * D[p]
    S = M @ Hd
    assert np.abs(S - S.T).max() < 1e-12 * np.abs(S).max()
    Ms = np.linalg.cholesky(M)
    A = np.linalg.solve(Ms, np.linalg.solve(Ms, S).T).T
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.min() > -1e-10 and ev.max() < 1 + 1e-10
    # linearity of the oracle's H
    v1, C1 = rng.standard_normal((P, 3)), rng.standard_normal((P, 3, 3))
    v2, C2 = rng.standard_normal((P, 3)), rng.standard_normal((P, 3, 3))
    a1 = oracle.apply_H(x, v1, C1, m, h)
    a2 = oracle.apply_H(x, v2, C2, m, h)
    a3 = oracle.apply_H(x, 2 * v1 - 3 * v2, 2 * C1 - 3 * C2, m, h)
    assert np.abs(a3[0] - (2 * a1[0] - 3 * a2[0])).max() < 1e-12 * 10
    assert np.abs(a3[1] - (2 * a1[1] - 3 * a2[1])).max() < 1e-11 * 10


# ------------------------------------------------ friction projection ----

def test_undesirable_closed_forms():
    """Sec. 2.4 projection cases, worked by hand."""
    n = np.array([0.0, 0.0, 1.0])
    dC = np.arange(9.0)
    # separating change (dv.n > 0): all undesirable
    w, wc = oracle.undesirable([0.3, -0.2, 0.5], dC, n, 0.4)
    np.testing.assert_allclose(w, [0.3, -0.2, 0.5])
    np.testing.assert_allclose(wc.ravel(), dC)
    # compressive, inside the cone (|t| = 0.5 <= mu*|dn| = 0.4*2 = 0.8): nothing
    w, _ = oracle.undesirable([0.3, 0.4, -2.0], dC, n, 0.4)
    np.testing.assert_allclose(w, 0.0, atol=1e-16)
    # compressive, outside the cone: tangential excess beyond mu*|dn|
    w, _ = oracle.undesirable([3.0, 4.0, -1.0], dC, n, 0.5)
    np.testing.assert_allclose(w, np.array([3.0, 4.0, 0.0]) * (1 - 0.5 / 5.0), atol=1e-15)
    # frictionless: the whole tangential part
    w, _ = oracle.undesirable([3.0, 4.0, -1.0], dC, n, 0.0)
    np.testing.assert_allclose(w, [3.0, 4.0, 0.0], atol=1e-15)
    # tie dv.n = 0 goes to the compressive branch; zero tangential part -> 0
    w, _ = oracle.undesirable([0.0, 0.0, 0.0], dC, n, 0.3)
    np.testing.assert_allclose(w, 0.0)
    # interior node (n = 0): dv.n = 0, tangential = dv, s = 0 -> W = dv
    w, _ = oracle.undesirable([1.0, -2.0, 3.0], dC, np.zeros(3), 0.3)
    np.testing.assert_allclose(w, [1.0, -2.0, 3.0])
    # Sec. 2.3 rule: zero unless separating, then everything incl. dC
    w, wc = oracle.undesirable([3.0, 4.0, -1.0], dC, n, 0.3, flags=oracle.FLAG_SEP23)
    np.testing.assert_allclose(w, 0.0)
    np.testing.assert_allclose(wc, 0.0)
    w, wc = oracle.undesirable([3.0, 4.0, 1.0], dC, n, 0.3, flags=oracle.FLAG_SEP23)
    np.testing.assert_allclose(w, [3.0, 4.0, 1.0])
    np.testing.assert_allclose(wc.ravel(), dC)
    # tilted normal: result must be orthogonal to n (tangential) and on the cone edge
    nn = np.array([1.0, 2.0, 2.0]) / 3.0
    dv = np.array([0.7, -1.9, 0.4])
    dn = dv @ nn
    assert dn < 0
    w, _ = oracle.undesirable(dv, dC, nn, 0.2)
    t = dv - dn * nn
    assert abs(w @ nn) < 1e-15
    kept = t - w
    np.testing.assert_allclose(np.linalg.norm(kept), 0.2 * (-dn), rtol=1e-14)


# ------------------------------------------------------- Sec. 3.1 ----

def test_gap1d_matrix_matches_printed_closed_form():
    """Sec. 3.1: G = H - I of two mirrored particles in one linear-hat cell
    [-1, 1] equals the printed matrix [[x^2-1, -x], [x^3-x, -x^2]]."""
    for row in _rows("gap1d_G.txt"):
        xg = row[0]
        Gm = row[1:].reshape(2, 2)
        xs = np.array([-xg, xg])  # listed particle at -x
        for v0, B0 in ((1.0, 0.0), (0.0, 1.0), (0.37, -1.3)):
            vo, Bo = oracle.apic1d_linear(xs, np.array([v0, -v0]), np.array([B0, B0]), np.ones(2), h=2.0, x0=-1.0)
            got = np.array([vo[0] - v0, Bo[0] - B0])
            np.testing.assert_allclose(got, Gm @ np.array([v0, B0]), atol=1e-14)
        # PIC: B = 0 and no affine term -> (x^2 - 1) v
        vo, _ = oracle.apic1d_linear(xs, np.array([1.0, -1.0]), np.zeros(2), np.ones(2), h=2.0, x0=-1.0)
        # with B = 0 APIC still adds B-coupling only through B, so v-part matches G11
        assert abs((vo[0] - 1.0) - Gm[0, 0]) < 1e-14


# ----------------------------------------------- symmetry / invariance ----

def test_two_cubes_mirror_and_momentum():
    """Two equal cubes approaching head-on, mirror-symmetric about the node
    plane x = 0.5 = 16 h: the step is mirror-equivariant and nets zero
    linear momentum (to 1e-12 of the scale)."""
    s = scenes.two_cubes(mu=0.0, n_iter=4)
    vo, Co, st = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, 0.0, 4)
    Mx = np.diag([-1.0, 1.0, 1.0])
    xm = s.x @ Mx + np.array([1.0, 0, 0])
    # partner index of every particle under the mirror
    key = {tuple(np.round(p, 9)): i for i, p in enumerate(s.x)}
    part = np.array([key[tuple(np.round(p, 9))] for p in xm])
    np.testing.assert_allclose(vo[part], vo @ Mx, atol=1e-12)
    np.testing.assert_allclose(Co[part], np.einsum("ab,pbc,cd->pad", Mx, Co, Mx), atol=1e-10)
    sP = _scale_P(s.m, s.v)
    assert np.abs(st["P_out"]).max() < 1e-12 * sP
    assert st["multibody_nodes"] > 0
    # the facing layers are slowed: relative normal velocity reduced
    face_l = (s.body == 0) & (s.nrm[:, 0] > 0.5)
    assert vo[face_l, 0].mean() < 1.0 - 1e-3


def test_separating_adhesion_decays_with_iterations():
    """Sec. 2.3: for bodies moving apart, each augury iteration removes more of
    the undesirable (adhesive) change, so the largest change shrinks with N."""
    s = scenes.two_cubes(mu=0.3, approach=False)
    prev = None
    for N in (0, 1, 3, 10):
        vo, Co, _ = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, 0.3, N)
        adh = np.abs(vo - s.v).max()
        if prev is not None:
            assert adh < prev
        prev = adh
    assert prev < 0.05


def test_shift_and_permutation_invariance():
    """The grid is x_i = h * i (App. B): shifting every x by an integer
    multiple of h leaves the step unchanged; permuting axes permutes it."""
    s = scenes.random_cloud(150, n_bodies=3, seed=41, h=0.125, n_iter=2)
    base = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, 0.3, 2)
    sh = oracle.contact_step(s.x + s.h * np.array([3, -7, 11]), s.v, s.C, s.m, s.nrm, s.body, s.h, 0.3, 2)
    np.testing.assert_allclose(sh[0], base[0], atol=1e-12)
    np.testing.assert_allclose(sh[1], base[1], atol=1e-10)
    perm = [2, 0, 1]
    Pm = np.eye(3)[perm]
    pr = oracle.contact_step(s.x @ Pm.T, s.v @ Pm.T, np.einsum("ab,pbc,dc->pad", Pm, s.C, Pm), s.m, s.nrm @ Pm.T,
                             s.body, s.h, 0.3, 2)
    np.testing.assert_allclose(pr[0], base[0] @ Pm.T, atol=1e-12)
    np.testing.assert_allclose(pr[1], np.einsum("ab,pbc,dc->pad", Pm, base[1], Pm), atol=1e-10)


def test_mu_pair_uniform_equals_scalar():
    """A uniform pair table reduces the per-particle blend to the scalar mu."""
    s = scenes.random_cloud(150, n_bodies=3, seed=51, h=0.15, n_iter=3)
    a = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, 0.25, 3)
    b = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, 0.0, 3, mu_pair=np.full((3, 3), 0.25))
    np.testing.assert_allclose(a[0], b[0], atol=1e-13)


def test_mu_pair_two_rigid_bodies_use_the_cross_coefficient():
    """Two rigid bodies, one series term (N = 1): only particles whose stencil
    reaches the other body are projected (elsewhere Delta = 0, App. A), and
    for them the blend of the pair table is mu(0, 1) whatever the diagonal.
    So a table with very different diagonal entries gives exactly the scalar
    step with mu = mu(0, 1) -- and a blend that counted the particle's own
    body, or the other body's self-friction, would not."""
    s = scenes.two_cubes(mu=0.2, n_iter=1)
    a = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, 0.2, 1)
    b = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, 0.0, 1,
                            mu_pair=np.array([[0.9, 0.2], [0.2, 0.05]]))
    np.testing.assert_allclose(b[0], a[0], atol=1e-13)
    np.testing.assert_allclose(b[1], a[1], atol=1e-10)
    # and the cross coefficient does matter here
    c = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, 0.0, 1,
                            mu_pair=np.array([[0.9, 0.6], [0.6, 0.05]]))
    assert np.abs(c[0] - a[0]).max() > 1e-3


# ------------------------------------------------- planted mistakes ----

MISTAKES = [
    # (original snippet, planted replacement, which pin catches it)
    ("N[1] = 0.25 * (a + b);", "N[1] = 0.125 * (a + b);", "pou"),
    ("aff += C[9 * p + 3 * a + b] * s.r[q][b];", "aff += C[9 * p + 3 * b + a] * s.r[q][b];", "momentum"),
    ("const double s = std::min(nt, -mu * dn);", "const double s = std::min(nt, mu * dn);", "cone"),
    ("for (size_t k = 0; k < nv; ++k) dv[k] += Hv[k] - Wv[k];", "for (size_t k = 0; k < nv; ++k) dv[k] += Hv[k] + Wv[k];", "series"),
    ("s.r[q][1] = h * (double)key.j - x[3 * p + 1];", "s.r[q][1] = x[3 * p + 1] - h * (double)key.j;", "affine"),
]


def test_planted_mistakes(tmp_path):
    """Each planted mistake in a copy of the oracle fails at least one pin."""
    import ctypes

    src = open(os.path.join(os.path.dirname(oracle.__file__), "apic_oracle.cpp")).read()
    s = scenes.random_cloud(60, n_bodies=2, seed=61, h=0.2, n_iter=2)
    sa = scenes.random_cloud(60, n_bodies=2, seed=62, h=0.2, affine=True)
    for k, (old, new, _) in enumerate(MISTAKES):
        assert old in src, old
        path = tmp_path / f"bad{k}.cpp"
        path.write_text(src.replace(old, new))
        so = tmp_path / f"bad{k}.so"
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", str(path), "-o", str(so)])
        lib = ctypes.CDLL(str(so))
        P = ctypes.c_void_p
        lib.oracle_contact_step.argtypes = [ctypes.c_int64, ctypes.c_int32, P, P, P, P, P, P, ctypes.c_double,
                                            ctypes.c_double, P, ctypes.c_int32, ctypes.c_uint32, P, P, P]
        lib.oracle_weights.argtypes = [ctypes.c_double, P, P]
        failures = 0
        # pou
        il, N = np.zeros(1, np.int64), np.zeros(4)
        lib.oracle_weights(0.3, il.ctypes.data, N.ctypes.data)
        failures += abs(N.sum() - 1) > 1e-12
        # cone
        lib.oracle_undesirable.argtypes = [P, P, P, ctypes.c_double, ctypes.c_uint32, P, P]
        dv, dC, nn = np.array([3.0, 4.0, -1.0]), np.zeros(9), np.array([0, 0, 1.0])
        w, wc = np.zeros(3), np.zeros(9)
        lib.oracle_undesirable(dv.ctypes.data, dC.ctypes.data, nn.ctypes.data, 0.5, 0, w.ctypes.data, wc.ctypes.data)
        failures += np.abs(w - np.array([3.0, 4.0, 0.0]) * 0.9).max() > 1e-12
        # momentum + affine through the full step
        for sc, check in ((s, "mom"), (sa, "aff")):
            vo, Co, st = np.zeros((sc.n, 3)), np.zeros((sc.n, 3, 3)), np.zeros(13)
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (sc.x, sc.v, sc.C, sc.m, sc.nrm)]
            body = np.ascontiguousarray(sc.body, np.int32)
            lib.oracle_contact_step(sc.n, 2, body.ctypes.data, *[a.ctypes.data for a in arrs], sc.h, 0.3, None, 2, 0,
                                    vo.ctypes.data, Co.ctypes.data, st.ctypes.data)
            if check == "mom":
                sP = _scale_P(sc.m, sc.v)
                sL = _scale_L(sc.x, sc.m, sc.v, sc.C, sc.h)
                failures += np.abs(st[3:6] - st[0:3]).max() > 1e-12 * sP or np.abs(st[9:12] - st[6:9]).max() > 1e-12 * sL
            else:
                failures += np.abs(vo - sc.v).max() > 1e-10
        assert failures > 0, f"planted mistake not caught: {new}"


def test_separation_rule_is_a_step_and_the_cone_rule_is_continuous():
    """Sec. 2.3's separation rule switches W between 0 and Delta at dn = 0, and
    the series drives the particles of an active contact there; Sec. 2.4's cone
    projection is continuous.  So under seeded relative changes of v and C the
    oracle's output moves in proportion to the change with the cone rule (ten
    times the change, ten times the effect), but jumps with the separation rule
    at a change of only 1e-8.  The GPU tests compare the separation rule beyond
    the oracle's own envelope for this reason (tests/discontinuity.py)."""
    import discontinuity

    s = scenes.four_bodies(scale=0.02)
    vs = np.abs(s.v).max()
    moved = {}
    for flags in (0, oracle.FLAG_SEP23):
        def run(v, C, flags=flags):
            return oracle.contact_step(s.x, v, C, s.m, s.nrm, s.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies,
                                       flags=flags)[:2]
        for eps in (1e-8, 1e-7):
            for seed in range(3):
                ev = discontinuity.envelope(run, s.v, s.C, eps=eps, trials=1, seed=seed)[2]
                moved[flags, eps, seed] = ev.max() / vs
    for seed in range(3):  # cone rule: linear in the change, to 10%
        ratio = moved[0, 1e-7, seed] / moved[0, 1e-8, seed]
        assert 9.0 < ratio < 11.0, (seed, ratio)
        assert moved[0, 1e-8, seed] < 1e-7
    cone = max(moved[0, 1e-8, k] for k in range(3))
    step = max(moved[oracle.FLAG_SEP23, 1e-8, k] for k in range(3))
    assert step > 10 * cone, (step, cone)
