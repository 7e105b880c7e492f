"""Pins of the oracle's normals from a body's grid mass.

Callers with neither normals nor a surface mesh get n_p = -g_p / |g_p|,
with g_p the gradient (in cell units) of body b's grid mass interpolated
at x_p, where |g_p| exceeds a threshold times the interpolated mass rho_p,
and 0 inside the body.  The paper's normals come from the FE surface
(Sec. 2.3), so the construction is a reading; what it is built from is
fixed by App. B: the weights, their derivatives and eq. massToGrid over one
body.  These pins would each catch a plausible mistake: a flipped sign, a
wrong derivative, swapped gradient components, the total grid mass in place
of the body's own, interior particles given a normal.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle

H = 0.1


def _lattice_box(n, s, shift):
    I, J, K = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ijk = np.stack([I.ravel(), J.ravel(), K.ravel()], 1)
    return ijk, ijk * s + np.asarray(shift, np.float64)


def test_weight_derivatives():
    """dN/dxi of the App. B functions: zero sum (they sum to one), sum of
    dN_k (k - 1) = 1 (they reproduce xi), central differences of the
    weights, and the values at t = 0 and t = 1/2 worked out by hand from
    (1-t)^2/4, (2-t^2)/4, (1+2t-t^2)/4, t^2/4."""
    rng = np.random.default_rng(3)
    for xi in np.concatenate([rng.uniform(-7, 7, 50), [0.0, 2.5, -3.0]]):
        dN = oracle.weight_grads(xi)
        assert abs(dN.sum()) < 1e-15
        assert abs(np.dot(dN, np.arange(4) - 1.0) - 1.0) < 1e-14
    for xi in rng.uniform(-7, 7, 50):
        t = xi - np.floor(xi)
        if t < 1e-3 or t > 1 - 1e-3:
            continue
        eps = 1e-6
        Np = oracle.weights(xi + eps)[1]
        Nm = oracle.weights(xi - eps)[1]
        assert np.abs((Np - Nm) / (2 * eps) - oracle.weight_grads(xi)).max() < 1e-8
    assert np.abs(oracle.weight_grads(4.0) - [-0.5, 0.0, 0.5, 0.0]).max() < 1e-15
    assert np.abs(oracle.weight_grads(4.5) - [-0.25, -0.25, 0.25, 0.25]).max() < 1e-15


@pytest.mark.parametrize("shift", [(0.013, -0.021, 0.007), (0.0, 0.0, 0.0), (-1.234, 5.5, 0.05)])
def test_face_normals_of_a_lattice_box_are_exact(shift):
    """A box lattice at spacing h/2: away from edges the lattice repeats
    every h along the face, so every node of a layer gets the same mass and
    the in-face gradient components vanish; the outward face normal comes
    out exactly on each of the six faces."""
    n = 24
    ijk, x = _lattice_box(n, H / 2, shift)
    nrm, ratio = oracle.mass_normals(x, np.ones(len(x)), np.zeros(len(x), np.int32), H)
    lo, hi = 9, n - 10  # 4h clear of every edge (the stencil reaches 2h, node masses 2h more)
    for ax in range(3):
        others = [a for a in range(3) if a != ax]
        inner = np.all((ijk[:, others] >= lo) & (ijk[:, others] <= hi), axis=1)
        for side, layer in ((-1.0, 0), (1.0, n - 1)):
            sel = inner & (ijk[:, ax] == layer)
            assert sel.sum() > 0
            want = np.zeros(3)
            want[ax] = side
            assert np.abs(nrm[sel] - want).max() < 1e-12, (ax, side)


def test_deep_interior_has_no_normal():
    """Where every node of a particle's stencil has the full interior mass
    (8 layers in at spacing h/2), the gradient vanishes: ratio ~ 0, n = 0."""
    n = 24
    ijk, x = _lattice_box(n, H / 2, (0.013, 0.02, -0.03))
    nrm, ratio = oracle.mass_normals(x, np.ones(len(x)), np.zeros(len(x), np.int32), H)
    depth = np.minimum(ijk, n - 1 - ijk).min(axis=1)
    deep = depth >= 8
    assert deep.sum() > 0
    assert ratio[deep].max() < 1e-12
    assert np.all(nrm[deep] == 0.0)
    # and the outermost layer is on the surface
    assert np.all(np.linalg.norm(nrm[depth == 0], axis=1) > 0.999)


def test_threshold_splits_zero_and_unit():
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 1, (3000, 3))
    body = rng.integers(0, 3, 3000).astype(np.int32)
    m = rng.uniform(0.5, 2, 3000)
    for thr in (0.0, 0.3, 0.7):
        nrm, ratio = oracle.mass_normals(x, m, body, H, threshold=thr)
        ln = np.linalg.norm(nrm, axis=1)
        on = ratio > thr
        assert np.all(ln[~on] == 0.0)
        assert np.abs(ln[on] - 1.0).max() < 1e-14


def test_integer_shift_and_axis_permutation():
    rng = np.random.default_rng(6)
    x = rng.uniform(-0.5, 0.5, (2000, 3)) * [1.0, 0.7, 0.4]
    body = (x[:, 0] > 0.05).astype(np.int32)
    m = rng.uniform(0.5, 1.5, 2000)
    n0, r0 = oracle.mass_normals(x, m, body, H, threshold=0.0)
    n1, r1 = oracle.mass_normals(x + np.array([3, -5, 7]) * H, m, body, H, threshold=0.0)
    assert np.abs(n1 - n0).max() < 1e-12 and np.abs(r1 - r0).max() < 1e-12
    perm = [2, 0, 1]
    n2, r2 = oracle.mass_normals(x[:, perm], m, body, H, threshold=0.0)
    assert np.abs(n2 - n0[:, perm]).max() < 1e-12 and np.abs(r2 - r0).max() < 1e-12


def test_bodies_see_only_their_own_mass():
    """Two interpenetrating bodies: each body's normals are those it has
    alone (the construction uses the body's own grid mass)."""
    rng = np.random.default_rng(7)
    a = rng.uniform(0, 0.6, (1500, 3))
    b = rng.uniform(0.3, 0.9, (1500, 3))
    x = np.concatenate([a, b])
    m = rng.uniform(0.5, 1.5, 3000)
    body = np.repeat(np.array([0, 1], np.int32), 1500)
    both, _ = oracle.mass_normals(x, m, body, H)
    alone_a, _ = oracle.mass_normals(a, m[:1500], np.zeros(1500, np.int32), H)
    alone_b, _ = oracle.mass_normals(b, m[1500:], np.zeros(1500, np.int32), H)
    assert np.abs(both[:1500] - alone_a).max() < 1e-12
    assert np.abs(both[1500:] - alone_b).max() < 1e-12


MISTAKES = [
    ("dN[0] = 0.25 * da;", "dN[0] = -0.25 * da;"),
    ("gr[0] += dN[0][kx] * N[1][ky] * N[2][kz] * mi;", "gr[0] += N[0][kx] * dN[1][ky] * N[2][kz] * mi;"),
    ("const double* mbb = &mb[(size_t)body[p] * G];", "const double* mbb = &mb[0];"),
    ("? -gr[a] / len : 0.0;", "? gr[a] / len : 0.0;"),
    ("const double db = 2.0 - 4.0 * t;", "const double db = 2.0 - 2.0 * t;"),
]


def test_planted_mistakes(tmp_path):
    """Each planted mistake in a copy of the oracle fails at least one of
    the pins above."""
    src = open(os.path.join(os.path.dirname(oracle.__file__), "apic_oracle.cpp")).read()
    n = 24
    ijk, xb = _lattice_box(n, H / 2, (0.013, -0.021, 0.007))
    rng = np.random.default_rng(8)
    xa, xc = rng.uniform(0, 0.6, (800, 3)), rng.uniform(0.3, 0.9, (800, 3))
    for k, (old, new) in enumerate(MISTAKES):
        assert old in src, old
        path = tmp_path / f"bad{k}.cpp"
        path.write_text(src.replace(old, new))
        so = tmp_path / f"bad{k}.so"
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", str(path), "-o", str(so)])
        lib = ctypes.CDLL(str(so))
        P = ctypes.c_void_p
        lib.oracle_weight_grads.argtypes = [ctypes.c_double, P]
        lib.oracle_mass_normals.argtypes = [ctypes.c_int64, ctypes.c_int32, P, P, P, ctypes.c_double,
                                            ctypes.c_double, P, P]

        def mn(x, body, nb):
            x = np.ascontiguousarray(x, np.float64)
            body = np.ascontiguousarray(body, np.int32)
            m = np.ones(len(x))
            out, r = np.zeros_like(x), np.zeros(len(x))
            lib.oracle_mass_normals(len(x), nb, body.ctypes.data, x.ctypes.data, m.ctypes.data, H, 0.5,
                                    out.ctypes.data, r.ctypes.data)
            return out

        failures = 0
        dN = np.zeros(4)
        lib.oracle_weight_grads(4.3, dN.ctypes.data)
        failures += abs(dN.sum()) > 1e-12 or abs(np.dot(dN, np.arange(4) - 1.0) - 1.0) > 1e-12
        nb_ = mn(xb, np.zeros(len(xb)), 1)
        for ax in range(3):  # the + face of each axis
            others = [a for a in range(3) if a != ax]
            sel = np.all((ijk[:, others] >= 9) & (ijk[:, others] <= n - 10), axis=1) & (ijk[:, ax] == n - 1)
            failures += np.abs(nb_[sel] - np.eye(3)[ax]).max() > 1e-12
        both = mn(np.concatenate([xa, xc]), np.repeat([0, 1], 800), 2)
        failures += np.abs(both[:800] - mn(xa, np.zeros(800), 1)).max() > 1e-12
        failures += np.abs(both[800:] - mn(xc, np.zeros(800), 1)).max() > 1e-12
        assert failures > 0, f"planted mistake not caught: {new}"
