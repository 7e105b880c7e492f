"""ctypes binding of the FP64 oracle (``apic_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use it; the CUDA library never imports it.  Argument
marshalling only: every number is computed by the C++ oracle.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "apic_oracle.cpp")
_LIB = os.path.join(_HERE, "libapic_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (plain -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fno-fast-math", _SRC, "-o", tmp]
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            d, i64, i32, u32 = C.c_double, C.c_int64, C.c_int32, C.c_uint32
            P = C.c_void_p
            lib.oracle_flag_pic.restype = u32
            lib.oracle_flag_sep23.restype = u32
            lib.oracle_weights.argtypes = [d, P, P]
            lib.oracle_weights.restype = None
            lib.oracle_undesirable.argtypes = [P, P, P, d, u32, P, P]
            lib.oracle_undesirable.restype = None
            lib.oracle_D.argtypes = [i64, P, d, P]
            lib.oracle_D.restype = C.c_int
            lib.oracle_p2g_grid.argtypes = [i64, P, P, P, P, d, u32, P, P, P]
            lib.oracle_p2g_grid.restype = i64
            lib.oracle_g2p_from_grid.argtypes = [i64, P, d, u32, i64, P, P, P, P, P]
            lib.oracle_g2p_from_grid.restype = C.c_int
            lib.oracle_apply_H.argtypes = [i64, P, P, P, P, d, u32, P, P]
            lib.oracle_apply_H.restype = C.c_int
            lib.oracle_momentum.argtypes = [i64, P, P, P, P, d, P, P]
            lib.oracle_momentum.restype = C.c_int
            lib.oracle_contact_step.argtypes = [i64, i32, P, P, P, P, P, P, d, d, P, i32, u32, P, P, P]
            lib.oracle_contact_step.restype = C.c_int
            lib.oracle_apic1d_linear.argtypes = [i64, P, P, P, P, d, d, P, P]
            lib.oracle_apic1d_linear.restype = C.c_int
            lib.oracle_weight_grads.argtypes = [d, P]
            lib.oracle_weight_grads.restype = None
            lib.oracle_mass_normals.argtypes = [i64, i32, P, P, P, d, d, P, P]
            lib.oracle_mass_normals.restype = C.c_int
            lib.oracle_node_normals.argtypes = [i64, P, i64, P, P]
            lib.oracle_node_normals.restype = C.c_int
            lib.oracle_augury_steps.argtypes = [i64, i32, P, P, P, P, P, P, P, P, i64, P, P, P, P, i64, P, d, d, P,
                                                i32, u32, d, d, i32, i32, P]
            lib.oracle_augury_steps.restype = C.c_int
            _lib = lib
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data


FLAG_PIC = 1 << 0  # the tests check these against the values the library exports
FLAG_SEP23 = 1 << 1


def weights(xi: float):
    """App. B weights: (i_left, N[4]) for the nodes i-1..i+2 covering xi = x/h."""
    lib = _load()
    il = np.zeros(1, np.int64)
    N = np.zeros(4, np.float64)
    lib.oracle_weights(float(xi), _ptr(il), _ptr(N))
    return int(il[0]), N


def undesirable(dv, dC, nrm, mu, flags=0):
    lib = _load()
    dv, dC, nrm = _f64(dv, 3), _f64(dC, 9), _f64(nrm, 3)
    dvu, dCu = np.zeros(3), np.zeros(9)
    lib.oracle_undesirable(_ptr(dv), _ptr(dC), _ptr(nrm), float(mu), int(flags), _ptr(dvu), _ptr(dCu))
    return dvu, dCu.reshape(3, 3)


def D_tensor(x, h):
    lib = _load()
    x = _f64(x, (-1, 3))
    D = np.zeros((x.shape[0], 3, 3))
    if lib.oracle_D(x.shape[0], _ptr(x), float(h), _ptr(D)) != 0:
        raise ValueError("oracle_D: invalid arguments")
    return D


def p2g_grid(x, v, Cm, m, h, flags=0):
    """P2G only: (node_ijk[G,3], m_i[G], p_i[G,3])."""
    lib = _load()
    x, v, Cm, m = _f64(x, (-1, 3)), _f64(v, (-1, 3)), _f64(Cm, (-1, 3, 3)), _f64(m, -1)
    n = x.shape[0]
    ijk = np.zeros((64 * max(n, 1), 3), np.int64)
    mass = np.zeros(64 * max(n, 1))
    mom = np.zeros((64 * max(n, 1), 3))
    G = lib.oracle_p2g_grid(n, _ptr(x), _ptr(v), _ptr(Cm), _ptr(m), float(h), int(flags), _ptr(ijk), _ptr(mass), _ptr(mom))
    if G < 0:
        raise ValueError("oracle_p2g_grid: invalid arguments")
    return ijk[:G].copy(), mass[:G].copy(), mom[:G].copy()


def g2p_from_grid(x, h, node_ijk, vgrid, Cin=None, flags=0):
    lib = _load()
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    node_ijk = np.ascontiguousarray(np.asarray(node_ijk, np.int64).reshape(-1, 3))
    vgrid = _f64(vgrid, (-1, 3))
    Cin = np.zeros((n, 3, 3)) if Cin is None else _f64(Cin, (-1, 3, 3))
    vout, Cout = np.zeros((n, 3)), np.zeros((n, 3, 3))
    rc = lib.oracle_g2p_from_grid(n, _ptr(x), float(h), int(flags), node_ijk.shape[0], _ptr(node_ijk), _ptr(vgrid), _ptr(Cin), _ptr(vout), _ptr(Cout))
    if rc != 0:
        raise ValueError("oracle_g2p_from_grid: invalid arguments")
    return vout, Cout


def apply_H(x, v, Cm, m, h, flags=0):
    lib = _load()
    x, v, Cm, m = _f64(x, (-1, 3)), _f64(v, (-1, 3)), _f64(Cm, (-1, 3, 3)), _f64(m, -1)
    vout, Cout = np.zeros_like(v), np.zeros_like(Cm)
    if lib.oracle_apply_H(x.shape[0], _ptr(x), _ptr(v), _ptr(Cm), _ptr(m), float(h), int(flags), _ptr(vout), _ptr(Cout)) != 0:
        raise ValueError("oracle_apply_H: invalid arguments")
    return vout, Cout


def momentum(x, v, Cm, m, h):
    lib = _load()
    x, v, Cm, m = _f64(x, (-1, 3)), _f64(v, (-1, 3)), _f64(Cm, (-1, 3, 3)), _f64(m, -1)
    P, L = np.zeros(3), np.zeros(3)
    if lib.oracle_momentum(x.shape[0], _ptr(x), _ptr(v), _ptr(Cm), _ptr(m), float(h), _ptr(P), _ptr(L)) != 0:
        raise ValueError("oracle_momentum: invalid arguments")
    return P, L


def contact_step(x, v, Cm, m, nrm, body, h, mu, n_iter, n_bodies=None, mu_pair=None, flags=0):
    """The full contact step.  Returns (v_out[n,3], C_out[n,3,3], stats dict)."""
    lib = _load()
    x, v, Cm, m, nrm = _f64(x, (-1, 3)), _f64(v, (-1, 3)), _f64(Cm, (-1, 3, 3)), _f64(m, -1), _f64(nrm, (-1, 3))
    body = np.ascontiguousarray(np.asarray(body, np.int32).reshape(-1))
    n = x.shape[0]
    if n_bodies is None:
        n_bodies = int(body.max()) + 1 if n else 1
    mp = None if mu_pair is None else _f64(mu_pair, (n_bodies, n_bodies))
    vout, Cout = np.zeros((n, 3)), np.zeros((n, 3, 3))
    st = np.zeros(13)
    rc = lib.oracle_contact_step(n, int(n_bodies), _ptr(body), _ptr(x), _ptr(v), _ptr(Cm), _ptr(m), _ptr(nrm),
                                 float(h), float(mu), _ptr(mp), int(n_iter), int(flags), _ptr(vout), _ptr(Cout), _ptr(st))
    if rc != 0:
        raise ValueError("oracle_contact_step: invalid arguments")
    stats = dict(P_in=st[0:3].copy(), P_out=st[3:6].copy(), L_in=st[6:9].copy(), L_out=st[9:12].copy(),
                 multibody_nodes=int(st[12]))
    return vout, Cout, stats


def apic1d_linear(x, v, B, m, h, x0=0.0):
    lib = _load()
    x, v, B, m = _f64(x, -1), _f64(v, -1), _f64(B, -1), _f64(m, -1)
    vout, Bout = np.zeros_like(v), np.zeros_like(B)
    if lib.oracle_apic1d_linear(x.shape[0], _ptr(x), _ptr(v), _ptr(B), _ptr(m), float(h), float(x0), _ptr(vout), _ptr(Bout)) != 0:
        raise ValueError("oracle_apic1d_linear: invalid arguments")
    return vout, Bout


def node_normals(x, tri):
    """Area-weighted, normalised node normals from boundary triangles
    (Sec. 2.3); 0 for nodes on no face."""
    lib = _load()
    x = _f64(x, (-1, 3))
    tri = np.ascontiguousarray(np.asarray(tri, np.int32).reshape(-1, 3))
    out = np.zeros_like(x)
    if lib.oracle_node_normals(x.shape[0], _ptr(x), tri.shape[0], tri.ctypes.data, _ptr(out)) != 0:
        raise ValueError("oracle_node_normals: a triangle index is outside [0, n)")
    return out


def weight_grads(xi):
    """Derivatives dN_k/dxi (k = 0..3) of the App. B weights at xi = x/h."""
    lib = _load()
    out = np.zeros(4)
    lib.oracle_weight_grads(float(xi), out.ctypes.data)
    return out


MASS_NORMAL_THRESHOLD = 0.5  # |grad rho| h / rho above which a particle is on the surface


def mass_normals(x, m, body, h, n_bodies=None, threshold=MASS_NORMAL_THRESHOLD):
    """Normals from each body's grid mass: n = -grad rho / |grad rho| where
    |grad rho| h > threshold rho, else 0.  Returns (nrm [n,3], ratio [n]),
    ratio = |grad rho| h / rho."""
    lib = _load()
    x = _f64(x, (-1, 3))
    m = _f64(m, -1)
    body = np.ascontiguousarray(np.asarray(body, np.int32).reshape(-1))
    if n_bodies is None:
        n_bodies = int(body.max()) + 1 if body.size else 1
    nrm = np.zeros_like(x)
    ratio = np.zeros(x.shape[0])
    if lib.oracle_mass_normals(x.shape[0], int(n_bodies), body.ctypes.data, _ptr(x), _ptr(m), float(h),
                               float(threshold), _ptr(nrm), _ptr(ratio)) != 0:
        raise ValueError("oracle_mass_normals: invalid arguments")
    return nrm, ratio


def augury_steps(x, v, Cm, m, body, springs, rest, stiffness, tri, h, mu, n_iter, dt, tau, n_steps, av=None,
                 aC=None, gravity=None, fixed=None, n_bodies=None, mu_pair=None, flags=0, init=True):
    """Augury dynamics (Sec. 2.2, eq. Newmark read as velocity Verlet) with a
    linear-spring foreground.  Returns (x, v, C[n,3,3], av, aC[n,3,3],
    energy dict) after n_steps; inputs are not modified."""
    lib = _load()
    x, v, Cm, m = _f64(x, (-1, 3)).copy(), _f64(v, (-1, 3)).copy(), _f64(Cm, (-1, 3, 3)).copy(), _f64(m, -1)
    n = x.shape[0]
    av = np.zeros((n, 3)) if av is None else _f64(av, (-1, 3)).copy()
    aC = np.zeros((n, 3, 3)) if aC is None else _f64(aC, (-1, 3, 3)).copy()
    body = np.ascontiguousarray(np.asarray(body, np.int32).reshape(-1))
    if n_bodies is None:
        n_bodies = int(body.max()) + 1
    sp = np.ascontiguousarray(np.asarray(springs, np.int32).reshape(-1, 2))
    rest, stiffness = _f64(rest, -1), _f64(stiffness, -1)
    tri = np.ascontiguousarray(np.asarray(tri, np.int32).reshape(-1, 3))
    g = None if gravity is None else _f64(gravity, 3)
    fx = None if fixed is None else np.ascontiguousarray(np.asarray(fixed, np.uint8).reshape(-1))
    mp = None if mu_pair is None else _f64(mu_pair, (n_bodies, n_bodies))
    en = np.zeros(3)
    rc = lib.oracle_augury_steps(n, int(n_bodies), _ptr(body), _ptr(x), _ptr(v), _ptr(Cm), _ptr(av), _ptr(aC),
                                 _ptr(m), None if fx is None else fx.ctypes.data, sp.shape[0], sp.ctypes.data,
                                 _ptr(rest), _ptr(stiffness), _ptr(g), tri.shape[0], tri.ctypes.data if len(tri) else None,
                                 float(h), float(mu), _ptr(mp), int(n_iter), int(flags), float(dt), float(tau),
                                 int(n_steps), 1 if init else 0, _ptr(en))
    if rc != 0:
        raise ValueError("oracle_augury_steps: invalid arguments")
    return x, v, Cm, av, aC, dict(kinetic=en[0], springs=en[1], gravity=en[2])
