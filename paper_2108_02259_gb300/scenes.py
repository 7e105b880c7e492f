"""Seeded synthetic contact scenes shaped like the paper's workloads.

This module only makes inputs: node clouds of finite-element-like bodies
(lattice boxes, lattice balls, ellipsoids), their masses, outward normals,
rigid-body velocities and the matching affine matrices C = skew(omega).  It
holds none of the contact method's arithmetic and is shared by the oracle
tests, the CUDA tests and the benchmark.

Conventions (same as the library): x[n,3] float64, v[n,3], C[n,3,3] with
C[p, a, b] = d v_a / d x_b, m[n], nrm[n,3] (unit outward normal for surface
nodes, zero for interior nodes), body[n] int32.

Normals follow Sec. 2.3 of the paper (area-weighted outward normals of the
boundary faces adjacent to a node): on a lattice box a face node gets the
face normal, an edge node the normalised sum of two, a corner node of three;
on a ball or ellipsoid the normal is the normalised gradient of the implicit
surface at the node.  Interior nodes get 0.
"""
from __future__ import annotations

import os
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2108_0225


@dataclass
class Scene:
    x: np.ndarray
    v: np.ndarray
    C: np.ndarray
    m: np.ndarray
    nrm: np.ndarray
    body: np.ndarray
    n_bodies: int
    h: float
    mu: float
    n_iter: int
    mu_pair: np.ndarray | None = None
    name: str = ""
    info: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def astype(self, dt) -> "Scene":
        """Copy with v, C, m, nrm in dtype dt (x stays float64)."""
        return Scene(self.x.copy(), self.v.astype(dt), self.C.astype(dt), self.m.astype(dt),
                     self.nrm.astype(dt), self.body.copy(), self.n_bodies, self.h, self.mu,
                     self.n_iter, None if self.mu_pair is None else self.mu_pair.copy(),
                     self.name, dict(self.info))


def skew(w):
    """Matrix of the cross product: skew(w) @ r == cross(w, r)."""
    w = np.asarray(w, np.float64)
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def haar_rotation(rng) -> np.ndarray:
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def random_direction(rng) -> np.ndarray:
    d = rng.standard_normal(3)
    return d / np.linalg.norm(d)


def _box_lattice(nx, ny, nz, s):
    """Lattice box centred at 0 with spacing s, and its area-weighted normals."""
    I, J, K = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    I, J, K = I.ravel(), J.ravel(), K.ravel()
    pts = np.stack([(I - (nx - 1) / 2) * s, (J - (ny - 1) / 2) * s, (K - (nz - 1) / 2) * s], 1)
    nrm = np.zeros_like(pts)
    for ax, (idx, nmax) in enumerate(((I, nx), (J, ny), (K, nz))):
        nrm[idx == 0, ax] -= 1.0
        nrm[idx == nmax - 1, ax] += 1.0
    ln = np.linalg.norm(nrm, axis=1)
    nz_ = ln > 0
    nrm[nz_] /= ln[nz_, None]
    return pts, nrm


def _implicit_lattice(count, s, axes, shape, jitter, rng):
    """The `count` lattice points (spacing s) innermost in an ellipsoid or box
    with semi-axis ratios `axes`; surface points get outward normals."""
    axes = np.asarray(axes, np.float64)
    vol_unit = (4.0 / 3.0 * np.pi) if shape == "ellipsoid" else 8.0
    R = (count * s**3 / (vol_unit * np.prod(axes))) ** (1.0 / 3.0) * 1.15
    ext = np.ceil(R * axes / s).astype(int) + 2
    gi = [np.arange(-e, e + 1) for e in ext]
    I, J, K = np.meshgrid(*gi, indexing="ij")
    lat = np.stack([I.ravel(), J.ravel(), K.ravel()], 1)
    pts = lat * s

    def level(p):
        q = p / (axes * R)
        if shape == "ellipsoid":
            return np.sqrt((q**2).sum(1))
        return np.abs(q).max(1)

    lev = level(pts)
    order = np.argsort(lev, kind="stable")[:count]
    lat, pts, lev = lat[order], pts[order], lev[order]
    # surface = lattice points with a missing 6-neighbour
    occ = np.zeros(tuple(2 * ext + 3), bool)
    li = lat + ext + 1
    occ[li[:, 0], li[:, 1], li[:, 2]] = True
    surf = np.zeros(count, bool)
    for d in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
        nb = li + np.array(d)
        surf |= ~occ[nb[:, 0], nb[:, 1], nb[:, 2]]
    nrm = np.zeros_like(pts)
    if shape == "ellipsoid":
        g = pts / (axes * R) ** 2
    else:
        q = pts / (axes * R)
        g = np.zeros_like(pts)
        amax = np.abs(q).max(1, keepdims=True)
        g = np.where(np.abs(q) >= amax - 1e-12, np.sign(q), 0.0)
    g = g / np.maximum(np.linalg.norm(g, axis=1, keepdims=True), 1e-300)
    nrm[surf] = g[surf]
    if jitter > 0:
        pts = pts + rng.uniform(-jitter, jitter, pts.shape)
    return pts, nrm


def _rigid(pts, nrm, R, center, v0, w):
    x = pts @ R.T + center
    n = nrm @ R.T
    v = v0 + np.cross(w, x - center)
    C = np.broadcast_to(skew(w), (x.shape[0], 3, 3)).copy()
    return x, n, v, C


def _assemble(parts, h, mu, n_iter, name, mu_pair=None, info=None):
    x = np.concatenate([p[0] for p in parts])
    nrm = np.concatenate([p[1] for p in parts])
    v = np.concatenate([p[2] for p in parts])
    C = np.concatenate([p[3] for p in parts])
    m = np.concatenate([p[4] for p in parts])
    body = np.concatenate([np.full(p[0].shape[0], b, np.int32) for b, p in enumerate(parts)])
    return Scene(x, v, C, m, nrm, body, len(parts), h, mu, n_iter, mu_pair, name, info or {})


def two_cubes(mu: float = 0.3, n_iter: int = 10, approach: bool = True) -> Scene:
    """Two 8x8x8-node cubes (spacing 1/32, 1/512 mass per node), centres at
    x = 0.35 and 0.65 moving head-on at +-1 (C = 0), h = 1/32."""
    s = 1.0 / 32
    pts, nrm = _box_lattice(8, 8, 8, s)
    sign = 1.0 if approach else -1.0
    parts = []
    for cx, vx in ((0.35, sign), (0.65, -sign)):
        x = pts + np.array([cx, 0.5, 0.5])
        v = np.tile([vx, 0.0, 0.0], (x.shape[0], 1))
        parts.append((x, nrm.copy(), v, np.zeros((x.shape[0], 3, 3)), np.full(x.shape[0], 1.0 / 512)))
    return _assemble(parts, 1.0 / 32, mu, n_iter, "two_cubes_8x8x8_h1/32")


def four_bodies(seed: int = SEED_BASE + 2, scale: float = 1.0, mu: float = 0.3, n_iter: int = 8,
                h: float = 1.0 / 256) -> Scene:
    """Two lattice boxes (50x40x25 nodes) and two lattice balls (50,000
    nodes), spacing h/2, jittered by U(-0.1h, 0.1h), Haar-random rotations,
    random rigid velocities |v| <= 2 and |omega| <= 5, placed as two facing
    pairs with surface gaps U(0, 2h).  `scale` < 1 shrinks the node counts
    (for tests); 1 gives 200,000 nodes."""
    rng = np.random.default_rng(seed)
    s = h / 2
    jit = 0.1 * h
    nb = max(int(round(50 * scale ** (1 / 3))), 2), max(int(round(40 * scale ** (1 / 3))), 2), max(int(round(25 * scale ** (1 / 3))), 2)
    nball = int(nb[0] * nb[1] * nb[2])
    shapes = []
    for kind in ("box", "ball", "box", "ball"):
        if kind == "box":
            pts, nrm = _box_lattice(*nb, s)
            pts = pts + rng.uniform(-jit, jit, pts.shape)
        else:
            pts, nrm = _implicit_lattice(nball, s, (1, 1, 1), "ellipsoid", jit, rng)
        shapes.append((pts, nrm))
    parts = []
    for pair in range(2):
        A, B = shapes[2 * pair], shapes[2 * pair + 1]
        RA, RB = haar_rotation(rng), haar_rotation(rng)
        pa, pb = A[0] @ RA.T, B[0] @ RB.T
        gap = rng.uniform(0, 2 * h)
        yc = 0.3 + 0.4 * pair
        ca = np.array([0.5 - pa[:, 0].max() - gap / 2, yc, 0.5])
        cb = np.array([0.5 - pb[:, 0].min() + gap / 2, yc, 0.5])
        for (pts, nrm), R, c, side in (((A[0], A[1]), RA, ca, 1.0), ((B[0], B[1]), RB, cb, -1.0)):
            v0 = random_direction(rng) * rng.uniform(0, 2)
            v0[0] = side * abs(v0[0])  # the pair approaches along x
            w = random_direction(rng) * rng.uniform(0, 5)
            x, n, v, Cm = _rigid(pts, nrm, R, c, v0, w)
            m = np.full(x.shape[0], 1.0 / x.shape[0])
            parts.append((x, n, v, Cm, m))
    return _assemble(parts, h, mu, n_iter, f"four_bodies_{sum(p[0].shape[0] for p in parts)}_h1/{round(1 / h)}",
                     info=dict(seed=seed))


def eight_bodies(seed: int = SEED_BASE + 3, per_body: int = 500_000, n_iter: int = 8,
                 h: float = 1.0 / 512) -> Scene:
    """Eight tetrahedral-mesh-like node clouds: jittered lattices (spacing
    h/2, jitter U(-h/8, h/8)) inside ellipsoids or boxes with axis ratios
    U(0.6, 1), the `per_body` innermost points each; four approaching pairs
    whose surfaces overlap by up to h; lognormal masses (sigma 0.3) scaled to
    unit mass per body; mu(b, b') ~ U[0.1, 0.5], symmetric."""
    rng = np.random.default_rng(seed)
    s = h / 2
    parts = []
    centres = [(0.3, 0.3), (0.3, 0.7), (0.7, 0.3), (0.7, 0.7)]
    for pair in range(4):
        shp = []
        for _ in range(2):
            kind = "ellipsoid" if rng.uniform() < 0.5 else "box"
            axes = rng.uniform(0.6, 1.0, 3)
            pts, nrm = _implicit_lattice(per_body, s, axes, kind, 0.25 * s, rng)
            R = haar_rotation(rng)
            shp.append((pts @ R.T, nrm @ R.T))
        overlap = rng.uniform(0, h)
        yc, zc = centres[pair]
        ca = np.array([0.5 - shp[0][0][:, 0].max() + overlap / 2, yc, zc])
        cb = np.array([0.5 - shp[1][0][:, 0].min() - overlap / 2, yc, zc])
        for (pts, nrm), c, side in ((shp[0], ca, 1.0), (shp[1], cb, -1.0)):
            v0 = random_direction(rng) * rng.uniform(0, 2)
            v0[0] = side * abs(v0[0])
            w = random_direction(rng) * rng.uniform(0, 5)
            x = pts + c
            v = v0 + np.cross(w, pts)
            Cm = np.broadcast_to(skew(w), (x.shape[0], 3, 3)).copy()
            m = rng.lognormal(0.0, 0.3, x.shape[0])
            m = m / m.sum()
            parts.append((x, nrm, v, Cm, m))
    nb = len(parts)
    mp = rng.uniform(0.1, 0.5, (nb, nb))
    mp = np.triu(mp) + np.triu(mp, 1).T
    return _assemble(parts, h, 0.3, n_iter, f"eight_bodies_{nb * per_body}_h1/{round(1 / h)}",
                     mu_pair=mp, info=dict(seed=seed))


def random_cloud(n: int, n_bodies: int = 2, seed: int = 0, h: float = 0.1, affine: bool = False,
                 spread: float = 1.0, mu: float = 0.3, n_iter: int = 3, origin=(0.0, 0.0, 0.0),
                 interior_frac: float = 0.3) -> Scene:
    """Random non-affine state on a random cloud (test input): uniform
    positions in a cube of side `spread`, random masses in [0.5, 1.5],
    random unit normals (a fraction zeroed as interior), and either random
    v, C or one shared affine field v = v0 + L x, C = L."""
    rng = np.random.default_rng(seed)
    x = np.asarray(origin) + rng.uniform(0, spread, (n, 3))
    m = rng.uniform(0.5, 1.5, n)
    nrm = rng.standard_normal((n, 3))
    nrm /= np.maximum(np.linalg.norm(nrm, axis=1, keepdims=True), 1e-300)
    nrm[rng.uniform(size=n) < interior_frac] = 0.0
    body = rng.integers(0, n_bodies, n).astype(np.int32)
    if affine:
        v0 = rng.standard_normal(3)
        L = rng.standard_normal((3, 3))
        v = v0 + x @ L.T
        Cm = np.broadcast_to(L, (n, 3, 3)).copy()
    else:
        v = rng.standard_normal((n, 3))
        Cm = rng.standard_normal((n, 3, 3)) / h
    return Scene(x, v, Cm, m, nrm, body, n_bodies, h, mu, n_iter, None, f"random_cloud_{n}", dict(seed=seed))


def multi_body_scene(rng, total_nodes: int, n_bodies: int, h: float, mu: float = 0.3, n_iter: int = 8,
                     name: str = "") -> Scene:
    """`n_bodies` lattice boxes and balls (alternating) of total_nodes /
    n_bodies nodes each, spacing h/2, jitter U(-0.1h, 0.1h), Haar-random
    rotations, rigid velocities |v| <= 2, |omega| <= 5, placed as approaching
    pairs along x (gaps U(0, 2h)) stacked along y."""
    s = h / 2
    per = max(int(total_nodes // n_bodies), 8)
    parts = []
    y = 0.0
    for b in range(0, n_bodies, 2):
        pair = []
        for k in range(b, min(b + 2, n_bodies)):
            if k % 2 == 0:
                e = max(int(round(per ** (1 / 3))), 2)
                pts, nrm = _box_lattice(e, e, max(per // (e * e), 1), s)
                pts = pts + rng.uniform(-0.1 * h, 0.1 * h, pts.shape)
            else:
                pts, nrm = _implicit_lattice(per, s, (1, 1, 1), "ellipsoid", 0.1 * h, rng)
            R = haar_rotation(rng)
            pair.append((pts @ R.T, nrm @ R.T))
        ext = max(np.ptp(p[0][:, 1]) for p in pair)
        yc = y + ext / 2 + 2 * h
        y = yc + ext / 2 + 4 * h
        gap = rng.uniform(0, 2 * h)
        ca = np.array([-pair[0][0][:, 0].max() - gap / 2, yc, 0.0])
        centres = [ca]
        if len(pair) == 2:
            centres.append(np.array([-pair[1][0][:, 0].min() + gap / 2, yc, 0.0]))
        for (pts, nrm), c, side in zip(pair, centres, (1.0, -1.0)):
            v0 = random_direction(rng) * rng.uniform(0, 2)
            v0[0] = side * abs(v0[0])
            w = random_direction(rng) * rng.uniform(0, 5)
            x = pts + c
            v = v0 + np.cross(w, pts)
            Cm = np.broadcast_to(skew(w), (x.shape[0], 3, 3)).copy()
            parts.append((x, nrm, v, Cm, np.full(x.shape[0], 1.0 / x.shape[0])))
    return _assemble(parts, h, mu, n_iter, name)


def batch_of_scenes(n_scenes: int = 64, seed: int = SEED_BASE + 4, min_nodes: float = 1e3, max_nodes: float = 2e5,
                    bodies=(2, 6), hs=(1.0 / 64, 1.0 / 128, 1.0 / 256), mu: float = 0.3, n_iter: int = 8):
    """Independent scenes of uneven size: ln P ~ U(ln min, ln max), bodies ~
    U{bodies}, h uniform over `hs`, node spacing h/2."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_scenes):
        P = int(np.exp(rng.uniform(np.log(min_nodes), np.log(max_nodes))))
        nb = int(rng.integers(bodies[0], bodies[1] + 1))
        h = float(hs[int(rng.integers(0, len(hs)))])
        out.append(multi_body_scene(rng, P, nb, h, mu, n_iter, name=f"scene{i}_{P}_{nb}b_h1/{round(1 / h)}"))
    return out


def served_simulations(n_sims: int = 256, seed: int = SEED_BASE + 5, min_nodes: float = 2e3,
                       max_nodes: float = 1e6, bodies=(2, 8), n_iter: int = 8, threads: int | None = None):
    """Simulations for the serving benchmark, each drawn on its own: ln P ~
    U(ln min, ln max) nodes, U{bodies} bodies, h in {1/128, 1/256, 1/512} by
    size (so that bodies span about 20-40 cells), friction mu ~ U[0, 0.5],
    and a shift of the whole scene by whole cells.  Simulation k draws from
    the generator seeded with (seed, k), so the set does not depend on how
    many threads build it (numpy releases the GIL in its array kernels)."""
    from concurrent.futures import ThreadPoolExecutor

    def one(k):
        rng = np.random.default_rng([seed, k])
        P = int(np.exp(rng.uniform(np.log(min_nodes), np.log(max_nodes))))
        nb = int(rng.integers(bodies[0], bodies[1] + 1))
        h = 1.0 / 128 if P < 2e4 else 1.0 / 256 if P < 2e5 else 1.0 / 512
        s = multi_body_scene(rng, P, nb, h, 0.3, n_iter, name=f"sim{k}_{P}_{nb}b")
        shift = rng.integers(-50, 50, 3) * s.h
        return Scene(s.x + shift, s.v, s.C, s.m, s.nrm, s.body, s.n_bodies, s.h, float(rng.uniform(0, 0.5)),
                     n_iter, None, s.name)

    workers = threads if threads is not None else min(16, os.cpu_count() or 1)
    with ThreadPoolExecutor(max(1, workers)) as ex:
        return list(ex.map(one, range(n_sims)))


# ----------------------------------------------------------- surface meshes
# Boundary triangulations for the node-normal construction of Sec. 2.3.
# Triangles are wound counter-clockwise seen from outside.

def cube_surface_mesh(side: float = 1.0):
    """Cube [0, side]^3: 8 corners then 6 face centres; each face is four
    triangles around its centre (so every corner sees each of its three faces
    through two triangles of equal area)."""
    c = np.array([[i, j, k] for k in (0, 1) for j in (0, 1) for i in (0, 1)], np.float64) * side
    faces = [  # corner ids counter-clockwise seen from outside, and the outward axis
        ([0, 2, 3, 1], (0, 0, -1)), ([4, 5, 7, 6], (0, 0, 1)),
        ([0, 1, 5, 4], (0, -1, 0)), ([2, 6, 7, 3], (0, 1, 0)),
        ([0, 4, 6, 2], (-1, 0, 0)), ([1, 3, 7, 5], (1, 0, 0)),
    ]
    x = [*c]
    tri = []
    for ids, _ in faces:
        centre = len(x)
        x.append(c[ids].mean(axis=0))
        for a in range(4):
            tri.append([centre, ids[a], ids[(a + 1) % 4]])
    return np.array(x), np.array(tri, np.int32)


def icosphere(level: int = 0, radius: float = 1.0):
    """Unit icosahedron subdivided `level` times, vertices projected to the
    sphere; outward winding."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
         (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11),
         (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    x = [np.array(p, np.float64) / np.linalg.norm(p) for p in v]
    for _ in range(level):
        mid = {}

        def midpoint(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                p = x[a] + x[b]
                x.append(p / np.linalg.norm(p))
                mid[key] = len(x) - 1
            return mid[key]

        nf = []
        for a, b, c in f:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = nf
    return np.array(x) * radius, np.array(f, np.int32)


def box_lattice_surface(nx: int, ny: int, nz: int, spacing: float = 1.0, origin=(0.0, 0.0, 0.0)):
    """All nodes of an nx x ny x nz lattice (x fastest) and the triangles of
    its boundary (each boundary quad split in two).  Interior nodes are on
    no triangle."""
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    x = np.stack([ii.T.ravel(), jj.T.ravel(), kk.T.ravel()], 1).astype(np.float64) * spacing + np.asarray(origin)

    def nid(i, j, k):
        return (k * ny + j) * nx + i

    tri = []

    def quad(a, b, c, d):  # counter-clockwise seen from outside
        tri.append([a, b, c])
        tri.append([a, c, d])

    for j in range(ny - 1):
        for k in range(nz - 1):
            quad(nid(0, j, k), nid(0, j, k + 1), nid(0, j + 1, k + 1), nid(0, j + 1, k))  # -x
            i = nx - 1
            quad(nid(i, j, k), nid(i, j + 1, k), nid(i, j + 1, k + 1), nid(i, j, k + 1))  # +x
    for i in range(nx - 1):
        for k in range(nz - 1):
            quad(nid(i, 0, k), nid(i + 1, 0, k), nid(i + 1, 0, k + 1), nid(i, 0, k + 1))  # -y
            j = ny - 1
            quad(nid(i, j, k), nid(i, j, k + 1), nid(i + 1, j, k + 1), nid(i + 1, j, k))  # +y
    for i in range(nx - 1):
        for j in range(ny - 1):
            quad(nid(i, j, 0), nid(i, j + 1, 0), nid(i + 1, j + 1, 0), nid(i + 1, j, 0))  # -z
            k = nz - 1
            quad(nid(i, j, k), nid(i + 1, j, k), nid(i + 1, j + 1, k), nid(i, j + 1, k))  # +z
    return x, np.array(tri, np.int32)


# ----------------------------------------------------- elastic foreground
# Inputs of the augury dynamics driver (Sec. 2.2): lattice bodies held
# together by linear springs (a stand-in for the paper's finite elements),
# with boundary triangles for the Sec. 2.3 normals.

@dataclass
class ElasticScene:
    scene: Scene               # x, v, C, m, body, h, mu, n_iter (nrm unused: built from tri)
    springs: np.ndarray        # [S, 2] int32 node pairs
    rest: np.ndarray           # [S] rest lengths
    stiffness: np.ndarray      # [S] spring constants
    tri: np.ndarray            # [T, 3] int32 boundary triangles, outward winding
    gravity: np.ndarray        # [3]
    dt: float
    tau: float


def lattice_springs(nx: int, ny: int, nz: int, spacing: float, k_axis: float, k_diag: float, offset: int = 0):
    """Springs of an nx x ny x nz lattice (x fastest): the 3 axis neighbours
    and the 2 diagonals of every lattice-cell face.  Returns (pairs, rest, k)."""
    idx = np.arange(nx * ny * nz).reshape(nz, ny, nx) + offset
    pairs, rest, ks = [], [], []

    def add(a, b, L, k):
        p = np.stack([a.ravel(), b.ravel()], 1)
        pairs.append(p)
        rest.append(np.full(len(p), L))
        ks.append(np.full(len(p), k))

    add(idx[:, :, :-1], idx[:, :, 1:], spacing, k_axis)
    add(idx[:, :-1, :], idx[:, 1:, :], spacing, k_axis)
    add(idx[:-1, :, :], idx[1:, :, :], spacing, k_axis)
    d = spacing * np.sqrt(2.0)
    add(idx[:, :-1, :-1], idx[:, 1:, 1:], d, k_diag)   # xy faces
    add(idx[:, :-1, 1:], idx[:, 1:, :-1], d, k_diag)
    add(idx[:-1, :, :-1], idx[1:, :, 1:], d, k_diag)   # xz faces
    add(idx[:-1, :, 1:], idx[1:, :, :-1], d, k_diag)
    add(idx[:-1, :-1, :], idx[1:, 1:, :], d, k_diag)   # yz faces
    add(idx[:-1, 1:, :], idx[1:, :-1, :], d, k_diag)
    return (np.concatenate(pairs).astype(np.int32), np.concatenate(rest), np.concatenate(ks))


def elastic_pair(n_side: int = 6, spacing: float = 1 / 32, v0: float = 1.0, wave_speed: float = 12.0,
                 gap_cells: float = 1.0, mu: float = 0.0, n_iter: int = 4, tilt: float = 0.0,
                 courant: float = 0.1) -> ElasticScene:
    """Two identical elastic lattice cubes (n_side^3 nodes, unit mass each)
    approaching head on along x at +-v0, mirror images of each other about
    the plane x = 0.5, which is a grid-node plane (h = 2 * spacing, the paper's
    background grid of twice the element size).  `tilt` rotates the second
    cube about the x axis (radians), breaking the symmetry.  Springs give a
    long-wave sound speed of about `wave_speed`; dt = courant * spacing / wave_speed."""
    h = 2.0 * spacing
    side = (n_side - 1) * spacing
    x0, t0 = box_lattice_surface(n_side, n_side, n_side, spacing)
    x0 = x0 - x0.mean(axis=0)
    gap = gap_cells * h
    c0 = np.array([0.5 - gap / 2 - side / 2, 0.5, 0.5])
    c1 = np.array([0.5 + gap / 2 + side / 2, 0.5, 0.5])
    xa = x0 + c0
    ca, sa = np.cos(tilt), np.sin(tilt)
    R = np.array([[1, 0, 0], [0, ca, -sa], [0, sa, ca]])
    xb = (x0 * np.array([-1.0, 1.0, 1.0])) @ R.T + c1  # mirrored lattice (then tilted)
    nb = len(x0)
    x = np.vstack([xa, xb])
    tri = np.vstack([t0, t0[:, ::-1] + nb]).astype(np.int32)  # mirroring flips the winding
    m = np.full(2 * nb, 1.0 / nb)
    rho = (1.0 / nb) / spacing ** 3
    k_axis = rho * wave_speed ** 2 * spacing  # E ~ k / spacing for a cubic lattice, c = sqrt(E / rho)
    pa, ra, kk = lattice_springs(n_side, n_side, n_side, spacing, k_axis, 0.5 * k_axis)
    springs = np.vstack([pa, pa + nb]).astype(np.int32)
    rest = np.concatenate([ra, ra])
    stiff = np.concatenate([kk, kk])
    v = np.zeros_like(x)
    v[:nb, 0], v[nb:, 0] = v0, -v0
    body = np.repeat(np.arange(2), nb).astype(np.int32)
    sc = Scene(x, v, np.zeros((2 * nb, 9)), m, np.zeros_like(x), body, 2, h, mu, n_iter, None,
               f"elastic_pair_{n_side}", dict(spacing=spacing, wave_speed=wave_speed, tilt=tilt))
    dt = courant * spacing / wave_speed
    return ElasticScene(sc, springs, rest, stiff, tri, np.zeros(3), dt, dt)
