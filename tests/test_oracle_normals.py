"""Pins of the oracle's node normals (Sec. 2.3: area-weighted outward normals
of the boundary faces adjacent to a node, normalised) against closed forms
and symmetries.  Each case would catch a plausible mistake: weighting by face
count instead of area, a flipped cross product, a missing normalisation,
interior nodes given a normal."""
import numpy as np
import pytest

import oracle
from paper_2108_02259_gb300 import scenes


def test_cube_corners_and_face_centres():
    x, tri = scenes.cube_surface_mesh(2.0)
    n = oracle.node_normals(x, tri)
    signs = np.array([[i, j, k] for k in (-1, 1) for j in (-1, 1) for i in (-1, 1)], np.float64)
    assert np.abs(n[:8] - signs / np.sqrt(3.0)).max() < 1e-15
    axes = np.array([[0, 0, -1], [0, 0, 1], [0, -1, 0], [0, 1, 0], [-1, 0, 0], [1, 0, 0]], np.float64)
    assert np.abs(n[8:] - axes).max() < 1e-15


def test_area_weighting_not_face_count():
    """A node shared by a horizontal triangle of area 2 (normal +z) and a
    vertical one of area 1 (normal +x): n = (1, 0, 2)/sqrt(5).  Averaging
    unit normals per face would give (1, 0, 1)/sqrt(2)."""
    x = np.array([[0, 0, 0], [2, 0, 0], [0, 2, 0], [0, 0, -1]], np.float64)
    tri = [[0, 1, 2], [0, 3, 2]]
    n = oracle.node_normals(x, tri)
    want = np.array([1.0, 0.0, 2.0]) / np.sqrt(5.0)
    assert np.abs(n[0] - want).max() < 1e-15
    assert np.abs(n[2] - want).max() < 1e-15
    assert np.abs(n[1] - [0, 0, 1]).max() < 1e-15
    assert np.abs(n[3] - [1, 0, 0]).max() < 1e-15


def test_planar_mesh_has_the_plane_normal():
    rng = np.random.default_rng(4)
    x, tri = scenes.box_lattice_surface(6, 5, 2)
    top = tri[np.all(x[tri][:, :, 2] == 1.0, axis=1)]  # the +z face only
    R = np.linalg.qr(rng.normal(size=(3, 3)))[0]
    n = oracle.node_normals(x @ R.T + 0.3, top)
    on = np.unique(top)
    assert np.abs(n[on] - R[:, 2]).max() < 1e-13
    off = np.setdiff1d(np.arange(len(x)), on)
    assert np.all(n[off] == 0.0)


def test_icosahedron_vertices_are_radial_and_icosphere_converges():
    x, tri = scenes.icosphere(0)
    assert np.abs(oracle.node_normals(x, tri) - x).max() < 1e-15  # 5-fold symmetry at every vertex
    prev = None
    for level in (2, 3, 4):
        x, tri = scenes.icosphere(level)
        err = np.arccos(np.clip((oracle.node_normals(x, tri) * x).sum(1), -1, 1)).max()
        if prev is not None:
            assert err < 0.6 * prev  # first order: the error halves with the edge length
        prev = err
    assert prev < 7e-3


def test_winding_rotation_translation():
    rng = np.random.default_rng(9)
    x, tri = scenes.icosphere(2)
    x = x * rng.uniform(0.5, 1.5, size=(1, 3))  # an ellipsoid
    n = oracle.node_normals(x, tri)
    assert np.abs(oracle.node_normals(x, tri[:, ::-1]) + n).max() < 1e-15
    R = np.linalg.qr(rng.normal(size=(3, 3)))[0]
    if np.linalg.det(R) < 0:
        R[:, 0] *= -1
    assert np.abs(oracle.node_normals(x @ R.T + [3.0, -2.0, 7.5], tri) - n @ R.T).max() < 1e-13


def test_interior_nodes_degenerate_faces_and_bad_indices():
    x, tri = scenes.box_lattice_surface(5, 4, 6)
    n = oracle.node_normals(x, tri)
    interior = np.array([(0 < i < 4) and (0 < j < 3) and (0 < k < 5)
                         for k in range(6) for j in range(4) for i in range(5)])
    assert np.all(n[interior] == 0.0)
    assert np.allclose(np.linalg.norm(n[~interior], axis=1), 1.0, atol=1e-15)
    assert np.all(((x[~interior] - x.mean(0)) * n[~interior]).sum(1) > 0)  # outward
    # zero-area triangles (collinear corners, a repeated corner) add nothing;
    # nodes on them alone keep n = 0
    x2 = np.vstack([x, [[10, 10, 10], [11, 10, 10], [12, 10, 10]]])
    m = len(x)
    n2 = oracle.node_normals(x2, np.vstack([tri, [[m, m + 1, m + 2], [0, 1, 0]]]))
    assert np.all(n2[m:] == 0.0)
    assert np.all(n2[:m] == n)
    with pytest.raises(ValueError):
        oracle.node_normals(x, np.vstack([tri, [[0, 1, len(x)]]]))
    with pytest.raises(ValueError):
        oracle.node_normals(x, np.vstack([tri, [[0, -1, 2]]]))
