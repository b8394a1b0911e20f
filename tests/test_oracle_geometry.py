"""Pins for oracle/geometry.py: exact volumes and areas of the cube meshes,
a hand-counted edge set, and affine reproduction of the shape functions."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import geometry as G


def test_cube_volumes_and_shape_gradients():
    m = W.cube_mesh(4)
    Dm, Dminv, V = G.shape_matrices(m.nodes, m.tets)
    assert np.all(V > 0)
    assert V.sum() == pytest.approx(1.0, rel=1e-14)
    np.testing.assert_allclose(V, (1 / 4) ** 3 / 6, rtol=1e-12)    # every Kuhn tet is 1/6 hex
    g = G.shape_gradients(Dminv)
    # sum_a x_a (x) grad N_a reproduces any affine field's gradient exactly
    A = np.array([[0.3, -0.2, 0.1], [0.05, 0.4, -0.3], [0.2, 0.1, -0.1]])
    x = m.nodes @ A.T + np.array([1.0, 2.0, 3.0])
    F = np.einsum("eai,eaj->eij", x[m.tets], g)
    np.testing.assert_allclose(F, np.broadcast_to(A, F.shape), atol=1e-12)
    np.testing.assert_allclose(G.deformation_gradient(x, m.tets, Dminv), F, atol=1e-12)


def test_single_hex_edges_hand_count():
    """One Kuhn-split cube: 12 cube edges, 6 face diagonals, 1 body diagonal."""
    m = W.cube_mesh(1)
    e = G.unique_edges(m.tets)
    assert len(e) == 19
    assert G.mean_edge_length(m.nodes, m.tets) == pytest.approx(
        (12 + 6 * math.sqrt(2) + math.sqrt(3)) / 19, rel=1e-14)


def test_cube_boundary_and_lumped_areas():
    n = 8
    m = W.cube_mesh(n)
    faces = G.boundary_faces(m.tets)
    assert len(faces) == 6 * n * n * 2
    A = G.lumped_areas(m.nodes, faces, m.n_nodes)
    assert A.sum() == pytest.approx(6.0, rel=1e-13)
    X = m.nodes
    h = 1.0 / n
    interior_top = (np.abs(X[:, 2] - 1) < 1e-12) & (X[:, 0] > 1e-9) & (X[:, 0] < 1 - 1e-9) \
        & (X[:, 1] > 1e-9) & (X[:, 1] < 1 - 1e-9)
    np.testing.assert_allclose(A[interior_top], h * h, rtol=1e-12)
    inside = np.all((X > 1e-9) & (X < 1 - 1e-9), axis=1)
    assert np.all(A[inside] == 0)


def test_penalty_candidates_and_values():
    m = W.cube_mesh(4)
    fixed = G.fixed_dof_mask(m.n_nodes, m.fixed_nodes, m.fixed_mask)
    E = np.full(m.n_tets, 2.0)
    k, h_bar, Emax = G.penalty_stiffness(m.nodes, m.tets, E, fixed, 10.0)
    A = G.lumped_areas(m.nodes, G.boundary_faces(m.tets), m.n_nodes)
    cand = k > 0
    # candidates: boundary nodes minus the fully fixed bottom face
    X = m.nodes
    on_b = np.any((X < 1e-9) | (X > 1 - 1e-9), axis=1)
    assert np.array_equal(cand, on_b & (X[:, 2] > 1e-9))
    np.testing.assert_allclose(k[cand], 10.0 * 2.0 * A[cand] / h_bar, rtol=1e-14)


def test_fixed_dof_mask_bits():
    mask = G.fixed_dof_mask(5, np.array([1, 3]), np.array([0b101, 0b010], dtype=np.uint8))
    assert mask[1].tolist() == [True, False, True]
    assert mask[3].tolist() == [False, True, False]
    assert not mask[[0, 2, 4]].any()
