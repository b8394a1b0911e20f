"""Mesh geometry for linear tets, FP64 (oracle; test infrastructure only).

Linear tetrahedra with one-point (exact) integration, as in the paper's
volumetric FEM of Sec. III-A:

    Dm = [X1-X0, X2-X0, X3-X0]    (columns),   V = det(Dm) / 6 > 0,
    F  = Ds Dm^-1,  Ds = [x1-x0, x2-x0, x3-x0],
    grad N_a = Dm^-T e_a (a = 1..3),  grad N_0 = -(grad N_1 + grad N_2 + grad N_3).

Contact penalty reading (the paper only says collisions are resolved through a
thin collision layer, Sec. III-A; no law is given):

    k_i = c_kappa * E_max,i * A_i / h_bar

for every boundary node i that is not fully fixed, where A_i is one third of
the area of the boundary triangles (faces seen by exactly one tet) touching i,
E_max,i is the largest Young's modulus among tets at i and h_bar is the mean
length of the unique mesh edges.
"""
from __future__ import annotations

import numpy as np


def shape_matrices(X, tets):
    """Dm (Nt,3,3), Dm^-1 (Nt,3,3), V (Nt,)."""
    x0 = X[tets[:, 0]]
    Dm = np.stack([X[tets[:, 1]] - x0, X[tets[:, 2]] - x0, X[tets[:, 3]] - x0], axis=2)
    V = np.linalg.det(Dm) / 6.0
    return Dm, np.linalg.inv(Dm), V


def shape_gradients(Dminv):
    """grad N_a for a = 0..3, shape (Nt, 4, 3). Row a-1 of Dm^-1 is grad N_a."""
    g123 = Dminv                          # (Nt, 3, 3): [a-1, :] = grad N_a
    g0 = -g123.sum(axis=1, keepdims=True)
    return np.concatenate([g0, g123], axis=1)


def deformation_gradient(x, tets, Dminv):
    """F = Ds(x) Dm^-1 for current positions x (Nn, 3)."""
    x0 = x[tets[:, 0]]
    Ds = np.stack([x[tets[:, 1]] - x0, x[tets[:, 2]] - x0, x[tets[:, 3]] - x0], axis=2)
    return Ds @ Dminv


def boundary_faces(tets):
    """Triangles that belong to exactly one tet, as sorted vertex triples."""
    faces = np.concatenate([tets[:, [0, 1, 2]], tets[:, [0, 1, 3]],
                            tets[:, [0, 2, 3]], tets[:, [1, 2, 3]]], axis=0)
    faces = np.sort(faces, axis=1)
    uniq, counts = np.unique(faces, axis=0, return_counts=True)
    return uniq[counts == 1]


def lumped_areas(X, faces, n_nodes):
    """A_i = sum over boundary triangles at i of area / 3."""
    a = X[faces[:, 1]] - X[faces[:, 0]]
    b = X[faces[:, 2]] - X[faces[:, 0]]
    area = 0.5 * np.linalg.norm(np.cross(a, b), axis=1)
    A = np.zeros(n_nodes)
    for k in range(3):
        np.add.at(A, faces[:, k], area / 3.0)
    return A


def unique_edges(tets):
    pairs = np.concatenate([tets[:, [0, 1]], tets[:, [0, 2]], tets[:, [0, 3]],
                            tets[:, [1, 2]], tets[:, [1, 3]], tets[:, [2, 3]]], axis=0)
    return np.unique(np.sort(pairs, axis=1), axis=0)


def mean_edge_length(X, tets):
    e = unique_edges(tets)
    return float(np.mean(np.linalg.norm(X[e[:, 1]] - X[e[:, 0]], axis=1)))


def node_max_modulus(tets, tet_E, n_nodes):
    Emax = np.zeros(n_nodes)
    for k in range(4):
        np.maximum.at(Emax, tets[:, k], tet_E)
    return Emax


def fixed_dof_mask(n_nodes, fixed_nodes, fixed_mask):
    """Boolean (Nn, 3): True where the displacement component is prescribed."""
    m = np.zeros((n_nodes, 3), dtype=bool)
    fixed_nodes = np.asarray(fixed_nodes, dtype=np.int64)
    if fixed_mask is None:
        m[fixed_nodes, :] = True
    else:
        bits = np.asarray(fixed_mask, dtype=np.uint8)
        for c in range(3):
            m[fixed_nodes, c] |= ((bits >> c) & 1).astype(bool)
    return m


def penalty_stiffness(X, tets, tet_E, fixed, c_kappa):
    """k_i (Nn,) per the reading in the module docstring; 0 for non-candidates.
    Returns (k, h_bar, E_max per node)."""
    n = len(X)
    faces = boundary_faces(tets)
    A = lumped_areas(X, faces, n)
    h_bar = mean_edge_length(X, tets)
    Emax = node_max_modulus(tets, tet_E, n)
    on_boundary = np.zeros(n, dtype=bool)
    on_boundary[faces.ravel()] = True
    candidate = on_boundary & ~fixed.all(axis=1)
    k = np.where(candidate, c_kappa * Emax * A / h_bar, 0.0)
    return k, h_bar, Emax
