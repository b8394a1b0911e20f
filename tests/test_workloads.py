"""Sanity of the seeded input generators (sizes, conformity, orientation,
determinism, initial-contact placement)."""
import math

import numpy as np
import pytest

import workloads as W


def _faces(tets):
    F = np.sort(np.concatenate([tets[:, [0, 1, 2]], tets[:, [0, 1, 3]],
                                tets[:, [0, 2, 3]], tets[:, [1, 2, 3]]]), axis=1)
    return np.unique(F, axis=0, return_counts=True)


def _vols(m):
    X, T = m.nodes, m.tets
    return np.einsum("ij,ij->i", X[T[:, 1]] - X[T[:, 0]],
                     np.cross(X[T[:, 2]] - X[T[:, 0]], X[T[:, 3]] - X[T[:, 0]])) / 6


def test_cube_sizes():
    m, ind = W.cube_sphere()
    assert (m.n_tets, m.n_nodes, len(m.fixed_nodes)) == (3072, 729, 81)
    assert np.all(_vols(m) > 0)
    _, c = _faces(m.tets)
    assert c.max() == 2
    np.testing.assert_allclose(ind.origin, [0.5, 0.5, 1.3])
    assert ind.n_steps == 10 and ind.depth_schedule[-1] == pytest.approx(0.05)


def test_fingertip_mesh():
    m, ind = W.fingertip_sphere()
    assert 8000 < m.n_nodes < 10000 and 35000 < m.n_tets < 45000
    v = _vols(m)
    assert v.min() > 0
    _, c = _faces(m.tets)
    assert c.max() == 2                                   # conforming
    ns = m.meta["n_surface"]
    n, mm = m.meta["n_cap"], m.meta["m_axial"]
    assert ns == 4 * n * (mm + 1) + (n + 1) ** 2 + (n // 2 - 1) * 4 * n
    quads = 4 * n * mm + 3 * n * n
    assert np.count_nonzero(c == 1) == 2 * (2 * quads) + 2 * 4 * n * 3   # outer+core+base rim
    # volume of the faceted shell below the smooth one, within 1%
    R, Lc = 7.0, 33.0
    exact = math.pi * (R**2 - 4**2) * Lc + 2 / 3 * math.pi * (R**3 - 4**3)
    assert abs(v.sum() / exact - 1) < 1e-2
    # fixed = innermost layer at radius 4
    Xf = m.nodes[m.fixed_nodes]
    rad = np.where(Xf[:, 2] <= Lc, np.hypot(Xf[:, 0], Xf[:, 1]),
                   np.linalg.norm(Xf - [0, 0, Lc], axis=1))
    np.testing.assert_allclose(rad, 4.0, atol=1e-9)
    assert set(np.unique(m.tet_material)) == {0, 1}
    assert W.fingertip_tet_count(7.0, 40.0, 0.88) == m.n_tets


def test_fingertip_indenter_touches_first_node():
    m, ind = W.fingertip_sphere()
    X = m.nodes[: m.meta["n_surface"]]
    t = W.entry_times(ind, X)
    assert abs(t.min()) < 1e-12
    d = np.linalg.norm(X - ind.origin, axis=1)
    assert d.min() == pytest.approx(4.0, abs=1e-9)
    assert ind.n_steps == 20 and ind.depth_schedule[-1] == pytest.approx(2.0)


def test_draws_are_seeded_and_touch():
    m = W.fingertip_mesh()
    a = W.draw_indentations(m, 12, seed=5)
    b = W.draw_indentations(m, 12, seed=5)
    for x, y in zip(a, b):
        assert x.shape == y.shape
        np.testing.assert_array_equal(x.pose, y.pose)
    X = m.nodes[: m.meta["n_surface"]]
    for ind in a:
        assert abs(W.entry_times(ind, X).min()) < 1e-9
        R = ind.rotation
        np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-12)
        assert np.linalg.det(R) == pytest.approx(1.0)
        assert 0.5 <= ind.depth_schedule[-1] <= 3.0
    assert {ind.shape for ind in W.draw_indentations(m, 30, seed=9)} == {0, 1, 2}


def test_uneven_sizes_log_uniform():
    sizes = [s[2] for s in W.uneven_fingertips(64, build=False)]
    assert min(sizes) > 3e3 and max(sizes) < 3e5
