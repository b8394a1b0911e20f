"""Pins for oracle/contact.py: constructed points at known distance, brute-force
surface sampling for the box, eikonal property and finite differences."""
import numpy as np
import pytest

from oracle import contact as C

RNG = np.random.default_rng(11)


def _rot():
    q, _ = np.linalg.qr(RNG.standard_normal((3, 3)))
    return q * np.sign(np.linalg.det(q))


def _fd_check(shape, origin, R, params, x):
    phi, g, H = C.sdf(shape, origin, R, params, x)
    eps = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = eps
        pp, gp, _ = C.sdf(shape, origin, R, params, x + e)
        pm, gm, _ = C.sdf(shape, origin, R, params, x - e)
        np.testing.assert_allclose((pp - pm) / (2 * eps), g[:, k], atol=1e-7)
        np.testing.assert_allclose((gp - gm) / (2 * eps), H[:, :, k], atol=2e-5)
    np.testing.assert_allclose(np.linalg.norm(g, axis=1), 1.0, atol=1e-12)


def test_sphere_known_distances():
    c = np.array([0.3, -0.2, 1.0])
    dirs = RNG.standard_normal((20, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    s = RNG.uniform(0.1, 2.0, 20)
    x = c + s[:, None] * dirs
    phi, g, _ = C.sdf(C.SPHERE, c, np.eye(3), [0.7, 0, 0], x)
    np.testing.assert_allclose(phi, s - 0.7, atol=1e-14)
    np.testing.assert_allclose(g, dirs, atol=1e-14)
    _fd_check(C.SPHERE, c, np.eye(3), [0.7, 0, 0], x)


def test_cylinder_known_distances():
    R = _rot()
    c = np.array([1.0, 2.0, -1.0])
    ax, p1, p2 = R[:, 2], R[:, 0], R[:, 1]
    t = RNG.uniform(-5, 5, 20)
    ang = RNG.uniform(0, 2 * np.pi, 20)
    rho = RNG.uniform(0.2, 3.0, 20)
    radial = np.cos(ang)[:, None] * p1 + np.sin(ang)[:, None] * p2
    x = c + t[:, None] * ax + rho[:, None] * radial
    phi, g, _ = C.sdf(C.CYLINDER, c, R, [1.1, 0, 0], x)
    np.testing.assert_allclose(phi, rho - 1.1, atol=1e-13)
    np.testing.assert_allclose(g, radial, atol=1e-12)
    _fd_check(C.CYLINDER, c, R, [1.1, 0, 0], x)


def test_box_against_surface_sampling():
    """Unsigned distance to a densely sampled box surface, sign from containment."""
    R = _rot()
    c = np.array([0.1, 0.2, 0.3])
    h = np.array([0.5, 0.3, 0.8])
    n = 120
    u = np.linspace(-1, 1, n)
    U, V = np.meshgrid(u, u, indexing="ij")
    pts = []
    for ax in range(3):
        o = [a for a in range(3) if a != ax]
        for sgn in (-1, 1):
            p = np.zeros((n * n, 3))
            p[:, ax] = sgn * h[ax]
            p[:, o[0]] = U.ravel() * h[o[0]]
            p[:, o[1]] = V.ravel() * h[o[1]]
            pts.append(p)
    surf_local = np.concatenate(pts)
    x_local = RNG.uniform(-1.5, 1.5, (40, 3)) * h
    x = c + x_local @ R.T
    phi, _, _ = C.sdf(C.BOX, c, R, h, x)
    dist = np.min(np.linalg.norm(x_local[:, None, :] - surf_local[None], axis=2), axis=1)
    inside = np.all(np.abs(x_local) < h, axis=1)
    ref = np.where(inside, -dist, dist)
    spacing = 2 * h.max() / (n - 1)
    np.testing.assert_allclose(phi, ref, atol=spacing)


def test_box_derivatives_off_kinks():
    R = _rot()
    c = np.zeros(3)
    h = np.array([0.5, 0.3, 0.8])
    # points outside near a face, an edge and a corner, and inside near a face
    loc = np.array([[0.9, 0.0, 0.1], [0.7, 0.5, 0.2], [0.7, 0.6, 1.0], [0.0, 0.1, 0.7],
                    [0.45, -0.1, 0.2]])
    _fd_check(C.BOX, c, R, h, loc @ R.T)


def test_plane():
    R = _rot()
    c = np.array([0.0, 0.0, 1.0])
    x = RNG.standard_normal((10, 3))
    phi, g, H = C.sdf(C.PLANE, c, R, [0, 0, 0], x)
    np.testing.assert_allclose(phi, (x - c) @ R[:, 2], atol=1e-14)
    assert np.abs(H).max() == 0


def test_penalty_consistency():
    c = np.array([0.0, 0.0, 0.0])
    x = RNG.uniform(-1, 1, (30, 3))
    k = RNG.uniform(0.5, 2.0, 30)
    k[::7] = 0.0
    e, g, Hx, gn, act = C.penalty(C.SPHERE, c, np.eye(3), [0.8, 0, 0], x, k)
    phi, n, _ = C.sdf(C.SPHERE, c, np.eye(3), [0.8, 0, 0], x)
    assert np.array_equal(act, (phi < 0) & (k > 0))
    assert np.all(e[~act] == 0) and np.all(g[~act] == 0)
    eps = 1e-6
    for d in range(3):
        dx = np.zeros(3)
        dx[d] = eps
        ep = C.penalty(C.SPHERE, c, np.eye(3), [0.8, 0, 0], x + dx, k)
        em = C.penalty(C.SPHERE, c, np.eye(3), [0.8, 0, 0], x - dx, k)
        np.testing.assert_allclose((ep[0] - em[0]) / (2 * eps), g[:, d], atol=1e-7)
        np.testing.assert_allclose((ep[1] - em[1]) / (2 * eps), Hx[:, :, d], atol=1e-5)
    np.testing.assert_allclose(gn, (k * act)[:, None, None] * np.einsum("ni,nj->nij", n, n))
