"""Pins for oracle/solver.py: finite differences of the assembled energy,
frame invariance, the linear patch test, the uniaxial closed form at small and
large strain, global force and moment balance, Hertz (loose) and brute-force
minimisation on tiny meshes."""
import math

import numpy as np
import pytest
from scipy.optimize import minimize

import workloads as W
from oracle import Problem
from tests.closed_forms import hertz_force, uniaxial_plane

RNG = np.random.default_rng(3)


def _far_sphere():
    ind = W.cube_sphere_indenter()
    ind.origin = np.array([50.0, 50.0, 50.0])
    return ind


@pytest.fixture(scope="module")
def cube3():
    m = W.cube_mesh(3)
    X = m.nodes.copy()
    interior = np.all((X > 1e-9) & (X < 1 - 1e-9), axis=1)
    X[interior] += RNG.uniform(-0.08, 0.08, (interior.sum(), 3))   # unstructured interior
    m.nodes = X
    return m


def test_gradient_and_tangent_match_finite_differences(cube3):
    ind = W.cube_sphere_indenter(radius=0.4, depth=0.1, n_steps=1)
    p = Problem(cube3, ind)
    u = 0.03 * RNG.standard_normal((p.n, 3))
    u[p.fixed] = 0.0
    step = 1
    g, _ = p.gradient(u, step)
    assert np.count_nonzero(p.contact_terms(u, step)[4]) > 0     # some contact active
    eps = 1e-7
    for idx in RNG.choice(3 * p.n, 25, replace=False):
        du = np.zeros(3 * p.n)
        du[idx] = eps
        du = du.reshape(-1, 3)
        fd = (p.energy(u + du, step)[0] - p.energy(u - du, step)[0]) / (2 * eps)
        assert fd == pytest.approx(g.ravel()[idx], rel=1e-6, abs=1e-6 * np.abs(g).max())
    K = p.hessian(u, step)
    v = RNG.standard_normal((p.n, 3))
    h = 1e-6
    fd = (p.gradient(u + h * v, step)[0] - p.gradient(u - h * v, step)[0]) / (2 * h)
    np.testing.assert_allclose(K @ v.ravel(), fd.ravel(), rtol=1e-5, atol=1e-5 * np.abs(fd).max())
    assert abs(K - K.T).max() < 1e-8 * abs(K).max()


def test_rigid_motion_is_force_free(cube3):
    p = Problem(cube3, _far_sphere())
    q, _ = np.linalg.qr(RNG.standard_normal((3, 3)))
    Q = q * np.sign(np.linalg.det(q))
    u = p.X @ Q.T - p.X + np.array([0.3, -1.0, 2.0])
    e, _ = p.elastic_energy(u)
    g = p.elastic_gradient(u)
    ref = np.abs(p.elastic_gradient(0.01 * p.X)).max()         # 1% strain for scale
    assert abs(e) < 1e-10
    assert np.abs(g).max() < 1e-12 * ref * 1e4


def test_linear_patch_test(cube3):
    """All boundary nodes follow an affine map; the interior must follow it too."""
    m = cube3
    X = m.nodes
    bnd = np.nonzero(np.any((X < 1e-9) | (X > 1 - 1e-9), axis=1))[0].astype(np.int32)
    A = np.array([[0.04, 0.01, -0.02], [0.0, -0.03, 0.02], [0.01, 0.02, 0.05]])
    t = np.array([0.01, -0.02, 0.03])
    m2 = W.Mesh(X, m.tets, m.tet_material, m.materials, bnd, None)
    vals = X[bnd] @ A.T + t
    ind = _far_sphere()
    ind.depth_schedule = np.array([0.0, 0.0])
    p = Problem(m2, ind, dirichlet_values=vals)
    r = p.solve(tol=1e-10)
    assert r.converged
    np.testing.assert_allclose(r.u, X @ A.T + t, atol=1e-12)


def _uniaxial(strain, c_kappa):
    m = W.cube_mesh(4, E=1e6, nu=0.3, fix="rollers")
    p = Problem(m, W.plane_indenter(1.0, strain, 4), c_kappa=c_kappa)
    # the penalty has an FP64 floor of about c_kappa*E*eps_mach/(P h_bar) relative
    r = p.solve(tol=1e-9)
    assert r.converged
    return m, p, r


@pytest.mark.parametrize("strain", [0.01, 0.2])
def test_uniaxial_plane_closed_form(strain):
    """Rollers + frictionless plane: homogeneous state, closed form exact up to
    the O(1/c_kappa) penalty effect at the top edges (whose lumped area also
    counts side faces). Direct check at c_kappa = 1e3, then a Richardson
    extrapolation in 1/c_kappa checked against the rigid (gap-free) limit."""
    E, nu = 1e6, 0.3
    m, p, r1 = _uniaxial(strain, 1e3)
    X = m.nodes
    lz, lt, pzz = uniaxial_plane(strain, E, nu, p.h_bar, 1e3)
    np.testing.assert_allclose(r1.u[:, 2], (lz - 1) * X[:, 2], atol=5e-4 * strain)
    np.testing.assert_allclose(r1.u[:, 0], (lt - 1) * X[:, 0], atol=5e-4 * strain)
    assert r1.step_force[-1, 2] == pytest.approx(pzz, rel=5e-4)
    _, _, r2 = _uniaxial(strain, 2e3)
    u = 2 * r2.u - r1.u
    f = 2 * r2.step_force[-1, 2] - r1.step_force[-1, 2]
    lz, lt, pzz = uniaxial_plane(strain, E, nu, p.h_bar, np.inf)
    np.testing.assert_allclose(u[:, 2], (lz - 1) * X[:, 2], atol=1e-6 * strain)
    np.testing.assert_allclose(u[:, 0], (lt - 1) * X[:, 0], atol=1e-6 * strain)
    np.testing.assert_allclose(u[:, 1], (lt - 1) * X[:, 1], atol=1e-6 * strain)
    assert f == pytest.approx(pzz, rel=1e-6)


def test_uniaxial_closed_form_small_strain_limit():
    """sigma -> E eps and lateral strain -> -nu eps as eps -> 0."""
    E, nu = 1e6, 0.3
    eps = 1e-5
    lz, lt, pzz = uniaxial_plane(eps, E, nu, 0.1, 1e12)
    assert (lz - 1) == pytest.approx(-eps, rel=1e-6)
    assert pzz / (lz - 1) == pytest.approx(E, rel=1e-4)
    assert -(lt - 1) / (lz - 1) == pytest.approx(nu, rel=1e-4)
    lz, lt, pzz = uniaxial_plane(0.01, E, nu, 0.1, 1e12)
    assert lt - 1 == pytest.approx(0.003016, abs=2e-6)
    assert pzz == pytest.approx(-10078, abs=2)


@pytest.fixture(scope="module")
def cube_sphere_solution():
    m, ind = W.cube_sphere()
    p = Problem(m, ind)
    return p, p.solve()


def test_cube_sphere_equilibrium(cube_sphere_solution):
    p, r = cube_sphere_solution
    assert r.converged
    assert np.all(r.residual <= 1e-10 * r.scale)
    fc = r.nodal_contact.sum(axis=0)
    react = r.reactions.sum(axis=0)
    np.testing.assert_allclose(fc + react, 0.0, atol=1e-8 * np.linalg.norm(fc))
    x = p.X + r.u
    moment = np.cross(x, r.nodal_contact + r.reactions).sum(axis=0)
    assert np.linalg.norm(moment) < 1e-8 * np.linalg.norm(fc)
    # frictionless sphere over the centre: mostly vertical (the Kuhn split is
    # not mirror symmetric, so a small lateral part remains)
    assert abs(fc[0]) < 1e-2 * abs(fc[2]) and abs(fc[1]) < 1e-2 * abs(fc[2])


def test_cube_sphere_hertz_loose(cube_sphere_solution):
    p, r = cube_sphere_solution
    d = p.depths
    F = -r.step_force[:, 2]
    FH = hertz_force(1e6, 0.3, 0.3, d)
    assert F[-1] == pytest.approx(FH[-1], rel=0.25)
    slope = np.polyfit(np.log(d[4:]), np.log(F[4:]), 1)[0]
    assert 1.35 <= slope <= 1.65


def test_brute_force_single_tet_under_plane():
    """One tet, base fixed, apex pushed by a plane: generic minimiser vs Newton."""
    nodes = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0.3, 0.25, 0.9]], dtype=float)
    m = W.Mesh(nodes, np.array([[0, 1, 2, 3]], dtype=np.int32), np.zeros(1, dtype=np.int32),
               np.array([[1000.0, 0.3]]), np.array([0, 1, 2], dtype=np.int32))
    ind = W.plane_indenter(0.9, 0.2, 3)
    p = Problem(m, ind, c_kappa=50.0)
    r = p.solve(tol=1e-12)
    assert r.converged

    def f(v):
        u = np.zeros((4, 3))
        u[3] = v
        e, minJ = p.energy(u, p.K)
        return e if minJ > 0 else 1e30
    best = minimize(f, np.zeros(3), method="Nelder-Mead",
                    options=dict(xatol=1e-12, fatol=1e-16, maxiter=40000, maxfev=40000))
    np.testing.assert_allclose(r.u[3], best.x, atol=2e-6)


def test_brute_force_one_hex_under_sphere():
    m = W.cube_mesh(1, E=500.0, nu=0.35)
    ind = W.cube_sphere_indenter(radius=0.9, depth=0.12, n_steps=3)
    ind.origin = np.array([0.45, 0.4, 2.5])
    ind = W.place_at_contact(ind, m.nodes)
    p = Problem(m, ind, c_kappa=20.0)
    r = p.solve(tol=1e-12)
    assert r.converged
    free = ~p.fixed

    def f(v):
        u = np.zeros((p.n, 3))
        u[free] = v
        e, minJ = p.energy(u, p.K)
        return e if minJ > 0 else 1e30

    def grad(v):
        u = np.zeros((p.n, 3))
        u[free] = v
        return p.gradient(u, p.K)[0][free]
    best = minimize(f, np.zeros(free.sum()), jac=grad, method="BFGS",
                    options=dict(gtol=1e-12, maxiter=10000))
    np.testing.assert_allclose(r.u[free], best.x, atol=1e-7)


def test_newton_converges_quadratically_near_solution(cube_sphere_solution):
    """Restart the last step from a perturbed solution: residual ratios shrink
    like |R_k+1| ~ C |R_k|^2 once close (exact tangent)."""
    p, r = cube_sphere_solution
    u = r.u + 1e-5 * RNG.standard_normal(r.u.shape) * (~p.fixed)
    norms = []
    for _ in range(4):
        g, _ = p.gradient(u, p.K)
        gf = g.ravel()[p.free]
        norms.append(np.linalg.norm(gf))
        d, proj = p._direction(u, p.K, gf)
        du = np.zeros(3 * p.n)
        du[p.free] = d
        u = u + du.reshape(-1, 3)
    # 420 -> 3e-2 -> 2e-7 -> roundoff: each step squares the relative error
    assert norms[1] < 1e-3 * norms[0] and norms[2] < 1e-4 * norms[1], norms
