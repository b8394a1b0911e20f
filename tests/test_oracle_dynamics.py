"""Pins for the oracle's dynamic stepping (backward Euler, lumped mass;
Sec. III-A: implicit time integration with a 1e-4 s step).

Each pin is fixed by mechanics, not by the oracle's own formulas:
  - total lumped mass = density * volume of the cube (closed form);
  - a free body given a uniform velocity translates rigidly, u_k = k dt v0;
  - a free body conserves linear momentum, and its centre of mass moves
    uniformly;
  - the angular-momentum identity of backward Euler for a free spinning body
    (internal forces of a frame-invariant energy exert no torque);
  - momentum balance under contact: sum m (v_k - v_{k-1}) / dt equals the
    resultant contact force;
  - the apex of one tet, free along z only, follows the textbook backward-Euler
    recurrence of a linear oscillator at small amplitude;
  - density -> 0 recovers the quasi-static solution;
  - finite differences of the incremental potential."""
import numpy as np
import pytest

import workloads as W
from oracle import Problem

RNG = np.random.default_rng(11)


def _far_plane(n_steps):
    return W.plane_indenter(50.0, 0.0, n_steps)


def _momentum(p, v):
    return (p.mass[:, None] * v).sum(axis=0)


def test_total_lumped_mass_is_density_times_volume():
    m = W.cube_mesh(3, length=2.0)
    X = m.nodes.copy()
    interior = np.all((X > 1e-9) & (X < 2 - 1e-9), axis=1)
    X[interior] += RNG.uniform(-0.1, 0.1, (interior.sum(), 3))
    m.nodes = X
    rho = 3.7
    p = Problem(m, _far_plane(1), dt=1e-3, density=rho)
    assert p.mass.sum() == pytest.approx(rho * 8.0, rel=1e-13)
    assert np.all(p.mass > 0)


def test_free_body_uniform_velocity_translates_rigidly():
    m = W.cube_mesh(2, fix="none")
    dt, K = 1e-3, 6
    v0 = np.tile(np.array([0.3, -0.2, 0.5]), (m.n_nodes, 1))
    p = Problem(m, _far_plane(K), dt=dt, density=2.0)
    r = p.solve(tol=1e-12, v0=v0)
    assert r.converged
    for k, uk in enumerate(r.step_u, start=1):
        np.testing.assert_allclose(uk, k * dt * v0, rtol=1e-10, atol=1e-14)


def test_free_body_conserves_linear_momentum():
    m = W.cube_mesh(2, fix="none")
    dt, K = 1e-3, 8
    v0 = 0.5 * RNG.standard_normal((m.n_nodes, 3))
    p = Problem(m, _far_plane(K), dt=dt, density=1.0)
    r = p.solve(tol=1e-12, v0=v0)
    assert r.converged
    P0 = _momentum(p, v0)
    for k, (uk, vk) in enumerate(zip(r.step_u, p.step_v), start=1):
        np.testing.assert_allclose(_momentum(p, vk), P0, rtol=0, atol=1e-9 * np.abs(P0).max())
        cm = (p.mass[:, None] * uk).sum(axis=0)
        np.testing.assert_allclose(cm, k * dt * P0, rtol=0, atol=1e-11)
    # the body deforms (non-uniform start), so elastic forces did act
    assert np.linalg.norm(r.u - r.u.mean(axis=0)) > 1e-5


def test_free_spinning_body_angular_momentum_identity():
    """x_k = X + u_k, v_k = (u_k - u_{k-1}) / dt. With m (v_k - v_{k-1}) / dt =
    -grad E(x_k) and sum x_k x grad E(x_k) = 0 for a rotation-invariant E,
    L_k - L_{k-1} = dt sum m v_k x v_{k-1}, L = sum m x x v."""
    m = W.cube_mesh(2, fix="none")
    dt, K = 2e-3, 10
    c = m.nodes.mean(axis=0)
    omega = np.array([0.4, -1.0, 3.0])
    v0 = np.cross(omega, m.nodes - c)
    p = Problem(m, _far_plane(K), dt=dt, density=1.0)
    r = p.solve(tol=1e-12, v0=v0)
    assert r.converged
    x_prev, v_prev = m.nodes.copy(), v0
    L_prev = (p.mass[:, None] * np.cross(x_prev, v_prev)).sum(axis=0)
    for uk, vk in zip(r.step_u, p.step_v):
        x = m.nodes + uk
        L = (p.mass[:, None] * np.cross(x, vk)).sum(axis=0)
        rhs = dt * (p.mass[:, None] * np.cross(vk, v_prev)).sum(axis=0)
        np.testing.assert_allclose(L - L_prev, rhs, rtol=0, atol=1e-9 * np.abs(L).max())
        L_prev, v_prev = L, vk
    # backward Euler dissipates: kinetic energy of the spin falls
    ke0 = 0.5 * (p.mass * (v0 ** 2).sum(axis=1)).sum()
    ke = 0.5 * (p.mass * (p.step_v[-1] ** 2).sum(axis=1)).sum()
    assert ke < ke0


def test_momentum_balance_under_contact():
    m = W.cube_mesh(3, fix="none")
    ind = W.place_at_contact(W.cube_sphere_indenter(radius=0.3, depth=0.04, n_steps=4), m.nodes)
    dt = 1e-3
    p = Problem(m, ind, dt=dt, density=1.0)
    r = p.solve(tol=1e-10)      # FP64 rounding floor of this residual: ~5e-12 * scale
    assert r.converged
    v_prev = np.zeros((p.n, 3))
    for k, vk in enumerate(p.step_v):
        lhs = _momentum(p, vk - v_prev) / dt
        f = r.step_force[k]
        assert np.linalg.norm(f) > 0
        np.testing.assert_allclose(lhs, f, rtol=0, atol=1e-8 * np.linalg.norm(f))
        v_prev = vk
    assert r.step_force[-1][2] < 0      # the sphere pushes the body down


def test_single_tet_apex_follows_linear_backward_euler():
    """Apex free along z only: a one-DOF oscillator m z'' = -k z. Backward
    Euler gives z_{n+1} = (z_n + dt v_n) / (1 + w^2 dt^2), v_{n+1} = (z_{n+1}
    - z_n) / dt, w^2 = k / m, k the linear stiffness at rest."""
    nodes = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0.3, 0.25, 0.9]], dtype=float)
    m = W.Mesh(nodes, np.array([[0, 1, 2, 3]], dtype=np.int32), np.zeros(1, dtype=np.int32),
               np.array([[1000.0, 0.3]]), np.array([0, 1, 2, 3], dtype=np.int32),
               np.array([7, 7, 7, 3], dtype=np.uint8))
    dt, K, rho = 0.01, 30, 1.0
    p = Problem(m, _far_plane(K), dt=dt, density=rho)
    k = p.hessian(np.zeros((4, 3)), 1)[11, 11]
    mass = p.mass[3]
    assert mass == pytest.approx(rho * 0.9 / 6.0 / 4.0, rel=1e-13)
    w2 = k / mass
    assert 0.2 < np.sqrt(w2) * dt < 2.0       # a step where backward Euler damps visibly
    v0 = np.zeros((4, 3))
    v0[3, 2] = 1e-4
    r = p.solve(tol=1e-13, v0=v0)
    assert r.converged
    z, v = 0.0, 1e-4
    ref = []
    for _ in range(K):
        zn = (z + dt * v) / (1.0 + w2 * dt * dt)
        v = (zn - z) / dt
        z = zn
        ref.append(z)
    got = np.array([uk[3, 2] for uk in r.step_u])
    ref = np.array(ref)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-4 * np.abs(ref).max())
    assert np.all(np.abs(np.array([uk[3, :2] for uk in r.step_u])) == 0.0)
    assert abs(ref[-1]) < 0.5 * np.abs(ref).max()   # the amplitude decays


def test_vanishing_density_recovers_quasi_static():
    m = W.cube_mesh(3)
    ind = W.place_at_contact(W.cube_sphere_indenter(radius=0.3, depth=0.04, n_steps=4), m.nodes)
    qs = Problem(m, ind).solve(tol=1e-12)
    dyn = Problem(m, ind, dt=1e-4, density=1e-16).solve(tol=1e-12)
    assert qs.converged and dyn.converged
    assert np.linalg.norm(dyn.u - qs.u) <= 1e-8 * np.linalg.norm(qs.u)
    np.testing.assert_allclose(dyn.step_force, qs.step_force, rtol=1e-7)


def test_incremental_potential_finite_differences():
    m = W.cube_mesh(2)
    ind = W.place_at_contact(W.cube_sphere_indenter(radius=0.4, depth=0.1, n_steps=1), m.nodes)
    p = Problem(m, ind, dt=1e-3, density=50.0)
    u = 0.02 * RNG.standard_normal((p.n, 3))
    u[p.fixed] = 0.0
    p.u_tilde = u + 0.01 * RNG.standard_normal((p.n, 3))
    e_in, g_in, _ = p.inertia_terms(u)
    assert e_in > 0 and np.all(g_in[p.fixed] == 0.0)
    g, _ = p.gradient(u, 1)
    eps = 1e-7
    for idx in RNG.choice(3 * p.n, 20, replace=False):
        du = np.zeros(3 * p.n)
        du[idx] = eps
        du = du.reshape(-1, 3)
        fd = (p.energy(u + du, 1)[0] - p.energy(u - du, 1)[0]) / (2 * eps)
        if p.fixed.ravel()[idx]:
            continue
        assert fd == pytest.approx(g.ravel()[idx], rel=1e-6, abs=1e-6 * np.abs(g).max())
    H = p.hessian(u, 1)
    v = RNG.standard_normal((p.n, 3)) * ~p.fixed
    h = 1e-6
    fd = (p.gradient(u + h * v, 1)[0] - p.gradient(u - h * v, 1)[0]) / (2 * h)
    np.testing.assert_allclose(H @ v.ravel(), fd.ravel(), rtol=1e-5, atol=1e-5 * np.abs(fd).max())
    p.u_tilde = None
