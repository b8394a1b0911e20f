"""Pins for the oracle's lagged, smoothed Coulomb friction (the paper's contact
model is isotropic Coulomb, Sec. III-A; reading in oracle/solver.py).

  - the smoothed magnitude f0: value and slope continuous at the smoothing slip,
    slope 0 at rest and 1 in sliding;
  - finite differences: potential -> force -> Hessian; the Hessian is PSD;
  - the force is tangent to the contact, opposes the slip, and equals mu fn in
    sliding (Coulomb's law), less below the smoothing slip;
  - a plane dragged across a block: once every contact node slides, the
    tangential resultant equals mu times the normal resultant of the previous
    step (the lagged normal force), exactly;
  - with a large coefficient the contact nodes stick to the moving plane;
  - re-solving each step with the normal forces refreshed at its own end state
    (friction passes) converges to Coulomb's law with the step's own normal
    forces: the per-node mismatch contracts pass by pass;
  - mu_f = 0 is the frictionless solve."""
import numpy as np
import pytest

import workloads as W
from oracle import Problem, contact

RNG = np.random.default_rng(41)


def test_f0_is_c1_with_unit_sliding_slope():
    eps = 0.3
    h = 1e-7
    f = lambda y: contact.friction_f0(y, eps)   # noqa: E731
    assert f(0.0) == pytest.approx(eps / 3)
    assert f(eps - 1e-12) == pytest.approx(f(eps + 1e-12), abs=1e-11)
    slope = lambda y: (f(y + h) - f(y - h)) / (2 * h)   # noqa: E731
    assert slope(eps - 1e-5) == pytest.approx(1.0, abs=1e-4)
    assert slope(eps + 1e-5) == pytest.approx(1.0, abs=1e-6)
    assert slope(2 * h) == pytest.approx(0.0, abs=1e-5)
    ys = np.linspace(0, 2 * eps, 101)[1:-1]
    s = np.array([slope(y) for y in ys])
    assert np.all(np.diff(s) >= -1e-6) and s.max() <= 1 + 1e-6


def _random_state(n=12, eps=0.05):
    n_ = RNG.standard_normal((n, 3))
    n_ /= np.linalg.norm(n_, axis=1)[:, None]
    x0 = RNG.standard_normal((n, 3))
    dc = RNG.standard_normal(3) * 0.05
    fn = RNG.uniform(0.0, 2.0, n)
    fn[:2] = 0.0
    # half the nodes below the smoothing slip, half above
    x = x0 + dc + RNG.standard_normal((n, 3)) * np.where(np.arange(n) % 2 == 0, 0.2 * eps, 4 * eps)[:, None]
    return x, x0, dc, n_, fn


def test_friction_derivatives_and_psd():
    mu, eps = 0.783, 0.05
    x, x0, dc, nrm, fn = _random_state(eps=eps)
    e, g, H = contact.friction(x, x0, dc, nrm, fn, mu, eps)
    h = 1e-7
    for i in range(len(x)):
        for k in range(3):
            d = np.zeros_like(x)
            d[i, k] = h
            fd = (contact.friction(x + d, x0, dc, nrm, fn, mu, eps)[0].sum()
                  - contact.friction(x - d, x0, dc, nrm, fn, mu, eps)[0].sum()) / (2 * h)
            assert fd == pytest.approx(g[i, k], rel=1e-6, abs=1e-7)
            fdg = (contact.friction(x + d, x0, dc, nrm, fn, mu, eps)[1][i]
                   - contact.friction(x - d, x0, dc, nrm, fn, mu, eps)[1][i]) / (2 * h)
            np.testing.assert_allclose(H[i][:, k], fdg, rtol=1e-5, atol=1e-5 * np.abs(H).max())
    w = np.linalg.eigvalsh(H)
    assert w.min() >= -1e-12 * np.abs(w).max()


def test_coulomb_law_direction_and_magnitude():
    mu, eps = 0.6, 0.05
    x, x0, dc, nrm, fn = _random_state(eps=eps)
    _, g, _ = contact.friction(x, x0, dc, nrm, fn, mu, eps)
    r = x - x0 - dc
    s = r - np.einsum("ni,ni->n", nrm, r)[:, None] * nrm
    y = np.linalg.norm(s, axis=1)
    force = -g                                     # friction force on the node
    np.testing.assert_allclose(np.einsum("ni,ni->n", force, nrm), 0.0, atol=1e-12)
    assert np.all(np.einsum("ni,ni->n", force, s) <= 1e-15)          # opposes the slip
    mag = np.linalg.norm(force, axis=1)
    slide = (y >= eps) & (fn > 0)
    stick = (y < eps) & (fn > 0)
    assert slide.any() and stick.any()
    np.testing.assert_allclose(mag[slide], mu * fn[slide], rtol=1e-12)
    assert np.all(mag[stick] < mu * fn[stick])
    assert np.all(mag[fn == 0] == 0.0)


def _dragged_plane(mu_f, n_steps=8, tilt=0.05, depth=0.2):
    """Cube (bottom fixed) under a rigid plane moving along a = (1, 0, -tilt)
    (normalised): it presses and drags at the same time."""
    m = W.cube_mesh(3, E=1.0e3, nu=0.3)
    ind = W.plane_indenter(1.0, depth, n_steps)
    a = np.array([1.0, 0.0, -tilt])
    ind.direction = a / np.linalg.norm(a)
    return m, ind, Problem(m, ind, mu_f=mu_f)


def test_dragged_plane_tangential_force_is_mu_times_lagged_normal_force():
    mu = 0.783
    m, ind, p = _dragged_plane(mu)
    r = p.solve(tol=1e-10)
    assert r.converged
    Fz = r.step_force[:, 2]                       # normal: plane normal is -z
    Fx = r.step_force[:, 0]
    assert np.all(Fz < 0) and np.all(Fx[1:] > 0)  # pushed down, dragged along +x
    assert Fx[0] == 0.0                           # no normal force yet at the start of step 1
    # the resultant is slightly below mu |Fz| where slips are not all parallel
    np.testing.assert_allclose(Fx[1:], mu * np.abs(Fz[:-1]), rtol=1e-3)
    assert np.all(Fx[1:] <= mu * np.abs(Fz[:-1]))
    # every contact node slides at the last step (premise of the exact law)
    p.set_friction_lag(r.step_u[-2], p.K)
    f = p.fric
    rr = (m.nodes + r.u) - f["x_start"] - f["dc"]
    s = rr - np.einsum("ni,ni->n", f["normal"], rr)[:, None] * f["normal"]
    y = np.linalg.norm(s, axis=1)
    assert np.all(y[f["fn"] > 0] >= p.fric_eps)
    # Coulomb per node: the tangential nodal forces of the last step sum in
    # magnitude to mu times the lagged normal forces, which sum to |Fz| of the
    # step before
    ft = np.linalg.norm(r.nodal_contact[:, :2], axis=1)
    assert ft.sum() == pytest.approx(mu * abs(Fz[-2]), rel=1e-9)
    np.testing.assert_allclose(ft, mu * f["fn"], rtol=1e-9, atol=1e-12 * ft.max())
    p.fric = None


def test_large_coefficient_sticks_contact_nodes_to_the_plane():
    m, ind, p = _dragged_plane(50.0, n_steps=4, tilt=0.2, depth=0.05)
    r = p.solve(tol=1e-10)
    assert r.converged
    # nodes pressed at the end of step 1 stick from step 2 on (step 1 itself
    # starts without normal force, hence without friction)
    p.set_friction_lag(r.step_u[0], 2)
    inside = p.fric["fn"] > 0
    assert inside.sum() >= 9
    ux_plane = (ind.depth_schedule[-1] - ind.depth_schedule[0]) * ind.direction[0]
    np.testing.assert_allclose(r.u[inside, 0] - r.step_u[0][inside, 0], ux_plane, atol=2 * p.fric_eps)
    p.fric = None


def _current_state_mismatch(p, r, mu):
    """max_i | |f_t,i| - mu fn_i(u_end) | / max |f_t|: Coulomb's law with the
    normal forces of the converged end state, indenter at the last pose."""
    p.set_friction_lag(r.step_u[-2], p.K)
    p.refresh_friction(r.u, p.K)
    ft = np.linalg.norm(r.nodal_contact[:, :2], axis=1)
    out = float(np.abs(ft - mu * p.fric["fn"]).max() / ft.max())
    p.fric = None
    return out


def test_friction_passes_converge_to_the_current_normal_forces():
    mu = 0.783
    m, ind, _ = _dragged_plane(mu)
    errs, fx = [], []
    for passes in (1, 3, 8):
        p = Problem(m, ind, mu_f=mu, friction_passes=passes)
        r = p.solve(tol=1e-10)
        assert r.converged
        errs.append(_current_state_mismatch(p, r, mu))
        fx.append(r.step_force[-1, 0])
        if passes == 1:
            it1 = r.newton_iters.copy()
        else:
            # every pass after the first costs at least one Newton iteration
            assert np.all(r.newton_iters[1:] > it1[1:])
    assert errs[0] > 0.1 and errs[1] < 0.25 * errs[0] and errs[2] < 1e-3
    # the lagged normal force trails the load: refreshed, the drag grows
    assert fx[0] < fx[1] < fx[2]


def test_zero_coefficient_is_frictionless():
    m, ind, p = _dragged_plane(0.0, n_steps=4)
    r0 = p.solve(tol=1e-10)
    r1 = Problem(m, ind).solve(tol=1e-10)
    np.testing.assert_array_equal(r0.u, r1.u)
    assert np.all(np.abs(r0.step_force[:, 0]) < 1e-9 * np.abs(r0.step_force[:, 2]).max())
