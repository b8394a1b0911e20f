"""GPU parity of the lagged, smoothed Coulomb friction (the paper's contact
model is isotropic Coulomb, Sec. III-A) against the FP64 oracle, through the
C ABI: a plane dragged across a cube (sliding), the stick limit, the batched
engines, friction passes, and Coulomb's law checked on the GPU's own outputs.

Tolerances as for the frictionless solve: rel-L2(u) <= 1e-4 and step forces
<= 1e-3 at a GPU residual of 1e-6."""
import numpy as np
import pytest

import workloads as W
from oracle import Problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2103_16747_b300 as F
    return F


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _dragged_plane(n=4, n_steps=8, tilt=0.05, depth=0.2):
    m = W.cube_mesh(n, E=1.0e3, nu=0.3)
    ind = W.plane_indenter(1.0, depth, n_steps)
    a = np.array([1.0, 0.0, -tilt])
    ind.direction = a / np.linalg.norm(a)
    return m, ind


def _opt(F, mu, passes=1):
    opt = F.fem_default_options()
    opt.mu_f = mu
    opt.friction_passes = passes
    return opt


def _solve(F, m, ind, mu, n_parts=None, passes=1):
    s = F.IndentationSolver(m)
    if n_parts:
        F.fem_repartition(s.handle, n_parts)
    s.set_indenter(ind)
    return s.solve(1e-6, _opt(F, mu, passes))


@pytest.mark.parametrize("n_parts", [None, 3])
def test_dragged_plane_matches_oracle(F, n_parts):
    mu = 0.783
    m, ind = _dragged_plane()
    ref = Problem(m, ind, mu_f=mu).solve(tol=1e-10)
    assert ref.converged
    out = _solve(F, m, ind, mu, n_parts)
    st = out["stats"]
    assert out["rc"] == 0 and st.steps_done == ind.n_steps and st.residual <= 1e-6 * st.scale
    e_u = rel(out["u"], ref.u)
    e_f = max(rel(out["step_force"][k], ref.step_force[k]) for k in range(1, ind.n_steps))
    print(f"parts={n_parts}: rel-L2(u)={e_u:.2e} max rel F={e_f:.2e} newton={st.newton_iters} cg={st.cg_iters}")
    assert e_u <= 1e-4 and e_f <= 1e-3
    assert rel(out["nodal_contact"], ref.nodal_contact) <= 1e-3
    # Coulomb's law on the GPU's own outputs: in full sliding the tangential
    # nodal forces sum in magnitude to mu times the previous step's normal force
    Fz = out["step_force"][:, 2]
    ft = np.linalg.norm(out["nodal_contact"][:, :2], axis=1).sum()
    assert ft == pytest.approx(mu * abs(Fz[-2]), rel=1e-5)
    # friction drags the body: without it the tangential force vanishes
    out0 = _solve(F, m, ind, 0.0)
    assert abs(out0["step_force"][-1, 0]) < 1e-6 * abs(out0["step_force"][-1, 2])
    assert out["step_force"][-1, 0] > 0.5 * mu * abs(Fz[-2])


def test_stick_limit_matches_oracle(F):
    m, ind = _dragged_plane(n_steps=4, tilt=0.2, depth=0.05)
    ref = Problem(m, ind, mu_f=50.0).solve(tol=1e-10)
    out = _solve(F, m, ind, 50.0)
    assert out["rc"] == 0
    assert rel(out["u"], ref.u) <= 1e-4
    assert max(rel(out["step_force"][k], ref.step_force[k]) for k in range(1, 4)) <= 1e-3


def test_sphere_with_friction_matches_oracle(F):
    m, ind = W.cube_sphere()
    ref = Problem(m, ind, mu_f=0.783).solve(tol=1e-10)
    assert ref.converged
    out = _solve(F, m, ind, 0.783)
    assert out["rc"] == 0
    e_u = rel(out["u"], ref.u)
    print(f"cube sphere with friction: rel-L2(u)={e_u:.2e}")
    assert e_u <= 1e-4
    assert max(rel(out["step_force"][k], ref.step_force[k]) for k in range(1, 10)) <= 1e-3


@pytest.mark.parametrize("engine", [(1, 0), (2, 0), (1, 3)])
def test_batch_with_friction_matches_oracle(F, engine):
    mu = 0.783
    m, ind = _dragged_plane()
    ref = Problem(m, ind, mu_f=mu).solve(tol=1e-10)
    h = F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes)
    opt = _opt(F, mu)
    opt.batch_engine, opt.batch_parts = engine
    out = [np.zeros((m.n_nodes, 3)) for _ in range(2)]
    frc = [np.zeros((ind.n_steps, 3)) for _ in range(2)]
    rc, st = F.fem_solve_batch([h, h], [ind, ind], 1e-6, opt, out, frc)
    assert rc == 0
    for k in range(2):
        assert rel(out[k], ref.u) <= 1e-4
        assert max(rel(frc[k][j], ref.step_force[j]) for j in range(1, ind.n_steps)) <= 1e-3
    assert np.array_equal(out[0], out[1])
    F.fem_destroy_mesh(h)


@pytest.mark.parametrize("n_parts", [None, 3])
def test_friction_passes_match_oracle(F, n_parts):
    """Each load step re-solved with the normal forces refreshed at its own
    converged state: parity with the oracle's passes, and the passes approach
    Coulomb's law with the step's own normal forces."""
    mu, passes = 0.783, 6
    m, ind = _dragged_plane()
    p = Problem(m, ind, mu_f=mu, friction_passes=passes)
    ref = p.solve(tol=1e-10)
    assert ref.converged
    out = _solve(F, m, ind, mu, n_parts, passes)
    st = out["stats"]
    assert out["rc"] == 0 and st.steps_done == ind.n_steps
    e_u = rel(out["u"], ref.u)
    e_f = max(rel(out["step_force"][k], ref.step_force[k]) for k in range(1, ind.n_steps))
    one = _solve(F, m, ind, mu, n_parts, 1)
    print(f"parts={n_parts} passes={passes}: rel-L2(u)={e_u:.2e} max rel F={e_f:.2e} "
          f"newton={st.newton_iters} (one pass {one['stats'].newton_iters})")
    assert e_u <= 1e-4 and e_f <= 1e-3
    assert rel(out["nodal_contact"], ref.nodal_contact) <= 1e-3
    assert st.newton_iters > one["stats"].newton_iters
    # Coulomb with the end state's normal forces (oracle's refresh at the GPU's u)
    p.set_friction_lag(out["u"], p.K)
    p.refresh_friction(out["u"], p.K)
    ft = np.linalg.norm(out["nodal_contact"][:, :2], axis=1)
    assert np.abs(ft - mu * p.fric["fn"]).max() <= 0.01 * ft.max()
    p.fric = None
    # passes without friction change nothing
    a, b = _solve(F, m, ind, 0.0, n_parts, 1), _solve(F, m, ind, 0.0, n_parts, passes)
    assert np.array_equal(a["u"], b["u"]) and a["stats"].newton_iters == b["stats"].newton_iters


@pytest.mark.parametrize("engine", [(1, 2), (2, 2)])
def test_batch_friction_passes_match_oracle(F, engine):
    """Friction passes in the CTA-group engine and in thread-block clusters."""
    mu, passes = 0.783, 4
    m, ind = _dragged_plane()
    ref = Problem(m, ind, mu_f=mu, friction_passes=passes).solve(tol=1e-10)
    h = F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes)
    opt = _opt(F, mu, passes)
    opt.batch_engine, opt.batch_parts = engine
    out = [np.zeros((m.n_nodes, 3)) for _ in range(2)]
    frc = [np.zeros((ind.n_steps, 3)) for _ in range(2)]
    rc, st = F.fem_solve_batch([h, h], [ind, ind], 1e-6, opt, out, frc)
    assert rc == 0
    for k in range(2):
        assert rel(out[k], ref.u) <= 1e-4
        assert max(rel(frc[k][j], ref.step_force[j]) for j in range(1, ind.n_steps)) <= 1e-3
    F.fem_destroy_mesh(h)


def test_friction_options_are_validated(F):
    m, ind = _dragged_plane()
    s = F.IndentationSolver(m)
    s.set_indenter(ind)
    for field, value in (("mu_f", -0.1), ("friction_eps", 0.0), ("mu_f", float("nan")),
                         ("friction_passes", 0), ("friction_passes", 65)):
        opt = F.fem_default_options()
        setattr(opt, field, value)
        assert s.solve(1e-6, opt, check=False)["rc"] == F.FEM_ERR_ARG


def test_fingertip_with_friction_matches_oracle(F):
    import os
    here = os.path.dirname(os.path.abspath(__file__))
    path = os.path.join(here, "golden", "fingertip_sphere_friction_oracle.npz")
    if not os.path.exists(path):
        pytest.skip("golden file missing: run tests/golden/make_golden.py friction")
    from tests.golden.make_golden import FRICTION_MU, mesh_digest
    g = np.load(path)
    m, ind = W.fingertip_sphere()
    assert str(g["digest"]) == mesh_digest(m, ind), "workload generator changed: regenerate golden"
    out = _solve(F, m, ind, FRICTION_MU)
    st = out["stats"]
    assert out["rc"] == 0 and st.steps_done == 20
    e_u = rel(out["u"], g["u"])
    e_f = [rel(out["step_force"][k], g["step_force"][k]) for k in range(1, 20)]
    print(f"fingertip with friction: rel-L2(u)={e_u:.2e} max rel F={max(e_f):.2e} newton={st.newton_iters} "
          f"cg={st.cg_iters} kernel={st.kernel_ms:.1f} ms")
    assert e_u <= 1e-4
    assert max(e_f) <= 1e-3
