"""GPU parity of dynamic stepping (backward Euler with a lumped mass, one
load step = one time step; Sec. III-A) against the FP64 oracle, through the
C ABI.

Tolerances as for the quasi-static solve: relative L2 nodal displacement
error <= 1e-4 and relative contact-force error <= 1e-3 at every step, the GPU
converged to ||R_free|| <= 1e-6 * scale. The cube cases use a density at
which the inertia term is of the order of the stiffness, so that the dynamic
answer differs clearly from the quasi-static one."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import Problem

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2103_16747_b300 as F
    return F


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _opt(F, dt, density):
    opt = F.fem_default_options()
    opt.dt = dt
    opt.density = density
    return opt


def _check(out, ref, n_steps):
    st = out["stats"]
    assert out["rc"] == 0 and st.steps_done == n_steps
    assert st.residual <= 1e-6 * st.scale
    e_u = rel(out["u"], ref.u)
    e_f = [rel(out["step_force"][k], ref.step_force[k]) for k in range(n_steps)]
    print(f"rel-L2(u)={e_u:.2e} max rel F={max(e_f):.2e} newton={st.newton_iters} cg={st.cg_iters}")
    assert e_u <= 1e-4
    assert max(e_f) <= 1e-3


@pytest.fixture(scope="module")
def cube_dyn():
    m, ind = W.cube_sphere()
    return m, ind, Problem(m, ind, dt=1e-3, density=1.0).solve(tol=1e-10), Problem(m, ind).solve(tol=1e-10)


@pytest.mark.parametrize("n_parts", [None, 5])
def test_dynamic_cube_matches_oracle(F, cube_dyn, n_parts):
    m, ind, ref, qs = cube_dyn
    assert rel(ref.u, qs.u) > 1e-2          # inertia matters at this density and step
    s = F.IndentationSolver(m)
    if n_parts:
        F.fem_repartition(s.handle, n_parts)
    s.set_indenter(ind)
    out = s.solve(1e-6, _opt(F, 1e-3, 1.0))
    _check(out, ref, ind.n_steps)
    # the same mesh handle solves quasi-statically again with dt = 0
    out_qs = s.solve(1e-6)
    assert rel(out_qs["u"], qs.u) <= 1e-4


def test_dynamic_free_body_matches_oracle_and_momentum(F):
    """No fixed node: only the mass term makes the problem well posed. Centre
    of mass: sum_i m_i u_i,K = dt^2 sum_{k<=K} sum_{j<=k} F_j from the GPU's
    own step forces."""
    m = W.cube_mesh(4, fix="none")
    ind = W.place_at_contact(W.cube_sphere_indenter(radius=0.3, depth=0.05, n_steps=6), m.nodes)
    dt, rho = 1e-3, 1.0
    p = Problem(m, ind, dt=dt, density=rho)
    ref = p.solve(tol=1e-10)
    assert ref.converged
    s = F.IndentationSolver(m)
    s.set_indenter(ind)
    out = s.solve(1e-6, _opt(F, dt, rho))
    _check(out, ref, ind.n_steps)
    Fc = out["step_force"]
    expect = dt * dt * np.cumsum(np.cumsum(Fc, axis=0), axis=0)[-1]
    cm = (p.mass[:, None] * out["u"]).sum(axis=0)
    assert np.linalg.norm(cm - expect) <= 1e-4 * np.linalg.norm(expect)


@pytest.mark.parametrize("engine", [(1, 0), (2, 0), (1, 3)])
def test_dynamic_batch_matches_oracle(F, cube_dyn, engine):
    m, ind, ref, _ = cube_dyn
    h = F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes)
    opt = _opt(F, 1e-3, 1.0)
    opt.batch_engine, opt.batch_parts = engine
    out = [np.zeros((m.n_nodes, 3)) for _ in range(2)]
    frc = [np.zeros((ind.n_steps, 3)) for _ in range(2)]
    rc, st = F.fem_solve_batch([h, h], [ind, ind], 1e-6, opt, out, frc)
    assert rc == 0
    for k in range(2):
        assert st[k].steps_done == ind.n_steps and st[k].residual <= 1e-6 * st[k].scale
        assert rel(out[k], ref.u) <= 1e-4
        assert max(rel(frc[k][j], ref.step_force[j]) for j in range(ind.n_steps)) <= 1e-3
    assert np.array_equal(out[0], out[1])
    F.fem_destroy_mesh(h)


@pytest.fixture(scope="module")
def fingertip_dynamic_golden():
    path = os.path.join(HERE, "golden", "fingertip_sphere_dynamic_oracle.npz")
    if not os.path.exists(path):
        pytest.skip("golden file missing: run tests/golden/make_golden.py dynamic")
    g = np.load(path)
    m, ind = W.fingertip_sphere()
    from tests.golden.make_golden import DYN_DENSITY, DYN_DT, mesh_digest
    assert str(g["digest"]) == mesh_digest(m, ind), "workload generator changed: regenerate golden"
    return m, ind, g, DYN_DT, DYN_DENSITY


def test_dynamic_fingertip_matches_oracle(F, fingertip_dynamic_golden):
    m, ind, g, dt, rho = fingertip_dynamic_golden
    s = F.IndentationSolver(m)
    s.set_indenter(ind)
    out = s.solve(1e-6, _opt(F, dt, rho))
    st = out["stats"]
    assert out["rc"] == 0 and st.steps_done == 20
    e_u = rel(out["u"], g["u"])
    e_f = [rel(out["step_force"][k], g["step_force"][k]) for k in range(20)]
    print(f"dynamic fingertip: rel-L2(u)={e_u:.2e} max rel F={max(e_f):.2e} newton={st.newton_iters} "
          f"cg={st.cg_iters} kernel={st.kernel_ms:.1f} ms")
    assert e_u <= 1e-4
    assert max(e_f) <= 1e-3


def test_dynamic_options_are_validated(F):
    m, ind = W.cube_sphere()
    s = F.IndentationSolver(m)
    s.set_indenter(ind)
    for dt, rho in ((-1e-3, 1.0), (1e-3, 0.0), (float("nan"), 1.0)):
        out = s.solve(1e-6, _opt(F, dt, rho), check=False)
        assert out["rc"] == F.FEM_ERR_ARG
