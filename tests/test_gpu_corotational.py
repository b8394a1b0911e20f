"""GPU parity of the co-rotational linear-elastic law (model 1; the law the
paper's simulator uses for the skin, Sec. III-A) against the FP64 oracle,
through the C ABI: the FP64 residual and energy, the FP32 tangent product,
full solves (all co-rotational, and both laws mixed in one mesh), the
homogeneous uniaxial closed form under prescribed displacements, element
stress and the calibrated co-rotational fingertip against its stored oracle
solution.

Tolerances as for the neo-Hookean law: residual 1e-10 relative, tangent
product 2e-5, solves rel-L2(u) <= 1e-4 and step forces <= 1e-3."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import Problem
from oracle.material import cauchy, von_mises

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


def _mixed_cube():
    """Cube whose tets draw one of two materials at random: neo-Hookean and
    co-rotational."""
    m, ind = W.cube_sphere()
    rng = np.random.default_rng(31)
    m.materials = np.array([[1.0e6, 0.3, 0.0], [2.0e6, 0.35, 1.0]])
    m.tet_material = rng.integers(0, 2, m.n_tets).astype(np.int32)
    return m, ind


def _case(name):
    if name == "cube":
        m, ind = W.cube_sphere()
        return W.with_model(m, 1), ind, 0.01, 10
    if name == "mixed":
        m, ind = _mixed_cube()
        return m, ind, 0.01, 10
    m, ind = W.fingertip_sphere()
    return W.with_model(m, 1), ind, 0.05, 20


def _solver(F, m, ind):
    s = F.IndentationSolver(m)
    s.set_indenter(ind)
    return s


@pytest.mark.parametrize("name", ["cube", "mixed", "fingertip"])
def test_fp64_residual_matches_oracle(F, name):
    m, ind, amp, step = _case(name)
    rng = np.random.default_rng(5)
    u = 0.2 * amp * rng.standard_normal((m.n_nodes, 3))
    p = Problem(m, ind)
    u[p.fixed] = 0.0
    s = _solver(F, m, ind)
    R, fc, (e_el, e_c) = s.eval_residual(u, step)
    g, fco = p.gradient(u, step)
    assert rel(R, g) < 1e-10
    assert rel(fc, fco) < 1e-10
    ee, _ = p.elastic_energy(u)
    assert e_el == pytest.approx(ee, rel=1e-11)


@pytest.mark.parametrize("tangent", ["projected", "exact"])
@pytest.mark.parametrize("name", ["cube", "mixed", "fingertip"])
def test_fp32_tangent_product_matches_oracle(F, name, tangent):
    m, ind, amp, step = _case(name)
    rng = np.random.default_rng(9)
    u = amp * rng.standard_normal((m.n_nodes, 3))
    p = Problem(m, ind)
    u[p.fixed] = 0.0
    v = rng.standard_normal((m.n_nodes, 3))
    s = _solver(F, m, ind)
    opt = F.fem_default_options()
    opt.tangent = F.FEM_TANGENT_PROJECTED if tangent == "projected" else F.FEM_TANGENT_EXACT
    y = s.apply_tangent(u, step, v, opt)
    # oracle: projected tangent with the Gauss-Newton contact block, or the exact
    # tangent with the exact contact Hessian (indenter curvature included)
    K = p.hessian(u, step, projected=(tangent == "projected"))
    free = p.free
    vv = v.ravel() * free
    yo = (K @ vv) * free
    assert rel(y.ravel(), yo) < 2e-5


@pytest.mark.parametrize("name", ["cube", "mixed"])
def test_cube_solve_matches_oracle(F, name):
    m, ind, _, _ = _case(name)
    ref = Problem(m, ind).solve(tol=1e-10)
    assert ref.converged
    out = _solver(F, m, ind).solve(1e-6)
    st = out["stats"]
    assert out["rc"] == 0 and st.steps_done == 10 and st.residual <= 1e-6 * st.scale
    e_u = rel(out["u"], ref.u)
    e_f = max(rel(out["step_force"][k], ref.step_force[k]) for k in range(10))
    print(f"{name}: rel-L2(u)={e_u:.2e} max rel F={e_f:.2e} newton={st.newton_iters} cg={st.cg_iters}")
    assert e_u <= 1e-4 and e_f <= 1e-3
    # the law matters here: the neo-Hookean answer is measurably different
    nh = W.with_model(m, 0)
    out_nh = _solver(F, nh, ind).solve(1e-6)
    assert rel(out_nh["u"], ref.u) > 1e-3


def test_uniaxial_closed_form_on_gpu(F):
    """Rollers + prescribed top face, 20% compression: the co-rotational law
    gives l_t - 1 = -nu (l_z - 1) exactly at any strain."""
    from tests.test_oracle_corotational import corot_cube_uniaxial
    strain, E, nu = -0.2, 1.0e3, 0.3
    m, vals = corot_cube_uniaxial(4, strain, E, nu)
    ind = W.plane_indenter(50.0, 0.0, 4)
    s = _solver(F, m, ind)
    s.set_dirichlet_values(vals)
    out = s.solve(1e-8)
    assert out["rc"] == 0
    X = m.nodes
    np.testing.assert_allclose(out["u"][:, 2], strain * X[:, 2], atol=1e-6)
    np.testing.assert_allclose(out["u"][:, 0], -nu * strain * X[:, 0], atol=1e-6)
    np.testing.assert_allclose(out["u"][:, 1], -nu * strain * X[:, 1], atol=1e-6)


def test_element_stress_matches_oracle(F):
    m, ind = _mixed_cube()
    rng = np.random.default_rng(4)
    u = 0.02 * rng.standard_normal((m.n_nodes, 3))
    p = Problem(m, ind)
    u[p.fixed] = 0.0
    sig_ref = cauchy(p.F(u), p.mu, p.lam, p.model)
    vm_ref = von_mises(sig_ref)
    h = F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes)
    sig, vm = F.fem_element_stress(h, u, m.n_tets)
    F.fem_destroy_mesh(h)
    ref6 = np.stack([sig_ref[:, 0, 0], sig_ref[:, 1, 1], sig_ref[:, 2, 2],
                     sig_ref[:, 1, 2], sig_ref[:, 0, 2], sig_ref[:, 0, 1]], axis=1)
    assert np.abs(sig - ref6).max() <= 1e-9 * np.abs(ref6).max()
    assert np.abs(vm - vm_ref).max() <= 1e-9 * vm_ref.max()


@pytest.fixture(scope="module")
def fingertip_calibrated_golden():
    path = os.path.join(HERE, "golden", "fingertip_calibrated_oracle.npz")
    if not os.path.exists(path):
        pytest.skip("golden file missing: run tests/golden/make_golden.py corot")
    g = np.load(path)
    m, ind = W.fingertip_calibrated()
    from tests.golden.make_golden import mesh_digest
    assert str(g["digest"]) == mesh_digest(m, ind), "workload generator changed: regenerate golden"
    return m, ind, g


def test_fingertip_calibrated_matches_oracle(F, fingertip_calibrated_golden):
    """The paper's calibrated co-rotational shell (E=1.55 MPa, nu=0.316)."""
    m, ind, g = fingertip_calibrated_golden
    out = _solver(F, m, ind).solve(1e-6)
    st = out["stats"]
    assert out["rc"] == 0 and st.steps_done == 20
    e_u = rel(out["u"], g["u"])
    e_f = [rel(out["step_force"][k], g["step_force"][k]) for k in range(20)]
    print(f"co-rotational fingertip: rel-L2(u)={e_u:.2e} max rel F={max(e_f):.2e} "
          f"newton={st.newton_iters} cg={st.cg_iters} kernel={st.kernel_ms:.1f} ms")
    assert e_u <= 1e-4
    assert max(e_f) <= 1e-3
    rn, scale, _ = Problem(m, ind).residual_norm(out["u"], 20)
    assert rn <= 1e-6 * scale
