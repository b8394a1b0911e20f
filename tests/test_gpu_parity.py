"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Tolerances (parity rule of the indentation problem): relative L2 nodal
displacement error <= 1e-4 and relative contact-force error <= 1e-3 at every
load step, the GPU converged to ||R_free|| <= 1e-6 * scale. Single passes: the
FP64 residual to 1e-10 relative (same arithmetic, different summation order),
the FP32 tangent product to 2e-5 relative (FP32 rounding of F, the SVD and the
products)."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import Problem, material
from tests.closed_forms import uniaxial_plane

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


def _solver(F, mesh, ind, n_parts=None):
    s = F.IndentationSolver(mesh)
    if n_parts:
        F.fem_repartition(s.handle, n_parts)
    s.set_indenter(ind)
    return s


def test_barrier_timeout_is_reported_and_context_survives(F):
    assert F.fem_debug_barrier_timeout(0.05) == F.FEM_ERR_TIMEOUT
    m, ind = W.cube_sphere()
    s = _solver(F, m, ind)
    out = s.solve(1e-6)
    assert out["rc"] == 0


@pytest.mark.parametrize("workload", ["cube", "fingertip"])
def test_fp64_residual_matches_oracle(F, workload):
    rng = np.random.default_rng(5)
    if workload == "cube":
        m, ind = W.cube_sphere()
        u = 0.002 * rng.standard_normal((m.n_nodes, 3))
        step = 10
    else:
        m, ind = W.fingertip_sphere()
        u = 0.02 * rng.standard_normal((m.n_nodes, 3))
        step = 20
    p = Problem(m, ind)
    u[p.fixed] = 0.0
    s = _solver(F, m, ind)
    R, fc, (e_el, e_c) = s.eval_residual(u, step)
    g, fco = p.gradient(u, step)
    assert np.count_nonzero(np.linalg.norm(fco, axis=1)) > 0
    assert rel(R, g) < 1e-10
    assert rel(fc, fco) < 1e-10
    ee, _ = p.elastic_energy(u)
    ec = float(p.contact_terms(u, step)[0].sum())
    assert e_el == pytest.approx(ee, rel=1e-11)
    assert e_c == pytest.approx(ec, rel=1e-9)


@pytest.mark.parametrize("tangent", ["projected", "exact"])
@pytest.mark.parametrize("workload", ["cube", "fingertip"])
def test_fp32_tangent_product_matches_oracle(F, workload, tangent):
    rng = np.random.default_rng(9)
    if workload == "cube":
        m, ind = W.cube_sphere()
        u = 0.01 * rng.standard_normal((m.n_nodes, 3))
        step = 10
    else:
        m, ind = W.fingertip_sphere()
        u = 0.05 * rng.standard_normal((m.n_nodes, 3))
        step = 20
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


def _cube_reference():
    m, ind = W.cube_sphere()
    return m, ind, Problem(m, ind).solve(tol=1e-10)


@pytest.fixture(scope="module")
def cube_ref():
    return _cube_reference()


@pytest.mark.parametrize("n_parts", [None, 7, 2])
def test_cube_sphere_solve_parity(F, cube_ref, n_parts):
    m, ind, ref = cube_ref
    s = _solver(F, m, ind, n_parts)
    out = s.solve(1e-6)
    st = out["stats"]
    assert out["rc"] == 0 and st.steps_done == 10
    assert st.residual <= 1e-6 * st.scale
    e_u = rel(out["u"], ref.u)
    e_f = [rel(out["step_force"][k], ref.step_force[k]) for k in range(10)]
    print(f"cube parts={n_parts}: rel-L2(u)={e_u:.2e} max rel F={max(e_f):.2e} "
          f"newton={st.newton_iters} cg={st.cg_iters}")
    assert e_u <= 1e-4
    assert max(e_f) <= 1e-3
    assert rel(out["nodal_contact"], ref.nodal_contact) <= 1e-3


@pytest.mark.parametrize("degree", range(1, 9))
def test_every_preconditioner_degree_matches_oracle(F, cube_ref, degree):
    """Block-Jacobi (degree 1) and its Chebyshev polynomials of degree 2-8:
    the preconditioner changes the PCG path, not the equilibrium. Odd and even
    degrees publish their halo epochs with opposite parities; the reduction
    slots alternate by publication count in both. Single path on 15 parts and
    the CTA-group engine (two solves of 3 parts in one launch)."""
    m, ind, ref = cube_ref
    opt = F.fem_default_options()
    opt.precond_degree = degree
    s = _solver(F, m, ind, 15)
    out = s.solve(1e-6, opt)
    st = out["stats"]
    assert out["rc"] == 0 and st.residual <= 1e-6 * st.scale
    assert rel(out["u"], ref.u) <= 1e-4
    assert max(rel(out["step_force"][k], ref.step_force[k]) for k in range(10)) <= 1e-3
    h = F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes)
    opt.batch_engine, opt.batch_parts = 1, 3
    u = [np.zeros((m.n_nodes, 3)) for _ in range(2)]
    f = [np.zeros((ind.n_steps, 3)) for _ in range(2)]
    rc, _ = F.fem_solve_batch([h, h], [ind, ind], 1e-6, opt, u, f)
    F.fem_destroy_mesh(h)
    assert rc == 0
    assert np.array_equal(u[0], u[1])
    assert rel(u[0], ref.u) <= 1e-4
    print(f"degree {degree}: newton={st.newton_iters} cg={st.cg_iters} products={st.tangent_products}")


def test_deterministic_bitwise(F):
    m, ind = W.cube_sphere()
    s = _solver(F, m, ind)
    a = s.solve(1e-6)
    b = s.solve(1e-6)
    assert np.array_equal(a["u"], b["u"])
    assert np.array_equal(a["step_force"], b["step_force"])
    assert a["stats"].cg_iters == b["stats"].cg_iters


def test_uniaxial_closed_form_on_gpu(F):
    """Rollers + frictionless plane on the unit cube, 10% compression:
    homogeneous state, closed form up to the O(1/c_kappa) edge effect."""
    E, nu, ck, strain = 1e6, 0.3, 1e3, 0.1
    m = W.cube_mesh(4, E=E, nu=nu, fix="rollers")
    ind = W.plane_indenter(1.0, strain, 4)
    s = _solver(F, m, ind)
    opt = F.fem_default_options()
    opt.c_kappa = ck
    out = s.solve(1e-7, opt)
    h_bar = s.info().h_bar
    lz, lt, pzz = uniaxial_plane(strain, E, nu, h_bar, ck)
    X = m.nodes
    np.testing.assert_allclose(out["u"][:, 2], (lz - 1) * X[:, 2], atol=5e-4 * strain)
    np.testing.assert_allclose(out["u"][:, 0], (lt - 1) * X[:, 0], atol=5e-4 * strain)
    assert out["step_force"][-1, 2] == pytest.approx(pzz, rel=5e-4)


def test_patch_test_on_gpu(F):
    rng = np.random.default_rng(3)
    m = W.cube_mesh(3)
    X = m.nodes.copy()
    interior = np.all((X > 1e-9) & (X < 1 - 1e-9), axis=1)
    X[interior] += rng.uniform(-0.08, 0.08, (interior.sum(), 3))
    bnd = np.nonzero(~interior)[0].astype(np.int32)
    A = np.array([[0.04, 0.01, -0.02], [0.0, -0.03, 0.02], [0.01, 0.02, 0.05]])
    t = np.array([0.01, -0.02, 0.03])
    m2 = W.Mesh(X, m.tets, m.tet_material, m.materials, bnd, None)
    ind = W.cube_sphere_indenter()
    ind.origin = np.array([50.0, 50.0, 50.0])
    ind.depth_schedule = np.array([0.0, 0.0])
    s = _solver(F, m2, ind)
    s.set_dirichlet_values(X[bnd] @ A.T + t)
    out = s.solve(1e-8)
    np.testing.assert_allclose(out["u"], X @ A.T + t, atol=1e-9)


def test_no_contact_gives_zero(F):
    m, ind = W.cube_sphere()
    ind.origin = ind.origin + np.array([0.0, 0.0, 1.0])   # stays 0.95 above the top
    s = _solver(F, m, ind)
    out = s.solve(1e-6)
    assert out["rc"] == 0
    assert np.abs(out["u"]).max() == 0.0
    assert np.abs(out["step_force"]).max() == 0.0


def test_single_tet(F):
    nodes = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0.3, 0.25, 0.9]], dtype=float)
    m = W.Mesh(nodes, np.array([[0, 1, 2, 3]], dtype=np.int32), np.zeros(1, dtype=np.int32),
               np.array([[1000.0, 0.3]]), np.array([0, 1, 2], dtype=np.int32))
    ind = W.plane_indenter(0.9, 0.2, 3)
    ref = Problem(m, ind, c_kappa=50.0).solve(tol=1e-12)
    s = _solver(F, m, ind)
    opt = F.fem_default_options()
    opt.c_kappa = 50.0
    out = s.solve(1e-8, opt)
    assert rel(out["u"], ref.u) < 1e-5


def test_not_converged_status(F):
    m, ind = W.cube_sphere()
    s = _solver(F, m, ind)
    opt = F.fem_default_options()
    opt.max_newton = 1
    out = s.solve(1e-6, opt, check=False)
    assert out["rc"] == F.FEM_ERR_NOT_CONVERGED
    assert out["stats"].steps_done == 0 and out["stats"].newton_iters == 1
    assert np.isfinite(out["u"]).all()


@pytest.fixture(scope="module")
def fingertip_golden():
    path = os.path.join(HERE, "golden", "fingertip_sphere_oracle.npz")
    if not os.path.exists(path):
        pytest.skip("golden file missing: run tests/golden/make_golden.py")
    g = np.load(path)
    m, ind = W.fingertip_sphere()
    from tests.golden.make_golden import mesh_digest
    assert str(g["digest"]) == mesh_digest(m, ind), "workload generator changed: regenerate golden"
    return m, ind, g


def test_fingertip_sphere_parity(F, fingertip_golden):
    m, ind, g = fingertip_golden
    s = _solver(F, m, ind)
    out = s.solve(1e-6)
    st = out["stats"]
    assert out["rc"] == 0 and st.steps_done == 20
    e_u = rel(out["u"], g["u"])
    e_f = [rel(out["step_force"][k], g["step_force"][k]) for k in range(20)]
    print(f"fingertip: rel-L2(u)={e_u:.2e} max rel F={max(e_f):.2e} newton={st.newton_iters} "
          f"cg={st.cg_iters} kernel={st.kernel_ms:.1f} ms")
    assert e_u <= 1e-4
    assert max(e_f) <= 1e-3
    # certify: the oracle's own FP64 residual of the GPU displacement
    rn, scale, _ = Problem(m, ind).residual_norm(out["u"], 20)
    assert rn <= 1e-6 * scale


def test_fp64_reciprocals_meet_their_error_bound(F):
    """The element kernels take FP64 1/x and 1/sqrt(x) from the FP32 hardware
    value refined by one Newton-Raphson step; one step squares FP32's relative
    error (<= ~2e-7), so both stay within 1e-13 of the FP64 values wherever x
    and 1/x are FP32-normal."""
    rng = np.random.default_rng(17)
    x = 10.0 ** rng.uniform(-30, 30, 200000)
    x = np.concatenate([x, 1.0 + rng.uniform(-1e-3, 1e-3, 1000), [1.0, 2.0, 0.5, 3.0, 1e-37, 1e37]])
    r, q = F.fem_debug_reciprocals(x)
    assert np.max(np.abs(r * x - 1.0)) < 1e-13
    assert np.max(np.abs(q * np.sqrt(x) - 1.0)) < 1e-13
