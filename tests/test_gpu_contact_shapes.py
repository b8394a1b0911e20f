"""GPU parity of the non-spherical indenters: an infinite cylinder lying across
the surface (axis normal to the approach) and the edge of a box whose faces
meet at +-45 degrees to the approach (the paper presses objects with edges as
well as round ones into the sensor, Sec. III-C).

Each shape is checked like the sphere: the FP64 residual and the FP32 tangent
product of one pass against the oracle at a state where the contact is active
(for the box, with pressed nodes on both sides of its medial plane, where the
signed distance's gradient jumps from one face to the other), full solves of
the unit cube on the single-solve path and on both batched engines against
the oracle's direct solve, and one random-draw fingertip case per shape
against the oracle's stored solution.

Tolerances as everywhere: relative L2 nodal displacement error <= 1e-4,
relative contact-force error <= 1e-3 at every load step, GPU residual <=
1e-6 * scale; one pass: FP64 residual to 1e-10, FP32 tangent product to
2e-5."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import Problem, contact

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
CASES = {"cylinder": W.cube_cylinder, "box_edge": W.cube_box_edge}


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2103_16747_b300 as F
    return F


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def cube_refs():
    out = {}
    for name, make in CASES.items():
        m, ind = make()
        r = Problem(m, ind).solve(tol=1e-10)
        assert r.converged
        out[name] = (m, ind, r)
    return out


def _active_state(name, cube_refs, seed):
    """The oracle's equilibrium at the last load step plus a small random
    perturbation (no node sits exactly on a medial plane)."""
    m, ind, r = cube_refs[name]
    rng = np.random.default_rng(seed)
    p = Problem(m, ind)
    u = r.u + 0.005 * np.abs(r.u).max() * rng.standard_normal(r.u.shape)
    u[p.fixed] = 0.0
    phi, n, _ = contact.sdf(ind.shape, p.origin_at(ind.n_steps), ind.rotation, ind.params, m.nodes + u)
    act = (phi < 0) & (p.k > 0)
    assert act.sum() >= 3
    if ind.shape == W.BOX:
        # the active nodes' normals: both faces that meet at the edge
        face = np.argmax(np.abs(n[act] @ ind.rotation), axis=1)
        assert set(face.tolist()) >= {0, 1}, face
    return m, ind, p, u


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_residual_matches_oracle(F, cube_refs, name):
    m, ind, p, u = _active_state(name, cube_refs, 21)
    s = F.IndentationSolver(m)
    s.set_indenter(ind)
    R, fc, (e_el, e_c) = s.eval_residual(u, ind.n_steps)
    g, fco = p.gradient(u, ind.n_steps)
    assert rel(R, g) < 1e-10
    assert rel(fc, fco) < 1e-10
    assert e_el == pytest.approx(p.elastic_energy(u)[0], rel=1e-11)
    assert e_c == pytest.approx(float(p.contact_terms(u, ind.n_steps)[0].sum()), rel=1e-9)
    s.close()


@pytest.mark.parametrize("tangent", ["projected", "exact"])
@pytest.mark.parametrize("name", list(CASES))
def test_fp32_tangent_product_matches_oracle(F, cube_refs, name, tangent):
    m, ind, p, u = _active_state(name, cube_refs, 22)
    v = np.random.default_rng(23).standard_normal((m.n_nodes, 3))
    s = F.IndentationSolver(m)
    s.set_indenter(ind)
    opt = F.fem_default_options()
    opt.tangent = F.FEM_TANGENT_PROJECTED if tangent == "projected" else F.FEM_TANGENT_EXACT
    y = s.apply_tangent(u, ind.n_steps, v, opt)
    # oracle: projected tangent with the Gauss-Newton contact block, or the exact
    # tangent with the exact contact Hessian (indenter curvature included)
    K = p.hessian(u, ind.n_steps, projected=(tangent == "projected"))
    yo = (K @ (v.ravel() * p.free)) * p.free
    assert rel(y.ravel(), yo) < 2e-5
    s.close()


def _check_solve(u, forces, nodal, st, m, ind, r, label):
    e_u = rel(u, r.u)
    e_f = [rel(forces[k], r.step_force[k]) for k in range(ind.n_steps)]
    print(f"{label}: rel-L2(u)={e_u:.2e} max rel F={max(e_f):.2e} newton={st.newton_iters} cg={st.cg_iters}")
    assert st.steps_done == ind.n_steps
    assert st.residual <= 1e-6 * st.scale
    assert e_u <= 1e-4
    assert max(e_f) <= 1e-3
    if nodal is not None:
        assert rel(nodal, r.nodal_contact) <= 1e-3
    rn, scale, _ = Problem(m, ind).residual_norm(u, ind.n_steps)
    assert rn <= 1e-6 * scale


@pytest.mark.parametrize("n_parts", [None, 7])
@pytest.mark.parametrize("name", list(CASES))
def test_cube_solve_matches_oracle(F, cube_refs, name, n_parts):
    m, ind, r = cube_refs[name]
    s = F.IndentationSolver(m)
    if n_parts:
        F.fem_repartition(s.handle, n_parts)
    s.set_indenter(ind)
    out = s.solve(1e-6)
    assert out["rc"] == 0
    _check_solve(out["u"], out["step_force"], out["nodal_contact"], out["stats"], m, ind, r,
                 f"cube {name} parts={n_parts}")
    s.close()


@pytest.mark.parametrize("engine", [(1, 0), (2, 0)])
def test_cube_shapes_in_one_batch_match_oracle(F, cube_refs, engine):
    """Sphere, cylinder and box edge on the cube as three jobs of one launch."""
    m, sph = W.cube_sphere()
    ref_s = Problem(m, sph).solve(tol=1e-10)
    jobs = [(m, sph, ref_s)] + [cube_refs[n] for n in CASES]
    h = F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes)
    out = [np.zeros((m.n_nodes, 3)) for _ in jobs]
    frc = [np.zeros((j[1].n_steps, 3)) for j in jobs]
    opt = F.fem_default_options()
    opt.batch_engine, opt.batch_parts = engine
    rc, st = F.fem_solve_batch([h] * len(jobs), [j[1] for j in jobs], 1e-6, opt, out, frc)
    F.fem_destroy_mesh(h)
    assert rc == 0, [x.status for x in st]
    for k, (mm, ind, r) in enumerate(jobs):
        _check_solve(out[k], frc[k], None, st[k], mm, ind, r, f"batch {engine} job {k}")


def _golden(kind):
    path = os.path.join(HERE, "golden", f"fingertip_{kind}_oracle.npz")
    if not os.path.exists(path):
        pytest.skip("golden file missing: run tests/golden/make_golden.py")
    g = np.load(path)
    m, ind = W.fingertip_shape_draw(W.CYLINDER if kind == "cylinder" else W.BOX)
    from tests.golden.make_golden import mesh_digest
    assert str(g["digest"]) == mesh_digest(m, ind), "workload generator changed: regenerate golden"
    return m, ind, g


class _Ref:
    def __init__(self, g):
        self.u, self.step_force, self.nodal_contact = g["u"], g["step_force"], g["nodal_contact"]


@pytest.mark.parametrize("kind", ["cylinder", "box_edge"])
def test_fingertip_draw_matches_golden(F, kind):
    """One cylinder and one box-edge draw of the random-indentation workload on
    the 38,880-tet fingertip: the single-solve path and the CTA-group engine
    against the oracle's direct solve."""
    m, ind, g = _golden(kind)
    r = _Ref(g)
    s = F.IndentationSolver(m)
    s.set_indenter(ind)
    out = s.solve(1e-6)
    assert out["rc"] == 0
    _check_solve(out["u"], out["step_force"], out["nodal_contact"], out["stats"], m, ind, r,
                 f"fingertip {kind} single")
    s.close()
    h = F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes)
    u = [np.zeros((m.n_nodes, 3))]
    f = [np.zeros((ind.n_steps, 3))]
    opt = F.fem_default_options()
    rc, st = F.fem_solve_batch([h], [ind], 1e-6, opt, u, f)
    F.fem_destroy_mesh(h)
    assert rc == 0
    _check_solve(u[0], f[0], None, st[0], m, ind, r, f"fingertip {kind} batch")
