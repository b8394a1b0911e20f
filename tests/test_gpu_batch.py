"""Batched solves on the GPU, both engines (CTA groups of one cooperative
launch; thread-block clusters), jobs taken from a queue: parity with the FP64
oracle, a job's result bitwise independent of the rest of the batch and of the
slot that ran it, uneven meshes in one launch."""
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


ENGINES = [(1, 0), (2, 0)]        # (FEM_BATCH_GROUPS, automatic parts), (FEM_BATCH_CLUSTERS, automatic)


def _batch(F, meshes, handles, inds, tol=1e-6, max_newton=None, engine=(1, 0), fp16=False):
    out = [np.zeros((m.n_nodes, 3)) for m in meshes]
    frc = [np.zeros((d.n_steps, 3)) for d in inds]
    opt = F.fem_default_options()
    opt.tangent_fp16 = int(fp16)
    if max_newton is not None:
        opt.max_newton = max_newton
    opt.batch_engine, opt.batch_parts = engine
    rc, st = F.fem_solve_batch(handles, inds, tol, opt, out, frc)
    return rc, out, frc, st


@pytest.mark.parametrize("engine", ENGINES + [(1, 3), (2, 4)])
def test_batch_cube_matches_oracle(F, engine):
    m, ind = W.cube_sphere()
    h = F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes)
    ref = Problem(m, ind).solve(tol=1e-10)
    rc, out, frc, st = _batch(F, [m] * 3, [h] * 3, [ind] * 3, engine=engine)
    assert rc == 0
    for k in range(3):
        assert st[k].steps_done == 10 and st[k].residual <= 1e-6 * st[k].scale
        assert rel(out[k], ref.u) <= 1e-4
        assert max(rel(frc[k][s], ref.step_force[s]) for s in range(10)) <= 1e-3
    # identical jobs give bitwise identical results whichever CTA ran them
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])
    F.fem_destroy_mesh(h)


@pytest.mark.parametrize("engine", ENGINES)
def test_batch_fp16_tangent_holds_for_any_stiffness(F, engine):
    """With tangent_fp16 the batched engines store the tangent in FP16 with a
    per-tet scale. The penalty stiffness scales with E, so the displacements of
    the cube do not depend on E: the cube at E = 1e9 (tangent entries far above
    FP16's range unscaled) and at E = 1e3 must both match the oracle at E = 1e6."""
    m6, ind = W.cube_sphere()
    ref = Problem(m6, ind).solve(tol=1e-10)
    for E in (1.0e3, 1.0e9):
        m = W.cube_mesh(8, E=E, nu=0.3)
        h = F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes)
        rc, out, frc, st = _batch(F, [m], [h], [ind], engine=engine, fp16=True)
        F.fem_destroy_mesh(h)
        assert rc == 0 and st[0].residual <= 1e-6 * st[0].scale
        assert rel(out[0], ref.u) <= 1e-4
        # forces scale with E
        assert rel(frc[0][-1] * (1.0e6 / E), ref.step_force[-1]) <= 1e-3


@pytest.mark.parametrize("engine", ENGINES)
def test_batch_fingertip_matches_golden_and_is_mix_independent(F, engine):
    g = np.load(os.path.join(HERE, "golden", "fingertip_sphere_oracle.npz"))
    m, ind = W.fingertip_sphere()
    draws = W.draw_indentations(m, 5, seed=77)
    h = F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes)
    # deep random draws need more Newton iterations in their last load steps
    # than the default cap allows
    rc, out, frc, st = _batch(F, [m] * 6, [h] * 6, [ind] + draws, max_newton=200, engine=engine)
    assert rc == 0, [s.status for s in st]
    e_u = rel(out[0], g["u"])
    e_f = max(rel(frc[0][s], g["step_force"][s]) for s in range(20))
    print(f"batch fingertip {engine}: rel-L2(u)={e_u:.2e} max rel F={e_f:.2e} newton={st[0].newton_iters} "
          f"cg={st[0].cg_iters} kernel={st[0].kernel_ms:.1f} ms")
    assert e_u <= 1e-4 and e_f <= 1e-3
    # the same job alone: bitwise identical to its result inside the mix
    rc1, out1, frc1, _ = _batch(F, [m], [h], [draws[2]], max_newton=200, engine=engine)
    assert rc1 == 0
    assert np.array_equal(out1[0], out[3]) and np.array_equal(frc1[0], frc[3])
    # every draw certified by the oracle's own FP64 residual
    for k, d in enumerate(draws):
        rn, scale, _ = Problem(m, d).residual_norm(out[k + 1], d.n_steps)
        assert rn <= 1e-6 * scale, (k, rn, scale)
    F.fem_destroy_mesh(h)


@pytest.mark.parametrize("engine", ENGINES)
def test_batch_uneven_meshes(F, engine):
    jobs = W.uneven_fingertips(3, seed=5, tet_min=4e3, tet_max=2e4)
    meshes = [m for m, _ in jobs]
    inds = [d for _, d in jobs]
    handles = [F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes) for m in meshes]
    rc, out, frc, st = _batch(F, meshes, handles, inds, max_newton=200, engine=engine)
    assert rc == 0, [s.status for s in st]
    for k, (m, d) in enumerate(jobs):
        rn, scale, _ = Problem(m, d).residual_norm(out[k], d.n_steps)
        assert rn <= 1e-6 * scale
    if engine == (1, 0):
        # size classes: each solve's partition comes from its own mesh, so a
        # solve alone gives bitwise its result in the uneven mix
        for k in range(len(jobs)):
            rc1, o1, f1, _ = _batch(F, [meshes[k]], [handles[k]], [inds[k]], max_newton=200, engine=engine)
            assert rc1 == 0 and np.array_equal(o1[0], out[k]) and np.array_equal(f1[0], frc[k]), k
    for h in handles:
        F.fem_destroy_mesh(h)


@pytest.mark.parametrize("engine", ENGINES)
def test_batch_plan_replays_captured_graph(F, engine):
    """A plan captures the batch once as a CUDA graph; every run replays it
    with new indenters and gives bitwise the results of a one-shot batch."""
    import dataclasses
    m, _ = W.cube_sphere()
    h = F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes)
    inds_all = []
    for r, d, dx, dy in ((0.25, 0.04, 0.0, 0.0), (0.3, 0.05, 0.1, -0.05), (0.35, 0.03, -0.1, 0.1),
                         (0.3, 0.06, 0.05, 0.05)):
        base = W.cube_sphere_indenter(radius=r, depth=d, n_steps=10)
        inds_all.append(dataclasses.replace(base, origin=base.origin + np.array([dx, dy, 0.0])))
    opt = F.fem_default_options()
    opt.batch_engine, opt.batch_parts = engine
    plan = F.FemBatch([h] * 4, [10] * 4, opt)
    info = plan.info()
    assert info.graph == 1 and info.slots >= 1 and info.parts >= 1
    for order in ([0, 1, 2, 3], [3, 2, 1, 0]):
        inds = [inds_all[k] for k in order]
        out = [np.zeros((m.n_nodes, 3)) for _ in inds]
        frc = [np.zeros((10, 3)) for _ in inds]
        rc, st = plan.run(inds, 1e-6, out, frc)
        assert rc == 0 and all(x.steps_done == 10 for x in st)
        rc2, ref, ref_f, _ = _batch(F, [m] * 4, [h] * 4, inds, engine=engine)
        assert rc2 == 0
        for k in range(4):
            assert np.array_equal(out[k], ref[k]) and np.array_equal(frc[k], ref_f[k]), (order, k)
    plan.close()
    F.fem_destroy_mesh(h)


def test_result_independent_of_the_launch_layout(F):
    """A job's shared-memory layout (chunk size, placement) is planned for the
    whole launch: the cube alone and next to a fingertip runs under different
    layouts. The node sums walk each node's list in the same order whatever
    the chunking, so the cube gives the same bits in both launches."""
    cube, cind = W.cube_sphere()
    tip, tind = W.fingertip_sphere()
    hc = F.fem_create_mesh(cube.nodes, cube.tets, cube.tet_material, cube.materials, cube.fixed_nodes)
    ht = F.fem_create_mesh(tip.nodes, tip.tets, tip.tet_material, tip.materials, tip.fixed_nodes)
    opt = F.fem_default_options()
    opt.batch_engine, opt.batch_parts = F.FEM_BATCH_GROUPS, 0
    alone = F.FemBatch([hc], [cind.n_steps], opt)
    mixed = F.FemBatch([hc, ht], [cind.n_steps, tind.n_steps], opt)
    ia, im = alone.info(), mixed.info()
    print(f"alone: smem {ia.smem_bytes} B, mixed: smem {im.smem_bytes} B, global/CTA {im.global_bytes_per_cta} B")
    assert ia.smem_bytes != im.smem_bytes
    oa = [np.zeros((cube.n_nodes, 3))]
    fa = [np.zeros((cind.n_steps, 3))]
    om = [np.zeros((cube.n_nodes, 3)), np.zeros((tip.n_nodes, 3))]
    fm = [np.zeros((cind.n_steps, 3)), np.zeros((tind.n_steps, 3))]
    rc, _ = alone.run([cind], 1e-6, oa, fa)
    assert rc == 0
    rc, st = mixed.run([cind, tind], 1e-6, om, fm)
    assert rc == 0
    assert np.array_equal(oa[0], om[0]) and np.array_equal(fa[0], fm[0])
    alone.close()
    mixed.close()
    F.fem_destroy_mesh(hc)
    F.fem_destroy_mesh(ht)
