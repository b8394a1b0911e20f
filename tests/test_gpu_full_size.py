"""Parity at full size, in the launch configurations the benchmarks time: the
256 random fingertip indentations of the batched workload (groups of 37 CTAs),
the three largest meshes of the 64-mesh uneven workload (175k-186k tets, the
largest the benchmarks run; size classes at 1,000 tets per CTA, which puts each
of them on every SM) also on the single-solve path, and the request server on
the serving workload's 16-mesh pool in all three launch shapes. The oracle cannot
solve all of these in test time, so each answer is checked through properties
that hold at any size: the oracle's own FP64 residual at the GPU displacement
is within the solve tolerance of its scale at the last load step, and the
GPU's last-step resultant contact force equals the oracle's resultant
(Sec. III-A: nodal contact forces summed) at that displacement."""
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


@pytest.fixture(scope="module")
def largest():
    jobs = W.uneven_fingertips(64, seed=1003)
    order = np.argsort([-m.n_tets for m, _ in jobs])[:3]
    return [jobs[k] for k in order]


def _certify(m, d, u, force):
    p = Problem(m, d)
    rn, scale, _ = p.residual_norm(u, d.n_steps)
    assert rn <= 1e-6 * scale, (rn, scale)
    _, fc = p.gradient(u, d.n_steps)
    ref = fc.sum(axis=0)
    assert np.linalg.norm(force - ref) <= 1e-8 * np.linalg.norm(ref), (force, ref)


def test_largest_uneven_meshes_batched_and_single(F, largest):
    assert min(m.n_tets for m, _ in largest) > 170000
    meshes = [m for m, _ in largest]
    inds = [d for _, d in largest]
    handles = [F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes) for m in meshes]
    opt = F.fem_default_options()
    opt.max_newton = 400
    opt.batch_engine, opt.batch_parts, opt.batch_tets_per_cta = 1, 0, 1000
    out = [np.zeros((m.n_nodes, 3)) for m in meshes]
    frc = [np.zeros((d.n_steps, 3)) for d in inds]
    rc, st = F.fem_solve_batch(handles, inds, 1e-6, opt, out, frc, check=False)
    assert rc == 0, [s.status for s in st]
    for k, (m, d) in enumerate(largest):
        assert st[k].steps_done == d.n_steps and st[k].residual <= 1e-6 * st[k].scale
        _certify(m, d, out[k], frc[k][-1])
    # the single-solve path on the same meshes (its own partition of 148 parts)
    for k, (m, d) in enumerate(largest):
        F.fem_set_indenter(handles[k], d.shape, d.pose, np.asarray(d.params), d.direction, d.depth_schedule)
        u = np.zeros((m.n_nodes, 3))
        f = np.zeros((d.n_steps, 3))
        rc1, s1 = F.fem_solve(handles[k], d.n_steps, 1e-6, opt, u, f, None, check=False)
        assert rc1 == 0 and s1.steps_done == d.n_steps
        _certify(m, d, u, f[-1])
        # two converged answers of the same problem: within the conditioning
        # of the tangent times the residual tolerance of each other
        assert np.linalg.norm(u - out[k]) <= 1e-3 * np.linalg.norm(out[k])
    for h in handles:
        F.fem_destroy_mesh(h)


def test_fingertip_256_draws_in_the_benchmark_slot_shape(F):
    """The 256 random indentations of the batched fingertip workload, in the
    slot shape its benchmark times (groups of 37 CTAs, FP32 tangent, at most
    400 Newton iterations per load step): every solve converges, every 8th
    draw and the two hardest (62, 176) are certified by the oracle's residual
    and resultant force, and a draw alone gives bitwise its result in the
    256-solve mix."""
    m, _ = W.fingertip_sphere()
    draws = W.draw_indentations(m, 256, seed=1002)
    h = F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes)
    opt = F.fem_default_options()
    opt.max_newton = 400
    opt.batch_engine, opt.batch_parts = 1, 37
    out = [np.zeros((m.n_nodes, 3)) for _ in draws]
    frc = [np.zeros((d.n_steps, 3)) for d in draws]
    rc, st = F.fem_solve_batch([h] * len(draws), draws, 1e-6, opt, out, frc, check=False)
    assert rc == 0, [k for k, s in enumerate(st) if s.status != 0]
    assert all(s.steps_done == 20 and s.residual <= 1e-6 * s.scale for s in st)
    for k in sorted(set(range(0, 256, 8)) | {62, 176}):
        _certify(m, draws[k], out[k], frc[k][-1])
    u1 = [np.zeros((m.n_nodes, 3))]
    f1 = [np.zeros((20, 3))]
    rc1, _ = F.fem_solve_batch([h], [draws[62]], 1e-6, opt, u1, f1, check=False)
    assert rc1 == 0 and np.array_equal(u1[0], out[62]) and np.array_equal(f1[0], frc[62])
    F.fem_destroy_mesh(h)


def test_request_server_on_the_serving_pool(F):
    """The request server on the serving workload's pool (16 fingertips of
    6k-168k tets, the default 1,300 tets per CTA: size classes, the large-mesh
    group beside the 64-CTA class, and the whole-GPU group for the largest),
    one request per mesh submitted at once: every result converges and is
    certified by the oracle's residual and resultant force."""
    jobs = W.uneven_fingertips(16, seed=1004)
    pool = [m for m, _ in jobs]
    handles = [F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes) for m in pool]
    opt = F.fem_default_options()
    opt.max_newton = 400
    srv = F.FemServer(handles, 20, opt, result_bytes=1 << 30)
    info = srv.info()
    assert info.n_shapes == 3
    draws = [W.draw_indentations(m, 4, seed=2000 + k)[0] for k, m in enumerate(pool)]
    srv.start(300.0)
    ids = []
    for k, d in enumerate(draws):
        rc, rid = srv.submit(k, d, 1e-6)
        assert rc == 0
        ids.append(rid)
    for k, rid in enumerate(ids):
        rc, u, f, st, _ = srv.result(rid, pool[k].n_nodes, 20, wait_ms=200000)
        assert rc == 0 and st.steps_done == 20, (k, rc)
        _certify(pool[k], draws[k], u, f[-1])
    assert srv.stop() == 0
    srv.close()
    for h in handles:
        F.fem_destroy_mesh(h)
