"""Request server (continuous batching) on the GPU: a request's result is
bitwise the same alone and inside a burst of mixed requests (also when it is
suspended for a whole-GPU pass and resumed), matches the FP64 oracle, and
requests submitted after stop are rejected."""
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


def test_server_alone_equals_mix_and_matches_oracle(F):
    cube, cube_ind = W.cube_sphere()
    pool = [cube] + [m for m, _ in W.uneven_fingertips(3, seed=21, tet_min=4e3, tet_max=2e4)]
    handles = [F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes) for m in pool]
    draws = {k: W.draw_indentations(pool[k], 3, seed=100 + k) for k in range(1, len(pool))}
    opt = F.fem_default_options()
    opt.max_newton = 200
    srv = F.FemServer(handles, 20, opt, result_bytes=64 << 20)
    info = srv.info()
    assert info.n_ctas >= 1 and info.result_slots >= 1
    srv.start(120.0)

    def wait(rid, k, n_steps):
        rc, u, f, st, t = srv.result(rid, pool[k].n_nodes, n_steps, wait_ms=100000)
        assert rc != F.FEM_PENDING
        return rc, u, f, st, t

    # alone
    rc, rid = srv.submit(2, draws[2][0], 1e-6)
    assert rc == 0
    rc_a, u_a, f_a, st_a, _ = wait(rid, 2, 20)
    # a deep random draw may exhaust max_newton: the comparison below holds
    # for whatever the solver reached
    assert rc_a in (F.FEM_OK, F.FEM_ERR_NOT_CONVERGED)
    # a burst over the whole pool, the same request among them
    burst = [(0, cube_ind)] + [(k, d) for k in range(1, len(pool)) for d in draws[k]]
    ids = []
    for k, d in burst:
        rc, rid = srv.submit(k, d, 1e-6)
        assert rc == 0
        ids.append((rid, k, d))
    res = [wait(rid, k, d.n_steps) for rid, k, d in ids]
    for (rid, k, d), r in zip(ids, res):
        assert r[0] in (F.FEM_OK, F.FEM_ERR_NOT_CONVERGED), (k, r[0])
    assert res[0][0] == F.FEM_OK and sum(r[0] == F.FEM_OK for r in res) >= len(res) - 2
    j = [i for i, (_, k, d) in enumerate(ids) if k == 2 and d is draws[2][0]][0]
    assert res[j][0] == rc_a and np.array_equal(res[j][1], u_a) and np.array_equal(res[j][2], f_a)
    # the cube request against the oracle
    ref = Problem(cube, cube_ind).solve(tol=1e-10)
    u0, f0 = res[0][1], res[0][2]
    assert np.linalg.norm(u0 - ref.u) / np.linalg.norm(ref.u) <= 1e-4
    assert np.linalg.norm(f0[-1] - ref.step_force[-1]) / np.linalg.norm(ref.step_force[-1]) <= 1e-3
    # every converged fingertip request certified by the oracle's FP64 residual
    for (rid, k, d), r in zip(ids[1:], res[1:]):
        if r[0] == F.FEM_OK:
            rn, scale, _ = Problem(pool[k], d).residual_norm(r[1], d.n_steps)
            assert rn <= 1e-6 * scale
    assert srv.stop() == 0
    rc, _ = srv.submit(0, cube_ind, 1e-6)
    assert rc == F.FEM_ERR_BUSY
    info = srv.info()
    assert info.completed == 1 + len(burst) and info.admitted == info.completed
    srv.close()
    for h in handles:
        F.fem_destroy_mesh(h)


def test_server_whole_gpu_passes_for_large_meshes(F):
    """Meshes too large for a 64-CTA class (here: more than 64 x 100 tets)
    are served in whole-GPU passes between runs of the persistent launch: a
    large request's result equals a direct fem_solve, a small one's result
    equals the same request served alone."""
    cube, cube_ind = W.cube_sphere()
    pool = [cube] + [m for m, _ in W.uneven_fingertips(2, seed=21, tet_min=8e3, tet_max=1.2e4)]
    assert all(m.n_tets > 6400 for m in pool[1:])
    handles = [F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes) for m in pool]
    draws = {k: W.draw_indentations(pool[k], 2, seed=300 + k) for k in range(1, len(pool))}
    opt = F.fem_default_options()
    opt.max_newton = 200
    opt.batch_tets_per_cta = 100
    # direct single solves of the large requests (reference)
    ref = {}
    for k in range(1, len(pool)):
        for j, d in enumerate(draws[k]):
            s = F.IndentationSolver(pool[k])
            s.set_indenter(d)
            r = s.solve(1e-6, opt, check=False)
            ref[(k, j)] = (r["rc"], r["u"], r["step_force"])
            s.close()
    srv = F.FemServer(handles, 20, opt, result_bytes=32 << 20)
    srv.start(120.0)
    rc, rid = srv.submit(0, cube_ind, 1e-6)
    alone = srv.result(rid, cube.n_nodes, 10, wait_ms=100000)
    assert alone[0] == 0
    ids = []
    for rep in range(2):
        rc, rid = srv.submit(0, cube_ind, 1e-6)
        ids.append((rid, 0, None))
        for k in range(1, len(pool)):
            for j, d in enumerate(draws[k]):
                rc, rid = srv.submit(k, d, 1e-6)
                assert rc == 0
                ids.append((rid, k, j))
    for rid, k, j in ids:
        n_steps = 10 if k == 0 else 20
        r = srv.result(rid, pool[k].n_nodes, n_steps, wait_ms=100000)
        assert r[0] != F.FEM_PENDING
        if k == 0:
            assert r[0] == 0 and np.array_equal(r[1], alone[1]) and np.array_equal(r[2], alone[2])
        else:
            rc_ref, u_ref, f_ref = ref[(k, j)]
            assert r[0] == rc_ref and np.array_equal(r[1], u_ref) and np.array_equal(r[2], f_ref), (k, j)
    assert srv.stop() == 0
    srv.close()
    for h in handles:
        F.fem_destroy_mesh(h)


def test_running_solves_yield_to_a_whole_gpu_pass(F):
    """A whole-GPU pass waits one load step, not the rest of the running
    solves: they leave between load steps and resume after the pass from their
    own state. Each resumed request gives bitwise the result it gives served
    alone, the large request bitwise that of a direct fem_solve."""
    tip, tip_ind = W.fingertip_sphere()
    big = W.fingertip_mesh(R=8.0, h=0.75)       # 81,408 tets: beyond 64 x 700
    pool = [tip, big]
    assert big.n_tets > 64 * 700 > tip.n_tets
    handles = [F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes) for m in pool]
    small = W.draw_indentations(tip, 4, seed=411)
    big_ind = W.draw_indentations(big, 1, seed=412)[0]
    opt = F.fem_default_options()
    opt.max_newton = 400
    opt.batch_tets_per_cta = 700
    s = F.IndentationSolver(big)
    s.set_indenter(big_ind)
    ref_big = s.solve(1e-6, opt, check=False)
    s.close()
    srv = F.FemServer(handles, 20, opt, result_bytes=256 << 20)
    srv.start(300.0)
    alone = []
    for d in small:
        rc, rid = srv.submit(0, d, 1e-6)
        assert rc == 0
        alone.append(srv.result(rid, tip.n_nodes, 20, wait_ms=200000))
    assert srv.info().suspended == 0
    # the small requests start, then the large one arrives while they run
    ids = []
    for d in small:
        rc, rid = srv.submit(0, d, 1e-6)
        assert rc == 0
        ids.append(rid)
    import time
    time.sleep(0.02)
    rc, rid_big = srv.submit(1, big_ind, 1e-6)
    assert rc == 0
    for rid, a in zip(ids, alone):
        r = srv.result(rid, tip.n_nodes, 20, wait_ms=200000)
        assert r[0] == a[0] and np.array_equal(r[1], a[1]) and np.array_equal(r[2], a[2])
    rb = srv.result(rid_big, big.n_nodes, 20, wait_ms=200000)
    assert rb[0] == ref_big["rc"] and np.array_equal(rb[1], ref_big["u"])
    assert np.array_equal(rb[2], ref_big["step_force"])
    info = srv.info()
    print(f"suspended solves: {info.suspended}")
    assert info.suspended >= 1
    assert srv.stop() == 0
    srv.close()
    for h in handles:
        F.fem_destroy_mesh(h)


@pytest.mark.parametrize("physics", ["dynamic", "friction", "friction_passes", "corotational"])
def test_server_physics_options_match_oracle(F, physics):
    """The served path runs every physics option: dynamic stepping, Coulomb
    friction (one and several passes per load step) and the co-rotational
    law, each against the FP64 oracle."""
    m, ind = W.cube_sphere()
    opt = F.fem_default_options()
    kw = {}
    if physics == "dynamic":
        opt.dt, opt.density = 1e-3, 1.0
        kw = {"dt": 1e-3, "density": 1.0}
    elif physics in ("friction", "friction_passes"):
        opt.mu_f = 0.783
        kw = {"mu_f": 0.783}
        if physics == "friction_passes":
            opt.friction_passes = 3
            kw["friction_passes"] = 3
    else:
        m = W.with_model(m, 1)
    ref = Problem(m, ind, **kw).solve(tol=1e-10)
    assert ref.converged
    h = F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes)
    srv = F.FemServer([h], ind.n_steps, opt, result_bytes=16 << 20)
    srv.start(60.0)
    rc, rid = srv.submit(0, ind, 1e-6)
    assert rc == 0
    rc, u, f, st, _ = srv.result(rid, m.n_nodes, ind.n_steps, wait_ms=60000)
    assert rc == F.FEM_OK
    assert np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u) <= 1e-4
    k0 = 1 if physics.startswith("friction") else 0
    for k in range(k0, ind.n_steps):
        assert np.linalg.norm(f[k] - ref.step_force[k]) / np.linalg.norm(ref.step_force[k]) <= 1e-3
    assert srv.stop() == 0
    srv.close()
    F.fem_destroy_mesh(h)
