"""Request server (continuous batching) on the GPU: a request's result is
bitwise the same alone and inside a burst of mixed requests (also when it is
suspended for a change of launch shape and resumed), matches the FP64 oracle, and
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


def _batch_reference(F, mesh, handle, draws, opt, parts):
    """The batched group engine on one mesh cut into `parts` parts: the same
    partition and kernel as the server's large-mesh group."""
    bo = F.fem_options.from_buffer_copy(opt)
    bo.batch_engine, bo.batch_parts = 1, parts
    out = []
    for d in draws:
        u = [np.zeros((mesh.n_nodes, 3))]
        f = [np.zeros((d.n_steps, 3))]
        rc, _ = F.fem_solve_batch([handle], [d], 1e-6, bo, u, f, check=False)
        out.append((rc, u[0], f[0]))
    return out


def test_server_large_meshes_in_their_own_launch_shape(F):
    """Meshes too large for a 64-CTA class (here: more than 64 x 100 tets)
    are served by other launch shapes of the persistent kernel: the large
    ones (parts of at most 100 tets on the SMs the largest class leaves) by
    one group beside that class's groups, the huge ones by one group of every
    SM. A large or huge request's result equals the batched engine's on the
    same number of parts, a small one's result equals the same request served
    alone."""
    cube, cube_ind = W.cube_sphere()
    pool = [cube] + [m for m, _ in W.uneven_fingertips(3, seed=21, tet_min=6.6e3, tet_max=1.2e4)]
    assert all(m.n_tets > 6400 for m in pool[1:])
    handles = [F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes) for m in pool]
    draws = {k: W.draw_indentations(pool[k], 2, seed=300 + k) for k in range(1, len(pool))}
    opt = F.fem_default_options()
    opt.max_newton = 200
    opt.batch_tets_per_cta = 100
    srv = F.FemServer(handles, 20, opt, result_bytes=32 << 20)
    info = srv.info()
    assert info.n_shapes == 3 and info.large_class >= 0 and info.huge_class >= 0
    lc, hc = info.large_class, info.huge_class
    p_large, p_huge = info.class_parts[lc], info.class_parts[hc]
    assert p_large * 100 < 9216 and p_large * 100 >= 8208
    assert info.class_groups[lc] == 0 and info.shape_groups[1][lc] == 1 and info.shape_groups[2][hc] == 1
    assert info.shape_ctas[1] == p_large + sum(info.class_parts[c] * info.shape_groups[1][c] for c in range(lc))
    assert info.shape_ctas[2] == p_huge
    parts_of = {k: (p_huge if pool[k].n_tets > p_large * 100 else p_large) for k in range(1, len(pool))}
    ref = {}
    for k in range(1, len(pool)):
        for j, r in enumerate(_batch_reference(F, pool[k], handles[k], draws[k], opt, parts_of[k])):
            ref[(k, j)] = r
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
    info = srv.info()
    print(f"launches {info.launches}, suspended {info.suspended}, parts large {p_large} huge {p_huge}")
    assert info.launches >= 3
    assert srv.stop() == 0
    srv.close()
    for h in handles:
        F.fem_destroy_mesh(h)


def test_running_solves_yield_to_the_large_mesh_shape(F):
    """A change of launch shape waits one load step, not the rest of the
    running solves: they leave between load steps and resume in the next
    launch from their own state. A short request A (4 load steps) and a long
    one C run on the two groups of the fingertip's class, and a huge request B
    that arrived between them asks for the other shape: when A is done, B is
    older than C, so C leaves mid-solve and resumes after B. Each request
    gives bitwise the result it gives served alone, B bitwise that of the
    batched engine on the huge-mesh group's part count."""
    import dataclasses
    import time
    tip, tip_ind = W.fingertip_sphere()
    big = W.fingertip_mesh(R=8.0, h=0.75)       # 81,408 tets: beyond 64 x 700
    pool = [tip, big]
    assert big.n_tets > 64 * 700 > tip.n_tets
    handles = [F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes) for m in pool]
    d_a, d_c = W.draw_indentations(tip, 2, seed=411)
    d_a = dataclasses.replace(d_a, depth_schedule=d_a.depth_schedule[:4].copy())
    big_ind = W.draw_indentations(big, 1, seed=412)[0]
    opt = F.fem_default_options()
    opt.max_newton = 400
    opt.batch_tets_per_cta = 700
    srv = F.FemServer(handles, 20, opt, result_bytes=256 << 20)
    info = srv.info()
    big_class = max(info.large_class, info.huge_class)
    assert info.n_shapes == 2 and big_class == 1 and info.class_groups[0] == 2
    ref_big = _batch_reference(F, big, handles[1], [big_ind], opt, info.class_parts[big_class])[0]
    srv.start(300.0)
    alone = []
    for d in (d_a, d_c):
        rc, rid = srv.submit(0, d, 1e-6)
        assert rc == 0
        alone.append(srv.result(rid, tip.n_nodes, d.n_steps, wait_ms=200000))
    assert srv.info().suspended == 0
    launches0 = srv.info().launches
    rc, rid_a = srv.submit(0, d_a, 1e-6)
    time.sleep(0.005)
    rc, rid_big = srv.submit(1, big_ind, 1e-6)
    rc, rid_c = srv.submit(0, d_c, 1e-6)
    assert rc == 0
    for rid, d, a in ((rid_a, d_a, alone[0]), (rid_c, d_c, alone[1])):
        r = srv.result(rid, tip.n_nodes, d.n_steps, wait_ms=200000)
        assert r[0] == a[0] and np.array_equal(r[1], a[1]) and np.array_equal(r[2], a[2])
    rb = srv.result(rid_big, big.n_nodes, 20, wait_ms=200000)
    assert rb[0] == ref_big[0] and np.array_equal(rb[1], ref_big[1])
    assert np.array_equal(rb[2], ref_big[2])
    info = srv.info()
    print(f"suspended solves: {info.suspended}, launches {info.launches - launches0}")
    assert info.suspended >= 1
    assert info.launches - launches0 >= 2
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


def test_stop_while_shapes_change_returns_every_request(F):
    """Stop while the server changes launch shapes (large, huge and small
    requests interleaved, so solves are being suspended and resumed): stop
    returns, every request comes back finished or FEM_ERR_TIMEOUT (not run, or
    suspended when the session closed), none stays pending, and a finished
    small request equals the same request served alone."""
    import time
    cube, cube_ind = W.cube_sphere()
    pool = [cube] + [m for m, _ in W.uneven_fingertips(3, seed=21, tet_min=6.6e3, tet_max=1.2e4)]
    handles = [F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes) for m in pool]
    draws = {k: W.draw_indentations(pool[k], 2, seed=500 + k) for k in range(1, len(pool))}
    opt = F.fem_default_options()
    opt.max_newton = 200
    opt.batch_tets_per_cta = 100
    srv = F.FemServer(handles, 20, opt, result_bytes=32 << 20)
    assert srv.info().n_shapes == 3
    srv.start(120.0)
    rc, rid = srv.submit(0, cube_ind, 1e-6)
    alone = srv.result(rid, cube.n_nodes, 10, wait_ms=100000)
    assert alone[0] == 0
    launches0 = srv.info().launches
    ids = []
    for rep in range(3):
        for k in range(1, len(pool)):
            for d in draws[k]:
                rc, rid = srv.submit(k, d, 1e-6)
                assert rc == 0
                ids.append((rid, k))
        rc, rid = srv.submit(0, cube_ind, 1e-6)
        assert rc == 0
        ids.append((rid, 0))
    time.sleep(0.3)
    t0 = time.perf_counter()
    assert srv.stop() == 0
    assert time.perf_counter() - t0 < 60.0
    seen = {}
    for rid, k in ids:
        n_steps = 10 if k == 0 else 20
        r = srv.result(rid, pool[k].n_nodes, n_steps, wait_ms=0)
        assert r[0] in (F.FEM_OK, F.FEM_ERR_NOT_CONVERGED, F.FEM_ERR_TIMEOUT), r[0]
        seen[r[0]] = seen.get(r[0], 0) + 1
        if k == 0 and r[0] == F.FEM_OK:
            assert np.array_equal(r[1], alone[1]) and np.array_equal(r[2], alone[2])
    info = srv.info()
    print(f"statuses {seen}, launches {info.launches - launches0}, suspended {info.suspended}")
    assert info.launches - launches0 >= 2
    rc, _ = srv.submit(0, cube_ind, 1e-6)
    assert rc == F.FEM_ERR_BUSY
    srv.close()
    for h in handles:
        F.fem_destroy_mesh(h)
