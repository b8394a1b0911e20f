"""The allocation-free residual entry point, for callers that may not allocate
device memory while running (e.g. a control loop with a no-allocation rule after
start-up): it must give the same results as fem_eval_residual and as the FP64
oracle, call after call, while reusing the library's fixed device scratch block
and allocating nothing; a mesh too large for the block is refused with its sizes.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test."""
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("workload", ["cube", "fingertip"])
def test_noalloc_residual_matches_regular_entry_point(F, workload):
    rng = np.random.default_rng(17)
    if workload == "cube":
        mesh, ind = W.cube_sphere()
        scale, step = 0.002, 10
    else:
        mesh, ind = W.fingertip_sphere()
        scale, step = 0.02, 20
    s = F.IndentationSolver(mesh)
    s.set_indenter(ind)
    p = Problem(mesh, ind)
    n = mesh.n_nodes
    for call in range(2):                      # two calls in a row share the scratch block
        u = scale * rng.standard_normal((n, 3))
        u[mesh.fixed_nodes] = 0.0
        R_ref = np.zeros((n, 3))
        fc_ref = np.zeros((n, 3))
        e_ref = F.fem_eval_residual(s.handle, u, step, None, R_ref, fc_ref)
        R = np.full((n, 3), np.nan)
        fc = np.full((n, 3), np.nan)
        e = F.fem_eval_residual_noalloc(s.handle, u, step, None, R, fc)
        assert _rel(R, R_ref) <= 1e-10, call
        assert _rel(fc, fc_ref) <= 1e-10, call
        assert e[0] == pytest.approx(e_ref[0], rel=1e-10)
        assert e[1] == pytest.approx(e_ref[1], rel=1e-10, abs=1e-300)
        # and against the FP64 oracle directly
        g, fco = p.gradient(u, step)
        assert _rel(R, g) <= 1e-10, call
        assert _rel(fc, fco) <= 1e-10, call
        assert e[0] == pytest.approx(p.elastic_energy(u)[0], rel=1e-11)
    s.close()


def test_noalloc_calls_allocate_no_device_memory(F):
    """After one warm-up call (which looks up the block's address), further
    calls leave the device's free memory unchanged: the entry point allocates
    nothing."""
    import torch
    mesh, ind = W.cube_sphere()
    s = F.IndentationSolver(mesh)
    s.set_indenter(ind)
    n = mesh.n_nodes
    u = 0.002 * np.random.default_rng(3).standard_normal((n, 3))
    u[mesh.fixed_nodes] = 0.0
    R = np.zeros((n, 3))
    F.fem_eval_residual_noalloc(s.handle, u, 10, None, R, None)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    R2 = np.zeros((n, 3))
    for _ in range(5):
        F.fem_eval_residual_noalloc(s.handle, u, 10, None, R2, None)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert np.array_equal(R, R2)
    s.close()


def test_noalloc_refuses_a_mesh_beyond_the_block(F):
    """A cube of 46^3 = 97,336 nodes needs more than the fixed block: the call
    returns FEM_ERR_TOO_LARGE with the sizes and the node limit in the message
    and writes nothing."""
    mesh = W.cube_mesh(45)
    assert mesh.n_nodes == 97336
    s = F.IndentationSolver(mesh)
    s.set_indenter(W.cube_sphere_indenter())
    R = np.full((mesh.n_nodes, 3), 7.0)
    with pytest.raises(F.FemError) as ei:
        F.fem_eval_residual_noalloc(s.handle, np.zeros((mesh.n_nodes, 3)), 1, None, R, None)
    assert ei.value.code == F.FEM_ERR_TOO_LARGE
    msg = F.fem_last_error()
    assert "97336 nodes" in msg and "at most" in msg, msg
    assert np.all(R == 7.0)
    s.close()
