"""The allocation-free residual entry point, for callers that may not allocate
device memory while running (e.g. a control loop with a no-allocation rule after
start-up): it must give the same results as fem_eval_residual, call after call,
while reusing the library's fixed device scratch block.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

import workloads as W

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
    s.close()
