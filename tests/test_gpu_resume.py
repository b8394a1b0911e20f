"""Checkpoint and resume of a solve (fem_solve_range): the state after load step
k is the pair of converged displacements (u_k, u_{k-1}); a solve split into
ranges, each resumed from the state the previous range returned, must give
bitwise the displacements and step forces of one fem_solve: quasi-static on
the fingertip, backward-Euler dynamics (the velocity comes from the state) and
lagged friction (frozen from u_k) on the cube."""
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


def _case(F, name):
    opt = F.fem_default_options()
    if name == "fingertip":
        m, ind = W.fingertip_sphere()
        return m, ind, opt, [8]
    m, ind = W.cube_sphere()
    if name == "dynamic":
        opt.dt, opt.density = 1e-3, 1.0            # inertia comparable to the cube's stiffness
    elif name == "friction":
        opt.mu_f = 0.5
    return m, ind, opt, [3, 7]


@pytest.mark.parametrize("name", ["fingertip", "dynamic", "friction"])
def test_split_solve_is_bitwise_the_full_solve(F, name):
    m, ind, opt, cuts = _case(F, name)
    K = ind.n_steps
    s = F.IndentationSolver(m)
    s.set_indenter(ind)
    full = s.solve(1e-6, opt)
    assert full["rc"] == 0 and full["stats"].steps_done == K
    u = prev = None
    forces = np.zeros((K, 3))
    bounds = [0] + cuts + [K]
    for a, b in zip(bounds[:-1], bounds[1:]):
        out_u = np.zeros((m.n_nodes, 3))
        out_prev = np.zeros((m.n_nodes, 3))
        f = np.zeros((K, 3))
        rc, st = F.fem_solve_range(s.handle, a + 1, b, 1e-6, opt, u, prev, out_u, out_prev, f)
        assert rc == 0 and st.steps_done == b
        assert np.all(f[:a] == 0.0) and np.all(f[b:] == 0.0)
        forces[a:b] = f[a:b]
        assert np.array_equal(st.newton_per_step[a:b], full["stats"].newton_per_step[a:b])
        u, prev = out_u, out_prev
    assert np.array_equal(u, full["u"])
    assert np.array_equal(forces, full["step_force"])
    s.close()


def test_range_arguments_are_checked(F):
    m, ind = W.cube_sphere()
    s = F.IndentationSolver(m)
    s.set_indenter(ind)
    u = np.zeros((m.n_nodes, 3))
    for first, last, u0 in ((0, 3, None), (4, 3, u), (1, 11, None), (2, 5, None)):
        rc, _ = F.fem_solve_range(s.handle, first, last, 1e-6, None, u0, None, u, check=False)
        assert rc == F.FEM_ERR_ARG, (first, last)
    s.close()
