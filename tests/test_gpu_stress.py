"""Element stress output on the GPU (Cauchy stress and von Mises per tet,
FP64) against the oracle's definition sigma = P F^T / J, at the fingertip's
solved displacement (large strain) and at a small random displacement."""
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


@pytest.mark.parametrize("state", ["solved", "small"])
def test_element_stress_matches_oracle(F, state):
    m, ind = W.fingertip_sphere()
    if state == "solved":
        u = np.load(os.path.join(HERE, "golden", "fingertip_sphere_oracle.npz"))["u"]
    else:
        rng = np.random.default_rng(8)
        u = 1e-4 * rng.standard_normal((m.n_nodes, 3))
        u[m.fixed_nodes] = 0.0
    p = Problem(m, ind)
    Fd = p.F(u)
    sig_ref = cauchy(Fd, p.mu, p.lam)
    vm_ref = von_mises(sig_ref)
    h = F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes)
    sig, vm = F.fem_element_stress(h, u, m.n_tets)
    F.fem_destroy_mesh(h)
    ref6 = np.stack([sig_ref[:, 0, 0], sig_ref[:, 1, 1], sig_ref[:, 2, 2],
                     sig_ref[:, 1, 2], sig_ref[:, 0, 2], sig_ref[:, 0, 1]], axis=1)
    scale = np.abs(ref6).max()
    err = np.abs(sig - ref6).max() / scale
    print(f"{state}: max |sigma| {scale:.3e}, max rel err {err:.2e}, max von Mises {vm_ref.max():.3e}")
    assert err <= 1e-9
    assert np.abs(vm - vm_ref).max() <= 1e-9 * vm_ref.max()
