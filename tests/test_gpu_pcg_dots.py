"""The PCG's dot-product reductions against exactly rounded sums.

The PCG holds its vectors in FP32 and forms (r,u), (w,u) and (r,r) with
error-free FP32 products (product plus its fma-computed rounding error) summed
in compensated FP32 pairs per thread, per CTA and over the CTAs. Each
compensated addition is exact up to about 2^-44 of the magnitudes involved, and
a sum passes through fewer than 48 of them (per thread, shuffle tree, warps,
CTA slots), so

    |dot_gpu - dot_exact| <= 48 * 2^-44 * sum_i |a_i b_i|  (< 3e-12 sum |a_i b_i|),

where dot_exact is the correctly rounded sum of the exact products of the
FP32-rounded vectors (math.fsum over FP64 products, which are exact for FP32
factors). Plain FP32 accumulation misses that bound by orders of magnitude on
the same vectors, so the bound tells the two apart."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import Problem

pytestmark = pytest.mark.gpu
BOUND = 48 * 2.0 ** -44


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2103_16747_b300 as F
    return F


def _exact(a, b):
    return math.fsum((a * b).tolist())


def _fp32_naive(a, b):
    acc = np.float32(0.0)
    for x, y in zip(a.astype(np.float32), b.astype(np.float32)):
        acc = np.float32(acc + x * y)
    return float(acc)


@pytest.mark.parametrize("workload", ["cube", "fingertip"])
def test_pcg_dots_meet_the_compensated_bound(F, workload):
    m, ind = W.cube_sphere() if workload == "cube" else W.fingertip_sphere()
    free = Problem(m, ind).free
    rng = np.random.default_rng(31)
    n = 3 * m.n_nodes
    # magnitudes spread over six decades, signs mixed: a hard case for plain sums
    r = rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 3, n)
    u = rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 3, n)
    w = rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 3, n)
    s = F.IndentationSolver(m)
    got = F.fem_debug_pcg_dots(s.handle, r.reshape(-1, 3), u.reshape(-1, 3), w.reshape(-1, 3))
    s.close()
    r32, u32, w32 = (x.astype(np.float32).astype(np.float64) * free for x in (r, u, w))
    worst = 0.0
    for k, (a, b) in enumerate(((r32, u32), (w32, u32), (r32, r32))):
        ref = _exact(a, b)
        mag = math.fsum(np.abs(a * b).tolist())
        err = abs(got[k] - ref)
        worst = max(worst, err / mag)
        assert err <= BOUND * mag, (k, got[k], ref, err / mag)
        if k == 2:
            assert abs(got[k] / ref - 1.0) <= BOUND
    # plain FP32 accumulation of the same (r,u) is far outside the bound
    naive = _fp32_naive(r32[free], u32[free])
    ref = _exact(r32, u32)
    mag = math.fsum(np.abs(r32 * u32).tolist())
    print(f"{workload}: worst compensated error {worst:.2e} of sum|ab|; plain FP32 {abs(naive - ref) / mag:.2e}")
    assert abs(naive - ref) > 100 * BOUND * mag
