"""The FEM_CHECKED build: the same kernels with every index they read from the
mesh's device arrays bounded and the element forces and stored tangents
checked for NaN/Inf (a stand-in for a memory checker). On valid inputs it must
report a clean check word and give the production results; a NaN displacement
handed to the FP64 evaluation must come back as FEM_ERR_CHECK naming the
non-finite check, with the context still usable.

The checked library is built on first use (nvcc, about a minute) and loaded in
a child process (FEM_B300_CHECKED=1), since a process loads one build."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np
sys.path.insert(0, ".")
import workloads as W
from oracle import Problem
import paper_2103_16747_b300 as F

out = {"checked": F.fem_build_checked()}

def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

# one tet, six tets (one Kuhn-split hex), the cube: solves against the oracle
one = W.Mesh(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0.3, 0.25, 0.9]], dtype=float),
             np.array([[0, 1, 2, 3]], dtype=np.int32), np.zeros(1, dtype=np.int32),
             np.array([[1000.0, 0.3]]), np.array([0, 1, 2], dtype=np.int32))
six = W.cube_mesh(1)
cases = {"one_tet": (one, W.plane_indenter(0.9, 0.2, 3), 50.0),
         "six_tets": (six, W.plane_indenter(1.0, 0.05, 3), 100.0),
         "cube": W.cube_sphere() + (100.0,)}
for name, (m, ind, ck) in cases.items():
    s = F.IndentationSolver(m)
    s.set_indenter(ind)
    opt = F.fem_default_options()
    opt.c_kappa = ck
    r = s.solve(1e-8 if name != "cube" else 1e-6, opt, check=False)
    ref = Problem(m, ind, c_kappa=ck).solve(tol=1e-12 if name == "one_tet" else 1e-10)
    assert ref.converged, name
    out[name] = {"rc": int(r["rc"]), "rel_u": rel(r["u"], ref.u), "msg": F.fem_last_error()}
    s.close()
# both batched engines on two cube jobs
m, ind = W.cube_sphere()
h = F.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes)
ref = Problem(m, ind).solve(tol=1e-10)
for eng in (1, 2):
    opt = F.fem_default_options()
    opt.batch_engine = eng
    u = [np.zeros((m.n_nodes, 3)) for _ in range(2)]
    rc, _ = F.fem_solve_batch([h, h], [ind, ind], 1e-6, opt, u, check=False)
    out[f"batch_engine_{eng}"] = {"rc": int(rc), "rel_u": max(rel(x, ref.u) for x in u), "msg": F.fem_last_error()}
F.fem_destroy_mesh(h)
# fingertip: FP64 residual and tangent product on a valid state
m, ind = W.fingertip_sphere()
s = F.IndentationSolver(m)
s.set_indenter(ind)
u = 0.02 * np.random.default_rng(5).standard_normal((m.n_nodes, 3))
u[m.fixed_nodes] = 0.0
R, fc, e = s.eval_residual(u, 20)
g, _ = Problem(m, ind).gradient(u, 20)
y = s.apply_tangent(u, 20, np.ones((m.n_nodes, 3)))
out["fingertip_eval"] = {"rel_R": rel(R, g), "finite_y": bool(np.isfinite(y).all())}
# a NaN displacement: the kernel's non-finite check fires
u[17, 1] = np.nan
try:
    s.eval_residual(u, 20)
    out["nan"] = {"rc": 0, "msg": ""}
except F.FemError as err:
    out["nan"] = {"rc": int(err.code), "msg": F.fem_last_error()}
# the context is still usable and the word was cleared
u[17, 1] = 0.0
R2, _, _ = s.eval_residual(u, 20)
out["after_nan"] = {"rel_R": rel(R2, Problem(m, ind).gradient(u, 20)[0])}
s.close()
print("RESULT " + json.dumps(out))
'''


@pytest.fixture(scope="module")
def checked_lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import importlib.util
    spec = importlib.util.spec_from_file_location("fem_b300_build", os.path.join(ROOT, "paper_2103_16747_b300",
                                                                                   "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build(checked=True)


def test_production_build_is_not_the_checked_one():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2103_16747_b300 as F
    assert F.fem_build_checked() == 0


def test_checked_build_is_clean_on_valid_inputs_and_flags_nan(checked_lib):
    env = dict(os.environ, FEM_B300_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("RESULT ")][-1]
    out = json.loads(line[len("RESULT "):])
    print(json.dumps(out, indent=1))
    assert out["checked"] == 1
    for name in ("one_tet", "six_tets", "cube", "batch_engine_1", "batch_engine_2"):
        assert out[name]["rc"] == 0, (name, out[name]["msg"])
        assert out[name]["rel_u"] <= 1e-4, name
    assert out["fingertip_eval"]["rel_R"] < 1e-10 and out["fingertip_eval"]["finite_y"]
    assert out["nan"]["rc"] == -10 and "non-finite" in out["nan"]["msg"], out["nan"]
    assert out["after_nan"]["rel_R"] < 1e-10
