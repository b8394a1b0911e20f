"""CPU-only checks of the C-ABI library: it builds, loads, exports every symbol
include/fem.h declares, and rejects malformed inputs on the host before any
CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    from paper_2103_16747_b300 import _lib
    hdr = open(os.path.join(ROOT, "include", "fem.h")).read()
    declared = set(re.findall(r"^\s*(?:int|void|const char\*)\s+(fem_\w+)\s*\(", hdr, re.M))
    assert declared == set(_lib.EXPORTS)
    raw = ctypes.CDLL(_lib.LIB_PATH)
    for name in declared:
        assert hasattr(raw, name), name


def test_default_options():
    from paper_2103_16747_b300 import _lib as L
    o = L.fem_default_options()
    assert o.c_kappa == 100.0 and o.max_cg == 2000 and o.tangent == L.FEM_TANGENT_ADAPTIVE
    assert o.cg_rtol_max == 0.2 and o.cg_rtol_min == 1e-2
    assert o.batch_engine == L.FEM_BATCH_AUTO and o.batch_parts == 0
    assert o.precond_degree == 5 and o.precond_ratio == 120.0
    assert o.dt == 0.0 and o.density == 1.1e-9
    assert o.mu_f == 0.0 and o.friction_eps == 0.01 and o.friction_passes == 1
    assert o.tangent_fp16 == 0


@pytest.mark.parametrize("field,value", [("batch_engine", 3), ("batch_parts", -1), ("batch_parts", 300),
                                         ("tangent", 7), ("max_cg", 0), ("precond_degree", 0),
                                         ("precond_degree", 9), ("precond_ratio", 1.0),
                                         ("dt", -1e-4), ("dt", float("inf")), ("friction_passes", 0),
                                         ("friction_passes", 65), ("tangent_fp16", 2), ("tangent_fp16", -1)])
def test_batch_options_are_checked_before_any_device_call(field, value):
    """Invalid options are rejected on the host (no mesh is touched)."""
    from paper_2103_16747_b300 import _lib as L
    o = L.fem_default_options()
    setattr(o, field, value)
    ind = W.cube_sphere_indenter()
    rc, _ = L.fem_solve_batch([None], [ind], 1e-6, o, [np.zeros((8, 3))], check=False)
    assert rc == L.FEM_ERR_ARG and "fem_options" in L.fem_last_error()


def test_cluster_engine_takes_powers_of_two_up_to_16():
    from paper_2103_16747_b300 import _lib as L
    o = L.fem_default_options()
    o.batch_engine, o.batch_parts = L.FEM_BATCH_CLUSTERS, 3
    rc, _ = L.fem_solve_batch([None], [W.cube_sphere_indenter()], 1e-6, o, [np.zeros((8, 3))], check=False)
    assert rc == L.FEM_ERR_ARG and "fem_options" in L.fem_last_error()


@pytest.mark.parametrize("case", ["index", "repeat", "inverted", "flat", "nan", "material", "model", "mask",
                                  "sizes"])
def test_host_validation(case):
    from paper_2103_16747_b300 import _lib as L
    m = W.cube_mesh(2)
    nodes, tets, mats = m.nodes.copy(), m.tets.copy(), m.materials.copy()
    fixed, mask = m.fixed_nodes, None
    want = L.FEM_ERR_ARG
    if case == "index":
        tets[3, 1] = len(nodes)
    elif case == "repeat":
        tets[0, 1] = tets[0, 0]
        want = L.FEM_ERR_DEGENERATE_TET
    elif case == "inverted":
        tets[0, [2, 3]] = tets[0, [3, 2]]
        want = L.FEM_ERR_DEGENERATE_TET
    elif case == "flat":
        nodes[tets[0, 3]] = nodes[tets[0, 0]] + 0.5 * (nodes[tets[0, 1]] - nodes[tets[0, 0]]) \
            + 0.5 * (nodes[tets[0, 2]] - nodes[tets[0, 0]])
        want = L.FEM_ERR_DEGENERATE_TET
    elif case == "nan":
        nodes[4, 2] = np.inf
        want = L.FEM_ERR_NONFINITE
    elif case == "material":
        mats[0, 1] = 0.5
    elif case == "model":
        mats = np.column_stack([mats, [2.0]])
    elif case == "mask":
        mask = np.full(len(fixed), 9, dtype=np.uint8)
    elif case == "sizes":
        tets = tets[:0]
    with pytest.raises(L.FemError) as ei:
        L.fem_create_mesh(nodes, tets, m.tet_material[: len(tets)], mats, fixed, mask)
    assert ei.value.code == want, str(ei.value)
    assert L.fem_last_error()


def test_no_device_is_an_error_not_a_fallback():
    """Without a GPU the valid call fails loudly with FEM_ERR_CUDA."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2103_16747_b300 import _lib as L
    m = W.cube_mesh(2)
    with pytest.raises(L.FemError) as ei:
        L.fem_create_mesh(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes)
    assert ei.value.code == L.FEM_ERR_CUDA


@pytest.mark.parametrize("workload,n_parts", [("cube", 7), ("cube", 37), ("fingertip", 148), ("fingertip", 37),
                                              ("fingertip", 1), ("large", 148), ("large", 64)])
def test_host_plan_is_thread_independent_and_owners_are_balanced(workload, n_parts):
    """Mesh preparation and partition plan on the host, without a GPU: the plan
    on host threads equals the one-thread plan; every tet is evaluated by exactly
    one part that holds it; owned counts stay within a few tets of the mean
    (the owner of a tet is not simply the part of its smallest node); node->tet
    lists are ascending in local tet index (the chunked gathers rely on it)."""
    from paper_2103_16747_b300 import _lib as L
    if workload == "cube":
        m = W.cube_mesh(8)
    elif workload == "fingertip":
        m = W.fingertip_sphere()[0]
    else:   # the largest fingertip of the uneven batch: R = 9 mm, about 204k tets
        m = W.fingertip_mesh(R=9.0, h=W.fingertip_for_tets(2e5, 9.0))
    r = L.fem_debug_plan_check(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes, n_parts)
    assert r["identical"] == 1 and r["owners_valid"] == 1 and r["lists_ascending"] == 1
    mean = len(m.tets) / n_parts
    assert r["max_owned"] <= 1.05 * mean + 8
    assert r["max_part_tets"] >= r["max_owned"]
    if workload == "fingertip" and n_parts == 148:
        # the single-solve kernel's gathers take one thread per owned node component
        assert r["max_owned_nodes"] <= 256 // 3
        # halo tets make a part's list well longer than its owned share
        assert r["max_part_tets"] > 1.5 * r["max_owned"]


def test_host_plan_check_reports_bad_input():
    from paper_2103_16747_b300 import _lib as L
    m = W.cube_mesh(2)
    tets = m.tets.copy()
    tets[0, [1, 2]] = tets[0, [2, 1]]   # inverted
    with pytest.raises(RuntimeError):
        L.fem_debug_plan_check(m.nodes, tets, m.tet_material, m.materials, m.fixed_nodes, 2)
    with pytest.raises(RuntimeError):
        L.fem_debug_plan_check(m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes, 0)


def test_host_plan_from_concurrent_threads_and_a_forked_child():
    """The host worker pool serves one job at a time: concurrent callers (ctypes
    releases the GIL) run their items on their own thread and still get the
    same plan; a forked child runs without the parent's pool threads."""
    import os
    import threading
    from paper_2103_16747_b300 import _lib as L
    m = W.fingertip_sphere()[0]
    args = (m.nodes, m.tets, m.tet_material, m.materials, m.fixed_nodes, 148)
    ref = L.fem_debug_plan_check(*args)
    out = [None] * 6

    def work(k):
        out[k] = [L.fem_debug_plan_check(*args) for _ in range(3)]
    ts = [threading.Thread(target=work, args=(k,)) for k in range(6)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert all(r == ref for rs in out for r in rs)
    if hasattr(os, "fork"):
        import warnings
        with warnings.catch_warnings():
            warnings.simplefilter("ignore", DeprecationWarning)
            pid = os.fork()
        if pid == 0:
            r = L.fem_debug_plan_check(*args)
            os._exit(0 if r == ref else 1)
        _, status = os.waitpid(pid, 0)
        assert os.WIFEXITED(status) and os.WEXITSTATUS(status) == 0


def test_ctypes_structures_match_the_c_header(tmp_path):
    """Every structure the binding declares has the size and field offsets of
    the C header's (a mismatch would hand the library shifted options). The
    offsets come from a small C program compiled against include/fem.h."""
    import shutil
    import subprocess
    from paper_2103_16747_b300 import _lib as L
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    here = os.path.dirname(os.path.abspath(__file__))
    include = os.path.join(os.path.dirname(here), "include")
    structs = [v for v in vars(L).values()
               if isinstance(v, type) and issubclass(v, ctypes.Structure) and v.__name__.startswith("fem_")]
    assert len(structs) >= 8
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "fem.h"', 'int main(void) {']
    for st in structs:
        lines.append(f'  printf("{st.__name__} sizeof %zu\\n", sizeof({st.__name__}));')
        for name, _ in st._fields_:
            lines.append(f'  printf("{st.__name__} {name} %zu\\n", offsetof({st.__name__}, {name}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", include, str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for st in structs:
        assert got[(st.__name__, "sizeof")] == ctypes.sizeof(st), st.__name__
        for name, _ in st._fields_:
            assert got[(st.__name__, name)] == getattr(st, name).offset, (st.__name__, name)


def test_binding_signatures_match_the_header():
    """Each function the header declares is bound with as many arguments as it
    takes and with its return kind (int status, void, or a C string)."""
    import ctypes
    from paper_2103_16747_b300 import _lib as L
    here = os.path.dirname(os.path.abspath(__file__))
    text = open(os.path.join(os.path.dirname(here), "include", "fem.h")).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    decls = re.findall(r"^\s*(int|void|const char\s*\*)\s*(fem_\w+)\s*\(([^;]*?)\)\s*;", text, flags=re.M | re.S)
    assert len(decls) >= 25
    for ret, name, params in decls:
        params = params.strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        f = getattr(L.lib, name)
        assert len(f.argtypes) == n, (name, len(f.argtypes), n)
        want = {"int": ctypes.c_int, "void": None}.get(ret.replace(" ", ""), ctypes.c_char_p)
        assert f.restype == want, (name, f.restype, want)


def test_product_and_oracle_share_no_code():
    """The CUDA path and the oracle are independent: no product module imports
    the oracle, no oracle module imports the product, and the product's C/CUDA
    sources include nothing from the oracle. Importing the product leaves the
    oracle unloaded."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.join(root, "paper_2103_16747_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b|#include\s+\"[^\"]*oracle", text, re.M), f
    for dirpath, _, files in os.walk(os.path.join(root, "oracle")):
        for f in files:
            if f.endswith(".py"):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+paper_2103_16747_b300\b", text, re.M), f
    code = "import sys, paper_2103_16747_b300; print(any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules))"
    out = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, check=True)
    assert out.stdout.strip() == "False"


def test_bench_reference_line_keeps_the_contract():
    """`bench.py --impl reference` runs the oracle on the host cores (no GPU) and
    prints one JSON line with the metric, the timing keys, a cpu_baseline that
    describes the run and an e2e with no host-device copies."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["n_gpus"] == 1 and "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_documented_option_defaults_are_the_defaults():
    """Every numeric "(default N)" in the header's fem_options comments is what
    fem_default_options sets."""
    from paper_2103_16747_b300 import _lib as L
    here = os.path.dirname(os.path.abspath(__file__))
    text = open(os.path.join(os.path.dirname(here), "include", "fem.h")).read()
    body = text[:text.index("} fem_options;")]
    body = body[body.rindex("typedef struct {"):]
    fields = list(re.finditer(r"^\s*(?:double|int32_t|int64_t)\s+(\w+);", body, re.M))
    o = L.fem_default_options()
    checked = 0
    for k, f in enumerate(fields):
        end = fields[k + 1].start() if k + 1 < len(fields) else len(body)
        m = re.search(r"default\s+(-?\d[\d.]*(?:e[-+]?\d+)?)", body[f.start():end])
        if m:
            assert getattr(o, f.group(1)) == pytest.approx(float(m.group(1)), rel=1e-12), f.group(1)
            checked += 1
    assert checked >= 12
