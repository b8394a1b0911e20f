"""ctypes binding of the C ABI in include/fem.h (argument marshalling only).

Every function keeps the C name and order of arguments. Arrays may be NumPy
arrays (host) or torch tensors (host or CUDA); they are passed as raw pointers
after a dtype/contiguity check. Nothing here computes any part of the solve and
there is no CPU fallback: if the CUDA library is missing, importing this module
raises ImportError.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# FEM_B300_CHECKED=1 selects the checked build (bounds- and NaN-checked kernels)
LIB_PATH = os.path.join(_HERE, "libfem_b300_checked.so" if os.environ.get("FEM_B300_CHECKED") == "1"
                        else "libfem_b300.so")

FEM_OK = 0
FEM_MODEL_NEO_HOOKEAN = 0
FEM_MODEL_COROTATED = 1
FEM_ERR_ARG = -1
FEM_ERR_DEGENERATE_TET = -2
FEM_ERR_NONFINITE = -3
FEM_ERR_OOM = -4
FEM_ERR_NOT_CONVERGED = -5
FEM_ERR_TIMEOUT = -6
FEM_ERR_CUDA = -7
FEM_ERR_TOO_LARGE = -8
FEM_ERR_CHECK = -10
FEM_ERR_BUSY = -9
FEM_PENDING = 1
ERR_NAMES = {0: "FEM_OK", -1: "FEM_ERR_ARG", -2: "FEM_ERR_DEGENERATE_TET", -3: "FEM_ERR_NONFINITE",
             -4: "FEM_ERR_OOM", -5: "FEM_ERR_NOT_CONVERGED", -6: "FEM_ERR_TIMEOUT", -7: "FEM_ERR_CUDA",
             -8: "FEM_ERR_TOO_LARGE", -9: "FEM_ERR_BUSY", -10: "FEM_ERR_CHECK", 1: "FEM_PENDING"}

FEM_SPHERE, FEM_CYLINDER, FEM_BOX, FEM_PLANE = 0, 1, 2, 3
FEM_MAX_STEPS = 256
FEM_TANGENT_PROJECTED, FEM_TANGENT_EXACT, FEM_TANGENT_ADAPTIVE, FEM_TANGENT_ABS = 0, 1, 2, 3
FEM_BATCH_AUTO, FEM_BATCH_GROUPS, FEM_BATCH_CLUSTERS = 0, 1, 2
PHASES = ("eval", "tangent", "pcg_init", "pcg_reduce", "product_element", "vector_update", "halo_wait", "total",
          "pcg_scalar", "product_gather")

# Every symbol include/fem.h declares.
EXPORTS = ("fem_default_options", "fem_create_mesh", "fem_set_indenter", "fem_set_dirichlet_values",
           "fem_solve", "fem_solve_range", "fem_solve_batch", "fem_destroy_mesh", "fem_last_error", "fem_build_checked",
           "fem_mesh_info_get", "fem_repartition",
           "fem_eval_residual", "fem_eval_residual_noalloc", "fem_apply_tangent",
           "fem_debug_barrier_timeout", "fem_debug_pcg_dots", "fem_debug_reciprocals", "fem_debug_plan_check", "fem_debug_pick_shape", "fem_batch_create", "fem_batch_run", "fem_batch_info_get",
           "fem_batch_destroy", "fem_batch_tune", "fem_server_create", "fem_server_start", "fem_server_submit",
           "fem_server_result", "fem_server_stop", "fem_server_info_get", "fem_server_destroy",
           "fem_element_stress")


class fem_material(C.Structure):
    _fields_ = [("E", C.c_double), ("nu", C.c_double), ("model", C.c_int32), ("reserved", C.c_int32)]


class fem_options(C.Structure):
    _fields_ = [("c_kappa", C.c_double), ("max_newton", C.c_int32), ("max_cg", C.c_int32),
                ("cg_rtol_max", C.c_double), ("cg_rtol_min", C.c_double),
                ("max_backtracks", C.c_int32), ("tangent", C.c_int32),
                ("barrier_timeout_s", C.c_double), ("batch_engine", C.c_int32), ("batch_parts", C.c_int32),
                ("batch_tets_per_cta", C.c_int32), ("precond_degree", C.c_int32),
                ("precond_ratio", C.c_double), ("dt", C.c_double), ("density", C.c_double),
                ("mu_f", C.c_double), ("friction_eps", C.c_double), ("friction_passes", C.c_int32),
                ("tangent_fp16", C.c_int32)]


class fem_stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("steps_done", C.c_int32), ("newton_iters", C.c_int32),
                ("cg_iters", C.c_int32), ("backtracks", C.c_int32), ("active_contacts", C.c_int32),
                ("residual", C.c_double), ("scale", C.c_double), ("energy", C.c_double),
                ("kernel_ms", C.c_double), ("exact_newton_iters", C.c_int32),
                ("phase_ms", C.c_double * 10), ("phase_max_ms", C.c_double * 10),
                ("phase_min_ms", C.c_double * 10),
                ("newton_per_step", C.c_int32 * FEM_MAX_STEPS),
                ("cg_per_step", C.c_int32 * FEM_MAX_STEPS),
                ("residual_per_step", C.c_double * FEM_MAX_STEPS), ("tangent_products", C.c_int64),
                ("step_end_ms", C.c_double * FEM_MAX_STEPS)]


class fem_indenter(C.Structure):
    _fields_ = [("shape", C.c_int32), ("pose", C.c_double * 12), ("params", C.c_double * 3),
                ("dir", C.c_double * 3), ("depth_schedule", C.c_void_p), ("n_steps", C.c_int32)]


class fem_mesh_info(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_tets", C.c_int64), ("n_parts", C.c_int32),
                ("part_tets", C.c_int64), ("max_owned_nodes", C.c_int32),
                ("max_local_nodes", C.c_int32), ("max_part_tets", C.c_int32),
                ("smem_bytes", C.c_int32), ("resident", C.c_int32), ("h_bar", C.c_double), ("scale_floor", C.c_double),
                ("n_candidates", C.c_int64), ("device_bytes", C.c_int64)]


class fem_batch_info(C.Structure):
    _fields_ = [("engine", C.c_int32), ("parts", C.c_int32), ("slots", C.c_int32), ("graph", C.c_int32),
                ("smem_bytes", C.c_int32), ("global_bytes_per_cta", C.c_int32), ("resident_tangent", C.c_int32),
                ("workspace_bytes", C.c_int64)]


class fem_tune_report(C.Structure):
    _fields_ = [("n_candidates", C.c_int32), ("engine", C.c_int32 * 16), ("parts", C.c_int32 * 16),
                ("tets_per_cta", C.c_int32 * 16), ("rate", C.c_double * 16), ("best", C.c_int32)]


class fem_server_info(C.Structure):
    _fields_ = [("n_classes", C.c_int32), ("class_parts", C.c_int32 * 8), ("class_groups", C.c_int32 * 8),
                ("n_ctas", C.c_int32), ("result_slots", C.c_int32), ("admitted", C.c_int64),
                ("completed", C.c_int64), ("rejected", C.c_int64), ("workspace_bytes", C.c_int64),
                ("suspended", C.c_int64), ("launches", C.c_int64), ("large_class", C.c_int32),
                ("huge_class", C.c_int32), ("n_shapes", C.c_int32), ("shape_ctas", C.c_int32 * 3),
                ("shape_groups", (C.c_int32 * 8) * 3)]


class FemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing; build it with `python -m paper_2103_16747_b300.build`")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    sig = {
        "fem_default_options": (None, [C.POINTER(fem_options)]),
        "fem_create_mesh": (C.c_int, [P, C.c_int64, P, C.c_int64, P, P, C.c_int32, P, C.c_int64, P, P,
                                      C.POINTER(P)]),
        "fem_set_indenter": (C.c_int, [P, C.c_int, P, P, P, P, C.c_int32]),
        "fem_set_dirichlet_values": (C.c_int, [P, P]),
        "fem_solve": (C.c_int, [P, C.c_int32, C.c_double, C.POINTER(fem_options), P, P, P,
                                C.POINTER(fem_stats)]),
        "fem_solve_batch": (C.c_int, [P, P, C.c_int32, C.c_double, C.POINTER(fem_options), P, P, P]),
        "fem_solve_range": (C.c_int, [P, C.c_int32, C.c_int32, P, P, C.c_double, C.POINTER(fem_options), P, P, P, P,
                                      C.POINTER(fem_stats)]),
        "fem_destroy_mesh": (None, [P]),
        "fem_last_error": (C.c_char_p, []),
        "fem_build_checked": (C.c_int, []),
        "fem_mesh_info_get": (C.c_int, [P, C.POINTER(fem_mesh_info)]),
        "fem_repartition": (C.c_int, [P, C.c_int32]),
        "fem_eval_residual": (C.c_int, [P, P, C.c_int32, C.POINTER(fem_options), P, P, P]),
        "fem_eval_residual_noalloc": (C.c_int, [P, P, C.c_int32, C.POINTER(fem_options), P, P, P]),
        "fem_apply_tangent": (C.c_int, [P, P, C.c_int32, C.POINTER(fem_options), P, P]),
        "fem_debug_barrier_timeout": (C.c_int, [C.c_double]),
        "fem_debug_pcg_dots": (C.c_int, [P, P, P, P, P]),
        "fem_debug_reciprocals": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
        "fem_debug_plan_check": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                           C.c_int32, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p]),
        "fem_debug_pick_shape": (C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                           C.c_int32, C.c_void_p]),
        "fem_batch_create": (C.c_int, [P, P, C.c_int32, C.POINTER(fem_options), C.POINTER(P)]),
        "fem_batch_run": (C.c_int, [P, P, C.c_double, P, P, P]),
        "fem_batch_info_get": (C.c_int, [P, C.POINTER(fem_batch_info)]),
        "fem_batch_destroy": (None, [P]),
        "fem_batch_tune": (C.c_int, [P, P, C.c_int32, C.c_double, C.POINTER(fem_options), C.c_int32,
                                     C.POINTER(fem_options), C.POINTER(fem_tune_report)]),
        "fem_server_create": (C.c_int, [P, C.c_int32, C.c_int32, C.POINTER(fem_options), C.c_int64, C.POINTER(P)]),
        "fem_server_start": (C.c_int, [P, C.c_double]),
        "fem_server_submit": (C.c_int, [P, C.c_int32, P, C.c_double, C.POINTER(C.c_int64)]),
        "fem_server_result": (C.c_int, [P, C.c_int64, C.c_int32, P, P, C.POINTER(fem_stats), P]),
        "fem_server_stop": (C.c_int, [P]),
        "fem_server_info_get": (C.c_int, [P, C.POINTER(fem_server_info)]),
        "fem_server_destroy": (None, [P]),
        "fem_element_stress": (C.c_int, [P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def fem_last_error() -> str:
    return lib.fem_last_error().decode()


def fem_build_checked() -> int:
    """1 for the FEM_CHECKED build (bounds- and NaN-checked kernels), else 0."""
    return int(lib.fem_build_checked())


def _check(rc):
    if rc != FEM_OK:
        raise FemError(rc, fem_last_error())
    return rc


def _ptr(x, dtype, keep):
    """Raw pointer of a contiguous array of the given numpy dtype (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):                       # torch tensor, host or device
        import torch
        want = {np.float64: torch.float64, np.int32: torch.int32, np.uint8: torch.uint8}[dtype]
        if x.dtype != want or not x.is_contiguous():
            raise TypeError(f"tensor must be contiguous {want}")
        keep.append(x)
        return C.c_void_p(x.data_ptr())
    a = np.ascontiguousarray(x, dtype=dtype)
    keep.append(a)
    return C.c_void_p(a.ctypes.data)


def _out_ptr(x, dtype, keep):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return _ptr(x, dtype, keep)
    if not (isinstance(x, np.ndarray) and x.dtype == dtype and x.flags.c_contiguous and x.flags.writeable):
        raise TypeError("output arrays must be writeable C-contiguous numpy arrays of the right dtype")
    keep.append(x)
    return C.c_void_p(x.ctypes.data)


def fem_default_options() -> fem_options:
    o = fem_options()
    lib.fem_default_options(C.byref(o))
    return o


def fem_create_mesh(nodes, tets, tet_material, materials, fixed_nodes, fixed_mask=None,
                    cuda_stream=None):
    """Returns an opaque handle (c_void_p). ``materials``: (M, 2) array of (E, nu),
    or (M, 3) with a third column FEM_MODEL_* (0 neo-Hookean, 1 co-rotational).
    ``cuda_stream``: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
    keep = []
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    mats = np.asarray(materials, dtype=np.float64)
    mats = mats.reshape(-1, mats.shape[-1] if mats.ndim == 2 else 2)
    model = mats[:, 2].astype(np.int32) if mats.shape[1] > 2 else np.zeros(len(mats), dtype=np.int32)
    mat_arr = (fem_material * len(mats))(*[fem_material(float(e), float(n), int(md), 0)
                                            for (e, n), md in zip(mats[:, :2], model)])
    fixed = np.ascontiguousarray(fixed_nodes if fixed_nodes is not None else [], dtype=np.int32)
    stream = getattr(cuda_stream, "cuda_stream", cuda_stream)
    out = C.c_void_p()
    rc = lib.fem_create_mesh(_ptr(nodes, np.float64, keep), nodes.shape[0],
                             _ptr(tets, np.int32, keep), tets.shape[0],
                             _ptr(tet_material, np.int32, keep), C.cast(mat_arr, C.c_void_p), len(mats),
                             _ptr(fixed, np.int32, keep) if len(fixed) else None, len(fixed),
                             _ptr(fixed_mask, np.uint8, keep),
                             C.c_void_p(stream) if stream else None, C.byref(out))
    _check(rc)
    return out


def fem_set_indenter(mesh, shape, pose, params, direction, depth_schedule):
    keep = []
    d = np.ascontiguousarray(depth_schedule, dtype=np.float64)
    return _check(lib.fem_set_indenter(mesh, int(shape), _ptr(pose, np.float64, keep),
                                       _ptr(params, np.float64, keep), _ptr(direction, np.float64, keep),
                                       _ptr(d, np.float64, keep), len(d)))


def fem_set_dirichlet_values(mesh, values):
    keep = []
    return _check(lib.fem_set_dirichlet_values(mesh, _ptr(values, np.float64, keep)))


def fem_solve(mesh, load_steps, tol, opt=None, out_disp=None, out_contact_force=None,
              out_nodal_contact=None, check=True):
    """Runs the solve; outputs are written into the given arrays (numpy or torch,
    host or device). Returns (rc, fem_stats)."""
    keep = []
    st = fem_stats()
    rc = lib.fem_solve(mesh, int(load_steps), float(tol), C.byref(opt) if opt is not None else None,
                       _out_ptr(out_disp, np.float64, keep), _out_ptr(out_contact_force, np.float64, keep),
                       _out_ptr(out_nodal_contact, np.float64, keep), C.byref(st))
    if check:
        _check(rc)
    return rc, st


def fem_solve_range(mesh, first_step, last_step, tol, opt=None, u0=None, u0_prev=None, out_disp=None,
                    out_prev_disp=None, out_contact_force=None, out_nodal_contact=None, check=True):
    """Load steps first_step..last_step from the saved state (u0, u0_prev);
    returns (rc, fem_stats). (out_disp, out_prev_disp) is the state to resume
    the next range from."""
    keep = []
    st = fem_stats()
    rc = lib.fem_solve_range(mesh, int(first_step), int(last_step), _ptr(u0, np.float64, keep),
                             _ptr(u0_prev, np.float64, keep), float(tol), C.byref(opt) if opt is not None else None,
                             _out_ptr(out_disp, np.float64, keep), _out_ptr(out_prev_disp, np.float64, keep),
                             _out_ptr(out_contact_force, np.float64, keep),
                             _out_ptr(out_nodal_contact, np.float64, keep), C.byref(st))
    if check:
        _check(rc)
    return rc, st


def _indenter_array(indenters, keep):
    n = len(indenters)
    arr = (fem_indenter * n)()
    for i, d in enumerate(indenters):
        sched = np.ascontiguousarray(d.depth_schedule, dtype=np.float64)
        keep.append(sched)
        arr[i].shape = int(d.shape)
        arr[i].pose[:] = [float(v) for v in np.asarray(d.pose, dtype=np.float64)]
        prm = np.zeros(3) if d.params is None else np.asarray(d.params, dtype=np.float64)
        arr[i].params[:] = [float(v) for v in prm]
        arr[i].dir[:] = [float(v) for v in np.asarray(d.direction, dtype=np.float64)]
        arr[i].depth_schedule = sched.ctypes.data
        arr[i].n_steps = len(sched)
    return arr


def _mesh_array(meshes):
    return (C.c_void_p * len(meshes))(*[m.value if isinstance(m, C.c_void_p) else m for m in meshes])


def _batch_outputs(n, out_disp, out_contact_force, keep):
    disp = (C.c_void_p * n)(*[_out_ptr(a, np.float64, keep).value for a in out_disp])
    forces = None
    if out_contact_force is not None:
        forces = (C.c_void_p * n)(*[_out_ptr(a, np.float64, keep).value for a in out_contact_force])
    return disp, forces


def fem_solve_batch(meshes, indenters, tol, opt=None, out_disp=None, out_contact_force=None, check=True):
    """Batched solves. ``meshes``: list of handles (repeats allowed);
    ``indenters``: objects with shape/pose/params/direction/depth_schedule;
    ``out_disp`` / ``out_contact_force``: lists of arrays (numpy or torch, host
    or device). Returns (rc, list of fem_stats)."""
    n = len(meshes)
    keep = []
    mesh_arr = _mesh_array(meshes)
    ind_arr = _indenter_array(indenters, keep)
    disp, forces = _batch_outputs(n, out_disp, out_contact_force, keep)
    stats = (fem_stats * n)()
    rc = lib.fem_solve_batch(C.cast(mesh_arr, C.c_void_p), C.cast(ind_arr, C.c_void_p), n, float(tol),
                             C.byref(opt) if opt is not None else None, C.cast(disp, C.c_void_p),
                             C.cast(forces, C.c_void_p) if forces is not None else None,
                             C.cast(stats, C.c_void_p))
    if check:
        _check(rc)
    return rc, list(stats)


def fem_batch_tune(meshes, indenters, tol, opt=None, proxy_steps=2):
    """Autotune the batch slot shape; returns (options, report)."""
    keep = []
    n = len(meshes)
    ind_arr = _indenter_array(indenters, keep)
    out = fem_options()
    rep = fem_tune_report()
    _check(lib.fem_batch_tune(C.cast(_mesh_array(meshes), C.c_void_p), C.cast(ind_arr, C.c_void_p), n, float(tol),
                              C.byref(opt) if opt is not None else None, int(proxy_steps), C.byref(out),
                              C.byref(rep)))
    return out, rep


class FemServer:
    """Request server (fem_server_*): continuous batching on a resident mesh
    pool. ``submit`` returns a request id; ``result`` waits for it."""

    def __init__(self, meshes, max_steps, opt=None, result_bytes=256 << 20):
        self.n_nodes = None
        h = C.c_void_p()
        _check(lib.fem_server_create(C.cast(_mesh_array(meshes), C.c_void_p), len(meshes), int(max_steps),
                                     C.byref(opt) if opt is not None else None, int(result_bytes), C.byref(h)))
        self.handle = h

    def start(self, max_seconds):
        _check(lib.fem_server_start(self.handle, float(max_seconds)))

    def submit(self, mesh_index, indenter, tol):
        keep = []
        arr = _indenter_array([indenter], keep)
        rid = C.c_int64()
        rc = lib.fem_server_submit(self.handle, int(mesh_index), C.cast(arr, C.c_void_p), float(tol), C.byref(rid))
        return rc, rid.value

    def result(self, request_id, n_nodes, n_steps, wait_ms=0):
        """(rc, u (n_nodes, 3), forces (n_steps, 3), fem_stats, times) or
        (FEM_PENDING, None, ...) while it runs."""
        u = np.zeros((n_nodes, 3))
        f = np.zeros((n_steps, 3))
        st = fem_stats()
        t = np.zeros(3)
        rc = lib.fem_server_result(self.handle, int(request_id), int(wait_ms), C.c_void_p(u.ctypes.data),
                                   C.c_void_p(f.ctypes.data), C.byref(st), C.c_void_p(t.ctypes.data))
        if rc == FEM_PENDING:
            return rc, None, None, None, None
        return rc, u, f, st, t

    def info(self) -> fem_server_info:
        i = fem_server_info()
        _check(lib.fem_server_info_get(self.handle, C.byref(i)))
        return i

    def stop(self):
        return lib.fem_server_stop(self.handle)

    def close(self):
        if self.handle:
            lib.fem_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FemBatch:
    """A reusable batch plan (fem_batch_create): fixed meshes, load-step
    counts and options; ``run`` replays the captured batch with new
    indenters."""

    def __init__(self, meshes, n_steps, opt=None):
        n = len(meshes)
        self.n = n
        steps = np.ascontiguousarray(n_steps, dtype=np.int32)
        h = C.c_void_p()
        _check(lib.fem_batch_create(C.cast(_mesh_array(meshes), C.c_void_p), C.c_void_p(steps.ctypes.data), n,
                                    C.byref(opt) if opt is not None else None, C.byref(h)))
        self.handle = h

    def info(self) -> fem_batch_info:
        i = fem_batch_info()
        _check(lib.fem_batch_info_get(self.handle, C.byref(i)))
        return i

    def run(self, indenters, tol, out_disp, out_contact_force=None, check=True):
        keep = []
        ind_arr = _indenter_array(indenters, keep)
        disp, forces = _batch_outputs(self.n, out_disp, out_contact_force, keep)
        stats = (fem_stats * self.n)()
        rc = lib.fem_batch_run(self.handle, C.cast(ind_arr, C.c_void_p), float(tol), C.cast(disp, C.c_void_p),
                               C.cast(forces, C.c_void_p) if forces is not None else None, C.cast(stats, C.c_void_p))
        if check:
            _check(rc)
        return rc, list(stats)

    def close(self):
        if self.handle:
            lib.fem_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fem_element_stress(mesh, u, n_tets, out_cauchy=None, out_von_mises=None):
    """Cauchy stress (n_tets, 6: xx yy zz yz xz xy) and von Mises stress
    (n_tets,) at displacement u (caller orders). Returns (sigma, von_mises)."""
    keep = []
    sig = np.zeros((n_tets, 6)) if out_cauchy is None else out_cauchy
    vm = np.zeros(n_tets) if out_von_mises is None else out_von_mises
    _check(lib.fem_element_stress(mesh, _ptr(u, np.float64, keep), _out_ptr(sig, np.float64, keep),
                                  _out_ptr(vm, np.float64, keep)))
    return sig, vm


def fem_destroy_mesh(mesh):
    lib.fem_destroy_mesh(mesh)


def fem_mesh_info_get(mesh) -> fem_mesh_info:
    info = fem_mesh_info()
    _check(lib.fem_mesh_info_get(mesh, C.byref(info)))
    return info


def fem_repartition(mesh, n_parts):
    return _check(lib.fem_repartition(mesh, int(n_parts)))


def fem_eval_residual(mesh, u, step, opt=None, out_R=None, out_fc=None):
    keep = []
    e = (C.c_double * 2)()
    rc = lib.fem_eval_residual(mesh, _ptr(u, np.float64, keep), int(step),
                               C.byref(opt) if opt is not None else None,
                               _out_ptr(out_R, np.float64, keep), _out_ptr(out_fc, np.float64, keep), e)
    _check(rc)
    return float(e[0]), float(e[1])


def fem_eval_residual_noalloc(mesh, u, step, opt=None, out_R=None, out_fc=None):
    """As fem_eval_residual, for callers that may not allocate device memory:
    the library's fixed scratch block replaces every per-call buffer."""
    keep = []
    e = (C.c_double * 2)()
    rc = lib.fem_eval_residual_noalloc(mesh, _ptr(u, np.float64, keep), int(step),
                                       C.byref(opt) if opt is not None else None,
                                       _out_ptr(out_R, np.float64, keep), _out_ptr(out_fc, np.float64, keep), e)
    _check(rc)
    return float(e[0]), float(e[1])


def fem_apply_tangent(mesh, u, step, p, out_y, opt=None):
    keep = []
    return _check(lib.fem_apply_tangent(mesh, _ptr(u, np.float64, keep), int(step),
                                        C.byref(opt) if opt is not None else None,
                                        _ptr(p, np.float64, keep), _out_ptr(out_y, np.float64, keep)))


def fem_debug_pcg_dots(mesh, r, u, w):
    """(r,u), (w,u), (r,r) over the free DOFs as the PCG's reductions form them."""
    keep = []
    out = np.zeros(3)
    _check(lib.fem_debug_pcg_dots(mesh, _ptr(r, np.float64, keep), _ptr(u, np.float64, keep),
                                  _ptr(w, np.float64, keep), C.c_void_p(out.ctypes.data)))
    return out


def fem_debug_barrier_timeout(timeout_s):
    return lib.fem_debug_barrier_timeout(float(timeout_s))


def fem_debug_plan_check(nodes, tets, tet_material, materials, fixed_nodes, n_parts):
    """Host-only check of mesh preparation and partitioning (no CUDA call): a
    dict with the fields of fem_debug_plan_check's out[8]."""
    keep = []
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    mats = np.asarray(materials, dtype=np.float64)
    mats = mats.reshape(-1, mats.shape[-1] if mats.ndim == 2 else 2)
    model = mats[:, 2].astype(np.int32) if mats.shape[1] > 2 else np.zeros(len(mats), dtype=np.int32)
    mat_arr = (fem_material * len(mats))(*[fem_material(float(e), float(n), int(md), 0)
                                            for (e, n), md in zip(mats[:, :2], model)])
    fixed = np.ascontiguousarray(fixed_nodes if fixed_nodes is not None else [], dtype=np.int32)
    out = np.zeros(8, dtype=np.int64)
    _check(lib.fem_debug_plan_check(_ptr(nodes, np.float64, keep), nodes.shape[0], _ptr(tets, np.int32, keep),
                                    tets.shape[0], _ptr(tet_material, np.int32, keep), C.cast(mat_arr, C.c_void_p),
                                    len(mats), _ptr(fixed, np.int32, keep) if len(fixed) else None, len(fixed),
                                    int(n_parts), C.c_void_p(out.ctypes.data)))
    keys = ("identical", "owners_valid", "max_owned", "min_owned", "max_part_tets", "workers", "max_owned_nodes",
            "lists_ascending")
    return dict(zip(keys, (int(v) for v in out)))


def fem_debug_pick_shape(shape_groups, cur, requests):
    """The request server's next launch shape (host rule, no CUDA call).
    shape_groups: [n_shapes][n_classes] groups per class in each shape;
    cur: the live shape; requests: (id, class) of the unfinished requests."""
    g = np.ascontiguousarray(shape_groups, dtype=np.int32)
    ids = np.ascontiguousarray([r[0] for r in requests], dtype=np.int64)
    cls = np.ascontiguousarray([r[1] for r in requests], dtype=np.int32)
    out = C.c_int32(-1)
    _check(lib.fem_debug_pick_shape(g.shape[0], g.shape[1], C.c_void_p(g.ctypes.data), int(cur),
                                    C.c_void_p(ids.ctypes.data) if len(ids) else None,
                                    C.c_void_p(cls.ctypes.data) if len(cls) else None, len(ids), C.byref(out)))
    return out.value


def fem_debug_reciprocals(x):
    """(1/x, 1/sqrt(x)) as the element kernels compute them in FP64 (x > 0)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    r = np.zeros_like(x)
    q = np.zeros_like(x)
    _check(lib.fem_debug_reciprocals(C.c_void_p(x.ctypes.data), x.size, C.c_void_p(r.ctypes.data),
                                     C.c_void_p(q.ctypes.data)))
    return r, q
