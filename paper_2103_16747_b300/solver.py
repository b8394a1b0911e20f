"""Convenience layer over the C ABI: holds a mesh handle and marshals mesh /
indenter objects (anything with the attributes used below) into fem_* calls.
All arithmetic happens in the CUDA library."""
from __future__ import annotations

import numpy as np

from . import _lib as L


class IndentationSolver:
    """One resident mesh (one solve slot) on the current CUDA device."""

    def __init__(self, mesh, cuda_stream=None):
        self.n_nodes = int(mesh.nodes.shape[0])
        self.handle = L.fem_create_mesh(mesh.nodes, mesh.tets, mesh.tet_material, mesh.materials,
                                        mesh.fixed_nodes, mesh.fixed_mask, cuda_stream)
        self.n_steps = 0

    def close(self):
        if self.handle:
            L.fem_destroy_mesh(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        return L.fem_mesh_info_get(self.handle)

    def set_indenter(self, ind):
        L.fem_set_indenter(self.handle, ind.shape, ind.pose, np.asarray(ind.params, dtype=np.float64),
                           ind.direction, ind.depth_schedule)
        self.n_steps = len(ind.depth_schedule)

    def set_dirichlet_values(self, values):
        L.fem_set_dirichlet_values(self.handle, values)

    def solve(self, tol=1e-6, opt=None, out_disp=None, out_force=None, out_nodal=None, check=True):
        """Host outputs by default; pass preallocated (torch/numpy) arrays to
        write elsewhere (device outputs avoid the host copies)."""
        if out_disp is None:
            out_disp = np.zeros((self.n_nodes, 3))
        if out_force is None:
            out_force = np.zeros((self.n_steps, 3))
        if out_nodal is None:
            out_nodal = np.zeros((self.n_nodes, 3))
        rc, st = L.fem_solve(self.handle, self.n_steps, tol, opt, out_disp, out_force, out_nodal, check=check)
        return {"rc": rc, "u": out_disp, "step_force": out_force, "nodal_contact": out_nodal, "stats": st}

    def eval_residual(self, u, step, opt=None):
        R = np.zeros((self.n_nodes, 3))
        fc = np.zeros((self.n_nodes, 3))
        e = L.fem_eval_residual(self.handle, np.ascontiguousarray(u, dtype=np.float64), step, opt, R, fc)
        return R, fc, e

    def apply_tangent(self, u, step, p, opt=None):
        y = np.zeros((self.n_nodes, 3))
        L.fem_apply_tangent(self.handle, np.ascontiguousarray(u, dtype=np.float64), step,
                            np.ascontiguousarray(p, dtype=np.float64), y, opt)
        return y


def solve_indentation(mesh, ind, tol=1e-6, opt=None, cuda_stream=None):
    s = IndentationSolver(mesh, cuda_stream)
    try:
        s.set_indenter(ind)
        return s.solve(tol, opt)
    finally:
        s.close()
