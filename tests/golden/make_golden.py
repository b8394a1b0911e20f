"""Write the oracle's reference solutions of the single-fingertip sphere
indentation (R=7 mm, L=40 mm two-layer fingertip, sphere r=4 mm, 2 mm in 20
load steps):

  fingertip_sphere_oracle.npz          quasi-static load steps
  fingertip_sphere_dynamic_oracle.npz  the same schedule as 20 backward-Euler
                                       time steps of DYN_DT s, from rest, with
                                       the lumped mass of density DYN_DENSITY
                                       (mm, N, s units: t/mm^3)
  fingertip_calibrated_oracle.npz      quasi-static, the calibrated preset: one
                                       co-rotational shell (E=1.55 MPa, nu=0.316)
                                       over the fixed core, same load
  fingertip_sphere_friction_oracle.npz quasi-static with Coulomb friction
                                       mu_f = FRICTION_MU (the paper's calibrated
                                       coefficient)
  fingertip_cylinder_oracle.npz        quasi-static, one cylinder draw of the
                                       random-indentation workload (r 3.2 mm,
                                       axis normal to the approach, 1.57 mm)
  fingertip_box_edge_oracle.npz        quasi-static, one box-edge draw (20 mm
                                       cube, faces at +-45 deg, 1.90 mm)

Calls only ``oracle/`` and the seeded input generators; the GPU parity tests
compare against the stored arrays because the full oracle solve takes minutes.
Run from the repository root:
    python tests/golden/make_golden.py [static|dynamic|corot|friction|cylinder|box]
"""
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import Problem  # noqa: E402


def mesh_digest(mesh, ind):
    h = hashlib.sha256()
    for a in (mesh.nodes, mesh.tets, mesh.tet_material, mesh.fixed_nodes, ind.pose,
              ind.params, ind.direction, ind.depth_schedule):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


# time step of the paper's implicit integration (Sec. III-A) and a skin-like density
DYN_DT = 1e-4
DYN_DENSITY = 1.1e-9
# Coulomb coefficient calibrated in the paper (Sec. III-A)
FRICTION_MU = 0.783


def main(kind="static"):
    mesh, ind = W.fingertip_sphere()
    t = time.time()
    if kind == "dynamic":
        r = Problem(mesh, ind, dt=DYN_DT, density=DYN_DENSITY).solve(tol=1e-10)
        name = "fingertip_sphere_dynamic_oracle.npz"
    elif kind == "friction":
        r = Problem(mesh, ind, mu_f=FRICTION_MU).solve(tol=1e-10)
        name = "fingertip_sphere_friction_oracle.npz"
    elif kind in ("cylinder", "box"):
        mesh, ind = W.fingertip_shape_draw(W.CYLINDER if kind == "cylinder" else W.BOX)
        r = Problem(mesh, ind).solve(tol=1e-10)
        name = f"fingertip_{'cylinder' if kind == 'cylinder' else 'box_edge'}_oracle.npz"
    elif kind == "corot":
        mesh, ind = W.fingertip_calibrated()
        r = Problem(mesh, ind).solve(tol=1e-10)
        name = "fingertip_calibrated_oracle.npz"
    else:
        r = Problem(mesh, ind).solve(tol=1e-10)
        name = "fingertip_sphere_oracle.npz"
    assert r.converged
    out = os.path.join(HERE, name)
    np.savez_compressed(out, u=r.u, step_force=r.step_force, nodal_contact=r.nodal_contact,
                        reactions=r.reactions, residual=r.residual, scale=r.scale,
                        newton_iters=r.newton_iters, digest=np.array(mesh_digest(mesh, ind)))
    print(f"wrote {out} in {time.time() - t:.1f} s; newton {r.newton_iters.tolist()}")


if __name__ == "__main__":
    for k in (sys.argv[1:] or ["static", "dynamic", "corot", "friction", "cylinder", "box"]):
        main(k)
