"""Write the oracle's reference solution of the single-fingertip sphere
indentation (R=7 mm, L=40 mm two-layer fingertip, sphere r=4 mm, 2 mm in 20
load steps) to ``fingertip_sphere_oracle.npz``.

Calls only ``oracle/`` and the seeded input generators; the GPU parity tests
compare against the stored arrays because the full oracle solve takes minutes.
Run from the repository root:  python tests/golden/make_golden.py
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


def main():
    mesh, ind = W.fingertip_sphere()
    t = time.time()
    r = Problem(mesh, ind).solve(tol=1e-10)
    assert r.converged
    out = os.path.join(HERE, "fingertip_sphere_oracle.npz")
    np.savez_compressed(out, u=r.u, step_force=r.step_force, nodal_contact=r.nodal_contact,
                        reactions=r.reactions, residual=r.residual, scale=r.scale,
                        newton_iters=r.newton_iters, digest=np.array(mesh_digest(mesh, ind)))
    print(f"wrote {out} in {time.time() - t:.1f} s; newton {r.newton_iters.tolist()}")


if __name__ == "__main__":
    main()
