"""Seeded synthetic inputs for the tet-FEM indentation path.

The only module shared by the CPU oracle and the CUDA path: it builds meshes and
indenter poses and holds none of the method's arithmetic. Seeds follow
``numpy.random.Generator(PCG64(1000 + workload index))``.

Workloads (sizes from the indentation problem of Sec. III-A of the paper, on
synthetic geometry):
  * ``cube_sphere``        unit cube 8x8x8 hexes x 6 tets (3072 tets, 729 nodes),
                           E=1e6, nu=0.3, bottom fixed; sphere r=0.3 pressed 0.05
                           deep in 10 load steps.
  * ``fingertip_sphere``   two-layer half-capsule fingertip (R=7 mm, L=40 mm, 1 mm
                           skin E=1.5 MPa nu=0.45 over 2 mm inner E=0.2 MPa
                           nu=0.48, core surface fixed; ~39k tets / ~8.7k nodes);
                           sphere r=4 mm pressed 2 mm normal to a seeded skin point
                           in 20 load steps.
  * ``fingertip_draws``    random sphere / cylinder / box-edge indentations of the
                           same fingertip.
  * ``uneven_fingertips``  fingertips with R~U[5,10] and a log-uniform tet count.
  * ``with_model``         a copy of a mesh whose materials carry an element-law
                           id (third column: 0 neo-Hookean, 1 co-rotational).
  * ``fingertip_calibrated`` the fingertip geometry as one co-rotational shell
                           (skin and inner layer alike: E=1.55 MPa, nu=0.316, the
                           paper's calibrated simulator parameters, Sec. III-A) over
                           the fixed core, with the single-fingertip sphere load.
"""
from __future__ import annotations

import math

import numpy as np

from .indenters import (BOX, CYLINDER, PLANE, SHAPE_NAMES, SPHERE, Indenter,  # noqa: F401
                        cube_box_edge_indenter, cube_cylinder_indenter,
                        cube_sphere_indenter, draw_indentations, entry_times,
                        fingertip_sphere_indentation, linear_schedule,
                        place_at_contact, plane_indenter)
from .meshgen import (INNER, SKIN, Mesh, cube_mesh, fingertip_for_tets,  # noqa: F401
                      fingertip_mesh, fingertip_tet_count)

SEED_BASE = 1000


def cube_sphere():
    """Unit cube with a sphere pressed into the top face."""
    return cube_mesh(8), cube_sphere_indenter()


def with_model(mesh, model):
    """Copy of ``mesh`` with an element-law id per material (an int, or one per
    material) in a third materials column."""
    import copy
    m = copy.copy(mesh)
    mats = np.asarray(mesh.materials, dtype=np.float64)[:, :2]
    ids = np.broadcast_to(np.asarray(model, dtype=np.float64), (len(mats),))
    m.materials = np.column_stack([mats, ids])
    return m


def fingertip_calibrated(seed: int = SEED_BASE + 1):
    """Calibrated co-rotational shell over the rigid core, sphere indentation."""
    mesh = with_model(fingertip_mesh(E_skin=1.55, nu_skin=0.316, E_inner=1.55, nu_inner=0.316), 1)
    return mesh, fingertip_sphere_indentation(mesh, seed=seed)


def fingertip_sphere(seed: int = SEED_BASE + 1):
    """The single-fingertip sphere indentation."""
    mesh = fingertip_mesh()
    return mesh, fingertip_sphere_indentation(mesh, seed=seed)


def cube_cylinder():
    """Unit cube with a cylinder pressed across the top face (axis normal to the
    approach)."""
    return cube_mesh(8), place_at_contact(cube_cylinder_indenter(), cube_mesh(8).nodes)


def cube_box_edge():
    """Unit cube with the edge of a box pressed into the top face (faces at
    +-45 degrees to the approach)."""
    return cube_mesh(8), place_at_contact(cube_box_edge_indenter(), cube_mesh(8).nodes)


def fingertip_shape_draw(shape: int, seed: int = SEED_BASE + 5, min_depth: float = 1.5):
    """The fingertip with the first random indentation (the draws of
    ``fingertip_draws``, from ``seed``) of the given shape that goes at least
    ``min_depth`` mm deep: a fixed cylinder or box-edge case of the random-draw
    workload."""
    mesh = fingertip_mesh()
    rng = np.random.Generator(np.random.PCG64(seed))
    for _ in range(1000):
        from .indenters import draw_indentation
        ind = draw_indentation(mesh, rng)
        if ind.shape == shape and ind.depth_schedule[-1] >= min_depth:
            return mesh, ind
    raise RuntimeError("no draw of that shape")


def fingertip_draws(n: int = 256, seed: int = SEED_BASE + 2, n_steps: int = 20):
    """n random indentations of the fingertip."""
    mesh = fingertip_mesh()
    return mesh, draw_indentations(mesh, n, seed, n_steps)


def uneven_fingertips(n: int = 64, seed: int = SEED_BASE + 3, tet_min: float = 5e3,
                      tet_max: float = 2e5, build: bool = True):
    """n fingertip meshes with R~U[5,10] and tets log-uniform in [tet_min, tet_max],
    each with one random indentation."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n):
        R = rng.uniform(5.0, 10.0)
        target = math.exp(rng.uniform(math.log(tet_min), math.log(tet_max)))
        h = fingertip_for_tets(target, R)
        sub = int(rng.integers(0, 2**31 - 1))
        if build:
            mesh = fingertip_mesh(R=R, h=h)
            ind = draw_indentations(mesh, 1, sub)[0]
            out.append((mesh, ind))
        else:
            out.append((R, h, fingertip_tet_count(R, 40.0, h), sub))
    return out
