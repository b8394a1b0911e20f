"""FP64 CPU oracle for the quasi-static tetrahedral-FEM indentation solve.

TEST INFRASTRUCTURE ONLY. This package is imported solely by ``tests/``, by
``__graft_entry__.smoke()`` and by the ``cpu_baseline`` / reference legs of
``bench.py``. The product path (the CUDA library and its Python binding) never
imports, links or calls anything here, and nothing here imports the product.

What it computes (Sec. III-A of the paper: a volumetric tet mesh, a per-element
hyperelastic constitutive model, rigid indenters driven into the fingertip,
nodal displacements and nodal contact forces as outputs):

  * ``material``  compressible neo-Hookean and co-rotational energies, first
                  Piola-Kirchhoff stress and its exact derivative dP/dF, the
                  eigenvalue-clamped (PSD-projected) derivative, Cauchy and von
                  Mises stress;
  * ``geometry``  reference shape matrices, volumes, shape-function gradients,
                  boundary faces, lumped nodal areas, mean edge length and the
                  contact penalty stiffness per node;
  * ``contact``   signed distance, gradient and Hessian of sphere, cylinder,
                  box and plane indenters; the smoothed Coulomb friction
                  potential with its force and PSD Hessian;
  * ``solver``    assembly of the global energy, gradient and sparse tangent,
                  and Newton's method with a direct sparse solve, an Armijo line
                  search with a J>0 guard, over prescribed load steps; optional
                  backward-Euler inertia with lumped mass, lagged friction and
                  friction passes that refresh the normal forces within a step.

Readings taken where the paper is silent (it names "Neo-Hookean" without a
formula and gives no penalty law) are written next to each function. Every
function is pinned by tests under ``tests/`` against closed forms, finite
differences, invariants or brute force (no function here is "parity
unpinned").
"""
from . import contact, geometry, material, solver  # noqa: F401
from .solver import Problem, SolveResult  # noqa: F401
