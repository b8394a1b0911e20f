"""FP64 CPU oracle for the quasi-static tetrahedral-FEM indentation solve.

TEST INFRASTRUCTURE ONLY. This package is imported solely by ``tests/``, by
``__graft_entry__.smoke()`` and by the ``cpu_baseline`` / reference legs of
``bench.py``. The product path (the CUDA library and its Python binding) never
imports, links or calls anything here, and nothing here imports the product.

What it computes (Sec. III-A of the paper: a volumetric tet mesh, a per-element
hyperelastic constitutive model, rigid indenters driven into the fingertip,
nodal displacements and nodal contact forces as outputs):

  * ``material``  compressible neo-Hookean energy, first Piola-Kirchhoff stress
                  and its exact derivative dP/dF, and the eigenvalue-clamped
                  (PSD-projected) derivative;
  * ``geometry``  reference shape matrices, volumes, shape-function gradients,
                  boundary faces, lumped nodal areas, mean edge length and the
                  contact penalty stiffness per node;
  * ``contact``   signed distance, gradient and Hessian of sphere, cylinder,
                  box and plane indenters;
  * ``solver``    assembly of the global energy, gradient and sparse tangent,
                  and Newton's method with a direct sparse solve, an Armijo line
                  search with a J>0 guard, over prescribed load steps.

Readings taken where the paper is silent (it names "Neo-Hookean" without a
formula and gives no penalty law) are written next to each function. Every
function is pinned by tests under ``tests/`` against closed forms, finite
differences, invariants or brute force (no function here is "parity
unpinned").
"""
from . import contact, geometry, material, solver  # noqa: F401
from .solver import Problem, SolveResult  # noqa: F401
