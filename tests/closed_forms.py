"""Closed-form solutions used to pin the oracle (and, through it, the GPU path).

Uniaxial compression of a cube on rollers by a frictionless rigid plane:
  the deformation is homogeneous, F = diag(lt, lt, lz). The lateral faces are
  traction free, so P_xx = mu (lt - 1/lt) + lam ln J / lt = 0 with J = lt^2 lz.
  The top face carries P_zz = mu (lz - 1/lz) + lam ln J / lz (reference area 1,
  so the plate force is P_zz). A penalty spring k_i = c_kappa E A_i / h_bar
  balances the nodal traction P_zz A_i at every top node, so the plate
  penetrates the top face by g = -P_zz h_bar / (c_kappa E) and lz = 1 - delta + g.
  (Nodes on the top edges also carry side-face area in A_i; with c_kappa large
  the gap is negligible there and everywhere, so the state stays homogeneous to
  within ~g.)
  At small strain this gives sigma = E eps and lateral strain -nu eps (isotropic
  linear elasticity), which the tests check separately.

Hertz contact of a rigid sphere on an elastic half-space (K. L. Johnson,
Contact Mechanics, 1985, Sec. 4.2): F = 4/3 E* sqrt(R) d^(3/2), E* = E/(1-nu^2).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import fsolve


def lame(E, nu):
    return E / (2 * (1 + nu)), E * nu / ((1 + nu) * (1 - 2 * nu))


def uniaxial_plane(delta, E, nu, h_bar, c_kappa):
    """(lz, lt, P_zz) of the rollers + rigid plane problem at plate travel delta."""
    mu, lam = lame(E, nu)

    def eqs(v):
        lz, lt = v
        lnJ = math.log(lt * lt * lz)
        pxx = mu * (lt - 1 / lt) + lam * lnJ / lt
        pzz = mu * (lz - 1 / lz) + lam * lnJ / lz
        return [pxx / E, lz - (1 - delta) + pzz * h_bar / (c_kappa * E)]

    lz, lt = fsolve(eqs, [1 - delta, 1 + nu * delta], xtol=1e-14)
    lnJ = math.log(lt * lt * lz)
    pzz = mu * (lz - 1 / lz) + lam * lnJ / lz
    return float(lz), float(lt), float(pzz)


def hertz_force(E, nu, R, d):
    return 4.0 / 3.0 * E / (1 - nu * nu) * math.sqrt(R) * np.asarray(d) ** 1.5
