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
from scipy.optimize import brentq


def lame(E, nu):
    return E / (2 * (1 + nu)), E * nu / ((1 + nu) * (1 - 2 * nu))


def uniaxial_plane(delta, E, nu, h_bar, c_kappa):
    """(lz, lt, P_zz) of the rollers + rigid plane problem at plate travel delta.

    Two nested bracketed roots. For a given lz, the traction-free lateral faces
    fix lt: mu (lt^2 - 1) + lam (2 ln lt + ln lz) = 0 (lt P_xx = 0), strictly
    increasing in lt. The plate then fixes lz: lz - (1 - delta) + P_zz h_bar /
    (c_kappa E) = 0, negative at lz = 1 - delta (compression) and equal to delta
    at lz = 1 (no strain). Both equations' residuals are asserted."""
    mu, lam = lame(E, nu)
    if delta == 0.0:
        return 1.0, 1.0, 0.0

    def lateral(lz):
        return brentq(lambda lt: mu * (lt * lt - 1.0) + lam * (2.0 * math.log(lt) + math.log(lz)),
                      1e-3, 10.0, xtol=1e-15, rtol=4 * np.finfo(float).eps, maxiter=500)

    def pzz_of(lz):
        lt = lateral(lz)
        lnJ = math.log(lt * lt * lz)
        return mu * (lz - 1 / lz) + lam * lnJ / lz

    def plate(lz):
        return lz - (1.0 - delta) + pzz_of(lz) * h_bar / (c_kappa * E)

    lo, hi = (1.0 - delta, 1.0) if delta > 0 else (1.0, 1.0 - delta)
    lz = brentq(plate, lo, hi, xtol=1e-15, rtol=4 * np.finfo(float).eps, maxiter=500)
    lt = lateral(lz)
    lnJ = math.log(lt * lt * lz)
    pxx = mu * (lt - 1 / lt) + lam * lnJ / lt
    pzz = mu * (lz - 1 / lz) + lam * lnJ / lz
    assert abs(pxx) <= 1e-9 * E, pxx
    assert abs(lz - (1.0 - delta) + pzz * h_bar / (c_kappa * E)) <= 1e-13, lz
    return float(lz), float(lt), float(pzz)


def hertz_force(E, nu, R, d):
    return 4.0 / 3.0 * E / (1 - nu * nu) * math.sqrt(R) * np.asarray(d) ** 1.5
