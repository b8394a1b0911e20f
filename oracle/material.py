"""Compressible neo-Hookean material, FP64 (oracle; test infrastructure only).

The paper (Sec. III-A) names a Neo-Hookean model for the skin without giving its
form. Reading used here: the standard compressible form

    Psi(F) = mu/2 (I1 - 3) - mu ln J + lam/2 (ln J)^2,   I1 = tr(F^T F), J = det F,

with Lame parameters mu = E / (2(1+nu)), lam = E nu / ((1+nu)(1-2nu)). It reduces
to isotropic linear elasticity at small strain.

    P(F)   = dPsi/dF = mu (F - F^-T) + lam ln J F^-T
    dP     = mu dF + (mu - lam ln J) F^-T dF^T F^-T + lam tr(F^-1 dF) F^-T

Matrices over vec(F) use row-major flattening: index 3*i + j holds F[i, j].
All functions take batches: F has shape (..., 3, 3).
"""
from __future__ import annotations

import numpy as np


def lame(E, nu):
    """(mu, lam) from Young's modulus and Poisson's ratio."""
    E = np.asarray(E, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


def energy_density(F, mu, lam):
    """Psi(F) per element; NaN where J <= 0."""
    J = np.linalg.det(F)
    with np.errstate(invalid="ignore", divide="ignore"):
        lnJ = np.where(J > 0, np.log(np.where(J > 0, J, 1.0)), np.nan)
    I1 = np.einsum("...ij,...ij->...", F, F)
    return 0.5 * mu * (I1 - 3.0) - mu * lnJ + 0.5 * lam * lnJ * lnJ


def pk1(F, mu, lam):
    """First Piola-Kirchhoff stress P(F)."""
    J = np.linalg.det(F)
    FinvT = np.swapaxes(np.linalg.inv(F), -1, -2)
    lnJ = np.log(J)
    mu = np.asarray(mu)[..., None, None]
    lam = np.asarray(lam)[..., None, None]
    return mu * (F - FinvT) + lam * lnJ[..., None, None] * FinvT


def dpdf(F, mu, lam):
    """Exact dP/dF as a (..., 9, 9) matrix C with dP_ij = C[3i+j, 3k+l] dF_kl.

    C[ij,kl] = mu d_ik d_jl + (mu - lam ln J) FiT_il FiT_kj + lam FiT_ij FiT_kl,
    FiT = F^-T."""
    J = np.linalg.det(F)
    FiT = np.swapaxes(np.linalg.inv(F), -1, -2)
    lnJ = np.log(J)
    mu = np.asarray(mu, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    c = mu - lam * lnJ
    eye = np.eye(3)
    t_id = np.einsum("ik,jl->ijkl", eye, eye)
    t_tr = np.einsum("...il,...kj->...ijkl", FiT, FiT)
    t_vol = np.einsum("...ij,...kl->...ijkl", FiT, FiT)
    C = (mu[..., None, None, None, None] * t_id
         + c[..., None, None, None, None] * t_tr
         + lam[..., None, None, None, None] * t_vol)
    return C.reshape(C.shape[:-4] + (9, 9))


def project_psd(C):
    """Clamp the negative eigenvalues of each symmetric 9x9 matrix to zero."""
    Cs = 0.5 * (C + np.swapaxes(C, -1, -2))
    w, Q = np.linalg.eigh(Cs)
    w = np.maximum(w, 0.0)
    return np.einsum("...ik,...k,...jk->...ij", Q, w, Q)


def cauchy(F, mu, lam):
    """Cauchy stress sigma = P F^T / J (Sec. III-A of the paper reports element
    stress tensors; this is their true-stress form). Computed from pk1, the
    definition, so that a mistake in either shows in the pins below."""
    J = np.linalg.det(F)
    return pk1(F, mu, lam) @ np.swapaxes(F, -1, -2) / J[..., None, None]


def von_mises(sigma):
    """Equivalent stress sqrt(3/2 s:s) of the deviator s = sigma - tr(sigma)/3 I."""
    tr = np.trace(sigma, axis1=-2, axis2=-1)
    s = sigma - tr[..., None, None] / 3.0 * np.eye(3)
    return np.sqrt(1.5 * np.einsum("...ij,...ij->...", s, s))
