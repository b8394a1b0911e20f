"""Element laws, FP64 (oracle; test infrastructure only): compressible
neo-Hookean (model 0) and co-rotational linear elasticity (model 1).

The paper (Sec. III-A) names a Neo-Hookean model for the skin without giving its
form. Reading used here: the standard compressible form

    Psi(F) = mu/2 (I1 - 3) - mu ln J + lam/2 (ln J)^2,   I1 = tr(F^T F), J = det F,

with Lame parameters mu = E / (2(1+nu)), lam = E nu / ((1+nu)(1-2nu)). It reduces
to isotropic linear elasticity at small strain.

    P(F)   = dPsi/dF = mu (F - F^-T) + lam ln J F^-T
    dP     = mu dF + (mu - lam ln J) F^-T dF^T F^-T + lam tr(F^-1 dF) F^-T

Co-rotational linear elasticity (model 1). The paper's simulator models the
skin with a co-rotational linear-elastic law (Sec. III-A) and does not print
its form. Reading used here: the standard energy

    Psi(F) = mu ||F - R||_F^2 + lam/2 (tr(R^T F) - 3)^2,   F = R S (polar),

that is mu ||S - I||^2 + lam/2 (tr S - 3)^2, with the same Lame parameters. Then

    P(F) = 2 mu (F - R) + lam (tr S - 3) R,
    dP   = 2 mu dF + (lam (tr S - 3) - 2 mu) dR + lam tr(R^T dF) R,
    dR   = R [w]_x,  (tr S I - S) w = axial(R^T dF - dF^T R),

where [w]_x is the cross-product matrix and axial([a]_x) = a. The formula for
dR comes from differentiating F = R S and keeping the antisymmetric part, using
[w]_x S + S [w]_x = [(tr S I - S) w]_x for symmetric S. It is valid for
det F > 0, the only states the solver accepts.

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


NEO_HOOKEAN, COROTATED = 0, 1


def polar(F):
    """(R, S) with F = R S, R a rotation, S symmetric positive definite, from
    the SVD F = W diag(s) Z^T: R = W Z^T, S = Z diag(s) Z^T (det F > 0)."""
    W, s, Zt = np.linalg.svd(F)
    R = W @ Zt
    S = np.swapaxes(Zt, -1, -2) @ (s[..., :, None] * Zt)
    return R, S


def corot_energy_density(F, mu, lam):
    """Psi(F) of the co-rotational law; NaN where det F <= 0."""
    J = np.linalg.det(F)
    R, S = polar(F)
    E = S - np.eye(3)
    trE = np.trace(E, axis1=-2, axis2=-1)
    psi = mu * np.einsum("...ij,...ij->...", E, E) + 0.5 * lam * trE * trE
    return np.where(J > 0, psi, np.nan)


def corot_pk1(F, mu, lam):
    R, S = polar(F)
    trE = np.trace(S, axis1=-2, axis2=-1) - 3.0
    mu = np.asarray(mu)[..., None, None]
    lam = np.asarray(lam)[..., None, None]
    return 2.0 * mu * (F - R) + lam * trE[..., None, None] * R


def _cross_matrix(w):
    z = np.zeros(w.shape[:-1])
    return np.stack([np.stack([z, -w[..., 2], w[..., 1]], -1),
                     np.stack([w[..., 2], z, -w[..., 0]], -1),
                     np.stack([-w[..., 1], w[..., 0], z], -1)], -2)


def corot_dpdf(F, mu, lam):
    """Exact dP/dF of the co-rotational law as (..., 9, 9), column 3k+l = dP
    for dF = e_k e_l^T, through the polar-decomposition derivative above."""
    R, S = polar(F)
    trS = np.trace(S, axis1=-2, axis2=-1)
    mu = np.asarray(mu, dtype=np.float64)[..., None, None]
    lam = np.asarray(lam, dtype=np.float64)[..., None, None]
    Minv = np.linalg.inv(trS[..., None, None] * np.eye(3) - S)
    cols = []
    for k in range(3):
        for l in range(3):
            dF = np.zeros(F.shape)
            dF[..., k, l] = 1.0
            RtdF = np.swapaxes(R, -1, -2) @ dF
            Aq = RtdF - np.swapaxes(RtdF, -1, -2)
            a = np.stack([Aq[..., 2, 1], Aq[..., 0, 2], Aq[..., 1, 0]], -1)
            w = np.einsum("...ij,...j->...i", Minv, a)
            dR = R @ _cross_matrix(w)
            tr = np.trace(RtdF, axis1=-2, axis2=-1)[..., None, None]
            dP = 2.0 * mu * dF + (lam * (trS[..., None, None] - 3.0) - 2.0 * mu) * dR + lam * tr * R
            cols.append(dP.reshape(dP.shape[:-2] + (9,)))
    return np.stack(cols, -1)


def law_energy_density(F, mu, lam, model):
    """Psi(F) per element for a per-element model id (0 neo-Hookean, 1 co-rotational)."""
    model = np.asarray(model)
    out = energy_density(F, mu, lam)
    c = model == COROTATED
    if np.any(c):
        out = np.array(out, dtype=np.float64)
        out[c] = corot_energy_density(F[c], np.asarray(mu)[c], np.asarray(lam)[c])
    return out


def law_pk1(F, mu, lam, model):
    model = np.asarray(model)
    c = model == COROTATED
    out = np.zeros(F.shape)
    if np.any(~c):
        out[~c] = pk1(F[~c], np.asarray(mu)[~c], np.asarray(lam)[~c])
    if np.any(c):
        out[c] = corot_pk1(F[c], np.asarray(mu)[c], np.asarray(lam)[c])
    return out


def law_dpdf(F, mu, lam, model):
    model = np.asarray(model)
    c = model == COROTATED
    out = np.zeros(F.shape[:-2] + (9, 9))
    if np.any(~c):
        out[~c] = dpdf(F[~c], np.asarray(mu)[~c], np.asarray(lam)[~c])
    if np.any(c):
        out[c] = corot_dpdf(F[c], np.asarray(mu)[c], np.asarray(lam)[c])
    return out


def cauchy(F, mu, lam, model=None):
    """Cauchy stress sigma = P F^T / J (Sec. III-A of the paper reports element
    stress tensors; this is their true-stress form). Computed from the first
    Piola-Kirchhoff stress, the definition, so that a mistake in either shows
    in the pins."""
    J = np.linalg.det(F)
    P = pk1(F, mu, lam) if model is None else law_pk1(F, mu, lam, model)
    return P @ np.swapaxes(F, -1, -2) / J[..., None, None]


def von_mises(sigma):
    """Equivalent stress sqrt(3/2 s:s) of the deviator s = sigma - tr(sigma)/3 I."""
    tr = np.trace(sigma, axis1=-2, axis2=-1)
    s = sigma - tr[..., None, None] / 3.0 * np.eye(3)
    return np.sqrt(1.5 * np.einsum("...ij,...ij->...", s, s))
