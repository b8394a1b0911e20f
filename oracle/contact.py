"""Analytic signed distance of rigid indenters, FP64 (oracle; test infrastructure only).

The paper drives rigid indenters (spheres, cylinders, objects with edges) into
the fingertip (Sec. III-A, Sec. III-C). Contact here is node-versus-analytic
surface with a penalty: a candidate node at x with phi(x) < 0 (inside the
indenter) stores energy k/2 phi^2 (frictionless; the paper's Coulomb friction is
not part of this path).

Indenter description (identical to the library's): origin c, rotation R whose
columns are the local axes, shape parameters, all translated by d_k a at load
step k.
  sphere    radius r, centre c.                 phi = |x-c| - r
  cylinder  radius r, infinite, axis R e_z.      phi = |P_perp (x-c)| - r
  box       half extents h, local frame R.       exact box distance
  plane     outward face normal n = R e_z.       phi = (x-c).n (solid: phi<0)

Each function returns phi (N,), grad phi (N,3) and the Hessian (N,3,3).
"""
from __future__ import annotations

import numpy as np

SPHERE, CYLINDER, BOX, PLANE = 0, 1, 2, 3


def _outer(a, b):
    return np.einsum("ni,nj->nij", a, b)


def sdf(shape, origin, R, params, x):
    """Signed distance, gradient and Hessian at points x (N, 3)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    d = x - np.asarray(origin, dtype=np.float64)
    N = len(x)
    eye = np.broadcast_to(np.eye(3), (N, 3, 3))
    if shape == SPHERE:
        r = params[0]
        rho = np.linalg.norm(d, axis=1)
        n = d / rho[:, None]
        return rho - r, n, (eye - _outer(n, n)) / rho[:, None, None]
    if shape == CYLINDER:
        r = params[0]
        ax = R[:, 2]
        dp = d - np.outer(d @ ax, ax)
        rho = np.linalg.norm(dp, axis=1)
        n = dp / rho[:, None]
        Pax = np.outer(ax, ax)
        return rho - r, n, (eye - Pax[None] - _outer(n, n)) / rho[:, None, None]
    if shape == PLANE:
        nrm = R[:, 2]
        return d @ nrm, np.broadcast_to(nrm, (N, 3)).copy(), np.zeros((N, 3, 3))
    if shape == BOX:
        h = np.asarray(params[:3], dtype=np.float64)
        q = d @ R                                  # local coordinates
        closest = np.clip(q, -h, h)
        s = q - closest                            # nonzero on clamped axes only
        out_dist = np.linalg.norm(s, axis=1)
        outside = out_dist > 0
        phi = np.empty(N)
        g_loc = np.zeros((N, 3))
        H_loc = np.zeros((N, 3, 3))
        if outside.any():
            so = s[outside]
            do = out_dist[outside]
            n = so / do[:, None]
            clamped = (np.abs(q[outside]) > h).astype(np.float64)
            D = np.einsum("ni,ij->nij", clamped, np.eye(3))
            phi[outside] = do
            g_loc[outside] = n
            H_loc[outside] = (D - _outer(n, n)) / do[:, None, None]
        inside = ~outside
        if inside.any():
            qi = q[inside]
            gap = np.abs(qi) - h                   # <= 0 on every axis
            k = np.argmax(gap, axis=1)
            phi[inside] = gap[np.arange(len(k)), k]
            gi = np.zeros((len(k), 3))
            gi[np.arange(len(k)), k] = np.where(qi[np.arange(len(k)), k] >= 0, 1.0, -1.0)
            g_loc[inside] = gi
        grad = g_loc @ R.T
        H = np.einsum("ij,njk,lk->nil", R, H_loc, R)
        return phi, grad, H
    raise ValueError(shape)


def penalty(shape, origin, R, params, x, k):
    """Penalty energy per node, its gradient (= minus the contact force on the
    body), the exact Hessian and the Gauss-Newton Hessian k grad phi grad phi^T.
    Nodes with phi >= 0 or k == 0 contribute nothing."""
    phi, g, H = sdf(shape, origin, R, params, x)
    act = (phi < 0) & (k > 0)
    pm = np.where(act, phi, 0.0)
    energy = 0.5 * k * pm * pm
    grad = (k * pm)[:, None] * g
    gn = (k * act)[:, None, None] * _outer(g, g)
    hess = gn + (k * pm)[:, None, None] * H
    return energy, grad, hess, gn, act
