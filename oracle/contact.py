"""Analytic signed distance of rigid indenters, FP64 (oracle; test infrastructure only).

The paper drives rigid indenters (spheres, cylinders, objects with edges) into
the fingertip (Sec. III-A, Sec. III-C). Contact here is node-versus-analytic
surface with a penalty: a candidate node at x with phi(x) < 0 (inside the
indenter) stores energy k/2 phi^2. Coulomb friction (the paper's contact model is
isotropic Coulomb, Sec. III-A) is optional, as a lagged and smoothed dissipation
potential (``friction`` below).

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


def friction_f0(y, eps):
    """Smoothed Coulomb magnitude: f0(y) = y^2/eps - y^3/(3 eps^2) + eps/3 below
    the slip eps, y above; C1 at eps, f0' rises from 0 to 1 over [0, eps]."""
    y = np.asarray(y, dtype=np.float64)
    return np.where(y < eps, y * y / eps - y ** 3 / (3 * eps * eps) + eps / 3, y)


def friction(x, x_start, dc, normal, fn, mu_f, eps):
    """Lagged, smoothed Coulomb friction of the nodes against a translating
    rigid indenter. Reading of the paper's Coulomb contact (Sec. III-A) for
    load steps solved by energy minimisation: per node the dissipation
    potential

        D_i(x) = mu_f fn_i f0(|s_i|),  s_i = (I - n_i n_i^T)(x_i - x_start_i - dc),

    with the normal n_i and the normal force magnitude fn_i frozen at the start
    of the load step (x_start, indenter at its previous pose), and dc the
    indenter's translation over the step. A node sliding by more than eps
    carries a friction force of magnitude mu_f fn_i against its slip relative
    to the indenter; below eps it sticks elastically with stiffness 2 mu_f
    fn_i / eps.

    Returns energy per node (N,), gradient (N,3) and the Hessian (N,3,3)
      mu_f fn [ (f1/y) P - q s s^T ],  P = I - n n^T, f1 = f0',
      q = 1/(eps^2 y) below eps, 1/y^3 above (PSD: eigenvalues 2/eps - 2y/eps^2
      or 0 along s, f1/y across it, 0 along n)."""
    r = np.asarray(x, dtype=np.float64) - x_start - np.asarray(dc, dtype=np.float64)
    n = np.asarray(normal, dtype=np.float64)
    s = r - np.einsum("ni,ni->n", n, r)[:, None] * n
    y = np.linalg.norm(s, axis=1)
    w = mu_f * np.asarray(fn, dtype=np.float64)
    energy = w * friction_f0(y, eps)
    below = y < eps
    ysafe = np.where(y > 0, y, 1.0)
    f1_over_y = np.where(below, 2.0 / eps - y / (eps * eps), 1.0 / ysafe)
    grad = (w * f1_over_y)[:, None] * s
    shat = s / ysafe[:, None]
    q_y2 = np.where(below, y / (eps * eps), 1.0 / ysafe)     # q * y^2
    P = np.eye(3)[None] - _outer(n, n)
    hess = w[:, None, None] * (f1_over_y[:, None, None] * P - q_y2[:, None, None] * _outer(shat, shat))
    return energy, grad, hess
