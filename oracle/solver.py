"""Quasi-static Newton solve of the indentation problem, FP64 (oracle; test
infrastructure only).

At every load step k the equilibrium is a local minimiser of

    Pi_k(u) = sum_e V_e Psi(F_e(u)) + sum_{i candidate} k_i/2 min(0, phi_k(X_i+u_i))^2

subject to the prescribed displacements on fixed DOFs, where phi_k is the
indenter's signed distance with the indenter translated to origin + d_k a
(Sec. III-A of the paper: tet FEM with a per-element hyperelastic model, rigid
indenters driven into the body, nodal positions and nodal contact forces as
outputs). The paper solves a dynamic problem with its own GPU Newton solver;
this oracle solves the quasi-static problem plainly:

  1. element energy, gradient and exact tangent (material.py) assembled into a
     global sparse matrix (scipy.sparse COO -> CSR, duplicates summed);
  2. the Newton direction from a direct sparse LU solve (SuperLU, minimum
     degree ordering on K+K^T) of the exact
     tangent restricted to the free DOFs; if that direction is not a descent
     direction, the solve is repeated with the element-wise PSD-projected
     tangent plus the Gauss-Newton contact term;
  3. backtracking Armijo line search on Pi (c1 = 1e-4, halving) while the
     residual is above 1e-3 * scale, plain steps below that; every trial step
     must keep J > 0 in every tet;
  4. convergence when ||R_free||_2 <= tol * scale with
     scale = max(||f_c||_2, E_max h_bar^2 1e-3), f_c the nodal contact forces;
  5. load steps solved in order, each warm-started from the previous one.

Prescribed (Dirichlet) values, when given, are ramped linearly over the load
steps: at step k the fixed DOFs hold values * k / K.

Friction (mu_f > 0). The paper's contact is isotropic Coulomb (Sec. III-A).
Reading: at each load step the nodes' normal force magnitudes fn_i = k_i
max(0, -phi_i) and SDF normals n_i are taken at the start of the step (the
previous converged state, indenter at its previous pose) and frozen, and
Pi_k gains the smoothed dissipation potential sum_i mu_f fn_i f0(|s_i|) of
contact.friction, with s_i the tangential slip of node i relative to the
indenter's translation over the step and the smoothing slip
eps = fric_eps_rel * h_bar. The reported contact forces include the
friction forces. With friction_passes = n > 1 each load step is solved n times:
after each solve the normal forces and normals are frozen again at the
current state, with the indenter at this step's pose (the slip still counts
from the step's start); the passes converge to friction that uses the step's
own normal forces.

Dynamic stepping (dt > 0). The paper integrates the deformable body's dynamics
implicitly in time, with a time step of 1e-4 s (Sec. III-A). Reading: backward
(implicit) Euler with a lumped mass matrix, m_i = rho * sum over the tets at
node i of V_e / 4. Every load step is then one time step. Its solution is the
minimiser of the incremental potential

    Phi_k(u) = Pi_k(u) + sum_{i, free DOFs} m_i / (2 dt^2) (u_i - u~_i)^2,
    u~ = u_{k-1} + dt v_{k-1},

and the velocity is updated afterwards as v_k = (u_k - u_{k-1}) / dt. Setting
the gradient to zero gives m (v_k - v_{k-1}) / dt = -grad Pi_k(u_k), which is
backward Euler. Prescribed components carry no inertia term, because on them
the term would only be a constant. The body starts at rest unless a v0 is
given (only the oracle takes v0; the pins use it).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import contact, geometry, material


@dataclasses.dataclass
class SolveResult:
    u: np.ndarray                 # (Nn, 3) displacement at the last solved step
    step_force: np.ndarray        # (K, 3) resultant contact force on the body per step
    nodal_contact: np.ndarray     # (Nn, 3) nodal contact forces at the last step
    reactions: np.ndarray         # (Nn, 3) support forces on fixed DOFs, last step
    newton_iters: np.ndarray      # (K,)
    residual: np.ndarray          # (K,) final ||R_free||_2 per step
    scale: np.ndarray             # (K,) convergence scale per step
    converged: bool
    projected_directions: int     # Newton steps that needed the PSD fallback
    step_u: list                  # displacement after each step


class Problem:
    """One mesh + one indenter (+ optional prescribed values on fixed DOFs)."""

    def __init__(self, mesh, indenter, c_kappa: float = 100.0, dirichlet_values=None,
                 dt: float = 0.0, density: float = 1.1e-9, mu_f: float = 0.0,
                 fric_eps_rel: float = 0.01, friction_passes: int = 1):
        self.X = np.asarray(mesh.nodes, dtype=np.float64)
        self.tets = np.asarray(mesh.tets, dtype=np.int64)
        self.n = len(self.X)
        mats = np.asarray(mesh.materials, dtype=np.float64)
        tm = np.asarray(mesh.tet_material, dtype=np.int64)
        self.E = mats[tm, 0]
        self.mu, self.lam = material.lame(mats[tm, 0], mats[tm, 1])
        # element law per material: column 2 (if present) 0 neo-Hookean, 1 co-rotational
        self.model = (mats[tm, 2].astype(np.int64) if mats.shape[1] > 2
                      else np.zeros(len(tm), dtype=np.int64))
        _, self.Dminv, self.V = geometry.shape_matrices(self.X, self.tets)
        if np.any(self.V <= 0):
            raise ValueError("non-positive tet volume")
        self.grads = geometry.shape_gradients(self.Dminv)        # (Nt, 4, 3)
        self.fixed = geometry.fixed_dof_mask(self.n, mesh.fixed_nodes, mesh.fixed_mask)
        self.free = ~self.fixed.ravel()
        self.k, self.h_bar, _ = geometry.penalty_stiffness(
            self.X, self.tets, self.E, self.fixed, c_kappa)
        # lumped mass: a quarter of each tet's mass to each of its nodes
        self.dt = float(dt)
        self.mass = np.zeros(self.n)
        for a in range(4):
            np.add.at(self.mass, self.tets[:, a], 0.25 * float(density) * self.V)
        self.u_tilde = None      # inertial prediction u~ of the current time step (dt > 0)
        self.E_max = float(self.E.max())
        self.mu_f = float(mu_f)
        self.friction_passes = max(1, int(friction_passes))
        self.fric = None         # lagged friction state of the current load step
        self.scale_floor = self.E_max * self.h_bar ** 2 * 1e-3
        self.u_presc = np.zeros((self.n, 3))
        if dirichlet_values is not None:
            vals = np.asarray(dirichlet_values, dtype=np.float64).reshape(-1, 3)
            fn = np.asarray(mesh.fixed_nodes, dtype=np.int64)
            self.u_presc[fn] = vals
            self.u_presc[~self.fixed] = 0.0
        self.shape = int(indenter.shape)
        self.origin0 = np.asarray(indenter.origin, dtype=np.float64)
        self.R = np.asarray(indenter.rotation, dtype=np.float64)
        self.params = np.asarray(indenter.params, dtype=np.float64)
        self.a = np.asarray(indenter.direction, dtype=np.float64)
        self.depths = np.asarray(indenter.depth_schedule, dtype=np.float64)
        self.K = len(self.depths)
        self.fric_eps = float(fric_eps_rel) * self.h_bar
        # element -> global DOF map for assembly
        dof = (3 * self.tets[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 12)
        self._rows = np.repeat(dof, 12, axis=1).ravel()
        self._cols = np.tile(dof, (1, 12)).ravel()

    # ------------------------------------------------------------ pieces
    def origin_at(self, step: int) -> np.ndarray:
        """Indenter origin at load step ``step`` (1-based; 0 = initial contact)."""
        d = 0.0 if step == 0 else self.depths[step - 1]
        return self.origin0 + d * self.a

    def F(self, u):
        return geometry.deformation_gradient(self.X + u, self.tets, self.Dminv)

    def elastic_energy(self, u):
        F = self.F(u)
        J = np.linalg.det(F)
        if np.any(J <= 0):
            return np.inf, float(J.min())
        psi = material.law_energy_density(F, self.mu, self.lam, self.model)
        return float(np.sum(self.V * psi)), float(J.min())

    def elastic_gradient(self, u):
        """Nodal gradient of the elastic energy (Nn, 3): sum_e V_e P_e grad N_a."""
        P = material.law_pk1(self.F(u), self.mu, self.lam, self.model)
        fe = np.einsum("e,eij,eaj->eai", self.V, P, self.grads)
        g = np.zeros((self.n, 3))
        for a in range(4):
            np.add.at(g, self.tets[:, a], fe[:, a])
        return g

    def element_tangents(self, u, projected=False):
        """Element stiffness (Nt, 12, 12) = V B^T C B."""
        C = material.law_dpdf(self.F(u), self.mu, self.lam, self.model)
        if projected:
            C = material.project_psd(C)
        C4 = C.reshape(-1, 3, 3, 3, 3)
        Ke = np.einsum("e,eaj,eijkl,ebl->eaibk", self.V, self.grads, C4, self.grads,
                       optimize=True)
        return Ke.reshape(-1, 12, 12)

    def contact_terms(self, u, step):
        x = self.X + u
        return contact.penalty(self.shape, self.origin_at(step), self.R, self.params, x, self.k)

    def inertia_terms(self, u):
        """(energy, gradient (Nn,3), diagonal (Nn,3)) of the backward-Euler
        inertia term sum_free m_i/(2 dt^2) |u_i - u~_i|^2; zeros when
        quasi-static."""
        if self.dt <= 0.0 or self.u_tilde is None:
            z = np.zeros((self.n, 3))
            return 0.0, z, z
        w = np.where(self.fixed, 0.0, (self.mass / self.dt ** 2)[:, None])
        d = u - self.u_tilde
        return float(0.5 * np.sum(w * d * d)), w * d, w

    def set_friction_lag(self, u_start, step):
        """Freeze the friction state of load step ``step`` at the converged
        displacement u_start of the previous step (indenter at its previous pose)."""
        x0 = self.X + u_start
        phi, n, _ = contact.sdf(self.shape, self.origin_at(step - 1), self.R, self.params, x0)
        fn = np.where((phi < 0) & (self.k > 0), -self.k * phi, 0.0)
        self.fric = dict(x_start=x0, dc=self.origin_at(step) - self.origin_at(step - 1),
                         normal=n, fn=fn)

    def refresh_friction(self, u, step):
        """Freeze the normal forces and normals again at the current state u,
        indenter at this step's pose; the slip origin and translation stay."""
        x = self.X + u
        phi, n, _ = contact.sdf(self.shape, self.origin_at(step), self.R, self.params, x)
        self.fric["normal"] = n
        self.fric["fn"] = np.where((phi < 0) & (self.k > 0), -self.k * phi, 0.0)

    def friction_terms(self, u):
        """(energy, gradient (Nn,3), Hessian blocks (Nn,3,3)) of the lagged
        friction potential; zeros when frictionless."""
        if self.mu_f <= 0.0 or self.fric is None:
            return 0.0, np.zeros((self.n, 3)), np.zeros((self.n, 3, 3))
        f = self.fric
        e, g, H = contact.friction(self.X + u, f["x_start"], f["dc"], f["normal"], f["fn"],
                                   self.mu_f, self.fric_eps)
        return float(e.sum()), g, H

    def energy(self, u, step):
        Ee, minJ = self.elastic_energy(u)
        ec = self.contact_terms(u, step)[0]
        return Ee + float(ec.sum()) + self.inertia_terms(u)[0] + self.friction_terms(u)[0], minJ

    def gradient(self, u, step):
        """(R, f_c): full gradient of Pi (plus the inertia and friction terms
        when present) (Nn,3) and nodal contact forces on the body (normal
        penalty plus friction)."""
        _, gc, _, _, _ = self.contact_terms(u, step)
        gf = self.friction_terms(u)[1]
        return self.elastic_gradient(u) + gc + gf + self.inertia_terms(u)[1], -(gc + gf)

    def hessian(self, u, step, projected=False):
        """Global tangent (3Nn x 3Nn CSR). Exact: exact element tangent + exact
        contact Hessian. Projected: PSD element tangent + Gauss-Newton contact."""
        Ke = self.element_tangents(u, projected)
        K = sp.coo_matrix((Ke.ravel(), (self._rows, self._cols)),
                          shape=(3 * self.n, 3 * self.n)).tocsr()
        _, _, hc, gn, _ = self.contact_terms(u, step)
        blocks = gn if projected else hc
        idx = np.arange(self.n)
        r = (3 * idx[:, None, None] + np.arange(3)[None, :, None]).repeat(3, axis=2)
        c = (3 * idx[:, None, None] + np.arange(3)[None, None, :]).repeat(3, axis=1)
        K = K + sp.coo_matrix((blocks.ravel(), (r.ravel(), c.ravel())),
                              shape=K.shape).tocsr()
        w = self.inertia_terms(u)[2]
        if np.any(w):
            K = K + sp.diags(w.ravel())
        if self.mu_f > 0.0 and self.fric is not None:
            Hf = self.friction_terms(u)[2]
            K = K + sp.coo_matrix((Hf.ravel(), (r.ravel(), c.ravel())), shape=K.shape).tocsr()
        return K

    def residual_norm(self, u, step):
        """(||R_free||_2, scale, ||f_c||_2) at a given displacement (certification)."""
        g, fc = self.gradient(u, step)
        rn = float(np.linalg.norm(g.ravel()[self.free]))
        fcn = float(np.linalg.norm(fc))
        return rn, max(fcn, self.scale_floor), fcn

    # ------------------------------------------------------------ Newton
    def _direction(self, u, step, g_free):
        for projected in (False, True):
            K = self.hessian(u, step, projected)
            Kff = K[self.free][:, self.free].tocsc()
            try:
                lu = spla.splu(Kff, permc_spec="MMD_AT_PLUS_A",
                               options=dict(SymmetricMode=True))
                d = lu.solve(-g_free)
            except RuntimeError:
                continue
            if np.all(np.isfinite(d)) and float(g_free @ d) < 0:
                return d, projected
        raise RuntimeError("no descent direction")

    def solve(self, tol: float = 1e-10, load_steps: int | None = None,
              max_newton: int = 100, max_backtracks: int = 60, u0=None,
              verbose: bool = False, v0=None) -> SolveResult:
        K = self.K if not load_steps else int(load_steps)
        u = np.zeros((self.n, 3)) if u0 is None else np.array(u0, dtype=np.float64)
        vel = np.zeros((self.n, 3)) if v0 is None else np.array(v0, dtype=np.float64)
        vel[self.fixed] = 0.0
        self.step_v = []
        step_force = np.zeros((K, 3))
        iters = np.zeros(K, dtype=np.int64)
        resid = np.zeros(K)
        scales = np.zeros(K)
        n_proj = 0
        converged = True
        step_u = []
        fc = np.zeros((self.n, 3))
        g = np.zeros((self.n, 3))
        for step in range(1, K + 1):
            u_prev = u.copy()
            if self.dt > 0.0:
                self.u_tilde = u_prev + self.dt * vel
            if self.mu_f > 0.0:
                self.set_friction_lag(u_prev, step)
            u[self.fixed] = (self.u_presc * (step / K))[self.fixed]
            passes = self.friction_passes if self.mu_f > 0.0 else 1
            ok = False
            it_total = 0
            for pss in range(passes):
              if pss > 0:
                  if not ok:
                      break
                  self.refresh_friction(u, step)
              ok = False
              for it in range(max_newton + 1):
                  g, fc = self.gradient(u, step)
                  g_free = g.ravel()[self.free]
                  rn = float(np.linalg.norm(g_free))
                  scale = max(float(np.linalg.norm(fc)), self.scale_floor)
                  if verbose:
                      print(f"step {step} it {it} |R|={rn:.3e} scale={scale:.3e}")
                  if rn <= tol * scale:
                      ok = True
                      break
                  if it == max_newton:
                      break
                  d_free, proj = self._direction(u, step, g_free)
                  n_proj += int(proj)
                  du = np.zeros(3 * self.n)
                  du[self.free] = d_free
                  du = du.reshape(-1, 3)
                  slope = float(g_free @ d_free)
                  e0, _ = self.energy(u, step)
                  alpha = 1.0
                  accepted = False
                  for _ in range(max_backtracks):
                      ut = u + alpha * du
                      et, minJ = self.energy(ut, step)
                      if minJ > 0 and np.isfinite(et):
                          if rn <= 1e-3 * scale or et <= e0 + 1e-4 * alpha * slope:
                              accepted = True
                              break
                      alpha *= 0.5
                  if not accepted:
                      break
                  u = ut
              it_total += it
            iters[step - 1] = it_total
            resid[step - 1] = rn
            scales[step - 1] = scale
            step_force[step - 1] = fc.sum(axis=0)
            step_u.append(u.copy())
            if self.dt > 0.0:
                vel = np.where(self.fixed, 0.0, (u - u_prev) / self.dt)
                self.step_v.append(vel.copy())
            if not ok:
                converged = False
                break
        reactions = np.where(self.fixed, g, 0.0)
        self.u_tilde = None
        self.fric = None
        return SolveResult(u, step_force, fc, reactions, iters, resid, scales,
                           converged, n_proj, step_u)
