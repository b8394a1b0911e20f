"""Pins for the oracle's co-rotational linear-elastic law (model 1; the law
the paper's simulator uses for the skin, Sec. III-A).

  - finite differences: energy -> P, P -> dP/dF;
  - at F = I the tangent is the isotropic linear-elasticity tensor
    lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk);
  - rigid rotations carry no energy and no stress, exactly (unlike linear
    elasticity); left and right rotations leave the energy unchanged;
  - energy from the singular values, taken from the eigenvalues of F^T F;
  - a pure stretch: P_zz = E (l_z - 1) with l_t - 1 = -nu (l_z - 1) laterally
    free, at any strain;
  - on the assembled problem: a cube on rollers under a prescribed top
    displacement takes that homogeneous state."""
import numpy as np
import pytest

import workloads as W
from oracle import Problem, material as M

RNG = np.random.default_rng(21)


def _rot(rng):
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    return q * np.sign(np.linalg.det(q))


def _random_F(n, amp=0.3):
    F = np.eye(3) + amp * RNG.standard_normal((n, 3, 3))
    F[np.linalg.det(F) <= 0.2] = np.eye(3)
    return F


def test_pk1_and_tangent_match_finite_differences():
    F = _random_F(6)
    mu, lam = M.lame(np.full(6, 1000.0), np.full(6, 0.35))
    P = M.corot_pk1(F, mu, lam)
    C = M.corot_dpdf(F, mu, lam)
    h = 1e-6
    for k in range(3):
        for l in range(3):
            d = np.zeros((6, 3, 3))
            d[:, k, l] = h
            fd = (M.corot_energy_density(F + d, mu, lam) - M.corot_energy_density(F - d, mu, lam)) / (2 * h)
            np.testing.assert_allclose(P[:, k, l], fd, rtol=1e-6, atol=1e-6 * np.abs(P).max())
            fdP = (M.corot_pk1(F + d, mu, lam) - M.corot_pk1(F - d, mu, lam)) / (2 * h)
            np.testing.assert_allclose(C[:, :, 3 * k + l], fdP.reshape(6, 9), rtol=1e-5,
                                       atol=1e-6 * np.abs(C).max())
    # a conservative law has a symmetric tangent
    np.testing.assert_allclose(C, np.swapaxes(C, -1, -2), atol=1e-9 * np.abs(C).max())


def test_tangent_at_rest_is_linear_elasticity():
    mu, lam = 3.0, 7.0
    C = M.corot_dpdf(np.eye(3)[None], np.array([mu]), np.array([lam]))[0]
    d = np.eye(3)
    ref = (lam * np.einsum("ij,kl->ijkl", d, d)
           + mu * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)))
    np.testing.assert_allclose(C, ref.reshape(9, 9), atol=1e-12)
    # both laws share the small-strain limit
    np.testing.assert_allclose(M.dpdf(np.eye(3)[None], mu, lam)[0], ref.reshape(9, 9), atol=1e-12)


def test_rotations_are_free_and_invariant():
    mu, lam = np.full(4, 2.0), np.full(4, 5.0)
    Q = np.stack([_rot(RNG) for _ in range(4)])
    assert np.abs(M.corot_energy_density(Q, mu, lam)).max() < 1e-24
    assert np.abs(M.corot_pk1(Q, mu, lam)).max() < 1e-13
    F = _random_F(4)
    Q2 = np.stack([_rot(RNG) for _ in range(4)])
    e = M.corot_energy_density(F, mu, lam)
    np.testing.assert_allclose(M.corot_energy_density(Q @ F, mu, lam), e, rtol=1e-12)
    np.testing.assert_allclose(M.corot_energy_density(F @ Q2, mu, lam), e, rtol=1e-12)
    np.testing.assert_allclose(M.corot_pk1(Q @ F, mu, lam), Q @ M.corot_pk1(F, mu, lam), atol=1e-12)


def test_energy_from_singular_values():
    F = _random_F(5, 0.4)
    mu, lam = np.full(5, 1.5), np.full(5, 4.0)
    s = np.sqrt(np.linalg.eigvalsh(np.swapaxes(F, -1, -2) @ F))
    psi = mu * ((s - 1) ** 2).sum(-1) + 0.5 * lam * (s.sum(-1) - 3) ** 2
    np.testing.assert_allclose(M.corot_energy_density(F, mu, lam), psi, rtol=1e-12)


@pytest.mark.parametrize("lz", [0.6, 0.9, 1.3])
def test_pure_stretch_uniaxial(lz):
    E, nu = 2.0e3, 0.3
    mu, lam = M.lame(E, nu)
    lt = 1.0 - nu * (lz - 1.0)
    Q = _rot(RNG)
    F = Q @ np.diag([lt, lt, lz])          # any rotation of the stretched state
    P = np.linalg.solve(Q, M.corot_pk1(F[None], np.array([mu]), np.array([lam]))[0])
    assert P[2, 2] == pytest.approx(E * (lz - 1.0), rel=1e-12)
    assert abs(P[0, 0]) < 1e-9 * E and abs(P[1, 1]) < 1e-9 * E
    assert np.abs(P - np.diag(np.diag(P))).max() < 1e-9 * E


def corot_cube_uniaxial(n=3, strain=-0.2, E=1.0e3, nu=0.3):
    """Unit cube, symmetry rollers on x=0, y=0, z=0, top face z=1 prescribed
    u_z = strain, all co-rotational."""
    m = W.cube_mesh(n, E=E, nu=nu, fix="rollers")
    m.materials = np.array([[E, nu, 1.0]])
    X = m.nodes
    top = np.nonzero(X[:, 2] > 1 - 1e-9)[0]
    fixed = list(m.fixed_nodes)
    mask = list(m.fixed_mask)
    for t in top:
        if t in fixed:
            mask[fixed.index(t)] |= 4
        else:
            fixed.append(int(t))
            mask.append(4)
    m.fixed_nodes = np.array(fixed, dtype=np.int32)
    m.fixed_mask = np.array(mask, dtype=np.uint8)
    vals = np.zeros((len(fixed), 3))
    vals[:, 2] = np.where(X[fixed, 2] > 1 - 1e-9, strain, 0.0)
    return m, vals


def test_cube_on_rollers_takes_homogeneous_uniaxial_state():
    strain, E, nu = -0.2, 1.0e3, 0.3
    m, vals = corot_cube_uniaxial(3, strain, E, nu)
    ind = W.plane_indenter(50.0, 0.0, 4)       # far away: no contact
    p = Problem(m, ind, dirichlet_values=vals)
    r = p.solve(tol=1e-10)          # FP64 rounding floor of this residual: ~5e-12 * scale
    assert r.converged
    X = m.nodes
    lz = 1.0 + strain
    np.testing.assert_allclose(r.u[:, 2], strain * X[:, 2], atol=1e-10)
    np.testing.assert_allclose(r.u[:, 0], -nu * strain * X[:, 0], atol=1e-10)
    np.testing.assert_allclose(r.u[:, 1], -nu * strain * X[:, 1], atol=1e-10)
    # the top-face reactions sum to the nominal stress times the face area
    top = X[:, 2] > 1 - 1e-9
    assert r.reactions[top, 2].sum() == pytest.approx(E * (lz - 1.0), rel=1e-9)
