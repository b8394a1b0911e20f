"""Pins for oracle/material.py: textbook limits, finite differences, frame
invariance and an independent principal-stretch eigen-analysis."""
import numpy as np
import pytest

from oracle import material as M

RNG = np.random.default_rng(7)


def _rand_F(scale=0.2, n=8):
    F = np.eye(3) + scale * RNG.standard_normal((n, 3, 3))
    F[np.linalg.det(F) <= 0] = np.eye(3)
    return F


def test_lame_textbook():
    mu, lam = M.lame(1.0, 0.25)
    assert mu == pytest.approx(0.4) and lam == pytest.approx(0.4)
    mu, lam = M.lame(2.6, 0.3)      # G = E/2.6
    assert mu == pytest.approx(1.0)
    assert lam == pytest.approx(2.6 * 0.3 / (1.3 * 0.4))


def test_rest_state():
    F = np.eye(3)[None]
    assert M.energy_density(F, 1.0, 2.0)[0] == pytest.approx(0.0, abs=1e-15)
    assert np.abs(M.pk1(F, 1.0, 2.0)).max() < 1e-15


def test_small_strain_tangent_is_linear_elasticity():
    """dP/dF at F = I equals lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk)."""
    mu, lam = 0.7, 1.9
    C = M.dpdf(np.eye(3)[None], np.array([mu]), np.array([lam]))[0]
    d = np.eye(3)
    ref = (lam * np.einsum("ij,kl->ijkl", d, d) + mu * np.einsum("ik,jl->ijkl", d, d)
           + mu * np.einsum("il,jk->ijkl", d, d)).reshape(9, 9)
    np.testing.assert_allclose(C, ref, atol=1e-14)


@pytest.mark.parametrize("scale", [0.05, 0.3])
def test_pk1_is_energy_gradient(scale):
    F = _rand_F(scale)
    mu, lam = 1.3, 5.0
    P = M.pk1(F, np.full(len(F), mu), np.full(len(F), lam))
    eps = 1e-6
    for i in range(3):
        for j in range(3):
            dF = np.zeros((3, 3))
            dF[i, j] = eps
            fd = (M.energy_density(F + dF, mu, lam) - M.energy_density(F - dF, mu, lam)) / (2 * eps)
            np.testing.assert_allclose(P[:, i, j], fd, rtol=1e-7, atol=1e-8)


@pytest.mark.parametrize("scale", [0.05, 0.3])
def test_dpdf_is_pk1_derivative(scale):
    F = _rand_F(scale)
    n = len(F)
    mu, lam = np.full(n, 1.3), np.full(n, 5.0)
    C = M.dpdf(F, mu, lam)
    eps = 1e-6
    for _ in range(4):
        dF = RNG.standard_normal((3, 3))
        fd = (M.pk1(F + eps * dF, mu, lam) - M.pk1(F - eps * dF, mu, lam)) / (2 * eps)
        lin = np.einsum("nab,b->na", C, dF.ravel()).reshape(n, 3, 3)
        np.testing.assert_allclose(lin, fd, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(C, np.swapaxes(C, 1, 2), atol=1e-12)   # major symmetry


def test_frame_invariance():
    F = _rand_F(0.3)
    q, _ = np.linalg.qr(RNG.standard_normal((3, 3)))
    Q = q * np.sign(np.linalg.det(q))
    QF = np.einsum("ij,njk->nik", Q, F)
    np.testing.assert_allclose(M.energy_density(QF, 1.0, 3.0), M.energy_density(F, 1.0, 3.0),
                               rtol=1e-12, atol=1e-14)
    P = M.pk1(F, np.ones(len(F)), np.full(len(F), 3.0))
    np.testing.assert_allclose(M.pk1(QF, np.ones(len(F)), np.full(len(F), 3.0)),
                               np.einsum("ij,njk->nik", Q, P), atol=1e-12)


def _principal_eigs(s, mu, lam):
    """Eigenvalues of dP/dF at F = U diag(s) V^T from the principal-stretch
    decomposition (Teran et al. 2005; Smith et al. 2018): for each pair i<j the
    two values mu +/- c/(s_i s_j), c = mu - lam ln J, and the eigenvalues of the
    3x3 block A = diag(mu + c/s_i^2) + lam (1/s)(1/s)^T."""
    J = np.prod(s)
    c = mu - lam * np.log(J)
    out = []
    for i, j in [(0, 1), (0, 2), (1, 2)]:
        out += [mu + c / (s[i] * s[j]), mu - c / (s[i] * s[j])]
    inv = 1.0 / s
    A = np.diag(mu + c * inv * inv) + lam * np.outer(inv, inv)
    out += list(np.linalg.eigvalsh(A))
    return np.sort(out)


@pytest.mark.parametrize("s", [(1.0, 1.0, 1.0), (0.8, 0.9, 0.7), (1.3, 0.6, 1.05), (0.5, 0.5, 0.95)])
def test_dpdf_spectrum_matches_principal_analysis(s):
    s = np.array(s)
    mu, lam = 0.5, 12.0
    q1, _ = np.linalg.qr(RNG.standard_normal((3, 3)))
    q2, _ = np.linalg.qr(RNG.standard_normal((3, 3)))
    U = q1 * np.sign(np.linalg.det(q1))
    V = q2 * np.sign(np.linalg.det(q2))
    F = U @ np.diag(s) @ V.T
    C = M.dpdf(F[None], np.array([mu]), np.array([lam]))[0]
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(C)), _principal_eigs(s, mu, lam),
                               rtol=1e-10, atol=1e-10)
    Cp = M.project_psd(C[None])[0]
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(Cp)),
                               np.maximum(_principal_eigs(s, mu, lam), 0.0), atol=1e-10)


def test_projection_is_identity_on_psd():
    F = np.diag([1.1, 1.05, 1.1])[None]          # stretched: c < mu s_i s_j, exact tangent PD
    C = M.dpdf(F, np.array([1.0]), np.array([4.0]))
    assert np.linalg.eigvalsh(C[0]).min() > 0
    np.testing.assert_allclose(M.project_psd(C), C, atol=1e-12)
