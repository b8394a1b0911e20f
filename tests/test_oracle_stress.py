"""Pins of the oracle's element stress output (Cauchy stress, von Mises)
against closed forms: the linear-elastic small-strain limit, a hydrostatic
stretch, frame rotation and symmetry."""
import numpy as np

from oracle.material import cauchy, lame, von_mises


def test_small_strain_limit_is_linear_elasticity():
    mu, lam = lame(1.0e6, 0.3)
    rng = np.random.default_rng(3)
    for _ in range(5):
        H = 1e-7 * rng.standard_normal((3, 3))
        eps = 0.5 * (H + H.T)
        lin = lam * np.trace(eps) * np.eye(3) + 2 * mu * eps
        sig = cauchy(np.eye(3) + H, mu, lam)
        assert np.abs(sig - lin).max() <= 1e-6 * np.abs(lin).max()


def test_hydrostatic_stretch():
    mu, lam = lame(2.0e5, 0.45)
    for s in (0.8, 1.0, 1.3):
        sig = cauchy(s * np.eye(3), mu, lam)
        p = (mu * (s * s - 1.0) + lam * np.log(s ** 3)) / s ** 3
        assert np.allclose(sig, p * np.eye(3), rtol=1e-12, atol=1e-9 * max(abs(p), 1.0))
        assert von_mises(sig) <= 1e-9 * max(abs(p), 1.0)


def test_uniaxial_von_mises_equals_the_stress():
    # a uniaxial Cauchy stress state: von Mises = |sigma_11|
    sig = np.diag([7.0, 0.0, 0.0])
    assert abs(von_mises(sig) - 7.0) <= 1e-12


def test_rotation_and_symmetry():
    mu, lam = lame(1.5e6, 0.45)
    rng = np.random.default_rng(4)
    F = np.eye(3) + 0.2 * rng.standard_normal((3, 3))
    if np.linalg.det(F) <= 0:
        F[0] *= -1
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    R = q * np.sign(np.linalg.det(q))
    s0 = cauchy(F, mu, lam)
    s1 = cauchy(R @ F, mu, lam)
    assert np.allclose(s0, s0.T, atol=1e-9 * np.abs(s0).max())
    assert np.allclose(s1, R @ s0 @ R.T, atol=1e-9 * np.abs(s0).max())
    assert abs(von_mises(s1) - von_mises(s0)) <= 1e-9 * von_mises(s0)
