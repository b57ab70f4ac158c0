"""Pins of the oracle's constitutive pieces.

* Eq. (Crot): an isotropic tensor is invariant under any rotation; a cubic tensor rotated about
  [001] follows the textbook closed forms C'11 = C11 - 2 D s^2 c^2, C'12 = C12 + 2 D s^2 c^2,
  C'66 = C44 + 2 D s^2 c^2 with D = C11 - C12 - 2 C44; 90 degree rotations leave it unchanged.
* Eq. (zener): z = 2 C1212 / (C1111 - C1122) = 1 is isotropy.
* Eq. (PFFani): beta = 0 gives A = I; A has eigenvalue 1 along n_pl and 1 + beta across it.
* Sec. 2.1: g(0) = 1 + k, g(1) = k, g' = dg/dphi (finite differences).
* Spectral split: psi+ + psi- = psi_o, sigma+- = d psi+- / d eps and the tangent = d sigma / d eps
  (central differences), pure tension has psi- = 0.
"""
import numpy as np
import pytest

from oracle import material as mat

RNG = np.random.default_rng(1)


def _rand_rot():
    q = RNG.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def test_isotropic_invariant_under_rotation():
    lam, mu = 0.7, 0.4
    C = mat.cubic_tensor(lam + 2 * mu, lam, mu)
    d = np.eye(3)
    ref = lam * np.einsum("ij,kl->ijkl", d, d) + mu * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d))
    np.testing.assert_allclose(C, ref, atol=1e-15)
    for _ in range(5):
        np.testing.assert_allclose(mat.rotate_stiffness(C, _rand_rot()), C, atol=1e-13)


@pytest.mark.parametrize("theta", [0.3, 0.7854, 1.2, 2.9])
def test_cubic_rotation_about_z_closed_form(theta):
    c11, c12, c44 = 1.0, 0.6, 0.5
    c, s = np.cos(theta), np.sin(theta)
    R = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])
    Cr = mat.rotate_stiffness(mat.cubic_tensor(c11, c12, c44), R)
    D = c11 - c12 - 2 * c44
    assert abs(Cr[0, 0, 0, 0] - (c11 - 2 * D * s * s * c * c)) < 1e-14
    assert abs(Cr[0, 0, 1, 1] - (c12 + 2 * D * s * s * c * c)) < 1e-14
    assert abs(Cr[0, 1, 0, 1] - (c44 + 2 * D * s * s * c * c)) < 1e-14
    assert abs(Cr[2, 2, 2, 2] - c11) < 1e-14
    # major and minor symmetries survive the rotation
    np.testing.assert_allclose(Cr, np.transpose(Cr, (2, 3, 0, 1)), atol=1e-15)
    np.testing.assert_allclose(Cr, np.transpose(Cr, (1, 0, 2, 3)), atol=1e-15)


def test_cubic_invariant_under_quarter_turns():
    C = mat.cubic_tensor(1.0, 0.6, 0.5)
    Rz = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1.0]])
    Rx = np.array([[1, 0, 0], [0, 0, -1], [0, 1, 0.0]])
    np.testing.assert_allclose(mat.rotate_stiffness(C, Rz), C, atol=1e-15)
    np.testing.assert_allclose(mat.rotate_stiffness(C, Rx), C, atol=1e-15)


def test_zener_one_is_isotropic():
    c11, c12 = 24.0, 8.0
    c44 = 1.0 * (c11 - c12) / 2.0          # Eq. (zener) with z = 1
    C = mat.cubic_tensor(c11, c12, c44)
    np.testing.assert_allclose(mat.rotate_stiffness(C, _rand_rot()), C, atol=1e-12)


def test_cleavage_tensor():
    R = _rand_rot()
    np.testing.assert_allclose(mat.cleavage_tensor(R, [1, 0, 0], 0.0, 3), np.eye(3), atol=0)
    beta = 2.0
    A = mat.cleavage_tensor(R, [0, 1, 0], beta, 3)
    n = R @ np.array([0, 1.0, 0])
    np.testing.assert_allclose(A @ n, n, atol=1e-14)
    t = np.cross(n, RNG.standard_normal(3))
    np.testing.assert_allclose(A @ t, (1 + beta) * t, atol=1e-13)
    th = 0.4
    R2 = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    A2 = mat.cleavage_tensor(R2, [1, 0, 0], beta, 2)
    n2 = np.array([np.cos(th), np.sin(th)])
    np.testing.assert_allclose(A2, np.eye(2) + beta * (np.eye(2) - np.outer(n2, n2)), atol=1e-15)


def test_degradation():
    k = 1e-6
    assert mat.degradation(0.0, k) == 1.0 + k and mat.degradation(1.0, k) == k
    for phi in (0.1, 0.5, 0.93):
        h = 1e-6
        fd = (mat.degradation(phi + h, k) - mat.degradation(phi - h, k)) / (2 * h)
        assert abs(fd - mat.degradation_prime(phi)) < 1e-9


def sc(a):
    return float(np.asarray(a).reshape(-1)[0])


def _fields(eps2):
    e = np.asarray(eps2, float).reshape(2, 2, 1, 1, 1)
    return e


@pytest.mark.parametrize("eps", [[[0.3, 0.1], [0.1, -0.2]], [[0.5, 0.0], [0.0, 0.2]],
                                 [[-0.4, 0.05], [0.05, -0.1]], [[0.1, 0.3], [0.3, 0.1]]])
def test_split_energy_stress_tangent(eps):
    lam, mu = np.full((1, 1, 1), 0.577), np.full((1, 1, 1), 0.385)
    e = _fields(eps)
    pp, pm, sp_, sm_ = mat.split_parts(e, lam, mu)
    psi_o = 0.5 * lam * np.trace(e[:, :, 0, 0, 0]) ** 2 + mu * np.sum(e * e)
    assert abs(sc(pp + pm) - sc(psi_o)) < 1e-14
    h = 1e-6
    for part, sig in ((0, sp_), (1, sm_)):
        for i in range(2):
            for j in range(2):
                dE = np.zeros_like(e)
                dE[i, j] += 0.5 * h
                dE[j, i] += 0.5 * h
                fp = mat.split_parts(e + dE, lam, mu)[part]
                fm = mat.split_parts(e - dE, lam, mu)[part]
                fd = sc((fp - fm) / (2 * h))
                w = 1.0                             # dE is symmetric with dE:sigma = h sigma_ij
                assert abs(fd - w * sc(sig[i, j])) < 1e-8
    g = np.full((1, 1, 1), 0.37)
    for _ in range(3):
        dE = RNG.standard_normal((2, 2, 1, 1, 1))
        dE = 0.5 * (dE + np.swapaxes(dE, 0, 1))
        an = mat.split_tangent_apply(e, dE, lam, mu, g)
        s = lambda x: (lambda r: g * r[2] + r[3])(mat.split_parts(x, lam, mu))
        fd = (s(e + h * dE) - s(e - h * dE)) / (2 * h)
        np.testing.assert_allclose(an, fd, atol=1e-7)


def test_split_pure_tension_and_compression():
    lam, mu = np.full((1, 1, 1), 0.5), np.full((1, 1, 1), 0.3)
    pp, pm, _, _ = mat.split_parts(_fields([[0.2, 0.0], [0.0, 0.1]]), lam, mu)
    assert sc(pm) == 0.0 and sc(pp) > 0
    pp, pm, _, _ = mat.split_parts(_fields([[-0.2, 0.0], [0.0, -0.1]]), lam, mu)
    assert sc(pp) == 0.0 and sc(pm) > 0
