"""Pins of the oracle's spectral operators (Sec. 4.1, Eq. (GFourier)) against closed forms.

* gradient of a trigonometric polynomial is known exactly; the Nyquist mode has zero derivative
  (the Nyquist reading);
* the spectral divergence is minus the adjoint of the gradient (integration by parts);
* G^ is an orthogonal projection: idempotent, self-adjoint, G^(uniform) = 0;
* compatible fields pass through G^ unchanged (the projection property of the Galerkin operator);
* an Airy-stress (divergence-free) field is annihilated by G^.
"""
import numpy as np
import pytest

from oracle import spectral as sp

RNG = np.random.default_rng(0)


def _grid_xyz(shape):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.astype(float), y.astype(float), z.astype(float)


@pytest.mark.parametrize("shape,k,m", [((1, 16, 32), 3, 5), ((1, 8, 8), 1, 3), ((4, 8, 16), 7, -2)])
def test_gradient_of_trig_polynomial(shape, k, m):
    nz, ny, nx = shape
    x, y, _ = _grid_xyz(shape)
    arg = 2 * np.pi * (k * x / nx + m * y / ny)
    u = np.sin(arg)
    g = sp.grad(u, 3 if nz > 1 else 2)
    np.testing.assert_allclose(g[0], 2 * np.pi * k / nx * np.cos(arg), atol=1e-12)
    np.testing.assert_allclose(g[1], 2 * np.pi * m / ny * np.cos(arg), atol=1e-12)


def test_nyquist_mode_has_zero_derivative():
    shape = (1, 8, 16)
    x, y, _ = _grid_xyz(shape)
    u = np.cos(np.pi * x) + 0.5 * np.cos(np.pi * y)
    g = sp.grad(u, 2)
    assert np.abs(g).max() < 1e-13


@pytest.mark.parametrize("shape,d", [((1, 16, 8), 2), ((4, 8, 8), 3)])
def test_divergence_is_minus_adjoint_of_gradient(shape, d):
    u = RNG.standard_normal(shape)
    q = RNG.standard_normal((d,) + shape)
    lhs = np.sum(sp.grad(u, d) * q)
    rhs = -np.sum(u * sp.div(q, d))
    assert abs(lhs - rhs) < 1e-11 * max(1.0, abs(lhs))


@pytest.mark.parametrize("shape,d", [((1, 16, 32), 2), ((4, 8, 16), 3)])
def test_galerkin_projection_properties(shape, d):
    T = RNG.standard_normal((d, d) + shape)
    S = RNG.standard_normal((d, d) + shape)
    GT = sp.galerkin_G(T, d)
    np.testing.assert_allclose(sp.galerkin_G(GT, d), GT, atol=1e-13)         # idempotent
    a = np.sum(GT * S)
    b = np.sum(T * sp.galerkin_G(S, d))
    assert abs(a - b) < 1e-11 * np.sum(np.abs(T * S))                          # self-adjoint
    U = np.ones((d, d) + shape) * RNG.standard_normal((d, d, 1, 1, 1))
    assert np.abs(sp.galerkin_G(U, d)).max() < 1e-13                          # kills the mean
    u = RNG.standard_normal((d,) + shape)
    Fu = sp.sym_grad_vec(u, d)                                                # compatible field
    np.testing.assert_allclose(sp.galerkin_G(Fu, d), Fu, atol=1e-12)


def test_galerkin_annihilates_airy_stress():
    shape = (1, 16, 32)
    chi = RNG.standard_normal(shape)
    xi = sp.xi_tilde(shape)
    X = sp.fft(chi)
    d2 = lambda a, b: sp.ifft_real(-xi[a] * xi[b] * X)
    sig = np.empty((2, 2) + shape)
    sig[0, 0] = d2(1, 1)
    sig[1, 1] = d2(0, 0)
    sig[0, 1] = sig[1, 0] = -d2(0, 1)
    assert np.abs(sp.galerkin_G(sig, 2)).max() < 1e-12 * np.abs(sig).max()


def test_threaded_fft_backend_gives_the_same_transform():
    """The scipy.fft backend (used only to time the CPU baseline on all host cores) computes the
    same DFT as numpy.fft, to rounding."""
    rng = np.random.default_rng(9)
    u = rng.standard_normal((4, 8, 16))
    ref_f, ref_g = sp.fft(u), sp.grad(u, 3)
    try:
        sp.set_fft_workers(2)
        f, g = sp.fft(u), sp.grad(u, 3)
    finally:
        sp.set_fft_workers(None)
    assert np.abs(f - ref_f).max() < 1e-12 and np.abs(g - ref_g).max() < 1e-12
