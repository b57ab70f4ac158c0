"""Spectral operators on a periodic voxel grid (oracle; test infrastructure only).

Fields live on numpy arrays of shape (nz, ny, nx) (nz = 1 for 2D); spatial direction a = 0, 1, 2
(x, y, z) maps to numpy axis 2 - a. Tensors carry leading component axes, e.g. (d, d, nz, ny, nx).

Frequencies (Sec. 4.1, "complex frequency vector"): xi_a = 2 pi k_a / n_a with k_a in FFT order,
grid spacing h = 1. In every odd-order derivative, and in G^, the Nyquist frequency k_a = n_a / 2
is set to zero (xi~); this keeps the derivative of a real field real and makes the spectral
gradient exactly skew-adjoint. It is a reading: the paper does not say how the Nyquist mode is
handled.
"""
from __future__ import annotations

import numpy as np


def xi_tilde(shape):
    """Return [xi~_x, xi~_y, xi~_z], each broadcastable to ``shape`` = (nz, ny, nx)."""
    out = []
    for a in range(3):
        n = shape[2 - a]
        k = np.fft.fftfreq(n) * n
        xi = 2.0 * np.pi * k / n
        if n % 2 == 0:
            xi[np.isclose(k, -n / 2)] = 0.0
        sh = [1, 1, 1]
        sh[2 - a] = n
        out.append(xi.reshape(sh))
    return out


# FFT backend: None runs numpy.fft (one thread); an integer n runs scipy.fft with n worker threads.
# Both compute the same DFT; the switch exists so that the CPU baseline can also be timed on all
# host cores. Every test runs with the default.
_WORKERS = None


def set_fft_workers(n):
    """Select the FFT backend (None: numpy.fft, single-threaded; n >= 1: scipy.fft, n threads)."""
    global _WORKERS
    _WORKERS = None if n is None else int(n)


def fft(u):
    if _WORKERS:
        import scipy.fft
        return scipy.fft.fftn(u, axes=(-3, -2, -1), workers=_WORKERS)
    return np.fft.fftn(u, axes=(-3, -2, -1))


def ifft_real(U):
    if _WORKERS:
        import scipy.fft
        return scipy.fft.ifftn(U, axes=(-3, -2, -1), workers=_WORKERS).real
    return np.fft.ifftn(U, axes=(-3, -2, -1)).real


def grad(u, dim):
    """Spectral gradient F^-1[i xi~ F[u]] of a scalar field: shape (dim, *grid)."""
    xi = xi_tilde(u.shape)
    U = fft(u)
    return np.stack([ifft_real(1j * xi[a] * U) for a in range(dim)])


def div(q, dim):
    """Spectral divergence F^-1[sum_a i xi~_a F[q_a]] of a vector field q (dim, *grid)."""
    xi = xi_tilde(q.shape[1:])
    acc = 0.0
    for a in range(dim):
        acc = acc + 1j * xi[a] * fft(q[a])
    return ifft_real(acc)


def galerkin_G(T, dim):
    """Apply the Fourier-Galerkin operator of Eq. (GFourier) to a tensor field T (d, d, *grid).

    G^_ijkl = delta_ik xi_j xi_l / (xi . xi) for xi != 0 and G^ = 0 at xi = 0, i.e.
    (G^ : T^)_ij = (T^ xi)_i xi_j / |xi|^2. Frequencies with xi~ = 0 (the mean and pure-Nyquist
    modes) are mapped to zero.
    """
    xi = xi_tilde(T.shape[2:])
    xi = xi[:dim]
    That = fft(T)
    xi2 = sum(x * x for x in xi)
    inv = np.where(xi2 > 0, 1.0 / np.where(xi2 > 0, xi2, 1.0), 0.0)
    Txi = [sum(That[i, l] * xi[l] for l in range(dim)) for i in range(dim)]
    out = np.empty_like(That)
    for i in range(dim):
        for j in range(dim):
            out[i, j] = Txi[i] * xi[j] * inv
    return ifft_real(out)


def sym_grad_vec(u, dim):
    """Displacement gradient F^-1[i xi~_j F[u_i]] of a vector field u (dim, *grid): (d, d, *grid)."""
    xi = xi_tilde(u.shape[1:])
    out = np.empty((dim, dim) + u.shape[1:])
    for i in range(dim):
        Ui = fft(u[i])
        for j in range(dim):
            out[i, j] = ifft_real(1j * xi[j] * Ui)
    return out
