"""Independent evaluation of the residuals R1, R2, R3 (Sec. 4.1, Eq. (aniSystem_CrackLength)).

Written separately from ``solver``: real-to-complex FFTs (numpy.fft.rfftn), its own frequency
vectors and its own contractions. A converged state of the staggered solve must make all three
residuals vanish:

  R1 = F^-1{ G^ : F[ sigma(eps, phi) ] }                              (equilibrium, Eq. (GFourier))
  R2 = g'(phi) H + Gc/l phi - F^-1[ i xi . F[ Gc l A . F^-1[ i xi phi^ ] ] ]   (damage)
  R3 = int Gc [ phi^2 / (2 l) + l/2 A : (grad phi (x) grad phi) ] - tau^n       (control)

with H = max(psi_o(eps) + psi_ini, H^{n-1}) (Eq. (HistoryNumIni)).
"""
from __future__ import annotations

import numpy as np

from . import material as mat


def _freq(shape):
    """i xi~ factors on the rfftn half-grid of a (nz, ny, nx) field, x last (halved)."""
    nz, ny, nx = shape
    out = []
    for n, last in ((nx, True), (ny, False), (nz, False)):
        k = np.arange(n // 2 + 1) if last else np.fft.fftfreq(n) * n
        xi = 2.0 * np.pi * k / n
        if n % 2 == 0:
            xi = np.where(np.abs(np.abs(k) - n / 2) < 0.25, 0.0, xi)
        out.append(xi)
    kx, ky, kz = out
    return [kx[None, None, :], ky[None, :, None], kz[:, None, None]]


def _r(u):
    return np.fft.rfftn(u, axes=(-3, -2, -1))


def _ir(U, shape):
    return np.fft.irfftn(U, s=shape, axes=(-3, -2, -1))


def _gradient(phi, d):
    xi = _freq(phi.shape)
    P = _r(phi)
    return [_ir(1j * xi[a] * P, phi.shape) for a in range(d)]


def r1_equilibrium(sig, d):
    """F^-1[(sigma^ xi) (x) xi / |xi|^2] for a stress field sig (d, d, *grid)."""
    shape = sig.shape[2:]
    xi = _freq(shape)[:d]
    S = [[_r(sig[i, j]) for j in range(d)] for i in range(d)]
    xi2 = sum(x * x for x in xi)
    safe = np.where(xi2 > 0, xi2, 1.0)
    out = np.zeros_like(sig)
    for i in range(d):
        s_xi = sum(S[i][l] * xi[l] for l in range(d))
        for j in range(d):
            out[i, j] = _ir(np.where(xi2 > 0, s_xi * xi[j] / safe, 0.0), shape)
    return out


def r2_damage(phi, H, Gc, A, ell, d):
    grads = _gradient(phi, d)
    xi = _freq(phi.shape)
    flux_hat = 0.0
    for a in range(d):
        q_a = Gc * ell * sum(A[a, b] * grads[b] for b in range(d))
        flux_hat = flux_hat + 1j * xi[a] * _r(q_a)
    divq = _ir(flux_hat, phi.shape)
    return mat.degradation_prime(phi) * H + Gc / ell * phi - divq


def r3_control(phi, Gc, A, ell, tau, d):
    grads = _gradient(phi, d)
    quad = sum(A[a, b] * grads[a] * grads[b] for a in range(d) for b in range(d))
    return float(np.sum(Gc * (phi * phi / (2.0 * ell) + 0.5 * ell * quad))) - tau


def check_state(model, st, H_prev):
    """Relative residuals (|R1|/|sigma|, |R2|/|2H|, |R3|/tau) of a committed state."""
    d = model.d
    eps, phi = st.eps, st.phi
    sig = model.stress(eps, phi)
    drive = model.drive(eps)
    H = np.maximum(drive + st.psi_ini, H_prev) if model.p.history else drive + st.psi_ini
    r1 = r1_equilibrium(sig, d)
    r2 = r2_damage(phi, H, model.Gc, model.A, model.p.ell, d)
    r3 = r3_control(phi, model.Gc, model.A, model.p.ell, st.tau, d)
    n = lambda a: float(np.sqrt(np.sum(a * a)))
    return n(r1) / n(sig), n(r2) / n(2.0 * H), abs(r3) / st.tau
