"""Monolithic Newton-Raphson increment with BiCGSTAB (oracle; FP64, test infrastructure only).

This is the paper's own solver of one increment (Sec. 4.1, Eqs. (schemeSys)-(relax)), written
from its equations. The unknowns are q = (F~, phi, E): the displacement-gradient fluctuation at
the actual load (eps = f E + sym F~), the damage and the load factor. The residuals are those of
Eq. (aniSystem_CrackLength):
    R1 = G^ * [ g(phi) C^r : eps ]                                   equilibrium (Eq. (GFourier))
    R2 = g'(phi) H + Gc/l phi - div(Gc l A grad phi)                 damage, Eq. (gamFunct)
    R3 = D(phi) - tau^n                                              control, Eq. (CrackLenght_ani)
with H = max(psi_o + psi_ini, H^n) (Eq. (HistoryNumIni); psi_o + psi_ini without history). The
Jacobian applied to dq = (dF, dphi, dE) is Eq. (aniCrackLength_linearization):
    J1 = G^ * [ g C^r : deps + g'(phi) sigma_o dphi ],   deps = sym dF + f dE   (Eq. (linSig))
    J2 = g'(phi) dH/deps : deps + (Gc/l + 2 H) dphi - div(Gc l A grad dphi)
    J3 = sum Gc/l phi dphi + Gc l grad(phi) . A grad(dphi)
with sigma_o = C^r : eps and dH/deps = sigma_o where the drive is on the loading branch,
psi_o + psi_ini >= H^n, else 0 (Eq. (Delta_history), whose printed condition psi_o > max(psi_o,
H^n) can never hold; ties count as loading, so at q_0 = q^n the voxels that set H^n stay coupled). Each Newton step solves J dq = -R by BiCGSTAB (the system is not symmetric),
right-preconditioned on the damage block by the FFT Helmholtz inverse (abar + bbar |xi~|^2)^-1
used by the staggered solver; q <- q + alpha dq with the under-relaxation of Eq. (relax), read
as alpha^n = max(theta, Sigma^{n-1} / max_j Sigma^j), theta = 0.3. The iteration stops on the
three ratios of Eq. (errors_crack) (strain change in the degraded energy norm, as in the
staggered oracle).

Only the model without the energy split is linearised here (the paper's Sec. 4.1 model).
The converged state solves the same three equations as the staggered fixed point of
``solver.increment``, so the two agree to the solver tolerances; ``tests/test_oracle_newton.py``
pins that, and the Jacobian against finite differences of the residual.
"""
from __future__ import annotations

import math

import numpy as np

from . import material as mat
from . import spectral as sp
from .solver import energy_norm, macro_stress


def _sym(T):
    return 0.5 * (T + np.swapaxes(T, 0, 1))


class Linearisation:
    """Fields of the residual and Jacobian at q = (F~, phi, E)."""

    def __init__(self, model, F, phi, E, H_prev, psi_ini):
        p = model.p
        self.model, self.phi, self.E = model, phi, E
        self.eps = model.fB * E + _sym(F)
        self.sig_o = model.contract(self.eps)                         # undamaged stress C^r : eps
        psi = 0.5 * np.einsum("ijzyx,ijzyx->zyx", self.eps, self.sig_o)
        drive = psi + psi_ini
        if p.history:
            self.H = np.maximum(drive, H_prev)
            self.active = (drive >= H_prev).astype(np.float64)
        else:
            self.H = drive
            self.active = np.ones_like(drive)
        self.g = mat.degradation(phi, p.k_res)
        self.gp = mat.degradation_prime(phi)
        self.K = model.Gc * p.ell * model.A                          # Gc l A, (d, d, *grid)

    def flux_div(self, v):
        d = self.model.d
        return sp.div(np.einsum("ijzyx,jzyx->izyx", self.K, sp.grad(v, d)), d)


def residual(model, lin, tau):
    d, p = model.d, model.p
    R1 = sp.galerkin_G(lin.g * lin.sig_o, d)
    R2 = lin.gp * lin.H + model.Gc / p.ell * lin.phi - lin.flux_div(lin.phi)
    R3 = model.dissipation(lin.phi) - tau
    return R1, R2, R3


def jacobian_apply(model, lin, dF, dphi, dE):
    d, p = model.d, model.p
    deps = _sym(dF) + model.fB * dE
    J1 = sp.galerkin_G(lin.g * model.contract(deps) + lin.gp * lin.sig_o * dphi, d)
    dH = lin.active * np.einsum("ijzyx,ijzyx->zyx", lin.sig_o, deps)
    J2 = lin.gp * dH + (model.Gc / p.ell + 2.0 * lin.H) * dphi - lin.flux_div(dphi)
    gr = sp.grad(lin.phi, d)
    Agr = np.einsum("ijzyx,jzyx->izyx", lin.K, sp.grad(dphi, d))
    J3 = float(np.sum(model.Gc / p.ell * lin.phi * dphi) + np.sum(gr * Agr))
    return J1, J2, J3


# ---- vectors q = (F, phi, E) ----------------------------------------------------------------------

def _vdot(a, b):
    return float(np.sum(a[0] * b[0]) + np.sum(a[1] * b[1]) + a[2] * b[2])


def _vaxpy(y, alpha, x):
    return (y[0] + alpha * x[0], y[1] + alpha * x[1], y[2] + alpha * x[2])


def _vnorm(a):
    return math.sqrt(max(_vdot(a, a), 0.0))


def bicgstab(apply, b, precond, tol, maxit):
    """Right-preconditioned BiCGSTAB (van der Vorst) from x = 0; stops when |r| <= tol |b|.

    The shadow residual is a fixed random vector, not b: at a converged state the right-hand side
    is almost only the control row (-R3 = dtau), and J has no E-E entry, so with rhat = b the
    first step divides by (b, J b) ~ 0."""
    zero = (np.zeros_like(b[0]), np.zeros_like(b[1]), 0.0)
    x, r = zero, b
    nb = _vnorm(b)
    if nb == 0.0:
        return x, 0
    rng = np.random.default_rng(0)
    rhat = (rng.standard_normal(b[0].shape), rng.standard_normal(b[1].shape), 1.0)
    rho = alpha = omega = 1.0
    v = p = zero
    for it in range(1, maxit + 1):
        rho_new = _vdot(rhat, r)
        if rho_new == 0.0:
            raise RuntimeError("BiCGSTAB breakdown (rho = 0)")
        beta = (rho_new / rho) * (alpha / omega)
        p = _vaxpy(r, beta, _vaxpy(p, -omega, v))
        phat = precond(p)
        v = apply(phat)
        alpha = rho_new / _vdot(rhat, v)
        s = _vaxpy(r, -alpha, v)
        if _vnorm(s) <= tol * nb:
            return _vaxpy(x, alpha, phat), it
        shat = precond(s)
        t = apply(shat)
        omega = _vdot(t, s) / _vdot(t, t)
        x = _vaxpy(_vaxpy(x, alpha, phat), omega, shat)
        r = _vaxpy(s, -omega, t)
        if _vnorm(r) <= tol * nb:
            return x, it
        rho = rho_new
    raise RuntimeError(f"BiCGSTAB did not converge: |r|/|b| = {_vnorm(r) / nb:.3e}")


def increment(model, st, dtau, theta=0.3, max_newton=50, max_lin=2000):
    """One dissipation increment by Newton-Raphson from the committed state ``st``.

    Returns (new state, stats) in the form of ``solver.increment``; raises RuntimeError when
    Newton does not converge within ``max_newton`` steps."""
    p = model.p
    if p.split:
        raise ValueError("the monolithic Newton scheme is linearised for the model without split")
    if not st.E > 0.0:
        # psi_o is quadratic in E, so at E = 0 the Jacobian has no coupling from E to the damage
        # and the control row cannot fix dE: start from a state with E > 0
        raise ValueError("Newton increment needs a committed state with E > 0")
    d = model.d
    tau = st.tau + dtau
    E = st.E
    F = E * st.F1
    phi = st.phi.copy()
    alpha = 1.0 if st.Sigma_max <= 0.0 else max(theta, st.Sigma / st.Sigma_max)
    xi = sp.xi_tilde(model.grid)
    xi2 = sum(x * x for x in xi[:d])
    stats = {"newton_iters": 0, "lin_iters": 0}
    err = math.inf
    for k in range(max_newton):
        lin = Linearisation(model, F, phi, E, st.H, st.psi_ini)
        R1, R2, R3 = residual(model, lin, tau)
        abar = float((model.Gc / p.ell + 2.0 * lin.H).mean())
        bbar = float((model.Gc * p.ell * np.trace(model.A)).mean() / d)
        denom = abar + bbar * xi2

        def precond(v):
            return (v[0], sp.ifft_real(sp.fft(v[1]) / denom), v[2])

        def apply(v):
            return jacobian_apply(model, lin, *v)

        # inexact Newton: the linear tolerance follows the last error (quadratic phase kept)
        tol_lin = max(1e-14, min(1e-4, 0.01 * err))
        dq, it = bicgstab(apply, (-R1, -R2, -R3), precond, tol_lin, max_lin)
        stats["lin_iters"] += it
        stats["newton_iters"] = k + 1
        dF, dphi, dE = dq
        F = F + alpha * dF
        phi = phi + alpha * dphi
        E = E + alpha * dE
        eps = model.fB * E + _sym(F)
        deps = alpha * (_sym(dF) + model.fB * dE)
        D = model.dissipation(phi)
        err = max(energy_norm(model, deps, phi) / max(energy_norm(model, eps, phi), 1e-300),
                  alpha * math.sqrt(float(np.sum(dphi * dphi))) / max(math.sqrt(float(np.sum(phi * phi))), 1e-300),
                  abs(D - tau) / tau)
        if err < p.tol_stag:
            break
    else:
        raise RuntimeError("Newton-Raphson did not converge (err %.3e)" % err)
    lin = Linearisation(model, F, phi, E, st.H, st.psi_ini)
    new = st.copy()
    new.phi, new.H, new.eps, new.E, new.tau = phi, lin.H, lin.eps, E, tau
    new.F1 = F / E if E > 0.0 else st.F1.copy()
    sig = model.stress(lin.eps, phi)
    Sigma = macro_stress(model, sig)
    new.T = st.T + 0.5 * (Sigma + st.Sigma) * (E - st.E)
    new.Sigma = Sigma
    new.Sigma_max = max(st.Sigma_max, Sigma)
    new.n = st.n + 1
    new.fractured = bool(new.Sigma_max > 0 and Sigma <= p.fracture_ratio * new.Sigma_max)
    rec = dict(n=new.n, E=E, Sigma=Sigma, D=model.dissipation(phi), Emec=model.elastic_energy(lin.eps, phi),
               T=new.T, Gamma=model.crack_surface(phi), tau=tau, **stats)
    new.curve.append(rec)
    return new, stats
