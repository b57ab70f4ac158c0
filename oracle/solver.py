"""Staggered FFT phase-field-fracture solve under dissipation control (oracle; FP64, test only).

What one increment n computes (Sec. 2.1 Eq. (SystemDisany), Sec. 4.1):
  find the strain fluctuation eps~, the damage phi and the load factor E with
    (a) equilibrium   G^ : F[ g(phi) C^r : (eps~ + f E) ] = 0                       (R1 = 0)
    (b) damage        g'(phi) H + gamma_f'(phi) = 0, H = max(psi_o + psi_ini, H^{n-1})  (R2 = 0)
    (c) control       D(phi) = int Gc gamma_f = tau^n                                  (R3 = 0)
  with gamma_f' of Eq. (gamFunct), D of Eq. (CrackLenght_ani), H of Eq. (HistoryNumIni).

The paper solves (a)-(c) monolithically by Newton-Raphson + BiCGSTAB. This oracle (like the CUDA
library) uses the staggered fixed point of the same equations, which has the same solution:
  repeat
    1. at fixed phi solve (a) at unit load E = 1 for eps1 = f + sym(F~1) (Fourier-Galerkin CG on
       the displacement-gradient fluctuation F~1, Sec. 4.1 / Eq. (GFourier));
       the problem is positively homogeneous of degree 1 in E, so eps(E) = E eps1 and
       psi_o(eps(E)) = E^2 psi1 (also with the spectral split, for E >= 0);
    2. find E >= 0 with D(phi(E)) = tau^n, where phi(E) solves (b) with
       H_E = max(E^2 psi1 + psi_ini, H^{n-1}): (Gc/l + 2 H_E) phi - div(Gc l A grad phi) = 2 H_E;
    3. phi <- phi(E)
  until max(|d eps|/|eps|, |d phi|/|phi|, |D - tau|/tau) < tol   (the three quantities of
  Eq. (errors_crack)).

Toughness (Sec. 4.2, Eqs. (JaviGc), (ABC)): G = V / A_g (T^F - 1/2 Sigma^F E^F) with the
trapezoid sum T^n = sum 1/2 (Sigma^j + Sigma^{j-1})(E^j - E^{j-1}), Sigma = <sigma> : f, and F the
first increment with Sigma^F <= rho max_j Sigma^j (rho = 0.01: the coalescence point of Sec. 4.2 is
not formalised in the paper; this is the reading used).

Crack-tip enrichment (Sec. 4.3): phi_o - l^2 div(A grad phi_o) = phi_disc (Eqs. (damini),
(daminiAni); the printed "l nabla^2" is read as l^2 for dimensional consistency),
phi_ini = phi_M phi_o / max phi_o, psi_ini = -gamma_f'(phi_ini) / g'(phi_ini) clipped at 0
(Eq. (Enini), read without the stray factors), H^0 = psi_ini, tau^0 = D(phi_ini).
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

from . import material as mat
from . import spectral as sp


@dataclass
class Params:
    ell: float
    k_res: float = 1e-6
    split: int = 0
    history: bool = True
    f6: tuple = (0.0, 1.0, 0.0, 0.0, 0.0, 0.0)
    tol_mech: float = 1e-12
    tol_dmg: float = 1e-12
    tol_root: float = 1e-13
    tol_stag: float = 1e-10
    max_mech: int = 20000
    max_dmg: int = 20000
    max_root: int = 200
    max_stag: int = 300
    fracture_ratio: float = 0.01


class Model:
    """Static per-RVE data: per-voxel stiffness, toughness, cleavage tensor, crack geometry."""

    def __init__(self, micro, params):
        self.micro, self.p = micro, params
        d = micro.dim
        self.d = d
        nx, ny, nz = micro.n
        self.grid = (nz, ny, nx)
        self.V = float(nx * ny * nz)
        gid = micro.grain_id
        crack = micro.crack
        self.crack_mask = crack.mask(micro.n)
        mult = np.where(self.crack_mask, crack.stiffness, 1.0)
        Cg = np.stack([mat.rotate_stiffness(mat.cubic_tensor(*micro.C_cubic[g]), micro.R[g])[:d, :d, :d, :d]
                       for g in range(micro.n_grains)])
        self.C = Cg[gid] * mult[..., None, None, None, None]          # (*grid, d, d, d, d)
        self.Gc = micro.Gc[gid].astype(np.float64)
        Ag = np.stack([mat.cleavage_tensor(micro.R[g], micro.cleave_n[g], micro.beta[g], d)
                       for g in range(micro.n_grains)])
        self.A = np.moveaxis(Ag[gid], (-2, -1), (0, 1))               # (d, d, *grid)
        self.isotropic_damage = bool(np.all(micro.beta == 0.0))
        if params.split:
            c11, c12, c44 = micro.C_cubic.T
            if not np.allclose(c44, 0.5 * (c11 - c12), rtol=1e-12, atol=0):
                raise ValueError("the spectral split is defined for isotropic phases only")
            self.lam = c12[gid] * mult
            self.mu = c44[gid] * mult
        self.f = mat.tensor_from_voigt6(params.f6, d)
        self.fB = self.f.reshape(d, d, 1, 1, 1) * np.ones((1, 1) + self.grid)

    # ---- constitutive ----
    def contract(self, T):
        return np.einsum("zyxijkl,klzyx->ijzyx", self.C, T)

    def stress(self, eps, phi):
        g = mat.degradation(phi, self.p.k_res)
        if self.p.split:
            _, _, sp_, sm_ = mat.split_parts(eps, self.lam, self.mu)
            return g * sp_ + sm_
        return g * self.contract(eps)

    def drive(self, eps):
        """Crack driving energy density: psi_o = 1/2 eps:C:eps, or psi+ with the split."""
        if self.p.split:
            return mat.split_parts(eps, self.lam, self.mu)[0]
        return 0.5 * np.einsum("ijzyx,ijzyx->zyx", eps, self.contract(eps))

    def elastic_energy(self, eps, phi):
        g = mat.degradation(phi, self.p.k_res)
        if self.p.split:
            pp, pm, _, _ = mat.split_parts(eps, self.lam, self.mu)
            return float(np.sum(g * pp + pm))
        return float(np.sum(g * self.drive(eps)))

    # ---- fracture functional ----
    def gamma_density(self, phi):
        gr = sp.grad(phi, self.d)
        Agr = np.einsum("ijzyx,jzyx->izyx", self.A, gr)
        return phi * phi / (2.0 * self.p.ell) + 0.5 * self.p.ell * np.einsum("izyx,izyx->zyx", gr, Agr)

    def dissipation(self, phi):
        """D(phi) of Eq. (CrackLenght_ani), h = 1."""
        return float(np.sum(self.Gc * self.gamma_density(phi)))

    def crack_surface(self, phi):
        """Gamma(phi) of Eq. (CrackLenghtreal) (with A in the anisotropic case)."""
        return float(np.sum(self.gamma_density(phi)))

    def gamma_prime(self, phi):
        """gamma_f'(phi) = Gc/l phi - div(Gc l A grad phi), Eq. (gamFunct)."""
        gr = sp.grad(phi, self.d)
        q = self.Gc * self.p.ell * np.einsum("ijzyx,jzyx->izyx", self.A, gr)
        return self.Gc / self.p.ell * phi - sp.div(q, self.d)


def dot(a, b):
    return float(np.sum(a * b))


def norm(a):
    return math.sqrt(dot(a, a))


def cg(apply, b, x0, tol, scale, maxit, precond=None):
    """Plain (preconditioned) conjugate gradients; stops when |r| <= tol * scale."""
    x = x0.copy()
    r = b - apply(x)
    z = precond(r) if precond else r
    p = z.copy()
    rz = dot(r, z)
    it = 0
    while norm(r) > tol * scale:
        if it >= maxit:
            raise RuntimeError(f"CG did not converge: |r|/scale = {norm(r) / scale:.3e}")
        q = apply(p)
        alpha = rz / dot(p, q)
        x += alpha * p
        r -= alpha * q
        z = precond(r) if precond else r
        rz_new = dot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    return x, it


# ---- mechanics -----------------------------------------------------------------------------------

def mech_solve(model, phi, F0):
    """Unit-load equilibrium at fixed phi: returns the gradient fluctuation F~1 and CG iterations.

    Without split: CG on G^[C_phi : F~] = -G^[C_phi : f] (C_phi = g(phi) C^r), over
    compatible fields, Frobenius inner product. With the split: Newton on G^[sigma(f + sym F~)] = 0
    with the exact tangent, each step solved by CG.
    """
    d, p = model.d, model.p
    g = mat.degradation(phi, p.k_res)
    G = lambda T: sp.galerkin_G(T, d)
    if not p.split:
        Cphi = lambda T: g * model.contract(0.5 * (T + np.swapaxes(T, 0, 1)))
        sig_f = Cphi(model.fB)
        b = -G(sig_f)
        return cg(lambda T: G(Cphi(T)), b, F0, p.tol_mech, norm(sig_f), p.max_mech)
    x = F0.copy()
    total = 0
    for _ in range(100):
        eps = model.fB + 0.5 * (x + np.swapaxes(x, 0, 1))
        sig = model.stress(eps, phi)
        R = G(sig)
        nR, ns = norm(R), norm(sig)
        if nR <= p.tol_mech * ns:
            return x, total
        K = lambda T: G(mat.split_tangent_apply(eps, T, model.lam, model.mu, g))
        dx, it = cg(K, -R, np.zeros_like(x), 1e-3, nR, p.max_mech)
        total += it
        x = x + dx
    raise RuntimeError("Newton (split) did not converge")


# ---- damage ---------------------------------------------------------------------------------------

def damage_operator(model, H):
    d, l = model.d, model.p.ell
    a = model.Gc / l + 2.0 * H
    K = model.Gc * l * model.A                      # (d, d, *grid)

    def L(v):
        gr = sp.grad(v, d)
        return a * v - sp.div(np.einsum("ijzyx,jzyx->izyx", K, gr), d)

    xi = sp.xi_tilde(model.grid)
    xi2 = sum(x * x for x in xi[:d])
    abar = float(a.mean())
    bbar = float((model.Gc * l * np.trace(model.A)).mean() / d)
    denom = abar + bbar * xi2
    M = lambda r: sp.ifft_real(sp.fft(r) / denom)
    return L, M


def damage_solve(model, H, phi0):
    """Solve (Gc/l + 2H) phi - div(Gc l A grad phi) = 2H by FFT-preconditioned CG."""
    L, M = damage_operator(model, H)
    rhs = 2.0 * H
    s = norm(rhs)
    if s == 0.0:
        return np.zeros_like(H), 0
    return cg(L, rhs, phi0, model.p.tol_dmg, s, model.p.max_dmg, precond=M)


# ---- crack-tip enrichment -----------------------------------------------------------------------

def initial_crack(model):
    """Return phi_ini, psi_ini (Sec. 4.3)."""
    micro, d, l = model.micro, model.d, model.p.ell
    crack = micro.crack
    phi_disc = np.zeros(model.grid)
    if crack.kind == 0:
        return phi_disc.copy(), phi_disc.copy()
    nx = micro.n[0]
    if crack.kind == 1:                                   # CTE: the two tip voxels (lines in 3D)
        for x in (crack.x0 % nx, (crack.x0 + crack.length - 1) % nx):
            phi_disc[:, crack.row, x] = 1.0
    else:                                                 # CPFE: every crack voxel
        phi_disc[model.crack_mask] = 1.0
    xi = sp.xi_tilde(model.grid)
    xi2 = sum(x * x for x in xi[:d])
    if model.isotropic_damage:
        phi_o = sp.ifft_real(sp.fft(phi_disc) / (1.0 + l * l * xi2))
    else:
        Kl = l * l * model.A

        def Lc(v):
            return v - sp.div(np.einsum("ijzyx,jzyx->izyx", Kl, sp.grad(v, d)), d)
        bb = float((l * l * np.trace(model.A)).mean() / d)
        Mc = lambda r: sp.ifft_real(sp.fft(r) / (1.0 + bb * xi2))
        phi_o, _ = cg(Lc, phi_disc, np.zeros_like(phi_disc), 1e-14, norm(phi_disc), 20000, precond=Mc)
    phi_ini = crack.phi_M * phi_o / phi_o.max()
    gp = model.gamma_prime(phi_ini)
    psi_ini = np.maximum(0.0, -gp / mat.degradation_prime(phi_ini))
    return phi_ini, psi_ini


# ---- dissipation control ---------------------------------------------------------------------------

@dataclass
class State:
    phi: np.ndarray
    H: np.ndarray
    psi_ini: np.ndarray
    F1: np.ndarray                 # unit-load displacement-gradient fluctuation (warm start)
    eps: np.ndarray                # total strain at the committed load
    E: float = 0.0
    tau: float = 0.0
    T: float = 0.0
    Sigma: float = 0.0
    Sigma_max: float = 0.0
    n: int = 0
    fractured: bool = False
    tau0: float = 0.0              # D(phi^0), the functional of the initial crack
    Gamma0: float = 0.0            # Gamma(phi^0), its crack surface
    curve: list = field(default_factory=list)

    def copy(self):
        return dataclasses.replace(self, phi=self.phi.copy(), H=self.H.copy(), psi_ini=self.psi_ini.copy(),
                                   F1=self.F1.copy(), eps=self.eps.copy(), curve=list(self.curve))


def init_state(model):
    phi_ini, psi_ini = initial_crack(model)
    d = model.d
    z = np.zeros((d, d) + model.grid)
    st = State(phi=phi_ini, H=psi_ini.copy(), psi_ini=psi_ini, F1=z.copy(), eps=z.copy())
    st.tau = model.dissipation(phi_ini)
    st.tau0 = st.tau
    st.Gamma0 = model.crack_surface(phi_ini)
    return st


def history_field(model, E, psi1, psi_ini, H_prev):
    drive = E * E * psi1 + psi_ini
    return np.maximum(drive, H_prev) if model.p.history else drive


def arc_length(model, psi1, psi_ini, H_prev, tau, phi_warm, E_guess, stats):
    """Smallest E >= 0 with D(phi(E)) = tau (the control equation R3 = 0).

    D(phi(E)) is non-decreasing in E and D(phi(0)) = tau^{n-1} < tau, so the root is bracketed
    by stepping away from the previous load factor (steps growing x4), then refined by Illinois
    regula falsi until |D - tau| <= tol_root * tau.
    """
    p = model.p
    cache = {"phi": phi_warm}

    def evaluate(E):
        H = history_field(model, E, psi1, psi_ini, H_prev)
        phi, it = damage_solve(model, H, cache["phi"])
        stats["dmg_iters"] += it
        stats["root_evals"] += 1
        cache["phi"] = phi
        return model.dissipation(phi) - tau, phi, H

    if E_guess <= 0.0:
        E_guess = math.sqrt(float(np.mean(model.Gc)) / (p.ell * max(float(psi1.mean()), 1e-300))) * 0.05
    E0 = E_guess
    f0, phi, H = evaluate(E0)
    if abs(f0) <= p.tol_root * tau:
        return E0, phi, H, f0 + tau
    h = 1e-3 * E0
    if f0 < 0.0:
        lo, flo = E0, f0
        hi = lo + h
        fhi, phi, H = evaluate(hi)
        while fhi <= 0.0:
            lo, flo, h = hi, fhi, 4.0 * h
            hi = lo + h
            fhi, phi, H = evaluate(hi)
    else:
        hi, fhi = E0, f0
        lo = max(0.0, hi - h)
        flo, phi, H = evaluate(lo)
        while flo >= 0.0:
            if lo == 0.0:
                return 0.0, phi, H, flo + tau
            hi, fhi, h = lo, flo, 4.0 * h
            lo = max(0.0, hi - h)
            flo, phi, H = evaluate(lo)
    side = 0
    for _ in range(p.max_root):
        E = (lo * fhi - hi * flo) / (fhi - flo)
        fE, phi, H = evaluate(E)
        if abs(fE) <= p.tol_root * tau or (hi - lo) <= 1e-15 * hi:
            return E, phi, H, fE + tau
        if fE > 0.0:
            hi, fhi = E, fE
            if side == 1:
                flo *= 0.5
            side = 1
        else:
            lo, flo = E, fE
            if side == -1:
                fhi *= 0.5
            side = -1
    raise RuntimeError("arc-length root did not converge")


def macro_stress(model, sig):
    """Sigma = <sigma> : f."""
    return float(np.einsum("ij,ij->", sig.mean(axis=(2, 3, 4)), model.f))


def anderson_mix(X, Gv, rcond=1e-10):
    """Anderson acceleration (type II) of the staggered fixed point phi -> Phi(phi).

    X, Gv: the last m+1 inputs phi_j and outputs Phi(phi_j), residuals r_j = Phi_j - phi_j,
    dF_i = r_{i+1} - r_i, dG_i = Phi_{i+1} - Phi_i. The mixing weights minimise
    |r_k - dF gamma|: gamma = pinv(dF^T dF) dF^T r_k (pseudo-inverse of the small Gram matrix with
    relative cutoff ``rcond`` on its eigenvalues, numpy.linalg.lstsq). Returns Phi_k - dG gamma.
    """
    R = [g - x for x, g in zip(X, Gv)]
    if len(R) < 2:
        return Gv[-1].copy()
    dF = np.stack([(R[i + 1] - R[i]).ravel() for i in range(len(R) - 1)], 1)
    dG = np.stack([(Gv[i + 1] - Gv[i]).ravel() for i in range(len(R) - 1)], 1)
    M = dF.T @ dF
    gam = np.linalg.lstsq(M, dF.T @ R[-1].ravel(), rcond=rcond)[0]
    return (Gv[-1].ravel() - dG @ gam).reshape(Gv[-1].shape)


def energy_norm(model, eps, phi):
    """|eps|_{gC} = sqrt(sum eps : g(phi) C : eps): the norm of the staggered strain test (Eq.
    (errors_crack) does not fix the norm; weighting by the degraded stiffness keeps the fully
    cracked voxels, whose strain is ill-determined at k << 1, from dominating it)."""
    g = mat.degradation(phi, model.p.k_res)
    return math.sqrt(max(float(np.sum(g * np.einsum("ijzyx,ijzyx->zyx", eps, model.contract(eps)))), 0.0))


def increment(model, st, dtau, anderson_m=5, accept_unconverged=False):
    """One dissipation increment from the committed state ``st``; returns (new state, stats).

    The staggered map phi -> Phi(phi) (mechanics at phi, then the control root) is iterated to
    its fixed point with Anderson acceleration (memory ``anderson_m``; 0 = plain iteration), the
    acceleration of staggered PFF schemes of Storvik et al. cited in Sec. 4.1. The fixed point,
    hence the committed state, does not depend on the acceleration.
    """
    p = model.p
    tau = st.tau + dtau
    phi = st.phi.copy()
    F1 = st.F1.copy()
    eps_prev = st.eps
    E = st.E
    stats = {"mech_iters": 0, "dmg_iters": 0, "root_evals": 0, "stag_iters": 0}
    X, Gv = [], []
    best, k_best = math.inf, 0
    stats["stagnated"] = False
    for k in range(p.max_stag):
        F1, it = mech_solve(model, phi, F1)
        stats["mech_iters"] += it
        eps1 = model.fB + 0.5 * (F1 + np.swapaxes(F1, 0, 1))
        psi1 = model.drive(eps1)
        E, phi_new, H, D = arc_length(model, psi1, st.psi_ini, st.H, tau, phi, E, stats)
        eps = E * eps1
        err = max(energy_norm(model, eps - eps_prev, phi) / max(energy_norm(model, eps, phi), 1e-300),
                  norm(phi_new - phi) / max(norm(phi_new), 1e-300),
                  abs(D - tau) / tau)
        eps_prev = eps
        stats["stag_iters"] = k + 1
        if err < p.tol_stag:
            phi = phi_new
            break
        # noise floor: accept when the error has not improved for 20 iterations and is within
        # 1000 x tol (the conditioning of cracked voxels, k << 1, bounds how far the staggered
        # error can fall in floating point)
        if err < best:
            best, k_best = err, k
        if k - k_best >= 20 and err <= 1000.0 * p.tol_stag:
            phi = phi_new
            stats["stagnated"] = True
            break
        if anderson_m > 0:
            X.append(phi)
            Gv.append(phi_new)
            X, Gv = X[-(anderson_m + 1):], Gv[-(anderson_m + 1):]
            phi = anderson_mix(X, Gv)
        else:
            phi = phi_new
    else:
        if not accept_unconverged:
            raise RuntimeError("staggered iteration did not converge")
        phi = phi_new
        stats["unconverged"] = True
    new = st.copy()
    new.phi, new.H, new.F1, new.eps, new.E, new.tau = phi, H, F1, eps, E, tau
    sig = model.stress(eps, phi)
    Sigma = macro_stress(model, sig)
    new.T = st.T + 0.5 * (Sigma + st.Sigma) * (E - st.E)
    new.Sigma = Sigma
    new.Sigma_max = max(st.Sigma_max, Sigma)
    new.n = st.n + 1
    new.fractured = bool(new.Sigma_max > 0 and Sigma <= p.fracture_ratio * new.Sigma_max)
    rec = dict(n=new.n, E=E, Sigma=Sigma, D=model.dissipation(phi), Emec=model.elastic_energy(eps, phi),
               T=new.T, Gamma=model.crack_surface(phi), tau=tau, **stats)
    new.curve.append(rec)
    return new, stats


def crack_area(model):
    """A_g of Eq. (JaviGc0): the surface the fracture creates, without the pre-crack (h = 1)."""
    micro = model.micro
    nx, ny, nz = micro.n
    a0 = micro.crack.length if micro.crack.kind != 0 else 0
    return (nx - a0) * (nz if micro.dim == 3 else 1)


def toughness(model, st):
    """Eq. (JaviGc) with Eq. (ABC): G = V / A_g (T^F - 1/2 Sigma^F E^F)."""
    return model.V / crack_area(model) * (st.T - 0.5 * st.Sigma * st.E)


def toughness_functional(model, st):
    """Toughness from the dissipation functional instead of the load curve (Sec. 5.1, the
    comparison with the variational model): (D(phi^F) - D(phi^0)) / A_g, D of Eq.
    (CrackLenght_ani) and D(phi^0) = tau^0 the functional of the initial crack."""
    return (model.dissipation(st.phi) - st.tau0) / crack_area(model)


def instantaneous_toughness(model, Gamma0, curve):
    """Eq. (Gmed): G^n = V (T^n - T^{n-1}) / (Gamma^n - Gamma^{n-1}) for each committed increment,
    with T^0 = 0 and Gamma^0 the crack surface (Eq. (CrackLenghtreal)) of the initial crack."""
    out, T0, G0 = [], 0.0, Gamma0
    for rec in curve:
        dG = rec["Gamma"] - G0
        out.append(model.V * (rec["T"] - T0) / dG if dG != 0.0 else float("nan"))
        T0, G0 = rec["T"], rec["Gamma"]
    return out


def params_from_workload(w, **kw):
    return Params(ell=w.ell, k_res=w.k_res, split=w.split, f6=tuple(w.f), **kw)


def increment_with_cutback(model, st, dtau, depth=0):
    """One increment; if the staggered iteration does not converge, two increments of half the
    dissipation instead (recursively, up to four levels), each its own point of the load curve."""
    try:
        return increment(model, st, dtau)
    except RuntimeError as e:
        if "staggered" not in str(e):
            raise
        if depth >= 4:
            return increment(model, st, dtau, accept_unconverged=True)
    st1, s1 = increment_with_cutback(model, st, 0.5 * dtau, depth + 1)
    if st1.fractured:
        return st1, s1
    st2, s2 = increment_with_cutback(model, st1, 0.5 * dtau, depth + 1)
    return st2, {k: s1.get(k, 0) + s2.get(k, 0) for k in s2 if k != "stagnated"}


def run(w, n_inc=None, params=None, stop_at_fracture=True, callback=None):
    """Full toughness run of a synth.Workload: returns (model, final state, G or None)."""
    p = params or params_from_workload(w)
    model = Model(w.micro, p)
    st = init_state(model)
    for _ in range(n_inc or w.n_inc):
        st, _ = increment_with_cutback(model, st, w.dtau)
        if callback:
            callback(model, st)
        if st.fractured and stop_at_fracture:
            break
    G = toughness(model, st) if st.fractured else None
    return model, st, G
