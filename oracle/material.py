"""Constitutive pieces of the PFF model (oracle; test infrastructure only).

* Cubic lattice stiffness and its rotation C^r_ijkl = R_im R_jn R_kp R_lq C_mnpq (Eq. (Crot), Sec. 2.2).
* Plane strain: the in-plane block C_ijkl, i,j,k,l in {x, y} (eps_zz = eps_xz = eps_yz = 0).
* Cleavage tensor A_f = I + beta (I - n_pl (x) n_pl) (Eq. (PFFani)), n_pl the weak-plane normal
  rotated to sample axes and, in 2D, projected on the RVE plane (not renormalised).
* Degradation g(phi) = (1 - phi)^2 + k and g'(phi) = -2 (1 - phi) (Sec. 2.1, Eq. (desgast)); the
  printed "- k" is read as the usual residual stiffness "+ k".
* Spectral tension/compression split (isotropic phases only; not part of the paper's model, which
  uses psi_o = 1/2 C : eps : eps): psi+- = lam/2 <tr eps>+-^2 + mu tr(eps+-^2) with
  eps+- = sum_a <e_a>+- n_a (x) n_a, and its tangent by the Daleckii-Krein divided-difference
  formula for spectral matrix functions.
"""
from __future__ import annotations

import numpy as np


def cubic_tensor(c1111, c1122, c1212):
    """Fourth-order cubic stiffness in lattice axes (tensor constants, shear not doubled)."""
    C = np.zeros((3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    if i == j == k == l:
                        C[i, j, k, l] = c1111
                    elif i == j and k == l:
                        C[i, j, k, l] = c1122
                    elif i != j and ((i == k and j == l) or (i == l and j == k)):
                        C[i, j, k, l] = c1212
    return C


def rotate_stiffness(C, R):
    """Eq. (Crot): C^r_ijkl = R_im R_jn R_kp R_lq C_mnpq."""
    return np.einsum("im,jn,kp,lq,mnpq->ijkl", R, R, R, R, C)


def cleavage_tensor(R, n_lattice, beta, dim):
    """Eq. (PFFani): A = I + beta (I - n_pl (x) n_pl), n_pl = (R n)[:dim] (projection in 2D)."""
    n = (R @ np.asarray(n_lattice, np.float64))[:dim]
    eye = np.eye(dim)
    return eye + beta * (eye - np.outer(n, n))


def degradation(phi, k):
    return (1.0 - phi) ** 2 + k


def degradation_prime(phi):
    return -2.0 * (1.0 - phi)


def tensor_from_voigt6(f6, dim):
    """(xx, yy, zz, yz, xz, xy) tensor components -> symmetric dim x dim matrix."""
    xx, yy, zz, yz, xz, xy = f6
    F = np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]], np.float64)
    return F[:dim, :dim]


# ---- spectral split ----------------------------------------------------------------------------

def _pos(x):
    return np.maximum(x, 0.0)


def _neg(x):
    return np.minimum(x, 0.0)


def _eig(eps):
    """eps (d, d, *grid) -> eigenvalues (*grid, d), eigenvectors (*grid, d, d) (columns)."""
    d = eps.shape[0]
    m = np.moveaxis(eps.reshape(d, d, -1), 2, 0)
    m = 0.5 * (m + np.swapaxes(m, 1, 2))
    w, v = np.linalg.eigh(m)
    return w, v


def split_parts(eps, lam, mu):
    """Return psi+, psi-, sigma+, sigma- for a strain field eps (d, d, *grid).

    lam, mu are per-voxel Lame fields (*grid). In plane strain the out-of-plane eigenvalue is 0
    and contributes to neither part, so the in-plane eigen-decomposition is exact.
    """
    d = eps.shape[0]
    grid = eps.shape[2:]
    w, v = _eig(eps)
    lamf, muf = lam.reshape(-1), mu.reshape(-1)
    tr = w.sum(-1)
    out = []
    for part in (_pos, _neg):
        ep = part(w)
        psi = 0.5 * lamf * part(tr) ** 2 + muf * (ep * ep).sum(-1)
        epsp = np.einsum("nia,na,nja->nij", v, ep, v)
        sig = 2.0 * muf[:, None, None] * epsp
        for i in range(d):
            sig[:, i, i] += lamf * part(tr)
        out.append((psi.reshape(grid), np.moveaxis(sig, 0, 2).reshape((d, d) + grid)))
    (psp, sgp), (psm, sgm) = out
    return psp, psm, sgp, sgm


def _divided_difference(fun, dfun, wa, wb):
    same = wa == wb
    den = np.where(same, 1.0, wa - wb)
    return np.where(same, dfun(wa), (fun(wa) - fun(wb)) / den)


def split_tangent_apply(eps, deps, lam, mu, g):
    """Directional derivative of sigma = g sigma+ + sigma- at eps in direction deps.

    d sigma+- = lam H(+-tr) tr(deps) I + 2 mu D[eps+-](deps), with the Daleckii-Krein formula
    D[F](deps) = sum_ab f^[1](e_a, e_b) (n_a . deps . n_b) n_a (x) n_b, f = <.>+- .
    """
    d = eps.shape[0]
    grid = eps.shape[2:]
    w, v = _eig(eps)
    dm = np.moveaxis(deps.reshape(d, d, -1), 2, 0)
    dm = 0.5 * (dm + np.swapaxes(dm, 1, 2))
    proj = np.einsum("nia,nij,njb->nab", v, dm, v)
    trd = np.einsum("nii->n", dm)
    tr = w.sum(-1)
    lamf, muf, gf = lam.reshape(-1), mu.reshape(-1), g.reshape(-1)
    heav_p = lambda x: (x > 0).astype(np.float64)
    heav_m = lambda x: (x < 0).astype(np.float64)
    total = np.zeros_like(dm)
    for fun, dfun, heav, weight in ((_pos, heav_p, heav_p, gf), (_neg, heav_m, heav_m, np.ones_like(gf))):
        dd = _divided_difference(fun, dfun, w[:, :, None], w[:, None, :])
        dF = np.einsum("nia,nab,njb->nij", v, dd * proj, v)
        part = 2.0 * muf[:, None, None] * dF
        for i in range(d):
            part[:, i, i] += lamf * heav(tr) * trd
        total += weight[:, None, None] * part
    return np.moveaxis(total, 0, 2).reshape((d, d) + grid)
