"""Pins of the oracle's solver against results fixed independently of it.

P2  homogeneous RVE, no damage: zero fluctuation, sigma = g C : f uniform, no CG iteration.
P3  laminates with even layer widths (no Nyquist content): the exact 1D laminate solution
    (normal load: Reuss 1/<1/M>; parallel load: closed form of the uniform-sigma_xx problem).
P4  brute force: the unit-load equilibrium equals the minimiser of the elastic energy over
    displacements assembled with dense DFT derivative matrices (numpy.linalg.lstsq); the damage
    solve equals a dense direct solve of the same operator (numpy.linalg.solve).
P5  crack-tip enrichment is a fixed point: a damage solve with H = psi_ini returns phi_ini, and
    psi_ini vanishes away from the two tips (homogeneous Gc; A = I and A of Eq. (PFFani) with
    beta = 2). The anisotropic (Eq. (daminiAni)) and CPFE enrichments equal a dense direct solve.
P6  1D AT2 profile: with phi pinned to 1 at one voxel the damage solve approaches exp(-|x|/l)
    and Gamma -> 1 as l/h grows (Sec. 2.1, Eqs. (CrackLenght), (CrackLenghtreal)).
P7  uniform branch of a homogeneous uncracked RVE: phi = sqrt(2 l tau/(Gc V)),
    H = Gc phi/(2 l (1-phi)), E = sqrt(H/psi1), Sigma = g(phi) M E, T by trapezoid.
P8  without history the model is variational, so the external work V T^n equals the change of
    E_mec + D + int g psi_ini up to the quadrature error of the load curve (Sec. 5.1: the two
    toughness measures coincide without history); the gap vanishes as the increment shrinks.
R   converged increments make the independently coded residuals R1, R2, R3 vanish (also with the
    spectral split).
S   spectral split at system level: stress, drive and energy of a homogeneous cell against
    Miehe's closed form (tension, compression, mixed signs); the split equilibrium of a damaged
    laminate against its closed form in tension and in compression.
"""
import math

import numpy as np
import pytest

import synth
from oracle import material as mat
from oracle import residuals as res
from oracle import solver as S

RNG = np.random.default_rng(2)


# ---- dense brute-force helpers (explicit DFT matrices, no FFT) ----------------------------------

def _xi1d(n):
    k = np.arange(n)
    k = np.where(k > n // 2, k - n, k)
    xi = 2 * np.pi * k / n
    if n % 2 == 0:
        xi[n // 2] = 0.0
    return xi


def _deriv1d(n):
    j = np.arange(n)
    F = np.exp(-2j * np.pi * np.outer(j, j) / n)
    Finv = np.conj(F) / n
    return np.real(Finv @ np.diag(1j * _xi1d(n)) @ F)


def _deriv(shape, a):
    nz, ny, nx = shape
    mats = [np.eye(nz), np.eye(ny), np.eye(nx)]
    mats[2 - a] = _deriv1d(shape[2 - a])
    return np.kron(np.kron(mats[0], mats[1]), mats[2])


def _micro_random(n, dim, n_grains=3, seed=5):
    rng = np.random.default_rng(seed)
    m = synth.voronoi(n, n_grains, seed, C=(1.0, 0.6, 0.5), orientation="inplane" if dim == 2 else "so3",
                      beta=1.5, sigma_Gc=0.3)
    m.C_cubic[0] = synth.iso_constants(3.0, 0.25)
    return m


@pytest.mark.parametrize("n,dim", [((8, 4), 2), ((4, 4, 2), 3)])
def test_mech_solve_matches_dense_energy_minimiser(n, dim):
    m = _micro_random(n, dim)
    w = synth.Workload(m, ell=1.5)
    p = S.Params(ell=1.5, f6=(0.2, 1.0, -0.3, 0.1, 0.05, 0.4), tol_mech=1e-14)
    model = S.Model(m, p)
    phi = RNG.uniform(0.0, 0.8, model.grid)
    F1, _ = S.mech_solve(model, phi, np.zeros((dim, dim) + model.grid))
    eps_cg = model.fB + 0.5 * (F1 + np.swapaxes(F1, 0, 1))
    # dense: u (dim x N) -> eps = f + sym grad u; minimise sum 1/2 eps : C_phi : eps
    N = int(np.prod(model.grid))
    D = [_deriv(model.grid, a) for a in range(dim)]
    B = np.zeros((dim * dim * N, dim * N))
    for i in range(dim):
        for j in range(dim):
            row = (i * dim + j) * N
            B[row:row + N, j * N:(j + 1) * N] += 0.5 * D[i]
            B[row:row + N, i * N:(i + 1) * N] += 0.5 * D[j]
    g = mat.degradation(phi, p.k_res).reshape(-1)
    Cv = model.C.reshape(N, dim * dim, dim * dim) * g[:, None, None]
    Cbig = np.zeros((dim * dim * N, dim * dim * N))
    for a in range(dim * dim):
        for b in range(dim * dim):
            Cbig[a * N:(a + 1) * N, b * N:(b + 1) * N] = np.diag(Cv[:, a, b])
    fvec = np.repeat(model.f.reshape(-1), N)
    K = B.T @ Cbig @ B
    u = np.linalg.lstsq(K, -B.T @ Cbig @ fvec, rcond=1e-13)[0]
    eps_dense = (fvec + B @ u).reshape((dim, dim) + model.grid)
    np.testing.assert_allclose(eps_cg, eps_dense, atol=1e-10)


@pytest.mark.parametrize("n,dim", [((8, 8), 2), ((4, 4, 4), 3)])
def test_damage_solve_matches_dense_direct_solve(n, dim):
    m = _micro_random(n, dim)
    p = S.Params(ell=1.7, tol_dmg=1e-14)
    model = S.Model(m, p)
    H = RNG.uniform(0.0, 3.0, model.grid)
    phi, _ = S.damage_solve(model, H, np.zeros(model.grid))
    N = int(np.prod(model.grid))
    D = [_deriv(model.grid, a) for a in range(dim)]
    a = (model.Gc / p.ell + 2 * H).reshape(-1)
    L = np.diag(a)
    for i in range(dim):
        for j in range(dim):
            L += D[i].T @ np.diag((model.Gc * p.ell * model.A[i, j]).reshape(-1)) @ D[j]
    ref = np.linalg.solve(L, 2 * H.reshape(-1)).reshape(model.grid)
    np.testing.assert_allclose(phi, ref, atol=1e-12)
    # D(phi) by its definition with dense derivative matrices
    gr = [(Di @ ref.reshape(-1)).reshape(model.grid) for Di in D]
    quad = sum(model.A[i, j] * gr[i] * gr[j] for i in range(dim) for j in range(dim))
    Dref = np.sum(model.Gc * (ref ** 2 / (2 * p.ell) + 0.5 * p.ell * quad))
    assert abs(model.dissipation(phi) - Dref) < 1e-12 * Dref


def test_homogeneous_no_damage_uniform_stress():
    m = synth.homogeneous((16, 8), E=2.0, nu=0.25)
    p = S.Params(ell=2.0, f6=(0.3, 1.0, 0.0, 0.0, 0.0, 0.2))
    model = S.Model(m, p)
    for phi in (np.zeros(model.grid), np.full(model.grid, 0.37)):
        F1, it = S.mech_solve(model, phi, np.zeros((2, 2) + model.grid))
        assert it == 0 and np.abs(F1).max() == 0.0
        lam, mu = m.C_cubic[0, 1], m.C_cubic[0, 2]
        f = model.f
        sig_ref = mat.degradation(phi[0, 0, 0], p.k_res) * (lam * np.trace(f) * np.eye(2) + 2 * mu * f)
        sig = model.stress(model.fB, phi)
        np.testing.assert_allclose(sig, sig_ref.reshape(2, 2, 1, 1, 1) * np.ones_like(sig), rtol=1e-14)


def test_laminate_reuss_and_parallel_closed_forms():
    widths = [6, 10, 8, 8]
    phases = [(1.0, 0.3, 1.0), (5.0, 0.2, 1.0), (2.0, 0.35, 1.0), (0.5, 0.3, 1.0)]
    m = synth.laminate((32, 8), "x", widths, phases)
    C = np.array([synth.iso_constants(E, nu) for (E, nu, _) in phases])
    M_layer = np.repeat(C[:, 0], widths)
    lam_layer = np.repeat(C[:, 1], widths)
    # normal load (e_x (x) e_x): sigma_xx uniform = 1 / <1/M>  (Reuss)
    model = S.Model(m, S.Params(ell=2.0, f6=(1, 0, 0, 0, 0, 0), k_res=0.0))
    phi = np.zeros(model.grid)
    F1, _ = S.mech_solve(model, phi, np.zeros((2, 2) + model.grid))
    sig = model.stress(model.fB + 0.5 * (F1 + np.swapaxes(F1, 0, 1)), phi)
    reuss = 1.0 / np.mean(1.0 / M_layer)
    np.testing.assert_allclose(sig[0, 0], reuss, rtol=1e-12)
    np.testing.assert_allclose(sig[0, 1], 0.0, atol=1e-12)
    np.testing.assert_allclose(sig[1, 1][0, 0], lam_layer * reuss / M_layer, rtol=1e-12)
    # parallel load (e_y (x) e_y): sigma_xx = c uniform, eps_xx = (c - lam)/M with <eps_xx> = 0
    model = S.Model(m, S.Params(ell=2.0, f6=(0, 1, 0, 0, 0, 0), k_res=0.0))
    F1, _ = S.mech_solve(model, phi, np.zeros((2, 2) + model.grid))
    eps = model.fB + 0.5 * (F1 + np.swapaxes(F1, 0, 1))
    sig = model.stress(eps, phi)
    c = np.mean(lam_layer / M_layer) / np.mean(1.0 / M_layer)
    exx = (c - lam_layer) / M_layer
    np.testing.assert_allclose(eps[0, 0][0, 0], exx, atol=1e-12)
    np.testing.assert_allclose(sig[0, 0], c, rtol=1e-12)
    Syy = np.mean(lam_layer * exx + M_layer)
    assert abs(S.macro_stress(model, sig) - Syy) < 1e-12 * Syy


def test_cte_is_fixed_point_of_damage_solve():
    crack = synth.Crack(synth.CRACK_CTE, row=16, x0=4, length=10, phi_M=0.8)
    m = synth.homogeneous((32, 32), crack=crack)
    model = S.Model(m, S.Params(ell=2.0, tol_dmg=1e-14))
    st = S.init_state(model)
    assert abs(st.phi.max() - 0.8) < 1e-15
    phi, _ = S.damage_solve(model, st.psi_ini, np.zeros(model.grid))
    np.testing.assert_allclose(phi, st.phi, atol=1e-12)
    off = np.ones(model.grid, bool)
    off[0, 16, 4] = off[0, 16, 13] = False
    assert np.abs(st.psi_ini[off]).max() < 1e-12 * st.psi_ini.max()


def test_at2_profile_and_unit_crack_surface():
    """Continuum limit l/h -> infinity with n/l -> infinity (n = 8 l^2): the Nyquist-zeroed
    gradient leaves the checkerboard mode unpenalised, so a point pin carries a (-1)^x component
    of amplitude ~2 l/n that must vanish too."""
    errs, gammas = [], []
    for ell in (4.0, 8.0, 16.0, 32.0):
        n = int(8 * ell * ell)
        m = synth.homogeneous((n, 1))
        model = S.Model(m, S.Params(ell=ell, tol_dmg=1e-14))
        H = np.zeros(model.grid)
        H[0, 0, 0] = 1e12
        phi, _ = S.damage_solve(model, H, np.zeros(model.grid))
        x = np.arange(n)
        prof = np.exp(-np.minimum(x, n - x) / ell)
        errs.append(np.abs(phi[0, 0] - prof).max())
        gammas.append(abs(model.crack_surface(phi) - 1.0))
    assert all(a > b for a, b in zip(errs, errs[1:])) and errs[-1] < 0.015
    assert all(a > b for a, b in zip(gammas, gammas[1:])) and gammas[-1] < 0.002


def _uniform_case(history=True, k=1e-6):
    m = synth.homogeneous((8, 8), E=1.0, nu=0.3, Gc=1.0)
    return S.Model(m, S.Params(ell=2.0, k_res=k, history=history, tol_root=1e-14))


def test_uniform_branch_closed_form():
    model = _uniform_case()
    st = S.init_state(model)
    assert st.tau == 0.0
    V, Gc, ell, k = model.V, 1.0, 2.0, 1e-6
    M = synth.iso_constants(1.0, 0.3)[0]
    dtau = 0.05 * V
    T, Sig0, E0 = 0.0, 0.0, 0.0
    for n in range(1, 5):
        st, _ = S.increment(model, st, dtau)
        tau = n * dtau
        phi = math.sqrt(2 * ell * tau / (Gc * V))
        H = Gc * phi / (2 * ell * (1 - phi))
        E = math.sqrt(H / (0.5 * M))
        Sig = ((1 - phi) ** 2 + k) * M * E
        T += 0.5 * (Sig + Sig0) * (E - E0)
        Sig0, E0 = Sig, E
        assert abs(st.phi.mean() - phi) < 1e-12 and np.ptp(st.phi) < 1e-12
        assert abs(st.E - E) < 1e-11 * E
        assert abs(st.Sigma - Sig) < 1e-11 * Sig
        assert abs(st.T - T) < 1e-11 * T


def test_instantaneous_toughness_uniform_branch():
    """Eq. (Gmed) on the uniform branch, where every quantity is closed form: with phi uniform the
    crack surface is Gamma = V phi^2 / (2 l) (no gradient term), T follows the closed-form load
    curve of the test above, and G^n = V (T^n - T^{n-1}) / (Gamma^n - Gamma^{n-1})."""
    model = _uniform_case()
    st = S.init_state(model)
    assert st.Gamma0 == 0.0
    V, Gc, ell, k = model.V, 1.0, 2.0, 1e-6
    M = synth.iso_constants(1.0, 0.3)[0]
    dtau = 0.05 * V
    T, Sig0, E0, Gam0, ref = 0.0, 0.0, 0.0, 0.0, []
    for n in range(1, 5):
        st, _ = S.increment(model, st, dtau)
        phi = math.sqrt(2 * ell * n * dtau / (Gc * V))
        E = math.sqrt(Gc * phi / (ell * (1 - phi) * M))
        Sig = ((1 - phi) ** 2 + k) * M * E
        Tn = T + 0.5 * (Sig + Sig0) * (E - E0)
        Gam = V * phi * phi / (2 * ell)
        ref.append(V * (Tn - T) / (Gam - Gam0))
        T, Sig0, E0, Gam0 = Tn, Sig, E, Gam
    got = S.instantaneous_toughness(model, st.Gamma0, st.curve)
    assert np.allclose(got, ref, rtol=1e-10, atol=0), (got, ref)


def test_residual_energy_is_half_sigma_e():
    """E_res of Eq. (JaviGc) is read as 1/2 Sigma^F E^F (Eq. (ABC)): at an equilibrium state the
    stored energy is 1/2 V <sigma : eps> = 1/2 V E <sigma> : f, because the periodic fluctuation
    does no work against a divergence-free stress (Hill-Mandel). With it the load-curve toughness
    equals (V T - E_mec) / A_g."""
    w = synth.small_cases()["fibre64x16"]
    model = S.Model(w.micro, S.params_from_workload(w, tol_stag=1e-11))
    st = S.init_state(model)
    for _ in range(3):
        st, _ = S.increment(model, st, w.dtau)
        rec = st.curve[-1]
        assert abs(rec["Emec"] - 0.5 * model.V * st.Sigma * st.E) < 1e-8 * rec["Emec"]
    g_work = S.toughness(model, st)
    assert abs(g_work - (model.V * st.T - st.curve[-1]["Emec"]) / S.crack_area(model)) < 1e-8 * abs(g_work)


def test_work_and_functional_toughness_agree_without_history():
    """Sec. 5.1: for the model without history (variational up to the enrichment term) the
    load-curve measure and the functional measure of the toughness coincide; their gap is the
    trapezoid error of the curve plus the change of the enrichment energy int g(phi) psi_ini, and
    the first part shrinks when the increment does."""
    crack = synth.Crack(synth.CRACK_CTE, row=8, x0=0, length=4, phi_M=0.8)
    m = synth.homogeneous((16, 16), crack=crack)
    gaps = []
    for steps, dtau in ((6, 0.2), (12, 0.1), (24, 0.05)):
        model = S.Model(m, S.Params(ell=2.0, history=False, tol_stag=1e-11))
        st = S.init_state(model)
        k = model.p.k_res
        ini0 = float(np.sum(mat.degradation(st.phi, k) * st.psi_ini))
        for _ in range(steps):
            st, _ = S.increment(model, st, dtau)
        ini = float(np.sum(mat.degradation(st.phi, k) * st.psi_ini))
        A_g = S.crack_area(model)
        assert A_g == 12
        gaps.append(S.toughness(model, st) - S.toughness_functional(model, st) - (ini - ini0) / A_g)
    assert abs(gaps[0]) > 1.9 * abs(gaps[1]) > 3.6 * abs(gaps[2]), gaps
    assert abs(gaps[2]) < 0.03 * abs(S.toughness_functional(model, st))


def test_no_history_energy_balance_second_order():
    """Without history the damage equation g'(phi)(psi_o + psi_ini) + gamma_f' = 0 is the
    stationarity of Psi = E_mec + D + int g(phi) psi_ini, so the external work V T equals the
    change of Psi up to the trapezoid error."""
    crack = synth.Crack(synth.CRACK_CTE, row=8, x0=0, length=4, phi_M=0.8)
    m = synth.homogeneous((16, 16), crack=crack)
    gaps, works = [], []
    for steps, dtau in ((6, 0.2), (12, 0.1), (24, 0.05)):
        model = S.Model(m, S.Params(ell=2.0, history=False, tol_stag=1e-11))
        st = S.init_state(model)
        k = model.p.k_res
        psi0 = st.tau + float(np.sum(mat.degradation(st.phi, k) * st.psi_ini))
        for _ in range(steps):
            st, _ = S.increment(model, st, dtau)
        rec = st.curve[-1]
        psi = rec["Emec"] + rec["D"] + float(np.sum(mat.degradation(st.phi, k) * st.psi_ini))
        gaps.append(model.V * st.T - (psi - psi0))
        works.append(model.V * st.T)
    # the gap is the quadrature error of the load curve: it vanishes at least linearly
    assert gaps[0] / gaps[1] > 1.9 and gaps[1] / gaps[2] > 1.9, gaps
    assert abs(gaps[2]) < 0.005 * works[2]


def test_plate_one_voxel_thick_equals_plane_strain():
    """A 3D plate one voxel thick (the RVEs of Sec. 5) with grains rotated about z only and the
    load e_y (x) e_y is a plane-strain problem: xi_z = 0 leaves no zz fluctuation, cubic symmetry
    about z decouples the anti-plane shears, and the cleavage tensor acts on an in-plane gradient.
    So its increments equal those of the 2D model on the same grains, exactly up to rounding."""
    import dataclasses
    crack = synth.Crack(synth.CRACK_CTE, row=8, x0=0, length=4, phi_M=0.8)
    m3 = synth.polycrystal_plate((32, 16), 8, 17, zener=4.0, beta=2.0, orientation="inplane", crack=crack)
    m2 = dataclasses.replace(m3, n=(32, 16, 1), dim=2)
    out = []
    for m in (m3, m2):
        model = S.Model(m, S.Params(ell=2.0, tol_stag=1e-11))
        st = S.init_state(model)
        for _ in range(2):
            st, _ = S.increment(model, st, 0.4)
        out.append((st, model))
    (s3, m3_), (s2, _) = out
    assert m3_.d == 3 and m3_.grid == (1, 16, 32)
    for k in ("E", "Sigma", "D", "T", "Gamma", "Emec"):
        a, b = s3.curve[-1][k], s2.curve[-1][k]
        assert abs(a - b) <= 1e-9 * abs(b), (k, a, b)
    assert np.max(np.abs(s3.phi.reshape(-1) - s2.phi.reshape(-1))) < 1e-9
    # the anti-plane shears and the zz strain stay zero
    assert np.max(np.abs(s3.eps[2])) < 1e-12 and np.max(np.abs(s3.eps[:, 2])) < 1e-12


def test_laguerre_without_spread_is_voronoi():
    """The power-weighted tessellation with equal radii is the plain periodic Voronoi one."""
    from scipy.spatial import cKDTree
    gid, seeds, radii, _ = synth.laguerre_ids((48, 32), 12, 3, sigma_size=0.0)
    assert np.allclose(radii, radii[0])
    tree = cKDTree(seeds, boxsize=[48, 32])
    X, Y = np.meshgrid(np.arange(48) + 0.5, np.arange(32) + 0.5)
    _, ref = tree.query(np.stack([X.ravel(), Y.ravel()], -1))
    assert np.array_equal(gid.ravel(), ref)
    # with spread, larger radii claim larger grains on average
    gid, seeds, radii, _ = synth.laguerre_ids((256, 256), 60, 4, sigma_size=0.25)
    size = np.bincount(gid.ravel(), minlength=60)
    assert np.corrcoef(radii, size)[0, 1] > 0.5


def test_converged_increments_zero_residuals():
    w = synth.small_cases()["fibre64x16"]
    model = S.Model(w.micro, S.params_from_workload(w, tol_stag=1e-11))
    st = S.init_state(model)
    for _ in range(3):
        H_prev = st.H
        st, _ = S.increment(model, st, w.dtau)
        r1, r2, r3 = res.check_state(model, st, H_prev)
        assert r1 < 1e-10 and r2 < 1e-9 and r3 < 1e-11, (r1, r2, r3)


# ---- crack-tip enrichment with anisotropic damage, CPFE, and the split at system level -----------

def _dense_helmholtz(model, ell, phi_disc):
    """Dense direct solve of phi - l^2 div(A grad phi) = phi_disc with explicit DFT derivative
    matrices: the spectral divergence is -D^T, so the operator is I + l^2 sum_ij D_i^T A_ij D_j."""
    dim = model.d
    N = int(np.prod(model.grid))
    D = [_deriv(model.grid, a) for a in range(dim)]
    L = np.eye(N)
    for i in range(dim):
        for j in range(dim):
            L += ell * ell * D[i].T @ np.diag(model.A[i, j].reshape(-1)) @ D[j]
    return np.linalg.solve(L, phi_disc.reshape(-1)).reshape(model.grid), D


def _dense_gamma_prime(model, ell, phi, D):
    """gamma_f'(phi) = Gc/l phi + sum_ij D_i^T (Gc l A_ij) D_j phi (Eq. (gamFunct), dense)."""
    out = (model.Gc / ell * phi).reshape(-1)
    for i in range(model.d):
        for j in range(model.d):
            out = out + D[i].T @ ((model.Gc * ell * model.A[i, j]).reshape(-1) * (D[j] @ phi.reshape(-1)))
    return out.reshape(model.grid)


def _tip_source(micro):
    """phi_disc written from the crack's definition (Sec. 4.3): 1 at the first and last voxel of
    the crack row (every z), 0 elsewhere."""
    nx, ny, nz = micro.n
    c = micro.crack
    src = np.zeros((nz, ny, nx))
    src[:, c.row, c.x0 % nx] = 1.0
    src[:, c.row, (c.x0 + c.length - 1) % nx] = 1.0
    return src


@pytest.mark.parametrize("n,dim", [((16, 8), 2), ((8, 4, 4), 3)])
def test_anisotropic_cte_matches_dense_solve(n, dim):
    """Eq. (daminiAni) with the cleavage tensor of Eq. (PFFani), beta = 2 (the anisotropic branch
    of the enrichment solves it by PCG). Against a dense direct solve of the same operator:
    phi_ini = phi_M phi_o / max phi_o and psi_ini = max(0, gamma'/(2 (1 - phi_ini))) of Eq.
    (Enini). Catches l A in place of l^2 A, A^T or I in place of A, a wrong tip voxel, a dropped
    Gc in gamma'."""
    crack = synth.Crack(synth.CRACK_CTE, row=n[1] // 2, x0=2, length=6, phi_M=0.8)
    m = synth.voronoi(n, 4, 21, orientation="inplane" if dim == 2 else "so3", beta=2.0, sigma_Gc=0.3,
                      crack=crack)
    ell = 1.7
    model = S.Model(m, S.Params(ell=ell))
    assert not model.isotropic_damage
    phi_ini, psi_ini = S.initial_crack(model)
    phi_o, D = _dense_helmholtz(model, ell, _tip_source(m))
    ref = 0.8 * phi_o / phi_o.max()
    np.testing.assert_allclose(phi_ini, ref, rtol=0, atol=1e-12)
    gp = _dense_gamma_prime(model, ell, ref, D)
    np.testing.assert_allclose(psi_ini, np.maximum(0.0, gp / (2.0 * (1.0 - ref))), rtol=0,
                               atol=1e-11 * np.abs(psi_ini).max())


@pytest.mark.parametrize("n,dim", [((16, 16), 2), ((8, 8, 4), 3)])
def test_anisotropic_cte_is_fixed_point_of_damage_solve(n, dim):
    """With uniform Gc and beta != 0, gamma'(phi_ini) = Gc/l (phi_ini - l^2 div(A grad phi_ini))
    is a non-negative multiple of the tip source, so H = psi_ini makes phi_ini the solution of the
    damage equation at E = 0 (Eqs. (Enini), (HistoryNumIni)) exactly, and psi_ini vanishes off
    the tips."""
    crack = synth.Crack(synth.CRACK_CTE, row=n[1] // 2, x0=3, length=6, phi_M=0.8)
    m = synth.voronoi(n, 5, 23, orientation="inplane" if dim == 2 else "so3", beta=2.0, crack=crack)
    model = S.Model(m, S.Params(ell=2.0, tol_dmg=1e-14))
    assert not model.isotropic_damage
    st = S.init_state(model)
    phi, _ = S.damage_solve(model, st.psi_ini, np.zeros(model.grid))
    np.testing.assert_allclose(phi, st.phi, rtol=0, atol=1e-11)
    off = _tip_source(m) == 0.0
    assert np.abs(st.psi_ini[off]).max() < 1e-10 * st.psi_ini.max()


@pytest.mark.parametrize("beta", [0.0, 2.0])
def test_cpfe_initial_crack_matches_dense_solve(beta):
    """CPFE (Sec. 4.3): phi_disc = 1 on every voxel of the crack row, so the source is the crack
    mask itself (written here from the row and the span, not from the oracle's mask). Dense solve
    of Eq. (damini) / (daminiAni) as above; psi_ini of Eq. (Enini)."""
    crack = synth.Crack(synth.CRACK_CPFE, row=5, x0=13, length=6, phi_M=0.98)
    m = synth.voronoi((16, 10), 3, 29, beta=beta, crack=crack)
    ell = 1.5
    model = S.Model(m, S.Params(ell=ell))
    phi_ini, psi_ini = S.initial_crack(model)
    src = np.zeros(model.grid)
    for x in range(13, 19):
        src[0, 5, x % 16] = 1.0
    assert src.sum() == 6
    phi_o, D = _dense_helmholtz(model, ell, src)
    ref = 0.98 * phi_o / phi_o.max()
    np.testing.assert_allclose(phi_ini, ref, rtol=0, atol=1e-12)
    gp = _dense_gamma_prime(model, ell, ref, D)
    np.testing.assert_allclose(psi_ini, np.maximum(0.0, gp / (2.0 * (1.0 - ref))), rtol=0,
                               atol=1e-11 * np.abs(psi_ini).max())


def _miehe_closed_form(e, lam, mu, g):
    """Miehe's split for a diagonal plane-strain strain diag(a, b) (principal axes x, y, eps_zz = 0):
    psi+- = lam/2 <a + b>+-^2 + mu (<a>+-^2 + <b>+-^2), sigma = g sigma+ + sigma- with
    sigma+- = lam <tr>+- I + 2 mu diag(<a>+-, <b>+-)."""
    a, b = e
    pos, neg = (lambda v: max(v, 0.0)), (lambda v: min(v, 0.0))
    tr = a + b
    pp = 0.5 * lam * pos(tr) ** 2 + mu * (pos(a) ** 2 + pos(b) ** 2)
    pm = 0.5 * lam * neg(tr) ** 2 + mu * (neg(a) ** 2 + neg(b) ** 2)
    sp_ = np.diag([lam * pos(tr) + 2 * mu * pos(a), lam * pos(tr) + 2 * mu * pos(b)])
    sm_ = np.diag([lam * neg(tr) + 2 * mu * neg(a), lam * neg(tr) + 2 * mu * neg(b)])
    return pp, pm, g * sp_ + sm_


@pytest.mark.parametrize("f6", [(0, 1, 0, 0, 0, 0), (0, -1, 0, 0, 0, 0), (-0.5, 1, 0, 0, 0, 0),
                                (0.3, -1, 0, 0, 0, 0)])
def test_split_model_energies_and_stress_closed_form(f6):
    """Model.stress / drive / elastic_energy with the spectral split on a homogeneous RVE at a
    uniform damage: uniaxial tension, uniaxial compression and two mixed-sign strains against
    Miehe's closed form. Catches g (sigma+ + sigma-) in place of g sigma+ + sigma-, psi_o in
    place of psi+ as the drive, and a degraded psi-."""
    m = synth.homogeneous((8, 8), E=1.3, nu=0.27)
    model = S.Model(m, S.Params(ell=2.0, split=1, f6=f6))
    phi = np.full(model.grid, 0.41)
    g = (1 - 0.41) ** 2 + model.p.k_res
    _, lam, mu = synth.iso_constants(1.3, 0.27)
    E = 0.7
    eps = E * model.fB
    pp, pm, sig = _miehe_closed_form((E * f6[0], E * f6[1]), lam, mu, g)
    got = model.stress(eps, phi)
    np.testing.assert_allclose(got[:, :, 0, 0, 0], sig, rtol=1e-13, atol=1e-15)
    assert np.ptp(got) < 1e-14 or np.allclose(got, got[:, :, :1, :1, :1], rtol=1e-14, atol=0)
    np.testing.assert_allclose(model.drive(eps), pp, rtol=1e-13, atol=1e-16)
    assert abs(model.elastic_energy(eps, phi) - model.V * (g * pp + pm)) <= 1e-13 * model.V * (pp + pm)
    # the unit-load equilibrium of a homogeneous cell is the uniform strain (no fluctuation)
    F1, _ = S.mech_solve(model, phi, np.zeros((2, 2) + model.grid))
    assert np.abs(F1).max() < 1e-14


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_split_laminate_closed_form(sign):
    """Layers stacked along x with damage constant per layer, load f = sign e_x (x) e_x - 0.25 e_y (x) e_y.
    Compatibility leaves eps_yy = -0.25 and eps_xy = 0 uniform and eps_xx = a_k per layer with
    <a_k> = sign; equilibrium makes sigma_xx uniform. Tension (sign = +1, tr > 0 in every layer):
    g_k (lam_k (a_k - 1/4) + 2 mu_k a_k) = c. Compression (sign = -1, a_k < 0 and tr < 0): the
    degradation drops out, lam_k (a_k - 1/4) + 2 mu_k a_k = c. So the Newton solve of the split
    equilibrium has a closed form in both regimes."""
    widths = [6, 10, 8, 8]
    phases = [(1.0, 0.3, 1.0), (4.0, 0.2, 1.0), (2.0, 0.35, 1.0), (0.7, 0.25, 1.0)]
    m = synth.laminate((32, 8), "x", widths, phases)
    model = S.Model(m, S.Params(ell=2.0, split=1, f6=(sign, -0.25, 0, 0, 0, 0), tol_mech=1e-13))
    phi_layer = np.repeat([0.1, 0.5, 0.3, 0.7], widths)
    phi = np.broadcast_to(phi_layer, model.grid).copy()
    C = np.array([synth.iso_constants(E, nu) for (E, nu, _) in phases])
    lam = np.repeat(C[:, 1], widths)
    mu = np.repeat(C[:, 2], widths)
    g = (1 - phi_layer) ** 2 + model.p.k_res if sign > 0 else np.ones_like(phi_layer)
    M = lam + 2 * mu
    # a_k = (c / g_k + lam_k / 4) / M_k with mean(a) = sign
    c = (sign - np.mean(lam / (4 * M))) / np.mean(1.0 / (g * M))
    a = (c / g + lam / 4) / M
    tr = a - 0.25
    assert (np.all(tr > 0) and np.all(a > 0)) if sign > 0 else (np.all(tr < 0) and np.all(a < 0))
    F1, it = S.mech_solve(model, phi, np.zeros((2, 2) + model.grid))
    assert it > 0
    eps = model.fB + 0.5 * (F1 + np.swapaxes(F1, 0, 1))
    np.testing.assert_allclose(eps[0, 0][0, 0], a, rtol=0, atol=1e-11)
    np.testing.assert_allclose(eps[1, 1], -0.25, rtol=0, atol=1e-11)
    np.testing.assert_allclose(eps[0, 1], 0.0, atol=1e-11)
    sig = model.stress(eps, phi)
    np.testing.assert_allclose(sig[0, 0], c, rtol=1e-10)


def test_split_converged_increments_zero_residuals():
    """Increments of the cracked homogeneous cell with the spectral split: the independently coded
    residuals R1-R3 (with the split stress and psi+ as the history drive) vanish."""
    w = synth.replace(synth.small_cases()["homog32"], split=1)
    model = S.Model(w.micro, S.params_from_workload(w, tol_stag=1e-11))
    st = S.init_state(model)
    for _ in range(2):
        H_prev = st.H
        st, _ = S.increment(model, st, w.dtau)
        r1, r2, r3 = res.check_state(model, st, H_prev)
        assert r1 < 1e-10 and r2 < 1e-9 and r3 < 1e-11, (r1, r2, r3)
