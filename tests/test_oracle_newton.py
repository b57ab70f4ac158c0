"""Pins of the oracle's monolithic Newton-Raphson increment (Sec. 4.1).

N1  the Jacobian of Eq. (aniCrackLength_linearization) is the derivative of the residuals of Eq.
    (aniSystem_CrackLength): central differences in a random compatible direction, away from the
    history switch (where max(., H^n) has no derivative);
N2  BiCGSTAB solves a small non-symmetric system to numpy.linalg.solve's answer;
N3  a converged Newton increment equals the converged staggered increment from the same state
    (both solve the same three equations; the two algorithms share no solver code);
N4  the states the scheme cannot start from are refused.
"""
import numpy as np
import pytest

import synth
from oracle import newton as NR
from oracle import solver as S
from oracle import spectral as sp


def _state(name, n=1, **tol):
    w = synth.small_cases()[name]
    kw = dict(tol_mech=1e-13, tol_dmg=1e-13, tol_root=1e-13, tol_stag=1e-11)
    kw.update(tol)
    model = S.Model(w.micro, S.params_from_workload(w, **kw))
    st = S.init_state(model)
    for _ in range(n):
        st, _ = S.increment(model, st, w.dtau)
    return w, model, st


@pytest.mark.parametrize("name", ["homog32", "poly32"])
def test_jacobian_matches_finite_differences(name):
    w, model, st = _state(name)
    d = model.d
    tau = st.tau + w.dtau
    # a point off the history switch: more load and damage than the committed state
    F, phi, E = 1.05 * st.E * st.F1, 1.01 * st.phi, 1.05 * st.E
    rng = np.random.default_rng(0)
    u = rng.standard_normal((d,) + model.grid)
    dF = np.stack([sp.grad(u[i], d) for i in range(d)])        # compatible: grad of a displacement
    dphi = 1e-2 * rng.standard_normal(model.grid)
    dE = 0.3
    lin = NR.Linearisation(model, F, phi, E, st.H, st.psi_ini)
    assert lin.active.all()
    J = NR.jacobian_apply(model, lin, dF, dphi, dE)
    h = 1e-5
    lp = NR.Linearisation(model, F + h * dF, phi + h * dphi, E + h * dE, st.H, st.psi_ini)
    lm = NR.Linearisation(model, F - h * dF, phi - h * dphi, E - h * dE, st.H, st.psi_ini)
    Rp, Rm = NR.residual(model, lp, tau), NR.residual(model, lm, tau)
    for i in range(2):
        fd = (Rp[i] - Rm[i]) / (2 * h)
        assert np.linalg.norm(fd - J[i]) <= 1e-7 * np.linalg.norm(J[i]), i
    assert abs((Rp[2] - Rm[2]) / (2 * h) - J[2]) <= 1e-7 * abs(J[2])
    # a dropped coupling term would show: each off-diagonal block is far from zero
    J0 = NR.jacobian_apply(model, lin, 0 * dF, 0 * dphi, dE)
    assert np.linalg.norm(J0[0]) > 1e-3 * np.linalg.norm(J[0]) and np.linalg.norm(J0[1]) > 0


def test_bicgstab_solves_a_nonsymmetric_system():
    rng = np.random.default_rng(3)
    n1, n2 = 7, 5
    n = 2 * n1 + n2 + 1
    A = np.eye(n) * 4 + rng.standard_normal((n, n))
    pack = lambda v: np.concatenate([v[0].ravel(), v[1].ravel(), [v[2]]])
    unpack = lambda z: (z[:2 * n1].reshape(2, n1), z[2 * n1:2 * n1 + n2].copy(), float(z[-1]))
    b = unpack(rng.standard_normal(n))
    x, it = NR.bicgstab(lambda v: unpack(A @ pack(v)), b, lambda v: v, 1e-13, 500)
    assert np.allclose(pack(x), np.linalg.solve(A, pack(b)), rtol=0, atol=1e-11)


@pytest.mark.parametrize("name", ["homog32", "fibre64x16", "poly32"])
def test_newton_increment_equals_staggered_increment(name):
    w, model, st = _state(name)
    for _ in range(2):
        a, _ = S.increment(model, st, w.dtau)
        b, stats = NR.increment(model, st, w.dtau)
        assert stats["newton_iters"] <= 10
        for k in ("E", "Sigma", "D", "T", "Gamma", "Emec"):
            x, y = a.curve[-1][k], b.curve[-1][k]
            assert abs(x - y) <= 1e-9 * abs(x), (k, x, y)
        assert np.linalg.norm(a.phi - b.phi) <= 1e-9 * np.linalg.norm(a.phi)
        assert np.linalg.norm(a.H - b.H) <= 1e-9 * np.linalg.norm(a.H)
        st = a


def test_newton_refuses_states_it_cannot_start_from():
    w, model, st = _state("homog32", n=0)
    with pytest.raises(ValueError):
        NR.increment(model, st, w.dtau)                   # E = 0: no E coupling in J
    w = synth.small_cases()["homog32"]
    m = S.Model(w.micro, S.Params(ell=2.0, split=1))
    st = S.init_state(m)
    st.E = 0.1
    with pytest.raises(ValueError):
        NR.increment(m, st, w.dtau)                       # split: not linearised
