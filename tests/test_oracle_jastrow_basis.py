"""Pins for the oracle's AO-expanded Jastrow terms (App., Eqs. onebody_J_inhom and threebody_jas):
U = sum_e sum_mu xi_mu psi^J_mu(r_e) + sum_{i<j} sum_{mu,nu} Xi_{mu nu} psi^J_mu(r_i) psi^J_nu(r_j),
read as terms of the Jastrow exponent, Xi symmetric.

Checked against: the closed form of one normalised s Gaussian, the matrix identity
U = xi.s + (s^T Xi s - sum_e phi_e^T Xi phi_e) / 2 (s = sum_e phi_e) evaluated with numpy, O(h^4)
finite differences in electron and nuclear coordinates, the translational sum rule, and a replay
of the Metropolis chain from the Philox generator and the oracle's own log|Psi|.
"""
import copy
import math

import numpy as np
import pytest

import oracle
from paper_2511_05222_gb300 import systems as S

NOJ = S.Jastrow(enable_J1=False, enable_J2=False)


def _rich(f, h):
    """Richardson-extrapolated central difference, O(h^4)."""
    return (4 * (f(h / 2) - f(-h / 2)) / h - (f(h) - f(-h)) / (2 * h)) / 3


@pytest.fixture(scope="module")
def water_jb():
    """Water with a seeded medium Jastrow basis and coefficients three times the defaults, so that
    the AO-expanded terms are a sizeable part of grad ln Psi and E_L."""
    sx = S.make_system(0)
    return S.with_jastrow_basis(sx, S.jastrow_basis(sx, 7, xi_scale=0.3, same_scale=0.09, pair_scale=0.03))


def _single_s(alpha, beta, xi):
    """One electron on a proton; determinant orbital exp(-alpha r^2); one s Jastrow function
    exp(-beta r^2) on the proton with coefficient xi."""
    sx = S.custom_system("H", [1], [[0.0, 0.0, 0.0]], [(0, 0, [alpha], [1.0])], 1, 0, [[1.0]], None,
                         copy.copy(NOJ))
    jb = S.JastrowBasis(np.array([0], np.int32), np.array([0], np.int32), np.array([1], np.int32),
                        np.array([[beta, 0.0, 0.0]]), np.array([[1.0, 0.0, 0.0]]), np.array([xi]), np.zeros((1, 1)))
    return S.with_jastrow_basis(sx, jb)


@pytest.mark.parametrize("alpha,beta,xi", [(0.4, 0.7, 0.35), (1.3, 0.2, -0.8)])
def test_one_s_function_closed_form(alpha, beta, xi):
    """J = xi N e^{-b r^2}, N = (2b/pi)^{3/4}: ln Psi, its gradient and Laplacian, and
    E_L = -1/2 (lap ln Psi + |grad ln Psi|^2) - 1/r with ln D = -a r^2 + const."""
    sx = _single_s(alpha, beta, xi)
    o = oracle.Oracle(sx)
    rng = np.random.default_rng(1)
    pos = rng.standard_normal((6, 1, 3)) * 0.9
    out = o.eval(pos, want=("logpsi", "grad_lnpsi", "lap_lnpsi", "EL", "parts"))
    r = pos[:, 0, :]
    r2 = (r ** 2).sum(-1)
    N = (2 * beta / math.pi) ** 0.75
    Jv = xi * N * np.exp(-beta * r2)
    gJ = (-2 * beta * Jv)[:, None] * r
    lJ = Jv * (4 * beta ** 2 * r2 - 6 * beta)
    np.testing.assert_allclose(out["parts"][:, 4], Jv, rtol=1e-13, atol=1e-15)
    g = -2 * alpha * r + gJ
    np.testing.assert_allclose(out["grad_lnpsi"][:, 0, :], g, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(out["lap_lnpsi"][:, 0], -6 * alpha + lJ, rtol=1e-12, atol=1e-13)
    EL = -0.5 * (-6 * alpha + lJ + (g ** 2).sum(-1)) - 1.0 / np.sqrt(r2)
    np.testing.assert_allclose(out["EL"], EL, rtol=1e-12)


def _jastrow_functions(sx, pts):
    """Values of the Jastrow basis functions at pts (n, 3), through an oracle system whose
    determinant basis is the Jastrow basis (AO values are pinned by quadrature and by finite
    differences elsewhere)."""
    jb = sx.jastrow.basis
    shells = [(int(c), int(l), list(jb.shell_exp[s, :jb.shell_nprim[s]]), list(jb.shell_coef[s, :jb.shell_nprim[s]]))
              for s, (c, l) in enumerate(zip(jb.shell_center, jb.shell_l))]
    C = np.zeros((jb.MJ, 1))
    C[0, 0] = 1.0
    aux = S.custom_system("jb", sx.Z, sx.R, shells, 1, 0, C, None, copy.copy(NOJ))
    return oracle.Oracle(aux).ao_eval(pts)[:, :, 0]


def test_pair_and_one_body_terms_by_the_matrix_identity(water_jb):
    """The Jastrow value added by the AO-expanded terms equals xi.s + (s^T Xi s - sum_e phi_e^T Xi phi_e)/2,
    with every phi_e from the basis evaluation; the one-body and pair parts are checked apart."""
    sx = water_jb
    jb = sx.jastrow.basis
    pos = S.initial_walkers(sx, 5, seed=4)
    base = copy.deepcopy(sx)
    base.jastrow.basis = None
    J0 = oracle.Oracle(base).eval(pos, want=("parts",))["parts"][:, 4]
    for xi, Xi in [(jb.xi, jb.Xi), (jb.xi, 0 * jb.Xi), (0 * jb.xi, jb.Xi)]:
        s2 = copy.deepcopy(sx)
        s2.jastrow.basis = S.JastrowBasis(jb.shell_center, jb.shell_l, jb.shell_nprim, jb.shell_exp, jb.shell_coef,
                                          xi, Xi)
        J1 = oracle.Oracle(s2).eval(pos, want=("parts",))["parts"][:, 4]
        for w in range(pos.shape[0]):
            phi = _jastrow_functions(sx, pos[w])  # (Ne, MJ)
            s = phi.sum(0)
            U = xi @ s + 0.5 * (s @ Xi @ s - np.einsum("em,mn,en->", phi, Xi, phi))
            assert abs((J1[w] - J0[w]) - U) < 1e-12 * max(1.0, abs(U)), (w, J1[w] - J0[w], U)
        assert np.abs(J1 - J0).max() > 1e-2  # the term is not negligible


def test_derivatives_by_finite_differences(water_jb):
    """grad and lap of ln Psi, E_L, dE_L/dr_e, d ln Psi/dR and dE_L/dR, with the Jastrow functions
    moving with their nuclei, against O(h^4) central differences."""
    sx = water_jb
    o = oracle.Oracle(sx)
    pos = S.initial_walkers(sx, 4, seed=23)
    out = o.eval(pos, want=("grad_lnpsi", "lap_lnpsi", "EL", "parts", "dlnpsi_dR", "dEL_dR"))
    wv = o.eval_warp(pos)
    h = 1e-4
    lap_fd = np.zeros((4, sx.Ne))
    for e in range(sx.Ne):
        for d in range(3):
            def f(t, what, e=e, d=d):
                p = pos.copy()
                p[:, e, d] += t
                return o.eval(p, want=(what,))[what]
            np.testing.assert_allclose(_rich(lambda t: f(t, "logpsi"), h), out["grad_lnpsi"][:, e, d],
                                       rtol=1e-7, atol=1e-7)
            lap_fd[:, e] += _rich(lambda t: f(t, "grad_lnpsi")[:, e, d], h)
            if (e + d) % 3 == 0:
                fdE = _rich(lambda t: f(t, "EL"), h)
                np.testing.assert_allclose(wv["dEL_dr"][:, e, d], fdE, rtol=1e-6, atol=1e-6 * np.abs(fdE).max())
    np.testing.assert_allclose(lap_fd, out["lap_lnpsi"], rtol=1e-7, atol=1e-7)
    V = out["parts"][:, 1] + out["parts"][:, 2] + out["parts"][:, 3]
    EL = -0.5 * (lap_fd + (out["grad_lnpsi"] ** 2).sum(-1)).sum(1) + V
    np.testing.assert_allclose(EL, out["EL"], rtol=1e-6)

    def with_R(I, d, t):
        s = copy.deepcopy(sx)
        s.R = s.R.copy()
        s.R[I, d] += t
        return oracle.Oracle(s)
    for I in range(sx.K):
        for d in range(3):
            fdE = _rich(lambda t: with_R(I, d, t).eval(pos, want=("EL",))["EL"], h)
            fdl = _rich(lambda t: with_R(I, d, t).eval(pos, want=("logpsi",))["logpsi"], h)
            np.testing.assert_allclose(out["dEL_dR"][:, I, d], fdE, rtol=1e-5, atol=1e-5)
            np.testing.assert_allclose(out["dlnpsi_dR"][:, I, d], fdl, rtol=1e-6, atol=1e-6)


def test_translational_sum_rules(water_jb):
    """Moving every nucleus and electron together changes nothing: sum_I d/dR_I + sum_e d/dr_e = 0
    for ln Psi and for E_L."""
    o = oracle.Oracle(water_jb)
    pos = S.initial_walkers(water_jb, 8, seed=5)
    out = o.eval(pos, want=("dlnpsi_dR", "grad_lnpsi", "dEL_dR"))
    wv = o.eval_warp(pos)
    t1 = out["dlnpsi_dR"].sum(1) + out["grad_lnpsi"].sum(1)
    t2 = out["dEL_dR"].sum(1) + wv["dEL_dr"].sum(1)
    assert np.abs(t1).max() < 1e-10 * np.abs(out["grad_lnpsi"]).max()
    assert np.abs(t2).max() < 1e-9 * np.abs(out["dEL_dR"]).max()


def test_move_jastrow_difference_equals_the_change_of_J(water_jb):
    """The sampler's Jastrow difference for a single-electron move equals the change of the
    evaluated Jastrow value J, for moves of every electron (the two-body, e-n and AO-expanded
    terms together, and the AO-expanded terms alone)."""
    base = copy.deepcopy(water_jb)
    base.jastrow = copy.copy(water_jb.jastrow)
    only = copy.deepcopy(water_jb)
    only.jastrow = S.Jastrow(enable_J1=False, enable_J2=False, basis=water_jb.jastrow.basis)
    rng = np.random.default_rng(9)
    for sx in (base, only):
        o = oracle.Oracle(sx)
        pos = S.initial_walkers(sx, 2, seed=12)
        for w in range(2):
            for e in range(sx.Ne):
                new = pos[w].copy()
                new[e] += 0.6 * rng.standard_normal(3)
                J = o.eval(np.stack([pos[w], new]), want=("parts",))["parts"][:, 4]
                dJ = o.move_jastrow_diff(pos[w], e, new[e])
                assert abs(dJ - (J[1] - J[0])) < 1e-11 * max(1.0, abs(J[0])), (w, e, dJ, J[1] - J[0])


def _u01(x):
    return float(int(x) >> 11) * (1.0 / 9007199254740992.0)


def test_metropolis_chain_replayed_from_log_psi(water_jb):
    """One sweep of the oracle's chain equals a replay that draws the Gaussian proposal and the
    acceptance uniform from the Philox4x64-10 generator (pinned to numpy's; counter (wid, sweep, e, 0 or 1)) and accepts when
    u < |Psi(r')/Psi(r)|^2 with ln|Psi| from the oracle's evaluation: the move's Jastrow
    difference carries the AO-expanded terms."""
    sx = water_jb
    o = oracle.Oracle(sx)
    W, key = 3, (5222, 77)
    pos0 = S.initial_walkers(sx, W, seed=8)
    st = o.new_state(pos0, key=key)
    o.sample(st, 1, sigma=0.45, refresh_k=10 ** 9)
    rep = pos0.copy()
    nacc = 0
    for w in range(W):
        for e in range(sx.Ne):
            prev = np.array([w, 0, e, 0], np.uint64)
            r = oracle.philox4x64_10(prev, key)
            u1, u2, u3, u4 = (_u01(x) for x in r)
            a = math.sqrt(-2.0 * math.log(1.0 - u1))
            b = math.sqrt(-2.0 * math.log(1.0 - u3))
            xi3 = np.array([a * math.cos(2 * math.pi * u2), a * math.sin(2 * math.pi * u2),
                            b * math.cos(2 * math.pi * u4)])
            new = rep[w].copy()
            new[e] += 0.45 * xi3
            lp = o.eval(np.stack([rep[w], new]), want=("logpsi",))["logpsi"]
            p = math.exp(2.0 * (lp[1] - lp[0]))
            u = _u01(oracle.philox4x64_10(np.array([w, 0, e, 1], np.uint64), key)[0])
            assert abs(u - p) > 1e-9 * p  # the decision is not a tie at this precision
            if u < p:
                rep[w] = new
                nacc += 1
    np.testing.assert_allclose(st["pos"], rep, rtol=0, atol=1e-12)
    assert 0 < nacc < W * sx.Ne
