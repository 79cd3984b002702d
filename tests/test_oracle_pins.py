"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Every function of the oracle is checked here against something other than itself:
closed forms (single-Gaussian hydrogen, two-electron product states, Kato cusps), exact
Gaussian-integral expectation values, brute-force determinants, quadrature, finite
differences (Richardson-extrapolated), correlated-sampling finite differences, invariances,
and numpy's own Philox generator.
"""
import copy
import dataclasses
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import estimators
from paper_2511_05222_gb300 import systems as S

NOJ = S.Jastrow(enable_J1=False, enable_J2=False)


def hydrogen(alpha, jastrow=NOJ):
    return S.custom_system("H", [1], [[0, 0, 0]], [(0, 0, [alpha], [1.0])], 1, 0, [[1.0]], None, jastrow)


# ------------------------------------------------------------------ Philox (RNG reading P8)
def test_philox_matches_numpy():
    """numpy.random.Philox is Philox4x64-10; it increments the counter before each block."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        ctr = rng.integers(0, 2 ** 63, size=4, dtype=np.uint64)
        key = rng.integers(0, 2 ** 63, size=2, dtype=np.uint64)
        prev = ctr.copy()
        prev[0] -= np.uint64(1)  # no borrow: ctr[0] > 0 with overwhelming probability
        ref = np.random.Philox(counter=[int(x) for x in prev], key=[int(x) for x in key]).random_raw(4)
        np.testing.assert_array_equal(oracle.philox4x64_10(ctr, key), ref)
    # carry across counter words
    ref = np.random.Philox(counter=np.array([2 ** 64 - 1, 5, 0, 0], np.uint64), key=[1, 2]).random_raw(4)
    np.testing.assert_array_equal(oracle.philox4x64_10([0, 6, 0, 0], [1, 2]), ref)


# ------------------------------------------------------------------ H1, H3, cusps (App. A E_L)
@pytest.mark.parametrize("alpha", [0.3, 1.0, 4.7])
def test_h1_hydrogen_single_gaussian(alpha):
    """E_L = 3a - 2a^2 r^2 - 1/r for psi = exp(-a r^2), one proton, no Jastrow."""
    o = oracle.Oracle(hydrogen(alpha))
    pos = np.random.default_rng(1).normal(size=(50, 1, 3))
    r = np.linalg.norm(pos[:, 0], axis=1)
    out = o.eval(pos, want=("EL",))
    np.testing.assert_allclose(out["EL"], 3 * alpha - 2 * alpha ** 2 * r ** 2 - 1 / r, rtol=1e-12, atol=1e-12)


def two_electron(a1, a2, jas, RA=(0, 0, 0), RB=(1.4, 0.2, -0.3)):
    return S.custom_system("H2", [1, 1], [RA, RB], [(0, 0, [a1], [1.0]), (1, 0, [a2], [1.0])], 1, 1,
                           [[1.0], [0.0]], [[0.0], [1.0]], jas)


def test_h3_two_electron_product_state_with_pade():
    """Up electron in a Gaussian on A, down electron in a Gaussian on B, Pade e-e Jastrow
    a r/(1+F r) with a = 1/2: E_L written out from lap(phi1 phi2 e^u)/(phi1 phi2 e^u)."""
    a1, a2 = 0.8, 1.3
    jas = S.Jastrow(enable_J1=False, enable_J2=True)
    sysx = two_electron(a1, a2, jas)
    o = oracle.Oracle(sysx)
    rng = np.random.default_rng(3)
    pos = rng.normal(size=(40, 2, 3))
    A, B = sysx.R
    r1, r2 = pos[:, 0], pos[:, 1]
    d = r1 - r2
    r12 = np.linalg.norm(d, axis=1)
    n = d / r12[:, None]
    a, F = 0.5, 0.8
    up = a / (1 + F * r12) ** 2
    upp = -2 * a * F / (1 + F * r12) ** 3
    g1 = -2 * a1 * (r1 - A)
    g2 = -2 * a2 * (r2 - B)
    kin = (3 * a1 - 2 * a1 ** 2 * ((r1 - A) ** 2).sum(1)) + (3 * a2 - 2 * a2 ** 2 * ((r2 - B) ** 2).sum(1))
    kin += -0.5 * (2 * (upp + 2 * up / r12) + 2 * up ** 2 + 2 * up * (n * g1).sum(1) - 2 * up * (n * g2).sum(1))
    V = 1 / r12 - sum(1.0 / np.linalg.norm(pos[:, e] - R, axis=1) for e in range(2) for R in (A, B))
    V += 1.0 / np.linalg.norm(A - B)
    out = o.eval(pos, want=("EL",))
    np.testing.assert_allclose(out["EL"], kin + V, rtol=1e-11, atol=1e-11)


def test_kato_cusps_keep_EL_finite():
    """The e-n term chi = -Z r/(1+b r) and the e-e terms (1/2 antiparallel, 1/4 parallel)
    carry Kato's cusp slopes, so E_L stays finite at coalescence; without them it diverges."""
    def el_at(sysx, pos):
        return oracle.Oracle(sysx).eval(pos, want=("EL",))["EL"]

    # electron-nucleus
    base = np.array([[[0.3, -0.2, 0.5]]])
    for jas, bounded in ((S.Jastrow(enable_J2=False), True), (NOJ, False)):
        sx = hydrogen(1.1, jas)
        vals = [el_at(sx, base * t)[0] for t in (1e-3, 1e-5, 1e-7)]
        spread = abs(vals[-1] - vals[0])
        assert (spread < 1e-2) if bounded else (spread > 1e5)
    # electron-electron, antiparallel (a = 1/2)
    sx = two_electron(0.7, 0.9, S.Jastrow(enable_J1=False))
    sn = two_electron(0.7, 0.9, NOJ)
    p0 = np.array([0.2, 0.1, -0.1])
    dirv = np.array([0.6, -0.8, 0.0])
    vals = [el_at(sx, np.array([[p0, p0 + t * dirv]]))[0] for t in (1e-3, 1e-5, 1e-7)]
    valn = [el_at(sn, np.array([[p0, p0 + t * dirv]]))[0] for t in (1e-3, 1e-5, 1e-7)]
    assert abs(vals[-1] - vals[0]) < 1e-2 and abs(valn[-1] - valn[0]) > 1e5
    # parallel spins (a = 1/4): two up electrons in s and p orbitals on one centre
    sp = S.custom_system("He*", [2], [[0, 0, 0]], [(0, 0, [0.9], [1.0]), (0, 1, [0.6], [1.0])], 2, 0,
                         np.array([[1, 0], [0, 1], [0, 0], [0, 0]], float), None, S.Jastrow(enable_J1=False))
    vals = [el_at(sp, np.array([[p0, p0 + t * dirv]]))[0] for t in (1e-3, 1e-5, 1e-7)]
    assert abs(vals[-1] - vals[0]) < 1e-2


# ------------------------------------------------------------------ H4 brute-force determinants
def leibniz(A):
    n = A.shape[0]
    tot = 0.0
    for p in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if p[i] > p[j])
        tot += (-1) ** inv * np.prod([A[i, p[i]] for i in range(n)])
    return tot


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_lu_against_leibniz_and_cofactors(n):
    rng = np.random.default_rng(n)
    for _ in range(20):
        A = rng.normal(size=(n, n))
        inv, la, sg, rc = oracle.lu_inverse(A)
        det = leibniz(A)
        assert rc == 0
        assert sg == np.sign(det)
        assert abs(la - math.log(abs(det))) < 1e-12
        cof = np.zeros((n, n))
        for i in range(n):
            for j in range(n):
                minor = np.delete(np.delete(A, i, 0), j, 1)
                cof[i, j] = (-1) ** (i + j) * (leibniz(minor) if n > 1 else 1.0)
        np.testing.assert_allclose(inv, cof.T / det, rtol=1e-11, atol=1e-11)
    inv, la, sg, rc = oracle.lu_inverse(np.zeros((n, n)))
    assert rc == 1 and sg == 0.0


# ------------------------------------------------------------------ AOs (convention P1)
def _sphere_quadrature(nth=10, nph=20):
    x, w = np.polynomial.legendre.leggauss(nth)
    ph = np.arange(nph) * 2 * np.pi / nph
    ct, P = np.meshgrid(x, ph, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(P), st * np.sin(P), ct], -1).reshape(-1, 3)
    wts = (np.repeat(w, nph) * 2 * np.pi / nph)
    return dirs, wts


def test_ao_normalisation_by_quadrature(sys0):
    """Integral of psi_mu psi_nu over space for AOs on one centre, by radial (log grid,
    Simpson) x Gauss-Legendre/trapezoid angular quadrature, equals the Gaussian-product
    overlap of the input generator (diagonal = 1)."""
    o = oracle.Oracle(sys0)
    dirs, wa = _sphere_quadrature()
    t = np.linspace(np.log(1e-5), np.log(12.0), 3001)
    r = np.exp(t)
    wr = np.full(t.size, 2.0)
    wr[1:-1:2] = 4.0
    wr[0] = wr[-1] = 1.0
    wr *= (t[1] - t[0]) / 3 * r ** 3  # dr = r dt, r^2 dr
    centre = sys0.R[0]
    pts = centre + (r[:, None, None] * dirs[None]).reshape(-1, 3)
    vals = o.ao_eval(pts)[:, :, 0].reshape(r.size, dirs.shape[0], -1)
    on_o = [mu for mu in range(14)]  # the 14 AOs of the O atom come first
    G = np.einsum("r,a,ram,ran->mn", wr, wa, vals[:, :, on_o], vals[:, :, on_o])
    np.testing.assert_allclose(np.diag(G), 1.0, atol=1e-8)
    np.testing.assert_allclose(G, sys0.S[np.ix_(on_o, on_o)], atol=1e-8)


def test_ao_derivatives_by_finite_differences(sys0):
    o = oracle.Oracle(sys0)
    rng = np.random.default_rng(5)
    pts = sys0.R[rng.integers(0, 3, 8)] + 0.6 * rng.normal(size=(8, 3))
    h = 1e-4
    base = o.ao_eval(pts)

    def fd(comp):
        g = np.zeros((pts.shape[0], o.M, 3))
        for d in range(3):
            e = np.zeros(3)
            e[d] = h
            p1, m1 = o.ao_eval(pts + e)[:, :, comp], o.ao_eval(pts - e)[:, :, comp]
            p2, m2 = o.ao_eval(pts + 2 * e)[:, :, comp], o.ao_eval(pts - 2 * e)[:, :, comp]
            g[:, :, d] = (8 * (p1 - m1) - (p2 - m2)) / (12 * h)
        return g

    def check(a, b):
        scale = np.abs(b).max() + 1e-300
        assert np.abs(a - b).max() / scale < 1e-7

    check(fd(0), base[:, :, 1:4])
    gx, gy, gz = fd(1), fd(2), fd(3)
    check(gx[:, :, 0] + gy[:, :, 1] + gz[:, :, 2], base[:, :, 4])
    hess = {(0, 0): 5, (1, 1): 6, (2, 2): 7, (0, 1): 8, (0, 2): 9, (1, 2): 10}
    grads = [gx, gy, gz]
    for (a, b), k in hess.items():
        check(grads[a][:, :, b], base[:, :, k])
    check(fd(4), base[:, :, 11:14])


# ------------------------------------------------------------------ wavefunction derivatives
def _rich(f, h):
    """Richardson-extrapolated central difference, O(h^4)."""
    return (4 * (f(h / 2) - f(-h / 2)) / h - (f(h) - f(-h)) / (2 * h)) / 3


def test_I1_translational_identity(sys1):
    o = oracle.Oracle(sys1)
    pos = S.initial_walkers(sys1, 16, seed=3)
    out = o.eval(pos, want=("dlnpsi_dR", "grad_lnpsi", "dEL_dR", "EL"))
    tot = out["dlnpsi_dR"].sum(1) + out["grad_lnpsi"].sum(1)
    assert np.abs(tot).max() < 1e-9 * max(1.0, np.abs(out["grad_lnpsi"]).max())
    # E_L: sum over nuclei of dE_L/dR_I equals minus the derivative under a rigid shift of
    # all electrons.
    for d in range(3):
        def shifted(t):
            p = pos.copy()
            p[:, :, d] += t
            return o.eval(p, want=("EL",))["EL"]
        fd = _rich(shifted, 2e-5)
        np.testing.assert_allclose(out["dEL_dR"][:, :, d].sum(1), -fd, rtol=1e-6,
                                   atol=1e-6 * np.abs(fd).max())


def test_I2_fd_gradient_laplacian_and_EL(sys0):
    o = oracle.Oracle(sys0)
    pos = S.initial_walkers(sys0, 4, seed=11)
    out = o.eval(pos, want=("grad_lnpsi", "lap_lnpsi", "EL", "parts"))
    h = 1e-4
    lap_fd = np.zeros((4, sys0.Ne))
    for e in range(sys0.Ne):
        for d in range(3):
            def f(t):
                p = pos.copy()
                p[:, e, d] += t
                return o.eval(p, want=("logpsi",))["logpsi"]
            g = _rich(f, h)
            np.testing.assert_allclose(g, out["grad_lnpsi"][:, e, d], rtol=1e-7, atol=1e-7)

            def gd(t):
                p = pos.copy()
                p[:, e, d] += t
                return o.eval(p, want=("grad_lnpsi",))["grad_lnpsi"][:, e, d]
            lap_fd[:, e] += _rich(gd, h)
    np.testing.assert_allclose(lap_fd, out["lap_lnpsi"], rtol=1e-7, atol=1e-7)
    # E_L = -1/2 sum_e (lap ln Psi + |grad ln Psi|^2) + V
    V = out["parts"][:, 1] + out["parts"][:, 2] + out["parts"][:, 3]
    EL = -0.5 * (lap_fd + (out["grad_lnpsi"] ** 2).sum(-1)).sum(1) + V
    np.testing.assert_allclose(EL, out["EL"], rtol=1e-6)


def _with_R(sysx, I, d, t):
    s = copy.deepcopy(sysx)
    s.R = s.R.copy()
    s.R[I, d] += t
    return oracle.Oracle(s)


def _with_C(sysx, sg, mu, i, t):
    s = copy.deepcopy(sysx)
    s.C_up, s.C_dn = s.C_up.copy(), s.C_dn.copy()
    (s.C_up if sg == 0 else s.C_dn)[mu, i] += t
    return oracle.Oracle(s)


def test_nuclear_derivatives_by_finite_differences(sys0):
    o = oracle.Oracle(sys0)
    pos = S.initial_walkers(sys0, 24, seed=2)
    out = o.eval(pos, want=("dlnpsi_dR", "dEL_dR"))
    for I in range(sys0.K):
        for d in range(3):
            fdE = _rich(lambda t: _with_R(sys0, I, d, t).eval(pos, want=("EL",))["EL"], 1e-4)
            fdl = _rich(lambda t: _with_R(sys0, I, d, t).eval(pos, want=("logpsi",))["logpsi"], 1e-4)
            np.testing.assert_allclose(out["dEL_dR"][:, I, d], fdE, rtol=1e-5, atol=1e-5)
            np.testing.assert_allclose(out["dlnpsi_dR"][:, I, d], fdl, rtol=1e-6, atol=1e-6)


def test_orbital_derivatives_by_finite_differences(sys0):
    o = oracle.Oracle(sys0)
    pos = S.initial_walkers(sys0, 24, seed=4)
    out = o.eval(pos, want=("O", "dEL_dC"))
    M, n = sys0.M, sys0.n_up
    for sg, mu, i in [(0, 0, 0), (0, 7, 3), (1, 13, 4), (1, 22, 1), (0, 18, 2)]:
        idx = sg * M * n + mu * n + i
        fdl = _rich(lambda t: _with_C(sys0, sg, mu, i, t).eval(pos, want=("logpsi",))["logpsi"], 1e-4)
        fdE = _rich(lambda t: _with_C(sys0, sg, mu, i, t).eval(pos, want=("EL",))["EL"], 1e-4)
        np.testing.assert_allclose(out["O"][:, idx], fdl, rtol=1e-7, atol=1e-7)
        np.testing.assert_allclose(out["dEL_dC"][:, idx], fdE, rtol=1e-6, atol=1e-6)


# ------------------------------------------------------------------ X1 / X2: correlated sampling
def _reweighted_energy(o, pos, logpsi0):
    out = o.eval(pos, want=("EL", "logpsi"))
    w = np.exp(2 * (out["logpsi"] - logpsi0))
    return (w * out["EL"]).sum() / w.sum()


def _one_block_sums(sysx, o, pos, e_ref):
    out = o.eval(pos, want=("EL", "dlnpsi_dR", "dEL_dR", "O"))
    sums = estimators.new_sums(4, sysx.K, o.nO)
    blk = np.arange(pos.shape[0]) * 4 // pos.shape[0]
    estimators.accumulate(sums, blk, out["EL"], out["dlnpsi_dR"], out["dEL_dR"], out["O"], e_ref)
    return estimators.finish(sums, e_ref), out


def test_X1_forces_equal_correlated_sampling_derivative(sys0):
    """With w = (Psi_R'/Psi_R)^2 on fixed walkers, dE/dR of the reweighted mean equals
    <dE_L/dR> + 2(<E_L dlnPsi/dR> - E <dlnPsi/dR>) exactly, i.e. -F (Eqs. hf, pulay)."""
    o = oracle.Oracle(sys0)
    pos = S.initial_walkers(sys0, 64, seed=9)
    res, _ = _one_block_sums(sys0, o, pos, e_ref=-70.0)
    logpsi0 = o.eval(pos, want=("logpsi",))["logpsi"]
    F = res["F"].reshape(sys0.K, 3)
    for I in range(sys0.K):
        for d in range(3):
            fd = _rich(lambda t: _reweighted_energy(_with_R(sys0, I, d, t), pos, logpsi0), 1e-4)
            assert abs(-F[I, d] - fd) < 1e-6 * max(1.0, abs(fd))


def test_X2_orbital_gradient_equals_correlated_sampling_derivative(sys0):
    """dE/dC of the reweighted mean equals <dE_L/dC> + B exactly, with B = 2(<E_L O> - E<O>)."""
    o = oracle.Oracle(sys0)
    pos = S.initial_walkers(sys0, 64, seed=10)
    res, _ = _one_block_sums(sys0, o, pos, e_ref=-70.0)
    ext = o.eval(pos, want=("dEL_dC", "logpsi"))
    M, n = sys0.M, sys0.n_up
    for sg, mu, i in [(0, 2, 1), (1, 16, 3), (0, 23, 4)]:
        idx = sg * M * n + mu * n + i
        fd = _rich(lambda t: _reweighted_energy(_with_C(sys0, sg, mu, i, t), pos, ext["logpsi"]), 1e-4)
        exact = ext["dEL_dC"][:, idx].mean() + res["dEdC"][idx]
        assert abs(exact - fd) < 1e-6 * max(1.0, abs(fd))


# ------------------------------------------------------------------ invariants I3, I4, I5
def test_I3_CtO_identity_and_B_projection(sys1):
    o = oracle.Oracle(sys1)
    pos = S.initial_walkers(sys1, 32, seed=6)
    res, out = _one_block_sums(sys1, o, pos, e_ref=-150.0)
    M, n = sys1.M, sys1.n_up
    O = out["O"].reshape(-1, 2, M, n)
    for sg, C in ((0, sys1.C_up), (1, sys1.C_dn)):
        np.testing.assert_allclose(np.einsum("mj,wmi->wji", C, O[:, sg]), np.broadcast_to(np.eye(n), (32, n, n)),
                                   atol=1e-9)
        Bs = res["dEdC"].reshape(2, M, n)[sg]
        # C^T B = 0, hence B Q = B with Q = 1 - C C^T S (Eq. Q_projector)
        assert np.abs(C.T @ Bs).max() < 1e-9 * np.abs(Bs).max()
        Q = np.eye(M) - C @ C.T @ sys1.S
        np.testing.assert_allclose(Q.T @ Bs, Bs, atol=1e-9 * np.abs(Bs).max())


def test_I4_orbital_rotation_and_exchange(sys0):
    o = oracle.Oracle(sys0)
    pos = S.initial_walkers(sys0, 16, seed=12)
    out = o.eval(pos, want=("EL", "dlnpsi_dR", "dEL_dR", "O", "sign"))
    rng = np.random.default_rng(0)
    n, M = sys0.n_up, sys0.M
    G = rng.normal(size=(n, n))
    s2 = copy.deepcopy(sys0)
    s2.C_up = sys0.C_up @ G
    out2 = oracle.Oracle(s2).eval(pos, want=("EL", "dlnpsi_dR", "dEL_dR", "O"))
    np.testing.assert_allclose(out2["EL"], out["EL"], rtol=1e-9)
    np.testing.assert_allclose(out2["dlnpsi_dR"], out["dlnpsi_dR"], rtol=1e-8, atol=1e-8)
    np.testing.assert_allclose(out2["dEL_dR"], out["dEL_dR"], rtol=1e-7, atol=1e-7)
    O1 = out["O"].reshape(-1, 2, M, n)[:, 0]
    O2 = out2["O"].reshape(-1, 2, M, n)[:, 0]
    np.testing.assert_allclose(O2, O1 @ np.linalg.inv(G).T, rtol=1e-8, atol=1e-8)
    # swap two up electrons
    p = pos.copy()
    p[:, [0, 1]] = p[:, [1, 0]]
    out3 = o.eval(p, want=("EL", "sign"))
    np.testing.assert_allclose(out3["EL"], out["EL"], rtol=1e-11)
    np.testing.assert_array_equal(out3["sign"], -out["sign"])


def test_I5_total_force_vanishes(sys0):
    """Translational invariance: the nuclear-nuclear forces cancel exactly, and the sampled
    total force sum_I F_I vanishes within its jackknife error bar."""
    R, Z = sys0.R, sys0.Z
    Fnn = np.zeros_like(R)
    for I in range(sys0.K):
        for J in range(sys0.K):
            if I != J:
                d = R[I] - R[J]
                Fnn[I] += Z[I] * Z[J] * d / np.linalg.norm(d) ** 3
    assert np.abs(Fnn.sum(0)).max() < 1e-12
    o = oracle.Oracle(sys0)
    W, nb = 1024, 32
    st = o.new_state(S.initial_walkers(sys0, W, seed=31), key=(5222, 0))
    o.sample(st, 30)
    sums = estimators.new_sums(nb, sys0.K, o.nO)
    blk = np.arange(W) * nb // W
    for _ in range(20):
        o.sample(st, 2)
        o.force_refresh(st)
        out = o.eval(st["pos"], want=("EL", "dlnpsi_dR", "dEL_dR", "O"))
        estimators.accumulate(sums, blk, out["EL"], out["dlnpsi_dR"], out["dEL_dR"], out["O"], -76.0)
    tot, err = estimators.jackknife(sums, -76.0, lambda E, F, B: F.reshape(-1, 3).sum(0))
    assert np.all(np.abs(tot) < 4.5 * err + 1e-12), (tot, err)


# ------------------------------------------------------------------ H2: sampling
def test_h2_sampled_gaussian_expectations():
    """|psi|^2 for psi = exp(-a r^2) gives <E_L> = 3a/2 - 2 sqrt(2a/pi) and <r^2> = 3/(4a)."""
    a = 0.35
    o = oracle.Oracle(hydrogen(a))
    W = 3000
    st = o.new_state(np.random.default_rng(1).normal(size=(W, 1, 3)), key=(5222, 77))
    o.sample(st, 100, sigma=0.8)
    accE = np.zeros(W)
    accr = np.zeros(W)
    nm = 60
    for _ in range(nm):
        o.sample(st, 3, sigma=0.8)
        accE += o.eval(st["pos"], want=("EL",))["EL"]
        accr += (st["pos"] ** 2).sum(axis=(1, 2))
    Ew, rw = accE / nm, accr / nm  # independent chains: per-walker time averages
    for vals, exact in ((Ew, 1.5 * a - 2 * math.sqrt(2 * a / math.pi)), (rw, 3 / (4 * a))):
        err = vals.std(ddof=1) / math.sqrt(W)
        assert abs(vals.mean() - exact) < 4.5 * err, (vals.mean(), exact, err)


def test_sherman_morrison_matches_fresh_inverse(sys1):
    o = oracle.Oracle(sys1)
    st = o.new_state(S.initial_walkers(sys1, 16, seed=21), key=(5222, 1))
    o.sample(st, 2, refresh_k=10 ** 9)
    fresh = o.refresh(st["pos"])
    assert np.abs(st["B"] - fresh).max() < 1e-9 * np.abs(fresh).max()
    assert st["nacc"].sum() > 0


def test_refresh_cadence_and_counter(sys0):
    o = oracle.Oracle(sys0)
    st = o.new_state(S.initial_walkers(sys0, 4, seed=1))
    o.sample(st, 3, refresh_k=7)
    assert st["counter"] == (3 * sys0.Ne) % 7
    o.force_refresh(st)
    assert st["counter"] == 0
    np.testing.assert_allclose(st["B"], o.refresh(st["pos"]), rtol=0, atol=0)


def test_lowering_k_between_calls_re_inverts_first(sys0):
    """A call whose k is at or below the moves already made since the last re-inversion starts
    with one: the chain is the one of an explicit re-inversion before the call."""
    o = oracle.Oracle(sys0)
    pos = S.initial_walkers(sys0, 6, seed=2)
    a = o.new_state(pos, key=(5222, 3))
    b = o.new_state(pos, key=(5222, 3))
    for st in (a, b):
        o.sample(st, 1, refresh_k=26)
    assert a["counter"] == sys0.Ne >= 7
    o.force_refresh(b)
    o.sample(a, 2, refresh_k=7)
    o.sample(b, 2, refresh_k=7)
    np.testing.assert_array_equal(a["pos"], b["pos"])
    np.testing.assert_array_equal(a["B"], b["B"])
    np.testing.assert_array_equal(a["nacc"], b["nacc"])
    assert a["counter"] == b["counter"] == (2 * sys0.Ne) % 7


def test_kinetic_energy_from_the_P_rows(sys0):
    """The kinetic energy as sum_i P_ei B_ie + lap J_e + |grad J_e|^2 with P = lap(phi) + 2 grad J .
    grad(phi) contracted from the AO rows, the Jastrow derivatives written out in closed form here
    (Pade pairs and e-n cusp terms), the AO values and derivatives from the oracle's AO evaluation
    (pinned by quadrature and finite differences): equal to the oracle's kinetic energy."""
    o = oracle.Oracle(sys0)
    j = sys0.jastrow
    pos = S.initial_walkers(sys0, 5, seed=21)
    ekin = o.eval(pos, want=("parts",))["parts"][:, 0]
    R, Z = sys0.R, np.asarray(sys0.Z, float)
    for w in range(pos.shape[0]):
        r = pos[w]
        ao = o.ao_eval(r)  # (Ne, M, 14): value, gradient, Laplacian, ...
        gJ = np.zeros((sys0.Ne, 3))
        lJ = np.zeros(sys0.Ne)
        for e in range(sys0.Ne):
            for q in range(sys0.Ne):
                if q == e:
                    continue
                par = (q < sys0.n_up) == (e < sys0.n_up)
                a, F = (j.a_par, j.F_par) if par else (j.a_anti, j.F_anti)
                d = r[e] - r[q]
                x = np.linalg.norm(d)
                u1, u2 = a / (1 + F * x) ** 2, -2 * a * F / (1 + F * x) ** 3
                gJ[e] += u1 * d / x
                lJ[e] += u2 + 2 * u1 / x
            for I in range(sys0.K):
                d = r[e] - R[I]
                x = np.linalg.norm(d)
                c1, c2 = -Z[I] / (1 + j.b_en * x) ** 2, 2 * Z[I] * j.b_en / (1 + j.b_en * x) ** 3
                gJ[e] += c1 * d / x
                lJ[e] += c2 + 2 * c1 / x
        total = 0.0
        for sg, C in ((0, sys0.C_up), (1, sys0.C_dn)):
            es = range(0, sys0.n_up) if sg == 0 else range(sys0.n_up, sys0.Ne)
            v = ao[list(es)]
            A = v[:, :, 0] @ C
            B = np.linalg.inv(A)  # B[i, el]
            P = v[:, :, 4] @ C + 2 * np.einsum("ek,emk->em", gJ[list(es)], v[:, :, 1:4]) @ C
            total += np.einsum("ei,ie->", P, B)
        total += lJ.sum() + (gJ ** 2).sum()
        assert abs(-0.5 * total - ekin[w]) < 1e-10 * max(1.0, abs(ekin[w])), (w, -0.5 * total, ekin[w])


# ------------------------------------------------------------------ jackknife
def test_jackknife_of_a_mean_is_the_block_standard_error():
    rng = np.random.default_rng(0)
    nb, per = 16, 50
    x = rng.normal(size=nb * per) + 3.0
    sums = estimators.new_sums(nb, 1, 1)
    blk = np.repeat(np.arange(nb), per)
    z = np.zeros((x.size, 1, 3))
    estimators.accumulate(sums, blk, x, z, z, np.zeros((x.size, 1)), 0.0)
    res = estimators.finish(sums, 0.0)
    bm = x.reshape(nb, per).mean(1)
    assert abs(res["E"] - x.mean()) < 1e-12
    assert abs(res["E_err"] - bm.std(ddof=1) / math.sqrt(nb)) < 1e-12


def test_jackknife_covariance_of_means_is_the_block_covariance():
    """When the estimators reduce to plain sample means (E_L averaging to E_ref inside every
    block, so that F = -<dE_L/dR> and B = 2 <(E_L - E_ref) O>), the delete-one-block jackknife
    covariance equals the textbook covariance of the block means divided by the block count."""
    rng = np.random.default_rng(1)
    nb, per, K, nO = 8, 40, 2, 5
    e_ref = -1.5
    n = nb * per
    dEL = rng.normal(size=(n, K, 3))
    O = rng.normal(size=(n, nO))
    dev = rng.normal(size=n // 2)
    EL = e_ref + np.stack([dev, -dev], 1).ravel()  # +d, -d pairs: every block averages to e_ref
    blk = np.repeat(np.arange(nb), per)
    sums = estimators.new_sums(nb, K, nO)
    estimators.accumulate(sums, blk, EL, np.zeros((n, K, 3)), dEL, O, e_ref)
    cF, cB = estimators.jackknife_covariance(sums, e_ref)
    for x, c in ((-dEL.reshape(n, -1), cF), (2.0 * (EL - e_ref)[:, None] * O, cB)):
        bm = x.reshape(nb, per, -1).mean(1)
        ref = np.cov(bm, rowvar=False, ddof=1) / nb
        np.testing.assert_allclose(c, ref, rtol=1e-10, atol=1e-14)
    res = estimators.finish(sums, e_ref)
    np.testing.assert_allclose(np.sqrt(np.diag(cB)), res["dEdC_err"], rtol=1e-12)


# ------------------------------------------------------------------ space warp (SWCT)
def test_electron_derivatives_of_EL_by_finite_differences(sys0):
    """dE_L/dr_e against O(h^4) central differences of E_L, and the exact translational sum
    rule sum_I dE_L/dR_I + sum_e dE_L/dr_e = 0."""
    o = oracle.Oracle(sys0)
    pos = S.initial_walkers(sys0, 6, seed=13)
    w = o.eval_warp(pos)
    for e, d in [(0, 0), (2, 1), (5, 2), (9, 0), (4, 1)]:
        def f(t):
            p = pos.copy()
            p[:, e, d] += t
            return o.eval(p, want=("EL",))["EL"]
        fd = _rich(f, 1e-4)
        np.testing.assert_allclose(w["dEL_dr"][:, e, d], fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())
    out = o.eval(pos, want=("dEL_dR",))
    tot = out["dEL_dR"].sum(1) + w["dEL_dr"].sum(1)
    assert np.abs(tot).max() < 1e-9 * np.abs(w["dEL_dr"]).max()


def _omega(R, r):
    """Space-warp weights omega_a(r) = |r - R_a|^-4 / sum_b |r - R_b|^-4, (npts, K)."""
    k = ((r[:, None, :] - R[None, :, :]) ** 2).sum(-1) ** -2
    return k / k.sum(1, keepdims=True)


def test_space_warp_vectors_are_derivatives_along_the_warp(sys0):
    """dE_L^sw/dR_a and d ln Psi^sw/dR_a are the total derivatives when nucleus a moves by t e_d
    and every electron by omega_a(r_e) t e_d (plus half the log-Jacobian of that electron map
    for ln Psi); they sum to zero over the nuclei (the warp of every nucleus together is a rigid
    translation)."""
    o = oracle.Oracle(sys0)
    pos = S.initial_walkers(sys0, 5, seed=14)
    w = o.eval_warp(pos)
    assert np.abs(w["dEL_sw"].sum(1)).max() < 1e-9 * np.abs(w["dEL_sw"]).max()
    assert np.abs(w["dlnpsi_sw"].sum(1)).max() < 1e-9 * np.abs(w["dlnpsi_sw"]).max()
    W, Ne = pos.shape[:2]
    om = _omega(sys0.R, pos.reshape(-1, 3)).reshape(W, Ne, sys0.K)
    for a, d in [(0, 0), (1, 2), (2, 1)]:
        def dom(t):  # d omega_a / d r_d at each electron, by central differences of the weights
            p = pos.reshape(-1, 3).copy()
            p[:, d] += t
            return _omega(sys0.R, p)[:, a].reshape(W, Ne)
        gom = _rich(dom, 1e-5)

        def moved(t, what):
            p = pos.copy()
            p[:, :, d] += om[:, :, a] * t
            out = _with_R(sys0, a, d, t).eval(p, want=(what,))[what]
            if what == "logpsi":
                out = out + 0.5 * np.log1p(t * gom).sum(1)
            return out
        fdE = _rich(lambda t: moved(t, "EL"), 1e-4)
        fdl = _rich(lambda t: moved(t, "logpsi"), 1e-4)
        np.testing.assert_allclose(w["dEL_sw"][:, a, d], fdE, rtol=1e-5, atol=1e-5 * np.abs(fdE).max())
        np.testing.assert_allclose(w["dlnpsi_sw"][:, a, d], fdl, rtol=1e-6, atol=1e-6 * np.abs(fdl).max())


# ------------------------------------------------------------------ reweighted (guided) sampling
def test_guided_sampling_with_eps_zero_is_plain_sampling(sys0):
    o = oracle.Oracle(sys0)
    pos = S.initial_walkers(sys0, 32, seed=31)
    a, b = o.new_state(pos, key=(5222, 0)), o.new_state(pos, key=(5222, 0))
    o.sample(a, 5)
    o.sample(b, 5, eps=0.0)
    np.testing.assert_array_equal(a["pos"], b["pos"])
    np.testing.assert_array_equal(o.guide_weight(a["pos"], 0.0), np.ones(32))


def test_guided_weights_and_estimates(sys0):
    """Weights |Psi/Psi_G|^2 = min(1, 1/(eps^2 S)) with S the summed squares of the inverse
    Slater entries (S from an independent numpy inversion of the oracle's Slater matrices), and
    the reweighted estimates from a |Psi_G|^2 chain agree with plain |Psi|^2 sampling within
    their statistical errors (the reweighting identity of the appendix)."""
    o = oracle.Oracle(sys0)
    W, nb = 1024, 16
    pos = S.initial_walkers(sys0, W, seed=32)
    st0 = o.new_state(pos, key=(5222, 0))
    o.sample(st0, 30)
    ao = o.ao_eval(st0["pos"].reshape(-1, 3))[:, :, 0].reshape(W, sys0.Ne, -1)
    Sx = (np.linalg.inv(ao[:, :sys0.n_up] @ sys0.C_up) ** 2).sum((1, 2)) + \
         (np.linalg.inv(ao[:, sys0.n_up:] @ sys0.C_dn) ** 2).sum((1, 2))
    eps = 1.0 / math.sqrt(np.quantile(Sx, 0.8))  # the guide is active on ~20% of |Psi|^2 samples
    wt = o.guide_weight(st0["pos"], eps)
    np.testing.assert_allclose(wt, np.minimum(1.0, 1.0 / (eps ** 2 * Sx)), rtol=1e-9)
    assert 0.1 < (wt < 1).mean() < 0.3
    e_ref = -76.0
    blk = np.arange(W) * nb // W
    res = {}
    for name, e in (("plain", 0.0), ("guided", eps)):
        st = o.new_state(pos, key=(5222, 7 if e else 8))
        o.sample(st, 30, eps=e)
        sums = estimators.new_sums(nb, sys0.K, o.nO)
        for _ in range(8):
            o.sample(st, 2, eps=e)
            out = o.eval(st["pos"], want=("EL", "dlnpsi_dR", "dEL_dR", "O"))
            estimators.accumulate(sums, blk, out["EL"], out["dlnpsi_dR"], out["dEL_dR"], out["O"], e_ref,
                                  weight=o.guide_weight(st["pos"], e) if e else None)
        res[name] = estimators.finish(sums, e_ref)
    p, g = res["plain"], res["guided"]
    assert abs(p["E"] - g["E"]) < 4.0 * math.hypot(p["E_err"], g["E_err"])
    dF = np.abs(p["F"] - g["F"]) / np.hypot(p["F_err"], g["F_err"])
    assert np.median(dF) < 1.5 and dF.max() < 5.0


def _u01(x):
    return float(int(x) >> 11) * (1.0 / 9007199254740992.0)


def test_guided_chain_replayed_from_log_psi_and_fresh_inverses(sys0):
    """Two sweeps of the oracle's guided chain equal a replay that draws the proposal and the
    acceptance uniform from Philox4x64-10 (counter (wid, sweep, e, 0 or 1), pinned to numpy's
    generator) and accepts when u < |Psi(r')/Psi(r)|^2 (g'/g)^2, with ln|Psi| from the oracle's
    evaluation and g = max(1, eps sqrt(S)), S the summed squares of inverses taken afresh by numpy
    from the oracle's Slater matrices at both configurations. The chain itself tracks S through
    its Sherman-Morrison updates, so a dropped term of that update, or of (g'/g)^2, changes a
    decision here."""
    o = oracle.Oracle(sys0)
    W, key, sigma, sweeps = 6, (5222, 91), 0.45, 2

    def s_inv(x):  # (n, Ne, 3) -> S per configuration
        n = x.shape[0]
        ao = o.ao_eval(x.reshape(-1, 3))[:, :, 0].reshape(n, sys0.Ne, -1)
        return (np.linalg.inv(ao[:, :sys0.n_up] @ sys0.C_up) ** 2).sum((1, 2)) + \
               (np.linalg.inv(ao[:, sys0.n_up:] @ sys0.C_dn) ** 2).sum((1, 2))

    pos0 = S.initial_walkers(sys0, W, seed=33)
    eps = 3.0 / math.sqrt(np.median(s_inv(pos0)))  # the guide is active on many of the configurations
    st = o.new_state(pos0, key=key)
    o.sample(st, sweeps, sigma=sigma, refresh_k=10 ** 9, eps=eps)
    rep = pos0.copy()
    nacc, active = 0, 0
    for w in range(W):
        for sw in range(sweeps):
            for e in range(sys0.Ne):
                r = oracle.philox4x64_10(np.array([w, sw, e, 0], np.uint64), key)
                u1, u2, u3, u4 = (_u01(x) for x in r)
                a = math.sqrt(-2.0 * math.log(1.0 - u1))
                b = math.sqrt(-2.0 * math.log(1.0 - u3))
                xi3 = np.array([a * math.cos(2 * math.pi * u2), a * math.sin(2 * math.pi * u2),
                                b * math.cos(2 * math.pi * u4)])
                new = rep[w].copy()
                new[e] += sigma * xi3
                both = np.stack([rep[w], new])
                lp = o.eval(both, want=("logpsi",))["logpsi"]
                g = np.maximum(1.0, eps * np.sqrt(s_inv(both)))
                active += int(g[0] > 1.0 or g[1] > 1.0)
                p = math.exp(2.0 * (lp[1] - lp[0])) * (g[1] / g[0]) ** 2
                u = _u01(oracle.philox4x64_10(np.array([w, sw, e, 1], np.uint64), key)[0])
                assert abs(u - p) > 1e-8 * p  # the decision is not a tie at this precision
                if u < p:
                    rep[w] = new
                    nacc += 1
    np.testing.assert_allclose(st["pos"], rep, rtol=0, atol=1e-12)
    assert 0 < nacc < W * sweeps * sys0.Ne
    assert active > W * sweeps * sys0.Ne // 4  # the guiding factor took part in many decisions


# ------------------------------------------------------------------ exponential two-body form
def _with_exp_j2(sysx):
    s = copy.deepcopy(sysx)
    s.jastrow = dataclasses.replace(sysx.jastrow, two_body_exp=True)
    return s


def test_exponential_two_body_term_cusp_and_derivatives(sys0):
    """Eq. twobody_v_exp, u(r) = (a/F)(1 - exp(-F r)): its slope at coalescence is a, so the
    e-e cusp keeps E_L finite; the gradient and Laplacian of ln Psi, E_L and dE_L/dr_e follow
    from O(h^4) central differences; at F -> 0 the form tends to the linear a r, as the Pade
    form does."""
    # cusp: antiparallel pair
    sx = two_electron(0.7, 0.9, S.Jastrow(enable_J1=False, two_body_exp=True))
    p0 = np.array([0.2, 0.1, -0.1])
    dirv = np.array([0.6, -0.8, 0.0])
    o2 = oracle.Oracle(sx)
    vals = [o2.eval(np.array([[p0, p0 + t * dirv]]), want=("EL",))["EL"][0] for t in (1e-3, 1e-5, 1e-7)]
    assert abs(vals[-1] - vals[0]) < 1e-2
    # small F: exponential and Pade forms agree to O(F)
    for exp_form in (True, False):
        s = two_electron(0.7, 0.9, S.Jastrow(enable_J1=False, F_anti=1e-7, two_body_exp=exp_form))
        lp = oracle.Oracle(s).eval(np.array([[p0, p0 + 0.5 * dirv]]), want=("logpsi",))["logpsi"][0]
        if exp_form:
            lp_exp = lp
        else:
            assert abs(lp - lp_exp) < 1e-6
    # derivatives by finite differences on water with the exponential form
    sx = _with_exp_j2(sys0)
    o = oracle.Oracle(sx)
    pos = S.initial_walkers(sx, 4, seed=17)
    out = o.eval(pos, want=("grad_lnpsi", "lap_lnpsi", "EL", "parts"))
    wv = o.eval_warp(pos)
    h = 1e-4
    for e, d in [(0, 0), (3, 2), (8, 1)]:
        def f(t, what):
            p = pos.copy()
            p[:, e, d] += t
            return o.eval(p, want=(what,))[what]
        np.testing.assert_allclose(_rich(lambda t: f(t, "logpsi"), h), out["grad_lnpsi"][:, e, d], rtol=1e-7, atol=1e-7)
        fdE = _rich(lambda t: f(t, "EL"), h)
        np.testing.assert_allclose(wv["dEL_dr"][:, e, d], fdE, rtol=1e-6, atol=1e-6 * np.abs(fdE).max())
    lap_fd = np.zeros((4, sx.Ne))
    for e in range(sx.Ne):
        for d in range(3):
            def gd(t):
                p = pos.copy()
                p[:, e, d] += t
                return o.eval(p, want=("grad_lnpsi",))["grad_lnpsi"][:, e, d]
            lap_fd[:, e] += _rich(gd, h)
    np.testing.assert_allclose(lap_fd, out["lap_lnpsi"], rtol=1e-7, atol=1e-7)
    V = out["parts"][:, 1] + out["parts"][:, 2] + out["parts"][:, 3]
    EL = -0.5 * (lap_fd + (out["grad_lnpsi"] ** 2).sum(-1)).sum(1) + V
    np.testing.assert_allclose(EL, out["EL"], rtol=1e-6)
