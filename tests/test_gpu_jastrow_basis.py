"""AO-expanded Jastrow terms (App., Eqs. onebody_J_inhom and threebody_jas: the inhomogeneous one-body
term and the three/four-body pair term over a separate Jastrow basis) on the GPU against the oracle:
per-walker outputs in FP64 (1e-10 normwise), space-warp vectors, FP64 chains and estimators following
the oracle's chain (plain, and guided with the space-warp estimator), mixed-precision local energies (1e-5)
and estimators (within 0.1 of their error bars, paired with FP64), and ragged batches. Water and C2OH6 run
on the one-warp-per-walker kernels unless a test forces the walker-group kernels (group=True)."""
import numpy as np
import pytest

import oracle
from oracle import estimators
from paper_2511_05222_gb300 import systems as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_05222_gb300 import vmcf  # noqa: E402

TOL64 = 1e-10
ALL = ("EL", "logpsi", "dlnpsi_dR", "dEL_dR", "O", "dEL_dC")
NO_DC = ("EL", "logpsi", "dlnpsi_dR", "dEL_dR", "O")


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def gpu_eval(system, pos, want):
    out = vmcf.vmcf_evaluate(system, dev(pos), want=want)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def with_jb(cfg, seed=3, scale=1.0):
    """Workload cfg with a seeded medium Jastrow basis (coefficients scale x the defaults)."""
    sx = S.make_system(cfg)
    return S.with_jastrow_basis(sx, S.jastrow_basis(sx, seed, 0.1 * scale, 0.03 * scale, 0.01 * scale))


@pytest.fixture(scope="module")
def water_jb():
    return with_jb(0, scale=3.0)


@pytest.fixture(scope="module")
def c2oh6_jb():
    return with_jb(1)


@pytest.mark.parametrize("W,group", [(1, False), (37, False), (37, True)])
def test_evaluate_fp64_water(water_jb, W, group):
    pos = S.initial_walkers(water_jb, W, seed=5)
    ref = oracle.Oracle(water_jb).eval(pos, want=ALL)
    g = vmcf.System(water_jb, vmcf.FP64, force_group=group)
    for want in (NO_DC, ALL):
        got = gpu_eval(g, pos, want)
        for k in want:
            assert rel(got[k], ref[k]) < TOL64, (k, rel(got[k], ref[k]))


def test_evaluate_fp64_c2oh6(c2oh6_jb):
    pos = S.initial_walkers(c2oh6_jb, 24, seed=6)
    ref = oracle.Oracle(c2oh6_jb).eval(pos, want=ALL)
    got = gpu_eval(vmcf.System(c2oh6_jb, vmcf.FP64), pos, ALL)
    for k in ALL:
        assert rel(got[k], ref[k]) < TOL64, (k, rel(got[k], ref[k]))


@pytest.mark.parametrize("group", [0, 32, 256])
def test_evaluate_fp64_c9o4h8(group):
    """94 electrons, 243 Jastrow-basis functions: more functions than threads per walker group
    for 32- and 128-thread groups."""
    sx = with_jb(4)
    pos = S.initial_walkers(sx, 3, seed=7)
    ref = oracle.Oracle(sx).eval(pos, want=NO_DC)
    g = vmcf.System(sx, vmcf.FP64)
    if group:
        g.set_tuning("measure_group_size", group)
    got = gpu_eval(g, pos, NO_DC)
    for k in NO_DC:
        assert rel(got[k], ref[k]) < TOL64, (k, rel(got[k], ref[k]))


@pytest.mark.parametrize("cfg,group", [(0, False), (1, False), (1, True)])
def test_warp_vectors_fp64(cfg, group, water_jb, c2oh6_jb):
    sx = water_jb if cfg == 0 else c2oh6_jb
    pos = S.initial_walkers(sx, 17, seed=21)
    ref = oracle.Oracle(sx).eval_warp(pos)
    got = vmcf.vmcf_evaluate_warp(vmcf.System(sx, vmcf.FP64, force_group=group), dev(pos))
    torch.cuda.synchronize()
    for k in ("dEL_dr", "dEL_sw", "dlnpsi_sw"):
        assert rel(got[k].cpu().numpy(), ref[k]) < TOL64, (k, rel(got[k].cpu().numpy(), ref[k]))


@pytest.mark.parametrize("kref,group", [(26, False), (7, False), (26, True)])
def test_fp64_chain_and_estimators_follow_the_oracle(water_jb, kref, group):
    W, nb, warm, meas, e_ref = 128, 8, 3, 2, -76.0
    pos = S.initial_walkers(water_jb, W, seed=9)
    o = oracle.Oracle(water_jb)
    st = o.new_state(pos, key=(5222, 0))
    o.sample(st, warm, refresh_k=kref)
    g = vmcf.System(water_jb, vmcf.FP64, force_group=group)
    wk = vmcf.Walkers(g, pos, key=(5222, 0), nblocks=nb)
    wk.sample(warm, 0.3, kref, measure=False)
    ok = st["margin"] >= 1e-9
    assert ok.sum() >= W - 2
    assert np.abs(wk.positions()[ok] - st["pos"][ok]).max() < 1e-9
    wk.reset_accumulators(e_ref)
    wk.sample(meas, 0.3, kref, measure=True)
    sums = estimators.new_sums(nb, water_jb.K, o.nO)
    blk = np.arange(W) * nb // W
    for _ in range(meas):
        o.sample(st, 1, refresh_k=kref)
        o.force_refresh(st)
        out = o.eval(st["pos"], want=("EL", "dlnpsi_dR", "dEL_dR", "O"))
        estimators.accumulate(sums, blk, out["EL"], out["dlnpsi_dR"], out["dEL_dR"], out["O"], e_ref)
    ok = st["margin"] >= 1e-9
    assert np.abs(wk.positions()[ok] - st["pos"][ok]).max() < 1e-9
    if ok.all():
        ref = estimators.finish(sums, e_ref)
        got = wk.reduce_estimators()
        assert abs(got["E"] - ref["E"]) < 1e-10 * abs(ref["E"])
        assert rel(got["F"].ravel(), ref["F"]) < 1e-9
        assert rel(got["dEdC"], ref["dEdC"]) < 1e-9


@pytest.mark.parametrize("group", [False, True])
def test_mixed_local_energy(c2oh6_jb, group):
    """Mixed precision on walkers drawn from |Psi|^2 (20 oracle sweeps): per-walker E_L within 1e-5 of
    max(|E_L|, |mean E_L|) for nearly every walker, median 1e-6."""
    o = oracle.Oracle(c2oh6_jb)
    st = o.new_state(S.initial_walkers(c2oh6_jb, 128, seed=8), key=(5222, 8))
    o.sample(st, 20)
    pos = st["pos"]
    ref = o.eval(pos, want=("EL",))["EL"]
    got = gpu_eval(vmcf.System(c2oh6_jb, vmcf.MIXED, force_group=group), pos, ("EL",))["EL"]
    r = np.abs(got - ref) / np.maximum(np.abs(ref), abs(ref.mean()))
    assert np.median(r) < 1e-6
    assert np.mean(r < 1e-5) > 0.98, np.sort(r)[-8:]


@pytest.mark.parametrize("precision,group", [(vmcf.FP64, True), (vmcf.MIXED, True), (vmcf.FP64, False),
                                             (vmcf.MIXED, False)])
def test_batch_with_jastrow_basis_follows_the_single_path(water_jb, c2oh6_jb, precision, group):
    """A ragged batch holding systems with and without the AO-expanded terms, on either kernel family: same
    chains (bit for bit) and walker sums (FP64 1e-12, mixed 1e-5) as each walker set sampled alone."""
    specs = [(water_jb, 48), (c2oh6_jb, 32), (S.make_system(0), 24)]
    systems = [vmcf.System(sx, precision, force_group=group) for sx, _ in specs]

    def walkers():
        return [vmcf.Walkers(systems[g], S.initial_walkers(sx, W, seed=30 + g), key=(5222, 400 + g), nblocks=4)
                for g, (sx, W) in enumerate(specs)]
    wa, wb = walkers(), walkers()
    batch = vmcf.Batch(systems, wa)
    batch.sample(2, measure=False)
    for g, w in enumerate(wa):
        w.reset_accumulators(-100.0)
        wb[g].sample(2, measure=False)
        wb[g].reset_accumulators(-100.0)
    batch.sample(2, measure=True)
    for w in wb:
        w.sample(2, measure=True)
    tol = 1e-12 if precision == vmcf.FP64 else 1e-5
    for g in range(len(specs)):
        np.testing.assert_array_equal(wa[g].positions(), wb[g].positions())
        assert rel(wa[g].block_sums(), wb[g].block_sums()) < tol


def test_invalid_jastrow_coefficients_are_rejected(water_jb):
    jb = water_jb.jastrow.basis
    bad = S.with_jastrow_basis(S.make_system(0), S.JastrowBasis(jb.shell_center, jb.shell_l, jb.shell_nprim,
                                                                  jb.shell_exp, jb.shell_coef, jb.xi, jb.Xi + np.triu(
                                                                      np.full_like(jb.Xi, 1e-3), 1)))
    with pytest.raises(vmcf.VmcfError):
        vmcf.System(bad, vmcf.FP64)
    nan = S.with_jastrow_basis(S.make_system(0), S.JastrowBasis(jb.shell_center, jb.shell_l, jb.shell_nprim,
                                                                  jb.shell_exp, jb.shell_coef, jb.xi * np.nan, jb.Xi))
    with pytest.raises(vmcf.VmcfError):
        vmcf.System(nan, vmcf.FP64)


@pytest.mark.parametrize("cfg", [0, 1])
def test_mixed_estimators_within_a_tenth_of_their_error_bars(cfg, water_jb, c2oh6_jb):
    """Mixed-precision sampling with the AO-expanded terms; the FP64 path measures the same
    configurations after every sweep (paired). E, every force component and every dE/dC element of
    the mixed path lie within 0.1 x the FP64 path's jackknife error bar."""
    sx = water_jb if cfg == 0 else c2oh6_jb
    W = 4096
    gm = vmcf.System(sx, vmcf.MIXED)
    g64 = vmcf.System(sx, vmcf.FP64)
    wm = vmcf.Walkers(gm, S.initial_walkers(sx, W, seed=12), key=(5222, 60 + cfg), nblocks=32)
    wm.sample(20, measure=False)
    w64 = vmcf.Walkers(g64, wm.positions(), key=(5222, 60 + cfg), nblocks=32)
    e_ref = {0: -76.0, 1: -150.0}[cfg]
    wm.reset_accumulators(e_ref)
    w64.reset_accumulators(e_ref)
    for _ in range(6):
        wm.sample(1, measure=True)
        w64.set_positions(wm.positions())
        w64.measure()
    em, e64 = wm.reduce_estimators(), w64.reduce_estimators()
    assert abs(em["E"] - e64["E"]) <= 0.1 * e64["E_err"], (em["E"], e64["E"], e64["E_err"])
    dF = np.abs(em["F"] - e64["F"]) / e64["F_err"]
    assert dF.max() <= 0.1, dF.max()
    ok = e64["dEdC_err"] > 0
    dB = np.abs(em["dEdC"] - e64["dEdC"])[ok] / e64["dEdC_err"][ok]
    assert dB.max() <= 0.1, dB.max()


def test_guided_space_warp_chain_follows_the_oracle(water_jb):
    """Reweighted (guided) FP64 sampling of a system with the AO-expanded terms and the space-warp
    estimator on: the chain, the weighted plain estimators and the weighted space-warp forces as the
    oracle's."""
    W, nb, warm, meas, e_ref = 96, 8, 3, 2, -76.0
    o = oracle.Oracle(water_jb)
    st = o.new_state(S.initial_walkers(water_jb, W, seed=43), key=(5222, 0))
    o.sample(st, 8)
    pos = st["pos"].copy()
    Bf = o.refresh(pos)
    eps = 1.0 / np.sqrt(np.quantile((Bf ** 2).sum(1), 0.5))
    st = o.new_state(pos, key=(5222, 0))
    o.sample(st, warm, eps=eps)
    g = vmcf.System(water_jb, vmcf.FP64, space_warp=True)
    wk = vmcf.Walkers(g, pos, key=(5222, 0), nblocks=nb)
    wk.set_guiding(eps)
    wk.sample(warm, measure=False)
    wk.reset_accumulators(e_ref)
    wk.sample(meas, measure=True)
    plain = estimators.new_sums(nb, water_jb.K, o.nO)
    warp = estimators.new_sums(nb, water_jb.K, o.nO)
    blk = np.arange(W) * nb // W
    for _ in range(meas):
        o.sample(st, 1, eps=eps)
        o.force_refresh(st)
        out = o.eval(st["pos"], want=("EL", "dlnpsi_dR", "dEL_dR", "O"))
        wv = o.eval_warp(st["pos"])
        wt = o.guide_weight(st["pos"], eps)
        estimators.accumulate(plain, blk, out["EL"], out["dlnpsi_dR"], out["dEL_dR"], out["O"], e_ref, weight=wt)
        estimators.accumulate(warp, blk, out["EL"], wv["dlnpsi_sw"], wv["dEL_sw"], out["O"], e_ref, weight=wt)
    ok = st["margin"] >= 1e-9
    assert np.abs(wk.positions()[ok] - st["pos"][ok]).max() < 1e-9
    if ok.all():
        ref, refw = estimators.finish(plain, e_ref), estimators.finish(warp, e_ref)
        got, gotw = wk.reduce_estimators(), wk.reduce_warp()
        assert abs(got["E"] - ref["E"]) < 1e-10 * abs(ref["E"])
        assert rel(got["F"].ravel(), ref["F"]) < 1e-9
        assert rel(got["dEdC"], ref["dEdC"]) < 1e-9
        assert rel(gotw["F"].ravel(), refw["F"]) < 1e-9


@pytest.mark.parametrize("case", ["one electron, one s function", "water, one p shell"])
def test_smallest_jastrow_bases(case):
    """Jastrow bases of 1 and 3 functions (rows padded to 4 in the products with Xi), in FP64 against the
    oracle: the one-electron case on a proton and water with a single p shell on oxygen."""
    if case.startswith("one"):
        sx = S.custom_system("H", [1], [[0.0, 0.0, 0.0]], [(0, 0, [0.6], [1.0])], 1, 0, [[1.0]], None,
                             S.Jastrow(enable_J1=False, enable_J2=False))
        jb = S.JastrowBasis(np.array([0], np.int32), np.array([0], np.int32), np.array([1], np.int32),
                            np.array([[0.5, 0.0, 0.0]]), np.array([[1.0, 0.0, 0.0]]), np.array([0.4]), np.array([[0.0]]))
    else:
        sx = S.make_system(0)
        rng = np.random.default_rng(5)
        G = rng.standard_normal((3, 3)) * 0.2
        jb = S.JastrowBasis(np.array([0], np.int32), np.array([1], np.int32), np.array([1], np.int32),
                            np.array([[0.8, 0.0, 0.0]]), np.array([[1.0, 0.0, 0.0]]), rng.uniform(-0.3, 0.3, 3),
                            G + G.T)
    sx = S.with_jastrow_basis(sx, jb)
    pos = S.initial_walkers(sx, 9, seed=3)
    ref = oracle.Oracle(sx).eval(pos, want=NO_DC)
    got = gpu_eval(vmcf.System(sx, vmcf.FP64), pos, NO_DC)
    for k in NO_DC:
        assert rel(got[k], ref[k]) < TOL64, (k, rel(got[k], ref[k]))
