"""Edge cases of the CUDA path, through the C ABI, against the FP64 oracle: an empty walker set
(no work and no error), the largest system the one-warp-per-walker kernels take (32 electrons
and 16 orbitals per spin: every lane holds an electron and the register rows are full), an
open-shell system (n_up = n_dn + 1) in both kernel families, a run of zero sweeps, a walker count
that fills no CTA, warp or jackknife block evenly, and a re-inversion interval k lowered between
calls below the moves already made since the last re-inversion (single path and batch), and walker-group
sweeps with and without the proposal pass (the same chains)."""
import numpy as np
import pytest

import oracle
from paper_2511_05222_gb300 import systems as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_05222_gb300 import vmcf  # noqa: E402

KEYS = ("EL", "logpsi", "dlnpsi_dR", "dEL_dR", "O")


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def gpu_eval(system, pos, want=KEYS):
    out = vmcf.vmcf_evaluate(system, torch.as_tensor(np.ascontiguousarray(pos), device="cuda"), want=want)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def molecule(name, Z, n_up, n_dn, seed):
    """A covalent-walk molecule of the seeded recipe with the given spin split."""
    Z = np.asarray(Z, np.int32)
    R = S.covalent_walk(list(Z), np.random.default_rng([7000, seed, 0]))
    c, l, npr, e, co = S.basis_rule(Z, np.random.default_rng([7000, seed, 1]))
    sx = S.System(name, Z, R, c, l, npr, e, co, n_up, n_dn, np.zeros((0, 0)), np.zeros((0, 0)), S.Jastrow())
    Sm = S.overlap_matrix(sx)
    rng = np.random.default_rng([7000, seed, 2])
    sx.C_up = S.orthonormal_orbitals(Sm, n_up, rng)
    sx.C_dn = S.orthonormal_orbitals(Sm, n_dn, rng)
    sx.S = Sm
    return sx


@pytest.mark.parametrize("force_group", [False, True])
def test_empty_walker_set_is_no_work(sys0, force_group):
    g = vmcf.System(sys0, vmcf.FP64, force_group=force_group)
    out = gpu_eval(g, np.zeros((0, sys0.Ne, 3)), want=KEYS)
    for k in KEYS:
        assert out[k].shape[0] == 0
    warp = vmcf.vmcf_evaluate_warp(g, torch.zeros((0, sys0.Ne, 3), dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert all(v.shape[0] == 0 for v in warp.values())


def test_full_warp_system_matches_the_oracle():
    """C2O2H4: 32 electrons, 16 orbitals per spin, 76 AOs."""
    sx = molecule("C2O2H4", [6, 6, 8, 8, 1, 1, 1, 1], 16, 16, seed=1)
    assert (sx.Ne, sx.n_up) == (32, 16)
    o = oracle.Oracle(sx)
    st = o.new_state(S.initial_walkers(sx, 96, seed=3), key=(5222, 11))
    o.sample(st, 10)
    pos = st["pos"]
    ref = o.eval(pos, want=KEYS)
    for force_group in (False, True):
        got = gpu_eval(vmcf.System(sx, vmcf.FP64, force_group=force_group), pos)
        for k in KEYS:
            assert rel(got[k], ref[k]) < 1e-10, (force_group, k, rel(got[k], ref[k]))
    got = gpu_eval(vmcf.System(sx, vmcf.MIXED), pos, ("EL",))["EL"]
    r = np.abs(got - ref["EL"]) / np.maximum(np.abs(ref["EL"]), abs(ref["EL"].mean()))
    assert np.median(r) < 1e-6
    assert np.mean(r < 1e-5) > 0.95, np.sort(r)[-10:]
    # a short FP64 chain on the small-system kernels follows the oracle's
    wk = vmcf.Walkers(vmcf.System(sx, vmcf.FP64), pos, key=(5222, 12), nblocks=4)
    wk.sample(2, 0.3, 26)
    st2 = o.new_state(pos, key=(5222, 12))
    o.sample(st2, 2, sigma=0.3, refresh_k=26)
    ok = st2["margin"] >= 1e-9
    assert ok.sum() >= 94
    assert np.abs(wk.positions()[ok] - st2["pos"][ok]).max() < 1e-9


@pytest.mark.parametrize("force_group", [False, True])
def test_open_shell_system_matches_the_oracle(force_group):
    """CH3 radical: 9 electrons, 5 up and 4 down (spin blocks of different size)."""
    sx = molecule("CH3", [6, 1, 1, 1], 5, 4, seed=2)
    pos = S.initial_walkers(sx, 48, seed=4)
    ref = oracle.Oracle(sx).eval(pos, want=KEYS)
    got = gpu_eval(vmcf.System(sx, vmcf.FP64, force_group=force_group), pos)
    for k in KEYS:
        assert rel(got[k], ref[k]) < 1e-10, (k, rel(got[k], ref[k]))


def test_zero_sweeps_leave_the_walkers_unchanged(sys0):
    pos = S.initial_walkers(sys0, 32, seed=6)
    wk = vmcf.Walkers(vmcf.System(sys0, vmcf.MIXED), pos, nblocks=4)
    before = wk.counters()
    wk.sample(0, 0.3, 26)
    np.testing.assert_array_equal(wk.positions(), pos)
    assert wk.counters() == before


def _block_map(W, nb):
    blk = np.zeros(W, int)
    for b in range(nb):
        blk[(W * b) // nb:(W * (b + 1)) // nb] = b
    return blk


@pytest.mark.parametrize("force_group", [False, True])
def test_ragged_walker_count_chain_and_estimators(sys0, force_group):
    """37 walkers in 5 jackknife blocks of 7 or 8 (a count that fills no CTA, warp or block evenly):
    the FP64 chain and the measured estimators follow the oracle."""
    from oracle import estimators

    W, nb, warm, meas, e_ref = 37, 5, 2, 2, -76.0
    pos = S.initial_walkers(sys0, W, seed=12)
    o = oracle.Oracle(sys0)
    st = o.new_state(pos, key=(5222, 13))
    o.sample(st, warm)
    wk = vmcf.Walkers(vmcf.System(sys0, vmcf.FP64, force_group=force_group), pos, key=(5222, 13), nblocks=nb)
    wk.sample(warm, measure=False)
    wk.reset_accumulators(e_ref)
    wk.sample(meas, measure=True)
    sums = estimators.new_sums(nb, sys0.K, o.nO)
    blk = _block_map(W, nb)
    for _ in range(meas):
        o.sample(st, 1)
        o.force_refresh(st)
        out = o.eval(st["pos"], want=("EL", "dlnpsi_dR", "dEL_dR", "O"))
        estimators.accumulate(sums, blk, out["EL"], out["dlnpsi_dR"], out["dEL_dR"], out["O"], e_ref)
    assert st["margin"].min() >= 1e-9
    assert np.abs(wk.positions() - st["pos"]).max() < 1e-9
    np.testing.assert_array_equal(wk.block_sums()[:, 0], sums["n"])
    ref = estimators.finish(sums, e_ref)
    got = wk.reduce_estimators()
    assert abs(got["E"] - ref["E"]) < 1e-10 * abs(ref["E"])
    assert rel(got["F"].ravel(), ref["F"]) < 1e-9
    assert rel(got["dEdC"], ref["dEdC"]) < 1e-9
    assert abs(got["E_err"] - ref["E_err"]) < 1e-8 * ref["E_err"]


@pytest.mark.parametrize("force_group", [False, True])
def test_lowering_k_between_calls_follows_the_oracle(sys0, force_group):
    """k = 26 for one sweep (10 moves since the re-inversion), then k = 7: both the library and the
    oracle re-invert before the first move of the second call."""
    W = 48
    pos = S.initial_walkers(sys0, W, seed=14)
    o = oracle.Oracle(sys0)
    st = o.new_state(pos, key=(5222, 15))
    o.sample(st, 1, refresh_k=26)
    o.sample(st, 2, refresh_k=7)
    wk = vmcf.Walkers(vmcf.System(sys0, vmcf.FP64, force_group=force_group), pos, key=(5222, 15), nblocks=4)
    wk.sample(1, 0.3, 26)
    wk.sample(2, 0.3, 7)
    ok = st["margin"] >= 1e-9
    assert ok.sum() >= W - 1
    assert np.abs(wk.positions()[ok] - st["pos"][ok]).max() < 1e-9


def test_batch_lowering_k_between_calls_follows_the_single_path(sys0):
    systems = [vmcf.System(sys0, vmcf.FP64, force_group=True) for _ in range(2)]
    pos = [S.initial_walkers(sys0, 32, seed=30 + g) for g in range(2)]
    wa = [vmcf.Walkers(systems[g], pos[g], key=(5222, 40 + g), nblocks=4) for g in range(2)]
    wb = [vmcf.Walkers(systems[g], pos[g], key=(5222, 40 + g), nblocks=4) for g in range(2)]
    batch = vmcf.Batch(systems, wa)
    batch.sample(1, 0.3, 26)
    batch.sample(2, 0.3, 7)
    for w in wb:
        w.sample(1, 0.3, 26)
        w.sample(2, 0.3, 7)
    for g in range(2):
        np.testing.assert_array_equal(wa[g].positions(), wb[g].positions())


@pytest.mark.parametrize("cfg,precision", [(0, vmcf.FP64), (0, vmcf.MIXED), (4, vmcf.MIXED)])
def test_group_proposal_pass_changes_no_chain(cfg, precision):
    """Walker-group sweeps with their proposals formed ahead by the proposal pass (the default) and drawn inside
    the move kernel: the same chains bit for bit (the same draws, orbital rows and Jastrow changes), across
    re-inversions inside a sweep (k = 7) and measured sweeps, and the same walker sums to rounding."""
    sx = S.make_system(cfg)
    W = 48 if cfg == 0 else 8
    pos = S.initial_walkers(sx, W, seed=31)
    runs = []
    for prepass in (1, 0):
        g = vmcf.System(sx, precision, force_group=True)
        g.set_tuning("group_proposal_pass", prepass)
        if precision == vmcf.MIXED:  # the FP32 SIMT rows (the tensor-core rows differ from them by rounding)
            g.set_tuning("tensor_core_rows", 0)
        wk = vmcf.Walkers(g, pos, key=(5222, 77), nblocks=4)
        wk.sample(2, 0.3, 7, measure=False)
        wk.reset_accumulators(-100.0)
        wk.sample(2, 0.3, 7, measure=True)
        runs.append((wk.positions(), wk.block_sums(), wk.counters()))
    (pa, sa, ca), (pb, sb, cb) = runs
    np.testing.assert_array_equal(pa, pb)
    assert ca["accepted"] == cb["accepted"] and ca["refreshes"] == cb["refreshes"]
    assert rel(sa, sb) < (1e-12 if precision == vmcf.FP64 else 1e-5)


@pytest.mark.parametrize("cfg,precision,W,nb", [(0, vmcf.MIXED, 512, 64), (1, vmcf.FP64, 300, 7), (0, vmcf.FP64, 4100, 4097)])
def test_device_estimator_finish_matches_the_host_finish(cfg, precision, W, nb):
    """vmcf_reduce_estimators finishes the estimators and their jackknife errors on the device (up to 4096
    blocks; beyond, on the host): the same values as the host routine vmcf_finish_estimators applied to
    the same block sums, to 1e-12 (the same operations in the same order; only the FMA contraction of the
    two compilers differs). 4097 blocks take the host path."""
    from paper_2511_05222_gb300 import distributed
    sx = S.make_system(cfg)
    g = vmcf.System(sx, precision)
    wk = vmcf.Walkers(g, S.initial_walkers(sx, W, seed=41), key=(5222, 41), nblocks=nb)
    wk.sample(2, measure=False)
    wk.reset_accumulators(-70.0 if cfg == 0 else -150.0)
    wk.sample(2, measure=True)
    got = wk.reduce_estimators()
    ref = distributed.finish_estimators(wk.block_sums(), sx.K, g.M, sx.n_up, sx.n_dn, wk.e_ref)
    assert abs(got["E"] - ref["E"]) <= 1e-12 * abs(ref["E"])
    assert abs(got["E_err"] - ref["E_err"]) <= 1e-12 * ref["E_err"]
    for k in ("F", "F_err", "dEdC", "dEdC_err"):
        a, b = np.ravel(got[k]), np.ravel(ref[k])
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), k


@pytest.mark.parametrize("precision", [vmcf.FP64, vmcf.MIXED])
@pytest.mark.parametrize("force_group", [False, True])
def test_refresh_residual(precision, force_group):
    """vmcf_refresh_residual: exactly 0 right after a re-inversion (the walker set's creation runs the
    same kernel on the same positions), and after a sweep of Sherman-Morrison updates without one
    (k = 1000 > the 10 moves) of the order of the working precision: FP64 below 1e-8; mixed above 0,
    on average below 1e-3. The call leaves the walker set unchanged: its chain continues as that of
    a walker set that never made it."""
    sx = S.make_system(0)
    pos = S.initial_walkers(sx, 64, seed=51)
    g = vmcf.System(sx, precision, force_group=force_group)
    wk = vmcf.Walkers(g, pos, key=(5222, 51), nblocks=4)
    r0 = wk.refresh_residual()
    assert r0["max"] == 0.0 and r0["mean"] == 0.0
    wk.sample(1, 0.3, 1000, measure=False)
    r1 = wk.refresh_residual()
    assert r1["mean"] <= r1["max"]
    if precision == vmcf.FP64:
        assert r1["max"] < 1e-8, r1
    else:
        assert r1["max"] > 0.0 and r1["mean"] < 1e-3, r1
    wk.sample(2, 0.3, 1000, measure=False)
    wk2 = vmcf.Walkers(vmcf.System(sx, precision, force_group=force_group), pos, key=(5222, 51), nblocks=4)
    wk2.sample(3, 0.3, 1000, measure=False)
    np.testing.assert_array_equal(wk.positions(), wk2.positions())
