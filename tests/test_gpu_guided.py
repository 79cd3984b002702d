"""Reweighted (guided) sampling on the GPU against the oracle: chains of |Psi_G|^2 (Psi_G = Psi
max(1, eps sqrt(S))) follow the oracle's in FP64 on both kernel families, the weighted estimators
match the oracle's, and mixed precision stays within a tenth of the FP64 error bars."""
import math

import numpy as np
import pytest

import oracle
from oracle import estimators
from paper_2511_05222_gb300 import systems as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_05222_gb300 import vmcf  # noqa: E402


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def guide_eps(o, pos, q=0.8):
    """eps putting the guide's threshold at the q-quantile of S over the given walkers."""
    B = o.refresh(pos)
    return 1.0 / math.sqrt(np.quantile((B ** 2).sum(1), q))


@pytest.mark.parametrize("force_group", [False, True])
def test_guided_fp64_chain_and_estimators_match_the_oracle(force_group):
    sys0 = S.make_system(0)
    W, nb, warm, meas, e_ref = 128, 8, 4, 3, -76.0
    pos = S.initial_walkers(sys0, W, seed=41)
    o = oracle.Oracle(sys0)
    st = o.new_state(pos, key=(5222, 0))
    o.sample(st, 10)
    pos = st["pos"].copy()
    eps = guide_eps(o, pos)
    st = o.new_state(pos, key=(5222, 0))
    o.sample(st, warm, eps=eps)
    g = vmcf.System(sys0, vmcf.FP64, force_group=force_group)
    wk = vmcf.Walkers(g, pos, key=(5222, 0), nblocks=nb)
    wk.set_guiding(eps)
    wk.sample(warm, measure=False)
    wk.reset_accumulators(e_ref)
    wk.sample(meas, measure=True)
    sums = estimators.new_sums(nb, sys0.K, o.nO)
    blk = np.arange(W) * nb // W
    for _ in range(meas):
        o.sample(st, 1, eps=eps)
        o.force_refresh(st)
        out = o.eval(st["pos"], want=("EL", "dlnpsi_dR", "dEL_dR", "O"))
        estimators.accumulate(sums, blk, out["EL"], out["dlnpsi_dR"], out["dEL_dR"], out["O"], e_ref,
                              weight=o.guide_weight(st["pos"], eps))
    ok = st["margin"] >= 1e-9
    assert ok.all(), int((~ok).sum())
    assert np.abs(wk.positions() - st["pos"]).max() < 1e-9
    assert wk.counters()["accepted"] == int(st["nacc"].sum())
    ref = estimators.finish(sums, e_ref)
    got = wk.reduce_estimators()
    np.testing.assert_allclose(wk.block_sums()[:, 0], sums["n"], rtol=1e-12)
    assert abs(got["E"] - ref["E"]) < 1e-10 * abs(ref["E"])
    assert rel(got["F"].ravel(), ref["F"]) < 1e-9
    assert rel(got["dEdC"], ref["dEdC"]) < 1e-9
    assert abs(got["E_err"] - ref["E_err"]) < 1e-8 * ref["E_err"]


@pytest.mark.parametrize("cfg", [0, 1])
def test_guided_mixed_estimators_within_a_tenth_of_their_error_bars(cfg):
    sysx = S.make_system(cfg)
    W = 4096
    pos = S.initial_walkers(sysx, W, seed=42)
    gm = vmcf.System(sysx, vmcf.MIXED)
    g64 = vmcf.System(sysx, vmcf.FP64)
    wm = vmcf.Walkers(gm, pos, key=(5222, cfg), nblocks=32)
    wm.sample(20, measure=False)
    eps = guide_eps(oracle.Oracle(sysx), wm.positions()[:512])
    wm.set_guiding(eps)
    wm.sample(10, measure=False)
    w64 = vmcf.Walkers(g64, wm.positions(), key=(5222, cfg), nblocks=32)
    w64.set_guiding(eps)
    e_ref = {0: -76.0, 1: -150.0}[cfg]
    wm.reset_accumulators(e_ref)
    w64.reset_accumulators(e_ref)
    for _ in range(6):
        wm.sample(1, measure=True)
        w64.set_positions(wm.positions())
        w64.measure()
    em, e64 = wm.reduce_estimators(), w64.reduce_estimators()
    assert abs(em["E"] - e64["E"]) <= 0.1 * e64["E_err"]
    dF = np.abs(em["F"] - e64["F"]) / e64["F_err"]
    assert dF.max() <= 0.1, dF.max()
    ok = e64["dEdC_err"] > 0
    dB = np.abs(em["dEdC"] - e64["dEdC"])[ok] / e64["dEdC_err"][ok]
    assert dB.max() <= 0.1, dB.max()
    n = wm.block_sums()[:, 0].sum()
    assert n < 6 * W  # the sample count is the sum of the weights, below one per sample
