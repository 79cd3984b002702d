"""Space-warp (SWCT) force estimator on the GPU against the oracle: per-walker electron
derivatives of E_L and warped force vectors (FP64, 1e-10 normwise), estimators from sampling
on both kernel families (FP64 against the oracle's chain), and mixed precision within a tenth
of the error bar of the FP64 path on the same configurations."""
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


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("cfg,W", [(0, 37), (1, 24), (4, 4)])
def test_warp_vectors_fp64(cfg, W):
    sysx = S.make_system(cfg)
    pos = S.initial_walkers(sysx, W, seed=21)
    ref = oracle.Oracle(sysx).eval_warp(pos)
    got = vmcf.vmcf_evaluate_warp(vmcf.System(sysx, vmcf.FP64), dev(pos))
    torch.cuda.synchronize()
    for k in ("dEL_dr", "dEL_sw", "dlnpsi_sw"):
        assert rel(got[k].cpu().numpy(), ref[k]) < 1e-10, (k, rel(got[k].cpu().numpy(), ref[k]))


@pytest.mark.parametrize("force_group", [False, True])
def test_warp_forces_from_sampling_match_the_oracle(force_group):
    sys0 = S.make_system(0)
    W, nb, warm, meas, e_ref = 128, 8, 3, 3, -76.0
    pos = S.initial_walkers(sys0, W, seed=22)
    o = oracle.Oracle(sys0)
    st = o.new_state(pos, key=(5222, 0))
    o.sample(st, warm)
    g = vmcf.System(sys0, vmcf.FP64, force_group=force_group, space_warp=True)
    wk = vmcf.Walkers(g, pos, key=(5222, 0), nblocks=nb)
    wk.sample(warm, measure=False)
    wk.reset_accumulators(e_ref)
    wk.sample(meas, measure=True)
    sums = estimators.new_sums(nb, sys0.K, o.nO)
    plain = estimators.new_sums(nb, sys0.K, o.nO)
    blk = np.arange(W) * nb // W
    for _ in range(meas):
        o.sample(st, 1)
        o.force_refresh(st)
        out = o.eval(st["pos"], want=("EL", "dlnpsi_dR", "dEL_dR", "O"))
        wv = o.eval_warp(st["pos"])
        estimators.accumulate(sums, blk, out["EL"], wv["dlnpsi_sw"], wv["dEL_sw"], out["O"], e_ref)
        estimators.accumulate(plain, blk, out["EL"], out["dlnpsi_dR"], out["dEL_dR"], out["O"], e_ref)
    assert st["margin"].min() >= 1e-9
    assert np.abs(wk.positions() - st["pos"]).max() < 1e-9
    ref, ref_plain = estimators.finish(sums, e_ref), estimators.finish(plain, e_ref)
    got = wk.reduce_warp()
    assert rel(got["F"].ravel(), ref["F"]) < 1e-9
    assert rel(got["F_err"].ravel(), ref["F_err"]) < 1e-7
    est = wk.reduce_estimators()  # the plain estimators are unchanged by the extra sums
    assert rel(est["F"].ravel(), ref_plain["F"]) < 1e-9
    assert abs(est["E"] - ref_plain["E"]) < 1e-10 * abs(ref_plain["E"])


@pytest.mark.parametrize("cfg", [0, 1])
def test_mixed_warp_forces_within_a_tenth_of_their_error_bars(cfg):
    sysx = S.make_system(cfg)
    W = 4096
    pos = S.initial_walkers(sysx, W, seed=23)
    gm = vmcf.System(sysx, vmcf.MIXED, space_warp=True)
    g64 = vmcf.System(sysx, vmcf.FP64, space_warp=True)
    wm = vmcf.Walkers(gm, pos, key=(5222, cfg), nblocks=32)
    wm.sample(20, measure=False)
    w64 = vmcf.Walkers(g64, wm.positions(), key=(5222, cfg), nblocks=32)
    e_ref = {0: -76.0, 1: -150.0}[cfg]
    wm.reset_accumulators(e_ref)
    w64.reset_accumulators(e_ref)
    for _ in range(6):
        wm.sample(1, measure=True)
        w64.set_positions(wm.positions())
        w64.measure()
    fm, f64 = wm.reduce_warp(), w64.reduce_warp()
    d = np.abs(fm["F"] - f64["F"]) / f64["F_err"]
    assert d.max() <= 0.1, d.max()
    # the warp removes most of the variance of the forces near the nuclei
    plain = w64.reduce_estimators()
    assert np.median(f64["F_err"] / plain["F_err"]) < 0.7
