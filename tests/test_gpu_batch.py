"""Ragged batches of geometries (vmcf_batch_*): every sweep of several molecules of different
sizes is one replay of a captured graph of persistent kernels (walker-group kernels) and, for the
geometries that fit them, branches of the small-system kernels. Batching must not change any
walker's chain or contribution: positions follow the single-geometry path and the oracle's
Markov chain, and the per-geometry walker sums give the same estimators."""
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


@pytest.fixture(scope="module")
def ragged():
    """Water plus the first three covalent-walk molecules of the ragged-batch generator: 10,
    38, 76 and 42 electrons, 24 to 174 AOs; the 76-electron one runs with 128 threads per
    walker."""
    rb = S.make_ragged_batch(3)
    return [(S.make_system(0), 96)] + [(s, W) for s, W in rb]


def _walkers(systems, specs, seed0, nb=4):
    out = []
    for g, (sx, W) in enumerate(specs):
        pos = S.initial_walkers(sx, W, seed=seed0 + g)
        out.append(vmcf.Walkers(systems[g], pos, key=(5222, 300 + g), nblocks=nb))
    return out


@pytest.mark.parametrize("precision", [vmcf.FP64, vmcf.MIXED])
def test_batch_follows_the_single_geometry_path(ragged, precision):
    """Same chains and sums as vmcf_sample on each walker set alone (positions bit for bit;
    walker sums to rounding: FP64 1e-12; mixed 1e-5; in mixed precision both form the O sums on
    the tensor cores)."""
    specs = [(sx, W) for (sx, _), W in zip(ragged, (64, 40, 56, 24))]
    systems = [vmcf.System(sx, precision, force_group=True) for sx, _ in specs]
    wa = _walkers(systems, specs, 20)
    wb = _walkers(systems, specs, 20)
    batch = vmcf.Batch(systems, wa)
    info = batch.info()
    assert info["buckets"] == 3 and info["launches"] >= 4  # the 38- and 42-electron molecules share one
    assert info["geometries"][2]["sweep"] == (128, 1) and info["geometries"][2]["evaluation"] == (256, 1)
    e_ref = [-76.0, -150.0, -160.0, -300.0]
    batch.sample(3, measure=False)
    for g, w in enumerate(wa):
        w.reset_accumulators(e_ref[g])
        wb[g].sample(3, measure=False)
        wb[g].reset_accumulators(e_ref[g])
    batch.sample(2, measure=True)
    batch.sample(1, measure=True)  # a second call replays the same graph from the uploaded clocks
    for w in wb:
        w.sample(3, measure=True)
    tol = 1e-12 if precision == vmcf.FP64 else 1e-5
    for g in range(len(specs)):
        np.testing.assert_array_equal(wa[g].positions(), wb[g].positions())
        ca, cb = wa[g].counters(), wb[g].counters()
        assert ca["accepted"] == cb["accepted"] and ca["moves"] == cb["moves"]
        sa, sb = wa[g].block_sums(), wb[g].block_sums()
        np.testing.assert_array_equal(sa[:, 0], sb[:, 0])
        assert rel(sa, sb) < tol, (g, rel(sa, sb))
        ea, eb = wa[g].reduce_estimators(), wb[g].reduce_estimators()
        assert abs(ea["E"] - eb["E"]) <= tol * abs(eb["E"])
        assert np.all(np.abs(ea["F"] - eb["F"]) <= 0.01 * eb["F_err"] + 1e-12)


@pytest.mark.parametrize("small", [False, True])
def test_batch_estimators_match_the_oracle(ragged, small):
    """Three geometries of different sizes in one ragged FP64 batch (water, 10 electrons, on the
    walker-group kernels or (small) on the small-system kernels in a branch of the batch graph; a
    38- and a 76-electron molecule on walker-group kernels of 32 and 128 threads per walker): every
    geometry's chain and estimators as the oracle's."""
    specs = [(ragged[0][0], 128), (ragged[1][0], 32), (ragged[2][0], 16)]
    nbs, keys, e_refs = (8, 4, 4), [(5222, 0), (5222, 10), (5222, 11)], (-76.0, -150.0, -300.0)
    warm, meas = 3, 3
    systems = [vmcf.System(sx, vmcf.FP64, force_group=not (small and g == 0)) for g, (sx, _) in enumerate(specs)]
    pos = [S.initial_walkers(sx, W, seed=10 + g) for g, (sx, W) in enumerate(specs)]
    wk = [vmcf.Walkers(systems[g], pos[g], key=keys[g], nblocks=nbs[g]) for g in range(3)]
    batch = vmcf.Batch(systems, wk)
    batch.sample(warm, measure=False)
    for g, w in enumerate(wk):
        w.reset_accumulators(e_refs[g])
    batch.sample(meas, measure=True)
    for g, (sx, W) in enumerate(specs):
        o = oracle.Oracle(sx)
        st = o.new_state(pos[g], key=keys[g])
        o.sample(st, warm)
        nb = nbs[g]
        sums = estimators.new_sums(nb, sx.K, o.nO)
        blk = np.zeros(W, dtype=np.int64)
        for b in range(nb):
            blk[(W * b) // nb:(W * (b + 1)) // nb] = b
        for _ in range(meas):
            o.sample(st, 1)
            o.force_refresh(st)
            out = o.eval(st["pos"], want=("EL", "dlnpsi_dR", "dEL_dR", "O"))
            estimators.accumulate(sums, blk, out["EL"], out["dlnpsi_dR"], out["dEL_dR"], out["O"], e_refs[g])
        assert st["margin"].min() >= 1e-9, g  # every decision clear of a tie: the chains are the same
        assert np.abs(wk[g].positions() - st["pos"]).max() < 1e-9, g
        ref = estimators.finish(sums, e_refs[g])
        got = wk[g].reduce_estimators()
        assert abs(got["E"] - ref["E"]) < 1e-10 * abs(ref["E"]), g
        assert rel(got["F"].ravel(), ref["F"]) < 1e-9, g
        assert rel(got["dEdC"], ref["dEdC"]) < 1e-9, g
        assert abs(got["E_err"] - ref["E_err"]) < 1e-8 * ref["E_err"], g
    if small:
        assert batch.info()["geometries"][0]["bucket"] == -1


@pytest.mark.parametrize("kref", [26, 7])
@pytest.mark.parametrize("precision", [vmcf.FP64, vmcf.MIXED])
def test_small_path_geometries_in_a_batch_follow_the_single_path(ragged, precision, kref):
    """Water and C2OH6 on the small-system kernels (one graph branch each: proposals, runs of moves
    with the re-inversions every k moves read from the device chain clock, the measurement) beside
    two walker-group geometries: every chain bit for bit as vmcf_sample on the walker set alone, the
    walker sums to rounding. k = 7 puts re-inversions inside sweeps at positions that change from
    sweep to sweep."""
    specs = [(ragged[0][0], 64), (S.make_system(1), 48), (ragged[1][0], 40), (ragged[3][0], 24)]
    systems = [vmcf.System(sx, precision, force_group=g >= 2) for g, (sx, _) in enumerate(specs)]
    wa = _walkers(systems, specs, 60)
    wb = _walkers(systems, specs, 60)
    batch = vmcf.Batch(systems, wa)
    info = batch.info()
    assert [geo["bucket"] for geo in info["geometries"]][:2] == [-1, -1]
    e_ref = [-76.0, -150.0, -150.0, -300.0]
    batch.sample(3, 0.3, kref, measure=False)
    for g, w in enumerate(wb):
        w.sample(3, 0.3, kref, measure=False)
        w.reset_accumulators(e_ref[g])
        wa[g].reset_accumulators(e_ref[g])
    batch.sample(2, 0.3, kref, measure=True)
    batch.sample(1, 0.3, kref, measure=False)
    batch.sample(1, 0.3, kref, measure=True)
    for w in wb:
        w.sample(2, 0.3, kref, measure=True)
        w.sample(1, 0.3, kref, measure=False)
        w.sample(1, 0.3, kref, measure=True)
    tol = 1e-12 if precision == vmcf.FP64 else 1e-5
    for g in range(len(specs)):
        np.testing.assert_array_equal(wa[g].positions(), wb[g].positions())
        ca, cb = wa[g].counters(), wb[g].counters()
        assert ca["accepted"] == cb["accepted"] and ca["moves"] == cb["moves"]
        assert ca["refreshes"] == cb["refreshes"] and ca["sweeps"] == cb["sweeps"]
        sa, sb = wa[g].block_sums(), wb[g].block_sums()
        np.testing.assert_array_equal(sa[:, 0], sb[:, 0])
        assert rel(sa, sb) < tol, (g, rel(sa, sb))


def test_launch_shape_and_autotuning_leave_the_chains_unchanged(ragged):
    """Two batches over identical walker sets: one autotuned, one with every bucket forced to
    one walker group per CTA (128 threads for sweeps, 256 for evaluations). Autotuning runs the
    same number of sweeps whatever it picks, and no shape changes a chain beyond FP64 rounding."""
    specs = [(sx, W) for (sx, _), W in zip(ragged, (64, 40, 48, 24))]
    systems = [vmcf.System(sx, vmcf.FP64, force_group=True) for sx, _ in specs]
    wa = _walkers(systems, specs, 40)
    wb = _walkers(systems, specs, 40)
    ba = vmcf.Batch(systems, wa)
    bb = vmcf.Batch(systems, wb)
    ba.autotune()
    bb.autotune()
    for g in range(len(specs)):
        bb.set_shape(g, 0, 128, 1)
        bb.set_shape(g, 1, 256, 1)
    info = ba.info()
    for geo in info["geometries"]:
        for ph in ("sweep", "evaluation"):
            assert geo[ph] in ((32, 1), (32, 2), (32, 4), (32, 8), (128, 1), (128, 2), (256, 1))
    for w in wa + wb:
        w.reset_accumulators(-100.0)
    ba.sample(2, measure=True)
    bb.sample(2, measure=True)
    for g in range(len(specs)):
        assert np.abs(wa[g].positions() - wb[g].positions()).max() < 1e-12
        assert wa[g].counters()["accepted"] == wb[g].counters()["accepted"]
        assert rel(wa[g].block_sums(), wb[g].block_sums()) < 1e-11


def test_batch_rejects_mixed_precisions(ragged):
    a = vmcf.System(ragged[0][0], vmcf.FP64, force_group=True)
    b = vmcf.System(ragged[1][0], vmcf.MIXED, force_group=True)
    wa = vmcf.Walkers(a, S.initial_walkers(ragged[0][0], 16, seed=1), nblocks=2)
    wb = vmcf.Walkers(b, S.initial_walkers(ragged[1][0], 16, seed=1), nblocks=2)
    with pytest.raises(vmcf.VmcfError):
        vmcf.Batch([a, b], [wa, wb])
