"""Stored oracle values of the water workload (tests/golden/water_oracle.txt, written by
tests/golden/make_golden.py from the oracle alone).

CPU: the seeded generator still gives the stored walker positions, and the oracle still gives
the stored values (a change to either shows here and needs the stored file rewritten with the
passage that justifies it). GPU: the FP64 CUDA path, through the C ABI, against the stored
values: evaluation in both kernel families within 1e-10 (normwise per tensor), the chain's
positions within 1e-9 with the same accepted-move counts, and the measured estimators of the
64 stored configurations."""
import importlib.util
from pathlib import Path

import numpy as np
import pytest

from paper_2511_05222_gb300 import systems as S

_spec = importlib.util.spec_from_file_location("make_golden", Path(__file__).parent / "golden" / "make_golden.py")
golden = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(golden)

EVAL_KEYS = ("EL", "logpsi", "dlnpsi_dR", "dEL_dR", "O")


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def stored():
    return golden.read()


def test_generator_gives_the_stored_positions(stored):
    _, pos, _ = golden.water_inputs()
    np.testing.assert_array_equal(pos, stored["pos"])


def test_oracle_reproduces_the_stored_values(stored):
    now = golden.compute()
    assert set(now) == set(stored)
    np.testing.assert_array_equal(now["chain_nacc"], stored["chain_nacc"])
    for k in stored:
        # libm may differ by an ulp between hosts; everything else is fixed
        assert rel(now[k], stored[k]) < 1e-12, (k, rel(now[k], stored[k]))


@pytest.mark.gpu
@pytest.mark.parametrize("force_group", [False, True])
def test_fp64_cuda_path_matches_the_stored_values(stored, force_group):
    torch = pytest.importorskip("torch")
    from paper_2511_05222_gb300 import vmcf

    sysx, _, pos64 = golden.water_inputs()
    g = vmcf.System(sysx, vmcf.FP64, force_group=force_group)
    dev = torch.as_tensor(np.ascontiguousarray(stored["pos"]), dtype=torch.float64, device="cuda")
    out = vmcf.vmcf_evaluate(g, dev, want=EVAL_KEYS)
    torch.cuda.synchronize()
    for k in EVAL_KEYS:
        got = out[k].cpu().numpy().reshape(stored[k].shape)
        assert rel(got, stored[k]) < 1e-10, (k, rel(got, stored[k]))

    wk = vmcf.Walkers(g, stored["pos"], key=golden.CHAIN_KEY, nblocks=3)
    wk.sample(3, 0.3, 26, measure=False)
    assert np.abs(wk.positions() - stored["chain_pos"]).max() < 1e-9
    assert wk.counters()["accepted"] == int(stored["chain_nacc"].sum())

    est = vmcf.Walkers(g, pos64, nblocks=8)
    est.reset_accumulators(golden.E_REF)
    est.measure()
    got = est.reduce_estimators()
    assert abs(got["E"] - stored["est_E"]) < 1e-10 * abs(stored["est_E"])
    assert abs(got["E_err"] - stored["est_E_err"]) < 1e-8 * stored["est_E_err"]
    assert rel(got["F"].ravel(), stored["est_F"]) < 1e-9
    assert rel(got["F_err"].ravel(), stored["est_F_err"]) < 1e-7
    assert rel(got["dEdC"], stored["est_dEdC"]) < 1e-9


@pytest.mark.gpu
def test_mixed_local_energy_matches_the_stored_values(stored):
    """Mixed precision: every walker's E_L within 1e-5 relative of the stored FP64 value."""
    torch = pytest.importorskip("torch")
    from paper_2511_05222_gb300 import vmcf

    sysx, _, _ = golden.water_inputs()
    g = vmcf.System(sysx, vmcf.MIXED)
    dev = torch.as_tensor(np.ascontiguousarray(stored["pos"]), dtype=torch.float64, device="cuda")
    got = vmcf.vmcf_evaluate(g, dev, want=("EL",))["EL"].cpu().numpy()
    assert (np.abs(got - stored["EL"]) / np.abs(stored["EL"])).max() < 1e-5
