"""vmcf_system_set_geometry: a system moved to new nuclear positions and orbital coefficients evaluates,
samples and reduces exactly as a system built at them (App. "Wavefunction Ansatz": the same basis, charges and
Jastrow factor at another geometry), on both kernel families; invalid geometries are refused and leave the
system as it was; walker sets and batches pick the change up."""
import copy

import numpy as np
import pytest

from paper_2511_05222_gb300 import systems as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_05222_gb300 import vmcf  # noqa: E402

OUT = ("EL", "logpsi", "dlnpsi_dR", "dEL_dR", "O")


def moved(sx, seed=4, dR=0.05, dC=0.02):
    """The same molecule with nuclei displaced by up to dR bohr and the orbital coefficients perturbed."""
    rng = np.random.default_rng(seed)
    out = copy.copy(sx)
    out.R = sx.R + rng.uniform(-dR, dR, sx.R.shape)
    out.C_up = sx.C_up + dC * rng.standard_normal(sx.C_up.shape)
    out.C_dn = sx.C_dn + dC * rng.standard_normal(sx.C_dn.shape)
    out.S = None  # the overlap belongs to the old geometry
    return out


def evaluate(g, pos):
    out = vmcf.vmcf_evaluate(g, torch.as_tensor(pos, device="cuda"), want=OUT)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("precision,group", [(vmcf.FP64, False), (vmcf.FP64, True), (vmcf.MIXED, False)])
def test_moved_system_evaluates_as_a_new_one(precision, group):
    sx0 = S.make_system(1)
    sx1 = moved(sx0)
    pos = S.initial_walkers(sx1, 37, seed=2)
    a = vmcf.System(sx0, precision, force_group=group)
    a.set_geometry(sx1.R, sx1.C_up, sx1.C_dn)
    got = evaluate(a, pos)
    ref = evaluate(vmcf.System(sx1, precision, force_group=group), pos)
    for k in OUT:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)


def test_invalid_geometry_is_refused_and_changes_nothing():
    sx0 = S.make_system(0)
    pos = S.initial_walkers(sx0, 9, seed=3)
    g = vmcf.System(sx0, vmcf.FP64)
    before = evaluate(g, pos)
    R = sx0.R.copy()
    R[1] = R[0]  # two nuclei at one position
    with pytest.raises(vmcf.VmcfError):
        g.set_geometry(R, sx0.C_up, sx0.C_dn)
    with pytest.raises(vmcf.VmcfError):
        g.set_geometry(sx0.R, sx0.C_up * np.nan, sx0.C_dn)
    C = sx0.C_up.copy()
    C[:, 1] = C[:, 0]  # dependent columns
    with pytest.raises(vmcf.VmcfError):
        g.set_geometry(sx0.R, C, sx0.C_dn)
    after = evaluate(g, pos)
    for k in OUT:
        np.testing.assert_array_equal(after[k], before[k], err_msg=k)


@pytest.mark.parametrize("precision", [vmcf.FP64, vmcf.MIXED])
def test_walkers_follow_the_moved_system(precision):
    """Walkers re-inverted after the move sample the same chains (bit for bit) and sums (FP64 1e-12, mixed 1e-5)
    as walkers of a new system."""
    sx0 = S.make_system(0)
    sx1 = moved(sx0, seed=6)
    pos = S.initial_walkers(sx1, 64, seed=7)
    a = vmcf.System(sx0, precision)
    wa = vmcf.Walkers(a, S.initial_walkers(sx0, 64, seed=8), key=(5222, 3), nblocks=4)
    wa.sample(2, measure=False)
    a.set_geometry(sx1.R, sx1.C_up, sx1.C_dn)
    wa.set_positions(pos)
    b = vmcf.System(sx1, precision)
    wb = vmcf.Walkers(b, pos, key=(5222, 3), nblocks=4)
    # the same chain clocks: both walker sets start the comparison at sweep 2 with fresh inverses
    wb.sample(2, measure=False)
    wb.set_positions(pos)
    for w in (wa, wb):
        w.reset_accumulators(-76.0)
        w.sample(3, measure=True)
    np.testing.assert_array_equal(wa.positions(), wb.positions())
    # sums to the rounding of the CTAs' shared-memory accumulation order (as between a batch and the single path)
    a, b = wa.block_sums(), wb.block_sums()
    tol = 1e-12 if precision == vmcf.FP64 else 1e-5
    assert np.abs(a - b).max() / np.abs(b).max() < tol


def test_batch_notices_the_move():
    """A ragged batch built before the move samples as the single path after it (bit for bit)."""
    specs = [(S.make_system(0), 32), (S.make_system(1), 16)]
    moved0 = moved(specs[0][0], seed=9)
    systems = [vmcf.System(sx, vmcf.MIXED) for sx, _ in specs]
    wa = [vmcf.Walkers(g, S.initial_walkers(sx, W, seed=40 + i), key=(5222, 500 + i), nblocks=4)
          for i, (g, (sx, W)) in enumerate(zip(systems, specs))]
    batch = vmcf.Batch(systems, wa)
    batch.sample(1, measure=False)
    systems[0].set_geometry(moved0.R, moved0.C_up, moved0.C_dn)
    pos = wa[0].positions()
    wa[0].set_positions(pos)
    # the single path at the new geometry, on the same chain clock (one sweep done, fresh inverses)
    ws = vmcf.Walkers(vmcf.System(moved0, vmcf.MIXED), pos, key=(5222, 500), nblocks=4)
    ws.sample(1, measure=False)
    ws.set_positions(pos)
    batch.sample(2, measure=False)
    ws.sample(2, measure=False)
    np.testing.assert_array_equal(wa[0].positions(), ws.positions())
