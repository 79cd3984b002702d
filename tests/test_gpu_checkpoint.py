"""Checkpoint and resume of walker sets through the C ABI (vmcf_walkers_save / vmcf_walkers_load):
a walker set that loads a checkpoint taken in the middle of a run (between a re-inversion and the
next, with sums accumulated) continues every chain bit for bit and its sums to rounding, in both
precisions and both kernel families; a checkpoint of another walker count is refused."""
import numpy as np
import pytest

from paper_2511_05222_gb300 import systems as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_05222_gb300 import vmcf  # noqa: E402


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("force_group", [False, True])
@pytest.mark.parametrize("precision", [vmcf.FP64, vmcf.MIXED])
def test_resume_continues_the_chains_and_sums(sys0, precision, force_group):
    W, nb, e_ref = 64, 4, -76.0
    g = vmcf.System(sys0, precision, force_group=force_group)
    a = vmcf.Walkers(g, S.initial_walkers(sys0, W, seed=20), key=(5222, 21), nblocks=nb)
    a.sample(3, 0.3, 7)  # k = 7: the checkpoint falls between re-inversions
    a.reset_accumulators(e_ref)
    a.sample(2, 0.3, 7, measure=True)
    a.sample(1, 0.3, 7)
    state = a.save()
    h = vmcf.WalkersState.from_buffer_copy(state[:vmcf.ctypes.sizeof(vmcf.WalkersState)])
    assert (h.W, h.nblocks, h.sweep, h.measured, h.e_ref) == (W, nb, 6, 2, e_ref)
    assert h.counter == sys0.Ne % 7  # one unmeasured sweep since the measurement's fresh inverses
    a.sample(2, 0.3, 7, measure=True)
    a.sample(1, 0.3, 7)

    b = vmcf.Walkers(g, S.initial_walkers(sys0, W, seed=99), key=(1, 1), nblocks=nb)
    b.load(state)
    assert b.e_ref == e_ref
    b.sample(2, 0.3, 7, measure=True)
    b.sample(1, 0.3, 7)

    np.testing.assert_array_equal(b.positions(), a.positions())
    assert b.counters() == a.counters()
    assert rel(b.block_sums(), a.block_sums()) < (1e-12 if precision == vmcf.FP64 else 1e-5)
    ea, eb = a.reduce_estimators(), b.reduce_estimators()
    assert abs(ea["E"] - eb["E"]) <= (1e-12 if precision == vmcf.FP64 else 1e-6) * abs(ea["E"])


def test_a_checkpoint_of_another_walker_set_is_refused(sys0):
    g = vmcf.System(sys0, vmcf.MIXED)
    a = vmcf.Walkers(g, S.initial_walkers(sys0, 32, seed=1), nblocks=4)
    b = vmcf.Walkers(g, S.initial_walkers(sys0, 48, seed=1), nblocks=4)
    pos_b = b.positions()
    with pytest.raises(vmcf.VmcfError) as ei:
        b.load(a.save())
    assert ei.value.code == -1
    np.testing.assert_array_equal(b.positions(), pos_b)  # nothing changed
    with pytest.raises(vmcf.VmcfError):
        b.load(b.save()[:100])  # truncated
