"""Host-side rejection of bad determinant inputs at vmcf_init_system (no GPU needed: every case is
refused before the first CUDA call): linearly dependent orbital columns, two nuclei at the same
position, invalid shells, non-finite coefficients, bad spin counts."""
import copy

import numpy as np
import pytest

from paper_2511_05222_gb300 import systems as S
from paper_2511_05222_gb300 import vmcf

EINVAL = -1


@pytest.fixture(scope="module")
def water():
    return S.make_system(0)


def _expect(sysx, text, precision=vmcf.FP64):
    with pytest.raises(vmcf.VmcfError) as ei:
        vmcf.System(sysx, precision)
    assert ei.value.code == EINVAL, str(ei.value)
    assert text in str(ei.value), str(ei.value)


def test_dependent_orbital_columns_are_rejected(water):
    sx = copy.copy(water)
    C = water.C_up.copy()
    C[:, 4] = 0.5 * C[:, 0] - 2.0 * C[:, 2]
    sx.C_up = C
    _expect(sx, "linearly dependent")
    sx = copy.copy(water)
    C = water.C_dn.copy()
    C[:, 1] = C[:, 3]
    sx.C_dn = C
    _expect(sx, "C_dn")


def test_coincident_nuclei_are_rejected(water):
    sx = copy.copy(water)
    R = water.R.copy()
    R[2] = R[1]
    sx.R = R
    _expect(sx, "same position")


@pytest.mark.parametrize("field,value", [("shell_l", 3), ("shell_center", 5), ("shell_exp", -0.5)])
def test_bad_determinant_shells_are_rejected(water, field, value):
    sx = copy.copy(water)
    arr = getattr(water, field).copy()
    if field == "shell_exp":
        arr[2, 1] = value
    else:
        arr[2] = value
    setattr(sx, field, arr)
    with pytest.raises(vmcf.VmcfError) as ei:
        vmcf.System(sx, vmcf.FP64)
    assert ei.value.code == EINVAL


def test_non_finite_orbital_coefficients_are_rejected(water):
    sx = copy.copy(water)
    C = water.C_up.copy()
    C[3, 2] = np.nan
    sx.C_up = C
    _expect(sx, "not finite")


def test_independent_columns_pass(water):
    """The check accepts orbitals far from orthonormal (scaled, mixed columns)."""
    sx = copy.copy(water)
    G = np.random.default_rng(0).normal(size=(water.n_up, water.n_up)) + 3 * np.eye(water.n_up)
    sx.C_up = water.C_up @ G * 1e-3
    # passes validation; only the GPU step can fail on a machine without one
    try:
        vmcf.System(sx, vmcf.FP64)
    except vmcf.VmcfError as e:
        assert e.code != EINVAL, str(e)
