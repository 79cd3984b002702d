"""Host-side checks of the AO-expanded Jastrow input at vmcf_init_system (no GPU needed: every case
here is rejected before the first CUDA call): Xi must be symmetric, the coefficients finite, the
Jastrow-basis shells valid, at most 1024 Jastrow-basis functions, and the work space must fit the
shared-memory plan."""
import numpy as np
import pytest

from paper_2511_05222_gb300 import systems as S
from paper_2511_05222_gb300 import vmcf

EINVAL, ENOTSUP = -1, -6


def _replace(jb, **kw):
    f = dict(shell_center=jb.shell_center, shell_l=jb.shell_l, shell_nprim=jb.shell_nprim, shell_exp=jb.shell_exp,
             shell_coef=jb.shell_coef, xi=jb.xi, Xi=jb.Xi)
    f.update(kw)
    return S.JastrowBasis(**f)


@pytest.fixture(scope="module")
def water():
    return S.make_system(0)


def _expect(sysx, code, text, precision=vmcf.FP64):
    with pytest.raises(vmcf.VmcfError) as ei:
        vmcf.System(sysx, precision)
    assert ei.value.code == code, str(ei.value)
    assert text in str(ei.value), str(ei.value)


def test_asymmetric_pair_coefficients_are_rejected(water):
    jb = S.jastrow_basis(water, 1)
    Xi = jb.Xi.copy()
    Xi[0, 1] += 1e-6
    _expect(S.with_jastrow_basis(water, _replace(jb, Xi=Xi)), EINVAL, "symmetric")


def test_non_finite_coefficients_are_rejected(water):
    jb = S.jastrow_basis(water, 1)
    xi = jb.xi.copy()
    xi[3] = np.inf
    _expect(S.with_jastrow_basis(water, _replace(jb, xi=xi)), EINVAL, "not finite")
    Xi = jb.Xi.copy()
    Xi[2, 2] = np.nan
    _expect(S.with_jastrow_basis(water, _replace(jb, Xi=Xi)), EINVAL, "not finite")


@pytest.mark.parametrize("field,value", [("shell_l", 3), ("shell_center", 7), ("shell_exp", -1.0)])
def test_bad_jastrow_shells_are_rejected(water, field, value):
    jb = S.jastrow_basis(water, 1)
    arr = getattr(jb, field).copy()
    if field == "shell_exp":
        arr[0, 0] = value
    else:
        arr[0] = value
    _expect(S.with_jastrow_basis(water, _replace(jb, **{field: arr})), EINVAL, "Jastrow basis")


def _big_basis(sysx, nshell_d):
    """nshell_d uncontracted d shells on nucleus 0 (5 functions each)."""
    ns = nshell_d
    ex = np.zeros((ns, S.MAXPRIM))
    co = np.zeros((ns, S.MAXPRIM))
    ex[:, 0] = np.geomspace(0.2, 2.0, ns)
    co[:, 0] = 1.0
    MJ = 5 * ns
    return S.JastrowBasis(np.zeros(ns, np.int32), np.full(ns, 2, np.int32), np.ones(ns, np.int32), ex, co,
                          np.zeros(MJ), np.zeros((MJ, MJ)))


def test_more_than_1024_jastrow_functions_are_not_supported(water):
    _expect(S.with_jastrow_basis(water, _big_basis(water, 205)), ENOTSUP, "1024")


def test_a_jastrow_basis_beyond_the_shared_memory_plan_is_not_supported():
    """C9O4H8 in FP64 already uses most of a CTA's shared memory for the evaluation; 700 more
    Jastrow-basis functions do not fit, and the plan says so instead of launching."""
    sys4 = S.make_system(4)
    _expect(S.with_jastrow_basis(sys4, _big_basis(sys4, 140)), ENOTSUP, "shared-memory plan")
