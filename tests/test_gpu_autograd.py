"""VMCForces (torch.autograd.Function over libvmcf) on fixed walkers: the R-gradient equals
central finite differences of the correlated-sampling energy, and the C-gradient plus
<dE_L/dC> equals the same finite differences in C (both exact identities); both agree with
the FP64 oracle's estimators."""
import copy

import numpy as np
import pytest

import oracle
from oracle import estimators
from paper_2511_05222_gb300 import systems as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_05222_gb300 import vmcf  # noqa: E402
from paper_2511_05222_gb300.autograd import vmc_energy  # noqa: E402


def reweighted_energy(sysx, pos_dev, logpsi0):
    out = vmcf.vmcf_evaluate(vmcf.System(sysx, vmcf.FP64), pos_dev, want=("EL", "logpsi"))
    el, lp = out["EL"].cpu().numpy(), out["logpsi"].cpu().numpy()
    w = np.exp(2 * (lp - logpsi0))
    return (w * el).sum() / w.sum()


def rich(f, h):
    return (4 * (f(h / 2) - f(-h / 2)) / h - (f(h) - f(-h)) / (2 * h)) / 3


def test_autograd_forces_and_orbital_gradient(sys1):
    W = 256
    o = oracle.Oracle(sys1)
    st = o.new_state(S.initial_walkers(sys1, W, seed=17), key=(5222, 1))
    o.sample(st, 10)
    pos = torch.as_tensor(st["pos"], device="cuda")
    R = torch.tensor(sys1.R, dtype=torch.float64, requires_grad=True)
    Cu = torch.tensor(sys1.C_up, requires_grad=True)
    Cd = torch.tensor(sys1.C_dn, requires_grad=True)
    E = vmc_energy(R, Cu, Cd, sys1, pos, vmcf.FP64, 16)
    E.backward()
    # oracle estimators on the same walkers (uniform weights)
    ref = o.eval(st["pos"], want=("EL", "dlnpsi_dR", "dEL_dR", "O", "dEL_dC"))
    sums = estimators.new_sums(16, sys1.K, o.nO)
    estimators.accumulate(sums, np.arange(W) * 16 // W, ref["EL"], ref["dlnpsi_dR"], ref["dEL_dR"], ref["O"], 0.0)
    fin = estimators.finish(sums, 0.0)
    assert abs(E.item() - fin["E"]) < 1e-10 * abs(fin["E"])
    np.testing.assert_allclose(R.grad.numpy().ravel(), -fin["F"], rtol=1e-8, atol=1e-8 * np.abs(fin["F"]).max())
    gC = np.concatenate([Cu.grad.numpy().ravel(), Cd.grad.numpy().ravel()])
    np.testing.assert_allclose(gC, fin["dEdC"], rtol=1e-8, atol=1e-8 * np.abs(fin["dEdC"]).max())
    # correlated-sampling finite differences on the GPU
    lp0 = vmcf.vmcf_evaluate(vmcf.System(sys1, vmcf.FP64), pos, want=("logpsi",))["logpsi"].cpu().numpy()
    for I, d in [(0, 0), (2, 1), (5, 2)]:
        def f(t):
            s = copy.deepcopy(sys1)
            s.R = s.R.copy()
            s.R[I, d] += t
            return reweighted_energy(s, pos, lp0)
        fd = rich(f, 1e-4)
        assert abs(R.grad[I, d].item() - fd) < 1e-6 * max(1.0, abs(fd)), (I, d, R.grad[I, d].item(), fd)
    dEL_dC = ref["dEL_dC"].mean(0)
    M, n = sys1.M, sys1.n_up
    for sg, mu, i in [(0, 3, 2), (1, 40, 7)]:
        def f(t):
            s = copy.deepcopy(sys1)
            s.C_up, s.C_dn = s.C_up.copy(), s.C_dn.copy()
            (s.C_up if sg == 0 else s.C_dn)[mu, i] += t
            return reweighted_energy(s, pos, lp0)
        fd = rich(f, 1e-4)
        idx = sg * M * n + mu * n + i
        assert abs(gC[idx] + dEL_dC[idx] - fd) < 1e-6 * max(1.0, abs(fd)), (sg, mu, i, gC[idx], dEL_dC[idx], fd)
