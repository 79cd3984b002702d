"""VMCForces (torch.autograd.Function over libvmcf) on fixed walkers, at the size of the
differentiation workload: the C2OH6 system, 16384 fixed walkers, forces on all 9 nuclei and the
full dE/dC (72 x 13 per spin).

- FP64: the R-gradient equals central finite differences of the correlated-sampling energy
  (Richardson-extrapolated over dR = 1e-4 and 5e-5), and the C-gradient plus <dE_L/dC> equals
  central finite differences in C with dC = 1e-5, element by element (both exact identities of
  the reweighted energy on fixed walkers); E, F and dE/dC agree with the FP64 oracle's
  estimators on the same walkers to 1e-10.
- Mixed precision: every force component and every dE/dC element of the mixed path within 0.1 x
  the FP64 error bar of the FP64 values (the same estimator accuracy)."""
import copy
import time

import numpy as np
import pytest

import oracle
from oracle import estimators
from paper_2511_05222_gb300 import systems as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_05222_gb300 import vmcf  # noqa: E402
from paper_2511_05222_gb300.autograd import vmc_energy  # noqa: E402

TOL64 = 1e-10


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def reweighted_energy(sysx, pos_dev, logpsi0):
    """Correlated-sampling energy of the fixed walkers under the parameters of sysx:
    sum_w q_w E_L,w / sum_w q_w, q_w = |Psi'(x_w) / Psi(x_w)|^2 (FP64 GPU evaluation)."""
    out = vmcf.vmcf_evaluate(vmcf.System(sysx, vmcf.FP64), pos_dev, want=("EL", "logpsi"))
    el, lp = out["EL"].cpu().numpy(), out["logpsi"].cpu().numpy()
    w = np.exp(2 * (lp - logpsi0))
    return (w * el).sum() / w.sum()


def rich(f, h):
    return (4 * (f(h / 2) - f(-h / 2)) / h - (f(h) - f(-h)) / (2 * h)) / 3


@pytest.fixture(scope="module")
def fixed_walkers(sys1):
    """16384 C2OH6 walkers after two sweeps of the oracle's chain, and the oracle's per-walker
    outputs on them."""
    W = 16384
    o = oracle.Oracle(sys1)
    st = o.new_state(S.initial_walkers(sys1, W, seed=17), key=(5222, 2))
    o.sample(st, 2)
    ref = o.eval(st["pos"], want=("EL", "dlnpsi_dR", "dEL_dR", "O", "dEL_dC"))
    return st["pos"], ref


def params(sysx):
    return (torch.tensor(sysx.R, dtype=torch.float64, requires_grad=True),
            torch.tensor(sysx.C_up, requires_grad=True), torch.tensor(sysx.C_dn, requires_grad=True))


def test_autograd_forces_and_orbital_gradient_config_scale(sys1, fixed_walkers):
    pos_h, ref = fixed_walkers
    W, nb = pos_h.shape[0], 64
    pos = torch.as_tensor(pos_h, device="cuda")
    R, Cu, Cd = params(sys1)
    E = vmc_energy(R, Cu, Cd, sys1, pos, vmcf.FP64, nb)
    E.backward()
    gR = R.grad.numpy().ravel()
    gC = np.concatenate([Cu.grad.numpy().ravel(), Cd.grad.numpy().ravel()])
    # the oracle's estimators on the same walkers (uniform weights, the library's blocks)
    sums = estimators.new_sums(nb, sys1.K, sys1.M * sys1.Ne)
    blk = np.zeros(W, int)
    for b in range(nb):
        blk[(W * b) // nb:(W * (b + 1)) // nb] = b
    estimators.accumulate(sums, blk, ref["EL"], ref["dlnpsi_dR"], ref["dEL_dR"], ref["O"], 0.0)
    fin = estimators.finish(sums, 0.0)
    assert abs(E.item() - fin["E"]) < TOL64 * abs(fin["E"])
    assert rel(-gR, fin["F"]) < TOL64, rel(-gR, fin["F"])
    assert rel(gC, fin["dEdC"]) < TOL64, rel(gC, fin["dEdC"])

    # correlated-sampling finite differences on the GPU: every nuclear coordinate
    lp0 = vmcf.vmcf_evaluate(vmcf.System(sys1, vmcf.FP64), pos, want=("logpsi",))["logpsi"].cpu().numpy()
    t0 = time.perf_counter()
    fdR = np.zeros(3 * sys1.K)
    for I in range(sys1.K):
        for d in range(3):
            def f(t):
                s = copy.deepcopy(sys1)
                s.R = s.R.copy()
                s.R[I, d] += t
                return reweighted_energy(s, pos, lp0)
            fdR[3 * I + d] = rich(f, 1e-4)
    np.testing.assert_allclose(gR, fdR, rtol=0, atol=1e-6 * max(1.0, np.abs(fdR).max()))
    # every orbital coefficient, dC = 1e-5: FD = B + <dE_L/dC> exactly on fixed walkers
    M, nu, nd = sys1.M, sys1.n_up, sys1.n_dn
    dC = 1e-5
    fdC = np.zeros(M * (nu + nd))
    base = copy.deepcopy(sys1)
    for sg, n in ((0, nu), (1, nd)):
        for mu in range(M):
            for i in range(n):
                vals = []
                for t in (dC, -dC):
                    s = copy.copy(base)
                    s.C_up, s.C_dn = base.C_up.copy(), base.C_dn.copy()
                    (s.C_up if sg == 0 else s.C_dn)[mu, i] += t
                    vals.append(reweighted_energy(s, pos, lp0))
                fdC[sg * M * nu + mu * n + i] = (vals[0] - vals[1]) / (2 * dC)
    print(f"finite differences: {time.perf_counter() - t0:.1f} s for {4 * 3 * sys1.K + 2 * fdC.size} evaluations "
          f"of {W} walkers")
    exact = gC + ref["dEL_dC"].mean(0)
    np.testing.assert_allclose(exact, fdC, rtol=0, atol=1e-6 * max(1.0, np.abs(fdC).max()))


def test_autograd_mixed_within_a_tenth_of_the_fp64_error_bars(sys1, fixed_walkers):
    """The mixed-precision VMCForces on the same 16384 walkers: every force component and every
    dE/dC element within 0.1 x the FP64 jackknife error bar of the FP64 gradient."""
    pos = torch.as_tensor(fixed_walkers[0], device="cuda")
    out = {}
    for prec in (vmcf.FP64, vmcf.MIXED):
        R, Cu, Cd = params(sys1)
        E = vmc_energy(R, Cu, Cd, sys1, pos, prec, 64)
        E.backward()
        out[prec] = (E.item(), R.grad.numpy().ravel(), np.concatenate([Cu.grad.numpy().ravel(),
                                                                       Cd.grad.numpy().ravel()]))
    from paper_2511_05222_gb300.autograd import VMCForces  # noqa: F401
    g = vmcf.System(sys1, vmcf.FP64)
    wk = vmcf.Walkers(g, pos, nblocks=64)
    wk.reset_accumulators(0.0)
    wk.measure()
    err = wk.reduce_estimators()
    (E64, gR64, gC64), (Em, gRm, gCm) = out[vmcf.FP64], out[vmcf.MIXED]
    assert abs(Em - E64) <= 0.1 * err["E_err"], (Em, E64, err["E_err"])
    dF = np.abs(gRm - gR64) / err["F_err"].ravel()
    assert dF.max() <= 0.1, dF.max()
    ok = err["dEdC_err"] > 0
    dB = np.abs(gCm - gC64)[ok] / err["dEdC_err"][ok]
    assert dB.max() <= 0.1, dB.max()
