"""Algorithmic work of one walker-evaluation, by pipe, for the roofline.

One walker-eval = one measured sweep of one walker: Ne single-electron Metropolis moves
(AO row, MO row, determinant and Jastrow ratios, Sherman-Morrison update on acceptance)
followed by one evaluation of E_L, d ln Psi/dR, dE_L/dR and O with its walker sums.

Only what the method has to compute is counted (one AO evaluation per electron with all
derivatives, one MO contraction, one inversion per spin, one adjoint sweep); recomputation
done by an implementation is not counted, so it lowers the achieved fraction. The MO
contraction of the evaluation is two rows per electron: the Slater row and the row of
P = lap(phi) + 2 grad J . grad(phi), which is linear in C (one AO coefficient per function);
the gradient and Laplacian rows themselves are never needed, since the kinetic term is
sum_i P_ei B_ie + lap J + |grad J|^2 and the determinant drift comes out of the force terms. Counts are
flops (an FMA is 2) split by the pipe that executes them in mixed mode: FP64 (inversion,
ratio dot products) and FP32 (everything else), plus exponentials (one per primitive per
electron per pass) counted separately for the SFU.
"""
from __future__ import annotations


def per_walker_eval(K: int, M: int, n_up: int, n_dn: int, nprim: int, acc: float = 0.5, MJ: int = 0,
                    nJprim: int = 0, kref: int = 26) -> dict:
    """MJ, nJprim: functions and primitives of the Jastrow basis of the AO-expanded Jastrow terms
    (0: none). Those add, per move, one Jastrow-basis evaluation at r' and the product Xi dphi with
    its dot products; per evaluation, the basis with all derivatives at every electron, t0 = xi + Xi s,
    u_e = Xi psi^J(r_e) and p_e = Xi w_e for every electron, and the force terms.
    kref: moves between FP64 re-inversions. A measured sweep re-inverts (Ne - 1) // kref times during its
    moves (a re-inversion that would fall on the last move is the evaluation's own, counted there):
    each rebuilds the Slater matrices (AO values and MO rows of every electron) and inverts both blocks."""
    Ne = n_up + n_dn
    ns = [n_up] * n_up + [n_dn] * n_dn  # orbital count seen by each electron
    move = {
        "exp": Ne * nprim,
        "fp32": sum(3 * nprim + 3 * M + 2 * M * n + (Ne - 1 + K) * 16 + acc * 4 * n * n for n in ns),
        "fp64": sum(2 * n for n in ns),
    }
    spins = [n for n in (n_up, n_dn) if n > 0]
    measure = {
        "exp": Ne * nprim,
        "fp32": (Ne * (8 * nprim + 40 * M)                       # AO value, gradient, Laplacian, Hessian, grad-Laplacian
                 + Ne * 8 * M                                    # AO coefficients lap psi + 2 grad J . grad psi of the P row
                 + sum(4 * M * n for n in ns)                    # MO rows: Slater row and P = lap phi + 2 grad J . grad phi
                 + 25 * (Ne * (Ne - 1) // 2) + 25 * Ne * K       # Jastrow and potentials
                 + sum(2 * n for n in ns)                        # kinetic ratio sum_i P_ei B_ie
                 + sum(4 * n ** 3 for n in spins)                # adjoint weights B P B
                 + sum(4 * M * n for n in ns) + 36 * Ne * M      # back-projection, force contraction, determinant drift
                 + 40 * Ne * K                                   # e-n Jastrow and V_en derivatives
                 + sum(2 * M * n for n in ns)                    # O
                 + sum(4 * M * n for n in spins) + 18 * K),      # walker sums
        "fp64": sum(2 * n ** 3 for n in spins),                  # Gauss-Jordan inversion per spin
    }
    n_ref = (Ne - 1) // kref
    spins0 = [n for n in (n_up, n_dn) if n > 0]
    move["exp"] += n_ref * Ne * nprim
    move["fp32"] += n_ref * sum(3 * nprim + 3 * M + 2 * M * n for n in ns)
    move["fp64"] += n_ref * sum(2 * n ** 3 for n in spins0)
    if MJ:
        move["exp"] += Ne * nJprim
        move["fp32"] += Ne * (3 * nJprim + 3 * MJ + 2 * MJ * MJ + 4 * MJ)
        measure["exp"] += Ne * nJprim
        measure["fp32"] += Ne * (8 * nJprim + 40 * MJ) + 2 * MJ * MJ + 4 * Ne * MJ * MJ + Ne * 46 * MJ
    total = {k: move[k] + measure[k] for k in move}
    return {"move": move, "measure": measure, "total": total}


def roofline_time(work: dict, peaks: dict) -> tuple[str, float]:
    """Binding pipe and the time (s) one unit of `work` needs at the measured peaks."""
    t = {"fp32": work["fp32"] / (peaks["fp32_tflops"] * 1e12),
         "fp64": work["fp64"] / (peaks["fp64_tflops"] * 1e12),
         "sfu": work["exp"] / (peaks["exp_gops"] * 1e9)}
    bound = max(t, key=t.get)
    return bound, t[bound]
