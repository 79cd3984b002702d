"""Walker-reduced estimators, written out plainly in numpy (test infrastructure).

Energy: the MCMC mean of E_L (App. A, Eq. eval-observable).
Forces (Eqs. hf, pulay): F_I = -<dE_L/dR_I> - 2 <(E_L - E) d ln Psi / dR_I>, with E the
same-sample mean, i.e. the covariance form -2 (<E_L d> - E <d>).
Orbital gradient (App. A, Eq. fc-vmc-eval, read as dE/dC): B = 2 (<E_L O> - E <O>). The
paper prints this with a leading minus sign, the generalised-force convention; the
quantity handed to the Z-vector equations is dE/dC, so the sign here is +.
Error bars: delete-one-block jackknife over contiguous walker blocks (Sec. II, last
paragraph; App. A, computational details).

Sums are kept with a reference energy E_ref subtracted from E_L before it multiplies
d ln Psi / dR or O; the finished estimators do not depend on E_ref except by rounding.
"""
from __future__ import annotations

import numpy as np

FIELDS = ("n", "sE", "sE2", "sdEL", "sd", "sEd", "sO", "sEO")


def new_sums(nblocks: int, K: int, nO: int) -> dict:
    return {"n": np.zeros(nblocks), "sE": np.zeros(nblocks), "sE2": np.zeros(nblocks),
            "sdEL": np.zeros((nblocks, K * 3)), "sd": np.zeros((nblocks, K * 3)),
            "sEd": np.zeros((nblocks, K * 3)), "sO": np.zeros((nblocks, nO)), "sEO": np.zeros((nblocks, nO))}


def accumulate(sums: dict, block_of_walker: np.ndarray, EL, dlnpsi_dR, dEL_dR, O, e_ref: float,
               weight=None) -> None:
    """Add one measured sweep (one sample per walker) to the block sums. weight: per-walker
    reweighting factors |Psi/Psi_G|^2 of a guided chain (App., reweighting: every average becomes
    sum(W O) / sum(W), so each sum, the sample count included, takes the factor W); None: 1."""
    W = EL.shape[0]
    dl = dlnpsi_dR.reshape(W, -1)
    de = dEL_dR.reshape(W, -1)
    c = EL - e_ref
    wt = np.ones(W) if weight is None else np.asarray(weight, dtype=np.float64)
    for w in range(W):
        b = block_of_walker[w]
        q = wt[w]
        sums["n"][b] += q
        sums["sE"][b] += q * EL[w]
        sums["sE2"][b] += q * EL[w] * EL[w]
        sums["sdEL"][b] += q * de[w]
        sums["sd"][b] += q * dl[w]
        sums["sEd"][b] += q * c[w] * dl[w]
        sums["sO"][b] += q * O[w]
        sums["sEO"][b] += q * c[w] * O[w]


def _estimate(t: dict, e_ref: float):
    n = t["n"]
    E = t["sE"] / n
    F = -(t["sdEL"] / n + 2.0 * (t["sEd"] / n - (E - e_ref) * t["sd"] / n))
    B = 2.0 * (t["sEO"] / n - (E - e_ref) * t["sO"] / n)
    return E, F, B


def jackknife(sums: dict, e_ref: float, fn):
    """Value and delete-one-block jackknife error of fn(E, F, B)."""
    tot = {k: v.sum(axis=0) for k, v in sums.items()}
    val = np.asarray(fn(*_estimate(tot, e_ref)))
    nb = sums["n"].shape[0]
    th = np.array([fn(*_estimate({k: tot[k] - sums[k][b] for k in FIELDS}, e_ref)) for b in range(nb)])
    return val, np.sqrt((nb - 1) / nb * ((th - th.mean(axis=0)) ** 2).sum(axis=0))


def finish(sums: dict, e_ref: float):
    """Estimates from all blocks and delete-one-block jackknife error bars."""
    tot = {k: v.sum(axis=0) for k, v in sums.items()}
    E, F, B = _estimate(tot, e_ref)
    nb = sums["n"].shape[0]
    jk = [_estimate({k: tot[k] - sums[k][b] for k in FIELDS}, e_ref) for b in range(nb)]
    Ej = np.array([x[0] for x in jk])
    Fj = np.array([x[1] for x in jk])
    Bj = np.array([x[2] for x in jk])
    f = (nb - 1) / nb
    err = lambda a: np.sqrt(f * ((a - a.mean(axis=0)) ** 2).sum(axis=0))
    return {"E": E, "E_err": err(Ej), "F": F, "F_err": err(Fj), "dEdC": B, "dEdC_err": err(Bj),
            "var_EL": tot["sE2"] / tot["n"] - E * E}


def jackknife_covariance(sums: dict, e_ref: float):
    """Delete-one-block jackknife covariance matrices of the forces and of B = dE/dC (the
    Cov(B) of the error-propagation appendix, "Error propagation"):
    Cov = (nb - 1)/nb sum_b (theta_b - mean)(theta_b - mean)^T over the leave-one-out
    estimates theta_b. Returns (Cov_F [3K][3K], Cov_B [nO][nO])."""
    tot = {k: v.sum(axis=0) for k, v in sums.items()}
    nb = sums["n"].shape[0]
    jk = [_estimate({k: tot[k] - sums[k][b] for k in FIELDS}, e_ref) for b in range(nb)]
    out = []
    for idx in (1, 2):
        th = np.array([x[idx] for x in jk])
        d = th - th.mean(axis=0)
        out.append((nb - 1) / nb * d.T @ d)
    return out[0], out[1]
