"""Writes the stored oracle values under tests/golden/ (run from the repository root:
`python tests/golden/make_golden.py`). It calls only the FP64 CPU oracle and the seeded input
generator; no stored value comes from the CUDA library.

water_oracle.txt -- the water workload (O + 2 H, 10 electrons, 24 AOs; the seeded generator's
system 0) at three seeded walker configurations:
  EL         local energy E_L = H Psi / Psi (App. A)
  logpsi     ln|Psi| of the Jastrow-Slater wavefunction (App. A, wavefunction ansatz)
  dlnpsi_dR  d ln|Psi| / dR_I at fixed electrons (the Pulay term's derivative, Eq. pulay)
  dEL_dR     dE_L / dR_I at fixed electrons (the Hellmann-Feynman term, Eq. hf)
  O          d ln|Psi| / dC^s_{mu i} = sum_e psi_mu(r_e) (A^s)^-1_{i e} (App. A, Eq. fc-vmc-eval),
             spin up [M][n_up] then spin down [M][n_dn]
and a short Metropolis chain of the same walkers (single-electron Gaussian moves, step 0.3 bohr,
acceptance |Psi'/Psi|^2, Philox4x64-10 streams keyed by (5222, 7), inverses rebuilt every 26
attempted moves):
  chain_pos  positions after three sweeps
  chain_nacc accepted moves per walker
and the walker-reduced estimators of 64 seeded walker configurations in 8 contiguous blocks
with E_ref = -76: E, the forces (Eqs. hf, pulay) and dE/dC (Eq. fc-vmc-eval), with the
delete-one-block jackknife errors of E and of the forces.
"""
from __future__ import annotations

import sys
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
from oracle import estimators  # noqa: E402
from paper_2511_05222_gb300 import systems as S  # noqa: E402

OUT = Path(__file__).resolve().parent / "water_oracle.txt"
EVAL_SEED, EST_SEED, CHAIN_KEY, E_REF = 11, 12, (5222, 7), -76.0


def water_inputs():
    """The seeded system, the three evaluation walkers and the 64 estimator walkers."""
    sysx = S.make_system(0)
    return sysx, S.initial_walkers(sysx, 3, EVAL_SEED), S.initial_walkers(sysx, 64, EST_SEED)


def compute():
    sysx, pos, pos64 = water_inputs()
    orc = oracle.Oracle(sysx, nthreads=1)
    out = orc.eval(pos, want=("EL", "logpsi", "dlnpsi_dR", "dEL_dR", "O"))
    vals = {"pos": pos, "EL": out["EL"], "logpsi": out["logpsi"], "dlnpsi_dR": out["dlnpsi_dR"],
            "dEL_dR": out["dEL_dR"], "O": out["O"]}
    st = orc.new_state(pos, key=CHAIN_KEY)
    orc.sample(st, 3, sigma=0.3, refresh_k=26)
    # every acceptance decision of the stored chain is clear of a tie, so that a rounding
    # difference cannot flip one
    assert st["margin"].min() >= 1e-6, st["margin"]
    vals["chain_pos"] = st["pos"]
    vals["chain_nacc"] = st["nacc"].astype(np.float64)
    e64 = orc.eval(pos64, want=("EL", "dlnpsi_dR", "dEL_dR", "O"))
    sums = estimators.new_sums(8, sysx.K, orc.nO)
    estimators.accumulate(sums, np.arange(64) // 8, e64["EL"], e64["dlnpsi_dR"], e64["dEL_dR"], e64["O"], E_REF)
    fin = estimators.finish(sums, E_REF)
    for k in ("E", "E_err", "F", "F_err", "dEdC"):
        vals["est_" + k] = np.asarray(fin[k], dtype=np.float64)
    return vals


def write(vals: dict, path: Path = OUT) -> None:
    lines = ["# Oracle values of the water workload; written by tests/golden/make_golden.py (see its",
             "# docstring for what each block is and the passage of arXiv:2511.05222 that defines it).",
             "# Format: '[name] shape...' then the values in C order, four per line."]
    for k, v in vals.items():
        a = np.asarray(v, dtype=np.float64)
        lines.append(f"[{k}] " + " ".join(str(d) for d in a.shape))
        flat = [repr(float(x)) for x in a.ravel()]
        for i in range(0, len(flat), 4):
            lines.append(" ".join(flat[i:i + 4]))
    path.write_text("\n".join(lines) + "\n")


def read(path: Path = OUT) -> dict:
    out, name, shape, buf = {}, None, None, []
    for line in path.read_text().splitlines():
        if line.startswith("#") or not line.strip():
            continue
        if line.startswith("["):
            if name is not None:
                out[name] = np.array(buf, dtype=np.float64).reshape(shape)
            head = line.split()
            name, shape, buf = head[0][1:-1], tuple(int(x) for x in head[1:]), []
        else:
            buf.extend(float(x) for x in line.split())
    if name is not None:
        out[name] = np.array(buf, dtype=np.float64).reshape(shape)
    return out


if __name__ == "__main__":
    write(compute())
    print(f"wrote {OUT}")
