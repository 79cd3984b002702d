"""Orbital rows of the walker-group proposal pass on the tensor cores.

The proposal pass forms, for every (walker, electron), the orbital row phi(r'_e) = psi(r'_e) C of the
electron's spin at its proposed position (App. A, "Computing derivatives"). In mixed precision the
walker-group kernels form these rows as a tcgen05 GEMM over tiles of 128 (walker, electron) pairs, the
AO values and C split into bf16 hi/lo parts (hi.hi + hi.lo + lo.hi, FP32 accumulation in tensor
memory). Checked here, through the C ABI:
- against the FP32 SIMT proposal pass of the same system on the same walkers: the proposals, acceptance
  uniforms and electron-nucleus Jastrow changes bit for bit (same arithmetic), the rows within 1e-4 of
  the largest row entry (each split product carries a relative error of at most 3 2^-18; the sums run
  over M <= 224 AOs);
- against the oracle: its FP64 AO values at the proposals drawn from the same Philox counters with the
  sampler's Box-Muller rule, contracted with C (numpy), within 1e-3 of the largest entry (the mixed
  proposals take the normals in float, which moves r' by up to ~1e-7 bohr; near a nucleus the rows'
  gradients scale that up);
on walker counts whose pair counts end in a ragged last tile, on the 94-electron system and on water
run on the walker-group kernels, and on an open-shell system (different orbital counts per spin).
"""
import numpy as np
import pytest

import oracle
from paper_2511_05222_gb300 import systems as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_05222_gb300 import vmcf  # noqa: E402

SIGMA = 0.3
KEY = (5222, 91)


def oracle_rows(sysx, pos, sweep):
    """FP64 proposals r' = r + sigma xi (xi: Box-Muller on the four uniforms of Philox counter
    (walker id, sweep, electron, 0), 1 - u inside the log) and the rows psi(r') C of each electron's
    spin, from the oracle's AO values."""
    W, Ne = pos.shape[:2]
    rn = np.empty_like(pos)
    for w in range(W):
        for e in range(Ne):
            x = oracle.philox4x64_10([w, sweep, e, 0], KEY)
            u = (x >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
            a, b = np.sqrt(-2.0 * np.log(1.0 - u[0])), np.sqrt(-2.0 * np.log(1.0 - u[2]))
            xi = np.array([a * np.cos(2 * np.pi * u[1]), a * np.sin(2 * np.pi * u[1]), b * np.cos(2 * np.pi * u[3])])
            rn[w, e] = pos[w, e] + SIGMA * xi
    psi = oracle.Oracle(sysx).ao_eval(rn.reshape(-1, 3))[:, :, 0].reshape(W, Ne, -1)
    nup = sysx.C_up.shape[1]
    rows = [psi[:, :nup] @ sysx.C_up, psi[:, nup:] @ sysx.C_dn]
    return rn, rows


def normwise(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("cfg,W", [(4, 37), (4, 256), (0, 203)])
def test_tensor_core_rows_match_simt_and_oracle(cfg, W):
    sysx = S.make_system(cfg)
    pos = S.initial_walkers(sysx, W, seed=17)
    g = vmcf.System(sysx, vmcf.MIXED, force_group=True)
    wk = vmcf.Walkers(g, pos, key=KEY, nblocks=2)  # the seeded positions; the next sweep is sweep 0
    out = {}
    for tc in (1, 0):
        g.set_tuning("tensor_core_rows", tc)
        out[tc] = wk.group_proposals(SIGMA)
    a, b = out[1], out[0]
    for k in ("rnew", "u", "dchi"):
        np.testing.assert_array_equal(a[k], b[k])
    nup, ndn = sysx.C_up.shape[1], sysx.C_dn.shape[1]
    blocks = [(slice(0, nup), nup), (slice(nup, nup + ndn), ndn)]
    for sl, n in blocks:
        ra, rb = a["rows"][:, sl, :n], b["rows"][:, sl, :n]
        assert np.isfinite(ra).all()
        err = normwise(ra, rb)
        assert err < 1e-4, err
        assert np.median(np.abs(ra - rb) / np.abs(rb).max()) < 1e-5
    rn, rows_o = oracle_rows(sysx, pos, 0)
    assert np.abs(a["rnew"] - rn).max() < 1e-5
    for (sl, n), ro in zip(blocks, rows_o):
        err = normwise(a["rows"][:, sl, :n], ro)
        assert err < 1e-3, err


def ch3_radical():
    """CH3 radical of the covalent-walk recipe: 9 electrons, 5 up and 4 down."""
    Z = np.asarray([6, 1, 1, 1], np.int32)
    R = S.covalent_walk(list(Z), np.random.default_rng([7000, 2, 0]))
    c, l, npr, e, co = S.basis_rule(Z, np.random.default_rng([7000, 2, 1]))
    sx = S.System("CH3", Z, R, c, l, npr, e, co, 5, 4, np.zeros((0, 0)), np.zeros((0, 0)), S.Jastrow())
    Sm = S.overlap_matrix(sx)
    rng = np.random.default_rng([7000, 2, 2])
    sx.C_up = S.orthonormal_orbitals(Sm, 5, rng)
    sx.C_dn = S.orthonormal_orbitals(Sm, 4, rng)
    sx.S = Sm
    return sx


def test_tensor_core_rows_open_shell():
    """5 up and 4 down electrons: the down rows have fewer orbitals than the up rows (zero rows of
    the padded C^dn operand), and the pair counts of the two spins differ."""
    sysx = ch3_radical()
    W = 61
    pos = S.initial_walkers(sysx, W, seed=5)
    g = vmcf.System(sysx, vmcf.MIXED, force_group=True)
    wk = vmcf.Walkers(g, pos, key=KEY, nblocks=2)
    a = wk.group_proposals(SIGMA)
    g.set_tuning("tensor_core_rows", 0)
    b = wk.group_proposals(SIGMA)
    rn, rows_o = oracle_rows(sysx, pos, 0)
    assert np.abs(a["rnew"] - rn).max() < 1e-5
    for sl, n, ro in ((slice(0, 5), 5, rows_o[0]), (slice(5, 9), 4, rows_o[1])):
        assert normwise(a["rows"][:, sl, :n], b["rows"][:, sl, :n]) < 1e-4
        assert normwise(a["rows"][:, sl, :n], ro) < 1e-3


def test_tensor_core_rows_switch():
    """The tuning key is refused where the rows have no tensor-core form (FP64 systems, the one-warp
    kernels)."""
    sysx = S.make_system(0)
    with pytest.raises(RuntimeError):
        vmcf.System(sysx, vmcf.FP64, force_group=True).set_tuning("tensor_core_rows", 1)
    with pytest.raises(RuntimeError):
        vmcf.System(sysx, vmcf.MIXED).set_tuning("tensor_core_rows", 1)
