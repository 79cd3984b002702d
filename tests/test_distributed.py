"""Sharded walkers over 2 ranks (gloo, CPU): each rank samples its own walkers with global
walker ids, the block sums are gathered, and the host finish of libvmcf gives the same
estimators as one process holding all walkers. The chains are produced by the oracle's
sampler (the GPU is not needed for the host-side logic under test)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2511_05222_gb300 import systems as S
from paper_2511_05222_gb300 import distributed as D

W_TOTAL, NB_LOCAL, E_REF = 48, 4, -76.0


def block_sums(o, sysx, pos, wid0_unused, nb):
    """Block sums in the library's layout from oracle per-walker outputs (blocks: contiguous
    walker ranges [W b / nb, W (b + 1) / nb))."""
    out = o.eval(pos, want=("EL", "dlnpsi_dR", "dEL_dR", "O"))
    W = pos.shape[0]
    c = out["EL"] - E_REF
    dl = out["dlnpsi_dR"].reshape(W, -1)
    de = out["dEL_dR"].reshape(W, -1)
    rows = []
    for b in range(nb):
        sl = slice(W * b // nb, W * (b + 1) // nb)
        rows.append(np.concatenate([[sl.stop - sl.start, out["EL"][sl].sum(), (out["EL"][sl] ** 2).sum()],
                                    de[sl].sum(0), dl[sl].sum(0), (c[sl, None] * dl[sl]).sum(0),
                                    out["O"][sl].sum(0), (c[sl, None] * out["O"][sl]).sum(0)]))
    return np.array(rows)


def run_shard(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sysx = S.make_system(0)
    o = oracle.Oracle(sysx, nthreads=1)
    Wl = W_TOTAL // world
    pos_all = S.initial_walkers(sysx, W_TOTAL, seed=3)
    st = o.new_state(pos_all[rank * Wl:(rank + 1) * Wl], key=(5222, 0), wid0=rank * Wl)
    o.sample(st, 3)
    o.force_refresh(st)
    blocks = D.gather_block_sums(block_sums(o, sysx, st["pos"], rank * Wl, NB_LOCAL))
    est = D.finish_estimators(blocks, sysx.K, sysx.M, sysx.n_up, sysx.n_dn, E_REF)
    q.put((rank, st["pos"], est))
    dist.barrier()
    dist.destroy_process_group()


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_rank_estimators_equal_one_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=run_shard, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        r, pos, est = q.get(timeout=300)
        res[r] = (pos, est)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # one process, all walkers, same global ids and the same block partition
    sysx = S.make_system(0)
    o = oracle.Oracle(sysx, nthreads=1)
    st = o.new_state(S.initial_walkers(sysx, W_TOTAL, seed=3), key=(5222, 0), wid0=0)
    o.sample(st, 3)
    o.force_refresh(st)
    np.testing.assert_array_equal(np.concatenate([res[0][0], res[1][0]]), st["pos"])
    blocks = np.concatenate([block_sums(o, sysx, st["pos"][r * 24:(r + 1) * 24], 0, NB_LOCAL) for r in range(2)])
    one = D.finish_estimators(blocks, sysx.K, sysx.M, sysx.n_up, sysx.n_dn, E_REF)
    for r in range(2):
        for k in ("E", "E_err", "F", "F_err", "dEdC", "dEdC_err"):
            np.testing.assert_array_equal(res[r][1][k], one[k])


def test_host_finish_matches_the_numpy_finish():
    """vmcf_finish_estimators (C++) against oracle/estimators.finish (numpy) on the same sums."""
    from oracle import estimators
    sysx = S.make_system(0)
    o = oracle.Oracle(sysx, nthreads=1)
    pos = S.initial_walkers(sysx, 64, seed=4)
    nb = 8
    blocks = block_sums(o, sysx, pos, 0, nb)
    got = D.finish_estimators(blocks, sysx.K, sysx.M, sysx.n_up, sysx.n_dn, E_REF)
    sums = estimators.new_sums(nb, sysx.K, o.nO)
    out = o.eval(pos, want=("EL", "dlnpsi_dR", "dEL_dR", "O"))
    estimators.accumulate(sums, np.arange(64) * nb // 64, out["EL"], out["dlnpsi_dR"], out["dEL_dR"], out["O"], E_REF)
    ref = estimators.finish(sums, E_REF)
    assert abs(got["E"] - ref["E"]) < 1e-12 * abs(ref["E"])
    assert abs(got["E_err"] - ref["E_err"]) < 1e-9 * ref["E_err"]
    np.testing.assert_allclose(got["F"].ravel(), ref["F"], rtol=1e-9, atol=1e-9 * np.abs(ref["F"]).max())
    np.testing.assert_allclose(got["dEdC"], ref["dEdC"], rtol=1e-9, atol=1e-9 * np.abs(ref["dEdC"]).max())
    np.testing.assert_allclose(got["F_err"].ravel(), ref["F_err"], rtol=1e-8)


def test_host_covariance_factor_matches_the_numpy_covariance():
    """vmcf_finish_covariance (C++ low-rank factor b, Cov = b b^T) against the oracle's
    jackknife covariance matrices; the diagonal is the square of the error bars."""
    from oracle import estimators
    sysx = S.make_system(0)
    o = oracle.Oracle(sysx, nthreads=1)
    pos = S.initial_walkers(sysx, 64, seed=5)
    nb = 8
    blocks = block_sums(o, sysx, pos, 0, nb)
    Ff, Bf = D.finish_covariance(blocks, sysx.K, sysx.M, sysx.n_up, sysx.n_dn, E_REF)
    sums = estimators.new_sums(nb, sysx.K, o.nO)
    out = o.eval(pos, want=("EL", "dlnpsi_dR", "dEL_dR", "O"))
    estimators.accumulate(sums, np.arange(64) * nb // 64, out["EL"], out["dlnpsi_dR"], out["dEL_dR"], out["O"], E_REF)
    cF, cB = estimators.jackknife_covariance(sums, E_REF)
    np.testing.assert_allclose(Ff @ Ff.T, cF, rtol=0, atol=1e-9 * np.abs(cF).max())
    np.testing.assert_allclose(Bf @ Bf.T, cB, rtol=0, atol=1e-9 * np.abs(cB).max())
    est = D.finish_estimators(blocks, sysx.K, sysx.M, sysx.n_up, sysx.n_dn, E_REF)
    np.testing.assert_allclose(np.sqrt(np.diag(Bf @ Bf.T)), est["dEdC_err"], rtol=1e-9, atol=1e-300)
    assert np.linalg.matrix_rank(Bf) <= nb - 1  # the deviations from their mean sum to zero


def test_host_warp_finish_matches_the_numpy_finish():
    """vmcf_finish_warp (C++) against the oracle's estimators fed the space-warp vectors."""
    from oracle import estimators
    sysx = S.make_system(0)
    o = oracle.Oracle(sysx, nthreads=1)
    W, nb = 64, 8
    pos = S.initial_walkers(sysx, W, seed=6)
    base = block_sums(o, sysx, pos, 0, nb)
    out = o.eval(pos, want=("EL",))
    wv = o.eval_warp(pos)
    c = out["EL"] - E_REF
    de, dl = wv["dEL_sw"].reshape(W, -1), wv["dlnpsi_sw"].reshape(W, -1)
    extra = [np.concatenate([de[sl].sum(0), dl[sl].sum(0), (c[sl, None] * dl[sl]).sum(0)])
             for sl in (slice(W * b // nb, W * (b + 1) // nb) for b in range(nb))]
    blocks = np.concatenate([base, np.array(extra)], 1)
    got = D.finish_warp(blocks, sysx.K, sysx.M, sysx.n_up, sysx.n_dn, E_REF)
    sums = estimators.new_sums(nb, sysx.K, o.nO)
    estimators.accumulate(sums, np.arange(W) * nb // W, out["EL"], wv["dlnpsi_sw"], wv["dEL_sw"],
                          np.zeros((W, o.nO)), E_REF)
    ref = estimators.finish(sums, E_REF)
    np.testing.assert_allclose(got["F"].ravel(), ref["F"], rtol=1e-9, atol=1e-9 * np.abs(ref["F"]).max())
    np.testing.assert_allclose(got["F_err"].ravel(), ref["F_err"], rtol=1e-8)


def _gather_or_die(rank, world, port, q):
    """Rank 1 fails before the exchange (an exception on the host, no GPU involved); rank 0's
    gather must end with an error instead of waiting forever."""
    import datetime
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        q.put((1, "failed"))
        raise SystemExit(3)  # leaves between steps, before the collective
    try:
        D.gather_block_sums(np.zeros((NB_LOCAL, 8)))
        q.put((0, "gathered"))
    except Exception as e:  # noqa: BLE001 - any error is the detection we want
        q.put((0, "error: " + type(e).__name__))


def test_a_rank_that_fails_before_the_exchange_ends_the_gather_with_an_error():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_gather_or_die, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
    assert res[1] == "failed" and procs[1].exitcode == 3
    assert res[0].startswith("error"), res[0]
