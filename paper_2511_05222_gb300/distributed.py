"""Several GPUs, one process each: walkers are sharded, and the only exchange is the FP64
block sums of the estimators, gathered once at the end (host side, torch.distributed on any
backend). Each rank samples its own walkers with global walker ids wid0 = rank * W_local, so
the Philox streams, and hence the chains, are the ones a single GPU would draw for the same
global walker set.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import vmcf


def gather_block_sums(local_blocks: np.ndarray, group=None) -> np.ndarray:
    """All ranks' block sums side by side ([world * nblocks][L]), rank order."""
    import torch
    import torch.distributed as dist
    t = torch.as_tensor(np.ascontiguousarray(local_blocks, dtype=np.float64))
    ws = dist.get_world_size(group)
    out = [torch.empty_like(t) for _ in range(ws)]
    dist.all_gather(out, t, group=group)
    return torch.cat(out, 0).numpy()


def finish_estimators(blocks: np.ndarray, K: int, M: int, n_up: int, n_dn: int, e_ref: float) -> dict:
    """vmcf_finish_estimators on host block sums (no GPU involved)."""
    L = vmcf.lib()
    L.vmcf_finish_estimators.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int] + [ctypes.c_int] * 4 + \
        [ctypes.c_double] + [ctypes.POINTER(ctypes.c_double)] * 6
    blocks = np.ascontiguousarray(blocks, dtype=np.float64)
    nO = M * (n_up + n_dn)
    E, Ee = np.zeros(1), np.zeros(1)
    F, Fe = np.zeros(3 * K), np.zeros(3 * K)
    B, Be = np.zeros(nO), np.zeros(nO)
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    rc = L.vmcf_finish_estimators(dp(blocks), blocks.shape[0], K, M, n_up, n_dn, float(e_ref), dp(E), dp(Ee), dp(F),
                                  dp(Fe), dp(B), dp(Be))
    if rc != 0:
        raise vmcf.VmcfError(rc, "vmcf_finish_estimators")
    return {"E": float(E[0]), "E_err": float(Ee[0]), "F": F.reshape(K, 3), "F_err": Fe.reshape(K, 3), "dEdC": B,
            "dEdC_err": Be}


def finish_covariance(blocks: np.ndarray, K: int, M: int, n_up: int, n_dn: int, e_ref: float):
    """vmcf_finish_covariance on host block sums: factors (F [3K][nb], B [nO][nb]) with
    Cov = factor @ factor.T (no GPU involved)."""
    L = vmcf.lib()
    L.vmcf_finish_covariance.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int] + [ctypes.c_int] * 4 + \
        [ctypes.c_double] + [ctypes.POINTER(ctypes.c_double)] * 2
    blocks = np.ascontiguousarray(blocks, dtype=np.float64)
    nb = blocks.shape[0]
    Ff = np.zeros((3 * K, nb))
    Bf = np.zeros((M * (n_up + n_dn), nb))
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    rc = L.vmcf_finish_covariance(dp(blocks), nb, K, M, n_up, n_dn, float(e_ref), dp(Ff), dp(Bf))
    if rc != 0:
        raise vmcf.VmcfError(rc, "vmcf_finish_covariance")
    return Ff, Bf


def finish_warp(blocks: np.ndarray, K: int, M: int, n_up: int, n_dn: int, e_ref: float) -> dict:
    """vmcf_finish_warp on host block sums that carry the space-warp fields (no GPU involved)."""
    L = vmcf.lib()
    blocks = np.ascontiguousarray(blocks, dtype=np.float64)
    F, Fe = np.zeros(3 * K), np.zeros(3 * K)
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    rc = L.vmcf_finish_warp(dp(blocks), blocks.shape[0], blocks.shape[1], K, M, n_up, n_dn, float(e_ref), dp(F), dp(Fe))
    if rc != 0:
        raise vmcf.VmcfError(rc, "vmcf_finish_warp")
    return {"F": F.reshape(K, 3), "F_err": Fe.reshape(K, 3)}


def sharded_estimators(walkers: "vmcf.Walkers", group=None) -> dict:
    """Estimators over the walkers of all ranks: gather block sums, finish on the host."""
    s = walkers.system
    blocks = gather_block_sums(walkers.block_sums(), group)
    return finish_estimators(blocks, s.K, s.M, s.n_up, s.n_dn, walkers.e_ref)
