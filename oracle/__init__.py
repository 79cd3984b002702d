"""Plain FP64 CPU oracle for the VMC hot path (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import this
package. It shares no code with the CUDA library; the seeded input generator
(`paper_2511_05222_gb300.systems`) is the only module both sides read, and it holds none
of the method's arithmetic.

Parity is pinned for every function here (see tests/test_oracle_pins.py): closed forms
(single-Gaussian hydrogen, two-electron product states), brute-force determinants,
finite differences, correlated-sampling finite differences, invariances and exact
Gaussian-integral expectation values.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "vmc_oracle.cpp"
_LIB_DIR = _HERE / "_build"
_LIB = _LIB_DIR / "liboracle.so"
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_u32p = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> Path:
    """Compile the oracle with plain flags: -O2, no fast-math, no FMA contraction."""
    if _LIB.exists() and not force and _LIB.stat().st_mtime >= _SRC.stat().st_mtime:
        return _LIB
    _LIB_DIR.mkdir(exist_ok=True)
    tmp = _LIB.with_suffix(f".{os.getpid()}.tmp")
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", str(_SRC), "-o", str(tmp)]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(str(build()))
        L = _lib
        L.osys_create.restype = ctypes.c_void_p
        L.osys_create.argtypes = [ctypes.c_int, _ip, _dp, ctypes.c_int, _ip, _ip, _ip, _dp, _dp, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int]
        L.osys_destroy.argtypes = [ctypes.c_void_p]
        L.osys_nao.argtypes = [ctypes.c_void_p]
        L.osys_norm_coefs.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int]
        L.osys_ao_eval.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, _dp]
        L.oracle_lu_inverse.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp]
        L.oracle_philox4x64_10.argtypes = [_u64p, _u64p, _u64p]
        L.osys_eval.restype = ctypes.c_int
        L.osys_eval.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_int] + [_dp] * 10
        L.osys_eval_warp.restype = ctypes.c_int
        L.osys_eval_warp.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _dp]
        L.osys_refresh.restype = ctypes.c_int
        L.osys_refresh.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, _dp, ctypes.c_int]
        L.osys_sample.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, _dp, ctypes.c_uint64, ctypes.c_uint64,
                                  ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                  _ip, _u32p, _u32p, _dp, ctypes.c_int, ctypes.c_double]
        L.osys_set_jastrow_basis.restype = ctypes.c_int
        L.osys_set_jastrow_basis.argtypes = [ctypes.c_void_p, ctypes.c_int, _ip, _ip, _ip, _dp, _dp, ctypes.c_int,
                                             _dp, _dp]
        L.osys_move_jastrow_diff.restype = ctypes.c_double
        L.osys_move_jastrow_diff.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int, _dp]
        L.osys_guide_weight.restype = ctypes.c_int
        L.osys_guide_weight.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_double, _dp, ctypes.c_int]
    return _lib


def _p(a, t=_dp):
    return None if a is None else a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def philox4x64_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, np.uint64)
    lib().oracle_philox4x64_10(_p(c, _u64p), _p(k, _u64p), _p(out, _u64p))
    return out


def lu_inverse(A: np.ndarray):
    A = _f64(A)
    n = A.shape[0]
    inv = np.zeros_like(A)
    la, sg = np.zeros(1), np.zeros(1)
    rc = lib().oracle_lu_inverse(n, _p(A), _p(inv), _p(la), _p(sg))
    return inv, float(la[0]), float(sg[0]), rc


class Oracle:
    """FP64 evaluation and Metropolis sampling of one system."""

    def __init__(self, sys, nthreads: int = 0):
        self.sys = sys
        self.nthreads = nthreads
        L = lib()
        j = sys.jastrow
        self._keep = [np.ascontiguousarray(sys.Z, np.int32), _f64(sys.R),
                      np.ascontiguousarray(sys.shell_center, np.int32), np.ascontiguousarray(sys.shell_l, np.int32),
                      np.ascontiguousarray(sys.shell_nprim, np.int32), _f64(sys.shell_exp), _f64(sys.shell_coef),
                      _f64(sys.C_up), _f64(sys.C_dn),
                      np.array([j.F_anti, j.F_par, j.a_anti, j.a_par, j.b_en], np.float64)]
        Z, R, c, l, npr, e, co, Cu, Cd, jp = self._keep
        self.h = L.osys_create(sys.K, _p(Z, _ip), _p(R), sys.nshell, _p(c, _ip), _p(l, _ip), _p(npr, _ip),
                               _p(e), _p(co), e.shape[1], sys.n_up, sys.n_dn, _p(Cu), _p(Cd), _p(jp),
                               int(j.enable_J1), int(j.enable_J2), int(bool(getattr(j, "two_body_exp", False))))
        jb = getattr(j, "basis", None)
        self.MJ = 0
        if jb is not None:
            jk = [np.ascontiguousarray(jb.shell_center, np.int32), np.ascontiguousarray(jb.shell_l, np.int32),
                  np.ascontiguousarray(jb.shell_nprim, np.int32), _f64(jb.shell_exp), _f64(jb.shell_coef),
                  _f64(jb.xi), _f64(jb.Xi)]
            self._keep += jk
            self.MJ = L.osys_set_jastrow_basis(self.h, jb.nshell, _p(jk[0], _ip), _p(jk[1], _ip), _p(jk[2], _ip),
                                               _p(jk[3]), _p(jk[4]), jk[3].shape[1], _p(jk[5]), _p(jk[6]))
        self.M = L.osys_nao(self.h)
        self.K, self.Ne = sys.K, sys.Ne
        self.nO = self.M * (sys.n_up + sys.n_dn)
        self.nB = sys.n_up ** 2 + sys.n_dn ** 2

    def __del__(self):
        try:
            lib().osys_destroy(self.h)
        except Exception:
            pass

    def norm_coefs(self) -> np.ndarray:
        out = np.zeros_like(self._keep[6])
        lib().osys_norm_coefs(self.h, _p(out), out.shape[1])
        return out

    def ao_eval(self, pts: np.ndarray) -> np.ndarray:
        """(npts, M, 14): value, grad (3), Laplacian, Hessian (xx yy zz xy xz yz), grad Laplacian (3)."""
        pts = _f64(pts).reshape(-1, 3)
        out = np.zeros((pts.shape[0], self.M, 14))
        lib().osys_ao_eval(self.h, pts.shape[0], _p(pts), _p(out))
        return out

    def eval(self, pos: np.ndarray, want=("EL",)):
        """Per-walker outputs for positions (W, Ne, 3). `want` selects among EL, logpsi, sign,
        dlnpsi_dR, dEL_dR, O, dEL_dC, grad_lnpsi, lap_lnpsi, parts."""
        pos = _f64(pos)
        W = pos.shape[0]
        K, Ne, nO = self.K, self.Ne, self.nO
        shapes = {"EL": (W,), "logpsi": (W,), "sign": (W,), "dlnpsi_dR": (W, K, 3), "dEL_dR": (W, K, 3),
                  "O": (W, nO), "dEL_dC": (W, nO), "grad_lnpsi": (W, Ne, 3), "lap_lnpsi": (W, Ne),
                  "parts": (W, 5)}
        out = {k: np.zeros(shapes[k]) for k in want}
        order = ["EL", "logpsi", "sign", "dlnpsi_dR", "dEL_dR", "O", "dEL_dC", "grad_lnpsi", "lap_lnpsi", "parts"]
        nsing = lib().osys_eval(self.h, W, _p(pos), self.nthreads, *[_p(out.get(k)) for k in order])
        out["n_singular"] = nsing
        return out

    def eval_warp(self, pos: np.ndarray) -> dict:
        """Electron derivatives dE_L/dr (W, Ne, 3) and the space-warp force vectors
        dE_L^sw/dR, d ln Psi^sw/dR (W, K, 3) for positions (W, Ne, 3)."""
        pos = _f64(pos)
        W = pos.shape[0]
        out = {"dEL_dr": np.zeros((W, self.Ne, 3)), "dEL_sw": np.zeros((W, self.K, 3)),
               "dlnpsi_sw": np.zeros((W, self.K, 3))}
        out["n_singular"] = lib().osys_eval_warp(self.h, W, _p(pos), self.nthreads, _p(out["dEL_dr"]),
                                                 _p(out["dEL_sw"]), _p(out["dlnpsi_sw"]))
        return out

    def move_jastrow_diff(self, pos: np.ndarray, e: int, rn) -> float:
        """The change of the Jastrow exponent that the sampler uses when electron e of the walker
        at pos (Ne, 3) moves to rn (3,)."""
        pos = _f64(pos)
        rn = _f64(rn)
        return float(lib().osys_move_jastrow_diff(self.h, _p(pos), int(e), _p(rn)))

    def guide_weight(self, pos: np.ndarray, eps: float) -> np.ndarray:
        """Reweighting factors |Psi / Psi_G|^2 (W,) of the guided sampling at positions (W, Ne, 3)."""
        pos = _f64(pos)
        wt = np.zeros(pos.shape[0])
        lib().osys_guide_weight(self.h, pos.shape[0], _p(pos), float(eps), _p(wt), self.nthreads)
        return wt

    def refresh(self, pos: np.ndarray) -> np.ndarray:
        pos = _f64(pos)
        B = np.zeros((pos.shape[0], self.nB))
        lib().osys_refresh(self.h, pos.shape[0], _p(pos), _p(B), self.nthreads)
        return B

    def sample(self, state: dict, n_sweeps: int, sigma: float = 0.3, refresh_k: int = 26, eps: float = 0.0):
        """Advance a sampler state in place. state: pos (W,Ne,3), B (W,nB), wid0, key (k0,k1),
        sweep, counter, nacc (W,), nsing (W,), margin (W,). eps > 0 samples |Psi_G|^2 (guided)."""
        W = state["pos"].shape[0]
        cnt = np.array([state["counter"]], np.int32)
        lib().osys_sample(self.h, W, _p(state["pos"]), _p(state["B"]), state["wid0"], state["key"][0],
                          state["key"][1], state["sweep"], n_sweeps, sigma, refresh_k, _p(cnt, _ip),
                          _p(state["nacc"], _u32p), _p(state["nsing"], _u32p), _p(state["margin"]),
                          self.nthreads, float(eps))
        state["counter"] = int(cnt[0])
        state["sweep"] += n_sweeps

    def new_state(self, pos: np.ndarray, key=(5222, 1), wid0: int = 0) -> dict:
        pos = _f64(pos).copy()
        W = pos.shape[0]
        return {"pos": pos, "B": self.refresh(pos), "wid0": wid0, "key": tuple(int(k) for k in key), "sweep": 0,
                "counter": 0, "nacc": np.zeros(W, np.uint32), "nsing": np.zeros(W, np.uint32),
                "margin": np.full(W, np.inf)}

    def force_refresh(self, state: dict) -> None:
        """The forced re-inversion before a measurement (skipped when already fresh)."""
        if state["counter"] != 0:
            state["B"] = self.refresh(state["pos"])
            state["counter"] = 0
