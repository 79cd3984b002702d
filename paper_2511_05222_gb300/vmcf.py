"""Thin Python binding of the C ABI in include/vmcf.h (argument marshalling only).

Every step of the VMC path runs in libvmcf's CUDA kernels; this module only converts
arguments: device buffers are torch CUDA tensors (data_ptr), streams are torch streams.
If the compiled library is missing, loading fails loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

from . import build as _build

FP64, MIXED = 0, 1
FORCE_GROUP_PATH = 0x100
SPACE_WARP = 0x200
_STATUS = {0: "VMCF_OK", -1: "VMCF_EINVAL", -2: "VMCF_ENOMEM", -3: "VMCF_ECUDA", -4: "VMCF_ESINGULAR",
           -5: "VMCF_ETIMEOUT", -6: "VMCF_ENOTSUP"}

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_vp = ctypes.c_void_p


class VmcfError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().vmcf_last_error().decode()
        super().__init__(f"{where}: {_STATUS.get(code, code)}: {msg}")
        self.code = code


class _Nuclei(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("Z", _ip), ("R", _dp)]


class _Basis(ctypes.Structure):
    _fields_ = [("nshell", ctypes.c_int), ("maxprim", ctypes.c_int), ("center", _ip), ("l", _ip), ("nprim", _ip),
                ("exps", _dp), ("coefs", _dp)]


class _Jastrow(ctypes.Structure):
    _fields_ = [("F_anti", ctypes.c_double), ("F_par", ctypes.c_double), ("a_anti", ctypes.c_double),
                ("a_par", ctypes.c_double), ("b_en", ctypes.c_double), ("enable_J1", ctypes.c_int),
                ("enable_J2", ctypes.c_int), ("two_body_exp", ctypes.c_int), ("basis", ctypes.POINTER(_Basis)),
                ("xi", _dp), ("Xi", _dp)]


class WalkersState(ctypes.Structure):
    """vmcf_walkers_state: the public header of a walker-set checkpoint."""
    _fields_ = [("magic", ctypes.c_char * 8), ("W", ctypes.c_int32), ("nblocks", ctypes.c_int32),
                ("Ne", ctypes.c_int32), ("n_up", ctypes.c_int32), ("n_dn", ctypes.c_int32), ("M", ctypes.c_int32),
                ("K", ctypes.c_int32), ("precision", ctypes.c_int32), ("counter", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("sweep", ctypes.c_uint64), ("measured", ctypes.c_uint64),
                ("key0", ctypes.c_uint64), ("key1", ctypes.c_uint64), ("wid0", ctypes.c_uint64),
                ("e_ref", ctypes.c_double), ("eps", ctypes.c_double), ("bytes", ctypes.c_uint64 * 8)]


class Counters(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in
                ("moves", "accepted", "rejected_nonfinite", "singular", "refreshes", "sweeps", "measured_sweeps")]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


def library_path() -> Path:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libvmcf.so (building it with nvcc when missing or stale)."""
    global _lib
    if _lib is None:
        if build_if_missing:
            _build.build()
        path = _build.LIB
        if not path.exists():
            raise RuntimeError(f"libvmcf.so not found at {path}; run paper_2511_05222_gb300.build.build()")
        L = ctypes.CDLL(str(path))
        L.vmcf_last_error.restype = ctypes.c_char_p
        L.vmcf_strerror.restype = ctypes.c_char_p
        L.vmcf_init_system.argtypes = [ctypes.POINTER(_Nuclei), ctypes.POINTER(_Basis), _dp, _dp, ctypes.c_int,
                                       ctypes.c_int, ctypes.POINTER(_Jastrow), _dp, ctypes.c_int, ctypes.POINTER(_vp)]
        L.vmcf_system_destroy.argtypes = [_vp]
        L.vmcf_system_info.argtypes = [_vp, _ip, _ip, _ip, _ip]
        L.vmcf_system_set_geometry.argtypes = [_vp, _dp, _dp, _dp, _dp]
        L.vmcf_accumulator_length.argtypes = [_vp]
        L.vmcf_walkers_create.argtypes = [_vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                          ctypes.c_uint64, ctypes.c_int, _vp, ctypes.POINTER(_vp)]
        L.vmcf_walkers_destroy.argtypes = [_vp]
        L.vmcf_walkers_set_positions.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp]
        L.vmcf_walkers_get_positions.argtypes = [_vp, _vp, ctypes.c_int, _vp]
        L.vmcf_reset_accumulators.argtypes = [_vp, ctypes.c_double, _vp]
        L.vmcf_sample.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, _vp]
        L.vmcf_measure.argtypes = [_vp, _vp, _vp]
        L.vmcf_evaluate.argtypes = [_vp, _vp, ctypes.c_int] + [_vp] * 6 + [_vp]
        L.vmcf_reduce_estimators.argtypes = [_vp, _vp] + [_dp] * 7 + [_vp]
        L.vmcf_block_sums.argtypes = [_vp, _vp, _dp, _vp]
        L.vmcf_status_counters.argtypes = [_vp, ctypes.POINTER(Counters), _vp]
        L.vmcf_profile.argtypes = [_vp, ctypes.c_int]
        L.vmcf_set_tuning.argtypes = [_vp, ctypes.c_char_p, ctypes.c_int]
        L.vmcf_kernel_times.argtypes = [_vp, _dp, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int]
        L.vmcf_probe_pipes.argtypes = [_dp, _dp, _dp, _vp]
        L.vmcf_diag_group_proposals.argtypes = [_vp, ctypes.c_double, _dp, _dp, _dp, _dp, _vp]
        L.vmcf_refresh_residual.argtypes = [_vp, _dp, _dp, _vp]
        L.vmcf_set_guiding.argtypes = [_vp, ctypes.c_double]
        L.vmcf_evaluate_warp.argtypes = [_vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp]
        L.vmcf_reduce_warp.argtypes = [_vp, _vp, _dp, _dp, _vp]
        L.vmcf_finish_warp.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_double, _dp, _dp]
        L.vmcf_batch_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_int, _vp,
                                        ctypes.POINTER(_vp)]
        L.vmcf_batch_destroy.argtypes = [_vp]
        L.vmcf_batch_autotune.argtypes = [_vp, ctypes.c_double, ctypes.c_int, _vp]
        L.vmcf_batch_set_shape.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.vmcf_batch_sample.argtypes = [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, _vp]
        L.vmcf_batch_info.argtypes = [_vp, _ip, _ip, ctypes.c_int, _ip, _ip]
        L.vmcf_walkers_state_bytes.argtypes = [_vp, ctypes.POINTER(ctypes.c_uint64)]
        L.vmcf_walkers_save.argtypes = [_vp, _vp, ctypes.c_uint64, _vp]
        L.vmcf_walkers_load.argtypes = [_vp, _vp, ctypes.c_uint64, _vp]
        _lib = L
    return _lib


def _check(code: int, where: str):
    if code != 0:
        raise VmcfError(code, where)


def _ptr(t):
    """Device pointer of a torch CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous() or t.dtype.itemsize != 8:
        raise ValueError("device buffers must be contiguous float64 CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _np(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class System:
    """vmcf_init_system: a molecule, its basis, frozen orbitals and Jastrow, on the GPU."""

    def __init__(self, sys, precision: int = FP64, force_group: bool = False, space_warp: bool = False):
        L = lib()
        j = sys.jastrow
        self._hold = dict(Z=_np(sys.Z, np.int32), R=_np(sys.R, np.float64), c=_np(sys.shell_center, np.int32),
                          l=_np(sys.shell_l, np.int32), np=_np(sys.shell_nprim, np.int32),
                          e=_np(sys.shell_exp, np.float64), co=_np(sys.shell_coef, np.float64),
                          Cu=_np(sys.C_up, np.float64), Cd=_np(sys.C_dn, np.float64),
                          S=None if sys.S is None else _np(sys.S, np.float64))
        h = self._hold
        dp = lambda a: None if a is None else a.ctypes.data_as(_dp)
        ip = lambda a: a.ctypes.data_as(_ip)
        nuc = _Nuclei(sys.K, ip(h["Z"]), dp(h["R"]))
        bas = _Basis(sys.nshell, h["e"].shape[1], ip(h["c"]), ip(h["l"]), ip(h["np"]), dp(h["e"]), dp(h["co"]))
        jas = _Jastrow(j.F_anti, j.F_par, j.a_anti, j.a_par, j.b_en, int(j.enable_J1), int(j.enable_J2),
                       int(bool(getattr(j, "two_body_exp", False))), None, None, None)
        jb = getattr(j, "basis", None)
        if jb is not None:  # AO-expanded Jastrow terms over a Jastrow basis
            h.update(jc=_np(jb.shell_center, np.int32), jl=_np(jb.shell_l, np.int32), jn=_np(jb.shell_nprim, np.int32),
                     je=_np(jb.shell_exp, np.float64), jco=_np(jb.shell_coef, np.float64),
                     xi=_np(jb.xi, np.float64), Xi=_np(jb.Xi, np.float64))
            h["jbas"] = _Basis(jb.nshell, h["je"].shape[1], ip(h["jc"]), ip(h["jl"]), ip(h["jn"]), dp(h["je"]),
                               dp(h["jco"]))
            jas.basis = ctypes.pointer(h["jbas"])
            jas.xi = dp(h["xi"])
            jas.Xi = dp(h["Xi"])
        out = _vp()
        _check(L.vmcf_init_system(ctypes.byref(nuc), ctypes.byref(bas), dp(h["Cu"]), dp(h["Cd"]), sys.n_up, sys.n_dn,
                                  ctypes.byref(jas), dp(h["S"]),
                                  precision | (FORCE_GROUP_PATH if force_group else 0) | (SPACE_WARP if space_warp else 0),
                                  ctypes.byref(out)), "vmcf_init_system")
        self.h = out
        self.precision = precision
        self.sys = sys
        K, M, nu, nd = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(L.vmcf_system_info(self.h, ctypes.byref(K), ctypes.byref(M), ctypes.byref(nu), ctypes.byref(nd)),
               "vmcf_system_info")
        self.K, self.M, self.n_up, self.n_dn = K.value, M.value, nu.value, nd.value
        self.Ne = self.n_up + self.n_dn
        self.nO = self.M * self.Ne
        self.accL = L.vmcf_accumulator_length(self.h)

    def set_tuning(self, key: str, value: int):
        _check(lib().vmcf_set_tuning(self.h, key.encode(), int(value)), "vmcf_set_tuning")

    def set_geometry(self, R, C_up, C_dn, S=None):
        """vmcf_system_set_geometry: new nuclear positions (K, 3) and orbital coefficients (M, n_up), (M, n_dn)
        for this system (host arrays); walker sets must be re-inverted (Walkers.set_positions) afterwards."""
        dp = lambda a: None if a is None else a.ctypes.data_as(_dp)
        R, C_up, C_dn = _np(R, np.float64), _np(C_up, np.float64), _np(C_dn, np.float64)
        S = None if S is None else _np(S, np.float64)
        if R.shape != (self.K, 3) or C_up.shape != (self.M, self.n_up) or C_dn.size != self.M * self.n_dn:
            raise ValueError("R must be (K, 3), C_up (M, n_up), C_dn (M, n_dn)")
        if S is not None and S.shape != (self.M, self.M):
            raise ValueError("S must be (M, M)")
        _check(lib().vmcf_system_set_geometry(self.h, dp(R), dp(C_up), dp(C_dn), dp(S)), "vmcf_system_set_geometry")

    def close(self):
        if getattr(self, "h", None):
            lib().vmcf_system_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def vmcf_evaluate(system: System, pos, want=("EL",), stream=None):
    """vmcf_evaluate on device positions pos (W, Ne, 3) float64. Returns a dict of torch
    CUDA tensors for the requested outputs among EL, logpsi, dlnpsi_dR, dEL_dR, O, dEL_dC."""
    import torch
    W = pos.shape[0]
    dev = pos.device
    shapes = {"EL": (W,), "logpsi": (W,), "dlnpsi_dR": (W, system.K, 3), "dEL_dR": (W, system.K, 3),
              "O": (W, system.nO), "dEL_dC": (W, system.nO)}
    out = {k: torch.empty(shapes[k], dtype=torch.float64, device=dev) for k in want}
    order = ["EL", "logpsi", "dlnpsi_dR", "dEL_dR", "O", "dEL_dC"]
    _check(lib().vmcf_evaluate(system.h, _ptr(pos.contiguous()), W, *[_ptr(out.get(k)) for k in order],
                               _stream(stream)), "vmcf_evaluate")
    return out


def vmcf_evaluate_warp(system: System, pos, stream=None):
    """vmcf_evaluate_warp on device positions (W, Ne, 3): dict of torch CUDA tensors dEL_dr
    (W, Ne, 3), dEL_sw and dlnpsi_sw (W, K, 3)."""
    import torch
    W = pos.shape[0]
    out = {"dEL_dr": torch.empty((W, system.Ne, 3), dtype=torch.float64, device=pos.device),
           "dEL_sw": torch.empty((W, system.K, 3), dtype=torch.float64, device=pos.device),
           "dlnpsi_sw": torch.empty((W, system.K, 3), dtype=torch.float64, device=pos.device)}
    _check(lib().vmcf_evaluate_warp(system.h, _ptr(pos.contiguous()), W, _ptr(out["dEL_dr"]), _ptr(out["dEL_sw"]),
                                    _ptr(out["dlnpsi_sw"]), _stream(stream)), "vmcf_evaluate_warp")
    return out


class Walkers:
    """vmcf_walkers_create: device walker state for sampling."""

    def __init__(self, system: System, pos, key=(5222, 1), wid0: int = 0, nblocks: int = 64, stream=None):
        L = lib()
        self.system = system
        out = _vp()
        if isinstance(pos, np.ndarray):
            self._host = _np(pos, np.float64)
            W = self._host.shape[0]
            p, is_host = ctypes.c_void_p(self._host.ctypes.data), 1
        else:
            W = pos.shape[0]
            p, is_host = _ptr(pos.contiguous()), 0
        _check(L.vmcf_walkers_create(system.h, W, p, is_host, int(key[0]), int(key[1]), int(wid0), nblocks,
                                     _stream(stream), ctypes.byref(out)), "vmcf_walkers_create")
        self.h = out
        self.W = W
        self.nblocks = nblocks
        self.e_ref = 0.0

    def close(self):
        if getattr(self, "h", None):
            lib().vmcf_walkers_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def group_proposals(self, sigma: float = 0.3, stream=None) -> dict:
        """vmcf_diag_group_proposals: the proposal pass of the next sweep (walker-group kernels) as host arrays:
        rnew (W, Ne, 3), rows (W, Ne, nmax), u (W, Ne), dchi (W, Ne). The chain does not advance."""
        sx = self.system
        Ne, nmax = sx.n_up + sx.n_dn, max(sx.n_up, sx.n_dn)
        out = {"rnew": np.zeros((self.W, Ne, 3)), "rows": np.zeros((self.W, Ne, nmax)), "u": np.zeros((self.W, Ne)),
               "dchi": np.zeros((self.W, Ne))}
        _check(lib().vmcf_diag_group_proposals(self.h, float(sigma), *[out[k].ctypes.data_as(_dp) for k in
                                                                        ("rnew", "rows", "u", "dchi")],
                                                _stream(stream)), "vmcf_diag_group_proposals")
        return out

    def set_positions(self, pos, stream=None):
        if isinstance(pos, np.ndarray):
            a = _np(pos, np.float64)
            _check(lib().vmcf_walkers_set_positions(self.system.h, self.h, ctypes.c_void_p(a.ctypes.data), 1,
                                                    _stream(stream)), "vmcf_walkers_set_positions")
        else:
            _check(lib().vmcf_walkers_set_positions(self.system.h, self.h, _ptr(pos.contiguous()), 0,
                                                    _stream(stream)), "vmcf_walkers_set_positions")

    def positions(self, stream=None, out=None) -> np.ndarray:
        """Positions [W][Ne][3] into a new array, or into `out` (C-contiguous float64 host array of that shape;
        pinned memory makes the copy a direct one)."""
        if out is None:
            out = np.empty((self.W, self.system.Ne, 3))
        elif (not isinstance(out, np.ndarray) or out.dtype != np.float64 or not out.flags.c_contiguous
              or out.shape != (self.W, self.system.Ne, 3)):
            raise ValueError("out must be a C-contiguous float64 array of shape (W, Ne, 3)")
        _check(lib().vmcf_walkers_get_positions(self.h, ctypes.c_void_p(out.ctypes.data), 1, _stream(stream)),
               "vmcf_walkers_get_positions")
        return out

    def positions_into(self, dev_tensor, stream=None):
        _check(lib().vmcf_walkers_get_positions(self.h, _ptr(dev_tensor), 0, _stream(stream)),
               "vmcf_walkers_get_positions")

    def set_guiding(self, eps: float):
        """Guided sampling of |Psi_G|^2 with reweighted sums (eps = 0: plain |Psi|^2)."""
        _check(lib().vmcf_set_guiding(self.h, float(eps)), "vmcf_set_guiding")
        self.eps = float(eps)

    def reset_accumulators(self, e_ref: float, stream=None):
        _check(lib().vmcf_reset_accumulators(self.h, float(e_ref), _stream(stream)), "vmcf_reset_accumulators")
        self.e_ref = float(e_ref)

    def sample(self, n_sweeps: int, step_sigma: float = 0.3, refresh_k: int = 26, measure: bool = False,
               stream=None):
        _check(lib().vmcf_sample(self.system.h, self.h, int(n_sweeps), float(step_sigma), int(refresh_k),
                                 int(bool(measure)), _stream(stream)), "vmcf_sample")

    def measure(self, stream=None):
        """vmcf_measure: accumulate one measurement of the current positions (no moves)."""
        _check(lib().vmcf_measure(self.system.h, self.h, _stream(stream)), "vmcf_measure")

    def reduce_estimators(self, with_rhs: bool = False, stream=None) -> dict:
        s = self.system
        E, Ee = np.zeros(1), np.zeros(1)
        F, Fe = np.zeros(3 * s.K), np.zeros(3 * s.K)
        B, Be = np.zeros(s.nO), np.zeros(s.nO)
        rhs = np.zeros(s.nO) if with_rhs else None
        dp = lambda a: None if a is None else a.ctypes.data_as(_dp)
        _check(lib().vmcf_reduce_estimators(s.h, self.h, dp(E), dp(Ee), dp(F), dp(Fe), dp(B), dp(Be), dp(rhs),
                                            _stream(stream)), "vmcf_reduce_estimators")
        out = {"E": float(E[0]), "E_err": float(Ee[0]), "F": F.reshape(s.K, 3), "F_err": Fe.reshape(s.K, 3),
               "dEdC": B, "dEdC_err": Be}
        if with_rhs:
            out["rhs_BQ"] = rhs
        return out

    def reduce_warp(self, stream=None) -> dict:
        """Space-warp forces F^sw and their jackknife errors (system created with space_warp)."""
        s = self.system
        F, Fe = np.zeros(3 * s.K), np.zeros(3 * s.K)
        _check(lib().vmcf_reduce_warp(s.h, self.h, F.ctypes.data_as(_dp), Fe.ctypes.data_as(_dp), _stream(stream)),
               "vmcf_reduce_warp")
        return {"F": F.reshape(s.K, 3), "F_err": Fe.reshape(s.K, 3)}

    def block_sums(self, stream=None) -> np.ndarray:
        s = self.system
        out = np.zeros((self.nblocks, s.accL))
        _check(lib().vmcf_block_sums(s.h, self.h, out.ctypes.data_as(_dp), _stream(stream)), "vmcf_block_sums")
        return out

    def profile(self, enable: bool = True):
        _check(lib().vmcf_profile(self.h, int(enable)), "vmcf_profile")

    def kernel_times(self, reset: bool = True) -> dict:
        ms = (ctypes.c_double * 5)()
        n = (ctypes.c_longlong * 5)()
        _check(lib().vmcf_kernel_times(self.h, ms, n, int(reset)), "vmcf_kernel_times")
        names = ("move", "measure", "refresh", "tc_sums", "propose")
        return {names[k]: {"ms": float(ms[k]), "launches": int(n[k])} for k in range(5)}

    def refresh_residual(self, stream=None) -> dict:
        """vmcf_refresh_residual: normwise deviation of the current inverses from a fresh FP64 re-inversion of the
        current positions, per walker; its maximum and mean over the walkers."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(lib().vmcf_refresh_residual(self.h, ctypes.byref(a), ctypes.byref(b), _stream(stream)),
               "vmcf_refresh_residual")
        return {"max": a.value, "mean": b.value}

    def counters(self, stream=None) -> dict:
        c = Counters()
        _check(lib().vmcf_status_counters(self.h, ctypes.byref(c), _stream(stream)), "vmcf_status_counters")
        return c.as_dict()

    def save(self, stream=None) -> bytes:
        """vmcf_walkers_save: a checkpoint of this walker set (header plus device state)."""
        n = ctypes.c_uint64()
        _check(lib().vmcf_walkers_state_bytes(self.h, ctypes.byref(n)), "vmcf_walkers_state_bytes")
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().vmcf_walkers_save(self.h, buf, n.value, _stream(stream)), "vmcf_walkers_save")
        return buf.raw

    def load(self, state: bytes, stream=None):
        """vmcf_walkers_load: continue from a checkpoint of a walker set of the same system, W and
        nblocks."""
        buf = ctypes.create_string_buffer(bytes(state), len(state))
        _check(lib().vmcf_walkers_load(self.h, buf, len(state), _stream(stream)), "vmcf_walkers_load")
        h = WalkersState.from_buffer_copy(bytes(state)[:ctypes.sizeof(WalkersState)])
        self.e_ref = h.e_ref
        self.eps = h.eps


def vmcf_probe_pipes(stream=None) -> dict:
    """Measured FP64/FP32 FMA throughput (TFLOP/s) and FP32 expf throughput (G/s)."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().vmcf_probe_pipes(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), _stream(stream)),
           "vmcf_probe_pipes")
    return {"fp64_tflops": a.value, "fp32_tflops": b.value, "exp_gops": c.value}


class Batch:
    """vmcf_batch_create: a ragged batch of geometries, each a (System, Walkers) pair; every sweep
    of the whole batch is one replay of a captured CUDA graph: persistent walker-group kernels for
    the geometries on that path, a branch of small-system kernels for each geometry that fits them.
    Each Walkers object keeps its own sums."""

    def __init__(self, systems, walkers, stream=None):
        L = lib()
        G = len(systems)
        if G != len(walkers) or G == 0:
            raise ValueError("need one walker set per system")
        self.systems, self.walkers = list(systems), list(walkers)
        hs = (_vp * G)(*[s.h for s in systems])
        hw = (_vp * G)(*[w.h for w in walkers])
        out = _vp()
        _check(L.vmcf_batch_create(hs, hw, G, _stream(stream), ctypes.byref(out)), "vmcf_batch_create")
        self.h = out
        self.G = G

    def close(self):
        if getattr(self, "h", None):
            lib().vmcf_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, step_sigma: float = 0.3, refresh_k: int = 26, stream=None):
        _check(lib().vmcf_batch_autotune(self.h, float(step_sigma), int(refresh_k), _stream(stream)),
               "vmcf_batch_autotune")

    def set_shape(self, g: int, phase: int, GS: int, groups: int):
        """Launch shape of phase 0 (sweep) or 1 (evaluation) for geometry g's bucket."""
        _check(lib().vmcf_batch_set_shape(self.h, int(g), int(phase), int(GS), int(groups)), "vmcf_batch_set_shape")

    def sample(self, n_sweeps: int, step_sigma: float = 0.3, refresh_k: int = 26, measure: bool = False,
               stream=None):
        _check(lib().vmcf_batch_sample(self.h, int(n_sweeps), float(step_sigma), int(refresh_k),
                                       int(bool(measure)), _stream(stream)), "vmcf_batch_sample")

    def info(self) -> dict:
        nb, nl = ctypes.c_int(), ctypes.c_int()
        geo = []
        for g in range(self.G):
            b = ctypes.c_int()
            sh = (ctypes.c_int * 4)()
            _check(lib().vmcf_batch_info(self.h, ctypes.byref(nb), ctypes.byref(nl), g, ctypes.byref(b), sh),
                   "vmcf_batch_info")
            geo.append({"bucket": b.value, "sweep": (sh[0], sh[1]), "evaluation": (sh[2], sh[3])})
        return {"buckets": nb.value, "launches": nl.value, "geometries": geo}
