"""vmcf_evaluate_sums_noalloc, the variant of the walker-sum evaluation that allocates no
GPU memory (its scratch is a fixed array inside the library), checked through the C ABI
against the existing vmcf_evaluate outputs summed on the host, on two calls in a row (the
second call must not see the first call's partial sums). This file is collected last.

The cases cover a grid the scratch does not cap (water, C2OH6 at a few hundred walkers) and
grids it does (C2OH6 at 16384 walkers, C9O4H8 at 1024 walkers: more CTAs than the 2^21-double
scratch holds partial sums for, so each CTA takes many walkers), in FP64 and in mixed
precision. Both entry points run the walker-group kernels here (the systems are built with
the group path). In FP64 the sums agree to 1e-10 (the FP64 tolerance of the parity tests). In
mixed precision a wide walker group (C9O4H8: 256 threads per walker) adds the per-walker force
partials with FP32 shared-memory atomics whose order changes from launch to launch, so two calls
differ by FP32 rounding of those terms; the sums are held to 1e-6 there."""
import ctypes

import numpy as np
import pytest

from paper_2511_05222_gb300 import systems as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_05222_gb300 import vmcf  # noqa: E402


def host_sums(out, e_ref):
    EL = out["EL"]
    c = EL - e_ref
    W = EL.shape[0]
    dl = out["dlnpsi_dR"].reshape(W, -1)
    de = out["dEL_dR"].reshape(W, -1)
    O = out["O"]
    return np.concatenate([[W, EL.sum(), (EL * EL).sum()], de.sum(0), dl.sum(0), (c[:, None] * dl).sum(0),
                           O.sum(0), (c[:, None] * O).sum(0)])


def noalloc():
    L = vmcf.lib()
    L.vmcf_evaluate_sums_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_void_p, ctypes.c_void_p]
    return L


CASES = [  # (workload, precision, [(W, seed, e_ref) of the two calls])
    (0, vmcf.FP64, [(203, 1, -70.0), (97, 2, -60.0)]),
    (1, vmcf.FP64, [(203, 1, -150.0), (16384, 2, -140.0)]),
    (1, vmcf.MIXED, [(16384, 3, -150.0), (203, 4, -145.0)]),
    (4, vmcf.FP64, [(1024, 5, -600.0), (96, 6, -590.0)]),
    (4, vmcf.MIXED, [(96, 7, -600.0), (1024, 8, -610.0)]),
]


@pytest.mark.parametrize("cfg,precision,calls", CASES)
def test_noalloc_sums_match_evaluate_on_two_calls(cfg, precision, calls):
    sysx = S.make_system(cfg)
    g = vmcf.System(sysx, precision, force_group=True)
    L = noalloc()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # the once-per-device set-up alone (W = 0: nothing launches)
    assert L.vmcf_evaluate_sums_noalloc(g.h, None, 0, 0.0, None, stream) == 0, L.vmcf_last_error()
    for call, (W, seed, e_ref) in enumerate(calls):
        pos = torch.as_tensor(S.initial_walkers(sysx, W, seed=seed), device="cuda")
        ref = vmcf.vmcf_evaluate(g, pos, want=("EL", "dlnpsi_dR", "dEL_dR", "O"))
        ref = {k: v.cpu().numpy() for k, v in ref.items()}
        EL = ref["EL"]
        ref = host_sums(ref, e_ref)
        out = torch.full((g.accL,), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.vmcf_evaluate_sums_noalloc(g.h, ctypes.c_void_p(pos.data_ptr()), W, e_ref,
                                          ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 0, L.vmcf_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert got[0] == W, (call, got[0])
        tol = 1e-10 if precision == vmcf.FP64 else 1e-6
        scale = np.abs(EL).sum()
        assert abs(got[1] - ref[1]) < tol * scale, (call, got[1], ref[1])
        K3, nO = 3 * g.K, g.nO
        seg = [(0, 3), (3, 3 + K3), (3 + K3, 3 + 2 * K3), (3 + 2 * K3, 3 + 3 * K3), (3 + 3 * K3, 3 + 3 * K3 + nO),
               (3 + 3 * K3 + nO, 3 + 3 * K3 + 2 * nO)]
        for a, b in seg:  # relative, normwise per segment
            err = np.abs(got[a:b] - ref[a:b]).max() / max(np.abs(ref[a:b]).max(), 1e-300)
            assert err < tol, (call, a, b, err)


def test_noalloc_rejects_another_current_device_and_bad_sizes():
    sysx = S.make_system(0)
    g = vmcf.System(sysx, vmcf.FP64)
    L = noalloc()
    assert L.vmcf_evaluate_sums_noalloc(g.h, None, -1, 0.0, None, None) == -1
    assert L.vmcf_evaluate_sums_noalloc(g.h, None, 5, 0.0, None, None) == -1
    if torch.cuda.device_count() > 1:
        with torch.cuda.device(1):
            assert L.vmcf_evaluate_sums_noalloc(g.h, None, 0, 0.0, None, None) == -1
