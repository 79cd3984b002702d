"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every entry point
that include/*.h declares (no compute call is made here)."""
import re
from pathlib import Path

from paper_2511_05222_gb300 import vmcf

HEADER = Path(__file__).resolve().parents[1] / "include" / "vmcf.h"


def test_library_exports_every_declared_symbol():
    L = vmcf.lib()
    declared = set()
    for h in sorted(HEADER.parent.glob("*.h")):
        declared |= set(re.findall(r"\b(vmcf_[a-z_]+)\s*\(", h.read_text()))
    assert len(declared) >= 14
    assert {"vmcf_probe_pipes", "vmcf_kernel_times", "vmcf_evaluate_sums_noalloc"} <= declared
    missing = [n for n in sorted(declared) if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings_and_error_text():
    L = vmcf.lib()
    assert L.vmcf_strerror(0) == b"ok"
    assert L.vmcf_strerror(-4) == b"singular Slater matrix"
    assert L.vmcf_strerror(12345) == b"unknown status"


def test_invalid_arguments_are_rejected_without_touching_the_gpu():
    import ctypes
    L = vmcf.lib()
    out = ctypes.c_void_p()
    # NULL inputs: rejected before any CUDA call
    rc = L.vmcf_init_system(None, None, None, None, 1, 1, None, None, 0, ctypes.byref(out))
    assert rc == -1 and out.value is None
    assert b"NULL" in L.vmcf_last_error()
    assert L.vmcf_sample(None, None, 1, 0.3, 26, 0, None) == -1
    assert L.vmcf_evaluate(None, None, 1, None, None, None, None, None, None, None) == -1


def test_checkpoint_header_layout_matches_the_c_struct(tmp_path):
    """The ctypes mirror of vmcf_walkers_state has the C struct's size and field offsets."""
    import ctypes
    import subprocess

    fields = [f[0] for f in vmcf.WalkersState._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "vmcf.h"\nint main(void) {\n'
                   '  printf("%zu\\n", sizeof(vmcf_walkers_state));\n' +
                   "".join(f'  printf("%zu\\n", offsetof(vmcf_walkers_state, {f}));\n' for f in fields) +
                   "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", str(HEADER.parent), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got[0] == ctypes.sizeof(vmcf.WalkersState)
    assert got[1:] == [getattr(vmcf.WalkersState, f).offset for f in fields]


def test_a_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without libvmcf.so the binding raises instead of computing anything."""
    import pytest

    monkeypatch.setattr(vmcf, "_lib", None)
    monkeypatch.setattr(vmcf._build, "LIB", tmp_path / "libvmcf.so")
    with pytest.raises(RuntimeError, match="libvmcf.so not found"):
        vmcf.lib(build_if_missing=False)
