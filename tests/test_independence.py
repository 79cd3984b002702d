"""The oracle and the CUDA path share no code (CPU, reads the sources): the oracle includes only
standard headers and imports neither the package nor its library; nothing in the package imports,
links or runs the oracle; only the tests, the smoke check and the benchmark's CPU legs name it."""
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]
PKG = ROOT / "paper_2511_05222_gb300"


def test_the_oracle_includes_only_standard_headers():
    src = (ROOT / "oracle" / "vmc_oracle.cpp").read_text()
    includes = re.findall(r'#include\s*[<"]([^>"]+)[>"]', src)
    assert includes and all("/" not in h and not h.endswith((".h", ".cuh")) or h == "omp.h" for h in includes), includes


def test_the_oracle_imports_nothing_of_the_package():
    for f in (ROOT / "oracle").glob("*.py"):
        text = f.read_text()
        assert not re.search(r"^\s*(import|from)\s+(paper_2511_05222_gb300|\.\.)", text, re.M), f
        # the only shared library it loads is its own, built from vmc_oracle.cpp
        assert "libvmcf" not in text, f
        assert text.count("CDLL(") == text.count("ctypes.CDLL(str(build()))"), f


def test_the_package_never_uses_the_oracle():
    for f in list(PKG.rglob("*.py")) + list(PKG.rglob("*.cu")) + list(PKG.rglob("*.cuh")) + list(PKG.rglob("*.h")):
        if "_build" in f.parts:
            continue
        code = f.read_text()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", code, re.M), f
        assert "liboracle" not in code and "vmc_oracle" not in code, f


def test_only_tests_smoke_and_the_benchmark_cpu_legs_name_the_oracle():
    users = []
    for f in ROOT.rglob("*.py"):
        rel = f.relative_to(ROOT)
        if rel.parts[0] in ("tests", "oracle", "_work", "gpurun_out", "baseline") or "_build" in rel.parts:
            continue
        if re.search(r"^\s*(import|from)\s+oracle\b", f.read_text(), re.M):
            users.append(str(rel))
    assert sorted(users) == ["__graft_entry__.py", "bench.py"], users
