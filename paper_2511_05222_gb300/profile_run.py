"""One measured sweep of a workload, for profiler captures of the hot-path kernels.

    python -m paper_2511_05222_gb300.profile_run --workload c9o4h8 --walkers 1024 [--precision mixed|fp64]
        [--group-path] [--jastrow-basis]

Builds the system, creates the walkers (one refresh launch), resets the sums and runs one measured sweep (the
Metropolis kernel, then the measurement kernel, plus the tensor-core sums on the small-system path).
"""
from __future__ import annotations

import argparse

WORKLOADS = {"water": 0, "c2oh6": 1, "c9o4h8": 4}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c9o4h8", choices=sorted(WORKLOADS))
    ap.add_argument("--walkers", type=int, default=1024)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--group-path", action="store_true", help="force the walker-group kernels")
    ap.add_argument("--jastrow-basis", action="store_true",
                    help="add the AO-expanded Jastrow terms (seeded medium Jastrow basis)")
    args = ap.parse_args(argv)
    import torch
    from . import systems as S
    from . import vmcf
    sysx = S.make_system(WORKLOADS[args.workload])
    if args.jastrow_basis:
        sysx = S.with_jastrow_basis(sysx)
    g = vmcf.System(sysx, vmcf.MIXED if args.precision == "mixed" else vmcf.FP64, force_group=args.group_path)
    wk = vmcf.Walkers(g, S.initial_walkers(sysx, args.walkers, seed=1), key=(5222, 4), nblocks=16)
    wk.reset_accumulators(-600.0 if WORKLOADS[args.workload] == 4 else -100.0)
    wk.sample(1, measure=True)
    torch.cuda.synchronize()
    print("ok", wk.counters())
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
