#!/usr/bin/env python
"""Throughput of the VMC hot path: walker-evaluations per second.

A step is one measured sweep over all walkers of the workload: every electron of every
walker attempts one Metropolis move (Sherman-Morrison update on acceptance), the inverses
are rebuilt in FP64, and E_L, d ln Psi/dR, dE_L/dR and O are evaluated and accumulated into
the walker sums behind E, the forces and dE/dC. value = walkers x steps / device time.

Default workload: C2OH6 (26 electrons, 72 AOs, 9 nuclei), 16384 walkers per GPU, Gaussian
step 0.3 bohr, re-inversion every 26 moves, mixed precision; the FP64 GPU path is timed on
the same workload for comparison. Inputs are synthetic (seeded generator). L2 is flushed
between timed steps (the walker state, 32 MB, would otherwise stay in the 129 MB L2).
The headline steps are timed without per-kernel instrumentation; the kernel split and the
roofline of the dominant kernel come from a second timed region of the same length with an
event pair around every kernel. The default line also carries a "c9o4h8" block: the
94-electron workload (C9O4H8, 222 AOs, 65536 walkers per GPU) measured the same way, mixed and
FP64, and a "ragged64" block: the ragged batch of 64 geometries (10-94 electrons, 148608 walkers)
sampled together, one captured graph per sweep (--no-large skips both).

--impl reference times the CPU oracle (the plain FP64 C++ reference implementation) on
the host cores, on a bounded sample of the same workload.
Multi-GPU: launched by torch.distributed.run, one process per GPU; each rank owns its own
walkers (weak scaling, no data-path collective); the timed region is bracketed by barriers
and the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

WORKLOADS = {
    "c2oh6": dict(cfg=1, walkers=16384, name="C2OH6 all-electron, 26 e-, 72 AOs, 9 nuclei"),
    "water": dict(cfg=0, walkers=1024, name="H2O all-electron, 10 e-, 24 AOs, 3 nuclei"),
    "c9o4h8": dict(cfg=4, walkers=65536, name="C9O4H8 all-electron, 94 e-, 222 AOs, 21 nuclei"),
    "ragged64": dict(cfg=3, walkers=0, name="ragged batch: 64 covalent-walk H/C/O molecules, 3-21 nuclei, "
                                           "10-94 e-, 24-212 AOs, 512-4096 walkers each"),
}
METRIC = "walker-evals/s (E_L+forces+dE/dC) at 26 e⁻, mixed vs FP64 GPU; % of roofline"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return int(os.environ.get("RANK", "0")), ws, int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """SM clocks and throttle reasons sampled in the background during a timed region: through the
    driver's NVML library every 10 ms (read-only queries), else nvidia-smi every 200 ms."""
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # nvmlClocksEventReason bits (nvml.h): SwPowerCap, HwSlowdown, SwThermalSlowdown, HwThermalSlowdown
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}

    def __init__(self, index: int, period_s: float = 0.01):
        self.index = index
        self.period = period_s
        self.lines: list[str] = []
        self.samples: list[tuple[float, float, int]] = []
        self.proc = None
        self.th = None
        self.stop_ev = threading.Event()
        self.source = None

    def _nvml(self):
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            return None
        h = ctypes.c_void_p()
        bus = None
        try:
            import torch
            p = torch.cuda.get_device_properties(self.index)
            bus = "%08x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
        except Exception:
            bus = None
        if bus is None or lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)) != 0:
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index), ctypes.byref(h)) != 0:
                return None
        reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        return lib, h, reasons

    def _poll(self, lib, h, reasons):
        import ctypes
        cur, mx, r = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        while not self.stop_ev.is_set():
            if (lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(cur)) == 0 and      # NVML_CLOCK_SM
                    lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0 and
                    reasons(h, ctypes.byref(r)) == 0):
                self.samples.append((float(cur.value), float(mx.value), int(r.value)))
            self.stop_ev.wait(self.period)

    def __enter__(self):
        try:
            nv = self._nvml()
        except (OSError, AttributeError):
            nv = None
        if nv is not None:
            self.source = "nvml, every %g ms" % (self.period * 1e3)
            self.th = threading.Thread(target=self._poll, args=nv, daemon=True)
            self.th.start()
            return self
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
            self.source = "nvidia-smi, every 200 ms"
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        self.stop_ev.set()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        elif self.th is not None:
            self.th.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], [], set()
        for c, m, r in self.samples:
            sm.append(c)
            mx.append(m)
            reasons.update(n for n, b in self.BITS.items() if r & b)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 6:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "source": self.source}


def oracle_steps(sysx, walkers: int, budget_s: float, max_s: float, key=(5222, 1)):
    """Time the FP64 CPU oracle on `walkers` walkers of the workload: equilibrate briefly,
    then measured sweeps (sweep + re-inversion + evaluation + walker sums) until budget_s."""
    import oracle
    from oracle import estimators
    from paper_2511_05222_gb300 import systems as S
    o = oracle.Oracle(sysx)
    st = o.new_state(S.initial_walkers(sysx, walkers, seed=99), key=key)
    o.sample(st, 2)
    nb = 8
    sums = estimators.new_sums(nb, sysx.K, o.nO)
    blk = np.arange(walkers) * nb // walkers
    t0 = time.perf_counter()
    steps, per = 0, []
    while True:
        t1 = time.perf_counter()
        o.sample(st, 1)
        o.force_refresh(st)
        out = o.eval(st["pos"], want=("EL", "dlnpsi_dR", "dEL_dR", "O"))
        estimators.accumulate(sums, blk, out["EL"], out["dlnpsi_dR"], out["dEL_dR"], out["O"], -150.0)
        per.append(time.perf_counter() - t1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or el + per[-1] > max_s:
            break
    return walkers * steps / sum(per), steps, sum(per)


ROOT = os.path.dirname(os.path.abspath(__file__))


def measure_source_sha1() -> str:
    """Hash of the measurement kernel's source (its function text and the shared device header)."""
    import hashlib
    ks = open(os.path.join(ROOT, "paper_2511_05222_gb300/csrc/kernels_small.cuh")).read()
    a = ks.index("template <typename T, int NM, bool JB>\n__global__ void __launch_bounds__(256, 2) measure_small(")
    b = ks.index("// Layout conversion between the ABI")
    dev = open(os.path.join(ROOT, "paper_2511_05222_gb300/csrc/vmcf_device.cuh")).read()
    return hashlib.sha1((ks[a:b] + dev).encode()).hexdigest()


def profiled_traffic():
    """DRAM bytes per launch of the measurement kernel from the committed ncu summary, or None
    when the kernel source changed since it was captured."""
    try:
        txt = open(os.path.join(ROOT, "profiles/measure_small_c2oh6.md")).read()
    except OSError:
        return None
    import re
    m = re.search(r"source-sha1: ([0-9a-f]+)", txt)
    r = re.search(r"\| DRAM read \| ([0-9.]+) Mbyte", txt)
    w = re.search(r"\| DRAM write \| ([0-9.]+) (K|M)byte", txt)
    if not (m and r and w) or m.group(1) != measure_source_sha1():
        return None
    return float(r.group(1)) * 1e6 + float(w.group(1)) * (1e3 if w.group(2) == "K" else 1e6)


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def run_reference(args, wl):
    rank, ws, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2511_05222_gb300 import systems as S
    sysx = S.make_system(wl["cfg"])
    sample_w = 128 if wl["cfg"] != 4 else 8
    vals = []
    for _ in range(args.warmup):
        oracle_steps(sysx, sample_w, 0.0, 1e9)
    tot_w, tot_t = 0, 0.0
    for _ in range(args.steps):
        v, n, t = oracle_steps(sysx, sample_w, 0.0, 1e9)
        vals.append(v)
        tot_w += sample_w * n
        tot_t += t
    value = tot_w / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "walker-evals/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "walkers_per_step": sample_w, "precision": "fp64 (CPU oracle)"},
            "cpu_baseline": {"value": value, "unit": "walker-evals/s", "cores": cores(), "kind": "oracle",
                             "sample": f"{sample_w} walkers x 1 measured sweep per step"},
            "e2e": {"value": value, "unit": "walker-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def shard_geometries(plan, ws):
    """Geometries per rank: longest-processing-time-first by N_e^3 x W."""
    load = [0.0] * ws
    own = [[] for _ in range(ws)]
    for g in sorted(range(len(plan)), key=lambda g: -(sum(plan[g][0]) ** 3) * plan[g][1]):
        r = min(range(ws), key=lambda r: load[r])
        own[r].append(g)
        load[r] += sum(plan[g][0]) ** 3 * plan[g][1]
    return [sorted(o) for o in own]


def run_ragged(args, wl, embedded=False):
    """One step = one measured sweep of every geometry of the ragged batch, as one replay of
    the batch's captured graph (persistent kernels, autotuned launch shapes). embedded: called
    from the default measurement (process group and device already set up); the line is
    returned instead of printed."""
    import torch
    from paper_2511_05222_gb300 import systems as S
    from paper_2511_05222_gb300 import vmcf, workmodel

    rank, ws, local = dist_env()
    if ws > 1 and not embedded:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    plan = S.ragged_batch_plan(64)
    mine = shard_geometries(plan, ws)[rank]
    geos = S.make_ragged_batch(64, only=set(mine))
    systems = [vmcf.System(sx, vmcf.MIXED) for sx, _ in geos]  # small geometries on the small-system kernels
    walkers = [vmcf.Walkers(systems[i], S.initial_walkers(sx, W, seed=g), key=(5222, 3000 + g), nblocks=64,
                            stream=stream) for i, ((sx, W), g) in enumerate(zip(geos, mine))]
    batch = vmcf.Batch(systems, walkers, stream=stream)
    batch.sample(max(1, args.equil // 2), 0.3, 26, measure=False, stream=stream)
    batch.autotune(0.3, 26, stream=stream)
    for w in walkers:  # E_ref: each geometry's mean local energy after equilibration
        w.reset_accumulators(0.0, stream=stream)
        w.measure(stream=stream)
        w.reset_accumulators(w.reduce_estimators(stream=stream)["E"], stream=stream)
    for _ in range(args.warmup):
        batch.sample(1, 0.3, 26, measure=True, stream=stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    barrier()
    with ClockSampler(local) as clk:
        for a, b in ev:
            flush.fill_(1.0)
            a.record(stream)
            batch.sample(1, 0.3, 26, measure=True, stream=stream)
            b.record(stream)
        barrier()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    if ws > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    total_w = sum(W for _, W in plan)
    value = total_w * args.steps / (ms * 1e-3)
    peaks = vmcf.vmcf_probe_pipes(stream=stream)
    t_roof, acc_n, acc_d = 0.0, 0, 0
    for (sx, W), w, sy in zip(geos, walkers, systems):
        c = w.counters(stream=stream)
        acc_n += c["accepted"]
        acc_d += c["moves"]
        wk = workmodel.per_walker_eval(sx.K, sy.M, sx.n_up, sx.n_dn, int(sx.shell_nprim.sum()),
                                       c["accepted"] / max(1, c["moves"]))
        t_roof += W * workmodel.roofline_time(wk["total"], peaks)[1]
    info = batch.info()
    shapes = {ph: sorted({gi[ph] for gi in info["geometries"]}) for ph in ("sweep", "evaluation")}
    line = {"metric": METRIC, "value": value, "unit": "walker-evals/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": wl["name"], "geometries": len(plan), "walkers_total": total_w,
                       "geometries_per_rank": len(mine), "step_sigma": 0.3, "refresh_every": 26,
                       "precision": "mixed (FP32 + FP64 inverse/ratio/sums)",
                       "l2": "flushed (256 MB write) between timed steps",
                       "buckets": info["buckets"], "persistent_kernels_per_sweep": info["launches"],
                       "launch_shapes": {ph: [f"{a}x{b}" for a, b in v] for ph, v in shapes.items()}},
            "roofline": {"bound": "alu", "pipe": "whole step, per geometry", "frac": t_roof * ws / (ms * 1e-3 / args.steps)
                         if ws == 1 else None, "peak_source": "measured in this run by vmcf_probe_pipes"},
            "gpu_launches": args.steps * (info["launches"] + 1), "clocks": clk.summary(),
            "acceptance": acc_n / max(1, acc_d)}
    if embedded:
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="vmcf", choices=["vmcf", "reference"])
    ap.add_argument("--workload", default="c2oh6", choices=sorted(WORKLOADS))
    ap.add_argument("--walkers", type=int, default=0, help="walkers per GPU (default: the workload's)")
    ap.add_argument("--equil", type=int, default=10, help="unmeasured sweeps before the warm-up steps")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                    help="precision of the headline measurement (default mixed)")
    ap.add_argument("--group-path", action="store_true", help="run a small system on the walker-group kernels")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 GPU comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end measurement")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the C9O4H8 (94 e-, 65536 walkers) block of the default line")
    ap.add_argument("--jastrow-basis", action="store_true",
                    help="add the AO-expanded Jastrow terms (seeded medium Jastrow basis) to the workload")
    ap.add_argument("--tuning", action="append", default=[], metavar="KEY=VALUE",
                    help="vmcf_set_tuning on the measured system, e.g. tensor_core_rows=0 (repeatable)")
    args = ap.parse_args()
    tunings = [(kv.split("=")[0], int(kv.split("=")[1])) for kv in args.tuning]
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl)
    if args.workload == "ragged64":
        return run_ragged(args, wl)

    import torch
    from paper_2511_05222_gb300 import systems as S
    from paper_2511_05222_gb300 import vmcf, workmodel

    rank, ws, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    nb = 64

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    def max_over_ranks(x: float) -> float:
        if ws == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2

    def timed_steps(wk, K, profile=False):
        """K measured sweeps, each bracketed by CUDA events on the launching stream, L2 flushed
        before each. With profile, the library also records an event pair around every kernel it
        launches (a second timed region, used only for the per-kernel split)."""
        if profile:
            wk.kernel_times(reset=True)
            wk.profile(True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        barrier()
        for a, b in ev:
            flush.fill_(1.0)
            a.record(stream)
            wk.sample(1, 0.3, 26, measure=True, stream=stream)
            b.record(stream)
        barrier()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        kt = None
        if profile:
            kt = wk.kernel_times(reset=True)
            wk.profile(False)
        return ms, kt

    peaks = vmcf.vmcf_probe_pipes(stream=stream)

    def workload_line(sysx, W, steps, warmup, fp64_steps, jb=None, prec=vmcf.MIXED, group=False, seed=0):
        """Headline measurement of one workload: the precision's walker-evals/s over `steps` timed
        sweeps without instrumentation, then the same number of sweeps with per-kernel events for
        the kernel split and the roofline of the dominant kernel; the FP64 GPU path on the same
        (equilibrated) configurations."""
        pos0 = S.initial_walkers(sysx, W, seed=seed)
        g = vmcf.System(sysx, prec, force_group=group)
        for k, v in tunings:
            g.set_tuning(k, v)
        wk = vmcf.Walkers(g, pos0, key=(5222, 1), wid0=rank * W, nblocks=nb, stream=stream)
        wk.sample(args.equil, 0.3, 26, measure=False, stream=stream)
        wk.reset_accumulators(0.0, stream=stream)
        wk.measure(stream=stream)  # E_ref: the mean local energy after equilibration
        e_ref = wk.reduce_estimators(stream=stream)["E"]
        wk.reset_accumulators(e_ref, stream=stream)
        for _ in range(warmup):
            wk.sample(1, 0.3, 26, measure=True, stream=stream)
        with ClockSampler(local) as clk:
            ms, _ = timed_steps(wk, steps)
        ms = max_over_ranks(ms)
        ms_prof, kt = timed_steps(wk, steps, profile=True)
        value = ws * W * steps / (ms * 1e-3)
        cnt = wk.counters(stream=stream)
        acc = cnt["accepted"] / max(1, cnt["moves"])
        est = wk.reduce_estimators(stream=stream)
        work = workmodel.per_walker_eval(sysx.K, g.M, sysx.n_up, sysx.n_dn, int(sysx.shell_nprim.sum()), acc,
                                         jb.MJ if jb else 0, int(jb.shell_nprim.sum()) if jb else 0)
        # the work model's "move" covers a sweep's proposals and moves together
        ktw = dict(kt, move={"ms": kt["move"]["ms"] + kt["propose"]["ms"], "launches": kt["move"]["launches"]})
        dom = max(("move", "measure"), key=lambda k: ktw[k]["ms"])
        t_launch = ktw[dom]["ms"] / max(1, ktw[dom]["launches"]) * 1e-3
        bound, _ = workmodel.roofline_time(work[dom], peaks)
        pipe_flops = {"fp32": work[dom]["fp32"], "fp64": work[dom]["fp64"], "sfu": work[dom]["exp"]}[bound]
        peak = {"fp32": peaks["fp32_tflops"], "fp64": peaks["fp64_tflops"], "sfu": peaks["exp_gops"] / 1e3}[bound]
        achieved = pipe_flops * W / t_launch / 1e12
        # the one-warp-per-walker kernel family, else walker groups (32 threads up to 24 orbitals per spin)
        small = sysx.Ne <= 32 and max(sysx.n_up, sysx.n_dn) <= 16 and not group
        wide = max(sysx.n_up, sysx.n_dn) > 24
        jbf = "1" if jb else "0"  # walker-group kernels: instance with (1) or without (0) the AO-expanded Jastrow terms
        nmx = max(sysx.n_up, sysx.n_dn)
        nm = 8 if nmx <= 8 else (14 if nmx <= 14 else 16)  # register-row width of the one-warp-per-walker kernels
        tn = "float" if prec == vmcf.MIXED else "double"
        kname = ({"move": f"move_small<{tn}, {nm}, 2, 0>",
                  "measure": f"measure_small<{tn}, {nm}, {jbf}>"}[dom] if small else
                 {"move": f"move_kernel<{tn}, {128 if wide else 32}, {jbf}>",
                  "measure": f"measure_kernel<{tn}, {256 if wide else 32}, {jbf}>"}[dom])
        traffic = (profiled_traffic() if (dom == "measure" and small and jb is None and prec == vmcf.MIXED and W == 16384)
                   else None)
        roofline = {"bound": "alu", "pipe": bound, "kernel": kname, "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s" if bound != "sfu" else "Texp/s", "frac": achieved / peak,
                    "peak_source": "measured in this run by vmcf_probe_pipes (register-only FMA/exp kernels)",
                    "traffic": traffic,
                    "traffic_source": ("DRAM bytes of the committed ncu capture profiles/measure_small_c2oh6.md "
                                       "(its kernel-source hash matches this build)") if traffic else None,
                    "launch_ms": t_launch * 1e3,
                    "kernel_times_source": "per-kernel CUDA events over a second timed region of the same "
                                           f"{steps} steps ({ms_prof / steps:.3f} ms per step with the events)",
                    "kernel_share": {k: kt[k]["ms"] / max(1e-9, sum(v["ms"] for v in kt.values())) for k in kt},
                    "whole_step_frac": workmodel.roofline_time(work["total"], peaks)[1] * W / (ms * 1e-3 / steps)}
        out = {"value": value, "ms_per_step": ms / steps, "steps": steps, "warmup": warmup, "roofline": roofline,
               "gpu_launches": sum(v["launches"] for v in kt.values()), "clocks": clk.summary(),
               "acceptance": acc, "estimates": {"E": est["E"], "E_err": est["E_err"]}, "walkers_per_gpu": W,
               "electrons": sysx.Ne, "aos": g.M}
        if fp64_steps and prec == vmcf.MIXED:
            pos_eq = wk.positions(stream=stream)
            del wk, g
            g64 = vmcf.System(sysx, vmcf.FP64, force_group=group)
            wk64 = vmcf.Walkers(g64, pos_eq, key=(5222, 1), wid0=rank * W, nblocks=nb, stream=stream)
            wk64.reset_accumulators(e_ref, stream=stream)
            wk64.sample(1, 0.3, 26, measure=True, stream=stream)
            ms64, _ = timed_steps(wk64, fp64_steps)
            ms64 = max_over_ranks(ms64)
            v64 = ws * W * fp64_steps / (ms64 * 1e-3)
            out["fp64_gpu"] = {"value": v64, "ms_per_step": ms64 / fp64_steps, "steps": fp64_steps}
            out["mixed_over_fp64"] = value / v64
            del wk64, g64
        return out

    W = args.walkers or wl["walkers"]
    sysx = S.make_system(wl["cfg"])
    jb = None
    if args.jastrow_basis:
        sysx = S.with_jastrow_basis(sysx)
        jb = sysx.jastrow.basis
    prec = vmcf.MIXED if args.precision == "mixed" else vmcf.FP64
    head = workload_line(sysx, W, args.steps, args.warmup, 0 if args.no_fp64 else args.steps, jb, prec,
                         args.group_path, seed=rank)
    line = {"metric": METRIC, "value": head["value"], "unit": "walker-evals/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if prec == vmcf.MIXED else "f64", "data": "synthetic",
            "config": {"workload": wl["name"] + (f" + AO-expanded Jastrow ({jb.MJ} Jastrow-basis functions)" if jb else ""),
                       "walkers_per_gpu": W, "electrons": sysx.Ne, "aos": head["aos"],
                       "step_sigma": 0.3, "refresh_every": 26,
                       "precision": "mixed (FP32 + FP64 inverse/ratio/sums)" if prec == vmcf.MIXED else "fp64",
                       "l2": "flushed (256 MB write) between timed steps"},
            "roofline": head["roofline"], "gpu_launches": head["gpu_launches"], "clocks": head["clocks"],
            "acceptance": head["acceptance"], "estimates": head["estimates"]}
    if "fp64_gpu" in head:
        line["fp64_gpu"] = head["fp64_gpu"]
        line["mixed_over_fp64"] = head["mixed_over_fp64"]

    # ---- end to end through the C ABI with host buffers
    if not args.no_e2e:
        g = vmcf.System(sysx, prec, force_group=args.group_path)
        pos0 = S.initial_walkers(sysx, W, seed=rank)
        wk = vmcf.Walkers(g, pos0, key=(5222, 1), wid0=rank * W, nblocks=nb, stream=stream)
        wk.sample(args.equil, 0.3, 26, measure=False, stream=stream)
        wk.reset_accumulators(head["estimates"]["E"], stream=stream)
        host = torch.empty((W, sysx.Ne, 3), dtype=torch.float64, pin_memory=True).numpy()
        host[:] = wk.positions(stream=stream)
        ke = max(2, args.steps // 2)
        barrier()
        t0 = time.perf_counter()
        for _ in range(ke):
            wk.set_positions(host, stream=stream)          # H2D, inverses rebuilt
            wk.sample(1, 0.3, 26, measure=True, stream=stream)
            _ = wk.reduce_estimators(stream=stream)         # estimators finished on the device, D2H of the results
            wk.positions(stream=stream, out=host)           # D2H positions (pinned) for the next step
        barrier()
        te = max_over_ranks(time.perf_counter() - t0)
        h2d = W * sysx.Ne * 3 * 8
        # positions, and the estimators with their errors (E, F [3K], dE/dC [nO], each with its error bar) plus
        # status flags; beyond 4096 jackknife blocks the block sums themselves come back instead
        d2h = W * sysx.Ne * 3 * 8 + (8 * (2 + 6 * sysx.K + 2 * g.M * sysx.Ne) + 12 if nb <= 4096 else nb * g.accL * 8)
        line["e2e"] = {"value": ws * W * ke / te, "unit": "walker-evals/s", "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h, "steps": ke}
        del wk, g

    # ---- the 94-electron workload (C9O4H8, 65536 walkers per GPU), mixed and FP64, beside the headline
    if args.workload == "c2oh6" and not args.no_large and not args.jastrow_basis and not args.walkers:
        big = WORKLOADS["c9o4h8"]
        blk = workload_line(S.make_system(big["cfg"]), big["walkers"], 5, 3, 0 if args.no_fp64 else 2, seed=rank)
        blk["workload"] = big["name"]
        line["c9o4h8"] = blk

    # ---- the ragged batch (64 geometries of 10-94 electrons, one captured graph per sweep), beside the headline
    if args.workload == "c2oh6" and not args.no_large and not args.jastrow_basis and not args.walkers:
        rg = run_ragged(argparse.Namespace(steps=3, warmup=1, equil=args.equil), WORKLOADS["ragged64"], embedded=True)
        line["ragged64"] = {k: rg[k] for k in ("value", "ms_per_step", "steps", "warmup", "roofline", "gpu_launches",
                                               "clocks", "acceptance")}
        line["ragged64"]["workload"] = rg["config"]["workload"]
        line["ragged64"]["walkers_total"] = rg["config"]["walkers_total"]

    # ---- CPU oracle baseline (rank 0, N = 1 only)
    if not args.no_cpu and ws == 1:
        v, n, t = oracle_steps(sysx, 256 if wl["cfg"] != 4 else 16, 10.0, 30.0)
        line["cpu_baseline"] = {"value": v, "unit": "walker-evals/s", "cores": cores(), "kind": "oracle",
                                "sample": f"{256 if wl['cfg'] != 4 else 16} walkers x {n} measured sweeps "
                                          f"({t:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
