"""Benchmark: PALMAD discords over [minL, maxL] on one series per GPU.

Metric: points x lengths per second, sum over lengths m of (n - m + 1)
divided by the time of one full MERLIN run (every length, every DRAG call the
schedule makes, exact results).  The default workload is the 100k-point noisy
sine with five injected anomalies, lengths 128..256, top-3 (seeded synthetic
data shaped like the paper's periodic series).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Our arm prints one JSON line (rank 0) with the device-resident throughput
(`value`), the host-pointer end-to-end throughput (`e2e`), the roofline of
the dominant kernel, the clocks seen during the timed region and the FP64
oracle timed on the host cores (`cpu_baseline`).  The reference arm
(`--impl reference`) times the FP64 oracle on a bounded sample of the same
workload on the host cores.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2304_01660_gb300 import synth  # noqa: E402

METRIC = "points x lengths / s (all lengths minL..maxL, exact discords)"
UNIT = "points*lengths/s"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x FMA x max SM clock
L2_FLUSH_BYTES = 512 << 20
# DRAM bytes (read + write) per launch of a kernel from an ncu capture of the
# current kernel source (profiles/); None once the kernel changes.
TRAFFIC_PER_LAUNCH: dict[str, float | None] = {
    "refine_sweep": 105.408512e6 + 130.19904e6,  # profiles/k_sweep_sine100k.md
}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """Samples SM clock and throttle reasons with nvidia-smi while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.t = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            if self.t:
                self.t.join(timeout=2)

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(w: synth.Workload, budget_s: float = 20.0) -> dict:
    """FP64 oracle (as it stands) on the first lengths of the workload, as
    many as fit in about ``budget_s`` seconds, on the host cores."""
    import oracle
    T, minL, maxL, K = w.series[0], w.minL[0], w.maxL[0], w.topK
    n = len(T)
    t0 = time.perf_counter()
    done = 0
    units = 0
    # MERLIN from minL over a growing prefix of the length range; the sample
    # is the largest prefix finished within the budget.
    for hi in range(minL, maxL + 1):
        t1 = time.perf_counter()
        oracle.merlin(T, minL, hi, K, True)
        el = time.perf_counter() - t1
        done = hi - minL + 1
        units = sum(n - m + 1 for m in range(minL, hi + 1))
        last = el
        if time.perf_counter() - t0 + 2.2 * el > budget_s:
            break
    return {"value": units / last, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"MERLIN over lengths {minL}..{minL + done - 1} of {w.name} ({done} of {maxL - minL + 1} "
                      f"lengths, {last:.1f} s)"}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    T, minL, K = w.series[0], w.minL[0], w.topK
    n = len(T)
    units = n - minL + 1
    for _ in range(args.warmup):
        oracle.merlin(T, minL, minL, K, True)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.merlin(T, minL, minL, K, True)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = units * args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n": n, "minL": minL, "maxL": w.maxL[0], "topK": K,
                   "sample": f"one step = MERLIN at the first length (m={minL}) only"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"MERLIN at m={minL} of {w.name} per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, w):
    import torch
    import torch.distributed as dist
    from paper_2304_01660_gb300 import _build, palmad

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        _build.build()  # one rank compiles; the others wait for it
    if world > 1:
        dist.barrier()

    T, minL, maxL, K = w.series[0], w.minL[0], w.maxL[0], w.topK
    n = len(T)
    L = maxL - minL + 1
    units = w.units
    stream = torch.cuda.current_stream()
    ctx = palmad.Context(local, stream.cuda_stream)
    T_dev = torch.from_numpy(T).cuda()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    prof = 0 if args.no_events else 1
    forms = {"plain": palmad.palmad_default_options(profile=prof),
             "batched": palmad.palmad_default_options(profile=prof, batch_lengths=args.batch),
             "mixed": palmad.palmad_default_options(profile=prof, batch_lengths=args.batch, precision=1)}
    forms = {f: o for f, o in forms.items() if f in args.forms.split(",")}
    best = args.form if args.form in forms else next(iter(forms))

    def step(form):
        return ctx.palmad_find_discords_device(T_dev, minL, maxL, K, forms[form])

    ref = None
    for form in forms:
        for _ in range(args.warmup):
            out = step(form)
            res = {k: v.cpu().numpy() for k, v in out.items()}
            if ref is None:
                ref = res
            elif not all(np.array_equal(ref[k], res[k]) for k in ref):
                raise RuntimeError(f"{form} results differ from the first run")

    def timed(form):
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        acc = {"launches": 0, "kernel_ms": {}, "flops": {"select": 0.0, "refine_direct": 0.0, "refine_sweep": 0.0},
               "pairs": {"select": 0, "refine": 0, "fp64": 0}}
        with ClockSampler(local) as clk:
            for s in range(args.steps):
                flush.zero_()
                ev[s][0].record(stream)
                step(form)
                ev[s][1].record(stream)
                st = ctx.palmad_get_stats()
                acc["launches"] += sum(st["launches"].values())
                for k2, v in st["kernel_ms"].items():
                    acc["kernel_ms"][k2] = acc["kernel_ms"].get(k2, 0.0) + v
                acc["flops"]["select"] += st["select_flops"]
                acc["flops"]["refine_direct"] += st["refine_flops"]
                acc["flops"]["refine_sweep"] += st["sweep_flops"]
                acc["pairs"]["select"] += st["select_pairs"]
                acc["pairs"]["refine"] += st["refine_pairs"]
                acc["pairs"]["fp64"] += st["fp64_pairs"]
            torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        tot = sum(a.elapsed_time(b) for a, b in ev)
        t = torch.tensor([tot], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        acc["total_ms"] = float(t.item())
        acc["clocks"] = clk.summary()
        acc["stats"] = ctx.palmad_get_stats()
        return acc

    results = {form: timed(form) for form in forms}
    R = results[best]
    total_ms = R["total_ms"]
    value = units * args.steps * world / (total_ms / 1e3)
    last_stats = R["stats"]
    kernel_ms, flops, pairs, launches = R["kernel_ms"], R["flops"], R["pairs"], R["launches"]

    class _Clk:
        def summary(self):
            return R["clocks"]
    clk = _Clk()

    # End to end through the host-pointer entry: upload, all lengths, results.
    T_pin = torch.from_numpy(T).pin_memory()
    T_host = T_pin.numpy()
    torch.cuda.synchronize()
    e2e_times = []
    for s in range(0 if args.no_e2e else max(1, args.steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.palmad_find_discords(T_host, minL, maxL, K, forms[best])
        e2e_times.append(time.perf_counter() - t0)
    e2e_t = torch.tensor([sum(e2e_times)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_value = units * len(e2e_times) * world / float(e2e_t.item()) if e2e_times else None

    if rank == 0:
        peaks = _peaks()
        # FP32 / FP64 FMA throughput measured on this GPU after the timed region
        fp_peaks = {}
        for kind in ("fp32", "fp32x2", "fp64"):
            try:
                fp_peaks[kind] = palmad.palmad_measure_peak(local, kind)
            except Exception:
                fp_peaks[kind] = None
        meas = max([v for k2, v in fp_peaks.items() if k2 != "fp64" and v] or [0.0])
        peak = meas if meas > 0 else FP32_PEAK_TFLOPS
        peak_src = ("measured: best of scalar and packed (f32x2) FMA chains on this GPU (palmad_measure_peak)"
                    if meas > 0 else "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (measurement failed)")
        # dominant kernel by event time over the timed region
        dom = max(kernel_ms, key=lambda k2: kernel_ms[k2]) if any(kernel_ms.values()) else "none"
        launches_per = {k2: v for k2, v in last_stats["launches"].items()}
        if dom in flops and kernel_ms.get(dom, 0) > 0:
            ach = flops[dom] / (kernel_ms[dom] / 1e3) / 1e12
            roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": TRAFFIC_PER_LAUNCH.get(dom), "peak_source": peak_src}
        else:
            roof = {"kernel": dom, "bound": "alu", "achieved": None, "peak": peak, "unit": "TFLOP/s",
                    "frac": None, "traffic": None, "peak_source": peak_src}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3+f32" if best == "mixed" else "f32",
            "data": "synthetic",
            "config": {"workload": w.name, "n": n, "minL": minL, "maxL": maxL, "topK": K,
                       "form": {"plain": "plain FP32", "batched": f"batched W={args.batch} FP32",
                                "mixed": f"mixed precision (tensor-core direct refine) + batched W={args.batch}"}[best],
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * n,
                    "d2h_bytes_per_step": L * K * 16 + L * 16},
            "gpu_launches": launches,
            "roofline": roof,
            "clocks": clk.summary(),
            "kernel_ms_per_step": {k2: v / args.steps for k2, v in kernel_ms.items() if v},
            "kernel_tflops": {k2: flops[k2] / (kernel_ms[k2] / 1e3) / 1e12 for k2 in flops if kernel_ms.get(k2, 0) > 0},
            "pairs_per_step": {k2: v / args.steps for k2, v in pairs.items()},
            "launches_per_step": launches_per,
            "drag_calls_per_step": last_stats["drag_calls"],
            "passes_per_step": last_stats["device_passes"],
            "reruns_per_step": last_stats["reruns"],
            "forms": {f: {"value": units * args.steps * world / (r["total_ms"] / 1e3), "ms_per_step": r["total_ms"] / args.steps,
                          "launches_per_step": r["launches"] / args.steps,
                          "passes_per_step": r["stats"]["device_passes"]} for f, r in results.items()},
            "max_fp32_rho_err": last_stats["max_fp32_rho_err"],
            "hbm_peak_gbs": peaks.get("hbm_gbs"),
            "fma_peaks_tflops": fp_peaks,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w, args.cpu_budget)
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="sine100k", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-pointer end-to-end leg")
    ap.add_argument("--no-events", action="store_true", help="no per-launch CUDA events (profiler runs)")
    ap.add_argument("--form", choices=["plain", "batched", "mixed"], default="mixed", help="form reported as `value`")
    ap.add_argument("--batch", type=int, default=16, help="lengths per pass of the batched form")
    ap.add_argument("--forms", default="plain,batched,mixed", help="forms to time (comma separated)")
    args = ap.parse_args(argv)
    w = synth.workload(args.workload)
    if args.impl == "reference":
        return run_reference(args, w)
    return run_ours(args, w)


if __name__ == "__main__":
    sys.exit(main())
