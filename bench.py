"""Benchmark: PALMAD discords over [minL, maxL] on one series per GPU.

Metric: points x lengths per second, the sum over lengths m of (n - m + 1)
divided by the time of one full MERLIN run (every length, every DRAG call the
schedule makes, exact results, the discord heatmap of Eq. 10 included when
the workload asks for it).  The default workload is the largest one-GPU
configuration: one 10^6-point series of quasi-periodic beats, lengths
100..1000, top-1 per length plus the full heatmap (seeded synthetic data
shaped like the paper's ECG series).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload beats1m|rw250k|sine100k|tiny]

Our arm prints one JSON line (rank 0): `value` is the mixed-precision form
(tensor-core direct refine) with the pass configuration the autotuner picks
for this workload (lengths per pass, speculation margin, select cap, refine
segment, refine-form split; tuning time reported apart), series resident in
HBM.  `forms` gives the plain FP32 form and the untuned 16-lengths-per-pass
form beside it on the same workload; `e2e` is the host-pointer entry
(upload, all lengths, results and heatmap back); `parity` checks the timed
run against values the FP64 oracle wrote (tests/golden/); `roofline`,
`clocks` and `cpu_baseline` as the contract asks.  The reference arm
(`--impl reference`) times the FP64 oracle on a sample of the same workload
on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
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
L2_FLUSH_BYTES = 512 << 20
FIXTURE = os.path.join(ROOT, "tests", "golden", "beats1m_windows.json")
# DRAM bytes (read + write) per evaluated pair of a kernel, from an ncu
# capture of a bounded case of this workload: (sha256[:16] of the kernel's
# source file at the capture, bytes per pair).  The bench scales it to its own launches by their pair
# counts; a source that no longer matches reports null.
# k_refine_tcs: beats1m m = 150..157, one launch of 54 684 tiles of 128 x 256
# survivor-column pairs, 37.6 MB read + 159.4 MB written (the chunk maxima).
TRAFFIC: dict[str, tuple[str, float]] = {
    "refine_direct_tc": ("aa47512157115605", 197.0e6 / (54684 * 128 * 256)),
}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def _src_hash(rel: str) -> str:
    import hashlib
    try:
        return hashlib.sha256(open(os.path.join(ROOT, rel), "rb").read()).hexdigest()[:16]
    except OSError:
        return ""


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


# ------------------------------------------------------------ FP64 oracle leg

def _oracle_sample_plan(w: synth.Workload):
    """Lengths and thresholds of the oracle sample.  For beats1m: the 20
    evenly spaced lengths of the oracle fixture, each at the largest
    nearest-neighbour distance the oracle found among that length's fixture
    windows (near the top of the distance distribution, where MERLIN's
    thresholds sit).  Other workloads: 8 evenly spaced lengths at the 99.9th
    percentile of the oracle's distances of 64 seeded windows."""
    T, minL, maxL = w.series[0], w.minL[0], w.maxL[0]
    if w.name.startswith("beats1m") and os.path.exists(FIXTURE):
        rows = json.load(open(FIXTURE))["windows"]
        by_m = {}
        for x in rows:
            by_m.setdefault(x["m"], []).append(x["nn"])
        return [(m, max(v)) for m, v in sorted(by_m.items())]
    import oracle
    rng = np.random.default_rng(5)
    plan = []
    for m in np.linspace(minL, maxL, 8).round().astype(int):
        N = len(T) - int(m) + 1
        d = [oracle.nn_one(T, int(m), int(i))[0] for i in rng.integers(0, N, size=64)]
        plan.append((int(m), float(np.quantile(d, 0.999))))
    return plan


def oracle_sample(w: synth.Workload, budget_s: float, seed: int = 17) -> dict:
    """The FP64 oracle's range-discord test (Sec. 2.1's definition, one
    window at a time) on seeded random windows of the sampled lengths, in
    random length order until the time budget is spent.  Each (length,
    window) is one unit of the metric, so units / CPU seconds is the
    oracle's points x lengths / s, extrapolated from the sample."""
    import oracle
    T = w.series[0]
    plan = _oracle_sample_plan(w)
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(plan))
    per = 96
    units, spent, lengths = 0, 0.0, []
    for q in order:
        m, r = plan[q]
        N = len(T) - m + 1
        wins = rng.integers(0, N, size=per)
        t0 = time.perf_counter()
        oracle.range_discord_windows(T, m, r, wins)
        spent += time.perf_counter() - t0
        units += per
        lengths.append(m)
        if spent > budget_s:
            break
    return {"value": units / spent, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"extrapolated: the oracle's range-discord test of {units} seeded random (length, window) units "
                      f"({per} windows at each of {len(lengths)} sampled lengths of {w.name}, m in "
                      f"{min(lengths)}..{max(lengths)}), threshold per length = the largest oracle nearest-neighbour "
                      f"distance among that length's fixture windows; {spent:.1f} s of oracle time"}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    budget = 4.0
    for _ in range(args.warmup):
        oracle_sample(w, budget, seed=99)
    vals, times = [], []
    for s in range(args.steps):
        t0 = time.perf_counter()
        cb = oracle_sample(w, budget, seed=1000 + s)
        times.append(time.perf_counter() - t0)
        vals.append(cb["value"])
    tot = sum(times)
    # the step's units are its sampled units; the rate is the units' harmonic mean
    value = float(len(vals) / sum(1.0 / v for v in vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n": len(w.series[0]), "minL": w.minL[0], "maxL": w.maxL[0], "topK": w.topK,
                   "sample": "one step = the FP64 oracle's range-discord test on about 4 s of seeded random "
                             "(length, window) units of the workload, extrapolated per unit"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cb["cores"], "kind": "oracle", "sample": cb["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------- parity

def schedule_ok(nn, idx, r, minL) -> bool:
    """Final r of every length from the closed forms of Sec. 2.2 applied to
    the returned distances (the same check as the full-size GPU tests)."""
    K = idx.shape[1]
    got = (idx >= 0).sum(axis=1)
    sched = np.where(got > 0, nn[np.arange(len(nn)), np.maximum(got - 1, 0)], 0.0)
    for l in range(len(r)):
        if r[l] <= 0.0:
            continue
        if l == 0:
            k = math.log2(2 * math.sqrt(minL) / r[0])
        elif l <= 4:
            k = math.log(r[l] / (0.99 * sched[l - 1])) / math.log(0.99)
        else:
            last = sched[l - 5:l]
            mu, sd = last.mean(), last.std(ddof=1)
            k = (mu - 2 * sd - r[l]) / (sd if sd > 0 else 0.01 * mu)
        if abs(k - round(k)) > 1e-6 or round(k) < 0 or (got[l] == K and sched[l] < r[l]):
            return False
    return True


def parity_check(w, res, heat) -> dict:
    """The timed run's outputs against the oracle fixture: every fixture
    window (length m, start i, the oracle's brute-force nearest-neighbour
    distance) is a range discord exactly when that distance is >= the run's
    final r at m, and its heatmap entry is then distance^2 / (2m)."""
    out = {"schedule_closed_forms": bool(schedule_ok(res["nn"], res["idx"], res["r"], w.minL[0]))}
    if not w.name.startswith("beats1m") or heat is None or not os.path.exists(FIXTURE):
        out["fixture"] = None
        return out
    rows = [x for x in json.load(open(FIXTURE))["windows"] if w.minL[0] <= x["m"] <= w.maxL[0]]
    bad, pos = 0, 0
    ms = sorted({x["m"] for x in rows})
    hrows = {m: heat[m - w.minL[0]].cpu().numpy() for m in ms}
    for x in rows:
        m, i, nn = x["m"], x["i"], x["nn"]
        r = res["r"][m - w.minL[0]]
        h = float(hrows[m][i])
        if nn >= r:
            pos += 1
            ok = h > 0 and abs(math.sqrt(h * 2 * m) - nn) <= 1e-5 * nn
        else:
            ok = h == 0.0
        bad += not ok
    out.update({"fixture": "tests/golden/beats1m_windows.json (FP64 oracle, brute-force nearest neighbour)",
                "windows_checked": len(rows), "windows_discord": pos, "mismatches": bad})
    return out


# ----------------------------------------------------------------- our arm

def run_ours(args, w):
    import torch
    import torch.distributed as dist
    from paper_2304_01660_gb300 import _build, palmad
    from paper_2304_01660_gb300 import dist as pdist

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
    heat = torch.empty((L, n - minL + 1), dtype=torch.float32, device="cuda") if w.heatmap else None
    prof = 0 if args.no_events else 1

    # the headline form's configuration, tuned on this series (not timed),
    # or given with --options (profiling runs)
    mixed_base = palmad.palmad_default_options(precision=1, batch_lengths=args.batch)
    if args.options:
        kv = {"precision": 1}
        kv.update({k: int(v) for k, v in (item.split("=") for item in args.options.split(","))})
        tuned = palmad.palmad_default_options(**kv)
        tune_rep = {"tune_ms": 0.0, "candidates": 0, "block_lo": 0, "block_hi": 0, "best_ms": None, "default_ms": None,
                    "chosen": {k: getattr(tuned, k) for k in palmad.TUNED_FIELDS}, "given": args.options}
    else:
        tuned, tune_rep = ctx.palmad_autotune(T_dev, minL, maxL, K, mixed_base)
    tuned.profile = prof
    forms = {
        "mixed_tuned": tuned,
        "plain": palmad.palmad_default_options(profile=prof),
        f"mixed_w{args.batch}": palmad.palmad_default_options(profile=prof, precision=1, batch_lengths=args.batch),
        # the k-th neighbour variant (k = 2) with the tuned configuration (its own form; off by default)
        "knn2": palmad.palmad_default_options(**{**{k: getattr(tuned, k) for k in palmad.TUNED_FIELDS},
                                                 "profile": prof, "knn_k": 2}),
    }
    forms = {f: o for f, o in forms.items() if f == "mixed_tuned" or f.split("_")[0] in args.forms.split(",")}
    chosen = tune_rep["chosen"]
    side_steps, side_warm = min(args.steps, args.side_steps), min(args.warmup, 1)

    def step(form):
        return ctx.palmad_find_discords_device(T_dev, minL, maxL, K, forms[form], heatmap_dev=heat)

    def timed(form, steps, warm):
        first = None
        for _ in range(warm):
            out = step(form)
            first = {k: v.cpu().numpy() for k, v in out.items()}
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        acc = {"launches": 0, "kernel_ms": {}, "flops": {"select": 0.0, "refine_direct": 0.0, "refine_sweep": 0.0},
               "pairs": {"select": 0, "refine": 0, "fp64": 0, "hint": 0}}
        with ClockSampler(local) as clk:
            for s in range(steps):
                flush.zero_()
                ev[s][0].record(stream)
                out = step(form)
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
                acc["pairs"]["hint"] += st["hint_pairs"]
                acc["pairs"]["direct"] = acc["pairs"].get("direct", 0) + st["direct_pairs"]
            torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        # job time: the slowest rank's
        total_ms = pdist.max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), device="cuda")
        acc.update(total_ms=total_ms, steps=steps, warmup=warm, clocks=clk.summary(),
                   stats=ctx.palmad_get_stats(), out={k: v.cpu().numpy() for k, v in out.items()}, first=first)
        return acc

    results = {}
    results["mixed_tuned"] = timed("mixed_tuned", args.steps, args.warmup)
    parity = parity_check(w, results["mixed_tuned"]["out"], heat)
    for f in forms:
        if f != "mixed_tuned":
            results[f] = timed(f, side_steps, side_warm)
    R = results["mixed_tuned"]
    ref_out = R["out"]
    parity["forms_identical"] = all(
        all(np.array_equal(ref_out[k], r["out"][k]) for k in ref_out) for f, r in results.items() if f != "knn2")
    total_ms = R["total_ms"]
    value = units * args.steps * world / (total_ms / 1e3)
    last_stats = R["stats"]
    kernel_ms, flops, pairs, launches = R["kernel_ms"], R["flops"], R["pairs"], R["launches"]

    # End to end through the host-pointer entry: upload, all lengths, results
    # and the heatmap back into pinned host memory.
    T_pin = torch.from_numpy(T).pin_memory()
    heat_host = torch.empty((L, n - minL + 1), dtype=torch.float32).pin_memory() if w.heatmap else None
    torch.cuda.synchronize()
    e2e_times = []
    e2e_steps = 0 if args.no_e2e else min(args.steps, args.side_steps)
    for s in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.palmad_find_discords(T_pin.numpy(), minL, maxL, K, forms["mixed_tuned"],
                                 heatmap=w.heatmap, heat_out=heat_host.numpy() if heat_host is not None else None)
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = pdist.max_over_ranks(sum(e2e_times), device="cuda")
    e2e_value = units * len(e2e_times) * world / e2e_s if e2e_times else None
    heat_bytes = 4 * L * (n - minL + 1) if w.heatmap else 0

    if rank == 0:
        peaks = _peaks()
        fp_peaks = {}
        for kind in ("fp32", "fp32x2", "fp64"):
            try:
                fp_peaks[kind] = palmad.palmad_measure_peak(local, kind)
            except Exception:
                fp_peaks[kind] = None
        meas = max([v for k2, v in fp_peaks.items() if k2 != "fp64" and v] or [0.0])
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        peak = meas if meas > 0 else sms * 128 * 2 * 2.070e9 / 1e12
        peak_src = ("measured: best of scalar and packed (f32x2) FMA chains on this GPU (palmad_measure_peak)"
                    if meas > 0 else f"derived: {sms} SMs x 128 FP32 lanes x 2 flop x 2070 MHz (measurement failed)")
        dom = max(kernel_ms, key=lambda k2: kernel_ms[k2]) if any(kernel_ms.values()) else "none"
        launches_per = dict(last_stats["launches"])
        tensor = dom == "refine_direct" and tuned.precision == 1
        src = {"refine_sweep": "paper_2304_01660_gb300/csrc/k_sweep.cu",
               "refine_direct": "paper_2304_01660_gb300/csrc/k_refine_tcs.cu" if tensor
               else "paper_2304_01660_gb300/csrc/k_refine.cu"}.get(dom, "")
        trf = TRAFFIC.get(dom if not tensor else "refine_direct_tc")
        traffic = None
        if trf and trf[0] == _src_hash(src) and launches_per.get(dom):
            dpairs = pairs.get("direct", 0) if dom == "refine_direct" else pairs.get("refine", 0) - pairs.get("direct", 0)
            traffic = trf[1] * dpairs / args.steps / launches_per[dom]
        if dom in flops and kernel_ms.get(dom, 0) > 0:
            ach = flops[dom] / (kernel_ms[dom] / 1e3) / 1e12
            if tensor:
                # a contraction on the tensor cores: the measured bf16 dense peak,
                # sustained (the kernel runs inside a seconds-long step)
                tpk = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
                roof = {"kernel": "refine_direct (tcgen05: k_refine_tcs, survivor-major, windows up to 256; "
                                  "k_refine_tc, column-major, longer windows)", "bound": "tensor", "achieved": ach,
                        "peak": tpk, "unit": "TFLOP/s", "frac": ach / tpk if tpk else None, "traffic": traffic,
                        "traffic_unit": "bytes per launch",
                        "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS bf16, of measured)",
                        "flops_per_pair": "2m per survivor-column dot product (algorithmic)",
                        "executed_tensor_tflops": 3 * ach,
                        "executed_frac": 3 * ach / tpk if tpk else None,
                        "note": "each FP32 product runs as three BF16 MMAs (hi*hi + hi*lo + lo*hi)"}
            else:
                roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                        "frac": ach / peak, "traffic": traffic, "traffic_unit": "bytes per launch",
                        "peak_source": peak_src,
                        "flops_per_pair": "8 per recurrence pair + 2m per direct dot product (seeds)"}
        else:
            roof = {"kernel": dom, "bound": "alu", "achieved": None, "peak": peak, "unit": "TFLOP/s",
                    "frac": None, "traffic": traffic, "peak_source": peak_src}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3+f32", "data": "synthetic",
            "config": {"workload": w.name, "n": n, "minL": minL, "maxL": maxL, "topK": K, "heatmap": w.heatmap,
                       "form": "mixed precision (tensor-core direct refine) with the autotuned pass configuration "
                               f"(lengths per pass {max(1, chosen['batch_lengths'])}, speculation margin "
                               f"{chosen['spec_scale'] or 100}%, select cap {chosen['select_cap'] or 1024}, refine "
                               f"segment {chosen['refine_seg'] or 'auto'}, direct form below "
                               f"{chosen['direct_below'] or 'auto'} survivors (windows up to 256; "
                               f"{chosen['direct_below_long'] or chosen['direct_below'] or 'auto'} for longer), "
                               f"direct refine in {chosen['tc_chunks'] or 1} column chunks, refine strips of "
                               f"{chosen['refine_rows'] or 128} rows)",
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * n,
                    "d2h_bytes_per_step": L * K * 16 + L * 16 + heat_bytes, "steps": len(e2e_times),
                    "note": "host-pointer entry; the heatmap comes back into pinned host memory"},
            "gpu_launches": launches,
            "roofline": roof,
            "clocks": R["clocks"],
            "parity": parity,
            "tuning": {k: tune_rep.get(k) for k in ("tune_ms", "candidates", "block_lo", "block_hi", "best_ms",
                                                    "default_ms", "chosen", "given")},
            "forms": {f: {"value": units * r["steps"] * world / (r["total_ms"] / 1e3),
                          "ms_per_step": r["total_ms"] / r["steps"], "steps": r["steps"], "warmup": r["warmup"],
                          "passes_per_step": r["stats"]["device_passes"], "reruns_per_step": r["stats"]["reruns"],
                          "clocks": r["clocks"]} for f, r in results.items()},
            "kernel_ms_per_step": {k2: v / args.steps for k2, v in kernel_ms.items() if v},
            "kernel_tflops": {k2: flops[k2] / (kernel_ms[k2] / 1e3) / 1e12 for k2 in flops if kernel_ms.get(k2, 0) > 0},
            "pairs_per_step": {k2: v / args.steps for k2, v in pairs.items()},
            "launches_per_step": launches_per,
            "drag_calls_per_step": last_stats["drag_calls"],
            "passes_per_step": last_stats["device_passes"],
            "reruns_per_step": last_stats["reruns"],
            "survivors_per_step": last_stats["survivors"],
            "hint_kills_per_step": last_stats["hint_kills"],
            "max_fp32_rho_err": last_stats["max_fp32_rho_err"],
            "hbm_peak_gbs": peaks.get("hbm_gbs"),
            "fma_peaks_tflops": fp_peaks,
        }
        if "plain" in results:
            line["mixed_vs_plain"] = results["plain"]["total_ms"] / results["plain"]["steps"] / (total_ms / args.steps)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = oracle_sample(w, args.cpu_budget)
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="beats1m", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-pointer end-to-end leg")
    ap.add_argument("--no-events", action="store_true", help="no per-launch CUDA events (profiler runs)")
    ap.add_argument("--batch", type=int, default=16, help="lengths per pass of the untuned batched form")
    ap.add_argument("--side-steps", type=int, default=2,
                    help="timed steps of the secondary forms and of the end-to-end leg")
    ap.add_argument("--forms", default="plain,mixed",
                    help="secondary forms to time beside the tuned one: plain, mixed (16 lengths per pass), "
                         "knn2 (the k-th neighbour variant, k = 2)")
    ap.add_argument("--options", default=None,
                    help="k=v,...: options of the headline form instead of the autotuner's (profiling runs)")
    ap.add_argument("--lengths", default=None,
                    help="LO:HI: only lengths LO..HI of the workload (bounded cases for profiling)")
    args = ap.parse_args(argv)
    w = synth.workload(args.workload)
    if args.lengths:
        lo, hi = (int(v) for v in args.lengths.split(":"))
        if not (w.minL[0] <= lo <= hi <= w.maxL[0]) or len(w.series) != 1:
            ap.error("--lengths must lie within the workload's single-series length range")
        w.minL, w.maxL = [lo], [hi]
        w.name = f"{w.name}[m={lo}..{hi}]"
        args.no_cpu_baseline = True
    if args.impl == "reference":
        return run_reference(args, w)
    return run_ours(args, w)


if __name__ == "__main__":
    sys.exit(main())
