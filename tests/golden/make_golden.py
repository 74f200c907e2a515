"""Write the stored expected values under tests/golden/.

Every value here comes from the FP64 oracle (``oracle/``) run on the seeded
synthetic inputs of ``paper_2304_01660_gb300.synth``; nothing is taken from the
CUDA path.  The paper prints no worked example with numeric discords, so the
fixtures are regression anchors for the oracle (checked on CPU) and cached
expectations for the GPU parity tests.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2304_01660_gb300 import synth  # noqa: E402


def tiny():
    w = synth.workload("tiny")
    T = w.series[0]
    res = oracle.merlin(T, w.minL[0], w.maxL[0], w.topK, True)
    return {
        "workload": "tiny", "n": len(T), "minL": w.minL[0], "maxL": w.maxL[0], "topK": w.topK,
        "exclusive": True,
        "idx": res["idx"].tolist(), "nn": res["nn"].tolist(), "count": res["count"].tolist(),
        "r": res["r"].tolist(), "calls": res["calls"].tolist(),
    }


def drag_cases():
    out = []
    for n, m, seed, r in [(1500, 24, 31, 4.0), (1200, 60, 32, 6.5)]:
        T = synth.random_walk(n, seed)
        idx, nn = oracle.drag(T, m, r)
        out.append({"n": n, "m": m, "seed": seed, "r": r, "idx": idx.tolist(), "nn": nn.tolist()})
    return out


def beats1m_windows(lengths=20, random_windows=8, seed=11):
    """Nearest non-self match (brute force, oracle.nn_one) of chosen windows
    of the 1M-point beats series at evenly spaced lengths of 100..1000.  The
    windows are the recipe's own: one starting half a window before every
    abnormal beat (the series' planted anomalies) plus seeded random ones.
    Whatever threshold a run ends with at a length, a window is a range
    discord there exactly when this distance is >= it, and its heatmap
    entry is then distance^2 / (2m) (Eq. 10)."""
    import numpy as np
    w = synth.workload("beats1m")
    T = w.series[0]
    n, minL, maxL = len(T), w.minL[0], w.maxL[0]
    rng = np.random.default_rng(seed)
    ms = sorted({int(round(minL + q * (maxL - minL) / (lengths - 1))) for q in range(lengths)})
    rows = []
    for m in ms:
        N = n - m + 1
        wins = [min(max(0, c - m // 2), N - 1) for c in w.notes["odd_beats"]]
        wins += [int(x) for x in rng.integers(0, N, size=random_windows)]
        for i in wins:
            nn, j = oracle.nn_one(T, m, i)
            rows.append({"m": m, "i": i, "nn": nn, "j": j})
    return {"workload": "beats1m", "n": n, "minL": minL, "maxL": maxL,
            "source": "oracle.nn_one (FP64 brute force over every non-self match)", "windows": rows}


if __name__ == "__main__":
    with open(os.path.join(HERE, "tiny_merlin.json"), "w") as f:
        json.dump(tiny(), f, indent=1)
    with open(os.path.join(HERE, "drag_random_walk.json"), "w") as f:
        json.dump(drag_cases(), f, indent=1)
    if "--beats1m" in sys.argv[1:]:  # minutes of CPU: written only when asked
        with open(os.path.join(HERE, "beats1m_windows.json"), "w") as f:
            json.dump(beats1m_windows(), f, indent=1)
    print("wrote golden fixtures")
