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


if __name__ == "__main__":
    with open(os.path.join(HERE, "tiny_merlin.json"), "w") as f:
        json.dump(tiny(), f, indent=1)
    with open(os.path.join(HERE, "drag_random_walk.json"), "w") as f:
        json.dump(drag_cases(), f, indent=1)
    print("wrote golden fixtures")
