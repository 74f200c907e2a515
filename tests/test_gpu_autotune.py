"""The autotuner changes how fast a call runs, never what it returns.

palmad_autotune times candidate pass configurations (lengths per pass, the
batched form's speculation margin, select cap, refine segment, refine-form
split) on a block of lengths of the caller's series; a find call with
autotune = 1 uses the tuned options of its workload bucket.  Both must give
results identical to the default options, and the report must describe
what was timed.
"""
import numpy as np
import pytest

from paper_2304_01660_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2304_01660_gb300 import _build, palmad
    _build.build()
    c = palmad.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_tuned_options_give_identical_results(ctx, precision):
    import torch
    from paper_2304_01660_gb300 import palmad
    w = synth.workload("sine100k")
    T = torch.from_numpy(w.series[0]).cuda()
    minL, maxL, K = w.minL[0], w.maxL[0], w.topK
    base = palmad.palmad_default_options(precision=precision)
    tuned, rep = ctx.palmad_autotune(T, minL, maxL, K, base)
    assert rep["candidates"] >= 8 and rep["tune_ms"] > 0
    assert minL <= rep["block_lo"] <= rep["block_hi"] <= maxL
    assert rep["best_ms"] <= rep["default_ms"]
    assert tuned.precision == precision and tuned.exclusive_topk == 1
    want = ctx.palmad_find_discords_device(T, minL, maxL, K, base)
    got = ctx.palmad_find_discords_device(T, minL, maxL, K, tuned)
    for k in want:
        assert torch.equal(want[k], got[k]), k
    # autotune = 1: the bucket's tuned options are found in the context
    auto = palmad.palmad_default_options(precision=precision, autotune=1)
    got2 = ctx.palmad_find_discords_device(T, minL, maxL, K, auto)
    assert ctx.palmad_get_stats()["tune_ms"] == 0.0  # cached: no tuning in this call
    for k in want:
        assert torch.equal(want[k], got2[k]), k


def test_autotune_on_first_use_of_a_bucket(ctx):
    """A bucket with no tuned options tunes inside the call, on the call's
    own series, and reports the time; results stay identical."""
    from paper_2304_01660_gb300 import palmad
    T = synth.random_walk(30000, 91)
    want = ctx.palmad_find_discords(T, 40, 70, 2)
    got = ctx.palmad_find_discords(T, 40, 70, 2, palmad.palmad_default_options(autotune=1))
    assert ctx.palmad_get_stats()["tune_ms"] > 0.0
    for k in want:
        np.testing.assert_array_equal(got[k], want[k])
