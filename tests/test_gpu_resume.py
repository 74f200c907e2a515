"""Checkpoint / resume per length: a MERLIN run resumed at length m0 from
the schedule inputs of the lengths before it returns exactly the rows
m0..maxL of the uninterrupted FP64 oracle run (same r sequence, discords,
distances, counts and heatmap rows)."""
import numpy as np
import pytest

import oracle
from paper_2304_01660_gb300 import palmad

from test_gpu_parity import NN_RTOL, SERIES, _opts, ctx  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("W", [0, 16])
@pytest.mark.parametrize("name,minL,maxL,K,excl", [("sine4000", 50, 70, 3, True), ("rw3000", 10, 40, 2, True)])
def test_resume_matches_uninterrupted_oracle_run(ctx, W, name, minL, maxL, K, excl):
    T = SERIES[name]()
    full = oracle.merlin(T, minL, maxL, K, excl, heatmap=True)
    sched = palmad.schedule_inputs(full["idx"], full["nn"])
    for m0 in (minL, minL + 1, minL + 3, minL + 5, minL + 9):
        l0 = m0 - minL
        hist = sched[max(0, l0 - 5):l0]
        got = ctx.palmad_find_discords_resume(T, minL, m0, maxL, K, hist, _opts(batch_lengths=W, exclusive_topk=int(excl)),
                                              heatmap=True)
        np.testing.assert_array_equal(got["idx"], full["idx"][l0:])
        np.testing.assert_allclose(got["nn"], full["nn"][l0:], rtol=NN_RTOL, atol=0)
        np.testing.assert_array_equal(got["count"], full["count"][l0:])
        np.testing.assert_allclose(got["r"], full["r"][l0:], rtol=1e-9, atol=0)
        want_heat = full["heatmap"][l0:, :len(T) - m0 + 1]
        np.testing.assert_allclose(got["heatmap"], want_heat, rtol=2 * NN_RTOL, atol=0)


def test_resume_argument_errors(ctx):
    T = SERIES["rw3000"]()
    with pytest.raises(palmad.PalmadError):
        ctx.palmad_find_discords_resume(T, 12, 10, 20, 1, [])             # m0 < minL_sched
    with pytest.raises(palmad.PalmadError):
        ctx.palmad_find_discords_resume(T, 10, 13, 20, 1, [1.0, -1.0, 2.0])  # negative history
