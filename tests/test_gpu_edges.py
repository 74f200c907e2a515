"""Degenerate and boundary cases of the whole MERLIN path against the FP64
oracle, in the FP32 form and in the mixed-precision batched form."""
import numpy as np
import pytest

import oracle
from paper_2304_01660_gb300 import synth

from test_gpu_parity import _check_merlin, _opts, ctx  # noqa: F401

pytestmark = pytest.mark.gpu

FORMS = [dict(), dict(precision=1, batch_lengths=8, direct_below=129)]


def _merlin(ctx, T, minL, maxL, K, form, excl=True):
    got = ctx.palmad_find_discords(T, minL, maxL, K, _opts(exclusive_topk=int(excl), **form), heatmap=True)
    want = oracle.merlin(T, minL, maxL, K, excl, heatmap=True)
    _check_merlin(got, want, heat=True)
    np.testing.assert_allclose(got["r"], want["r"], rtol=1e-9, atol=0)
    np.testing.assert_array_equal(got["count"], want["count"])


@pytest.mark.parametrize("form", FORMS)
def test_smallest_window_length(ctx, form):
    """m = 3, the smallest length the problem allows (Eq. 2)."""
    _merlin(ctx, synth.random_walk(700, 81), 3, 9, 2, form)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("K,excl", [(16, True), (16, False), (100, False)])
def test_large_topk(ctx, form, K, excl):
    _merlin(ctx, synth.random_walk(700, 82), 12, 15, K, form, excl)


@pytest.mark.parametrize("form", FORMS)
def test_n_equals_twice_maxL(ctx, form):
    _merlin(ctx, synth.random_walk(2 * 40, 83), 30, 40, 1, form)


@pytest.mark.parametrize("form", FORMS)
def test_constant_series(ctx, form):
    """Every window flat: every distance is 0, the schedule falls to r = 0
    and every window with a non-self match is a range discord."""
    _merlin(ctx, np.full(600, 3.25, dtype=np.float32), 10, 14, 2, form)


@pytest.mark.parametrize("form", FORMS)
def test_large_offset_series(ctx, form):
    """A random walk sitting on a large offset (mean far from zero)."""
    T = (synth.random_walk(1800, 84).astype(np.float64) + 5.0e4).astype(np.float32)
    _merlin(ctx, T, 16, 24, 2, form)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("excl", [True, False])
def test_large_topk_against_brute_force(ctx, form, excl):
    """K = 60 near the packing limit of exclusive picks: the schedule shrinks
    r through hundreds of DRAG calls.  Whenever a length reaches K picks they
    equal greedy top-K over the brute-force matrix profile (the result does
    not depend on r), which the oracle computes quickly."""
    T = synth.random_walk(1500, 82)
    minL, maxL, K = 20, 24, 60
    got = ctx.palmad_find_discords(T, minL, maxL, K, _opts(exclusive_topk=int(excl), **form))
    for l in range(maxL - minL + 1):
        m = minL + l
        mp, _ = oracle.matrix_profile(T, m)
        ok = np.isfinite(mp)
        wi, wn = oracle.topk(np.nonzero(ok)[0], mp[ok], m, K, excl)
        if (got["idx"][l] >= 0).sum() == K:
            np.testing.assert_array_equal(got["idx"][l], wi)
            np.testing.assert_allclose(got["nn"][l], wn, rtol=1e-5, atol=0)
        assert (got["idx"][l] >= 0).sum() == (wi >= 0).sum() or got["r"][l] > 0


@pytest.mark.parametrize("form", FORMS + [dict(precision=1)])
@pytest.mark.parametrize("m", [900, 1000])
def test_widest_windows_drag(ctx, form, m):
    """Windows padded to 1024, the widest the tensor-core refine takes: the
    sweep's top-row seed pass runs its longest k range."""
    from test_gpu_parity import _check_drag, _thresholds
    for T in (synth.random_walk(3200, 71), synth.workload("sine100k").series[0][:3400]):
        mp, _ = oracle.matrix_profile(T, m)
        for r in _thresholds(mp, (0.2, 0.9, 1.0)):
            _check_drag(ctx, T, m, float(r), _opts(**form))


@pytest.mark.parametrize("form", FORMS)
def test_widest_windows_merlin(ctx, form):
    _merlin(ctx, synth.random_walk(3200, 71), 994, 1000, 2, form)
