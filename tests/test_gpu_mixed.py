"""GPU parity of the mixed-precision form (tensor-core direct refine) against
the FP64 oracle, and against the FP32 form.

The mixed form must return exactly what the FP32 form returns: the tensor
cores only change which FP32-side values bound the pruning and the FP64
re-check; every kept decision and every reported distance is FP64.  Most
cases set direct_below = 129, which routes every survivor to the direct
form, so the tcgen05 kernel sees every lane shape; the m >= 520 cases use
its 32-survivor variant (kpad > 512).
"""
import numpy as np
import pytest

import oracle
from paper_2304_01660_gb300 import synth

from test_gpu_parity import NN_RTOL, SERIES, _check_drag, _check_merlin, _opts, _thresholds, ctx  # noqa: F401

pytestmark = pytest.mark.gpu

MIXED = 1
ALL_TC = dict(precision=MIXED, direct_below=129)
ALL_SEED = dict(precision=MIXED, tc_seed_min=1)   # every swept strip seeded on the tensor cores


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("name", list(SERIES))
@pytest.mark.parametrize("m", [8, 37, 100, 256])
def test_mixed_drag_matches_oracle(ctx, name, m, form):
    """form 0: survivor-major tiles (windows up to 256); 1: column-major."""
    T = SERIES[name]()
    mp, _ = oracle.matrix_profile(T, m)
    for r in _thresholds(mp, (0.5, 0.9, 0.99, 1.0)):
        _check_drag(ctx, T, m, float(r), _opts(**ALL_TC, tc_form=form))


_MANY = {}


def _many_groups_case(m):
    """40 000-point random walk and a threshold near the 95th percentile of
    sampled nearest-neighbour distances (midway between two sampled values),
    with the oracle's range discords (cached per m)."""
    if m not in _MANY:
        T = synth.random_walk(40000, 63)
        N = len(T) - m + 1
        idx = np.random.default_rng(m).choice(N, size=200, replace=False)
        d = np.sort([oracle.nn_one(T, m, int(i))[0] for i in idx])
        r = float(0.5 * (d[189] + d[190]))
        _MANY[m] = (T, r, oracle.drag(T, m, r))
    return _MANY[m]


@pytest.mark.parametrize("chunks", [0, 3])
@pytest.mark.parametrize("m", [64, 200])
def test_mixed_survivor_major_many_groups(ctx, m, chunks):
    """Thousands of direct survivors (several 256-survivor groups, two MMA
    halves each), five 8192-column work items per group, a ragged last tile,
    and column chunks that do not align with the work items."""
    T, r, (wi, wn) = _many_groups_case(m)
    assert len(wi) > 512
    gi, gn = ctx.palmad_drag(T, m, r, _opts(**ALL_TC, tc_form=2, tc_chunks=chunks))
    np.testing.assert_array_equal(gi, wi)
    np.testing.assert_allclose(gn, wn, rtol=NN_RTOL, atol=0)


@pytest.mark.parametrize("m", [520, 600])
def test_mixed_drag_long_windows(ctx, m):
    """kpad > 512: 32 survivors per MMA."""
    T = synth.random_walk(3000, 61)
    mp, _ = oracle.matrix_profile(T, m)
    for r in _thresholds(mp, (0.2, 0.9, 1.0)):
        _check_drag(ctx, T, m, float(r), _opts(**ALL_TC))
    _check_drag(ctx, T, m, 0.0, _opts(**ALL_TC))


@pytest.mark.parametrize("group", [0, 128, 256])
@pytest.mark.parametrize("name", list(SERIES))
def test_mixed_chunks_and_groups_match_oracle(ctx, name, group):
    """The direct refine in column chunks, live survivors re-packed between
    chunks, with 64 / 128 / 256 survivors per MMA (256 only fits windows up to
    128, so m = 200 falls back to 128)."""
    T = SERIES[name]()
    for m in (8, 100, 200):
        mp, _ = oracle.matrix_profile(T, m)
        for r in _thresholds(mp, (0.5, 0.99, 1.0)):
            _check_drag(ctx, T, m, float(r), _opts(**ALL_TC, tc_chunks=4, tc_group=group))


@pytest.mark.parametrize("chunks", [3, 8])
def test_mixed_chunked_merlin_matches_oracle(ctx, chunks):
    """A 20 000-point series spans several 2048-column chunks."""
    T = synth.random_walk(20000, 62)
    got = ctx.palmad_find_discords(T, 40, 60, 2, _opts(precision=MIXED, direct_below=16, tc_chunks=chunks,
                                                        batch_lengths=4), heatmap=True)
    want = oracle.merlin(T, 40, 60, 2, True, heatmap=True)
    _check_merlin(got, want, heat=True)


def test_mixed_drag_degenerate_thresholds(ctx):
    T = SERIES["rw3000"]()
    m = 20
    N = len(T) - m + 1
    assert _check_drag(ctx, T, m, 0.0, _opts(**ALL_TC)) == N
    assert _check_drag(ctx, T, m, 2 * np.sqrt(m) + 1.0, _opts(precision=MIXED)) == 0


@pytest.mark.parametrize("route", [0, 129])
@pytest.mark.parametrize("W", [0, 16])
@pytest.mark.parametrize("name,minL,maxL,K,excl", [
    ("rw3000", 10, 40, 2, True),
    ("sine4000", 50, 70, 3, True),
    ("flat2200", 16, 30, 1, False),
])
def test_mixed_merlin_matches_oracle(ctx, route, W, name, minL, maxL, K, excl):
    T = SERIES[name]()
    got = ctx.palmad_find_discords(T, minL, maxL, K, _opts(precision=MIXED, exclusive_topk=int(excl), batch_lengths=W,
                                                           direct_below=route), heatmap=True)
    want = oracle.merlin(T, minL, maxL, K, excl, heatmap=True)
    _check_merlin(got, want, heat=True)


def test_mixed_refine_rounds_and_mixed_lengths(ctx):
    """Many refine rounds (tiny pool) and lanes of different kpad in one pass."""
    series = [SERIES["rw3000"](), SERIES["sine4000"](), synth.random_walk(2600, 50)]
    mins, maxs = [10, 40, 100], [30, 60, 140]
    outs = ctx.palmad_find_discords_batch(series, mins, maxs, 2, _opts(batch_lengths=8, pool_slots=64, **ALL_TC))
    for T, a, b, o in zip(series, mins, maxs, outs):
        _check_merlin(o, oracle.merlin(T, a, b, 2, True))


def test_mixed_equals_fp32_full_size(ctx):
    """sine100k, all 129 lengths, batched: identical results in the FP32
    form, the mixed form, and the mixed form with every survivor on the
    tensor cores."""
    w = synth.workload("sine100k")
    T = w.series[0]
    args = (T, w.minL[0], w.maxL[0], w.topK)
    a = ctx.palmad_find_discords(*args, _opts(batch_lengths=16), heatmap=True)
    for o in (_opts(batch_lengths=16, precision=MIXED), _opts(batch_lengths=16, **ALL_TC)):
        b = ctx.palmad_find_discords(*args, o, heatmap=True)
        for k in ("idx", "nn", "count", "r", "heatmap"):
            np.testing.assert_array_equal(a[k], b[k])
    st = ctx.palmad_get_stats()
    assert st["refine_pairs"] > 0


@pytest.mark.parametrize("name", ["rw3000", "sine4000", "flat2200"])
def test_fp32_direct_form_matches_oracle(ctx, name):
    """Every survivor on the FP32 direct form (direct_below = 129)."""
    T = SERIES[name]()
    for m in (8, 37, 100):
        mp, _ = oracle.matrix_profile(T, m)
        for r in _thresholds(mp, (0.5, 0.99)):
            _check_drag(ctx, T, m, float(r), _opts(direct_below=129))


@pytest.mark.parametrize("name", list(SERIES))
@pytest.mark.parametrize("m", [8, 37, 100, 300])
def test_tc_seeds_drag_matches_oracle(ctx, name, m):
    """Tensor-core top-row seeds for every refine strip of the sweep."""
    T = SERIES[name]()
    if len(T) < 2 * m:
        pytest.skip("series too short")
    mp, _ = oracle.matrix_profile(T, m)
    seeded = 0
    for r in _thresholds(mp, (0.5, 0.9, 0.99, 1.0)):
        _check_drag(ctx, T, m, float(r), _opts(**ALL_SEED))
        seeded += ctx.palmad_get_stats()["seed_pairs"]
    assert seeded > 0  # the tensor-core seeds did run


@pytest.mark.parametrize("W", [0, 16])
@pytest.mark.parametrize("name,minL,maxL,K,excl", [
    ("rw3000", 10, 40, 2, True),
    ("sine4000", 50, 70, 3, True),
    ("flat2200", 16, 30, 1, False),
])
def test_tc_seeds_merlin_matches_oracle(ctx, W, name, minL, maxL, K, excl):
    T = SERIES[name]()
    got = ctx.palmad_find_discords(T, minL, maxL, K, _opts(exclusive_topk=int(excl), batch_lengths=W, **ALL_SEED),
                                   heatmap=True)
    assert ctx.palmad_get_stats()["seed_pairs"] > 0
    _check_merlin(got, oracle.merlin(T, minL, maxL, K, excl, heatmap=True), heat=True)


@pytest.mark.parametrize("cap", [1, 5, 40])
def test_tc_seeds_row_cap_and_rounds(ctx, cap):
    """Seed rows clipped to a small cap (the rest seed on the CUDA cores),
    with many refine rounds and lanes of different lengths."""
    series = [SERIES["rw3000"](), SERIES["sine4000"](), synth.random_walk(2600, 50)]
    mins, maxs = [10, 40, 100], [30, 60, 140]
    outs = ctx.palmad_find_discords_batch(series, mins, maxs, 2, _opts(batch_lengths=8, pool_slots=256,
                                                                          seed_rows_max=cap, **ALL_SEED))
    assert ctx.palmad_get_stats()["seed_pairs"] > 0
    for T, a, b, o in zip(series, mins, maxs, outs):
        _check_merlin(o, oracle.merlin(T, a, b, 2, True))


def test_tc_seeds_equal_fp32_full_size(ctx):
    """sine100k: tensor-core seeds (default and every strip) give the FP32
    form's results exactly, and seeds are in fact computed."""
    w = synth.workload("sine100k")
    T = w.series[0]
    args = (T, w.minL[0], w.maxL[0], w.topK)
    a = ctx.palmad_find_discords(*args, _opts(batch_lengths=16), heatmap=True)
    for o in (_opts(batch_lengths=16, precision=MIXED, tc_seed_min=16), _opts(batch_lengths=16, **ALL_SEED)):
        b = ctx.palmad_find_discords(*args, o, heatmap=True)
        for k in ("idx", "nn", "count", "r", "heatmap"):
            np.testing.assert_array_equal(a[k], b[k])
        assert ctx.palmad_get_stats()["seed_pairs"] > 0


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["rw3000", "sine4000", "flat2200"])
def test_long_refine_segments(ctx, prec, name):
    """2048-column refine segments (automatic on long passes), forced here."""
    T = SERIES[name]()
    for m in (8, 100):
        mp, _ = oracle.matrix_profile(T, m)
        for r in _thresholds(mp, (0.5, 0.99)):
            _check_drag(ctx, T, m, float(r), _opts(precision=prec, refine_seg=2048))
    got = ctx.palmad_find_discords(T, 16, 40, 2, _opts(precision=prec, refine_seg=2048, batch_lengths=8), heatmap=True)
    _check_merlin(got, oracle.merlin(T, 16, 40, 2, True, heatmap=True), heat=True)
