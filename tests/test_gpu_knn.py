"""GPU parity of the k-th neighbour variant (the top-k discord definition of
Sec. 2.1 read literally: the distance of a window is the k-th smallest
distance to its non-self matches) against the FP64 oracle, per length and
through MERLIN, in the FP32, mixed and direct forms."""
import numpy as np
import pytest

import oracle
from paper_2304_01660_gb300 import synth

from test_gpu_parity import NN_RTOL, SERIES, _check_merlin, _opts, ctx  # noqa: F401

pytestmark = pytest.mark.gpu

FORMS = [dict(), dict(precision=1), dict(precision=1, direct_below=129)]


def _thresholds(d, qs):
    """Thresholds midway between consecutive distinct finite k-distances
    (no window within rounding distance of r)."""
    v = np.unique(d[np.isfinite(d)])
    return [0.5 * (v[min(int(q * (len(v) - 1)), len(v) - 2)] + v[min(int(q * (len(v) - 1)), len(v) - 2) + 1])
            for q in qs]


def _check(ctx, T, m, k, r, opts, profile=None):
    gi, gn = ctx.palmad_drag(T, m, r, opts)
    wi, wn = oracle.drag_knn(T, m, k, r, profile)
    np.testing.assert_array_equal(gi, wi)
    np.testing.assert_allclose(gn, wn, rtol=NN_RTOL, atol=0)
    return len(wi)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("k", [2, 3, 16])
@pytest.mark.parametrize("name,m", [("rw3000", 20), ("sine4000", 60), ("flat2200", 16)])
def test_knn_drag_matches_oracle(ctx, form, k, name, m):
    T = SERIES[name]()
    d = oracle.knn_profile(T, m, k)
    for r in _thresholds(d, (0.5, 0.95, 1.0)) + [0.0]:
        _check(ctx, T, m, k, float(r), _opts(knn_k=k, **form), d)


def test_knn_1_is_the_nearest_neighbour(ctx):
    T = SERIES["rw3000"]()
    mp, _ = oracle.matrix_profile(T, 25)
    r = float(np.quantile(mp, 0.9))
    a = ctx.palmad_drag(T, 25, r, _opts(knn_k=1))
    b = ctx.palmad_drag(T, 25, r, _opts())
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


@pytest.mark.parametrize("k", [2, 3, 6])
def test_knn_fewer_than_k_matches(ctx, k):
    """n = 2m + 5: windows with fewer than k non-self matches are never
    range k-discords, even at r = 0."""
    m = 40
    T = synth.random_walk(2 * m + 5, 47)
    assert _check(ctx, T, m, k, 0.0, _opts(knn_k=k)) == len(oracle.drag_knn(T, m, k, 0.0)[0])


def test_knn_twin_anomaly(ctx):
    """A burst planted twice: exact twins hide it from the nearest neighbour,
    the second neighbour finds it (same series as the oracle's pin)."""
    rng = np.random.default_rng(40)
    p, m = 50, 30
    x = np.tile(np.sin(2 * np.pi * np.arange(p) / p), 40) + rng.normal(0, 0.02, 40 * p)
    burst = rng.normal(0, 1, 40)
    x[600:640] = burst
    x[1400:1440] = burst
    x = x.astype(np.float32)
    d = oracle.knn_profile(x, m, 2)
    r = float(_thresholds(d, (0.99,))[0])
    _check(ctx, x, m, 2, r, _opts(knn_k=2), d)
    gi, _ = ctx.palmad_drag(x, m, r, _opts(knn_k=2))
    assert all(570 < i < 640 or 1370 < i < 1440 for i in gi)


@pytest.mark.parametrize("W,k,prec", [(0, 2, 0), (8, 4, 1)])
def test_knn_merlin_matches_oracle(ctx, W, k, prec):
    T = SERIES["sine4000"]()
    got = ctx.palmad_find_discords(T, 50, 62, 2, _opts(knn_k=k, batch_lengths=W, precision=prec), heatmap=True)
    want = oracle.merlin(T, 50, 62, 2, True, heatmap=True, knn=k)
    _check_merlin(got, want, heat=True)


def test_knn_option_range(ctx):
    from paper_2304_01660_gb300 import palmad
    T = SERIES["rw3000"]()
    for bad in (-1, 17):
        with pytest.raises(palmad.PalmadError):
            ctx.palmad_drag(T, 20, 1.0, _opts(knn_k=bad))
