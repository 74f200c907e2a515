"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bar: discord indices and counts bit-exact; nearest-neighbour distances within
1e-5 relative (the tolerance the method's exactness claim allows; the GPU
recomputes final distances in FP64, so the observed error is ~1e-12); final
r per length within 1e-9 relative (host FP64 arithmetic on those distances).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2304_01660_gb300 import synth

pytestmark = pytest.mark.gpu

NN_RTOL = 1e-5
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def ctx():
    from paper_2304_01660_gb300 import _build, palmad
    _build.build()
    c = palmad.Context(0)
    yield c
    c.close()


def _opts(**kw):
    from paper_2304_01660_gb300 import palmad
    return palmad.palmad_default_options(**kw)


def _flat_series(n, seed):
    x = synth.random_walk(n, seed).astype(np.float64)
    x[300:420] = 5.0          # a flat stretch (flat windows of every length <= 120)
    x[900:960] = -2.0
    return x.astype(np.float32)


SERIES = {
    "rw3000": lambda: synth.random_walk(3000, 41),
    "rw2999": lambda: synth.random_walk(2999, 42),
    "rw_offset": lambda: (synth.random_walk(2500, 43).astype(np.float64) * 0.5 + 1000.0).astype(np.float32),
    "sine4000": lambda: synth.noisy_sine(4000, 60.0, 0.1, seed=44, anomalies=[(1700, 70), (3100, 50)]),
    "flat2200": lambda: _flat_series(2200, 45),
}


def _thresholds(mp, qs):
    """Thresholds at the given quantiles of the profile, each placed midway
    between two consecutive distinct profile values, so that no window lies
    within rounding distance of r (d == r is a tie two correct FP64
    evaluations may break differently)."""
    v = np.unique(mp[np.isfinite(mp)])
    out = []
    for q in qs:
        k = min(int(q * (len(v) - 1)), len(v) - 2)
        out.append(0.5 * (v[k] + v[k + 1]))
    return out


def _check_drag(ctx, T, m, r, opts=None):
    gi, gn = ctx.palmad_drag(T, m, r, opts)
    wi, wn = oracle.drag(T, m, r)
    np.testing.assert_array_equal(gi, wi)
    np.testing.assert_allclose(gn, wn, rtol=NN_RTOL, atol=0)
    return len(wi)


@pytest.mark.parametrize("name", list(SERIES))
@pytest.mark.parametrize("m", [8, 37, 100])
def test_drag_matches_oracle(ctx, name, m):
    T = SERIES[name]()
    mp, _ = oracle.matrix_profile(T, m)
    for r in _thresholds(mp, (0.5, 0.9, 0.99, 1.0)):
        _check_drag(ctx, T, m, float(r))


def test_drag_degenerate_thresholds(ctx):
    T = SERIES["rw3000"]()
    m = 20
    N = len(T) - m + 1
    # r <= 0: every window with a non-self match is a range discord
    assert _check_drag(ctx, T, m, 0.0) == N
    assert _check_drag(ctx, T, m, -3.0) == N
    # r above the largest possible distance: none
    assert _check_drag(ctx, T, m, 2 * math.sqrt(m) + 1.0) == 0


def test_drag_n_equals_2m(ctx):
    m = 64
    T = synth.random_walk(2 * m, 46)
    n_found = _check_drag(ctx, T, m, 0.0)
    assert n_found == 2  # windows 0 and m, each other's only non-self match


@pytest.mark.parametrize("cap", [1, 32, 100000])
def test_drag_select_cap_does_not_change_results(ctx, cap):
    T = SERIES["sine4000"]()
    mp, _ = oracle.matrix_profile(T, 50)
    r = float(_thresholds(mp, (0.95,))[0])
    _check_drag(ctx, T, 50, r, _opts(select_cap=cap))


@pytest.mark.parametrize("name", list(SERIES))
@pytest.mark.parametrize("m", [8, 100])
def test_drag_tall_refine_strips_match_oracle(ctx, name, m):
    """256-row refine strips (refine_rows = 256): rows up to 255 recurrence
    steps from a direct dot product, every survivor through the sweep."""
    T = SERIES[name]()
    mp, _ = oracle.matrix_profile(T, m)
    for r in _thresholds(mp, (0.5, 0.95, 1.0)):
        _check_drag(ctx, T, m, r, _opts(refine_rows=256, direct_below=1))
        _check_drag(ctx, T, m, r, _opts(refine_rows=256, precision=1))


def test_drag_hints_off_matches_oracle(ctx):
    T = SERIES["sine4000"]()
    for m in (37, 100):
        mp, _ = oracle.matrix_profile(T, m)
        for r in _thresholds(mp, (0.9, 0.99)):
            _check_drag(ctx, T, m, r, _opts(no_hints=1))


def test_drag_golden_fixtures(ctx):
    for case in json.load(open(os.path.join(HERE, "golden", "drag_random_walk.json"))):
        T = synth.random_walk(case["n"], case["seed"])
        gi, gn = ctx.palmad_drag(T, case["m"], case["r"])
        assert gi.tolist() == case["idx"]
        np.testing.assert_allclose(gn, case["nn"], rtol=NN_RTOL)


def _check_merlin(got, want, heat=False):
    np.testing.assert_array_equal(got["idx"], want["idx"])
    np.testing.assert_allclose(got["nn"], want["nn"], rtol=NN_RTOL, atol=0)
    np.testing.assert_array_equal(got["count"], want["count"])
    np.testing.assert_allclose(got["r"], want["r"], rtol=1e-9, atol=1e-12)
    if heat:
        np.testing.assert_allclose(got["heatmap"], want["heatmap"], rtol=2 * NN_RTOL, atol=0)


def test_merlin_golden_tiny(ctx):
    g = json.load(open(os.path.join(HERE, "golden", "tiny_merlin.json")))
    T = synth.workload("tiny").series[0]
    got = ctx.palmad_find_discords(T, g["minL"], g["maxL"], g["topK"])
    assert got["idx"].tolist() == g["idx"]
    np.testing.assert_allclose(got["nn"], g["nn"], rtol=NN_RTOL)
    assert got["count"].tolist() == g["count"]
    np.testing.assert_allclose(got["r"], g["r"], rtol=1e-9)


@pytest.mark.parametrize("name,minL,maxL,K,excl", [
    ("rw3000", 10, 30, 3, True),
    ("rw2999", 16, 24, 2, False),
    ("rw_offset", 30, 45, 1, True),
    ("sine4000", 40, 60, 2, True),
    ("flat2200", 20, 28, 2, True),
])
def test_merlin_matches_oracle(ctx, name, minL, maxL, K, excl):
    T = SERIES[name]()
    got = ctx.palmad_find_discords(T, minL, maxL, K, _opts(exclusive_topk=int(excl)), heatmap=True)
    want = oracle.merlin(T, minL, maxL, K, excl, heatmap=True)
    _check_merlin(got, want, heat=True)


@pytest.mark.parametrize("W", [4, 16])
@pytest.mark.parametrize("name,minL,maxL,K,excl", [
    ("rw3000", 10, 40, 3, True),
    ("sine4000", 40, 75, 2, True),
    ("flat2200", 20, 45, 2, False),
])
def test_merlin_batched_matches_oracle(ctx, W, name, minL, maxL, K, excl):
    """Batched form: W lengths per pass at a speculative r, exact replay."""
    T = SERIES[name]()
    got = ctx.palmad_find_discords(T, minL, maxL, K, _opts(exclusive_topk=int(excl), batch_lengths=W), heatmap=True)
    want = oracle.merlin(T, minL, maxL, K, excl, heatmap=True)
    _check_merlin(got, want, heat=True)


@pytest.mark.parametrize("W", [0, 8])
def test_refine_rounds_match_oracle(ctx, W):
    """A tiny survivor pool forces many refine rounds per pass (lanes split
    across rounds, strips split across rounds)."""
    series = [SERIES["rw3000"](), SERIES["sine4000"](), synth.random_walk(2600, 50)]
    mins, maxs = [10, 40, 14], [30, 60, 36]
    outs = ctx.palmad_find_discords_batch(series, mins, maxs, 2, _opts(batch_lengths=W, pool_slots=64))
    for T, a, b, o in zip(series, mins, maxs, outs):
        _check_merlin(o, oracle.merlin(T, a, b, 2, True))
    T = SERIES["rw3000"]()
    mp, _ = oracle.matrix_profile(T, 25)
    r = float(_thresholds(mp, (0.3,))[0])
    _check_drag(ctx, T, 25, r, _opts(pool_slots=100))


def test_merlin_options_do_not_change_results(ctx):
    T = SERIES["rw3000"]()
    base = ctx.palmad_find_discords(T, 12, 20, 2)
    for o in (_opts(band_rel=0.05), _opts(band_rel=1e-6), _opts(select_cap=1), _opts(profile=1),
              _opts(no_hints=1), _opts(refine_rows=256), _opts(batch_lengths=8, spec_scale=10),
              _opts(batch_lengths=8, spec_scale=400)):
        _check_merlin(ctx.palmad_find_discords(T, 12, 20, 2, o), base)


def test_device_entry_equals_host_entry(ctx):
    import torch
    T = SERIES["sine4000"]()
    host = ctx.palmad_find_discords(T, 40, 50, 2)
    dev = ctx.palmad_find_discords_device(torch.from_numpy(T).cuda(), 40, 50, 2)
    np.testing.assert_array_equal(dev["idx"].cpu().numpy(), host["idx"])
    np.testing.assert_array_equal(dev["nn"].cpu().numpy(), host["nn"])
    np.testing.assert_array_equal(dev["count"].cpu().numpy(), host["count"])
    np.testing.assert_array_equal(dev["r"].cpu().numpy(), host["r"])


@pytest.mark.parametrize("W", [0, 8])
def test_batch_entry_equals_oracle(ctx, W):
    series = [SERIES["rw3000"](), SERIES["sine4000"](), synth.random_walk(1800, 47), synth.random_walk(2500, 49)]
    mins, maxs = [10, 40, 30, 12], [24, 58, 33, 40]
    outs = ctx.palmad_find_discords_batch(series, mins, maxs, 2, _opts(batch_lengths=W))
    for T, a, b, o in zip(series, mins, maxs, outs):
        want = oracle.merlin(T, a, b, 2, True)
        _check_merlin(o, want)


def test_affine_invariance(ctx):
    T = SERIES["sine4000"]()
    T2 = (3.7 * T.astype(np.float64) - 11.0).astype(np.float32)
    a = ctx.palmad_find_discords(T, 40, 46, 2)
    b = ctx.palmad_find_discords(T2, 40, 46, 2)
    np.testing.assert_array_equal(a["idx"], b["idx"])
    np.testing.assert_allclose(a["nn"], b["nn"], rtol=1e-4)


def test_errors_are_reported(ctx):
    from paper_2304_01660_gb300 import palmad
    T = synth.random_walk(500, 48)
    bad = T.copy()
    bad[123] = np.nan
    with pytest.raises(palmad.PalmadError) as e:
        ctx.palmad_find_discords(bad, 10, 12, 1)
    assert e.value.status == -2
    for args in ((T, 2, 5, 1), (T, 10, 9, 1), (T, 10, 300, 1), (T, 10, 12, 0), (T, 10, 12, 2000)):
        with pytest.raises(palmad.PalmadError) as e:
            ctx.palmad_find_discords(*args)
        assert e.value.status == -1
    # the context stays usable after an error
    _check_drag(ctx, T, 10, 2.0)


# ------------------------------------------------------------ full-size sampled

@pytest.fixture(scope="module")
def sine100k(ctx):
    w = synth.workload("sine100k")
    T = w.series[0]
    res = ctx.palmad_find_discords(T, w.minL[0], w.maxL[0], w.topK, heatmap=True)
    return w, T, res


def test_full_size_schedule_closed_forms(sine100k):
    """The final r of every length follows Algorithm 1 from the returned
    distances (readings R6-R8 of the oracle header)."""
    w, T, res = sine100k
    minL, K = w.minL[0], w.topK
    sched = res["nn"][:, K - 1]
    r = res["r"]
    for l in range(len(r)):
        if l == 0:
            k = math.log2(2 * math.sqrt(minL) / r[0])
            assert abs(k - round(k)) < 1e-9
        elif l <= 4:
            k = math.log(r[l] / (0.99 * sched[l - 1])) / math.log(0.99)
            assert abs(k - round(k)) < 1e-6 and round(k) >= 0
        else:
            last = sched[l - 5:l]
            mu, sd = last.mean(), last.std(ddof=1)
            k = (mu - 2 * sd - r[l]) / sd
            assert abs(k - round(k)) < 1e-6 and round(k) >= 0
        assert res["nn"][l, K - 1] >= r[l]


def test_full_size_batched_equals_plain(ctx, sine100k):
    """The batched form returns exactly the plain form's results."""
    w, T, plain = sine100k
    got = ctx.palmad_find_discords(T, w.minL[0], w.maxL[0], w.topK, _opts(batch_lengths=16), heatmap=True)
    for k in ("idx", "nn", "count", "r", "heatmap"):
        np.testing.assert_array_equal(got[k], plain[k])


def test_full_size_sampled_against_brute_force(sine100k):
    w, T, res = sine100k
    minL, K = w.minL[0], w.topK
    rng = np.random.default_rng(7)
    L = res["idx"].shape[0]
    for l in sorted(set([0, 1, 5, L // 2, L - 1])):
        m = minL + l
        N = len(T) - m + 1
        for q in range(K):
            i = int(res["idx"][l, q])
            nn, j = oracle.nn_one(T, m, i)
            assert res["nn"][l, q] == pytest.approx(nn, rel=NN_RTOL)
        heat = res["heatmap"][l]
        for i in rng.integers(0, N, size=12):
            nn, _ = oracle.nn_one(T, m, int(i))
            assert nn <= res["nn"][l, 0] * (1 + 1e-9)  # nothing beats the top-1 discord
            if nn >= res["r"][l]:
                assert heat[i] == pytest.approx(nn * nn / (2 * m), rel=2 * NN_RTOL)
            else:
                assert heat[i] == 0.0
        # anomalies planted at known places: the top-1 discord touches one
        starts = w.notes["anomaly_starts"]
        i1 = int(res["idx"][l, 0])
        assert any(s - m < i1 < s + 150 for s in starts)
