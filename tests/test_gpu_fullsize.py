"""GPU parity at the full sizes of the precision, batched and heatmap
workloads, in the form the benchmark times (mixed precision, 16 lengths per
pass) and, where it fits the test budget, the plain FP32 form:

* rw250k   (n = 250 000 random walk, m = 64..512, top-1): at 12 evenly spaced
  lengths the oracle's range discords at the run's final r equal the
  heatmap's nonzero positions, the count and the top-K, with the nnDist of
  every range discord within 1e-5;
* batch256 (256 series of 5 000..60 000 points): 8 seeded series, each at 4
  evenly spaced lengths, against the oracle's range discords at the final r;
* beats1m  (n = 10^6, m = 100..1000, top-1 plus the 3.6 GB heatmap): the
  oracle cannot evaluate a whole length here (a single length holds up to
  3.3e5 range discords, each a brute-force row of 10^6 windows), so at 10
  evenly spaced lengths the top-1 pick and 64 windows per length (seeded
  random ones, seeded ones among the heatmap's nonzero entries, and one
  before every planted abnormal beat) are checked one by one against the
  oracle's brute-force nearest neighbour: a window is a range discord
  exactly when its distance is >= the final r, and its heatmap entry is
  then distance^2 / (2m).

Every workload also checks the final r of every length against the closed
forms of the schedule (Sec. 2.2) applied to the returned distances.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2304_01660_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

NN_RTOL = 1e-5
W_BENCH = 16


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


def _bench_form():
    return _opts(batch_lengths=W_BENCH, precision=1)


def _check_schedule(nn, idx, r, minL):
    """Final r per length from the closed forms of Sec. 2.2 (readings R6-R8):
    2 sqrt(minL) / 2^k, 0.99^(k+1) nnDist_{m-1}, mean - 2 sd - k sd."""
    K = idx.shape[1]
    got = (idx >= 0).sum(axis=1)
    sched = np.where(got > 0, nn[np.arange(len(nn)), np.maximum(got - 1, 0)], 0.0)
    for l in range(len(r)):
        if r[l] <= 0.0:
            continue
        if l == 0:
            k = math.log2(2 * math.sqrt(minL) / r[0])
            assert abs(k - round(k)) < 1e-9, (l, r[l])
        elif l <= 4:
            k = math.log(r[l] / (0.99 * sched[l - 1])) / math.log(0.99)
            assert abs(k - round(k)) < 1e-6 and round(k) >= 0, (l, r[l])
        else:
            last = sched[l - 5:l]
            mu, sd = last.mean(), last.std(ddof=1)
            step = sd if sd > 0 else 0.01 * mu
            k = (mu - 2 * sd - r[l]) / step
            assert abs(k - round(k)) < 1e-6 and round(k) >= 0, (l, r[l])
        if got[l] == K:
            assert sched[l] >= r[l]


def _check_length(T, m, r, count, idx_row, nn_row, K, heat_row=None):
    """Oracle range discords at (m, r) against one length's outputs."""
    oi, on = oracle.range_discords(T, m, r)
    assert count == len(oi), (m, count, len(oi))
    if heat_row is not None:
        N = len(T) - m + 1
        nz = np.nonzero(heat_row[:N])[0]
        np.testing.assert_array_equal(nz, oi)
        assert not np.any(heat_row[N:])
        np.testing.assert_allclose(np.sqrt(heat_row[oi].astype(np.float64) * 2 * m), on, rtol=NN_RTOL)
    wi, wn = oracle.topk(oi, on, m, K, True)
    np.testing.assert_array_equal(idx_row, wi)
    np.testing.assert_allclose(nn_row, wn, rtol=NN_RTOL, atol=0)


# --------------------------------------------------------------------- rw250k

@pytest.fixture(scope="module")
def rw250k(ctx):
    w = synth.workload("rw250k")
    T = w.series[0]
    res = ctx.palmad_find_discords(T, w.minL[0], w.maxL[0], w.topK, _bench_form(), heatmap=True)
    return w, T, res


def test_rw250k_schedule(rw250k):
    w, T, res = rw250k
    _check_schedule(res["nn"], res["idx"], res["r"], w.minL[0])


def test_rw250k_lengths_equal_oracle(rw250k):
    w, T, res = rw250k
    minL, K = w.minL[0], w.topK
    L = res["idx"].shape[0]
    for l in np.linspace(0, L - 1, 12).round().astype(int):
        m = minL + int(l)
        _check_length(T, m, res["r"][l], res["count"][l], res["idx"][l], res["nn"][l], K, res["heatmap"][l])


def test_rw250k_plain_form_is_identical(ctx, rw250k):
    w, T, res = rw250k
    got = ctx.palmad_find_discords(T, w.minL[0], w.maxL[0], w.topK, _opts(), heatmap=True)
    for k in ("idx", "nn", "count", "r", "heatmap"):
        np.testing.assert_array_equal(got[k], res[k])


# ------------------------------------------------------------------- batch256

def test_batch256_sampled_series_equal_oracle(ctx):
    w = synth.workload("batch256")
    outs = ctx.palmad_find_discords_batch(w.series, w.minL, w.maxL, w.topK, _bench_form())
    rng = np.random.default_rng(256)
    for s in sorted(rng.choice(len(w.series), size=8, replace=False).tolist()):
        T, minL, o = w.series[s], w.minL[s], outs[s]
        _check_schedule(o["nn"], o["idx"], o["r"], minL)
        L = o["idx"].shape[0]
        for l in np.linspace(0, L - 1, 4).round().astype(int):
            _check_length(T, minL + int(l), o["r"][l], o["count"][l], o["idx"][l], o["nn"][l], w.topK)


# -------------------------------------------------------------------- beats1m

@pytest.fixture(scope="module")
def beats1m(ctx):
    import torch
    w = synth.workload("beats1m")
    T = w.series[0]
    minL, maxL, K = w.minL[0], w.maxL[0], w.topK
    L, W = maxL - minL + 1, len(T) - minL + 1
    Td = torch.from_numpy(T).cuda()
    heat = torch.empty((L, W), dtype=torch.float32, device="cuda")
    res = ctx.palmad_find_discords_device(Td, minL, maxL, K, _bench_form(), heatmap_dev=heat)
    out = {k: v.cpu().numpy() for k, v in res.items()}
    yield w, T, out, heat
    del heat
    torch.cuda.empty_cache()


def test_beats1m_schedule(beats1m):
    w, T, res, _ = beats1m
    _check_schedule(res["nn"], res["idx"], res["r"], w.minL[0])


def test_beats1m_plain_form_is_identical(ctx, beats1m):
    import torch
    w, T, res, heat = beats1m
    minL, maxL, K = w.minL[0], w.maxL[0], w.topK
    heat2 = torch.empty_like(heat)
    got = ctx.palmad_find_discords_device(torch.from_numpy(T).cuda(), minL, maxL, K, _opts(), heatmap_dev=heat2)
    for k in ("idx", "nn", "count", "r"):
        np.testing.assert_array_equal(got[k].cpu().numpy(), res[k])
    assert torch.equal(heat2, heat)
    del heat2
    torch.cuda.empty_cache()


def test_beats1m_sampled_windows_against_brute_force(beats1m):
    w, T, res, heat = beats1m
    minL, K = w.minL[0], w.topK
    L = res["idx"].shape[0]
    rng = np.random.default_rng(1000)
    for l in np.linspace(0, L - 1, 10).round().astype(int):
        l = int(l)
        m = minL + l
        N = len(T) - m + 1
        r = res["r"][l]
        row = heat[l, :N].cpu().numpy()
        # the count is the heatmap's number of nonzero entries
        assert res["count"][l] == int(np.count_nonzero(row))
        top = res["nn"][l, 0]
        for q in range(K):
            i = int(res["idx"][l, q])
            nn, _ = oracle.nn_one(T, m, i)
            assert res["nn"][l, q] == pytest.approx(nn, rel=NN_RTOL)
            assert nn >= r
        nz = np.nonzero(row)[0]
        wins = rng.integers(0, N, size=24).tolist()
        wins += rng.choice(nz, size=min(24, len(nz)), replace=False).tolist()
        wins += [min(max(0, c - m // 2), N - 1) for c in w.notes["odd_beats"][:16]]
        for i in wins:
            nn, _ = oracle.nn_one(T, m, int(i))
            assert nn <= top * (1 + 1e-9)  # nothing beats the top-1 discord
            if nn >= r:
                assert row[i] == pytest.approx(nn * nn / (2 * m), rel=2 * NN_RTOL), (m, i)
            else:
                assert row[i] == 0.0, (m, i, nn, r)
