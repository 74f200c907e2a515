"""Pins for the FP64 oracle against things other than itself.

Each pin is chosen so a plausible slip in the oracle (a dropped term, a sign,
an off-by-one in the exclusion zone, a transposed operand, a wrong schedule
factor) fails at least one of them:

* window statistics  -- numpy mean / std (ddof=0) and the Eq. 7-8 recurrence
  lemma of the appendix (a different formula from the oracle's two-pass);
* distance           -- scipy z-scores + Euclidean norm (library), the
  dot-product form of Eq. 6 evaluated independently, closed forms
  (x vs -x is 2 sqrt(m), x vs a x + b is 0), symmetry and the 2 sqrt(m) bound;
* nearest neighbour  -- pure-Python brute force on tiny series, exact zero on
  an exactly periodic series, invariance under T -> aT + b, the n = 2m case;
* range discords     -- the set one DRAG call returns: {i : MP(i) >= r} with
  nnDist = MP(i), against the C brute force and the pure-Python one;
* top-K / MERLIN     -- greedy top-K over the brute-force profile, the r
  schedule's closed forms (2 sqrt(minL) / 2^k, 0.99^k, mean - 2 sd - k sd),
  the success condition and the heatmap of Eq. 10.
"""
import math

import numpy as np
import pytest
import scipy.stats

import oracle
from paper_2304_01660_gb300 import synth


def _rw(n, seed):
    return synth.random_walk(n, seed)


# ---------------------------------------------------------------- statistics

def test_stats_match_numpy():
    T = _rw(500, 1) * 3.0 + 100.0
    for m in (3, 7, 32):
        mu, sd = oracle.stats(T, m)
        W = np.lib.stride_tricks.sliding_window_view(T.astype(np.float64), m)
        np.testing.assert_allclose(mu, W.mean(axis=1), rtol=1e-13, atol=1e-11)
        np.testing.assert_allclose(sd, W.std(axis=1, ddof=0), rtol=1e-11)


def test_stats_recurrence_lemma():
    """Eq. 7-8: mu_{m+1} = (m mu_m + t_{i+m})/(m+1),
    sigma^2_{m+1} = m/(m+1) (sigma^2_m + (mu_m - t_{i+m})^2/(m+1))."""
    T = _rw(800, 2)
    t = T.astype(np.float64)
    m0, m1 = 10, 60
    mu, sd = oracle.stats(T, m0)
    var = sd ** 2
    for m in range(m0, m1):
        N1 = len(T) - (m + 1) + 1
        x = t[m:m + N1]
        mu_n = (m * mu[:N1] + x) / (m + 1)
        var_n = m / (m + 1) * (var[:N1] + (mu[:N1] - x) ** 2 / (m + 1))
        mu_o, sd_o = oracle.stats(T, m + 1)
        np.testing.assert_allclose(mu_o, mu_n, rtol=1e-12, atol=1e-10)
        np.testing.assert_allclose(sd_o ** 2, var_n, rtol=1e-9)
        mu, var = mu_n, var_n


# ------------------------------------------------------------------ distance

def test_dist_matches_scipy_zscore():
    T = _rw(300, 3)
    rng = np.random.default_rng(0)
    for m in (4, 16, 50):
        for _ in range(20):
            i, j = rng.integers(0, len(T) - m + 1, size=2)
            a = scipy.stats.zscore(T[i:i + m].astype(np.float64))
            b = scipy.stats.zscore(T[j:j + m].astype(np.float64))
            assert oracle.dist(T, m, i, j) == pytest.approx(np.linalg.norm(a - b), rel=1e-10, abs=1e-10)


def test_dist_matches_eq6_dot_product_form():
    """ED^2_norm = 2m (1 - (X.Y - m mu_X mu_Y) / (m sigma_X sigma_Y))."""
    T = _rw(400, 4) + 50.0
    rng = np.random.default_rng(1)
    for m in (5, 33, 100):
        for _ in range(20):
            i, j = rng.integers(0, len(T) - m + 1, size=2)
            X, Y = T[i:i + m].astype(np.float64), T[j:j + m].astype(np.float64)
            mx, my = X.mean(), Y.mean()
            sx, sy = X.std(), Y.std()
            d2 = 2 * m * (1 - (X @ Y - m * mx * my) / (m * sx * sy))
            assert oracle.dist(T, m, i, j) ** 2 == pytest.approx(max(d2, 0.0), rel=1e-7, abs=1e-7)


def test_dist_closed_forms_and_bounds():
    rng = np.random.default_rng(5)
    m = 24
    x = rng.standard_normal(m)
    T = np.concatenate([x, -x, 2.5 * x + 7.0]).astype(np.float32)
    # anti-correlated windows are at the maximum distance 2 sqrt(m) (Sec. 2.2)
    assert oracle.dist(T, m, 0, m) == pytest.approx(2 * math.sqrt(m), rel=1e-6)
    # an affine copy is at distance 0
    assert oracle.dist(T, m, 0, 2 * m) == pytest.approx(0.0, abs=1e-5)
    # identity, symmetry and the 2 sqrt(m) bound
    R = _rw(200, 6)
    for i, j in [(0, 50), (10, 140), (77, 3)]:
        assert oracle.dist(R, m, i, i) == 0.0
        assert oracle.dist(R, m, i, j) == pytest.approx(oracle.dist(R, m, j, i), rel=1e-14)
        assert 0.0 <= oracle.dist(R, m, i, j) <= 2 * math.sqrt(m) + 1e-12


def test_dist_flat_windows():
    """Reading R2: two flat windows are at 0, flat vs non-flat at sqrt(2m)."""
    m = 8
    T = np.concatenate([np.full(m, 3.0), np.full(m, -1.0), np.arange(m, dtype=float)]).astype(np.float32)
    assert oracle.dist(T, m, 0, m) == 0.0
    assert oracle.dist(T, m, 0, 2 * m) == pytest.approx(math.sqrt(2 * m))


# ------------------------------------------------------- nearest neighbour

def _py_profile(T, m):
    """Pure-Python brute force: z-scores by hand, every non-self pair."""
    N = len(T) - m + 1
    Z = []
    for i in range(N):
        w = [float(v) for v in T[i:i + m]]
        mu = sum(w) / m
        sd = math.sqrt(sum((v - mu) ** 2 for v in w) / m)
        Z.append([(v - mu) / sd for v in w])
    mp, idx = [], []
    for i in range(N):
        best, arg = math.inf, -1
        for j in range(N):
            if abs(i - j) < m:
                continue
            d = math.sqrt(sum((a - b) ** 2 for a, b in zip(Z[i], Z[j])))
            if d < best:
                best, arg = d, j
        mp.append(best)
        idx.append(arg)
    return np.array(mp), np.array(idx)


@pytest.mark.parametrize("n,m,seed", [(40, 4, 0), (60, 7, 1), (75, 12, 2)])
def test_profile_matches_python_brute_force(n, m, seed):
    T = _rw(n, seed)
    mp, idx = oracle.matrix_profile(T, m)
    ref, ridx = _py_profile(T, m)
    np.testing.assert_allclose(mp, ref, rtol=1e-9, atol=1e-9)
    fin = np.isfinite(ref)
    assert np.all(np.abs(idx[fin] - np.arange(len(T) - m + 1)[fin]) >= m)
    # the returned neighbour realises the minimum
    for i in np.nonzero(fin)[0]:
        assert oracle.dist(T, m, i, idx[i]) == pytest.approx(mp[i], rel=1e-12, abs=1e-12)


def test_nn_one_matches_profile_rows():
    T = _rw(500, 15)
    for m in (8, 40):
        mp, idx = oracle.matrix_profile(T, m)
        for i in (0, 7, 250, len(T) - m):
            nn, j = oracle.nn_one(T, m, i)
            assert nn == pytest.approx(mp[i], rel=1e-14)
            assert oracle.dist(T, m, i, j) == pytest.approx(mp[i], rel=1e-12)


def test_profile_exact_repetition_is_zero():
    rng = np.random.default_rng(9)
    pat = rng.standard_normal(37)
    T = np.tile(pat, 8).astype(np.float32)
    mp, _ = oracle.matrix_profile(T, 20)
    assert np.all(mp < 1e-5)


def test_profile_affine_invariance():
    T = _rw(300, 10)
    mp, _ = oracle.matrix_profile(T, 16)
    mp2, _ = oracle.matrix_profile((3.7 * T.astype(np.float64) - 11.0).astype(np.float32), 16)
    np.testing.assert_allclose(mp, mp2, rtol=1e-4, atol=1e-4)


def test_profile_n_equals_2m():
    """n = 2m: only windows 0 and m have a non-self match, each other."""
    m = 16
    T = _rw(2 * m, 11)
    mp, idx = oracle.matrix_profile(T, m)
    assert idx[0] == m and idx[m] == 0
    assert mp[0] == pytest.approx(oracle.dist(T, m, 0, m))
    assert np.all(np.isinf(mp[1:m])) and np.all(idx[1:m] == -1)


# ------------------------------------------------------------------- DRAG

@pytest.mark.parametrize("n,m,seed", [(400, 8, 12), (600, 20, 13), (300, 30, 14)])
def test_drag_equals_thresholded_profile(n, m, seed):
    T = _rw(n, seed)
    mp, _ = oracle.matrix_profile(T, m)
    fin = np.isfinite(mp)
    qs = np.quantile(mp[fin], [0.0, 0.5, 0.9, 0.99, 1.0])
    for r in list(qs) + [0.0, -1.0, 1e-9, mp[fin].max() + 1.0, 2 * math.sqrt(m)]:
        idx, nn = oracle.drag(T, m, r)
        want = np.nonzero(fin & (mp >= r))[0] if r > 0 else np.nonzero(fin)[0]
        np.testing.assert_array_equal(idx, want)
        np.testing.assert_allclose(nn, mp[want], rtol=1e-12, atol=1e-12)
        assert np.all(nn >= r)


@pytest.mark.parametrize("n,m,seed", [(60, 7, 1), (75, 12, 2)])
def test_range_discords_match_python_brute_force(n, m, seed):
    """Sec. 2.1's definition written out in Python: every window whose nearest
    non-self match is at least r away, with that distance."""
    T = _rw(n, seed)
    ref, _ = _py_profile(T, m)
    fin = np.isfinite(ref)
    for q in (0.0, 0.3, 0.7, 0.95):
        r = float(np.quantile(ref[fin], q))
        idx, nn = oracle.range_discords(T, m, r)
        want = np.nonzero(fin & (ref >= r))[0]
        # a window within rounding of r may fall on either side
        near = np.abs(ref - r) <= 1e-9 * max(1.0, r)
        assert set(idx.tolist()) ^ set(want.tolist()) <= set(np.nonzero(near)[0].tolist())
        np.testing.assert_allclose(nn, ref[idx], rtol=1e-9, atol=1e-9)


def test_range_discord_windows_is_the_same_test():
    T = _rw(800, 16)
    m = 20
    mp, _ = oracle.matrix_profile(T, m)
    r = float(np.quantile(mp[np.isfinite(mp)], 0.9))
    idx, nn = oracle.range_discords(T, m, r)
    wins = np.arange(0, len(T) - m + 1, 7)
    got = oracle.range_discord_windows(T, m, r, wins)
    want = np.full(len(wins), np.nan)
    pos = {int(i): v for i, v in zip(idx, nn)}
    for q, i in enumerate(wins):
        if int(i) in pos:
            want[q] = pos[int(i)]
    np.testing.assert_array_equal(np.isnan(got), np.isnan(want))
    np.testing.assert_array_equal(got[~np.isnan(got)], want[~np.isnan(want)])
    with pytest.raises(ValueError):
        oracle.range_discord_windows(T, m, r, [len(T)])


def test_drag_on_sine_finds_injected_anomaly():
    n, m = 3000, 40
    x = synth.noisy_sine(n, 50.0, 0.05, seed=3, anomalies=[(1500, 45)])
    mp, _ = oracle.matrix_profile(x, m)
    top = int(np.nanargmax(np.where(np.isfinite(mp), mp, -1)))
    assert 1500 - m < top < 1500 + 45
    idx, nn = oracle.drag(x, m, 0.99 * mp[top])
    assert top in idx.tolist()


# --------------------------------------------------------- top-K and MERLIN

def _greedy(mp, m, K, exclusive=True):
    order = sorted(np.nonzero(np.isfinite(mp))[0].tolist(), key=lambda i: (-mp[i], i))
    picks = []
    for i in order:
        if len(picks) == K:
            break
        if not exclusive or all(abs(i - p) >= m for p in picks):
            picks.append(i)
    return picks


def test_topk_greedy_exclusion():
    rng = np.random.default_rng(3)
    idx = np.arange(200)
    nn = rng.random(200)
    for K in (1, 3, 7):
        for excl in (True, False):
            oi, on = oracle.topk(idx, nn, 10, K, excl)
            want = _greedy(nn, 10, K, excl)
            assert oi.tolist() == want
            np.testing.assert_array_equal(on, nn[want])


@pytest.mark.parametrize("K,exclusive", [(1, True), (3, True), (2, False)])
def test_merlin_against_brute_force(K, exclusive):
    T = _rw(700, 21)
    minL, maxL = 10, 22
    res = oracle.merlin(T, minL, maxL, K, exclusive, heatmap=True)
    sched = []
    for l, m in enumerate(range(minL, maxL + 1)):
        mp, _ = oracle.matrix_profile(T, m)
        fin = np.isfinite(mp)
        picks = _greedy(mp, m, K, exclusive)
        # top-K equals greedy over the whole profile (independent of r)
        assert res["idx"][l].tolist() == picks
        np.testing.assert_allclose(res["nn"][l], mp[picks], rtol=1e-12)
        r = res["r"][l]
        kth = mp[picks[-1]]
        # success: the K-th pick clears the final r ...
        assert kth >= r
        # ... the count is the number of range discords at the final r ...
        assert res["count"][l] == int(np.sum(fin & (mp >= r)))
        # ... and the heatmap row is nnDist^2 / (2m) on them (Eq. 10)
        row = res["heatmap"][l]
        want = np.where(fin & (mp >= r), mp ** 2 / (2 * m), 0.0)
        want = np.concatenate([want, np.zeros(len(row) - len(want))])
        np.testing.assert_allclose(row, want.astype(np.float32), rtol=1e-6)
        calls = res["calls"][l]
        # closed forms of the r schedule (Algorithm 1 with readings R6/R7)
        if l == 0:
            r0 = 2 * math.sqrt(minL)
            assert r == pytest.approx(r0 / 2 ** (calls - 1), rel=1e-15)
            prev = r0 / 2 ** (calls - 2) if calls > 1 else None
        elif l <= 4:
            base = 0.99 * sched[-1]
            assert r == pytest.approx(base * 0.99 ** (calls - 1), rel=1e-12)
            prev = base * 0.99 ** (calls - 2) if calls > 1 else None
        else:
            last5 = np.array(sched[-5:])
            mu, sd = last5.mean(), last5.std(ddof=1)
            assert r == pytest.approx(mu - 2 * sd - (calls - 1) * sd, rel=1e-9, abs=1e-12)
            prev = mu - 2 * sd - (calls - 2) * sd if calls > 1 else None
        if prev is not None:
            # the previous, higher r failed: fewer than K greedy picks above it
            assert kth < prev
        sched.append(kth)


def test_merlin_sine_anomaly_is_top_discord():
    n = 4000
    x = synth.noisy_sine(n, 60.0, 0.05, seed=8, anomalies=[(2000, 70)])
    res = oracle.merlin(x, 50, 56, 1)
    for l in range(7):
        i = res["idx"][l, 0]
        assert 2000 - (50 + l) < i < 2070


# ------------------------------------------------- stored oracle fixtures

def test_golden_fixtures_reproduce():
    """The committed fixtures (written by tests/golden/make_golden.py from the
    oracle alone) still match the oracle."""
    import json
    import os
    here = os.path.join(os.path.dirname(__file__), "golden")
    g = json.load(open(os.path.join(here, "tiny_merlin.json")))
    w = synth.workload("tiny")
    res = oracle.merlin(w.series[0], g["minL"], g["maxL"], g["topK"], g["exclusive"])
    assert res["idx"].tolist() == g["idx"]
    np.testing.assert_allclose(res["nn"], g["nn"], rtol=1e-12)
    assert res["count"].tolist() == g["count"]
    np.testing.assert_allclose(res["r"], g["r"], rtol=1e-12)
    for case in json.load(open(os.path.join(here, "drag_random_walk.json"))):
        T = synth.random_walk(case["n"], case["seed"])
        idx, nn = oracle.drag(T, case["m"], case["r"])
        assert idx.tolist() == case["idx"]
        np.testing.assert_allclose(nn, case["nn"], rtol=1e-12)


# ------------------------------------------------------------ Eq. 11 interest

def _sparse_heat(L, W, seed, density=0.05):
    rng = np.random.default_rng(seed)
    h = np.where(rng.random((L, W)) < density, rng.random((L, W)), 0.0).astype(np.float32)
    h[:, 5] = 0.25   # equal along m: the smallest length wins the tie
    h[:, 9] = 0.0
    h[2, 9] = h[4, 9] = 0.75
    return h


def test_interest_is_columnwise_max_with_first_length():
    """Eq. 11 per index reduces to numpy's column max and first argmax."""
    h = _sparse_heat(7, 300, 1)
    got = oracle.interest(h, 40, 3)
    np.testing.assert_array_equal(got["score"], h.max(axis=0))
    np.testing.assert_array_equal(got["best_m"], 40 + h.argmax(axis=0))
    assert got["best_m"][5] == 40 and got["best_m"][9] == 42


def test_interest_plain_topk_is_a_sort():
    """Without the overlap rule the picks are the K largest positive scores,
    ties to the lower index (numpy lexsort)."""
    h = _sparse_heat(5, 400, 2)
    s = h.max(axis=0)
    order = np.lexsort((np.arange(len(s)), -s))
    order = [i for i in order if s[i] > 0][:25]
    got = oracle.interest(h, 10, 25, exclusive=False)
    np.testing.assert_array_equal(got["idx"], order)
    np.testing.assert_array_equal(got["value"], s[order])


def test_interest_exclusive_hand_example():
    h = np.zeros((3, 40), np.float32)
    h[0, 10] = 0.9                 # length 20: window [10, 30)
    h[2, 28] = 0.8                 # length 22: [28, 50) overlaps [10, 30): skipped
    h[1, 31] = 0.7                 # length 21: [31, 52) clear of [10, 30)
    h[0, 0] = 0.6                  # length 20: [0, 20) overlaps [10, 30): skipped
    got = oracle.interest(h, 20, 4)
    assert got["idx"].tolist() == [10, 31, -1, -1]
    assert got["m"].tolist() == [20, 21, 0, 0]
    got = oracle.interest(h, 20, 4, exclusive=False)
    assert got["idx"].tolist() == [10, 28, 31, 0]


def test_interest_empty_heatmap():
    got = oracle.interest(np.zeros((4, 50), np.float32), 8, 2)
    assert got["idx"].tolist() == [-1, -1] and got["value"].tolist() == [0.0, 0.0]


def test_interest_top1_is_a_per_length_top1():
    """The most interesting discord (Eq. 11) is the per-length top-1 discord
    whose nnDist^2 / (2m) (Eq. 10) is largest."""
    T = synth.random_walk(1500, 3)
    minL, maxL = 20, 27
    res = oracle.merlin(T, minL, maxL, 1, True, heatmap=True)
    got = oracle.interest(res["heatmap"], minL, 1)
    ms = np.arange(minL, maxL + 1)
    val = (res["nn"][:, 0] ** 2 / (2 * ms)).astype(np.float32)
    l = int(np.argmax(val))
    assert got["idx"][0] == res["idx"][l, 0]
    assert got["value"][0] == val[l]


# ------------------------------------ k-th neighbour variant (reading R14)

def _py_knn(T, m, k):
    """numpy brute force: z-scores by numpy, every non-self distance of a row
    sorted; the R2 convention for flat windows; inf where a window has fewer
    than k non-self matches."""
    T = np.asarray(T, dtype=np.float64)
    N = len(T) - m + 1
    W = np.lib.stride_tricks.sliding_window_view(T, m)
    mu, sd = W.mean(axis=1), W.std(axis=1)
    flat = sd <= 2.0 ** -22 * np.abs(mu)
    Z = (W - mu[:, None]) / np.where(flat, 1.0, sd)[:, None]
    out = np.full(N, np.inf)
    for i in range(N):
        j = np.array([j for j in range(N) if abs(i - j) >= m], dtype=np.int64)
        if len(j) < k:
            continue
        d2 = ((Z[j] - Z[i]) ** 2).sum(axis=1)
        d2 = np.where(flat[j] & flat[i], 0.0, np.where(flat[j] | flat[i], 2.0 * m, d2))
        out[i] = math.sqrt(np.sort(d2)[k - 1])
    return out


@pytest.mark.parametrize("k", [1, 2, 4, 7])
@pytest.mark.parametrize("n,m,seed", [(60, 5, 30), (90, 9, 31)])
def test_knn_matches_numpy_brute_force(n, m, seed, k):
    T = _rw(n, seed)
    np.testing.assert_allclose(oracle.knn_profile(T, m, k), _py_knn(T, m, k), rtol=1e-9, atol=1e-9)


def test_knn_with_flat_windows():
    T = np.concatenate([_rw(40, 32), np.full(20, 2.5), _rw(40, 33)]).astype(np.float32)
    for k in (1, 3):
        np.testing.assert_allclose(oracle.knn_profile(T, 6, k), _py_knn(T, 6, k), rtol=1e-9, atol=1e-9)


def test_knn_k1_is_the_matrix_profile():
    T = _rw(400, 34)
    for m in (6, 25):
        mp, _ = oracle.matrix_profile(T, m)
        np.testing.assert_array_equal(oracle.knn_profile(T, m, 1), mp)


def test_knn_nondecreasing_in_k():
    T = _rw(300, 35)
    prev = oracle.knn_profile(T, 12, 1)
    for k in range(2, 9):
        cur = oracle.knn_profile(T, 12, k)
        assert np.all(cur >= prev)
        prev = cur


def test_knn_exact_copies_closed_form():
    """A pattern tiled exactly: window i has an exact copy at every non-self
    j = i (mod p), so its k-distance is 0 for k up to that number of copies
    and positive beyond it."""
    p, m = 23, 9
    T = np.tile(_rw(p, 36), 9).astype(np.float32)
    N = len(T) - m + 1
    copies = np.array([sum(1 for j in range(i % p, N, p) if abs(i - j) >= m) for i in range(N)])
    for k in (1, 2, 5, 8):
        d = oracle.knn_profile(T, m, k)
        assert np.all(d[copies >= k] == 0.0)
        assert np.all(d[copies < k] > 1e-3)


def test_knn_fewer_than_k_matches():
    """n = 2m + 5: the middle windows have few non-self matches; a window
    with fewer than k has no k-distance and is never a range k-discord."""
    m = 10
    T = _rw(2 * m + 5, 37)
    N = len(T) - m + 1
    cnt = np.array([sum(1 for j in range(N) if abs(i - j) >= m) for i in range(N)])
    for k in (1, 2, 3, 6):
        d = oracle.knn_profile(T, m, k)
        assert np.array_equal(np.isfinite(d), cnt >= k)
        idx, _ = oracle.drag_knn(T, m, k, 0.0)
        assert idx.tolist() == np.nonzero(cnt >= k)[0].tolist()


def test_drag_knn_is_the_thresholded_profile():
    T = _rw(500, 38)
    m = 15
    for k in (2, 5):
        d = oracle.knn_profile(T, m, k)
        fin = np.isfinite(d)
        for r in (np.quantile(d[fin], 0.5), np.quantile(d[fin], 0.95), 0.0, -1.0):
            idx, nn = oracle.drag_knn(T, m, k, r)
            want = np.nonzero(fin & ((d >= r) | (r <= 0)))[0]
            assert idx.tolist() == want.tolist()
            np.testing.assert_array_equal(nn, d[want])


@pytest.mark.parametrize("k", [2, 4])
def test_merlin_knn_against_brute_force(k):
    """MERLIN on the k-distance: the picks are greedy top-K over the numpy
    k-distance profile (the same lemma as for k = 1: the range discords at r
    are an upper set of the profile), and the count is that of the profile
    at the final r."""
    T = _rw(500, 39)
    minL, maxL, K = 10, 18, 2
    res = oracle.merlin(T, minL, maxL, K, True, heatmap=True, knn=k)
    for l, m in enumerate(range(minL, maxL + 1)):
        d = _py_knn(T, m, k)
        picks = _greedy(d, m, K, True)
        assert res["idx"][l].tolist() == picks
        np.testing.assert_allclose(res["nn"][l], d[picks], rtol=1e-9)
        r = res["r"][l]
        assert res["count"][l] == int(np.sum(np.isfinite(d) & (d >= r)))


def test_knn_finds_a_twin_anomaly():
    """Twin freak: a burst that occurs twice hides from the nearest-neighbour
    distance (each copy matches the other exactly) but not from the second
    neighbour."""
    rng = np.random.default_rng(40)
    p, m = 50, 30
    x = np.tile(np.sin(2 * np.pi * np.arange(p) / p), 40) + rng.normal(0, 0.02, 40 * p)
    burst = rng.normal(0, 1, 40)
    x[600:640] = burst
    x[1400:1440] = burst
    x = x.astype(np.float32)
    d1, d2 = oracle.knn_profile(x, m, 1), oracle.knn_profile(x, m, 2)
    inside = list(range(600, 611)) + list(range(1400, 1411))  # windows within a copy
    far = [i for i in range(len(d1)) if not (570 < i < 640 or 1370 < i < 1440)]
    assert np.all(d1[inside] == 0.0)
    assert d2[inside].min() > d2[far].max()


def test_drag_knn_with_a_given_profile():
    T = _rw(300, 41)
    d = oracle.knn_profile(T, 12, 3)
    r = float(np.quantile(d, 0.8))
    a = oracle.drag_knn(T, 12, 3, r)
    b = oracle.drag_knn(T, 12, 3, r, d)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
