"""The no-allocation top-K entry point against the oracle and the existing
entry points.

palmad_topk_profile_noalloc serves callers that cannot call cudaMalloc (for
example while another allocator owns all device memory, or on a path that
cannot take cudaMalloc's implicit device synchronisation): it uses a fixed
device array of the library instead of allocated scratch.  Its results are
compared element by element with the oracle's greedy top-K (oracle.topk) on
the same profile: exclusive and plain picks, r <= 0 (every finite entry),
+inf and NaN holes, exact ties (the lower index wins), K = 1 and K = 1024,
a profile of exactly PALMAD_NOALLOC_MAX_WINDOWS windows, and a small profile
right after a large one on the same stream (the shared array keeps the
earlier call's entries).  This file is named to run last, so a failure here
cannot hide any other test's result.  It builds the library itself, so it
also runs alone in a fresh process.
"""
import numpy as np
import pytest

import oracle
from paper_2304_01660_gb300 import synth

pytestmark = pytest.mark.gpu

NN_RTOL = 1e-5


@pytest.fixture(scope="module")
def lib():
    from paper_2304_01660_gb300 import _build, palmad
    _build.build()
    return palmad


def _profile(N, seed, holes=True, ties=True):
    """Distances with +inf / NaN holes and exact ties."""
    rng = np.random.default_rng(seed)
    p = rng.gamma(4.0, 1.5, size=N)
    if ties:
        p[rng.integers(0, N, size=N // 50)] = 9.5  # many exact ties
        p[rng.integers(0, N, size=8)] = p.max()     # ties at the top
    if holes:
        p[rng.integers(0, N, size=N // 40)] = np.inf
        p[rng.integers(0, N, size=N // 40)] = np.nan
    return p


def _want(prof, m, r, K, exclusive):
    keep = np.isfinite(prof) & ((r <= 0.0) | (prof >= r))
    idx = np.nonzero(keep)[0]
    oi, on = oracle.topk(idx, prof[idx], m, K, exclusive)
    return oi, on, len(idx)


def _check(lib, prof_dev, prof, m, r, K, exclusive):
    import torch
    gi, gn, gc = lib.palmad_topk_profile_noalloc(prof_dev, m, r, K, exclusive=exclusive)
    torch.cuda.synchronize()
    oi, on, cnt = _want(prof, m, r, K, exclusive)
    np.testing.assert_array_equal(gi.cpu().numpy(), oi)
    np.testing.assert_array_equal(gn.cpu().numpy(), on)  # values are copied, not computed
    assert int(gc.item()) == cnt


@pytest.mark.parametrize("exclusive", [True, False])
@pytest.mark.parametrize("K", [1, 7, 1024])
def test_noalloc_matches_oracle_topk(lib, exclusive, K):
    import torch
    N, m = 20000, 37
    prof = _profile(N, 70 + K)
    d = torch.from_numpy(prof).cuda()
    fin = prof[np.isfinite(prof)]
    for r in (float(np.quantile(fin, 0.9)), 9.5, 0.0, -1.0, float(fin.max()) + 1.0):
        _check(lib, d, prof, m, r, K, exclusive)


def test_noalloc_at_the_size_limit_then_small(lib):
    """N exactly at the cap, then a much smaller profile on the same stream
    with no synchronisation in between: the second call must not see the
    first call's entries left in the shared array."""
    import torch
    big = _profile(lib.NOALLOC_MAX_WINDOWS, 81)
    small = _profile(1000, 82)
    db, ds = torch.from_numpy(big).cuda(), torch.from_numpy(small).cuda()
    rb = float(np.quantile(big[np.isfinite(big)], 0.5))
    gi1, gn1, gc1 = lib.palmad_topk_profile_noalloc(db, 50, rb, 64, exclusive=True)
    gi2, gn2, gc2 = lib.palmad_topk_profile_noalloc(ds, 50, 0.0, 64, exclusive=False)
    torch.cuda.synchronize()
    for (gi, gn, gc), (prof, r, excl) in (((gi1, gn1, gc1), (big, rb, True)), ((gi2, gn2, gc2), (small, 0.0, False))):
        oi, on, cnt = _want(prof, 50, r, 64, excl)
        np.testing.assert_array_equal(gi.cpu().numpy(), oi)
        np.testing.assert_array_equal(gn.cpu().numpy(), on)
        assert int(gc.item()) == cnt


def test_noalloc_topk_matches_existing_entry_points(lib):
    """On a real nearest-neighbour profile, two calls in a row give the top-K
    and count that MERLIN's entry returns at its final r."""
    import torch
    T = synth.noisy_sine(6000, 70.0, 0.1, seed=61, anomalies=[(2100, 80), (4500, 60)])
    K = 3
    with lib.Context(0) as ctx:
        for m in (48, 63):  # two calls in a row
            want = ctx.palmad_find_discords(T, m, m, K)  # top-K at MERLIN's final r for this length
            r = float(want["r"][0])
            idx, nn = ctx.palmad_drag(T, m, 0.0)         # exact nearest-neighbour profile
            prof = np.full(len(T) - m + 1, np.inf)
            prof[idx] = nn
            got_idx, got_nn, got_cnt = lib.palmad_topk_profile_noalloc(
                torch.from_numpy(prof).cuda(), m, r, K, exclusive=True)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(got_idx.cpu().numpy(), want["idx"][0])
            np.testing.assert_allclose(got_nn.cpu().numpy(), want["nn"][0], rtol=NN_RTOL, atol=0)
            assert int(got_cnt.item()) == int(want["count"][0])


def test_noalloc_rejects_oversized_profiles(lib):
    import torch
    big = torch.zeros(lib.NOALLOC_MAX_WINDOWS + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.PalmadError) as e:
        lib.palmad_topk_profile_noalloc(big, 10, 1.0, 1)
    assert e.value.status == -8
