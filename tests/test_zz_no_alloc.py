"""The no-allocation top-K entry point against the existing entry points.

palmad_topk_profile_noalloc serves callers that cannot call cudaMalloc (for
example while another allocator owns all device memory, or on a path that
cannot take cudaMalloc's implicit device synchronisation): it uses a fixed
device array of the library instead of allocated scratch.  This file is
named to run last, so a failure here cannot hide any other test's result.
It builds the library itself, so it also runs alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2304_01660_gb300 import synth

pytestmark = pytest.mark.gpu

NN_RTOL = 1e-5


def test_noalloc_topk_matches_existing_entry_points():
    import torch

    from paper_2304_01660_gb300 import _build, palmad
    _build.build()
    T = synth.noisy_sine(6000, 70.0, 0.1, seed=61, anomalies=[(2100, 80), (4500, 60)])
    K = 3
    with palmad.Context(0) as ctx:
        for m in (48, 63):  # two calls in a row
            want = ctx.palmad_find_discords(T, m, m, K)  # top-K at MERLIN's final r for this length
            r = float(want["r"][0])
            idx, nn = ctx.palmad_drag(T, m, 0.0)         # exact nearest-neighbour profile
            prof = np.full(len(T) - m + 1, np.inf)
            prof[idx] = nn
            got_idx, got_nn, got_cnt = palmad.palmad_topk_profile_noalloc(
                torch.from_numpy(prof).cuda(), m, r, K, exclusive=True)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(got_idx.cpu().numpy(), want["idx"][0])
            np.testing.assert_allclose(got_nn.cpu().numpy(), want["nn"][0], rtol=NN_RTOL, atol=0)
            assert int(got_cnt.item()) == int(want["count"][0])


def test_noalloc_rejects_oversized_profiles():
    import torch

    from paper_2304_01660_gb300 import _build, palmad
    _build.build()
    big = torch.zeros(palmad.NOALLOC_MAX_WINDOWS + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(palmad.PalmadError) as e:
        palmad.palmad_topk_profile_noalloc(big, 10, 1.0, 1)
    assert e.value.status == -8
