"""GPU parity of the Eq. 11 discord ranking (palmad_discord_interest)
against the FP64 oracle's: bit-exact on the same heatmap (the ranking is a
maximum and a sort of float32 values), and end to end from the device
heatmap of a MERLIN run against the oracle's MERLIN heatmap."""
import numpy as np
import pytest

import oracle
from paper_2304_01660_gb300 import synth

from test_gpu_parity import SERIES, _opts, ctx  # noqa: F401

pytestmark = pytest.mark.gpu


def _run(heat, minL, K, excl):
    import torch
    from paper_2304_01660_gb300 import palmad
    out = palmad.palmad_discord_interest(torch.from_numpy(heat).cuda(), minL, K, excl)
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("excl", [True, False])
@pytest.mark.parametrize("L,W,density,K", [(1, 1, 1.0, 1), (3, 1000, 0.01, 5), (17, 4099, 0.002, 40),
                                           (64, 100003, 0.0005, 64), (5, 777, 0.0, 3)])
def test_interest_matches_oracle_on_random_heatmaps(excl, L, W, density, K):
    rng = np.random.default_rng(L * 7 + W)
    heat = np.where(rng.random((L, W)) < density, rng.random((L, W)), 0.0).astype(np.float32)
    if W > 10:
        heat[:, 3] = 0.5            # ties along m
        heat[0, 7] = heat[0, 8] = 0.875  # ties across indices
    got, want = _run(heat, 30, K, excl), oracle.interest(heat, 30, K, excl)
    for k in ("score", "best_m", "idx", "m", "value"):
        np.testing.assert_array_equal(got[k], want[k], err_msg=k)


@pytest.mark.parametrize("name,minL,maxL", [("sine4000", 50, 70), ("rw3000", 10, 40)])
def test_interest_end_to_end(ctx, name, minL, maxL):
    import torch
    T = SERIES[name]()
    L, W = maxL - minL + 1, len(T) - minL + 1
    heat = torch.zeros((L, W), dtype=torch.float32, device="cuda")
    ctx.palmad_find_discords_device(torch.from_numpy(T).cuda(), minL, maxL, 2, _opts(batch_lengths=8), heatmap_dev=heat)
    h = heat.cpu().numpy()
    got = _run(h, minL, 6, True)
    same = oracle.interest(h, minL, 6, True)
    for k in ("score", "best_m", "idx", "m", "value"):
        np.testing.assert_array_equal(got[k], same[k], err_msg=k)
    want = oracle.interest(oracle.merlin(T, minL, maxL, 2, True, heatmap=True)["heatmap"], minL, 6, True)
    np.testing.assert_array_equal(got["idx"], want["idx"])
    np.testing.assert_array_equal(got["m"], want["m"])
    np.testing.assert_allclose(got["value"], want["value"], rtol=2e-5)
