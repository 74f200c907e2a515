"""One DRAG call split over ranks (the cluster DRAG of the paper's related
work, Sec. 1) against the FP64 oracle.

Each rank runs candidate select over its rows (palmad_drag_select_shard),
the ranks AND their candidate bitmaps, each refines the common candidates
against its columns (palmad_drag_refine_shard), and the ranks take the
elementwise minimum.  The range discords of the combined result must equal
the oracle's exactly (indices) and within 1e-5 in distance, for 2 and 3
shards emulated in one process, and for two gloo ranks that both use GPU 0
(ordinary host arrays exchanged, no peer memory).  A single shard must give
exactly what palmad_drag gives.
"""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2304_01660_gb300 import synth

pytestmark = pytest.mark.gpu

NN_RTOL = 1e-5


def _flat_series(n, seed):
    x = synth.random_walk(n, seed).astype(np.float64)
    x[300:420] = 5.0
    return x.astype(np.float32)


SERIES = {
    "rw3000": lambda: synth.random_walk(3000, 41),
    "sine4000": lambda: synth.noisy_sine(4000, 60.0, 0.1, seed=44, anomalies=[(1700, 70), (3100, 50)]),
    "flat2200": lambda: _flat_series(2200, 45),
}


def _thresholds(mp, qs):
    v = np.unique(mp[np.isfinite(mp)])
    return [0.5 * (v[min(int(q * (len(v) - 1)), len(v) - 2)] + v[min(int(q * (len(v) - 1)), len(v) - 2) + 1])
            for q in qs]


@pytest.fixture(scope="module")
def ctx():
    from paper_2304_01660_gb300 import _build, palmad
    _build.build()
    c = palmad.Context(0)
    yield c
    c.close()


def _emulated(ctx, T, m, r, world):
    from paper_2304_01660_gb300 import dist as pdist
    N = len(T) - m + 1
    slices = [pdist.column_slice(N, k, world) for k in range(world)]
    bits = None
    for lo, hi in slices:
        b = ctx.palmad_drag_select_shard(T, m, r, lo, hi)
        bits = b if bits is None else (bits & b)
    nn = None
    for lo, hi in slices:
        part = ctx.palmad_drag_refine_shard(T, m, r, bits, lo, hi)
        nn = part if nn is None else np.minimum(nn, part)
    keep = np.isfinite(nn) & (nn >= 0.0) & ((r <= 0.0) | (nn >= r))
    idx = np.nonzero(keep)[0]
    return idx, nn[idx]


@pytest.mark.parametrize("name", list(SERIES))
@pytest.mark.parametrize("m", [16, 60])
@pytest.mark.parametrize("world", [1, 2, 3])
def test_sharded_drag_equals_oracle(ctx, name, m, world):
    T = SERIES[name]()
    mp, _ = oracle.matrix_profile(T, m)
    for r in _thresholds(mp, (0.5, 0.95, 1.0)) + [0.0]:
        gi, gn = _emulated(ctx, T, m, r, world)
        wi, wn = oracle.range_discords(T, m, r)
        np.testing.assert_array_equal(gi, wi)
        np.testing.assert_allclose(gn, wn, rtol=NN_RTOL, atol=0)
        if world == 1:
            di, dn = ctx.palmad_drag(T, m, r)
            np.testing.assert_array_equal(gi, di)
            np.testing.assert_array_equal(gn, dn)


def test_shard_arguments_are_checked(ctx):
    from paper_2304_01660_gb300 import palmad
    T = SERIES["rw3000"]()
    N = len(T) - 20 + 1
    for lo, hi in ((-1, 10), (10, 5), (0, N + 1)):
        with pytest.raises(palmad.PalmadError) as e:
            ctx.palmad_drag_select_shard(T, 20, 3.0, lo, hi)
        assert e.value.status == -1
    bits = ctx.palmad_drag_select_shard(T, 20, 3.0, 0, N)
    with pytest.raises(palmad.PalmadError) as e:
        ctx.palmad_drag_refine_shard(T, 20, 3.0, bits, 5, 2)
    assert e.value.status == -1
    with pytest.raises(palmad.PalmadError) as e:
        ctx.palmad_drag_select_shard(T, 20, 3.0, 0, N, palmad.palmad_default_options(knn_k=2))
    assert e.value.status == -6


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, T, m, r, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2304_01660_gb300 import dist as pdist
        from paper_2304_01660_gb300 import palmad
        with palmad.Context(0) as c:
            idx, nn = pdist.sharded_drag(c, T, m, r, rank, world)
        q.put((rank, idx.tolist(), nn.tolist()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_on_one_gpu(ctx):
    import torch.multiprocessing as mp
    T = SERIES["sine4000"]()
    m = 48
    mp_, _ = oracle.matrix_profile(T, m)
    r = _thresholds(mp_, (0.97,))[0]
    spawn = mp.get_context("spawn")
    q = spawn.Queue()
    port = _free_port()
    procs = [spawn.Process(target=_rank, args=(k, 2, port, T, m, r, q)) for k in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    wi, wn = oracle.range_discords(T, m, r)
    for _, gi, gn in got:
        np.testing.assert_array_equal(np.array(gi, dtype=np.int64), wi)
        np.testing.assert_allclose(gn, wn, rtol=NN_RTOL, atol=0)
