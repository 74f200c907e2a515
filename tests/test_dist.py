"""Multi-rank host logic on CPU ranks (gloo, world size 2).

The exchange steps of a sharded DRAG (bitmap AND after select, nnDist min
after refine) are checked against the unsharded result: each rank computes
the nearest-neighbour distances over its own column slice with the FP64
oracle's distance, and after the MIN exchange every rank holds the full
brute-force profile; a bitmap of windows pruned at r by either rank, ANDed,
equals the unsharded pruning.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2304_01660_gb300 import dist as pdist
from paper_2304_01660_gb300 import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        T = synth.random_walk(300, 71)
        m, r = 12, 2.5
        N = len(T) - m + 1
        mu, sd = oracle.stats(T, m)
        Z = np.stack([(T[i:i + m].astype(np.float64) - mu[i]) / sd[i] for i in range(N)])
        lo, hi = pdist.column_slice(N, rank, world)
        # partial nearest neighbours over this rank's columns
        nn = np.full(N, np.inf)
        for i in range(N):
            for j in range(lo, hi):
                if abs(i - j) >= m:
                    nn[i] = min(nn[i], np.linalg.norm(Z[i] - Z[j]))
        nn_t = torch.from_numpy(nn.copy())
        pdist.nn_min_(nn_t)
        # candidate bitmap: a window stays a candidate unless this rank saw a pair with d < r
        alive = nn >= r
        words = np.zeros((N + 31) // 32, dtype=np.int64)
        for i in range(N):
            if alive[i]:
                words[i // 32] |= 1 << (i % 32)
        bits = torch.from_numpy(words.astype(np.int32))
        pdist.candidate_and_(bits)
        tmax = pdist.max_over_ranks(float(rank + 1))
        owned = pdist.shard_balanced([5, 1, 3, 3, 2, 8, 1], rank, world)
        allowned = pdist.gather_objects(owned, world)
        q.put((rank, nn_t.numpy(), bits.numpy(), tmax, allowned))
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def results():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out, key=lambda x: x[0])


def test_nn_min_exchange_gives_full_profile(results):
    import oracle
    T = synth.random_walk(300, 71)
    mp_full, _ = oracle.matrix_profile(T, 12)
    for _, nn, _, _, _ in results:
        np.testing.assert_allclose(nn, mp_full, rtol=1e-12)


def test_bitmap_and_equals_unsharded_pruning(results):
    import oracle
    T = synth.random_walk(300, 71)
    mp_full, _ = oracle.matrix_profile(T, 12)
    alive = mp_full >= 2.5
    for _, _, bits, _, _ in results:
        got = np.array([(int(bits[i // 32]) >> (i % 32)) & 1 for i in range(len(alive))], dtype=bool)
        np.testing.assert_array_equal(got, alive)


def test_max_over_ranks_and_sharding(results):
    for _, _, _, tmax, allowned in results:
        assert tmax == 2.0
        flat = sorted(i for part in allowned for i in part)
        assert flat == list(range(7))
        loads = [sum([5, 1, 3, 3, 2, 8, 1][i] for i in part) for part in allowned]
        assert max(loads) - min(loads) <= 1


def test_shard_balanced_single_rank():
    assert pdist.shard_balanced([3, 1, 2], 0, 1) == [0, 1, 2]
    assert pdist.column_slice(10, 1, 3) == (4, 8)


class _OracleShards:
    """Stand-in for a library context on CPU ranks: the two shard entry
    points computed from the FP64 oracle's distances (select over the rank's
    rows prunes windows i and j of every pair i < j <= ..., j >= i + m with
    d < r; refine gives -1 or the minimum over the rank's columns)."""

    def __init__(self):
        import oracle
        self.oracle = oracle

    def _z(self, T, m):
        mu, sd = self.oracle.stats(T, m)
        N = len(T) - m + 1
        return np.stack([(T[i:i + m].astype(np.float64) - mu[i]) / sd[i] for i in range(N)])

    def palmad_drag_select_shard(self, T, m, r, lo, hi, options=None):
        Z = self._z(T, m)
        N = len(Z)
        alive = np.ones(N, dtype=bool)
        for i in range(lo, hi):
            for j in range(i + m, N):
                if np.linalg.norm(Z[i] - Z[j]) < r:
                    alive[i] = alive[j] = False
        words = np.zeros((N + 31) // 32, dtype=np.uint64)
        for i in np.nonzero(alive)[0]:
            words[i // 32] |= np.uint64(1) << np.uint64(i % 32)
        return words.astype(np.uint32)

    def palmad_drag_refine_shard(self, T, m, r, bits, lo, hi, options=None):
        Z = self._z(T, m)
        N = len(Z)
        out = np.full(N, np.inf)
        for i in range(N):
            if not (int(bits[i // 32]) >> (i % 32)) & 1:
                continue
            best = np.inf
            for j in range(lo, hi):
                if abs(i - j) >= m:
                    d = np.linalg.norm(Z[i] - Z[j])
                    if d < r:
                        best = -1.0
                        break
                    best = min(best, d)
            out[i] = best
        return out


def _sharded_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        T = synth.random_walk(260, 72)
        idx, nn = pdist.sharded_drag(_OracleShards(), T, 10, 2.2, rank, world)
        q.put((rank, idx, nn))
    finally:
        dist.destroy_process_group()


def test_sharded_drag_exchange_on_cpu_ranks():
    """sharded_drag's two exchanges (bitmap AND, distance MIN) give every
    rank the unsharded range discords (two gloo ranks)."""
    import oracle
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    T = synth.random_walk(260, 72)
    wi, wn = oracle.range_discords(T, 10, 2.2)
    assert len(wi) > 0
    for _, gi, gn in out:
        np.testing.assert_array_equal(gi, wi)
        np.testing.assert_allclose(gn, wn, rtol=1e-9)

