"""Trial sharding across ranks: a run split into per-rank trial blocks and
merged for PML/TVaR gives the single-process result exactly.  Runs as two
gloo ranks on the CPU (the oracle computes each block's YLT)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1308_2066_gb300.sharding import layer_shard, trial_shard


def test_shards_cover_every_trial_once():
    for n in (0, 1, 7, 10, 1000, 1_000_003):
        for world in (1, 2, 3, 8):
            blocks = [trial_shard(n, world, r) for r in range(world)]
            assert blocks[0][0] == 0
            for (b0, c0), (b1, _) in zip(blocks, blocks[1:]):
                assert b0 + c0 == b1
            assert sum(c for _, c in blocks) == n
            assert max(c for _, c in blocks) - min(c for _, c in blocks) <= 1
    with pytest.raises(ValueError):
        trial_shard(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n_trials, q):
    import torch
    import torch.distributed as dist
    import oracle
    import workloads as W
    from paper_1308_2066_gb300.sharding import gather_ylt, trial_shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = W.plain_tiny(n_trials=n_trials, timestamps=False)
    wl.layers[0].agg_l = float("inf")
    b, c = trial_shard(n_trials, world, rank)
    local = oracle.simulate_layer(wl, trials=np.arange(b, b + c), threads=1).ylt
    full = gather_ylt(torch.from_numpy(local)).numpy()
    pml, tv = oracle.risk_measures(full, [100.0, 250.0, 10.0], [0.99, 0.9])
    q.put((rank, full, pml, tv))
    dist.destroy_process_group()


@pytest.mark.parametrize("n_trials", [3000, 3001])
def test_two_rank_run_equals_single_run(orc, n_trials):
    import workloads as W
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, n_trials, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    wl = W.plain_tiny(n_trials=n_trials, timestamps=False)
    wl.layers[0].agg_l = float("inf")
    whole = orc.simulate_layer(wl).ylt
    pml, tv = orc.risk_measures(whole, [100.0, 250.0, 10.0], [0.99, 0.9])
    for _, full, p, t in got:
        np.testing.assert_array_equal(full, whole)
        np.testing.assert_array_equal(p, pml)
        np.testing.assert_array_equal(t, tv)


def test_layer_shards_partition_and_balance():
    g = np.random.default_rng(3)
    for n in (0, 1, 5, 64):
        work = list(g.integers(1, 1000, size=n))
        for world in (1, 2, 3, 8):
            parts = [layer_shard(work, world, r) for r in range(world)]
            flat = sorted(i for p in parts for i in p)
            assert flat == list(range(n))
            if n >= world:
                loads = [sum(work[i] for i in p) for p in parts]
                # greedy in decreasing order: no rank exceeds the mean by more than the largest layer
                assert max(loads) <= sum(work) / world + max(work)
    with pytest.raises(ValueError):
        layer_shard([1, 2], 2, 5)


def _layer_rank_main(rank, world, port, q):
    import torch.distributed as dist
    import oracle
    import workloads as W
    from paper_1308_2066_gb300.sharding import gather_results, layer_shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = W.portfolio(n_trials=400, n_layers=6, pool=24, max_j=8, nnz_range=(200, 800),
                     catalog=5000, mean_events=30)
    work = [len(L.elts) for L in wl.layers]
    local = {}
    for i in layer_shard(work, world, rank):
        r = oracle.simulate_layer(wl, i, threads=1)
        pml, tv = oracle.risk_measures(r.ylt, [100.0, 10.0], [0.95])
        local[i] = (list(pml), list(tv))
    q.put((rank, gather_results(local, len(wl.layers))))
    dist.destroy_process_group()


def test_two_rank_layer_split_equals_single_run(orc):
    import workloads as W
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_layer_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    wl = W.portfolio(n_trials=400, n_layers=6, pool=24, max_j=8, nnz_range=(200, 800),
                     catalog=5000, mean_events=30)
    for _, res in got:
        for i in range(len(wl.layers)):
            r = orc.simulate_layer(wl, i)
            pml, tv = orc.risk_measures(r.ylt, [100.0, 10.0], [0.95])
            assert res[i] == (list(pml), list(tv))
