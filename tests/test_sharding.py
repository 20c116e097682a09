"""Trial sharding across ranks: a run split into per-rank trial blocks and
merged for PML/TVaR gives the single-process result exactly.  Runs as two
gloo ranks on the CPU (the oracle computes each block's YLT)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1308_2066_gb300.sharding import trial_shard


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
