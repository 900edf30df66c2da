"""The N > 1 path on CPU: two gloo ranks run the replica helpers the benchmark
uses (barrier, max of elapsed times, sum of units, job rate) and fit disjoint
shards of one batch of independent surfaces with the oracle; the shards'
results equal the single-process results item by item, so no collective is
needed on the data path."""
import json
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2104_14547_gb300 import replicas, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _item_loss(s, t):
    from oracle import oracle as O
    S = O.surface_eval(s.p, s.q, s.U, s.V, s.ctrl, s.u, s.v)
    T = O.surface_eval(t.p, t.q, t.U, t.V, t.ctrl, t.u, t.v)
    loss, g = O.mse(S, T, S.size)
    dctrl, _, _ = O.surface_vjp(s.p, s.q, s.U, s.V, s.ctrl, s.u, s.v, g)
    return float(loss), float(np.abs(dctrl).sum())


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    rk = replicas.init("gloo")
    res = {"rank": rk.rank, "world": rk.world}
    replicas.barrier()
    res["max"] = replicas.max_over_ranks(rank + 0.5)
    res["sum"] = replicas.sum_over_ranks(10.0 * (rank + 1))
    res["rate"] = replicas.job_rate(100.0 * (rank + 1), float(rank + 1))
    surfs, targets = synth.bicubic_batch(5, batch=5, net=6, grid=9)
    lo, hi = replicas.shard_range(len(surfs), rank, world)
    res["items"] = list(range(lo, hi))
    res["losses"] = [_item_loss(surfs[k], targets[k]) for k in range(lo, hi)]
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
        json.dump(res, fh)
    replicas.barrier()
    replicas.finalize()


def test_two_gloo_ranks(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, x in enumerate(res):
        assert x["rank"] == r and x["world"] == world
        assert x["max"] == 1.5                      # slowest rank
        assert x["sum"] == 30.0                     # all ranks' units
        assert x["rate"] == pytest.approx(300.0 / 2.0)
    items = res[0]["items"] + res[1]["items"]
    assert items == list(range(5))                  # disjoint shards covering the batch
    surfs, targets = synth.bicubic_batch(5, batch=5, net=6, grid=9)
    whole = [_item_loss(s, t) for s, t in zip(surfs, targets)]
    sharded = res[0]["losses"] + res[1]["losses"]
    assert sharded == [list(x) for x in whole]      # bit-identical per item


def test_shard_range_properties():
    for count in (0, 1, 5, 256, 1001):
        for world in (1, 2, 3, 8):
            spans = [replicas.shard_range(count, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == count
            for (a, b), (c, d) in zip(spans, spans[1:]):
                assert b == c
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        replicas.shard_range(4, 2, 2)
    assert len({replicas.shard_seed(0, r) for r in range(8)}) == 8
    assert replicas.shard_seed(0, 0) == 0


def test_single_process_defaults(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    r = replicas.env()
    assert (r.rank, r.world, r.local) == (0, 1, 0)
    assert replicas.max_over_ranks(3.0) == 3.0
    assert replicas.job_rate(10.0, 2.0) == 5.0
