"""The benchmark's multi-process path on CPU: two gloo ranks initialise the
process group the way torchrun does, agree on the slowest rank's time
(max over ranks), the total work (sum) and a check every rank passed (min),
the ensemble's channels split over the ranks cover every channel once with
balanced work, and the reference arm prints exactly one JSON line from rank 0
while rank 1 exits without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist, r, ws, local = bench.dist_init()
    got = bench.max_over_ranks(10.0 + 3.0 * r, dist)
    tot = bench.sum_over_ranks(10.0 + 3.0 * r, dist)
    low = bench.min_over_ranks(10.0 + 3.0 * r, dist)
    dist.barrier()
    q.put((r, ws, (got, tot, low)))
    dist.destroy_process_group()


def test_max_over_ranks_with_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get() for _ in range(2))
    assert [r for r, _, _ in res] == [0, 1]
    assert all(ws == 2 and got == (13.0, 23.0, 10.0) for _, ws, got in res)


def test_reference_arm_under_torchrun_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "2", "--warmup", "1", "--cells", "20000"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_ensemble_shards_cover_every_channel_once(world):
    sys.path.insert(0, ROOT)
    import numpy as np
    from paper_1912_04791_gb300 import workloads as W
    E = W.riemann_ensemble(512, seed=21)
    shards = [W.shard_ensemble(E, r, world) for r in range(world)]
    # every channel in exactly one shard, with its own cells
    assert sum(len(S.n_cells) for S in shards) == len(E.n_cells)
    assert sum(int(S.n_cells.sum()) for S in shards) == int(E.n_cells.sum())
    key = lambda S: sorted(zip(S.n_cells.tolist(), S.Ag.tolist()))
    assert sorted(sum((key(S) for S in shards), [])) == key(E)
    for S in shards:
        o = S.offsets
        for c in range(len(S.n_cells)):
            src = int(np.flatnonzero((E.n_cells == S.n_cells[c]) & (E.Ag == S.Ag[c]))[0])
            for a, b in zip(S.channel(c), E.channel(src)):
                assert np.array_equal(a, b)
    # list scheduling: no rank holds more than the mean plus the largest channel's work
    work = lambda S: float((S.n_cells.astype(float) ** 2 / S.length).sum())
    loads = [work(S) for S in shards]
    biggest = float((E.n_cells.astype(float) ** 2 / E.length).max())
    assert max(loads) <= sum(loads) / world + biggest
    with pytest.raises(ValueError):
        W.shard_ensemble(E, world, world)
