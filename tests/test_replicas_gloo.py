"""Multi-rank host logic of bench.py on CPU: two gloo ranks (world size 2, 127.0.0.1).

The path runs as independent replicas, one per GPU, with no exchange step; what the ranks share is the
timing rule (the job takes as long as its slowest rank) and the assignment of batched-SCF molecules to
ranks (disjoint sets of the same size distribution). Both are checked here without a GPU.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, root, out):
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch.distributed as tdist

    import bench
    tdist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        slowest = bench.max_over_ranks(1.0 + 3.5 * rank)
        members = bench.batch_members(8, rank)
        everyone = [None] * ws
        tdist.all_gather_object(everyone, members)
        out.put((rank, slowest, bench._dist(), everyone))
    finally:
        tdist.destroy_process_group()


def _run(ws):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, ROOT, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(res, key=lambda r: r[0])


def test_two_gloo_ranks_time_and_batch_assignment():
    res = _run(2)
    for rank, slowest, dist, everyone in res:
        assert slowest == pytest.approx(4.5)          # max over ranks, seen by every rank
        assert dist == (2, rank)
        seeds = [s for m in everyone for _, s in m]
        assert len(seeds) == len(set(seeds)) == 16    # disjoint molecule sets, 8 per rank
        for m in everyone:
            assert len(m) == 8 and all(1 <= w <= 8 for w, _ in m)
    assert res[0][3] == res[1][3]                      # every rank sees the same assignment


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(2.25) == 2.25
    assert bench.batch_members(4, 0) == bench.batch_members(4, 0)
    assert [s for _, s in bench.batch_members(4, 1)] == [1004, 1005, 1006, 1007]
