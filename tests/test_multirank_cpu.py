"""The multi-GPU path without GPUs: two gloo ranks on the CPU.

The path shards by forest: each rank advances its own forest and the only
collective combines per-rank scalars (max of times, sum of work).  Here two
ranks build their rank's layout with the library's host services and the
oracle, combine through bench.aggregate over gloo, and check the result
against what each rank reports.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        import paper_1703_03116_gb300 as fc
        w = bench.rank_workload(rank)
        w.lmax, w.mx = 4, 8  # small layout, same recipe
        F = oracle.initial_forest(w)
        leaves = F.leaves()
        desc = fc.make_desc(domain=fc.WALLS, mx=w.mx, lmin=w.lmin, lmax=w.lmax,
                            velocity=w.velocity)
        fc.layout_check(desc, leaves)
        updates = bench.cell_updates(leaves, w.lmin, w.mx)
        fake_ms = 10.0 + rank  # per-rank time
        agg = bench.aggregate([fake_ms, updates], ["max", "sum"], dist, "cpu")
        out[rank] = (updates, agg[0], agg[1], float(w.parts[0].centre[0]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_by_forest():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn", join=True)
    per = [out[r] for r in range(world)]
    total = sum(p[0] for p in per)
    for updates, ms_max, upd_sum, _ in per:
        assert ms_max == 10.0 + (world - 1)  # max over ranks
        assert upd_sum == total               # whole-job work
    # the ranks advance different forests (seeded by rank)
    assert per[0][3] != per[1][3]
