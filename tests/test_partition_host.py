"""The partition of one forest over ranks (Sec. 3), host side, without a GPU.

- fc_layout_partition splits the field (Morton) order into contiguous ranges
  of nearly equal work (a level-l leaf weighs 2^(l - lmin)).
- fc_layout_halo's mirrors suffice: the oracle's Alg. 1 (which locates every
  ghost cell geometrically, independently of the library's neighbour tables)
  run on a field that holds only a rank's leaves and mirrors -- every other
  leaf poisoned -- fills the rank's own leaves exactly as on the whole field.
  A missing mirror, or one missing behind a coarse neighbour (the
  interpolation reads the coarse leaf's copied and averaged ghosts), would
  let the poison through.
- Two gloo ranks exchange the halo over torch.distributed with host buffers,
  following the library's exchange lists: each side's lists match the
  other's, and after one exchange each rank holds its mirrors' values.
"""
import os
import socket

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
fc = pytest.importorskip("paper_1703_03116_gb300")
from paper_1703_03116_gb300.partition import (exchange_plan, halo_exchange,  # noqa: E402
                                              layout_halo, layout_partition)
from gpu_helpers import desc_for  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _layout(kind):
    if kind == "walls":
        w = synth.swirl(3, lmin=2, lmax=5, mx=8)
    elif kind == "periodic":
        w = synth.swirl(4, lmin=2, lmax=5, mx=8)
        w.domain = "periodic"
    else:
        w = synth.sphere(seed=2, lmin=1, lmax=3, mx=8)
    ref = oracle.initial_forest(w)
    return w, ref


@pytest.mark.parametrize("kind", ["walls", "periodic", "sphere"])
@pytest.mark.parametrize("nranks", [2, 3, 5])
def test_partition_is_contiguous_and_balanced(kind, nranks):
    w, ref = _layout(kind)
    lv = ref.leaves()  # field order
    desc = desc_for(fc, w, fc.F64)
    part = layout_partition(desc, lv, nranks)
    assert part[0] == 0 and part[-1] == nranks - 1
    assert np.all(np.diff(part) >= 0)  # contiguous ranges of the field order
    wgt = 2.0 ** (lv[:, 2] - w.lmin)
    work = np.array([wgt[part == r].sum() for r in range(nranks)])
    assert np.all(work > 0)
    assert work.max() - work.min() <= 2 * wgt.max()


def _poisoned_fill(w, lv, q, keep, poison):
    F = oracle.Forest(oracle.params_for(w), lv)
    qq = np.array(q)
    qq[~keep] = poison
    F.set_q(qq)
    F.fill_ghosts()
    return F.get_q_full()


@pytest.mark.parametrize("kind", ["walls", "periodic", "sphere"])
@pytest.mark.parametrize("nranks", [2, 3, 4])
def test_mirrors_hold_everything_the_owned_ghost_fill_reads(kind, nranks):
    w, ref = _layout(kind)
    lv = ref.leaves()
    desc = desc_for(fc, w, fc.F64)
    part = layout_partition(desc, lv, nranks)
    q = synth.random_field((len(lv), w.mx, w.mx), seed=7) + 0.5
    full = _poisoned_fill(w, lv, q, np.ones(len(lv), bool), 0.0)
    for r in range(nranks):
        mirrors = layout_halo(desc, lv, part, r)
        assert not np.any(part[mirrors] == r)
        keep = part == r
        keep[mirrors] = True
        own = part == r
        for poison in (np.nan, 1e30):
            got = _poisoned_fill(w, lv, q, keep, poison)
            np.testing.assert_array_equal(got[own], full[own])
        # and they are needed: dropping a mirror that is a same-size face
        # neighbour of an owned leaf lets the poison into that leaf's ghosts
        nb = fc.layout_neighbours(desc, lv)
        face = [int(nb[k, d, 1]) for k in np.flatnonzero(own) for d in range(4)
                if nb[k, d, 0] == 1 and not own[nb[k, d, 1]]]
        assert face, "a partition of a connected layout has a face across ranks"
        keep2 = keep.copy()
        keep2[face[0]] = False
        got = _poisoned_fill(w, lv, q, keep2, np.nan)
        assert np.isnan(got[own]).any()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as orc
        import paper_1703_03116_gb300 as fcl
        import synth as syn
        from gpu_helpers import desc_for as dfor
        from paper_1703_03116_gb300.partition import (exchange_plan as plan_of,
                                                      halo_exchange as exch, layout_partition as lp)
        w = syn.swirl(3, lmin=2, lmax=5, mx=8)
        ref = orc.initial_forest(w)
        lv = ref.leaves()
        desc = dfor(fcl, w, fcl.F64)
        part = lp(desc, lv, world)
        plan = plan_of(desc, lv, part, rank)
        # the lists agree pairwise: what this rank sends a peer is what that
        # peer receives from it (gathered from every rank)
        mine = {p: (s.tolist(), r.tolist()) for p, (s, r) in plan.items()}
        every = [None] * world
        dist.all_gather_object(every, mine)
        agree = all(every[a][b][0] == every[b][a][1] for a in range(world) for b in range(world)
                    if a != b)
        # a global field, held by each rank at its own leaves only
        q = syn.random_field((len(lv), 8, 8), seed=11) + 0.5
        local = np.full_like(q, np.nan)
        local[part == rank] = q[part == rank]
        flat = torch.from_numpy(local.reshape(len(lv), -1))
        exch(dist, plan, lambda p: (len(plan[p][0]), len(plan[p][1])),
             lambda p: flat[torch.from_numpy(plan[p][0])].contiguous().view(-1),
             lambda p, buf: flat.index_copy_(0, torch.from_numpy(plan[p][1]),
                                             buf.view(len(plan[p][1]), -1)),
             lambda p, n: torch.empty(n * 64, dtype=torch.float64))
        mirrors = set(int(k) for k in range(len(lv)) if part[k] != rank and
                      not np.isnan(local[k]).all())
        want = set(int(k) for _, (_, r) in plan.items() for k in r)
        held = part == rank
        for k in want:
            held[k] = True
        ok_values = bool(np.array_equal(local[held], q[held]))
        out[rank] = (agree, mirrors == want, ok_values, len(want))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_exchange_the_halo_with_host_buffers():
    import torch.multiprocessing as mp
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn", join=True)
    for r in range(world):
        agree, mirrors_ok, values_ok, n = out[r]
        assert agree and mirrors_ok and values_ok and n > 0, (r, out[r])
