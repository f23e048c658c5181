"""Partitioned forests (Sec. 3: partitioning and parallel ghost filling).

The leaves, in field (Morton) order, are split into contiguous ranges of
equal work; each rank's part (``fc_forest_create_part``) holds its leaves and
its mirrors.  After every update the owners send the new interiors of the
patches other ranks mirror (``fc_halo_pack`` / ``fc_halo_unpack``), in the
order of the multirate recursion (Sec. 4), so every part's next ghost fill
reads what the unpartitioned forest would.  This module only sequences the
library's calls and moves the packed buffers: within one process between
partitions on one GPU (a device copy into the receiver's buffer), or between
processes with ``torch.distributed`` point-to-point messages.  All
arithmetic runs in the library's kernels.
"""
from __future__ import annotations

import ctypes
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import _lib
from ._lib import Desc, check, load
from .forest import Forest, _iarr, _ip, _stream


def layout_partition(desc: Desc, leaves, nranks: int) -> np.ndarray:
    """Rank of each leaf (the caller's order): contiguous ranges of the field
    order with equal work, a level-l leaf weighing 2^(l - lmin)."""
    leaves = _iarr(leaves).reshape(-1, 5)
    out = np.zeros(len(leaves), dtype=np.int32)
    check(load().fc_layout_partition(ctypes.byref(desc), len(leaves), _ip(leaves), int(nranks),
                                     _ip(out)))
    return out


def layout_halo(desc: Desc, leaves, part, rank: int) -> np.ndarray:
    """Indices (into ``leaves``, field order) of rank's mirrors under part."""
    leaves = _iarr(leaves).reshape(-1, 5)
    part = _iarr(part)
    out = np.zeros(len(leaves), dtype=np.int32)
    n = ctypes.c_int()
    check(load().fc_layout_halo(ctypes.byref(desc), len(leaves), _ip(leaves), _ip(part),
                                int(rank), ctypes.byref(n), _ip(out)))
    return out[:n.value]


def exchange_plan(desc: Desc, leaves, part, rank: int) -> Dict[int, Tuple[np.ndarray, np.ndarray]]:
    """What rank exchanges with each other rank, as indices into ``leaves``:
    {peer: (sent, received)}, sent = rank's leaves that peer mirrors,
    received = rank's mirrors that peer owns, both ordered by (level, field
    order) -- the order of the packed buffers of fc_halo_pack(peer, -1)."""
    leaves = _iarr(leaves).reshape(-1, 5)
    part = _iarr(part)
    nranks = int(part.max()) + 1
    mirrors = {r: layout_halo(desc, leaves, part, r) for r in range(nranks)}
    plan = {}
    for peer in range(nranks):
        if peer == rank:
            continue
        sent = [k for k in mirrors[peer] if part[k] == rank]
        recv = [k for k in mirrors[rank] if part[k] == peer]
        # level-major, field order within a level (mirror lists are in field order)
        sent.sort(key=lambda k: leaves[k, 2])
        recv.sort(key=lambda k: leaves[k, 2])
        plan[peer] = (np.asarray(sent, dtype=np.int64), np.asarray(recv, dtype=np.int64))
    return plan


class Part(Forest):
    """One rank's part of a partitioned layout (fc_forest_create_part)."""

    def __init__(self, desc: Desc, leaves, part, rank: int):
        L = load()
        self.desc = desc
        leaves = _iarr(leaves).reshape(-1, 5)
        self.part = _iarr(part)
        self.rank = int(rank)
        self.nranks = int(self.part.max()) + 1
        h = ctypes.c_void_p()
        check(L.fc_forest_create_part(ctypes.byref(desc), len(leaves), _ip(leaves),
                                      _ip(self.part), self.rank, ctypes.byref(h)))
        self._h = h

    def halo_count(self, peer: int, level: int = -1) -> Tuple[int, int]:
        ns, nr = ctypes.c_int(), ctypes.c_int()
        check(load().fc_halo_count(self._h, int(peer), int(level), ctypes.byref(ns),
                                   ctypes.byref(nr)))
        return ns.value, nr.value

    def halo_pack(self, peer: int, level: int, dst, stream=None):
        assert dst.is_cuda and dst.is_contiguous()
        check(load().fc_halo_pack(self._h, int(peer), int(level),
                                  ctypes.c_void_p(dst.data_ptr()), _stream(stream)))

    def halo_unpack(self, peer: int, level: int, src, stream=None):
        assert src.is_cuda and src.is_contiguous()
        check(load().fc_halo_unpack(self._h, int(peer), int(level),
                                    ctypes.c_void_p(src.data_ptr()), _stream(stream)))


def _substeps(lmin: int, lmax: int, t0: float, dtc: float) -> List[Tuple[int, float, float]]:
    """The coarse-first recursion of a coarse multirate step (Sec. 4)."""
    out = []

    def rec(L, t, dt):
        out.append((L, t, dt))
        if L < lmax:
            rec(L + 1, t, 0.5 * dt)
            rec(L + 1, t + 0.5 * dt, 0.5 * dt)

    rec(lmin, t0, dtc)
    return out


class _Driver:
    """Stepping schedule shared by the in-process and the distributed runs:
    each update on every local part, then the exchange of what it changed."""

    parts: List[Part]

    def exchange(self, level: int):
        raise NotImplementedError

    def step_global(self, t: float, dt: float):
        for p in self.parts:
            p.step_global(t, dt)
        self.exchange(-1)

    def advance_level(self, level: int, t: float, dt: float):
        for p in self.parts:
            p.advance_level(level, t, dt)
        self.exchange(level)

    def step_multirate(self, t: float, dt_coarse: float):
        d = self.parts[0].desc
        for (L, tl, dtl) in _substeps(d.lmin, d.lmax, t, dt_coarse):
            self.advance_level(L, tl, dtl)


class VirtualPartitions(_Driver):
    """k partitions of one layout on one GPU, each with its own patch store;
    the exchange packs on the owner into a buffer that the receiver unpacks
    (what a peer copy into the receiving GPU's memory does across GPUs)."""

    def __init__(self, desc: Desc, leaves, nparts: int, part=None):
        import torch
        self.torch = torch
        self.leaves = _iarr(leaves).reshape(-1, 5)
        self.part = layout_partition(desc, self.leaves, nparts) if part is None else _iarr(part)
        self.parts = [Part(desc, self.leaves, self.part, r) for r in range(nparts)]
        self.owned = [np.flatnonzero(self.part == r) for r in range(nparts)]
        self.mx = desc.mx
        self.tdt = torch.float32 if desc.dtype == _lib.F32 else torch.float64

    def exchange(self, level: int):
        torch = self.torch
        for a, pa in enumerate(self.parts):
            for b, pb in enumerate(self.parts):
                if a == b:
                    continue
                ns, _ = pa.halo_count(b, level)
                if ns == 0:
                    continue
                buf = torch.empty(ns * self.mx * self.mx, dtype=self.tdt, device="cuda")
                pa.halo_pack(b, level, buf)
                pb.halo_unpack(a, level, buf)

    def set_q(self, q):
        """q: the whole layout's field (leaves in the order given)."""
        for r, p in enumerate(self.parts):
            p.set_q(np.ascontiguousarray(np.asarray(q)[self.owned[r]]))
        self.exchange(-1)

    def get_q(self) -> np.ndarray:
        out = np.empty((len(self.leaves), self.mx, self.mx))
        for r, p in enumerate(self.parts):
            out[self.owned[r]] = p.get_q()
        return out

    def mass(self) -> np.ndarray:
        return sum(p.mass() for p in self.parts)

    def close(self):
        for p in self.parts:
            p.close()


def halo_exchange(dist, plan: Dict[int, Tuple[np.ndarray, np.ndarray]], level_counts: Callable,
                  pack: Callable, unpack: Callable, make: Callable):
    """One exchange with every peer over torch.distributed point-to-point
    messages: for each peer, pack(peer) -> a buffer sent to it; a buffer of
    make(peer) elements received from it -> unpack(peer, buf).  All sends and
    receives are posted before any is waited on (no ordering deadlock)."""
    reqs, inbox = [], {}
    for peer in sorted(plan):
        ns, nr = level_counts(peer)
        if ns:
            reqs.append(dist.isend(pack(peer), dst=peer))
        if nr:
            buf = make(peer, nr)
            inbox[peer] = buf
            reqs.append(dist.irecv(buf, src=peer))
    for r in reqs:
        r.wait()
    for peer, buf in inbox.items():
        unpack(peer, buf)


class DistributedPart(_Driver):
    """This process's part of a layout partitioned over the ranks of a
    torch.distributed group (one GPU each); exchanges by point-to-point
    messages into the receiving GPU's own memory."""

    def __init__(self, desc: Desc, leaves, dist, part=None):
        import torch
        self.torch, self.dist = torch, dist
        self.leaves = _iarr(leaves).reshape(-1, 5)
        n = dist.get_world_size()
        self.rank = dist.get_rank()
        self.part = layout_partition(desc, self.leaves, n) if part is None else _iarr(part)
        self.parts = [Part(desc, self.leaves, self.part, self.rank)]
        self.plan = exchange_plan(desc, self.leaves, self.part, self.rank)
        self.owned = np.flatnonzero(self.part == self.rank)
        self.mx = desc.mx
        self.tdt = torch.float32 if desc.dtype == _lib.F32 else torch.float64

    def exchange(self, level: int):
        torch, P, cells = self.torch, self.parts[0], self.mx * self.mx

        def pack(peer):
            ns, _ = P.halo_count(peer, level)
            buf = torch.empty(ns * cells, dtype=self.tdt, device="cuda")
            P.halo_pack(peer, level, buf)
            torch.cuda.current_stream().synchronize()  # the message reads it
            return buf

        halo_exchange(self.dist, self.plan, lambda peer: P.halo_count(peer, level), pack,
                      lambda peer, buf: P.halo_unpack(peer, level, buf),
                      lambda peer, nr: torch.empty(nr * cells, dtype=self.tdt, device="cuda"))

    def set_q(self, q):
        self.parts[0].set_q(np.ascontiguousarray(np.asarray(q)[self.owned]))
        self.exchange(-1)

    def mass(self) -> np.ndarray:
        torch = self.torch
        m = torch.tensor(self.parts[0].mass(), dtype=torch.float64, device="cuda")
        self.dist.all_reduce(m)
        return m.cpu().numpy()
