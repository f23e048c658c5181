"""Python view of one fc_forest handle (marshalling only; all work is in libfc.so)."""
from __future__ import annotations

import ctypes
from typing import Callable, Optional, Sequence

import numpy as np

from . import _lib
from ._lib import Desc, check, load

_NP = {_lib.F32: np.float32, _lib.F64: np.float64}


def make_desc(domain: int = _lib.WALLS, mx: int = 32, lmin: int = 2, lmax: int = 6,
              dtype: int = _lib.F64, velocity=("swirl", 4.0), order: int = 2,
              limiter: int = 1, transverse: int = 2, nforests: int = 1, mbc: int = 2,
              indicator: int = 0, smooth: int = 0, reflux: int = 0, brick=(1, 1)) -> Desc:
    """brick: (blocks per row, blocks per column) of the FC_DOMAIN_BRICK domain."""
    d = Desc()
    d.domain, d.nforests, d.mx, d.mbc, d.lmin, d.lmax, d.dtype = (
        domain, nforests, mx, mbc, lmin, lmax, dtype)
    d.brick_nx, d.brick_ny = int(brick[0]), int(brick[1])
    if velocity[0] == "const":
        d.vel_kind = _lib.VEL_CONST
        d.vel[0], d.vel[1] = float(velocity[1]), float(velocity[2])
    elif velocity[0] == "swirl":
        d.vel_kind = _lib.VEL_SWIRL
        d.vel[0] = float(velocity[1])
    elif velocity[0] == "rotation":
        d.vel_kind = _lib.VEL_ROTATION
        for k in range(3):
            d.vel[k] = float(velocity[1 + k])
    elif velocity[0] == "deform":  # Sec. 5.3: (k, T, T_f)
        d.vel_kind = _lib.VEL_DEFORM
        for k in range(3):
            d.vel[k] = float(velocity[1 + k])
    else:
        raise ValueError(f"unknown velocity {velocity!r}")
    d.order, d.limiter, d.transverse = order, limiter, transverse
    d.indicator, d.smooth, d.reflux = indicator, smooth, reflux
    return d


def _iarr(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _stream(s) -> Optional[int]:
    if s is None:
        return None
    return int(getattr(s, "cuda_stream", s)) or None


def uniform_leaves(level: int, nforests: int = 1, nblocks: int = 1) -> np.ndarray:
    n = 1 << level
    ys, xs = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    one = np.stack([np.zeros(n * n, int), np.zeros(n * n, int), np.full(n * n, level),
                    xs.ravel(), ys.ravel()], axis=1)
    out = []
    for f in range(nforests):
        for b in range(nblocks):
            blk = one.copy()
            blk[:, 0] = f
            blk[:, 1] = b
            out.append(blk)
    return _iarr(np.concatenate(out))


class Forest:
    """An adaptive forest of patches resident on the GPU."""

    def __init__(self, desc: Desc, leaves):
        L = load()
        self.desc = desc
        leaves = _iarr(leaves).reshape(-1, 5)
        h = ctypes.c_void_p()
        check(L.fc_forest_create(ctypes.byref(desc), len(leaves), _ip(leaves), ctypes.byref(h)))
        self._h = h

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load().fc_forest_destroy(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----------------------------------------------------------------- layout
    @property
    def mx(self) -> int:
        return self.desc.mx

    @property
    def dtype(self):
        return _NP[self.desc.dtype]

    def __len__(self) -> int:
        n = ctypes.c_int()
        check(load().fc_forest_num_leaves(self._h, ctypes.byref(n)))
        return n.value

    def leaves(self) -> np.ndarray:
        out = np.zeros((len(self), 5), dtype=np.int32)
        check(load().fc_forest_leaves(self._h, _ip(out)))
        return out

    # ----------------------------------------------------------------- field
    def set_q(self, q, stream=None):
        """q: host array (n, mx, mx) or a contiguous CUDA tensor of the forest dtype."""
        n, mx = len(self), self.mx
        if hasattr(q, "is_cuda") and q.is_cuda:
            assert q.is_contiguous() and q.numel() == n * mx * mx
            assert q.element_size() == np.dtype(self.dtype).itemsize
            check(load().fc_forest_set_q(self._h, ctypes.c_void_p(q.data_ptr()), 1,
                                         _stream(stream)))
        else:
            a = np.ascontiguousarray(q, dtype=self.dtype).reshape(n, mx, mx)
            check(load().fc_forest_set_q(self._h, a.ctypes.data_as(ctypes.c_void_p), 0,
                                         _stream(stream)))

    def poison(self, value: float, stream=None):
        """Test aid (fc_forest_poison): value into every ghost cell of both
        state buffers and every time-interpolation tile cell."""
        check(load().fc_forest_poison(self._h, float(value), _stream(stream)))

    def get_q(self, out=None, stream=None, full: bool = False):
        """Interior (or, with full=True, ghost-including) field, host or device."""
        n = len(self)
        side = self.mx + 4 if full else self.mx
        fn = load().fc_forest_get_q_full if full else load().fc_forest_get_q
        if out is not None and hasattr(out, "is_cuda") and out.is_cuda:
            assert out.is_contiguous() and out.numel() == n * side * side
            check(fn(self._h, ctypes.c_void_p(out.data_ptr()), 1, _stream(stream)))
            return out
        a = np.empty((n, side, side), dtype=self.dtype)
        check(fn(self._h, a.ctypes.data_as(ctypes.c_void_p), 0, _stream(stream)))
        return a

    def capacity(self, out=None, stream=None):
        """Interior cell capacities (n, mx, mx) in FP64: h^2, or kappa on the sphere."""
        n, mx = len(self), self.mx
        if out is not None and hasattr(out, "is_cuda") and out.is_cuda:
            assert out.is_contiguous() and out.numel() == n * mx * mx
            check(load().fc_forest_get_capacity(self._h, ctypes.c_void_p(out.data_ptr()), 1,
                                                _stream(stream)))
            return out
        a = np.empty((n, mx, mx))
        check(load().fc_forest_get_capacity(self._h, a.ctypes.data_as(ctypes.c_void_p), 0,
                                            _stream(stream)))
        return a

    # ----------------------------------------------------------------- stepping
    def fill_ghosts(self, stream=None):
        check(load().fc_fill_ghosts(self._h, _stream(stream)))

    def advance_level(self, level: int, t: float, dt: float, stream=None):
        check(load().fc_advance_level(self._h, level, t, dt, _stream(stream)))

    def step_global(self, t: float, dt: float, stream=None):
        check(load().fc_step_global(self._h, t, dt, _stream(stream)))

    def step_multirate(self, t: float, dt_coarse: float, stream=None):
        check(load().fc_step_multirate(self._h, t, dt_coarse, _stream(stream)))

    def tag(self, stream=None) -> np.ndarray:
        out = np.zeros(len(self))
        check(load().fc_tag(self._h, _dp(out), _stream(stream)))
        return out

    def tag_regrid(self, tau_r: float, tau_c: float, lmax_f: Optional[Sequence[int]] = None,
                   stream=None) -> int:
        ch = ctypes.c_int()
        lm = None
        if lmax_f is not None:
            self._lm = _iarr(lmax_f)
            lm = _ip(self._lm)
        check(load().fc_tag_regrid(self._h, tau_r, tau_c, lm, ctypes.byref(ch), _stream(stream)))
        return ch.value

    def autotune(self, stream=None) -> dict:
        """Tune level substeps per launch size; returns {bucket: (variant, warps, fused, ns)}."""
        rep = np.zeros((32, 4), dtype=np.int32)
        check(load().fc_autotune(self._h, _ip(rep), _stream(stream)))
        return {b: tuple(int(v) for v in rep[b]) for b in range(32) if rep[b, 0] >= 0}

    def set_advance_variant(self, variant: int, warps: int = 4):
        """Force 0 staged / 1 walk / 2 walk1 / 3 band for every launch; -1
        restores the tuned choice (warps 2, 4, 8; 16 for band)."""
        check(load().fc_set_advance_variant(self._h, variant, warps))

    def set_limits(self, walk_ctas: int = 0, wait_polls: int = -1):
        """Cap the walk grid (0: residency) and set the update kernels' bounded
        wait (polls; negative: default) -- see fc_set_limits."""
        check(load().fc_set_limits(self._h, int(walk_ctas), int(wait_polls)))

    def set_velocity_scale(self, scale: float):
        check(load().fc_set_velocity_scale(self._h, float(scale)))

    def adjoint_step_global(self, t: float, dt: float, lam, dscale, stream=None):
        """In place: lam (CUDA tensor, field layout) <- adjoint of the step's input;
        dscale (CUDA float64 tensor, 1 element) += velocity-scale derivative."""
        assert lam.is_cuda and lam.is_contiguous() and dscale.is_cuda
        check(load().fc_adjoint_step_global(self._h, t, dt, ctypes.c_void_p(lam.data_ptr()),
                                            ctypes.c_void_p(dscale.data_ptr()), _stream(stream)))

    def adjoint_advance(self, level: int, t: float, dt: float, lam, lam_old, dscale,
                        stream=None):
        """Adjoint of fc_advance_level(level, t, dt) from the state before it:
        lam (CUDA tensor, field layout) in place; lam_old (same, or None when
        level-1 is not time-interpolated) accumulates the older states' share;
        dscale (CUDA float64, 1 element) += the velocity-scale derivative."""
        assert lam.is_cuda and lam.is_contiguous() and dscale.is_cuda
        lo = None
        if lam_old is not None:
            assert lam_old.is_cuda and lam_old.is_contiguous()
            lo = ctypes.c_void_p(lam_old.data_ptr())
        check(load().fc_adjoint_advance(self._h, level, t, dt, ctypes.c_void_p(lam.data_ptr()),
                                        lo, ctypes.c_void_p(dscale.data_ptr()),
                                        _stream(stream)))

    def info(self) -> dict:
        """Leaf counts per level, device bytes held, captured graphs (fc_forest_info)."""
        i = _lib.Info()
        check(load().fc_forest_info(self._h, ctypes.byref(i)))
        out = {n: getattr(i, n) for n, _ in _lib.Info._fields_ if n != "leaves_per_level"}
        out["leaves_per_level"] = list(i.leaves_per_level)
        return out

    def adjoint_step_multirate(self, t: float, dt_coarse: float, lam, dscale, stream=None):
        """Adjoint of one coarse multirate step from the current state (left
        unchanged): lam (CUDA tensor, field layout) in place, dscale += the
        velocity-scale derivative (CUDA float64 tensor, 1 element)."""
        assert lam.is_cuda and lam.is_contiguous() and dscale.is_cuda
        check(load().fc_adjoint_step_multirate(self._h, t, dt_coarse,
                                               ctypes.c_void_p(lam.data_ptr()),
                                               ctypes.c_void_p(dscale.data_ptr()),
                                               _stream(stream)))

    def step_multirate_record(self, t: float, dt_coarse: float, slot: int, stream=None):
        """fc_step_multirate that also keeps, in tape `slot`, what the step's
        reverse reads (see adjoint_step_multirate_taped)."""
        check(load().fc_step_multirate_record(self._h, t, dt_coarse, slot, _stream(stream)))

    def adjoint_step_multirate_taped(self, t: float, dt_coarse: float, slot: int, lam, dscale,
                                     stream=None):
        """Adjoint of the coarse step recorded in tape `slot` (the state is
        neither read nor changed): lam and dscale as in adjoint_step_multirate."""
        assert lam.is_cuda and lam.is_contiguous() and dscale.is_cuda
        check(load().fc_adjoint_step_multirate_taped(self._h, t, dt_coarse, slot,
                                                     ctypes.c_void_p(lam.data_ptr()),
                                                     ctypes.c_void_p(dscale.data_ptr()),
                                                     _stream(stream)))

    def release_tapes(self):
        """Free the tapes of recorded steps."""
        check(load().fc_tape_release(self._h))

    def fused_fill(self, enable: bool = True):
        """Multirate substeps fill each patch's ghosts inside the update kernel (default on)."""
        check(load().fc_set_fused_fill(self._h, 1 if enable else 0))

    def graphs(self, enable: bool = True):
        """Replay coarse multirate steps from captured CUDA graphs (default on)."""
        check(load().fc_set_graphs(self._h, 1 if enable else 0))

    def timers(self, enable: bool = True):
        check(load().fc_timers_enable(self._h, 1 if enable else 0))

    def read_timer(self, phase: int, reset: bool = True):
        """(ms, launches, algorithmic bytes) of phase 0 advance, 1 fill, 2 regrid, 3 other."""
        ms, n, b = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
        check(load().fc_timers_read(self._h, phase, ctypes.byref(ms), ctypes.byref(n),
                                    ctypes.byref(b), 1 if reset else 0))
        return ms.value, n.value, b.value

    def mass(self, stream=None) -> np.ndarray:
        out = np.zeros(self.desc.nforests)
        check(load().fc_forest_mass(self._h, _dp(out), _stream(stream)))
        return out


def initial_forest(desc: Desc, q0: Callable[[np.ndarray], np.ndarray],
                   lmax_f: Optional[Sequence[int]] = None, tau_r: float = 0.05,
                   tau_c: float = 0.0125, stream=None) -> Forest:
    """Adaptive initial layout: start uniform at lmin, then (lmax - lmin) times
    set q0 on the current leaves and tag/regrid; finally set q0 once more.

    ``q0(leaves)`` returns the initial field (n, mx, mx) for a leaf array.
    """
    nb = (6 if desc.domain == _lib.SPHERE else
          desc.brick_nx * desc.brick_ny if desc.domain == _lib.BRICK else 1)
    F = Forest(desc, uniform_leaves(desc.lmin, desc.nforests, nb))
    for _ in range(desc.lmax - desc.lmin):
        F.set_q(q0(F.leaves()), stream=stream)
        F.tag_regrid(tau_r, tau_c, lmax_f, stream=stream)
    F.set_q(q0(F.leaves()), stream=stream)
    return F


_ALLOCATOR = None  # the callbacks in use (kept alive while the library holds them)


def set_allocator(alloc=None, release=None) -> None:
    """Route every device allocation of the library through alloc(bytes, stream)
    -> int pointer and release(ptr, bytes, stream) (fc_set_allocator); no
    arguments restores the stream-ordered pool.  Only while no forest exists."""
    global _ALLOCATOR
    if alloc is None:
        check(load().fc_set_allocator(None, None, None))
        _ALLOCATOR = None
        return

    def a(nbytes, stream, user):
        try:
            return int(alloc(int(nbytes), stream or 0)) or None
        except Exception:
            return None

    def r(ptr, nbytes, stream, user):
        try:
            release(int(ptr), int(nbytes), stream or 0)
        except Exception:
            pass

    cb = (_lib.ALLOC_FN(a), _lib.FREE_FN(r))
    check(load().fc_set_allocator(ctypes.cast(cb[0], ctypes.c_void_p),
                                  ctypes.cast(cb[1], ctypes.c_void_p), None))
    _ALLOCATOR = cb


def torch_allocator():
    """(alloc, release) over torch's CUDA caching allocator, for set_allocator."""
    import torch

    def alloc(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, torch.cuda.current_device(), stream)

    def release(ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(ptr)

    return alloc, release


def layout_check(desc: Desc, leaves) -> None:
    leaves = _iarr(leaves).reshape(-1, 5)
    check(load().fc_layout_check(ctypes.byref(desc), len(leaves), _ip(leaves)))


def layout_neighbours(desc: Desc, leaves) -> np.ndarray:
    leaves = _iarr(leaves).reshape(-1, 5)
    out = np.zeros((len(leaves), 8, 6), dtype=np.int32)  # kind 4: beyond a cube vertex
    check(load().fc_layout_neighbours(ctypes.byref(desc), len(leaves), _ip(leaves), _ip(out)))
    return out


def layout_reflux(desc: Desc, leaves) -> np.ndarray:
    """Refluxing's pairing (host): (n, 4, mx, 5) ints (kind, leaf across, its
    face, j0, j1) per leaf, face and face cell; see fc_layout_reflux."""
    leaves = _iarr(leaves).reshape(-1, 5)
    out = np.zeros((len(leaves), 4, desc.mx, 5), dtype=np.int32)
    check(load().fc_layout_reflux(ctypes.byref(desc), len(leaves), _ip(leaves), _ip(out)))
    return out


def layout_regrid(desc: Desc, leaves, delta, tau_r: float, tau_c: float,
                  lmax_f: Optional[Sequence[int]] = None) -> np.ndarray:
    leaves = _iarr(leaves).reshape(-1, 5)
    d = np.ascontiguousarray(delta, dtype=np.float64)
    cap = 4 * len(leaves) + 64
    while True:
        out = np.zeros((cap, 5), dtype=np.int32)
        nout = ctypes.c_int()
        lm = _iarr(lmax_f) if lmax_f is not None else None
        st = load().fc_layout_regrid(ctypes.byref(desc), len(leaves), _ip(leaves), _dp(d),
                                     tau_r, tau_c, _ip(lm) if lm is not None else None,
                                     cap, _ip(out), ctypes.byref(nout))
        if st == _lib.FC_OK:
            return out[:nout.value]
        if nout.value > cap:
            cap = nout.value
            continue
        check(st)
