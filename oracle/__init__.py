"""CPU oracle (plain C, FP64) for the patch-AMR wave-propagation method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA path; the two meet only in the seeded inputs of ``synth``.

The C sources are compiled here with gcc (``-ffp-contract=off`` so that the
arithmetic is the same on every host) into ``oracle/liboracle.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SO_OMP = os.path.join(_HERE, "liboracle_omp.so")  # the same sources, patch loops over threads
_SRC = ["forest.c", "ghost.c", "claw.c", "drive.c", "adjoint.c", "sphere.c"]
_HDR = ["oracle.h", "internal.h"]

WALLS, PERIODIC, SPHERE, BRICK = 0, 1, 2, 3
VEL_CONST, VEL_SWIRL, VEL_ROTATION, VEL_DEFORM = 0, 1, 2, 3


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle into liboracle.so (skipped when up to date); with
    openmp=True the same sources into liboracle_omp.so with -fopenmp, whose
    patch loops run on all host threads (for the all-cores CPU baseline)."""
    so = _SO_OMP if openmp else _SO
    srcs = [os.path.join(_HERE, s) for s in _SRC]
    deps = srcs + [os.path.join(_HERE, h) for h in _HDR]
    if not force and os.path.exists(so):
        so_t = os.path.getmtime(so)
        if all(os.path.getmtime(d) <= so_t for d in deps):
            return so
    tmp = so + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
           "-Wall", *(["-fopenmp"] if openmp else []), *srcs, "-lm", "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, so)
    return so


class _Params(ctypes.Structure):
    _fields_ = [
        ("domain", ctypes.c_int), ("nforests", ctypes.c_int),
        ("mx", ctypes.c_int), ("mbc", ctypes.c_int),
        ("lmin", ctypes.c_int), ("lmax", ctypes.c_int),
        ("vel_kind", ctypes.c_int), ("vel", ctypes.c_double * 4),
        ("order", ctypes.c_int), ("limiter", ctypes.c_int),
        ("transverse", ctypes.c_int), ("vel_scale", ctypes.c_double),
        ("indicator", ctypes.c_int), ("smooth", ctypes.c_int),
        ("reflux", ctypes.c_int), ("brick", ctypes.c_int * 2),
    ]


_lib = None
_libs = {}


def use_openmp(on: bool = True) -> None:
    """Select the library that forests created from now on use: the OpenMP
    build (patch loops on all host threads) or the plain one."""
    global _lib
    _lib = _load(on)


def threads() -> int:
    """Host threads the OpenMP build's patch loops use (1 for the plain build)."""
    if _lib is None or _lib is not _libs.get(True):
        return 1
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def lib():
    global _lib
    if _lib is None:
        _lib = _load(False)
    return _lib


def _load(openmp: bool):
    if openmp in _libs:
        return _libs[openmp]
    so = build(openmp=openmp)
    L = ctypes.CDLL(so)
    vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    L.or_create.restype = vp
    L.or_create.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, ip]
    L.or_destroy.argtypes = [vp]
    L.or_num_leaves.argtypes = [vp]
    L.or_get_leaves.argtypes = [vp, ip]
    for f in ("or_set_q", "or_get_q", "or_get_q_full", "or_set_q_full"):
        getattr(L, f).argtypes = [vp, dp]
    L.or_fill_ghosts.argtypes = [vp]
    L.or_step_global.argtypes = [vp, ctypes.c_double, ctypes.c_double]
    L.or_step_multirate.argtypes = [vp, ctypes.c_double, ctypes.c_double]
    L.or_tag.argtypes = [vp, dp]
    L.or_regrid.argtypes = [vp, ctypes.c_double, ctypes.c_double, ip, ip]
    L.or_mass.argtypes = [vp, dp]
    L.or_adjoint_global.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp,
                                    dp, dp]
    L.or_adjoint_step_global.argtypes = [vp, ctypes.c_double, ctypes.c_double, dp, dp]
    L.or_adjoint_multirate.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp,
                                       dp, dp, dp]
    L.or_adjoint_step_multirate.argtypes = [vp, ctypes.c_double, ctypes.c_double, dp, dp]
    L.or_set_params.argtypes = [vp, ctypes.POINTER(_Params)]
    L.or_sphere_centres.argtypes = [vp, dp]
    L.or_get_kappa.argtypes = [vp, dp]
    L.or_get_kappa_full.argtypes = [vp, dp]
    L.or_reflux_pairs.argtypes = [vp, ip]
    L.or_sphere_edge_fluxes.argtypes = [vp, ctypes.c_double, dp, dp]
    L.or_single_grid_periodic.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, dp,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_int]
    for f in ("or_u_edge", "or_v_edge"):
        getattr(L, f).restype = ctypes.c_double
        getattr(L, f).argtypes = [ctypes.POINTER(_Params), ctypes.c_double, ctypes.c_double,
                                  ctypes.c_long, ctypes.c_long, ctypes.c_int, ctypes.c_int]
    L.or_mc_phi.restype = ctypes.c_double
    L.or_mc_phi.argtypes = [ctypes.c_double]
    L.or_minmod.restype = ctypes.c_double
    L.or_minmod.argtypes = [ctypes.c_double, ctypes.c_double]
    L.or_last_error.restype = ctypes.c_char_p
    _libs[openmp] = L
    return L


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


class OracleError(RuntimeError):
    pass


def _check(rc: int):
    if rc != 0:
        raise OracleError(lib().or_last_error().decode())


def params(domain: int, mx: int, mbc: int, lmin: int, lmax: int, velocity,
           order: int = 2, limiter: int = 1, transverse: int = 2,
           nforests: int = 1, indicator: int = 0, smooth: int = 0,
           reflux: int = 0, brick=(1, 1)) -> _Params:
    p = _Params()
    p.domain, p.nforests, p.mx, p.mbc, p.lmin, p.lmax = domain, nforests, mx, mbc, lmin, lmax
    if velocity[0] == "const":
        p.vel_kind = VEL_CONST
        p.vel[0], p.vel[1] = float(velocity[1]), float(velocity[2])
    elif velocity[0] == "swirl":
        p.vel_kind = VEL_SWIRL
        p.vel[0] = float(velocity[1])
    elif velocity[0] == "rotation":
        p.vel_kind = VEL_ROTATION
        for k in range(3):
            p.vel[k] = float(velocity[1 + k])
    elif velocity[0] == "deform":  # Sec. 5.3: (kappa, T, T_f)
        p.vel_kind = VEL_DEFORM
        for k in range(3):
            p.vel[k] = float(velocity[1 + k])
    else:
        raise ValueError(velocity)
    p.order, p.limiter, p.transverse = order, limiter, transverse
    p.vel_scale = 1.0
    p.indicator, p.smooth, p.reflux = indicator, smooth, reflux
    p.brick[0], p.brick[1] = int(brick[0]), int(brick[1])
    return p


def uniform_leaves(level: int, nforests: int = 1, nblocks: int = 1) -> np.ndarray:
    n = 1 << level
    out = [(f, b, level, x, y) for f in range(nforests) for b in range(nblocks)
           for y in range(n) for x in range(n)]
    return np.asarray(out, dtype=np.int32).reshape(-1, 5)


class Forest:
    """One oracle forest (owner of a C handle)."""

    def __init__(self, prm: _Params, leaves: np.ndarray):
        self.prm = prm
        self.L = lib()  # the build (plain or OpenMP) this forest lives in
        leaves = np.ascontiguousarray(leaves, dtype=np.int32).reshape(-1, 5)
        h = self.L.or_create(ctypes.byref(prm), len(leaves), _iptr(leaves))
        if not h:
            raise OracleError(self.L.or_last_error().decode())
        self.h = h

    def _check(self, rc: int):
        if rc != 0:
            raise OracleError(self.L.or_last_error().decode())

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.or_destroy(h)
            self.h = None

    @property
    def mx(self) -> int:
        return self.prm.mx

    @property
    def S(self) -> int:
        return self.prm.mx + 2 * self.prm.mbc

    def __len__(self) -> int:
        return self.L.or_num_leaves(self.h)

    def leaves(self) -> np.ndarray:
        out = np.zeros((len(self), 5), dtype=np.int32)
        self.L.or_get_leaves(self.h, _iptr(out))
        return out

    def set_q(self, q: np.ndarray):
        q = np.ascontiguousarray(q, dtype=np.float64).reshape(len(self), self.mx, self.mx)
        self.L.or_set_q(self.h, _dptr(q))

    def get_q(self) -> np.ndarray:
        out = np.zeros((len(self), self.mx, self.mx))
        self.L.or_get_q(self.h, _dptr(out))
        return out

    def get_q_full(self) -> np.ndarray:
        out = np.zeros((len(self), self.S, self.S))
        self.L.or_get_q_full(self.h, _dptr(out))
        return out

    def set_q_full(self, q: np.ndarray):
        q = np.ascontiguousarray(q, dtype=np.float64).reshape(len(self), self.S, self.S)
        self.L.or_set_q_full(self.h, _dptr(q))

    def fill_ghosts(self):
        self._check(self.L.or_fill_ghosts(self.h))

    def step_global(self, t: float, dt: float):
        self._check(self.L.or_step_global(self.h, t, dt))

    def step_multirate(self, t: float, dt_coarse: float):
        self._check(self.L.or_step_multirate(self.h, t, dt_coarse))

    def tag(self) -> np.ndarray:
        out = np.zeros(len(self))
        self._check(self.L.or_tag(self.h, _dptr(out)))
        return out

    def regrid(self, tau_r: float, tau_c: float,
               lmax_f: Optional[Sequence[int]] = None) -> int:
        changed = np.zeros(1, dtype=np.int32)
        lm = None
        if lmax_f is not None:
            lm_arr = np.ascontiguousarray(lmax_f, dtype=np.int32)
            lm = _iptr(lm_arr)
        self._check(self.L.or_regrid(self.h, tau_r, tau_c, lm, _iptr(changed)))
        return int(changed[0])

    def mass(self) -> np.ndarray:
        out = np.zeros(self.prm.nforests)
        self.L.or_mass(self.h, _dptr(out))
        return out

    def adjoint_global(self, nsteps: int, t0: float, dt: float, q_target: np.ndarray):
        """(loss, dL/dq0, dL/dscale) of L = 1/2 |q_N - q_target|^2 after nsteps
        global steps from the current state (which is left unchanged)."""
        qt = np.ascontiguousarray(q_target, dtype=np.float64).reshape(len(self), self.mx, self.mx)
        g = np.zeros_like(qt)
        gs = np.zeros(1)
        loss = np.zeros(1)
        self._check(self.L.or_adjoint_global(self.h, nsteps, t0, dt, _dptr(qt), _dptr(g), _dptr(gs),
                                       _dptr(loss)))
        return float(loss[0]), g, float(gs[0])

    def adjoint_step_global(self, t: float, dt: float, lam: np.ndarray):
        """Adjoint of one global step at the current state: returns (lam_n, dscale)."""
        lam = np.ascontiguousarray(lam, dtype=np.float64).reshape(len(self), self.mx, self.mx).copy()
        ds = np.zeros(1)
        self._check(self.L.or_adjoint_step_global(self.h, t, dt, _dptr(lam), _dptr(ds)))
        return lam, float(ds[0])

    def adjoint_multirate(self, ncoarse: int, t0: float, dtc: float, q_target: np.ndarray):
        """(loss, dL/dq0, dL/dscale) after ncoarse coarse multirate steps from the
        current state (which is left unchanged)."""
        qt = np.ascontiguousarray(q_target, dtype=np.float64).reshape(len(self), self.mx, self.mx)
        g = np.zeros_like(qt)
        gs = np.zeros(1)
        loss = np.zeros(1)
        self._check(self.L.or_adjoint_multirate(self.h, ncoarse, t0, dtc, _dptr(qt), _dptr(g),
                                          _dptr(gs), _dptr(loss)))
        return float(loss[0]), g, float(gs[0])

    def adjoint_step_multirate(self, t: float, dtc: float, lam: np.ndarray):
        """Adjoint of one coarse multirate step at the current state: (lam_n, dscale)."""
        lam = np.ascontiguousarray(lam, dtype=np.float64).reshape(len(self), self.mx, self.mx).copy()
        ds = np.zeros(1)
        self._check(self.L.or_adjoint_step_multirate(self.h, t, dtc, _dptr(lam), _dptr(ds)))
        return lam, float(ds[0])

    def sphere_centres(self) -> np.ndarray:
        """Unit-sphere positions of the interior cell centres, (n, mx, mx, 3)."""
        out = np.zeros((len(self), self.mx, self.mx, 3))
        self.L.or_sphere_centres(self.h, _dptr(out))
        return out

    def kappa(self) -> np.ndarray:
        """Cell capacities (spherical areas) of the interior cells, (n, mx, mx)."""
        out = np.zeros((len(self), self.mx, self.mx))
        self.L.or_get_kappa(self.h, _dptr(out))
        return out

    def reflux_pairs(self) -> np.ndarray:
        """What refluxing exchanges per (leaf, face, face cell): (n, 4, mx, 5) of
        (kind, leaf across, its face, j0, j1); see or_reflux_pairs."""
        out = np.zeros((len(self), 4, self.mx, 5), dtype=np.int32)
        self.L.or_reflux_pairs(self.h, _iptr(out))
        return out

    def kappa_full(self) -> np.ndarray:
        """Cell capacities over the extended range (ghost cells included), (n, S, S)."""
        out = np.zeros((len(self), self.S, self.S))
        self.L.or_get_kappa_full(self.h, _dptr(out))
        return out

    def edge_fluxes(self, t: float = 0.0):
        """Edge volume fluxes at time t over the extended index range:
        x-edges (n, S, S+1) [row j, edge i - 1/2] and y-edges (n, S+1, S)
        [edge j - 1/2, column i], both with index -mbc at 0."""
        S = self.S
        px = np.zeros((len(self), S, S + 1))
        py = np.zeros((len(self), S + 1, S))
        self.L.or_sphere_edge_fluxes(self.h, t, _dptr(px), _dptr(py))
        return px, py

    def set_velocity_scale(self, s: float):
        """Scale every edge speed (the parameter of the velocity-scale gradient)."""
        self.prm.vel_scale = float(s)
        self.L.or_set_params(self.h, ctypes.byref(self.prm))


def single_grid_periodic(prm: _Params, q: np.ndarray, t0: float, dt: float,
                         nsteps: int) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.float64).copy()
    N = q.shape[0]
    _check(lib().or_single_grid_periodic(ctypes.byref(prm), N, _dptr(q), t0, dt, nsteps))
    return q


def edge_speeds(prm: _Params, h: float, t: float, n: int):
    """Edge speeds of the single-grid scheme at velocity time t on an n x n grid
    of cell width h: u at the x-edges (i - 1/2, j), shape (n, n + 1) [j, i],
    and v at the y-edges (i, j - 1/2), shape (n + 1, n) [j, i]."""
    L = lib()
    u = np.array([[L.or_u_edge(ctypes.byref(prm), h, t, 0, 0, i, j) for i in range(n + 1)]
                  for j in range(n)])
    v = np.array([[L.or_v_edge(ctypes.byref(prm), h, t, 0, 0, i, j) for i in range(n)]
                  for j in range(n + 1)])
    return u, v


def mc_phi(theta: float) -> float:
    return lib().or_mc_phi(float(theta))


def minmod(a: float, b: float) -> float:
    return lib().or_minmod(float(a), float(b))


# ---------------------------------------------------------------- workloads

_DOMAIN = {"walls": WALLS, "periodic": PERIODIC, "sphere": SPHERE, "brick": BRICK}
_LIMITER = {"none": (2, 0), "lw": (2, 0), "mc": (2, 1), "first": (1, 0)}


_INDICATOR = {"gradient": 0, "maxmin": 1}


def params_for(w, nforests: int = 1, lmax: Optional[int] = None) -> _Params:
    order, lim = _LIMITER[w.limiter]
    return params(_DOMAIN[w.domain], w.mx, w.mbc, w.lmin,
                  w.lmax if lmax is None else lmax, w.velocity, order=order,
                  limiter=lim, transverse=w.transverse, nforests=nforests,
                  indicator=_INDICATOR[w.indicator], smooth=int(w.smooth),
                  reflux=int(w.reflux), brick=w.brick)


def initial_forest(workloads, lmax: Optional[int] = None) -> Forest:
    """Build the initial adaptive forest of one or more workloads.

    Start every forest uniformly at lmin, then (lmax_f - lmin) times: set the
    analytic field at the cell centres, tag, refine/coarsen/balance; finally
    set the analytic field on the final layout.
    """
    import synth
    if not isinstance(workloads, (list, tuple)):
        workloads = [workloads]
    w0 = workloads[0]
    nf = len(workloads)
    lmax_all = max(w.lmax for w in workloads) if lmax is None else lmax
    prm = params_for(w0, nforests=nf, lmax=lmax_all)
    sphere = w0.domain == "sphere"
    nb = 6 if sphere else w0.brick[0] * w0.brick[1] if w0.domain == "brick" else 1
    leaves = np.concatenate([uniform_leaves(w0.lmin, 1, nb) + np.array([f, 0, 0, 0, 0], np.int32)
                             for f in range(nf)])
    F = Forest(prm, leaves)
    lmax_f = [w.lmax for w in workloads]

    def set_analytic():
        lv = F.leaves()
        if sphere:
            X = F.sphere_centres()
            q = np.empty(X.shape[:3])
            for f, w in enumerate(workloads):
                sel = lv[:, 0] == f
                q[sel] = synth.evaluate_sphere(w, X[sel])
            F.set_q(q)
            return
        x, y = synth.cell_centres(lv, w0.mx)
        q = np.empty(x.shape)
        for f, w in enumerate(workloads):
            sel = lv[:, 0] == f
            q[sel] = synth.evaluate(w, x[sel], y[sel])
        F.set_q(q)

    for _ in range(lmax_all - w0.lmin):
        set_analytic()
        F.regrid(w0.tau_refine, w0.tau_coarsen, lmax_f)
    set_analytic()
    return F
