"""Seeded synthetic inputs for the patch-AMR advection workloads.

This module is the one piece shared by the CPU oracle and the CUDA path.  It
holds no arithmetic of the method: it draws seeded parameters (numpy PCG64)
and evaluates the analytic initial fields at points that the caller supplies.
Every workload is synthetic; the paper's own runs also start from analytic
tracer fields (a piecewise-constant disc pattern in the replicated-domain test,
a slotted disk on the sphere), so nothing here stands in for a dataset.

Workloads (unit square = one block; cubed sphere = six blocks):

* ``uniform_periodic``: one periodic tree refined uniformly to level 3,
  16x16 patches (a 128^2 grid), constant velocity (1, 0.5), MC limiter with
  transverse corrections, CFL 0.9, 100 steps.  q0 = four Gaussians
  (amplitude U[0.5,1], width U[0.03,0.08], centre U[0,1]^2, periodic distance)
  plus a square pulse of value 1 (side 0.25, corner U[0,0.75]^2).
* ``swirl``: one walled tree, levels 2..6, 32x32 patches, swirl velocity with
  period T=4, q0 = 1 inside a radius-0.2 disc (centre U[0.2,0.8]^2), else 0.
* ``ensemble``: many independent swirl forests, each with its own disc and a
  maximum level drawn from {4,5,6}.
* ``adjoint``: the swirl forest plus a target field from a disc whose centre is
  shifted by a seeded offset of at most 0.05.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

__all__ = [
    "Gaussians", "Disc", "SquarePulse", "Workload", "uniform_periodic",
    "swirl", "ensemble", "adjoint_target", "smooth_periodic", "cell_centres", "sphere_deform",
    "evaluate", "random_field", "time_step",
]


@dataclasses.dataclass
class Gaussians:
    amp: np.ndarray      # (k,)
    width: np.ndarray    # (k,)
    centre: np.ndarray   # (k, 2)
    periodic: bool = True


@dataclasses.dataclass
class SquarePulse:
    corner: np.ndarray   # (2,)
    side: float = 0.25
    periodic: bool = True


@dataclasses.dataclass
class Disc:
    centre: np.ndarray   # (2,)
    radius: float = 0.2


@dataclasses.dataclass
class DiscUnion:
    """1 inside any of the discs (periodic distances in the unit block), else 0."""
    centres: np.ndarray  # (k, 2)
    radius: float = 0.3


@dataclasses.dataclass
class Workload:
    """One forest's problem description (parameters only, no numerics)."""
    name: str
    domain: str          # "periodic" | "walls" | "sphere"
    mx: int
    mbc: int
    lmin: int
    lmax: int
    velocity: tuple      # ("const", u, v) | ("swirl", T)
    limiter: str         # "none" | "mc" | "lw"
    transverse: int      # 0, 1 (fluctuations), 2 (fluctuations + corrections)
    cfl: float
    parts: list          # list of Gaussians / SquarePulse / Disc
    steps: Optional[int] = None
    t_final: Optional[float] = None
    regrid_every: int = 0
    tau_refine: float = 0.05
    tau_coarsen: float = 0.0125
    seed: int = 0
    indicator: str = "gradient"  # regrid indicator: "gradient" | "maxmin" (Sec. 5.1)
    smooth: bool = False         # smooth grading of the target levels (Sec. 3.3)
    reflux: bool = False         # conservative coarse/fine correction (off in the paper)
    dt_lmin: Optional[float] = None  # fixed time step of level lmin (else from the CFL number)
    brick: tuple = (1, 1)        # "brick" domain: blocks per row and per column


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_periodic(seed: int = 0, level: int = 3, mx: int = 16,
                     steps: int = 100) -> Workload:
    g = _rng(seed)
    k = 4
    amp = g.uniform(0.5, 1.0, k)
    width = g.uniform(0.03, 0.08, k)
    centre = g.uniform(0.0, 1.0, (k, 2))
    corner = g.uniform(0.0, 0.75, 2)
    return Workload(
        name=f"uniform periodic level {level} mx={mx}", domain="periodic",
        mx=mx, mbc=2, lmin=level, lmax=level, velocity=("const", 1.0, 0.5),
        limiter="mc", transverse=2, cfl=0.9,
        parts=[Gaussians(amp, width, centre), SquarePulse(corner)],
        steps=steps, seed=seed)


def smooth_periodic(seed: int = 0, level: int = 2, mx: int = 16,
                    velocity=("const", 1.0, 0.5), limiter="none") -> Workload:
    """Gaussians only (smooth), for convergence studies."""
    g = _rng(seed)
    k = 4
    amp = g.uniform(0.5, 1.0, k)
    width = g.uniform(0.08, 0.12, k)
    centre = g.uniform(0.0, 1.0, (k, 2))
    return Workload(
        name="smooth periodic", domain="periodic", mx=mx, mbc=2, lmin=level,
        lmax=level, velocity=velocity, limiter=limiter, transverse=2, cfl=0.9,
        parts=[Gaussians(amp, width, centre)], seed=seed)


def swirl(seed: int = 0, lmin: int = 2, lmax: int = 6, mx: int = 32,
          period: float = 4.0, regrid_every: int = 4) -> Workload:
    g = _rng(seed)
    centre = g.uniform(0.2, 0.8, 2)
    return Workload(
        name=f"swirl levels {lmin}-{lmax} mx={mx}", domain="walls", mx=mx,
        mbc=2, lmin=lmin, lmax=lmax, velocity=("swirl", period),
        limiter="mc", transverse=2, cfl=0.9, parts=[Disc(centre)],
        t_final=period, regrid_every=regrid_every, seed=seed)


def ensemble(n: int = 256, seed: int = 0, lmin: int = 2, mx: int = 32,
             levels=(4, 5, 6)) -> List[Workload]:
    """n independent swirl forests with seeded discs and maximum levels."""
    g = _rng(seed)
    out = []
    sub_seeds = g.integers(0, 2**31 - 1, n)
    lmaxes = g.choice(np.asarray(levels), n)
    for f in range(n):
        out.append(swirl(int(sub_seeds[f]), lmin=lmin, lmax=int(lmaxes[f]),
                         mx=mx))
    return out


def adjoint_target(w: Workload, seed: int = 0, max_shift: float = 0.05) -> Workload:
    """The same workload with its disc centre moved by a seeded offset."""
    g = _rng(seed + 7919)
    ang = g.uniform(0.0, 2 * np.pi)
    r = g.uniform(0.0, max_shift)
    parts = []
    for p in w.parts:
        if isinstance(p, Disc):
            parts.append(Disc(p.centre + r * np.array([np.cos(ang), np.sin(ang)]),
                              p.radius))
        else:
            parts.append(p)
    return dataclasses.replace(w, parts=parts, name=w.name + " (target)")


@dataclasses.dataclass
class CosineBell:
    centre: np.ndarray   # (3,) unit vector
    radius: float = 0.5  # great-circle radius
    height: float = 1.0


@dataclasses.dataclass
class SlottedCylinder:
    centre: np.ndarray   # (3,) unit vector
    along: np.ndarray    # (3,) unit tangent at the centre: direction the slot opens to
    radius: float = 0.5
    slot: float = 0.1    # slot width


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def brick(seed: int = 0, n: int = 1, lmin: int = 4, lmax: int = 7, mx: int = 32,
          steps: int = 160) -> Workload:
    """Sec. 5.1's replicated problem: a periodic brick of 2^n x 2^n unit
    blocks, each an adaptive quadtree holding the same tracer field (1 inside
    one of five discs of radius 0.3, else 0; the paper shows the discs only
    in a figure, so their centres are seeded, with periodic distances in the
    block), the constant velocity (0.5, 0.5) of the streamfunction
    -(x - y)/2, CFL 0.64 at the finest level, global steps, the spread
    indicator with tau_r = 0.25, tau_c = 0.001, smooth grading, a regrid
    every 2^(lmax - lmin) steps."""
    g = _rng(seed)
    centres = g.uniform(0.0, 1.0, (5, 2))
    k = 1 << n
    return Workload(
        name=f"brick {k}x{k} levels {lmin}-{lmax} mx={mx}", domain="brick", mx=mx, mbc=2,
        lmin=lmin, lmax=lmax, velocity=("const", 0.5, 0.5), limiter="mc", transverse=2,
        cfl=0.64, parts=[DiscUnion(centres, 0.3)], steps=steps,
        regrid_every=1 << (lmax - lmin), tau_refine=0.25, tau_coarsen=0.001,
        indicator="maxmin", smooth=True, seed=seed, brick=(k, k))


def sphere(seed: int = 0, lmin: int = 1, lmax: int = 7, mx: int = 32) -> Workload:
    """Cubed-sphere workload: solid-body rotation about a seeded axis with
    |omega| = 2 pi (one revolution in t = 1), two cosine bells (great-circle
    radius 0.5, height 1) and a slotted cylinder (radius 0.5, slot width 0.1,
    seeded orientation), centres seeded on the sphere."""
    g = _rng(seed)
    axis = _unit(g.normal(size=3))
    omega = 2.0 * np.pi * axis
    cs = [_unit(g.normal(size=3)) for _ in range(3)]
    t = g.normal(size=3)
    along = _unit(t - np.dot(t, cs[2]) * cs[2])
    return Workload(
        name=f"cubed sphere levels {lmin}-{lmax} mx={mx}", domain="sphere", mx=mx, mbc=2,
        lmin=lmin, lmax=lmax, velocity=("rotation", *omega), limiter="mc", transverse=2,
        cfl=0.9, parts=[CosineBell(cs[0]), CosineBell(cs[1]), SlottedCylinder(cs[2], along)],
        t_final=1.0, regrid_every=4, seed=seed)


def sphere_deform(seed: int = 0, lmin: int = 2, lmax: int = 4, mx: int = 32) -> Workload:
    """The paper's cubed-sphere run (Sec. 5.3) in synthetic form: the
    deformational streamfunction with kappa = 2, T = 0.5, T_f = 5, run to
    t = 0.5 with the fixed level-lmin step 2.5e-3 (halved per finer level),
    moving two slotted cylinders (radius 0.5, on the equator around
    longitudes 5 pi / 6 and 7 pi / 6, slots opening to the north; the centres
    are nudged by a seeded few hundredths of a radian)."""
    g = _rng(seed)
    parts = []
    for lon in (5.0 * np.pi / 6.0, 7.0 * np.pi / 6.0):
        lon = lon + g.uniform(-0.02, 0.02)
        lat = g.uniform(-0.02, 0.02)
        c = np.array([np.cos(lat) * np.cos(lon), np.cos(lat) * np.sin(lon), np.sin(lat)])
        north = np.array([-np.sin(lat) * np.cos(lon), -np.sin(lat) * np.sin(lon), np.cos(lat)])
        parts.append(SlottedCylinder(c, north))
    return Workload(
        name=f"cubed sphere deformational flow levels {lmin}-{lmax} mx={mx}", domain="sphere",
        mx=mx, mbc=2, lmin=lmin, lmax=lmax, velocity=("deform", 2.0, 0.5, 5.0), limiter="mc",
        transverse=2, cfl=0.9, parts=parts, t_final=0.5, regrid_every=1,
        indicator="maxmin", tau_refine=0.25, tau_coarsen=0.001, dt_lmin=2.5e-3, seed=seed)


def evaluate_sphere(w: Workload, X: np.ndarray) -> np.ndarray:
    """Initial field of a sphere workload at unit vectors X (..., 3)."""
    X = np.asarray(X, dtype=np.float64)
    q = np.zeros(X.shape[:-1])
    for p in w.parts:
        r = np.arccos(np.clip(X @ p.centre, -1.0, 1.0))  # great-circle distance
        if isinstance(p, CosineBell):
            q = q + np.where(r < p.radius,
                             0.5 * p.height * (1.0 + np.cos(np.pi * r / p.radius)), 0.0)
        elif isinstance(p, SlottedCylinder):
            side = np.cross(p.centre, p.along)
            slot = (np.abs(X @ side) < 0.5 * p.slot) & (X @ p.along > -0.5 * p.radius)
            q = q + ((r < p.radius) & ~slot).astype(np.float64)
        else:
            raise TypeError(type(p))
    return q


def evaluate(w: Workload, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Initial field of workload ``w`` at points (x, y) (unit-square coords)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    q = np.zeros(np.broadcast(x, y).shape)
    for p in w.parts:
        if isinstance(p, Gaussians):
            for a, s, c in zip(p.amp, p.width, p.centre):
                dx = x - c[0]
                dy = y - c[1]
                if p.periodic:
                    dx = dx - np.round(dx)
                    dy = dy - np.round(dy)
                q = q + a * np.exp(-(dx * dx + dy * dy) / (s * s))
        elif isinstance(p, SquarePulse):
            dx = x - p.corner[0]
            dy = y - p.corner[1]
            if p.periodic:
                dx = np.mod(dx, 1.0)
                dy = np.mod(dy, 1.0)
            inside = (dx >= 0) & (dx < p.side) & (dy >= 0) & (dy < p.side)
            q = q + inside.astype(np.float64)
        elif isinstance(p, DiscUnion):
            inside = np.zeros(q.shape, dtype=bool)
            for c in p.centres:
                dx = x - c[0]
                dy = y - c[1]
                dx = dx - np.round(dx)
                dy = dy - np.round(dy)
                inside |= (dx * dx + dy * dy) < p.radius * p.radius
            q = q + inside.astype(np.float64)
        elif isinstance(p, Disc):
            dx = x - p.centre[0]
            dy = y - p.centre[1]
            q = q + ((dx * dx + dy * dy) < p.radius * p.radius).astype(np.float64)
        else:
            raise TypeError(type(p))
    return q


# cubed-sphere block convention of the C interface: block b is the cube face
# with outward normal n, block point (x, y) at n + (2x-1) ex + (2y-1) ey
_CUBE = {0: ((0, 0, 1), (1, 0, 0), (0, 1, 0)), 1: ((0, 0, -1), (1, 0, 0), (0, -1, 0)),
         2: ((1, 0, 0), (0, 1, 0), (0, 0, 1)), 3: ((-1, 0, 0), (0, -1, 0), (0, 0, 1)),
         4: ((0, 1, 0), (-1, 0, 0), (0, 0, 1)), 5: ((0, -1, 0), (1, 0, 0), (0, 0, 1))}


def sphere_cell_centres(leaves: np.ndarray, mx: int) -> np.ndarray:
    """Unit-sphere positions (n, mx, mx, 3) of the cell centres of cubed-sphere
    leaves (equiangular gnomonic grid on each face), where the initial field
    is evaluated."""
    leaves = np.asarray(leaves)
    x, y = cell_centres(leaves, mx)
    ta = np.tan((x - 0.5) * np.pi / 2)[..., None]
    tb = np.tan((y - 0.5) * np.pi / 2)[..., None]
    frames = np.array([_CUBE[int(b)] for b in leaves[:, 1]], dtype=np.float64)  # (n, 3, 3)
    P = (frames[:, None, None, 0, :] + ta * frames[:, None, None, 1, :]
         + tb * frames[:, None, None, 2, :])
    return P / np.linalg.norm(P, axis=-1, keepdims=True)


def cell_centres(leaves: np.ndarray, mx: int):
    """Cell-centre coordinates of every interior cell of every leaf.

    ``leaves`` is an (n, >=5) integer array whose columns 2..4 are
    (level, ix, iy) of a quadrant in a unit block.  Returns x, y of shape
    (n, mx, mx) indexed [leaf][j][i].
    """
    leaves = np.asarray(leaves)
    lev = leaves[:, 2].astype(np.float64)
    ix = leaves[:, 3].astype(np.float64)
    iy = leaves[:, 4].astype(np.float64)
    h = 1.0 / (mx * np.exp2(lev))
    i = np.arange(mx, dtype=np.float64) + 0.5
    x = (ix[:, None, None] * mx + i[None, None, :]) * h[:, None, None]
    y = (iy[:, None, None] * mx + i[None, :, None]) * h[:, None, None]
    x = np.broadcast_to(x, (len(leaves), mx, mx))
    y = np.broadcast_to(y, (len(leaves), mx, mx))
    return np.ascontiguousarray(x), np.ascontiguousarray(y)


def time_step(w: Workload, lmax: Optional[int] = None):
    """(number of coarse steps, coarse dt) landing exactly on ``w.t_final``.

    dt_CFL = cfl * h_finest / (largest speed; 1 for the swirl).  A coarse step
    is 2^(lmax - lmin) steps of the finest level.  This is a parameter choice
    shared by both implementations, not part of either.
    """
    L = w.lmax if lmax is None else lmax
    if w.dt_lmin is not None:  # a fixed step of the coarsest level
        n = int(round(w.t_final / w.dt_lmin))
        return n, w.t_final / n
    h_f = 1.0 / (w.mx * 2 ** L)
    if w.velocity[0] == "deform":  # speed <= kappa + 2 pi / |T_f|
        h_f = 0.7 * (np.pi / 2) / (w.mx * 2 ** L)
        smax = abs(w.velocity[1]) + 2.0 * np.pi / abs(w.velocity[3])
    elif w.velocity[0] == "rotation":
        # unit sphere: a block spans pi/2 radians; the smallest equiangular
        # cell side is about 0.7 of the nominal one; speed <= |omega|
        h_f = 0.7 * (np.pi / 2) / (w.mx * 2 ** L)
        smax = float(np.linalg.norm(w.velocity[1:4]))
    elif w.velocity[0] == "const":
        smax = max(abs(w.velocity[1]), abs(w.velocity[2]))
    else:
        smax = 1.0
    dt_cfl = w.cfl * h_f / smax
    ratio = 2 ** (L - w.lmin)
    n = int(np.ceil(w.t_final / (ratio * dt_cfl)))
    return n, w.t_final / n


def random_field(shape, seed: int = 0, lo: float = 0.0, hi: float = 1.0):
    return _rng(seed).uniform(lo, hi, shape)
