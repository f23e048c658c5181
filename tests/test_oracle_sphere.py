"""Pins of the oracle's cubed sphere (Sec. 2.4 multiblock indexing, Sec. 5.3).

Each check compares the oracle with a fact fixed by geometry or by the
mathematics of the method, not with the oracle itself:
  * the capacities of all cells tile the unit sphere: sum = 4 pi;
  * capacities are additive under refinement (cells are bounded by great
    circles, which equiangular grid lines are);
  * the edge volume fluxes of a solid-body rotation are divergence free, so
    a constant state stays constant (capacity form, Sec. 5.3);
  * the index-space fold across cube edges continues cell rows: ghost
    layers filled with the cell-centre coordinates sit one and two cell
    widths beyond the boundary cell, on the far side;
  * the rotation carries a cosine bell to where the rotation matrix puts it
    (direction and angle of the transport);
  * the error after one revolution falls under refinement.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.filterwarnings("ignore")

OMEGA = 2.0 * np.pi * np.array([0.3, -0.5, 0.81]) / np.linalg.norm([0.3, -0.5, 0.81])


def _sphere(level, mx=8, omega=OMEGA, lmax=None):
    prm = oracle.params(oracle.SPHERE, mx, 2, level, level if lmax is None else lmax,
                        ("rotation", *omega))
    return oracle.Forest(prm, oracle.uniform_leaves(level, 1, 6))


def _rotate(v, omega, t):
    """Rodrigues' rotation of v by angle |omega| t about omega."""
    w = np.linalg.norm(omega)
    k = omega / w
    a = w * t
    return v * np.cos(a) + np.cross(k, v) * np.sin(a) + k * np.dot(k, v) * (1 - np.cos(a))


@pytest.mark.parametrize("level", [0, 1, 2])
def test_capacities_tile_the_sphere(level):
    F = _sphere(level)
    kap = F.kappa()
    assert np.all(kap > 0)
    assert abs(kap.sum() - 4 * np.pi) < 1e-12 * 4 * np.pi
    # the six faces are congruent
    per_face = kap.reshape(6, -1).sum(axis=1)
    assert np.allclose(per_face, 4 * np.pi / 6, rtol=1e-13, atol=0)


def test_capacities_tile_an_adaptive_sphere():
    F = oracle.initial_forest(synth.sphere(seed=3, lmin=1, lmax=3, mx=8))
    assert len(np.unique(F.leaves()[:, 2])) >= 2
    assert abs(F.kappa().sum() - 4 * np.pi) < 1e-12 * 4 * np.pi


def _block_array(F, values):
    """Scatter per-leaf interior arrays of a uniform forest into per-block
    global arrays (6, N mx, N mx), indexed [b, global j, global i]."""
    lv = F.leaves()
    mx = F.mx
    n = 1 << int(lv[0, 2])
    out = np.zeros((6, n * mx, n * mx))
    for p, (_, b, _, x, y) in enumerate(lv):
        out[b, y * mx:(y + 1) * mx, x * mx:(x + 1) * mx] = values[p]
    return out


def test_capacities_are_additive_under_refinement():
    coarse = _block_array(_sphere(1), _sphere(1).kappa())
    fine = _block_array(_sphere(2), _sphere(2).kappa())
    summed = fine[:, 0::2, 0::2] + fine[:, 1::2, 0::2] + fine[:, 0::2, 1::2] + fine[:, 1::2, 1::2]
    assert np.allclose(summed, coarse, rtol=1e-11, atol=0)


def test_cell_centres_are_on_the_sphere_and_distinct():
    F = _sphere(1)
    X = F.sphere_centres().reshape(-1, 3)
    assert np.allclose(np.linalg.norm(X, axis=1), 1.0, atol=1e-15)
    # no two cells share a centre (blocks do not overlap)
    key = np.round(X * 1e9).astype(np.int64)
    assert len(np.unique(key, axis=0)) == len(X)


def _fill_with_coordinates(F):
    """Fill ghosts three times with the x, y, z cell-centre coordinates as
    data; return the full arrays stacked as (n, S, S, 3)."""
    X = F.sphere_centres()
    out = []
    for k in range(3):
        F.set_q(X[..., k].copy())
        F.fill_ghosts()
        out.append(F.get_q_full())
    return np.stack(out, axis=-1)


@pytest.mark.parametrize("level", [0, 1])
def test_fold_continues_cell_rows_across_cube_edges(level):
    F = _sphere(level)
    mx, mbc = F.mx, 2
    G = _fill_with_coordinates(F)
    assert np.all(np.isfinite(G))
    worst = 0.0
    for p in range(len(F)):
        # four sides: (ghost index, boundary index, inward index) along the row
        for side in range(4):
            for k in range(mx):
                def at(d):  # d < 0: ghost layer -d; d >= 0: interior, d cells in
                    if side == 0:
                        return G[p, mbc + k, mbc + d]
                    if side == 1:
                        return G[p, mbc + k, mbc + mx - 1 - d]
                    if side == 2:
                        return G[p, mbc + d, mbc + k]
                    return G[p, mbc + mx - 1 - d, mbc + k]
                width = np.linalg.norm(at(0) - at(1))
                for d in (1, 2):
                    g = at(-d)
                    # distance from the boundary cell grows with the layer
                    r = np.linalg.norm(g - at(0)) / width
                    worst = max(worst, abs(r - d) / d)
                    # and the ghost lies on the far side of the boundary cell
                    assert np.dot(g - at(0), at(0) - at(1)) > 0
    assert worst < 0.35, worst


def test_three_valent_corner_ghosts_are_finite_and_bounded():
    F = oracle.initial_forest(synth.sphere(seed=1, lmin=1, lmax=3, mx=8))
    q = F.get_q()
    F.fill_ghosts()
    full = F.get_q_full()
    assert np.all(np.isfinite(full))
    # every ghost value is a convex combination of interior values
    assert full.min() >= q.min() - 1e-12 and full.max() <= q.max() + 1e-12


def test_constant_state_is_preserved_on_an_adaptive_sphere():
    w = synth.sphere(seed=2, lmin=1, lmax=3, mx=8)
    F = oracle.initial_forest(w)
    F.set_q(np.ones((len(F), F.mx, F.mx)))
    n, dt = synth.time_step(w)
    for s in range(3):
        F.step_multirate(s * dt, dt)
    q = F.get_q()
    assert np.abs(q - 1.0).max() < 1e-13


def _bell_run(level, t_end, mx=8):
    c0 = np.array([0.6, 0.48, -0.64])
    c0 = c0 / np.linalg.norm(c0)
    w = synth.Workload(name="bell", domain="sphere", mx=mx, mbc=2, lmin=level, lmax=level,
                       velocity=("rotation", *OMEGA), limiter="mc", transverse=2, cfl=0.9,
                       parts=[synth.CosineBell(c0)], t_final=t_end, regrid_every=0, seed=0)
    F = _sphere(level, mx)
    X = F.sphere_centres()
    F.set_q(synth.evaluate_sphere(w, X))
    n, dt = synth.time_step(w)
    for s in range(n):
        F.step_global(s * dt, dt)
    return F, w, X, c0


def test_rotation_moves_the_bell_where_the_rotation_puts_it():
    F, w, X, c0 = _bell_run(2, 0.25)
    q, kap = F.get_q(), F.kappa()
    m = (kap * q)[..., None] * X
    centroid = m.reshape(-1, 3).sum(axis=0)
    centroid /= np.linalg.norm(centroid)
    expect = _rotate(c0, OMEGA, 0.25)
    angle = np.arccos(np.clip(np.dot(centroid, expect), -1, 1))
    assert angle < 0.01, angle
    # the opposite sense of rotation would be far away
    wrong = _rotate(c0, -OMEGA, 0.25)
    assert np.arccos(np.clip(np.dot(centroid, wrong), -1, 1)) > 0.5


def test_error_after_one_revolution_falls_under_refinement():
    errs, drift = [], []
    for level in (1, 2):
        F, w, X, c0 = _bell_run(level, 1.0)
        exact = synth.evaluate_sphere(w, X)
        kap = F.kappa()
        errs.append((kap * np.abs(F.get_q() - exact)).sum() / (kap * np.abs(exact)).sum())
        drift.append(abs((kap * (F.get_q() - exact)).sum()))
    # about second order in the smooth bell
    assert errs[1] < 0.3 * errs[0], errs
    # the mass defect (ghost metrics from each block's own mapping) is a
    # truncation error and also shrinks
    assert drift[1] < 0.6 * drift[0], drift


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_capacities_match_the_solid_angle_closed_form(level):
    """Every capacity over the extended range (ghost cells: the patch's own
    mapping continued past its block) equals the solid angle of its
    rectangle [X1, X2] x [Y1, Y2] on the face plane at unit distance,
    X = tan((x - 1/2) pi/2): F(X2, Y2) - F(X1, Y2) - F(X2, Y1) + F(X1, Y1)
    with F(X, Y) = arctan(X Y / sqrt(1 + X^2 + Y^2)), evaluated in extended
    precision (the four O(1) terms cancel to the cell's O(h^2) area)."""
    mx, mbc = 8, 2
    S = mx + 2 * mbc
    F = oracle.Forest(oracle.params(oracle.SPHERE, mx, mbc, level, level,
                                    ("rotation", 0.0, 0.0, 1.0)),
                      oracle.uniform_leaves(level, nblocks=6))
    K = F.kappa_full()
    ld = np.longdouble
    for p, (_, _, l, x0, y0) in enumerate(F.leaves()):
        h = 1.0 / (mx * 2 ** int(l))
        e = ((x0 * mx + np.arange(S + 1) - mbc) * h).astype(ld)
        g = ((y0 * mx + np.arange(S + 1) - mbc) * h).astype(ld)
        X = np.tan((e - ld(0.5)) * ld(np.pi) / ld(2))
        Y = np.tan((g - ld(0.5)) * ld(np.pi) / ld(2))
        Fxy = np.arctan(X[None, :] * Y[:, None] / np.sqrt(ld(1) + X[None, :] ** 2 + Y[:, None] ** 2))
        A = (Fxy[1:, 1:] - Fxy[1:, :-1] - Fxy[:-1, 1:] + Fxy[:-1, :-1]).astype(np.float64)
        assert np.abs(K[p] - A).max() <= 5e-14 * A.max()
