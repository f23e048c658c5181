"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, an exact invariant, a textbook special case, a hand-computed table, or a
brute-force property.  None of them retypes the oracle's own formulas.
"""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ helpers

def to_grid(F, q):
    """Assemble a uniform single-tree forest's leaf data into one array."""
    lv = F.leaves()
    mx = F.mx
    n = (1 << int(lv[0, 2])) * mx
    G = np.zeros((n, n))
    for p, (_, _, _, x, y) in enumerate(lv):
        G[y * mx:(y + 1) * mx, x * mx:(x + 1) * mx] = q[p]
    return G


def from_grid(F, G):
    lv = F.leaves()
    mx = F.mx
    return np.stack([G[y * mx:(y + 1) * mx, x * mx:(x + 1) * mx] for (_, _, _, x, y) in lv])


def uniform_forest(domain, level, mx, velocity, order=2, limiter=1, transverse=2):
    prm = oracle.params(domain, mx, 2, level, level, velocity, order=order,
                        limiter=limiter, transverse=transverse)
    return oracle.Forest(prm, oracle.uniform_leaves(level))


def squares(lv):
    """Closed squares of the leaves in units of the finest level."""
    L = int(lv[:, 2].max())
    s = (1 << (L - lv[:, 2])).astype(np.int64)
    x0 = lv[:, 3].astype(np.int64) * s
    y0 = lv[:, 4].astype(np.int64) * s
    return x0, x0 + s, y0, y0 + s, 1 << L


def balanced(lv, periodic):
    """Brute force: every pair of leaves whose closed squares meet differs by <= 1 level."""
    x0, x1, y0, y1, R = squares(lv)
    lev = lv[:, 2]
    shifts = [(a, b) for a in (-1, 0, 1) for b in (-1, 0, 1)] if periodic else [(0, 0)]
    for k in range(len(lv)):
        for sx, sy in shifts:
            touch = ((x0[k] <= x1 + sx * R) & (x0 + sx * R <= x1[k]) &
                     (y0[k] <= y1 + sy * R) & (y0 + sy * R <= y1[k]))
            touch[k] = False if (sx, sy) == (0, 0) else touch[k]
            if np.any(touch & (np.abs(lev - lev[k]) > 1)):
                return False
    return True


def covers_unit_square(lv):
    x0, x1, y0, y1, R = squares(lv)
    area = np.sum((x1 - x0) * (y1 - y0))
    return area == R * R


# ------------------------------------------------------------------ limiter tables

def test_limiter_tables_match_hand_values():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "limiters.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) >= 15
    for kind, a, b, want in rows:
        if kind == "mc":
            got = oracle.mc_phi(float(a))
        else:
            got = oracle.minmod(float(a), float(b))
        assert got == float(want), (kind, a, b, got, want)


# ------------------------------------------------------------------ scheme special cases

def test_first_order_ctu_closed_form():
    """Order 1 + transverse fluctuations = Colella's corner-transport upwind
    scheme, whose one-step stencil for u, v > 0 is
    Q - nu u (Q - Q_{i-1}) - nu v (Q - Q_{j-1})
      + nu^2 u v (Q - Q_{i-1} - Q_{j-1} + Q_{i-1,j-1})   (FVMHP Sec. 20.3)."""
    N = 32
    q = synth.random_field((N, N), seed=3)
    for (u, v) in [(0.7, 0.4), (-0.6, -0.9)]:
        prm = oracle.params(oracle.PERIODIC, N, 2, 0, 0, ("const", u, v), order=1,
                            limiter=0, transverse=1)
        h = 1.0 / N
        dt = 0.8 * h
        got = oracle.single_grid_periodic(prm, q, 0.0, dt, 1)
        nu = dt / h
        sx = -1 if u > 0 else 1  # upwind neighbour offset
        sy = -1 if v > 0 else 1
        Qi = np.roll(q, -sx, axis=1)   # Q at i + sx
        Qj = np.roll(q, -sy, axis=0)
        Qij = np.roll(Qi, -sy, axis=0)
        au, av = abs(u), abs(v)
        want = (q - nu * au * (q - Qi) - nu * av * (q - Qj)
                + nu * nu * au * av * (q - Qi - Qj + Qij))
        assert np.max(np.abs(got - want)) < 1e-14


def test_lax_wendroff_1d_closed_form():
    """Unlimited second order with v = 0 is the Lax-Wendroff scheme
    Q - nu u/2 (Q_{i+1} - Q_{i-1}) + (nu u)^2/2 (Q_{i+1} - 2Q + Q_{i-1})."""
    N = 32
    q = synth.random_field((N, N), seed=4)
    for u in (0.8, -0.55):
        prm = oracle.params(oracle.PERIODIC, N, 2, 0, 0, ("const", u, 0.0), order=2,
                            limiter=0, transverse=2)
        h = 1.0 / N
        dt = 0.9 * h
        got = oracle.single_grid_periodic(prm, q, 0.0, dt, 1)
        c = u * dt / h
        qp, qm = np.roll(q, -1, axis=1), np.roll(q, 1, axis=1)
        want = q - 0.5 * c * (qp - qm) + 0.5 * c * c * (qp - 2 * q + qm)
        assert np.max(np.abs(got - want)) < 1e-14


def test_mc_limited_1d_is_tvd_and_bounded():
    """The MC-limited 1D scheme is total-variation diminishing (Harten), so it
    creates no new extrema and its TV never grows."""
    N = 64
    q = synth.random_field((N, N), seed=5)
    prm = oracle.params(oracle.PERIODIC, N, 2, 0, 0, ("const", 0.0, 0.75), order=2,
                        limiter=1, transverse=2)
    h = 1.0 / N
    dt = 0.95 * h / 0.75
    cur = q.copy()
    tv = np.sum(np.abs(np.diff(cur, axis=0, append=cur[:1])), axis=0)
    for _ in range(30):
        cur = oracle.single_grid_periodic(prm, cur, 0.0, dt, 1)
        tv2 = np.sum(np.abs(np.diff(cur, axis=0, append=cur[:1])), axis=0)
        assert np.all(tv2 <= tv + 1e-12)
        tv = tv2
    assert cur.min() >= q.min() - 1e-14 and cur.max() <= q.max() + 1e-14


def test_exact_diagonal_shift_and_return():
    """(u, v) = (1, 1) at Courant number 1: every correction vanishes and the
    corner-transport scheme moves data by exactly one cell diagonally, so
    after N steps the periodic field returns bit for bit (Sec. 8 pin)."""
    mx, level = 16, 3
    F = uniform_forest(oracle.PERIODIC, level, mx, ("const", 1.0, 1.0))
    w = synth.uniform_periodic(1)
    x, y = synth.cell_centres(F.leaves(), mx)
    q0 = (synth.evaluate(w, x, y) > 0.9).astype(np.float64)  # {0,1} data
    F.set_q(q0)
    N = mx << level
    dt = 1.0 / N
    F.step_global(0.0, dt)
    G0, G1 = to_grid(F, q0), to_grid(F, F.get_q())
    assert np.array_equal(G1, np.roll(np.roll(G0, 1, axis=0), 1, axis=1))
    for n in range(1, N):
        F.step_global(n * dt, dt)
    assert np.array_equal(F.get_q(), q0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_uniform_forest_equals_single_grid_bitwise(seed):
    """64 patches of 16^2 with same-level copies = one 128^2 periodic grid."""
    w = synth.uniform_periodic(seed)
    F = oracle.initial_forest(w)
    assert len(F) == 64
    q0 = F.get_q()
    h = 1.0 / 128
    dt = w.cfl * h / 1.0
    for n in range(w.steps):
        F.step_global(n * dt, dt)
    G = oracle.single_grid_periodic(oracle.params_for(w), to_grid(F, q0), 0.0, dt, w.steps)
    assert np.array_equal(to_grid(F, F.get_q()), G)


# ------------------------------------------------------------------ invariants

def test_mass_conserved_uniform_periodic():
    w = synth.uniform_periodic(0)
    F = oracle.initial_forest(w)
    m0 = F.mass()[0]
    dt = w.cfl / 128
    for n in range(w.steps):
        F.step_global(n * dt, dt)
    assert abs(F.mass()[0] - m0) <= 1e-13 * abs(m0)


def test_mass_conserved_walls_swirl_single_level():
    """Swirl normal velocity vanishes on the walls; flux form conserves."""
    w = synth.swirl(0, lmin=3, lmax=3, mx=16)
    F = oracle.initial_forest(w)
    m0 = F.mass()[0]
    dt = 0.9 / 128
    for n in range(40):
        F.step_global(n * dt, dt)
    assert abs(F.mass()[0] - m0) <= 1e-13 * abs(m0)


@pytest.mark.parametrize("velocity", [("const", 0.8, -0.3), ("swirl", 4.0)])
@pytest.mark.parametrize("mode", ["global", "multirate"])
def test_constant_state_preserved(velocity, mode):
    w = synth.swirl(2, lmin=2, lmax=4, mx=8)
    F = oracle.initial_forest(w)
    lv = F.leaves()
    assert len(set(lv[:, 2])) == 3  # an adaptive layout
    prm = oracle.params(oracle.WALLS, 8, 2, 2, 4, velocity)
    G = oracle.Forest(prm, lv)
    c = 0.7
    G.set_q(np.full((len(lv), 8, 8), c))
    dtc = 0.9 / (8 * 16) * 4
    for n in range(3):
        if mode == "global":
            for k in range(4):
                G.step_global((4 * n + k) * dtc / 4, dtc / 4)
        else:
            G.step_multirate(n * dtc, dtc)
    err = np.max(np.abs(G.get_q() - c))
    if velocity[0] == "const":
        assert err == 0.0
    else:
        assert err <= 1e-14


# ------------------------------------------------------------------ ghost fill

def adaptive_walls_forest(seed=2, lmin=2, lmax=4, mx=8):
    w = synth.swirl(seed, lmin=lmin, lmax=lmax, mx=mx)
    F = oracle.initial_forest(w)
    return w, F


def test_initial_layout_is_balanced_and_covers():
    for seed in range(4):
        _, F = adaptive_walls_forest(seed, 2, 5, 8)
        lv = F.leaves()
        assert covers_unit_square(lv)
        assert balanced(lv, periodic=False)
        assert lv[:, 2].max() == 5


def test_ghost_fill_reproduces_linear_data():
    """Copy, average (Eq. ghost_coarse) and interpolation (Eq. ghost_fine) are
    exact on linear data: the four fine centres average to the coarse centre,
    and minmod slopes of a linear field are its exact differences.  Dyadic
    coefficients keep every operation exact in FP64."""
    _, F = adaptive_walls_forest(1, 2, 5, 8)
    lv = F.leaves()
    mx, mbc, S = 8, 2, 12
    a, b, c = 0.5, 0.375, -0.25

    def lin(x, y):
        return a + b * x + c * y

    x, y = synth.cell_centres(lv, mx)
    F.set_q(lin(x, y))
    F.fill_ghosts()
    Q = F.get_q_full()
    checked = 0
    idx = np.arange(-mbc, mx + mbc)
    for p, (_, _, l, ix, iy) in enumerate(lv):
        h = 1.0 / (mx * 2 ** l)
        xc = (ix * mx + idx + 0.5) * h
        yc = (iy * mx + idx + 0.5) * h
        for jj in range(S):
            for ii in range(S):
                if mbc <= ii < mx + mbc and mbc <= jj < mx + mbc:
                    continue
                X, Y = xc[ii], yc[jj]
                if min(X, Y, 1 - X, 1 - Y) <= 4 * h:  # stencils near walls use BC data
                    continue
                assert Q[p, jj, ii] == lin(X, Y), (p, ii, jj)
                checked += 1
    assert checked > 1000


def test_ghost_fill_leaves_no_invalid_value():
    """Executable Proposition 1: with all ghosts poisoned (NaN) before the
    fill, Alg. 1 on a 2:1 balanced layout with mbc <= mx/4 leaves none."""
    for seed in range(3):
        _, F = adaptive_walls_forest(seed, 2, 5, 8)
        F.set_q(synth.random_field((len(F), 8, 8), seed=seed))
        F.fill_ghosts()
        assert np.all(np.isfinite(F.get_q_full()))


def test_ghost_fill_exterior_is_extrapolation():
    """Walls: exterior ghosts equal the nearest cell of the owner, including
    the exterior corner of a patch in a domain corner."""
    F = uniform_forest(oracle.WALLS, 1, 8, ("const", 0.5, 0.5))
    F.set_q(synth.random_field((4, 8, 8), seed=9))
    F.fill_ghosts()
    Q = F.get_q_full()
    lv = F.leaves()
    p = [k for k in range(4) if lv[k, 3] == 0 and lv[k, 4] == 0][0]
    assert np.all(Q[p, :2, :2] == Q[p, 2, 2])        # corner block = cell (0,0)
    assert np.all(Q[p, 2:10, 0] == Q[p, 2:10, 2])   # left wall rows
    assert np.all(Q[p, 0, 2:10] == Q[p, 2, 2:10])   # bottom wall columns


def test_multirate_run_stays_finite_and_bounded():
    """Multirate substeps with time interpolation: no NaN canary reaches a
    solution value; a {0,1} disc stays within small over/undershoots."""
    w, F = adaptive_walls_forest(3, 2, 4, 8)
    n, dtc = synth.time_step(w, 4)
    for k in range(6):
        F.step_multirate(k * dtc, dtc)
    q = F.get_q()
    assert np.all(np.isfinite(q))
    assert q.min() > -0.2 and q.max() < 1.2


# ------------------------------------------------------------------ regrid

def test_refine_then_coarsen_is_identity_and_conservative():
    """Interpolation followed by averaging returns the coarse data exactly
    (the four d_k sum to zero) and both steps conserve mass."""
    prm = oracle.params(oracle.WALLS, 8, 2, 1, 2, ("const", 1.0, 0.0))
    F = oracle.Forest(prm, oracle.uniform_leaves(1))
    q0 = np.round(synth.random_field((4, 8, 8), seed=11) * 64) / 64  # dyadic data
    F.set_q(q0)
    m0 = F.mass()[0]
    F.regrid(-1.0, -1.0)  # refine every leaf
    assert len(F) == 16 and set(F.leaves()[:, 2]) == {2}
    assert abs(F.mass()[0] - m0) <= 1e-15
    F.regrid(np.inf, np.inf)  # coarsen every family
    assert len(F) == 4
    assert np.array_equal(F.get_q(), q0)


def test_regrid_balances_deep_corner_refinement():
    """Refining only the corner leaf repeatedly forces a graded layout."""
    prm = oracle.params(oracle.WALLS, 8, 2, 0, 5, ("const", 1.0, 0.0))
    F = oracle.Forest(prm, oracle.uniform_leaves(0))
    for _ in range(5):
        lv = F.leaves()
        x, y = synth.cell_centres(lv, 8)
        # a single nonzero cell, the one at the origin corner
        F.set_q(np.where((x == x.min()) & (y == y.min()), 1.0, 0.0))
        F.regrid(0.05, 0.0125)
    lv = F.leaves()
    assert lv[:, 2].max() == 5
    assert covers_unit_square(lv)
    assert balanced(lv, periodic=False)


def test_regrid_follows_tags():
    """Leaves whose indicator exceeds tau_r are refined; quiet families coarsen."""
    w, F = adaptive_walls_forest(0, 2, 4, 8)
    F.set_q(np.zeros((len(F), 8, 8)))
    # a zero field: every complete family coarsens, one level per regrid
    for _ in range(2):
        F.regrid(0.05, 0.0125)
        assert balanced(F.leaves(), periodic=False)
    assert set(F.leaves()[:, 2]) == {2}
    # one hot cell: its leaf is refined (and the layout stays balanced)
    lv = F.leaves()
    x, y = synth.cell_centres(lv, 8)
    hot = (np.abs(x - 0.53) < 0.03) & (np.abs(y - 0.47) < 0.03)
    F.set_q(hot.astype(np.float64))
    tagged = lv[np.any(hot, axis=(1, 2))]
    F.regrid(0.05, 0.0125)
    new = F.leaves()
    for (f, b, l, ix, iy) in tagged:
        kids = [(f, b, l + 1, 2 * ix + cx, 2 * iy + cy) for cx in (0, 1) for cy in (0, 1)]
        assert all(any((new == k).all(axis=1)) for k in map(np.array, kids))
    assert balanced(new, periodic=False)


# ------------------------------------------------------------------ convergence

def _smooth_error(level, limiter):
    w = synth.smooth_periodic(0, level=level, mx=16, limiter=limiter)
    F = oracle.initial_forest(w)
    N = 16 << level
    T = 0.25
    nsteps = int(np.ceil(T / (0.9 / N)))
    dt = T / nsteps
    for n in range(nsteps):
        F.step_global(n * dt, dt)
    x, y = synth.cell_centres(F.leaves(), 16)
    exact = synth.evaluate(w, x - 1.0 * T, y - 0.5 * T)
    return np.mean(np.abs(F.get_q() - exact))


@pytest.mark.parametrize("limiter,order_min", [("none", 1.9), ("mc", 1.6)])
def test_second_order_convergence(limiter, order_min):
    e = [_smooth_error(l, limiter) for l in (2, 3, 4)]
    orders = [np.log2(e[k] / e[k + 1]) for k in range(2)]
    assert min(orders) >= order_min, (e, orders)
