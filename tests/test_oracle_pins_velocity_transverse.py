"""Pins of three oracle pieces that the other pins cannot see.

- The swirl's edge speeds (Sec. 5.1: the velocity comes from a
  streamfunction): compared with the analytic velocity
  u = sin^2(pi x) sin(2 pi y) cos(pi t/T), v = -sin^2(pi y) sin(2 pi x) cos(pi t/T)
  at the edge midpoints, where the corner difference of psi is a centred
  difference (error O(h^2)); the discrete divergence of every cell vanishes.
- The transverse propagation of correction waves (the published unsplit
  wave-propagation method the paper runs through Clawpack, Sec. 5): the
  one-step impulse response of the unlimited scheme at dyadic Courant
  numbers, derived by hand in tests/golden/ctu_impulse_response.txt,
  compared exactly.  A flipped sign or factor in the corrections' transverse
  terms changes a third-order term that no smooth-data or linear-data pin
  sees; the impulse response shows it in its corner coefficients.
- The undivided gradient indicator of Sec. 3.1's tagging: on linear and
  quadratic data with dyadic coefficients it takes exact closed-form values.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ swirl edge speeds

def _swirl_speeds(N, t, T=4.0):
    prm = oracle.params(oracle.WALLS, N, 2, 0, 0, ("swirl", T))
    return oracle.edge_speeds(prm, 1.0 / N, t, N)


def _analytic(N, t, T=4.0):
    """Analytic velocity at the edge midpoints: x-edges (I h, (J + 1/2) h),
    y-edges ((I + 1/2) h, J h)."""
    h = 1.0 / N
    ct = np.cos(np.pi * t / T)
    I = np.arange(N + 1)[None, :] * h
    Jc = (np.arange(N)[:, None] + 0.5) * h
    u = np.sin(np.pi * I) ** 2 * np.sin(2 * np.pi * Jc) * ct
    Ic = (np.arange(N)[None, :] + 0.5) * h
    J = np.arange(N + 1)[:, None] * h
    v = -np.sin(np.pi * J) ** 2 * np.sin(2 * np.pi * Ic) * ct
    return u, v


@pytest.mark.parametrize("t", [0.0, 1.0, 3.0])
def test_swirl_edge_speeds_converge_to_analytic_velocity(t):
    errs = []
    for N in (16, 32, 64, 128):
        u, v = _swirl_speeds(N, t)
        ua, va = _analytic(N, t)
        errs.append(max(np.max(np.abs(u - ua)), np.max(np.abs(v - va))))
        # the leading error is relative O(h^2): already small at N = 16
        assert errs[-1] < 0.05
    ratios = [errs[k] / errs[k + 1] for k in range(3)]
    assert all(3.6 < r < 4.4 for r in ratios), (errs, ratios)


def test_swirl_edge_speeds_vanish_at_half_period_and_reverse():
    N = 32
    u1, v1 = _swirl_speeds(N, 1.0)   # t = T/4
    u2, v2 = _swirl_speeds(N, 2.0)   # t = T/2: cos(pi/2) = 0
    u3, v3 = _swirl_speeds(N, 3.0)   # t = 3T/4: the reversed flow
    assert np.max(np.abs(u2)) < 1e-15 and np.max(np.abs(v2)) < 1e-15
    scale = np.max(np.abs(u1))
    assert scale > 0.5
    assert np.max(np.abs(u3 + u1)) < 1e-15 * 8 and np.max(np.abs(v3 + v1)) < 1e-15 * 8
    # the sense of rotation at t = 0, from v = -sin^2(pi y) sin(2 pi x):
    # downward near x = 1/4, y = 1/2 and upward near x = 3/4
    u0, v0 = _swirl_speeds(N, 0.0)
    mid = N // 2
    assert v0[mid, N // 4] < -0.9 and v0[mid, 3 * N // 4] > 0.9


def test_swirl_edge_speeds_are_discretely_divergence_free_with_closed_walls():
    for N in (16, 64):
        for t in (0.0, 0.7, 2.9):
            u, v = _swirl_speeds(N, t)
            div = (u[:, 1:] - u[:, :-1]) + (v[1:, :] - v[:-1, :])
            assert np.max(np.abs(div)) < 1e-14, (N, t)
            # no normal velocity through the walls
            assert np.max(np.abs(u[:, [0, N]])) < 1e-30
            assert np.max(np.abs(v[[0, N], :])) < 1e-30


# ------------------------------------------------------------------ transverse propagation

def _impulse_tables():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "ctu_impulse_response.txt"))
            if l.strip() and not l.startswith("#")]
    tables = {}
    for r in rows:
        tr, an, ad, bn, bd, dx, dy, vn, vd = map(int, r)
        key = (tr, Fraction(an, ad), Fraction(bn, bd))
        tables.setdefault(key, {})[(dx, dy)] = Fraction(vn, vd)
    return tables


def test_impulse_tables_are_consistent():
    """The stored tables themselves: unit sum and the second-order moments."""
    for (tr, a, b), tab in _impulse_tables().items():
        assert sum(tab.values()) == 1
        # the response moves the unit mass by (a, b): first moments of the
        # response are +a, +b
        assert sum(dx * c for (dx, dy), c in tab.items()) == a
        assert sum(dy * c for (dx, dy), c in tab.items()) == b
        if tr > 0:
            assert sum(dx * dx * c for (dx, dy), c in tab.items()) == a * a
            assert sum(dy * dy * c for (dx, dy), c in tab.items()) == b * b
            assert sum(dx * dy * c for (dx, dy), c in tab.items()) == a * b


@pytest.mark.parametrize("key", sorted(_impulse_tables().keys()))
def test_unlimited_impulse_response_matches_hand_derivation(key):
    tr, a, b = key
    want = _impulse_tables()[key]
    N = 16
    h = 1.0 / N
    dt = h / 2  # nu = 1/2: u = 2a, v = 2b
    u, v = float(2 * a), float(2 * b)
    prm = oracle.params(oracle.PERIODIC, N, 2, 0, 0, ("const", u, v), order=2, limiter=0,
                        transverse=tr)
    i0, j0 = 7, 9
    q = np.zeros((N, N))
    q[j0, i0] = 1.0
    got = oracle.single_grid_periodic(prm, q, 0.0, dt, 1)
    expect = np.zeros((N, N))
    for (dx, dy), c in want.items():
        expect[j0 + dy, i0 + dx] = float(c)
    # dyadic data and coefficients: the oracle's sums are exact
    assert np.array_equal(got, expect), np.argwhere(got != expect)


# ------------------------------------------------------------------ gradient indicator

def _uniform_walls(level, mx):
    prm = oracle.params(oracle.WALLS, mx, 2, level, level + 1, ("const", 1.0, 0.0))
    return oracle.Forest(prm, oracle.uniform_leaves(level))


def _centres(F, mx):
    lv = F.leaves()
    h = 1.0 / (mx << lv[:, 2])
    i = np.arange(mx)
    x = (lv[:, 3, None] * mx + i[None, :] + 0.5) * h[:, None]
    y = (lv[:, 4, None] * mx + i[None, :] + 0.5) * h[:, None]
    return np.broadcast_to(x[:, None, :], (len(lv), mx, mx)), \
        np.broadcast_to(y[:, :, None], (len(lv), mx, mx)), h


def test_gradient_indicator_on_linear_data_is_h_times_gradient_norm():
    """q = k (3 x + 4 y): half the centred difference vector has length 5 k h
    in every interior cell (ghosts copied from neighbours or extrapolated at
    walls only lower it), so each leaf's indicator is exactly 5 k h."""
    mx = 8
    for level in (1, 2, 3):
        F = _uniform_walls(level, mx)
        x, y, h = _centres(F, mx)
        k = 0.125
        F.set_q(k * (3 * x + 4 * y))
        d = F.tag()
        assert np.array_equal(d, 5 * k * h), (level, d[:4], 5 * k * h[:4])


def test_gradient_indicator_on_quadratic_data_is_the_leaf_maximum():
    """q = c x^2: half the centred x-difference is 2 c x h at a cell centre x,
    so a leaf away from the right wall takes the value at its last column's
    centre (its neighbour supplies the ghost), x = x0 + (mx - 1/2) h."""
    mx, level, c = 8, 2, 0.75
    F = _uniform_walls(level, mx)
    x, y, h = _centres(F, mx)
    F.set_q(c * x * x)
    d = F.tag()
    lv = F.leaves()
    inner = lv[:, 3] < (1 << level) - 1
    xlast = (lv[:, 3] * mx + mx - 0.5) * h
    assert np.array_equal(d[inner], (2 * c * xlast * h)[inner])
    # at the right wall the extrapolated ghost lowers the last column: the
    # maximum moves one column in
    xprev = (lv[:, 3] * mx + mx - 1.5) * h
    right = ~inner
    assert np.array_equal(d[right], (2 * c * xprev * h)[right])
