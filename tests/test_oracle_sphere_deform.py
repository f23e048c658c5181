"""Pins of the oracle's deformational flow on the cubed sphere (the
streamfunction of Sec. 5.3, time dependent; edge volume fluxes = differences
of psi between edge end points), against facts fixed independently of it:
  * each edge flux approximates, to second order in the cell size, the arc
    length times the normal component of the published velocity of this
    flow, written from its components (u = kappa sin^2(rho') sin(2 theta)
    cos(pi t/T) + 2 pi cos(theta)/T_f, v = kappa sin(2 rho') cos(theta)
    cos(pi t/T), rho' = rho - 2 pi t/T) on a cube mapping built here with
    numpy;
  * at t = T/2 the deformation vanishes: the fluxes are those of the
    solid-body rotation about the z axis with |omega| = 2 pi/T_f;
  * psi differences cancel around every cell: a constant state stays
    constant on an adaptive forest, global and multirate;
  * with T_f = T the background rotation carries the pattern back: a smooth
    tracer returns to its start at t = T, closer on the finer grid; with the
    rotation reversed it does not.
"""
import numpy as np
import pytest

import oracle
import synth
from synth import _CUBE

K, T, TF = 2.0, 0.5, 5.0
MX, MBC = 8, 2


def _forest(level, velocity=("deform", K, T, TF), lmax=None):
    prm = oracle.params(oracle.SPHERE, MX, MBC, level, level if lmax is None else lmax, velocity)
    return oracle.Forest(prm, oracle.uniform_leaves(level, nblocks=6))


def _corners(leaves):
    """Unit-sphere corner points (n, S+1, S+1, 3) [j][i] over the extended range."""
    S = MX + 2 * MBC
    out = []
    for _, b, l, x0, y0 in leaves:
        h = 1.0 / (MX * 2 ** int(l))
        k = np.arange(S + 1) - MBC
        X, Y = np.meshgrid((x0 * MX + k) * h, (y0 * MX + k) * h)
        fr = np.array(_CUBE[int(b)], dtype=np.float64)
        P = (fr[0] + np.tan((X - 0.5) * np.pi / 2)[..., None] * fr[1]
             + np.tan((Y - 0.5) * np.pi / 2)[..., None] * fr[2])
        out.append(P / np.linalg.norm(P, axis=-1, keepdims=True))
    return np.array(out)


def _velocity(X, t, tf=TF):
    lam = np.arctan2(X[..., 1], X[..., 0])
    th = np.arcsin(np.clip(X[..., 2], -1.0, 1.0))
    lp = lam - 2.0 * np.pi * t / T
    c = np.cos(np.pi * t / T)
    u = K * np.sin(lp) ** 2 * np.sin(2 * th) * c + 2.0 * np.pi * np.cos(th) / tf
    v = K * np.sin(2 * lp) * np.cos(th) * c
    e_lam = np.stack([-np.sin(lam), np.cos(lam), 0.0 * lam], -1)
    e_th = np.stack([-np.sin(th) * np.cos(lam), -np.sin(th) * np.sin(lam), np.cos(th)], -1)
    return u[..., None] * e_lam + v[..., None] * e_th


def _edge_estimate(A, B, C, t):
    """arc length x normal velocity at the midpoint of the arc A-B, the normal
    pointing to the side of C"""
    M = A + B
    M /= np.linalg.norm(M, axis=-1, keepdims=True)
    d = B - A
    ell = 2.0 * np.arcsin(np.linalg.norm(d, axis=-1) / 2.0)
    n = np.cross(d / np.linalg.norm(d, axis=-1, keepdims=True), M)
    n *= np.sign(np.sum(n * (C - A), -1))[..., None]
    return ell * np.sum(_velocity(M, t) * n, -1)


def _flux_errors(level, t, ghosts=False):
    F = _forest(level)
    px, py = F.edge_fluxes(t)
    N = _corners(F.leaves())
    # interior edges, or every edge of the extended range but the outermost
    # (whose neighbouring corner for the normal's side lies outside)
    a, b = (0, MX + 2 * MBC - 1) if ghosts else (MBC, MBC + MX)
    # x-edge (i, j) runs from corner (i, j) to (i, j+1); positive flux toward +x
    wx = _edge_estimate(N[:, a:b, a:b + 1], N[:, a + 1:b + 1, a:b + 1], N[:, a:b, a + 1:b + 2], t)
    # y-edge (i, j) runs from corner (i, j) to (i+1, j); positive flux toward +y
    wy = _edge_estimate(N[:, a:b + 1, a:b], N[:, a:b + 1, a + 1:b + 1], N[:, a + 1:b + 2, a:b], t)
    ex = np.abs(px[:, a:b, a:b + 1] - wx).max() / np.abs(wx).max()
    ey = np.abs(py[:, a:b + 1, a:b] - wy).max() / np.abs(wy).max()
    return max(ex, ey)


@pytest.mark.parametrize("t", [0.0, 0.13, 0.41])
@pytest.mark.parametrize("ghosts", [False, True])
def test_edge_fluxes_follow_the_published_velocity(t, ghosts):
    """(with ghosts: the edges of the ghost cells too, the patch's own mapping
    extended past its block)"""
    e2, e3 = _flux_errors(2, t, ghosts), _flux_errors(3, t, ghosts)
    assert e2 < 1e-3
    assert e3 < 0.3 * e2  # second order: about 1/4


def test_half_period_is_the_solid_body_rotation():
    d = _forest(2)
    r = _forest(2, velocity=("rotation", 0.0, 0.0, 2.0 * np.pi / TF))
    pd, qd = d.edge_fluxes(0.5 * T)
    pr, qr = r.edge_fluxes(0.0)
    scale = max(np.abs(pr).max(), np.abs(qr).max())
    assert np.abs(pd - pr).max() < 1e-13 * scale
    assert np.abs(qd - qr).max() < 1e-13 * scale


@pytest.mark.parametrize("mode", ["global", "multirate"])
def test_constant_state_on_an_adaptive_forest(mode):
    w = synth.sphere_deform(seed=1, lmin=1, lmax=3, mx=8)
    F = oracle.initial_forest(w)
    assert len(np.unique(F.leaves()[:, 2])) > 1
    F.set_q(np.ones((len(F), MX, MX)))
    dtc = 4 * w.dt_lmin
    for n in range(2):
        if mode == "global":
            for s in range(4):
                F.step_global(n * dtc + s * dtc / 4, dtc / 4)
        else:
            F.step_multirate(n * dtc, dtc)
    assert np.abs(F.get_q() - 1.0).max() < 1e-12


def _bells(X):
    q = np.full(X.shape[:-1], 0.1)
    for lon in (5.0 * np.pi / 6.0, 7.0 * np.pi / 6.0):
        c = np.array([np.cos(lon), np.sin(lon), 0.0])
        r = np.arccos(np.clip(X @ c, -1.0, 1.0))
        q = q + np.where(r < 0.5, 0.45 * (1.0 + np.cos(np.pi * r / 0.5)), 0.0)
    return q


def _return_error(level, tf_sign):
    period = 5.0  # T = T_f: the background rotation brings the pattern back
    F = _forest(level, velocity=("deform", K, period, tf_sign * period))
    q0 = _bells(F.sphere_centres())
    F.set_q(q0)
    h = 0.7 * (np.pi / 2) / (MX * 2 ** level)
    n = int(np.ceil(period / (0.8 * h / (K + 2.0 * np.pi / period))))
    for s in range(n):
        F.step_global(s * period / n, period / n)
    kap = F.kappa()
    return np.sum(kap * np.abs(F.get_q() - q0)) / np.sum(kap * np.abs(q0))


def test_tracer_returns_after_one_period():
    e2, e3 = _return_error(2, 1.0), _return_error(3, 1.0)
    wrong = _return_error(2, -1.0)
    assert e3 < 0.6 * e2
    assert wrong > 1.5 * e2


def test_uniform_run_matches_the_papers_advance_count():
    """Tab. sphere_details, uniform level 2 on the six blocks: 19200 patch
    advances (16 patches per block, steps of 2.5e-3 to t = 0.5)."""
    w = synth.sphere_deform(lmin=2, lmax=2, mx=32)
    n, dtc = synth.time_step(w)
    assert len(oracle.uniform_leaves(2, nblocks=6)) * n == 19200
    assert dtc == pytest.approx(2.5e-3, rel=1e-15)
