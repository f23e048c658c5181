"""Pins of the oracle's adjoint against its (separately pinned) forward map.

* The unlimited scheme on a uniform periodic forest is linear, so the step
  map applied to v IS its Jacobian times v: <S v, w> = <v, S^T w> exactly.
* On an adaptive walled forest with the MC limiter the map is piecewise
  linear; on smooth data a central difference with a small step stays on one
  linear piece and must agree with the adjoint's directional derivative.
"""
import numpy as np

import oracle
import synth


def test_adjoint_dot_product_linear_uniform():
    for velocity in (("swirl", 4.0), ("const", 0.7, -0.45)):
        prm = oracle.params(oracle.PERIODIC, 8, 2, 2, 2, velocity, order=2, limiter=0,
                            transverse=2)
        F = oracle.Forest(prm, oracle.uniform_leaves(2))
        n = len(F)
        v = synth.random_field((n, 8, 8), seed=1) - 0.5
        w = synth.random_field((n, 8, 8), seed=2) - 0.5
        dt = 0.9 / 32
        F.set_q(v)
        F.step_global(0.1, dt)
        Jv = F.get_q()
        F.set_q(np.zeros((n, 8, 8)))
        lam, _ = F.adjoint_step_global(0.1, dt, w)
        a, b = np.sum(Jv * w), np.sum(v * lam)
        assert abs(a - b) <= 1e-13 * abs(a)


def _smooth_adaptive(nsteps=4):
    w = synth.swirl(3, lmin=2, lmax=4, mx=8)
    F = oracle.initial_forest(w)
    x, y = synth.cell_centres(F.leaves(), 8)
    q0 = synth.evaluate(synth.smooth_periodic(1), x, y) + 0.3 * np.sin(3 * x + 1) * np.cos(2 * y)
    qt = synth.evaluate(synth.smooth_periodic(2), x, y)
    F.set_q(q0)
    return F, q0, qt, 0.9 / 128, nsteps


def _loss(F, q, qt, dt, nsteps, scale=1.0):
    F.set_q(q)
    F.set_velocity_scale(scale)
    for k in range(nsteps):
        F.step_global(k * dt, dt)
    r = 0.5 * np.sum((F.get_q() - qt) ** 2)
    F.set_velocity_scale(1.0)
    return r


def test_adjoint_matches_central_differences_adaptive_mc():
    F, q0, qt, dt, n = _smooth_adaptive()
    loss, g, gs = F.adjoint_global(n, 0.0, dt, qt)
    assert abs(loss - _loss(F, q0, qt, dt, n)) <= 1e-14 * loss
    for seed in (5, 6):
        d = synth.random_field(q0.shape, seed=seed) - 0.5
        eps = 1e-7
        fd = (_loss(F, q0 + eps * d, qt, dt, n) - _loss(F, q0 - eps * d, qt, dt, n)) / (2 * eps)
        assert abs(fd - np.sum(g * d)) <= 1e-6 * abs(fd)
    eps = 1e-6
    fds = (_loss(F, q0, qt, dt, n, 1 + eps) - _loss(F, q0, qt, dt, n, 1 - eps)) / (2 * eps)
    assert abs(fds - gs) <= 1e-6 * abs(fds)


def _loss_mr(F, q, qt, dtc, ncoarse, scale=1.0):
    F.set_q(q)
    F.set_velocity_scale(scale)
    for k in range(ncoarse):
        F.step_multirate(k * dtc, dtc)
    r = 0.5 * np.sum((F.get_q() - qt) ** 2)
    F.set_velocity_scale(1.0)
    return r


def test_multirate_adjoint_matches_central_differences():
    """Multirate (coarse-first recursion with time-interpolated coarse
    ghosts) on an adaptive MC forest of three levels: the adjoint's
    directional derivatives match central differences."""
    F, q0, qt, _, _ = _smooth_adaptive()
    assert len(set(F.leaves()[:, 2])) == 3
    dtc = 4 * 0.9 / 128  # ratio 4 between levels 2 and 4
    n = 2
    loss, g, gs = F.adjoint_multirate(n, 0.0, dtc, qt)
    assert abs(loss - _loss_mr(F, q0, qt, dtc, n)) <= 1e-14 * loss
    for seed in (7, 8):
        d = synth.random_field(q0.shape, seed=seed) - 0.5
        eps = 1e-7
        fd = (_loss_mr(F, q0 + eps * d, qt, dtc, n) - _loss_mr(F, q0 - eps * d, qt, dtc, n)) / (
            2 * eps)
        assert abs(fd - np.sum(g * d)) <= 1e-6 * abs(fd), (fd, np.sum(g * d))
    eps = 1e-6
    fds = (_loss_mr(F, q0, qt, dtc, n, 1 + eps) - _loss_mr(F, q0, qt, dtc, n, 1 - eps)) / (2 * eps)
    assert abs(fds - gs) <= 1e-6 * abs(fds), (fds, gs)


def test_multirate_adjoint_single_level_is_the_global_adjoint():
    """With one level a coarse multirate step is one global step."""
    prm = oracle.params(oracle.WALLS, 8, 2, 3, 3, ("swirl", 4.0))
    F = oracle.Forest(prm, oracle.uniform_leaves(3))
    q = synth.random_field((len(F), 8, 8), seed=3)
    lam = synth.random_field((len(F), 8, 8), seed=4) - 0.5
    F.set_q(q)
    a, da = F.adjoint_step_multirate(0.2, 0.01, lam)
    b, db = F.adjoint_step_global(0.2, 0.01, lam)
    np.testing.assert_array_equal(a, b)
    assert da == db
