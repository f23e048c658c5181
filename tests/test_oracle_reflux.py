"""Pins of the oracle's refluxing (conservative coarse/fine correction,
Berger and Colella 1989; an extension: the paper's scheme has none), against
facts fixed by construction:
  * first order, one constant speed, no transverse terms: a coarse cell on a
    face where the flow leaves the finer side changes by
    -nu |s| (q - A), A the mean of the fine boundary cells across the face
    over the fine substeps (closed form, each of the four face directions,
    global and multirate stepping);
  * total mass is conserved to rounding on adaptive forests (periodic and
    walls, constant and swirling velocity, both steppings), and drifts
    without the correction;
  * on a uniform forest (no coarse/fine face) the correction changes nothing;
  * on the cubed sphere (cube edges: the block of lower index keeps its
    flux) mass is conserved to rounding, and a constant state stays constant
    wherever all fluxes of a step belong to one velocity field.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import synth

MX = 8
# level-1 leaves, with (0, 0) refined into its four level-2 children
LEAVES = np.array([(0, 0, 1, 0, 1), (0, 0, 1, 1, 0), (0, 0, 1, 1, 1),
                   (0, 0, 2, 0, 0), (0, 0, 2, 1, 0), (0, 0, 2, 0, 1), (0, 0, 2, 1, 1)],
                  dtype=np.int32)

# (speed (u, v), coarse leaf (x, y) at level 1, the coarse cells on the face
# as (i, j) of k, the fine leaf (x', y') at level 2 and its boundary cell and
# the cell upwind of it as (i, j) of r, for coarse cell k and fine row r)
CASES = {
    # fine on the -x side of coarse leaf (1, 0), flow in +x
    "+x": ((1.0, 0.0), (1, 0), lambda k: (0, k), lambda k: (1, (2 * k) // MX),
           lambda r: (MX - 1, r), lambda r: (MX - 2, r)),
    # fine on the +x side (through the periodic wrap) of coarse leaf (1, 0), flow in -x
    "-x": ((-1.0, 0.0), (1, 0), lambda k: (MX - 1, k), lambda k: (0, (2 * k) // MX),
           lambda r: (0, r), lambda r: (1, r)),
    # fine on the -y side of coarse leaf (0, 1), flow in +y
    "+y": ((0.0, 1.0), (0, 1), lambda k: (k, 0), lambda k: ((2 * k) // MX, 1),
           lambda r: (r, MX - 1), lambda r: (r, MX - 2)),
    # fine on the +y side (through the periodic wrap) of coarse leaf (0, 1), flow in -y
    "-y": ((0.0, -1.0), (0, 1), lambda k: (k, MX - 1), lambda k: ((2 * k) // MX, 0),
           lambda r: (r, 0), lambda r: (r, 1)),
}


def _first_order(vel, reflux, lmin=1, lmax=2):
    return oracle.params(oracle.PERIODIC, MX, 2, lmin, lmax, ("const",) + tuple(vel),
                         order=1, limiter=0, transverse=0, reflux=reflux)


def _index(F):
    return {(int(l), int(x), int(y)): p for p, (_, _, l, x, y) in enumerate(F.leaves())}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("mode", ["global", "multirate"])
def test_first_order_closed_form(case, mode):
    vel, cxy, ccell, fleaf, fcell, fup = CASES[case]
    rng = np.random.Generator(np.random.PCG64(7))
    out = {}
    for reflux in (0, 1):
        F = oracle.Forest(_first_order(vel, reflux), LEAVES)
        q0 = rng.uniform(0.5, 1.5, (len(F), MX, MX)) if reflux == 0 else q0
        F.set_q(q0)
        h_c = 1.0 / (2 * MX)
        dt_c = 0.5 * h_c  # Courant number 1/2 on both levels under multirate
        if mode == "global":
            F.step_global(0.0, 0.5 * dt_c)
        else:
            F.step_multirate(0.0, dt_c)
        out[reflux] = F.get_q()
    idx = _index(F)
    pc = idx[(1,) + cxy]
    s = abs(vel[0]) + abs(vel[1])
    for k in range(MX):
        ci, cj = ccell(k)
        pf = idx[(2,) + fleaf(k)]
        r0 = 2 * k - ((2 * k) // MX) * MX
        vals = []
        for r in (r0, r0 + 1):
            bi, bj = fcell(r)
            ui, uj = fup(r)
            qb, qu = q0[pf, bj, bi], q0[pf, uj, ui]
            vals.append(qb)
            if mode == "multirate":  # the boundary cell after the first fine substep
                nu_f = 0.5  # (dt_c / 2) / (h_c / 2)
                vals.append(qb - nu_f * s * (qb - qu))
        A = float(np.mean(vals))
        nu_c = (0.5 * dt_c if mode == "global" else dt_c) / h_c
        q = q0[pc, cj, ci]
        want = q - nu_c * s * (q - A)
        assert abs(out[1][pc, cj, ci] - want) < 1e-14, (case, mode, k)
        # without the correction the coarse cell used its own (averaged) ghost
        assert abs(out[0][pc, cj, ci] - want) > 1e-6, (case, mode, k)


def _mass_run(w, mode, steps):
    F = oracle.initial_forest(w)
    nco, dtc = synth.time_step(w)
    dt = dtc / 2 ** (w.lmax - w.lmin)
    m0 = F.mass().sum()
    t = 0.0
    for _ in range(steps):
        if mode == "global":
            F.step_global(t, dt)
            t += dt
        else:
            F.step_multirate(t, dtc)
            t += dtc
    return (F.mass().sum() - m0) / m0


@pytest.mark.parametrize("domain,velocity", [("periodic", ("const", 1.0, 0.5)),
                                             ("periodic", ("swirl", 4.0)),
                                             ("walls", ("swirl", 4.0))])
@pytest.mark.parametrize("mode", ["global", "multirate"])
def test_mass_conserved_on_adaptive_forests(domain, velocity, mode):
    w = dataclasses.replace(synth.swirl(seed=1, lmin=2, lmax=4, mx=8), domain=domain,
                            velocity=velocity)
    steps = 4 if mode == "global" else 2
    drift = _mass_run(w, mode, steps)
    fixed = _mass_run(dataclasses.replace(w, reflux=True), mode, steps)
    assert abs(drift) > 1e-6  # the forest has coarse/fine faces that leak
    assert abs(fixed) < 5e-15


@pytest.mark.parametrize("mode", ["global", "multirate"])
def test_uniform_forest_unchanged(mode):
    w = synth.uniform_periodic(seed=3, level=2, mx=8)
    res = []
    for reflux in (False, True):
        F = oracle.initial_forest(dataclasses.replace(w, reflux=reflux))
        dtc = 0.5 / (w.mx * 2 ** w.lmax)
        for n in range(3):
            (F.step_global if mode == "global" else F.step_multirate)(n * dtc, dtc)
        res.append(F.get_q())
    assert np.array_equal(res[0], res[1])


def _sphere_run(w, mode, steps, const=False):
    F = oracle.initial_forest(w)
    if const:
        F.set_q(np.ones((len(F), w.mx, w.mx)))
    kap = F.kappa()
    m0 = np.sum(kap * F.get_q())
    dtc = w.dt_lmin if w.dt_lmin else synth.time_step(w)[1]
    n = 2 ** (w.lmax - w.lmin)
    for s in range(steps):
        if mode == "global":
            for r in range(n):
                F.step_global(s * dtc + r * dtc / n, dtc / n)
        else:
            F.step_multirate(s * dtc, dtc)
    return (np.sum(kap * F.get_q()) - m0) / m0, F


SPHERES = {
    "rotation uniform": lambda: synth.sphere(seed=1, lmin=2, lmax=2, mx=8),
    "rotation adaptive": lambda: synth.sphere(seed=1, lmin=1, lmax=3, mx=8),
    "deformational adaptive": lambda: synth.sphere_deform(seed=1, lmin=1, lmax=3, mx=8),
}


@pytest.mark.parametrize("name", sorted(SPHERES))
@pytest.mark.parametrize("mode", ["global", "multirate"])
def test_sphere_mass_conserved(name, mode):
    """On the cubed sphere each side of a cube edge computes that edge's flux
    from its own ghost cells; with the block of lower index keeping its flux
    (and the fine side at coarse/fine faces) mass is conserved to rounding."""
    w = SPHERES[name]()
    drift, F = _sphere_run(w, mode, 3)
    fixed, _ = _sphere_run(dataclasses.replace(w, reflux=True), mode, 3)
    assert abs(drift) > 1e-7
    assert abs(fixed) < 5e-15


@pytest.mark.parametrize("name,mode", [("rotation adaptive", "global"),
                                       ("rotation adaptive", "multirate"),
                                       ("deformational adaptive", "global")])
def test_sphere_constant_state_kept(name, mode):
    """Where every flux of a step belongs to one velocity field (a steady
    flow, or all levels at one time), the exchanged fluxes describe the same
    edges: a constant state stays constant.  (A mismatched cell along a cube
    edge or a coarse/fine face would move it: the fluxes vary along edges.)"""
    w = dataclasses.replace(SPHERES[name](), reflux=True)
    _, F = _sphere_run(w, mode, 3, const=True)
    assert np.abs(F.get_q() - 1.0).max() < 1e-13


def test_rejected_where_not_stated():
    F = oracle.Forest(_first_order((1.0, 0.0), 1), LEAVES)
    F.set_q(np.ones((len(F), MX, MX)))
    with pytest.raises(oracle.OracleError):
        F.adjoint_step_global(0.0, 0.01, np.ones((len(F), MX, MX)))
