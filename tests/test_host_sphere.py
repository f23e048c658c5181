"""CPU tests of the library's cubed-sphere host side (Sec. 2.4 multiblock
indexing): the face transforms and neighbour kinds of the neighbour table,
compared with the oracle's brute-force ghost fill, and the regrid layout
(refine, 2:1 balance across cube edges and vertices, coarsen), compared with
the oracle's."""
import numpy as np
import pytest

import oracle
import synth

fc = pytest.importorskip("paper_1703_03116_gb300")

DIRS = [(-1, 0), (1, 0), (0, -1), (0, 1), (-1, -1), (1, -1), (-1, 1), (1, 1)]


def sphere_desc(w, lmax=None):
    return fc.make_desc(domain=fc.SPHERE, mx=w.mx, lmin=w.lmin,
                        lmax=w.lmax if lmax is None else lmax, dtype=fc.F64,
                        velocity=w.velocity)


def apply_code(a, x, y):
    u, v = (y, x) if a & 1 else (x, y)
    return (-u if a & 2 else u), (-v if a & 4 else v)


def region_cells(d, mx):
    ox, oy = DIRS[d]
    xs = range(-2, 0) if ox < 0 else (range(mx, mx + 2) if ox > 0 else range(mx))
    ys = range(-2, 0) if oy < 0 else (range(mx, mx + 2) if oy > 0 else range(mx))
    return [(i, j) for j in ys for i in xs]


def oracle_ids(F):
    """Fill the oracle's ghosts with data = field index of each interior cell
    (leaf * mx^2 + j * mx + i); returns the full arrays."""
    mx = F.mx
    ids = np.arange(len(F) * mx * mx, dtype=np.float64).reshape(len(F), mx, mx)
    F.set_q(ids)
    F.fill_ghosts()
    return F.get_q_full()


@pytest.mark.parametrize("level", [0, 1, 2])
def test_face_transforms_match_oracle_copies(level):
    w = synth.sphere(seed=0, lmin=level, lmax=level, mx=8)
    F = oracle.Forest(oracle.params_for(w), oracle.uniform_leaves(level, 1, 6))
    lv = F.leaves()
    mx = 8
    full = oracle_ids(F)
    nb = fc.layout_neighbours(sphere_desc(w), lv)
    nsame = ncorner3 = 0
    N = 1 << level
    for k, (f, b, l, x, y) in enumerate(lv):
        for d in range(8):
            kind, n0, n1, a, fx, fy = nb[k, d]
            ox, oy = DIRS[d]
            beyond_x = not (0 <= x + ox < N)
            beyond_y = not (0 <= y + oy < N)
            if beyond_x and beyond_y:  # past a cube vertex: only three blocks meet
                assert kind == 4
                ncorner3 += 1
                continue
            assert kind == 1
            nsame += 1
            if beyond_x or beyond_y:
                assert lv[n0, 1] != b  # across a cube edge
            for (i, j) in region_cells(d, mx):
                u, v = apply_code(a, x * mx + i, y * mx + j)
                gx, gy = u + fx, v + fy
                li, lj = gx - lv[n0, 3] * mx, gy - lv[n0, 4] * mx
                assert 0 <= li < mx and 0 <= lj < mx
                assert full[k, j + 2, i + 2] == n0 * mx * mx + lj * mx + li
    assert ncorner3 == 6 * 4  # every face has four cube-vertex corners
    assert nsame == 8 * len(lv) - 24


def adaptive_sphere(seed, lmin=1, lmax=3, mx=8):
    w = synth.sphere(seed=seed, lmin=lmin, lmax=lmax, mx=mx)
    return w, oracle.initial_forest(w)


@pytest.mark.parametrize("seed", range(3))
def test_adaptive_tables_match_oracle(seed):
    w, F = adaptive_sphere(seed)
    lv = F.leaves()
    assert len(np.unique(lv[:, 2])) >= 2
    d = sphere_desc(w)
    fc.layout_check(d, lv)
    nb = fc.layout_neighbours(d, lv)
    mx = w.mx
    # per-leaf constant data: copies and (area-weighted) averages return the
    # source leaf's value
    F.set_q(np.repeat(np.arange(len(lv), dtype=np.float64), mx * mx).reshape(len(lv), mx, mx))
    F.fill_ghosts()
    full = F.get_q_full()
    kinds = np.zeros(5, int)
    for k, (f, b, l, x, y) in enumerate(lv):
        for r in range(8):
            kind, n0, n1, a, fx, fy = nb[k, r]
            kinds[kind] += 1
            if kind in (1, 2):
                for (i, j) in region_cells(r, mx):
                    u, v = apply_code(a, x * mx + i, y * mx + j)
                    gx, gy = u + fx, v + fy  # level-l index in the neighbour block
                    if kind == 1:
                        src = n0
                    else:  # the fine leaf holding the fine cells (2 gx, 2 gy)
                        src = [n for n in (n0, n1) if n >= 0 and
                               0 <= 2 * gx - lv[n, 3] * mx < mx and 0 <= 2 * gy - lv[n, 4] * mx < mx]
                        assert len(src) == 1
                        src = src[0]
                        assert lv[src, 2] == l + 1
                    assert abs(full[k, j + 2, i + 2] - src) < 1e-12 * max(1, src)
            elif kind == 3:
                # the coarse leaf holds every transformed ghost cell, and sees
                # this leaf as a finer neighbour
                assert lv[n0, 2] == l - 1
                for (i, j) in region_cells(r, mx):
                    u, v = apply_code(a, x * mx + i, y * mx + j)
                    ic, jc = (u + fx) // 2 - lv[n0, 3] * mx, (v + fy) // 2 - lv[n0, 4] * mx
                    assert 0 <= ic < mx and 0 <= jc < mx
                back = nb[n0]
                assert any(back[q, 0] == 2 and k in (back[q, 1], back[q, 2]) for q in range(8))
            elif kind == 0:
                raise AssertionError("the sphere has no exterior")
    assert kinds[1] > 0 and kinds[2] > 0 and kinds[3] > 0 and kinds[4] > 0


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("taus", [(0.05, 0.0125), (0.2, 0.15), (-1.0, -1.0), (np.inf, np.inf)])
def test_regrid_layout_matches_oracle(seed, taus):
    w, F = adaptive_sphere(seed, lmin=1, lmax=4)
    lv = F.leaves()
    F.set_q(synth.random_field((len(lv), w.mx, w.mx), seed=seed) ** 6)
    delta = F.tag()
    got = fc.layout_regrid(sphere_desc(w), lv, delta, *taus)
    F.regrid(*taus)
    assert np.array_equal(got, F.leaves())


def test_balance_across_a_cube_vertex_matches_oracle():
    """Refine only the leaf of face 0 at one cube vertex, four times: the 2:1
    balance must spread onto all three faces that meet there, as the
    oracle's brute-force balance (closed boxes on the cube) does."""
    w = synth.sphere(seed=0, lmin=1, lmax=5, mx=8)
    F = oracle.Forest(oracle.params_for(w), oracle.uniform_leaves(1, 1, 6))
    d = sphere_desc(w)
    for _ in range(4):
        lv = F.leaves()
        n = 1 << lv[:, 2]
        hot = (lv[:, 1] == 0) & (lv[:, 3] == n - 1) & (lv[:, 4] == n - 1)
        q = np.zeros((len(lv), 8, 8))
        q[hot, 6, 6] = 1.0  # a spike inside the vertex leaf only
        F.set_q(q)
        delta = F.tag()
        assert delta[hot][0] == 0.5 and np.all(delta[~hot] < 0.25)
        got = fc.layout_regrid(d, lv, delta, 0.25, -1.0)
        F.regrid(0.25, -1.0)
        assert np.array_equal(got, F.leaves())
        fc.layout_check(d, got)
    lv = F.leaves()
    assert lv[:, 2].max() == 5
    near = lv[lv[:, 2] >= 3]
    assert set(near[:, 1]) >= {0, 2, 4}  # +Z, +X, +Y meet at (1, 1, 1)


def test_input_generator_centres_match_the_oracle():
    """The seeded input generator places sphere cell centres by the block
    convention of the C interface; the oracle by its own face frames."""
    w, F = adaptive_sphere(0)
    X = synth.sphere_cell_centres(F.leaves(), w.mx)
    np.testing.assert_allclose(X, F.sphere_centres(), rtol=0, atol=1e-15)


@pytest.mark.parametrize("case", ["walls", "periodic", "sphere rotation", "sphere deformational",
                                  "sphere uniform"])
def test_reflux_pairing_matches_oracle(case):
    """What refluxing exchanges per face cell (the finer leaf's face and its
    two cells across, or across a cube edge the same-level leaf's face and
    cell), from the product's neighbour table and index transforms, equals
    what the oracle finds by locating points beyond each face."""
    import dataclasses
    if case in ("walls", "periodic"):
        w = dataclasses.replace(synth.swirl(3, lmin=2, lmax=5, mx=8), domain=case)
    elif case == "sphere rotation":
        w = synth.sphere(seed=1, lmin=1, lmax=3, mx=8)
    elif case == "sphere uniform":  # the six level-0 leaves: every face lies on a cube edge
        w = synth.sphere(seed=1, lmin=0, lmax=0, mx=8)
    else:
        w = synth.sphere_deform(seed=2, lmin=1, lmax=4, mx=8)
    F = oracle.initial_forest(w)
    lv = F.leaves()
    ref = F.reflux_pairs()
    dom = {"walls": fc.WALLS, "periodic": fc.PERIODIC, "sphere": fc.SPHERE}[w.domain]
    d = fc.make_desc(domain=dom, mx=w.mx, lmin=w.lmin, lmax=w.lmax, dtype=fc.F64,
                     velocity=w.velocity)
    got = fc.layout_reflux(d, lv)
    assert (ref[..., 0] == 1).sum() > 0 or w.lmax == w.lmin
    if w.domain == "sphere":
        assert (ref[..., 0] == 2).sum() > 0
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("taus", [(0.3, 0.05), (0.6, 0.2)])
def test_graded_regrid_on_the_sphere_matches_oracle(seed, taus):
    """The paper's regrid policy (spread indicator, smooth grading) on the
    cubed sphere: the leaves touching a leaf come from the neighbour table's
    face and corner entries, across cube edges and, at a cube vertex, through
    the two face neighbours there; the oracle intersects closed boxes on the
    cube.  Same leaves, same order."""
    import dataclasses
    w, F0 = adaptive_sphere(seed, lmin=1, lmax=4)
    w = dataclasses.replace(w, indicator="maxmin", smooth=True)
    F = oracle.Forest(oracle.params_for(w), F0.leaves())
    lv = F.leaves()
    F.set_q(synth.random_field((len(lv), w.mx, w.mx), seed=seed) ** 3)
    delta = F.tag()
    d = sphere_desc(w)
    d.indicator, d.smooth = 1, 1
    got = fc.layout_regrid(d, lv, delta, *taus)
    F.regrid(*taus)
    assert np.array_equal(got, F.leaves())


def test_graded_regrid_at_a_cube_vertex_matches_oracle():
    """A spike in the leaf of face 0 at a cube vertex, smooth grading on: the
    leaves of the three faces that meet at the vertex are graded together,
    on the host as in the oracle."""
    import dataclasses
    w = dataclasses.replace(synth.sphere(seed=0, lmin=1, lmax=4, mx=8), indicator="maxmin",
                            smooth=True)
    F = oracle.Forest(oracle.params_for(w), oracle.uniform_leaves(1, 1, 6))
    d = sphere_desc(w)
    d.indicator, d.smooth = 1, 1
    for _ in range(2):
        lv = F.leaves()
        n = 1 << lv[:, 2]
        hot = (lv[:, 1] == 0) & (lv[:, 3] == n - 1) & (lv[:, 4] == n - 1)
        q = np.zeros((len(lv), 8, 8))
        q[hot, 6, 6] = 1.0
        F.set_q(q)
        delta = F.tag()
        got = fc.layout_regrid(d, lv, delta, 0.5, 0.0)
        F.regrid(0.5, 0.0)
        assert np.array_equal(got, F.leaves())
    assert len(np.unique(F.leaves()[:, 1][F.leaves()[:, 2] > 1])) >= 3
