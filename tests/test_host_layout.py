"""CPU tests of the library's host side: exported symbols, layout checks,
neighbour tables and the regrid layout (compared with the oracle)."""
import os
import re

import numpy as np
import pytest

import oracle
import synth

fc = pytest.importorskip("paper_1703_03116_gb300")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(fc_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = fc.load()
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(fc._lib.SIGNATURES), set(names) ^ set(fc._lib.SIGNATURES)


def desc_for(w, nforests=1, lmax=None, dtype=None):
    order, lim = {"none": (2, 0), "lw": (2, 0), "mc": (2, 1), "first": (1, 0)}[w.limiter]
    return fc.make_desc(domain={"walls": fc.WALLS, "periodic": fc.PERIODIC}[w.domain], mx=w.mx,
                        lmin=w.lmin, lmax=w.lmax if lmax is None else lmax,
                        dtype=fc.F64 if dtype is None else dtype, velocity=w.velocity,
                        order=order, limiter=lim, transverse=w.transverse, nforests=nforests)


def test_layout_check_accepts_and_rejects():
    w = synth.swirl(1, lmin=2, lmax=5, mx=8)
    F = oracle.initial_forest(w)
    lv = F.leaves()
    d = desc_for(w)
    fc.layout_check(d, lv)
    # drop one leaf: no longer tiles the block
    with pytest.raises(fc.FcError, match="PRECONDITION"):
        fc.layout_check(d, lv[1:])
    # refine one finest leaf twice: 2:1 balance broken
    k = int(np.argmax(lv[:, 2]))
    f, b, l, x, y = lv[k]
    kids = [(f, b, l + 1, 2 * x + (c & 1), 2 * y + (c >> 1)) for c in range(4)]
    g = kids[0]
    grand = [(f, b, l + 2, 2 * g[3] + (c & 1), 2 * g[4] + (c >> 1)) for c in range(4)]
    bad = np.concatenate([np.delete(lv, k, axis=0), np.array(kids[1:] + grand)])
    d2 = desc_for(w, lmax=l + 2)
    with pytest.raises(fc.FcError, match="balanced"):
        fc.layout_check(d2, bad)


def brute_holder(lv, f, b, L, X, Y, periodic):
    """Leaf holding the level-L quadrant (X, Y), by scanning every leaf."""
    n = 1 << L
    if periodic:
        X %= n
        Y %= n
    elif not (0 <= X < n and 0 <= Y < n):
        return None
    for k, (ff, bb, l, x, y) in enumerate(lv):
        if ff != f or bb != b:
            continue
        if l <= L:
            if (X >> (L - l)) == x and (Y >> (L - l)) == y:
                return k
    return "finer"


@pytest.mark.parametrize("domain", ["walls", "periodic"])
def test_neighbour_table_matches_brute_force(domain):
    w = synth.swirl(4, lmin=2, lmax=5, mx=8)
    if domain == "periodic":
        w.domain = "periodic"
    F = oracle.initial_forest(w)
    lv = F.leaves()
    check_neighbours_by_brute_force(fc.layout_neighbours(desc_for(w), lv), lv,
                                    domain == "periodic")


def test_deep_layout_matches_brute_force():
    """A layout refined towards one point down to level 12.  A map of its
    finest-level cells would hold 4^12 entries, so leaves are looked up
    through the key map: the same neighbour table, the same regrid."""
    w = synth.swirl(0, lmin=2, lmax=12, mx=8)
    d = desc_for(w)
    lv = np.array([(0, 0, 2, x, y) for y in range(4) for x in range(4)], dtype=np.int32)
    px, py = 0.3141, 0.2718
    for _ in range(10):
        h = 2.0 ** -lv[:, 2].astype(float)
        inside = ((lv[:, 3] * h <= px) & (px < (lv[:, 3] + 1) * h) &
                  (lv[:, 4] * h <= py) & (py < (lv[:, 4] + 1) * h))
        lv = fc.layout_regrid(d, lv, inside.astype(float), 0.5, -1.0)
    assert lv[:, 2].max() == 12 and len(lv) < 400
    fc.layout_check(d, lv)
    check_neighbours_by_brute_force(fc.layout_neighbours(d, lv), lv, False)
    # coarsening everything back: families merge level by level, balanced
    for _ in range(10):
        lv = fc.layout_regrid(d, lv, np.zeros(len(lv)), 0.5, 0.25)
    assert len(lv) == 16 and set(lv[:, 2]) == {2}


def check_neighbours_by_brute_force(nb, lv, per):
    dirs = [(-1, 0), (1, 0), (0, -1), (0, 1), (-1, -1), (1, -1), (-1, 1), (1, 1)]
    kinds = np.zeros(4, int)
    for k, (f, b, l, x, y) in enumerate(lv):
        for d, (ox, oy) in enumerate(dirs):
            kind, n0, n1, a, fx, fy = nb[k, d]
            kinds[kind] += 1
            h = brute_holder(lv, f, b, l, x + ox, y + oy, per)
            if h is None:
                assert kind == 0
            elif h == "finer":
                assert kind == 2
                for n in (n0, n1):
                    if n >= 0:
                        assert lv[n, 2] == l + 1
                assert (n1 >= 0) == (ox == 0 or oy == 0)
            else:
                assert kind == (1 if lv[h, 2] == l else 3)
                assert n0 == h
            assert a == 0  # one block: identity orientation
    assert np.all(kinds[1:] > 0)


def test_twenty_same_block_cases():
    """Sec. 2.4: seen from the coarser grid there are 4 x (3 + 2) = 20 cases:
    per face one same-size and two fine-neighbour positions, per corner one
    same-size and one fine neighbour."""
    seen = set()
    for seed in range(6):
        w = synth.swirl(seed, lmin=2, lmax=5, mx=8)
        F = oracle.initial_forest(w)
        lv = F.leaves()
        nb = fc.layout_neighbours(desc_for(w), lv)
        for k in range(len(lv)):
            for d in range(8):
                kind, n0, n1 = nb[k, d, :3]
                if kind == 1:
                    seen.add((d, "same"))
                elif kind == 2:
                    if d < 4:
                        seen.add((d, "fine", 0))
                        seen.add((d, "fine", 1))
                    else:
                        seen.add((d, "fine"))
    assert len(seen) == 20


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("taus", [(0.05, 0.0125), (0.2, 0.15), (-1.0, -1.0), (np.inf, np.inf)])
def test_regrid_layout_matches_oracle(seed, taus):
    w = synth.swirl(seed, lmin=2, lmax=5, mx=8)
    F = oracle.initial_forest(w)
    lv = F.leaves()
    F.set_q(synth.random_field((len(lv), 8, 8), seed=seed) ** 6)
    delta = F.tag()
    got = fc.layout_regrid(desc_for(w), lv, delta, *taus)
    F.regrid(*taus)
    assert np.array_equal(got, F.leaves())


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("domain", ["walls", "periodic"])
@pytest.mark.parametrize("taus", [(0.3, 0.05), (0.6, 0.2)])
def test_graded_regrid_layout_matches_oracle(seed, domain, taus):
    """The paper's policy (spread indicator, smooth grading) on the host
    against the oracle's: the same leaves, in the same order."""
    w = synth.swirl(seed, lmin=2, lmax=5, mx=8)
    w.domain, w.indicator, w.smooth = domain, "maxmin", True
    F = oracle.initial_forest(w)
    lv = F.leaves()
    F.set_q(synth.random_field((len(lv), 8, 8), seed=seed) ** 3)
    delta = F.tag()
    d = desc_for(w)
    d.indicator, d.smooth = 1, 1
    got = fc.layout_regrid(d, lv, delta, *taus)
    F.regrid(*taus)
    assert np.array_equal(got, F.leaves())


@pytest.mark.parametrize("seed", range(3))
def test_graded_regrid_of_a_moved_disc_matches_oracle(seed):
    """Refinement and coarsening together: the disc moves off the layout
    adapted to it, so grading both adds a ring of refinement and holds back
    coarsening next to it."""
    w = synth.swirl(seed, lmin=2, lmax=5, mx=8)
    w.indicator, w.smooth = "maxmin", True
    F = oracle.initial_forest(w)
    lv = F.leaves()
    x, y = synth.cell_centres(lv, 8)
    F.set_q(synth.evaluate(synth.adjoint_target(w, seed=seed, max_shift=0.15), x, y))
    delta = F.tag()
    d = desc_for(w)
    d.indicator, d.smooth = 1, 1
    got = fc.layout_regrid(d, lv, delta, 0.5, 0.01)
    n_before = len(lv)
    F.regrid(0.5, 0.01)
    ref = F.leaves()
    assert np.array_equal(got, ref)
    parents = {tuple(r) for r in ref} - {tuple(r) for r in lv}
    assert any(r[2] < lv[:, 2].max() for r in ref) and len(parents) > 0 and n_before > 0


def test_regrid_layout_batched_forests_matches_oracle():
    ws = synth.ensemble(5, seed=3, lmin=2, mx=8, levels=(3, 4, 5))
    F = oracle.initial_forest(ws)
    lv = F.leaves()
    lmax_f = [w.lmax for w in ws]
    assert len(set(lv[:, 0])) == 5
    F.set_q(synth.random_field((len(lv), 8, 8), seed=1) ** 4)
    delta = F.tag()
    got = fc.layout_regrid(desc_for(ws[0], nforests=5, lmax=5), lv, delta, 0.05, 0.0125, lmax_f)
    F.regrid(0.05, 0.0125, lmax_f)
    assert np.array_equal(got, F.leaves())


def test_reflux_option_checked():
    """Refluxing is an option, 0 or 1, on the square domains and the sphere."""
    w = synth.swirl(1, lmin=2, lmax=3, mx=8)
    lv = oracle.initial_forest(w).leaves()
    d = desc_for(w)
    d.reflux = 1
    fc.layout_check(d, lv)
    d.reflux = 2
    with pytest.raises(fc.FcError, match="INVALID_ARG"):
        fc.layout_check(d, lv)
    s = fc.make_desc(domain=fc.SPHERE, mx=8, lmin=0, lmax=1,
                     velocity=("rotation", 0.0, 0.0, 1.0), reflux=1)
    fc.layout_check(s, fc.uniform_leaves(0, nblocks=6))


def test_deformational_flow_option_checked():
    """The deformational flow is for the sphere, with nonzero T and T_f."""
    lv = fc.uniform_leaves(1, nblocks=6)
    d = fc.make_desc(domain=fc.SPHERE, mx=8, lmin=1, lmax=2, velocity=("deform", 2.0, 0.5, 5.0))
    fc.layout_check(d, lv)
    d0 = fc.make_desc(domain=fc.SPHERE, mx=8, lmin=1, lmax=2, velocity=("deform", 2.0, 0.0, 5.0))
    with pytest.raises(fc.FcError, match="INVALID_ARG"):
        fc.layout_check(d0, lv)
    sq = fc.make_desc(domain=fc.PERIODIC, mx=8, lmin=1, lmax=2, velocity=("deform", 2.0, 0.5, 5.0))
    with pytest.raises(fc.FcError, match="INVALID_ARG"):
        fc.layout_check(sq, fc.uniform_leaves(1))


@pytest.mark.parametrize("domain", ["walls", "periodic"])
def test_finer_face_entries_order_their_halves(domain):
    """Refluxing reads the two finer leaves of a face entry as n0: the half of
    the face at the coarse leaf's cells 0..mx/2-1 along it, n1: the other
    half.  Checked on adaptive layouts against the leaves' coordinates."""
    import dataclasses
    w = dataclasses.replace(synth.swirl(3, lmin=2, lmax=5, mx=8), domain=domain)
    lv = oracle.initial_forest(w).leaves()
    nb = fc.layout_neighbours(desc_for(w), lv)
    seen = 0
    for k, (f, b, l, x, y) in enumerate(lv):
        for r in range(4):
            kind, n0, n1 = nb[k, r, 0], nb[k, r, 1], nb[k, r, 2]
            if kind != 2:
                continue
            seen += 1
            m = 1 << (l + 1)
            for half, n in ((0, n0), (1, n1)):
                fl = lv[n]
                assert fl[2] == l + 1
                if r < 2:  # -x / +x face: the fine column beside it, rows 2y + half
                    assert fl[4] == 2 * y + half
                    assert fl[3] == ((2 * x - 1) % m if r == 0 else (2 * x + 2) % m)
                else:      # -y / +y face: columns 2x + half
                    assert fl[3] == 2 * x + half
                    assert fl[4] == ((2 * y - 1) % m if r == 2 else (2 * y + 2) % m)
    assert seen > 10


@pytest.mark.parametrize("domain", ["walls", "periodic"])
def test_reflux_kernel_indexing_is_the_oracle_pairing(domain):
    """On the square domains the refluxing kernel pairs coarse face cell k of
    a finer face with fine leaf n0 (k < mx/2) or n1 (the face entry's two
    leaves), the fine leaf's opposite face (dir ^ 1) and its cells
    2k - half*mx and the next.  That indexing, applied to the neighbour
    table, equals the oracle's geometric pairing."""
    import dataclasses
    w = dataclasses.replace(synth.swirl(4, lmin=2, lmax=5, mx=8), domain=domain)
    F = oracle.initial_forest(w)
    lv = F.leaves()
    ref = F.reflux_pairs()
    nb = fc.layout_neighbours(desc_for(w), lv)
    mx = w.mx
    got = np.full_like(ref, -1)
    got[..., 0] = 0
    for k in range(len(lv)):
        for d in range(4):
            kind, n0, n1 = nb[k, d, 0], nb[k, d, 1], nb[k, d, 2]
            if kind != 2:
                continue
            for c in range(mx):
                half = 1 if c >= mx // 2 else 0
                jf = 2 * c - half * mx
                got[k, d, c] = (1, n1 if half else n0, d ^ 1, jf, jf + 1)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.filterwarnings("ignore:This process .* is multi-threaded")
def test_tables_built_on_host_threads_concurrently_and_after_fork():
    """The neighbour tables are built in pieces by a pool of host threads.
    Calls from several threads at once (one takes the pool, the others run
    on their callers) and a call in a forked child (whose pool has no
    threads) all give the table of a lone call."""
    import multiprocessing as mp
    import threading

    w = synth.swirl(4, lmin=2, lmax=6, mx=8)
    lv = oracle.initial_forest(w).leaves()
    assert len(lv) >= 256  # several pieces
    d = desc_for(w)
    want = fc.layout_neighbours(d, lv)
    got = [None] * 6

    def run(i):
        for _ in range(20):
            got[i] = fc.layout_neighbours(d, lv)

    th = [threading.Thread(target=run, args=(i,)) for i in range(len(got))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for g in got:
        np.testing.assert_array_equal(g, want)
    ctx = mp.get_context("fork")
    with ctx.Pool(1) as pool:
        np.testing.assert_array_equal(pool.apply(fc.layout_neighbours, (d, lv)), want)


def test_large_ensemble_rows_equal_each_forest_built_alone():
    """The rows of a large ensemble (built in many pieces on the host worker
    pool) are, forest by forest, the rows of that forest built alone with
    its patch indices shifted: forests never touch, and the pieces are
    independent."""
    rng = np.random.default_rng(9)
    nf = 24
    d1 = fc.make_desc(domain=fc.PERIODIC, mx=8, lmin=2, lmax=6, dtype=fc.F32,
                      velocity=("swirl", 1.0), nforests=1)
    dn = fc.make_desc(domain=fc.PERIODIC, mx=8, lmin=2, lmax=6, dtype=fc.F32,
                      velocity=("swirl", 1.0), nforests=nf)
    parts = []
    for f in range(nf):
        lv = fc.uniform_leaves(2, 1, 1)
        for _ in range(4):
            lv = fc.layout_regrid(d1, lv, rng.random(len(lv)), 0.5, 0.1)
        lv = np.asarray(lv).copy()
        parts.append(lv)
    allv = np.concatenate([np.column_stack([np.full(len(p), f), p[:, 1:]])
                           for f, p in enumerate(parts)]).astype(np.int32)
    assert len(allv) > 8192  # several pieces of the pool
    big = fc.layout_neighbours(dn, allv)
    off = 0
    for f, p in enumerate(parts):
        one = fc.layout_neighbours(d1, p).copy()
        shifted = one.copy()
        for c in (1, 2):  # neighbour indices (field order) move by the forest's offset
            shifted[:, :, c] = np.where(one[:, :, c] >= 0, one[:, :, c] + off, -1)
        np.testing.assert_array_equal(big[off: off + len(p)], shifted)
        off += len(p)
