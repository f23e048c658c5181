"""The brick domain (Sec. 5.1's replicated problem): a periodic 2^n x 2^n
arrangement of unit blocks, each an adaptive quadtree, every block holding
the same tracer field.

- Oracle pin: the paper notes that with periodic outer faces each block runs
  the same problem.  The oracle's brick (blocks joined through its point
  location across block faces) must therefore reproduce, block by block and
  bit for bit, its periodic unit square (whose geometry is pinned elsewhere):
  the same leaves per block after regrids and the same field after steps.
- The library's host side: the neighbour table across block faces against a
  brute-force scan in the brick's frame, and the graded regrid layout equal
  to the oracle's.
"""
import numpy as np
import pytest

import oracle
import synth

fc = pytest.importorskip("paper_1703_03116_gb300")
from gpu_helpers import desc_for  # noqa: E402


def _per_block(lv, q, b):
    sel = lv[:, 1] == b
    return lv[sel][:, 2:], q[sel]


@pytest.mark.parametrize("n", [1, 2])
def test_oracle_brick_is_the_periodic_square_in_every_block(n):
    w = synth.brick(seed=3, n=n, lmin=2, lmax=4, mx=8, steps=8)
    w1 = synth.brick(seed=3, n=0, lmin=2, lmax=4, mx=8, steps=8)
    w1.domain = "periodic"
    B, S = oracle.initial_forest(w), oracle.initial_forest(w1)
    dt = w.cfl / (w.mx * 2 ** w.lmax) / 0.5
    for k in range(6):
        B.step_global(k * dt, dt)
        S.step_global(k * dt, dt)
        if k == 3:
            B.regrid(w.tau_refine, w.tau_coarsen)
            S.regrid(w.tau_refine, w.tau_coarsen)
    lb, qb = B.leaves(), B.get_q()
    ls, qs = S.leaves(), S.get_q()
    assert len(lb) == (1 << (2 * n)) * len(ls)
    for b in range(1 << (2 * n)):
        l1, q1 = _per_block(lb, qb, b)
        np.testing.assert_array_equal(l1, ls[:, 2:])
        np.testing.assert_array_equal(q1, qs)


def _brute_holder(index, nx, ny, b, L, X, Y, lmin):
    """Leaf of the brick holding the level-L quadrant (X, Y) of block b
    (coordinates may leave the block: the brick is periodic): place the
    quadrant in the brick's frame, wrap, and look for the leaf at every level
    from L down."""
    n = 1 << L
    GX = ((b % nx) * n + X) % (nx * n)
    GY = ((b // nx) * n + Y) % (ny * n)
    bb = (GY // n) * nx + GX // n
    X, Y = GX % n, GY % n
    for l in range(L, lmin - 1, -1):
        k = index.get((bb, l, X >> (L - l), Y >> (L - l)))
        if k is not None:
            return k
    return "finer"


@pytest.mark.parametrize("n", [1, 2])
def test_neighbour_table_across_block_faces_matches_brute_force(n):
    w = synth.brick(seed=4, n=n, lmin=2, lmax=4, mx=8)
    lv = oracle.initial_forest(w).leaves()
    nb = fc.layout_neighbours(desc_for(fc, w, fc.F64), lv)
    nx = ny = 1 << n
    index = {(int(r[1]), int(r[2]), int(r[3]), int(r[4])): k for k, r in enumerate(lv)}
    dirs = [(-1, 0), (1, 0), (0, -1), (0, 1), (-1, -1), (1, -1), (-1, 1), (1, 1)]
    crossing = 0
    for k, (f, b, l, x, y) in enumerate(lv):
        for d, (ox, oy) in enumerate(dirs):
            kind, n0, n1, a, fx, fy = nb[k, d]
            h = _brute_holder(index, nx, ny, b, l, x + ox, y + oy, w.lmin)
            assert kind != 0  # no exterior: the brick is periodic
            if h == "finer":
                assert kind == 2 and lv[n0, 2] == l + 1
            else:
                assert kind == (1 if lv[h, 2] == l else 3) and n0 == h
            assert a == 0  # blocks meet in the identity orientation
            if n0 >= 0 and lv[n0, 1] != b:
                crossing += 1
    assert crossing > 0


@pytest.mark.parametrize("seed", range(3))
def test_graded_regrid_layout_matches_oracle(seed):
    w = synth.brick(seed=seed, n=1, lmin=2, lmax=5, mx=8)
    F = oracle.initial_forest(w)
    lv = F.leaves()
    F.set_q(synth.random_field((len(lv), 8, 8), seed=seed) ** 3)
    delta = F.tag()
    got = fc.layout_regrid(desc_for(fc, w, fc.F64), lv, delta, 0.3, 0.05)
    F.regrid(0.3, 0.05)
    assert np.array_equal(got, F.leaves())


def test_brick_layout_checks():
    """Balance is checked across block faces: block 0 uniform at level 2 and
    block 1 uniform at level 4 are each balanced, but not where they meet."""
    w = synth.brick(seed=1, n=1, lmin=2, lmax=4, mx=8)
    lv = oracle.initial_forest(w).leaves()
    d = desc_for(fc, w, fc.F64)
    fc.layout_check(d, lv)

    def uniform(b, l):
        return [(0, b, l, x, y) for y in range(1 << l) for x in range(1 << l)]

    ok = np.array(uniform(0, 3) + uniform(1, 4) + uniform(2, 3) + uniform(3, 3))
    fc.layout_check(d, ok)
    bad = np.array(uniform(0, 2) + uniform(1, 4) + uniform(2, 3) + uniform(3, 3))
    with pytest.raises(fc.FcError, match="balanced"):
        fc.layout_check(d, bad)
    d.brick_nx = 0
    with pytest.raises(fc.FcError, match="INVALID_ARG"):
        fc.layout_check(d, lv)
