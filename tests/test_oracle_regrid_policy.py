"""Pins of the oracle's regrid policy of the paper's runs (Sec. 5.1: a patch
is tagged by the spread of its values, largest minus smallest; Sec. 3.3:
smooth grading of the target levels), against facts fixed by construction:
  * the spread of a linear field over a patch is |a| + |b| times the
    distance between its outermost cell centres;
  * grading one tagged patch at the coarsest level refines it together with
    every patch that touches it, and nothing else;
  * grading changes nothing when no patch is tagged, and when every patch is.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.filterwarnings("ignore")


def _forest(level, lmin, lmax, mx=8, domain=oracle.WALLS, indicator=1, smooth=1):
    prm = oracle.params(domain, mx, 2, lmin, lmax, ("const", 1.0, 0.5),
                        indicator=indicator, smooth=smooth)
    return oracle.Forest(prm, oracle.uniform_leaves(level))


def _centres(F):
    lv = F.leaves()
    mx = F.mx
    h = 2.0 ** -lv[:, 2].astype(float) / mx
    i = np.arange(mx) + 0.5
    x = lv[:, 3, None, None] * mx * h[:, None, None] + i[None, None, :] * h[:, None, None]
    y = lv[:, 4, None, None] * mx * h[:, None, None] + i[None, :, None] * h[:, None, None]
    return np.broadcast_to(x, (len(lv), mx, mx)), np.broadcast_to(y, (len(lv), mx, mx)), h


@pytest.mark.parametrize("a,b", [(0.7, -1.3), (-2.0, 0.0), (0.25, 0.5)])
def test_spread_of_a_linear_field(a, b):
    F = _forest(3, 2, 4)
    x, y, h = _centres(F)
    F.set_q(a * x + b * y + 0.3)
    got = F.tag()
    want = (abs(a) + abs(b)) * (F.mx - 1) * h
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15)


def _one_tagged(F, px, py):
    lv = F.leaves()
    q = np.zeros((len(lv), F.mx, F.mx))
    k = int(np.flatnonzero((lv[:, 3] == px) & (lv[:, 4] == py))[0])
    q[k, 0, 0] = 1.0  # spread 1 in that patch, 0 elsewhere
    F.set_q(q)


@pytest.mark.parametrize("px,py", [(1, 1), (0, 0), (3, 2)])
def test_grading_refines_the_touching_ring(px, py):
    graded, plain = _forest(2, 2, 4), _forest(2, 2, 4, smooth=0)
    for F in (graded, plain):
        _one_tagged(F, px, py)
        F.regrid(0.5, -1.0)
    ring = {(x, y) for x in range(px - 1, px + 2) for y in range(py - 1, py + 2)
            if 0 <= x < 4 and 0 <= y < 4}
    lv = graded.leaves()
    refined = {(int(x) // 2, int(y) // 2) for _, _, l, x, y in lv if l == 3}
    assert refined == ring
    assert len(lv) == 16 + 3 * len(ring)
    assert len(plain.leaves()) == 16 + 3


@pytest.mark.parametrize("tag_all", [False, True])
def test_grading_is_idle_when_all_or_nothing_is_tagged(tag_all):
    out = []
    for smooth in (0, 1):
        F = _forest(3, 2, 4, smooth=smooth)
        rng = np.random.default_rng(5)
        q = rng.random((len(F.leaves()), F.mx, F.mx)) if tag_all else np.zeros(
            (len(F.leaves()), F.mx, F.mx))
        F.set_q(q)
        F.regrid(0.5 if tag_all else 2.0, -1.0)
        out.append(F.leaves())
    np.testing.assert_array_equal(out[0], out[1])
