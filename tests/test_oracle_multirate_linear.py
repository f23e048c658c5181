"""Pin of the oracle's multirate time interpolation (Sec. 4: a fine level's
ghost cells from the coarser level interpolated linearly in time between its
states before and after its step), by exactness on linear data.

With a constant velocity (u, v) the exact solution of q0 = a x + b y + c is
a (x - u t) + b (y - v t) + c.  The wave-propagation step reproduces a linear
field exactly (every difference of it is constant, the MC limiter reads
theta = 1), the copies, averages and minmod interpolations of Alg. 1 are exact
on it, and the exact solution is linear in time, so linear interpolation in
time is exact too.  An adaptive forest stepped by the multirate recursion
must therefore return the translated field to rounding wherever the periodic
seam (where the linear field jumps) has not reached.  Without the time
interpolation (coarse ghosts frozen at the older state) the interior error
is about 5e-3 here.
"""
import numpy as np
import pytest

import oracle

MX = 8
A, B, C = 0.7, -0.4, 2.0


def _leaves():
    """Levels 2, 3, 4 nested around the centre of the periodic square."""
    out = []
    for y in range(4):
        for x in range(4):
            if not (1 <= x <= 2 and 1 <= y <= 2):
                out.append((0, 0, 2, x, y))
                continue
            for cy in range(2):
                for cx in range(2):
                    X, Y = 2 * x + cx, 2 * y + cy
                    if 3 <= X <= 4 and 3 <= Y <= 4:
                        out += [(0, 0, 4, 2 * X + dx, 2 * Y + dy) for dy in range(2)
                                for dx in range(2)]
                    else:
                        out.append((0, 0, 3, X, Y))
    return np.array(out, dtype=np.int32)


def _centres(lv):
    h = 1.0 / (MX * 2.0 ** lv[:, 2])
    i = np.arange(MX) + 0.5
    X = (lv[:, 3, None, None] * MX + i[None, None, :]) * h[:, None, None]
    Y = (lv[:, 4, None, None] * MX + i[None, :, None]) * h[:, None, None]
    return np.broadcast_to(X, (len(lv), MX, MX)), np.broadcast_to(Y, (len(lv), MX, MX))


@pytest.mark.parametrize("scheme", [(1, 0, 0), (2, 0, 2), (2, 1, 2), (2, 1, 1)])
@pytest.mark.parametrize("vel", [(1.0, 0.0), (1.0, 0.5), (-0.6, 0.8)])
@pytest.mark.parametrize("mode", ["global", "multirate"])
def test_linear_field_translates_exactly(scheme, vel, mode):
    order, limiter, transverse = scheme
    u, v = vel
    prm = oracle.params(oracle.PERIODIC, MX, 2, 2, 4, ("const", u, v), order=order,
                        limiter=limiter, transverse=transverse)
    F = oracle.Forest(prm, _leaves())
    X, Y = _centres(F.leaves())
    F.set_q(A * X + B * Y + C)
    dt_f = 0.8 / (MX * 2 ** 4) / max(abs(u), abs(v))
    if mode == "global":
        for s in range(4):
            F.step_global(s * dt_f, dt_f)
    else:
        F.step_multirate(0.0, 4 * dt_f)
    t = 4 * dt_f
    want = A * (X - u * t) + B * (Y - v * t) + C
    inner = (X > 0.25) & (X < 0.75) & (Y > 0.25) & (Y < 0.75)
    assert np.abs(F.get_q() - want)[inner].max() < 1e-13
