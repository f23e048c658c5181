"""The OpenMP build of the oracle (the all-cores CPU baseline) computes what
the plain build computes, bit for bit: its patch loops only split
independent per-patch work over host threads."""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture
def omp():
    try:
        oracle.use_openmp(True)
    except Exception as e:  # a compiler without OpenMP: nothing to compare
        pytest.skip(f"no OpenMP build: {e}")
    yield
    oracle.use_openmp(False)


def _run(w):
    F = oracle.initial_forest(w)
    _, dtc = synth.time_step(w)
    for n in range(3):
        F.step_multirate(n * dtc, dtc)
    F.regrid(w.tau_refine, w.tau_coarsen)
    F.step_global(3 * dtc, dtc / 4)
    return F.leaves(), F.get_q(), F.mass()


@pytest.mark.parametrize("kind", ["swirl", "sphere"])
def test_openmp_build_matches_plain_build_bitwise(kind, omp):
    w = (synth.swirl(1, lmin=2, lmax=4, mx=16) if kind == "swirl"
         else synth.sphere(seed=1, lmin=1, lmax=3, mx=8))
    oracle.use_openmp(False)
    a = _run(w)
    oracle.use_openmp(True)
    assert oracle.threads() >= 1
    b = _run(w)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
