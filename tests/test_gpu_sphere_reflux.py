"""Refluxing on the cubed sphere on the GPU (the conservative correction, an
extension of the paper's scheme) against the oracle's, through the C ABI.

On the sphere the library applies the host pairing (fc_layout_reflux, equal
to the oracle's geometric pairing): a coarse cell beside finer patches takes
their volume fluxes (time ratio 1/2 per substep under multirate stepping, 1
under global stepping), and a cell on a cube edge whose same-size neighbour
lies on the block of lower index takes that neighbour's flux.  Then FP64
mass (sum of kappa q) is conserved to rounding, where without the correction
it drifts.  FP64 parity with the oracle <= 1e-12; FP32 within the FP32
sphere bound of the other sphere tests.
"""
import dataclasses

import numpy as np
import pytest

import synth
from gpu_helpers import F64_TOL, pair, relerr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
fc = pytest.importorskip("paper_1703_03116_gb300")

SPHERES = {
    "rotation": lambda mx: synth.sphere(seed=1, lmin=1, lmax=3, mx=mx),
    "deformational": lambda mx: synth.sphere_deform(seed=1, lmin=1, lmax=3, mx=mx),
}


def _dt(w):
    return w.dt_lmin if getattr(w, "dt_lmin", None) else synth.time_step(w)[1]


@pytest.mark.parametrize("name", sorted(SPHERES))
@pytest.mark.parametrize("mx", [8, 16, 32])
@pytest.mark.parametrize("variant", [-1, 0])
def test_sphere_reflux_multirate_matches_oracle(name, mx, variant):
    """Default update (band) and staged, both recording the face fluxes."""
    w = dataclasses.replace(SPHERES[name](mx), reflux=True)
    dtc = _dt(w)
    t0 = 0.2 if name == "deformational" else 0.0
    for dtype, tol in ((fc.F64, F64_TOL), (fc.F32, 2e-4)):
        ref, gpu = pair(fc, w, dtype)
        gpu.set_advance_variant(variant, 8)
        for n in range(2):
            ref.step_multirate(t0 + n * dtc, dtc)
            gpu.step_multirate(t0 + n * dtc, dtc)
        err = relerr(gpu.get_q(), ref.get_q())
        print(f"sphere reflux multirate {name} mx={mx} variant {variant} dtype {dtype}: "
              f"rel err {err:.2e}")
        assert err <= tol


def test_sphere_reflux_global_steps_match_oracle():
    w = dataclasses.replace(SPHERES["rotation"](16), reflux=True)
    dt = _dt(w) / 4
    ref, gpu = pair(fc, w, fc.F64)
    for n in range(4):
        ref.step_global(n * dt, dt)
        gpu.step_global(n * dt, dt)
    assert relerr(gpu.get_q(), ref.get_q()) <= F64_TOL


@pytest.mark.parametrize("name", sorted(SPHERES))
@pytest.mark.parametrize("mode", ["multirate", "global"])
def test_sphere_mass_conserved_to_rounding(name, mode):
    drift = {}
    for reflux in (False, True):
        w = dataclasses.replace(SPHERES[name](16), reflux=reflux)
        dtc = _dt(w)
        dt = dtc if mode == "multirate" else dtc / 4
        _, gpu = pair(fc, w, fc.F64)
        m0 = gpu.mass().sum()
        for n in range(4):
            (gpu.step_multirate if mode == "multirate" else gpu.step_global)(n * dt, dt)
        drift[reflux] = (gpu.mass().sum() - m0) / m0
    print(f"sphere {name} {mode}: drift without {drift[False]:.2e}, with {drift[True]:.2e}")
    assert abs(drift[False]) > 1e-8
    assert abs(drift[True]) < 1e-13


def test_sphere_reflux_graphs_and_regrid_match_direct_launches():
    w = dataclasses.replace(synth.sphere(seed=0, lmin=1, lmax=4, mx=16), reflux=True)
    dtc = _dt(w)
    ref, a = pair(fc, w, fc.F32)
    b = fc.Forest(a.desc, ref.leaves())
    b.set_q(a.get_q())
    b.graphs(False)
    for n in range(6):
        a.step_multirate(n * dtc, dtc)
        b.step_multirate(n * dtc, dtc)
        if (n + 1) % 3 == 0:
            assert a.tag_regrid(w.tau_refine, w.tau_coarsen) == \
                b.tag_regrid(w.tau_refine, w.tau_coarsen)
    np.testing.assert_array_equal(a.get_q(), b.get_q())
