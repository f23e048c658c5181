"""Parity of the cubed sphere under the paper's deformational flow (Sec. 5.3,
a time-dependent streamfunction whose edge fluxes are refreshed before every
level substep) with the FP64 oracle, through the C ABI: multirate and global
stepping, both precisions, a start time away from zero (the captured steps
read it from device memory), a regrid, replayed graphs against direct
launches, and the constant state."""
import numpy as np
import pytest

import synth
from gpu_helpers import F64_TOL, pair, relerr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
fc = pytest.importorskip("paper_1703_03116_gb300")


@pytest.mark.parametrize("mx,lmin,lmax", [(8, 1, 3), (16, 1, 3), (32, 2, 3)])
@pytest.mark.parametrize("variant", [-1, 0])
def test_multirate_matches_oracle(mx, lmin, lmax, variant):
    """Default update (band) and staged under the refreshed fluxes."""
    w = synth.sphere_deform(seed=1, lmin=lmin, lmax=lmax, mx=mx)
    dtc = w.dt_lmin
    for dtype, tol in ((fc.F64, F64_TOL), (fc.F32, 2e-4)):
        ref, gpu = pair(fc, w, dtype)
        gpu.set_advance_variant(variant, 8)
        for s in range(2):
            t = 0.2 + s * dtc
            ref.step_multirate(t, dtc)
            gpu.step_multirate(t, dtc)
        err = relerr(gpu.get_q(), ref.get_q())
        print(f"deform multirate mx={mx} variant {variant} dtype {dtype}: rel err {err:.2e}")
        assert err <= tol


def test_global_steps_match_oracle():
    w = synth.sphere_deform(seed=2, lmin=1, lmax=3, mx=16)
    ref, gpu = pair(fc, w, fc.F64)
    dt = w.dt_lmin / 4
    for s in range(6):
        ref.step_global(0.1 + s * dt, dt)
        gpu.step_global(0.1 + s * dt, dt)
    assert relerr(gpu.get_q(), ref.get_q()) <= F64_TOL


def test_regrid_then_parity():
    w = synth.sphere_deform(seed=3, lmin=1, lmax=3, mx=16)
    ref, gpu = pair(fc, w, fc.F64)
    dtc = w.dt_lmin
    for s in range(3):
        ref.step_multirate(s * dtc, dtc)
        gpu.step_multirate(s * dtc, dtc)
        if s == 1:
            assert gpu.tag_regrid(w.tau_refine, w.tau_coarsen) == \
                ref.regrid(w.tau_refine, w.tau_coarsen)
    np.testing.assert_array_equal(gpu.leaves(), ref.leaves())
    assert relerr(gpu.get_q(), ref.get_q()) <= F64_TOL


def test_graphs_match_direct_launches():
    w = synth.sphere_deform(seed=4, lmin=1, lmax=3, mx=16)
    ref, a = pair(fc, w, fc.F32)
    b = fc.Forest(a.desc, ref.leaves())
    b.set_q(a.get_q())
    b.graphs(False)
    dtc = w.dt_lmin
    for s in range(4):
        a.step_multirate(s * dtc, dtc)
        b.step_multirate(s * dtc, dtc)
        if s == 1:
            assert a.tag_regrid(w.tau_refine, w.tau_coarsen) == \
                b.tag_regrid(w.tau_refine, w.tau_coarsen)
    np.testing.assert_array_equal(a.get_q(), b.get_q())


def test_constant_state():
    w = synth.sphere_deform(seed=5, lmin=1, lmax=3, mx=16)
    _, gpu = pair(fc, w, fc.F64)
    gpu.set_q(np.ones((len(gpu), 16, 16)))
    for s in range(3):
        gpu.step_multirate(s * w.dt_lmin, w.dt_lmin)
    assert np.abs(gpu.get_q() - 1.0).max() < 1e-12
