"""Parity of the cubed-sphere CUDA path with the FP64 oracle (Sec. 2.4
multiblock ghost fill, Sec. 5.3 capacity-form advection), through the C ABI.

FP64: max |gpu - oracle| / max |oracle| <= 1e-12.  The metrics come from the
same formulas evaluated by CUDA's and the host's math libraries, so unlike
the square domains the ghost fill is not bit-identical (the fine-to-coarse
average is area weighted).  FP32 (FP64 metrics, FP32 field and update):
bounds written per test, measured values printed.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import F64_TOL, pair, relerr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
fc = pytest.importorskip("paper_1703_03116_gb300")


def sphere(seed=0, lmin=1, lmax=3, mx=8):
    return synth.sphere(seed=seed, lmin=lmin, lmax=lmax, mx=mx)


@pytest.mark.parametrize("mx,lmax", [(8, 3), (16, 4), (32, 3)])
def test_fill_ghosts_fp64(mx, lmax):
    w = sphere(1, lmax=lmax, mx=mx)
    ref, gpu = pair(fc, w, fc.F64)
    q = synth.random_field((len(ref), mx, mx), seed=mx)
    ref.set_q(q)
    gpu.set_q(q)
    ref.fill_ghosts()
    gpu.fill_ghosts()
    a, b = gpu.get_q(full=True), ref.get_q_full()
    assert np.all(np.isfinite(a))
    err = relerr(a, b)
    print(f"sphere fill mx={mx}: rel err {err:.2e}")
    assert err <= 1e-14


def test_capacities_sum_to_the_sphere_area():
    w = sphere(2, lmax=4, mx=16)
    ref, gpu = pair(fc, w, fc.F64)
    one = np.ones((len(ref), 16, 16))
    ref.set_q(one)
    gpu.set_q(one)
    m_gpu, m_ref = gpu.mass()[0], ref.mass()[0]
    assert abs(m_gpu - 4 * np.pi) <= 1e-12 * 4 * np.pi
    assert abs(m_gpu - m_ref) <= 1e-13 * m_ref


@pytest.mark.parametrize("dtype,tol", [("f64", F64_TOL), ("f32", 2e-4)])
def test_global_steps(dtype, tol):
    w = sphere(3, lmax=4, mx=16)
    ref, gpu = pair(fc, w, fc.F64 if dtype == "f64" else fc.F32)
    n, dtc = synth.time_step(w)
    dt = dtc / 2 ** (w.lmax - w.lmin)
    for s in range(6):
        ref.step_global(s * dt, dt)
        gpu.step_global(s * dt, dt)
    err = relerr(gpu.get_q(), ref.get_q())
    print(f"sphere global steps {dtype}: rel err {err:.2e}")
    assert err <= tol


@pytest.mark.parametrize("mx,lmax", [(8, 4), (16, 4), (32, 3)])
@pytest.mark.parametrize("variant,warps", [(-1, 4), (0, 4), (3, 4), (3, 16)])
def test_multirate(mx, lmax, variant, warps):
    """The capacity-form update of every kernel that has one: the default
    (band, 8 warps), staged, band with 4 and 16 warps."""
    w = sphere(4, lmax=lmax, mx=mx)
    _, dtc = synth.time_step(w)
    for dtype, tol in ((fc.F64, F64_TOL), (fc.F32, 2e-4)):
        ref, gpu = pair(fc, w, dtype)
        gpu.set_advance_variant(variant, warps)
        for s in range(2):
            ref.step_multirate(s * dtc, dtc)
            gpu.step_multirate(s * dtc, dtc)
        err = relerr(gpu.get_q(), ref.get_q())
        print(f"sphere multirate mx={mx} variant {variant}/{warps} dtype={dtype}: rel err {err:.2e}")
        assert err <= tol
        m_gpu, m_ref = gpu.mass()[0], ref.mass()[0]
        assert abs(m_gpu - m_ref) <= (1e-12 if dtype == fc.F64 else 1e-5) * abs(m_ref)


def test_constant_state_is_preserved():
    w = sphere(5, lmax=4, mx=16)
    _, dtc = synth.time_step(w)
    for dtype, tol in ((fc.F64, 1e-13), (fc.F32, 2e-6)):
        _, gpu = pair(fc, w, dtype)
        gpu.set_q(np.ones((len(gpu), 16, 16)))
        for s in range(2):
            gpu.step_multirate(s * dtc, dtc)
        err = float(np.abs(gpu.get_q() - 1.0).max())
        print(f"sphere constant state dtype={dtype}: max |q - 1| {err:.2e}")
        assert err <= tol


def test_tag_regrid_matches_oracle():
    w = sphere(6, lmax=4, mx=8)
    ref, gpu = pair(fc, w, fc.F64)
    _, dtc = synth.time_step(w)
    for s in range(2):
        ref.step_multirate(s * dtc, dtc)
        gpu.step_multirate(s * dtc, dtc)
    np.testing.assert_allclose(gpu.tag(), ref.tag(), rtol=1e-11, atol=1e-14)
    gpu.tag_regrid(w.tau_refine, w.tau_coarsen)
    ref.regrid(w.tau_refine, w.tau_coarsen)
    assert np.array_equal(gpu.leaves(), ref.leaves())
    assert relerr(gpu.get_q(), ref.get_q()) <= F64_TOL
    # and stepping continues on the new layout (metrics rebuilt)
    ref.step_multirate(2 * dtc, dtc)
    gpu.step_multirate(2 * dtc, dtc)
    assert relerr(gpu.get_q(), ref.get_q()) <= F64_TOL


def test_velocity_scale_rescales_the_fluxes():
    w = sphere(7, lmax=3, mx=8)
    ref, gpu = pair(fc, w, fc.F64)
    ref.set_velocity_scale(-0.6)
    gpu.set_velocity_scale(-0.6)
    _, dtc = synth.time_step(w)
    for s in range(2):
        ref.step_multirate(s * dtc, dtc)
        gpu.step_multirate(s * dtc, dtc)
    assert relerr(gpu.get_q(), ref.get_q()) <= F64_TOL


def test_graphs_and_fused_fill_match_direct_launches():
    w = sphere(8, lmax=4, mx=16)
    _, dtc = synth.time_step(w)
    outs = []
    for graphs, fused in ((False, False), (False, True), (True, True)):
        _, gpu = pair(fc, w, fc.F32)
        gpu.graphs(graphs)
        gpu.fused_fill(fused)
        for s in range(3):
            gpu.step_multirate(s * dtc, dtc)
        outs.append(gpu.get_q())
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])


def test_adjoint_is_refused_on_the_sphere():
    w = sphere(0, lmax=2, mx=8)
    _, gpu = pair(fc, w, fc.F64)
    lam = torch.zeros(len(gpu) * 64, dtype=torch.float64, device="cuda")
    ds = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(fc.FcError):
        gpu.adjoint_step_global(0.0, 1e-3, lam, ds)


def test_full_size_sphere_one_coarse_step():
    """The benchmark's sphere workload (levels 1-7, 32^2 patches) for one
    coarse multirate step (64 finest-level substeps) plus a regrid, compared
    everywhere with the oracle."""
    w = synth.sphere(0)
    _, dtc = synth.time_step(w)
    for dtype, tol in ((fc.F64, F64_TOL), (fc.F32, 2e-4)):
        ref, gpu = pair(fc, w, dtype)
        assert ref.leaves()[:, 2].max() == 7
        ref.step_multirate(0.0, dtc)
        gpu.step_multirate(0.0, dtc)
        err = relerr(gpu.get_q(), ref.get_q())
        m_gpu, m_ref = gpu.mass()[0], ref.mass()[0]
        print(f"full-size sphere dtype {dtype}: {len(ref)} patches, rel err {err:.2e}, "
              f"mass rel diff {abs(m_gpu - m_ref) / abs(m_ref):.2e}")
        assert err <= tol
        if dtype == fc.F64:
            ref.regrid(w.tau_refine, w.tau_coarsen)
            gpu.tag_regrid(w.tau_refine, w.tau_coarsen)
            np.testing.assert_array_equal(gpu.leaves(), ref.leaves())
            assert relerr(gpu.get_q(), ref.get_q()) <= F64_TOL
