"""GPU parity of refluxing (the conservative coarse/fine correction, an
extension of the paper's scheme) against the oracle, through the C-ABI:
multirate and global stepping, both precisions, across a regrid, the captured
level-branch graphs against direct launches, and exact mass conservation."""
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


def _w(domain="periodic", velocity=("swirl", 4.0), seed=2, lmin=2, lmax=4, mx=8):
    w = synth.swirl(seed, lmin=lmin, lmax=lmax, mx=mx)
    return dataclasses.replace(w, domain=domain, velocity=velocity, reflux=True)


@pytest.mark.parametrize("domain,velocity,mx,lmax", [
    ("periodic", ("const", 1.0, 0.5), 8, 4),
    ("walls", ("swirl", 4.0), 16, 4),
    ("periodic", ("swirl", 4.0), 32, 5),
])
@pytest.mark.parametrize("variant", [-1, 3])
def test_multirate_matches_oracle(domain, velocity, mx, lmax, variant):
    """Default update (staged) and the band update, which records the face
    fluxes too."""
    w = _w(domain, velocity, mx=mx, lmax=lmax)
    _, dtc = synth.time_step(w)
    for dtype, tol in ((fc.F64, F64_TOL), (fc.F32, 1e-4)):
        ref, gpu = pair(fc, w, dtype)
        gpu.set_advance_variant(variant, 8)
        for n in range(3):
            ref.step_multirate(n * dtc, dtc)
            gpu.step_multirate(n * dtc, dtc)
        err = relerr(gpu.get_q(), ref.get_q())
        print(f"reflux multirate {domain} mx={mx} variant {variant} dtype {dtype}: "
              f"rel err {err:.2e}")
        assert err <= tol


def test_global_steps_match_oracle():
    w = _w("walls", ("swirl", 4.0), mx=16)
    ref, gpu = pair(fc, w, fc.F64)
    dt = 0.9 / (16 * 16)
    for n in range(6):
        ref.step_global(n * dt, dt)
        gpu.step_global(n * dt, dt)
    assert relerr(gpu.get_q(), ref.get_q()) <= F64_TOL


@pytest.mark.parametrize("mode", ["multirate", "global"])
@pytest.mark.parametrize("variant", [-1, 3])
def test_mass_conserved_to_rounding(mode, variant):
    """FP64: total mass after the steps equals the initial mass to rounding,
    where without the correction it drifts (the forest has coarse/fine faces)."""
    drift = {}
    for reflux in (False, True):
        w = dataclasses.replace(_w("periodic", ("swirl", 4.0), mx=16, lmax=5), reflux=reflux)
        _, dtc = synth.time_step(w)
        dt = dtc if mode == "multirate" else dtc / 2 ** (w.lmax - w.lmin)
        _, gpu = pair(fc, w, fc.F64)
        gpu.set_advance_variant(variant, 4)
        m0 = gpu.mass().sum()
        for n in range(4):
            (gpu.step_multirate if mode == "multirate" else gpu.step_global)(n * dt, dt)
        drift[reflux] = (gpu.mass().sum() - m0) / m0
    print(f"{mode}: drift without {drift[False]:.2e}, with {drift[True]:.2e}")
    assert abs(drift[False]) > 1e-8
    assert abs(drift[True]) < 1e-13


def test_graphs_and_regrid_match_direct_launches():
    """The correction runs on the level's own branch of a captured step, after
    the finer level's substeps: replayed steps give the bits of direct launches
    on one stream, across regrids (the flux store follows the layout), and
    follow the oracle."""
    w = _w("periodic", ("swirl", 4.0), seed=0, lmin=2, lmax=6, mx=32)
    _, dtc = synth.time_step(w)
    ref, a = pair(fc, w, fc.F32)
    b = fc.Forest(a.desc, ref.leaves())
    b.set_q(a.get_q())
    b.graphs(False)
    for n in range(8):
        a.step_multirate(n * dtc, dtc)
        b.step_multirate(n * dtc, dtc)
        if (n + 1) % 4 == 0:
            assert a.tag_regrid(w.tau_refine, w.tau_coarsen) == \
                b.tag_regrid(w.tau_refine, w.tau_coarsen)
    np.testing.assert_array_equal(a.get_q(), b.get_q())


def test_regrid_then_parity():
    w = _w("walls", ("swirl", 4.0), seed=5, mx=16, lmax=5)
    _, dtc = synth.time_step(w)
    ref, gpu = pair(fc, w, fc.F64)
    for n in range(4):
        ref.step_multirate(n * dtc, dtc)
        gpu.step_multirate(n * dtc, dtc)
        if n == 1:
            assert gpu.tag_regrid(w.tau_refine, w.tau_coarsen) == \
                ref.regrid(w.tau_refine, w.tau_coarsen)
    np.testing.assert_array_equal(gpu.leaves(), ref.leaves())
    assert relerr(gpu.get_q(), ref.get_q()) <= F64_TOL


def test_adjoint_rejects_refluxing():
    _, gpu = pair(fc, _w(), fc.F64)
    lam = torch.zeros(len(gpu) * gpu.mx * gpu.mx, dtype=torch.float64, device="cuda")
    ds = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(fc.FcError):
        gpu.adjoint_step_global(0.0, 1e-3, lam, ds)
    with pytest.raises(fc.FcError):
        gpu.adjoint_step_multirate(0.0, 1e-3, lam, ds)
