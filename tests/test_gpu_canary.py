"""Executable Prop. 1 (Sec. 2.3) on the device: every cell an update's
stencil reads is set by a rule of Alg. 1 before it is read.  Before every
coarse step (and before a regrid) every ghost cell of both state buffers and
every cell of the time-interpolation tiles is set to NaN (fc_forest_poison);
the steps must still match the oracle to FP64 tolerance with no NaN anywhere.
Covers the fused gathers of the staged and band updates (ghosts in shared
memory, the coarse neighbours' time-interpolated cells computed from the
sources listed in the neighbour entries), separate fill kernels, the walk,
and the regrid's remap (its tag fills the ghosts first)."""
import numpy as np
import pytest

import synth
from gpu_helpers import F64_TOL, pair, relerr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
fc = pytest.importorskip("paper_1703_03116_gb300")

NAN = float("nan")


def _run(w, variant, fused, steps=4, regrid_at=(1,)):
    ref, gpu = pair(fc, w, fc.F64)
    if variant >= 0:
        gpu.set_advance_variant(variant, 4)
    gpu.fused_fill(fused)
    _, dtc = synth.time_step(w)
    for n in range(steps):
        gpu.poison(NAN)
        ref.step_multirate(n * dtc, dtc)
        gpu.step_multirate(n * dtc, dtc)
        if n in regrid_at:
            gpu.poison(NAN)
            assert ref.regrid(w.tau_refine, w.tau_coarsen) == gpu.tag_regrid(w.tau_refine,
                                                                              w.tau_coarsen)
    q = gpu.get_q()
    assert np.isfinite(q).all()
    assert relerr(q, ref.get_q()) <= F64_TOL


@pytest.mark.parametrize("domain", ["walls", "periodic"])
@pytest.mark.parametrize("variant,fused", [(3, True), (0, True), (1, True), (3, False)])
def test_square_domains_read_only_filled_cells(domain, variant, fused):
    w = synth.swirl(4, lmin=2, lmax=4, mx=16)
    w.domain = domain
    _run(w, variant, fused)


@pytest.mark.parametrize("variant,fused", [(3, True), (0, True), (3, False)])
def test_sphere_reads_only_filled_cells(variant, fused):
    w = synth.sphere(seed=2, lmin=1, lmax=3, mx=8)
    _run(w, variant, fused, steps=3)


def test_full_size_swirl_reads_only_filled_cells():
    """The benchmark's forest (levels 2-6, 32^2), default kernel choice."""
    _run(synth.swirl(0), -1, True, steps=2, regrid_at=(0,))
