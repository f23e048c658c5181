"""Paths the default launches do not reach, through the C ABI.

- The walk kernels' persistent loop: with the grid capped at a few CTAs every
  warp loops over many groups of patches and its second tile buffer carries
  the prefetched group (walk) or the single buffer is reused (walk1).
  Compared with the FP64 oracle (<= 1e-12) and, in FP32, within the FP32
  multirate bound of the other parity tests (1e-4).
- The bounded wait for a tile copy giving up: with the wait limit at zero
  polls every update kernel gives up at once, waits (with the default limit)
  for its copies in flight and leaves; the next synchronising call reports
  FC_ERR_TIMEOUT, and with the limit restored the same forest steps exactly
  as the oracle does.
- A batched ensemble in FP32 (32 forests of mixed depth in one store, one
  launch per level substep for all) against the FP64 oracle.
"""
import numpy as np
import pytest

import synth
from gpu_helpers import F64_TOL, pair, relerr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
fc = pytest.importorskip("paper_1703_03116_gb300")


@pytest.mark.parametrize("ctas", [1, 3, 7])
@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("mx", [8, 16, 32])
def test_walk_persistent_loop_matches_oracle(ctas, variant, mx):
    ws = synth.ensemble(3, seed=13, lmin=2, mx=mx, levels=(4,) if mx == 32 else (4, 5))
    _, dtc = synth.time_step(ws[0], max(w.lmax for w in ws))
    for dtype, tol in ((fc.F64, F64_TOL), (fc.F32, 1e-4)):
        ref, gpu = pair(fc, ws, dtype)
        gpu.set_advance_variant(variant, 4)
        gpu.set_limits(walk_ctas=ctas)
        for n in range(2):
            ref.step_multirate(n * dtc, dtc)
            gpu.step_multirate(n * dtc, dtc)
        err = relerr(gpu.get_q(), ref.get_q())
        # every warp of the capped grid walked several groups
        groups = len(ref) // (32 // mx)
        print(f"walk variant {variant}, {ctas} CTAs, mx {mx}, dtype {dtype}: {len(ref)} patches "
              f"({groups} groups over {ctas * 4} warps), rel err {err:.2e}")
        assert groups >= 4 * ctas * 4
        assert err <= tol


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_bounded_wait_gives_up_then_recovers(variant):
    w = synth.swirl(2, lmin=2, lmax=4, mx=16)
    _, dtc = synth.time_step(w)
    ref, gpu = pair(fc, w, fc.F64)
    q0 = ref.get_q()
    gpu.set_advance_variant(variant, 4)
    gpu.set_limits(wait_polls=0)
    gpu.step_multirate(0.0, dtc)
    with pytest.raises(fc.FcError) as e:
        gpu.mass()
    assert e.value.status == 5  # FC_ERR_TIMEOUT
    # the error word was cleared by the call that reported it
    gpu.mass()
    gpu.set_limits(wait_polls=-1)
    gpu.set_q(q0)
    for n in range(2):
        ref.step_multirate(n * dtc, dtc)
        gpu.step_multirate(n * dtc, dtc)
    assert relerr(gpu.get_q(), ref.get_q()) <= F64_TOL


def test_batched_ensemble_fp32_matches_oracle():
    ws = synth.ensemble(32, seed=17, lmin=2, mx=16, levels=(3, 4))
    lmax = max(w.lmax for w in ws)
    _, dtc = synth.time_step(ws[0], lmax)
    lmax_f = [w.lmax for w in ws]
    ref, gpu = pair(fc, ws, fc.F32)
    assert len(set(lmax_f)) == 2 and len(ref) > 32 * 16
    gpu.autotune()
    for n in range(2):
        ref.step_multirate(n * dtc, dtc)
        gpu.step_multirate(n * dtc, dtc)
    err = relerr(gpu.get_q(), ref.get_q())
    print(f"batched FP32 ensemble: {len(ref)} patches in 32 forests, rel err {err:.2e}")
    assert err <= 1e-4
    ref.regrid(0.05, 0.0125, lmax_f)
    gpu.tag_regrid(0.05, 0.0125, lmax_f)
    # FP32 indicators may decide a leaf within rounding of a threshold
    # differently; the layouts agree on almost every leaf
    a = {tuple(r) for r in gpu.leaves()}
    b = {tuple(r) for r in ref.leaves()}
    assert len(a ^ b) <= 0.01 * len(b)
