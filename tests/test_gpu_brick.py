"""The brick domain on the GPU (Sec. 5.1's replicated problem: a periodic
brick of unit blocks joined face to face) against the oracle, through the C
ABI: the ghost fill across block faces bit for bit, global steps (the
paper's runs) and multirate steps with the graded spread regrid, FP64 within
1e-12 and FP32 within the FP32 bound of the square-domain tests; and every
block of the GPU's brick equal, bit for bit, to the GPU's single periodic
block (each block runs the same problem)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import F64_TOL, desc_for, pair, relerr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
fc = pytest.importorskip("paper_1703_03116_gb300")


@pytest.mark.parametrize("mx", [8, 16, 32])
def test_brick_fill_ghosts_bitwise(mx):
    w = synth.brick(seed=2, n=1, lmin=2, lmax=4 if mx < 32 else 3, mx=mx)
    ref, gpu = pair(fc, w, fc.F64)
    q = synth.random_field((len(ref), mx, mx), seed=mx)
    ref.set_q(q)
    gpu.set_q(q)
    ref.fill_ghosts()
    gpu.fill_ghosts()
    np.testing.assert_array_equal(gpu.get_q(full=True), ref.get_q_full())


@pytest.mark.parametrize("mode", ["global", "multirate"])
def test_brick_steps_and_regrid_match_oracle(mode):
    w = synth.brick(seed=5, n=1, lmin=2, lmax=4, mx=16)
    dtf = w.cfl / (w.mx * 2 ** w.lmax) / 0.5  # finest-level step at CFL 0.64
    for dtype, tol in ((fc.F64, F64_TOL), (fc.F32, 1e-4)):
        ref, gpu = pair(fc, w, dtype)
        for k in range(8):
            if mode == "global":
                ref.step_global(k * dtf, dtf)
                gpu.step_global(k * dtf, dtf)
            else:
                dtc = dtf * 2 ** (w.lmax - w.lmin)
                ref.step_multirate(k * dtc, dtc)
                gpu.step_multirate(k * dtc, dtc)
            if k == 3 and dtype == fc.F64:
                ref.regrid(w.tau_refine, w.tau_coarsen)
                gpu.tag_regrid(w.tau_refine, w.tau_coarsen)
                np.testing.assert_array_equal(gpu.leaves(), ref.leaves())
        err = relerr(gpu.get_q(), ref.get_q())
        print(f"brick {mode} dtype {dtype}: {len(ref)} leaves, rel err {err:.2e}")
        assert err <= tol


def test_every_block_runs_the_single_block_problem():
    w = synth.brick(seed=7, n=1, lmin=2, lmax=5, mx=16)
    w1 = synth.brick(seed=7, n=0, lmin=2, lmax=5, mx=16)
    w1.domain = "periodic"
    B = oracle.initial_forest(w)
    S = oracle.initial_forest(w1)
    gb = fc.Forest(desc_for(fc, w, fc.F32), B.leaves())
    gs = fc.Forest(desc_for(fc, w1, fc.F32), S.leaves())
    gb.set_q(B.get_q())
    gs.set_q(S.get_q())
    dtc = w.cfl / (w.mx * 2 ** w.lmax) / 0.5 * 2 ** (w.lmax - w.lmin)
    for k in range(8):
        gb.step_multirate(k * dtc, dtc)
        gs.step_multirate(k * dtc, dtc)
        if (k + 1) % 4 == 0:
            gb.tag_regrid(w.tau_refine, w.tau_coarsen)
            gs.tag_regrid(w.tau_refine, w.tau_coarsen)
    lb, qb = gb.leaves(), gb.get_q()
    ls, qs = gs.leaves(), gs.get_q()
    for b in range(4):
        sel = lb[:, 1] == b
        np.testing.assert_array_equal(lb[sel][:, 2:], ls[:, 2:])
        np.testing.assert_array_equal(qb[sel], qs)
