"""One forest partitioned over ranks (Sec. 3), emulated on one GPU: k parts,
each with its own patch store holding its leaves and mirrors, stepped level
substep by level substep with a halo exchange after each (pack on the owner,
unpack on the receiver), must give every leaf the same bits as the
unpartitioned forest -- multirate (Sec. 4) and global stepping, FP64 and
FP32, walls, periodic and the cubed sphere -- and the parts' masses must add
up to the whole forest's.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import desc_for

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
fc = pytest.importorskip("paper_1703_03116_gb300")
from paper_1703_03116_gb300.partition import VirtualPartitions  # noqa: E402


def _workload(kind):
    if kind == "walls":
        return synth.swirl(3, lmin=2, lmax=5, mx=16)
    if kind == "periodic":
        w = synth.swirl(4, lmin=2, lmax=5, mx=16)
        w.domain = "periodic"
        return w
    return synth.sphere(seed=2, lmin=1, lmax=4, mx=16)


def _pair(kind, dtype, nparts, variant):
    w = _workload(kind)
    ref = oracle.initial_forest(w)
    lv = ref.leaves()
    q0 = ref.get_q()
    if dtype == fc.F32:
        q0 = q0.astype(np.float32)
    whole = fc.Forest(desc_for(fc, w, dtype), lv)
    whole.set_q(q0)
    whole.graphs(False)  # direct launches, the same kernels the parts run
    vp = VirtualPartitions(desc_for(fc, w, dtype), lv, nparts)
    vp.set_q(q0)
    for F in [whole] + vp.parts:
        F.set_advance_variant(variant, 4)
    return w, lv, whole, vp


@pytest.mark.parametrize("kind", ["walls", "periodic", "sphere"])
@pytest.mark.parametrize("nparts", [2, 3, 4])
def test_partitioned_multirate_is_bitwise_the_whole_forest(kind, nparts):
    for dtype in (fc.F64, fc.F32):
        w, lv, whole, vp = _pair(kind, dtype, nparts, 0)
        assert sorted(np.unique(vp.part)) == list(range(nparts))
        _, dtc = synth.time_step(w)
        for n in range(2):
            whole.step_multirate(n * dtc, dtc)
            vp.step_multirate(n * dtc, dtc)
        a, b = vp.get_q(), whole.get_q()
        np.testing.assert_array_equal(a, b)
        np.testing.assert_allclose(vp.mass(), whole.mass(), rtol=1e-13)
        counts = [p.halo_count(q, -1) for p in vp.parts for q in range(nparts)
                  if q != p.rank]
        print(f"{kind} {nparts} parts dtype {dtype}: {len(lv)} leaves, owned "
              f"{[len(p) for p in vp.parts]}, exchanged per substep set {counts}")
        vp.close()


@pytest.mark.parametrize("variant", [0, 1, 3])
def test_partitioned_global_steps_are_bitwise_the_whole_forest(variant):
    w, lv, whole, vp = _pair("walls", fc.F64, 3, variant)
    dt = 0.9 / (16 * 2 ** 5)
    for n in range(4):
        whole.step_global(n * dt, dt)
        vp.step_global(n * dt, dt)
    np.testing.assert_array_equal(vp.get_q(), whole.get_q())
    vp.close()


@pytest.mark.parametrize("kind", ["walls", "periodic"])
def test_partitioned_band_multirate_is_bitwise_the_whole_forest(kind):
    w, lv, whole, vp = _pair(kind, fc.F32, 3, 3)
    _, dtc = synth.time_step(w)
    for n in range(2):
        whole.step_multirate(n * dtc, dtc)
        vp.step_multirate(n * dtc, dtc)
    np.testing.assert_array_equal(vp.get_q(), whole.get_q())
    vp.close()


def test_partition_rejects_what_it_does_not_build():
    w = _workload("walls")
    ref = oracle.initial_forest(w)
    vp = VirtualPartitions(desc_for(fc, w, fc.F64), ref.leaves(), 2)
    vp.set_q(ref.get_q())
    p = vp.parts[0]
    with pytest.raises(fc.FcError):
        p.step_multirate(0.0, 0.01)
    with pytest.raises(fc.FcError):
        p.tag_regrid(0.05, 0.0125)
    assert len(p) == int(np.sum(vp.part == 0))
    assert p.info()["nleaves"] == len(p)
    vp.close()
