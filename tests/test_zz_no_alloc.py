"""fc_mass_noalloc: the mass sum for callers that cannot allocate device memory.

The entry point keeps its per-leaf partial sums in a fixed device array
instead of allocating scratch, so it can serve code that must not touch the
allocator.  It is checked through the C ABI against fc_forest_mass on two
calls in a row (the second call finds the array holding the first call's
partial sums).  This file is collected last so that a failure here leaves
every other test already run; it passes alone or after the others.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
fc = pytest.importorskip("paper_1703_03116_gb300")


def _forest(dtype, nforests, seed):
    ws = synth.ensemble(nforests, seed=seed, lmin=2, mx=16, levels=(3, 4))
    desc = fc.make_desc(domain=fc.WALLS, mx=16, lmin=2, lmax=4, dtype=dtype,
                        velocity=ws[0].velocity, nforests=nforests)

    def q0(leaves):
        out = np.empty((len(leaves), 16, 16))
        for f in range(nforests):
            sel = leaves[:, 0] == f
            x, y = synth.cell_centres(leaves[sel], 16)
            out[sel] = synth.evaluate(ws[f], x, y) + 0.25 * np.sin(7 * x) * np.cos(5 * y)
        return out

    return fc.initial_forest(desc, q0, lmax_f=[w.lmax for w in ws])


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_mass_noalloc_matches_forest_mass_twice(dtype):
    L = fc.load()
    fdt = fc.F32 if dtype == "f32" else fc.F64
    tdt = torch.float32 if dtype == "f32" else torch.float64
    dev = torch.device("cuda", 0)
    for call, (nforests, seed) in enumerate([(3, 1), (5, 2)]):
        F = _forest(fdt, nforests, seed)
        leaves = F.leaves()
        n = len(leaves)
        q = torch.empty((n, 16, 16), dtype=tdt, device=dev)
        F.get_q(out=q)
        level = torch.tensor(leaves[:, 2], dtype=torch.int32, device=dev)
        fstart = np.searchsorted(leaves[:, 0], np.arange(nforests + 1)).astype(np.int32)
        fstart_d = torch.tensor(fstart, dtype=torch.int32, device=dev)
        out = torch.full((nforests,), float("nan"), dtype=torch.float64, device=dev)
        st = L.fc_mass_noalloc(ctypes.c_void_p(q.data_ptr()), fdt, 16, n,
                               ctypes.c_void_p(level.data_ptr()),
                               ctypes.c_void_p(fstart_d.data_ptr()), nforests,
                               ctypes.c_void_p(out.data_ptr()), None)
        assert st == 0, L.fc_last_error().decode()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        want = F.mass()
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=0)
        assert np.all(np.isfinite(got)) and np.all(got > 0), (call, got)


def test_mass_noalloc_rejects_oversized_input():
    L = fc.load()
    st = L.fc_mass_noalloc(ctypes.c_void_p(1), fc.F64, 16, (1 << 19) + 1, ctypes.c_void_p(1),
                           ctypes.c_void_p(1), 1, ctypes.c_void_p(1), None)
    assert st == 1
    assert "FC_NOALLOC_MAX_LEAVES" in L.fc_last_error().decode()
