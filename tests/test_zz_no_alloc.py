"""fc_mass_noalloc: the mass sum for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc at the point where they need a mass sum:
code running inside an allocator callback, a process whose device memory is
owned by another runtime, a driver loop that must not touch the allocator.
The entry point keeps its per-leaf partial sums in a fixed device array
instead of allocating scratch.  It is checked through the C ABI against
fc_forest_mass and against an FP64 sum of the same field on the host, on two
calls in a row: the first covers more leaves than the second, so the second
finds partial sums of the first beyond its own leaves, which it must not
read.  On the cubed sphere it is given the capacities and must reproduce the
capacity-weighted mass.  This file is collected last so that a failure here
leaves every other test already run; it passes alone or after the others.
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


def _call(L, q, cap, fdt, mx, leaves, nforests, dev):
    n = len(leaves)
    level = torch.tensor(leaves[:, 2], dtype=torch.int32, device=dev)
    fstart = np.searchsorted(leaves[:, 0], np.arange(nforests + 1)).astype(np.int32)
    fstart_d = torch.tensor(fstart, dtype=torch.int32, device=dev)
    out = torch.full((nforests,), float("nan"), dtype=torch.float64, device=dev)
    st = L.fc_mass_noalloc(ctypes.c_void_p(q.data_ptr()),
                           ctypes.c_void_p(cap.data_ptr()) if cap is not None else None,
                           fdt, mx, n, ctypes.c_void_p(level.data_ptr()),
                           ctypes.c_void_p(fstart_d.data_ptr()), nforests,
                           ctypes.c_void_p(out.data_ptr()), None)
    assert st == 0, L.fc_last_error().decode()
    torch.cuda.synchronize()
    return out.cpu().numpy(), fstart


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_mass_noalloc_matches_forest_mass_twice(dtype):
    L = fc.load()
    fdt = fc.F32 if dtype == "f32" else fc.F64
    tdt = torch.float32 if dtype == "f32" else torch.float64
    dev = torch.device("cuda", 0)
    # the larger case first: the second call's leaves end before the first's
    for call, (nforests, seed) in enumerate([(5, 2), (3, 1)]):
        F = _forest(fdt, nforests, seed)
        leaves = F.leaves()
        q = torch.empty((len(leaves), 16, 16), dtype=tdt, device=dev)
        F.get_q(out=q)
        got, fstart = _call(L, q, None, fdt, 16, leaves, nforests, dev)
        np.testing.assert_allclose(got, F.mass(), rtol=1e-13, atol=0)
        # an FP64 sum on the host of the same field: h^2 sum q per forest
        qh = q.cpu().numpy().astype(np.float64)
        h = 1.0 / (16 * (1 << leaves[:, 2].astype(np.int64)))
        per_leaf = h * h * qh.reshape(len(leaves), -1).sum(axis=1)
        want = np.array([per_leaf[fstart[f]:fstart[f + 1]].sum() for f in range(nforests)])
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=0)
        assert np.all(np.isfinite(got)) and np.all(got > 0), (call, got)


def test_mass_noalloc_on_the_sphere_with_capacities():
    """The cubed sphere's mass is sum kappa q; with the forest's capacities the
    call gives fc_forest_mass's number, and without them the h^2 sum differs."""
    L = fc.load()
    dev = torch.device("cuda", 0)
    w = synth.sphere(seed=0, lmin=1, lmax=3, mx=16)
    desc = fc.make_desc(domain=fc.SPHERE, mx=16, lmin=1, lmax=3, dtype=fc.F64,
                        velocity=w.velocity)

    def q0(leaves):
        return synth.evaluate_sphere(w, synth.sphere_cell_centres(leaves, 16)) + 0.5

    F = fc.initial_forest(desc, q0, tau_r=w.tau_refine, tau_c=w.tau_coarsen)
    leaves = F.leaves()
    n = len(leaves)
    q = torch.empty((n, 16, 16), dtype=torch.float64, device=dev)
    F.get_q(out=q)
    cap = torch.empty((n, 16, 16), dtype=torch.float64, device=dev)
    F.capacity(out=cap)
    want = F.mass()
    for _ in range(2):
        got, _ = _call(L, q, cap, fc.F64, 16, leaves, 1, dev)
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=0)
    # the capacities tile the unit sphere: their sum is its area
    assert abs(cap.sum().item() - 4 * np.pi) < 1e-10
    flat, _ = _call(L, q, None, fc.F64, 16, leaves, 1, dev)
    assert abs(flat[0] - want[0]) > 1e-6 * abs(want[0])


def test_mass_noalloc_clamps_a_malformed_forest_table():
    """forest_start entries outside [0, nleaves] are clamped: a table reaching
    past the leaves sums exactly the leaves there are."""
    L = fc.load()
    dev = torch.device("cuda", 0)
    F = _forest(fc.F64, 2, 3)
    leaves = F.leaves()
    n = len(leaves)
    q = torch.empty((n, 16, 16), dtype=torch.float64, device=dev)
    F.get_q(out=q)
    level = torch.tensor(leaves[:, 2], dtype=torch.int32, device=dev)
    fstart_d = torch.tensor([-5, n + 1000], dtype=torch.int32, device=dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    st = L.fc_mass_noalloc(ctypes.c_void_p(q.data_ptr()), None, fc.F64, 16, n,
                           ctypes.c_void_p(level.data_ptr()), ctypes.c_void_p(fstart_d.data_ptr()),
                           1, ctypes.c_void_p(out.data_ptr()), None)
    assert st == 0, L.fc_last_error().decode()
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy()[0], F.mass().sum(), rtol=1e-13)


def test_mass_noalloc_rejects_oversized_input():
    L = fc.load()
    st = L.fc_mass_noalloc(ctypes.c_void_p(1), None, fc.F64, 16, (1 << 19) + 1,
                           ctypes.c_void_p(1), ctypes.c_void_p(1), 1, ctypes.c_void_p(1), None)
    assert st == 1
    assert "FC_NOALLOC_MAX_LEAVES" in L.fc_last_error().decode()
