"""C-ABI calls of the boundary beyond stepping: the per-level adjoint
(fc_adjoint_advance), the forest summary (fc_forest_info) and the pluggable
device allocator (fc_set_allocator).

- fc_adjoint_advance is the transpose of one fc_advance_level call.  Chained
  in reverse over the substeps of a coarse multirate step (Sec. 4's
  coarse-first recursion), each from the forward state right before it, it
  must give the oracle's adjoint of the whole coarse step (FP64, field-
  normalised error <= 1e-12; only the order of the atomic sums differs).
- fc_set_allocator routes every device allocation through the caller's
  functions: with torch's caching allocator the results are bit-identical to
  the default pool's, every block comes back, and torch accounts the memory.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import F64_TOL, desc_for, relerr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
fc = pytest.importorskip("paper_1703_03116_gb300")

DEV = torch.device("cuda", 0)


def _substeps(lmin, lmax, t0, dtc):
    out = []

    def rec(L, t, dt):
        out.append((L, t, dt))
        if L < lmax:
            rec(L + 1, t, 0.5 * dt)
            rec(L + 1, t + 0.5 * dt, 0.5 * dt)

    rec(lmin, t0, dtc)
    return out


def _case(mx, lmax, seed=3):
    w = synth.swirl(seed, lmin=2, lmax=lmax, mx=mx)
    ref = oracle.initial_forest(w)
    x, y = synth.cell_centres(ref.leaves(), mx)
    q0 = synth.evaluate(synth.smooth_periodic(1), x, y) + 0.3 * np.sin(3 * x + 1) * np.cos(2 * y)
    ref.set_q(q0)
    return w, ref, q0


@pytest.mark.parametrize("mx,lmax", [(8, 4), (16, 4), (32, 3)])
def test_adjoint_advance_chained_over_a_coarse_step_matches_oracle(mx, lmax):
    w, ref, q0 = _case(mx, lmax)
    lv = ref.leaves()
    F = fc.Forest(desc_for(fc, w, fc.F64), lv)
    lam0 = synth.random_field(q0.shape, seed=11) - 0.5
    t0, dtc = 0.3, 0.9 / (mx * 2 ** lmax) * 2 ** (lmax - 2)
    lam_ref, ds_ref = ref.adjoint_step_multirate(t0, dtc, lam0)
    subs = _substeps(w.lmin, lmax, t0, dtc)
    q0d = torch.tensor(q0, dtype=torch.float64, device=DEV)
    lam = torch.tensor(lam0, dtype=torch.float64, device=DEV)
    lam_old = torch.zeros_like(lam)
    ds = torch.zeros(1, dtype=torch.float64, device=DEV)
    level = torch.tensor(lv[:, 2], device=DEV)
    for k in reversed(range(len(subs))):
        F.set_q(q0d)  # replay the forward to the state right before substep k
        for (L, t, dt) in subs[:k]:
            F.advance_level(L, t, dt)
        before = torch.empty_like(lam)
        F.get_q(out=before)
        L, t, dt = subs[k]
        F.adjoint_advance(L, t, dt, lam, lam_old, ds)
        after = torch.empty_like(lam)
        F.get_q(out=after)
        assert torch.equal(before, after)  # the forest is not advanced
        # level L's older state is its state before this substep
        sel = level == L
        lam[sel] += lam_old[sel]
        lam_old[sel] = 0
    err = relerr(lam.cpu().numpy(), lam_ref)
    print(f"chained fc_adjoint_advance, mx={mx}, {len(subs)} substeps: rel err {err:.2e}")
    assert err <= F64_TOL
    assert abs(float(ds) - ds_ref) <= 1e-12 * abs(ds_ref)
    assert float(lam_old.abs().max()) == 0.0


def test_adjoint_advance_rejects_missing_lam_old():
    w, ref, q0 = _case(8, 3)
    F = fc.Forest(desc_for(fc, w, fc.F64), ref.leaves())
    F.set_q(q0)
    dtc = 0.9 / (8 * 8) * 2
    F.advance_level(2, 0.0, dtc)  # level 3 now reads level 2 through the time interpolation
    lam = torch.zeros((len(F), 8, 8), dtype=torch.float64, device=DEV)
    ds = torch.zeros(1, dtype=torch.float64, device=DEV)
    with pytest.raises(fc.FcError):
        F.adjoint_advance(3, 0.0, 0.5 * dtc, lam, None, ds)


def test_forest_info_reports_levels_memory_graphs_and_tuning():
    w = synth.swirl(0, lmin=2, lmax=5, mx=16)
    ref = oracle.initial_forest(w)
    lv = ref.leaves()
    F = fc.Forest(desc_for(fc, w, fc.F32), lv)
    F.set_q(ref.get_q())
    i = F.info()
    assert i["nleaves"] == len(lv) and i["nforests"] == 1 and i["mx"] == 16
    assert (i["lmin"], i["lmax"], i["dtype"], i["domain"]) == (2, 5, fc.F32, fc.WALLS)
    want = np.bincount(lv[:, 2], minlength=21)
    assert i["leaves_per_level"] == list(want[:21])
    assert i["device_bytes"] >= 4 * len(lv) * 20 * 20 * 4
    assert i["graphs"] == 0 and i["tuned_buckets"] == 0
    F.autotune()
    _, dtc = synth.time_step(w)
    F.step_multirate(0.0, dtc)
    i2 = F.info()
    assert i2["graphs"] >= 1 and i2["tuned_buckets"] >= 1


def _run(dtype):
    """Layout, steps, a regrid and a multirate adjoint step; returns the results."""
    w = synth.swirl(1, lmin=2, lmax=4, mx=16)
    ref = oracle.initial_forest(w)
    F = fc.Forest(desc_for(fc, w, dtype), ref.leaves())
    F.set_q(ref.get_q())
    _, dtc = synth.time_step(w)
    for n in range(3):
        F.step_multirate(n * dtc, dtc)
    F.tag_regrid(w.tau_refine, w.tau_coarsen)
    F.step_multirate(3 * dtc, dtc)
    tdt = torch.float32 if dtype == fc.F32 else torch.float64
    q = torch.empty((len(F), 16, 16), dtype=tdt, device=DEV)
    F.get_q(out=q)
    lam = q.clone()
    ds = torch.zeros(1, dtype=torch.float64, device=DEV)
    F.adjoint_step_multirate(4 * dtc, dtc, lam, ds)
    out = (F.leaves(), q.cpu().numpy(), float(ds))
    F.close()
    del F
    torch.cuda.synchronize()
    return out


def test_allocator_hook_with_torch_caching_allocator():
    base = _run(fc.F64)
    alloc, release = fc.torch_allocator()
    seen = {"alloc": 0, "free": 0, "live": 0, "peak": 0}

    def a(nbytes, stream):
        p = alloc(nbytes, stream)
        seen["alloc"] += 1
        seen["live"] += nbytes
        seen["peak"] = max(seen["peak"], torch.cuda.memory_allocated())
        return p

    def r(ptr, nbytes, stream):
        seen["free"] += 1
        seen["live"] -= nbytes
        release(ptr, nbytes, stream)

    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    fc.set_allocator(a, r)
    try:
        hooked = _run(fc.F64)
    finally:
        fc.set_allocator()
    assert seen["alloc"] > 10 and seen["alloc"] == seen["free"] and seen["live"] == 0
    # torch saw the library's memory while the forest lived, and got it all back
    assert seen["peak"] > before + 4 * 100 * 20 * 20 * 8
    assert torch.cuda.memory_allocated() == before
    np.testing.assert_array_equal(hooked[0], base[0])
    np.testing.assert_array_equal(hooked[1], base[1])
    assert hooked[2] == base[2] or abs(hooked[2] - base[2]) <= 1e-13 * abs(base[2])


def test_allocator_cannot_change_while_a_forest_lives():
    w = synth.swirl(0, lmin=2, lmax=3, mx=8)
    F = fc.Forest(desc_for(fc, w, fc.F64), oracle.uniform_leaves(2))
    alloc, release = fc.torch_allocator()
    with pytest.raises(fc.FcError):
        fc.set_allocator(alloc, lambda p, n, s: release(p, n, s))
    F.close()
    fc.set_allocator()  # no forest: accepted


@pytest.mark.parametrize("domain", ["walls", "periodic", "sphere", "brick"])
@pytest.mark.parametrize("mx", [8, 32])
def test_every_coarse_region_lists_its_coarse_ghosts(domain, mx):
    """The update reads the ghosts of a coarser neighbour that its
    interpolation reaches from sources listed in the region's entry (written
    on the device after each upload); a region whose list is incomplete
    falls back to the coarse neighbour's own entries (same values, a longer
    read chain).  On random graded layouts of every domain kind, and after a
    regrid of the swirl forest, no region falls back."""
    rng = np.random.default_rng(5)
    nb = {"walls": 1, "periodic": 1, "sphere": 6, "brick": 4}[domain]
    dom = {"walls": fc.WALLS, "periodic": fc.PERIODIC, "sphere": fc.SPHERE, "brick": fc.BRICK}[domain]
    vel = ("rotation", 0.0, 0.0, 1.0) if domain == "sphere" else ("swirl", 1.0)
    kw = {"brick": (2, 2)} if domain == "brick" else {}  # noqa: E501
    desc = fc.make_desc(domain=dom, mx=mx, lmin=1, lmax=5, dtype=fc.F32, velocity=vel, **kw)
    lv = fc.uniform_leaves(1, 1, nb)
    for _ in range(6):
        lv = fc.layout_regrid(desc, lv, rng.random(len(lv)), 0.55, 0.1)
    F = fc.Forest(desc, lv)
    i = F.info()
    assert i["coarse_entries"] > 0 and i["coarse_unlisted"] == 0, i


def test_swirl_forest_lists_its_coarse_ghosts_after_regrids():
    w = synth.swirl(0)
    ref = oracle.initial_forest(w)
    F = fc.Forest(desc_for(fc, w, fc.F32), ref.leaves())
    F.set_q(ref.get_q())
    _, dtc = synth.time_step(w)
    for n in range(8):
        F.step_multirate(n * dtc, dtc)
        if (n + 1) % 4 == 0:
            F.tag_regrid(w.tau_refine, w.tau_coarsen)
            i = F.info()
            assert i["coarse_entries"] > 0 and i["coarse_unlisted"] == 0, i
