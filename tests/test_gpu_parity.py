"""Parity of the CUDA path with the FP64 oracle, through the C ABI.

FP64: max |gpu - oracle| / max |oracle| <= 1e-12 (the only differences are
rounding order and fused multiply-adds).  FP32: the same measure against the
FP64 oracle started from the same FP32-rounded data; the bound for each case
is written in the test and the measured value is printed.
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


@pytest.mark.parametrize("mx", [8, 16, 32])
@pytest.mark.parametrize("domain", ["walls", "periodic"])
def test_fill_ghosts_bitwise_fp64(mx, domain):
    """Alg. 1 on an adaptive layout: copy, average and interpolate take the
    same operations in the same order on both sides -> identical bits."""
    w = synth.swirl(3, lmin=2, lmax=5 if mx < 32 else 4, mx=mx)
    w.domain = domain
    ref, gpu = pair(fc, w, fc.F64)
    n = len(ref)
    q = synth.random_field((n, mx, mx), seed=mx)
    ref.set_q(q)
    gpu.set_q(q)
    ref.fill_ghosts()
    gpu.fill_ghosts()
    a, b = gpu.get_q(full=True), ref.get_q_full()
    assert np.all(np.isfinite(a))
    np.testing.assert_array_equal(a, b)


def test_fill_ghosts_fp32():
    w = synth.swirl(5, lmin=2, lmax=5, mx=16)
    ref, gpu = pair(fc, w, fc.F32)
    q = synth.random_field((len(ref), 16, 16), seed=2).astype(np.float32)
    ref.set_q(q.astype(np.float64))
    gpu.set_q(q)
    ref.fill_ghosts()
    gpu.fill_ghosts()
    err = relerr(gpu.get_q(full=True), ref.get_q_full())
    print(f"fp32 ghost fill rel err {err:.2e}")
    assert err <= 2e-7


@pytest.mark.parametrize("seed", [0, 1])
def test_uniform_periodic_100_steps(seed):
    """Uniform periodic level-3 forest of 16^2 patches, (u,v) = (1, 0.5),
    MC + transverse corrections, CFL 0.9, 100 global steps."""
    w = synth.uniform_periodic(seed)
    for dtype, tol in ((fc.F64, F64_TOL), (fc.F32, 2e-5)):
        ref, gpu = pair(fc, w, dtype)
        dt = w.cfl / 128
        for n in range(w.steps):
            ref.step_global(n * dt, dt)
            gpu.step_global(n * dt, dt)
        err = relerr(gpu.get_q(), ref.get_q())
        print(f"uniform periodic seed {seed} dtype {dtype}: rel err {err:.2e}")
        assert err <= tol


@pytest.mark.parametrize("mx,lmax", [(8, 5), (16, 4), (32, 4)])
def test_swirl_multirate(mx, lmax):
    w = synth.swirl(2, lmin=2, lmax=lmax, mx=mx)
    _, dtc = synth.time_step(w)
    for dtype, tol in ((fc.F64, F64_TOL), (fc.F32, 1e-4)):
        ref, gpu = pair(fc, w, dtype)
        for n in range(3):
            ref.step_multirate(n * dtc, dtc)
            gpu.step_multirate(n * dtc, dtc)
        err = relerr(gpu.get_q(), ref.get_q())
        print(f"swirl multirate mx={mx} lmax={lmax} dtype {dtype}: rel err {err:.2e}")
        assert np.all(np.isfinite(gpu.get_q()))
        assert err <= tol


def test_swirl_global_steps():
    w = synth.swirl(7, lmin=2, lmax=4, mx=16)
    ref, gpu = pair(fc, w, fc.F64)
    dt = 0.9 / (16 * 16)
    for n in range(8):
        ref.step_global(n * dt, dt)
        gpu.step_global(n * dt, dt)
    assert relerr(gpu.get_q(), ref.get_q()) <= F64_TOL


@pytest.mark.parametrize("scheme", [dict(limiter="none"), dict(limiter="first"),
                                    dict(transverse=0), dict(transverse=1)])
def test_scheme_options(scheme):
    w = synth.swirl(4, lmin=2, lmax=4, mx=8)
    for k, v in scheme.items():
        setattr(w, k, v)
    ref, gpu = pair(fc, w, fc.F64)
    dt = 0.45 / (8 * 16)   # transverse=0 needs CFL <= 1/2
    for n in range(4):
        ref.step_global(n * dt, dt)
        gpu.step_global(n * dt, dt)
    assert relerr(gpu.get_q(), ref.get_q()) <= F64_TOL


def test_tag_and_regrid_match_oracle():
    w = synth.swirl(1, lmin=2, lmax=5, mx=16)
    ref, gpu = pair(fc, w, fc.F64)
    _, dtc = synth.time_step(w)
    for n in range(2):
        ref.step_multirate(n * dtc, dtc)
        gpu.step_multirate(n * dtc, dtc)
    np.testing.assert_allclose(gpu.tag(), ref.tag(), rtol=1e-12, atol=1e-14)
    c_ref = ref.regrid(w.tau_refine, w.tau_coarsen)
    c_gpu = gpu.tag_regrid(w.tau_refine, w.tau_coarsen)
    assert c_gpu == c_ref and c_gpu > 0
    np.testing.assert_array_equal(gpu.leaves(), ref.leaves())
    assert relerr(gpu.get_q(), ref.get_q()) <= F64_TOL


def test_tag_in_single_precision_matches_oracle():
    """FP32 fields: the indicator is computed in FP32 (the square root of the
    patch maximum in FP64); it follows the FP64 oracle to the field's error."""
    w = synth.swirl(1, lmin=2, lmax=5, mx=16)
    ref, gpu = pair(fc, w, fc.F32)
    _, dtc = synth.time_step(w)
    for n in range(2):
        ref.step_multirate(n * dtc, dtc)
        gpu.step_multirate(n * dtc, dtc)
    t_ref, t_gpu = ref.tag(), gpu.tag()
    assert np.abs(t_gpu - t_ref).max() <= 1e-4 * np.abs(t_ref).max()
    assert np.array_equal(t_gpu > w.tau_refine, t_ref > w.tau_refine) or \
        np.min(np.abs(t_ref - w.tau_refine)) < 1e-4 * np.abs(t_ref).max()


@pytest.mark.parametrize("domain", ["walls", "periodic"])
def test_graded_spread_regrid_matches_oracle(domain):
    """The paper's regrid policy on the device (spread indicator, Sec. 5.1;
    smooth grading, Sec. 3.3): the same indicators as the oracle, the same
    layouts, and stepping continues alike, over three regrids."""
    w = synth.swirl(2, lmin=2, lmax=5, mx=16)
    w.domain, w.indicator, w.smooth = domain, "maxmin", True
    ref, gpu = pair(fc, w, fc.F64)
    _, dtc = synth.time_step(w)
    for n in range(6):
        ref.step_multirate(n * dtc, dtc)
        gpu.step_multirate(n * dtc, dtc)
        if n % 2 == 1:
            # a spread is the difference of two field values, each within the
            # field's tolerance: its error bound is absolute
            atol = 2 * F64_TOL * np.abs(ref.get_q()).max()
            np.testing.assert_allclose(gpu.tag(), ref.tag(), rtol=1e-12, atol=atol)
            c_ref = ref.regrid(0.3, 0.02)
            c_gpu = gpu.tag_regrid(0.3, 0.02)
            assert c_gpu == c_ref
            np.testing.assert_array_equal(gpu.leaves(), ref.leaves())
    assert relerr(gpu.get_q(), ref.get_q()) <= F64_TOL


def test_mass_matches_oracle():
    w = synth.swirl(0, lmin=2, lmax=5, mx=16)
    ref, gpu = pair(fc, w, fc.F64)
    m_ref, m_gpu = ref.mass(), gpu.mass()
    assert abs(m_gpu[0] - m_ref[0]) <= 1e-14 * abs(m_ref[0])


def test_batched_forests():
    ws = synth.ensemble(6, seed=11, lmin=2, mx=16, levels=(3, 4, 5))
    _, dtc = synth.time_step(ws[0], 5)
    ref, gpu = pair(fc, ws, fc.F64)
    lmax_f = [w.lmax for w in ws]
    for n in range(4):
        ref.step_multirate(n * dtc, dtc)
        gpu.step_multirate(n * dtc, dtc)
    assert relerr(gpu.get_q(), ref.get_q()) <= F64_TOL
    ref.regrid(0.05, 0.0125, lmax_f)
    gpu.tag_regrid(0.05, 0.0125, lmax_f)
    np.testing.assert_array_equal(gpu.leaves(), ref.leaves())
    np.testing.assert_allclose(gpu.mass(), ref.mass(), rtol=1e-13)


def test_single_patch_and_empty_levels():
    """One periodic patch (its own neighbour in every direction), and a run
    whose level range includes levels with no patches."""
    w = synth.uniform_periodic(0, level=0, mx=8, steps=10)
    ref, gpu = pair(fc, w, fc.F64)
    assert len(ref) == 1
    for n in range(10):
        ref.step_global(n * 0.9 / 8, 0.9 / 8)
        gpu.step_global(n * 0.9 / 8, 0.9 / 8)
    assert relerr(gpu.get_q(), ref.get_q()) <= F64_TOL
    w = synth.swirl(0, lmin=1, lmax=5, mx=8)
    w.parts = []  # zero field: the layout stays uniform at lmin
    ref, gpu = pair(fc, w, fc.F64)
    assert set(ref.leaves()[:, 2]) == {1}
    q = synth.random_field((len(ref), 8, 8), seed=3)
    ref.set_q(q)
    gpu.set_q(q)
    _, dtc = synth.time_step(w)
    ref.step_multirate(0.0, dtc)
    gpu.step_multirate(0.0, dtc)
    assert relerr(gpu.get_q(), ref.get_q()) <= F64_TOL


def test_full_size_swirl_one_coarse_step():
    """The benchmark workload (levels 2-6, 32^2 patches) for one coarse
    multirate step plus a regrid, compared everywhere with the oracle."""
    w = synth.swirl(0)
    _, dtc = synth.time_step(w)
    for dtype, tol in ((fc.F64, F64_TOL), (fc.F32, 1e-4)):
        ref, gpu = pair(fc, w, dtype)
        assert len(ref) > 300
        ref.step_multirate(0.0, dtc)
        gpu.step_multirate(0.0, dtc)
        err = relerr(gpu.get_q(), ref.get_q())
        print(f"full-size swirl dtype {dtype}: {len(ref)} patches, rel err {err:.2e}")
        assert err <= tol
        if dtype == fc.F64:
            ref.regrid(w.tau_refine, w.tau_coarsen)
            gpu.tag_regrid(w.tau_refine, w.tau_coarsen)
            np.testing.assert_array_equal(gpu.leaves(), ref.leaves())


def test_launch_counter_counts_kernels():
    w = synth.swirl(0, lmin=2, lmax=3, mx=8)
    ref, gpu = pair(fc, w, fc.F64)
    # 3 substeps (level 2 once, level 3 twice).  Separate fills: each substep a
    # copy/average fill and an update, level 3 also an interpolation fill.
    gpu.graphs(False)
    gpu.fused_fill(False)
    fc.launch_count(reset=True)
    gpu.step_multirate(0.0, 0.01)
    assert fc.launch_count() == 3 * 2 + 2
    # fused fill: one update per substep (the staged update fills its own
    # ghosts and computes the time-interpolated coarse cells it reads)
    gpu.fused_fill(True)
    fc.launch_count(reset=True)
    gpu.step_multirate(0.01, 0.01)
    assert fc.launch_count() == 1 + 1 + 1
    # graph replay: the same kernels plus the one that stores the step time
    gpu.graphs(True)
    for n in range(3):
        fc.launch_count(reset=True)
        gpu.step_multirate(0.01 * (n + 2), 0.01)
        assert fc.launch_count() == 1 + 1 + 1 + 1


@pytest.mark.parametrize("variant", [0, 1, 3])
def test_fused_fill_matches_separate_fills_bitwise(variant):
    w = synth.swirl(9, lmin=2, lmax=5, mx=16)
    _, dtc = synth.time_step(w)
    ref, a = pair(fc, w, fc.F64)
    b = fc.Forest(a.desc, ref.leaves())
    b.set_q(a.get_q())
    a.set_advance_variant(variant, 4)
    b.set_advance_variant(variant, 4)
    b.fused_fill(False)
    for n in range(3):
        a.step_multirate(n * dtc, dtc)
        b.step_multirate(n * dtc, dtc)
    np.testing.assert_array_equal(a.get_q(), b.get_q())


def test_graph_replay_matches_direct_launches():
    """Coarse steps replayed from captured CUDA graphs give the same bits as
    direct launches, across a regrid (which discards the captured steps)."""
    w = synth.swirl(6, lmin=2, lmax=5, mx=16)
    _, dtc = synth.time_step(w)
    ref, a = pair(fc, w, fc.F32)
    b = fc.Forest(a.desc, ref.leaves())
    b.set_q(a.get_q())
    b.graphs(False)
    for n in range(6):
        a.step_multirate(n * dtc, dtc)
        b.step_multirate(n * dtc, dtc)
        if n == 2:
            assert a.tag_regrid(0.05, 0.0125) == b.tag_regrid(0.05, 0.0125)
    np.testing.assert_array_equal(a.get_q(), b.get_q())


def test_level_branches_match_one_stream_over_many_steps():
    """The captured steps run each level on its own stream, every substep
    waiting only for the states it reads.  A missing wait would be a race:
    over 12 coarse steps of the full-size swirl forest (levels 2-6, 32^2),
    regridding every 4, the replayed steps must give the same bits as direct
    launches on one stream, and two replayed runs the same bits as each
    other."""
    w = synth.swirl(0)
    _, dtc = synth.time_step(w)
    ref, a = pair(fc, w, fc.F32)
    runs = [a]
    for graphs in (True, False):
        f = fc.Forest(a.desc, ref.leaves())
        f.set_q(a.get_q())
        f.graphs(graphs)
        runs.append(f)
    for n in range(12):
        for f in runs:
            f.step_multirate(n * dtc, dtc)
        if (n + 1) % 4 == 0:
            changed = [f.tag_regrid(w.tau_refine, w.tau_coarsen) for f in runs]
            assert len(set(changed)) == 1
    q = [f.get_q() for f in runs]
    np.testing.assert_array_equal(q[0], q[1])
    np.testing.assert_array_equal(q[0], q[2])


def test_timers_count_replayed_launches():
    w = synth.swirl(6, lmin=2, lmax=4, mx=16)
    _, dtc = synth.time_step(w)
    ref, gpu = pair(fc, w, fc.F32)
    gpu.timers(True)
    nlev = len(set(gpu.leaves()[:, 2]))
    substeps = sum(1 << (l - 2) for l in set(gpu.leaves()[:, 2]))
    for n in range(3):
        gpu.step_multirate(n * dtc, dtc)
        ms, launches, nbytes = gpu.read_timer(0, reset=True)
        assert launches == substeps and ms > 0 and nbytes > 0, (n, launches, substeps, nlev)


def test_timers_count_every_replay_across_regrids():
    """Several replays of the same graphs between reads, and a regrid (which
    drops the graphs) in between: every advance launch is counted once."""
    w = synth.swirl(6, lmin=2, lmax=4, mx=16)
    _, dtc = synth.time_step(w)
    _, gpu = pair(fc, w, fc.F32)
    gpu.step_multirate(0.0, dtc)  # capture outside the timed region
    gpu.timers(True)
    gpu.read_timer(0, reset=True)
    expect = 0
    for n in range(1, 9):
        expect += sum(1 << (l - 2) for l in set(gpu.leaves()[:, 2]))
        gpu.step_multirate(n * dtc, dtc)
        if n % 4 == 0:
            gpu.tag_regrid(w.tau_refine, w.tau_coarsen)
    ms, launches, nbytes = gpu.read_timer(0, reset=True)
    assert launches == expect and ms > 0 and nbytes > 0


@pytest.mark.parametrize("variant,warps", [(0, 4), (1, 2), (1, 4), (1, 8), (2, 4), (2, 8),
                                           (3, 2), (3, 4), (3, 8), (3, 16)])
@pytest.mark.parametrize("mx", [8, 16, 32])
def test_advance_variants_match_oracle(variant, warps, mx):
    """Every patch-update kernel (staged; walk with 2/4/8 warps per CTA;
    walk1; band with 1 to 16 rows a band) on an adaptive swirl forest, FP64
    and FP32, against the oracle."""
    w = synth.swirl(8, lmin=2, lmax=4 if mx == 32 else 5, mx=mx)
    _, dtc = synth.time_step(w)
    for dtype, tol in ((fc.F64, F64_TOL), (fc.F32, 1e-4)):
        ref, gpu = pair(fc, w, dtype)
        gpu.set_advance_variant(variant, warps)
        for n in range(2):
            ref.step_multirate(n * dtc, dtc)
            gpu.step_multirate(n * dtc, dtc)
        err = relerr(gpu.get_q(), ref.get_q())
        print(f"variant {variant} warps {warps} mx {mx} dtype {dtype}: rel err {err:.2e}")
        assert err <= tol


@pytest.mark.parametrize("scheme", [dict(limiter="none"), dict(limiter="first"),
                                    dict(transverse=1), dict(domain="periodic"),
                                    dict(velocity=("const", -0.7, 0.45))])
@pytest.mark.parametrize("variant", [1, 3])
def test_row_walk_variants_scheme_options(scheme, variant):
    """The scheme's options (limiter, transverse terms, boundaries, constant
    velocity of either sign) in the row-walking kernels (walk, band)."""
    w = synth.swirl(4, lmin=2, lmax=4, mx=16)
    for k, v in scheme.items():
        setattr(w, k, v)
    ref, gpu = pair(fc, w, fc.F64)
    gpu.set_advance_variant(variant, 4)
    dt = 0.45 / (16 * 16)
    for n in range(4):
        ref.step_global(n * dt, dt)
        gpu.step_global(n * dt, dt)
    assert relerr(gpu.get_q(), ref.get_q()) <= F64_TOL


def test_autotune_then_parity():
    ws = synth.ensemble(12, seed=5, lmin=2, mx=32, levels=(4, 5))
    _, dtc = synth.time_step(ws[0], 5)
    ref, gpu = pair(fc, ws, fc.F64)
    rep = gpu.autotune()
    assert len(rep) >= 2
    assert all(v[0] in (0, 1, 2, 3) and v[2] in (0, 1) and v[3] > 0 for v in rep.values())
    for n in range(2):
        ref.step_multirate(n * dtc, dtc)
        gpu.step_multirate(n * dtc, dtc)
    assert relerr(gpu.get_q(), ref.get_q()) <= F64_TOL


def _smooth_field(leaves, mx):
    """1 + sin(2 pi x) cos(2 pi y) / 2 at the cell centres of each leaf: a
    field that is nowhere constant."""
    lv = np.asarray(leaves)
    n = len(lv)
    h = 1.0 / (mx * 2.0 ** lv[:, 2])
    i = np.arange(mx) + 0.5
    x = (lv[:, 3, None] * mx + i[None, :]) * h[:, None]
    y = (lv[:, 4, None] * mx + i[None, :]) * h[:, None]
    return (1.0 + 0.5 * np.sin(2 * np.pi * x)[:, None, :] *
            np.cos(2 * np.pi * y)[:, :, None]).reshape(n, mx, mx)


@pytest.mark.parametrize("indicator", ["gradient", "maxmin"])
def test_regrid_interpolates_new_children_with_filled_ghosts(indicator):
    """New children take Eq. ghost_fine interpolation from their parent's
    cells, the stencil reaching the parent's first ghost layer at its edges:
    with either indicator the regrid fills the ghosts first, so on a field
    that is nowhere constant the remapped field equals the oracle's."""
    w = synth.swirl(3, lmin=2, lmax=4, mx=16)
    w.indicator = indicator
    ref, gpu = pair(fc, w, fc.F64)
    q = _smooth_field(ref.leaves(), w.mx)
    ref.set_q(q)
    gpu.set_q(q)
    _, dtc = synth.time_step(w)
    ref.step_multirate(0.0, dtc)
    gpu.step_multirate(0.0, dtc)
    # a threshold in the widest gap between the middle indicators (no leaf
    # within rounding of it)
    d = np.sort(ref.tag())
    k = len(d) // 4 + int(np.argmax(np.diff(d[len(d) // 4: 3 * len(d) // 4])))
    tau_r = 0.5 * (d[k] + d[k + 1])
    assert d[k + 1] - d[k] > 1e-9 * d[-1]
    assert ref.regrid(tau_r, -1.0) > 0
    gpu.tag_regrid(tau_r, -1.0)
    np.testing.assert_array_equal(gpu.leaves(), ref.leaves())
    assert relerr(gpu.get_q(), ref.get_q()) <= F64_TOL
