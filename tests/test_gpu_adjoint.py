"""The GPU adjoint (fc_adjoint_step_global, fc_adjoint_step_multirate, autograd
with sqrt(N) checkpoints) against the oracle's adjoint, the transpose identity
and finite differences.

FP64: relative error of the gradient <= 1e-10 against the oracle (the adjoint
sums ghost contributions with atomics, so only the rounding order differs).
FP32: <= 1e-3 against the FP64 oracle adjoint, as the config-5 tolerance.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import desc_for, relerr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
fc = pytest.importorskip("paper_1703_03116_gb300")
from paper_1703_03116_gb300.autograd import advect  # noqa: E402

DEV = torch.device("cuda", 0)


def _tensor(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def test_gpu_adjoint_transpose_identity_linear():
    """Unlimited scheme on a uniform periodic forest: the step is linear, so
    <S v, w> = <v, S^T w> to rounding."""
    w0 = synth.smooth_periodic(0, level=2, mx=16, velocity=("swirl", 4.0), limiter="none")
    F = fc.Forest(desc_for(fc, w0, fc.F64), oracle.uniform_leaves(2))
    n = len(F)
    v = _tensor(synth.random_field((n, 16, 16), seed=1) - 0.5, torch.float64)
    w = _tensor(synth.random_field((n, 16, 16), seed=2) - 0.5, torch.float64)
    dt = 0.9 / 64
    F.set_q(v)
    F.step_global(0.2, dt)
    Jv = torch.empty_like(v)
    F.get_q(out=Jv)
    F.set_q(torch.zeros_like(v))
    lam = w.clone()
    ds = torch.zeros(1, dtype=torch.float64, device=DEV)
    F.adjoint_step_global(0.2, dt, lam, ds)
    a, b = float((Jv * w).sum()), float((v * lam).sum())
    assert abs(a - b) <= 1e-13 * abs(a)


def _case(mx=8, lmax=4, seed=3):
    w = synth.swirl(seed, lmin=2, lmax=lmax, mx=mx)
    ref = oracle.initial_forest(w)
    x, y = synth.cell_centres(ref.leaves(), mx)
    q0 = synth.evaluate(synth.smooth_periodic(1), x, y) + 0.3 * np.sin(3 * x + 1) * np.cos(2 * y)
    qt = synth.evaluate(synth.smooth_periodic(2), x, y)
    ref.set_q(q0)
    return w, ref, q0, qt


@pytest.mark.parametrize("mx,lmax", [(8, 4), (16, 4), (32, 3)])
def test_gpu_adjoint_step_matches_oracle_fp64(mx, lmax):
    w, ref, q0, qt = _case(mx, lmax)
    F = fc.Forest(desc_for(fc, w, fc.F64), ref.leaves())
    F.set_q(q0)
    lam0 = synth.random_field(q0.shape, seed=9) - 0.5
    dt = 0.9 / (mx * 2 ** lmax)
    lam_ref, ds_ref = ref.adjoint_step_global(0.3, dt, lam0)
    lam = _tensor(lam0, torch.float64)
    ds = torch.zeros(1, dtype=torch.float64, device=DEV)
    F.adjoint_step_global(0.3, dt, lam, ds)
    assert relerr(lam.cpu().numpy(), lam_ref) <= 1e-12
    assert abs(float(ds) - ds_ref) <= 1e-12 * abs(ds_ref)


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-10), ("f32", 1e-3)])
def test_autograd_gradient_matches_oracle(dtype, tol):
    w, ref, q0, qt = _case(8, 4)
    nsteps, dt = 9, 0.9 / 128
    loss_ref, g_ref, gs_ref = ref.adjoint_global(nsteps, 0.0, dt, qt)
    fdt = fc.F64 if dtype == "f64" else fc.F32
    tdt = torch.float64 if dtype == "f64" else torch.float32
    F = fc.Forest(desc_for(fc, w, fdt), ref.leaves())
    q = _tensor(q0, tdt).requires_grad_(True)
    s = torch.ones((), dtype=tdt, device=DEV, requires_grad=True)
    qN = advect(q, s, F, 0.0, dt, nsteps)
    loss = 0.5 * ((qN - _tensor(qt, tdt)) ** 2).sum()
    loss.backward()
    err_q = relerr(q.grad.double().cpu().numpy(), g_ref)
    err_s = abs(float(s.grad) - gs_ref) / abs(gs_ref)
    print(f"{dtype}: loss {float(loss.detach()):.6e} vs {loss_ref:.6e}, grad q0 rel err {err_q:.2e}, "
          f"grad scale rel err {err_s:.2e}")
    assert err_q <= tol and err_s <= tol


def test_checkpoint_segments_give_the_same_gradient():
    w, ref, q0, qt = _case(8, 4)
    F = fc.Forest(desc_for(fc, w, fc.F64), ref.leaves())
    grads = []
    for seg in (1, 3, 0, 9):
        q = _tensor(q0, torch.float64).requires_grad_(True)
        s = torch.ones((), dtype=torch.float64, device=DEV, requires_grad=True)
        qN = advect(q, s, F, 0.0, 0.9 / 128, 9, segment=seg)
        (0.5 * ((qN - _tensor(qt, torch.float64)) ** 2).sum()).backward()
        grads.append((q.grad.cpu().numpy(), float(s.grad)))
    for g, gs in grads[1:]:
        assert relerr(g, grads[0][0]) <= 1e-12 and abs(gs - grads[0][1]) <= 1e-12 * abs(gs)


def test_autograd_central_differences_fp64():
    """The map is piecewise linear (limiter and interpolation slopes), so the
    step must stay on one piece: smooth data and a small step."""
    w, ref, q0, qt = _case(8, 4)
    F = fc.Forest(desc_for(fc, w, fc.F64), ref.leaves())
    nsteps, dt = 4, 0.9 / 128
    qt_t = _tensor(qt, torch.float64)

    def L(q, s):
        with torch.no_grad():
            qN = advect(q, s, F, 0.0, dt, nsteps)
            return float(0.5 * ((qN - qt_t) ** 2).sum())

    q = _tensor(q0, torch.float64).requires_grad_(True)
    s = torch.ones((), dtype=torch.float64, device=DEV, requires_grad=True)
    qN = advect(q, s, F, 0.0, dt, nsteps)
    (0.5 * ((qN - qt_t) ** 2).sum()).backward()
    d = _tensor(synth.random_field(q0.shape, seed=4) - 0.5, torch.float64)
    eps = 1e-7
    q0t = _tensor(q0, torch.float64)
    one = torch.ones((), dtype=torch.float64, device=DEV)
    fd = (L(q0t + eps * d, one) - L(q0t - eps * d, one)) / (2 * eps)
    assert abs(fd - float((q.grad * d).sum())) <= 1e-6 * abs(fd)
    fds = (L(q0t, one + 1e-6) - L(q0t, one - 1e-6)) / 2e-6
    assert abs(fds - float(s.grad)) <= 1e-6 * abs(fds)


# ---------------------------------------------------------------- multirate


@pytest.mark.parametrize("mx,lmax", [(8, 4), (16, 4), (32, 3)])
def test_gpu_multirate_adjoint_step_matches_oracle_fp64(mx, lmax):
    w, ref, q0, qt = _case(mx, lmax)
    F = fc.Forest(desc_for(fc, w, fc.F64), ref.leaves())
    F.set_q(q0)
    lam0 = synth.random_field(q0.shape, seed=11) - 0.5
    dtc = 0.9 / (mx * 2 ** lmax) * 2 ** (lmax - 2)
    lam_ref, ds_ref = ref.adjoint_step_multirate(0.3, dtc, lam0)
    lam = _tensor(lam0, torch.float64)
    ds = torch.zeros(1, dtype=torch.float64, device=DEV)
    F.adjoint_step_multirate(0.3, dtc, lam, ds)
    err = relerr(lam.cpu().numpy(), lam_ref)
    print(f"multirate adjoint step mx={mx}: rel err {err:.2e}, dscale {float(ds):.6e} vs {ds_ref:.6e}")
    assert err <= 1e-12
    assert abs(float(ds) - ds_ref) <= 1e-12 * abs(ds_ref)
    # the forest is left at the step's start state
    back = torch.empty_like(lam)
    F.get_q(out=back)
    np.testing.assert_array_equal(back.cpu().numpy(), q0)


@pytest.mark.parametrize("mx,lmax", [(8, 4), (16, 4), (32, 3)])
def test_recorded_step_and_taped_reverse_fp64(mx, lmax):
    """fc_step_multirate_record is fc_step_multirate (the same bits) and the
    taped reverse equals the oracle's adjoint of the step, for steps
    recorded into several slots and reversed in any order."""
    w, ref, q0, qt = _case(mx, lmax)
    dtc = 0.9 / (mx * 2 ** lmax) * 2 ** (lmax - 2)
    plain = fc.Forest(desc_for(fc, w, fc.F64), ref.leaves())
    rec = fc.Forest(desc_for(fc, w, fc.F64), ref.leaves())
    plain.set_q(q0)
    rec.set_q(q0)
    states = [q0]
    for k in range(3):
        plain.step_multirate(0.3 + k * dtc, dtc)
        rec.step_multirate_record(0.3 + k * dtc, dtc, k)
        np.testing.assert_array_equal(rec.get_q(), plain.get_q())
        states.append(plain.get_q())
    for k in (1, 2, 0):  # any order of the slots
        o = oracle.initial_forest(w)
        o.set_q(states[k])
        lam0 = synth.random_field(q0.shape, seed=20 + k) - 0.5
        lam_ref, ds_ref = o.adjoint_step_multirate(0.3 + k * dtc, dtc, lam0)
        lam = _tensor(lam0, torch.float64)
        ds = torch.zeros(1, dtype=torch.float64, device=DEV)
        rec.adjoint_step_multirate_taped(0.3 + k * dtc, dtc, k, lam, ds)
        err = relerr(lam.cpu().numpy(), lam_ref)
        print(f"taped reverse mx={mx} slot {k}: rel err {err:.2e}")
        assert err <= 1e-12
        assert abs(float(ds) - ds_ref) <= 1e-12 * abs(ds_ref)
    # the reverses left the recorded forest where its forward steps did
    np.testing.assert_array_equal(rec.get_q(), states[3])


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_forward_tape_and_recompute_give_the_same_gradient(dtype, tol):
    """advect's two multirate strategies -- every step recorded by the
    forward pass, or sqrt(N) checkpoints recomputed and recorded segment by
    segment -- give the same gradients (to the atomics' rounding order)."""
    w, ref, q0, qt = _case(16, 4)
    dtc = 0.9 / (16 * 2 ** 4) * 4
    F = fc.Forest(desc_for(fc, w, fc.F64 if dtype == "f64" else fc.F32), ref.leaves())
    tdt = torch.float64 if dtype == "f64" else torch.float32
    grads = {}
    for tape in ("forward", "recompute"):
        q = _tensor(q0, tdt).requires_grad_(True)
        s = torch.ones((), dtype=tdt, device=DEV, requires_grad=True)
        qN = advect(q, s, F, 0.1, dtc, 6, multirate=True, tape=tape)
        loss = 0.5 * ((qN - _tensor(qt, tdt)) ** 2).sum()
        loss.backward()
        grads[tape] = (q.grad.cpu().numpy(), float(s.grad))
    err = relerr(grads["forward"][0], grads["recompute"][0])
    print(f"tape vs recompute {dtype}: q0 gradient {err:.2e}")
    assert err <= tol
    assert abs(grads["forward"][1] - grads["recompute"][1]) <= tol * abs(grads["recompute"][1])
    # a later taped run takes the forest's tapes: the first backward refuses
    q1 = _tensor(q0, tdt).requires_grad_(True)
    s1 = torch.ones((), dtype=tdt, device=DEV, requires_grad=True)
    a = advect(q1, s1, F, 0.1, dtc, 3, multirate=True, tape="forward")
    b = advect(q1, s1, F, 0.1, dtc, 3, multirate=True, tape="forward")
    b.sum().backward(retain_graph=True)
    with pytest.raises(RuntimeError):
        a.sum().backward()


def test_taped_reverse_refuses_what_was_not_recorded():
    w, ref, q0, qt = _case(16, 4)
    dtc = 0.9 / (16 * 2 ** 4) * 4
    F = fc.Forest(desc_for(fc, w, fc.F64), ref.leaves())
    F.set_q(q0)
    lam = _tensor(q0, torch.float64)
    ds = torch.zeros(1, dtype=torch.float64, device=DEV)
    with pytest.raises(fc.FcError) as e:  # nothing recorded
        F.adjoint_step_multirate_taped(0.0, dtc, 0, lam, ds)
    assert e.value.status == 6  # FC_ERR_STATE
    F.step_multirate_record(0.0, dtc, 0)
    with pytest.raises(fc.FcError) as e:  # recorded with another step length
        F.adjoint_step_multirate_taped(0.0, 0.5 * dtc, 0, lam, ds)
    assert e.value.status == 6
    with pytest.raises(fc.FcError) as e:
        F.step_multirate_record(0.0, dtc, 64)  # past FC_MAX_TAPE_SLOTS
    assert e.value.status == 1  # FC_ERR_INVALID_ARG
    F.set_advance_variant(0, 4)  # the captured steps changed: the tape is stale
    with pytest.raises(fc.FcError) as e:
        F.adjoint_step_multirate_taped(0.0, dtc, 0, lam, ds)
    assert e.value.status == 6
    F.release_tapes()


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-10), ("f32", 1e-3)])
def test_autograd_multirate_gradient_matches_oracle(dtype, tol):
    w, ref, q0, qt = _case(8, 4)
    ncoarse, dtc = 5, 4 * 0.9 / 128
    loss_ref, g_ref, gs_ref = ref.adjoint_multirate(ncoarse, 0.0, dtc, qt)
    fdt = fc.F64 if dtype == "f64" else fc.F32
    tdt = torch.float64 if dtype == "f64" else torch.float32
    F = fc.Forest(desc_for(fc, w, fdt), ref.leaves())
    q = _tensor(q0, tdt).requires_grad_(True)
    s = torch.ones((), dtype=tdt, device=DEV, requires_grad=True)
    qN = advect(q, s, F, 0.0, dtc, ncoarse, multirate=True)
    loss = 0.5 * ((qN - _tensor(qt, tdt)) ** 2).sum()
    loss.backward()
    err_q = relerr(q.grad.double().cpu().numpy(), g_ref)
    err_s = abs(float(s.grad) - gs_ref) / abs(gs_ref)
    print(f"multirate {dtype}: loss {float(loss.detach()):.6e} vs {loss_ref:.6e}, grad q0 rel err "
          f"{err_q:.2e}, grad scale rel err {err_s:.2e}")
    assert err_q <= tol and err_s <= tol


def test_autograd_multirate_central_differences_fp64():
    w, ref, q0, qt = _case(8, 4)
    F = fc.Forest(desc_for(fc, w, fc.F64), ref.leaves())
    ncoarse, dtc = 3, 4 * 0.9 / 128
    qt_t = _tensor(qt, torch.float64)

    def L(q, s):
        with torch.no_grad():
            qN = advect(q, s, F, 0.0, dtc, ncoarse, multirate=True)
            return float(0.5 * ((qN - qt_t) ** 2).sum())

    q = _tensor(q0, torch.float64).requires_grad_(True)
    s = torch.ones((), dtype=torch.float64, device=DEV, requires_grad=True)
    qN = advect(q, s, F, 0.0, dtc, ncoarse, multirate=True)
    (0.5 * ((qN - qt_t) ** 2).sum()).backward()
    d = _tensor(synth.random_field(q0.shape, seed=5) - 0.5, torch.float64)
    eps = 1e-7
    q0t = _tensor(q0, torch.float64)
    one = torch.ones((), dtype=torch.float64, device=DEV)
    fd = (L(q0t + eps * d, one) - L(q0t - eps * d, one)) / (2 * eps)
    assert abs(fd - float((q.grad * d).sum())) <= 1e-6 * abs(fd)
    fds = (L(q0t, one + 1e-6) - L(q0t, one - 1e-6)) / 2e-6
    assert abs(fds - float(s.grad)) <= 1e-6 * abs(fds)


def _full_size(smooth):
    w = synth.swirl(0)
    tw = synth.adjoint_target(w)
    ref = oracle.initial_forest(w)
    lv = ref.leaves()
    x, y = synth.cell_centres(lv, w.mx)
    if smooth:
        q0 = synth.evaluate(synth.smooth_periodic(1), x, y) + 0.3 * np.sin(3 * x + 1) * np.cos(2 * y)
    else:
        q0 = synth.evaluate(w, x, y)
    qt = synth.evaluate(tw, x, y)
    ref.set_q(q0)
    _, dtc = synth.time_step(w)
    return w, ref, lv, q0, qt, dtc


def _gpu_grad(w, lv, q0, qt, dtc, dtype, ncoarse=2):
    fdt = fc.F64 if dtype == "f64" else fc.F32
    tdt = torch.float64 if dtype == "f64" else torch.float32
    F = fc.Forest(desc_for(fc, w, fdt), lv)
    q = _tensor(q0, tdt).requires_grad_(True)
    s = torch.ones((), dtype=tdt, device=DEV, requires_grad=True)
    qN = advect(q, s, F, 0.0, dtc, ncoarse, multirate=True)
    loss = 0.5 * ((qN - _tensor(qt, tdt)) ** 2).sum()
    loss.backward()
    return float(loss.detach()), q.grad.double().cpu().numpy(), float(s.grad)


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-10), ("f32", 1e-3)])
def test_full_size_multirate_adjoint_smooth(dtype, tol):
    """The adjoint workload's forest (swirl levels 2-6, 32^2 patches, frozen
    after the initial regrid) with smooth data, sqrt(N) checkpoints over 2
    coarse steps (32 finest substeps), against the FP64 oracle's adjoint."""
    w, ref, lv, q0, qt, dtc = _full_size(True)
    loss_ref, g_ref, gs_ref = ref.adjoint_multirate(2, 0.0, dtc, qt)
    loss, g, gs = _gpu_grad(w, lv, q0, qt, dtc, dtype)
    err_q = relerr(g, g_ref)
    l2 = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    err_s = abs(gs - gs_ref) / abs(gs_ref)
    print(f"full-size multirate adjoint, smooth data, {dtype}: {len(lv)} patches, grad q0 rel err "
          f"{err_q:.2e} (L2 {l2:.2e}), grad scale rel err {err_s:.2e}")
    assert err_s <= tol
    if dtype == "f64":
        assert err_q <= tol
    else:
        # FP32 rounding of the forward state (~1e-7) decides some limiter
        # near-ties differently over 474k cells x 32 substeps: pointwise
        # outliers, bounded in L2
        assert l2 <= 1e-2


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-10), ("f32", 1e-3)])
def test_full_size_multirate_adjoint_disc(dtype, tol):
    """The adjoint workload itself: disc data and the shifted-disc target.
    The flat regions of the disc make the limiter's piece a matter of
    rounding noise (the sign of W W_up when both are ~1e-17), so the gradient
    with respect to q0 is not unique there: the oracle's own gradient moves by
    ~3% in L2 when q0 is perturbed by 1e-15.  Compared: the loss and the
    velocity-scale derivative (unique), and the q0 gradient within that
    spread."""
    w, ref, lv, q0, qt, dtc = _full_size(False)
    loss_ref, g_ref, gs_ref = ref.adjoint_multirate(2, 0.0, dtc, qt)
    loss, g, gs = _gpu_grad(w, lv, q0, qt, dtc, dtype)
    err_l = abs(loss - loss_ref) / loss_ref
    err_s = abs(gs - gs_ref) / abs(gs_ref)
    l2 = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    print(f"full-size multirate adjoint, disc data, {dtype}: loss rel err {err_l:.2e}, grad scale "
          f"rel err {err_s:.2e}, grad q0 L2 rel diff {l2:.2e}")
    assert err_l <= (1e-12 if dtype == "f64" else 1e-5)
    assert err_s <= tol
    assert l2 <= 0.1


def _config5(smooth, ncoarse=25):
    """FP32 and FP64 gradients of the config-5 run (the swirl forest frozen
    after its initial regrid, levels 2-6, 32^2 patches, ncoarse coarse
    multirate steps, sqrt(N) checkpoints) and FP64 central differences
    (h = 1e-3) of the loss along three seeded smooth directions and of the
    velocity scale."""
    w, ref, lv, q0, qt, dtc = _full_size(smooth)
    loss32, g32, gs32 = _gpu_grad(w, lv, q0, qt, dtc, "f32", ncoarse)
    loss64, g64, gs64 = _gpu_grad(w, lv, q0, qt, dtc, "f64", ncoarse)
    F = fc.Forest(desc_for(fc, w, fc.F64), lv)
    qt_t = _tensor(qt, torch.float64)
    q0t = _tensor(q0, torch.float64)

    def L(q, s):
        with torch.no_grad():
            qN = advect(q, torch.tensor(s, dtype=torch.float64, device=DEV), F, 0.0, dtc,
                        ncoarse, multirate=True)
            return float(0.5 * ((qN - qt_t) ** 2).sum())

    h = 1e-3
    x, y = synth.cell_centres(lv, w.mx)
    rows = []
    for k in range(3):
        d = synth.evaluate(synth.smooth_periodic(20 + k), x, y)
        d = d / np.sqrt(np.sum(d * d))
        dt_ = _tensor(d, torch.float64)
        fd = (L(q0t + h * dt_, 1.0) - L(q0t - h * dt_, 1.0)) / (2 * h)
        rows.append((fd, float(np.sum(g64 * d)), float(np.sum(g32 * d))))
    fds = (L(q0t, 1.0 + h) - L(q0t, 1.0 - h)) / (2 * h)
    r = {"patches": len(lv), "loss": abs(loss32 - loss64) / loss64,
         "scale32": abs(gs32 - gs64) / abs(gs64), "scale_fd": abs(fds - gs64) / abs(fds),
         "q0_l2": np.linalg.norm(g32 - g64) / np.linalg.norm(g64),
         "dir32": [abs(b - c) / abs(b) for _, b, c in rows],
         "dir_fd": [abs(a - b) / abs(a) for a, b, _ in rows]}
    print(f"config 5 at size, {'smooth' if smooth else 'disc'} data ({len(lv)} patches, "
          f"{ncoarse} coarse steps): FP32 vs FP64 loss {r['loss']:.2e}, scale derivative "
          f"{r['scale32']:.2e}, q0 gradient L2 {r['q0_l2']:.2e}, directions "
          f"{['%.2e' % e for e in r['dir32']]}; FP64 adjoint vs central differences: scale "
          f"{r['scale_fd']:.2e}, directions {['%.2e' % e for e in r['dir_fd']]}")
    return r


def test_config5_disc_data_at_its_own_size():
    """The adjoint workload itself: disc data and the shifted-disc target over
    25 coarse steps.  The loss and the velocity-scale derivative are unique
    and meet 1e-3 (FP32 against FP64, and the FP64 adjoint against central
    differences).  The gradient with respect to q0 is not unique: in the
    disc's flat regions W = W_up = 0 puts every edge on the limiter's kink,
    the map is only positively homogeneous there, and the piece an adjoint
    takes is decided by rounding noise (FP32 and FP64 differ by O(1) in L2,
    and so do directional central differences) -- printed, not bounded."""
    r = _config5(False)
    assert r["loss"] <= 1e-4
    assert r["scale32"] <= 1e-3
    assert r["scale_fd"] <= 1e-3


def test_config5_smooth_data_at_its_own_size():
    """The same forest and 25 coarse steps from smooth data, where the map is
    differentiable almost everywhere on the path: the FP32 gradient with
    respect to q0 along smooth directions, and the FP64 adjoint against
    central differences."""
    r = _config5(True)
    assert r["loss"] <= 1e-4 and r["scale32"] <= 1e-3 and r["scale_fd"] <= 1e-3
    # measured: q0 gradient L2 5.6e-4, directions ~1e-7, differences ~1e-7
    assert r["q0_l2"] <= 1e-3
    assert max(r["dir32"]) <= 1e-5
    assert max(r["dir_fd"]) <= 1e-5
