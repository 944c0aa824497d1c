"""The adjoint step (lb_adjoint_step) and differentiable rollouts against the
FP64 oracle's complex-step derivatives (exact to rounding) and central finite
differences.

Tolerances: FP64 adjoint vs the oracle's transposed Jacobian <= 1e-12 relative
(element by element); FP32 adjoint vs FP64 adjoint <= 2e-4 relative (single
precision of a ~10-term chain of products); rollout gradients vs complex step
<= 1e-9 and vs central differences <= 1e-5 (the O(h^2) truncation of the
difference quotient)."""
import numpy as np
import pytest

from gpu_util import W_REST, lattice, oracle_params
from paper_1809_02390_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_02390_gb300 import build

    build.build()


def _flow_state(orc, p, nx, ny, seed):
    rng = np.random.default_rng(seed)
    rho = inputs.droplet(nx, ny, min(nx, ny) / 3, 3, p.rho_g, p.rho_l) * (1 + 0.02 * rng.uniform(-1, 1, (ny, nx)))
    return orc.init_eq(p, rho, 0.06 * rng.uniform(-1, 1, (ny, nx)), 0.06 * rng.uniform(-1, 1, (ny, nx)))


def _gpu_adjoint(lat, f_state, lam_in):
    from paper_1809_02390_gb300 import capi

    real = torch.float64 if lat.precision == "fp64" else torch.float32
    s = torch.from_numpy(np.ascontiguousarray(f_state)).to("cuda", lat.dtype)
    li = torch.from_numpy(np.ascontiguousarray(lam_in)).to("cuda", real)
    lo = torch.empty_like(li)
    dth = torch.zeros(3, dtype=torch.float64, device="cuda")
    n = capi.lb_adjoint_scratch_bytes(lat.p)
    scr = torch.empty(n, dtype=torch.uint8, device="cuda")
    capi.lb_adjoint_step(lat.h, s.data_ptr(), li.data_ptr(), lo.data_ptr(), dth.data_ptr(), scr.data_ptr(), n)
    torch.cuda.synchronize()
    return lo.double().cpu().numpy(), dth.cpu().numpy()


@pytest.mark.parametrize("nx,ny,eos", [(7, 6, "vdw"), (5, 9, "vdw"), (6, 6, "cs")])
def test_fp64_adjoint_equals_transposed_jacobian(orc, nx, ny, eos):
    """Every column of the step's Jacobian (state and parameters T, G2, lam) from
    the oracle by complex step; the GPU adjoint must equal J^T lam element-wise."""
    kw = dict(Tr=0.85, K_int=1.0) if eos == "vdw" else dict(eos="cs", a=1.0, b=4.0, Tr=0.8, K_int=2.0)
    p = oracle_params(**kw)
    f0 = _flow_state(orc, p, nx, ny, 5)
    rng = np.random.default_rng(9)
    lam = rng.standard_normal(f0.shape)
    h = 1e-30
    n = f0.size
    J = np.empty((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = h
        J[:, k] = orc.step_cs(p, f0, e.reshape(f0.shape), (0, 0, 0), 1)[1].ravel() / h
    Jt = np.stack([orc.step_cs(p, f0, None, h * np.eye(3)[k], 1)[1].ravel() / h for k in range(3)], 1)
    ref = (J.T @ lam.ravel()).reshape(f0.shape)
    ref_th = Jt.T @ lam.ravel()
    lkw = dict(Tr=kw["Tr"], G2=p.G2, lam=p.lam, rho_ref=0.0)
    if eos == "cs":
        lkw.update(eos="cs", eos_a=1.0, eos_b=4.0)
    lat = lattice(np.full((ny, nx), 2.0 if eos == "vdw" else 0.2), "fp64", **lkw)
    got, th = _gpu_adjoint(lat, f0, lam)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(th - ref_th).max() <= 1e-11 * np.abs(ref_th).max()


def test_fp32_adjoint_close_to_fp64(orc):
    p = oracle_params(Tr=0.85, K_int=1.0)
    f0 = _flow_state(orc, p, 64, 48, 2)
    lam = np.random.default_rng(1).standard_normal(f0.shape)
    l64 = lattice(np.full((48, 64), 2.0), "fp64", Tr=0.85, G2=p.G2, lam=p.lam, rho_ref=0.0)
    l32 = lattice(np.full((48, 64), 2.0), "fp32", Tr=0.85, G2=p.G2, lam=p.lam, rho_ref=0.0)
    a, ta = _gpu_adjoint(l64, f0, lam)
    b, tb = _gpu_adjoint(l32, f0, lam)
    assert np.abs(a - b).max() <= 2e-4 * np.abs(a).max()
    assert np.abs(ta - tb).max() <= 2e-4 * np.abs(ta).max()


def _loss_setup(n=24, steps=30):
    from paper_1809_02390_gb300.adjoint import RolloutSpec, initial_state

    spec = RolloutSpec(n, n, precision="fp64", Tr_ref=0.85, K_int_ref=1.0)
    theta0 = torch.tensor([0.85, spec.G2_ref, 1.0], dtype=torch.float64)
    rho0 = inputs.ellipse(n, n, 7.0, 4.5, 3.0, spec.rho_g, spec.rho_l, noise=0.01, seed=4)
    f0 = initial_state(spec, rho0, theta0)
    target = torch.from_numpy(inputs.droplet(n, n, 5.5, 3.0, spec.rho_g, spec.rho_l)).cuda()
    return spec, theta0, f0, target, steps


def _loss(spec, theta, f0, target, steps, every=None):
    from paper_1809_02390_gb300.adjoint import density, rollout

    out = rollout(theta, f0, spec, steps, every)
    return ((density(out, spec) - target) ** 2).sum()


def test_rollout_gradient_vs_central_differences():
    spec, theta0, f0, target, steps = _loss_setup()
    theta = theta0.clone().requires_grad_(True)
    f0r = f0.clone().requires_grad_(True)
    L = _loss(spec, theta, f0r, target, steps, every=7)  # ragged last segment
    L.backward()
    g = theta.grad.numpy()
    for k, hrel in enumerate((1e-5, 1e-5, 1e-5)):
        hk = hrel * float(theta0[k])
        tp, tm = theta0.clone(), theta0.clone()
        tp[k] += hk
        tm[k] -= hk
        with torch.no_grad():
            fd = (float(_loss(spec, tp, f0, target, steps)) - float(_loss(spec, tm, f0, target, steps))) / (2 * hk)
        assert g[k] == pytest.approx(fd, rel=1e-5)
    # Initial-state gradient along a random direction.
    v = torch.randn(f0.shape, dtype=torch.float64, device="cuda") * 1e-3
    eps = 1e-4
    with torch.no_grad():
        fd = (float(_loss(spec, theta0, f0 + eps * v, target, steps))
              - float(_loss(spec, theta0, f0 - eps * v, target, steps))) / (2 * eps)
    assert float((f0r.grad * v).sum()) == pytest.approx(fd, rel=1e-5)


def test_rollout_gradient_vs_oracle_complex_step(orc):
    """dL/d(Tr, G2, K_int) through 30 steps against the FP64 oracle differentiated
    by complex step (T = Tr Tc, lam = lam_ref (K_ref/K)^2)."""
    spec, theta0, f0, target, steps = _loss_setup(n=16, steps=20)
    theta = theta0.clone().requires_grad_(True)
    L = _loss(spec, theta, f0, target, steps, every=6)
    L.backward()
    g = theta.grad.numpy()
    p = oracle_params(Tr=0.85, K_int=1.0).as_dict()
    p.update(G2=float(theta0[1]), lam=spec.lam_ref)
    fabs = f0.double().cpu().numpy() + spec.rho_ref * W_REST[:, None, None]
    re, _ = orc.step_cs(p, fabs, None, (0, 0, 0), steps)
    resid = 2 * (re.sum(0) - target.cpu().numpy())
    h = 1e-30
    dT = orc.step_cs(p, fabs, None, (h, 0, 0), steps)[1].sum(0) / h
    dG = orc.step_cs(p, fabs, None, (0, h, 0), steps)[1].sum(0) / h
    dl = orc.step_cs(p, fabs, None, (0, 0, h), steps)[1].sum(0) / h
    ref = np.array([(resid * dT).sum() * spec.Tc, (resid * dG).sum(), (resid * dl).sum() * (-2 * spec.lam_ref)])
    assert np.allclose(g, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("nx,ny", [(45, 38), (33, 17), (130, 70), (1540, 644)])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_fused_segment_equals_single_steps(orc, precision, tol, nx, ny):
    """lb_adjoint_steps (fused, one kernel per step) against k calls of lb_adjoint_step,
    on small lattices where the fused FP32 step pulls the state directly and on one
    with several waves of tiles (1540 x 644, ragged) where it stages the state
    window by asynchronous copies."""
    from paper_1809_02390_gb300 import capi

    p = oracle_params(Tr=0.85, K_int=1.0)
    k = 5
    f0 = _flow_state(orc, p, nx, ny, 3)
    lat = lattice(np.full((ny, nx), 2.0), precision, Tr=0.85, G2=p.G2, lam=p.lam, rho_ref=0.0)
    real = torch.float64 if precision == "fp64" else torch.float32
    states = [torch.from_numpy(f0).to("cuda", lat.dtype)]
    capi.lb_set_state(lat.h, states[0].data_ptr())
    for _ in range(k - 1):
        lat.step(1)
        states.append(lat.state().clone())
    lam0 = torch.from_numpy(np.random.default_rng(2).standard_normal(f0.shape)).to("cuda", real)
    # k single steps
    ns = capi.lb_adjoint_scratch_bytes(lat.p)
    scr = torch.empty(ns, dtype=torch.uint8, device="cuda")
    a, b = lam0.clone(), torch.empty_like(lam0)
    th1 = torch.zeros(3, dtype=torch.float64, device="cuda")
    for st in reversed(states):
        capi.lb_adjoint_step(lat.h, st.data_ptr(), a.data_ptr(), b.data_ptr(), th1.data_ptr(), scr.data_ptr(), ns)
        a, b = b, a
    # one fused call
    ns2 = capi.lb_adjoint_steps_scratch_bytes(lat.p)
    scr2 = torch.empty(ns2, dtype=torch.uint8, device="cuda")
    c = lam0.clone()
    th2 = torch.zeros(3, dtype=torch.float64, device="cuda")
    capi.lb_adjoint_steps(lat.h, [t.data_ptr() for t in states], c.data_ptr(), th2.data_ptr(), scr2.data_ptr(), ns2)
    torch.cuda.synchronize()
    assert float((a - c).abs().max()) <= tol * float(a.abs().max())
    assert float((th1 - th2).abs().max()) <= tol * float(th1.abs().max())


def test_calibration_recovers_parameters():
    """Gradient-based calibration through the adjoint: a target density field made at
    reference (Tr, G2, K_int) is fitted from parameters perturbed by -4%, +5%, -7%;
    L-BFGS (the default) recovers each of the three within 2% (on the 256^2 benchmark
    case it recovers them exactly to the printed digits, where Adam with the same
    budget leaves K_int 19% off: the loss is ill-conditioned)."""
    from paper_1809_02390_gb300.adjoint import RolloutSpec, calibrate, density, initial_state, rollout

    n = 64
    spec = RolloutSpec(n, n, precision="fp32", Tr_ref=0.8, K_int_ref=1.0)
    ref = torch.tensor([0.8, spec.G2_ref, 1.0], dtype=torch.float64)
    rho0 = inputs.ellipse(n, n, 12 * 1.5 ** 0.5, 12 / 1.5 ** 0.5, 4.0, spec.rho_g, spec.rho_l, noise=0.01, seed=1)
    f0 = initial_state(spec, rho0, ref)
    with torch.no_grad():
        target = density(rollout(ref, f0, spec, 300), spec).detach()
    start = ref * torch.tensor([0.96, 1.05, 0.93], dtype=torch.float64)
    theta, losses = calibrate(spec, f0, target, start, 300, iterations=40)
    assert losses[-1] < 1e-4 * losses[0]
    assert float(((theta - ref) / ref).abs().max()) < 0.02
