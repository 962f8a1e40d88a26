"""GPU profile gradients (fresnel_grad_profile) and boundary-shape gradients
(fresnel_grad_shape), both through torch autograd, against the oracle's
hand-derived adjoints and against central differences."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_05978_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _maker(problems, grid, prec, tol, profile_key="coefs"):
    from paper_2010_05978_gb300 import BatchPlan

    def make(th):
        probs = []
        for q in problems:
            fam = dict(q["family"])
            prof = dict(fam["profile"])
            if profile_key == "hg":
                prof["b"], prof["q"] = float(th[0]), float(th[1])
            else:
                prof[profile_key] = th
            fam["profile"] = prof
            probs.append({"families": [fam], "lam": q["lam"], "z": q["z"]})
        return BatchPlan(probs, tol, precision=prec, grid=grid, output="occulter")
    return make


def _loss(u, keep_t):
    return (u.reshape(u.shape[0], -1)[:, keep_t].abs() ** 2).mean()


def fp32_gradient_bar(u_oc, keep, tol, occulter=True):
    """Relative bar (of max |g|) for an FP32 gradient of L = mean |u^oc|^2.

    The fast mode meets tol in relative L2 on the aperture field u^ap, whose
    magnitude is ~1; u^oc = 1 - u^ap is small in the shadow, so its error
    relative to itself is tol |u^ap| / |u^oc| (RMS over the kept targets).
    The gradient (2/M) Re sum conj(u^oc) du^oc/dtheta takes that error
    through the upstream gradient gamma = dL/du^oc, and the adjoint transform
    adds its own relative error ~tol.  Bar = 3 tol (1 + |u^ap| / |u^oc|), the
    factor 3 covering the loss's factor 2 and rounding.  For an aperture
    output (occulter=False) there is no cancellation: the bar is 6 tol."""
    u = u_oc.reshape(u_oc.shape[0], -1)[:, keep]
    rms_oc = float(np.sqrt(np.mean(np.abs(u) ** 2)))
    rms_ap = float(np.sqrt(np.mean(np.abs(1.0 - u) ** 2))) if occulter else rms_oc
    return 3.0 * tol * (1.0 + rms_ap / rms_oc)


def _gpu_loss_grad(theta, problems, grid, keep, prec, tol, key="coefs"):
    from paper_2010_05978_gb300.fresnel import profile_field
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    keep_t = torch.tensor(keep, device="cuda")
    u = profile_field(th, _maker(problems, grid, prec, tol, key))
    L = _loss(u, keep_t)
    L.backward()
    return float(L.detach()), th.grad.numpy().copy()


def _gpu_loss(theta, problems, grid, keep, prec, tol, key="coefs"):
    keep_t = torch.tensor(keep, device="cuda")
    u = _maker(problems, grid, prec, tol, key)(np.asarray(theta, dtype=np.float64)).eval()
    return float(_loss(u, keep_t))


@pytest.mark.parametrize("kind", ["small", "hg24_small"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_profile_gradient_matches_oracle_adjoint(kind, prec):
    from oracle import gradient as G
    theta, problems, grid, keep = W.spline_starshade(kind)
    L_ref, g_ref = G.loss_and_grad(theta, problems, grid, keep)
    tol = 1e-12 if prec == "fp64" else 1e-6
    L, g = _gpu_loss_grad(theta, problems, grid, keep, prec, tol)
    if prec == "fp64":
        bar = 1e-9
    else:
        u = _maker(problems, grid, "fp64", 1e-12)(np.asarray(theta, np.float64)).eval()
        bar = fp32_gradient_bar(u.cpu().numpy(), keep, tol)
    assert abs(L - L_ref) <= bar * L_ref
    assert np.max(np.abs(g - g_ref)) <= bar * np.max(np.abs(g_ref)), (g[:5], g_ref[:5])


def test_profile_gradient_central_differences_c4():
    """C4 at full size: 200 spline coefficients, 8 wavelengths, 256 x 256 pupil
    grid (51,431 kept targets); FP64 adjoint gradient against central
    differences of the FP64 loss (h = 1e-6) at a few coefficients, and the
    FP32 gradient against the FP64 one."""
    theta, problems, grid, keep = W.spline_starshade("c4")
    L, g = _gpu_loss_grad(theta, problems, grid, keep, "fp64", 1e-12)
    h = 1e-6
    for m in (5, 60, 120, 190):
        e = np.zeros_like(theta)
        e[m] = h
        fd = (_gpu_loss(theta + e, problems, grid, keep, "fp64", 1e-12) -
              _gpu_loss(theta - e, problems, grid, keep, "fp64", 1e-12)) / (2 * h)
        assert abs(g[m] - fd) <= 1e-6 * np.max(np.abs(g)), (m, g[m], fd)
    _, g32 = _gpu_loss_grad(theta, problems, grid, keep, "fp32", 1e-6)
    u = _maker(problems, grid, "fp64", 1e-12)(np.asarray(theta, np.float64)).eval()
    bar = fp32_gradient_bar(u.cpu().numpy(), keep, 1e-6)
    err = np.max(np.abs(g32 - g)) / np.max(np.abs(g))
    print("C4 FP32 gradient: error %.2e of max|g|, derived bar %.2e" % (err, bar))
    assert err <= bar


@pytest.mark.parametrize("key", ["hg", "A"])
def test_hg_and_table_profile_gradients(key):
    """Gradients w.r.t. the offset hyper-Gaussian's (b, q) and w.r.t. a
    tabulated A(r_l), against central differences of the FP64 loss."""
    theta_s, problems, grid, keep = W.spline_starshade("small")
    fam = problems[0]["family"]
    if key == "hg":
        theta = np.array([0.35, 4.0])
        prof = {"kind": "hg", "b": 0.35, "q": 4.0}
    else:
        r = 0.4 + 0.6 * (np.polynomial.legendre.leggauss(fam["m"])[0] + 1) / 2
        theta = np.exp(-((r - 0.4) / 0.35) ** 4)
        prof = {"kind": "table", "A": theta}
    problems = [dict(q, family=dict(q["family"], profile=prof)) for q in problems]
    L, g = _gpu_loss_grad(theta, problems, grid, keep, "fp64", 1e-12, key)
    h = 1e-6
    for m in range(min(len(theta), 3)):
        e = np.zeros_like(theta)
        e[m] = h
        fd = (_gpu_loss(theta + e, problems, grid, keep, "fp64", 1e-12, key) -
              _gpu_loss(theta - e, problems, grid, keep, "fp64", 1e-12, key)) / (2 * h)
        assert abs(g[m] - fd) <= 1e-6 * max(np.max(np.abs(g)), 1e-12), (m, g[m], fd)


# ------------------------------------------------------------------ boundary-shape gradients
def _shape_setup(kind):
    """(params, family, lz, grid): "small" an off-centre star with extra modes
    at F ~ 25; "c2" the C2 star r = 1 + 0.3 cos 5t at F = 100 (lz = 0.0169) on
    a reduced rule (32 panels x 16 x 48 radii) and a 64 x 64 grid over
    [-1.5, 1.5)^2."""
    if kind == "small":
        params = np.array(W.STAR_PARAMS, dtype=np.float64)
        params[3], params[4], params[6] = 0.02, -0.015, 0.01
        fam = W.fourier_family(params, 16, 8, 12, cx=0.05, cy=-0.03)
        return params, fam, 0.05, W.grid_spec(48, 48, 2.4 / 48, x0=0.013)
    params = np.array(W.STAR_PARAMS, dtype=np.float64)
    fam = W.fourier_family(params, 32, 16, 48)
    return params, fam, 1.3 ** 2 / 100.0, W.grid_spec(64, 64, 3.0 / 64)


def _shape_maker(fam0, lz, grid, prec, tol, output):
    from paper_2010_05978_gb300 import Plan

    def make(th):
        fam = dict(fam0, params=np.asarray(th, dtype=np.float64))
        return Plan([fam], lz, 1.0, tol, precision=prec, grid=grid, output=output)
    return make


def _shape_loss_grad(params, make):
    from paper_2010_05978_gb300.fresnel import shape_field
    th = torch.tensor(params, dtype=torch.float64, requires_grad=True)
    u = shape_field(th, make)
    L = (u.abs() ** 2).mean()
    L.backward()
    return float(L.detach()), th.grad.numpy().copy(), u.detach().cpu().numpy()


@pytest.mark.parametrize("output", ["aperture", "occulter"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_shape_gradient_matches_oracle_adjoint(prec, output):
    """dL/d(Fourier coefficients) of L = mean |u|^2 over the grid, GPU against
    the oracle's hand-derived adjoint of the direct sum (itself pinned by
    central differences), on an off-centre star with several modes."""
    import oracle
    from oracle import gradient as G
    params, fam, lz, grid = _shape_setup("small")
    xi, eta = oracle.grid_targets(grid["n1"], grid["n2"], grid["h"], grid["x0"], grid["y0"])
    L_ref, g_ref = G.shape_loss_and_grad(params, fam, lz, 1.0, xi, eta, output)
    tol = 1e-12 if prec == "fp64" else 1e-6
    L, g, u = _shape_loss_grad(params, _shape_maker(fam, lz, grid, prec, tol, output))
    if prec == "fp64":
        bar = 1e-9
    else:
        keep = np.ones(u.size, dtype=bool)
        bar = fp32_gradient_bar(u.reshape(1, -1), keep, tol, occulter=output == "occulter")
    assert abs(L - L_ref) <= bar * L_ref
    assert np.max(np.abs(g - g_ref)) <= bar * np.max(np.abs(g_ref)), (g[:5], g_ref[:5])


def test_shape_gradient_central_differences_c2_star():
    """The C2 star at F = 100 on a reduced rule: the FP64 shape gradient
    against central differences (h = 1e-6) of the FP64 GPU loss at r0 and the
    cos 5t, sin 5t and cos 3t coefficients, and the FP32 gradient against the
    FP64 one within the derived bar (aperture output: 6 tol)."""
    params, fam, lz, grid = _shape_setup("c2")
    make64 = _shape_maker(fam, lz, grid, "fp64", 1e-12, "aperture")
    L, g, _ = _shape_loss_grad(params, make64)

    def loss(th):
        u = make64(th).eval()
        return float((u.abs() ** 2).mean())
    h = 1e-6
    for k in (0, 5, 9, 10):
        e = np.zeros_like(params)
        e[k] = h
        fd = (loss(params + e) - loss(params - e)) / (2 * h)
        assert abs(g[k] - fd) <= 1e-6 * np.max(np.abs(g)), (k, g[k], fd)
    _, g32, u32 = _shape_loss_grad(params, _shape_maker(fam, lz, grid, "fp32", 1e-6, "aperture"))
    bar = fp32_gradient_bar(u32.reshape(1, -1), np.ones(u32.size, dtype=bool), 1e-6,
                            occulter=False)
    err = np.max(np.abs(g32 - g)) / np.max(np.abs(g))
    print("C2 star FP32 shape gradient: error %.2e of max|g|, bar %.2e" % (err, bar))
    assert err <= bar
