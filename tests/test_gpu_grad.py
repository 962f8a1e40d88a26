"""GPU profile gradients (fresnel_grad_profile through torch autograd) against
the oracle's hand-derived adjoint and against central differences."""
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


def _gpu_loss_grad(theta, problems, grid, keep, prec, tol, key="coefs"):
    from paper_2010_05978_gb300.fresnel import profile_field
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    keep_t = torch.tensor(keep, device="cuda")
    u = profile_field(th, _maker(problems, grid, prec, tol, key))
    L = _loss(u, keep_t)
    L.backward()
    return float(L), th.grad.numpy().copy()


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
    bar = 1e-9 if prec == "fp64" else 2e-4
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
    assert np.max(np.abs(g32 - g)) <= 1e-3 * np.max(np.abs(g))


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
