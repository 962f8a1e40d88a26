"""GPU parity of batched plans (fresnel_plan_many / fresnel_eval_many): many
independent problems (wavelengths, shapes) on one target grid."""
import numpy as np
import pytest

import oracle
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


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


BARS = {"fp64": (1e-12, 1e-10), "fp32": (1e-6, 1e-6)}


def _mixed_problems():
    hg = {"kind": "hg", "b": 0.35, "q": 4}
    return [
        {"families": [W.fourier_family([1.0], 32, 16, 24)], "lam": 0.05, "z": 1.0},
        {"families": [W.fourier_family(W.STAR_PARAMS, 32, 16, 32, cx=0.1)], "lam": 0.02, "z": 1.5},
        {"families": [W.petal_family(5, 0.4, 1.0, hg, 40, 30, 60, 40)], "lam": 0.07, "z": 1.0},
        {"families": [W.fourier_family([0.5], 16, 8, 8),
                      W.petal_family(3, 0.2, 0.9, hg, 20, 12, 0, 0, cx=-0.3)], "lam": 0.04, "z": 2.0},
    ]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("output", ["aperture", "occulter"])
def test_batch_matches_oracle_and_single_plans(prec, output):
    from paper_2010_05978_gb300 import BatchPlan, Plan
    probs = _mixed_problems()
    g = W.grid_spec(72, 50, 0.04, x0=0.02)
    tol, bar = BARS[prec]
    u = BatchPlan(probs, tol, precision=prec, grid=g, output=output).eval().cpu().numpy()
    assert u.shape == (len(probs), 50, 72)
    xi, eta = oracle.grid_targets(g["n1"], g["n2"], g["h"], g["x0"], g["y0"])
    for b, q in enumerate(probs):
        ref = oracle.field(q["families"], q["lam"], q["z"], xi, eta).reshape(50, 72)
        ap = u[b] if output == "aperture" else 1.0 - u[b]
        assert rel_l2(ap, ref) <= bar, b
        single = Plan(q["families"], q["lam"], q["z"], tol, precision=prec, grid=g,
                      output=output).eval().cpu().numpy()
        assert np.max(np.abs(single - u[b])) <= (1e-13 if prec == "fp64" else 2e-6) * np.max(np.abs(u[b]))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_starshade_wavelength_sweep_sampled(prec):
    """The 24-petal HG starshade at 8 wavelengths in [400, 1000] nm (uneven
    node counts), 512 x 512 pupil grid, occulter output, sampled targets."""
    from paper_2010_05978_gb300 import BatchPlan
    cfg = W.starshade_sweep(n_lambda=8)
    g = cfg["grid"]
    tol, bar = BARS[prec]
    u = BatchPlan(cfg["problems"], tol, precision=prec, grid=g, output="occulter",
                  recompute_nodes=True).eval().cpu().numpy().reshape(8, -1)
    xi, eta = oracle.grid_targets(g["n1"], g["n2"], g["h"])
    for b, q in enumerate(cfg["problems"]):
        idx = W.rng(3, 10 + b).choice(len(xi), 400, replace=False)
        ref = oracle.field(q["families"], q["lam"], q["z"], xi[idx], eta[idx], output="occulter")
        assert np.max(np.abs(u[b, idx] - ref)) <= 4 * bar, b
        assert rel_l2(1.0 - u[b, idx], 1.0 - ref) <= bar, b


def test_batch_repeated_evaluation_is_stable():
    """Recomputed nodes and sort each call: results repeat (FP64 bit-for-bit up
    to atomic order in split tiles) and the device status stays clean."""
    from paper_2010_05978_gb300 import BatchPlan
    probs = _mixed_problems()
    g = W.grid_spec(40, 40, 0.05)
    p = BatchPlan(probs, 1e-12, precision="fp64", grid=g, recompute_nodes=True)
    a = p.eval().cpu().numpy()
    for _ in range(3):
        b = p.eval().cpu().numpy()
    assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(a))
    p.check()


def test_single_eval_rejects_batched_plan():
    from paper_2010_05978_gb300 import BatchPlan, FresnelError
    from paper_2010_05978_gb300.fresnel import load_library
    probs = _mixed_problems()[:2]
    p = BatchPlan(probs, 1e-6, grid=W.grid_spec(16, 16, 0.1))
    out = torch.empty(256, dtype=torch.complex64, device="cuda")
    assert load_library().fresnel_eval(p.handle, None, 256, out.data_ptr()) == -1
    with pytest.raises(FresnelError):
        from paper_2010_05978_gb300.fresnel import _check
        _check(load_library().fresnel_eval(p.handle, None, 256, out.data_ptr()))
