"""Source-plane screens (Sec. 5: the weight of each areal node times the
source term s = A exp(2 pi i OPD / lambda)) on the GPU against the oracle's
screened direct sum, through every node path: the dilation rule in
double-float (FP32) and FP64, starshade petals in double-float, explicit
nodes, type 1 and type 3, and a batch of two wavelengths (one screen, the
phase scaled by each problem's 1/lambda)."""
import importlib

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
FL = importlib.import_module("oracle.field")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_05978_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def plan(*a, **k):
    from paper_2010_05978_gb300 import Plan
    return Plan(*a, **k)


BARS = {"fp64": (1e-12, 1e-10), "fp32": (1e-6, 1e-6)}


def smooth_screen(box, n1=41, n2=37, lam=0.02, scale=1.0):
    """A smooth amplitude and an OPD of about one wave (the FP32 screen phase
    carries ~1e-7 of its range), sampled on the box."""
    xs = np.linspace(box[0], box[1], n1)
    ys = np.linspace(box[2], box[3], n2)
    X, Y = np.meshgrid(xs / scale, ys / scale)
    amp = 0.8 + 0.2 * np.cos(1.3 * X) * np.sin(0.9 * Y + 0.3)
    opd = 0.3 * lam * (1.5 * X * Y + 0.8 * np.sin(2.1 * X - 0.4 * Y) + 0.3 * X * X)
    return {"amp": amp, "opd": opd, "box": box}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_screen_t3_star(prec):
    fam = [W.fourier_family(W.STAR_PARAMS, 32, 16, 48, cx=0.05, cy=-0.03)]
    lam, z = 0.02, 2.5
    sc = smooth_screen((-1.6, 1.6, -1.6, 1.6), lam=lam)
    xi, eta = W.disc_targets(3000, 1.5, 51)
    ref = FL.field(fam, lam, z, xi, eta, screen=sc)
    tol, bar = BARS[prec]
    p = plan(fam, lam, z, tol, precision=prec, box=(-1.5, 1.5, -1.5, 1.5), screen=sc)
    u = p.eval(torch.tensor(np.stack([xi, eta], 1), device="cuda")).cpu().numpy()
    assert rel_l2(u, ref) <= bar


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_screen_t1_grid_occulter(prec):
    fam = [W.fourier_family([1.0, 0.1, 0.0, 0.05, 0.0], 32, 16, 40)]
    lam, z = 0.01, 5.0
    sc = smooth_screen((-1.5, 1.5, -1.5, 1.5), 33, 35, lam=lam)
    g = W.grid_spec(96, 80, 0.03, x0=0.05, y0=-0.02)
    xi, eta = oracle.grid_targets(96, 80, 0.03, 0.05, -0.02)
    ref = FL.field(fam, lam, z, xi, eta, output="occulter", screen=sc).reshape(80, 96)
    tol, bar = BARS[prec]
    u = plan(fam, lam, z, tol, precision=prec, grid=g, output="occulter", screen=sc).eval()
    assert rel_l2(u.cpu().numpy(), ref) <= bar


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_screen_petals_and_explicit_nodes(prec):
    """Starshade petals (FP32: the double-float petal form) plus a family of
    explicit nodes in one plan."""
    hg = {"kind": "hg", "b": 0.5, "q": 2.5}
    petals = W.petal_family(6, 0.4, 1.0, hg, 24, 12, 20, 8, cx=0.1, cy=0.05)
    g = W.rng(52, 0)
    nodes = {"kind": "nodes", "x": g.uniform(-1.0, 1.0, 400), "y": g.uniform(-1.0, 1.0, 400),
             "w": g.normal(0, 1e-3, 400)}
    fam = [petals, nodes]
    lam, z = 0.02, 2.0
    sc = smooth_screen((-1.3, 1.3, -1.3, 1.3), 30, 30, lam=lam)
    xi, eta = W.disc_targets(2000, 1.2, 53)
    ref = FL.field(fam, lam, z, xi, eta, screen=sc)
    tol, bar = BARS[prec]
    p = plan(fam, lam, z, tol, precision=prec, box=(-1.2, 1.2, -1.2, 1.2), screen=sc)
    u = p.eval(torch.tensor(np.stack([xi, eta], 1), device="cuda")).cpu().numpy()
    assert rel_l2(u, ref) <= bar


def test_screen_batch_of_wavelengths():
    """One OPD screen, two wavelengths in a batched grid plan: the phase
    2 pi OPD / lambda follows each problem's lambda."""
    from paper_2010_05978_gb300 import BatchPlan
    fam = [W.fourier_family([1.0, 0.0, 0.08], 32, 16, 40)]
    sc = smooth_screen((-1.4, 1.4, -1.4, 1.4), 29, 29, lam=0.015)
    g = W.grid_spec(64, 64, 0.04)
    xi, eta = oracle.grid_targets(64, 64, 0.04)
    probs = [{"families": fam, "lam": lam, "z": 3.0} for lam in (0.01, 0.016)]
    u = BatchPlan(probs, 1e-12, precision="fp64", grid=g, screen=sc).eval().cpu().numpy()
    for b, q in enumerate(probs):
        ref = FL.field(fam, q["lam"], q["z"], xi, eta, screen=sc).reshape(64, 64)
        assert rel_l2(u[b], ref) <= 1e-10


def test_screen_rejected_by_line_integral_and_gradients():
    from paper_2010_05978_gb300 import FresnelError
    fam = [W.fourier_family([1.0], 32, 16, 16)]
    sc = smooth_screen((-1.3, 1.3, -1.3, 1.3), 9, 9)
    p = plan(fam, 0.02, 1.0, 1e-12, precision="fp64", box=(-1, 1, -1, 1), screen=sc)
    t = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(FresnelError):
        p.nsli(t)
    with pytest.raises(FresnelError):
        plan(fam, 0.02, 1.0, 1e-6, box=(-1, 1, -1, 1),
             screen={"amp": np.ones((3, 9)), "box": (-1, 1, -1, 1)})
    petals = W.petal_family(6, 0.4, 1.0, {"kind": "bspline", "coefs": np.full(8, 0.6)}, 12, 8)
    q = plan([petals], 0.02, 1.0, 1e-12, precision="fp64", grid=W.grid_spec(32, 32, 0.05),
             screen=sc)
    with pytest.raises(FresnelError):
        q.grad_profile(torch.ones((32, 32), dtype=torch.complex128, device="cuda"))
