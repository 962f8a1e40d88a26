"""GPU parity for starshade (petal) quadrature, Sec. 4.2: the CUDA path
through the C ABI against the CPU oracle's own starshade rule and direct sum."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import quadrature as Q

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


def plan(*a, **k):
    from paper_2010_05978_gb300 import Plan
    return Plan(*a, **k)


BARS = {"fp64": (1e-12, 1e-10), "fp32": (1e-6, 1e-6)}
HG = {"kind": "hg", "b": W.HG24["b"], "q": W.HG24["q"]}


def hg24(lam):
    F = W.HG24["R"] ** 2 / (lam * W.HG24["z"])
    m, n_p, n_d, m_d = W.starshade_resolution(F, W.HG24["n_petals"])
    return W.petal_family(24, 6.0, 14.0, HG, m, n_p, n_d, m_d)


def _random_bspline(n=20, stream=0):
    g = W.rng(4, stream)
    return {"kind": "bspline", "coefs": 0.5 + 0.4 * g.random(n)}


@pytest.mark.parametrize("fam", [
    hg24(600e-9),
    W.petal_family(7, 0.8, 2.0, _random_bspline(), 23, 11, 0, 0, cx=0.3, cy=-0.4),
    W.petal_family(5, 0.4, 1.0, {"kind": "table", "A": np.linspace(1.0, 0.1, 17)}, 17, 9, 31, 5),
    W.petal_family(3, 0.0, 1.0, {"kind": "hg", "b": 0.5, "q": 2.5}, 8, 4),
])
def test_petal_nodes_match_oracle(fam):
    p = plan([fam], 1e-6, 1e4, 1e-6, grid=W.grid_spec(64, 64, 0.05))
    x, y, w = (t.cpu().numpy() for t in p.nodes())
    ox, oy, ow = Q.family_nodes(fam)
    assert len(x) == len(ox)
    scale = fam["R"] + abs(fam["cx"]) + abs(fam["cy"])
    assert np.max(np.abs(x - ox)) < 4e-15 * scale and np.max(np.abs(y - oy)) < 4e-15 * scale
    assert np.max(np.abs(w - ow)) < 1e-13 * np.max(np.abs(ow))
    p.close()


def _grid_sample(g, count, stream):
    xi, eta = oracle.grid_targets(g["n1"], g["n2"], g["h"], g["x0"], g["y0"])
    idx = W.rng(3, stream).choice(len(xi), count, replace=False)
    return xi, eta, idx


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("lam", [400e-9, 1000e-9])
def test_starshade_t1_pupil_grid_sampled(prec, lam):
    """24-petal HG occulter, 512 x 512 grid over the 2.4 m pupil, sampled targets."""
    fam = [hg24(lam)]
    z = W.HG24["z"]
    g = W.grid_spec(512, 512, 2.4 / 512)
    xi, eta, idx = _grid_sample(g, 1500, 1)
    tol, bar = BARS[prec]
    u_ap = plan(fam, lam, z, tol, precision=prec, grid=g).eval().cpu().numpy().ravel()
    u_oc = plan(fam, lam, z, tol, precision=prec, grid=g,
                output="occulter").eval().cpu().numpy().ravel()
    ref = oracle.field(fam, lam, z, xi[idx], eta[idx])
    assert rel_l2(u_ap[idx], ref) <= bar
    # the paper's metric: absolute error of u^oc = 1 - u^ap (eq. bab)
    assert np.max(np.abs(u_oc[idx] - (1.0 - ref))) <= 4 * bar


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_starshade_t3_pupil_disc(prec):
    lam, z = 700e-9, W.HG24["z"]
    fam = [hg24(lam)]
    xi, eta = W.disc_targets(3000, 1.2, 7)
    t = torch.tensor(np.stack([xi, eta], 1), dtype=torch.float64, device="cuda")
    tol, bar = BARS[prec]
    u = plan(fam, lam, z, tol, precision=prec, box=(-1.2, 1.2, -1.2, 1.2),
             output="occulter").eval(t).cpu().numpy()
    ref = oracle.field(fam, lam, z, xi, eta, output="occulter")
    assert np.max(np.abs(u - ref)) <= 4 * bar
    assert rel_l2(1.0 - u, 1.0 - ref) <= bar


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_starshade_bspline_profile_off_centre_t1(prec):
    """Spline profile, no disc, translated shape, moderate Fresnel number (full grid)."""
    fam = [W.petal_family(7, 0.8, 2.0, _random_bspline(), 40, 24, 0, 0, cx=0.3, cy=-0.4)]
    lz = 0.2
    g = W.grid_spec(90, 70, 0.05, x0=0.1)
    xi, eta = oracle.grid_targets(g["n1"], g["n2"], g["h"], g["x0"], g["y0"])
    ref = oracle.field(fam, lz, 1.0, xi, eta).reshape(g["n2"], g["n1"])
    tol, bar = BARS[prec]
    u = plan(fam, lz, 1.0, tol, precision=prec, grid=g).eval().cpu().numpy()
    assert rel_l2(u, ref) <= bar


def _moved_starshade():
    """A 6-petal starshade with seeded small rigid motions of every petal
    (Sec. 5: perturbed starshades, moved petals plus root-arc patches)."""
    fam = W.petal_family(6, 0.4, 1.0, {"kind": "hg", "b": 0.5, "q": 2.5}, 40, 20, 64, 24,
                         cx=0.03, cy=-0.02)
    g = W.rng(61, 0)
    motion = np.column_stack([g.normal(0, 0.01, 6), g.normal(0, 0.006, 6), g.normal(0, 0.006, 6)])
    return dict(fam, motion=motion)


def test_moved_petal_nodes_match_oracle():
    fam = _moved_starshade()
    p = plan([fam], 0.05, 1.0, 1e-12, precision="fp64", grid=W.grid_spec(64, 64, 0.04))
    x, y, w = (t.cpu().numpy() for t in p.nodes())
    ox, oy, ow = Q.family_nodes(fam)
    assert len(x) == len(ox)
    assert np.max(np.abs(x - ox)) < 5e-15 and np.max(np.abs(y - oy)) < 5e-15
    assert np.max(np.abs(w - ow)) < 1e-15


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_moved_petals_field(prec):
    fam = [_moved_starshade()]
    tol, bar = BARS[prec]
    g = W.grid_spec(96, 96, 0.025)
    xi, eta = oracle.grid_targets(96, 96, 0.025)
    ref = oracle.field(fam, 0.05, 1.0, xi, eta, output="occulter").reshape(96, 96)
    u = plan(fam, 0.05, 1.0, tol, precision=prec, grid=g, output="occulter").eval()
    assert rel_l2(u.cpu().numpy(), ref) <= bar
    xs, es = W.disc_targets(2000, 1.2, 62)
    ref3 = oracle.field(fam, 0.05, 1.0, xs, es)
    p3 = plan(fam, 0.05, 1.0, tol, precision=prec, box=(-1.2, 1.2, -1.2, 1.2))
    u3 = p3.eval(torch.tensor(np.stack([xs, es], 1), device="cuda")).cpu().numpy()
    assert rel_l2(u3, ref3) <= bar


def test_moved_petals_rejected_by_profile_gradients():
    from paper_2010_05978_gb300 import FresnelError
    fam = W.petal_family(6, 0.4, 1.0, {"kind": "bspline", "coefs": np.full(8, 0.6)}, 12, 8)
    fam = dict(fam, motion=np.zeros((6, 3)))
    p = plan([fam], 0.05, 1.0, 1e-12, precision="fp64", grid=W.grid_spec(32, 32, 0.05))
    with pytest.raises(FresnelError):
        p.grad_profile(torch.ones((32, 32), dtype=torch.complex128, device="cuda"))
    with pytest.raises(FresnelError):   # a motion on a non-petal family
        plan([dict(W.fourier_family([1.0], 16, 8, 8), motion=np.zeros((16, 3)))], 0.05, 1.0,
             1e-6, grid=W.grid_spec(32, 32, 0.05))
