"""Four-step FFT lengths (transforms beyond one shared-memory pass) and the
Fresnel-number-1000 workload that needs them, against the CPU oracle."""
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


def plan(*a, **k):
    from paper_2010_05978_gb300 import Plan
    return Plan(*a, **k)


BARS = {"fp64": (1e-12, 1e-10), "fp32": (1e-6, 1e-6)}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("output", ["aperture", "occulter"])
def test_t1_four_step_matches_oracle(prec, output):
    """Type 1 on a ragged offset grid with every FFT length split in two."""
    fam = [W.fourier_family(W.STAR_PARAMS, 32, 16, 48, cx=0.05, cy=0.02)]
    lz = 0.05
    g = W.grid_spec(301, 250, 0.011, x0=0.13, y0=-0.07)
    xi, eta = oracle.grid_targets(g["n1"], g["n2"], g["h"], g["x0"], g["y0"])
    ref = oracle.field(fam, lz, 1.0, xi, eta, output=output).reshape(g["n2"], g["n1"])
    tol, bar = BARS[prec]
    p = plan(fam, lz, 1.0, tol, precision=prec, grid=g, output=output, fft_split_above=64)
    u = p.eval().cpu().numpy()
    ref_ap = ref if output == "aperture" else 1.0 - ref
    u_ap = u if output == "aperture" else 1.0 - u
    assert rel_l2(u_ap, ref_ap) <= bar
    one = plan(fam, lz, 1.0, tol, precision=prec, grid=g, output=output).eval().cpu().numpy()
    assert np.max(np.abs(one - u)) <= (1e-12 if prec == "fp64" else 2e-6) * np.max(np.abs(u))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_t3_four_step_matches_oracle(prec):
    fam = [W.fourier_family(W.STAR_PARAMS, 48, 16, 64, cx=0.02)]
    lz = 0.03
    xi, eta = W.disc_targets(5000, 1.5, 9)
    t = torch.tensor(np.stack([xi, eta], 1), dtype=torch.float64, device="cuda")
    tol, bar = BARS[prec]
    box = (-1.5, 1.5, -1.5, 1.5)
    u = plan(fam, lz, 1.0, tol, precision=prec, box=box, fft_split_above=100).eval(t).cpu().numpy()
    ref = oracle.field(fam, lz, 1.0, xi, eta)
    assert rel_l2(u, ref) <= bar


def test_random_star_F1000_t3_full_size_sampled():
    """F = 1000 random smooth aperture (640 x 16 x 1024 = 10,485,760 nodes),
    type 3 to 1e8 targets uniform in [-1.2, 1.2]^2 in FP32 fast mode: the FFT
    grid (~17k per side) takes the four-step path and the target binning its
    multi-block scan.  Sampled targets against the oracle's direct sum."""
    cfg = W.random_star()
    M = 100_000_000
    xi, eta = W.square_targets(M, 1.2, 5)
    t = torch.empty((M, 2), dtype=torch.float64, device="cuda")
    t[:, 0].copy_(torch.from_numpy(xi))
    t[:, 1].copy_(torch.from_numpy(eta))
    p = plan(cfg["families"], cfg["lam"], cfg["z"], 1e-6, precision="fp32",
             box=(-1.2, 1.2, -1.2, 1.2))
    info = p.info()
    assert info["nfft1"] > 13000 and info["n_nodes"] == 10_485_760
    u = p.eval(t)
    idx = W.rng(5, 7).choice(M, 300, replace=False)
    idx[:2] = [0, M - 1]
    got = u[torch.tensor(idx, device="cuda")].cpu().numpy()
    ref = oracle.field(cfg["families"], cfg["lam"], cfg["z"], xi[idx], eta[idx])
    assert rel_l2(got, ref) <= 1e-6
    del u, t
    p.close()
