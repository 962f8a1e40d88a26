"""GPU test of the spreading primitive (fresnel_spread) against a direct
numpy spreader written here: b[l2, l1] = sum_j c_j psi(l1 - g1_j) psi(l2 - g2_j)
on a periodic grid, psi the exponential-of-semicircle kernel."""
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


def psi(u, w, beta):
    z = 2.0 * u / w
    a = 1.0 - z * z
    return np.where(a > 0, np.exp(beta * (np.sqrt(np.maximum(a, 0.0)) - 1.0)), 0.0)


def numpy_spread(g1, g2, c, nf1, nf2, w, beta):
    grid = np.zeros((nf2, nf1), np.complex128)
    for o1 in range(-(w // 2) - 1, w // 2 + 2):
        l1 = np.floor(g1).astype(np.int64) + o1
        k1 = psi(l1 - g1, w, beta)
        for o2 in range(-(w // 2) - 1, w // 2 + 2):
            l2 = np.floor(g2).astype(np.int64) + o2
            k2 = psi(l2 - g2, w, beta)
            np.add.at(grid, (l2 % nf2, l1 % nf1), c * k1 * k2)
    return grid


def points(seed, n, nf1, nf2):
    g = W.rng(300 + seed, 0)
    g1 = g.uniform(0, nf1, n)
    g2 = g.uniform(0, nf2, n)
    # a dense cluster straddling the periodic corner (split tiles + wrap)
    m = n // 3
    g1[:m] = g.uniform(-1.0, 1.0, m)
    g2[:m] = g.uniform(-1.0, 1.0, m)
    # some coordinates far outside [0, nf) (taken modulo nf)
    g1[m:m + 50] += 5 * nf1
    g2[m + 50:m + 100] -= 3 * nf2
    c = (g.normal(size=n) + 1j * g.normal(size=n)).astype(np.complex64)
    return g1, g2, c


def to_dev(g1, g2, c):
    return (torch.tensor(g1, dtype=torch.float64, device="cuda"),
            torch.tensor(g2, dtype=torch.float64, device="cuda"),
            torch.tensor(c, dtype=torch.complex64, device="cuda"))


@pytest.mark.parametrize("w", [7, 8, 13])
def test_spread_matches_numpy(w):
    from paper_2010_05978_gb300.fresnel import fresnel_spread
    nf1, nf2 = 128, 96
    beta = 2.30 * w
    g1, g2, c = points(w, 6000, nf1, nf2)
    ref = numpy_spread(g1, g2, c.astype(np.complex128), nf1, nf2, w, beta)
    out = fresnel_spread(*to_dev(g1, g2, c), nf1, nf2, w, beta).cpu().numpy()
    err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    assert err < 2e-6, err


def test_spread_empty_and_bad_input():
    from paper_2010_05978_gb300 import FresnelError
    from paper_2010_05978_gb300.fresnel import fresnel_spread
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    ec = torch.empty(0, dtype=torch.complex64, device="cuda")
    out = torch.full((64, 64), 3.0 + 1j, dtype=torch.complex64, device="cuda")
    fresnel_spread(e, e, ec, 64, 64, 8, 18.4, out=out)
    assert torch.count_nonzero(out).item() == 0
    g1 = torch.tensor([1.0, float("nan")], dtype=torch.float64, device="cuda")
    g2 = torch.tensor([1.0, 2.0], dtype=torch.float64, device="cuda")
    cc = torch.ones(2, dtype=torch.complex64, device="cuda")
    with pytest.raises(FresnelError) as ex:
        fresnel_spread(g1, g2, cc, 64, 64, 8, 18.4)
    assert ex.value.status == -6
    with pytest.raises(FresnelError):
        fresnel_spread(g1, g2, cc, 60, 64, 8, 18.4)   # not a multiple of 32
