"""GPU test of fresnel_spread_noalloc, the spreading entry point for callers
that cannot allocate device memory (a framework that owns the memory pool
forbids allocations it does not make; an embedded caller forbids allocation
after start-up).  It must give
the same grid as fresnel_spread, which allocates its scratch, on two calls in
a row (the second call must not see the first call's leftover scratch).

The file name sorts last so that, in a run that stops at the first failure,
every other test has already run.  It also passes on its own in a fresh
process."""
import ctypes

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


def _inputs(seed, n, nf1, nf2):
    g = W.rng(400 + seed, 0)
    g1 = g.uniform(0, nf1, n)
    g2 = g.uniform(0, nf2, n)
    m = n // 4                       # dense cluster across the periodic corner
    g1[:m] = g.uniform(-1.5, 1.5, m)
    g2[:m] = g.uniform(-1.5, 1.5, m)
    c = (g.normal(size=n) + 1j * g.normal(size=n)).astype(np.complex64)
    return (torch.tensor(g1, dtype=torch.float64, device="cuda"),
            torch.tensor(g2, dtype=torch.float64, device="cuda"),
            torch.tensor(c, dtype=torch.complex64, device="cuda"))


def _call_noalloc_cabi(g1, g2, c, nf1, nf2, w, beta, out):
    """Direct C-ABI call (ctypes), no binding helper in between."""
    from paper_2010_05978_gb300 import fresnel
    lib = fresnel.load_library()
    st = torch.cuda.current_stream().cuda_stream
    return lib.fresnel_spread_noalloc(g1.data_ptr(), g2.data_ptr(), c.data_ptr(), g1.numel(),
                                      nf1, nf2, w, beta, out.data_ptr(), ctypes.c_void_p(st))


def test_noalloc_matches_allocating_spread_twice():
    from paper_2010_05978_gb300.fresnel import fresnel_spread
    cases = [(1, 40000, 256, 192, 8), (2, 25000, 128, 128, 7)]   # two calls in a row
    for seed, n, nf1, nf2, w in cases:
        g1, g2, c = _inputs(seed, n, nf1, nf2)
        beta = 2.30 * w
        ref = fresnel_spread(g1, g2, c, nf1, nf2, w, beta).cpu().numpy()
        out = torch.full((nf2, nf1), 7.0 - 3.0j, dtype=torch.complex64, device="cuda")
        assert _call_noalloc_cabi(g1, g2, c, nf1, nf2, w, beta, out) == 0
        got = out.cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 2e-6, (seed, err)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2010_05978_gb300 import fresnel
    lib = fresnel.load_library()
    n = 65537                      # one more than FRESNEL_SPREAD_NOALLOC_MAX_POINTS
    g1 = torch.zeros(n, dtype=torch.float64, device="cuda")
    c = torch.zeros(n, dtype=torch.complex64, device="cuda")
    out = torch.zeros((64, 64), dtype=torch.complex64, device="cuda")
    assert _call_noalloc_cabi(g1, g1, c, 64, 64, 8, 18.4, out) == -5
    assert "MAX_POINTS" in lib.fresnel_last_error().decode()
    g1 = torch.zeros(10, dtype=torch.float64, device="cuda")
    c = torch.zeros(10, dtype=torch.complex64, device="cuda")
    big = torch.zeros((4096, 2048 + 32), dtype=torch.complex64, device="cuda")
    assert _call_noalloc_cabi(g1, g1, c, 2048 + 32, 4096, 8, 18.4, big) == -5
