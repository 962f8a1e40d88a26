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


# ------------------------------------------------------------------ scattered-target batches
def _scattered_problems():
    return [
        {"families": [W.fourier_family(W.STAR_PARAMS, 32, 16, 32, cx=0.1)], "lam": 0.03, "z": 1.0},
        {"families": [W.fourier_family([1.0], 24, 16, 24)], "lam": 0.1, "z": 1.0},
        {"families": [W.petal_family(5, 0.4, 1.0, {"kind": "hg", "b": 0.35, "q": 4},
                                     30, 20, 40, 30)], "lam": 0.05, "z": 1.0},
    ]


def _targets(counts, half=1.5):
    xs, ys = [], []
    for i, m in enumerate(counts):
        x, y = W.square_targets(m, half, 11, 300 + i)
        xs.append(x)
        ys.append(y)
    xi, eta = np.concatenate(xs), np.concatenate(ys)
    t = torch.tensor(np.stack([xi, eta], 1), dtype=torch.float64, device="cuda")
    return xi, eta, t


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_scattered_batch_matches_oracle_and_single_plans(prec):
    from paper_2010_05978_gb300 import BatchPlan, Plan
    probs = _scattered_problems()
    counts = [700, 0, 40000]     # an empty problem and one large enough to bin (FP32)
    xi, eta, t = _targets(counts)
    tol, bar = BARS[prec]
    box = (-1.5, 1.5, -1.5, 1.5)
    p = BatchPlan(probs, tol, precision=prec, box=box, output="occulter")
    u = p.eval(t, counts).cpu().numpy()
    off = 0
    for b, q in enumerate(probs):
        m = counts[b]
        if m:
            sl = slice(off, off + m)
            idx = np.arange(off, off + m)[:: max(1, m // 300)]
            ref = oracle.field(q["families"], q["lam"], q["z"], xi[idx], eta[idx], output="occulter")
            assert rel_l2(1.0 - u[idx], 1.0 - ref) <= bar, b
            single = Plan(q["families"], q["lam"], q["z"], tol, precision=prec, box=box,
                          output="occulter").eval(t[sl].contiguous()).cpu().numpy()
            assert np.max(np.abs(single - u[sl])) <= (1e-13 if prec == "fp64" else 2e-6)
        off += m
    p.check()


def test_scattered_batch_graph_replay_and_recapture():
    from paper_2010_05978_gb300 import BatchPlan
    probs = _scattered_problems()
    p = BatchPlan(probs, 1e-12, precision="fp64", box=(-1.5, 1.5, -1.5, 1.5))
    counts = [300, 200, 100]
    xi, eta, t = _targets(counts)
    out = torch.empty(sum(counts), dtype=torch.complex128, device="cuda")
    a = p.eval(t, counts, out).cpu().numpy()
    for _ in range(3):                       # replays of the captured graph
        b = p.eval(t, counts, out).cpu().numpy()
        # equal up to the order of the atomic adds into shared spreading tiles
        assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(a))
    counts2 = [100, 300, 200]                # new counts: captured again
    xi2, eta2, t2 = _targets(counts2)
    c = p.eval(t2, counts2).cpu().numpy()
    ref = oracle.field(probs[1]["families"], probs[1]["lam"], 1.0, xi2[100:400], eta2[100:400])
    assert rel_l2(c[100:400], ref) <= 1e-10
    info = p.info()
    assert info["n_nodes"] == sum(len(oracle.nodes(q["families"])[0]) for q in probs)


def test_random_star_batch32_full_size_sampled():
    """32 uneven instances (1e5-2e6 nodes, F = 100..450, 1e5-1e7 targets each,
    5.5e7 in all) in one batched evaluation, FP32 fast mode; 20 sampled
    targets per instance against the oracle."""
    from paper_2010_05978_gb300 import BatchPlan
    probs, counts = W.random_star_batch()
    total = sum(counts)
    t = torch.empty((total, 2), dtype=torch.float64, device="cuda")
    samples = []
    off = 0
    for i, m in enumerate(counts):
        x, y = W.square_targets(m, 1.2, 5, 100 + i)
        t[off:off + m, 0].copy_(torch.from_numpy(x))
        t[off:off + m, 1].copy_(torch.from_numpy(y))
        idx = W.rng(5, 500 + i).choice(m, 20, replace=False)
        samples.append((off + idx, x[idx], y[idx]))
        off += m
    p = BatchPlan(probs, 1e-6, precision="fp32", box=(-1.2, 1.2, -1.2, 1.2))
    u = p.eval(t, counts)
    for (gidx, x, y), q in zip(samples, probs):
        got = u[torch.tensor(gidx, device="cuda")].cpu().numpy()
        ref = oracle.field(q["families"], q["lam"], q["z"], x, y)
        assert rel_l2(got, ref) <= 1e-6
    p.check()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_direct_column_dft_matches_fft_path(prec):
    """One wavelength of the sweep: its grid has one live tile row, so the
    column pass is the direct DFT over the live rows; the same plan forced
    onto the four-step FFT (no row pruning, FFT column pass) gives the same
    grid."""
    from paper_2010_05978_gb300 import Plan
    cfg = W.starshade_sweep(n_lambda=3)
    q, g = cfg["problems"][1], cfg["grid"]
    tol = 1e-12 if prec == "fp64" else 1e-6
    u = Plan(q["families"], q["lam"], q["z"], tol, precision=prec, grid=g,
             output="occulter").eval().cpu().numpy()
    v = Plan(q["families"], q["lam"], q["z"], tol, precision=prec, grid=g, output="occulter",
             fft_split_above=256).eval().cpu().numpy()
    assert rel_l2(1.0 - u, 1.0 - v) <= (1e-12 if prec == "fp64" else 2e-6)


@pytest.mark.parametrize("n", [512, 480])
def test_one_live_row_fp64_pruned_fft(n):
    """FP64 plan whose nodes occupy one tile row: the column pass is the
    pruned FFT (32-point DFTs of the twiddled live rows), for a power-of-two
    column length (n = 512: 1024) and one that is not (n = 480: 960); it
    equals the unpruned four-step FFT path and the oracle's direct sum."""
    from paper_2010_05978_gb300 import Plan
    cfg = W.starshade_sweep(n_lambda=3, n=n)
    q, g = cfg["problems"][1], cfg["grid"]
    p = Plan(q["families"], q["lam"], q["z"], 1e-12, precision="fp64", grid=g,
             output="occulter")
    assert p.info()["live_tile_rows"] == 1
    u = p.eval().cpu().numpy()
    v = Plan(q["families"], q["lam"], q["z"], 1e-12, precision="fp64", grid=g, output="occulter",
             fft_split_above=256).eval().cpu().numpy()
    assert rel_l2(1.0 - u, 1.0 - v) <= 1e-12
    xi, eta = oracle.grid_targets(g["n1"], g["n2"], g["h"])
    idx = W.rng(6, n).choice(len(xi), 300, replace=False)
    ref = oracle.field(q["families"], q["lam"], q["z"], xi[idx], eta[idx])
    assert rel_l2(1.0 - u.ravel()[idx], ref) <= 1e-10

