"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bars (relative L2 over the evaluated targets): <= 1e-10 in FP64 mode at
tol 1e-12, <= tol in FP32 fast mode (the requested tolerance itself).
"""
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


# ------------------------------------------------------------------ quadrature
@pytest.mark.parametrize("fam", [
    W.fourier_family([1.0], 64, 16, 16),
    W.fourier_family(W.STAR_PARAMS, 32, 16, 64, cx=0.2, cy=-0.1),
    W.fourier_family(list(W.random_star_params()), 40, 16, 24),
])
def test_nodes_match_oracle(fam):
    p = plan([fam], 0.1, 1.0, 1e-6, grid=W.grid_spec(64, 64, 0.05))
    x, y, w = (t.cpu().numpy() for t in p.nodes())
    ox, oy, ow = Q.family_nodes(fam)
    assert len(x) == len(ox)
    assert np.max(np.abs(x - ox)) < 5e-15 and np.max(np.abs(y - oy)) < 5e-15
    assert np.max(np.abs(w - ow)) < 1e-14 * np.max(np.abs(ow)) * 10
    p.close()


# ------------------------------------------------------------------ type 1 (grid)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_t1_disc_F10_full_grid(prec):
    """Unit disc, F = 10, 64 x 16 x 16 nodes, 100 x 100 grid over [-1.5, 1.5)^2."""
    cfg = W.disc()
    fam, g = cfg["families"], cfg["grid"]
    xi, eta = oracle.grid_targets(g["n1"], g["n2"], g["h"])
    ref = oracle.field(fam, cfg["lam"], cfg["z"], xi, eta).reshape(g["n2"], g["n1"])
    tol, bar = BARS[prec]
    u = plan(fam, cfg["lam"], cfg["z"], tol, precision=prec, grid=g).eval().cpu().numpy()
    assert u.shape == (g["n2"], g["n1"])
    assert rel_l2(u, ref) <= bar


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_t1_ragged_offset_grid(prec):
    """Odd, non-square grid (301 x 250) with an offset origin (pre-phase, Sec. 3.3)."""
    fam = [W.fourier_family(W.STAR_PARAMS, 32, 16, 48, cx=0.05, cy=0.02)]
    lz = 0.05
    g = W.grid_spec(301, 250, 0.011, x0=0.13, y0=-0.07)
    xi, eta = oracle.grid_targets(g["n1"], g["n2"], g["h"], g["x0"], g["y0"])
    ref = oracle.field(fam, lz, 1.0, xi, eta).reshape(g["n2"], g["n1"])
    tol, bar = BARS[prec]
    u = plan(fam, lz, 1.0, tol, precision=prec, grid=g).eval().cpu().numpy()
    assert rel_l2(u, ref) <= bar


def test_t1_folding_coarse_grid():
    """A grid coarser than the field (n < F): x~ must be folded mod 2 pi (Sec. 3.3)."""
    fam = [W.fourier_family([1.0], 64, 16, 48)]
    lz = 0.02   # F = 50
    g = W.grid_spec(16, 16, 0.2)
    xi, eta = oracle.grid_targets(16, 16, 0.2)
    ref = oracle.field(fam, lz, 1.0, xi, eta).reshape(16, 16)
    u = plan(fam, lz, 1.0, 1e-12, precision="fp64", grid=g).eval().cpu().numpy()
    assert rel_l2(u, ref) <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_t1_occulter_babinet(prec):
    cfg = W.disc()
    fam, g = cfg["families"], cfg["grid"]
    tol, _ = BARS[prec]
    ua = plan(fam, cfg["lam"], 1.0, tol, precision=prec, grid=g).eval().cpu().numpy()
    uo = plan(fam, cfg["lam"], 1.0, tol, precision=prec, grid=g,
              output="occulter").eval().cpu().numpy()
    np.testing.assert_allclose(uo, 1.0 - ua, atol=1e-12 if prec == "fp64" else 1e-6)


def test_t1_disc_closed_form_on_axis():
    """Disc at F = 10 with converged m = 64: the grid point (0, 0) equals 1 - e^{i 10 pi} = 0."""
    fam = [W.fourier_family([1.0], 64, 16, 64)]
    u = plan(fam, 0.1, 1.0, 1e-12, precision="fp64",
             grid=W.grid_spec(100, 100, 0.03)).eval().cpu().numpy()
    assert abs(u[50, 50] - oracle.closed_forms.disc_on_axis(1.0, 0.1)) < 1e-10


def test_multiple_families_add():
    f1 = W.fourier_family([0.5], 32, 16, 24, cx=-0.6)
    f2 = W.fourier_family([0.4, 0.0, 0.0, 0.05, 0.0], 32, 16, 24, cx=0.6, cy=0.2)
    g = W.grid_spec(96, 80, 0.03)
    xi, eta = oracle.grid_targets(96, 80, 0.03)
    ref = oracle.field([f1, f2], 0.05, 1.0, xi, eta).reshape(80, 96)
    u = plan([f1, f2], 0.05, 1.0, 1e-12, precision="fp64", grid=g).eval().cpu().numpy()
    assert rel_l2(u, ref) <= 1e-10


def test_explicit_nodes_and_line_rule_families():
    """NODES (negative weights allowed, Sec. 4.1) and LINE_RULE (kite via eq. ptr)."""
    X, Y, Wt, V = Q.ptr_line_rule(
        lambda s: (0.5 * np.cos(s) + 0.5 * np.cos(2 * s), np.sin(s)),
        lambda s: (-0.5 * np.sin(s) - np.sin(2 * s), np.cos(s)), 160)
    kite = {"kind": "line_rule", "X": X, "Y": Y, "W": Wt, "V": V, "m": 40}
    g = W.rng(7, 0)
    nodes = {"kind": "nodes", "x": g.uniform(-1, 1, 500), "y": g.uniform(-1, 1, 500),
             "w": g.normal(0, 1e-3, 500)}
    grid = W.grid_spec(64, 64, 0.045)
    xi, eta = oracle.grid_targets(64, 64, 0.045)
    for fams in ([kite], [nodes], [kite, nodes]):
        ref = oracle.field(fams, 0.1, 1.0, xi, eta).reshape(64, 64)
        u = plan(fams, 0.1, 1.0, 1e-12, precision="fp64", grid=grid).eval().cpu().numpy()
        assert rel_l2(u, ref) <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_eval_host_matches_device(prec):
    """Host-buffer entry point = device entry point (up to the order of the
    shared-memory atomic additions, which varies between runs)."""
    cfg = W.disc()
    tol, _ = BARS[prec]
    p = plan(cfg["families"], 0.1, 1.0, tol, precision=prec, grid=cfg["grid"])
    ud = p.eval().cpu().numpy()
    uh = p.eval_host()
    assert rel_l2(uh, ud) <= (1e-13 if prec == "fp64" else 2e-6)
    p3 = plan(cfg["families"], 0.1, 1.0, tol, precision=prec, box=(-1.5, 1.5, -1.5, 1.5))
    xi, eta = W.disc_targets(777, 1.5, 1)
    h = np.ascontiguousarray(np.stack([xi, eta], 1))
    u3d = p3.eval(torch.tensor(h, device="cuda")).cpu().numpy()
    u3h = p3.eval_host(h)
    assert rel_l2(u3h, u3d) <= (1e-13 if prec == "fp64" else 2e-6)


# ------------------------------------------------------------------ type 3 (scattered)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_t3_star_scattered(prec):
    fam = [W.fourier_family(W.STAR_PARAMS, 32, 16, 48, cx=0.03, cy=-0.02)]
    lz = 0.05
    xi, eta = W.disc_targets(3001, 1.5, 2)
    ref = oracle.field(fam, lz, 1.0, xi, eta)
    tol, bar = BARS[prec]
    p = plan(fam, lz, 1.0, tol, precision=prec, box=(-1.5, 1.5, -1.5, 1.5))
    t = torch.tensor(np.stack([xi, eta], 1), dtype=torch.float64, device="cuda")
    u = p.eval(t).cpu().numpy()
    assert rel_l2(u, ref) <= bar


def test_t3_offset_box_and_occulter():
    fam = [W.fourier_family([1.0, 0.1, 0.0], 32, 16, 40)]
    lz = 0.08
    g = W.rng(8, 0)
    xi, eta = g.uniform(0.2, 1.4, 1500), g.uniform(-1.1, -0.3, 1500)
    ref = 1.0 - oracle.field(fam, lz, 1.0, xi, eta)
    p = plan(fam, lz, 1.0, 1e-12, precision="fp64", output="occulter", box=(0.2, 1.4, -1.1, -0.3))
    t = torch.tensor(np.stack([xi, eta], 1), dtype=torch.float64, device="cuda")
    assert rel_l2(p.eval(t).cpu().numpy(), ref) <= 1e-10


@pytest.mark.parametrize("M", [40000, 777])
def test_t3_binned_path_matches_oracle_and_direct_path(M):
    """FP32 type-3 with target binning forced on (interpolation from
    shared-memory patches) and off (direct gathers): both must match the
    oracle and each other."""
    fam = [W.fourier_family(W.STAR_PARAMS, 48, 16, 64, cx=0.02)]
    lz = 0.03
    xi, eta = W.disc_targets(M, 1.5, 9)
    xi[:5], eta[:5] = 0.0, 0.0               # duplicates at the box centre
    xi[5], eta[5] = 1.5, 0.0                 # on the box edge
    t = torch.tensor(np.stack([xi, eta], 1), dtype=torch.float64, device="cuda")
    box = (-1.5, 1.5, -1.5, 1.5)
    u_binned = plan(fam, lz, 1.0, 1e-6, box=box, t3_binning=1).eval(t).cpu().numpy()
    u_direct = plan(fam, lz, 1.0, 1e-6, box=box, t3_binning=-1).eval(t).cpu().numpy()
    assert rel_l2(u_binned, u_direct) <= 1e-6
    idx = W.rng(9, 3).choice(len(xi), min(600, M), replace=False)
    idx[:6] = np.arange(6)
    ref = oracle.field(fam, lz, 1.0, xi[idx], eta[idx])
    assert rel_l2(u_binned[idx], ref) <= 1e-6


def test_t3_binned_path_flags_outside_targets():
    from paper_2010_05978_gb300 import FresnelError
    fam = [W.fourier_family([1.0], 16, 16, 16)]
    p = plan(fam, 0.1, 1.0, 1e-6, box=(-1, 1, -1, 1), t3_binning=1)
    xi, eta = W.square_targets(40000, 0.9, 5)
    xi[123] = 1.7
    t = torch.tensor(np.stack([xi, eta], 1), dtype=torch.float64, device="cuda")
    with pytest.raises(FresnelError) as e:
        p.eval(t)
    assert e.value.status == -6


def test_t3_empty_and_single_target():
    fam = [W.fourier_family([1.0], 16, 16, 16)]
    p = plan(fam, 0.1, 1.0, 1e-12, precision="fp64", box=(-1, 1, -1, 1))
    t0 = torch.empty((0, 2), dtype=torch.float64, device="cuda")
    assert p.eval(t0).shape == (0,)
    t1 = torch.tensor([[0.0, 0.0]], dtype=torch.float64, device="cuda")
    u = p.eval(t1).cpu().numpy()
    assert abs(u[0] - oracle.field(fam, 0.1, 1.0, [0.0], [0.0])[0]) < 1e-10


def test_t3_target_outside_box_is_reported():
    from paper_2010_05978_gb300 import FresnelError
    fam = [W.fourier_family([1.0], 16, 16, 16)]
    p = plan(fam, 0.1, 1.0, 1e-6, box=(-1, 1, -1, 1))
    t = torch.tensor([[0.0, 0.0], [1.5, 0.0]], dtype=torch.float64, device="cuda")
    with pytest.raises(FresnelError) as e:
        p.eval(t)
    assert e.value.status == -6
    # the plan stays usable after the error
    ok = torch.tensor([[0.5, 0.5]], dtype=torch.float64, device="cuda")
    p.eval(ok)


# ------------------------------------------------------------------ full-size workload
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_star_F100_t1_full_size_sampled(prec):
    """Star r = 1 + 0.3 cos 5t at F = 100, 524,288 nodes, 1000 x 1000 grid: sampled targets."""
    cfg = W.star()
    fam, g = cfg["families"], cfg["grid"]
    tol, bar = BARS[prec]
    u = plan(fam, cfg["lam"], 1.0, tol, precision=prec, grid=g,
             recompute_nodes=True).eval().cpu().numpy().ravel()
    xi, eta = oracle.grid_targets(g["n1"], g["n2"], g["h"])
    idx = W.rng(2, 7).choice(len(xi), 400, replace=False)
    ref = oracle.field(fam, cfg["lam"], 1.0, xi[idx], eta[idx])
    assert rel_l2(u[idx], ref) <= bar


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_star_F100_t3_full_size_sampled(prec):
    """Star at F = 100, 524,288 nodes, type 3 to 1e6 targets in the disc of
    radius 1.5 (the benchmark's launch configuration), in both precisions:
    fast mode at tol 1e-6 and FP64 at tol 1e-12 (bar 1e-10)."""
    cfg = W.star()
    fam = cfg["families"]
    tol, bar = BARS[prec]
    xi, eta = W.disc_targets(1000000, 1.5, 2)
    p = plan(fam, cfg["lam"], 1.0, tol, precision=prec, box=(-1.5, 1.5, -1.5, 1.5),
             recompute_nodes=True)
    t = torch.tensor(np.stack([xi, eta], 1), dtype=torch.float64, device="cuda")
    u = p.eval(t).cpu().numpy()
    idx = W.rng(2, 8).choice(len(xi), 400, replace=False)
    ref = oracle.field(fam, cfg["lam"], 1.0, xi[idx], eta[idx])
    assert rel_l2(u[idx], ref) <= bar


# ------------------------------------------------------------------ autotuned plans
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_autotuned_plans_match_oracle(prec):
    """autotune = 1 times candidate configurations on the device (sigma 5/4 or
    2 in FP64; binned or direct interpolation for FP32 type 3) and keeps the
    faster; the result must meet the same bar."""
    tol, bar = BARS[prec]
    cfg = W.disc()
    fam, g = cfg["families"], cfg["grid"]
    xi, eta = oracle.grid_targets(g["n1"], g["n2"], g["h"])
    p = plan(fam, cfg["lam"], cfg["z"], tol, precision=prec, grid=g, autotune=True)
    assert p.info()["sigma"] in (1.25, 2.0)
    ref = oracle.field(fam, cfg["lam"], cfg["z"], xi, eta).reshape(g["n2"], g["n1"])
    assert rel_l2(p.eval().cpu().numpy(), ref) <= bar
    fam3 = [W.fourier_family(W.STAR_PARAMS, 32, 16, 48)]
    x3, y3 = W.disc_targets(40000, 1.5, 12)
    t = torch.tensor(np.stack([x3, y3], 1), dtype=torch.float64, device="cuda")
    p3 = plan(fam3, 0.03, 1.0, tol, precision=prec, box=(-1.5, 1.5, -1.5, 1.5), autotune=True)
    # FP32: the autotuner fixed the interpolation mode, which info() reports
    assert p3.info()["t3_binning"] in ((1, -1) if prec == "fp32" else (0,))
    u3 = p3.eval(t).cpu().numpy()
    idx = np.arange(0, 40000, 97)
    assert rel_l2(u3[idx], oracle.field(fam3, 0.03, 1.0, x3[idx], y3[idx])) <= bar


# ------------------------------------------------------------------ line integral on the device
def test_nsli_matches_oracle_line_integral():
    """GPU eq. nsli against the oracle's, on the same boundary rule, including a
    target exactly on a boundary node (r = 0) and targets near the boundary."""
    fam = W.fourier_family(W.STAR_PARAMS, 32, 16, 8, cx=0.1, cy=-0.05)
    X, Y, Wt, V, _, _ = Q.family_line_rule(fam)
    xi, eta = W.disc_targets(2000, 1.6, 13)
    xi[0], eta[0] = X[17], Y[17]
    xi[1], eta[1] = 1.0001 * X[40], 1.0001 * Y[40]
    lz = 0.04
    from oracle import direct
    ref = direct.nsli(X, Y, Wt, V, xi, eta, lz)
    p = plan([fam], lz, 1.0, 1e-12, precision="fp64", box=(-1.6, 1.6, -1.6, 1.6))
    t = torch.tensor(np.stack([xi, eta], 1), dtype=torch.float64, device="cuda")
    u = p.nsli(t).cpu().numpy()
    assert np.max(np.abs(u - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("output", ["aperture", "occulter"])
def test_nsli_far_matches_oracle(output):
    """The far-target option (eq. li with the rounded winding number, the
    Appendix's remark on shadows) against the oracle's line_integral_far on
    a coarse rule (inexact winding numbers), near and far targets, inside
    and outside."""
    fam = W.fourier_family(W.STAR_PARAMS, 12, 4, 8, cx=0.1, cy=-0.05)
    X, Y, Wt, V, _, _ = Q.family_line_rule(fam)
    xi, eta = W.disc_targets(3000, 1.6, 15)
    lz, far = 0.04, 0.15
    from oracle import direct
    uap, uoc = direct.line_integral_far(X, Y, Wt, V, xi, eta, lz, far)
    ref = uoc if output == "occulter" else uap
    p = plan([fam], lz, 1.0, 1e-12, precision="fp64", box=(-1.6, 1.6, -1.6, 1.6),
             output=output, nsli_far=far)
    t = torch.tensor(np.stack([xi, eta], 1), dtype=torch.float64, device="cuda")
    u = p.nsli(t).cpu().numpy()
    assert np.max(np.abs(u - ref)) <= 1e-12
    # both kinds of target are present (the oracle copies eq. nsli's value
    # for near ones), and the option changed the far ones
    un = direct.nsli(X, Y, Wt, V, xi, eta, lz)
    un = 1.0 - un if output == "occulter" else un
    near = ref == un
    assert np.count_nonzero(near) > 10 and np.count_nonzero(~near) > 100
    assert np.min(np.abs(u - un)[~near]) > 1e-9 or np.median(np.abs(u - un)[~near]) > 1e-6


def test_nsli_agrees_with_areal_path():
    """Converged disc (F = 10, m = 64): the areal NUFFT path and the device line
    integral agree, and both match the Hankel closed form."""
    fam = [W.fourier_family([1.0], 64, 16, 64)]
    rho = np.linspace(0.0, 1.45, 40)
    xi, eta = rho * np.cos(0.7), rho * np.sin(0.7)
    t = torch.tensor(np.stack([xi, eta], 1), dtype=torch.float64, device="cuda")
    p = plan(fam, 0.1, 1.0, 1e-12, precision="fp64", box=(-1.5, 1.5, -1.5, 1.5))
    ua = p.eval(t).cpu().numpy()
    un = p.nsli(t).cpu().numpy()
    ref = oracle.closed_forms.disc_off_axis(1.0, 0.1, rho)
    assert np.max(np.abs(ua - un)) < 1e-9
    assert np.max(np.abs(un - ref)) < 1e-9


@pytest.mark.parametrize("tol,w", [(1e-7, 9), (1e-3, 5)])
def test_t3_fp32_kernel_widths(tol, w):
    """FP32 type 3 at the widths the tolerance picks (w = 9 gathers with 16
    lanes per target, w = 5 leaves lanes idle) against the oracle."""
    fam = [W.fourier_family(W.STAR_PARAMS, 32, 16, 48)]
    xi, eta = W.disc_targets(5000, 1.5, 14)
    t = torch.tensor(np.stack([xi, eta], 1), dtype=torch.float64, device="cuda")
    p = plan(fam, 0.04, 1.0, tol, precision="fp32", box=(-1.5, 1.5, -1.5, 1.5))
    assert p.info()["w"] == w
    u = p.eval(t).cpu().numpy()
    ref = oracle.field(fam, 0.04, 1.0, xi, eta)
    assert rel_l2(u, ref) <= max(tol, 1e-6)


@pytest.mark.parametrize("binning", [0, 1])
def test_eval_host_async_pinned_back_to_back(binning):
    """Host-buffer evaluations with sync_status off return once queued: two
    calls with different pinned target sets, then one check (stream
    synchronisation).  The second call's target copy must not overwrite the
    staged targets while the first evaluation still reads them.  With the
    binned interpolation (binning 1) the target sort runs on its own stream:
    it must wait for its evaluation's target copy, and the second sort must
    not overwrite the permutation the first interpolation still reads."""
    fam = [W.fourier_family(W.STAR_PARAMS, 32, 16, 48)]
    p = plan(fam, 0.05, 1.0, 1e-6, precision="fp32", box=(-1.5, 1.5, -1.5, 1.5),
             sync_status=False, t3_binning=binning)
    xa, ya = W.disc_targets(60000, 1.5, 21)
    xb, yb = W.disc_targets(60000, 1.5, 22)
    ha = torch.tensor(np.stack([xa, ya], 1), dtype=torch.float64).pin_memory()
    hb = torch.tensor(np.stack([xb, yb], 1), dtype=torch.float64).pin_memory()
    oa = torch.empty(60000, dtype=torch.complex64).pin_memory()
    ob = torch.empty(60000, dtype=torch.complex64).pin_memory()
    p.eval_host(ha.numpy(), oa.numpy())
    p.eval_host(hb.numpy(), ob.numpy())
    p.check()
    ua = p.eval(ha.cuda()).cpu().numpy()
    ub = p.eval(hb.cuda()).cpu().numpy()
    assert rel_l2(oa.numpy(), ua) <= 2e-6 and rel_l2(ob.numpy(), ub) <= 2e-6
    sel = np.arange(0, 60000, 997)
    ref = oracle.field(fam, 0.05, 1.0, xb[sel], yb[sel])
    assert rel_l2(ob.numpy()[sel], ref) <= 1e-6
