"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Every check here is CPU-only.  The planted-mistake tests at the end put a
plausible bug into a copy of the oracle (on the CPU) and confirm that at least
one pin catches it.
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import closed_forms as CF
from oracle import direct as D
from oracle import quadrature as Q

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ quadrature
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 16, 33])
def test_gauss_legendre_polynomial_exactness(n):
    """An n-point Gauss rule integrates x^k exactly on (0,1) for k <= 2n-1."""
    x, w = Q.gauss_legendre(n, 0.0, 1.0)
    for k in range(2 * n):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-14
    if n <= 5:  # and is not exact one degree higher (so it is the n-point rule)
        assert abs(np.sum(w * x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-8


@pytest.mark.parametrize("n", [256, 1024])
def test_gauss_legendre_large(n):
    x, w = Q.gauss_legendre(n, 0.0, 1.0)
    assert np.all(np.diff(x) > 0) and x[0] > 0 and x[-1] < 1
    assert abs(w.sum() - 1.0) < 1e-14
    # smooth integrand: int_0^1 cos(50 x) dx = sin(50)/50
    assert abs(np.sum(w * np.cos(50 * x)) - np.sin(50.0) / 50.0) < 1e-14


SHAPES = {
    "disc": [1.0],
    "star5": W.STAR_PARAMS,
    "random20": list(W.random_star_params()),
}


@pytest.mark.parametrize("name", sorted(SHAPES))
def test_line_rule_area_by_green(name):
    """(1/2) sum_i (X_i V_i - Y_i W_i) = area (Green's theorem on eq. vliq)."""
    params = SHAPES[name]
    X, Y, Wt, V = Q.fourier_line_rule(params, 64, 16)
    assert abs(0.5 * np.sum(X * V - Y * Wt) - CF.fourier_star_area(params)) < 1e-13


@pytest.mark.parametrize("name", sorted(SHAPES))
def test_areal_rule_area_and_moments(name):
    """Dilation rule (eqs. aqnod, aqwei): exact area, zero-free moments."""
    params = SHAPES[name]
    fam = W.fourier_family(params, 64, 16, 24)
    x, y, w = Q.family_nodes(fam)
    assert len(x) == 64 * 16 * 24
    area = CF.fourier_star_area(params)
    assert abs(w.sum() - area) < 1e-13
    assert abs(np.sum(w * (x * x + y * y)) - CF.fourier_star_second_moment(params)) < 1e-13
    if name in ("disc", "star5"):  # symmetric about the x axis and (disc) both axes
        assert abs(np.sum(w * y)) < 1e-14


def test_areal_rule_translated_centre():
    fam = W.fourier_family(W.STAR_PARAMS, 32, 16, 16, cx=0.7, cy=-0.4)
    x, y, w = Q.family_nodes(fam)
    area = CF.fourier_star_area(W.STAR_PARAMS)
    assert abs(w.sum() - area) < 1e-13
    assert abs(np.sum(w * x) - 0.7 * area) < 1e-13
    assert abs(np.sum(w * y) + 0.4 * area) < 1e-13


def test_kite_printed_radius_and_fresnel_number():
    """Sec. 4.1 prints R ~ 1.13 for the kite and F ~ 12.8 at lambda z = 0.1."""
    g = json.load(open(os.path.join(GOLDEN, "paper_printed.json")))["kite"]
    t = np.linspace(0, 2 * np.pi, 200001)
    R = np.max(np.hypot(0.5 * np.cos(t) + 0.5 * np.cos(2 * t), np.sin(t)))
    assert round(R, 2) == g["R_max_approx"]
    assert round(R * R / 0.1, 1) == g["fresnel_number_lz_0p1"]
    assert round(R * R / 0.01, 0) == g["fresnel_number_lz_0p01"]
    # kite area (Green): pi/2
    X, Y, Wt, V = Q.ptr_line_rule(
        lambda s: (0.5 * np.cos(s) + 0.5 * np.cos(2 * s), np.sin(s)),
        lambda s: (-0.5 * np.sin(s) - np.sin(2 * s), np.cos(s)), 200)
    x, y, w = Q.dilation_rule(X, Y, Wt, V, 8)
    assert abs(w.sum() - np.pi / 2) < 1e-13


# ------------------------------------------------------------------ field: closed forms
def test_disc_on_axis_dauger():
    """Appendix eq. dauger, R(theta) = R: u^ap(0) = 1 - e^{i pi R^2 / lz}."""
    for lz, m in ((0.1, 64), (0.25, 32), (1.0 / 30.0, 128)):
        fam = W.fourier_family([1.0], 64, 16, m)
        u = oracle.field([fam], lz, 1.0, [0.0], [0.0])[0]
        assert abs(u - CF.disc_on_axis(1.0, lz)) < 1e-12


def test_disc_off_axis_golden():
    """Direct sum vs the stored Hankel closed form of the disc at F = 10."""
    g = json.load(open(os.path.join(GOLDEN, "disc_F10_hankel.json")))
    rho = np.asarray(g["rho"])
    ref = np.asarray(g["u_re"]) + 1j * np.asarray(g["u_im"])
    fam = W.fourier_family([g["R"]], 64, 16, 64)
    u = oracle.field([fam], g["lambda_z"], 1.0, rho, 0.0 * rho)
    assert np.max(np.abs(u - ref)) < 1e-10
    # the same closed form along another direction (rotational symmetry)
    u2 = oracle.field([fam], g["lambda_z"], 1.0, rho * np.cos(1.0), rho * np.sin(1.0))
    assert np.max(np.abs(u2 - ref)) < 1e-10
    # the stored Hankel values carry ~1e-11 rounding (2 pi / lz times a 6000-term sum)
    assert abs(ref[0] - complex(*g["u_axis_dauger"])) < 5e-11


def test_nsli_matches_areal_direct_sum():
    """Appendix eq. nsli (a line integral) vs eq. faq (an areal sum): independent formulas."""
    fam = W.fourier_family(W.STAR_PARAMS, 128, 16, 96)
    X, Y, Wt, V, cx, cy = Q.family_line_rule(fam)
    g = W.rng(99, 3)
    xi = np.concatenate([[0.0, -1.5, 1.3, 0.0], g.uniform(-1.5, 1.5, 60)])
    eta = np.concatenate([[0.0, -1.5, 0.0, 1.0], g.uniform(-1.5, 1.5, 60)])
    un = D.nsli(X, Y, Wt, V, xi, eta, 0.1)
    ud = oracle.field([fam], 0.1, 1.0, xi, eta)
    assert np.max(np.abs(un - ud)) < 1e-11


def test_nsli_target_on_boundary_node():
    """NSLI with a target exactly on a boundary node (r^2 = 0 branch) stays finite and accurate."""
    fam = W.fourier_family([1.0], 64, 16, 64)
    X, Y, Wt, V, _, _ = Q.family_line_rule(fam)
    xi, eta = np.array([X[5]]), np.array([Y[5]])
    un = D.nsli(X, Y, Wt, V, xi, eta, 0.1)
    ref = CF.disc_off_axis(1.0, 0.1, [np.hypot(X[5], Y[5])])
    assert np.isfinite(un).all() and abs(un[0] - ref[0]) < 1e-10


@pytest.mark.parametrize("target", [(0.3, -0.2), (1.4, 0.9)])
def test_brute_force_adaptive_tiny(target):
    """Eq. fres by adaptive 2D quadrature on a tiny case (F ~ 1) vs the areal sum."""
    params = [1.0, 0.0, 0.0, 0.1, 0.05]
    fam = W.fourier_family(params, 32, 16, 32)
    bf = CF.brute_force_star(params, 1.0, *target)
    u = oracle.field([fam], 1.0, 1.0, [target[0]], [target[1]])[0]
    assert abs(bf - u) < 1e-11


# ------------------------------------------------------------------ field: invariants
def _star_field(params, lz, xi, eta, cx=0.0, cy=0.0, n_panels=96, m=64):
    fam = W.fourier_family(params, n_panels, 16, m, cx, cy)
    return oracle.field([fam], lz, 1.0, np.asarray(xi), np.asarray(eta))


def test_translation_invariance():
    """u_{Omega+d}(xi) = u_Omega(xi - d) (eq. fres depends on xi - x only)."""
    g = W.rng(98, 0)
    xi, eta = g.uniform(-1.5, 1.5, 20), g.uniform(-1.5, 1.5, 20)
    d = (0.31, -0.17)
    a = _star_field(W.STAR_PARAMS, 0.1, xi + d[0], eta + d[1], *d)
    b = _star_field(W.STAR_PARAMS, 0.1, xi, eta)
    assert np.max(np.abs(a - b)) < 1e-12


def test_scaling_invariance():
    """u_{s Omega}(s xi; s^2 lz) = u_Omega(xi; lz)."""
    s = 1.7
    params = np.asarray(W.STAR_PARAMS)
    g = W.rng(97, 0)
    xi, eta = g.uniform(-1.5, 1.5, 20), g.uniform(-1.5, 1.5, 20)
    a = _star_field(s * params, s * s * 0.1, s * xi, s * eta)
    b = _star_field(params, 0.1, xi, eta)
    assert np.max(np.abs(a - b)) < 1e-12


def test_reflection_symmetry():
    """A shape symmetric under y -> -y gives u(xi, -eta) = u(xi, eta); a rotated copy does not."""
    g = W.rng(96, 0)
    xi, eta = g.uniform(-1.5, 1.5, 16), g.uniform(-1.5, 1.5, 16)
    a = _star_field(W.STAR_PARAMS, 0.1, xi, eta)
    b = _star_field(W.STAR_PARAMS, 0.1, xi, -eta)
    assert np.max(np.abs(a - b)) < 1e-12
    p = list(W.STAR_PARAMS)
    p[9], p[10] = 0.3 * np.cos(0.5), 0.3 * np.sin(0.5)  # rotated star: no longer symmetric
    c = _star_field(p, 0.1, xi, eta)
    d = _star_field(p, 0.1, xi, -eta)
    assert np.max(np.abs(c - d)) > 1e-3


def test_five_fold_rotation_symmetry():
    th = 2 * np.pi / 5
    g = W.rng(95, 0)
    xi, eta = g.uniform(-1.5, 1.5, 16), g.uniform(-1.5, 1.5, 16)
    a = _star_field(W.STAR_PARAMS, 0.1, xi, eta)
    b = _star_field(W.STAR_PARAMS, 0.1, np.cos(th) * xi - np.sin(th) * eta,
                    np.sin(th) * xi + np.cos(th) * eta)
    assert np.max(np.abs(a - b)) < 1e-12


def test_babinet_output_option():
    """Eq. bab: the occulter field is 1 - the aperture field."""
    fam = W.fourier_family(W.STAR_PARAMS, 32, 16, 16)
    xi, eta = np.array([0.0, 0.4, 2.0]), np.array([0.0, -0.3, 1.0])
    ua = oracle.field([fam], 0.1, 1.0, xi, eta, output="aperture")
    uo = oracle.field([fam], 0.1, 1.0, xi, eta, output="occulter")
    assert np.max(np.abs(ua + uo - 1.0)) == 0.0


def test_split_identity_pins_sum3():
    """Eq. split: direct sum = (1/(i lz)) chirp(xi) * sum3(c), c_j = w_j chirp(x_j)."""
    fam = W.fourier_family(W.STAR_PARAMS, 32, 16, 24)
    x, y, w = Q.family_nodes(fam)
    lz = 0.05
    g = W.rng(94, 0)
    xi, eta = g.uniform(-1.5, 1.5, 50), g.uniform(-1.5, 1.5, 50)
    c = w * np.exp(1j * np.pi * (x * x + y * y) / lz)
    v = D.sum3(x, y, c, xi, eta, lz)
    u = np.exp(1j * np.pi * (xi * xi + eta * eta) / lz) * v / (1j * lz)
    ud = D.direct_sum(x, y, w, xi, eta, lz)
    assert np.max(np.abs(u - ud)) < 1e-11


# ------------------------------------------------------------------ starshade rule (Sec. 4.2)
HG = lambda a, b, q: (lambda r: np.exp(-((r - a) / b) ** q))
SMALL_FLOWER = dict(n_petals=5, a=0.4, R=1.0, profile={"kind": "hg", "b": 0.35, "q": 4})


def _small_flower(m=40, n_p=30, n_d=60, m_d=40, **kw):
    d = dict(SMALL_FLOWER)
    d.update(kw)
    return W.petal_family(d["n_petals"], d["a"], d["R"], d["profile"], m, n_p, n_d, m_d,
                          d.get("cx", 0.0), d.get("cy", 0.0))


def test_starshade_printed_node_count():
    """Table t:star: HG with 16 petals, m = 60, n_p = 30 has N = 37440 nodes."""
    with open(os.path.join(GOLDEN, "paper_printed.json")) as fh:
        g = json.load(fh)["starshade_node_counts"]["HG"]
    n_d = int(round(0.3 * g["N_p"] * g["n_p"]))
    fam = W.petal_family(g["N_p"], 12.5, 31.0, {"kind": "hg", "b": 12.5, "q": 6}, g["m"],
                         g["n_p"], n_d, g["m"])
    x, y, w = Q.family_nodes(fam)
    assert len(x) == len(y) == len(w) == g["N"]


@pytest.mark.parametrize("shape", ["paper_hg", "hg24", "small"])
def test_starshade_area_and_moments(shape):
    """Sum w = pi a^2 + 2 pi int A r dr; sum w |x|^2 likewise; first moments 0."""
    if shape == "paper_hg":
        a, R, b, q, Np, m, n_p = 12.5, 31.0, 12.5, 6, 16, 60, 30
    elif shape == "hg24":
        a, R, b, q, Np, m, n_p = 6.0, 14.0, 3.9, 6, 24, 40, 20
    else:
        a, R, b, q, Np, m, n_p = 0.4, 1.0, 0.35, 4, 5, 40, 30
    fam = W.petal_family(Np, a, R, {"kind": "hg", "b": b, "q": q}, m, n_p,
                         int(np.ceil(0.3 * Np * n_p)), m)
    x, y, w = Q.family_nodes(fam)
    area, mom = CF.flower_area_moments(a, R, HG(a, b, q))
    assert abs(w.sum() - area) < 1e-13 * area
    assert abs(np.sum(w * (x * x + y * y)) - mom) < 1e-13 * mom
    assert abs(np.sum(w * x)) < 1e-13 * area * R and abs(np.sum(w * y)) < 1e-13 * area * R


def test_bspline_profile_partition_of_unity_and_linear_precision():
    """Clamped cubic B-splines sum to 1 and reproduce r from its Greville abscissae."""
    a, R, n = 6.0, 14.0, 20
    r = np.linspace(a, R, 301)
    one = Q.petal_profile({"kind": "bspline", "coefs": np.ones(n)}, a, R, r)
    assert np.max(np.abs(one - 1.0)) < 1e-14
    t = Q.bspline_knots(a, R, n)
    greville = (t[1:n + 1] + t[2:n + 2] + t[3:n + 3]) / 3.0
    lin = Q.petal_profile({"kind": "bspline", "coefs": greville}, a, R, r)
    assert np.max(np.abs(lin - r)) < 1e-13 * R
    assert t[0] == t[3] == a and t[-1] == t[-4] == R and len(t) == n + 4
    assert np.allclose(np.diff(t[3:n + 1]), (R - a) / (n - 3))


def test_starshade_full_width_petals_make_a_disc():
    """A = 1 on [a, R]: the petals tile the annulus and the flower is the disc of radius R."""
    lz = 0.1
    fam = _small_flower(m=48, n_p=60, n_d=80, m_d=48,
                        profile={"kind": "bspline", "coefs": np.ones(12)})
    rho = np.array([0.0, 0.37, 0.8, 1.3])
    th = np.array([0.3, 1.1, 2.0, -0.7])
    u = oracle.field([fam], lz, 1.0, rho * np.cos(th), rho * np.sin(th))
    ref = CF.disc_off_axis(1.0, lz, rho)
    assert np.max(np.abs(u - ref)) < 1e-11


def test_starshade_on_axis_closed_form():
    lz = 0.05
    fam = _small_flower(m=64, n_p=20, n_d=80, m_d=64)
    u = oracle.field([fam], lz, 1.0, [0.0], [0.0])[0]
    ref = CF.flower_on_axis(0.4, 1.0, HG(0.4, 0.35, 4), lz)
    assert abs(u - ref) < 1e-11


@pytest.mark.parametrize("target", [(0.3, 0.1), (0.9, -0.4), (1.3, 0.6)])
def test_starshade_brute_force_off_axis(target):
    """Areal rule vs adaptive 2D integration over the region of eq. Omega."""
    lz = 0.5
    u = oracle.field([_small_flower()], lz, 1.0, [target[0]], [target[1]])[0]
    ref = CF.brute_force_flower(5, 0.4, 1.0, HG(0.4, 0.35, 4), lz, *target)
    assert abs(u - ref) < 1e-10


def test_starshade_rotation_and_translation():
    lz = 0.07
    fam = _small_flower()
    xi, eta = np.array([0.21, 0.83, -0.5]), np.array([0.05, -0.32, 0.61])
    rot = 2.0 * np.pi / 5
    u = oracle.field([fam], lz, 1.0, xi, eta)
    ur = oracle.field([fam], lz, 1.0, np.cos(rot) * xi - np.sin(rot) * eta,
                      np.sin(rot) * xi + np.cos(rot) * eta)
    assert np.max(np.abs(u - ur)) < 1e-12
    ut = oracle.field([_small_flower(cx=0.3, cy=-0.2)], lz, 1.0, xi + 0.3, eta - 0.2)
    assert np.max(np.abs(u - ut)) < 1e-12


def test_planted_starshade_printed_weight_index(monkeypatch):
    """The literal printed weight r_l what_l A(r_i) omegahat_i (A at the wrong
    radius) is caught by the area pin."""
    orig = Q.petal_profile

    def bad(profile, a, R, r):
        A = orig(profile, a, R, r)
        return A[np.arange(len(A)) % 7]          # A taken at another radius index
    fam = _small_flower()
    area, _ = CF.flower_area_moments(0.4, 1.0, HG(0.4, 0.35, 4))
    with monkeypatch.context() as mp:
        mp.setattr(Q, "petal_profile", bad)
        _, _, w = Q.family_nodes(fam)
    assert abs(w.sum() - area) > 1e-6


def test_planted_petals_off_centre(monkeypatch):
    """Petals centred half a period off (on pi (2k+1)/Np) fail the brute-force pin."""
    fam = _small_flower()
    x, y, w = Q.family_nodes(fam)
    n_disc = 60 * 40
    th = np.pi / 5
    xb, yb = x.copy(), y.copy()
    xb[n_disc:] = np.cos(th) * x[n_disc:] - np.sin(th) * y[n_disc:]
    yb[n_disc:] = np.sin(th) * x[n_disc:] + np.cos(th) * y[n_disc:]
    lz, target = 0.5, (0.9, -0.4)
    u = D.direct_sum(xb, yb, w, np.array([target[0]]), np.array([target[1]]), lz)[0]
    ref = CF.brute_force_flower(5, 0.4, 1.0, HG(0.4, 0.35, 4), lz, *target)
    assert abs(u - ref) > 1e-4


# ------------------------------------------------------------------ spline-profile gradient
def _spline_case(kind):
    return W.spline_starshade("hg24_small" if kind == "hg24" else kind)


def test_spline_loss_gradient_matches_central_differences():
    """Adjoint gradient of the mean pupil intensity w.r.t. the B-spline
    coefficients against central differences (h = 1e-6) of the loss itself."""
    from oracle import gradient as G
    for kind in ("hg24", "small"):
        theta, probs, grid, keep = _spline_case(kind)
        _check_gradient(G, theta, probs, grid, keep)


def _check_gradient(G, theta, probs, grid, keep):
    L, g = G.loss_and_grad(theta, probs, grid, keep)
    assert abs(L - G.loss(theta, probs, grid, keep)) < 1e-14
    h = 1e-6
    for m in (0, 3, 10, 17, 19):
        e = np.zeros_like(theta)
        e[m] = h
        fd = (G.loss(theta + e, probs, grid, keep) - G.loss(theta - e, probs, grid, keep)) / (2 * h)
        assert abs(g[m] - fd) <= 1e-7 * max(abs(fd), 1e-3), (m, g[m], fd)


def test_planted_gradient_without_node_motion(monkeypatch):
    """Dropping the node-position term of the adjoint (weights only) fails the
    central-difference pin."""
    from oracle import gradient as G
    theta, probs, grid, keep = _spline_case("small")
    orig = G.direct.adjoint_sums

    def bad(x, y, xi, eta, lz, g):
        P, Qx, Qy = orig(x, y, xi, eta, lz, g)
        return P, 0 * Qx, 0 * Qy
    with monkeypatch.context() as mp:
        mp.setattr(G.direct, "adjoint_sums", bad)
        _, g = G.loss_and_grad(theta, probs, grid, keep)
    e = np.zeros_like(theta)
    e[10] = 1e-6
    fd = (G.loss(theta + e, probs, grid, keep) - G.loss(theta - e, probs, grid, keep)) / 2e-6
    assert abs(g[10] - fd) > 1e-3 * abs(fd)


def _shape_case():
    fam = W.fourier_family(W.STAR_PARAMS, 16, 8, 12, cx=0.05, cy=-0.03)
    params = np.array(fam["params"])
    params[3], params[4] = 0.02, -0.015
    xi, eta = W.disc_targets(60, 1.2, 31)
    return params, fam, xi, eta


def _shape_fd(G, params, fam, xi, eta, out, k, h=1e-6):
    e = np.zeros_like(params)
    e[k] = h
    return (G.shape_loss(params + e, fam, 0.05, 1.0, xi, eta, out) -
            G.shape_loss(params - e, fam, 0.05, 1.0, xi, eta, out)) / (2 * h)


@pytest.mark.parametrize("out", ["aperture", "occulter"])
def test_shape_gradient_matches_central_differences(out):
    """Adjoint gradient of the mean |u|^2 w.r.t. every Fourier coefficient of an
    off-centre star boundary against central differences (h = 1e-6) of the
    loss itself."""
    from oracle import gradient as G
    params, fam, xi, eta = _shape_case()
    L, g = G.shape_loss_and_grad(params, fam, 0.05, 1.0, xi, eta, out)
    assert abs(L - G.shape_loss(params, fam, 0.05, 1.0, xi, eta, out)) < 1e-13
    for k in range(len(params)):
        fd = _shape_fd(G, params, fam, xi, eta, out, k)
        assert abs(g[k] - fd) <= 1e-7 * np.max(np.abs(g)), (k, g[k], fd)


def test_planted_shape_gradient_with_swapped_modes(monkeypatch):
    """Taking the cosine mode's derivative for the sine coefficient (and back)
    fails the central-difference pin."""
    from oracle import gradient as G
    params, fam, xi, eta = _shape_case()
    orig = G.fourier_mode

    def bad(kk, t):
        return orig(kk + 1 if kk % 2 == 1 else (kk - 1 if kk > 0 else 0), t)
    with monkeypatch.context() as mp:
        mp.setattr(G, "fourier_mode", bad)
        _, g = G.shape_loss_and_grad(params, fam, 0.05, 1.0, xi, eta, "aperture")
    fd = np.array([_shape_fd(G, params, fam, xi, eta, "aperture", k) for k in range(len(params))])
    assert np.max(np.abs(g - fd)) > 1e-3 * np.max(np.abs(fd))


# ------------------------------------------------------------------ planted mistakes
def _pins_fail(monkeypatch, patch):
    """Apply a plausible oracle bug and report whether the closed-form pins notice it."""
    with monkeypatch.context() as mp:
        patch(mp)
        failures = 0
        fam = W.fourier_family([1.0], 64, 16, 64)
        x, y, w = Q.family_nodes(fam)
        failures += abs(w.sum() - np.pi) > 1e-12
        u = oracle.field([fam], 0.1, 1.0, [0.0, 0.6], [0.0, 0.3])
        ref = CF.disc_off_axis(1.0, 0.1, [0.0, np.hypot(0.6, 0.3)])
        failures += np.max(np.abs(u - ref)) > 1e-10
        fs = W.fourier_family(W.STAR_PARAMS, 64, 16, 48)
        us = oracle.field([fs], 0.1, 1.0, [0.4], [0.25])
        X, Y, Wt, V, _, _ = Q.family_line_rule(fs)
        un = D.nsli(X, Y, Wt, V, np.array([0.4]), np.array([0.25]), 0.1)
        failures += abs(us[0] - un[0]) > 1e-11
        return failures > 0


def test_planted_dropped_alpha_in_weights(monkeypatch):
    orig = Q.dilation_rule

    def bad(X, Y, Wt, V, m, cx=0.0, cy=0.0):
        x, y, w = orig(X, Y, Wt, V, m, cx, cy)
        a, _ = Q.gauss_legendre(m, 0.0, 1.0)
        return x, y, w / np.tile(a, len(X))  # drops the alpha_l Jacobian factor
    assert _pins_fail(monkeypatch, lambda mp: mp.setattr(Q, "dilation_rule", bad))


def test_planted_phase_sign(monkeypatch):
    orig = D.direct_sum
    # conj of the integrand = wrong sign of the phase, same normalisation
    bad = lambda x, y, w, xi, eta, lz: -np.conj(orig(x, y, w, xi, eta, lz))
    assert _pins_fail(monkeypatch, lambda mp: mp.setattr(D, "direct_sum", bad))


def test_planted_transposed_coordinates(monkeypatch):
    orig = D.direct_sum
    bad = lambda x, y, w, xi, eta, lz: orig(x, y, w, eta, xi, lz)
    # disc is symmetric under the swap; the star target (0.4, 0.25) is not
    assert _pins_fail(monkeypatch, lambda mp: mp.setattr(D, "direct_sum", bad))


def test_planted_wrong_tangent(monkeypatch):
    orig = Q.fourier_line_rule

    def bad(params, n_panels, p, cx=0.0, cy=0.0):
        X, Y, Wt, V = orig(params, n_panels, p, cx, cy)
        return X, Y, V, Wt  # W and V swapped
    assert _pins_fail(monkeypatch, lambda mp: mp.setattr(Q, "fourier_line_rule", bad))


# ------------------------------------------------------------------ eq. li far from the boundary
def _disc_ptr(n, R=1.0):
    return Q.ptr_line_rule(lambda s: (R * np.cos(s), R * np.sin(s)),
                           lambda s: (-R * np.sin(s), R * np.cos(s)), n)


def test_line_integral_far_matches_nsli_on_a_converged_rule():
    """Eq. li with the rounded winding number (Appendix remark r:shadfix) and
    eq. nsli are the same integral: on a converged rule they agree at far
    targets inside (u_geom = 1) and outside (u_geom = 0) the disc, for u^ap
    and u^oc; near targets take eq. nsli unchanged."""
    from oracle import direct
    X, Y, Wt, V = _disc_ptr(240)
    xi = np.array([0.0, 0.35, -0.2, 1.7, -2.5, 0.995])
    eta = np.array([0.0, -0.3, 0.45, 0.4, 1.0, 0.0])
    uap, uoc = direct.line_integral_far(X, Y, Wt, V, xi, eta, 0.05, 0.25)
    un = direct.nsli(X, Y, Wt, V, xi, eta, 0.05)
    assert np.max(np.abs(uap - un)) < 1e-13
    assert np.max(np.abs(uoc - (1.0 - un))) < 1e-13
    assert uoc[-1] == 1.0 - un[-1]   # nearest node 0.005 away: eq. nsli
    # on axis the disc's closed form
    assert abs(uap[0] - CF.disc_on_axis(1.0, 0.05)) < 1e-13


def test_line_integral_far_uses_the_exact_winding_number():
    """With a coarse rule the quadrature's winding number (eq. geom) is not
    an integer; eq. li replaces it by the integer, so the two forms differ
    by exactly (round(w) - w), w = 1/(2 pi) sum (r x ds)/r^2 (eq. nsli =
    w - 1/(2 pi) sum e^{i pi r^2/lz} (r x ds)/r^2)."""
    from oracle import direct
    X, Y, Wt, V = _disc_ptr(9, R=1.0)
    xi, eta = np.array([0.3, 3.0]), np.array([0.1, -0.5])
    uap, uoc = direct.line_integral_far(X, Y, Wt, V, xi, eta, 0.1, 0.3)
    un = direct.nsli(X, Y, Wt, V, xi, eta, 0.1)
    for k in range(2):
        rx, ry = X - xi[k], Y - eta[k]
        w = np.sum((rx * V - ry * Wt) / (rx * rx + ry * ry)) / (2 * np.pi)
        assert abs(w - np.rint(w)) > 1e-9          # the coarse rule's winding is inexact
        assert abs((uap[k] - un[k]) - (np.rint(w) - w)) < 1e-13
        assert abs(uoc[k] - (1.0 - uap[k])) < 1e-13
    assert np.rint(np.sum(((X - 0.3) * V - (Y - 0.1) * Wt) / ((X - 0.3) ** 2 + (Y - 0.1) ** 2))
                   / (2 * np.pi)) == 1.0


# ------------------------------------------------------------------ source screens (Sec. 5)
def _field_module():
    import importlib
    return importlib.import_module("oracle.field")


def _screen_grid(f, box, n1, n2):
    xs = np.linspace(box[0], box[1], n1)
    ys = np.linspace(box[2], box[3], n2)
    X, Y = np.meshgrid(xs, ys)
    return f(X, Y)


def test_screen_interpolation_reproduces_quadratics():
    """Cubic convolution with a = -1/2 is exact for polynomials of degree <= 2
    inside the samples' interior (and not for cubics)."""
    FL = _field_module()
    box = (-1.2, 1.3, -1.1, 1.0)
    f = lambda x, y: 0.3 + 0.7 * x - 0.2 * y + 0.5 * x * x - 0.4 * x * y + 0.9 * y * y
    g = W.rng(41, 0)
    x, y = g.uniform(-0.95, 1.05, 2000), g.uniform(-0.85, 0.75, 2000)
    s = FL.screen_value({"amp": _screen_grid(f, box, 13, 11), "box": box}, 1.0, x, y)
    assert np.max(np.abs(s - f(x, y))) < 1e-13
    f3 = lambda x, y: x ** 3
    s3 = FL.screen_value({"amp": _screen_grid(f3, box, 13, 11), "box": box}, 1.0, x, y)
    assert np.max(np.abs(s3 - f3(x, y))) > 1e-5


def test_screen_amplitude_disc_on_axis_closed_form():
    """Disc of radius R under the amplitude screen A = 1 - r^2/R^2: on axis,
    u = (pi/(i lz)) int_0^{R^2} (1 - t/R^2) e^{i a t} dt (a = pi/lz), i.e.
    (pi/(i lz)) [E/(i a) - (R^2 e^{i a R^2}/(i a) - E/(i a)^2)/R^2], E = e^{i a R^2} - 1."""
    FL = _field_module()
    R, lz = 1.0, 0.1
    box = (-1.3, 1.3, -1.3, 1.3)
    amp = _screen_grid(lambda x, y: 1.0 - (x * x + y * y) / (R * R), box, 27, 27)
    u = FL.field([W.fourier_family([R], 64, 16, 64)], lz, 1.0, np.array([0.0]), np.array([0.0]),
                 screen={"amp": amp, "box": box})[0]
    a = np.pi / lz
    T = R * R
    E = np.exp(1j * a * T) - 1.0
    ref = (np.pi / (1j * lz)) * (E / (1j * a) - (T * np.exp(1j * a * T) / (1j * a) - E / (1j * a) ** 2) / T)
    assert abs(u - ref) < 1e-11


def test_screen_tilt_is_a_target_shift():
    """Linear OPD = tx x + ty y (a tilted incident wave) shifts the pattern by
    d = (tx z, ty z): u_s(xi) = e^{i pi (|xi|^2 - |xi - d|^2)/lz} u(xi - d),
    term by term in the discrete sum (linear OPD is interpolated exactly)."""
    FL = _field_module()
    fam = [W.fourier_family(W.STAR_PARAMS, 32, 16, 24)]
    lam, z, tx, ty = 0.02, 2.0, 0.03, -0.05
    box = (-1.6, 1.6, -1.6, 1.6)
    opd = _screen_grid(lambda x, y: tx * x + ty * y, box, 17, 17)
    xi, eta = W.disc_targets(60, 1.2, 42)
    us = FL.field(fam, lam, z, xi, eta, screen={"opd": opd, "box": box})
    d1, d2 = tx * z, ty * z
    u0 = FL.field(fam, lam, z, xi - d1, eta - d2)
    ph = np.exp(1j * np.pi * (xi ** 2 + eta ** 2 - (xi - d1) ** 2 - (eta - d2) ** 2) / (lam * z))
    assert np.max(np.abs(us - ph * u0)) < 1e-12


def test_screen_defocus_is_a_new_distance():
    """Quadratic OPD = -(x^2 + y^2)/(2D) (a converging wave, focus D) gives the
    field at the effective distance 1/z' = 1/z - 1/D on targets scaled by z'/z:
    u_s(xi; z) = (z'/z) e^{i pi (|xi|^2/z - |xi'|^2/z')/lam} u(xi'; z'), xi' = xi z'/z,
    term by term (the spherical incidence of Sec. 2 with the sign of D reversed)."""
    FL = _field_module()
    fam = [W.fourier_family([1.0, 0.1, 0.0, 0.05, 0.0], 32, 16, 24)]
    lam, z, D = 0.01, 3.0, 7.0
    box = (-1.5, 1.5, -1.5, 1.5)
    opd = _screen_grid(lambda x, y: -(x * x + y * y) / (2.0 * D), box, 21, 21)
    xi, eta = W.disc_targets(60, 1.0, 43)
    us = FL.field(fam, lam, z, xi, eta, screen={"opd": opd, "box": box})
    zp = 1.0 / (1.0 / z - 1.0 / D)
    xp, ep = xi * zp / z, eta * zp / z
    u0 = FL.field(fam, lam, zp, xp, ep)
    ref = (zp / z) * np.exp(1j * np.pi * ((xi ** 2 + eta ** 2) / z - (xp ** 2 + ep ** 2) / zp) / lam) * u0
    assert np.max(np.abs(us - ref)) < 1e-11


# ------------------------------------------------------------------ triangle unions (Sec. 4.3)
@pytest.mark.parametrize("level", [0, 1, 2, 3, 5])
def test_koch_area_closed_form(level):
    """Weights of the snowflake's triangle rules sum to the level-L area
    A_L = A_0 (1 + sum_{k=1}^L 3 4^(k-1) / 9^k), A_0 = 3 sqrt(3)/4 (side sqrt(3)),
    and the triangle counts are 1 + 3 sum_{k<L} 4^k (Sec. 4.3)."""
    fams = W.koch_families(level, 0.2)
    total = sum(Q.family_nodes(f)[2].sum() for f in fams)
    A0 = 3.0 * np.sqrt(3.0) / 4.0
    AL = A0 * (1.0 + sum(3.0 * 4.0 ** (k - 1) / 9.0 ** k for k in range(1, level + 1)))
    assert abs(total - AL) < 1e-13
    assert sum(len(f["tri"]) for f in fams) == 1 + 3 * sum(4 ** k for k in range(level))


def test_triangle_rule_polynomial_exactness():
    """The p x p triangle rule integrates x^a y^b (a + b <= 2p - 2) exactly:
    against Green's theorem, iint x^a y^b = oint x^(a+1)/(a+1) y^b dy over the
    counter-clockwise edges, each edge by a 12-point Gauss rule in t."""
    g = W.rng(44, 0)
    v = g.uniform(-1, 1, 6)
    if (v[2] - v[0]) * (v[5] - v[1]) - (v[3] - v[1]) * (v[4] - v[0]) < 0:
        v = v[[0, 1, 4, 5, 2, 3]]
    x, y, w = Q.triangle_rule(v[None, :], 4)
    t, wt = Q.gauss_legendre(12, 0.0, 1.0)
    P = v.reshape(3, 2)
    for a in range(7):
        for b in range(7 - a):
            exact = 0.0
            for k in range(3):
                p0, p1 = P[k], P[(k + 1) % 3]
                xs, ys = p0[0] + t * (p1[0] - p0[0]), p0[1] + t * (p1[1] - p0[1])
                exact += np.sum(wt * xs ** (a + 1) / (a + 1) * ys ** b) * (p1[1] - p0[1])
            assert abs(np.sum(w * x ** a * y ** b) - exact) < 1e-13 * max(1.0, abs(exact))


def test_square_from_two_triangles_fresnel_integrals():
    """A rectangle as two triangles: u^ap = F_x F_y / (2i), F = (C(u2) - C(u1))
    + i (S(u2) - S(u1)), u = sqrt(2/lz) (edge - target) (eq. fres separates)."""
    from scipy.special import fresnel
    x1, x2, y1, y2, lz = -0.4, 0.6, -0.5, 0.3, 0.05
    tri = np.array([[x1, y1, x2, y1, x2, y2], [x1, y1, x2, y2, x1, y2]])
    fam = [{"kind": "triangles", "tri": tri, "p": 120}]
    xi = np.array([0.0, 0.3, -0.7, 0.9, 0.1])
    eta = np.array([0.0, -0.2, 0.4, 0.6, -0.9])
    u = oracle.field(fam, lz, 1.0, xi, eta)

    def F(a, b, c):
        s2, c2 = fresnel(np.sqrt(2.0 / lz) * (b - c))
        s1, c1 = fresnel(np.sqrt(2.0 / lz) * (a - c))
        return (c2 - c1) + 1j * (s2 - s1)
    ref = F(x1, x2, xi) * F(y1, y2, eta) / 2j
    assert np.max(np.abs(u - ref)) < 1e-12


def test_triangle_rule_matches_polygon_line_rule():
    """The snowflake's base triangle two ways: the p x p triangle rule, and
    its three edges as a vector line rule (Gauss panels) dilated about the
    centroid (eqs. vliq, aqnod, aqwei): the fields agree once both converge."""
    tri = W.koch_triangles(0)[0]
    P = tri.reshape(3, 2)
    t, wt = Q.gauss_legendre(60, 0.0, 1.0)
    X = np.concatenate([P[k, 0] + t * (P[(k + 1) % 3, 0] - P[k, 0]) for k in range(3)])
    Y = np.concatenate([P[k, 1] + t * (P[(k + 1) % 3, 1] - P[k, 1]) for k in range(3)])
    Wt = np.concatenate([wt * (P[(k + 1) % 3, 0] - P[k, 0]) for k in range(3)])
    V = np.concatenate([wt * (P[(k + 1) % 3, 1] - P[k, 1]) for k in range(3)])
    line = {"kind": "line_rule", "X": X, "Y": Y, "W": Wt, "V": V, "m": 60}
    xi, eta = W.disc_targets(40, 1.0, 45)
    u1 = oracle.field([{"kind": "triangles", "tri": tri, "p": 60}], 0.25, 1.0, xi, eta)
    u2 = oracle.field([line], 0.25, 1.0, xi, eta)
    assert np.max(np.abs(u1 - u2)) < 1e-11


# ------------------------------------------------------------------ perturbed starshades (Sec. 5)
def _resolved_starshade(**kw):
    return W.petal_family(6, 0.4, 1.0, {"kind": "hg", "b": 0.5, "q": 2.5}, 48, 24, 96, 32, **kw)


def test_moved_petals_zero_motion_is_the_ideal_rule():
    fam = _resolved_starshade()
    x0, y0, w0 = Q.family_nodes(fam)
    x, y, w = Q.family_nodes(dict(fam, motion=np.zeros((6, 3))))
    n = len(x0)
    assert np.array_equal(x[:n], x0) and np.array_equal(y[:n], y0) and np.array_equal(w[:n], w0)
    assert len(x) == n + 6 * 48 * 8 and np.all(w[n:] == 0.0)


def test_moved_petals_common_translation_is_the_translated_starshade():
    """Every petal translated by the same T: the root-arc patches sweep the
    disc circle into its translate (adjacent patch sides cancel), so the
    construction equals the ideal starshade centred at T."""
    T = (0.013, -0.021)
    fam = _resolved_starshade()
    moved = dict(fam, motion=np.tile([0.0, T[0], T[1]], (6, 1)))
    xi, eta = W.disc_targets(30, 1.0, 60)
    u1 = oracle.field([moved], 0.1, 1.0, xi, eta)
    u2 = oracle.field([dict(fam, cx=T[0], cy=T[1])], 0.1, 1.0, xi, eta)
    assert np.max(np.abs(u1 - u2)) < 1e-11


def test_root_arc_patch_areas():
    """Pure translation T: the patch is the arc swept by T, signed area
    T x (g(1) - g(0)) (its chord); pure rotation about the centre: the two
    end segments cancel, area 0 (so rotations keep the starshade's area)."""
    a, Np = 0.4, 6
    for k in range(Np):
        th0, th1 = 2 * np.pi * (k - 0.5) / Np, 2 * np.pi * (k + 0.5) / Np
        ch = a * np.array([np.cos(th1) - np.cos(th0), np.sin(th1) - np.sin(th0)])
        T = np.array([0.02 * np.cos(k), -0.015 + 0.003 * k])
        w = Q.root_arc_patch(a, Np, k, (0.0, T[0], T[1]), 24, 8)[2]
        assert abs(w.sum() - (T[0] * ch[1] - T[1] * ch[0])) < 1e-15
        w = Q.root_arc_patch(a, Np, k, (0.01 * (k - 2), 0.0, 0.0), 24, 8)[2]
        assert abs(w.sum()) < 1e-15
    fam = _resolved_starshade()
    rot = np.column_stack([0.01 * np.arange(6) - 0.02, np.zeros(6), np.zeros(6)])
    assert abs(Q.family_nodes(dict(fam, motion=rot))[2].sum() - Q.family_nodes(fam)[2].sum()) < 1e-13


# ------------------------------------------------------------------ Fraunhofer limit
def _fraunhofer_disc_error(lz, R=1.0):
    """max |u - u_F| / max |u_F| for the disc, u_F = (1/(i lz)) e^{i pi rho^2/lz}
    pi R^2 2 J1(v)/v, v = 2 pi R rho / lz (the Airy pattern)."""
    from scipy import special
    fam = [W.fourier_family([R], 16, 16, 16)]
    rho = np.linspace(0.0, 3.0 * lz, 25)
    u = oracle.field(fam, lz, 1.0, rho * np.cos(0.3), rho * np.sin(0.3))
    v = 2 * np.pi * R * rho / lz
    airy = np.where(v > 0, 2 * special.j1(v) / np.where(v > 0, v, 1.0), 1.0)
    ref = np.exp(1j * np.pi * rho ** 2 / lz) / (1j * lz) * np.pi * R * R * airy
    return np.max(np.abs(u - ref)) / np.max(np.abs(ref))


def test_fraunhofer_limit_disc_airy():
    """For F = R^2/lz -> 0 the source chirp e^{i pi |x|^2/lz}, the last factor
    of eq. split, tends to 1 over the aperture, and u tends to the target
    chirp times the aperture's Fourier transform at xi/lz (the Fraunhofer
    limit, Sec. 4.1's remark on small Fresnel numbers).  The leading
    correction is pi R^2/(2 lz), so the error falls tenfold for a tenfold
    lz."""
    e3, e4 = _fraunhofer_disc_error(1e3), _fraunhofer_disc_error(1e4)
    assert e4 <= 0.6 * np.pi / 1e4
    assert 8.0 < e3 / e4 < 12.0


def _rect_fraunhofer_error(lz=1e3):
    """Off-centre rectangle [x0 -+ a] x [y0 -+ b] (two triangles): its Fourier
    transform is e^{-2 pi i q.c} sin(2 pi a qx)/(pi qx) sin(2 pi b qy)/(pi qy),
    whose shift phase fixes the sign of the xi.x term."""
    x0, y0, a, b = 0.3, -0.2, 0.5, 0.25
    P = [(x0 - a, y0 - b), (x0 + a, y0 - b), (x0 + a, y0 + b), (x0 - a, y0 + b)]
    tri = np.array([[*P[0], *P[1], *P[2]], [*P[0], *P[2], *P[3]]])
    fam = [{"kind": "triangles", "tri": tri, "p": 12}]
    g = W.rng(9, 0)
    xi, eta = g.uniform(-2, 2, 40) * lz, g.uniform(-2, 2, 40) * lz
    u = oracle.field(fam, lz, 1.0, xi, eta)
    qx, qy = xi / lz, eta / lz
    sx = np.sin(2 * np.pi * a * qx) / (np.pi * qx)
    sy = np.sin(2 * np.pi * b * qy) / (np.pi * qy)
    ref = (np.exp(1j * np.pi * (xi ** 2 + eta ** 2) / lz) / (1j * lz)
           * np.exp(-2j * np.pi * (qx * x0 + qy * y0)) * sx * sy)
    rmax2 = max(px * px + py * py for px, py in P)
    return np.max(np.abs(u - ref)) / (4 * a * b / lz), np.pi * rmax2 / lz


def test_fraunhofer_limit_offset_rectangle():
    err, bound = _rect_fraunhofer_error()
    assert err <= bound


def test_planted_mirrored_nodes_fail_the_rectangle_limit(monkeypatch):
    orig = D.direct_sum
    monkeypatch.setattr(D, "direct_sum", lambda x, y, w, xi, eta, lz: orig(-x, -y, w, xi, eta, lz))
    err, bound = _rect_fraunhofer_error()
    assert err > 100 * bound


def test_oracle_sums_do_not_depend_on_the_thread_count(tmp_path):
    """The C sums (direct, type 3, NSLI, the far-target line integral and the
    adjoint sums) parallelise over their outputs only, each output's sum in a
    fixed order, so one and four OpenMP threads give bit-identical results."""
    import subprocess
    import sys
    prog = (
        "import sys, numpy as np\n"
        "sys.path.insert(0, %r)\n"
        "import workloads as W\n"
        "from oracle import direct as D, quadrature as Q\n"
        "fam = W.fourier_family(W.STAR_PARAMS, 16, 16, 24)\n"
        "x, y, w = Q.family_nodes(fam)\n"
        "X, Y, Wt, V, _, _ = Q.family_line_rule(fam)\n"
        "g = W.rng(95, 0)\n"
        "xi, eta = g.uniform(-1.5, 1.5, 64), g.uniform(-1.5, 1.5, 64)\n"
        "c = w * np.exp(1j * np.pi * (x * x + y * y) / 0.05)\n"
        "far = D.line_integral_far(X, Y, Wt, V, xi, eta, 0.05, 0.2)\n"
        "adj = D.adjoint_sums(x[:64], y[:64], xi, eta, 0.05, c[:64])\n"
        "np.save(sys.argv[1], np.stack([D.direct_sum(x, y, w, xi, eta, 0.05),\n"
        "                               D.sum3(x, y, c, xi, eta, 0.05),\n"
        "                               D.nsli(X, Y, Wt, V, xi, eta, 0.05),\n"
        "                               far[0], far[1], adj[0]]))\n"
    ) % os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = {}
    for n in (1, 4):
        f = str(tmp_path / ("t%d.npy" % n))
        env = dict(os.environ, OMP_NUM_THREADS=str(n))
        subprocess.run([sys.executable, "-c", prog, f], check=True, env=env, timeout=300)
        out[n] = np.load(f)
    assert np.array_equal(out[1], out[4])


def test_triangle_rule_vertex_choice_and_orientation():
    """Sec. 4.3's triangle rule dilates about one vertex; the field it gives
    must not depend on which vertex (cyclic relabelling), and the reversed
    orientation negates every weight, hence the field."""
    v = [(0.05, -0.1), (0.9, 0.2), (0.3, 0.85)]
    xi, eta = np.array([0.0, 0.5, -0.7]), np.array([0.1, 0.4, 0.9])
    lz = 0.1

    def u(order):
        tri = np.array([[*v[order[0]], *v[order[1]], *v[order[2]]]])
        return oracle.field([{"kind": "triangles", "tri": tri, "p": 40}], lz, 1.0, xi, eta)

    ref = u((0, 1, 2))
    assert np.max(np.abs(u((1, 2, 0)) - ref)) < 1e-12
    assert np.max(np.abs(u((2, 0, 1)) - ref)) < 1e-12
    assert np.max(np.abs(u((0, 2, 1)) + ref)) < 1e-12
    x, y, w = Q.triangle_rule(np.array([[*v[0], *v[2], *v[1]]]), 5)
    area = 0.5 * ((v[1][0] - v[0][0]) * (v[2][1] - v[0][1]) - (v[1][1] - v[0][1]) * (v[2][0] - v[0][0]))
    assert abs(w.sum() + area) < 1e-15
