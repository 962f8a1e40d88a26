"""Seeded synthetic workloads shaped like the paper's experiments.

This module only describes inputs: boundary descriptions (panel families),
lambda*z, and target sets, drawn from numpy's seeded generators.  It holds
none of the method's arithmetic, and both the CUDA library and the CPU oracle
receive exactly these arrays.

Panel-family dicts (see oracle/quadrature.py and the C header
include/fresnel.h for how each side reads them):

    {"kind": "fourier", "params": [r0, a1, b1, ...], "n_panels": P, "p": p,
     "m": m, "cx": 0.0, "cy": 0.0}

Workloads (Fresnel number F = R^2 / (lambda z), Sec. 2 eq. fn):

* ``disc``  -- unit disc, F = 10 (lambda z = 0.1), 64 panels x 16 GL x m radial
               (m = 16: 16,384 nodes), 100 x 100 grid with h = 0.03 spanning
               [-1.5, 1.5)^2 (the paper's grid convention, Sec. 3.3).
* ``star``  -- r = 1 + 0.3 cos 5 theta, F = 100 with R = max r = 1.3
               (lambda z = 0.0169), 128 x 16 x 256 = 524,288 nodes;
               grid 1000 x 1000 with h = 0.003, and 1e6 scattered targets
               uniform in the disc of radius 1.5.
* ``starshade_sweep`` -- 24-petal offset hyper-Gaussian starshade
               (A(r) = exp(-((r - 6)/3.9)^6) on [6, 14] m, Sec. 4.2), z = 3.7e7 m,
               64 wavelengths evenly spaced in [400, 1000] nm (F = 13.2 .. 5.3);
               per wavelength m = max(30, ceil(3F)) radii and n_p = max(15,
               ceil(1.5F)) angles per petal, n_d = ceil(0.3 * 24 n_p) disc
               boundary nodes with m_d = m radii (14,040 .. 24,960 nodes);
               512 x 512 grid with h = 2.4/512 over the 2.4 m pupil, of which
               the 205,859 points with rho <= 1.2 are kept.
* ``random_star`` -- r = 1 + sum_{k=1}^{20} a_k cos(k theta + phi_k),
               a_k ~ U(0, 0.02), phi_k ~ U(0, 2 pi); F = 1000 with R = max r
               over 1e5 samples; 640 x 16 x 1024 = 10,485,760 nodes; scattered
               targets uniform in [-1.2, 1.2]^2 (1e8 at full size).
"""
import numpy as np

SEED0 = 20105978


def rng(config_id, stream=0):
    """numpy Generator seeded by the paper id, the workload id and a sub-stream."""
    return np.random.default_rng([SEED0 + int(config_id), int(stream)])


def fourier_family(params, n_panels, p, m, cx=0.0, cy=0.0):
    return {"kind": "fourier", "params": np.asarray(params, dtype=np.float64),
            "n_panels": int(n_panels), "p": int(p), "m": int(m),
            "cx": float(cx), "cy": float(cy)}


def grid_spec(n1, n2, h, x0=0.0, y0=0.0):
    return {"n1": int(n1), "n2": int(n2), "h": float(h), "x0": float(x0), "y0": float(y0)}


# ---------------------------------------------------------------- disc (F = 10)
def disc(m=16, n_panels=64, p=16, n=100, R=1.0):
    return {
        "name": "disc_F10",
        "families": [fourier_family([R], n_panels, p, m)],
        "lam": 0.1, "z": 1.0,
        "grid": grid_spec(n, n, 3.0 / n),
    }


# ---------------------------------------------------------------- star (F = 100)
STAR_PARAMS = [1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.3, 0.0]


def star(n_panels=128, p=16, m=256, n=1000, lz=1.3 ** 2 / 100.0):
    return {
        "name": "star5_F100",
        "families": [fourier_family(STAR_PARAMS, n_panels, p, m)],
        "lam": lz, "z": 1.0,
        "grid": grid_spec(n, n, 3.0 / n),
    }


def disc_targets(M, radius, config_id, stream=1):
    """M targets uniform in the disc |xi| <= radius: rho = radius sqrt(U), theta = 2 pi V."""
    g = rng(config_id, stream)
    u = g.random(M)
    v = g.random(M)
    rho = radius * np.sqrt(u)
    th = 2.0 * np.pi * v
    return rho * np.cos(th), rho * np.sin(th)


def square_targets(M, half, config_id, stream=1):
    """M targets uniform in [-half, half]^2."""
    g = rng(config_id, stream)
    return g.uniform(-half, half, M), g.uniform(-half, half, M)


# ---------------------------------------------------------------- random star (F = 1000)
def random_star_params(config_id=5, K=20, amax=0.02, stream=0):
    g = rng(config_id, stream)
    a = g.uniform(0.0, amax, K)
    ph = g.uniform(0.0, 2.0 * np.pi, K)
    params = [1.0]
    for k in range(K):
        # a cos(k t + ph) = a cos(ph) cos(k t) - a sin(ph) sin(k t)
        params += [a[k] * np.cos(ph[k]), -a[k] * np.sin(ph[k])]
    return np.asarray(params)


def max_radius(params, n=100000):
    th = 2.0 * np.pi * np.arange(n) / n
    params = np.asarray(params)
    r = np.full(n, params[0])
    for k in range(1, (len(params) - 1) // 2 + 1):
        r += params[2 * k - 1] * np.cos(k * th) + params[2 * k] * np.sin(k * th)
    return float(r.max())


def petal_family(n_petals, a, R, profile, m, n_p, n_d=0, m_d=0, cx=0.0, cy=0.0):
    """A starshade (disc r < a plus n_petals petals on [a, R]) as a panel family.

    profile: {"kind": "hg", "b": b, "q": q}, {"kind": "bspline", "coefs": [...]}
    or {"kind": "table", "A": [...]} (A at the m Gauss-Legendre radii).
    """
    prof = dict(profile)
    for key in ("coefs", "A"):
        if key in prof:
            prof[key] = np.asarray(prof[key], dtype=np.float64)
    return {"kind": "petals", "n_petals": int(n_petals), "a": float(a), "R": float(R),
            "m": int(m), "n_p": int(n_p), "n_d": int(n_d), "m_d": int(m_d),
            "profile": prof, "cx": float(cx), "cy": float(cy)}


HG24 = {"n_petals": 24, "a": 6.0, "R": 14.0, "b": 3.9, "q": 6.0, "z": 3.7e7}


def starshade_resolution(fresnel_number, n_petals):
    """(m, n_p, n_d, m_d) for a starshade at Fresnel number F (workload recipe)."""
    F = float(fresnel_number)
    m = max(30, int(np.ceil(3.0 * F)))
    n_p = max(15, int(np.ceil(1.5 * F)))
    n_d = int(np.ceil(0.3 * n_petals * n_p))
    return m, n_p, n_d, m


def starshade_sweep(n_lambda=64, lam_lo=400e-9, lam_hi=1000e-9, n=512, pupil=2.4):
    s = HG24
    lams = np.linspace(lam_lo, lam_hi, n_lambda)
    problems = []
    for lam in lams:
        F = s["R"] ** 2 / (lam * s["z"])
        m, n_p, n_d, m_d = starshade_resolution(F, s["n_petals"])
        fam = petal_family(s["n_petals"], s["a"], s["R"], {"kind": "hg", "b": s["b"], "q": s["q"]},
                           m, n_p, n_d, m_d)
        problems.append({"families": [fam], "lam": float(lam), "z": s["z"]})
    h = pupil / n
    return {"name": "hg24_sweep%d" % n_lambda, "problems": problems,
            "grid": grid_spec(n, n, h), "pupil_radius": 0.5 * pupil}


def spline_starshade(kind="c4", n_coef=None, lams=None, ngrid=None):
    """A starshade whose petal profile is a clamped uniform cubic B-spline.

    Coefficients: the design profile sampled at the spline's Greville
    abscissae (knot averages) plus seeded N(0, 1e-3^2) perturbations.
    kind "c4": the 24-petal HG occulter of ``starshade_sweep`` with 200
    coefficients, 8 wavelengths in [400, 1000] nm, the 256 x 256 pupil grid
    (h = 2.4/256), targets kept for rho <= 1.2 (51,431 points), per-wavelength
    resolution as in ``starshade_sweep``.  kind "hg24_small": the same
    occulter with 20 coefficients at 2 wavelengths on a 24 x 24 grid.  kind
    "small": a 5-petal shape seen far off axis (both the weight and the
    node-motion parts of the gradient matter there).
    Returns (theta, problems, grid, keep): problems = [{"family", "lam", "z"}]
    (family profile data = theta), keep = boolean mask over the grid targets
    (k1 fastest).
    """
    if kind == "small":
        a, R, Np, b, z, half = 0.4, 1.0, 5, 0.35, 1.0, 1.5
        n_coef, lams, ngrid = n_coef or 20, lams or (0.03, 0.05), ngrid or 16
        res = lambda lam: (30, 24, 40, 30)
        x0 = 0.013
    else:
        s = HG24
        a, R, Np, b, z, half = s["a"], s["R"], s["n_petals"], s["b"], s["z"], 1.2
        if kind == "c4":
            n_coef, ngrid = n_coef or 200, ngrid or 256
            lams = lams or tuple(np.linspace(400e-9, 1000e-9, 8))
            res = lambda lam: starshade_resolution(R * R / (lam * z), Np)
            x0 = 0.0
        else:
            n_coef, lams, ngrid = n_coef or 20, lams or (500e-9, 900e-9), ngrid or 24
            res = lambda lam: (40, 20, 144, 40)
            x0 = 0.013
    n = n_coef
    inner = np.linspace(a, R, n - 2)[1:-1]
    t = np.concatenate([[a] * 4, inner, [R] * 4])
    grev = (t[1:n + 1] + t[2:n + 2] + t[3:n + 3]) / 3.0
    theta = np.exp(-((grev - a) / b) ** 6) + 1e-3 * rng(4, 1).standard_normal(n)
    problems = [{"family": petal_family(Np, a, R, {"kind": "bspline", "coefs": theta}, *res(lam)),
                 "lam": float(lam), "z": z} for lam in lams]
    h = 2 * half / ngrid
    k = np.arange(-(ngrid // 2), ngrid - ngrid // 2)
    XI, ETA = np.meshgrid(x0 + h * k, h * k, indexing="xy")
    keep = (XI * XI + ETA * ETA <= half * half).ravel()
    return theta, problems, grid_spec(ngrid, ngrid, h, x0=x0), keep


def random_star(n_panels=640, p=16, m=1024, fresnel_number=1000.0, config_id=5):
    params = random_star_params(config_id)
    R = max_radius(params)
    return {
        "name": "randstar20_F1000",
        "families": [fourier_family(params, n_panels, p, m)],
        "lam": R * R / fresnel_number, "z": 1.0,
    }


def koch_triangles(level):
    """Triangles of the level-L Koch snowflake of maximum radius 1 (Sec. 4.3):
    the equilateral triangle of side sqrt(3) (vertices at angles 90, 210, 330
    degrees on the unit circle), then at each level k = 1..L one triangle of
    side sqrt(3)/3^k on the middle third of every boundary edge of the
    previous level, pointing outward.  Returns one (n_k, 6) array per level
    (rows v0, v1, v2 counter-clockwise), n_0 = 1, n_k = 3 * 4^(k-1)."""
    ang = np.pi / 2 + 2 * np.pi / 3 * np.arange(3)
    P = np.stack([np.cos(ang), np.sin(ang)], 1)
    out = [np.concatenate([P[0], P[1], P[2]])[None, :]]
    A, B = P, np.roll(P, -1, axis=0)            # counter-clockwise boundary edges
    c60, s60 = 0.5, np.sqrt(3.0) / 2.0
    for _ in range(level):
        c = A + (B - A) / 3.0
        d = A + 2.0 * (B - A) / 3.0
        u = d - c                               # outward apex: u turned 60 degrees clockwise
        e = c + np.stack([c60 * u[:, 0] + s60 * u[:, 1], -s60 * u[:, 0] + c60 * u[:, 1]], 1)
        out.append(np.concatenate([c, e, d], 1))
        A, B = (np.stack([A, c, e, d], 1).reshape(-1, 2), np.stack([c, e, d, B], 1).reshape(-1, 2))
    return out


def koch_families(level, lz, p_max=None):
    """The level-L snowflake as one TRIANGLES family per construction level,
    level k with p_k = max(1, ceil(s_k / (0.8 lz))) Gauss-Legendre points per
    direction, s_k = sqrt(3)/3^k its side (node spacing ~ lz; at lz = 0.01
    the largest triangle gets p = 217, the value Sec. 4.3 quotes)."""
    fams = []
    for k, tri in enumerate(koch_triangles(level)):
        pk = max(1, int(np.ceil(np.sqrt(3.0) / 3.0 ** k / (0.8 * lz))))
        if p_max is not None:
            pk = min(pk, p_max)
        fams.append({"kind": "triangles", "tri": tri, "p": pk})
    return fams


def random_star_batch(n=32, config_id=5):
    """32 uneven instances of the random smooth aperture: N_i log-uniform in
    [1e5, 2e6] nodes, F_i = 1000 sqrt(N_i / 1e7), a fresh shape each, M_i
    log-uniform in [1e5, 1e7] targets uniform in [-1.2, 1.2]^2.  Node layout
    as in ``random_star`` (boundary nodes : radii = 10 : 1, 16 per panel).
    Returns (problems, counts); targets of instance i from
    ``square_targets(counts[i], 1.2, config_id, 100 + i)``."""
    g = rng(config_id, 40)
    N = np.exp(g.uniform(np.log(1e5), np.log(2e6), n))
    M = np.exp(g.uniform(np.log(1e5), np.log(1e7), n)).astype(np.int64)
    problems = []
    for i in range(n):
        params = random_star_params(config_id, stream=100 + i)
        m = int(np.ceil(np.sqrt(N[i] / 10.0)))
        n_panels = int(np.ceil(N[i] / (16.0 * m)))
        F = 1000.0 * np.sqrt(N[i] / 1e7)
        R = max_radius(params)
        problems.append({"families": [fourier_family(params, n_panels, 16, m)],
                         "lam": R * R / F, "z": 1.0})
    return problems, [int(x) for x in M]
