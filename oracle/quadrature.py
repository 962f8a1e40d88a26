"""Areal quadrature, built the plain way (test infrastructure only; see oracle/__init__.py).

Everything is FP64 numpy, vectorised but with no blocking or fusion beyond the
formulas below, so each line can be checked against the paper by eye.

Panel-family description (plain dict, produced by ``workloads.py``):

``{"kind": "fourier", "params": [r0, a1, b1, a2, b2, ...], "n_panels": P,
   "p": p, "m": m, "cx": cx, "cy": cy}``
    Boundary r(t) = r0 + sum_k (a_k cos kt + b_k sin kt) about the centre
    (cx, cy), t in [0, 2pi) counter-clockwise; P panels of p Gauss-Legendre
    nodes on t; m radial Gauss-Legendre nodes in the dilation rule.

``{"kind": "line_rule", "X", "Y", "W", "V", "m", "cx", "cy"}``
    An explicit vector line rule (eq. vliq) plus m radial nodes.

``{"kind": "nodes", "x", "y", "w"}``
    An explicit areal rule (eq. aq).

``{"kind": "petals", "n_petals": Np, "a": a, "R": R, "m": m, "n_p": n_p,
   "n_d": n_d, "m_d": m_d, "profile": {...}, "cx": cx, "cy": cy}``
    The starshade rule of Sec. 4.2: the disc r < a (n_d-node periodic
    trapezoid boundary rule, m_d radii) plus Np petals whose angular width at
    radius r is 2 pi A(r) / Np (eq. Omega), each covered by m Gauss-Legendre
    radii on (a, R) times n_p Gauss-Legendre angles.  The profile A is
    ``{"kind": "hg", "b": b, "q": q}`` (offset hyper-Gaussian
    A = exp(-((r - a)/b)^q)), ``{"kind": "bspline", "coefs": [...]}`` (clamped
    uniform cubic B-spline on [a, R]) or ``{"kind": "table", "A": [...]}``
    (values at the m ascending Gauss-Legendre radii).  The whole shape is
    translated by (cx, cy).
"""
import numpy as np


def gauss_legendre(n, a=-1.0, b=1.0):
    """n-point Gauss-Legendre nodes/weights on (a, b) (the rule named in Sec. 3.1).

    The library primitive ``numpy.polynomial.legendre.leggauss`` supplies the
    rule on (-1, 1); the affine map to (a, b) scales the weights by (b-a)/2.
    """
    t, wt = np.polynomial.legendre.leggauss(int(n))
    x = 0.5 * (b - a) * (t + 1.0) + a
    return x, 0.5 * (b - a) * wt


def fourier_radius(params, t):
    """r(t) = r0 + sum_k (a_k cos kt + b_k sin kt) and its derivative r'(t)."""
    params = np.asarray(params, dtype=np.float64)
    r = np.full_like(t, params[0])
    dr = np.zeros_like(t)
    K = (len(params) - 1) // 2
    for k in range(1, K + 1):
        a, b = params[2 * k - 1], params[2 * k]
        r += a * np.cos(k * t) + b * np.sin(k * t)
        dr += k * (-a * np.sin(k * t) + b * np.cos(k * t))
    return r, dr


def fourier_line_rule(params, n_panels, p, cx=0.0, cy=0.0):
    """Vector line rule (X_i, Y_i, W_i, V_i) of eq. vliq on a Fourier star boundary.

    The boundary x(t) = (cx + r(t) cos t, cy + r(t) sin t) is traversed
    counter-clockwise for t in [0, 2pi).  As in eq. vliq1 the vector line
    integral is int f(x(t)) . x'(t) dt; here the t-integral is split into
    n_panels equal panels, each with a p-point Gauss-Legendre rule (the
    configurations' choice in place of the periodic trapezoid rule of
    eq. ptr), so W_i = what_i X'(t_i), V_i = what_i Y'(t_i).
    Boundary index i runs panel-major, node-minor.
    """
    tq, wq = gauss_legendre(p, 0.0, 2.0 * np.pi / n_panels)
    t = (np.arange(n_panels)[:, None] * (2.0 * np.pi / n_panels) + tq[None, :]).ravel()
    what = np.tile(wq, n_panels)
    r, dr = fourier_radius(params, t)
    X = cx + r * np.cos(t)
    Y = cy + r * np.sin(t)
    dX = dr * np.cos(t) - r * np.sin(t)
    dY = dr * np.sin(t) + r * np.cos(t)
    return X, Y, what * dX, what * dY


def ptr_line_rule(curve, dcurve, n):
    """Periodic trapezoid vector line rule, eq. ptr: t_i = 2 pi i / n, weights 2pi/n."""
    t = 2.0 * np.pi * np.arange(1, n + 1) / n
    X, Y = curve(t)
    dX, dY = dcurve(t)
    return X, Y, (2.0 * np.pi / n) * dX, (2.0 * np.pi / n) * dY


def dilation_rule(X, Y, W, V, m, cx=0.0, cy=0.0):
    """Areal rule by dilation about (cx, cy): eqs. aqnod and aqwei (Sec. 3.1).

    With alpha_l, wtilde_l the m-point Gauss-Legendre rule on (0, 1):
        x_{l + (i-1)m} = c + alpha_l (X_i - c)
        w_{l + (i-1)m} = alpha_l wtilde_l ((X_i - cx) V_i - (Y_i - cy) W_i)
    (the paper's formulas with the origin moved to c).  Nodes may fall outside
    a non-star-shaped domain and weights may be negative; nothing is clamped.
    Returned arrays are ordered with the radial index l fastest.
    """
    alpha, wt = gauss_legendre(m, 0.0, 1.0)
    dx = np.asarray(X) - cx
    dy = np.asarray(Y) - cy
    cross = dx * np.asarray(V) - dy * np.asarray(W)
    x = cx + alpha[None, :] * dx[:, None]
    y = cy + alpha[None, :] * dy[:, None]
    w = (alpha * wt)[None, :] * cross[:, None]
    return x.ravel(), y.ravel(), w.ravel()


def bspline_knots(a, R, n):
    """Clamped uniform cubic knot vector on [a, R] for n >= 4 coefficients."""
    inner = np.linspace(a, R, n - 2)[1:-1]
    return np.concatenate([[a] * 4, inner, [R] * 4])


def petal_profile(profile, a, R, r):
    """Apodisation A(r) of Sec. 4.2 on [a, R] (the profile dict of a petal family)."""
    kind = profile["kind"]
    if kind == "hg":
        return np.exp(-((r - a) / profile["b"]) ** profile["q"])
    if kind == "bspline":
        from scipy.interpolate import BSpline
        c = np.asarray(profile["coefs"], float)
        return BSpline(bspline_knots(a, R, len(c)), c, 3)(r)
    if kind == "table":
        return np.asarray(profile["A"], float)
    raise ValueError("unknown profile kind %r" % kind)


def starshade_rule(fam):
    """Areal rule for the starshade ("flower") of eq. Omega, Sec. 4.2.

    Disc part: the periodic trapezoid rule (eq. ptr) on the circle
    (a cos t, a sin t) with n_d nodes, dilated with m_d radii (eqs. aqnod,
    aqwei).  Petal part: (r_l, what_l) the m-point Gauss-Legendre rule on
    (a, R), (t_i, omegahat_i) the n_p-point Gauss-Legendre rule on
    [-pi/Np, pi/Np]; in petal k (centred on angle 2 pi k / Np, where
    P(Np theta) = 0) the node at (l, i) is
        r_l (cos(A(r_l) t_i + 2 pi k/Np), sin(A(r_l) t_i + 2 pi k/Np)),
    weight r_l what_l A(r_l) omegahat_i (area element r dr dtheta with
    theta = A(r) t; the printed A(r_i) is read as A(r_l)).
    Order: disc nodes (boundary-major, radius fastest), then petal k, angle
    i, radius l fastest.  N = n_d m_d + Np n_p m.
    """
    Np, a, R = int(fam["n_petals"]), float(fam["a"]), float(fam["R"])
    m, n_p = int(fam["m"]), int(fam["n_p"])
    n_d, m_d = int(fam.get("n_d", 0)), int(fam.get("m_d", 0))
    cx, cy = fam.get("cx", 0.0), fam.get("cy", 0.0)
    xs, ys, ws = [], [], []
    if n_d > 0:
        X, Y, W, V = ptr_line_rule(lambda t: (a * np.cos(t), a * np.sin(t)),
                                   lambda t: (-a * np.sin(t), a * np.cos(t)), n_d)
        x, y, w = dilation_rule(X, Y, W, V, m_d)
        xs.append(x)
        ys.append(y)
        ws.append(w)
    r, wr = gauss_legendre(m, a, R)
    t, wt = gauss_legendre(n_p, -np.pi / Np, np.pi / Np)
    A = petal_profile(fam["profile"], a, R, r)
    motion = fam.get("motion")
    motion = None if motion is None else np.asarray(motion, float).reshape(Np, 3)
    for k in range(Np):
        theta = A[None, :] * t[:, None] + 2.0 * np.pi * k / Np     # [i, l]
        px = (r[None, :] * np.cos(theta)).ravel()
        py = (r[None, :] * np.sin(theta)).ravel()
        if motion is not None:   # rigid motion about the centre, weights unchanged
            phi, tx, ty = motion[k]
            px, py = (np.cos(phi) * px - np.sin(phi) * py + tx,
                      np.sin(phi) * px + np.cos(phi) * py + ty)
        xs.append(px)
        ys.append(py)
        ws.append((wt[:, None] * (r * wr * A)[None, :]).ravel())
    if motion is not None:
        for k in range(Np):
            x, y, w = root_arc_patch(a, Np, k, motion[k], max(2 * n_p, 16), 8)
            xs.append(x)
            ys.append(y)
            ws.append(w)
    return cx + np.concatenate(xs), cy + np.concatenate(ys), np.concatenate(ws)


def root_arc_patch(a, Np, k, motion, qs, qt):
    """Sec. 5 (perturbed starshades, second construction): the signed region
    joining petal k's root arc on the disc circle r = a (angles 2 pi k/Np -
    pi/Np .. + pi/Np) to its rigidly moved image, as the ruled surface
    P(s, t) = (1 - t) g(s) + t M(g(s)), g the arc on s in (0, 1), M(x) =
    R(phi) x + (tx, ty), integrated on a qs x qt Gauss-Legendre product rule
    with the Jacobian dP/dt x dP/ds (positive where the petal has moved
    outward, leaving a gap; negative over an overlap).  About the origin;
    ordered s-major, t fastest."""
    phi, tx, ty = motion
    s, ws = gauss_legendre(qs, 0.0, 1.0)
    t, wt = gauss_legendre(qt, 0.0, 1.0)
    th = 2.0 * np.pi * (k - 0.5 + s) / Np
    g = np.stack([a * np.cos(th), a * np.sin(th)], 1)
    dg = (2.0 * np.pi / Np) * np.stack([-a * np.sin(th), a * np.cos(th)], 1)
    Rm = np.array([[np.cos(phi), -np.sin(phi)], [np.sin(phi), np.cos(phi)]])
    Mg = g @ Rm.T + np.array([tx, ty])
    dMg = dg @ Rm.T
    P = (1.0 - t)[None, :, None] * g[:, None, :] + t[None, :, None] * Mg[:, None, :]
    Pt = (Mg - g)[:, None, :]
    Ps = (1.0 - t)[None, :, None] * dg[:, None, :] + t[None, :, None] * dMg[:, None, :]
    J = Pt[..., 0] * Ps[..., 1] - Pt[..., 1] * Ps[..., 0]
    w = ws[:, None] * wt[None, :] * J
    return P[..., 0].ravel(), P[..., 1].ravel(), w.ravel()


def family_line_rule(fam):
    """The boundary vector line rule (X, Y, W, V) and centre of one panel family."""
    kind = fam["kind"]
    if kind == "fourier":
        cx, cy = fam.get("cx", 0.0), fam.get("cy", 0.0)
        return fourier_line_rule(fam["params"], fam["n_panels"], fam["p"], cx, cy) + (cx, cy)
    if kind == "line_rule":
        return (np.asarray(fam["X"], float), np.asarray(fam["Y"], float),
                np.asarray(fam["W"], float), np.asarray(fam["V"], float),
                fam.get("cx", 0.0), fam.get("cy", 0.0))
    raise ValueError("family kind %r has no line rule" % kind)


def triangle_rule(tri, p, cx=0.0, cy=0.0):
    """p x p areal rule of each triangle (Sec. 4.3): move vertex v0 to the
    origin, discretise the line integral along the opposite edge v1 -> v2
    with p Gauss-Legendre nodes (X_i = v1 + s_i (v2 - v1), tangent weights
    what_i (v2 - v1)) and apply the dilation rule (eqs. aqnod, aqwei) with the
    same p-point rule as radii: x = v0 + alpha_l (X_i - v0),
    w = alpha_l what_l ((X_i - v0) x tangent_i) = alpha_l what_l what_i (v1 - v0) x (v2 - v1).
    tri: (n, 6) rows (v0x, v0y, v1x, v1y, v2x, v2y).  Ordered triangle-major,
    edge node, radius fastest; all triangles at once (numpy broadcasting)."""
    tri = np.asarray(tri, float).reshape(-1, 6)
    s, ws = gauss_legendre(p, 0.0, 1.0)
    v0, v1, v2 = tri[:, 0:2], tri[:, 2:4], tri[:, 4:6]
    d1, e = v1 - v0, v2 - v1
    rel = d1[:, None, :] + s[None, :, None] * e[:, None, :]            # X_i - v0: (n, i, 2)
    cross = (d1[:, 0] * e[:, 1] - d1[:, 1] * e[:, 0])[:, None] * ws[None, :]   # (n, i)
    pts = v0[:, None, None, :] + s[None, None, :, None] * rel[:, :, None, :]   # (n, i, l, 2)
    w = cross[:, :, None] * (s * ws)[None, None, :]
    return cx + pts[..., 0].ravel(), cy + pts[..., 1].ravel(), w.ravel()


def family_nodes(fam):
    """Areal nodes and weights (x, y, w) of one panel family."""
    if fam["kind"] == "triangles":
        return triangle_rule(fam["tri"], fam["p"], fam.get("cx", 0.0), fam.get("cy", 0.0))
    if fam["kind"] == "nodes":
        return (np.asarray(fam["x"], float), np.asarray(fam["y"], float),
                np.asarray(fam["w"], float))
    if fam["kind"] == "petals":
        return starshade_rule(fam)
    X, Y, W, V, cx, cy = family_line_rule(fam)
    return dilation_rule(X, Y, W, V, fam["m"], cx, cy)
