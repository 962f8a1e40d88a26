"""Gradient of a starshade loss with respect to its spline petal profile
(test infrastructure only; see oracle/__init__.py).

Loss: L(theta) = mean over problems b and kept targets k of |u^oc_bk|^2,
with u^oc = 1 - u^ap (eq. bab) and u^ap the direct sum of eq. faq over the
starshade rule of Sec. 4.2 whose petal profile A(r) = sum_m theta_m B_m(r) is
a clamped uniform cubic B-spline.

Gradient by differentiating the direct sum by hand.  For real perturbations
of the weights and nodes,
    du_k = 1/(i lz) sum_j e^{i phi_jk} [dw_j + i (2 pi / lz) w_j (x_j - xi_k) . dx_j],
phi_jk = pi |x_j - xi_k|^2 / lz.  With dL = Re sum_k c_k du_k,
c_k = -2 conj(u^oc_k) / K (K kept targets over all problems):
    dL/dw_j = Re S_j,  dL/dx_j = Re(i (2 pi / lz) w_j T_j),
    S_j = P_j / (i lz),  T_j = Q_j / (i lz),
where P, Q are the adjoint sums of oracle/direct.c with g = c.  A petal node
(k, i, l) has w = r_l what_l A_l omegahat_i and angle A_l t_i + 2 pi k / Np,
so dw/dA_l = r_l what_l omegahat_i and dx/dA_l = r_l t_i (-sin, cos)(angle);
the disc does not depend on A.  Finally dL/dtheta_m = sum_b sum_l
dL/dA_l B_m(r_l).
"""
import numpy as np

from . import direct
from . import quadrature as Q
from .field import grid_targets


def bspline_basis(a, R, n, r):
    """B_m(r) for the n clamped uniform cubic B-splines on [a, R] (rows: r)."""
    from scipy.interpolate import BSpline
    t = Q.bspline_knots(a, R, n)
    out = np.empty((len(r), n))
    for m in range(n):
        e = np.zeros(n)
        e[m] = 1.0
        out[:, m] = BSpline(t, e, 3)(r)
    return out


def _problem_family(prob, theta):
    fam = dict(prob["family"])
    fam["profile"] = {"kind": "bspline", "coefs": np.asarray(theta, dtype=np.float64)}
    return fam


def _targets(grid, keep):
    xi, eta = grid_targets(grid["n1"], grid["n2"], grid["h"], grid.get("x0", 0.0),
                           grid.get("y0", 0.0))
    return xi[keep], eta[keep]


def loss(theta, problems, grid, keep):
    """L(theta): problems = [{"family": petal family (profile ignored), "lam", "z"}],
    keep = boolean mask over the grid's targets (k1 fastest)."""
    xi, eta = _targets(grid, keep)
    tot, K = 0.0, 0
    for prob in problems:
        x, y, w = Q.family_nodes(_problem_family(prob, theta))
        lz = prob["lam"] * prob["z"]
        u = 1.0 - direct.direct_sum(x, y, w, xi, eta, lz)
        tot += np.sum(np.abs(u) ** 2)
        K += len(xi)
    return tot / K


def loss_and_grad(theta, problems, grid, keep):
    """(L, dL/dtheta) by the adjoint of the direct sum (see module docstring)."""
    theta = np.asarray(theta, dtype=np.float64)
    xi, eta = _targets(grid, keep)
    K = len(xi) * len(problems)
    L = 0.0
    grad = np.zeros_like(theta)
    for prob in problems:
        fam = _problem_family(prob, theta)
        x, y, w = Q.family_nodes(fam)
        lz = prob["lam"] * prob["z"]
        uoc = 1.0 - direct.direct_sum(x, y, w, xi, eta, lz)
        L += np.sum(np.abs(uoc) ** 2)
        c = -2.0 * np.conj(uoc) / K
        P, Qx, Qy = direct.adjoint_sums(x, y, xi, eta, lz, c)
        S, Tx, Ty = P / (1j * lz), Qx / (1j * lz), Qy / (1j * lz)
        dLdw = S.real
        dLdx = (1j * (2.0 * np.pi / lz) * w * Tx).real
        dLdy = (1j * (2.0 * np.pi / lz) * w * Ty).real
        # petal part of the node list (the disc comes first)
        Np, a, R = fam["n_petals"], fam["a"], fam["R"]
        m, n_p = fam["m"], fam["n_p"]
        n_disc = fam.get("n_d", 0) * fam.get("m_d", 0)
        r, wr = Q.gauss_legendre(m, a, R)
        t, wt = Q.gauss_legendre(n_p, -np.pi / Np, np.pi / Np)
        A = Q.petal_profile(fam["profile"], a, R, r)
        dLdA = np.zeros(m)
        for k in range(Np):
            sl = slice(n_disc + k * n_p * m, n_disc + (k + 1) * n_p * m)
            ang = (A[None, :] * t[:, None] + 2.0 * np.pi * k / Np)        # [i, l]
            dw_dA = wt[:, None] * (r * wr)[None, :]
            dx_dA = -r[None, :] * t[:, None] * np.sin(ang)
            dy_dA = r[None, :] * t[:, None] * np.cos(ang)
            gw = dLdw[sl].reshape(n_p, m)
            gx = dLdx[sl].reshape(n_p, m)
            gy = dLdy[sl].reshape(n_p, m)
            dLdA += np.sum(gw * dw_dA + gx * dx_dA + gy * dy_dA, axis=0)
        grad += bspline_basis(a, R, len(theta), r).T @ dLdA
    return L / K, grad


# ---------------------------------------------------------------- shape gradient (Fourier boundary)
def fourier_mode(kk, t):
    """dr/dp and dr'/dp at t for the coefficient p = params[kk] of
    r(t) = r0 + sum_k (a_k cos kt + b_k sin kt), params = [r0, a1, b1, ...]."""
    if kk == 0:
        return np.ones_like(t), np.zeros_like(t)
    k = (kk + 1) // 2
    if kk % 2 == 1:
        return np.cos(k * t), -k * np.sin(k * t)
    return np.sin(k * t), k * np.cos(k * t)


def shape_loss(params, fam, lam, z, xi, eta, output="aperture"):
    """L(params) = mean over targets of |u|^2 for a Fourier-boundary family
    whose radius r(t) = r0 + sum_k (a_k cos kt + b_k sin kt) has coefficients
    params = [r0, a1, b1, ...] (the dilation rule of eqs. aqnod/aqwei on the
    Gauss-Legendre panel line rule); u = u^ap, or u^oc = 1 - u^ap (eq. bab)."""
    f = dict(fam, params=np.asarray(params, dtype=np.float64))
    x, y, w = Q.family_nodes(f)
    u = direct.direct_sum(x, y, w, xi, eta, lam * z)
    if output == "occulter":
        u = 1.0 - u
    return float(np.mean(np.abs(u) ** 2))


def shape_loss_and_grad(params, fam, lam, z, xi, eta, output="aperture"):
    """(L, dL/dparams) for shape_loss by the adjoint of the direct sum.

    The node and weight derivatives dL/dx_j, dL/dy_j, dL/dw_j are those of the
    module docstring (adjoint sums of eq. faq with c_k = 2 s conj(u_k) / M,
    s = -1 for the occulter field).  They are chained through the dilation
    rule written out for boundary node i and radius l,
        x = c + alpha_l (X_i - c),  w = alpha_l wtilde_l ((X_i - cx) V_i - (Y_i - cy) W_i),
    and through the line rule X_i - cx = r(t_i) cos t_i, Y_i - cy = r(t_i) sin t_i,
    W_i = what_i (r' cos t_i - r sin t_i), V_i = what_i (r' sin t_i + r cos t_i),
    by the product rule with dr/dp and dr'/dp of each Fourier coefficient p."""
    params = np.asarray(params, dtype=np.float64)
    cx, cy = fam.get("cx", 0.0), fam.get("cy", 0.0)
    n_panels, p, m = fam["n_panels"], fam["p"], fam["m"]
    lz = lam * z
    f = dict(fam, params=params)
    x, y, w = Q.family_nodes(f)
    u = direct.direct_sum(x, y, w, xi, eta, lz)
    sgn = 1.0
    if output == "occulter":
        u = 1.0 - u
        sgn = -1.0
    M = len(xi)
    L = float(np.mean(np.abs(u) ** 2))
    c = sgn * 2.0 * np.conj(u) / M
    P, Qx, Qy = direct.adjoint_sums(x, y, xi, eta, lz, c)
    S, Tx, Ty = P / (1j * lz), Qx / (1j * lz), Qy / (1j * lz)
    gw = S.real.reshape(-1, m)
    gx = (1j * (2.0 * np.pi / lz) * w * Tx).real.reshape(-1, m)
    gy = (1j * (2.0 * np.pi / lz) * w * Ty).real.reshape(-1, m)
    # boundary rule and its pieces (same construction as quadrature.fourier_line_rule)
    tq, wq = Q.gauss_legendre(p, 0.0, 2.0 * np.pi / n_panels)
    t = (np.arange(n_panels)[:, None] * (2.0 * np.pi / n_panels) + tq[None, :]).ravel()
    what = np.tile(wq, n_panels)
    r, dr = Q.fourier_radius(params, t)
    ct, st = np.cos(t), np.sin(t)
    DX, DY = r * ct, r * st                                   # X - cx, Y - cy
    Wb, Vb = what * (dr * ct - r * st), what * (dr * st + r * ct)
    alpha, wt = Q.gauss_legendre(m, 0.0, 1.0)
    # per boundary node: sums over radii of the derivatives wrt X - cx, Y - cy and the cross
    gX = gx @ alpha                                           # dL/d(X - cx)
    gY = gy @ alpha
    gC = gw @ (alpha * wt)                                    # dL/d((X-cx) V - (Y-cy) W)
    grad = np.zeros_like(params)
    for kk in range(len(params)):
        phi, dphi = fourier_mode(kk, t)
        dDX, dDY = phi * ct, phi * st
        dW = what * (dphi * ct - phi * st)
        dV = what * (dphi * st + phi * ct)
        dC = dDX * Vb + DX * dV - dDY * Wb - DY * dW
        grad[kk] = np.sum(gX * dDX + gY * dDY + gC * dC)
    return L, grad
