"""The oracle's whole field, eqs. fres/faq and bab (test infrastructure only)."""
import numpy as np

from . import quadrature
from . import direct


def nodes(families):
    """Concatenated areal rule (x, y, w) over a list of panel families (eq. aq)."""
    parts = [quadrature.family_nodes(f) for f in families]
    return tuple(np.concatenate([p[k] for p in parts]) for k in range(3))


def keys_kernel(s):
    """Cubic convolution kernel with a = -1/2 (Catmull-Rom):
    K(s) = 3/2 |s|^3 - 5/2 |s|^2 + 1 on |s| <= 1, -1/2 |s|^3 + 5/2 |s|^2 - 4 |s| + 2
    on 1 < |s| < 2, 0 beyond; interpolation with it reproduces polynomials of
    degree <= 2."""
    s = np.abs(s)
    return np.where(s <= 1.0, 1.5 * s ** 3 - 2.5 * s ** 2 + 1.0,
                    np.where(s < 2.0, -0.5 * s ** 3 + 2.5 * s ** 2 - 4.0 * s + 2.0, 0.0))


def screen_value(screen, lam, x, y):
    """Source term s = A exp(2 pi i OPD / lam) at (x, y) (Sec. 5: multiply w_j by
    the source term at each areal node): A and OPD sampled on the uniform grid
    of screen["box"] = (x0, x1, y0, y1) (arrays of n2 rows of n1 samples; a
    missing one is 1 / 0), interpolated by the cubic convolution kernel over
    the 4 x 4 nearest samples, with the stencil kept inside the samples (the
    coordinate clamped to [1, n - 2] sample spacings)."""
    x0, x1, y0, y1 = screen["box"]
    arrs = [screen.get(k) for k in ("amp", "opd")]
    n2, n1 = next(np.shape(a) for a in arrs if a is not None)
    u = np.clip((np.asarray(x, float) - x0) * (n1 - 1) / (x1 - x0), 1.0, n1 - 2.0)
    v = np.clip((np.asarray(y, float) - y0) * (n2 - 1) / (y1 - y0), 1.0, n2 - 2.0)
    i1 = np.minimum(np.floor(u).astype(int), n1 - 3)
    i2 = np.minimum(np.floor(v).astype(int), n2 - 3)

    def interp(a):
        a = np.asarray(a, float)
        tot = np.zeros(len(u))
        for db in (-1, 0, 1, 2):
            for da in (-1, 0, 1, 2):
                tot += keys_kernel(v - (i2 + db)) * keys_kernel(u - (i1 + da)) * a[i2 + db, i1 + da]
        return tot

    A = interp(arrs[0]) if arrs[0] is not None else 1.0
    opd = interp(arrs[1]) if arrs[1] is not None else 0.0
    return A * np.exp(2j * np.pi * opd / lam)


def field(families, lam, z, xi, eta, output="aperture", screen=None):
    """u at targets (xi_k, eta_k) by the direct sum of eq. faq over the oracle's own nodes.

    output="aperture" gives u^ap (eq. fres with 1/(i lambda z) normalisation,
    plane-wave phase e^{2 pi i z/lambda} dropped as in Sec. 2);
    output="occulter" gives u^oc = 1 - u^ap (Babinet, eq. bab).  screen: a
    source term (see screen_value) multiplying each node's weight; the sum is
    linear in the weights, so its real and imaginary parts are summed apart.
    """
    x, y, w = nodes(families)
    xi, eta = np.asarray(xi, float), np.asarray(eta, float)
    if screen is None:
        u = direct.direct_sum(x, y, w, xi, eta, lam * z)
    else:
        ws = w * screen_value(screen, lam, x, y)
        u = (direct.direct_sum(x, y, ws.real, xi, eta, lam * z)
             + 1j * direct.direct_sum(x, y, ws.imag, xi, eta, lam * z))
    if output == "occulter":
        return 1.0 - u
    if output != "aperture":
        raise ValueError(output)
    return u


def grid_targets(n1, n2, h, x0=0.0, y0=0.0):
    """Targets of Sec. 3.3's grid: (x0 + k1 h, y0 + k2 h), -n/2 <= k < n/2, k1 fastest."""
    k1 = np.arange(-(n1 // 2), n1 - n1 // 2)
    k2 = np.arange(-(n2 // 2), n2 - n2 // 2)
    XI, ETA = np.meshgrid(x0 + h * k1, y0 + h * k2, indexing="xy")
    return XI.ravel(), ETA.ravel()
