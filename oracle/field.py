"""The oracle's whole field, eqs. fres/faq and bab (test infrastructure only)."""
import numpy as np

from . import quadrature
from . import direct


def nodes(families):
    """Concatenated areal rule (x, y, w) over a list of panel families (eq. aq)."""
    parts = [quadrature.family_nodes(f) for f in families]
    return tuple(np.concatenate([p[k] for p in parts]) for k in range(3))


def field(families, lam, z, xi, eta, output="aperture"):
    """u at targets (xi_k, eta_k) by the direct sum of eq. faq over the oracle's own nodes.

    output="aperture" gives u^ap (eq. fres with 1/(i lambda z) normalisation,
    plane-wave phase e^{2 pi i z/lambda} dropped as in Sec. 2);
    output="occulter" gives u^oc = 1 - u^ap (Babinet, eq. bab).
    """
    x, y, w = nodes(families)
    u = direct.direct_sum(x, y, w, np.asarray(xi, float), np.asarray(eta, float), lam * z)
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
