"""ctypes wrappers around oracle/direct.c (test infrastructure only)."""
import ctypes
import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        d = ctypes.POINTER(ctypes.c_double)
        ll = ctypes.c_longlong
        _lib.oracle_direct.argtypes = [ll, d, d, d, ll, d, d, ctypes.c_double, d, d]
        _lib.oracle_nsli.argtypes = [ll, d, d, d, d, ll, d, d, ctypes.c_double, d, d]
        _lib.oracle_sum3.argtypes = [ll, d, d, d, d, ll, d, d, ctypes.c_double, d, d]
        _lib.oracle_adjoint.argtypes = [ll, d, d, ll, d, d, ctypes.c_double, d, d, d, d, d]
        _lib.oracle_max_threads.restype = ctypes.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def max_threads():
    """Number of OpenMP threads the oracle sums use."""
    return _load().oracle_max_threads()


def direct_sum(x, y, w, xi, eta, lz):
    """Eq. faq, unsplit: u_k = 1/(i lz) sum_j w_j exp(i pi |xi_k - x_j|^2 / lz)."""
    lib = _load()
    x, y, w, xi, eta = map(_c, (x, y, w, xi, eta))
    re = np.empty(len(xi))
    im = np.empty(len(xi))
    lib.oracle_direct(len(x), _p(x), _p(y), _p(w), len(xi), _p(xi), _p(eta), float(lz),
                      _p(re), _p(im))
    return re + 1j * im


def nsli(X, Y, W, V, xi, eta, lz):
    """Appendix eq. nsli: u^ap = 1/(2pi) sum_i (1 - e^{i pi r^2/lz}) / r^2 (r x ds)_i."""
    lib = _load()
    X, Y, W, V, xi, eta = map(_c, (X, Y, W, V, xi, eta))
    re = np.empty(len(xi))
    im = np.empty(len(xi))
    lib.oracle_nsli(len(X), _p(X), _p(Y), _p(W), _p(V), len(xi), _p(xi), _p(eta), float(lz),
                    _p(re), _p(im))
    return re + 1j * im


def line_integral_far(X, Y, W, V, xi, eta, lz, far):
    """Appendix remark r:shadfix: targets whose nearest boundary node is at
    least `far` away use the classical line integral eq. li,
        u^ap = -1/(2 pi) sum_i e^{i pi r^2/lz} (r x ds)_i / r^2 + u_geom,
    with u_geom the winding number of eq. geom, (1/(2 pi)) sum_i (r x ds)_i / r^2,
    rounded to an integer; the others use eq. nsli.  Returns (u^ap, u^oc),
    u^oc = (1 - u_geom) + 1/(2 pi) sum_i e^{i pi r^2/lz} (r x ds)_i / r^2 for
    far targets (no cancellation against 1 in a shadow) and 1 - u^ap
    otherwise.  Plain numpy, in chunks of targets.
    """
    X, Y, W, V = (np.asarray(a, float) for a in (X, Y, W, V))
    xi, eta = np.atleast_1d(np.asarray(xi, float)), np.atleast_1d(np.asarray(eta, float))
    uap = nsli(X, Y, W, V, xi, eta, lz)
    uoc = 1.0 - uap
    for s in range(0, len(xi), 256):
        rx = X[None, :] - xi[s:s + 256, None]
        ry = Y[None, :] - eta[s:s + 256, None]
        r2 = rx * rx + ry * ry
        cr = rx * V[None, :] - ry * W[None, :]
        far_k = r2.min(axis=1) >= far * far
        if far > 0 and np.any(far_k):
            k = np.nonzero(far_k)[0]
            inv = cr[k] / r2[k]
            ug = np.rint(inv.sum(axis=1) / (2.0 * np.pi))
            B = (np.exp(1j * np.pi * r2[k] / lz) * inv).sum(axis=1) / (2.0 * np.pi)
            uap[s + k] = ug - B
            uoc[s + k] = (1.0 - ug) + B
    return uap, uoc


def sum3(x, y, c, xi, eta, lz):
    """Eq. nufft3 evaluated exactly: v_k = sum_j c_j exp(-2 pi i (xi_k x_j + eta_k y_j)/lz)."""
    lib = _load()
    x, y, xi, eta = map(_c, (x, y, xi, eta))
    c = np.asarray(c, dtype=np.complex128)
    cr, ci = _c(c.real), _c(c.imag)
    re = np.empty(len(xi))
    im = np.empty(len(xi))
    lib.oracle_sum3(len(x), _p(x), _p(y), _p(cr), _p(ci), len(xi), _p(xi), _p(eta), float(lz),
                    _p(re), _p(im))
    return re + 1j * im


def adjoint_sums(x, y, xi, eta, lz, g):
    """P_j = sum_k g_k e^{i phi_jk} and Q_j = sum_k g_k e^{i phi_jk} (x_j - xi_k) (2-vector)."""
    lib = _load()
    x, y, xi, eta = map(_c, (x, y, xi, eta))
    g = np.asarray(g, dtype=np.complex128)
    gr, gi = _c(g.real), _c(g.imag)
    P = np.empty(2 * len(x))
    Qx = np.empty(2 * len(x))
    Qy = np.empty(2 * len(x))
    lib.oracle_adjoint(len(x), _p(x), _p(y), len(xi), _p(xi), _p(eta), float(lz), _p(gr), _p(gi),
                       _p(P), _p(Qx), _p(Qy))
    v = lambda a: a[0::2] + 1j * a[1::2]
    return v(P), v(Qx), v(Qy)
