"""Closed forms and brute force used to pin the oracle (test infrastructure only).

None of these share a formula with the areal-quadrature sum they check:
they come from the mathematics of eq. fres itself.
"""
import numpy as np
from scipy import integrate, special

from .quadrature import gauss_legendre


def disc_on_axis(R, lz):
    """u^ap at the centre of a disc of radius R.

    Appendix eq. dauger with R(theta) = R for every theta (a disc seen from its
    centre): u^ap = -(1/2pi) int_0^{2pi} (e^{i pi R^2/lz} - 1) dtheta
                  = 1 - e^{i pi R^2 / lz}.
    """
    return 1.0 - np.exp(1j * np.pi * R * R / lz)


def disc_off_axis(R, lz, rho, n_quad=4000):
    """u^ap at distance rho from the centre of a disc of radius R.

    Eq. fres in polar coordinates about the disc centre; the angular integral
    of e^{-2 pi i rho r cos(theta)/lz} is 2 pi J0(2 pi rho r / lz) (textbook
    Bessel integral), leaving the 1D Hankel-type integral
      u = (2 pi / (i lz)) e^{i pi rho^2/lz} int_0^R J0(2 pi rho r/lz) e^{i pi r^2/lz} r dr,
    done here by an n_quad-point Gauss-Legendre rule (scipy's J0).
    """
    rho = np.atleast_1d(np.asarray(rho, dtype=np.float64))
    r, wr = gauss_legendre(n_quad, 0.0, R)
    out = np.empty(rho.shape, dtype=np.complex128)
    for i, p in enumerate(rho):
        integrand = special.j0(2.0 * np.pi * p * r / lz) * np.exp(1j * np.pi * r * r / lz) * r
        out[i] = (2.0 * np.pi / (1j * lz)) * np.exp(1j * np.pi * p * p / lz) * np.sum(wr * integrand)
    return out


def fourier_star_area(params):
    """Area of r(theta) = r0 + sum_k (a_k cos k theta + b_k sin k theta).

    (1/2) int_0^{2pi} r^2 dtheta = pi (r0^2 + (1/2) sum_k (a_k^2 + b_k^2))  (Parseval).
    """
    params = np.asarray(params, dtype=np.float64)
    return np.pi * (params[0] ** 2 + 0.5 * np.sum(params[1:] ** 2))


def fourier_star_second_moment(params, n=4096):
    """int_Omega |x|^2 dA = (1/4) int_0^{2pi} r(theta)^4 dtheta, about the star centre.

    r^4 is a trigonometric polynomial of degree 4K, so the n-point periodic
    trapezoid rule is exact for n > 4K.
    """
    params = np.asarray(params, dtype=np.float64)
    K = (len(params) - 1) // 2
    assert n > 4 * K
    th = 2.0 * np.pi * np.arange(n) / n
    r = np.full_like(th, params[0])
    for k in range(1, K + 1):
        r += params[2 * k - 1] * np.cos(k * th) + params[2 * k] * np.sin(k * th)
    return 0.25 * (2.0 * np.pi / n) * np.sum(r ** 4)


def brute_force_star(params, lz, xi, eta, cx=0.0, cy=0.0, tol=1e-12):
    """Eq. fres by adaptive 2D integration over a Fourier star, polar about its centre.

    u = 1/(i lz) int_0^{2pi} int_0^{r(theta)} e^{i pi |xi - x|^2 / lz} r dr dtheta,
    real and imaginary parts by scipy.integrate.dblquad (adaptive Gauss-Kronrod).
    For tiny Fresnel numbers only: cost grows quickly with oscillation.
    """
    params = np.asarray(params, dtype=np.float64)
    K = (len(params) - 1) // 2

    def rmax(th):
        r = params[0]
        for k in range(1, K + 1):
            r += params[2 * k - 1] * np.cos(k * th) + params[2 * k] * np.sin(k * th)
        return r

    def phase(r, th):
        dx = xi - (cx + r * np.cos(th))
        dy = eta - (cy + r * np.sin(th))
        return np.pi * (dx * dx + dy * dy) / lz

    re, _ = integrate.dblquad(lambda r, th: np.cos(phase(r, th)) * r, 0.0, 2.0 * np.pi,
                              lambda th: 0.0, rmax, epsabs=tol, epsrel=tol)
    im, _ = integrate.dblquad(lambda r, th: np.sin(phase(r, th)) * r, 0.0, 2.0 * np.pi,
                              lambda th: 0.0, rmax, epsabs=tol, epsrel=tol)
    return (re + 1j * im) / (1j * lz)


def flower_area_moments(a, R, A):
    """Area and second moment of the starshade of eq. Omega (Sec. 4.2).

    At radius r the petals cover an angle N_p * 2 pi A(r) / N_p = 2 pi A(r),
    the disc the full 2 pi, so
        area = pi a^2 + 2 pi int_a^R A(r) r dr,
        int |x|^2 dA = pi a^4 / 2 + 2 pi int_a^R A(r) r^3 dr,
    the 1D integrals by adaptive Gauss-Kronrod (scipy quad).
    """
    opt = dict(epsabs=1e-14, epsrel=1e-14, limit=400)
    area = np.pi * a * a + 2.0 * np.pi * integrate.quad(lambda r: A(r) * r, a, R, **opt)[0]
    mom = 0.5 * np.pi * a ** 4 + 2.0 * np.pi * integrate.quad(lambda r: A(r) * r ** 3, a, R, **opt)[0]
    return area, mom


def flower_on_axis(a, R, A, lz):
    """u^ap at the centre of the starshade (eq. fres at xi = 0, polar coordinates).

    The angular integral at radius r gives 2 pi (disc) or 2 pi A(r) (petals), so
        u = 1 - e^{i pi a^2/lz} + (2 pi/(i lz)) int_a^R A(r) e^{i pi r^2/lz} r dr,
    the last integral by adaptive Gauss-Kronrod on its real and imaginary parts.
    """
    opt = dict(epsabs=1e-14, epsrel=1e-13, limit=2000)
    re = integrate.quad(lambda r: A(r) * np.cos(np.pi * r * r / lz) * r, a, R, **opt)[0]
    im = integrate.quad(lambda r: A(r) * np.sin(np.pi * r * r / lz) * r, a, R, **opt)[0]
    return 1.0 - np.exp(1j * np.pi * a * a / lz) + (2.0 * np.pi / (1j * lz)) * (re + 1j * im)


def brute_force_flower(n_petals, a, R, A, lz, xi, eta, tol=1e-11):
    """Eq. fres by adaptive 2D integration over the starshade of eq. Omega.

    Omega = {0 <= r <= R : P(N_p theta) in (-pi A(r), pi A(r))}, A = 1 on r < a:
    the disc r < a plus, for each k, the petal a < r < R,
    |theta - 2 pi k/N_p| < pi A(r)/N_p.  Each piece is integrated in polar
    coordinates (area element r dr dtheta) with scipy.integrate.dblquad.
    """
    def phase(r, th):
        dx = xi - r * np.cos(th)
        dy = eta - r * np.sin(th)
        return np.pi * (dx * dx + dy * dy) / lz

    def piece(r0, r1, lo, hi):
        re, _ = integrate.dblquad(lambda th, r: np.cos(phase(r, th)) * r, r0, r1, lo, hi,
                                  epsabs=tol, epsrel=tol)
        im, _ = integrate.dblquad(lambda th, r: np.sin(phase(r, th)) * r, r0, r1, lo, hi,
                                  epsabs=tol, epsrel=tol)
        return re + 1j * im

    total = piece(0.0, a, lambda r: 0.0, lambda r: 2.0 * np.pi)
    for k in range(n_petals):
        c = 2.0 * np.pi * k / n_petals
        total += piece(a, R, lambda r, c=c: c - np.pi * A(r) / n_petals,
                       lambda r, c=c: c + np.pi * A(r) / n_petals)
    return total / (1j * lz)
