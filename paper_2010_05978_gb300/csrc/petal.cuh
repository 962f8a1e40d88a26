// Petal apodisation profiles of the starshade rule (arXiv:2010.05978,
// Sec. 4.2, eq. Omega): petal angular width 2 pi A(r) / N_p on a < r < R.
// A(r) and its derivatives with respect to the profile parameters
// (params[5...] of a FRESNEL_FAMILY_PETALS family).
#pragma once
#include "internal.cuh"

namespace fres {

// Knot t_i of the clamped uniform cubic B-spline with n coefficients on [a, R]:
// a for i <= 3, R for i >= n, a + (i - 3) (R - a) / (n - 3) in between.
__device__ __forceinline__ double bspline_knot(int i, int n, double a, double R) {
    return i <= 3 ? a : (i >= n ? R : a + (i - 3) * ((R - a) / (n - 3)));
}

// Span mu (t_mu <= r < t_mu+1, 3 <= mu <= n - 1) and the four nonzero cubic
// basis values B_{mu-3..mu}(r) (Cox-de Boor recursion, triangular form).
__device__ __forceinline__ int bspline_basis4(double r, int n, double a, double R, double N[4]) {
    const double step = (R - a) / (n - 3);
    int mu = 3 + (int)floor((r - a) / step);
    mu = min(max(mu, 3), n - 1);
    double left[4], right[4];
    N[0] = 1.0;
    for (int j = 1; j <= 3; ++j) {
        left[j] = r - bspline_knot(mu + 1 - j, n, a, R);
        right[j] = bspline_knot(mu + j, n, a, R) - r;
        double saved = 0.0;
        for (int q = 0; q < j; ++q) {
            const double tmp = N[q] / (right[q + 1] + left[j - q]);
            N[q] = saved + right[q + 1] * tmp;
            saved = left[j - q] * tmp;
        }
        N[j] = saved;
    }
    return mu;
}

// A(r_l) at radius r (l: index of r among the family's m Gauss radii).
__device__ __forceinline__ double petal_profile(const FamilyDev& f, int l, double r) {
    const double* d = f.params + 5;
    if (f.profile == FRESNEL_PETAL_HG) return exp(-pow((r - f.pa) / d[0], d[1]));
    if (f.profile == FRESNEL_PETAL_TABLE) return d[l];
    double N[4];
    const int mu = bspline_basis4(r, (int)f.n_prof, f.pa, f.pR, N);
    return N[0] * d[mu - 3] + N[1] * d[mu - 2] + N[2] * d[mu - 1] + N[3] * d[mu];
}

// dA(r_l)/dparam for the (at most four) parameters A depends on: returns the
// count and fills idx (offsets into params[5...]) and val.
__device__ __forceinline__ int petal_profile_grad(const FamilyDev& f, int l, double r, int idx[4],
                                                  double val[4]) {
    const double* d = f.params + 5;
    if (f.profile == FRESNEL_PETAL_HG) {   // A = exp(-s^q), s = (r - a) / b
        const double s = (r - f.pa) / d[0], sq = pow(s, d[1]), A = exp(-sq);
        idx[0] = 0;
        val[0] = A * d[1] * sq / d[0];                  // dA/db
        idx[1] = 1;
        val[1] = s > 0.0 ? -A * sq * log(s) : 0.0;      // dA/dq
        return 2;
    }
    if (f.profile == FRESNEL_PETAL_TABLE) {
        idx[0] = l;
        val[0] = 1.0;
        return 1;
    }
    const int mu = bspline_basis4(r, (int)f.n_prof, f.pa, f.pR, val);
    for (int q = 0; q < 4; ++q) idx[q] = mu - 3 + q;
    return 4;
}

}  // namespace fres
