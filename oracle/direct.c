/*
 * Oracle O(NM) sums, plain FP64 C with OpenMP over targets.
 * TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the
 * CPU-baseline legs of bench.py; never linked into the CUDA library.
 *
 * Built with -O2 -ffp-contract=off so the arithmetic is exactly what is
 * written here.  Each target is summed by one thread in a fixed order
 * (blocks of ORACLE_BLOCK terms, block sums added in order), so the result
 * does not depend on the thread count.
 */
#include <math.h>
#include <stddef.h>

#define ORACLE_BLOCK 512

/*
 * Direct areal-quadrature sum, eq. faq (Sec. 3.1, first line, unsplit form):
 *   u_k = 1/(i lz) * sum_j w_j exp(i pi [(xi_k - x_j)^2 + (eta_k - y_j)^2] / lz)
 * with lz = lambda * z.  1/(i lz) = -i/lz, so
 *   Re u = (1/lz) sum w sin(phi),  Im u = -(1/lz) sum w cos(phi).
 */
void oracle_direct(long long n_nodes, const double* x, const double* y, const double* w,
                   long long n_targets, const double* xi, const double* eta, double lz,
                   double* u_re, double* u_im)
{
    const double k = M_PI / lz;
#pragma omp parallel for schedule(dynamic, 4)
    for (long long t = 0; t < n_targets; ++t) {
        double sc = 0.0, ss = 0.0;               /* sum w cos, sum w sin */
        for (long long j0 = 0; j0 < n_nodes; j0 += ORACLE_BLOCK) {
            long long j1 = j0 + ORACLE_BLOCK < n_nodes ? j0 + ORACLE_BLOCK : n_nodes;
            double bc = 0.0, bs = 0.0;
            for (long long j = j0; j < j1; ++j) {
                double dx = xi[t] - x[j];
                double dy = eta[t] - y[j];
                double phi = k * (dx * dx + dy * dy);
                bc += w[j] * cos(phi);
                bs += w[j] * sin(phi);
            }
            sc += bc;
            ss += bs;
        }
        u_re[t] = ss / lz;
        u_im[t] = -sc / lz;
    }
}

/*
 * Non-singular line integral (NSLI), Appendix eq. nsli:
 *   u^ap = 1/(2 pi) * sum_i (1 - exp(i pi r^2 / lz)) / r^2 * (rx V_i - ry W_i)
 * with (rx, ry) = (X_i - xi, Y_i - eta) and (W_i, V_i) the vector line weights
 * of eq. vliq; the factor is set to 0 where r^2 == 0 (any finite value is
 * allowed there because the cross product vanishes).
 */
void oracle_nsli(long long n_bdry, const double* X, const double* Y, const double* W,
                 const double* V, long long n_targets, const double* xi, const double* eta,
                 double lz, double* u_re, double* u_im)
{
    const double k = M_PI / lz;
#pragma omp parallel for schedule(dynamic, 4)
    for (long long t = 0; t < n_targets; ++t) {
        double sr = 0.0, si = 0.0;
        for (long long i0 = 0; i0 < n_bdry; i0 += ORACLE_BLOCK) {
            long long i1 = i0 + ORACLE_BLOCK < n_bdry ? i0 + ORACLE_BLOCK : n_bdry;
            double br = 0.0, bi = 0.0;
            for (long long i = i0; i < i1; ++i) {
                double rx = X[i] - xi[t];
                double ry = Y[i] - eta[t];
                double r2 = rx * rx + ry * ry;
                double cr = rx * V[i] - ry * W[i];
                double fr = 0.0, fi = 0.0;
                if (r2 != 0.0) {
                    fr = (1.0 - cos(k * r2)) / r2;
                    fi = -sin(k * r2) / r2;
                }
                br += fr * cr;
                bi += fi * cr;
            }
            sr += br;
            si += bi;
        }
        u_re[t] = sr / (2.0 * M_PI);
        u_im[t] = si / (2.0 * M_PI);
    }
}

/*
 * Exact 2D type-3 exponential sum of eq. nufft3 (the middle step of the
 * split form, eq. split):
 *   v_k = sum_j c_j exp(-2 pi i (xi_k x_j + eta_k y_j) / lz)
 * Used to check the NUFFT stage on its own.
 */
void oracle_sum3(long long n_nodes, const double* x, const double* y, const double* c_re,
                 const double* c_im, long long n_targets, const double* xi, const double* eta,
                 double lz, double* v_re, double* v_im)
{
    const double k = 2.0 * M_PI / lz;
#pragma omp parallel for schedule(dynamic, 4)
    for (long long t = 0; t < n_targets; ++t) {
        double sr = 0.0, si = 0.0;
        for (long long j0 = 0; j0 < n_nodes; j0 += ORACLE_BLOCK) {
            long long j1 = j0 + ORACLE_BLOCK < n_nodes ? j0 + ORACLE_BLOCK : n_nodes;
            double br = 0.0, bi = 0.0;
            for (long long j = j0; j < j1; ++j) {
                double phi = -k * (xi[t] * x[j] + eta[t] * y[j]);
                double cs = cos(phi), sn = sin(phi);
                br += c_re[j] * cs - c_im[j] * sn;
                bi += c_re[j] * sn + c_im[j] * cs;
            }
            sr += br;
            si += bi;
        }
        v_re[t] = sr;
        v_im[t] = si;
    }
}

/*
 * Adjoint sums for the gradient of a real loss of the field (derivative of
 * eq. faq with respect to the nodes and weights): for node j and complex
 * target coefficients g_k,
 *   P_j  = sum_k g_k exp(i phi_jk),
 *   Qx_j = sum_k g_k exp(i phi_jk) (x_j - xi_k),  Qy_j likewise with y, eta,
 * phi_jk = pi [(xi_k - x_j)^2 + (eta_k - y_j)^2] / lz.  One thread per node,
 * fixed-order blocked sums over targets.
 */
void oracle_adjoint(long long n_nodes, const double* x, const double* y, long long n_targets,
                    const double* xi, const double* eta, double lz, const double* g_re,
                    const double* g_im, double* P, double* Qx, double* Qy)
{
    const double k = M_PI / lz;
#pragma omp parallel for schedule(dynamic, 4)
    for (long long j = 0; j < n_nodes; ++j) {
        double acc[6] = {0, 0, 0, 0, 0, 0};   /* P re/im, Qx re/im, Qy re/im */
        for (long long t0 = 0; t0 < n_targets; t0 += ORACLE_BLOCK) {
            long long t1 = t0 + ORACLE_BLOCK < n_targets ? t0 + ORACLE_BLOCK : n_targets;
            double b[6] = {0, 0, 0, 0, 0, 0};
            for (long long t = t0; t < t1; ++t) {
                double dx = x[j] - xi[t];
                double dy = y[j] - eta[t];
                double phi = k * (dx * dx + dy * dy);
                double c = cos(phi), s = sin(phi);
                double er = g_re[t] * c - g_im[t] * s;   /* g exp(i phi) */
                double ei = g_re[t] * s + g_im[t] * c;
                b[0] += er;
                b[1] += ei;
                b[2] += er * dx;
                b[3] += ei * dx;
                b[4] += er * dy;
                b[5] += ei * dy;
            }
            for (int q = 0; q < 6; ++q) acc[q] += b[q];
        }
        P[2 * j] = acc[0];
        P[2 * j + 1] = acc[1];
        Qx[2 * j] = acc[2];
        Qx[2 * j + 1] = acc[3];
        Qy[2 * j] = acc[4];
        Qy[2 * j + 1] = acc[5];
    }
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
