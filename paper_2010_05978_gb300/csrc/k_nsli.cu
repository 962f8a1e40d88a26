// Non-singular line integral (arXiv:2010.05978, Appendix, eq. nsli): the
// aperture field from the boundary's vector line rule (X_i, Y_i, W_i, V_i)
// alone,
//   u^ap(xi) = 1/(2 pi) sum_i (1 - exp(i pi r_i^2 / lz)) / r_i^2 (rx_i V_i - ry_i W_i),
//   (rx, ry) = (X_i - xi, Y_i - eta),
// with the summand 0 where r = 0 (the cross product vanishes there).  An
// independent O(n M) FP64 evaluation used to check the areal path on the
// device; accurate up to the boundary itself.
//
// Option far > 0 (the Appendix's remark on shadows): a target whose nearest
// boundary node is at least far away takes the classical line integral
// eq. li instead,
//   u^ap = -1/(2 pi) sum_i e^{i pi r^2/lz} (r x ds)_i / r^2 + u_geom,
// with u_geom the winding number of eq. geom, 1/(2 pi) sum_i (r x ds)_i / r^2,
// rounded to an integer, and u^oc = (1 - u_geom) + 1/(2 pi) sum_i ... formed
// without subtracting from 1.
#include "internal.cuh"

namespace fres {

namespace {

constexpr int kNsliThreads = 256;

// One thread per target; the boundary nodes stream through shared memory in
// tiles of one node per thread.  bnd = (X, Y, W, V) absolute coordinates.
__global__ void __launch_bounds__(kNsliThreads)
k_nsli(const double4_32a* __restrict__ bnd, long long n, double lz, const double* __restrict__ targets,
       long long M, int occulter, double far2, double2* __restrict__ out) {
    __shared__ double4_32a tile[kNsliThreads];
    const double kq = kPi / lz;
    for (long long t0 = (long long)blockIdx.x * blockDim.x; t0 < M;
         t0 += (long long)gridDim.x * blockDim.x) {
        const long long t = t0 + threadIdx.x;
        const bool on = t < M;
        const double xi = on ? targets[2 * t] : 0.0, eta = on ? targets[2 * t + 1] : 0.0;
        double sr = 0.0, si = 0.0;            // eq. nsli sum
        double wsum = 0.0, br = 0.0, bi = 0.0;  // eq. geom and eq. li sums (far > 0)
        double r2min = INFINITY;
        for (long long i0 = 0; i0 < n; i0 += kNsliThreads) {
            __syncthreads();
            if (i0 + threadIdx.x < n) tile[threadIdx.x] = bnd[i0 + threadIdx.x];
            __syncthreads();
            const int cnt = (int)min((long long)kNsliThreads, n - i0);
            for (int i = 0; i < cnt; ++i) {
                const double4_32a b = tile[i];
                const double rx = b.x - xi, ry = b.y - eta;
                const double r2 = rx * rx + ry * ry;
                const double cr = rx * b.w - ry * b.z;
                if (r2 != 0.0) {
                    double s, c;
                    sincos(reduce_phase(kq * r2), &s, &c);
                    const double inv = cr / r2;
                    sr += (1.0 - c) * inv;
                    si -= s * inv;
                    if (far2 > 0.0) {
                        wsum += inv;
                        br += c * inv;
                        bi += s * inv;
                    }
                }
                r2min = fmin(r2min, r2);
            }
        }
        if (on) {
            double ur, ui;
            if (far2 > 0.0 && r2min >= far2) {   // eq. li with the exact winding number
                const double ug = rint(wsum / kTwoPi);
                ur = occulter ? (1.0 - ug) + br / kTwoPi : ug - br / kTwoPi;
                ui = occulter ? bi / kTwoPi : -bi / kTwoPi;
            } else {
                ur = sr / kTwoPi;
                ui = si / kTwoPi;
                if (occulter) {
                    ur = 1.0 - ur;
                    ui = -ui;
                }
            }
            out[t] = make_double2(ur, ui);
        }
    }
}

// (X, Y, W, V) of one family's boundary rule into the packed array.
__global__ void k_nsli_pack(FamilyDev f, double4_32a* __restrict__ dst) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= f.n_bdry) return;
    dst[i] = make_double4_32a(f.cx + f.bx[i], f.cy + f.by[i], f.bw[i], f.bv[i]);
}

}  // namespace

void launch_nsli(const FamilyDev* fams_host, int nfam, double lz, const double* targets,
                 long long M, int occulter, double far, double2* out, cudaStream_t st) {
    long long n = 0;
    for (int i = 0; i < nfam; ++i) n += fams_host[i].n_bdry;
    double4_32a* bnd = nullptr;
    if (cudaMallocAsync((void**)&bnd, sizeof(double4_32a) * (size_t)std::max(1LL, n), st) != cudaSuccess)
        return;
    long long off = 0;
    for (int i = 0; i < nfam; ++i) {
        const FamilyDev& f = fams_host[i];
        if (f.n_bdry > 0)
            k_nsli_pack<<<(int)((f.n_bdry + 255) / 256), 256, 0, st>>>(f, bnd + off);
        off += f.n_bdry;
    }
    if (M > 0) {
        const long long blocks = std::min<long long>((M + kNsliThreads - 1) / kNsliThreads, 152 * 8);
        k_nsli<<<(int)blocks, kNsliThreads, 0, st>>>(bnd, n, lz, targets, M, occulter, far * far,
                                                     out);
    }
    cudaFreeAsync(bnd, st);
}

}  // namespace fres
