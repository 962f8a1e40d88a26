// Internal declarations shared by the libfresnel translation units.
// Method: arXiv:2010.05978 (areal quadrature + NUFFT Fresnel diffraction).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/fresnel.h"

namespace fres {

constexpr int kMaxW = 16;          // widest spreading kernel supported
constexpr int kTile = 32;          // spreading tile edge (grid points)
constexpr int kMaxRadixStages = 32;
constexpr int kMaxCheb = 64;       // Chebyshev terms kept for psihat (type 3)
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double kPi = 3.141592653589793238462643383280;
constexpr double kTwoPiHi = 6.28318530717958623199592693709;    // fl(2 pi)
constexpr double kTwoPiLo = 2.44929359829470635445e-16;        // 2 pi - fl(2 pi)
constexpr double kInvTwoPi = 0.159154943091895335768883763373;

// Reduce an FP64 phase into [-pi, pi]: phi - 2 pi rint(phi / 2 pi), with 2 pi
// split into two doubles so the product n * 2 pi is carried to ~2^-106.
__device__ __forceinline__ double reduce_phase(double ph) {
    double n = rint(ph * kInvTwoPi);
    ph = fma(-n, kTwoPiHi, ph);
    return fma(-n, kTwoPiLo, ph);
}

// Device status word bits (read back by fresnel_check).
enum : unsigned {
    kStatusTargetOutside = 1u,     // a scattered target lay outside the plan's box
    kStatusNodeOutside = 2u,       // a node's support left the type-3 spreading grid
    kStatusNonFinite = 4u,         // a non-finite coordinate was met
    kStatusOverflow = 8u,          // a sort region was smaller than its records (batched plans)
    kStatusTimeout = 16u,          // a bounded device-side wait gave up (its work was skipped)
};

// Polls of a device-side wait before it gives up when fresnel_opts.max_spin = 0.
constexpr long long kDefaultMaxSpin = 1LL << 22;

template <typename T> struct Cx;
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<double> { using type = double2; };
template <typename T> using cx_t = typename Cx<T>::type;

// Node record after the chirp (Sec. 3.2 step 1) and the grid-coordinate
// split: first support cell s = floor(g - w/2) + 1 (wrapped into [0, nf) for
// type 1), fraction f = (g - w/2) - floor(g - w/2) in [0, 1), strength c.
template <typename T>
struct __align__(2 * sizeof(T) > 8 ? 16 : 8) NodeRec {
    int s1, s2;
    T f1, f2;
    T cre, cim;
};

// A spreading work item: nodes [begin, end) of the sorted record list that
// touch tile `tile`.  Tiles with more than the chunk cap of records are split
// into several consecutive chunks: the first clears the grid tile and raises
// the tile's ready flag, and every chunk adds its nonzero cells with global
// atomic adds (the others after waiting for the flag).  Unsplit tiles
// (including empty ones) are written with plain stores.  Chunks of split
// tiles come first in the list so the heaviest work starts first.
// split: 0 plain chunk; 1 padding (no records, does nothing); >= 2 a chunk
// of split tile number (split >> 1) - 1 (its ready flag), the tile's first
// chunk when split is odd.
struct Chunk {
    int tile;
    int begin, end;
    int split;
};
__host__ __device__ __forceinline__ int split_code(int split_index, bool first) {
    return ((split_index + 1) << 1) | (first ? 1 : 0);
}

// Radix plan of one FFT length.
struct FftPlan {
    int n;
    int nstages;
    int radix[kMaxRadixStages];
    // stage s: p = product of the earlier radices and ceil(2^32 / p), so that
    // i / p = umulhi(i, pmagic) exactly for i * p < 2^32 (p = 1: magic 0)
    int p[kMaxRadixStages];
    unsigned pmagic[kMaxRadixStages];
};

// One node family resident on the device.
struct FamilyDev {
    int kind;
    int n_panels, p, m;
    int K;                 // Fourier modes (kind FOURIER)
    int ptr;               // FOURIER on the periodic trapezoid rule (p = 1), t_q = 2 pi (q+1)/n_panels
    // PETALS (Sec. 4.2): bx, by, bc hold the first petal's u = r_l cos(A_l t_i),
    // v = r_l sin(A_l t_i), w = r_l what_l A_l omegahat_i at index i*m + l;
    // petal k is that petal rotated by rot[2k], rot[2k+1] = cos, sin(2 pi k/n_panels).
    int profile;
    long long n_prof;      // profile data values (at params + 5)
    double pa, pR;         // petal radii a < r < R
    double* rot;
    int prob;              // problem of a batched plan this family belongs to
    long long n_bdry;      // boundary nodes (PETALS: table entries p*m)
    long long n_nodes;     // areal nodes
    long long offset;      // first global node index
    double cx, cy;
    double* params;        // device copy of params
    double* bx;            // boundary X - cx   (n_bdry)
    double* by;            // boundary Y - cy
    double* bc;            // (X-cx) V - (Y-cy) W
    double* bw;            // the line rule's W, V (kept for the line integral, eq. nsli)
    double* bv;
    double* gl_p_t;        // p-point Gauss-Legendre nodes on (0,1)
    double* gl_p_w;
    double* gl_m_a;        // m-point Gauss-Legendre nodes alpha_l on (0,1)
    double* gl_m_aw;       // alpha_l * wtilde_l
    // FP32 fast mode (double-float "spoke" form of the dilation rule): with
    // x = c + alpha b_i the chirp phase is A0 + alpha (A1_i + alpha A2_i) and
    // the grid coordinate (minus w/2) is G0 + alpha G1_i per dimension.
    float* spoke;          // per boundary node: A1, A2, G1x, G1y as (hi, lo) pairs
    float* bcf;            // bc as FP32 (weights need only FP32)
    float* adf;            // alpha_l as (hi, lo)
    float* awf;            // alpha_l wtilde_l as FP32
    // FP32 fast mode, PETALS: per table entry (i, l) 8 floats: u, v, the
    // phase kq r_l^2 mod 2 pi (each hi, lo), the weight, a pad; per petal k
    // 18 floats: phase slopes P, Q and grid-coordinate slopes G1u, G1v, G2u,
    // G2v, then the petal's A0, G0x, G0y (each hi, lo), so that phase =
    // A0_k + R + u P + v Q and grid coordinate (minus w/2) = G0_k + u Gu + v Gv
    // (the constants differ between petals only when the petals are moved).
    float* ptab;
    float* pk;             // kPetalK floats per petal: the 12 slopes, then its A0, G0x, G0y
    double* shift;         // PETALS with a motion: per petal translation (tx, ty), else NULL
    float A0[2], G0x[2], G0y[2];
    // FP32 fast mode, TRIANGLES: per triangle 16 floats: v0 + c, v1 - v0 and
    // v2 - v1 (x, y of each as hi, lo) and (v1 - v0) x (v2 - v1) in FP32; per
    // family kq, -a1, -a2 (chirp) and U1, U2 (grid scale) as (hi, lo), with A0
    // = a0 and G0x, G0y the grid offsets minus w/2, so phase = kq |x|^2 -
    // a1 x - a2 y + a0 and grid coordinate (minus w/2) = U x + G0.
    float* tdf;
    float* wpf;            // the plain Gauss-Legendre weights what_i as FP32
    float tk[10];
};

constexpr int kPetalK = 18;   // floats per petal in FamilyDev::pk

// Everything a node kernel needs to turn (x, y, w) into a record.
struct ChirpParams {
    double kq;             // pi / lz
    double a1, a2, a0;     // phase = kq |x|^2 - a1 x - a2 y + a0 (pre-phase)
    int type3;
    // type 1: g = frac(x * u1) * nf1
    double u1, u2;
    // type 3: g = (x - C1) * inv_h1 + ng1 / 2
    double C1, C2, inv_h1, inv_h2;
    int nf1, nf2;          // spreading grid
    int w;
    int ntx, nty;          // tiles per dimension
    int tile_base;         // first tile of this problem in a batched plan (problem * ntx * nty)
    // type 1: the periodic grid is spread shifted by (sh1, sh2) cells (a node at
    // x~ = 0 lands mid-tile, so a cluster round the origin does not straddle
    // the wrap); the output tables undo it with exp(+2 pi i k sh / nf).
    int sh1, sh2;
    double screen_k;       // 2 pi / lambda of the problem (source screens)
};

// Piecewise-polynomial form of the spreading kernel: the value at
// cell a of a node with fractional offset f is a polynomial p_a(t) in
// t = 2 f - 1 (fitted once per plan on the Chebyshev points of each unit
// piece).  The kernel is even, so piece w - 1 - a is piece a mirrored:
// p_{w-1-a}(t) = p_a(-t).  Only the pieces a < ceil(w/2) are stored, split
// into even and odd parts in u = t^2: p_a(t) = E_a(u) + t O_a(u), giving the
// pair p_a, p_{w-1-a} = E_a -/+ ... from one evaluation of E_a and O_a.  Every
// piece is evaluated to the fixed degree kHornerDeg (the fit's own degree, at
// most kHornerDeg, zero-padded), so the fully unrolled Horner chains take
// their coefficients as constant operands.  deg < 0 means "evaluate exp/sqrt
// directly".  Passed by value, so it lives in the kernel-parameter constant
// bank (uniform access).  FP32 tables (HornerTab) go to degree 10, FP64
// tables (HornerTabD, the FP64 mode at any tolerance) to degree 14 (the
// fits level off at degree 9-14 for w <= 16: the end points' square roots).
constexpr int kHornerDeg = 10;
constexpr int kHornerEven = kHornerDeg / 2 + 1;        // t^0, t^2, ..., t^10
constexpr int kHornerOdd = (kHornerDeg + 1) / 2;       // t^1, t^3, ..., t^9
struct HornerTab {
    float e[(kMaxW + 1) / 2][kHornerEven];
    float o[(kMaxW + 1) / 2][kHornerOdd];
    int deg = -1;
};
constexpr int kHornerDegD = 14;
constexpr int kHornerEvenD = kHornerDegD / 2 + 1;      // t^0, t^2, ..., t^14
constexpr int kHornerOddD = (kHornerDegD + 1) / 2;     // t^1, t^3, ..., t^13
struct HornerTabD {
    double e[(kMaxW + 1) / 2][kHornerEvenD];
    double o[(kMaxW + 1) / 2][kHornerOddD];
    int deg = -1;
};
template <typename T> struct HornerFor { using type = HornerTab; };
template <> struct HornerFor<double> { using type = HornerTabD; };
template <typename T> using horner_t = typename HornerFor<T>::type;

struct KernelShape {
    int w;
    double beta;
    float betaf;
    HornerTab horner;
    HornerTabD hornerd;
};
template <typename T>
inline const horner_t<T>& horner_of(const KernelShape& ks) {
    if constexpr (sizeof(T) == 8) return ks.hornerd;
    else return ks.horner;
}

template <int W>
__device__ __forceinline__ void horner_eval(const HornerTab& h, float f, float* out) {
    const float t = 2.0f * f - 1.0f, u = t * t;
#pragma unroll
    for (int a = 0; a < (W + 1) / 2; ++a) {
        float E = h.e[a][kHornerEven - 1];
#pragma unroll
        for (int k = kHornerEven - 2; k >= 0; --k) E = fmaf(E, u, h.e[a][k]);
        float O = h.o[a][kHornerOdd - 1];
#pragma unroll
        for (int k = kHornerOdd - 2; k >= 0; --k) O = fmaf(O, u, h.o[a][k]);
        out[a] = fmaf(t, O, E);
        if (W - 1 - a != a) out[W - 1 - a] = fmaf(-t, O, E);
    }
}
template <int W>
__device__ __forceinline__ void horner_eval(const HornerTabD& h, double f, double* out) {
    const double t = 2.0 * f - 1.0, u = t * t;
#pragma unroll
    for (int a = 0; a < (W + 1) / 2; ++a) {
        double E = h.e[a][kHornerEvenD - 1];
#pragma unroll
        for (int k = kHornerEvenD - 2; k >= 0; --k) E = fma(E, u, h.e[a][k]);
        double O = h.o[a][kHornerOddD - 1];
#pragma unroll
        for (int k = kHornerOddD - 2; k >= 0; --k) O = fma(O, u, h.o[a][k]);
        out[a] = fma(t, O, E);
        if (W - 1 - a != a) out[W - 1 - a] = fma(-t, O, E);
    }
}

// Fourier transform of the exponential-of-semicircle spreading kernel
// psi(u) = exp(beta (sqrt(1 - (2u/w)^2) - 1)), |u| <= w/2 (grid points), at
// t radians per grid point:
//   psihat(t) = int psi(u) e^{-i t u} du = w int_0^1 psi(w s/2) cos(t w s/2) ds,
// evaluated by the q-point Gauss-Legendre rule (gq_t, gq_w) on (0, 1).
template <typename R>
__device__ __forceinline__ R kernel_ft(R t, int w, R beta, const R* gq_t, const R* gq_w, int q) {
    R acc = 0;
    R hw = (R)0.5 * (R)w;
    for (int i = 0; i < q; ++i) {
        R s = gq_t[i];
        acc += gq_w[i] * exp(beta * (sqrt((R)1 - s * s) - (R)1)) * cos(t * hw * s);
    }
    return (R)w * acc;
}

// The families of a plan for one node launch: family f owns blocks
// [blk0[f], blk0[f+1]); its problem's chirp parameters are cps[fams[f].prob].
// Source-plane screen (fresnel_opts.screen_*) on the device: n2 rows of n1
// samples in the plan's precision from (x0, y0) with spacings 1/ihx, 1/ihy;
// amp / opd NULL mean A = 1 / OPD = 0; n1 = 0: no screen.
struct ScreenDev {
    const void* amp = nullptr;
    const void* opd = nullptr;
    int n1 = 0, n2 = 0;
    double x0 = 0, y0 = 0, ihx = 0, ihy = 0;
};

struct FamTable {
    const FamilyDev* fams;
    const ChirpParams* cps;
    const int* blk0;
    int nfam;
    ScreenDev scr;
};
constexpr int kNodeThreads = 256;

// Per-problem regions of a batched plan's chunk list, split-tile list and
// sorted records (B + 1 entries each, absolute starts; sized at plan time).
// Chunk index space: every problem's split chunks first, then every
// problem's one-per-tile plain chunks.
// live (type 1 only, else NULL): per problem and tile row, 1 if any tile of
// the row holds records.  Tiles of dead rows get no chunk: the grid there is
// never written, and the FFT passes skip those rows (they are zero).
struct ScanLayout {
    const int* sc_off;
    const int* pl_off;
    const int* st_off;
    const long long* rec_off;
    int* live;
    int ntx, nty;
};
constexpr int kMaxTileRows = 256;   // nf2 <= 8192

// ------------------------------------------------------------------ launchers
// k_nodes.cu
void launch_gauss_legendre(int n, double* t01, double* w01, cudaStream_t st);
void launch_boundary(const FamilyDev& f, const ChirpParams& cp, cudaStream_t st);
// All families of a plan in one launch: records, tile counts (keys offset by
// each problem's tile_base) and, when dx != NULL, the FP64 nodes.
template <typename T>
void launch_nodes(const FamTable& ft, int nblocks, NodeRec<T>* rec, int* counts, double* dx,
                  double* dy, double* dw, unsigned* status, cudaStream_t st);
template <typename T>
void launch_scatter_fams(const FamTable& ft, int nblocks, const NodeRec<T>* rec, int* cursor,
                         NodeRec<T>* sorted, long long cap, unsigned* status, cudaStream_t st);
// One block per problem (B blocks): cursors, chunks and split tiles into the
// problem's regions of L; clears the counts.
void launch_scan_problems(int B, int ntiles, int* counts, int* cursor, Chunk* chunks,
                          int* split_tiles, const ScanLayout& L, int chunk_cap, unsigned* status,
                          cudaStream_t st);
// records + tile counts for points given by periodic grid coordinates (fresnel_spread)
void launch_records_from_coords(long long n, const double* g1, const double* g2, const float2* c,
                                const ChirpParams& cp, NodeRec<float>* rec, int* counts,
                                unsigned* status, cudaStream_t st);
// n_meta[0] = chunks, n_meta[1] = split tiles (listed in split_tiles)
void launch_scan_chunks(int ntiles, int* counts, int* cursor, Chunk* chunks, int* n_meta,
                        int* split_tiles, int chunk_cap, int max_chunks, int max_split,
                        cudaStream_t st);
template <typename T>
void launch_scatter(long long n, const ChirpParams& cp, const NodeRec<T>* rec, int* cursor,
                    NodeRec<T>* sorted, long long cap, unsigned* status, cudaStream_t st);
void launch_twiddles(int n, void* table, int is_double, cudaStream_t st);
// t1 output tables Ax[k1] = chirp(xi)/(i lz)/psihat(k1), Ay[k2] = chirp(eta)/psihat(k2),
// each times exp(2 pi i k shift / nf) for a grid spread shifted by shift cells
void launch_t1_tables(int n, int nf, double h, double x0, double lz, int w, double beta,
                      int with_ilz, int shift, void* table, int is_double, const double* gq_t,
                      const double* gq_w, int q, cudaStream_t st);
// t3 type-2 deconvolution factors 1/psihat(2 pi l / nfft), l in [-ng/2, ng/2)
void launch_t3_deconv(int ng, int nfft, int w, double beta, void* table, int is_double,
                      const double* gq_t, const double* gq_w, int q, cudaStream_t st);

// k_spread.cu
// work[0]: next chunk, work[1]: finished blocks (both return to 0 at exit);
// ready[0 .. max_split): the split tiles' ready flags (zero on entry, left
// zero); max_spin: polls of the ready wait (< 0: none).  Chunk tiles are
// global tile ids: problem = tile / ntiles (its grid is nf1 * nf2 cells
// after the previous problem's).
template <typename T>
void launch_spread(const NodeRec<T>* sorted, const Chunk* chunks, const int* n_meta,
                   int max_chunks, int* ready, int max_split, long long max_spin,
                   cx_t<T>* grid, int* work, unsigned* status, int nf1, int nf2, int ntx,
                   int ntiles, const KernelShape& ks, int nblocks, cudaStream_t st);
// Deterministic mode (fresnel_opts.deterministic): the same grid from exact
// fixed-point sums, bit for bit whatever the records' order within a tile
// and the split tiles' chunk order.  Three launches: the strengths' partial
// maxima into det_part[kDetPartials], the spreading pass, and the split
// tiles' conversion.  split_acc: max_split x 32 KB, zero on entry (left
// zero); tmax: records of the fullest tile (< kDetMaxTileRecords).
template <typename T>
void launch_spread_det(const NodeRec<T>* sorted, long long n_records, const Chunk* chunks,
                       const int* n_meta, int max_chunks, const int* split_tiles, int max_split,
                       unsigned long long* split_acc, double* det_part, int tmax, cx_t<T>* grid,
                       int* work, unsigned* status, int nf1, int nf2, int ntx, int ntiles,
                       const KernelShape& ks, cudaStream_t st);
constexpr int kDetPartials = 152 * 4;          // det_part entries
constexpr int kDetMaxTileRecords = 1 << 23;

// k_nsli.cu: non-singular line integral (Appendix, eq. nsli) over the
// boundary rules of the given families, FP64, one thread per target
void launch_nsli(const FamilyDev* fams_host, int nfam, double lz, const double* targets,
                 long long M, int occulter, double far, double2* out, cudaStream_t st);

// k_adjoint.cu (derivatives of type-1 plans with respect to petal profiles)
template <typename T>
void launch_adj_prologue(const void* gamma, const void* ax, const void* ay, void* out, int n1,
                         int n2, int B, int occulter, cudaStream_t st);
// mode 0: PETALS profiles (per-node dL/dA_l contributions); mode 1: Fourier
// boundary families (per-node dL/dr_i contributions)
template <typename T>
void launch_adj_nodes(const FamTable& ft, int nblocks, const void* bt, int nf1, int nf2,
                      const KernelShape& ks, double* contrib, int mode, cudaStream_t st);
void launch_adj_reduce(const FamilyDev* fams, const int* pf, const long long* gofs, int npf,
                       const double* contrib, double* grad, cudaStream_t st);
// Fourier families sf[0..nsf): dL/dr_i into rbuf (at bofs[f]), then dL/dp of
// each family's 1 + 2K coefficients into grad (at gofs[f])
void launch_adj_shape_reduce(const FamilyDev* fams, const int* sf, int nsf, int max_params,
                             long long n_bdry_total, const long long* bofs, const long long* gofs,
                             const double* contrib, double* rbuf, double* grad, cudaStream_t st);

// k_fft.cu
struct RowPassArgs {
    const void* in; void* out;
    long long in_stride, out_stride;   // elements between rows
    int nrows;
    int in_len;          // input elements per row
    int centered_in;     // 1: input index i holds mode i - in_len/2 (type 3 layout)
    const void* deconv_col;   // per-element factor along the row (centered_in), or NULL
    const void* deconv_row;   // per-row scalar factor (centered_in), or NULL
    int out_len;         // kept outputs: modes k in [-out_len/2, out_len - out_len/2), stored at k + out_len/2 (out_len == n: fftshifted)
    const void* twiddle;
    // rows of dead tile rows (live[(row / batch_rows) * nty + (row % batch_rows) / 32] == 0)
    // are skipped: neither read nor written.  NULL: every row is live.
    const int* live;
    int batch_rows, nty;
    // when not NULL: the nlist rows to transform (ascending), instead of
    // walking every row and skipping dead ones by their live flag
    const int* row_list;
    int nlist;
};
struct ColPassArgs {
    const void* in; void* out;
    int ncols;           // columns (contiguous dimension length of in/out)
    int in_len;          // input rows
    int centered_in;
    int out_len;         // kept output rows (centred as in RowPassArgs)
    const void* twiddle;
    // type-1 epilogue (final output) when ax != NULL: out[k2][k1] = F * ax[k1] * ay[k2], then Babinet
    const void* ax; const void* ay;
    int occulter;
    int out_is_final;    // 1: out has ncols columns of the final type (complex64/128)
    // batch of independent transforms: in/out of batch b start b * in_bstride /
    // out_bstride elements in; the epilogue tables of b at b * ncols / b * out_len
    int batch;
    long long in_bstride, out_bstride;
    // input row i of transform b is zero (not read) when live[b * nty + i / 32] == 0
    const int* live;
    int nty;
    // Four-step transforms of length fN = fa * fb beyond one shared-memory pass
    // (natural input index e = fb * a + b, output k = k1 + fa * k2):
    //  kFftRowStep1: A-point DFTs over a of every grid row o (nouter rows,
    //    in_stride apart; centred input with deconv as RowPassArgs), columns
    //    b < fb; output scratch[o * fN + k1 * fb + b];
    //  kFftColStep1: A-point DFTs over a down the grid columns (ncols), one
    //    outer index per b; output scratch[(k1 * fb + b) * ncols + c];
    //  kFftColStep2: B-point DFTs over b of scratch (outer index k1) with the
    //    twiddle w_N^(b k1); output row out_slot(k1 + fa * k2) (+ epilogue).
    //  kFftRowStep2: B-point DFTs of scratch rows (l, k1) (outer index l,
    //    "columns" k1 < fa, elements b at stride 1) with the twiddle
    //    w_N^(b k1); output grid row l at out_stride, slot out_slot(k1 + fa k2).
    int mode;
    int fa, fb, fN, nouter;
    long long in_stride, out_stride;
    const void* twN;
    const void* deconv_col;
    const void* deconv_row;
};
enum { kFftPlain = 0, kFftRowStep1 = 1, kFftColStep1 = 2, kFftColStep2 = 3, kFftRowStep2 = 4 };
template <typename T>
void launch_fft_rows(const FftPlan& fp, const RowPassArgs& a, cudaStream_t st);
template <typename T>
void launch_fft_cols(const FftPlan& fp, const ColPassArgs& a, cudaStream_t st);
// Type-1 column pass (kFftPlain layout with the output epilogue) as a direct
// DFT over the live rows only, for grids whose live band is a few tile rows:
// out[k][c] = sum_{r live} w_n^{k r} in[r][c] over the kept outputs k, with
// w_n^j from the n-point twiddle table.  Live rows beyond kDftMaxRows set
// kStatusOverflow.
constexpr int kDftMaxRows = 128;
template <typename T>
void launch_col_dft(const ColPassArgs& a, int n, unsigned* status, cudaStream_t st);
// k_col_dft_tc.cu: the same product (FP32 in and out) on the tensor cores,
// tcgen05 MMAs of kind::tf32 on split high / low TF32 operands, for plans whose
// problems have one live tile row (live_rows = 32)
bool col_dft_tc_supported(const ColPassArgs& a, int live_rows);
void launch_col_dft_tc(const ColPassArgs& a, int n, unsigned* status, cudaStream_t st);
// The same column pass for one live tile row (live_rows = 32) in FP64 as a
// pruned FFT: per output residue b modulo n / 32, a 32-point DFT of the live
// rows twiddled by w_n^{b j} (n a multiple of 32, at most 32768)
bool col_pfft_supported(int n, int live_rows);
void launch_col_pfft_d(const ColPassArgs& a, int n, unsigned* status, cudaStream_t st);
bool fft_supported(int n, int is_double, int* max_cols);
// Split of a length beyond one pass into fa * fb (both single-pass), or false.
bool fft_split(int n, int is_double, int* fa, int* fb);
FftPlan make_fft_plan(int n, int max_radix);

// k_interp.cu
struct InterpParams {
    double xi_c, eta_c;      // target box centre
    double K1, K2;           // tau = (xi - xi_c) * K  (grid units of the FFT grid)
    double sh1, sh2;         // s' h = (xi - xi_c) * sh  (argument of the kernel transform)
    double kq;               // pi / lz
    double p1, p2;           // post-phase: -2 pi C / lz
    double inv_lz;
    double inv_tmax;         // 1 / t_max of the Chebyshev series of psihat
    // FP32 fast mode, double-float (hi, lo) constants:
    //   g = xi K + G  (grid coordinate minus w/2), phase = xi (kq xi + p1) + eta (kq eta + p2)
    float dK1[2], dK2[2], dG1[2], dG2[2], dkq[2], dp1[2], dp2[2];
    float boxf[4];
    float shK1, shK2;        // (g + w/2) * shK = argument of psihat
    int nbin1, nbin2;        // kTargetBin x kTargetBin target bins per dimension of the FFT grid
    double box[4];
    int nfft1, nfft2;
    int occulter;
};
// Buffers of the binned FP32 type-3 interpolation: per-bin counts (zero on
// entry, left zero), bin starts, scatter cursors, the target permutation
// (>= M entries) and the dynamic bin counter (2 ints, zero, left zero).
struct T3Sort {
    int* counts;
    int* start;
    int* cursor;
    int* perm;
    int* work;
    int* partial;   // per 4096-bin chunk sums (bin counts too many to scan in one block)
};
constexpr int kTargetBin = 16;          // edge of a target bin (cells of the FFT grid)
constexpr int kBinScanStaged = 40000;   // bins scanned by one block in shared memory
constexpr int kBinChunk = 4096;         // bins per block of the multi-block scan
// FP32 binned path, step 1: bucket the targets by bin (count, scan, scatter
// into sort->perm; three or five launches).  w must satisfy
// interp_binned_width.
void launch_target_sort(const double* targets, long long M, const InterpParams& ip, int w,
                        const T3Sort* sort, cudaStream_t st);
// sort == NULL (or FP64, or a width without a binned kernel): one thread per
// target straight from global memory.  Otherwise the binned interpolation
// from sort->perm, which launch_target_sort has filled on the same stream.
template <typename T>
void launch_interp_w(const double* targets, long long M, const cx_t<T>* F, const InterpParams& ip,
                     const KernelShape& ks, const double* cheb, int ncheb,
                     void* out, unsigned* status, const T3Sort* sort, cudaStream_t st);
bool interp_binned_width(int w);
// psihat at the n even-half Chebyshev points of [-t_max, t_max] (plan time)
void launch_cheb_samples(int n, double tmax, int w, double beta, const double* gq_t,
                         const double* gq_w, int q, double* out, cudaStream_t st);

}  // namespace fres

// Thread-local error message + status helpers (api.cu).
fresnel_status fres_fail(fresnel_status s, const std::string& msg);
