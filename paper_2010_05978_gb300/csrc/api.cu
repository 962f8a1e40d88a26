// C ABI and plan runtime of libfresnel (declared in include/fresnel.h).
//
// A plan fixes the aperture (its panel families), lambda*z, the targets'
// layout (uniform grid: type-1 NUFFT, Sec. 3.3; scattered targets in a box:
// type-3 NUFFT, Sec. 3.2 of arXiv:2010.05978) and the tolerance, chooses the
// spreading kernel and grids, allocates every device buffer once, and builds
// the plan-time tables.  fresnel_eval then only launches kernels on the
// plan's stream:
//   nodes+chirp+count -> scan -> scatter   (skipped when nodes are cached)
//   spread -> FFT rows -> FFT columns (+ fused type-1 epilogue)
//   [type 3: -> interpolation + deconvolution + post-phase/chirp]
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "dfloat.cuh"
#include "internal.cuh"

using namespace fres;

static thread_local std::string g_last_error;

fresnel_status fres_fail(fresnel_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

#define FRES_CK(call)                                                                        \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fres_fail(e_ == cudaErrorMemoryAllocation ? FRESNEL_ERR_OOM               \
                                                             : FRESNEL_ERR_CUDA,             \
                             std::string(#call) + ": " + cudaGetErrorString(e_));            \
    } while (0)

namespace {

constexpr uint64_t kMagic = 0x46524553'4e454c31ull;   // "FRESNEL1"
constexpr int kMaxEvents = 16;
// FP32 type-3 target binning (kTargetBin x kTargetBin blocks of the FFT grid, interpolation
// from shared-memory patches) is chosen automatically only when the FFT grid
// would not stay in L2 and the target set is large.  Measured on the
// F = 100 star workload (29 MB grid, 1e6 targets): binned 0.18 ms against
// 0.126 ms for direct gathers from L2, so small grids gather directly.
constexpr long long kSortTargetsFrom = 32768;
constexpr long long kBinFromGridBytes = 64LL << 20;

// FFT along one dimension: one shared-memory pass, or four steps fa x fb
// (A-point transforms, twiddle, B-point transforms) for longer lengths.
struct FftDim {
    int n = 0;
    bool big = false;
    int fa = 0, fb = 0;
    FftPlan fp{}, fpa{}, fpb{};
    void* tw = nullptr;            // w_n table (for a four-step length, the w_N twiddles)
    void* twa = nullptr;
    void* twb = nullptr;
};

struct Plan {
    uint64_t magic = kMagic;
    int prec = FRESNEL_FP32_FAST, output = 0, tkind = 0;
    double lz = 0, tol = 0;       // lz: the first problem's lambda * z
    cudaStream_t st = nullptr;
    fresnel_opts opts{};
    int B = 1;                    // independent problems (fresnel_plan_many)
    std::vector<double> lzs;      // lambda * z per problem
    std::vector<ChirpParams> cps; // chirp / grid parameters per problem
    std::vector<FamilyDev> fams;
    long long N = 0;
    FamTable ft{};                // device copies of fams, cps and the block starts
    int node_blocks = 0;
    ScanLayout layout{};          // per-problem sort regions (device)
    KernelShape ks{};
    double sigma = 2.0;
    int nf1 = 0, nf2 = 0, nfft1 = 0, nfft2 = 0;
    int n1 = 0, n2 = 0;
    int ntx = 0, nty = 0, ntiles = 0;
    int chunk_cap = 0, max_chunks = 0, max_split = 0;
    int* ready = nullptr;         // split tiles' ready flags (zero between evaluations)
    unsigned long long* det_acc = nullptr;   // deterministic mode: split tiles' fixed-point sums
    double* det_part = nullptr;   // deterministic mode: the strengths' partial maxima
    int det_tmax = 0;             // records of the fullest tile
    bool col_dft = false;         // type-1 column pass as a direct DFT over the live rows
    int max_live_rows = 0;        // live tile rows of the fullest problem
    long long live_rows_total = 0;   // live tile rows summed over the problems
    int* row_list = nullptr;      // type 1, pruned: the spreading-grid rows of live tile rows
    int n_row_list = 0;
    long long n_records = 0;
    int spread_blocks = 0;
    ChirpParams cp{};
    InterpParams ip{};
    FftPlan fp1{}, fp2{};
    FftDim d1{}, d2{};            // FFT along x (rows) and y (columns)
    void* fscratch = nullptr;     // four-step intermediate
    std::vector<void*> allocs;
    long long bytes = 0;
    void* rec = nullptr;
    void* sorted = nullptr;
    int* counts = nullptr;
    int* cursor = nullptr;
    Chunk* chunks = nullptr;
    int* n_meta = nullptr;        // [chunks, split tiles]
    int* split_tiles = nullptr;
    int* work = nullptr;          // dynamic chunk counter + finished blocks
    void* grid = nullptr;
    void* inter = nullptr;
    void* F = nullptr;
    void* tw1 = nullptr;
    void* tw2 = nullptr;
    void* ax = nullptr;
    void* ay = nullptr;
    void* dec1 = nullptr;
    void* dec2 = nullptr;
    double* gq_t = nullptr;
    double* gq_w = nullptr;
    int gq_n = 0;
    int* tcounts = nullptr;       // type-3 target bins (zero between evaluations)
    int* tstart = nullptr;
    int* tcursor = nullptr;
    int* twork = nullptr;         // binned interpolation's dynamic bin counter
    int* tpartial = nullptr;      // chunk sums of the multi-block bin scan
    int* perm = nullptr;          // type-3 target permutation, grown on demand
    long long perm_cap = 0;
    double* cheb = nullptr;
    int ncheb = 0;
    unsigned* status = nullptr;
    bool nodes_ready = false;
    double* stage_tgt = nullptr;
    void* stage_out = nullptr;
    long long stage_cap = 0;
    // host-buffer evaluations: the targets' copy runs on cst while the node,
    // sort, spreading and FFT stages run on st; st waits for ev_h2d (wait_tgt)
    // only before the target-side kernels; cst waits for ev_free (the previous
    // evaluation done with stage_tgt) before overwriting it
    cudaStream_t cst = nullptr;
    cudaEvent_t ev_h2d = nullptr, ev_free = nullptr;
    cudaEvent_t wait_tgt = nullptr;
    // FP32 binned type 3: the target sort runs on sort_st, forked from st at
    // the start of an evaluation (ev_sort_fork: the previous evaluation's
    // interpolation is done with the sort buffers) and joined before the
    // interpolation (ev_sorted), so it overlaps the spreading and the FFT
    cudaStream_t sort_st = nullptr;
    cudaEvent_t ev_sort_fork = nullptr, ev_sorted = nullptr;
    int timing = 0;
    cudaEvent_t ev[kMaxEvents] = {};
    const char* ev_name[kMaxEvents] = {};
    int nev = 0;
    int launches = 0;
    int last_launches = 0;     // kernels launched by the most recent evaluation
    // scattered-target batches: one sub-plan per problem, evaluated as one
    // CUDA graph over kLanes internal streams
    std::vector<Plan*> subs;
    cudaStream_t lanes[4] = {};
    cudaEvent_t ev_fork = nullptr, ev_in = nullptr, ev_out = nullptr, ev_join[4] = {};
    cudaGraphExec_t gexec = nullptr;
    std::vector<long long> g_M;   // key of the captured graph: counts and pointers
    const void* g_t = nullptr;
    void* g_out = nullptr;
    // profile-gradient scratch (allocated on first use)
    void* adj_in = nullptr;       // B x n2 x n1: sgn conj(gamma) ax ay
    void* adj_rows = nullptr;     // B x n2 x nf1 after the row pass
    double* contrib = nullptr;    // per node dL/dA contribution
    int* pf = nullptr;            // PETALS families (indices into fams)
    long long* gofs = nullptr;    // their offsets in the gradient output
    int npf = 0;
    long long n_grad = 0;
    // shape-gradient lists (Fourier boundary families), allocated on first use
    bool shape_ready = false;
    int* sf = nullptr;            // Fourier families (indices into fams)
    long long* sbofs = nullptr;   // their first boundary node in rbuf
    long long* sgofs = nullptr;   // their first coefficient in the gradient output
    double* rbuf = nullptr;       // dL/dr_i per boundary node
    int nsf = 0, max_params = 0;
    long long n_sgrad = 0, n_sbdry = 0;

    size_t csize() const { return prec == FRESNEL_FP64 ? 16 : 8; }
    size_t rsize() const { return prec == FRESNEL_FP64 ? sizeof(NodeRec<double>) : sizeof(NodeRec<float>); }
};

fresnel_status dalloc(Plan* p, void** out, size_t bytes) {
    *out = nullptr;
    if (bytes == 0) bytes = 16;
    if (p->opts.max_device_bytes > 0 && p->bytes + (long long)bytes > p->opts.max_device_bytes)
        return fres_fail(FRESNEL_ERR_OOM, "plan would exceed max_device_bytes (" +
                                               std::to_string(p->opts.max_device_bytes) + ")");
    cudaError_t e = cudaMalloc(out, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fres_fail(FRESNEL_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    p->allocs.push_back(*out);
    p->bytes += (long long)bytes;
    return FRESNEL_OK;
}

#define FRES_TRY(x)                          \
    do {                                     \
        fresnel_status s_ = (x);             \
        if (s_ != FRESNEL_OK) return s_;     \
    } while (0)

void free_plan(Plan* p) {
    if (!p) return;
    cudaStreamSynchronize(p->st);
    for (Plan* q : p->subs) free_plan(q);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    for (cudaStream_t& l : p->lanes)
        if (l) cudaStreamDestroy(l);
    for (cudaEvent_t e : {p->ev_fork, p->ev_in, p->ev_out, p->ev_join[0], p->ev_join[1],
                          p->ev_join[2], p->ev_join[3], p->ev_h2d, p->ev_free})
        if (e) cudaEventDestroy(e);
    if (p->cst) {
        cudaStreamSynchronize(p->cst);
        cudaStreamDestroy(p->cst);
    }
    if (p->sort_st) {
        cudaStreamSynchronize(p->sort_st);
        cudaStreamDestroy(p->sort_st);
    }
    for (cudaEvent_t e : {p->ev_sort_fork, p->ev_sorted})
        if (e) cudaEventDestroy(e);
    for (void* a : p->allocs) cudaFree(a);
    if (p->perm) cudaFree(p->perm);
    for (int i = 0; i < kMaxEvents; ++i)
        if (p->ev[i]) cudaEventDestroy(p->ev[i]);
    p->magic = 0;
    delete p;
}

bool is_nice(long long n) {
    for (int f : {2, 3, 5})
        while (n % f == 0) n /= f;
    return n == 1;
}
int nice_size(double target, int mult) {
    long long n = (long long)std::ceil(target - 1e-9);
    if (n < mult) n = mult;
    n = (n + mult - 1) / mult * mult;
    while (!is_nice(n)) n += mult;
    return (int)n;
}

// Spreading-kernel choice: exponential of semicircle, width w grid points,
// shape beta, upsampling sigma.  The paper takes the NUFFT as a library and
// quotes only its upsampling (5/4 for eps >= 1e-9, else 2; Sec. 4.1); the
// width/shape rules follow the published FINUFFT method.  FP32 fast mode
// uses sigma = 2 (at 5/4 the deconvolution amplifies FP32 rounding by >1e2 at
// the band edge) and designs the kernel for tol/10, leaving room for FP32
// rounding under the requested tolerance.
void fit_horner(int w, double beta, HornerTab* h);
double fit_horner_d(int w, double beta, HornerTabD* h);

void choose_kernel(Plan* p) {
    double tk = p->tol;
    double sigma;
    if (p->prec == FRESNEL_FP32_FAST) {
        sigma = p->opts.sigma > 0 ? p->opts.sigma : 2.0;
        tk = p->tol / 10.0;
    } else {
        sigma = p->opts.sigma > 0 ? p->opts.sigma : (p->tol >= 1e-9 ? 1.25 : 2.0);
    }
    int w;
    double beta;
    if (std::fabs(sigma - 2.0) < 1e-12) {
        w = (int)std::ceil(std::log10(1.0 / tk)) + 1;
    } else {
        w = (int)std::ceil(-std::log(tk) / (kPi * std::sqrt(1.0 - 1.0 / sigma)));
    }
    if (p->opts.kernel_w > 0) w = p->opts.kernel_w;
    w = std::max(2, std::min(kMaxW, w));
    if (std::fabs(sigma - 2.0) < 1e-12) beta = 2.30 * w;
    else beta = 0.97 * kPi * (1.0 - 0.5 / sigma) * w;
    p->sigma = sigma;
    p->ks.w = w;
    p->ks.beta = beta;
    p->ks.betaf = (float)beta;
    p->ks.horner.deg = -1;
    p->ks.hornerd.deg = -1;
    if (p->prec == FRESNEL_FP32_FAST) {
        fit_horner(w, beta, &p->ks.horner);
    } else if (fit_horner_d(w, beta, &p->ks.hornerd) > 0.2 * p->tol) {
        p->ks.hornerd.deg = -1;   // the fit's floor is above this tolerance: exp/sqrt
    }
}

// Fit, for each of the unit pieces a < ceil(w/2) of the kernel (the others
// are their mirror images), a polynomial in t = 2 f - 1 (f the node's
// fractional offset): Chebyshev interpolation at deg + 1 points, converted to
// monomials in long double and split into even and odd parts.  The degree
// grows until the maximum error (on a fine grid) stops improving or drops
// below `stop`; the kernel's square-root end points set a floor near
// beta e^-beta / deg.  Returns the kept table's maximum error.
template <typename Tab, typename R, int kMaxDeg>
double fit_pieces(int w, double beta, int deg0, double stop, Tab* h) {
    auto psi = [&](long double z) -> long double {
        long double a = 1.0L - z * z;
        return a > 0 ? std::exp((long double)beta * (std::sqrt(a) - 1.0L)) : 0.0L;
    };
    // the kernel on each piece's error grid, once for every degree tried
    // (long double is software quad precision on some hosts)
    constexpr int kGrid = 400;
    std::vector<long double> gv((size_t)((w + 1) / 2) * (kGrid + 1));
    for (int a = 0; a < (w + 1) / 2; ++a)
        for (int i = 0; i <= kGrid; ++i) {
            const long double f = 0.5L * (-1.0L + i / (0.5L * kGrid) + 1.0L);
            gv[(size_t)a * (kGrid + 1) + i] = psi(((long double)a + 1.0L - 0.5L * w - f) * 2.0L / w);
        }
    double prev_err = 1e300, best_err = 1e300;
    Tab best{};
    best.deg = -1;
    for (int d = deg0; d <= kMaxDeg; ++d) {
        const int n = d + 1;
        Tab t{};
        t.deg = d;
        double err = 0.0;
        for (int a = 0; a < (w + 1) / 2; ++a) {
            auto g = [&](long double tt) {
                long double f = 0.5L * (tt + 1.0L);
                return psi(((long double)a + 1.0L - 0.5L * w - f) * 2.0L / w);
            };
            std::vector<long double> b(n), mono(n, 0.0L), T0(n, 0.0L), T1(n, 0.0L), T2(n);
            for (int k = 0; k < n; ++k) {
                long double acc = 0.0L;
                for (int i = 0; i < n; ++i) {
                    long double th = 3.14159265358979323846264338327950288L * (i + 0.5L) / n;
                    acc += g(std::cos(th)) * std::cos(k * th);
                }
                b[k] = (k == 0 ? 1.0L : 2.0L) * acc / n;
            }
            T0[0] = 1.0L;
            if (n > 1) T1[1] = 1.0L;
            for (int k = 0; k < n; ++k) {
                const std::vector<long double>& Tk = k == 0 ? T0 : T1;
                for (int j = 0; j < n; ++j) mono[j] += b[k] * Tk[j];
                if (k >= 1 && k + 1 < n) {   // T_{k+1} = 2 t T_k - T_{k-1}
                    for (int j = 0; j < n; ++j) T2[j] = (j > 0 ? 2.0L * T1[j - 1] : 0.0L) - T0[j];
                    T0 = T1;
                    T1 = T2;
                }
            }
            for (int j = 0; j < n; ++j) {
                if (j % 2 == 0) t.e[a][j / 2] = (R)mono[j];
                else t.o[a][j / 2] = (R)mono[j];
            }
            for (int i = 0; i <= kGrid; ++i) {
                long double tt = -1.0L + i / (0.5L * kGrid), acc = 0.0L;
                for (int j = n - 1; j >= 0; --j) acc = acc * tt + mono[j];
                err = std::max(err, (double)std::fabs(acc - gv[(size_t)a * (kGrid + 1) + i]));
            }
        }
        if (err < best_err) {
            best = t;
            best_err = err;
        }
        if (err < stop || err > 0.9 * prev_err) break;
        prev_err = err;
    }
    *h = best;
    return best_err;
}

void fit_horner(int w, double beta, HornerTab* h) {
    fit_pieces<HornerTab, float, kHornerDeg>(w, beta, 4, 1e-9, h);
}

double fit_horner_d(int w, double beta, HornerTabD* h) {
    return fit_pieces<HornerTabD, double, kHornerDegD>(w, beta, 6, 1e-16, h);
}

fresnel_status validate_family(const fresnel_family& f, long long* n_bdry, long long* n_nodes,
                               int* K) {
    if (!f.params || f.n_params <= 0) return fres_fail(FRESNEL_ERR_ARG, "family params missing");
    for (long long i = 0; i < f.n_params; ++i)
        if (!std::isfinite(f.params[i]))
            return fres_fail(FRESNEL_ERR_ARG, "family params contain a non-finite value");
    if (!std::isfinite(f.cx) || !std::isfinite(f.cy))
        return fres_fail(FRESNEL_ERR_ARG, "family centre not finite");
    if (f.motion) {
        if (f.kind != FRESNEL_FAMILY_PETALS)
            return fres_fail(FRESNEL_ERR_ARG, "a motion is for PETALS families only");
        if (f.n_panels < 1 || f.n_panels > 65536)
            return fres_fail(FRESNEL_ERR_ARG, "PETALS family needs 1<=n_panels<=65536");
        for (long long i = 0; i < 3LL * f.n_panels; ++i)
            if (!std::isfinite(f.motion[i]))
                return fres_fail(FRESNEL_ERR_ARG, "petal motion contains a non-finite value");
    }
    switch (f.kind) {
        case FRESNEL_FAMILY_FOURIER:
            if (f.n_panels < 1 || f.p < 1 || f.m < 1 || f.p > 4096 || f.m > 65536)
                return fres_fail(FRESNEL_ERR_ARG, "FOURIER family needs n_panels>=1, 1<=p<=4096, 1<=m<=65536");
            if (f.n_params % 2 != 1)
                return fres_fail(FRESNEL_ERR_ARG, "FOURIER params must be [r0, a1, b1, ...] (odd length)");
            *K = (int)((f.n_params - 1) / 2);
            *n_bdry = (long long)f.n_panels * f.p;
            *n_nodes = *n_bdry * f.m;
            return FRESNEL_OK;
        case FRESNEL_FAMILY_LINE_RULE:
            if (f.n_panels < 1 || f.p < 1 || f.m < 1 || f.m > 65536)
                return fres_fail(FRESNEL_ERR_ARG, "LINE_RULE family needs n_panels>=1, p>=1, 1<=m<=65536");
            if (f.n_params != 4LL * f.n_panels * f.p)
                return fres_fail(FRESNEL_ERR_ARG, "LINE_RULE params must hold 4 * n_panels * p values");
            *K = 0;
            *n_bdry = (long long)f.n_panels * f.p;
            *n_nodes = *n_bdry * f.m;
            return FRESNEL_OK;
        case FRESNEL_FAMILY_NODES:
            if (f.n_params % 3 != 0)
                return fres_fail(FRESNEL_ERR_ARG, "NODES params must hold 3 * N values");
            *K = 0;
            *n_bdry = 0;
            *n_nodes = f.n_params / 3;
            return FRESNEL_OK;
        case FRESNEL_FAMILY_TRIANGLES:
            if (f.n_panels < 1 || f.p < 1 || f.p > 4096)
                return fres_fail(FRESNEL_ERR_ARG, "TRIANGLES family needs n_panels>=1, 1<=p<=4096");
            if (f.n_params != 6LL * f.n_panels)
                return fres_fail(FRESNEL_ERR_ARG, "TRIANGLES params must hold 6 * n_panels values");
            *K = 0;
            *n_bdry = 0;
            *n_nodes = (long long)f.n_panels * f.p * f.p;
            return FRESNEL_OK;
        case FRESNEL_FAMILY_PETALS: {
            if (f.n_panels < 1 || f.p < 1 || f.m < 1 || f.n_panels > 65536 || f.p > 4096 ||
                f.m > 65536)
                return fres_fail(FRESNEL_ERR_ARG,
                                 "PETALS family needs 1<=n_panels<=65536, 1<=p<=4096, 1<=m<=65536");
            if (f.n_params < 5)
                return fres_fail(FRESNEL_ERR_ARG, "PETALS params must be [a, R, n_d, m_d, profile, ...]");
            const double a = f.params[0], R = f.params[1];
            const double n_d = f.params[2], m_d = f.params[3], prof = f.params[4];
            if (!(a >= 0.0) || !(R > a))
                return fres_fail(FRESNEL_ERR_ARG, "PETALS needs 0 <= a < R");
            if (n_d != std::floor(n_d) || n_d < 0 || n_d > 1e7 || m_d != std::floor(m_d) ||
                (n_d > 0 && (m_d < 1 || m_d > 65536)))
                return fres_fail(FRESNEL_ERR_ARG, "PETALS needs whole n_d in [0, 1e7] and m_d in [1, 65536]");
            const long long nprof = f.n_params - 5;
            if (prof == FRESNEL_PETAL_HG) {
                if (nprof != 2 || !(f.params[5] > 0.0) || !(f.params[6] > 0.0))
                    return fres_fail(FRESNEL_ERR_ARG, "PETAL_HG profile needs [b > 0, q > 0]");
            } else if (prof == FRESNEL_PETAL_BSPLINE) {
                if (nprof < 4 || nprof > (1 << 20))
                    return fres_fail(FRESNEL_ERR_ARG, "PETAL_BSPLINE profile needs 4 to 2^20 coefficients");
            } else if (prof == FRESNEL_PETAL_TABLE) {
                if (nprof != f.m)
                    return fres_fail(FRESNEL_ERR_ARG, "PETAL_TABLE profile needs m values");
            } else {
                return fres_fail(FRESNEL_ERR_ARG, "unknown petal profile");
            }
            *K = 0;
            *n_bdry = (long long)f.p * f.m;
            *n_nodes = (long long)f.n_panels * f.p * f.m;
            return FRESNEL_OK;
        }
        default:
            return fres_fail(FRESNEL_ERR_ARG, "unknown family kind");
    }
}

void ev_record(Plan* p, const char* name) {
    if (!p->timing || p->nev >= kMaxEvents) return;
    if (!p->ev[p->nev]) cudaEventCreate(&p->ev[p->nev]);
    p->ev_name[p->nev] = name;
    cudaEventRecord(p->ev[p->nev], p->st);
    p->nev++;
}

template <typename T>
fresnel_status run_nodes(Plan* p, double* dx, double* dy, double* dw) {
    launch_nodes<T>(p->ft, p->node_blocks, (NodeRec<T>*)p->rec, p->counts, dx, dy, dw, p->status,
                    p->st);
    p->launches++;
    return FRESNEL_OK;
}

template <typename T>
fresnel_status run_sort(Plan* p) {
    launch_scan_problems(p->B, p->ntiles, p->counts, p->cursor, p->chunks, p->split_tiles,
                         p->layout, p->chunk_cap, p->status, p->st);
    ev_record(p, "scan");
    launch_scatter_fams<T>(p->ft, p->node_blocks, (const NodeRec<T>*)p->rec, p->cursor,
                           (NodeRec<T>*)p->sorted, p->n_records, p->status, p->st);
    p->launches += 2;
    return FRESNEL_OK;
}

// Row pass (transforms along x) through one pass or the four-step path.
template <typename T>
void run_rows(Plan* p, RowPassArgs ra) {
    const FftDim& d = p->d1;
    if (!d.big) {
        ra.twiddle = d.tw;
        launch_fft_rows<T>(d.fp, ra, p->st);
        p->launches++;
        return;
    }
    ColPassArgs c1{};
    c1.mode = kFftRowStep1;
    c1.in = ra.in;
    c1.in_stride = ra.in_stride;
    c1.in_len = ra.in_len;
    c1.centered_in = ra.centered_in;
    c1.deconv_col = ra.deconv_col;
    c1.deconv_row = ra.deconv_row;
    c1.out = p->fscratch;
    c1.ncols = d.fb;
    c1.nouter = ra.nrows;
    c1.fa = d.fa;
    c1.fb = d.fb;
    c1.fN = d.n;
    c1.out_len = d.fa;
    c1.twiddle = d.twa;
    launch_fft_cols<T>(d.fpa, c1, p->st);
    // B-point transforms: groups of adjacent scratch rows (consecutive k1)
    // per block, so short transforms still fill the GPU
    ColPassArgs c2{};
    c2.mode = kFftRowStep2;
    c2.in = p->fscratch;
    c2.ncols = d.fa;
    c2.nouter = ra.nrows;
    c2.out = ra.out;
    c2.out_stride = ra.out_stride;
    c2.out_len = ra.out_len;
    c2.fa = d.fa;
    c2.fb = d.fb;
    c2.fN = d.n;
    c2.twN = d.tw;
    c2.twiddle = d.twb;
    launch_fft_cols<T>(d.fpb, c2, p->st);
    p->launches += 2;
}

// Column pass (transforms along y), likewise.
template <typename T>
void run_cols(Plan* p, ColPassArgs ca) {
    const FftDim& d = p->d2;
    if (!d.big) {
        ca.twiddle = d.tw;
        launch_fft_cols<T>(d.fp, ca, p->st);
        p->launches++;
        return;
    }
    ColPassArgs c1{};
    c1.mode = kFftColStep1;
    c1.in = ca.in;
    c1.ncols = ca.ncols;
    c1.in_len = ca.in_len;
    c1.centered_in = ca.centered_in;
    c1.out = p->fscratch;
    c1.nouter = d.fb;
    c1.fa = d.fa;
    c1.fb = d.fb;
    c1.fN = d.n;
    c1.out_len = d.fa;
    c1.twiddle = d.twa;
    launch_fft_cols<T>(d.fpa, c1, p->st);
    ColPassArgs c2{};
    c2.mode = kFftColStep2;
    c2.in = p->fscratch;
    c2.ncols = ca.ncols;
    c2.out = ca.out;
    c2.nouter = d.fa;
    c2.fa = d.fa;
    c2.fb = d.fb;
    c2.fN = d.n;
    c2.out_len = ca.out_len;
    c2.twN = d.tw;
    c2.twiddle = d.twb;
    c2.ax = ca.ax;
    c2.ay = ca.ay;
    c2.occulter = ca.occulter;
    launch_fft_cols<T>(d.fpb, c2, p->st);
    p->launches += 2;
}

template <typename T>
fresnel_status eval_impl(Plan* p, const double* d_targets, long long M, void* d_out) {
    p->launches = 0;
    p->nev = 0;
    ev_record(p, "start");
    // FP32 type 3 with binned interpolation: the target sort depends on the
    // targets and the plan's geometry only, so it runs on its own stream
    // beside the node, spreading and FFT stages (serially on st when stage
    // times are recorded, so that each stage is timed on its own)
    bool binned = false;
    if (p->tkind == FRESNEL_SCATTERED && M > 0 && sizeof(T) == 4) {
        const long long fbytes = (long long)p->nfft1 * p->nfft2 * (long long)sizeof(cx_t<T>);
        const bool want = p->opts.t3_binning > 0 ||
                          (p->opts.t3_binning == 0 && M >= kSortTargetsFrom &&
                           fbytes > kBinFromGridBytes);
        binned = want && M < (1LL << 31) && interp_binned_width(p->ks.w);
    }
    T3Sort sort{};
    const bool overlap = binned && !p->timing && p->sort_st;
    if (binned) {
        if (M > p->perm_cap) {   // grown once; later evaluations reuse it
            if (p->perm) cudaFree(p->perm);
            p->perm = nullptr;
            p->perm_cap = 0;
            FRES_CK(cudaMalloc((void**)&p->perm, sizeof(int) * (size_t)M));
            p->perm_cap = M;
        }
        sort = T3Sort{p->tcounts, p->tstart, p->tcursor, p->perm, p->twork, p->tpartial};
        p->launches += p->ip.nbin1 * p->ip.nbin2 <= kBinScanStaged ? 3 : 5;
    }
    if (overlap) {
        FRES_CK(cudaEventRecord(p->ev_sort_fork, p->st));
        FRES_CK(cudaStreamWaitEvent(p->sort_st, p->ev_sort_fork, 0));
        if (p->wait_tgt) FRES_CK(cudaStreamWaitEvent(p->sort_st, p->wait_tgt, 0));
        launch_target_sort(d_targets, M, p->ip, p->ks.w, &sort, p->sort_st);
        FRES_CK(cudaEventRecord(p->ev_sorted, p->sort_st));
    }
    if (p->opts.recompute_nodes || !p->nodes_ready) {
        FRES_TRY(run_nodes<T>(p, nullptr, nullptr, nullptr));
        ev_record(p, "nodes_chirp_count");
        FRES_TRY(run_sort<T>(p));
        ev_record(p, "scatter");
        p->nodes_ready = true;
    }
    if (p->opts.deterministic) {
        launch_spread_det<T>((const NodeRec<T>*)p->sorted, p->n_records, p->chunks, p->n_meta,
                             p->max_chunks, p->split_tiles, p->max_split, p->det_acc,
                             p->det_part, p->det_tmax, (cx_t<T>*)p->grid, p->work, p->status,
                             p->nf1, p->nf2, p->ntx, p->ntiles, p->ks, p->st);
        p->launches += p->max_split > 0 ? 3 : 2;
    } else {
        const long long spin = p->opts.max_spin == 0 ? kDefaultMaxSpin
                                                     : std::max(0LL, p->opts.max_spin);
        launch_spread<T>((const NodeRec<T>*)p->sorted, p->chunks, p->n_meta, p->max_chunks,
                         p->ready, p->max_split, spin, (cx_t<T>*)p->grid, p->work, p->status,
                         p->nf1, p->nf2, p->ntx, p->ntiles, p->ks, p->spread_blocks, p->st);
        p->launches += 1;
    }
    ev_record(p, "spread");
    if (p->tkind == FRESNEL_GRID) {
        RowPassArgs ra{};
        ra.in = p->grid;
        ra.out = p->inter;
        ra.in_stride = p->nf1;
        ra.out_stride = p->n1;
        ra.nrows = p->nf2 * p->B;
        ra.in_len = p->nf1;
        ra.centered_in = 0;
        ra.out_len = p->n1;
        ra.live = p->layout.live;
        ra.batch_rows = p->nf2;
        ra.nty = p->nty;
        ra.row_list = p->row_list;
        ra.nlist = p->n_row_list;
        run_rows<T>(p, ra);
        ev_record(p, "fft_rows");
        ColPassArgs ca{};
        ca.in = p->inter;
        ca.out = d_out;
        ca.ncols = p->n1;
        ca.in_len = p->nf2;
        ca.centered_in = 0;
        ca.out_len = p->n2;
        ca.twiddle = p->tw2;
        ca.ax = p->ax;
        ca.ay = p->ay;
        ca.occulter = p->output == FRESNEL_OCCULTER;
        ca.out_is_final = 1;
        ca.batch = p->B;
        ca.in_bstride = (long long)p->nf2 * p->n1;
        ca.out_bstride = (long long)p->n2 * p->n1;
        ca.live = p->layout.live;
        ca.nty = p->nty;
        if (p->col_dft) {
            ca.twiddle = p->d2.tw;
            // one live tile row: FP32 on the tensor cores (split-TF32
            // operands), FP64 as a pruned FFT; several: the direct FMA sum
            if (sizeof(T) == 4 && col_dft_tc_supported(ca, kTile * p->max_live_rows))
                launch_col_dft_tc(ca, p->nf2, p->status, p->st);
            else if (sizeof(T) == 8 && col_pfft_supported(p->nf2, kTile * p->max_live_rows))
                launch_col_pfft_d(ca, p->nf2, p->status, p->st);
            else
                launch_col_dft<T>(ca, p->nf2, p->status, p->st);
            p->launches++;
        } else {
            run_cols<T>(p, ca);
        }
        ev_record(p, "fft_cols_epilogue");
    } else {
        RowPassArgs ra{};
        ra.in = p->grid;
        ra.out = p->inter;
        ra.in_stride = p->nf1;
        ra.out_stride = p->nfft1;
        ra.nrows = p->nf2;
        ra.in_len = p->nf1;
        ra.centered_in = 1;
        ra.deconv_col = p->dec1;
        ra.deconv_row = p->dec2;
        ra.out_len = p->nfft1;
        run_rows<T>(p, ra);
        ev_record(p, "fft_rows");
        ColPassArgs ca{};
        ca.in = p->inter;
        ca.out = p->F;
        ca.ncols = p->nfft1;
        ca.in_len = p->nf2;
        ca.centered_in = 1;
        ca.out_len = p->nfft2;
        run_cols<T>(p, ca);
        ev_record(p, "fft_cols");
        if (M > 0) {
            if (p->wait_tgt) {   // the host targets' copy (fresnel_eval_host)
                FRES_CK(cudaStreamWaitEvent(p->st, p->wait_tgt, 0));
                p->wait_tgt = nullptr;
            }
            const T3Sort* sp = binned ? &sort : nullptr;
            if (overlap) {
                FRES_CK(cudaStreamWaitEvent(p->st, p->ev_sorted, 0));
            } else if (binned) {
                launch_target_sort(d_targets, M, p->ip, p->ks.w, sp, p->st);
                ev_record(p, "target_sort");
            }
            launch_interp_w<T>(d_targets, M, (const cx_t<T>*)p->F, p->ip, p->ks, p->cheb,
                               p->ncheb, d_out, p->status, sp, p->st);
            p->launches++;
        }
        ev_record(p, "interp_epilogue");
    }
    p->last_launches = p->launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fres_fail(FRESNEL_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return FRESNEL_OK;
}

fresnel_status read_status(Plan* p) {
    unsigned h = 0;
    FRES_CK(cudaMemcpyAsync(&h, p->status, sizeof(unsigned), cudaMemcpyDeviceToHost, p->st));
    FRES_CK(cudaStreamSynchronize(p->st));
    if (h) {
        FRES_CK(cudaMemsetAsync(p->status, 0, sizeof(unsigned), p->st));
        FRES_CK(cudaStreamSynchronize(p->st));
        std::string msg = "device check failed:";
        if (h & kStatusTargetOutside) msg += " target outside the plan's box;";
        if (h & kStatusNodeOutside) msg += " node support outside the type-3 grid;";
        if (h & kStatusNonFinite) msg += " non-finite coordinate;";
        if (h & kStatusOverflow) msg += " sort region overflow;";
        if (h & kStatusTimeout) {
            msg += " a split tile's chunk gave up waiting for the tile to be cleared"
                   " (fresnel_opts.max_spin);";
            return fres_fail(FRESNEL_ERR_TIMEOUT, msg);
        }
        return fres_fail(FRESNEL_ERR_DEVICE, msg);
    }
    return FRESNEL_OK;
}

struct Bounds {
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    void add(double x, double y) {
        xmin = std::min(xmin, x);
        xmax = std::max(xmax, x);
        ymin = std::min(ymin, y);
        ymax = std::max(ymax, y);
    }
};

fresnel_status copy_params(Plan* p, FamilyDev& f, const double* hparams, long long n) {
    FRES_TRY(dalloc(p, (void**)&f.params, sizeof(double) * n));
    FRES_CK(cudaMemcpyAsync(f.params, hparams, sizeof(double) * n, cudaMemcpyHostToDevice, p->st));
    return FRESNEL_OK;
}

template <typename T>
fresnel_status setup_nodes_family(Plan* p, FamilyDev& f, const double* hparams, long long n,
                                  Bounds& bb) {
    FRES_TRY(copy_params(p, f, hparams, n));
    for (long long j = 0; j < f.n_nodes; ++j) bb.add(hparams[j], hparams[f.n_nodes + j]);
    return FRESNEL_OK;
}

// A union of triangles: device vertices and the p-point Gauss-Legendre rule
// on (0, 1) as alpha (gl_m_a, also the edge parameters), alpha * what
// (gl_m_aw) and what (gl_p_w); nodes lie inside each triangle, so the
// translated vertices bound them.
fresnel_status setup_triangle_family(Plan* p, FamilyDev& f, const double* hparams, long long n,
                                     Bounds& bb) {
    FRES_TRY(copy_params(p, f, hparams, n));
    f.m = f.p;
    FRES_TRY(dalloc(p, (void**)&f.gl_m_a, sizeof(double) * f.p));
    FRES_TRY(dalloc(p, (void**)&f.gl_m_aw, sizeof(double) * f.p));
    FRES_TRY(dalloc(p, (void**)&f.gl_p_w, sizeof(double) * f.p));
    launch_gauss_legendre(f.p, f.gl_m_a, f.gl_p_w, p->st);
    std::vector<double> a(f.p), w(f.p);
    FRES_CK(cudaMemcpyAsync(a.data(), f.gl_m_a, sizeof(double) * f.p, cudaMemcpyDeviceToHost, p->st));
    FRES_CK(cudaMemcpyAsync(w.data(), f.gl_p_w, sizeof(double) * f.p, cudaMemcpyDeviceToHost, p->st));
    FRES_CK(cudaStreamSynchronize(p->st));
    for (int l = 0; l < f.p; ++l) w[l] *= a[l];
    FRES_CK(cudaMemcpyAsync(f.gl_m_aw, w.data(), sizeof(double) * f.p, cudaMemcpyHostToDevice, p->st));
    FRES_CK(cudaStreamSynchronize(p->st));
    for (long long t = 0; t < f.n_panels; ++t)
        for (int v = 0; v < 3; ++v)
            bb.add(f.cx + hparams[6 * t + 2 * v], f.cy + hparams[6 * t + 2 * v + 1]);
    return FRESNEL_OK;
}

// Device params, Gauss-Legendre rules and boundary line rule of a family
// used through the dilation rule (FOURIER, LINE_RULE, a starshade's disc),
// and the bounds of its nodes.
template <typename T>
fresnel_status setup_dilation_family(Plan* p, FamilyDev& f, const double* hparams, long long n,
                                     Bounds& bb) {
    const bool dbl = sizeof(T) == 8;
    const long long nb = f.n_bdry;
    FRES_TRY(copy_params(p, f, hparams, n));
    if (f.kind == FRESNEL_FAMILY_FOURIER && !f.ptr) {
        FRES_TRY(dalloc(p, (void**)&f.gl_p_t, sizeof(double) * f.p));
        FRES_TRY(dalloc(p, (void**)&f.gl_p_w, sizeof(double) * f.p));
        launch_gauss_legendre(f.p, f.gl_p_t, f.gl_p_w, p->st);
    }
    FRES_TRY(dalloc(p, (void**)&f.gl_m_a, sizeof(double) * f.m));
    FRES_TRY(dalloc(p, (void**)&f.gl_m_aw, sizeof(double) * f.m));
    launch_gauss_legendre(f.m, f.gl_m_a, f.gl_m_aw, p->st);
    // alpha_l * wtilde_l (eq. aqwei) formed on the host from the device rule
    std::vector<double> a(f.m), w(f.m);
    FRES_CK(cudaMemcpyAsync(a.data(), f.gl_m_a, sizeof(double) * f.m, cudaMemcpyDeviceToHost, p->st));
    FRES_CK(cudaMemcpyAsync(w.data(), f.gl_m_aw, sizeof(double) * f.m, cudaMemcpyDeviceToHost, p->st));
    FRES_CK(cudaStreamSynchronize(p->st));
    for (int l = 0; l < f.m; ++l) w[l] *= a[l];
    FRES_CK(cudaMemcpyAsync(f.gl_m_aw, w.data(), sizeof(double) * f.m, cudaMemcpyHostToDevice, p->st));
    FRES_TRY(dalloc(p, (void**)&f.bx, sizeof(double) * nb));
    FRES_TRY(dalloc(p, (void**)&f.by, sizeof(double) * nb));
    FRES_TRY(dalloc(p, (void**)&f.bc, sizeof(double) * nb));
    FRES_TRY(dalloc(p, (void**)&f.bw, sizeof(double) * nb));
    FRES_TRY(dalloc(p, (void**)&f.bv, sizeof(double) * nb));
    if (!dbl) {   // double-float radial rule for the FP32 spoke form
        std::vector<float> adf(2 * f.m), awf(f.m);
        for (int l = 0; l < f.m; ++l) {
            dflt s = df_host(a[l]);
            adf[2 * l] = s.hi;
            adf[2 * l + 1] = s.lo;
            awf[l] = (float)w[l];
        }
        FRES_TRY(dalloc(p, (void**)&f.adf, sizeof(float) * 2 * f.m));
        FRES_TRY(dalloc(p, (void**)&f.awf, sizeof(float) * f.m));
        FRES_CK(cudaMemcpyAsync(f.adf, adf.data(), sizeof(float) * 2 * f.m, cudaMemcpyHostToDevice, p->st));
        FRES_CK(cudaMemcpyAsync(f.awf, awf.data(), sizeof(float) * f.m, cudaMemcpyHostToDevice, p->st));
        FRES_CK(cudaStreamSynchronize(p->st));
    }
    launch_boundary(f, p->cp, p->st);
    // node bounds (type 3 sizing): nodes lie on segments from the centre to
    // the boundary nodes, so centre + boundary bounds them.
    std::vector<double> bx(nb), by(nb);
    FRES_CK(cudaMemcpyAsync(bx.data(), f.bx, sizeof(double) * nb, cudaMemcpyDeviceToHost, p->st));
    FRES_CK(cudaMemcpyAsync(by.data(), f.by, sizeof(double) * nb, cudaMemcpyDeviceToHost, p->st));
    FRES_CK(cudaStreamSynchronize(p->st));
    bb.add(f.cx, f.cy);
    for (long long i = 0; i < nb; ++i) bb.add(f.cx + bx[i], f.cy + by[i]);
    return FRESNEL_OK;
}

// Petal tables of a starshade family (Sec. 4.2) and the bounds of its nodes.
fresnel_status setup_petal_family(Plan* p, FamilyDev& f, const fresnel_family& hf, Bounds& bb) {
    const long long nb = f.n_bdry;
    FRES_TRY(copy_params(p, f, hf.params, hf.n_params));
    f.pa = hf.params[0];
    f.pR = hf.params[1];
    f.profile = (int)hf.params[4];
    f.n_prof = hf.n_params - 5;
    FRES_TRY(dalloc(p, (void**)&f.gl_p_t, sizeof(double) * f.p));
    FRES_TRY(dalloc(p, (void**)&f.gl_p_w, sizeof(double) * f.p));
    launch_gauss_legendre(f.p, f.gl_p_t, f.gl_p_w, p->st);
    FRES_TRY(dalloc(p, (void**)&f.gl_m_a, sizeof(double) * f.m));
    FRES_TRY(dalloc(p, (void**)&f.gl_m_aw, sizeof(double) * f.m));
    launch_gauss_legendre(f.m, f.gl_m_a, f.gl_m_aw, p->st);
    FRES_TRY(dalloc(p, (void**)&f.bx, sizeof(double) * nb));
    FRES_TRY(dalloc(p, (void**)&f.by, sizeof(double) * nb));
    FRES_TRY(dalloc(p, (void**)&f.bc, sizeof(double) * nb));
    FRES_TRY(dalloc(p, (void**)&f.rot, sizeof(double) * 2 * f.n_panels));
    launch_boundary(f, p->cp, p->st);
    std::vector<double> u(nb), v(nb), rot(2 * f.n_panels);
    FRES_CK(cudaMemcpyAsync(u.data(), f.bx, sizeof(double) * nb, cudaMemcpyDeviceToHost, p->st));
    FRES_CK(cudaMemcpyAsync(v.data(), f.by, sizeof(double) * nb, cudaMemcpyDeviceToHost, p->st));
    FRES_CK(cudaMemcpyAsync(rot.data(), f.rot, sizeof(double) * 2 * f.n_panels,
                            cudaMemcpyDeviceToHost, p->st));
    FRES_CK(cudaStreamSynchronize(p->st));
    FRES_CK(cudaGetLastError());
    std::vector<double> sh(2 * f.n_panels, 0.0);
    if (hf.motion) {   // rigid motions: rotation folded into rot, translation kept apart
        for (int k = 0; k < f.n_panels; ++k) {
            const double phi = hf.motion[3 * k], c = rot[2 * k], s = rot[2 * k + 1];
            const double cp = std::cos(phi), sp = std::sin(phi);
            rot[2 * k] = c * cp - s * sp;
            rot[2 * k + 1] = s * cp + c * sp;
            sh[2 * k] = hf.motion[3 * k + 1];
            sh[2 * k + 1] = hf.motion[3 * k + 2];
        }
        FRES_TRY(dalloc(p, (void**)&f.shift, sizeof(double) * 2 * f.n_panels));
        FRES_CK(cudaMemcpyAsync(f.rot, rot.data(), sizeof(double) * 2 * f.n_panels,
                                cudaMemcpyHostToDevice, p->st));
        FRES_CK(cudaMemcpyAsync(f.shift, sh.data(), sizeof(double) * 2 * f.n_panels,
                                cudaMemcpyHostToDevice, p->st));
        FRES_CK(cudaStreamSynchronize(p->st));
    }
    for (long long q = 0; q < nb; ++q) {
        if (!std::isfinite(u[q]) || !std::isfinite(v[q]))
            return fres_fail(FRESNEL_ERR_ARG, "petal profile gives a non-finite node");
        for (int k = 0; k < f.n_panels; ++k) {
            const double c = rot[2 * k], s = rot[2 * k + 1];
            bb.add(f.cx + sh[2 * k] + u[q] * c - v[q] * s, f.cy + sh[2 * k + 1] + u[q] * s + v[q] * c);
        }
    }
    return FRESNEL_OK;
}

// Root-arc patches of a starshade with moved petals (Sec. 5, second
// construction): for petal k the signed region between its root arc on the
// disc circle, root(s) = c + a (cos, sin)(2 pi k/N - pi/N + 2 pi s/N), and the
// moved base arc M_k(root(s)) = c + R(phi_k)(root(s) - c) + t_k, as
// P(s, t) = (1 - t) root(s) + t M_k(root(s)) with weight dP/dt x dP/ds on a
// qs x qt Gauss-Legendre product rule in (s, t).  Returns x..., y..., w...
// (FP64, host) for an explicit-node family.
fresnel_status petal_patches(Plan* p, const fresnel_family& hf, std::vector<double>* out) {
    const int N = hf.n_panels, qs = std::max(2 * hf.p, 16), qt = 8;
    const double a = hf.params[0];
    double* d = nullptr;
    FRES_TRY(dalloc(p, (void**)&d, sizeof(double) * 2 * (qs + qt)));
    launch_gauss_legendre(qs, d, d + qs, p->st);
    launch_gauss_legendre(qt, d + 2 * qs, d + 2 * qs + qt, p->st);
    std::vector<double> g(2 * (qs + qt));
    FRES_CK(cudaMemcpyAsync(g.data(), d, sizeof(double) * g.size(), cudaMemcpyDeviceToHost, p->st));
    FRES_CK(cudaStreamSynchronize(p->st));
    const double* ss = g.data();
    const double* ws = g.data() + qs;
    const double* tt = g.data() + 2 * qs;
    const double* wt = g.data() + 2 * qs + qt;
    const long long np = (long long)N * qs * qt;
    out->assign(3 * np, 0.0);
    double* X = out->data();
    double* Y = X + np;
    double* Wt = Y + np;
    long long j = 0;
    for (int k = 0; k < N; ++k) {
        const double phi = hf.motion[3 * k], tx = hf.motion[3 * k + 1], ty = hf.motion[3 * k + 2];
        const double cp = std::cos(phi), sp = std::sin(phi);
        for (int i = 0; i < qs; ++i) {
            const double th = kTwoPi * (k - 0.5 + ss[i]) / N;
            const double rx = a * std::cos(th), ry = a * std::sin(th);          // root - c
            const double dx = -a * std::sin(th) * kTwoPi / N, dy = a * std::cos(th) * kTwoPi / N;
            const double mx = rx * cp - ry * sp + tx, my = rx * sp + ry * cp + ty;   // M - c
            const double mdx = dx * cp - dy * sp, mdy = dx * sp + dy * cp;
            const double ptx = mx - rx, pty = my - ry;                             // dP/dt
            for (int l = 0; l < qt; ++l) {
                const double t = tt[l];
                const double psx = (1.0 - t) * dx + t * mdx, psy = (1.0 - t) * dy + t * mdy;
                X[j] = hf.cx + (1.0 - t) * rx + t * mx;
                Y[j] = hf.cy + (1.0 - t) * ry + t * my;
                Wt[j] = ws[i] * wt[l] * (ptx * psy - pty * psx);
                ++j;
            }
        }
    }
    return FRESNEL_OK;
}

template <typename T>
fresnel_status build_plan(Plan* p, const fresnel_problem* problems) {
    const bool dbl = sizeof(T) == 8;
    // ---------------- families: device copies, Gauss-Legendre rules, boundary rules
    long long off = 0;
    Bounds bb;
    for (int pb = 0; pb < p->B; ++pb)
    for (int fi = 0; fi < problems[pb].n_families; ++fi) {
        const fresnel_family& hf = problems[pb].families[fi];
        FamilyDev f{};
        f.prob = pb;
        long long nb = 0, nn = 0;
        int K = 0;
        FRES_TRY(validate_family(hf, &nb, &nn, &K));
        f.kind = hf.kind;
        f.n_panels = hf.n_panels;
        f.p = hf.p;
        f.m = hf.m;
        f.K = K;
        f.n_bdry = nb;
        f.n_nodes = nn;
        f.cx = hf.kind == FRESNEL_FAMILY_NODES ? 0.0 : hf.cx;
        f.cy = hf.kind == FRESNEL_FAMILY_NODES ? 0.0 : hf.cy;
        if (hf.kind == FRESNEL_FAMILY_NODES) {
            f.offset = off;
            off += nn;
            FRES_TRY(setup_nodes_family<T>(p, f, hf.params, hf.n_params, bb));
        } else if (hf.kind == FRESNEL_FAMILY_TRIANGLES) {
            f.offset = off;
            off += nn;
            FRES_TRY(setup_triangle_family(p, f, hf.params, hf.n_params, bb));
        } else if (hf.kind == FRESNEL_FAMILY_PETALS) {
            // the disc r < a: a FOURIER circle on the periodic trapezoid rule
            const int n_d = (int)hf.params[2], m_d = (int)hf.params[3];
            if (n_d > 0) {
                FamilyDev d{};
                d.prob = pb;
                d.kind = FRESNEL_FAMILY_FOURIER;
                d.ptr = 1;
                d.n_panels = n_d;
                d.p = 1;
                d.m = m_d;
                d.n_bdry = n_d;
                d.n_nodes = (long long)n_d * m_d;
                d.cx = hf.cx;
                d.cy = hf.cy;
                d.offset = off;
                off += d.n_nodes;
                FRES_TRY(setup_dilation_family<T>(p, d, hf.params, 1, bb));
                p->fams.push_back(d);
            }
            f.offset = off;
            off += nn;
            FRES_TRY(setup_petal_family(p, f, hf, bb));
            if (hf.motion) {   // root-arc patches, after the petals
                std::vector<double> pp;
                FRES_TRY(petal_patches(p, hf, &pp));
                FamilyDev pf{};
                pf.prob = pb;
                pf.kind = FRESNEL_FAMILY_NODES;
                pf.n_nodes = (long long)pp.size() / 3;
                p->fams.push_back(f);
                pf.offset = off;
                off += pf.n_nodes;
                FRES_TRY(setup_nodes_family<T>(p, pf, pp.data(), (long long)pp.size(), bb));
                p->fams.push_back(pf);
                continue;
            }
        } else {
            f.offset = off;
            off += nn;
            FRES_TRY(setup_dilation_family<T>(p, f, hf.params, hf.n_params, bb));
        }
        p->fams.push_back(f);
    }
    const double xmin = bb.xmin, xmax = bb.xmax, ymin = bb.ymin, ymax = bb.ymax;
    p->N = off;
    if (p->N < 1) return fres_fail(FRESNEL_ERR_ARG, "the quadrature has no nodes");
    if (p->N > (1LL << 30)) return fres_fail(FRESNEL_ERR_UNSUPPORTED, "more than 2^30 nodes");

    // ---------------- kernel and grids
    choose_kernel(p);
    const int w = p->ks.w;
    const double lz = p->lz;
    int cmax = 0;
    p->cp.kq = kPi / lz;
    p->cp.w = w;
    if (p->tkind == FRESNEL_GRID) {
        p->n1 = p->opts.grid_n1;
        p->n2 = p->opts.grid_n2;
        p->nf1 = nice_size(std::max({p->sigma * p->n1, 2.0 * w, 64.0}), kTile);
        p->nf2 = nice_size(std::max({p->sigma * p->n2, 2.0 * w, 64.0}), kTile);
        p->nfft1 = p->nf1;
        p->nfft2 = p->nf2;
        p->cp.type3 = 0;
        p->cp.u1 = p->opts.grid_h / lz;
        p->cp.u2 = p->opts.grid_h / lz;
        p->cp.a1 = kTwoPi * p->opts.grid_x0 / lz;
        p->cp.a2 = kTwoPi * p->opts.grid_y0 / lz;
        p->cp.a0 = 0.0;
    } else {
        const double* b = p->opts.box;
        double X1 = 0.5 * (xmax - xmin), X2 = 0.5 * (ymax - ymin);
        double C1 = 0.5 * (xmax + xmin), C2 = 0.5 * (ymax + ymin);
        X1 = std::max(X1, 1e-9 * std::max(1.0, std::fabs(C1)));
        X2 = std::max(X2, 1e-9 * std::max(1.0, std::fabs(C2)));
        double xic = 0.5 * (b[0] + b[1]), etac = 0.5 * (b[2] + b[3]);
        double S1 = kTwoPi * 0.5 * (b[1] - b[0]) / lz, S2 = kTwoPi * 0.5 * (b[3] - b[2]) / lz;
        S1 = std::max(S1, 1.0 / X1);
        S2 = std::max(S2, 1.0 / X2);
        const double sg = p->sigma;
        p->nf1 = nice_size(2.0 * sg * X1 * S1 / kPi + w + 2, kTile);
        p->nf2 = nice_size(2.0 * sg * X2 * S2 / kPi + w + 2, kTile);
        p->nfft1 = nice_size(sg * p->nf1, 2);
        p->nfft2 = nice_size(sg * p->nf2, 2);
        double hs1 = kPi / (sg * S1), hs2 = kPi / (sg * S2);
        double D1 = kTwoPi * xic / lz, D2 = kTwoPi * etac / lz;
        p->cp.type3 = 1;
        p->cp.C1 = C1;
        p->cp.C2 = C2;
        p->cp.inv_h1 = 1.0 / hs1;
        p->cp.inv_h2 = 1.0 / hs2;
        p->cp.a1 = D1;
        p->cp.a2 = D2;
        p->cp.a0 = D1 * C1 + D2 * C2;
        InterpParams& ip = p->ip;
        ip.xi_c = xic;
        ip.eta_c = etac;
        ip.K1 = hs1 * p->nfft1 / lz;
        ip.K2 = hs2 * p->nfft2 / lz;
        ip.sh1 = kTwoPi * hs1 / lz;
        ip.sh2 = kTwoPi * hs2 / lz;
        ip.kq = kPi / lz;
        ip.p1 = -kTwoPi * C1 / lz;
        ip.p2 = -kTwoPi * C2 / lz;
        ip.inv_lz = 1.0 / lz;
        for (int i = 0; i < 4; ++i) ip.box[i] = b[i];
        ip.nfft1 = p->nfft1;
        ip.nfft2 = p->nfft2;
        ip.nbin1 = (p->nfft1 + kTargetBin - 1) / kTargetBin;
        ip.nbin2 = (p->nfft2 + kTargetBin - 1) / kTargetBin;
        auto put = [](float* d, double v) {
            dflt s = df_host(v);
            d[0] = s.hi;
            d[1] = s.lo;
        };
        put(ip.dK1, ip.K1);
        put(ip.dK2, ip.K2);
        // grid coordinate in the fftshifted FFT grid, minus w/2
        put(ip.dG1, -xic * ip.K1 + 0.5 * p->nfft1 - 0.5 * w);
        put(ip.dG2, -etac * ip.K2 + 0.5 * p->nfft2 - 0.5 * w);
        put(ip.dkq, ip.kq);
        put(ip.dp1, ip.p1);
        put(ip.dp2, ip.p2);
        for (int i = 0; i < 4; ++i) ip.boxf[i] = (float)b[i];
        ip.shK1 = (float)(ip.sh1 / ip.K1);
        ip.shK2 = (float)(ip.sh2 / ip.K2);
        ip.occulter = p->output == FRESNEL_OCCULTER;
    }
    // FFT lengths: one shared-memory pass, or the four-step split
    for (FftDim* d : {&p->d1, &p->d2}) {
        d->n = d == &p->d1 ? p->nfft1 : p->nfft2;
        const bool forced = p->opts.fft_split_above > 0 && d->n > p->opts.fft_split_above;
        if (fft_supported(d->n, dbl, &cmax) && !forced) {
            d->fp = make_fft_plan(d->n, dbl ? 8 : 16);
        } else if (fft_split(d->n, dbl, &d->fa, &d->fb)) {
            d->big = true;
            d->fpa = make_fft_plan(d->fa, dbl ? 8 : 16);
            d->fpb = make_fft_plan(d->fb, dbl ? 8 : 16);
        } else {
            return fres_fail(FRESNEL_ERR_UNSUPPORTED, "FFT length " + std::to_string(d->n) +
                                                          " has no supported split");
        }
    }
    if ((p->d1.big || p->d2.big) && p->B > 1)
        return fres_fail(FRESNEL_ERR_UNSUPPORTED, "batched plans need single-pass FFT lengths");
    p->fp1 = p->d1.fp;
    p->fp2 = p->d2.fp;
    p->cp.nf1 = p->nf1;
    p->cp.nf2 = p->nf2;
    p->ntx = p->nf1 / kTile;
    p->nty = p->nf2 / kTile;
    p->ntiles = p->ntx * p->nty;
    p->cp.ntx = p->ntx;
    p->cp.nty = p->nty;
    p->cp.tile_base = 0;
    p->chunk_cap = dbl ? 256 : 512;
    if ((long long)p->B * p->ntiles >= (1LL << 31) ||
        (long long)p->B * p->nf1 * p->nf2 >= (1LL << 40))
        return fres_fail(FRESNEL_ERR_UNSUPPORTED, "batch too large");
    // per-problem chirp parameters: the grid is common, lambda z is not
    p->cps.assign(p->B, p->cp);
    for (int b = 0; b < p->B; ++b) {
        ChirpParams& c = p->cps[b];
        const double lzb = p->lzs[b];
        c.tile_base = b * p->ntiles;
        if (p->tkind == FRESNEL_GRID) {
            c.sh1 = p->nf1 / 2 + kTile / 2;   // x~ = 0 -> the middle of a tile
            c.sh2 = p->nf2 / 2 + kTile / 2;
            c.kq = kPi / lzb;
            c.u1 = p->opts.grid_h / lzb;
            c.u2 = p->opts.grid_h / lzb;
            c.a1 = kTwoPi * p->opts.grid_x0 / lzb;
            c.a2 = kTwoPi * p->opts.grid_y0 / lzb;
        }
    }

    // ---------------- FP32 fast mode: spoke coefficients and family constants
    if (!dbl) {
        for (FamilyDev& f : p->fams) {
            const ChirpParams& cp = p->cps[f.prob];
            if (f.kind == FRESNEL_FAMILY_NODES) continue;
            if (f.kind == FRESNEL_FAMILY_TRIANGLES) {   // double-float triangle tables
                const int np = f.p;
                std::vector<double> a(np), aw(np), wp(np);
                FRES_CK(cudaMemcpyAsync(a.data(), f.gl_m_a, sizeof(double) * np, cudaMemcpyDeviceToHost, p->st));
                FRES_CK(cudaMemcpyAsync(aw.data(), f.gl_m_aw, sizeof(double) * np, cudaMemcpyDeviceToHost, p->st));
                FRES_CK(cudaMemcpyAsync(wp.data(), f.gl_p_w, sizeof(double) * np, cudaMemcpyDeviceToHost, p->st));
                FRES_CK(cudaStreamSynchronize(p->st));
                std::vector<float> adf(2 * np), awf(np), wpf(np);
                for (int l = 0; l < np; ++l) {
                    const dflt d = df_host(a[l]);
                    adf[2 * l] = d.hi;
                    adf[2 * l + 1] = d.lo;
                    awf[l] = (float)aw[l];
                    wpf[l] = (float)wp[l];
                }
                FRES_TRY(dalloc(p, (void**)&f.adf, sizeof(float) * 2 * np));
                FRES_TRY(dalloc(p, (void**)&f.awf, sizeof(float) * np));
                FRES_TRY(dalloc(p, (void**)&f.wpf, sizeof(float) * np));
                FRES_TRY(dalloc(p, (void**)&f.tdf, sizeof(float) * 16 * (size_t)f.n_panels));
                FRES_CK(cudaMemcpyAsync(f.adf, adf.data(), sizeof(float) * 2 * np, cudaMemcpyHostToDevice, p->st));
                FRES_CK(cudaMemcpyAsync(f.awf, awf.data(), sizeof(float) * np, cudaMemcpyHostToDevice, p->st));
                FRES_CK(cudaMemcpyAsync(f.wpf, wpf.data(), sizeof(float) * np, cudaMemcpyHostToDevice, p->st));
                const double U1 = cp.type3 ? cp.inv_h1 : (double)cp.nf1 * cp.u1;
                const double U2 = cp.type3 ? cp.inv_h2 : (double)cp.nf2 * cp.u2;
                const double G0x = cp.type3 ? -cp.C1 * cp.inv_h1 + 0.5 * cp.nf1 - 0.5 * w
                                            : cp.sh1 - 0.5 * w;
                const double G0y = cp.type3 ? -cp.C2 * cp.inv_h2 + 0.5 * cp.nf2 - 0.5 * w
                                            : cp.sh2 - 0.5 * w;
                const double tk[5] = {cp.kq, -cp.a1, -cp.a2, U1, U2};
                for (int k = 0; k < 5; ++k) {
                    const dflt d = df_host(tk[k]);
                    f.tk[2 * k] = d.hi;
                    f.tk[2 * k + 1] = d.lo;
                }
                const dflt a0 = df_host(cp.a0), gx = df_host(G0x), gy = df_host(G0y);
                f.A0[0] = a0.hi;
                f.A0[1] = a0.lo;
                f.G0x[0] = gx.hi;
                f.G0x[1] = gx.lo;
                f.G0y[0] = gy.hi;
                f.G0y[1] = gy.lo;
                launch_boundary(f, cp, p->st);   // the per-triangle tables, once per plan
                FRES_CK(cudaStreamSynchronize(p->st));
                continue;
            }
            const double A0 = cp.kq * (f.cx * f.cx + f.cy * f.cy) - cp.a1 * f.cx - cp.a2 * f.cy + cp.a0;
            double G0x, G0y;
            if (!cp.type3) {
                G0x = (double)cp.nf1 * cp.u1 * f.cx - 0.5 * w + cp.sh1;
                G0y = (double)cp.nf2 * cp.u2 * f.cy - 0.5 * w + cp.sh2;
            } else {
                G0x = (f.cx - cp.C1) * cp.inv_h1 + 0.5 * cp.nf1 - 0.5 * w;
                G0y = (f.cy - cp.C2) * cp.inv_h2 + 0.5 * cp.nf2 - 0.5 * w;
            }
            if (f.kind == FRESNEL_FAMILY_PETALS) {
                FRES_TRY(dalloc(p, (void**)&f.ptab, sizeof(float) * 8 * f.n_bdry));
                FRES_TRY(dalloc(p, (void**)&f.pk, sizeof(float) * kPetalK * f.n_panels));
                // per petal: phase slopes E.d with E = 2 kq c_k - a, grid slopes
                // U d, and the constants at the petal's own centre c_k = c + t_k
                std::vector<double> rot(2 * f.n_panels), sh(2 * f.n_panels, 0.0);
                FRES_CK(cudaMemcpyAsync(rot.data(), f.rot, sizeof(double) * 2 * f.n_panels,
                                        cudaMemcpyDeviceToHost, p->st));
                if (f.shift)
                    FRES_CK(cudaMemcpyAsync(sh.data(), f.shift, sizeof(double) * 2 * f.n_panels,
                                            cudaMemcpyDeviceToHost, p->st));
                FRES_CK(cudaStreamSynchronize(p->st));
                const double U1 = cp.type3 ? cp.inv_h1 : (double)cp.nf1 * cp.u1;
                const double U2 = cp.type3 ? cp.inv_h2 : (double)cp.nf2 * cp.u2;
                std::vector<float> pk(kPetalK * f.n_panels);
                for (int k = 0; k < f.n_panels; ++k) {
                    const double c = rot[2 * k], sn = rot[2 * k + 1];
                    const double tx = sh[2 * k], ty = sh[2 * k + 1];
                    const double ckx = f.cx + tx, cky = f.cy + ty;
                    const double E1 = 2.0 * cp.kq * ckx - cp.a1, E2 = 2.0 * cp.kq * cky - cp.a2;
                    const double vals[9] = {c * E1 + sn * E2, c * E2 - sn * E1, c * U1, -sn * U1,
                                            sn * U2, c * U2,
                                            cp.kq * (ckx * ckx + cky * cky) - cp.a1 * ckx -
                                                cp.a2 * cky + cp.a0,
                                            G0x + U1 * tx, G0y + U2 * ty};
                    for (int v = 0; v < 9; ++v) {
                        const dflt d = df_host(vals[v]);
                        pk[kPetalK * k + 2 * v] = d.hi;
                        pk[kPetalK * k + 2 * v + 1] = d.lo;
                    }
                }
                FRES_CK(cudaMemcpyAsync(f.pk, pk.data(), sizeof(float) * kPetalK * f.n_panels,
                                        cudaMemcpyHostToDevice, p->st));
                FRES_CK(cudaStreamSynchronize(p->st));
            } else {
                FRES_TRY(dalloc(p, (void**)&f.spoke, sizeof(float) * 8 * f.n_bdry));
                FRES_TRY(dalloc(p, (void**)&f.bcf, sizeof(float) * f.n_bdry));
            }
            const dflt a0 = df_host(A0), gx = df_host(G0x), gy = df_host(G0y);
            f.A0[0] = a0.hi;
            f.A0[1] = a0.lo;
            f.G0x[0] = gx.hi;
            f.G0x[1] = gx.lo;
            f.G0y[0] = gy.hi;
            f.G0y[1] = gy.lo;
            launch_boundary(f, cp, p->st);   // spoke coefficients, once per plan
        }
    }

    // ---------------- source screen: samples in the plan's precision, k per problem
    if (p->opts.screen_n1 > 0) {
        const fresnel_opts& o = p->opts;
        const size_t ns = (size_t)o.screen_n1 * o.screen_n2;
        ScreenDev& sc = p->ft.scr;
        for (int k = 0; k < 2; ++k) {
            const double* src = k == 0 ? o.screen_amp : o.screen_opd;
            if (!src) continue;
            std::vector<T> h(src, src + ns);
            void* d = nullptr;
            FRES_TRY(dalloc(p, &d, sizeof(T) * ns));
            FRES_CK(cudaMemcpyAsync(d, h.data(), sizeof(T) * ns, cudaMemcpyHostToDevice, p->st));
            FRES_CK(cudaStreamSynchronize(p->st));
            (k == 0 ? sc.amp : sc.opd) = d;
        }
        sc.n1 = o.screen_n1;
        sc.n2 = o.screen_n2;
        sc.x0 = o.screen_box[0];
        sc.y0 = o.screen_box[2];
        sc.ihx = (o.screen_n1 - 1) / (o.screen_box[1] - o.screen_box[0]);
        sc.ihy = (o.screen_n2 - 1) / (o.screen_box[3] - o.screen_box[2]);
        for (int b = 0; b < p->B; ++b) p->cps[b].screen_k = kTwoPi / problems[b].lambda;
    }

    // ---------------- family table for the node and scatter launches
    {
        const int nfam = (int)p->fams.size();
        std::vector<int> blk0(nfam + 1, 0);
        for (int i = 0; i < nfam; ++i) {
            const long long nb = (p->fams[i].n_nodes + kNodeThreads - 1) / kNodeThreads;
            if ((long long)blk0[i] + nb >= (1LL << 31))
                return fres_fail(FRESNEL_ERR_UNSUPPORTED, "too many nodes for one launch");
            blk0[i + 1] = blk0[i] + (int)nb;
        }
        FamilyDev* d_f = nullptr;
        ChirpParams* d_c = nullptr;
        int* d_b = nullptr;
        FRES_TRY(dalloc(p, (void**)&d_f, sizeof(FamilyDev) * nfam));
        FRES_TRY(dalloc(p, (void**)&d_c, sizeof(ChirpParams) * p->B));
        FRES_TRY(dalloc(p, (void**)&d_b, sizeof(int) * (nfam + 1)));
        FRES_CK(cudaMemcpyAsync(d_f, p->fams.data(), sizeof(FamilyDev) * nfam, cudaMemcpyHostToDevice, p->st));
        FRES_CK(cudaMemcpyAsync(d_c, p->cps.data(), sizeof(ChirpParams) * p->B, cudaMemcpyHostToDevice, p->st));
        FRES_CK(cudaMemcpyAsync(d_b, blk0.data(), sizeof(int) * (nfam + 1), cudaMemcpyHostToDevice, p->st));
        FRES_CK(cudaStreamSynchronize(p->st));
        p->ft.fams = d_f;
        p->ft.cps = d_c;
        p->ft.blk0 = d_b;
        p->ft.nfam = nfam;
        p->node_blocks = blk0[nfam];
    }

    // ---------------- node pass once: exact record / chunk / slot counts
    FRES_TRY(dalloc(p, (void**)&p->status, sizeof(unsigned)));
    FRES_CK(cudaMemsetAsync(p->status, 0, sizeof(unsigned), p->st));
    FRES_TRY(dalloc(p, &p->rec, p->rsize() * p->N));
    const long long tt = (long long)p->B * p->ntiles;
    FRES_TRY(dalloc(p, (void**)&p->counts, sizeof(int) * tt));
    FRES_TRY(dalloc(p, (void**)&p->cursor, sizeof(int) * tt));
    FRES_TRY(dalloc(p, (void**)&p->work, 2 * sizeof(int)));
    FRES_CK(cudaMemsetAsync(p->counts, 0, sizeof(int) * tt, p->st));
    FRES_CK(cudaMemsetAsync(p->work, 0, 2 * sizeof(int), p->st));
    FRES_TRY(run_nodes<T>(p, nullptr, nullptr, nullptr));
    std::vector<int> hc(tt);
    FRES_CK(cudaMemcpyAsync(hc.data(), p->counts, sizeof(int) * tt, cudaMemcpyDeviceToHost, p->st));
    FRES_CK(cudaStreamSynchronize(p->st));
    FRES_CK(cudaGetLastError());
    // chunk cap: tiles with more records are split into chunks that run in
    // parallel and add into the tile with global atomics.  A cap of about the
    // records per eight chunks per resident spreading block keeps the load
    // balanced; when every tile is heavily loaded (N >> nf1 nf2: the Koch
    // snowflake's 67M nodes on a 2048^2 grid) a larger cap saves most of the
    // atomic tile additions.  Small plans keep the base cap.
    {
        long long total = 0;
        for (int c : hc) {
            total += c;
            p->det_tmax = std::max(p->det_tmax, c);
        }
        if (p->opts.deterministic && p->det_tmax >= kDetMaxTileRecords)
            return fres_fail(FRESNEL_ERR_UNSUPPORTED,
                             "deterministic mode: a spreading tile holds 2^23 or more records");
        const long long slots = 152LL * 4 * 8;
        const long long base = p->chunk_cap;
        p->chunk_cap = (int)std::max(base, std::min(total / slots, 1LL << 20));
    }
    // per-problem regions: every problem's split chunks, then its plain tiles
    std::vector<int> sc_off(p->B + 1, 0), pl_off(p->B + 1, 0), st_off(p->B + 1, 0);
    std::vector<long long> rec_off(p->B + 1, 0);
    // type 1: tile rows without records are neither spread nor transformed
    // (the four-step FFT path reads every row, so it keeps them all)
    const bool prune = p->tkind == FRESNEL_GRID && !p->d1.big && !p->d2.big;
    if (prune && p->nty > kMaxTileRows)
        return fres_fail(FRESNEL_ERR_UNSUPPORTED, "spreading grid too tall");
    int max_live_rows = 0;   // live tile rows of the fullest problem
    p->live_rows_total = 0;
    std::vector<int> rows;   // the row pass's work list (pruned plans)
    for (int b = 0; b < p->B; ++b) {
        long long nrec = 0, nsc = 0, nsplit = 0, nlive = 0;
        std::vector<char> live(p->nty, prune ? 0 : 1);
        for (int i = 0; i < p->ntiles; ++i)
            if (hc[(size_t)b * p->ntiles + i] > 0) live[i / p->ntx] = 1;
        for (int r = 0; r < p->nty; ++r) nlive += live[r] ? p->ntx : 0;
        int lr = 0;
        for (int r = 0; r < p->nty; ++r) lr += live[r] ? 1 : 0;
        max_live_rows = std::max(max_live_rows, lr);
        p->live_rows_total += lr;
        if (prune)
            for (int r = 0; r < p->nty; ++r)
                if (live[r])
                    for (int i = 0; i < kTile; ++i) rows.push_back(b * p->nf2 + r * kTile + i);
        for (int i = 0; i < p->ntiles; ++i) {
            const int c = hc[(size_t)b * p->ntiles + i];
            nrec += c;
            if (c > p->chunk_cap) {
                nsc += (c + p->chunk_cap - 1) / p->chunk_cap;
                ++nsplit;
            }
        }
        if (sc_off[b] + nsc + (long long)p->B * p->ntiles >= (1LL << 31) ||
            rec_off[b] + nrec >= (1LL << 31))
            return fres_fail(FRESNEL_ERR_UNSUPPORTED, "more than 2^31 records or chunks");
        sc_off[b + 1] = sc_off[b] + (int)nsc;
        st_off[b + 1] = st_off[b] + (int)nsplit;
        pl_off[b + 1] = pl_off[b] + (int)(nlive - nsplit);
        rec_off[b + 1] = rec_off[b] + nrec;
    }
    for (int b = 0; b <= p->B; ++b) pl_off[b] += sc_off[p->B];
    // narrow live band: the direct column DFT costs R complex multiply-adds
    // (4 FMA) per kept output, R n2 per column, against ~150 instructions per
    // point of the nf2-point transform (measured over three radix stages):
    // direct when R n2 <= 24 nf2 (e.g. one live tile row, 512 of 1024 modes)
    {
        p->max_live_rows = max_live_rows;
        const long long R = (long long)kTile * max_live_rows;
        p->col_dft = prune && R > 0 && R <= kDftMaxRows && R * p->n2 <= 24LL * p->nf2;
    }
    if (prune && !rows.empty() && (long long)p->nf2 * p->B < (1LL << 31)) {
        FRES_TRY(dalloc(p, (void**)&p->row_list, sizeof(int) * rows.size()));
        FRES_CK(cudaMemcpyAsync(p->row_list, rows.data(), sizeof(int) * rows.size(),
                                cudaMemcpyHostToDevice, p->st));
        p->n_row_list = (int)rows.size();
    }
    p->n_records = rec_off[p->B];
    p->max_chunks = pl_off[p->B];
    p->max_split = st_off[p->B];
    FRES_TRY(dalloc(p, &p->sorted, p->rsize() * std::max(1LL, p->n_records)));
    FRES_TRY(dalloc(p, (void**)&p->chunks, sizeof(Chunk) * p->max_chunks));
    FRES_TRY(dalloc(p, (void**)&p->n_meta, 2 * sizeof(int)));
    FRES_TRY(dalloc(p, (void**)&p->split_tiles, sizeof(int) * std::max(1, p->max_split)));
    FRES_TRY(dalloc(p, (void**)&p->ready, sizeof(int) * std::max(1, p->max_split)));
    FRES_CK(cudaMemsetAsync(p->ready, 0, sizeof(int) * std::max(1, p->max_split), p->st));
    if (p->opts.deterministic) {
        const size_t acc = sizeof(unsigned long long) * 4 * kTile * kTile * std::max(1, p->max_split);
        FRES_TRY(dalloc(p, (void**)&p->det_acc, acc));
        FRES_CK(cudaMemsetAsync(p->det_acc, 0, acc, p->st));
        FRES_TRY(dalloc(p, (void**)&p->det_part, sizeof(double) * kDetPartials));
    }
    {
        int* d_sc = nullptr;
        int* d_pl = nullptr;
        int* d_st = nullptr;
        long long* d_ro = nullptr;
        const size_t nb1 = (size_t)p->B + 1;
        FRES_TRY(dalloc(p, (void**)&d_sc, sizeof(int) * nb1));
        FRES_TRY(dalloc(p, (void**)&d_pl, sizeof(int) * nb1));
        FRES_TRY(dalloc(p, (void**)&d_st, sizeof(int) * nb1));
        FRES_TRY(dalloc(p, (void**)&d_ro, sizeof(long long) * nb1));
        FRES_CK(cudaMemcpyAsync(d_sc, sc_off.data(), sizeof(int) * nb1, cudaMemcpyHostToDevice, p->st));
        FRES_CK(cudaMemcpyAsync(d_pl, pl_off.data(), sizeof(int) * nb1, cudaMemcpyHostToDevice, p->st));
        FRES_CK(cudaMemcpyAsync(d_st, st_off.data(), sizeof(int) * nb1, cudaMemcpyHostToDevice, p->st));
        FRES_CK(cudaMemcpyAsync(d_ro, rec_off.data(), sizeof(long long) * nb1, cudaMemcpyHostToDevice, p->st));
        const int meta[2] = {p->max_chunks, p->max_split};
        FRES_CK(cudaMemcpyAsync(p->n_meta, meta, sizeof(meta), cudaMemcpyHostToDevice, p->st));
        FRES_CK(cudaStreamSynchronize(p->st));
        p->layout.sc_off = d_sc;
        p->layout.pl_off = d_pl;
        p->layout.st_off = d_st;
        p->layout.rec_off = d_ro;
        p->layout.ntx = p->ntx;
        p->layout.nty = p->nty;
        p->layout.live = nullptr;
        if (prune) {
            FRES_TRY(dalloc(p, (void**)&p->layout.live, sizeof(int) * p->nty * (size_t)p->B));
            FRES_CK(cudaMemsetAsync(p->layout.live, 0, sizeof(int) * p->nty * (size_t)p->B, p->st));
        }
    }
    FRES_TRY(run_sort<T>(p));
    p->nodes_ready = true;
    p->spread_blocks = 152 * 8;

    // ---------------- grids and tables
    const size_t cs = p->csize();
    FRES_TRY(dalloc(p, &p->grid, cs * (size_t)p->nf1 * p->nf2 * p->B));
    // kernel-transform quadrature: Gauss-Legendre on (0,1) with 2w + 16 points
    p->gq_n = std::min(64, 2 * w + 16);
    FRES_TRY(dalloc(p, (void**)&p->gq_t, sizeof(double) * p->gq_n));
    FRES_TRY(dalloc(p, (void**)&p->gq_w, sizeof(double) * p->gq_n));
    launch_gauss_legendre(p->gq_n, p->gq_t, p->gq_w, p->st);
    for (FftDim* d : {&p->d1, &p->d2}) {
        FRES_TRY(dalloc(p, &d->tw, cs * d->n));
        launch_twiddles(d->n, d->tw, dbl, p->st);
        if (d->big) {
            FRES_TRY(dalloc(p, &d->twa, cs * d->fa));
            launch_twiddles(d->fa, d->twa, dbl, p->st);
            FRES_TRY(dalloc(p, &d->twb, cs * d->fb));
            launch_twiddles(d->fb, d->twb, dbl, p->st);
        }
    }
    p->tw1 = p->d1.tw;
    p->tw2 = p->d2.tw;
    if (p->d1.big || p->d2.big) {   // four-step intermediate, shared by both passes
        const size_t rows = p->d1.big ? (size_t)p->nf2 * p->d1.n : 0;
        const size_t ncol = p->tkind == FRESNEL_GRID ? (size_t)p->n1 : (size_t)p->nfft1;
        const size_t cols = p->d2.big ? (size_t)p->d2.n * ncol : 0;
        FRES_TRY(dalloc(p, &p->fscratch, cs * std::max(rows, cols)));
    }
    if (p->tkind == FRESNEL_GRID) {
        FRES_TRY(dalloc(p, &p->inter, cs * (size_t)p->nf2 * p->n1 * p->B));
        FRES_TRY(dalloc(p, &p->ax, cs * p->n1 * p->B));
        FRES_TRY(dalloc(p, &p->ay, cs * p->n2 * p->B));
        for (int b = 0; b < p->B; ++b) {   // per problem: the chirp depends on lambda z
            launch_t1_tables(p->n1, p->nf1, p->opts.grid_h, p->opts.grid_x0, p->lzs[b], w,
                             p->ks.beta, 1, p->cps[b].sh1, (char*)p->ax + cs * p->n1 * b, dbl,
                             p->gq_t, p->gq_w, p->gq_n, p->st);
            launch_t1_tables(p->n2, p->nf2, p->opts.grid_h, p->opts.grid_y0, p->lzs[b], w,
                             p->ks.beta, 0, p->cps[b].sh2, (char*)p->ay + cs * p->n2 * b, dbl,
                             p->gq_t, p->gq_w, p->gq_n, p->st);
        }
    } else {
        FRES_TRY(dalloc(p, &p->inter, cs * (size_t)p->nf2 * p->nfft1));
        FRES_TRY(dalloc(p, &p->F, cs * (size_t)p->nfft2 * p->nfft1));
        const size_t rs = dbl ? 8 : 4;
        FRES_TRY(dalloc(p, &p->dec1, rs * p->nf1));
        FRES_TRY(dalloc(p, &p->dec2, rs * p->nf2));
        launch_t3_deconv(p->nf1, p->nfft1, w, p->ks.beta, p->dec1, dbl, p->gq_t, p->gq_w, p->gq_n, p->st);
        launch_t3_deconv(p->nf2, p->nfft2, w, p->ks.beta, p->dec2, dbl, p->gq_t, p->gq_w, p->gq_n, p->st);
        // Even Chebyshev series of psihat on [-t_max, t_max], t = (xi - xi_c) * sh.
        const double* b = p->opts.box;
        double tmax = std::max(0.5 * (b[1] - b[0]) * p->ip.sh1, 0.5 * (b[3] - b[2]) * p->ip.sh2);
        tmax = std::max(tmax * (1.0 + 1e-12), 1e-3);
        const int ns = kMaxCheb;
        double* d_s = nullptr;
        FRES_TRY(dalloc(p, (void**)&d_s, sizeof(double) * ns));
        launch_cheb_samples(ns, tmax, w, p->ks.beta, p->gq_t, p->gq_w, p->gq_n, d_s, p->st);
        std::vector<double> hs(ns), a(ns);
        FRES_CK(cudaMemcpyAsync(hs.data(), d_s, sizeof(double) * ns, cudaMemcpyDeviceToHost, p->st));
        FRES_CK(cudaStreamSynchronize(p->st));
        for (int j = 0; j < ns; ++j) {        // a_j = c_{2j}
            double acc = 0.0;
            for (int i = 0; i < ns; ++i) acc += hs[i] * std::cos(2.0 * j * kPi * (i + 0.5) / (2.0 * ns));
            a[j] = (j == 0 ? 1.0 : 2.0) * acc / ns;
        }
        // The coefficients fall geometrically to a roundoff plateau (~1e-16 of
        // a_0); the series ends at the first term below the arithmetic's
        // resolution (FP32 1e-10, FP64 1e-15): 9 and 11 terms for w = 8.
        const double cut = dbl ? 1e-15 : 1e-10;
        int nk = 1;
        while (nk < ns && std::fabs(a[nk]) >= cut * std::fabs(a[0])) ++nk;
        FRES_CK(cudaMemcpyAsync(d_s, a.data(), sizeof(double) * nk, cudaMemcpyHostToDevice, p->st));
        FRES_CK(cudaStreamSynchronize(p->st));
        p->cheb = d_s;
        p->ncheb = nk;
        const int nbins = p->ip.nbin1 * p->ip.nbin2;
        FRES_TRY(dalloc(p, (void**)&p->tpartial,
                        sizeof(int) * (size_t)((nbins + kBinChunk - 1) / kBinChunk)));
        FRES_TRY(dalloc(p, (void**)&p->tcounts, sizeof(int) * nbins));
        FRES_TRY(dalloc(p, (void**)&p->tstart, sizeof(int) * nbins));
        FRES_TRY(dalloc(p, (void**)&p->tcursor, sizeof(int) * nbins));
        FRES_TRY(dalloc(p, (void**)&p->twork, 2 * sizeof(int)));
        if (!dbl) {
            FRES_CK(cudaStreamCreateWithFlags(&p->sort_st, cudaStreamNonBlocking));
            FRES_CK(cudaEventCreateWithFlags(&p->ev_sort_fork, cudaEventDisableTiming));
            FRES_CK(cudaEventCreateWithFlags(&p->ev_sorted, cudaEventDisableTiming));
        }
        FRES_CK(cudaMemsetAsync(p->tcounts, 0, sizeof(int) * nbins, p->st));
        FRES_CK(cudaMemsetAsync(p->twork, 0, 2 * sizeof(int), p->st));
        p->ip.inv_tmax = 1.0 / tmax;
    }
    FRES_CK(cudaGetLastError());
    FRES_CK(cudaStreamSynchronize(p->st));
    return read_status(p);
}

Plan* as_plan(fresnel_plan_t h) {
    Plan* p = reinterpret_cast<Plan*>(h);
    if (!p || p->magic != kMagic) return nullptr;
    return p;
}

}  // namespace

struct fresnel_plan_s {};   // opaque handle type; the handle points at a Plan

namespace {
// The adjoint transform shared by the profile and shape gradients:
// btilde = FFT(sgn conj(gamma) ax ay) on the plan's spreading grid.
template <typename T>
fresnel_status adjoint_grid(Plan* p, const void* d_gamma) {
    const size_t cs = p->csize();
    if (!p->adj_in) {
        FRES_TRY(dalloc(p, &p->adj_in, cs * (size_t)p->n1 * p->n2 * p->B));
        FRES_TRY(dalloc(p, &p->adj_rows, cs * (size_t)p->n2 * p->nf1 * p->B));
        FRES_TRY(dalloc(p, (void**)&p->contrib, sizeof(double) * p->N));
    }
    launch_adj_prologue<T>(d_gamma, p->ax, p->ay, p->adj_in, p->n1, p->n2, p->B,
                           p->output == FRESNEL_OCCULTER, p->st);
    RowPassArgs ra{};
    ra.in = p->adj_in;
    ra.out = p->adj_rows;
    ra.in_stride = p->n1;
    ra.out_stride = p->nf1;
    ra.nrows = p->n2 * p->B;
    ra.in_len = p->n1;
    ra.centered_in = 1;
    ra.out_len = p->nf1;
    ra.twiddle = p->tw1;
    launch_fft_rows<T>(p->fp1, ra, p->st);
    ColPassArgs ca{};
    ca.in = p->adj_rows;
    ca.out = p->grid;
    ca.ncols = p->nf1;
    ca.in_len = p->n2;
    ca.centered_in = 1;
    ca.out_len = p->nf2;
    ca.twiddle = p->tw2;
    ca.out_is_final = 0;
    ca.batch = p->B;
    ca.in_bstride = (long long)p->n2 * p->nf1;
    ca.out_bstride = (long long)p->nf2 * p->nf1;
    launch_fft_cols<T>(p->fp2, ca, p->st);
    return FRESNEL_OK;
}

template <typename T>
fresnel_status grad_shape_impl(Plan* p, const void* d_gamma, double* d_grad) {
    if (!p->shape_ready) {
        std::vector<int> sf;
        std::vector<long long> bofs, gofs;
        long long boff = 0, goff = 0;
        int maxp = 0;
        for (int i = 0; i < (int)p->fams.size(); ++i) {
            const FamilyDev& f = p->fams[i];
            if (f.kind != FRESNEL_FAMILY_FOURIER || f.ptr) continue;
            sf.push_back(i);
            bofs.push_back(boff);
            gofs.push_back(goff);
            boff += f.n_bdry;
            goff += 1 + 2 * f.K;
            maxp = std::max(maxp, 1 + 2 * f.K);
        }
        const size_t nf = std::max<size_t>(1, sf.size());
        FRES_TRY(dalloc(p, (void**)&p->sf, sizeof(int) * nf));
        FRES_TRY(dalloc(p, (void**)&p->sbofs, sizeof(long long) * nf));
        FRES_TRY(dalloc(p, (void**)&p->sgofs, sizeof(long long) * nf));
        FRES_TRY(dalloc(p, (void**)&p->rbuf, sizeof(double) * std::max<long long>(1, boff)));
        if (!sf.empty()) {
            FRES_CK(cudaMemcpyAsync(p->sf, sf.data(), sizeof(int) * sf.size(), cudaMemcpyHostToDevice, p->st));
            FRES_CK(cudaMemcpyAsync(p->sbofs, bofs.data(), sizeof(long long) * sf.size(),
                                    cudaMemcpyHostToDevice, p->st));
            FRES_CK(cudaMemcpyAsync(p->sgofs, gofs.data(), sizeof(long long) * sf.size(),
                                    cudaMemcpyHostToDevice, p->st));
        }
        FRES_CK(cudaStreamSynchronize(p->st));
        p->nsf = (int)sf.size();
        p->n_sgrad = goff;
        p->n_sbdry = boff;
        p->max_params = maxp;
        p->shape_ready = true;
    }
    FRES_TRY(adjoint_grid<T>(p, d_gamma));
    launch_adj_nodes<T>(p->ft, p->node_blocks, p->grid, p->nf1, p->nf2, p->ks, p->contrib, 1, p->st);
    launch_adj_shape_reduce(p->ft.fams, p->sf, p->nsf, p->max_params, p->n_sbdry, p->sbofs,
                            p->sgofs, p->contrib, p->rbuf, d_grad, p->st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fres_fail(FRESNEL_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return FRESNEL_OK;
}

template <typename T>
fresnel_status grad_profile_impl(Plan* p, const void* d_gamma, double* d_grad) {
    if (!p->pf) {
        std::vector<int> pf;
        std::vector<long long> gofs;
        long long off = 0;
        for (int i = 0; i < (int)p->fams.size(); ++i)
            if (p->fams[i].kind == FRESNEL_FAMILY_PETALS) {
                pf.push_back(i);
                gofs.push_back(off);
                off += p->fams[i].n_prof;
            }
        FRES_TRY(dalloc(p, (void**)&p->pf, sizeof(int) * std::max<size_t>(1, pf.size())));
        FRES_TRY(dalloc(p, (void**)&p->gofs, sizeof(long long) * std::max<size_t>(1, gofs.size())));
        if (!pf.empty()) {
            FRES_CK(cudaMemcpyAsync(p->pf, pf.data(), sizeof(int) * pf.size(), cudaMemcpyHostToDevice, p->st));
            FRES_CK(cudaMemcpyAsync(p->gofs, gofs.data(), sizeof(long long) * gofs.size(),
                                    cudaMemcpyHostToDevice, p->st));
        }
        FRES_CK(cudaStreamSynchronize(p->st));
        p->npf = (int)pf.size();
        p->n_grad = off;
    }
    if (p->n_grad > 0) FRES_CK(cudaMemsetAsync(d_grad, 0, sizeof(double) * p->n_grad, p->st));
    FRES_TRY(adjoint_grid<T>(p, d_gamma));
    launch_adj_nodes<T>(p->ft, p->node_blocks, p->grid, p->nf1, p->nf2, p->ks, p->contrib, 0, p->st);
    launch_adj_reduce(p->ft.fams, p->pf, p->gofs, p->npf, p->contrib, d_grad, p->st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fres_fail(FRESNEL_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return FRESNEL_OK;
}

}  // namespace

namespace {
// A scattered-target batch: one sub-plan per problem (each sized for its own
// aperture and lambda z; all with the opts box), internal streams and events
// for the graph that evaluates them together.
fresnel_status plan_scattered_batch(const fresnel_problem* problems, int n, double tol,
                                    const fresnel_opts* opts, void* stream,
                                    fresnel_plan_t* out_plan);
fresnel_status read_batch_status(Plan* p);
fresnel_status plan_autotuned(const fresnel_problem* problems, int n, double tol,
                              const fresnel_opts* opts, void* stream, fresnel_plan_t* out_plan);
}  // namespace

extern "C" {

void fresnel_default_opts(fresnel_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = FRESNEL_FP32_FAST;
    o->output = FRESNEL_APERTURE;
    o->target_kind = FRESNEL_GRID;
    o->grid_n1 = o->grid_n2 = 100;
    o->grid_h = 0.03;
    o->box[0] = o->box[2] = -1.0;
    o->box[1] = o->box[3] = 1.0;
    o->sync_status = 1;
}

fresnel_status fresnel_plan_many(const fresnel_problem* problems, int n_problems, double tol,
                                 const fresnel_opts* opts, void* cuda_stream,
                                 fresnel_plan_t* out_plan) {
    if (!out_plan) return fres_fail(FRESNEL_ERR_ARG, "out_plan is NULL");
    *out_plan = nullptr;
    if (!problems || n_problems < 1) return fres_fail(FRESNEL_ERR_ARG, "no problems");
    if (n_problems > (1 << 20)) return fres_fail(FRESNEL_ERR_UNSUPPORTED, "more than 2^20 problems");
    for (int b = 0; b < n_problems; ++b) {
        const fresnel_problem& q = problems[b];
        if (!q.families || q.n_families < 1) return fres_fail(FRESNEL_ERR_ARG, "no families");
        const double lambda = q.lambda, z = q.z;
        if (!(lambda > 0) || !(z > 0) || !std::isfinite(lambda) || !std::isfinite(z) ||
            !std::isfinite(lambda * z) || !(lambda * z > 0))
            return fres_fail(FRESNEL_ERR_ARG, "lambda and z must be finite and > 0");
    }
    if (!opts) return fres_fail(FRESNEL_ERR_ARG, "opts is NULL");
    if (!(tol >= 1e-14 && tol <= 1e-1)) return fres_fail(FRESNEL_ERR_ARG, "tol must lie in [1e-14, 1e-1]");
    if (opts->precision != FRESNEL_FP64 && opts->precision != FRESNEL_FP32_FAST)
        return fres_fail(FRESNEL_ERR_ARG, "unknown precision");
    if (opts->precision == FRESNEL_FP32_FAST && tol < 1e-7)
        return fres_fail(FRESNEL_ERR_UNSUPPORTED, "FP32 fast mode reaches tol >= 1e-7 only; use FRESNEL_FP64");
    if (opts->output != FRESNEL_APERTURE && opts->output != FRESNEL_OCCULTER)
        return fres_fail(FRESNEL_ERR_ARG, "unknown output");
    if (opts->target_kind == FRESNEL_GRID) {
        if (opts->grid_n1 < 1 || opts->grid_n2 < 1 || !(opts->grid_h > 0) ||
            !std::isfinite(opts->grid_h) || !std::isfinite(opts->grid_x0) ||
            !std::isfinite(opts->grid_y0))
            return fres_fail(FRESNEL_ERR_ARG, "grid needs n1, n2 >= 1 and finite h > 0, x0, y0");
    } else if (opts->target_kind == FRESNEL_SCATTERED) {
        const double* b = opts->box;
        for (int i = 0; i < 4; ++i)
            if (!std::isfinite(b[i])) return fres_fail(FRESNEL_ERR_ARG, "box must be finite");
        if (!(b[0] <= b[1]) || !(b[2] <= b[3])) return fres_fail(FRESNEL_ERR_ARG, "box must have min <= max");
    } else {
        return fres_fail(FRESNEL_ERR_ARG, "unknown target_kind");
    }
    if (opts->sigma != 0 && !(opts->sigma >= 1.2 && opts->sigma <= 4.0))
        return fres_fail(FRESNEL_ERR_ARG, "sigma must be 0 (auto) or in [1.2, 4]");
    if (opts->kernel_w < 0 || opts->kernel_w == 1 || opts->kernel_w > kMaxW)
        return fres_fail(FRESNEL_ERR_ARG, "kernel_w must be 0 (auto) or in [2, 16]");
    if (opts->t3_binning < -1 || opts->t3_binning > 1)
        return fres_fail(FRESNEL_ERR_ARG, "t3_binning must be -1, 0 or 1");
    if (opts->fft_split_above < 0)
        return fres_fail(FRESNEL_ERR_ARG, "fft_split_above must be >= 0");
    if (!(opts->nsli_far >= 0.0) || !std::isfinite(opts->nsli_far))
        return fres_fail(FRESNEL_ERR_ARG, "nsli_far must be finite and >= 0");
    if (opts->screen_n1 || opts->screen_n2 || opts->screen_amp || opts->screen_opd) {
        const double* bx = opts->screen_box;
        if (opts->screen_n1 < 4 || opts->screen_n2 < 4)
            return fres_fail(FRESNEL_ERR_ARG, "a screen needs at least 4 x 4 samples");
        if (!opts->screen_amp && !opts->screen_opd)
            return fres_fail(FRESNEL_ERR_ARG, "a screen needs screen_amp and/or screen_opd");
        if ((long long)opts->screen_n1 * opts->screen_n2 > (1LL << 28))
            return fres_fail(FRESNEL_ERR_UNSUPPORTED, "screen larger than 2^28 samples");
        for (int i = 0; i < 4; ++i)
            if (!std::isfinite(bx[i])) return fres_fail(FRESNEL_ERR_ARG, "screen_box not finite");
        if (!(bx[1] > bx[0]) || !(bx[3] > bx[2]))
            return fres_fail(FRESNEL_ERR_ARG, "screen_box must have box[1] > box[0], box[3] > box[2]");
    }
    int dev = 0;
    FRES_CK(cudaGetDevice(&dev));
    if (opts->target_kind == FRESNEL_SCATTERED && n_problems > 1)
        return plan_scattered_batch(problems, n_problems, tol, opts, cuda_stream, out_plan);
    if (opts->autotune)
        return plan_autotuned(problems, n_problems, tol, opts, cuda_stream, out_plan);
    Plan* p = new Plan();
    p->prec = opts->precision;
    p->output = opts->output;
    p->tkind = opts->target_kind;
    p->B = n_problems;
    for (int b = 0; b < n_problems; ++b) p->lzs.push_back(problems[b].lambda * problems[b].z);
    p->lz = p->lzs[0];
    p->tol = tol;
    p->st = (cudaStream_t)cuda_stream;
    p->opts = *opts;
    fresnel_status s = p->prec == FRESNEL_FP64 ? build_plan<double>(p, problems)
                                               : build_plan<float>(p, problems);
    if (s != FRESNEL_OK) {
        std::string msg = g_last_error;
        cudaGetLastError();
        free_plan(p);
        g_last_error = msg;
        return s;
    }
    *out_plan = reinterpret_cast<fresnel_plan_t>(p);
    return FRESNEL_OK;
}

fresnel_status fresnel_plan(const fresnel_family* families, int n_families, double lambda,
                            double z, double tol, const fresnel_opts* opts, void* cuda_stream,
                            fresnel_plan_t* out_plan) {
    fresnel_problem one{families, n_families, lambda, z};
    return fresnel_plan_many(&one, 1, tol, opts, cuda_stream, out_plan);
}

fresnel_status fresnel_eval_many(fresnel_plan_t plan, void* d_out) {
    Plan* p = as_plan(plan);
    if (!p) return fres_fail(FRESNEL_ERR_ARG, "invalid plan handle");
    if (p->tkind != FRESNEL_GRID) return fres_fail(FRESNEL_ERR_ARG, "fresnel_eval_many needs a GRID plan");
    if (!d_out) return fres_fail(FRESNEL_ERR_ARG, "d_out is NULL");
    const long long M = (long long)p->n1 * p->n2;
    fresnel_status s = p->prec == FRESNEL_FP64 ? eval_impl<double>(p, nullptr, M, d_out)
                                               : eval_impl<float>(p, nullptr, M, d_out);
    if (s != FRESNEL_OK) return s;
    if (p->opts.sync_status) return read_status(p);
    return FRESNEL_OK;
}

fresnel_status fresnel_eval(fresnel_plan_t plan, const double* d_targets, long long M, void* d_out) {
    Plan* p = as_plan(plan);
    if (!p) return fres_fail(FRESNEL_ERR_ARG, "invalid plan handle");
    if (p->B != 1) return fres_fail(FRESNEL_ERR_ARG, "plan has several problems: use fresnel_eval_many");
    if (p->tkind == FRESNEL_GRID) {
        if (M != (long long)p->n1 * p->n2)
            return fres_fail(FRESNEL_ERR_ARG, "GRID plan: M must equal n1 * n2");
    } else {
        if (M < 0) return fres_fail(FRESNEL_ERR_ARG, "M must be >= 0");
        if (M > 0 && !d_targets) return fres_fail(FRESNEL_ERR_ARG, "d_targets is NULL");
    }
    if (M > 0 && !d_out) return fres_fail(FRESNEL_ERR_ARG, "d_out is NULL");
    fresnel_status s = p->prec == FRESNEL_FP64 ? eval_impl<double>(p, d_targets, M, d_out)
                                               : eval_impl<float>(p, d_targets, M, d_out);
    if (s != FRESNEL_OK) return s;
    if (p->opts.sync_status) return read_status(p);
    return FRESNEL_OK;
}

fresnel_status fresnel_eval_host(fresnel_plan_t plan, const double* h_targets, long long M,
                                 void* h_out) {
    Plan* p = as_plan(plan);
    if (!p) return fres_fail(FRESNEL_ERR_ARG, "invalid plan handle");
    if (p->B != 1) return fres_fail(FRESNEL_ERR_ARG, "plan has several problems: use fresnel_eval_many");
    if (M < 0) return fres_fail(FRESNEL_ERR_ARG, "M must be >= 0");
    if (M > 0 && !h_out) return fres_fail(FRESNEL_ERR_ARG, "h_out is NULL");
    if (p->tkind == FRESNEL_SCATTERED && M > 0 && !h_targets)
        return fres_fail(FRESNEL_ERR_ARG, "h_targets is NULL");
    if (p->tkind == FRESNEL_GRID && M != (long long)p->n1 * p->n2)
        return fres_fail(FRESNEL_ERR_ARG, "GRID plan: M must equal n1 * n2");
    if (M > p->stage_cap) {
        long long cap = M;
        if (p->tkind == FRESNEL_SCATTERED) FRES_TRY(dalloc(p, (void**)&p->stage_tgt, 16 * (size_t)cap));
        FRES_TRY(dalloc(p, &p->stage_out, p->csize() * (size_t)cap));
        p->stage_cap = cap;
    }
    if (p->tkind == FRESNEL_SCATTERED && M > 0) {
        // the copy overlaps the target-independent stages (nodes to FFT)
        if (!p->cst) {
            FRES_CK(cudaStreamCreateWithFlags(&p->cst, cudaStreamNonBlocking));
            FRES_CK(cudaEventCreateWithFlags(&p->ev_h2d, cudaEventDisableTiming));
            FRES_CK(cudaEventCreateWithFlags(&p->ev_free, cudaEventDisableTiming));
        }
        FRES_CK(cudaStreamWaitEvent(p->cst, p->ev_free, 0));
        FRES_CK(cudaMemcpyAsync(p->stage_tgt, h_targets, 16 * (size_t)M, cudaMemcpyHostToDevice, p->cst));
        FRES_CK(cudaEventRecord(p->ev_h2d, p->cst));
        p->wait_tgt = p->ev_h2d;
    }
    fresnel_status s = p->prec == FRESNEL_FP64 ? eval_impl<double>(p, p->stage_tgt, M, p->stage_out)
                                               : eval_impl<float>(p, p->stage_tgt, M, p->stage_out);
    p->wait_tgt = nullptr;
    if (s != FRESNEL_OK) return s;
    if (p->ev_free) FRES_CK(cudaEventRecord(p->ev_free, p->st));
    if (M > 0)
        FRES_CK(cudaMemcpyAsync(h_out, p->stage_out, p->csize() * (size_t)M, cudaMemcpyDeviceToHost, p->st));
    if (p->opts.sync_status) return read_status(p);
    return FRESNEL_OK;
}

fresnel_status fresnel_grad_profile(fresnel_plan_t plan, const void* d_gamma, double* d_grad) {
    Plan* p = as_plan(plan);
    if (!p) return fres_fail(FRESNEL_ERR_ARG, "invalid plan handle");
    if (p->tkind != FRESNEL_GRID)
        return fres_fail(FRESNEL_ERR_UNSUPPORTED, "profile gradients need a GRID plan");
    bool any = false;
    for (const FamilyDev& f : p->fams) any = any || f.kind == FRESNEL_FAMILY_PETALS;
    for (const FamilyDev& f : p->fams)
        if (f.shift)
            return fres_fail(FRESNEL_ERR_UNSUPPORTED, "profile gradients do not take moved petals");
    if (!any) return fres_fail(FRESNEL_ERR_ARG, "the plan has no PETALS family");
    if (p->d1.big || p->d2.big)
        return fres_fail(FRESNEL_ERR_UNSUPPORTED, "profile gradients need single-pass FFT lengths");
    if (!d_gamma || !d_grad) return fres_fail(FRESNEL_ERR_ARG, "d_gamma or d_grad is NULL");
    if (p->ft.scr.n1 > 0)
        return fres_fail(FRESNEL_ERR_UNSUPPORTED, "profile gradients do not take a source screen");
    fresnel_status s = p->prec == FRESNEL_FP64 ? grad_profile_impl<double>(p, d_gamma, d_grad)
                                               : grad_profile_impl<float>(p, d_gamma, d_grad);
    if (s != FRESNEL_OK) return s;
    if (p->opts.sync_status) return read_status(p);
    return FRESNEL_OK;
}

fresnel_status fresnel_grad_shape(fresnel_plan_t plan, const void* d_gamma, double* d_grad) {
    Plan* p = as_plan(plan);
    if (!p) return fres_fail(FRESNEL_ERR_ARG, "invalid plan handle");
    if (p->tkind != FRESNEL_GRID)
        return fres_fail(FRESNEL_ERR_UNSUPPORTED, "shape gradients need a GRID plan");
    bool any = false;
    for (const FamilyDev& f : p->fams) any = any || (f.kind == FRESNEL_FAMILY_FOURIER && !f.ptr);
    if (!any) return fres_fail(FRESNEL_ERR_ARG, "the plan has no FOURIER family");
    if (p->d1.big || p->d2.big)
        return fres_fail(FRESNEL_ERR_UNSUPPORTED, "shape gradients need single-pass FFT lengths");
    if (!d_gamma || !d_grad) return fres_fail(FRESNEL_ERR_ARG, "d_gamma or d_grad is NULL");
    if (p->ft.scr.n1 > 0)
        return fres_fail(FRESNEL_ERR_UNSUPPORTED, "shape gradients do not take a source screen");
    fresnel_status s = p->prec == FRESNEL_FP64 ? grad_shape_impl<double>(p, d_gamma, d_grad)
                                               : grad_shape_impl<float>(p, d_gamma, d_grad);
    if (s != FRESNEL_OK) return s;
    if (p->opts.sync_status) return read_status(p);
    return FRESNEL_OK;
}

fresnel_status fresnel_nsli(fresnel_plan_t plan, const double* d_targets, long long M,
                            void* d_out) {
    Plan* p = as_plan(plan);
    if (!p) return fres_fail(FRESNEL_ERR_ARG, "invalid plan handle");
    if (!p->subs.empty() || p->B != 1)
        return fres_fail(FRESNEL_ERR_ARG, "fresnel_nsli takes a one-problem plan");
    for (const FamilyDev& f : p->fams)
        if (f.kind != FRESNEL_FAMILY_FOURIER && f.kind != FRESNEL_FAMILY_LINE_RULE)
            return fres_fail(FRESNEL_ERR_UNSUPPORTED,
                             "the line integral needs FOURIER or LINE_RULE families only");
    if (p->ft.scr.n1 > 0)
        return fres_fail(FRESNEL_ERR_UNSUPPORTED, "the line integral cannot include a source screen");
    if (M < 0) return fres_fail(FRESNEL_ERR_ARG, "M must be >= 0");
    if (M > 0 && (!d_targets || !d_out)) return fres_fail(FRESNEL_ERR_ARG, "d_targets or d_out is NULL");
    launch_nsli(p->fams.data(), (int)p->fams.size(), p->lz, d_targets, M,
                p->output == FRESNEL_OCCULTER, p->opts.nsli_far, (double2*)d_out, p->st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fres_fail(FRESNEL_ERR_CUDA, std::string("line integral: ") + cudaGetErrorString(e));
    if (p->opts.sync_status) FRES_CK(cudaStreamSynchronize(p->st));
    return FRESNEL_OK;
}

fresnel_status fresnel_check(fresnel_plan_t plan) {
    Plan* p = as_plan(plan);
    if (!p) return fres_fail(FRESNEL_ERR_ARG, "invalid plan handle");
    if (!p->subs.empty()) return read_batch_status(p);
    return read_status(p);
}

fresnel_status fresnel_destroy(fresnel_plan_t plan) {
    if (!plan) return FRESNEL_OK;
    Plan* p = as_plan(plan);
    if (!p) return fres_fail(FRESNEL_ERR_ARG, "invalid plan handle");
    free_plan(p);
    return FRESNEL_OK;
}

const char* fresnel_last_error(void) { return g_last_error.c_str(); }

fresnel_status fresnel_get_info(fresnel_plan_t plan, fresnel_info* info) {
    Plan* p = as_plan(plan);
    if (!p || !info) return fres_fail(FRESNEL_ERR_ARG, "invalid plan handle or info");
    if (!p->subs.empty()) {   // batch: the first problem's shapes, totals over all
        FRES_TRY(fresnel_get_info(reinterpret_cast<fresnel_plan_t>(p->subs[0]), info));
        info->n_nodes = p->N;
        long long bytes = 0;
        int launches = 0;
        for (Plan* q : p->subs) {
            fresnel_info qi{};
            FRES_TRY(fresnel_get_info(reinterpret_cast<fresnel_plan_t>(q), &qi));
            bytes += q->bytes;
            launches += qi.launches_per_eval;
        }
        info->device_bytes = bytes;
        info->launches_per_eval = launches;
        for (size_t i = 1; i < p->subs.size(); ++i) {
            info->split_tiles += p->subs[i]->max_split;
            info->max_tile_records = std::max(info->max_tile_records, p->subs[i]->det_tmax);
            info->live_tile_rows += (int)std::min<long long>(p->subs[i]->live_rows_total, INT_MAX);
        }
        return FRESNEL_OK;
    }
    info->n_nodes = p->N;
    info->w = p->ks.w;
    info->beta = p->ks.beta;
    info->sigma = p->sigma;
    info->nf1 = p->nf1;
    info->nf2 = p->nf2;
    info->nfft1 = p->nfft1;
    info->nfft2 = p->nfft2;
    info->tile_x = kTile;
    info->tile_y = kTile;
    info->device_bytes = p->bytes;
    int nl = 4;   // spread, two FFT passes, (type 3) interpolation
    if (p->tkind == FRESNEL_GRID) nl = 3;
    if (p->opts.recompute_nodes) nl += 3;   // nodes, scan, scatter
    if (p->opts.deterministic) nl += 2;      // strengths' maxima, split tiles' conversion
    info->launches_per_eval = p->last_launches > 0 ? p->last_launches : nl;
    info->split_tiles = p->max_split;
    info->max_tile_records = p->det_tmax;
    info->t3_binning = p->opts.t3_binning;
    info->live_tile_rows = (int)std::min<long long>(p->live_rows_total, INT_MAX);
    return FRESNEL_OK;
}

fresnel_status fresnel_get_nodes(fresnel_plan_t plan, double* d_x, double* d_y, double* d_w) {
    Plan* p = as_plan(plan);
    if (!p) return fres_fail(FRESNEL_ERR_ARG, "invalid plan handle");
    if (!d_x || !d_y || !d_w) return fres_fail(FRESNEL_ERR_ARG, "node output arrays are NULL");
    if (!p->subs.empty())
        return fres_fail(FRESNEL_ERR_ARG, "scattered-target batch: nodes are per sub-plan");
    // Regenerates the nodes (and, harmlessly, the unsorted records and counts),
    // then re-runs the scan so the counts are reset and the cached sort stays valid.
    if (p->prec == FRESNEL_FP64) {
        FRES_TRY(run_nodes<double>(p, d_x, d_y, d_w));
        FRES_TRY(run_sort<double>(p));
    } else {
        FRES_TRY(run_nodes<float>(p, d_x, d_y, d_w));
        FRES_TRY(run_sort<float>(p));
    }
    FRES_CK(cudaGetLastError());
    return read_status(p);
}

int fresnel_set_timing(fresnel_plan_t plan, int enable) {
    Plan* p = as_plan(plan);
    if (!p) return 0;
    p->timing = enable ? 1 : 0;
    return p->timing;
}

int fresnel_stage_times(fresnel_plan_t plan, double* stage_ms, const char** names, int max_stages) {
    Plan* p = as_plan(plan);
    if (!p || !p->timing || p->nev < 2) return 0;
    cudaEventSynchronize(p->ev[p->nev - 1]);
    int n = 0;
    for (int i = 1; i < p->nev && n < max_stages; ++i, ++n) {
        float ms = 0;
        cudaEventElapsedTime(&ms, p->ev[i - 1], p->ev[i]);
        if (stage_ms) stage_ms[n] = ms;
        if (names) names[n] = p->ev_name[i];
    }
    return n;
}

}  // extern "C"

namespace {

fresnel_status plan_scattered_batch(const fresnel_problem* problems, int n, double tol,
                                    const fresnel_opts* opts, void* stream,
                                    fresnel_plan_t* out_plan) {
    Plan* p = new Plan();
    p->prec = opts->precision;
    p->output = opts->output;
    p->tkind = FRESNEL_SCATTERED;
    p->B = n;
    p->tol = tol;
    p->st = (cudaStream_t)stream;
    p->opts = *opts;
    fresnel_opts so = *opts;
    so.sync_status = 0;   // the batch reads every sub-plan's status itself
    auto fail = [&](fresnel_status st) {
        std::string msg = g_last_error;
        cudaGetLastError();
        free_plan(p);
        g_last_error = msg;
        return st;
    };
    for (int b = 0; b < n; ++b) {
        fresnel_plan_t h = nullptr;
        fresnel_status st = fresnel_plan_many(&problems[b], 1, tol, &so, stream, &h);
        if (st != FRESNEL_OK) {
            g_last_error = "problem " + std::to_string(b) + ": " + g_last_error;
            return fail(st);
        }
        p->subs.push_back(reinterpret_cast<Plan*>(h));
        p->N += p->subs.back()->N;
        p->lzs.push_back(p->subs.back()->lz);
        p->bytes += p->subs.back()->bytes;
    }
    p->lz = p->lzs[0];
    for (cudaStream_t& l : p->lanes)
        if (cudaStreamCreateWithFlags(&l, cudaStreamNonBlocking) != cudaSuccess)
            return fail(fres_fail(FRESNEL_ERR_CUDA, "cudaStreamCreate failed"));
    for (cudaEvent_t* e : {&p->ev_fork, &p->ev_in, &p->ev_out, &p->ev_join[0], &p->ev_join[1],
                           &p->ev_join[2], &p->ev_join[3]})
        if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess)
            return fail(fres_fail(FRESNEL_ERR_CUDA, "cudaEventCreate failed"));
    for (int b = 0; b < n; ++b) p->subs[b]->st = p->lanes[b % 4];
    *out_plan = reinterpret_cast<fresnel_plan_t>(p);
    return FRESNEL_OK;
}

// Grows a type-3 plan's target permutation ahead of graph capture (no
// allocation may happen while the evaluation is being captured).
fresnel_status ensure_perm(Plan* q, long long M) {
    if (q->prec != FRESNEL_FP32_FAST || M < kSortTargetsFrom || M <= q->perm_cap) return FRESNEL_OK;
    FRES_CK(cudaStreamSynchronize(q->st));
    if (q->perm) cudaFree(q->perm);
    q->perm = nullptr;
    q->perm_cap = 0;
    FRES_CK(cudaMalloc((void**)&q->perm, sizeof(int) * (size_t)M));
    q->perm_cap = M;
    return FRESNEL_OK;
}

// Captures the batch's evaluation on the internal lanes (fork from lane 0,
// problem b on lane b mod 4, join back) into p->gexec.
template <typename T>
fresnel_status capture_batch(Plan* p, const double* d_targets, const long long* M, void* d_out) {
    for (int b = 0; b < p->B; ++b) FRES_TRY(ensure_perm(p->subs[b], M[b]));
    if (p->gexec) {
        cudaGraphExecDestroy(p->gexec);
        p->gexec = nullptr;
    }
    FRES_CK(cudaStreamBeginCapture(p->lanes[0], cudaStreamCaptureModeRelaxed));
    fresnel_status st = FRESNEL_OK;
    cudaEventRecord(p->ev_fork, p->lanes[0]);
    for (int k = 1; k < 4; ++k) cudaStreamWaitEvent(p->lanes[k], p->ev_fork, 0);
    const size_t cs = p->csize();
    long long off = 0;
    for (int b = 0; b < p->B && st == FRESNEL_OK; ++b) {
        st = eval_impl<T>(p->subs[b], M[b] > 0 ? d_targets + 2 * off : nullptr, M[b],
                          M[b] > 0 ? (char*)d_out + cs * off : nullptr);
        off += M[b];
    }
    for (int k = 1; k < 4; ++k) {
        cudaEventRecord(p->ev_join[k], p->lanes[k]);
        cudaStreamWaitEvent(p->lanes[0], p->ev_join[k], 0);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(p->lanes[0], &g);
    if (st != FRESNEL_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess)
        return fres_fail(FRESNEL_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&p->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess)
        return fres_fail(FRESNEL_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    p->g_M.assign(M, M + p->B);
    p->g_t = d_targets;
    p->g_out = d_out;
    return FRESNEL_OK;
}

// Reads (and clears) every sub-plan's device status after the batch joined
// back into the caller's stream.
fresnel_status read_batch_status(Plan* p) {
    std::vector<unsigned> h(p->subs.size(), 0u);
    for (size_t b = 0; b < p->subs.size(); ++b)
        FRES_CK(cudaMemcpyAsync(&h[b], p->subs[b]->status, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                p->st));
    FRES_CK(cudaStreamSynchronize(p->st));
    for (size_t b = 0; b < p->subs.size(); ++b)
        if (h[b]) {
            FRES_CK(cudaMemsetAsync(p->subs[b]->status, 0, sizeof(unsigned), p->st));
            FRES_CK(cudaStreamSynchronize(p->st));
            std::string msg = "problem " + std::to_string(b) + ": device check failed:";
            if (h[b] & kStatusTargetOutside) msg += " target outside the plan's box;";
            if (h[b] & kStatusNodeOutside) msg += " node support outside the type-3 grid;";
            if (h[b] & kStatusNonFinite) msg += " non-finite coordinate;";
            if (h[b] & kStatusOverflow) msg += " sort region overflow;";
            return fres_fail(FRESNEL_ERR_DEVICE, msg);
        }
    return FRESNEL_OK;
}

}  // namespace

extern "C" {

fresnel_status fresnel_eval_many_scattered(fresnel_plan_t plan, const double* d_targets,
                                           const long long* M_each, void* d_out) {
    Plan* p = as_plan(plan);
    if (!p) return fres_fail(FRESNEL_ERR_ARG, "invalid plan handle");
    if (p->tkind != FRESNEL_SCATTERED)
        return fres_fail(FRESNEL_ERR_ARG, "fresnel_eval_many_scattered needs a SCATTERED plan");
    if (!M_each) return fres_fail(FRESNEL_ERR_ARG, "M_each is NULL");
    long long total = 0;
    for (int b = 0; b < p->B; ++b) {
        if (M_each[b] < 0) return fres_fail(FRESNEL_ERR_ARG, "M_each entries must be >= 0");
        total += M_each[b];
    }
    if (total > 0 && (!d_targets || !d_out))
        return fres_fail(FRESNEL_ERR_ARG, "d_targets or d_out is NULL");
    if (p->subs.empty()) return fresnel_eval(plan, d_targets, M_each[0], d_out);
    const bool same = p->gexec && p->g_t == d_targets && p->g_out == d_out &&
                      std::equal(p->g_M.begin(), p->g_M.end(), M_each);
    if (!same) {
        // the previous graph may still run on the lanes: capture after it
        FRES_CK(cudaStreamSynchronize(p->lanes[0]));
        FRES_TRY(p->prec == FRESNEL_FP64 ? capture_batch<double>(p, d_targets, M_each, d_out)
                                         : capture_batch<float>(p, d_targets, M_each, d_out));
    }
    FRES_CK(cudaEventRecord(p->ev_in, p->st));
    FRES_CK(cudaStreamWaitEvent(p->lanes[0], p->ev_in, 0));
    FRES_CK(cudaGraphLaunch(p->gexec, p->lanes[0]));
    FRES_CK(cudaEventRecord(p->ev_out, p->lanes[0]));
    FRES_CK(cudaStreamWaitEvent(p->st, p->ev_out, 0));
    if (p->opts.sync_status) return read_batch_status(p);
    return FRESNEL_OK;
}

}  // extern "C"

namespace {

// Device time (ms) of one evaluation of p, averaged over three after one
// warm-up; type 3 on `targets` (M pairs), type 1 on the plan's grid.
fresnel_status time_eval(Plan* p, const double* targets, long long M, void* out, float* ms) {
    cudaEvent_t a = nullptr, b = nullptr;
    FRES_CK(cudaEventCreate(&a));
    FRES_CK(cudaEventCreate(&b));
    fresnel_status st = FRESNEL_OK;
    auto one = [&]() {
        return p->prec == FRESNEL_FP64 ? eval_impl<double>(p, targets, M, out)
                                       : eval_impl<float>(p, targets, M, out);
    };
    st = one();
    if (st == FRESNEL_OK) {
        cudaEventRecord(a, p->st);
        for (int i = 0; i < 3 && st == FRESNEL_OK; ++i) st = one();
        cudaEventRecord(b, p->st);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(ms, a, b);
        *ms /= 3.0f;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st;
}

fresnel_status plan_autotuned(const fresnel_problem* problems, int n, double tol,
                              const fresnel_opts* opts, void* stream, fresnel_plan_t* out_plan) {
    fresnel_opts o = *opts;
    o.autotune = 0;
    std::vector<double> sigmas{opts->sigma};
    if (opts->precision == FRESNEL_FP64 && opts->sigma == 0 && opts->kernel_w == 0)
        sigmas = {1.25, 2.0};
    const bool scattered = opts->target_kind == FRESNEL_SCATTERED;
    const bool tune_bins = scattered && opts->precision == FRESNEL_FP32_FAST && opts->t3_binning == 0;
    // synthetic targets for type 3: 2^20 points spread evenly over the box
    const long long MT = scattered ? (1LL << 20) : 0;
    double* d_t = nullptr;
    void* d_out = nullptr;
    long long out_elems = 0;
    Plan* best = nullptr;
    float best_ms = 0.0f;
    int best_bins = opts->t3_binning;
    fresnel_status last = FRESNEL_OK;
    std::string last_msg;
    for (double sg : sigmas) {
        o.sigma = sg;
        fresnel_plan_t h = nullptr;
        fresnel_status st = fresnel_plan_many(problems, n, tol, &o, stream, &h);
        if (st != FRESNEL_OK) {
            last = st;
            last_msg = g_last_error;
            continue;
        }
        Plan* q = reinterpret_cast<Plan*>(h);
        const long long need = scattered ? MT : (long long)q->n1 * q->n2 * q->B;
        if (need > out_elems) {
            if (d_out) cudaFree(d_out);
            d_out = nullptr;
            if (cudaMalloc(&d_out, 16 * (size_t)need) != cudaSuccess) {
                cudaGetLastError();
                free_plan(q);
                last = fres_fail(FRESNEL_ERR_OOM, "autotune scratch");
                last_msg = g_last_error;
                break;
            }
            out_elems = need;
        }
        if (scattered && !d_t) {
            std::vector<double> ht(2 * MT);
            const double* bx = opts->box;
            const int side = 1024;   // 1024 x 1024 lattice, offset by a golden-ratio shift
            for (long long k = 0; k < MT; ++k) {
                const double u = ((k % side) + 0.618033988749895) / side;
                const double v = ((k / side) + 0.381966011250105) / side;
                ht[2 * k] = bx[0] + (bx[1] - bx[0]) * u;
                ht[2 * k + 1] = bx[2] + (bx[3] - bx[2]) * v;
            }
            if (cudaMalloc((void**)&d_t, sizeof(double) * 2 * MT) != cudaSuccess) {
                cudaGetLastError();
                free_plan(q);
                last = fres_fail(FRESNEL_ERR_OOM, "autotune targets");
                last_msg = g_last_error;
                break;
            }
            cudaMemcpy(d_t, ht.data(), sizeof(double) * 2 * MT, cudaMemcpyHostToDevice);
        }
        int bins = opts->t3_binning;
        float ms = 0.0f;
        if (tune_bins) {
            float m1 = 0.0f, m2 = 0.0f;
            q->opts.t3_binning = -1;
            st = time_eval(q, d_t, MT, d_out, &m1);
            if (st == FRESNEL_OK) {
                q->opts.t3_binning = 1;
                st = time_eval(q, d_t, MT, d_out, &m2);
            }
            bins = m2 < m1 ? 1 : -1;
            ms = std::min(m1, m2);
            q->opts.t3_binning = bins;
        } else {
            st = time_eval(q, d_t, MT, d_out, &ms);
        }
        cudaMemsetAsync(q->status, 0, sizeof(unsigned), q->st);   // synthetic run: no report
        if (st != FRESNEL_OK) {
            last = st;
            last_msg = g_last_error;
            free_plan(q);
            continue;
        }
        if (!best || ms < best_ms) {
            if (best) free_plan(best);
            best = q;
            best_ms = ms;
            best_bins = bins;
        } else {
            free_plan(q);
        }
    }
    if (d_t) cudaFree(d_t);
    if (d_out) cudaFree(d_out);
    if (!best) {
        g_last_error = last_msg;
        return last != FRESNEL_OK ? last : fres_fail(FRESNEL_ERR_ARG, "autotune found no plan");
    }
    best->opts.autotune = 1;
    best->opts.t3_binning = best_bins;
    cudaStreamSynchronize(best->st);
    *out_plan = reinterpret_cast<fresnel_plan_t>(best);
    return FRESNEL_OK;
}

}  // namespace
