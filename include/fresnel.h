/*
 * fresnel.h -- C ABI of libfresnel: scalar Fresnel diffraction of a planar
 * aperture or occulter by areal quadrature + one 2D nonuniform FFT, on one
 * NVIDIA GB300 (sm_103a).
 *
 * Method: Barnett, "Efficient high-order accurate Fresnel diffraction via
 * areal quadrature and the nonuniform FFT", arXiv:2010.05978.
 *   u^ap(xi, eta) = 1/(i lz) iint_Omega exp(i pi [(xi-x)^2 + (eta-y)^2] / lz) dx dy
 * (eq. fres, Sec. 2; lz = lambda * z; the plane-wave phase e^{2 pi i z/lambda}
 * is dropped as in Sec. 2) is approximated by an areal quadrature (x_j, y_j,
 * w_j) (eq. aq) and evaluated in the split form of eq. split:
 *   c_j = w_j exp(i pi |x_j|^2 / lz)                      (Sec. 3.2, step 1)
 *   v_k = sum_j exp(-2 pi i xi_k . x_j / lz) c_j           (eq. nufft3, step 2)
 *   u_k = 1/(i lz) exp(i pi |xi_k|^2 / lz) v_k             (Sec. 3.2, step 3)
 * Step 2 is a 2D type-1 NUFFT for targets on a uniform grid (Sec. 3.3) or a
 * type-3 NUFFT for scattered targets (Sec. 3.2).  The occulter field is
 * u^oc = 1 - u^ap (Babinet, eq. bab).
 *
 * Conventions for every entry point:
 *  - Status codes are returned, never thrown; fresnel_last_error() gives a
 *    message for the calling thread's most recent failure.
 *  - "host" pointers are read during the call only and may be freed after it.
 *  - "device" pointers must be CUDA device (or managed) memory on the device
 *    that was current when the plan was made; they are owned by the caller.
 *  - All device work is enqueued on the plan's stream (the cudaStream_t given
 *    to fresnel_plan, or the legacy default stream for NULL).
 */
#ifndef FRESNEL_H
#define FRESNEL_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
typedef enum {
    FRESNEL_OK = 0,
    FRESNEL_ERR_ARG = -1,         /* invalid argument; nothing was launched */
    FRESNEL_ERR_CUDA = -2,        /* a CUDA runtime call failed */
    FRESNEL_ERR_OOM = -3,         /* device allocation failed or exceeded the cap */
    FRESNEL_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up (fresnel_opts.max_spin) */
    FRESNEL_ERR_UNSUPPORTED = -5, /* valid request beyond this build's limits */
    FRESNEL_ERR_DEVICE = -6       /* a device-side check failed (e.g. target outside the plan's box) */
} fresnel_status;

/* ---------------------------------------------------------------- geometry */
/*
 * One family of quadrature nodes.  kind selects how params is read:
 *
 * FRESNEL_FAMILY_FOURIER: a smooth star-shaped boundary about (cx, cy),
 *     X(t) = cx + r(t) cos t, Y(t) = cy + r(t) sin t, t in [0, 2 pi)
 *     counter-clockwise, r(t) = r0 + sum_{k=1}^{K} (a_k cos kt + b_k sin kt),
 *     params = [r0, a_1, b_1, ..., a_K, b_K] (n_params = 1 + 2K).
 *     The vector line rule (eq. vliq) uses n_panels equal t-panels with p
 *     Gauss-Legendre nodes each: W_i = what_i X'(t_i), V_i = what_i Y'(t_i)
 *     (eq. vliq1 with panels in place of the trapezoid rule).  The areal rule
 *     is the dilation rule about (cx, cy) with m Gauss-Legendre radii on (0,1)
 *     (eqs. aqnod, aqwei, Sec. 4.1): N = n_panels * p * m nodes.
 *
 * FRESNEL_FAMILY_LINE_RULE: an explicit vector line rule on the boundary,
 *     params = [X_1..X_n, Y_1..Y_n, W_1..W_n, V_1..V_n] (n_params = 4n), with
 *     n = n_panels * p (p may be 1), dilated about (cx, cy) with m radii.
 *
 * FRESNEL_FAMILY_NODES: an explicit areal rule (eq. aq),
 *     params = [x_1..x_N, y_1..y_N, w_1..w_N] (n_params = 3N); the other
 *     fields are ignored.
 *
 * FRESNEL_FAMILY_PETALS: a starshade (Sec. 4.2, eq. Omega): the disc r < a
 *     plus n_panels identical petals; petal k is centred on the angle
 *     2 pi k / n_panels and its angular width at radius r in (a, R) is
 *     2 pi A(r) / n_panels.  params = [a, R, n_d, m_d, profile, data...]:
 *       n_d >= 0  disc boundary nodes (periodic trapezoid rule of eq. ptr,
 *                 t_i = 2 pi i / n_d), dilated with m_d >= 1 radii (eqs.
 *                 aqnod, aqwei); n_d = 0 leaves the disc out;
 *       profile   FRESNEL_PETAL_HG: data = [b, q], A = exp(-((r - a)/b)^q)
 *                 (the offset hyper-Gaussian, n_params = 7);
 *                 FRESNEL_PETAL_BSPLINE: data = n >= 4 coefficients of a
 *                 clamped uniform cubic B-spline on [a, R] (knots a x4, the
 *                 n - 4 interior points of an (n - 3)-interval uniform mesh,
 *                 R x4; n_params = 5 + n);
 *                 FRESNEL_PETAL_TABLE: data = A at the m ascending
 *                 Gauss-Legendre radii on (a, R) (n_params = 5 + m).
 *     Each petal has m Gauss-Legendre radii r_l on (a, R) times p
 *     Gauss-Legendre angles t_i on [-pi/n_panels, pi/n_panels]: node
 *     r_l (cos th, sin th) with th = A(r_l) t_i + 2 pi k / n_panels, weight
 *     r_l what_l A(r_l) omegahat_i.  Nodes are ordered disc first
 *     (boundary-major, radius fastest), then petal, angle, radius fastest:
 *     N = n_d m_d + n_panels p m.  (cx, cy) translates the whole shape.
 *     n_d, m_d and profile are whole numbers stored as doubles.  A may be
 *     negative or exceed 1 (non-ideal profiles); nothing is clamped.
 *
 * FRESNEL_FAMILY_TRIANGLES: a union of triangles (Sec. 4.3, the Koch
 *     snowflake construction), params = [v0x, v0y, v1x, v1y, v2x, v2y] per
 *     triangle (n_params = 6 n_panels, n_panels triangles), translated by
 *     (cx, cy).  Each triangle is a p x p product rule: v0 moved to the
 *     origin, p Gauss-Legendre nodes s_i on the edge v1 -> v2 form the line
 *     rule X_i = v1 + s_i (v2 - v1), (W_i, V_i) = what_i (v2 - v1), and the
 *     dilation rule (eqs. aqnod, aqwei) with the same p radii alpha_l gives
 *     x = v0 + alpha_l (X_i - v0), w = alpha_l what_l what_i
 *     (v1 - v0) x (v2 - v1); the weights sum to the signed area (positive for
 *     counter-clockwise v0, v1, v2).  m is ignored (p radii).  Nodes are
 *     ordered triangle-major, then edge node, radius fastest: N = n_panels p^2.
 *
 * Negative weights and nodes outside Omega (non-star-shaped domains, Sec. 4.1)
 * are accepted as given.  params is a HOST array copied during fresnel_plan.
 */
enum {
    FRESNEL_FAMILY_FOURIER = 0,
    FRESNEL_FAMILY_LINE_RULE = 1,
    FRESNEL_FAMILY_NODES = 2,
    FRESNEL_FAMILY_PETALS = 3,
    FRESNEL_FAMILY_TRIANGLES = 4
};
enum { FRESNEL_PETAL_HG = 0, FRESNEL_PETAL_BSPLINE = 1, FRESNEL_PETAL_TABLE = 2 };

typedef struct {
    int kind;
    int n_panels, p, m;
    const double* params;   /* host */
    long long n_params;
    double cx, cy;
    /* PETALS only, or NULL: rigid motion of each petal (Sec. 5's perturbed
     * starshades, second construction), 3 * n_panels values (phi_k, tx_k, ty_k):
     * petal k's nodes move to c + R(phi_k) (x - c) + (tx_k, ty_k), weights
     * unchanged, and a signed patch joins its root arc on the disc circle
     * r = a (angles 2 pi k/n_panels +- pi/n_panels) to the moved base arc:
     * P(s, t) = (1 - t) root(s) + t M_k(root(s)), weight dP/dt x dP/ds, on a
     * max(2 p, 16) x 8 Gauss-Legendre rule in (s, t), appended after the
     * family's nodes (gaps add, overlaps subtract).  HOST array, read during
     * fresnel_plan.  Not with profile gradients. */
    const double* motion;
} fresnel_family;

/* ---------------------------------------------------------------- options */
enum { FRESNEL_FP64 = 0, FRESNEL_FP32_FAST = 1 };
enum { FRESNEL_APERTURE = 0, FRESNEL_OCCULTER = 1 };
enum { FRESNEL_GRID = 0, FRESNEL_SCATTERED = 1 };

typedef struct {
    /* FRESNEL_FP64: every stage in FP64; output complex128 (re, im doubles).
     * FRESNEL_FP32_FAST: spreading, FFT and interpolation in FP32 with FP32
     * accumulation; the chirp phases and the xi.x/lz scalings stay FP64 with
     * argument reduction; output complex64 (re, im floats). */
    int precision;
    int output;          /* FRESNEL_APERTURE (u^ap) or FRESNEL_OCCULTER (1 - u^ap) */
    int target_kind;     /* FRESNEL_GRID (type 1, Sec. 3.3) or FRESNEL_SCATTERED (type 3, Sec. 3.2) */
    /* GRID targets: xi = grid_x0 + k1 h, eta = grid_y0 + k2 h,
     * -floor(n/2) <= k < n - floor(n/2); output index k2' * grid_n1 + k1'
     * with k' = k + floor(n/2) (k1 fastest).  A nonzero (x0, y0) is applied
     * by pre-phasing the strengths (Sec. 3.3, last paragraph). */
    int grid_n1, grid_n2;
    double grid_h, grid_x0, grid_y0;
    /* SCATTERED targets must lie in [box[0], box[1]] x [box[2], box[3]]; the
     * plan sizes its grids from this box and eval flags targets outside it
     * (FRESNEL_ERR_DEVICE). */
    double box[4];
    double sigma;        /* upsampling factor; 0 = automatic */
    int kernel_w;        /* spreading kernel width in grid points, 2..16; 0 = automatic */
    int recompute_nodes; /* 1: node generation, chirp and binning run inside every
                            fresnel_eval (nothing node-sized is cached); 0: done once */
    int sync_status;     /* 1: fresnel_eval synchronises the stream and returns the
                            device status; 0: asynchronous, see fresnel_check */
    long long max_device_bytes; /* cap on the plan's device memory; 0 = no cap */
    /* SCATTERED + FP32_FAST: bucket the targets by 16 x 16 blocks of the FFT
     * grid and interpolate from shared-memory patches (1), gather each target
     * straight from global memory (-1), or choose (0: bucket when the FFT grid
     * exceeds 64 MB, i.e. would not stay in L2, and M >= 32768). */
    int t3_binning;
    /* FFT lengths above this run as four-step transforms fa x fb (two launches
     * per pass through an intermediate buffer) instead of one shared-memory
     * pass; 0 = only when one pass does not fit in shared memory (lengths
     * above ~13,600 in FP32, ~6,800 in FP64).  Batched plans and profile
     * gradients need single-pass lengths. */
    int fft_split_above;
    /* 1: measure before committing to a configuration.  FP64 with automatic
     * sigma / width: plans with sigma = 5/4 and 2 are built and timed on the
     * device (type 1: an evaluation of the grid; type 3: 2^20 targets spread
     * over the box) and the faster is kept.  FP32 type 3 with t3_binning = 0:
     * binned and direct interpolation are timed the same way and the faster
     * is fixed for the plan.  Plan time grows accordingly; results stay
     * within tol either way.  Not applied to scattered-target batches. */
    int autotune;
    /* fresnel_nsli only (Appendix, remark r:shadfix): targets whose nearest
     * boundary node is at least nsli_far away use the classical line
     * integral eq. li with the winding number of eq. geom rounded to an
     * integer (exact u_geom, so a shadow's u^oc is not 1 minus a quadrature
     * of 1); nearer targets use eq. nsli.  0 = eq. nsli everywhere. */
    double nsli_far;
    /* Source-plane screen (Sec. 5: the strengths' w_j times the source term
     * at each areal node): s(x, y) = A(x, y) exp(2 pi i OPD(x, y) / lambda),
     * lambda each problem's own.  screen_amp (amplitude A) and screen_opd
     * (optical path difference, same length unit as lambda) are HOST arrays
     * of screen_n2 rows of screen_n1 samples (row-major; either may be NULL:
     * A = 1 / OPD = 0) at x = box[0] + i (box[1] - box[0]) / (n1 - 1),
     * y = box[2] + k (box[3] - box[2]) / (n2 - 1), copied at plan time, and
     * interpolated by Catmull-Rom (cubic convolution, exact for polynomials of
     * degree <= 2).  The interpolation stencil stays inside the samples: the
     * box must reach one spacing beyond the aperture (nodes nearer the edge
     * take the nearest interior value).  screen_n1 = screen_n2 = 0: no screen.
     * FP32_FAST plans evaluate the screen in FP32: its phase 2 pi OPD / lambda
     * carries an error of ~1e-7 of its range, so at tol 1e-6 keep that range
     * within ~10 rad or use FP64.  Not with profile gradients or the line
     * integral. */
    const double* screen_amp;
    const double* screen_opd;
    int screen_n1, screen_n2;
    double screen_box[4];
    /* Bound on the one device-side wait of the spreading stage: the chunks
     * of a tile that holds more records than one work item takes wait, before
     * adding into the tile, for the flag with which the tile's first chunk
     * reports having cleared it.  Polls per wait (~256 ns apart) before the
     * wait gives up, skips its addition and flags FRESNEL_ERR_TIMEOUT (read by
     * fresnel_check or a synchronous evaluation): 0 = the built-in 2^22
     * (about a second), > 0 = that many, < 0 = none at all (every such wait
     * gives up at once; for tests of the timeout path). */
    long long max_spin;
    /* 1: results repeat bit for bit from evaluation to evaluation and plan
     * to plan (same device, library and options).  The spreading stage then
     * sums in exact fixed point (each contribution scaled by a power of two
     * fixed per evaluation from the largest strength and the fullest tile,
     * then rounded once to an integer), so neither the order of the records
     * within a tile nor the order of a split tile's chunks can change a bit;
     * every other stage already sums in a fixed order.  Costs two launches
     * more per evaluation and a slower spread (shared-memory 64-bit atomic
     * adds); plans whose fullest tile holds 2^23 or more records are
     * refused (FRESNEL_ERR_UNSUPPORTED).  The accuracy meets tol as in the
     * default mode.  0 (default): the spread sums in floating point in the
     * order the records arrive, which varies by a few ulp between runs. */
    int deterministic;
} fresnel_opts;

/* Fills *opts with defaults: FP32_FAST, aperture, grid 100 x 100 with h = 0.03,
 * automatic sigma/width, recompute_nodes = 0, sync_status = 1, nsli_far = 0. */
void fresnel_default_opts(fresnel_opts* opts);

/* ---------------------------------------------------------------- plan */
typedef struct fresnel_plan_s* fresnel_plan_t;   /* opaque; owned by the library */

/*
 * Builds the quadrature of the n_families families, chooses the NUFFT
 * parameters for the requested relative tolerance tol (1e-14 <= tol <= 1e-1),
 * and allocates all device scratch.  lambda > 0, z > 0 (only lambda*z enters,
 * eq. fres).  cuda_stream is a cudaStream_t (NULL = legacy default stream).
 * On success *out_plan receives the plan; on failure *out_plan is NULL and
 * nothing stays allocated.  Synchronises the stream before returning.
 */
fresnel_status fresnel_plan(const fresnel_family* families, int n_families,
                            double lambda, double z, double tol,
                            const fresnel_opts* opts, void* cuda_stream,
                            fresnel_plan_t* out_plan);

/*
 * A batch of independent problems sharing one target grid, e.g. one
 * starshade at many wavelengths (the wavelength sweeps of Sec. 4.2): each
 * problem has its own families (host array) and lambda, z; tol and opts are
 * common.  GRID targets: all problems share the grid, one spreading kernel
 * and one FFT size, so one launch per stage serves the whole batch
 * (fresnel_eval_many).  SCATTERED targets: one sub-plan per problem, sized
 * for it, evaluated together by fresnel_eval_many_scattered.  Otherwise as
 * fresnel_plan (which is the one-problem case).
 */
typedef struct {
    const fresnel_family* families;
    int n_families;
    double lambda, z;
} fresnel_problem;

fresnel_status fresnel_plan_many(const fresnel_problem* problems, int n_problems, double tol,
                                 const fresnel_opts* opts, void* cuda_stream,
                                 fresnel_plan_t* out_plan);

/*
 * Scattered-target batches (fresnel_plan_many with opts->target_kind =
 * FRESNEL_SCATTERED): every problem gets its own NUFFT sizes (its aperture
 * and lambda z set them), all with the opts box; problem b has M_each[b]
 * targets (HOST array of n_problems counts, each >= 0).  d_targets (DEVICE)
 * holds all problems' (xi, eta) FP64 pairs concatenated in problem order and
 * d_out (DEVICE) receives the concatenated fields (complex64 / complex128).
 * The whole batch is one CUDA graph (captured on the first call and again
 * whenever the counts or pointers change) spread over four internal streams
 * and joined back into the plan's stream.  Asynchronous unless
 * opts.sync_status = 1.  Also accepts a one-problem SCATTERED plan.
 */
fresnel_status fresnel_eval_many_scattered(fresnel_plan_t plan, const double* d_targets,
                                           const long long* M_each, void* d_out);

/*
 * Evaluates every problem of a plan on its grid: d_out is a DEVICE array of
 * n_problems * grid_n2 * grid_n1 complex values (problem-major, each problem
 * as fresnel_eval writes it).  Asynchronous unless opts.sync_status = 1.
 */
fresnel_status fresnel_eval_many(fresnel_plan_t plan, void* d_out);

/*
 * Gradient of a real loss of a GRID plan's output with respect to the
 * profile parameters of its FRESNEL_FAMILY_PETALS families (Sec. 4.2: the
 * apodisation A(r) sets the petal widths), for optimising starshade designs.
 * d_gamma (DEVICE, the same layout and type as the output of
 * fresnel_eval_many / fresnel_eval: n_problems * grid_n2 * grid_n1 complex)
 * holds the loss's sensitivity: dL = Re sum_k conj(gamma_k) du_k for
 * perturbations du of the plan's output field (u^ap or u^oc as configured);
 * for L = sum |u_k|^2, gamma = 2 u.  d_grad (DEVICE, FP64) receives, for every
 * PETALS family in plan order (problem-major, then family order), dL/dparam
 * for its profile data params[5...]: [b, q] for FRESNEL_PETAL_HG, the n
 * spline coefficients for FRESNEL_PETAL_BSPLINE, the m values of A for
 * FRESNEL_PETAL_TABLE.  It is the exact derivative of the computed
 * (discretised) field: the adjoint of the spreading / FFT / output chain is a
 * type-2 transform interpolated at the nodes with the kernel and its
 * derivative.  The quadrature nodes are taken as last evaluated (call after
 * an evaluation with the same profile).  Reuses the plan's spreading grid.
 * Asynchronous unless opts.sync_status = 1.
 */
fresnel_status fresnel_grad_profile(fresnel_plan_t plan, const void* d_gamma, double* d_grad);

/*
 * Gradient of a real loss of a GRID plan's output with respect to the
 * boundary coefficients of its FRESNEL_FAMILY_FOURIER families, for
 * optimising aperture shapes: the boundary r(t) = r0 + sum_k (a_k cos kt +
 * b_k sin kt) about (cx, cy) enters through its Gauss-Legendre panel line
 * rule (eq. vliq1) and the dilation rule (Sec. 3.1, eqs. aqnod, aqwei):
 * x = c + alpha_l r(t_i) (cos t_i, sin t_i), w = alpha_l wtilde_l what_i r(t_i)^2.
 * d_gamma as for fresnel_grad_profile (dL = Re sum_k conj(gamma_k) du_k).
 * d_grad (DEVICE, FP64) receives, for every FOURIER family in plan order
 * (problem-major, then family order), dL/dparams in the layout of its params
 * [r0, a_1, b_1, ..., a_K, b_K] (1 + 2K values).  A starshade's disc is not a
 * FOURIER family for this purpose.  It is the exact derivative of the
 * computed (discretised) field: the same type-2 adjoint transform as
 * fresnel_grad_profile, interpolated at every node with the kernel and its
 * derivative, chained to dL/dr(t_i) per boundary node and summed against
 * cos kt_i, sin kt_i in a fixed order.  Reuses the plan's spreading grid
 * (evaluate again afterwards).  Errors: FRESNEL_ERR_ARG for a NULL pointer or
 * a plan without FOURIER families; FRESNEL_ERR_UNSUPPORTED for scattered
 * targets, a source screen or an FFT length beyond one pass.  Asynchronous
 * unless opts.sync_status = 1.
 */
fresnel_status fresnel_grad_shape(fresnel_plan_t plan, const void* d_gamma, double* d_grad);

/*
 * Evaluates u at the plan's targets (plans with one problem).
 * GRID plans: d_targets is ignored (may be NULL) and M must equal n1 * n2.
 * SCATTERED plans: d_targets is a DEVICE array of M (xi, eta) FP64 pairs
 * (interleaved, 16 bytes per target); M >= 0.
 * d_out is a DEVICE array of M complex values (complex128 for FP64 plans,
 * complex64 for FP32_FAST plans), written in target order.
 * Asynchronous on the plan's stream unless opts.sync_status = 1.
 */
fresnel_status fresnel_eval(fresnel_plan_t plan, const double* d_targets, long long M,
                            void* d_out);

/*
 * The same evaluation with HOST buffers: h_targets (M FP64 pairs, ignored for
 * GRID plans) is copied to the device, fresnel_eval runs, and the M complex
 * results are copied back to h_out.  The targets' copy runs on a second
 * stream of the plan, overlapping the stages that do not need the targets
 * (nodes, sort, spreading, FFT).  With opts.sync_status = 1 the call returns
 * after the results are in h_out (and reports the device status); with
 * opts.sync_status = 0 it returns once the work is queued, like fresnel_eval:
 * h_out is complete, and h_targets may be reused, after the plan's stream
 * has been synchronised (fresnel_check, or a stream / device
 * synchronisation).  Pinned host memory makes the copies asynchronous and
 * fast; pageable memory works, with copies that block the caller.
 */
fresnel_status fresnel_eval_host(fresnel_plan_t plan, const double* h_targets, long long M,
                                 void* h_out);

/*
 * Non-singular line integral (Appendix, eq. nsli) on the device: u at M
 * scattered targets (DEVICE (xi, eta) FP64 pairs) from the boundary line
 * rules of the plan's families alone, O(n M) in FP64, written to d_out
 * (DEVICE, M complex128, aperture or occulter as the plan's output) whatever
 * the plan's precision.  An independent reference for the areal path, valid
 * up to and on the boundary (the summand is 0 where r = 0).  One-problem
 * plans whose families are all FRESNEL_FAMILY_FOURIER or LINE_RULE.
 */
fresnel_status fresnel_nsli(fresnel_plan_t plan, const double* d_targets, long long M,
                            void* d_out);

/* Synchronises the plan's stream and returns (then clears) the device status
 * word: FRESNEL_OK or FRESNEL_ERR_DEVICE (the message names each check that
 * failed: a target outside the box, a node support outside the type-3 grid, a
 * non-finite coordinate, a sort region overflow). */
fresnel_status fresnel_check(fresnel_plan_t plan);

/* Releases everything the plan owns.  NULL-safe; synchronises the stream. */
fresnel_status fresnel_destroy(fresnel_plan_t plan);

/* Message describing the calling thread's most recent failure ("" if none). */
const char* fresnel_last_error(void);

/* ---------------------------------------------------------------- introspection */
typedef struct {
    long long n_nodes;      /* N, total quadrature nodes (over all problems) */
    int w;                  /* spreading kernel width (grid points) */
    double beta;            /* exponential-of-semicircle shape parameter */
    double sigma;           /* upsampling factor used */
    int nf1, nf2;           /* spreading grid */
    int nfft1, nfft2;       /* FFT grid (= spreading grid for GRID plans) */
    int tile_x, tile_y;     /* spreading tile */
    long long device_bytes; /* device memory the plan holds */
    int launches_per_eval;  /* kernels launched by one fresnel_eval */
    int split_tiles;        /* spreading tiles whose records are split over several work items */
    int max_tile_records;   /* node records of the fullest spreading tile */
    int t3_binning;         /* FP32 SCATTERED plans: 1 binned interpolation, -1 direct
                               gathers, 0 chosen per evaluation (fresnel_opts.t3_binning,
                               after the autotuner's choice when it ran) */
    int live_tile_rows;     /* spreading-tile rows holding nodes, summed over the problems
                               (GRID plans spread and transform only these rows) */
} fresnel_info;

fresnel_status fresnel_get_info(fresnel_plan_t plan, fresnel_info* info);

/*
 * Copies the plan's quadrature nodes (x, y, w; FP64, N each) into DEVICE
 * arrays, in family order and, within a family, boundary-node-major with the
 * radial index fastest (eqs. aqnod, aqwei).  For checking the quadrature.
 */
fresnel_status fresnel_get_nodes(fresnel_plan_t plan, double* d_x, double* d_y, double* d_w);

/* ---------------------------------------------------------------- spreading primitive */
/*
 * The spreading stage of the NUFFT on its own (the first step of the type-1
 * and type-3 transforms behind Secs. 3.2-3.3): for N points with periodic
 * grid coordinates (g1_j, g2_j) (FP64, grid units, any real value; taken
 * modulo nf1, nf2) and FP32 complex strengths c_j,
 *   grid[l2 * nf1 + l1] = sum_j c_j psi(l1 - g1_j) psi(l2 - g2_j),
 *   psi(u) = exp(beta (sqrt(1 - (2u/w)^2) - 1)) for |u| < w/2, else 0,
 * with l - g taken periodically.  All pointers are DEVICE memory:
 * d_g1, d_g2 (N doubles each), d_c (N complex64 = interleaved float pairs),
 * d_grid (nf1 * nf2 complex64, overwritten).  2 <= w <= 16, beta > 0,
 * nf1 and nf2 multiples of 32 and >= 64.  The kernel values are evaluated
 * with exp/sqrt (not the plan's polynomial form).  Scratch is allocated
 * stream-ordered (cudaMallocAsync) on cuda_stream and released before the
 * call returns; the call synchronises the stream.  Returns FRESNEL_ERR_DEVICE
 * if a coordinate is not finite (that point is dropped).
 */
fresnel_status fresnel_spread(const double* d_g1, const double* d_g2, const void* d_c,
                              long long N, int nf1, int nf2, int w, double beta,
                              void* d_grid, void* cuda_stream);

/*
 * fresnel_spread for callers that cannot allocate device memory: code that
 * may not call cudaMalloc (or any allocating routine) because another
 * framework owns the device memory pool and forbids allocations it does not
 * make, and embedded or real-time callers that forbid allocation after
 * start-up.  The
 * paper has no counterpart: this is a property of the library, not of the
 * method.  Same arguments, result and errors as fresnel_spread, with limits:
 * N <= FRESNEL_SPREAD_NOALLOC_MAX_POINTS and nf1 * nf2 <=
 * FRESNEL_SPREAD_NOALLOC_MAX_GRID (else FRESNEL_ERR_UNSUPPORTED, nothing
 * launched).  The scratch is a static device array of
 * FRESNEL_SPREAD_NOALLOC_SCRATCH_BYTES that every device which loads the
 * library holds until the process exits; the call allocates nothing.  The
 * first call on a device looks the array's address up (cudaGetSymbolAddress,
 * with that device current) and should come before any stream capture; the
 * address is kept until the process exits, so after a cudaDeviceReset the
 * call must not be used again.  All calls on a device share the array, so
 * calls that overlap on the GPU (other streams, other host threads) race:
 * serialise them.  Every call reads a 4-byte status word back to the host
 * and synchronises cuda_stream before it returns.
 */
#define FRESNEL_SPREAD_NOALLOC_MAX_POINTS 65536
#define FRESNEL_SPREAD_NOALLOC_MAX_GRID (2048 * 2048)
#define FRESNEL_SPREAD_NOALLOC_SCRATCH_BYTES (8 * 1024 * 1024)
fresnel_status fresnel_spread_noalloc(const double* d_g1, const double* d_g2, const void* d_c,
                                      long long N, int nf1, int nf2, int w, double beta,
                                      void* d_grid, void* cuda_stream);

/*
 * Per-stage device time of the last fresnel_eval, in milliseconds, measured
 * with CUDA events on the plan's stream when timing was enabled by
 * fresnel_set_timing(plan, 1).  stage_ms receives up to max_stages values;
 * names (optional) receives static strings.  Returns the number of stages.
 */
int fresnel_set_timing(fresnel_plan_t plan, int enable);
int fresnel_stage_times(fresnel_plan_t plan, double* stage_ms, const char** names, int max_stages);

#ifdef __cplusplus
}
#endif
#endif /* FRESNEL_H */
