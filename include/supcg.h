/*
 * supcg.h -- C ABI of libsupcg, a GB300 (sm_103a) implementation of the
 * data-parallel hot path of Superiorized Preconditioned Conjugate Gradient
 * (SupPCG) for 2-D parallel-beam tomography (Helou, Herman, Lin, Zibetti,
 * arXiv 1807.10151).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Image: ny rows x nx columns, row-major, FP32 unless the geometry's
 *    storage is SUPCG_BF16; element i*nx + j is pixel (i, j) (Sec. 3.1 puts
 *    pixel (i, j) at component c(i-1)+j).  Row 0 is the top row.  Pixel (i, j)
 *    has centre x_j = (j - (nx-1)/2) d, y_i = ((ny-1)/2 - i) d, d = pixel size.
 *  - Sinogram: n_views rows x n_bins columns, row-major.  Ray (v, u) is the
 *    line x cos(theta_v) + y sin(theta_v) = s_u, s_u = (u - (U-1)/2) ds + off
 *    (Sec. 2 data model R x = b + e; Sec. 4.1 acquisition shape).
 *  - R_{(v,u),(i,j)} is the length of ray (v, u) inside the closed pixel
 *    square (a line on an edge shared by two pixels gives each half).
 *  - "d_" pointers are device pointers owned by the caller; the library never
 *    frees them.  "h_" pointers are host pointers.  Batched arrays are `batch`
 *    images (or sinograms) stored back to back.
 *  - Work is enqueued on `stream` (a cudaStream_t, NULL = legacy default
 *    stream) and is asynchronous unless the entry point says otherwise.
 *  - Every entry point returns SUPCG_OK (0) or a negative supcg_status.  No
 *    entry point aborts the process or throws.  After an error the outputs
 *    are unspecified; the geometry stays valid.
 *  - Scratch memory is owned by the geometry object: allocated lazily on
 *    first use (cudaMalloc) and freed by supcg_destroy_geometry.  A geometry
 *    must not be used from two host threads at once.
 */
#ifndef SUPCG_H
#define SUPCG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct supcg_geometry_s *supcg_geometry;

typedef enum {
    SUPCG_OK = 0,
    SUPCG_ERR_ARG = -1,       /* invalid argument (null pointer, size, parameter range) */
    SUPCG_ERR_CUDA = -2,      /* a CUDA runtime/driver call failed                        */
    SUPCG_ERR_NOMEM = -3,     /* device or host allocation failed                         */
    SUPCG_ERR_BREAKDOWN = -4, /* CG breakdown: p^T h <= 0 or a non-finite scalar          */
    SUPCG_ERR_BACKTRACK = -5, /* S_TV backtracking exceeded max_trials (Algorithm 1)      */
    SUPCG_ERR_TIMEOUT = -6,   /* a bounded device-side wait expired                       */
    SUPCG_ERR_PRECOND = -7,   /* preconditioner parameters outside 1/2 < rho <= 1, mu >= 0 */
    SUPCG_ERR_UNSUPPORTED = -8/* geometry outside the kernels' supported range             */
} supcg_status;

typedef enum { SUPCG_F32 = 0, SUPCG_BF16 = 1 } supcg_storage;

/* Create a 2-D parallel-beam geometry (Sec. 2, Sec. 4.1).
 *   nx, ny          image size in pixels (1 .. 16384 each)
 *   pixel_size      d > 0 (the unit-square convention is d = 1/max(nx, ny))
 *   n_views         1 <= V <= 2^20
 *   angles          host array of V angles in radians, or NULL for v*pi/V
 *                   (V equally spaced angles in [0, pi), as in Sec. 4.1)
 *   n_bins          1 <= U <= 2^21 (bin indices stay below 2^22, where one FP32
 *                   addition rounded upward gives their ceiling exactly)
 *   bin_spacing     ds; <= 0 selects ds = d (ray spacing = pixel size, Sec. 4.1)
 *   det_center_offset  off, added to every s_u
 *   storage         SUPCG_F32 or SUPCG_BF16: element type of the images and
 *                   sinograms passed to supcg_project / supcg_backproject
 * The host copies everything it needs; `angles` may be freed afterwards.
 * cos/sin are evaluated in FP64 on the host and are exact at multiples of pi/2.
 * Errors: SUPCG_ERR_ARG, SUPCG_ERR_UNSUPPORTED (bins more than about 2.5 times
 * coarser or about 2 times finer than pixels: the projectors' shared-memory
 * windows have fixed maxima), SUPCG_ERR_CUDA, SUPCG_ERR_NOMEM. */
int supcg_create_geometry(int nx, int ny, double pixel_size, int n_views, const double *angles,
                          int n_bins, double bin_spacing, double det_center_offset,
                          int storage, supcg_geometry *out);

/* Tiling of the forward projector: rays (bins) per thread block, one of 32,
 * 64, 96, 128 (default: the largest whose staged box fits).  Results do not
 * depend on it (every ray sums its row terms in the same order).  Setting it
 * frees the geometry's scratch (rebuilt on next use).  Used by the autotuner.
 * Errors: SUPCG_ERR_ARG, SUPCG_ERR_UNSUPPORTED (box wider than 256 columns). */
int supcg_set_tiling(supcg_geometry g, int fwd_bins_per_block);
int supcg_get_tiling(supcg_geometry g, int *fwd_bins_per_block);

/* Tiling of the backprojector: thread blocks per 32 x 32 pixel tile (1 .. 8,
 * default 4), each summing a contiguous share of the views, combined per
 * pixel in a fixed order by the tile's last block.  More parts give a grid of
 * more, shorter blocks (a smaller idle tail when the last wave is partial) at
 * the cost of more partial sums.  The choice changes the order in which a
 * pixel's views are added, so results differ from one setting to another in
 * the last bits (each setting is deterministic and stays the exact transpose
 * of supcg_project).  Setting it frees the geometry's scratch.  Used by the
 * autotuner.  Errors: SUPCG_ERR_ARG. */
int supcg_set_bwd_parts(supcg_geometry g, int parts);
int supcg_get_bwd_parts(supcg_geometry g, int *parts);

/* Mirror pairs of views found at creation: views theta and pi - theta (cos of
 * opposite sign, sin equal, both within 1e-12; for the default angles v pi / V,
 * views v and V - v).  Such a pair's rays meet the left-right mirrored image
 * with the same weights, so the forward projector evaluates them once for both
 * views (the second view's cos is set to exactly minus the first's, a change of
 * at most 1e-12 in the geometry).  *pairs receives their number (0: none).
 * Errors: SUPCG_ERR_ARG. */
int supcg_get_mirror_pairs(supcg_geometry g, int *pairs);

/* Free the geometry and all scratch it owns (synchronises the device first). */
int supcg_destroy_geometry(supcg_geometry g);

/* Forward projection y = R x for `batch` images (the product R x of Sec. 2).
 *   d_x  [batch][ny][nx]   d_y [batch][V][U]   (storage type of the geometry)
 * Exact line-pixel intersection lengths, FP32 accumulation. */
int supcg_project(supcg_geometry g, const void *d_x, void *d_y, int batch, void *stream);

/* Backprojection x = R^T y (the transpose in the normal equations, Eq. (2.2)).
 * Uses bit-identical weights to supcg_project: it is the exact transpose of
 * the matrix applied there.  d_y [batch][V][U] -> d_x [batch][ny][nx]. */
int supcg_backproject(supcg_geometry g, const void *d_y, void *d_x, int batch, void *stream);

/* Preconditioner z = M g, M = F^-1 D F, D = h(w) of Eq. (3.2) with
 * h(w) = (|w| + mu)(rho + (1 - rho) cos w), w the radial frequency of the
 * ny x nx DFT clamped to pi.  d_g, d_z FP32 [batch][ny][nx]; may alias.
 * Accepted parameters: 1/2 < rho <= 1, mu finite and >= 0 (h(w) > 0 on [0, pi]: M
 * is symmetric positive definite).  Errors: SUPCG_ERR_PRECOND outside that range. */
int supcg_precondition(supcg_geometry g, double mu, double rho, const float *d_g, float *d_z,
                       int batch, void *stream);

/* Preconditioner z = M g for callers that must not allocate device memory:
 * code that runs under a fixed, pre-reserved memory budget, inside a host
 * framework that owns every allocation, or on a path where cudaMalloc is
 * forbidden because it can synchronise the device.  The paper has no
 * counterpart; this is a packaging of supcg_precondition for those callers.
 *   ny, nx   image size, each 1 .. 512 (larger sizes return
 *            SUPCG_ERR_UNSUPPORTED); d_g, d_z FP32 [ny][nx], caller-owned
 * It needs no geometry object and calls no allocating routine: its scratch
 * (4 MiB + 16 KiB of FP64 complex values) is one static device array that
 * the library reserves on every GPU that loads it, until the process exits.
 * The first call on each device (and the first after that device's context
 * has been replaced, e.g. by cudaDeviceReset) looks that array's device
 * address up (cudaGetSymbolAddress) and sets kernel attributes; make that
 * first call before any stream capture.  All calls share the array: calls whose work
 * overlaps on the GPU (for example on two streams) race and give wrong
 * results.  Asynchronous on `stream`.  Accepted parameters: 1/2 < rho <= 1,
 * mu finite and >= 0.  Errors: SUPCG_ERR_ARG, SUPCG_ERR_UNSUPPORTED,
 * SUPCG_ERR_PRECOND (rho or mu outside that range), SUPCG_ERR_CUDA. */
int supcg_precondition_noalloc(int ny, int nx, double mu, double rho, const float *d_g, float *d_z,
                               void *stream);

/* Total variation and its nonascending vector (Sec. 3.1) for one image:
 * d_tbar[p] = -dTV/dy_p where that partial derivative exists, else 0.
 * h_out[0] = TV(y), h_out[1] = ||tbar||^2 (FP64 reductions).  Synchronous. */
int supcg_tv_tbar(supcg_geometry g, const float *d_y, float *d_tbar, double *h_out, void *stream);

/* S_TV(x, l, a, gamma, K), Algorithm 1, in place: d_x <- x + s (one image).
 *   h_ell        in: l, out: l after the call
 *   h_trials     nullable host array of K ints: trials of each nonascending step
 *   max_trials   bound on each `repeat` loop (the paper gives none);
 *                exceeding it returns SUPCG_ERR_BACKTRACK.
 * Synchronous (reads the new l back). */
int supcg_superiorize(supcg_geometry g, float *d_x, double a, double gamma, int K,
                      long long max_trials, long long *h_ell, int *h_trials, void *stream);

/* Parameters of supcg_solve (Algorithm 3 inputs plus the preconditioner of Eq. (3.2)). */
typedef struct {
    int K;                 /* nonascending steps per S_TV call (Algorithm 1)             */
    double a;              /* step-length diminishing factor, 0 < a < 1                   */
    double gamma;          /* starting step length, >= 0 (0 with perturb=0: plain PCG)    */
    double mu, rho;        /* preconditioner parameters of Eq. (3.2); rho > 1/2           */
    double eps;            /* stop when f(x_{k-1/2}) <= eps; eps < 0: never (fixed budget) */
    int max_iter;          /* bound on executions of the while body of Algorithm 3        */
    long long max_trials;  /* bound on each backtracking loop of Algorithm 1 (e.g. 10000)  */
    int perturb;           /* 1: SupPCG; 0: skip S_TV (plain PCG)                         */
    int precondition;      /* 1: M of Eq. (3.2); 0: M = I (SupCG / CG)                     */
    int graph;             /* 1: replay each iteration as a captured CUDA graph            */
    double bayes_r;        /* > 0: minimise the Bayesian criterion of Eq. (2.3),
                            *   r^2 ||R x - b||^2 + ||x - mu_X||^2 (r = bayes_r, the
                            *   signal-to-noise ratio), instead of ||R x - b||^2; every f
                            *   (eps test, report, log) is then that criterion.  <= 0: least squares */
    double bayes_mu;       /* mu_X, the gray level of Eq. (2.3); NaN: estimated from b on the
                            *   device as the image average the data imply (mean over views of
                            *   sum_u b ds, over the image area)                              */
} supcg_params;

/* Outcome of a solve. */
typedef struct {
    int iters;          /* executions of the while body (steps 11-14)                    */
    int k;              /* the k returned by Algorithm 3                                 */
    long long ell;      /* l_k after the last body                                       */
    double f_last;      /* f(x_{k-1/2}) = ||R x_{k-1/2} - b||^2 of the returned image     */
    double f0;          /* f(x_0)                                                        */
    double tv_last;     /* TV(x_{k-1/2})  (0 unless perturb = 1 and iters > 0)            */
    int status;         /* SUPCG_OK or the error that stopped the iteration              */
    int n_fallback;     /* supcg_solve_learned: proposals rejected by the nonascent test  */
    int n_learned;      /* supcg_solve_learned: proposals accepted                        */
} supcg_report;

/* Number of doubles per iteration written to the optional log of supcg_solve:
 * f(x_{k+1/2}), TV(x_k), TV(x_{k+1/2}), l_{k+1}, alpha, beta, ||s_k||^2, trials. */
#define SUPCG_LOG_STRIDE 8

/* SupPCG(x0, a, gamma, K, eps), Algorithm 3 (steps 1-9 then the while loop;
 * U_PCG of Algorithm 2; S_TV of Algorithm 1), for one problem.
 *   d_b    FP32 [V][U] measured data b
 *   d_x    FP32 [ny][nx]; in: x_0, out: x_{k-1/2} (the image Algorithm 3 returns)
 *   d_log  nullable FP64 [max_iter][SUPCG_LOG_STRIDE] per-iteration metrics
 * CG scalars (alpha, beta, inner products, f) are reduced in FP64.
 * Synchronous: returns after the report has been read back. */
int supcg_solve(supcg_geometry g, const float *d_b, float *d_x, const supcg_params *p,
                supcg_report *rep, double *d_log, void *stream);

/* supcg_solve with HOST buffers: copies h_b and h_x (x_0) to the device,
 * solves, and copies x_{k-1/2} back into h_x.  Page-locked host memory gives
 * the fastest copies.  The device copies are allocated on the first call and
 * kept with the geometry until it is destroyed.  Synchronous. */
int supcg_solve_host(supcg_geometry g, const float *h_b, float *h_x, const supcg_params *p,
                     supcg_report *rep, void *stream);

/* Solve `count` independent problems of possibly different geometries in one
 * set of batched launches: every kernel of an iteration processes all
 * problems at once, and the iteration is replayed as one CUDA graph.
 *   gs[c], d_b[c], d_x[c]  geometry, data and image (in x_0, out x_{k-1/2}) of problem c
 *   reps   host array of `count` reports
 * All problems share the parameters p.  The scratch lives in gs[0].
 * Synchronous. */
int supcg_solve_batched(const supcg_geometry *gs, const float *const *d_b, float *const *d_x,
                        int count, const supcg_params *p, supcg_report *reps, void *stream);

/* Parameter sweep (Sec. 4.2, algorithmic parameter selection): `count` solves of
 * the same problem (geometry g, data d_b) in one set of batched launches, solve c
 * with the S_TV parameters K, a, gamma and the preconditioner parameters mu, rho
 * of ps[c]; every other field must equal ps[0]'s (the shared loop control), else
 * SUPCG_ERR_ARG.
 *   d_x[c]   FP32 [ny][nx] image of solve c (in x_0, out x_{k-1/2}), caller-owned
 *   d_ref    nullable FP32 [ny][nx] reference image (the phantom x-dagger): with it,
 *            the selective error of Eq. (4.1) with C = 1,
 *              SE(x) = sqrt(sum over (i,j) in S of (x_ij - ref_ij)^2),
 *            S = the pixels whose centres lie in the centred ellipse of horizontal
 *            semi-axis se_ax * nx and vertical semi-axis se_ay * ny pixels, is
 *            written for x_{k+1/2} of every while-body k (1-based) of solve c to
 *            d_se[c * max_iter + k - 1] (FP64, device, caller-owned, count * max_iter)
 *   reps     host array of `count` reports
 * The scratch lives in g (one workspace per solve).  Synchronous. */
int supcg_solve_sweep(supcg_geometry g, const float *d_b, float *const *d_x, int count,
                      const supcg_params *ps, const float *d_ref, double se_ax, double se_ay,
                      double *d_se, supcg_report *reps, void *stream);

/* ART for the Bayesian criterion of Eq. (2.3) and SupART (Sec. 3.4, the
 * row-action method of Herman, Hurwitz and Lent with pixel basis functions).
 * From x = mu_X and one auxiliary value u_i = 0 per ray, each ray i updates
 *     c = lambda (r (b_i - <R_i, x>) - u_i) / (1 + r^2 ||R_i||^2),
 *     x <- x + r c R_i,   u_i <- u_i + c
 * (a sweep over r R (x - mu_X) + u = r (b - R mu_X), whose minimum-norm
 * solution minimises r^2 ||R x - b||^2 + ||x - mu_X||^2); one iteration is a
 * full cycle through the rays.  The paper does not fix the order of the
 * rays: here the views in order and, within a view, the rays in the residue
 * classes u = c (mod S), c = 0 .. S-1, with S = floor(2 max_v E_v) + 1 the
 * smallest bin spacing at which two rays of a view share no pixel (E_v =
 * (d/ds)(|cos|+|sin|)/2 the footprint half-width in bins); the rays of one
 * class touch disjoint pixels, so the GPU runs each class in parallel and the
 * result is that of any sequential order of the class.  R is the projectors'
 * matrix (same entries).  SupART (K > 0): before every cycle x <- S_TV(x, l,
 * a, gamma, K), Algorithm 1, from l = 0.  Table 1 of the paper lists r = 5,
 * lambda = 1e-2 for ART and K = 10, a = 1 - 1e-5, gamma = 1e-2, r = 5,
 * lambda = 5e-2 for SupART. */
typedef struct {
    double r;               /* signal-to-noise ratio of Eq. (2.3), > 0                     */
    double lambda;          /* relaxation, 0 < lambda < 2                                  */
    double mu;              /* prior mean mu_X, the starting image; NaN: estimated from b
                               (the data's gray level, as for supcg_params.bayes_mu)       */
    int cycles;             /* iterations (full cycles through the rays), >= 0             */
    int K;                  /* SupART: S_TV steps before every cycle; 0: ART               */
    double a, gamma;        /* SupART: S_TV parameters (Algorithm 1)                       */
    long long max_trials;   /* SupART: bound on each S_TV `repeat` loop                    */
} supcg_art_params;

typedef struct {
    int cycles;             /* cycles completed                                            */
    long long ell;          /* l after the last S_TV (SupART)                              */
    double mu;              /* the prior mean used                                         */
    int status;             /* SUPCG_OK or the first error                                 */
} supcg_art_report;

/* ART / SupART on one problem: d_b FP32 [V][U] (caller-owned), d_x FP32 [ny][nx]
 * out (x after `cycles` cycles).  The per-ray values u_i and 1 / (1 + r^2 ||R_i||^2)
 * (FP64, 16 bytes per ray) are kept with the geometry.  Synchronous.  Errors:
 * SUPCG_ERR_ARG, SUPCG_ERR_BACKTRACK (S_TV), SUPCG_ERR_TIMEOUT, SUPCG_ERR_NOMEM,
 * SUPCG_ERR_CUDA. */
int supcg_art(supcg_geometry g, const float *d_b, float *d_x, const supcg_art_params *p,
              supcg_art_report *rep, void *stream);

/* ------------------------------------------------------------------------
 * Learned perturbation network (an addition to the paper's method: the paper
 * perturbs along the normalised negative TV gradient, Sec. 3.1; this network
 * proposes a direction from the iterate and that gradient, and the solver
 * accepts it only when it is nonascending for TV).
 *
 * Five 3x3 convolutions (zero padding), channels 2 -> 32 -> 32 -> 32 -> 32 -> 1,
 * ReLU after the first four, output added to the scaled input direction.
 * Input: the image x scaled to unit RMS and tbar (Sec. 3.1) scaled to unit
 * RMS; output: the proposed direction at unit-RMS scale.  BF16 weights and
 * activations, FP32 accumulation (tensor cores), FP32 master weights (Adam).
 * Parameters, as a flat FP32 array: for each layer W[cout][cin][3][3] then
 * b[cout].  A network is created for images of ny x nx and up to max_batch
 * images per call; it owns its device memory.
 * ------------------------------------------------------------------------ */
typedef struct supcg_cnn_s *supcg_cnn;

/* Create a network with seeded initial weights (last layer zero: the untrained
 * network returns the plain direction).  Errors: SUPCG_ERR_ARG, _NOMEM, _CUDA. */
int supcg_cnn_create(int ny, int nx, int max_batch, unsigned long long seed, supcg_cnn *out);
int supcg_cnn_destroy(supcg_cnn net);
/* Number of FP32 parameters (length of the flat array). */
int supcg_cnn_num_params(supcg_cnn net);
int supcg_cnn_get_params(supcg_cnn net, float *h_params);
int supcg_cnn_set_params(supcg_cnn net, const float *h_params);
/* Forward pass for `count` images: d_x, d_tbar, d_out FP32 [count][ny][nx]. */
int supcg_cnn_forward(supcg_cnn net, const float *d_x, const float *d_tbar, int count, float *d_out,
                      void *stream);
/* Gradients of the mean squared error between the output and d_target
 * (scaled per image to unit RMS inside the call) with respect to all
 * parameters (host array, flat layout);
 * *h_loss receives the loss.  Synchronous. */
int supcg_cnn_gradients(supcg_cnn net, const float *d_x, const float *d_tbar, const float *d_target, int count,
                        float *h_grads, double *h_loss, void *stream);
/* One Adam step (lr, beta1 0.9, beta2 0.999) on the same loss.  h_loss nullable
 * (when given, the call synchronises to read it). */
int supcg_cnn_train_step(supcg_cnn net, const float *d_x, const float *d_tbar, const float *d_target, int count,
                         double lr, double *h_loss, void *stream);

/* supcg_solve that also records x_k (the iterate S_TV receives) of every while
 * body into d_trace [max_iter][ny][nx] (FP32, caller-owned): training data for
 * the learned direction.  Synchronous. */
int supcg_solve_trace(supcg_geometry g, const float *d_b, float *d_x, const supcg_params *p,
                      supcg_report *rep, double *d_log, float *d_trace, void *stream);

/* SupPCG with the learned direction: every while body computes tbar at x_k
 * (Sec. 3.1), runs the network on (x_k, tbar), and tests the proposal t with
 * the exact one-sided directional derivative D_TV(x_k; t).  If D_TV < 0 (t is
 * nonascending for TV at x_k), one step along t/||t|| of length
 * 2^-j gamma * sum_{i<K} a^(l+i) is taken, j = 0, 1, ... until TV does not
 * increase (the test of Algorithm 1), and l advances by K + j, which keeps the
 * bound of Theorem 1; otherwise the plain K steps of Algorithm 1 run.  The network must
 * have been created for this geometry's image size; nx must be a multiple of
 * 4.  rep->n_learned / n_fallback count the two outcomes.  Synchronous. */
int supcg_solve_learned(supcg_geometry g, supcg_cnn net, const float *d_b, float *d_x,
                        const supcg_params *p, supcg_report *rep, double *d_log, void *stream);

/* The learned direction in a batched solve: `count` independent problems of
 * possibly different views and bins but the network's image size, solved as
 * supcg_solve_batched does (every kernel of an iteration over all problems,
 * one graph per iteration), with the network run once per iteration over
 * all problems' (x_k, tbar) as one batch.  Each problem's proposal is tested
 * and used as in supcg_solve_learned, so every problem's iterates equal those
 * of supcg_solve_learned on it alone.
 *   gs[c], d_b[c], d_x[c]  geometry, data and image (in x_0, out x_{k-1/2}) of problem c
 *   reps   host array of `count` reports (n_learned / n_fallback per problem)
 * Requires count <= the network's max_batch, every image ny x nx equal to the
 * network's and nx a multiple of 4.  The scratch (including the network's
 * input batch, 2 count ny nx floats) lives in gs[0].  Synchronous.  Errors:
 * SUPCG_ERR_ARG, SUPCG_ERR_UNSUPPORTED (image size), and those of supcg_solve. */
int supcg_solve_batched_learned(const supcg_geometry *gs, supcg_cnn net, const float *const *d_b,
                                float *const *d_x, int count, const supcg_params *p, supcg_report *reps,
                                void *stream);

/* Kernel kinds of supcg_solve_profiled. */
typedef enum {
    SUPCG_KIND_FORWARD = 0,  /* forward projector (R x with residual, R p with ||R p||^2)   */
    SUPCG_KIND_BACKWARD = 1, /* backprojector (R^T r, R^T q)                               */
    SUPCG_KIND_FFT = 2,      /* preconditioner passes                                      */
    SUPCG_KIND_STV = 3,      /* S_TV (Algorithm 1)                                         */
    SUPCG_KIND_VECTOR = 4,   /* axpys, inner products, transposes, staging, bookkeeping    */
    SUPCG_KIND_CNN = 5,      /* learned-direction network (supcg_solve_learned)            */
    SUPCG_KIND_COUNT = 6
} supcg_kernel_kind;

/* supcg_solve without graph replay and with a CUDA event pair around every
 * kernel launch (the same kernels and launch shapes as supcg_solve).
 *   h_ms        host [SUPCG_KIND_COUNT]: total device milliseconds per kind
 *   h_launches  host [SUPCG_KIND_COUNT]: launches per kind
 * Synchronous.  The events perturb the schedule slightly; use supcg_solve for
 * throughput and this call for the per-kernel breakdown. */
int supcg_solve_profiled(supcg_geometry g, const float *d_b, float *d_x, const supcg_params *p,
                         supcg_report *rep, double *h_ms, long long *h_launches, void *stream);

/* Number of kernels the library has enqueued in this process so far (a CUDA
 * graph replay counts every kernel node it launches). */
long long supcg_kernel_launches(void);

/* Bounded device-side waits.  The repeat loop of Algorithm 1 (S_TV) has no
 * bound in the paper; here it runs on the device in one cooperative launch
 * whose blocks meet at grid barriers, and ART's ray classes (Sec. 3.4) meet
 * at the same kind of barrier.  Each wait polls a flag at most `polls` times
 * (each poll sleeps about 64 ns; the default, 2^24 polls, is a second or
 * two) and then gives up: the kernel records SUPCG_ERR_TIMEOUT, leaves, and
 * the call returns that status (the context stays usable and the next call
 * starts from a clean barrier).  The setting is process-wide and read by
 * every call when it starts.  The paper has no counterpart.
 * Errors: SUPCG_ERR_ARG when polls < 1. */
int supcg_set_wait_limit(long long polls);

/* Test hook for the timeout path above: with extra_blocks > 0 every
 * cooperative grid barrier waits for extra_blocks more arrivals than its
 * launch has blocks, so no barrier is ever released and every wait runs to
 * the limit of supcg_set_wait_limit (no copy or memory access is left in
 * flight: the blocks only poll).  0 (the default) restores normal barriers.
 * Process-wide; for tests of the error path only.  The paper has no
 * counterpart.  Errors: SUPCG_ERR_ARG outside 0 .. 1024. */
int supcg_set_barrier_shortfall(int extra_blocks);

/* Human-readable name of a status code (static string). */
const char *supcg_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* SUPCG_H */
