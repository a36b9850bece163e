/*
 * SupPCG oracle: plain, slow, FP64 CPU reference of the method of
 * Helou, Herman, Lin, Zibetti, "Superiorization of preconditioned conjugate
 * gradient algorithms for tomographic image reconstruction" (arXiv 1807.10151).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * What each function follows (paper sections / equations / algorithms):
 *   - data model R x = b + e, R the projection (Radon) matrix ........ Sec. 2
 *   - least squares f(x) = ||Rx - b||^2, normal equations R^T R x = R^T b
 *                                                         Eq. (2.1), (2.2)
 *   - Bayesian criterion f(x) = r^2 ||Rx - b||^2 + ||x - mu_X||^2 ... Eq. (2.3)
 *   - acquisition shape (parallel rays, equally spaced angles in [0,pi),
 *     ray spacing = pixel size) ............................. Sec. 4.1
 *   - total variation TV(y) and the nonascending vector t ...... Sec. 3.1
 *   - S_TV(x, l, a, gamma, K) ................................... Algorithm 1
 *   - U_PCG(x, p, h) ............................................ Algorithm 2
 *   - M = F^-1 D F with h(w) = (|w|+mu)(rho+(1-rho)cos w) ....... Eq. (3.2)
 *   - SupPCG(x0, a, gamma, K, eps) .............................. Algorithm 3
 *   - ART for the Bayesian criterion (the row-action method of Herman,
 *     Hurwitz and Lent that Sec. 3.4 uses) and its superiorization SupART
 *                                                          Sec. 3.4, Eq. (2.3)
 *
 * The paper leaves the entries of R to its software package.  Here R_{ray,pixel}
 * is the Euclidean length of the intersection of the ray (a straight line) with
 * the closed pixel square, obtained by parametric slab clipping of the line
 * against the square (Liang-Barsky).  A line that runs exactly along an edge
 * shared by two pixels gives half of the edge length to each of them (and half
 * to a boundary pixel whose outer edge it runs along): the mean of the lengths
 * seen by lines just to either side.  The paper is silent on that case.
 *
 * Conventions (readings of the paper where it is silent):
 *   - image [ny][nx] row-major, component c(i-1)+j is pixel (i, j) (Sec. 3.1);
 *     row 0 is the top row; pixel (i, j) has centre
 *         x_j = (j - (nx-1)/2) d,   y_i = ((ny-1)/2 - i) d;
 *   - view v at angle theta_v; cos/sin are exact at integer multiples of pi/2;
 *   - bin u of every view at detector coordinate
 *         s_u = (u - (U-1)/2) ds + off;
 *   - ray (v, u) is the line { (x, y) : x cos theta_v + y sin theta_v = s_u }.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_NOMEM (-3)
#define ORC_ERR_BREAKDOWN (-4)
#define ORC_ERR_BACKTRACK (-5)

static const double ORC_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------ */
/* Geometry (Sec. 2, Sec. 4.1)                                          */
/* ------------------------------------------------------------------ */

/* cos/sin of a view angle, exact at integer multiples of pi/2 so that the
 * axis-aligned views of a uniformly sampled [0, pi) are exactly axis-aligned. */
static void view_cos_sin(double th, double *c, double *s)
{
    double q = th / (0.5 * ORC_PI);
    double r = nearbyint(q);
    if (fabs(q - r) < 1e-12) {
        long k = ((long)r % 4 + 4) % 4;
        static const double cc[4] = {1.0, 0.0, -1.0, 0.0};
        static const double ss[4] = {0.0, 1.0, 0.0, -1.0};
        *c = cc[k];
        *s = ss[k];
    } else {
        *c = cos(th);
        *s = sin(th);
    }
}

/* Length of  { x c + y s = sv }  inside the closed box [xl,xr] x [yb,yt]. */
static double line_box_length(double c, double s, double sv,
                              double xl, double xr, double yb, double yt)
{
    if (s == 0.0) { /* vertical line x = sv / c, c = +-1 */
        double x = sv / c;
        if (x > xl && x < xr) return yt - yb;
        if (x == xl || x == xr) return 0.5 * (yt - yb);
        return 0.0;
    }
    if (c == 0.0) { /* horizontal line y = sv / s, s = +-1 */
        double y = sv / s;
        if (y > yb && y < yt) return xr - xl;
        if (y == yb || y == yt) return 0.5 * (xr - xl);
        return 0.0;
    }
    /* point on the line closest to the origin, unit direction along it */
    double px = sv * c, py = sv * s;
    double dx = -s, dy = c;
    double ta = (xl - px) / dx, tb = (xr - px) / dx;
    double tc = (yb - py) / dy, td = (yt - py) / dy;
    double lo_x = ta < tb ? ta : tb, hi_x = ta < tb ? tb : ta;
    double lo_y = tc < td ? tc : td, hi_y = tc < td ? td : tc;
    double lo = lo_x > lo_y ? lo_x : lo_y;
    double hi = hi_x < hi_y ? hi_x : hi_y;
    return hi > lo ? hi - lo : 0.0;
}

typedef struct {
    int nx, ny;
    double d;
    int V;
    const double *theta;
    int U;
    double ds, off;
} orc_geom;

static double bin_coord(const orc_geom *g, int u)
{
    return ((double)u - 0.5 * (double)(g->U - 1)) * g->ds + g->off;
}

/* Walk one ray over the image; for every pixel with a nonzero intersection
 * call emit(pixel index, length).  Rows are visited top to bottom and, within
 * a row, columns left to right.  The candidate column range per row is a
 * superset (one extra column each side); the clipping decides. */
typedef void (*emit_fn)(void *ctx, int pix, double w);

static void walk_ray(const orc_geom *g, int v, int u, emit_fn emit, void *ctx)
{
    double c, s;
    view_cos_sin(g->theta[v], &c, &s);
    double sv = bin_coord(g, u);
    double d = g->d;
    double W = g->nx * d;
    for (int i = 0; i < g->ny; ++i) {
        /* edges as (integer - half-count) * d: a shared edge has one value */
        double yt = (0.5 * g->ny - i) * d, yb = (0.5 * g->ny - i - 1) * d;
        int j0, j1;
        if (c == 0.0) {
            j0 = 0;
            j1 = g->nx - 1;
        } else {
            double xa = (sv - yb * s) / c, xb = (sv - yt * s) / c;
            double xmin = xa < xb ? xa : xb, xmax = xa < xb ? xb : xa;
            j0 = (int)floor((xmin + 0.5 * W) / d) - 1;
            j1 = (int)floor((xmax + 0.5 * W) / d) + 1;
            if (j0 < 0) j0 = 0;
            if (j1 > g->nx - 1) j1 = g->nx - 1;
        }
        for (int j = j0; j <= j1; ++j) {
            double xl = (j - 0.5 * g->nx) * d, xr = (j + 1 - 0.5 * g->nx) * d;
            double w = line_box_length(c, s, sv, xl, xr, yb, yt);
            if (w > 0.0) emit(ctx, i * g->nx + j, w);
        }
    }
}

static void emit_count(void *ctx, int pix, double w)
{
    (void)pix;
    (void)w;
    ++*(long *)ctx;
}

typedef struct { int *col; double *val; long k; } fill_ctx;
static void emit_fill(void *ctx, int pix, double w)
{
    fill_ctx *f = (fill_ctx *)ctx;
    f->col[f->k] = pix;
    f->val[f->k] = w;
    ++f->k;
}

typedef struct { const double *x; double acc; } dot_ctx;
static void emit_dot(void *ctx, int pix, double w)
{
    dot_ctx *f = (dot_ctx *)ctx;
    f->acc += w * f->x[pix];
}

static orc_geom mkgeom(int nx, int ny, double d, int V, const double *theta,
                       int U, double ds, double off)
{
    orc_geom g;
    g.nx = nx; g.ny = ny; g.d = d; g.V = V; g.theta = theta;
    g.U = U; g.ds = ds; g.off = off;
    return g;
}

/* Number of nonzeros of each row of R (rows = rays v*U+u); rowptr[m+1]. */
long orc_csr_rowptr(int nx, int ny, double d, int V, const double *theta,
                    int U, double ds, double off, long *rowptr)
{
    orc_geom g = mkgeom(nx, ny, d, V, theta, U, ds, off);
    long m = (long)V * U;
#pragma omp parallel for schedule(dynamic, 16)
    for (long r = 0; r < m; ++r) {
        long cnt = 0;
        walk_ray(&g, (int)(r / U), (int)(r % U), emit_count, &cnt);
        rowptr[r + 1] = cnt;
    }
    rowptr[0] = 0;
    for (long r = 0; r < m; ++r) rowptr[r + 1] += rowptr[r];
    return rowptr[m];
}

/* Column indices and values of R given rowptr from orc_csr_rowptr. */
void orc_csr_fill(int nx, int ny, double d, int V, const double *theta,
                  int U, double ds, double off, const long *rowptr,
                  int *col, double *val)
{
    orc_geom g = mkgeom(nx, ny, d, V, theta, U, ds, off);
    long m = (long)V * U;
#pragma omp parallel for schedule(dynamic, 16)
    for (long r = 0; r < m; ++r) {
        fill_ctx f;
        f.col = col + rowptr[r];
        f.val = val + rowptr[r];
        f.k = 0;
        walk_ray(&g, (int)(r / U), (int)(r % U), emit_fill, &f);
    }
}

/* Explicit transpose of a CSR matrix (m rows, n columns) into CSR of R^T. */
void orc_csr_transpose(long m, long n, const long *rp, const int *ci,
                       const double *va, long *rpt, int *cit, double *vat)
{
    long nnz = rp[m];
    for (long j = 0; j <= n; ++j) rpt[j] = 0;
    for (long k = 0; k < nnz; ++k) rpt[ci[k] + 1]++;
    for (long j = 0; j < n; ++j) rpt[j + 1] += rpt[j];
    long *pos = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
    for (long j = 0; j < n; ++j) pos[j] = rpt[j];
    for (long r = 0; r < m; ++r)
        for (long k = rp[r]; k < rp[r + 1]; ++k) {
            long dst = pos[ci[k]]++;
            cit[dst] = (int)r;
            vat[dst] = va[k];
        }
    free(pos);
}

/* y = A x for a CSR matrix with `rows` rows. */
void orc_spmv(long rows, const long *rp, const int *ci, const double *va,
              const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (long r = 0; r < rows; ++r) {
        double acc = 0.0;
        for (long k = rp[r]; k < rp[r + 1]; ++k) acc += va[k] * x[ci[k]];
        y[r] = acc;
    }
}

/* Ray sums of selected rays (ray id = v*U + u) without storing R. */
void orc_project_rays(int nx, int ny, double d, int V, const double *theta,
                      int U, double ds, double off, const double *x,
                      long nrays, const long *rays, double *out)
{
    orc_geom g = mkgeom(nx, ny, d, V, theta, U, ds, off);
#pragma omp parallel for schedule(dynamic, 4)
    for (long k = 0; k < nrays; ++k) {
        dot_ctx c;
        c.x = x;
        c.acc = 0.0;
        walk_ray(&g, (int)(rays[k] / U), (int)(rays[k] % U), emit_dot, &c);
        out[k] = c.acc;
    }
}

/* Entries of R^T y at selected pixels (pixel id = i*nx + j), by clipping every
 * ray of every view against that pixel: the column of R, computed directly. */
void orc_backproject_pixels(int nx, int ny, double d, int V, const double *theta,
                            int U, double ds, double off, const double *y,
                            long npix, const long *pix, double *out)
{
    orc_geom g = mkgeom(nx, ny, d, V, theta, U, ds, off);
#pragma omp parallel for schedule(dynamic, 1)
    for (long k = 0; k < npix; ++k) {
        int i = (int)(pix[k] / nx), j = (int)(pix[k] % nx);
        double xl = (j - 0.5 * nx) * d, xr = (j + 1 - 0.5 * nx) * d;
        double yt = (0.5 * ny - i) * d, yb = (0.5 * ny - i - 1) * d;
        double acc = 0.0;
        for (int v = 0; v < V; ++v) {
            double c, s;
            view_cos_sin(theta[v], &c, &s);
            for (int u = 0; u < U; ++u) {
                double w = line_box_length(c, s, bin_coord(&g, u), xl, xr, yb, yt);
                if (w > 0.0) acc += w * y[(long)v * U + u];
            }
        }
        out[k] = acc;
    }
}

/* ------------------------------------------------------------------ */
/* Total variation and the nonascending vector (Sec. 3.1)               */
/* ------------------------------------------------------------------ */

/* TV(y) = sum_{i<l-1, j<c-1} sqrt((y_ij - y_i+1,j)^2 + (y_ij - y_i,j+1)^2). */
double orc_tv(int ny, int nx, const double *y)
{
    double tv = 0.0;
    for (int i = 0; i + 1 < ny; ++i)
        for (int j = 0; j + 1 < nx; ++j) {
            double a = y[i * nx + j] - y[(i + 1) * nx + j];
            double b = y[i * nx + j] - y[i * nx + j + 1];
            tv += sqrt(a * a + b * b);
        }
    return tv;
}

/* tbar_p = -dTV/dy_p where that partial derivative exists, 0 otherwise.
 * The partial w.r.t. y_p exists iff every TV term containing y_p has a
 * nonzero square root (sum of squares exactly nonzero).  Returns TV(y). */
double orc_tv_tbar(int ny, int nx, const double *y, double *tbar)
{
    long n = (long)ny * nx;
    double *grad = (double *)calloc((size_t)n, sizeof(double));
    char *undef = (char *)calloc((size_t)n, 1);
    double tv = 0.0;
    for (int i = 0; i + 1 < ny; ++i)
        for (int j = 0; j + 1 < nx; ++j) {
            long p = (long)i * nx + j, pd = p + nx, pr = p + 1;
            double a = y[p] - y[pd];
            double b = y[p] - y[pr];
            double q = a * a + b * b;
            if (q == 0.0) {
                undef[p] = undef[pd] = undef[pr] = 1;
                continue;
            }
            double T = sqrt(q);
            tv += T;
            grad[p] += (a + b) / T;
            grad[pd] += -a / T;
            grad[pr] += -b / T;
        }
    for (long p = 0; p < n; ++p) tbar[p] = undef[p] ? 0.0 : -grad[p];
    free(grad);
    free(undef);
    return tv;
}

/* One-sided directional derivative of TV at y along t:
 *   sum over terms with nonzero root of <grad_ij y, grad_ij t> / root
 * + sum over terms with zero root of ||grad_ij t||,
 * grad_ij the pair of forward differences of the TV term (i, j).  t is a
 * nonascending direction (Sec. 3.1 definition) whenever this is < 0. */
double orc_tv_dirderiv(int ny, int nx, const double *y, const double *t)
{
    double dd = 0.0;
    for (int i = 0; i + 1 < ny; ++i)
        for (int j = 0; j + 1 < nx; ++j) {
            long p = (long)i * nx + j, pd = p + nx, pr = p + 1;
            double a = y[p] - y[pd], b = y[p] - y[pr];
            double ta = t[p] - t[pd], tb = t[p] - t[pr];
            double q = a * a + b * b;
            if (q == 0.0) dd += sqrt(ta * ta + tb * tb);
            else dd += (a * ta + b * tb) / sqrt(q);
        }
    return dd;
}

/* S_TV(x, l, a, gamma, K), Algorithm 1.  Writes s = y - x and the new l.
 * The paper's `repeat` loop has no bound; here each `repeat` may take at most
 * max_trials trials (ORC_ERR_BACKTRACK otherwise).  trials_log[i] (nullable)
 * receives the number of trials of the i-th nonascending step. */
int orc_stv(int ny, int nx, const double *x, long ell_in, double a, double gamma,
            int K, long max_trials, double *s_out, long *ell_out, long *trials_log)
{
    long n = (long)ny * nx;
    double *y = (double *)malloc(sizeof(double) * (size_t)n);
    double *t = (double *)malloc(sizeof(double) * (size_t)n);
    double *yt = (double *)malloc(sizeof(double) * (size_t)n);
    if (!y || !t || !yt) { free(y); free(t); free(yt); return ORC_ERR_NOMEM; }
    memcpy(y, x, sizeof(double) * (size_t)n);
    long ell = ell_in;
    int rc = ORC_OK;
    for (int i = 0; i < K; ++i) {
        /* t in the nonascending set: normalised tbar, or zero */
        double tv_y = orc_tv_tbar(ny, nx, y, t);
        double nrm2 = 0.0;
        for (long p = 0; p < n; ++p) nrm2 += t[p] * t[p];
        double nrm = sqrt(nrm2);
        for (long p = 0; p < n; ++p) t[p] = (nrm != 0.0) ? t[p] / nrm : 0.0;
        long trials = 0;
        for (;;) {
            if (trials >= max_trials) { rc = ORC_ERR_BACKTRACK; goto done; }
            double gt = gamma * pow(a, (double)ell);
            for (long p = 0; p < n; ++p) yt[p] = y[p] + gt * t[p];
            ++ell;
            ++trials;
            if (orc_tv(ny, nx, yt) <= tv_y) break;
        }
        if (trials_log) trials_log[i] = trials;
        memcpy(y, yt, sizeof(double) * (size_t)n);
    }
done:
    for (long p = 0; p < n; ++p) s_out[p] = y[p] - x[p];
    *ell_out = ell;
    free(y); free(t); free(yt);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Preconditioner M = F^-1 D F, Eq. (3.2)                               */
/* ------------------------------------------------------------------ */

/* D[k1*nx + k2] = h(w_r), w_i = 2 pi k_i / N_i taken in [-pi, pi],
 * w_r = min(sqrt(w1^2 + w2^2), pi),  h(w) = (|w| + mu)(rho + (1-rho) cos w). */
void orc_precond_D(int ny, int nx, double mu, double rho, double *D)
{
    for (int k1 = 0; k1 < ny; ++k1)
        for (int k2 = 0; k2 < nx; ++k2) {
            int m1 = k1 < ny - k1 ? k1 : ny - k1;
            int m2 = k2 < nx - k2 ? k2 : nx - k2;
            double w1 = 2.0 * ORC_PI * m1 / ny, w2 = 2.0 * ORC_PI * m2 / nx;
            double wr = sqrt(w1 * w1 + w2 * w2);
            if (wr > ORC_PI) wr = ORC_PI;
            D[(long)k1 * nx + k2] = (wr + mu) * (rho + (1.0 - rho) * cos(wr));
        }
}

/* In-place 1-D DFT of `len` complex values at stride `st` (sign -1 forward,
 * +1 inverse, unscaled), by the defining sum with a libm twiddle table. */
static void dft1(double *re, double *im, int len, long st, int sign,
                 const double *cw, const double *sw, double *tr, double *ti)
{
    for (int k = 0; k < len; ++k) {
        double ar = 0.0, ai = 0.0;
        for (int q = 0; q < len; ++q) {
            long e = ((long)k * q) % len;
            double c = cw[e], s = sign * sw[e];
            double xr = re[q * st], xi = im[q * st];
            ar += xr * c - xi * s;
            ai += xr * s + xi * c;
        }
        tr[k] = ar;
        ti[k] = ai;
    }
    for (int k = 0; k < len; ++k) {
        re[k * st] = tr[k];
        im[k * st] = ti[k];
    }
}

static void dft2(double *re, double *im, int ny, int nx, int sign)
{
    int mx = nx > ny ? nx : ny;
    double *cx = malloc(sizeof(double) * nx), *sx = malloc(sizeof(double) * nx);
    double *cy = malloc(sizeof(double) * ny), *sy = malloc(sizeof(double) * ny);
    for (int e = 0; e < nx; ++e) { cx[e] = cos(2.0 * ORC_PI * e / nx); sx[e] = sin(2.0 * ORC_PI * e / nx); }
    for (int e = 0; e < ny; ++e) { cy[e] = cos(2.0 * ORC_PI * e / ny); sy[e] = sin(2.0 * ORC_PI * e / ny); }
#pragma omp parallel
    {
        double *tr = malloc(sizeof(double) * mx), *ti = malloc(sizeof(double) * mx);
#pragma omp for schedule(static)
        for (int i = 0; i < ny; ++i)
            dft1(re + (long)i * nx, im + (long)i * nx, nx, 1, sign, cx, sx, tr, ti);
#pragma omp for schedule(static)
        for (int j = 0; j < nx; ++j)
            dft1(re + j, im + j, ny, nx, sign, cy, sy, tr, ti);
        free(tr);
        free(ti);
    }
    free(cx); free(sx); free(cy); free(sy);
}

/* z = Re(F^-1 diag(D) F g) on the ny x nx grid (periodic, no padding). */
void orc_fourier_diag(int ny, int nx, const double *D, const double *g, double *z)
{
    long n = (long)ny * nx;
    double *re = malloc(sizeof(double) * n), *im = calloc((size_t)n, sizeof(double));
    memcpy(re, g, sizeof(double) * n);
    dft2(re, im, ny, nx, -1);
    for (long p = 0; p < n; ++p) { re[p] *= D[p]; im[p] *= D[p]; }
    dft2(re, im, ny, nx, +1);
    for (long p = 0; p < n; ++p) z[p] = re[p] / (double)n;
    free(re);
    free(im);
}

/* ------------------------------------------------------------------ */
/* SupPCG, Algorithm 3 (with U_PCG, Algorithm 2, and S_TV, Algorithm 1) */
/* ------------------------------------------------------------------ */

typedef struct {
    long m, n;
    const long *rp; const int *ci; const double *va;    /* R    (CSR) */
    const long *rpt; const int *cit; const double *vat; /* R^T  (CSR) */
    double r2, muX;   /* r2 > 0: Bayesian criterion of Eq. (2.3) with r^2 = r2, gray level muX */
} orc_op;

static double dotv(long n, const double *a, const double *b)
{
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* g = A x - y and f(x).  Least squares (Eq. (2.1), (2.2)): A = R^T R,
 * y = R^T b, f = ||R x - b||^2.  Bayesian (Eq. (2.3); half its gradient):
 * A = r^2 R^T R + I, y = r^2 R^T b + mu_X, f = r^2 ||R x - b||^2 + ||x - mu_X||^2. */
static double grad_ls(const orc_op *op, const double *x, const double *b,
                      double *r, double *g)
{
    orc_spmv(op->m, op->rp, op->ci, op->va, x, r);
    double f = 0.0;
    for (long i = 0; i < op->m; ++i) { r[i] -= b[i]; f += r[i] * r[i]; }
    orc_spmv(op->n, op->rpt, op->cit, op->vat, r, g);
    if (op->r2 > 0.0) {
        double fx = 0.0;
        for (long j = 0; j < op->n; ++j) {
            const double dx = x[j] - op->muX;
            g[j] = op->r2 * g[j] + dx;
            fx += dx * dx;
        }
        f = op->r2 * f + fx;
    }
    return f;
}

/* h = A p: R^T R p, or r^2 R^T R p + p for the Bayesian criterion. */
static void apply_A(const orc_op *op, const double *p, double *q, double *h)
{
    orc_spmv(op->m, op->rp, op->ci, op->va, p, q);
    orc_spmv(op->n, op->rpt, op->cit, op->vat, q, h);
    if (op->r2 > 0.0)
        for (long j = 0; j < op->n; ++j) h[j] = op->r2 * h[j] + p[j];
}

/*
 * SupPCG(x0, a, gamma, K, eps), Algorithm 3, with M = F^-1 diag(D) F.
 *   perturb = 0 skips step 11 (s_k = 0): plain PCG.
 *   max_iter bounds the number of executions of the while body (steps
 *   11-14); eps < 0 makes the while condition always true, so exactly
 *   max_iter bodies run (fixed-budget mode).
 * Outputs: x_half = x_{k-1/2} (the returned image), x_last = x_k, iters =
 * number of while-body executions, k_out = the returned k, ell_out = l_k.
 * Logs (nullable, max_iter entries, entry k-1 for body k):
 *   f(x_{k+1/2}), TV(x_k), TV(x_{k+1/2}), l_{k+1}, alpha, beta, ||s_k||.
 * init_log (nullable, 3 entries): f(x_0), alpha of step 6, ||p_0||.
 * r2 > 0 selects the Bayesian criterion of Eq. (2.3) (r^2 = r2, gray level muX)
 * in place of least squares: A, y and f as in grad_ls.
 */
int orc_suppcg(long m, long n,
               const long *rp, const int *ci, const double *va,
               const long *rpt, const int *cit, const double *vat,
               int ny, int nx, const double *b, const double *x0, const double *D,
               double a, double gamma, int K, double eps, int max_iter,
               long max_trials, int perturb,
               double *x_half, double *x_last, int *iters, int *k_out, long *ell_out,
               double *log_f, double *log_tv_k, double *log_tv_half, long *log_ell,
               double *log_alpha, double *log_beta, double *log_snorm, double *init_log,
               double r2, double muX)
{
    if ((long)ny * nx != n) return ORC_ERR_ARG;
    orc_op op = {m, n, rp, ci, va, rpt, cit, vat, r2, muX};
    size_t nb = sizeof(double) * (size_t)n, mb = sizeof(double) * (size_t)m;
    double *x = malloc(nb), *g = malloc(nb), *z = malloc(nb), *p = malloc(nb);
    double *h = malloc(nb), *s = malloc(nb), *r = malloc(mb), *q = malloc(mb);
    if (!x || !g || !z || !p || !h || !s || !r || !q) return ORC_ERR_NOMEM;
    int rc = ORC_OK;

    /* steps 1-7 */
    memcpy(x_half, x0, nb);                                  /* x_{1/2} = x_0        */
    double f_half = grad_ls(&op, x0, b, r, g);               /* g_0 = A x_0 - y      */
    orc_fourier_diag(ny, nx, D, g, z);                       /* z_0 = M g_0          */
    for (long i = 0; i < n; ++i) p[i] = -z[i];               /* p_0 = -z_0           */
    apply_A(&op, p, q, h);                                   /* h_0 = A p_0          */
    double pth = dotv(n, p, h);
    if (!(pth > 0.0)) { rc = ORC_ERR_BREAKDOWN; goto out; }
    double alpha = -dotv(n, g, p) / pth;                     /* step 6               */
    for (long i = 0; i < n; ++i) x[i] = x0[i] + alpha * p[i]; /* x_1                 */
    if (init_log) { init_log[0] = f_half; init_log[1] = alpha; init_log[2] = sqrt(dotv(n, p, p)); }
    int k = 1;                                               /* step 8               */
    long ell = 0;                                            /* step 9: l_1 = 0      */
    int body = 0;

    while (f_half > eps && body < max_iter) {                /* step 10              */
        double tv_k = log_tv_k ? orc_tv(ny, nx, x) : 0.0;
        if (perturb) {                                       /* step 11              */
            int st = orc_stv(ny, nx, x, ell, a, gamma, K, max_trials, s, &ell, NULL);
            if (st != ORC_OK) { rc = st; break; }
        } else {
            memset(s, 0, nb);
        }
        for (long i = 0; i < n; ++i) x_half[i] = x[i] + s[i]; /* step 12              */
        /* step 13: U_PCG(x_{k+1/2}, p_{k-1}, h_{k-1}), Algorithm 2 */
        f_half = grad_ls(&op, x_half, b, r, g);              /* 1: g = A x - y       */
        orc_fourier_diag(ny, nx, D, g, z);                   /* 2: z = M g           */
        double beta = dotv(n, z, h) / pth;                   /* 3                    */
        for (long i = 0; i < n; ++i) p[i] = -z[i] + beta * p[i]; /* 4                */
        apply_A(&op, p, q, h);                               /* 5: h = A p           */
        pth = dotv(n, p, h);
        if (!(pth > 0.0)) { rc = ORC_ERR_BREAKDOWN; break; }
        alpha = -dotv(n, g, p) / pth;                        /* 6                    */
        for (long i = 0; i < n; ++i) x[i] = x_half[i] + alpha * p[i]; /* 7           */
        if (log_f) log_f[body] = f_half;
        if (log_tv_k) log_tv_k[body] = tv_k;
        if (log_tv_half) log_tv_half[body] = orc_tv(ny, nx, x_half);
        if (log_ell) log_ell[body] = ell;
        if (log_alpha) log_alpha[body] = alpha;
        if (log_beta) log_beta[body] = beta;
        if (log_snorm) log_snorm[body] = sqrt(dotv(n, s, s));
        ++k;                                                 /* step 14              */
        ++body;
    }
    if (x_last) memcpy(x_last, x, nb);
    *iters = body;
    *k_out = k;
    *ell_out = ell;
out:
    free(x); free(g); free(z); free(p); free(h); free(s); free(r); free(q);
    return rc;
}

/* ------------------------------------------------------------------ */
/* ART for the Bayesian criterion (Sec. 3.4, Eq. (2.3))                  */
/* ------------------------------------------------------------------ */

/* The row-action method of Herman, Hurwitz and Lent named in Sec. 3.4 (a
 * Kaczmarz sweep over the consistent system r R y + u = r (b - R mu_X) in the
 * unknowns y = x - mu_X and one auxiliary value u_i per ray, whose
 * minimum-norm solution minimises r^2 ||R x - b||^2 + ||x - mu_X||^2, the
 * criterion of Eq. (2.3)).  Starting from x = mu_X, u = 0, ray i updates
 *     c   = lambda (r (b_i - <R_i, x>) - u_i) / (1 + r^2 ||R_i||^2),
 *     x  <- x + r c R_i,      u_i <- u_i + c,
 * with lambda the relaxation.  This function applies the updates for the rays
 * order[0 .. count-1] in that order (rows of the CSR R, ids v U + u). */
void orc_art_rays(const long *rp, const int *ci, const double *va, const long *order, long count,
                  const double *b, double r, double lam, double *x, double *uaux)
{
    for (long t = 0; t < count; ++t) {
        const long i = order[t];
        double dot = 0.0, nn = 0.0;
        for (long k = rp[i]; k < rp[i + 1]; ++k) {
            dot += va[k] * x[ci[k]];
            nn += va[k] * va[k];
        }
        const double c = lam * (r * (b[i] - dot) - uaux[i]) / (1.0 + r * r * nn);
        for (long k = rp[i]; k < rp[i + 1]; ++k) x[ci[k]] += r * c * va[k];
        uaux[i] += c;
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Learned perturbation: 3x3 convolution layers (test reference)        */
/* ------------------------------------------------------------------ */
/* The paper has no learned part; this is the plain definition of the
 * layers the GPU network uses, for parity and gradient checks:
 *   y[co][i][j] = bias[co] + sum_{ci, dy, dx} W[co][ci][dy][dx] x[ci][i+dy-1][j+dx-1]
 * (zero outside the image), optionally followed by max(0, .). */
void orc_conv3x3(int ny, int nx, int cin, int cout, const double *x, const double *W, const double *bias,
                 int relu, double *y)
{
    long n = (long)ny * nx;
#pragma omp parallel for schedule(static)
    for (int co = 0; co < cout; ++co)
        for (int i = 0; i < ny; ++i)
            for (int j = 0; j < nx; ++j) {
                double s = bias ? bias[co] : 0.0;
                for (int ci = 0; ci < cin; ++ci)
                    for (int dy = 0; dy < 3; ++dy)
                        for (int dx = 0; dx < 3; ++dx) {
                            int ii = i + dy - 1, jj = j + dx - 1;
                            if (ii < 0 || ii >= ny || jj < 0 || jj >= nx) continue;
                            s += W[((co * cin + ci) * 3 + dy) * 3 + dx] * x[ci * n + (long)ii * nx + jj];
                        }
                y[co * n + (long)i * nx + j] = (relu && s < 0.0) ? 0.0 : s;
            }
}

/* Gradients of a layer without activation: given dL/dy, write dL/dx (nullable),
 * dL/dW and dL/dbias (nullable) by the definition of the layer above. */
void orc_conv3x3_backward(int ny, int nx, int cin, int cout, const double *x, const double *W, const double *dy_,
                          double *dx_, double *dW, double *db)
{
    long n = (long)ny * nx;
    if (dx_) {
        for (long e = 0; e < (long)cin * n; ++e) dx_[e] = 0.0;
        for (int co = 0; co < cout; ++co)
            for (int i = 0; i < ny; ++i)
                for (int j = 0; j < nx; ++j) {
                    double g = dy_[co * n + (long)i * nx + j];
                    for (int ci = 0; ci < cin; ++ci)
                        for (int dy = 0; dy < 3; ++dy)
                            for (int dx = 0; dx < 3; ++dx) {
                                int ii = i + dy - 1, jj = j + dx - 1;
                                if (ii < 0 || ii >= ny || jj < 0 || jj >= nx) continue;
                                dx_[ci * n + (long)ii * nx + jj] += W[((co * cin + ci) * 3 + dy) * 3 + dx] * g;
                            }
                }
    }
    for (int co = 0; co < cout; ++co) {
        if (db) {
            double s = 0.0;
            for (long p = 0; p < n; ++p) s += dy_[co * n + p];
            db[co] = s;
        }
        for (int ci = 0; ci < cin; ++ci)
            for (int dy = 0; dy < 3; ++dy)
                for (int dx = 0; dx < 3; ++dx) {
                    double s = 0.0;
                    for (int i = 0; i < ny; ++i)
                        for (int j = 0; j < nx; ++j) {
                            int ii = i + dy - 1, jj = j + dx - 1;
                            if (ii < 0 || ii >= ny || jj < 0 || jj >= nx) continue;
                            s += dy_[co * n + (long)i * nx + j] * x[ci * n + (long)ii * nx + jj];
                        }
                    dW[((co * cin + ci) * 3 + dy) * 3 + dx] = s;
                }
    }
}
