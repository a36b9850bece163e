// C ABI of libsupcg: geometry objects, workspaces (batched problem
// descriptors and scratch), and the host-side schedule of SupPCG
// (Algorithm 3) as a fixed sequence of device launches per iteration,
// optionally replayed as one CUDA graph.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "internal.cuh"

using namespace supcg;

namespace supcg {

int cuda_fail(cudaError_t e, const char *what, const char *file, int line)
{
    if (getenv("SUPCG_DEBUG")) fprintf(stderr, "supcg: %s failed at %s:%d: %s\n", what, file, line, cudaGetErrorString(e));
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? SUPCG_ERR_NOMEM : SUPCG_ERR_CUDA;
}

static int round_up(int v, int m) { return (v + m - 1) / m * m; }

// ------------------------------------------------------------------ TMA map encoding
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// Tiled map of `rank` dimensions (innermost first), no swizzle, zero fill outside the tensor.
int encode_tiled(CUtensorMap *m, CUtensorMapDataType type, int rank, void *base, const cuuint64_t *dims,
                 const cuuint64_t *strides_bytes, const cuuint32_t *box)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn || rank < 1 || rank > 5) return SUPCG_ERR_CUDA;
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    CUresult r = fn(m, type, (cuuint32_t)rank, base, dims, strides_bytes, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? SUPCG_OK : SUPCG_ERR_CUDA;
}

// 2-D FP32 map over [outer][pitch] with logical extent inner x outer, box BW x rows.
static int encode_map(CUtensorMap *m, float *base, int inner, int outer, int pitch, int BW, int rows)
{
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch * 4};
    const cuuint32_t box[2] = {(cuuint32_t)BW, (cuuint32_t)rows};
    return encode_tiled(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box);
}

// ------------------------------------------------------------------ FFT plan
static int fft_factor(int n, int *rad)
{
    int k = 0;
    while (n % 4 == 0 && k < kMaxStages) { rad[k++] = 4; n /= 4; }
    while (n % 2 == 0 && k < kMaxStages) { rad[k++] = 2; n /= 2; }
    for (int p = 3; n > 1 && k < kMaxStages; p += 2)
        while (n % p == 0 && k < kMaxStages) { rad[k++] = p; n /= p; }
    return n == 1 ? k : -1;
}

} // namespace supcg

// ------------------------------------------------------------------ objects
enum { KT_FWD, KT_FWDA, KT_BWD, KT_BWD2, KT_VEC, KT_TR, KT_ROWS, KT_COLS, KT_SINO, KT_STV, KT_TV, KT_COUNT };

struct Workspace {
    int count = 0;
    std::vector<supcg_geometry> geoms;
    std::vector<unsigned> versions;   // the geometries' layout versions when this was built
    std::vector<Prob> hp;
    Prob *dp = nullptr;
    int *dprefix = nullptr;     // KT_COUNT x (count + 1)
    int blocks[KT_COUNT] = {};
    int smem_rows = 0, smem_cols = 0;
    int bwin = 0;
    int bw_max = 0;
    int bparts = 0;             // view parts of every problem's backprojector, 0 if they differ
    int mirror = 0;             // 1: some problem has mirror pairs of views
    std::vector<void *> allocs;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t body_exec = nullptr;
    double key[6] = {};         // parameters the captured body depends on
    int key_i[4] = {};
    int *trials_dev = nullptr;
    int trials_cap = 0;
    long long body_nodes = 0;
    float *lstage = nullptr;    // batched learned solve: the network's input batch (x, then tbar)
    size_t lstage_elems = 0;
    int *hdone = nullptr;       // eps mode: pinned copies of the problems' done flags

    Launch L(int kt, cudaStream_t st) const
    {
        Launch l;
        l.probs = dp;
        l.count = count;
        l.prefix = dprefix + kt * (count + 1);
        l.blocks = blocks[kt];
        l.bw_max = bw_max;
        l.bparts = bparts;
        l.mirror = mirror;
        l.st = st;
        return l;
    }
    ~Workspace()
    {
        if (body_exec) cudaGraphExecDestroy(body_exec);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        for (void *p : allocs) cudaFree(p);
        if (dp) cudaFree(dp);
        if (dprefix) cudaFree(dprefix);
        if (trials_dev) cudaFree(trials_dev);
        if (lstage) cudaFree(lstage);
        if (hdone) cudaFreeHost(hdone);
    }
};

struct supcg_geometry_s {
    int nx, ny, V, U, storage;
    double d, ds, off;
    std::vector<double> theta;
    std::vector<ViewP> views;
    std::vector<int> vlist;
    int nA, nB;
    int BU, BW, ntu;
    int nfw = 0;                    // forward warp items (see upload_block_order)
    int nfw_all = 0;                // the same when every view has its own items
    int nxp, nyp, Up;
    float cx, cy, uc, uc_hi, uc_lo;
    int bwin;
    FFTPlan fx, fy;
    ViewP *dviews = nullptr;
    int *dvlist = nullptr;
    // mirror pairs of views: views v and w = mirror[v] with cos_w = -cos_v and sin_w = sin_v
    // (theta and pi - theta).  Ray u of w meets pixel (i, nx-1-j) with the weight ray u of v
    // gives pixel (i, j), so the forward projector evaluates the weights once for both.
    // mirror[v] = w for the pair's first view (cos > 0), -2 for its second, -1 unpaired.
    std::vector<int> mirror;
    int *dmirror = nullptr;         // device copy: the partner of a pair's first view, else -1
    int npairs = 0;
    int *dborder = nullptr;         // forward warp items in launch order, at most V x ceil(U / 32)
    int *dborder_all = nullptr;     // the same with every view's items (no mirror pairing)
    float *host_db = nullptr, *host_dx = nullptr;   // supcg_solve_host's device copies of b and x (first use)
    double *art_u = nullptr, *art_rn = nullptr;     // ART's per-ray values (first use)
    int art_S = 1;                                  // ART: bin spacing of rays with disjoint pixels
    float4 *dtwx = nullptr, *dtwy = nullptr;   // double-float twiddles
    Workspace *ws_ops = nullptr;    // standalone operators, `ops_batch` images
    int ops_batch = 0;
    Workspace *ws_solve = nullptr;  // single-problem solve
    Workspace *ws_batch = nullptr;  // batched solve owned by this (first) geometry
    std::vector<supcg_geometry> batch_key;
    int bparts = kBwdViewParts;     // backprojector: view parts per pixel tile
    unsigned layout_version = 0;    // changed with the tiling: workspaces built before are stale
};

// Forward projector box width: the inner indices that one warp's 64 rays can
// touch over one chunk of rows, plus slack, rounded up to a multiple of 4 floats.
static int fwd_box_width(const supcg_geometry_s *g)
{
    double span = 0.0;
    for (const ViewP &vp : g->views)
        span = std::max(span, fabs((double)vp.a_tau) * 63.0 + fabs((double)vp.b_o) * (kRowsPerChunk - 1));
    // a multiple of 4 floats (16-byte rows), so that every staged box (kRowsPerChunk rows of
    // BW floats) starts 128-byte aligned
    static_assert((4 * kRowsPerChunk * 4) % 128 == 0, "boxes of 4k floats per row start 128-byte aligned");
    return round_up((int)ceil(span + 11.0), 4);
}

// Forward warp items in launch order, longest first.  An item is one warp's rays: the
// first 64 bins of a (view, bin tile) or the rest of the tile.  It lasts about as long
// as the rows that the union of its rays can meet (the row ranges of the kernel's
// fwd_row_range, here in FP64), weighted by the cost of a row in its view.  Block b runs items 2b and 2b + 1 of the list, so a
// block pairs items of about the same length (its warps finish together) and the
// grid starts the long blocks first and ends on short ones; with one block per
// (view, tile) a block lasted as long as its slower warp and a view's long central
// tiles could start last.  Entry: (vidx * ntu + tile) * 2 + half, vidx indexing the
// class-A-then-class-B view list.  PAIRED: the second view of a mirror pair has no
// items (its rays are summed by its first view's items); else every view has its own.
static std::vector<int> block_order(const supcg_geometry_s *g, bool pair)
{
    const int nv = g->V, ntu = g->ntu;
    const double uc = 0.5 * (g->U - 1) - g->off / g->ds;
    std::vector<int> ord;
    std::vector<double> cost;
    ord.reserve((size_t)nv * ntu * 2);
    for (int vi = 0; vi < nv; ++vi) {
        const int v = g->vlist[vi];
        if (pair && g->mirror[v] == -2) continue;   // the second view of a pair: projected with the first
        const bool paired = pair && g->mirror[v] >= 0;
        const ViewP &vp = g->views[v];
        const bool classB = vi >= g->nA;
        const int n_outer = classB ? g->nx : g->ny, n_inner = classB ? g->ny : g->nx;
        const double L = -(double)vp.hwq - 1.0, H = (double)n_inner + vp.hwq;
        for (int t = 0; t < ntu; ++t) {
            const int u_end = std::min(g->U, (t + 1) * g->BU);
            for (int half = 0; half < 2; ++half) {
                const int w0 = t * g->BU + 64 * half;
                if (w0 >= u_end) continue;
                int lo = n_outer, hi = -1;
                for (int u = w0; u < std::min(u_end, w0 + 64); ++u) {
                    const double base = (double)vp.a_tau * ((double)u - uc) + vp.g0;
                    int l, h;
                    if (fabs((double)vp.b_o) < 1e-20) {
                        const bool in = base >= L && base <= H;
                        l = in ? 0 : n_outer;
                        h = in ? n_outer - 1 : -1;
                    } else {
                        const double ra = (L - base) / vp.b_o, rb = (H - base) / vp.b_o;
                        l = std::max(0, (int)floor(std::min(ra, rb) - 1.0));
                        h = std::min(n_outer - 1, (int)ceil(std::max(ra, rb) + 1.0));
                    }
                    lo = std::min(lo, l);
                    hi = std::max(hi, h);
                }
                // per row: two candidates; three candidates near the diagonal cost half as much
                // again; axis-aligned views, whose rays cross every row, are weighted to start
                // first (the order measured fastest)
                const double per_row = ((vp.flags & kViewAxis) ? 2.0 : ((vp.flags & kViewFwd3) ? 1.5 : 1.0)) *
                                       (paired ? 1.3 : 1.0);   // a pair: one more load and sum per candidate
                ord.push_back((vi * ntu + t) * 2 + half);
                cost.push_back(16.0 + per_row * (double)std::max(0, hi - lo + 1));
            }
        }
    }
    std::vector<int> idx(ord.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<int> sorted(ord.size());
    for (size_t i = 0; i < idx.size(); ++i) sorted[i] = ord[idx[i]];
    return sorted;
}

// The forward projector's two item lists: with mirror pairs (the paired kernel) and
// with every view (the unpaired kernel, for launches in which no problem has mirror pairs).
static int upload_block_order(supcg_geometry_s *g)
{
    const std::vector<int> all = block_order(g, false);
    g->nfw_all = (int)all.size();
    SUPCG_CUDA_TRY(cudaMemcpy(g->dborder_all, all.data(), sizeof(int) * all.size(), cudaMemcpyHostToDevice));
    if (g->npairs == 0) {
        g->nfw = g->nfw_all;
        SUPCG_CUDA_TRY(cudaMemcpy(g->dborder, all.data(), sizeof(int) * all.size(), cudaMemcpyHostToDevice));
        return SUPCG_OK;
    }
    const std::vector<int> paired = block_order(g, true);
    g->nfw = (int)paired.size();
    SUPCG_CUDA_TRY(cudaMemcpy(g->dborder, paired.data(), sizeof(int) * paired.size(), cudaMemcpyHostToDevice));
    return SUPCG_OK;
}

static void free_ws(Workspace *&w)
{
    delete w;
    w = nullptr;
}

// ------------------------------------------------------------------ geometry
static void exact_cos_sin(double th, double *c, double *s)
{
    const double q = th / (0.5 * M_PI);
    const double r = nearbyint(q);
    if (fabs(q - r) < 1e-12) {
        const long k = (((long)r) % 4 + 4) % 4;
        const double cc[4] = {1.0, 0.0, -1.0, 0.0}, ss[4] = {0.0, 1.0, 0.0, -1.0};
        *c = cc[k];
        *s = ss[k];
    } else {
        *c = cos(th);
        *s = sin(th);
    }
}

// exp(-2 pi i k / n), k < n, as double-float pairs (cos h, cos l, sin h, sin l) of the FP64 values
static int upload_twiddles(int n, float4 **out)
{
    std::vector<float4> tw(n);
    for (int k = 0; k < n; ++k) {
        const double a = -2.0 * M_PI * (double)k / (double)n;
        const double c = cos(a), s = sin(a);
        const float ch = (float)c, sh = (float)s;
        tw[k] = make_float4(ch, (float)(c - (double)ch), sh, (float)(s - (double)sh));
    }
    SUPCG_CUDA_TRY(cudaMalloc(out, sizeof(float4) * n));
    SUPCG_CUDA_TRY(cudaMemcpy(*out, tw.data(), sizeof(float4) * n, cudaMemcpyHostToDevice));
    return SUPCG_OK;
}

extern "C" int supcg_create_geometry(int nx, int ny, double pixel_size, int n_views, const double *angles, int n_bins,
                                     double bin_spacing, double det_center_offset, int storage, supcg_geometry *out)
{
    if (!out) return SUPCG_ERR_ARG;
    *out = nullptr;
    if (nx < 1 || ny < 1 || nx > 16384 || ny > 16384 || n_views < 1 || n_bins < 1 || n_bins > (1 << 21) ||
        n_views > (1 << 20) || !(pixel_size > 0.0) || !isfinite(pixel_size) || !isfinite(det_center_offset) ||
        (storage != SUPCG_F32 && storage != SUPCG_BF16))
        return SUPCG_ERR_ARG;
    auto *g = new (std::nothrow) supcg_geometry_s();
    if (!g) return SUPCG_ERR_NOMEM;
    g->nx = nx; g->ny = ny; g->V = n_views; g->U = n_bins; g->storage = storage;
    g->d = pixel_size;
    g->ds = (bin_spacing > 0.0) ? bin_spacing : pixel_size;
    g->off = det_center_offset;
    g->theta.resize(n_views);
    for (int v = 0; v < n_views; ++v) {
        g->theta[v] = angles ? angles[v] : (double)v * M_PI / (double)n_views;
        if (!isfinite(g->theta[v])) { delete g; return SUPCG_ERR_ARG; }
    }
    // cos and sin of every view (exact on the axes), then the mirror pairs: a view with cos > 0
    // and one with cos < 0 whose cos and sin agree up to sign within 1e-12 (for V angles
    // v pi / V, v and V - v).  The second view's cos is set to exactly minus the first's, so
    // that both views' per-view constants are exact negatives (the geometry moves by ~1e-16).
    std::vector<double> vcos(n_views), vsin(n_views);
    for (int v = 0; v < n_views; ++v) exact_cos_sin(g->theta[v], &vcos[v], &vsin[v]);
    g->mirror.assign(n_views, -1);
    {
        std::vector<int> neg;
        for (int v = 0; v < n_views; ++v)
            if (vcos[v] < 0.0 && vsin[v] != 0.0) neg.push_back(v);
        std::sort(neg.begin(), neg.end(), [&](int x, int y) { return vsin[x] < vsin[y]; });
        for (int v = 0; v < n_views; ++v) {
            if (!(vcos[v] > 0.0) || vsin[v] == 0.0) continue;
            auto it = std::lower_bound(neg.begin(), neg.end(), vsin[v] - 1e-12,
                                       [&](int w, double val) { return vsin[w] < val; });
            for (; it != neg.end() && vsin[*it] <= vsin[v] + 1e-12; ++it) {
                const int w = *it;
                if (g->mirror[w] == -1 && fabs(vcos[w] + vcos[v]) <= 1e-12) {
                    g->mirror[v] = w;
                    g->mirror[w] = -2;
                    vcos[w] = -vcos[v];
                    vsin[w] = vsin[v];
                    ++g->npairs;
                    break;
                }
            }
        }
    }
    const double r = g->d / g->ds;
    const double cx = 0.5 * (nx - 1), cy = 0.5 * (ny - 1);
    const double uc = 0.5 * (n_bins - 1) - g->off / g->ds;
    g->cx = (float)cx; g->cy = (float)cy;
    g->uc = (float)uc;
    // exact split: every partial sum of u - uc_hi - cu_hi X - su_hi Y stays a
    // multiple of 2^-Q below 2^(24-Q) in magnitude
    const double mbound = (double)n_bins + 256.0 + fabs(uc) + r * (cx + cy + 4.0) + 8.0;
    const int Q = (int)floor(24.0 - log2(mbound)) - 1;
    if (Q < 4) { delete g; return SUPCG_ERR_UNSUPPORTED; }
    auto split = [](double v, int q, float *hi, float *lo) {
        const double h = ldexp(nearbyint(ldexp(v, q)), -q);
        *hi = (float)h;
        *lo = (float)(v - h);
    };
    split(uc, Q, &g->uc_hi, &g->uc_lo);
    g->views.resize(n_views);
    std::vector<int> A, B;
    double maxE = 0.0, span_bwd = 0.0, max_small = fabs((double)g->uc_lo);
    double mcl = 0.0, msl = 0.0;
    for (int v = 0; v < n_views; ++v) {
        const double c = vcos[v], s = vsin[v];
        const double ac = fabs(c), as = fabs(s);
        const double a = std::max(ac, as), b = std::min(ac, as);
        ViewP vp = {};
        const double cu = c * r, su = s * r;
        vp.cu = (float)cu;
        vp.su = (float)su;
        split(cu, Q - 1, &vp.cu_hi, &vp.cu_lo);
        split(su, Q - 1, &vp.su_hi, &vp.su_lo);
        mcl = std::max(mcl, fabs((double)vp.cu_lo));
        msl = std::max(msl, fabs((double)vp.su_lo));
        vp.E = (float)(r * (a + b) / 2.0);
        const double Sd = (b > 0.0) ? g->ds / (a * b) : 0.0, Pd = g->d / a;
        vp.Sn = (float)(Sd / Pd);
        vp.P = (float)Pd;
        const bool classB = as > ac;
        if (!classB) {
            vp.a_tau = (float)(1.0 / cu);
            vp.b_o = (float)(su / cu);
            vp.g0 = (float)(cx - (su / cu) * cy);
            A.push_back(v);
        } else {
            vp.a_tau = (float)(-1.0 / su);
            vp.b_o = (float)(cu / su);
            vp.g0 = (float)(cy - (cu / su) * cx);
            B.push_back(v);
        }
        vp.ESn = (float)(r * (a + b) / 2.0 * Sd / Pd);
        // candidate windows: a ray's footprint on a row (column) is (a+b)/(2a) pixels
        // either side of its centre, a pixel's footprint E bins either side of its
        // projected centre; 0.02 covers the rounding of the centres
        const double margin = 0.02;
        vp.hwq = (float)((a + b) / (2.0 * a) + margin);
        vp.hwu = (float)(r * (a + b) / 2.0 + margin);
        vp.flags = (b == 0.0 ? kViewAxis : 0) | (classB ? kViewClassB : 0) |
                   (2.0 * vp.hwq >= 2.0 ? kViewFwd3 : 0) | (2.0 * vp.hwu >= 2.0 ? kViewBwd3 : 0);
        g->views[v] = vp;
        maxE = std::max(maxE, (double)vp.E);
        span_bwd = std::max(span_bwd, (kBwdTileJ - 1) * fabs((double)vp.cu) + (kBwdTileI - 1) * fabs((double)vp.su));
    }
    max_small += mcl * (cx + 1.0) + msl * (cy + 1.0);
    // the three bins nearest a pixel's centre must cover its footprint, and a
    // backprojector tile's bins must fit its shared-memory window
    g->bwin = std::max(64, round_up((int)ceil(span_bwd + 11.0), 4));
    // (the centres include the small correction, so only the margin pads the windows)
    (void)max_small;
    if (maxE + 0.03 >= 1.5 || g->bwin > 256) { delete g; return SUPCG_ERR_UNSUPPORTED; }
    // ART's class spacing: two rays of a view S bins apart share no pixel when S > 2 E for every
    // view's footprint half-width E = (d/ds)(|cos| + |sin|)/2 (FP64, exact cos/sin on the axes)
    {
        double e2 = 0.0;
        for (int v = 0; v < n_views; ++v) {
            double c, s2;
            exact_cos_sin(g->theta[v], &c, &s2);
            e2 = std::max(e2, r * (fabs(c) + fabs(s2)));
        }
        g->art_S = (int)floor(e2) + 1;
    }
    g->nA = (int)A.size();
    g->nB = (int)B.size();
    g->vlist = A;
    g->vlist.insert(g->vlist.end(), B.begin(), B.end());
    // forward tiling: the widest box any view needs must fit 256 columns
    g->BU = 0;
    for (int bu : {128, 96, 64, 32}) {
        const int bw = fwd_box_width(g);
        if (bw <= 256) { g->BU = bu; g->BW = bw; break; }
    }
    if (!g->BU) { delete g; return SUPCG_ERR_UNSUPPORTED; }
    g->ntu = (n_bins + g->BU - 1) / g->BU;
    g->nxp = round_up(nx, 4);
    g->nyp = round_up(ny, 4);
    g->Up = round_up(n_bins, 4);
    // FFT plans
    g->fx.n = nx;
    g->fy.n = ny;
    g->fx.nst = fft_factor(nx, g->fx.radix);
    g->fy.nst = fft_factor(ny, g->fy.radix);
    if (g->fx.nst < 0 || g->fy.nst < 0) { delete g; return SUPCG_ERR_UNSUPPORTED; }
    int rc;
    if ((rc = upload_twiddles(nx, &g->dtwx)) || (rc = upload_twiddles(ny, &g->dtwy))) {
        supcg_destroy_geometry(g);
        return rc;
    }
    g->fx.tw = nullptr;
    g->fy.tw = nullptr;
    g->fx.twf = g->dtwx;
    g->fy.twf = g->dtwy;
    std::vector<int> dm(n_views);
    for (int v = 0; v < n_views; ++v) dm[v] = g->mirror[v] >= 0 ? g->mirror[v] : -1;
    if (cudaMalloc(&g->dviews, sizeof(ViewP) * n_views) != cudaSuccess ||
        cudaMalloc(&g->dmirror, sizeof(int) * n_views) != cudaSuccess ||
        cudaMalloc(&g->dvlist, sizeof(int) * n_views) != cudaSuccess ||
        cudaMalloc(&g->dborder, sizeof(int) * (size_t)n_views * ((n_bins + 31) / 32)) != cudaSuccess ||
        cudaMalloc(&g->dborder_all, sizeof(int) * (size_t)n_views * ((n_bins + 31) / 32)) != cudaSuccess) {
        supcg_destroy_geometry(g);
        return SUPCG_ERR_NOMEM;
    }
    if (cudaMemcpy(g->dviews, g->views.data(), sizeof(ViewP) * n_views, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g->dmirror, dm.data(), sizeof(int) * n_views, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g->dvlist, g->vlist.data(), sizeof(int) * n_views, cudaMemcpyHostToDevice) != cudaSuccess) {
        supcg_destroy_geometry(g);
        return SUPCG_ERR_CUDA;
    }
    if ((rc = upload_block_order(g))) {
        supcg_destroy_geometry(g);
        return rc;
    }
    *out = g;
    return SUPCG_OK;
}

extern "C" int supcg_set_tiling(supcg_geometry g, int fwd_bins_per_block)
{
    if (!g || fwd_bins_per_block < 32 || fwd_bins_per_block > 128 || fwd_bins_per_block % 32) return SUPCG_ERR_ARG;
    const int bw = fwd_box_width(g);
    if (bw > 256) return SUPCG_ERR_UNSUPPORTED;
    cudaDeviceSynchronize();
    g->BU = fwd_bins_per_block;
    g->BW = bw;
    g->ntu = (g->U + g->BU - 1) / g->BU;
    int rc = upload_block_order(g);
    if (rc) return rc;
    // workspaces hold launch shapes and TMA boxes of the old tiling (a batched workspace owned
    // by another geometry sees the version change)
    free_ws(g->ws_ops);
    free_ws(g->ws_solve);
    free_ws(g->ws_batch);
    g->ops_batch = 0;
    ++g->layout_version;
    return SUPCG_OK;
}

extern "C" int supcg_set_bwd_parts(supcg_geometry g, int parts)
{
    if (!g || parts < 1 || parts > kBwdMaxParts) return SUPCG_ERR_ARG;
    cudaDeviceSynchronize();
    g->bparts = parts;
    free_ws(g->ws_ops);
    free_ws(g->ws_solve);
    free_ws(g->ws_batch);
    g->ops_batch = 0;
    ++g->layout_version;
    return SUPCG_OK;
}

extern "C" int supcg_get_bwd_parts(supcg_geometry g, int *parts)
{
    if (!g || !parts) return SUPCG_ERR_ARG;
    *parts = g->bparts;
    return SUPCG_OK;
}

extern "C" int supcg_get_mirror_pairs(supcg_geometry g, int *pairs)
{
    if (!g || !pairs) return SUPCG_ERR_ARG;
    *pairs = g->npairs;
    return SUPCG_OK;
}

extern "C" int supcg_get_tiling(supcg_geometry g, int *fwd_bins_per_block)
{
    if (!g || !fwd_bins_per_block) return SUPCG_ERR_ARG;
    *fwd_bins_per_block = g->BU;
    return SUPCG_OK;
}

extern "C" int supcg_destroy_geometry(supcg_geometry g)
{
    if (!g) return SUPCG_ERR_ARG;
    cudaDeviceSynchronize();
    free_ws(g->ws_ops);
    free_ws(g->ws_solve);
    free_ws(g->ws_batch);
    if (g->dviews) cudaFree(g->dviews);
    if (g->dvlist) cudaFree(g->dvlist);
    if (g->dmirror) cudaFree(g->dmirror);
    if (g->dborder) cudaFree(g->dborder);
    if (g->dborder_all) cudaFree(g->dborder_all);
    if (g->host_db) cudaFree(g->host_db);
    if (g->host_dx) cudaFree(g->host_dx);
    if (g->art_u) cudaFree(g->art_u);
    if (g->art_rn) cudaFree(g->art_rn);
    if (g->dtwx) cudaFree(g->dtwx);
    if (g->dtwy) cudaFree(g->dtwy);
    delete g;
    return SUPCG_OK;
}

// ------------------------------------------------------------------ workspace
static int ws_create(const std::vector<supcg_geometry> &gs, Workspace **out)
{
    auto *w = new (std::nothrow) Workspace();
    if (!w) return SUPCG_ERR_NOMEM;
    w->count = (int)gs.size();
    w->geoms = gs;
    for (const supcg_geometry g : gs) w->versions.push_back(g->layout_version);
    w->hp.resize(w->count);
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int rc = stv_max_blocks_per_sm(&per_sm);
    if (rc) { delete w; return rc; }
    const int stv_cap = std::max(1, nsm * per_sm);
    if (w->count > stv_cap) { delete w; return SUPCG_ERR_UNSUPPORTED; }

    // blocks per problem for every kernel type
    std::vector<std::vector<int>> nb(KT_COUNT, std::vector<int>(w->count));
    long long stv_want = 0;
    std::vector<long long> npx(w->count);
    for (int c = 0; c < w->count; ++c) {
        const supcg_geometry g = gs[c];
        nb[KT_FWD][c] = (g->nfw + 1) / 2;
        nb[KT_FWDA][c] = (g->nfw_all + 1) / 2;
        nb[KT_BWD][c] = backward_blocks(g->nx, g->ny, 0, g->bparts);
        nb[KT_BWD2][c] = backward_blocks(g->nx, g->ny, 1, g->bparts);
        nb[KT_VEC][c] = (int)(((long long)g->ny * g->nxp + 1023) / 1024);
        nb[KT_TR][c] = ((g->ny + 31) / 32) * ((g->nx + 31) / 32);
        // FFT: enough blocks to fill the device, each a few row pairs / stored columns
        const int npairs = (g->ny + 1) / 2, hx = g->nx / 2 + 1;
        const int rpb = std::max(1, std::min(std::min(8, 2048 / g->nx), npairs / 256));
        const int cw = std::max(1, std::min(std::min(8, 2048 / g->ny), hx / 256));
        nb[KT_ROWS][c] = (npairs + rpb - 1) / rpb;
        nb[KT_COLS][c] = (hx + cw - 1) / cw;
        // (two transform buffers, then the twiddles when at most 2048 of them)
        w->smem_rows = std::max(w->smem_rows, 2 * rpb * g->nx * 16 + (g->nx <= kFftSmemTw ? g->nx * 16 : 0));
        w->smem_cols = std::max(w->smem_cols, 2 * cw * g->ny * 16 + (g->ny <= kFftSmemTw ? g->ny * 16 : 0));
        nb[KT_SINO][c] = (int)(((long long)g->V * g->Up + 1023) / 1024);
        npx[c] = (long long)g->nx * g->ny;
        nb[KT_STV][c] = (int)std::max(1LL, std::min<long long>((npx[c] + 1023) / 1024, stv_cap));
        stv_want += nb[KT_STV][c];
        nb[KT_TV][c] = (int)std::max(1LL, std::min<long long>((npx[c] + 1023) / 1024, 4096));
        w->hp[c].fft_rpb = rpb;
        w->hp[c].fft_cw = cw;
    }
    if (w->smem_rows > 200 * 1024 || w->smem_cols > 200 * 1024) { delete w; return SUPCG_ERR_UNSUPPORTED; }
    // co-residency of the cooperative S_TV launch: scale down to the device capacity
    // (proportional shares, at least one block each; the rounding-up of the minimum is
    // taken back from the largest shares)
    if (stv_want > stv_cap) {
        long long tot = 0;
        for (int c = 0; c < w->count; ++c) {
            nb[KT_STV][c] = (int)std::max(1LL, (long long)nb[KT_STV][c] * stv_cap / stv_want);
            tot += nb[KT_STV][c];
        }
        while (tot > stv_cap) {
            int big = 0;
            for (int c = 1; c < w->count; ++c)
                if (nb[KT_STV][c] > nb[KT_STV][big]) big = c;
            --nb[KT_STV][big];
            --tot;
        }
    }
    std::vector<int> hprefix(KT_COUNT * (w->count + 1));
    for (int kt = 0; kt < KT_COUNT; ++kt) {
        int acc = 0;
        for (int c = 0; c < w->count; ++c) {
            hprefix[kt * (w->count + 1) + c] = acc;
            acc += nb[kt][c];
        }
        hprefix[kt * (w->count + 1) + w->count] = acc;
        w->blocks[kt] = acc;
    }
    if (cudaMalloc(&w->dprefix, sizeof(int) * hprefix.size()) != cudaSuccess ||
        cudaMemcpy(w->dprefix, hprefix.data(), sizeof(int) * hprefix.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        delete w;
        return SUPCG_ERR_NOMEM;
    }

    // buffers: one allocation per problem, 256-byte aligned pieces
    for (int c = 0; c < w->count; ++c) {
        const supcg_geometry g = gs[c];
        Prob &P = w->hp[c];
        const size_t img = (size_t)g->ny * g->nxp, imgT = (size_t)g->nx * g->nyp, sino = (size_t)g->V * g->Up;
        const size_t mir = g->npairs > 0 ? 1 : 0;   // mirrored images only with mirror pairs
        int maxblk = 0;
        for (int kt = 0; kt < KT_COUNT; ++kt) maxblk = std::max(maxblk, nb[kt][c]);
        const size_t npart = std::max<size_t>(12 * (size_t)nb[KT_STV][c], 2 * (size_t)maxblk) + 64;
        auto al = [](size_t b) { return (b + 255) / 256 * 256; };
        const size_t sizes[] = {img * 4, imgT * 4, img * 4, imgT * 4, img * 4, img * 4, img * 4, img * 4,
                                sino * 4, sino * 4, sino * 4, (size_t)g->ny * g->nx * 16, sizeof(Scal),
                                npart * 8, 16 * 4, 4 * 4, (size_t)(g->ny / 2 + 1) * (g->nx / 2 + 1) * 8,
                                2 * (size_t)g->bparts * img * 8,
                                (size_t)std::max(nb[KT_BWD][c], nb[KT_BWD2][c]) * 4, img * 4, img * 4,
                                mir * img * 4, mir * imgT * 4, mir * img * 4, mir * imgT * 4,
                                img * 4, imgT * 4, mir * img * 4, mir * imgT * 4, sino * 8, sino * 8};
        constexpr int kPieces = sizeof(sizes) / sizeof(sizes[0]);
        size_t total = 0;
        for (size_t s : sizes) total += al(s);
        char *base = nullptr;
        if (cudaMalloc(&base, total) != cudaSuccess) { delete w; return SUPCG_ERR_NOMEM; }
        w->allocs.push_back(base);
        if (cudaMemset(base, 0, total) != cudaSuccess) { delete w; return SUPCG_ERR_CUDA; }
        char *ptrs[kPieces];
        size_t off = 0;
        for (int k = 0; k < kPieces; ++k) { ptrs[k] = base + off; off += al(sizes[k]); }
        P.x = (float *)ptrs[0]; P.xT = (float *)ptrs[1]; P.p = (float *)ptrs[2]; P.pT = (float *)ptrs[3];
        P.g = (float *)ptrs[4]; P.z = (float *)ptrs[5]; P.h = (float *)ptrs[6]; P.tbar = (float *)ptrs[7];
        P.r = (float *)ptrs[8]; P.q = (float *)ptrs[9]; P.bpad = (float *)ptrs[10];
        P.C = (double2 *)ptrs[11]; P.sc = (Scal *)ptrs[12]; P.partial = (double *)ptrs[13];
        P.counter = (unsigned *)ptrs[14]; P.bar = (unsigned *)ptrs[15]; P.Dtab = (float2 *)ptrs[16];
        P.bsplit = (float2 *)ptrs[17]; P.tilecnt = (unsigned *)ptrs[18]; P.xlo = (float *)ptrs[19];
        P.bparts = g->bparts;
        w->bparts = (c == 0 || w->bparts == g->bparts) ? g->bparts : 0;
        P.glo = (float *)ptrs[20];
        P.xm = mir ? (float *)ptrs[21] : nullptr;
        P.xmT = mir ? (float *)ptrs[22] : nullptr;
        P.pm = mir ? (float *)ptrs[23] : nullptr;
        P.pmT = mir ? (float *)ptrs[24] : nullptr;
        P.mirror = mir ? g->dmirror : nullptr;
        P.d = (float *)ptrs[25];
        P.dT = (float *)ptrs[26];
        P.dm = mir ? (float *)ptrs[27] : nullptr;
        P.dmT = mir ? (float *)ptrs[28] : nullptr;
        P.rd = (double *)ptrs[29];
        P.qd = (double *)ptrs[30];
        if (mir) w->mirror = 1;
        P.border = g->dborder;
        P.border_all = g->dborder_all;
        P.nfw_all = g->nfw_all;
        P.nx = g->nx; P.ny = g->ny; P.V = g->V; P.U = g->U;
        P.nxp = g->nxp; P.nyp = g->nyp; P.Up = g->Up;
        P.BU = g->BU; P.BW = g->BW; P.ntu = g->ntu; P.nfw = g->nfw; P.nA = g->nA; P.nB = g->nB;
        P.cx = g->cx; P.cy = g->cy; P.uc = g->uc; P.uc_hi = g->uc_hi; P.uc_lo = g->uc_lo;
        P.bwin = g->bwin;
        w->bwin = std::max(w->bwin, g->bwin);
        w->bw_max = std::max(w->bw_max, g->BW);
        P.views = g->dviews; P.vlist = g->dvlist;
        P.fx = g->fx; P.fy = g->fy;
        P.storage = g->storage;
        P.stv_blocks = nb[KT_STV][c];
        P.mu = 1e-5; P.rho = 0.8; P.precond = 1;
        P.r2 = 0.0;
        P.gray_scale = g->ds / ((double)g->V * g->nx * g->ny * g->d * g->d);
        int e = 0;
        // 2 w + c: image w (x, p, d) in layout c (rows, transposed); 6 + 2 w + c: its mirror
        float *imgs[3][2] = {{P.x, P.xT}, {P.p, P.pT}, {P.d, P.dT}};
        float *mimgs[3][2] = {{P.xm, P.xmT}, {P.pm, P.pmT}, {P.dm, P.dmT}};
        for (int wi = 0; wi < 3; ++wi) {
            e |= encode_map(&P.tm[2 * wi], imgs[wi][0], g->nx, g->ny, g->nxp, g->BW, kRowsPerChunk);
            e |= encode_map(&P.tm[2 * wi + 1], imgs[wi][1], g->ny, g->nx, g->nyp, g->BW, kRowsPerChunk);
            if (mir) {
                e |= encode_map(&P.tm[6 + 2 * wi], mimgs[wi][0], g->nx, g->ny, g->nxp, g->BW, kRowsPerChunk);
                e |= encode_map(&P.tm[7 + 2 * wi], mimgs[wi][1], g->ny, g->nx, g->nyp, g->BW, kRowsPerChunk);
            }
        }
        if (e) { delete w; return SUPCG_ERR_CUDA; }
    }
    if (cudaMalloc(&w->dp, sizeof(Prob) * w->count) != cudaSuccess) { delete w; return SUPCG_ERR_NOMEM; }
    if (cudaStreamCreateWithFlags(&w->cap_stream, cudaStreamNonBlocking) != cudaSuccess) { delete w; return SUPCG_ERR_CUDA; }
    *out = w;
    return SUPCG_OK;
}

int supcg::current_device(int *dev)
{
    SUPCG_CUDA_TRY(cudaGetDevice(dev));
    return (*dev >= 0 && *dev < kMaxDevices) ? SUPCG_OK : SUPCG_ERR_UNSUPPORTED;
}

int supcg::func_attrs_once(const void *func, int max_dyn_smem, int carveout)
{
    static std::mutex mu;
    static std::vector<std::pair<const void *, int>> done;   // (kernel, device) pairs already set
    int dev = 0;
    int rc = current_device(&dev);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(mu);
    for (const auto &d : done)
        if (d.first == func && d.second == dev) return SUPCG_OK;
    SUPCG_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn_smem));
    if (carveout >= 0) SUPCG_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout, carveout));
    done.emplace_back(func, dev);
    return SUPCG_OK;
}

// Bounded grid barriers: polls before giving up, and the test hook's extra blocks.
static std::atomic<long long> g_wait_limit{kSpinLimit};
static std::atomic<int> g_bar_extra{0};

// The batched workspace of `owner` serves `key` if it was built for these geometries
// at their current layout versions.
static bool batch_ws_current(supcg_geometry owner, const std::vector<supcg_geometry> &key)
{
    const Workspace *w = owner->ws_batch;
    if (!w || owner->batch_key != key) return false;
    for (size_t c = 0; c < key.size(); ++c)
        if (w->versions[c] != key[c]->layout_version) return false;
    return true;
}

static int ws_upload(Workspace *w, cudaStream_t st)
{
    for (Prob &P : w->hp) {
        P.wait_limit = g_wait_limit.load();
        P.bar_extra = g_bar_extra.load();
    }
    // synchronous copy from pageable memory: safe to modify hp afterwards
    SUPCG_CUDA_TRY(cudaStreamSynchronize(st));
    SUPCG_CUDA_TRY(cudaMemcpy(w->dp, w->hp.data(), sizeof(Prob) * w->count, cudaMemcpyHostToDevice));
    return SUPCG_OK;
}

static int ops_ws(supcg_geometry g, int batch, Workspace **out)
{
    if (!g->ws_ops || g->ops_batch != batch) {
        free_ws(g->ws_ops);
        std::vector<supcg_geometry> gs(batch, g);
        int rc = ws_create(gs, &g->ws_ops);
        if (rc) return rc;
        g->ops_batch = batch;
    }
    *out = g->ws_ops;
    return SUPCG_OK;
}

static size_t elem_size(int storage) { return storage == SUPCG_BF16 ? 2 : 4; }

// ------------------------------------------------------------------ operators
extern "C" int supcg_project(supcg_geometry g, const void *d_x, void *d_y, int batch, void *stream)
{
    if (!g || !d_x || !d_y || batch < 1) return SUPCG_ERR_ARG;
    Workspace *w;
    int rc = ops_ws(g, batch, &w);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t es = elem_size(g->storage);
    for (int b = 0; b < batch; ++b) {
        w->hp[b].in_user = (const char *)d_x + (size_t)b * g->nx * g->ny * es;
        w->hp[b].out_user = (char *)d_y + (size_t)b * g->V * g->U * es;
    }
    if ((rc = ws_upload(w, st))) return rc;
    if ((rc = launch_stage_in(w->L(KT_TR, st), 0))) return rc;
    return launch_forward(w->L(KT_FWD, st), w->L(KT_FWDA, st), 0, FWD_PLAIN);
}

extern "C" int supcg_backproject(supcg_geometry g, const void *d_y, void *d_x, int batch, void *stream)
{
    if (!g || !d_x || !d_y || batch < 1) return SUPCG_ERR_ARG;
    Workspace *w;
    int rc = ops_ws(g, batch, &w);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t es = elem_size(g->storage);
    for (int b = 0; b < batch; ++b) {
        w->hp[b].in_user = (const char *)d_y + (size_t)b * g->V * g->U * es;
        w->hp[b].out_user = (char *)d_x + (size_t)b * g->nx * g->ny * es;
    }
    if ((rc = ws_upload(w, st))) return rc;
    if ((rc = launch_stage_sino(w->L(KT_SINO, st), 0))) return rc;
    if ((rc = launch_backward(w->L(KT_BWD, st), BWD_PLAIN, w->bwin))) return rc;
    return launch_store_out(w->L(KT_VEC, st), 1);
}

static int check_precond(double mu, double rho)
{
    return (!(rho > 0.5) || !(rho <= 1.0) || !(mu >= 0.0) || !isfinite(mu)) ? SUPCG_ERR_PRECOND : SUPCG_OK;
}

static int enqueue_precond(Workspace *w, cudaStream_t st, int standalone)
{
    int rc;
    if ((rc = launch_fft_rows(w->L(KT_ROWS, st), 0, standalone, w->smem_rows))) return rc;
    if ((rc = launch_fft_cols(w->L(KT_COLS, st), standalone, w->smem_cols))) return rc;
    return launch_fft_rows(w->L(KT_ROWS, st), 1, standalone, w->smem_rows);
}

extern "C" int supcg_precondition(supcg_geometry g, double mu, double rho, const float *d_g, float *d_z, int batch,
                                  void *stream)
{
    if (!g || !d_g || !d_z || batch < 1) return SUPCG_ERR_ARG;
    int rc = check_precond(mu, rho);
    if (rc) return rc;
    Workspace *w;
    if ((rc = ops_ws(g, batch, &w))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    for (int b = 0; b < batch; ++b) {
        Prob &P = w->hp[b];
        P.in_user = d_g + (size_t)b * g->nx * g->ny;
        P.out_user = d_z + (size_t)b * g->nx * g->ny;
        P.mu = mu;
        P.rho = rho;
        P.storage = SUPCG_F32;
    }
    rc = ws_upload(w, st);
    for (int b = 0; b < batch; ++b) w->hp[b].storage = g->storage;
    if (rc) return rc;
    if ((rc = launch_stage_in(w->L(KT_TR, st), 1))) return rc;
    if ((rc = launch_fft_dtab(w->L(KT_VEC, st)))) return rc;
    if ((rc = enqueue_precond(w, st, 1))) return rc;
    return launch_store_out(w->L(KT_VEC, st), 2);
}

static int read_scal(const Prob &P, Scal *h, cudaStream_t st)
{
    SUPCG_CUDA_TRY(cudaMemcpyAsync(h, P.sc, sizeof(Scal), cudaMemcpyDeviceToHost, st));
    SUPCG_CUDA_TRY(cudaStreamSynchronize(st));
    return SUPCG_OK;
}

extern "C" int supcg_tv_tbar(supcg_geometry g, const float *d_y, float *d_tbar, double *h_out, void *stream)
{
    if (!g || !d_y || !d_tbar || !h_out) return SUPCG_ERR_ARG;
    Workspace *w;
    int rc = ops_ws(g, 1, &w);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Prob &P = w->hp[0];
    P.in_user = d_y;
    P.out_user = d_tbar;
    P.storage = SUPCG_F32;
    rc = ws_upload(w, st);
    P.storage = g->storage;
    if (rc) return rc;
    if ((rc = launch_stage_in(w->L(KT_TR, st), 0))) return rc;
    if ((rc = launch_tv_tbar(w->L(KT_TV, st)))) return rc;
    if ((rc = launch_store_out(w->L(KT_VEC, st), 3))) return rc;
    Scal s;
    if ((rc = read_scal(P, &s, st))) return rc;
    h_out[0] = s.tv_k;
    h_out[1] = s.snorm2;
    return SUPCG_OK;
}

static int check_stv(double a, double gamma, int K, long long max_trials)
{
    if (K < 0 || !(a > 0.0) || !(a <= 1.0) || !(gamma >= 0.0) || !isfinite(gamma) || max_trials < 1)
        return SUPCG_ERR_ARG;
    return SUPCG_OK;
}

extern "C" int supcg_superiorize(supcg_geometry g, float *d_x, double a, double gamma, int K, long long max_trials,
                                 long long *h_ell, int *h_trials, void *stream)
{
    if (!g || !d_x || !h_ell || *h_ell < 0) return SUPCG_ERR_ARG;
    int rc = check_stv(a, gamma, K, max_trials);
    if (rc) return rc;
    Workspace *w;
    if ((rc = ops_ws(g, 1, &w))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Prob &P = w->hp[0];
    P.in_user = d_x;
    P.out_user = d_x;
    P.storage = SUPCG_F32;
    rc = ws_upload(w, st);
    P.storage = g->storage;
    if (rc) return rc;
    if (K > w->trials_cap) {
        if (w->trials_dev) cudaFree(w->trials_dev);
        w->trials_dev = nullptr;
        w->trials_cap = 0;
        SUPCG_CUDA_TRY(cudaMalloc(&w->trials_dev, sizeof(int) * K));
        w->trials_cap = K;
    }
    Scal s0 = {};
    s0.ell = *h_ell;
    SUPCG_CUDA_TRY(cudaMemcpyAsync(P.sc, &s0, sizeof(Scal), cudaMemcpyHostToDevice, st));
    SUPCG_CUDA_TRY(cudaMemsetAsync(P.bar, 0, 2 * sizeof(unsigned), st));
    if ((rc = launch_stage_in(w->L(KT_TR, st), 0))) return rc;
    if ((rc = launch_stv(w->L(KT_STV, st), K, a, gamma, max_trials, K > 0 ? w->trials_dev : nullptr, 0))) return rc;
    if ((rc = launch_store_out(w->L(KT_VEC, st), 0))) return rc;
    Scal s;
    if ((rc = read_scal(P, &s, st))) return rc;
    if (h_trials && K > 0) SUPCG_CUDA_TRY(cudaMemcpy(h_trials, w->trials_dev, sizeof(int) * K, cudaMemcpyDeviceToHost));
    *h_ell = s.ell;
    return s.status;
}

// ------------------------------------------------------------------ launch accounting
static std::atomic<long long> g_launches{0};

struct Prof {
    std::vector<cudaEvent_t> ev;
    std::vector<int> kind;
};
static thread_local Prof *t_prof = nullptr;
static thread_local long long t_capture_count = 0;

#define LAUNCH(KIND, ST, CALL)                                                   \
    do {                                                                         \
        cudaEvent_t e0_ = nullptr;                                               \
        if (t_prof) {                                                            \
            SUPCG_CUDA_TRY(cudaEventCreate(&e0_));                               \
            SUPCG_CUDA_TRY(cudaEventRecord(e0_, ST));                            \
        }                                                                        \
        int rc_ = (CALL);                                                        \
        if (rc_) return rc_;                                                     \
        ++g_launches;                                                            \
        ++t_capture_count;                                                       \
        if (t_prof) {                                                            \
            cudaEvent_t e1_;                                                     \
            SUPCG_CUDA_TRY(cudaEventCreate(&e1_));                               \
            SUPCG_CUDA_TRY(cudaEventRecord(e1_, ST));                            \
            t_prof->ev.push_back(e0_);                                           \
            t_prof->ev.push_back(e1_);                                           \
            t_prof->kind.push_back(KIND);                                        \
        }                                                                        \
    } while (0)

extern "C" long long supcg_kernel_launches(void) { return g_launches.load(); }

extern "C" int supcg_set_wait_limit(long long polls)
{
    if (polls < 1) return SUPCG_ERR_ARG;
    g_wait_limit.store(polls);
    return SUPCG_OK;
}

extern "C" int supcg_set_barrier_shortfall(int extra_blocks)
{
    if (extra_blocks < 0 || extra_blocks > 1024) return SUPCG_ERR_ARG;
    g_bar_extra.store(extra_blocks);
    return SUPCG_OK;
}

// ------------------------------------------------------------------ ART / SupART (Sec. 3.4)
extern "C" int supcg_art(supcg_geometry g, const float *d_b, float *d_x, const supcg_art_params *p,
                         supcg_art_report *rep, void *stream)
{
    if (!g || !d_b || !d_x || !p || !rep) return SUPCG_ERR_ARG;
    if (!(p->r > 0.0) || !isfinite(p->r) || !(p->lambda > 0.0) || !(p->lambda < 2.0) || p->cycles < 0 ||
        p->K < 0 || (!isnan(p->mu) && !isfinite(p->mu)))
        return SUPCG_ERR_ARG;
    int rc;
    if (p->K > 0 && (rc = check_stv(p->a, p->gamma, p->K, p->max_trials))) return rc;
    Workspace *w;
    if ((rc = ops_ws(g, 1, &w))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t m = (size_t)g->V * g->U;
    if (!g->art_u) SUPCG_CUDA_TRY(cudaMalloc(&g->art_u, sizeof(double) * m));
    if (!g->art_rn) SUPCG_CUDA_TRY(cudaMalloc(&g->art_rn, sizeof(double) * m));
    Prob &P = w->hp[0];
    P.in_user = d_x;
    P.out_user = d_x;
    P.in_user2 = d_b;
    P.art_u = g->art_u;
    P.art_rn = g->art_rn;
    P.storage = SUPCG_F32;
    float *xlo = P.xlo;
    P.xlo = nullptr;   // ART's row actions and SupART's S_TV work on the FP32 image alone
    rc = ws_upload(w, st);
    P.storage = g->storage;
    P.xlo = xlo;
    if (rc) return rc;
    Scal s0 = {};
    s0.muX = isnan(p->mu) ? 0.0 : p->mu;
    SUPCG_CUDA_TRY(cudaMemcpyAsync(P.sc, &s0, sizeof(Scal), cudaMemcpyHostToDevice, st));
    SUPCG_CUDA_TRY(cudaMemsetAsync(P.bar, 0, 2 * sizeof(unsigned), st));
    SUPCG_CUDA_TRY(cudaMemsetAsync(P.counter, 0, 16 * sizeof(unsigned), st));
    LAUNCH(SUPCG_KIND_VECTOR, st, launch_stage_sino(w->L(KT_SINO, st), 1));   // b -> bpad
    if (isnan(p->mu)) LAUNCH(SUPCG_KIND_VECTOR, st, launch_gray(w->L(KT_SINO, st)));
    const int init_blocks = (int)std::min<size_t>(8192, (m + 1) / 2);
    LAUNCH(SUPCG_KIND_VECTOR, st, launch_art_init(w->dp, p->r, init_blocks, st));   // norms, u = 0, x = mu_X
    int cap = 0;
    if ((rc = art_max_blocks(&cap))) return rc;
    const int rays = (g->U + g->art_S - 1) / g->art_S;   // rays per class, one block each
    const int blocks = std::max(1, std::min(cap, rays));
    if (p->K == 0) {
        if (p->cycles > 0)
            LAUNCH(SUPCG_KIND_FORWARD, st, launch_art(w->dp, p->cycles, p->r, p->lambda, g->art_S, blocks, st));
    } else {
        for (int c = 0; c < p->cycles; ++c) {   // SupART: S_TV, then one cycle
            LAUNCH(SUPCG_KIND_STV, st, launch_stv(w->L(KT_STV, st), p->K, p->a, p->gamma, p->max_trials, nullptr, 0));
            LAUNCH(SUPCG_KIND_FORWARD, st, launch_art(w->dp, 1, p->r, p->lambda, g->art_S, blocks, st));
        }
    }
    LAUNCH(SUPCG_KIND_VECTOR, st, launch_store_out(w->L(KT_VEC, st), 0));
    Scal s;
    if ((rc = read_scal(P, &s, st))) return rc;
    rep->cycles = s.status ? 0 : p->cycles;
    rep->ell = s.ell;
    rep->mu = s.muX;
    rep->status = s.status;
    return s.status;
}

// ------------------------------------------------------------------ solve
static int check_params(const supcg_params *p)
{
    if (!p || p->max_iter < 0 || p->K < 0) return SUPCG_ERR_ARG;
    if (!isfinite(p->bayes_r) || (p->bayes_r > 0.0 && isinf(p->bayes_mu))) return SUPCG_ERR_ARG;
    if (p->perturb) {
        int rc = check_stv(p->a, p->gamma, p->K, p->max_trials);
        if (rc) return rc;
    }
    if (p->precondition) return check_precond(p->mu, p->rho);
    return SUPCG_OK;
}

// One while-body of Algorithm 3 (steps 10-14) over every problem of w.
static int enqueue_precond_k(Workspace *w, cudaStream_t st)
{
    LAUNCH(SUPCG_KIND_FFT, st, launch_fft_rows(w->L(KT_ROWS, st), 0, 0, w->smem_rows));
    LAUNCH(SUPCG_KIND_FFT, st, launch_fft_cols(w->L(KT_COLS, st), 0, w->smem_cols));
    LAUNCH(SUPCG_KIND_FFT, st, launch_fft_rows(w->L(KT_ROWS, st), 1, 0, w->smem_rows));
    return SUPCG_OK;
}

static int enqueue_body(Workspace *w, const supcg_params *p, cudaStream_t st, int want_snorm,
                        supcg_cnn_s *net = nullptr)
{
    int rc;
    LAUNCH(SUPCG_KIND_VECTOR, st, launch_xupdate(w->L(KT_VEC, st)));            // step 10 + deferred step 7
    const float *dir = nullptr;
    if (net && p->perturb && p->K > 0) {                                         // proposal of the network
        LAUNCH(SUPCG_KIND_STV, st, launch_tv_tbar(w->L(KT_TV, st)));
        if (w->count == 1) {
            LAUNCH(SUPCG_KIND_CNN, st, cnn_forward(net, w->hp[0].x, w->hp[0].tbar, 1, st));
        } else {                                                                 // one batch for all problems
            const size_t half = w->lstage_elems / 2;
            LAUNCH(SUPCG_KIND_VECTOR, st, launch_gather_xt(w->L(KT_VEC, st), w->lstage, w->lstage + half));
            LAUNCH(SUPCG_KIND_CNN, st, cnn_forward(net, w->lstage, w->lstage + half, w->count, st));
        }
        dir = cnn_output(net);
    }
    // r = R x - b and f at x_{k+1/2}: r moves with x, by alpha q for step 7 (q = R p from the
    // previous norm pass) and by R d for the displacement d of S_TV, which S_TV writes in the
    // projector's layouts; the same sums as projecting x, in one pass over d
    if (p->perturb && p->K > 0) {                                               // steps 11-12
        LAUNCH(SUPCG_KIND_STV, st, launch_stv(w->L(KT_STV, st), p->K, p->a, p->gamma, p->max_trials, nullptr,
                                              want_snorm, dir));
        LAUNCH(SUPCG_KIND_FORWARD, st, launch_forward(w->L(KT_FWD, st), w->L(KT_FWDA, st), 2, FWD_RUPD));
    } else {
        LAUNCH(SUPCG_KIND_VECTOR, st, launch_rupdate(w->L(KT_SINO, st)));
    }
    // g = R^T r, and h = R^T q of the previous step (A p for this step's beta; the previous alpha
    // took p^T A p from ||q||^2), one pass over the views for both
    LAUNCH(SUPCG_KIND_BACKWARD, st, launch_backward2(w->L(KT_BWD2, st), w->bwin));
    if (p->precondition) {                                                      // z = M g; its last pass
        if ((rc = enqueue_precond_k(w, st))) return rc;                         // also forms beta
    } else {
        LAUNCH(SUPCG_KIND_VECTOR, st, launch_beta(w->L(KT_VEC, st)));           // beta = z^T h / p^T h
    }
    LAUNCH(SUPCG_KIND_VECTOR, st, launch_pupdate(w->L(KT_TR, st)));             // p = -z + beta p, g^T p, p^T
    // q = R p, p^T h, alpha; its last block also logs the step and sets k <- k + 1 (step 14)
    LAUNCH(SUPCG_KIND_FORWARD, st, launch_forward(w->L(KT_FWD, st), w->L(KT_FWDA, st), 1, FWD_NORM));
    return SUPCG_OK;
}

// Steps 1-9 of Algorithm 3: the same schedule with beta = 0 and no S_TV.
static int enqueue_init(Workspace *w, const supcg_params *p, cudaStream_t st)
{
    int rc;
    LAUNCH(SUPCG_KIND_FORWARD, st, launch_forward(w->L(KT_FWD, st), w->L(KT_FWDA, st), 0, FWD_RESID));
    LAUNCH(SUPCG_KIND_BACKWARD, st, launch_backward(w->L(KT_BWD, st), BWD_G, w->bwin));
    if (p->precondition) {
        if ((rc = enqueue_precond_k(w, st))) return rc;
    } else {
        LAUNCH(SUPCG_KIND_VECTOR, st, launch_beta(w->L(KT_VEC, st)));
    }
    LAUNCH(SUPCG_KIND_VECTOR, st, launch_pupdate(w->L(KT_TR, st)));
    // (h = A p: in the next pass; the last block ends steps 1-9: init <- 0)
    LAUNCH(SUPCG_KIND_FORWARD, st, launch_forward(w->L(KT_FWD, st), w->L(KT_FWDA, st), 1, FWD_NORM));
    return SUPCG_OK;
}

// Selective-error logging of a sweep (Eq. (4.1)): reference image, per-problem logs, semi-axes in pixels.
struct SeLog {
    const float *ref = nullptr;
    double *logs = nullptr;   // [count][max_iter]
    double ax = 0.0, ay = 0.0;
};

// per (nullable): per-problem parameters of a sweep; each problem then takes its S_TV (K, a,
// gamma) and preconditioner (mu, rho) parameters from per[c] and everything else from p.
static int run_solve(Workspace *w, const float *const *d_b, float *const *d_x, const supcg_params *p,
                     supcg_report *reps, double *d_log, cudaStream_t st, float *d_trace = nullptr,
                     supcg_cnn_s *net = nullptr, const supcg_params *per = nullptr, const SeLog *se = nullptr)
{
    int rc;
    for (int c = 0; c < w->count; ++c) {
        Prob &P = w->hp[c];
        const supcg_params &q = per ? per[c] : *p;
        P.in_user = d_x[c];
        P.out_user = d_x[c];
        P.in_user2 = d_b[c];
        P.mu = q.mu;
        P.rho = q.rho;
        P.stv_own = per ? 1 : 0;
        P.stv_K = q.K;
        P.stv_a = q.a;
        P.stv_gamma = q.gamma;
        P.precond = p->precondition ? 1 : 0;
        P.r2 = p->bayes_r > 0.0 ? p->bayes_r * p->bayes_r : 0.0;
        P.storage = SUPCG_F32;
        P.log = (c == 0) ? d_log : nullptr;
        P.trace = (c == 0) ? d_trace : nullptr;
        P.se_ref = (se && se->ref) ? se->ref : nullptr;
        P.se_log = P.se_ref ? se->logs + (size_t)c * std::max(1, p->max_iter) : nullptr;
        P.se_ax = se ? se->ax * P.nx : 0.0;
        P.se_ay = se ? se->ay * P.ny : 0.0;
    }
    rc = ws_upload(w, st);
    for (int c = 0; c < w->count; ++c) w->hp[c].storage = w->geoms[c]->storage;
    if (rc) return rc;
    std::vector<Scal> s0(w->count);
    for (int c = 0; c < w->count; ++c) {
        const Prob &P = w->hp[c];
        s0[c] = Scal();
        s0[c].eps = p->eps;
        s0[c].init = 1;
        s0[c].muX = isnan(p->bayes_mu) ? 0.0 : p->bayes_mu;   // NaN: estimated from b below
        SUPCG_CUDA_TRY(cudaMemcpyAsync(P.sc, &s0[c], sizeof(Scal), cudaMemcpyHostToDevice, st));
        SUPCG_CUDA_TRY(cudaMemsetAsync(P.counter, 0, 16 * sizeof(unsigned), st));
        SUPCG_CUDA_TRY(cudaMemsetAsync(P.bar, 0, 2 * sizeof(unsigned), st));
        SUPCG_CUDA_TRY(cudaMemsetAsync(P.p, 0, sizeof(float) * (size_t)P.ny * P.nxp, st));
        SUPCG_CUDA_TRY(cudaMemsetAsync(P.h, 0, sizeof(float) * (size_t)P.ny * P.nxp, st));
    }
    LAUNCH(SUPCG_KIND_VECTOR, st, launch_stage_in(w->L(KT_TR, st), 0));
    LAUNCH(SUPCG_KIND_VECTOR, st, launch_stage_sino(w->L(KT_SINO, st), 1));
    if (p->bayes_r > 0.0 && isnan(p->bayes_mu)) LAUNCH(SUPCG_KIND_VECTOR, st, launch_gray(w->L(KT_SINO, st)));
    if (p->precondition) LAUNCH(SUPCG_KIND_VECTOR, st, launch_fft_dtab(w->L(KT_VEC, st)));
    if ((rc = enqueue_init(w, p, st))) return rc;

    const int want_snorm = d_log != nullptr;
    const bool eps_mode = p->eps >= 0.0;
    if (eps_mode && !w->hdone) SUPCG_CUDA_TRY(cudaMallocHost(&w->hdone, sizeof(int) * w->count));   // once per workspace
    int *hdone = w->hdone;
    bool use_graph = p->graph != 0 && t_prof == nullptr;
    if (use_graph) {
        const double key[6] = {p->a, p->gamma, (double)p->max_trials, (double)p->K, (double)p->perturb,
                               (double)p->precondition};
        const int key_i[4] = {want_snorm, 1, (int)((uintptr_t)d_trace & 0x7fffffff), (int)((uintptr_t)net & 0x7fffffff)};
        if (!w->body_exec || memcmp(key, w->key, sizeof(key)) || memcmp(key_i, w->key_i, sizeof(key_i))) {
            if (w->body_exec) cudaGraphExecDestroy(w->body_exec);
            w->body_exec = nullptr;
            cudaGraph_t graph = nullptr;
            if (cudaStreamBeginCapture(w->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                use_graph = false;
            } else {
                t_capture_count = 0;
                int brc = enqueue_body(w, p, w->cap_stream, want_snorm, net);
                w->body_nodes = t_capture_count;
                cudaError_t e = cudaStreamEndCapture(w->cap_stream, &graph);
                if (brc || e != cudaSuccess || cudaGraphInstantiate(&w->body_exec, graph, 0) != cudaSuccess) {
                    use_graph = false;
                    w->body_exec = nullptr;
                    (void)cudaGetLastError();
                }
                if (graph) cudaGraphDestroy(graph);
            }
            if (use_graph) {
                memcpy(w->key, key, sizeof(key));
                memcpy(w->key_i, key_i, sizeof(key_i));
            }
        }
    }
    for (int it = 0; it < p->max_iter; ++it) {
        if (use_graph) {
            SUPCG_CUDA_TRY(cudaGraphLaunch(w->body_exec, st));
            g_launches += w->body_nodes;
        } else if ((rc = enqueue_body(w, p, st, want_snorm, net))) return rc;
        if (eps_mode && (it % 8 == 7)) {   // stop launching once every problem has stopped
            for (int c = 0; c < w->count; ++c)
                SUPCG_CUDA_TRY(cudaMemcpyAsync(hdone + c, &w->hp[c].sc->done, sizeof(int), cudaMemcpyDeviceToHost, st));
            SUPCG_CUDA_TRY(cudaStreamSynchronize(st));
            bool all = true;
            for (int c = 0; c < w->count; ++c) all = all && hdone[c];
            if (all) break;
        }
    }
    LAUNCH(SUPCG_KIND_VECTOR, st, launch_store_out(w->L(KT_VEC, st), 0));
    std::vector<Scal> hs(w->count);
    for (int c = 0; c < w->count; ++c)
        SUPCG_CUDA_TRY(cudaMemcpyAsync(&hs[c], w->hp[c].sc, sizeof(Scal), cudaMemcpyDeviceToHost, st));
    SUPCG_CUDA_TRY(cudaStreamSynchronize(st));
    int worst = SUPCG_OK;
    for (int c = 0; c < w->count; ++c) {
        supcg_report &r = reps[c];
        r.iters = hs[c].k;
        r.k = hs[c].k + 1;
        r.ell = hs[c].ell;
        r.f_last = hs[c].f;
        r.f0 = hs[c].f0;
        r.tv_last = hs[c].tv_half;
        r.status = hs[c].status;
        r.n_fallback = hs[c].n_fallback;
        r.n_learned = hs[c].n_learned;
        if (hs[c].status && !worst) worst = hs[c].status;
    }
    return worst;
}

extern "C" int supcg_solve(supcg_geometry g, const float *d_b, float *d_x, const supcg_params *p, supcg_report *rep,
                           double *d_log, void *stream)
{
    if (!g || !d_b || !d_x || !rep) return SUPCG_ERR_ARG;
    int rc = check_params(p);
    if (rc) return rc;
    if (!g->ws_solve) {
        std::vector<supcg_geometry> gs(1, g);
        if ((rc = ws_create(gs, &g->ws_solve))) return rc;
    }
    return run_solve(g->ws_solve, &d_b, &d_x, p, rep, d_log, (cudaStream_t)stream);
}

extern "C" int supcg_solve_trace(supcg_geometry g, const float *d_b, float *d_x, const supcg_params *p,
                                 supcg_report *rep, double *d_log, float *d_trace, void *stream)
{
    if (!g || !d_b || !d_x || !rep || !d_trace) return SUPCG_ERR_ARG;
    int rc = check_params(p);
    if (rc) return rc;
    if (!g->ws_solve) {
        std::vector<supcg_geometry> gs(1, g);
        if ((rc = ws_create(gs, &g->ws_solve))) return rc;
    }
    return run_solve(g->ws_solve, &d_b, &d_x, p, rep, d_log, (cudaStream_t)stream, d_trace);
}

extern "C" int supcg_solve_learned(supcg_geometry g, supcg_cnn_s *net, const float *d_b, float *d_x,
                                   const supcg_params *p, supcg_report *rep, double *d_log, void *stream)
{
    if (!g || !net || !d_b || !d_x || !rep) return SUPCG_ERR_ARG;
    int rc = check_params(p);
    if (rc) return rc;
    int ny = 0, nx = 0;
    cnn_shape(net, &ny, &nx);
    if (ny != g->ny || nx != g->nx || g->nxp != g->nx) return SUPCG_ERR_UNSUPPORTED;
    if (!g->ws_solve) {
        std::vector<supcg_geometry> gs(1, g);
        if ((rc = ws_create(gs, &g->ws_solve))) return rc;
    }
    // run the network once outside any capture (kernel attributes are set on first use)
    Workspace *w = g->ws_solve;
    if ((rc = cnn_forward(net, w->hp[0].x, w->hp[0].tbar, 1, (cudaStream_t)stream))) return rc;
    SUPCG_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    return run_solve(w, &d_b, &d_x, p, rep, d_log, (cudaStream_t)stream, nullptr, net);
}

extern "C" int supcg_solve_profiled(supcg_geometry g, const float *d_b, float *d_x, const supcg_params *p,
                                    supcg_report *rep, double *h_ms, long long *h_launches, void *stream)
{
    if (!h_ms || !h_launches) return SUPCG_ERR_ARG;
    Prof prof;
    t_prof = &prof;
    int rc = supcg_solve(g, d_b, d_x, p, rep, nullptr, stream);
    t_prof = nullptr;
    for (int k = 0; k < SUPCG_KIND_COUNT; ++k) { h_ms[k] = 0.0; h_launches[k] = 0; }
    cudaStreamSynchronize((cudaStream_t)stream);
    for (size_t i = 0; i < prof.kind.size(); ++i) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, prof.ev[2 * i], prof.ev[2 * i + 1]) == cudaSuccess) {
            h_ms[prof.kind[i]] += ms;
            h_launches[prof.kind[i]] += 1;
        }
    }
    for (cudaEvent_t e : prof.ev) cudaEventDestroy(e);
    return rc;
}

extern "C" int supcg_solve_host(supcg_geometry g, const float *h_b, float *h_x, const supcg_params *p,
                                supcg_report *rep, void *stream)
{
    if (!g || !h_b || !h_x || !rep) return SUPCG_ERR_ARG;
    int rc = check_params(p);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nb = sizeof(float) * (size_t)g->V * g->U, nx = sizeof(float) * (size_t)g->nx * g->ny;
    // device copies kept with the geometry (like its workspace): no allocation per call
    if (!g->host_db) SUPCG_CUDA_TRY(cudaMalloc(&g->host_db, nb));
    if (!g->host_dx) SUPCG_CUDA_TRY(cudaMalloc(&g->host_dx, nx));
    float *db = g->host_db, *dx = g->host_dx;
    SUPCG_CUDA_TRY(cudaMemcpyAsync(db, h_b, nb, cudaMemcpyHostToDevice, st));
    SUPCG_CUDA_TRY(cudaMemcpyAsync(dx, h_x, nx, cudaMemcpyHostToDevice, st));
    rc = supcg_solve(g, db, dx, p, rep, nullptr, stream);
    if (rc == SUPCG_OK || rc < SUPCG_ERR_NOMEM) {
        SUPCG_CUDA_TRY(cudaMemcpyAsync(h_x, dx, nx, cudaMemcpyDeviceToHost, st));
    }
    SUPCG_CUDA_TRY(cudaStreamSynchronize(st));
    return rc;
}

extern "C" int supcg_solve_batched(const supcg_geometry *gs, const float *const *d_b, float *const *d_x, int count,
                                   const supcg_params *p, supcg_report *reps, void *stream)
{
    if (!gs || !d_b || !d_x || !reps || count < 1) return SUPCG_ERR_ARG;
    for (int c = 0; c < count; ++c)
        if (!gs[c] || !d_b[c] || !d_x[c]) return SUPCG_ERR_ARG;
    int rc = check_params(p);
    if (rc) return rc;
    supcg_geometry owner = gs[0];
    std::vector<supcg_geometry> key(gs, gs + count);
    if (!batch_ws_current(owner, key)) {
        free_ws(owner->ws_batch);
        if ((rc = ws_create(key, &owner->ws_batch))) return rc;
        owner->batch_key = key;
    }
    return run_solve(owner->ws_batch, d_b, d_x, p, reps, nullptr, (cudaStream_t)stream);
}

extern "C" int supcg_solve_batched_learned(const supcg_geometry *gs, supcg_cnn_s *net, const float *const *d_b,
                                           float *const *d_x, int count, const supcg_params *p, supcg_report *reps,
                                           void *stream)
{
    if (!gs || !net || !d_b || !d_x || !reps || count < 1) return SUPCG_ERR_ARG;
    int ny = 0, nx = 0, cap = 0;
    cnn_shape(net, &ny, &nx);
    cnn_capacity(net, &cap);
    if (count > cap) return SUPCG_ERR_ARG;
    for (int c = 0; c < count; ++c) {
        if (!gs[c] || !d_b[c] || !d_x[c]) return SUPCG_ERR_ARG;
        if (gs[c]->ny != ny || gs[c]->nx != nx || gs[c]->nxp != nx) return SUPCG_ERR_UNSUPPORTED;
    }
    int rc = check_params(p);
    if (rc) return rc;
    supcg_geometry owner = gs[0];
    std::vector<supcg_geometry> key(gs, gs + count);
    if (!batch_ws_current(owner, key)) {
        free_ws(owner->ws_batch);
        if ((rc = ws_create(key, &owner->ws_batch))) return rc;
        owner->batch_key = key;
    }
    Workspace *w = owner->ws_batch;
    const size_t need = 2 * (size_t)count * ny * nx;
    if (w->lstage_elems != need) {
        if (w->lstage) cudaFree(w->lstage);
        w->lstage = nullptr;
        w->lstage_elems = 0;
        if (cudaMalloc(&w->lstage, need * sizeof(float)) != cudaSuccess) return SUPCG_ERR_NOMEM;
        SUPCG_CUDA_TRY(cudaMemset(w->lstage, 0, need * sizeof(float)));
        w->lstage_elems = need;
    }
    // run the network once outside any capture (kernel attributes are set on first use)
    if ((rc = cnn_forward(net, w->lstage, w->lstage + need / 2, count, (cudaStream_t)stream))) return rc;
    SUPCG_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    return run_solve(w, d_b, d_x, p, reps, nullptr, (cudaStream_t)stream, nullptr, net);
}

extern "C" int supcg_solve_sweep(supcg_geometry g, const float *d_b, float *const *d_x, int count,
                                 const supcg_params *ps, const float *d_ref, double se_ax, double se_ay,
                                 double *d_se, supcg_report *reps, void *stream)
{
    if (!g || !d_b || !d_x || !ps || !reps || count < 1) return SUPCG_ERR_ARG;
    if (d_ref && (!d_se || !(se_ax > 0.0) || !(se_ay > 0.0))) return SUPCG_ERR_ARG;
    const supcg_params &p0 = ps[0];
    auto same_mu = [](double u, double v) { return (isnan(u) && isnan(v)) || u == v; };
    for (int c = 0; c < count; ++c) {
        if (!d_x[c]) return SUPCG_ERR_ARG;
        const supcg_params &q = ps[c];
        int rc = check_params(&q);
        if (rc) return rc;
        // what is not swept is shared: the launch schedule and the loop control
        if (q.perturb != p0.perturb || q.precondition != p0.precondition || q.eps != p0.eps ||
            q.max_iter != p0.max_iter || q.max_trials != p0.max_trials || q.graph != p0.graph ||
            q.bayes_r != p0.bayes_r || !same_mu(q.bayes_mu, p0.bayes_mu) || (p0.perturb && q.K < 1))
            return SUPCG_ERR_ARG;
    }
    std::vector<supcg_geometry> key(count, g);
    if (!batch_ws_current(g, key)) {
        free_ws(g->ws_batch);
        int rc = ws_create(key, &g->ws_batch);
        if (rc) return rc;
        g->batch_key = key;
    }
    std::vector<const float *> bs(count, d_b);
    SeLog se;
    se.ref = d_ref;
    se.logs = d_se;
    se.ax = se_ax;
    se.ay = se_ay;
    return run_solve(g->ws_batch, bs.data(), d_x, &p0, reps, nullptr, (cudaStream_t)stream, nullptr, nullptr, ps,
                     d_ref ? &se : nullptr);
}

extern "C" const char *supcg_status_string(int status)
{
    switch (status) {
    case SUPCG_OK: return "ok";
    case SUPCG_ERR_ARG: return "invalid argument";
    case SUPCG_ERR_CUDA: return "CUDA error";
    case SUPCG_ERR_NOMEM: return "out of memory";
    case SUPCG_ERR_BREAKDOWN: return "CG breakdown (p^T h <= 0 or non-finite scalar)";
    case SUPCG_ERR_BACKTRACK: return "S_TV backtracking exceeded max_trials";
    case SUPCG_ERR_TIMEOUT: return "bounded device wait expired";
    case SUPCG_ERR_PRECOND: return "preconditioner not positive definite";
    case SUPCG_ERR_UNSUPPORTED: return "geometry outside the supported range";
    default: return "unknown status";
    }
}
