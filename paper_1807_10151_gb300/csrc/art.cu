// ART for the Bayesian criterion of Eq. (2.3) and its superiorization SupART
// (Sec. 3.4: the row-action method of Herman, Hurwitz and Lent).
//
// The method sweeps the consistent system r R (x - mu_X) + u = r (b - R mu_X),
// one auxiliary value u_i per ray, whose minimum-norm solution minimises
// r^2 ||R x - b||^2 + ||x - mu_X||^2.  From x = mu_X, u = 0, ray i updates
//     c = lambda (r (b_i - <R_i, x>) - u_i) / (1 + r^2 ||R_i||^2),
//     x <- x + r c R_i,   u_i <- u_i + c,
// and a cycle visits every ray once.  A cycle here takes the views in order
// and, within a view, the rays in S residue classes u = c (mod S), S the
// smallest spacing at which two rays of one view touch no common pixel.  The
// rays of one class run in parallel, one block each: their supports are
// disjoint, so this equals any sequential order of the class; a grid barrier
// (bounded) separates consecutive classes.  A ray's entries are the
// projectors' (the same exact-split delta and trapezoid), evaluated once for
// the ray sum <R_i, x> (a Kahan-compensated FP32 sum per thread, the
// threads' sums added in FP64) and again for the update (FP32 FMA; this
// part's FP64 pipe is narrow).  One block per ray: its threads take a few
// rows each and issue all their loads before using them (the pixels sit in
// L2, and a long chain of dependent loads had dominated).
#include "internal.cuh"

namespace supcg {

constexpr int kArtThreads = 64;      // k_art_init: two warps, one ray each
constexpr int kArtRayThreads = 128;  // k_art: one block per ray of a class
constexpr int kArtRows = 4;          // rows per thread per group: their 4 x 3 loads issued together

// The per-ray constants of a ray's entries (the projectors' exact split).
struct ArtRay {
    float tau_hi, qh, hi_o, lo_o, hi_i, lo_i, c_in, dI;
    int lo, hi, n_inner, nc;
    bool cb, axis;
};

__device__ __forceinline__ ArtRay art_ray_setup(const Prob &P, const ViewP &vp, int u)
{
    ArtRay R;
    R.cb = (vp.flags & kViewClassB) != 0;
    R.axis = (vp.flags & kViewAxis) != 0;
    R.nc = (vp.flags & kViewFwd3) ? 3 : 2;
    const int n_outer = R.cb ? P.nx : P.ny;
    R.n_inner = R.cb ? P.ny : P.nx;
    R.tau_hi = bin_pos(u, P.uc_hi);                                      // exact
    const float base = __fmaf_rn(vp.a_tau, bin_pos(u, P.uc), vp.g0);    // ray centre at outer index 0
    fwd_row_range(vp, base, R.n_inner, n_outer, &R.lo, &R.hi);
    R.hi_o = R.cb ? vp.cu_hi : vp.su_hi;   // outer coordinate
    R.lo_o = R.cb ? vp.cu_lo : vp.su_lo;
    R.hi_i = R.cb ? vp.su_hi : vp.cu_hi;   // inner coordinate
    R.lo_i = R.cb ? vp.su_lo : vp.cu_lo;
    R.c_in = R.cb ? P.cy : P.cx;
    R.dI = R.cb ? -1.0f : 1.0f;
    R.qh = __fsub_rn(base, vp.hwq);
    return R;
}

// Row o of the ray: the pixel offsets and unit weights of its (up to three)
// candidates; weight 0 for candidates off the image or outside the footprint.
__device__ __forceinline__ void art_row(const Prob &P, const ViewP &vp, const ArtRay &R, int o, int *pix, float *w)
{
    const float of = __int2float_rn(o);
    const float Oc = R.cb ? __fsub_rn(of, P.cx) : __fsub_rn(P.cy, of);
    const float rbig = __fmaf_rn(-R.hi_o, Oc, R.tau_hi);                 // exact
    const float rsmall = __fmaf_rn(R.lo_o, Oc, P.uc_lo);
    const float qc = ceil_magic(__fmaf_rn(of, vp.b_o, R.qh));            // first candidate
    const int q0 = magic_int(qc);
    float I = R.cb ? __fsub_rn(R.c_in, magic_float(qc)) : __fsub_rn(magic_float(qc), R.c_in);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (k) I = __fadd_rn(I, R.dI);                                     // exact
        const float big = __fmaf_rn(-R.hi_i, I, rbig);                   // exact
        const float ad = fabsf(__fsub_rn(big, __fmaf_rn(R.lo_i, I, rsmall)));
        const int q = q0 + k;
        const bool in = k < R.nc && q >= 0 && q < R.n_inner;
        w[k] = in ? weight_unit(ad, vp.E, vp.Sn, vp.ESn, R.axis) : 0.0f;
        pix[k] = in ? (R.cb ? q * P.nxp + o : o * P.nxp + q) : 0;
    }
}

// f(pixel offset, unit weight) for every entry of ray (vp, u) with a nonzero
// weight, over the rows lane, lane + 32, ... (used where latency does not matter).
template <typename F>
__device__ __forceinline__ void art_ray(const Prob &P, const ViewP &vp, int u, int lane, F &&f)
{
    const ArtRay R = art_ray_setup(P, vp, u);
    for (int o = R.lo + lane; o <= R.hi; o += 32) {
        int pix[3];
        float w[3];
        art_row(P, vp, R, o, pix, w);
#pragma unroll
        for (int k = 0; k < 3; ++k)
            if (w[k] != 0.0f) f(pix[k], w[k]);
    }
}

// 1 / (1 + r^2 ||R_i||^2) for every ray (FP64), u = 0, and x = mu_X on the image
// (the starting point of the method).  One warp per ray, grid-stride.
__global__ void __launch_bounds__(kArtThreads) k_art_init(const Prob *__restrict__ probs, double r)
{
    const Prob &P = probs[0];
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (kArtThreads / 32) + (threadIdx.x >> 5), W = gridDim.x * (kArtThreads / 32);
    for (int i = gw; i < P.V * P.U; i += W) {
        const int v = i / P.U, u = i - v * P.U;
        const ViewP vp = P.views[v];
        double s = 0.0;
        art_ray(P, vp, u, lane, [&](int, float w) { s += (double)w * (double)w; });
        s = warp_sum(s);
        if (lane == 0) {
            const double pl = (double)vp.P;
            P.art_rn[i] = 1.0 / (1.0 + r * r * pl * pl * s);
            P.art_u[i] = 0.0;
        }
    }
    const float mu = (float)P.sc->muX;
    const size_t n = (size_t)P.ny * P.nxp;
    for (size_t e = (size_t)blockIdx.x * kArtThreads + threadIdx.x; e < n; e += (size_t)gridDim.x * kArtThreads) {
        const int j = (int)(e % P.nxp);
        P.x[e] = (j < P.nx) ? mu : 0.0f;   // the padding stays 0
    }
}

// `cycles` full ART cycles on P.x (one cooperative launch; every block takes
// part in every class barrier).  Block b takes the rays u = c + S (b + k nblocks)
// of class c; its threads split the ray's rows, kArtRows at a time, and load
// the rows' candidates before using them (the pixels were written by other
// blocks before the last barrier: read past L1).
__global__ void __launch_bounds__(kArtRayThreads) k_art(const Prob *__restrict__ probs, int cycles, double r,
                                                        double lam, int S)
{
    __shared__ int flag;
    __shared__ __align__(16) double red[40];
    __shared__ float sh_rc;
    const Prob &P = probs[0];
    Scal *sc = P.sc;
    const int t = threadIdx.x;
    float *x = P.x;
    for (int cyc = 0; cyc < cycles; ++cyc) {
        for (int v = 0; v < P.V; ++v) {
            const ViewP vp = P.views[v];
            for (int c = 0; c < S; ++c) {
                for (int u = c + S * blockIdx.x; u < P.U; u += S * gridDim.x) {   // block-uniform
                    const ArtRay R = art_ray_setup(P, vp, u);
                    const size_t i = (size_t)v * P.U + u;
                    double bi = 0.0, ui = 0.0, rni = 0.0;   // the ray's scalars, fetched while the sum runs
                    if (t == 0) {
                        bi = (double)P.bpad[(size_t)v * P.Up + u];
                        ui = P.art_u[i];
                        rni = P.art_rn[i];
                    }
                    float ks = 0.0f, kc = 0.0f;   // Kahan pair of the thread's terms of <R_i, x>
                    // a ray of at most kArtRows x kArtRayThreads rows: each thread's rows, weights and
                    // pixel values are gathered once and kept for the update (the class's other rays
                    // touch none of these pixels, so the values are still current then)
                    const bool one_group = R.hi - R.lo < kArtRows * kArtRayThreads;
                    int gpix[3 * kArtRows];
                    float gw[3 * kArtRows], gx[3 * kArtRows];
                    for (int o0 = R.lo + t; o0 <= R.hi; o0 += kArtRows * kArtRayThreads) {
                        int *pix = gpix;
                        float *w = gw, *xv = gx;
#pragma unroll
                        for (int q = 0; q < kArtRows; ++q) {
                            const int o = o0 + q * kArtRayThreads;
                            if (o <= R.hi) {
                                art_row(P, vp, R, o, pix + 3 * q, w + 3 * q);
                            } else {
                                w[3 * q] = w[3 * q + 1] = w[3 * q + 2] = 0.0f;
                                pix[3 * q] = pix[3 * q + 1] = pix[3 * q + 2] = 0;
                            }
                        }
#pragma unroll
                        for (int k = 0; k < 3 * kArtRows; ++k) xv[k] = (w[k] != 0.0f) ? __ldcg(x + pix[k]) : 0.0f;
#pragma unroll
                        for (int k = 0; k < 3 * kArtRows; ++k) {
                            const float y = __fmaf_rn(w[k], xv[k], -kc);
                            const float tt = __fadd_rn(ks, y);
                            kc = __fsub_rn(__fsub_rn(tt, ks), y);
                            ks = tt;
                        }
                    }
                    const double s = block_sum<kArtRayThreads>((double)ks - (double)kc, red);   // in thread 0
                    if (t == 0) {
                        const double cc = lam * (r * (bi - (double)vp.P * s) - ui) * rni;
                        P.art_u[i] = ui + cc;
                        sh_rc = (float)(r * cc * (double)vp.P);
                    }
                    __syncthreads();
                    const float rcf = sh_rc;
                    if (one_group) {
                        if (t <= R.hi - R.lo) {   // (threads past the ray's rows gathered nothing)
#pragma unroll
                            for (int k = 0; k < 3 * kArtRows; ++k)
                                if (gw[k] != 0.0f) x[gpix[k]] = __fmaf_rn(rcf, gw[k], gx[k]);
                        }
                    } else
                    for (int o0 = R.lo + t; o0 <= R.hi; o0 += kArtRows * kArtRayThreads) {
                        int pix[3 * kArtRows];
                        float w[3 * kArtRows], xv[3 * kArtRows];
#pragma unroll
                        for (int q = 0; q < kArtRows; ++q) {
                            const int o = o0 + q * kArtRayThreads;
                            if (o <= R.hi) {
                                art_row(P, vp, R, o, pix + 3 * q, w + 3 * q);
                            } else {
                                w[3 * q] = w[3 * q + 1] = w[3 * q + 2] = 0.0f;
                                pix[3 * q] = pix[3 * q + 1] = pix[3 * q + 2] = 0;
                            }
                        }
#pragma unroll
                        for (int k = 0; k < 3 * kArtRows; ++k) xv[k] = (w[k] != 0.0f) ? __ldcg(x + pix[k]) : 0.0f;
#pragma unroll
                        for (int k = 0; k < 3 * kArtRows; ++k)
                            if (w[k] != 0.0f) x[pix[k]] = __fmaf_rn(rcf, w[k], xv[k]);
                    }
                    __syncthreads();   // sh_rc and red are reused by the block's next ray
                }
                if (!coop_barrier(P.bar, gridDim.x + P.bar_extra, &sc->status, &flag, P.wait_limit)) return;   // bounded: SUPCG_ERR_TIMEOUT
            }
        }
    }
}

int art_max_blocks(int *out)
{
    int nsm = 0, per_sm = 0, dev = 0;
    SUPCG_CUDA_TRY(cudaGetDevice(&dev));
    SUPCG_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    SUPCG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_art, kArtRayThreads, 0));
    *out = nsm * per_sm;
    return SUPCG_OK;
}

int launch_art_init(const Prob *d_prob, double r, int blocks, cudaStream_t st)
{
    k_art_init<<<blocks, kArtThreads, 0, st>>>(d_prob, r);
    SUPCG_CUDA_TRY(cudaGetLastError());
    return SUPCG_OK;
}

int launch_art(const Prob *d_prob, int cycles, double r, double lam, int S, int blocks, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kArtRayThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SUPCG_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_art, d_prob, cycles, r, lam, S));
    return SUPCG_OK;
}

} // namespace supcg
