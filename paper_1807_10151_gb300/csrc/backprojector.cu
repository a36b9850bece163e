// The exact transpose R^T y of the forward projection (Eq. (2.2): normal
// equations R^T R x = R^T b).
//
// Backward (pixel-driven, gather over bins, no atomics).  A tile of 32 x 32
// pixels is shared by P.bparts blocks (the geometry's view parts, 1 .. 8),
// each taking a contiguous part of the view chunks; for chunks of 32 views the bins that the tile projects
// onto are staged in shared memory with 16-byte vector loads; every pixel
// gathers the two (three) bins nearest to its projected centre with the same
// weight evaluated on the same FP32 operands as the forward kernel.  The last
// block of a tile to finish adds the parts' double-float sums in part order.
#include "internal.cuh"

namespace supcg {

// The kernel's dynamic shared memory (the staged sinogram windows), indexed by
// 32-bit float offsets so that operand loads are plain shared-memory loads.
extern __shared__ __align__(128) float proj_dyn[];

// ============================================================ backward
constexpr int kBwdSplit = 2;                                             // thread groups splitting the views
constexpr int kBwdGroup = 128;                                           // threads per group
constexpr int kBwdThreads = kBwdSplit * kBwdGroup;
constexpr int kBwdRowStep = kBwdGroup / kBwdTileJ;                       // 4

// Tiles of 32 x 32 pixels, 8 per thread, over one sinogram or, DUAL, two (the
// solver's R^T r and R^T q in one pass: each pixel's weights evaluated once and
// applied to both; twice the sums per thread, so two blocks per SM instead of
// three).  Either way a pixel sums its views in the same order (same groups,
// folds and parts), so each output has the same bits as from the one-sinogram kernel.
template <bool DUAL>
struct BwdShape {
    static constexpr int NS = DUAL ? 2 : 1;                        // sinograms
    static constexpr int TI = kBwdTileI;                           // tile rows
    static constexpr int PX = TI * kBwdTileJ / kBwdGroup;          // pixels per thread
};

// Per pixel and view: the bins within hwu (half-width + margin) of the pixel's
// projected centre, two of them (three when the bins are finer than pixels),
// with a check of the staged window.  t[s * PX + e]: sinogram s, pixel e; the
// window of sinogram s starts qoff floats after that of sinogram 0.
template <bool AXIS, int NC, int PX, int NS>
__device__ __forceinline__ void bwd_view(const ViewP &vp, float pb0, const float *sm, int w_row, int lo,
                                         int bwin, int qoff, float *t, int *bad)
{
    const float E = vp.E, Sn = vp.Sn, ESn = vp.ESn;
#pragma unroll
    for (int e = 0; e < PX; ++e) {
        // delta = (u + pb) - small; pb = -uc_hi - cu_hi X - su_hi Y is exact, and so is
        // stepping it by su_hi per pixel row
        const float pb = __fmaf_rn((float)(kBwdRowStep * e), vp.su_hi, pb0);
        const float uc = ceil_magic(__fsub_rn(__fsub_rn(sm[e], pb), vp.hwu));
        int u0 = magic_int(uc);
        const int idx = u0 - lo;
        if (idx < 0 || idx > bwin - NC) {   // outside the staged window: never for a valid window
            *bad = 1;
            u0 = min(max(idx, 0), bwin - NC) + lo;
        }
        const float big0 = __fadd_rn(__int2float_rn(u0), pb);   // exact, as are big0 + 1 and big0 + 2
        const int wv = w_row + (u0 - lo);
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const float ad = fabsf(__fsub_rn(__fadd_rn(big0, (float)k), sm[e]));
            const float w = weight_unit(ad, E, Sn, ESn, AXIS);
#pragma unroll
            for (int s = 0; s < NS; ++s)   // the window holds P * y
                t[s * PX + e] = __fmaf_rn(w, proj_dyn[wv + s * qoff + k], t[s * PX + e]);
        }
    }
}

// The same for the thread's pixels in pairs (2h, 2h + 1), every FP32 step as one
// f32x2 instruction; only for windows that hold every candidate (no checks).
// sm2[h] = (small of pixel 2h, of pixel 2h + 1); t2[s * PX / 2 + h] the pairs'
// running sums for sinogram s.
template <bool AXIS, int NC, int PX, int NS>
__device__ __forceinline__ void bwd_view_x2(const ViewP &vp, float pb0, const uint64_t *sm2, int w_row, int lo,
                                            int qoff, uint64_t *t2)
{
    const float E = vp.E, Sn = vp.Sn, ESn = vp.ESn;
    const uint64_t su2 = pk2(vp.su_hi, vp.su_hi), hwu2 = pk2(vp.hwu, vp.hwu), pbb = pk2(pb0, pb0);
    const uint64_t mag2 = pk2(kCeilMagic, kCeilMagic);
#pragma unroll
    for (int h = 0; h < PX / 2; ++h) {
        const uint64_t st = pk2((float)(kBwdRowStep * 2 * h), (float)(kBwdRowStep * (2 * h + 1)));
        const uint64_t pb = fma2_rn(st, su2, pbb);                          // exact
        const uint64_t uc = add2_rp(sub2_rn(sub2_rn(sm2[h], pb), hwu2), mag2);
        float uca, ucb;
        upk2(uc, uca, ucb);
        const int wa = w_row + (magic_int(uca) - lo), wb = w_row + (magic_int(ucb) - lo);
        const uint64_t big0 = add2_rn(sub2_rn(uc, mag2), pb);              // exact, as are big0 + 1, + 2
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const uint64_t bk = k ? add2_rn(big0, pk2((float)k, (float)k)) : big0;
            float da, db;
            upk2(sub2_rn(bk, sm2[h]), da, db);
            const uint64_t w = pk2(weight_unit(fabsf(da), E, Sn, ESn, AXIS), weight_unit(fabsf(db), E, Sn, ESn, AXIS));
#pragma unroll
            for (int s = 0; s < NS; ++s)   // the window holds P * y
                t2[s * PX / 2 + h] =
                    fma2_rn(w, pk2(proj_dyn[wa + s * qoff + k], proj_dyn[wb + s * qoff + k]), t2[s * PX / 2 + h]);
        }
    }
}

// R^T y over one sinogram (mode BWD_G: y = r into g, BWD_H: y = q into h,
// BWD_PLAIN: y = the staged input into g), or, DUAL, over two in one pass:
// g from r and h from q (h = A p for the beta of the next step of Algorithm 2,
// deferred to this pass: alpha takes p^T A p from the forward projector's ||q||^2).
// FIXED_PARTS: the view parts per tile when every problem of the launch has that
// (default) number, so the part arithmetic is compile-time; 0: each problem's own.
template <bool DUAL, int FIXED_PARTS>
__global__ void __launch_bounds__(kBwdThreads, DUAL ? 2 : 3) k_backward(const Prob *__restrict__ probs,
                                                          const int *__restrict__ prefix, int count, int mode)
{
    constexpr int NS = BwdShape<DUAL>::NS, TI = BwdShape<DUAL>::TI, PX = BwdShape<DUAL>::PX;
    // proj_dyn: [2][NS][kBwdViewChunk][bwin] sinogram windows
    __shared__ ViewP vsh[2][kBwdViewChunk];
    __shared__ int ulo_sh[2][kBwdViewChunk];
    __shared__ int kind_sh[2][kBwdViewChunk];   // variant: three bins (1) / two bins (2), + 3 if a window check is needed; axis 3
    __shared__ float2 comb[kBwdGroup * NS * PX];   // second group's sums, combined by the first
    __shared__ __align__(16) double red[40];
    __shared__ int bad_sh;

    int local;
    const int pi = find_problem(prefix, count, blockIdx.x, &local);
    const Prob &P = probs[pi];
    if ((DUAL || mode != BWD_PLAIN) && P.sc->done) return;

    const int bwin = P.bwin;
    const int qoff = kBwdViewChunk * bwin;   // second sinogram's windows after the first's
    const int tiles_j = (P.nx + kBwdTileJ - 1) / kBwdTileJ;
    // part-major: every tile's first part, then its second, ...; the last part has the
    // fewest view chunks, so the grid's final (partial) wave holds the shortest blocks
    const int parts = FIXED_PARTS ? FIXED_PARTS : P.bparts;
    const int ntiles_p = (prefix[pi + 1] - prefix[pi]) / parts;
    const int vpart = local / ntiles_p, tile = local - vpart * ntiles_p;   // this block's part of the views
    const int ti = tile / tiles_j, tj = tile - ti * tiles_j;
    const int i0 = ti * TI, j0 = tj * kBwdTileJ;
    const int t = threadIdx.x;
    const int grp = t / kBwdGroup, tg = t - grp * kBwdGroup;   // group grp takes views vv = grp (mod kBwdSplit)
    const int lx = tg % kBwdTileJ, ly = tg / kBwdTileJ;
    const int j = j0 + lx;
    const float X = __fsub_rn(__int2float_rn(j), P.cx);
    float Y[PX];
#pragma unroll
    for (int e = 0; e < PX; ++e) Y[e] = __fsub_rn(P.cy, __int2float_rn(i0 + ly + kBwdRowStep * e));
    // per pixel: FP32 sum of up to four views (t2, pixels in pairs), folded into a Kahan-compensated
    // pair (part, comp) that runs over all views; FP64 only for the final value (the FP64 pipe is narrow)
    float part[NS * PX], comp[NS * PX];
    uint64_t t2[NS * PX / 2];
#pragma unroll
    for (int e = 0; e < NS * PX; ++e) part[e] = comp[e] = 0.0f;
#pragma unroll
    for (int h = 0; h < NS * PX / 2; ++h) t2[h] = pk2(0.0f, 0.0f);
    uint64_t Y2[PX / 2];
#pragma unroll
    for (int h = 0; h < PX / 2; ++h) Y2[h] = pk2(Y[2 * h], Y[2 * h + 1]);
    const uint64_t X2 = pk2(X, X);

    const float *sino0 = (!DUAL && mode == BWD_H) ? P.q : P.r;
    const float *sino1 = P.q;
    const int Up = P.Up;
    // tile corners in pixel-centre coordinates
    const float Xa = __fsub_rn(__int2float_rn(j0), P.cx), Xb = __fsub_rn(__int2float_rn(j0 + kBwdTileJ - 1), P.cx);
    const float Ya = __fsub_rn(P.cy, __int2float_rn(i0)), Yb = __fsub_rn(P.cy, __int2float_rn(i0 + TI - 1));
    if (t == 0) bad_sh = 0;

    const int nchunks = (P.V + kBwdViewChunk - 1) / kBwdViewChunk;
    // stage chunk c into buffer c&1
    auto stage = [&](int c) {
        const int buf = c & 1;
        const int v0 = c * kBwdViewChunk;
        if (t < kBwdViewChunk) {
            const int v = v0 + t;
            int lo = 0;
            int kind = 0;
            if (v < P.V) {
                const ViewP vp = P.views[v];
                vsh[buf][t] = vp;
                float m = fminf(fminf(det_coord(vp, Xa, Ya), det_coord(vp, Xa, Yb)),
                                fminf(det_coord(vp, Xb, Ya), det_coord(vp, Xb, Yb)));
                lo = (__float2int_rd(__fadd_rn(m, P.uc)) - 3) & ~3;
                // a pixel's first candidate is (up to rounding) linear in X and Y, so its values at
                // the tile's corners, with one bin of slack, bound it for every pixel of the tile;
                // they are computed exactly as each pixel's own
                const int nc = (vp.flags & kViewBwd3) ? 3 : 2;
                bool inside = true;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float Xc = (k & 1) ? Xb : Xa, Yc = (k & 2) ? Yb : Ya;
                    const float pbc = __fmaf_rn(-vp.cu_hi, Xc, __fmaf_rn(-vp.su_hi, Yc, -P.uc_hi));
                    const float smc = delta_small(vp, Xc, Yc, P.uc_lo);
                    const int q = magic_int(ceil_magic(__fsub_rn(__fsub_rn(smc, pbc), vp.hwu))) - lo;
                    inside = inside && q >= 1 && q <= bwin - nc - 1;
                }
                // axis-aligned views (two in a uniform set) always take the checked scalar path
                kind = ((vp.flags & kViewAxis) ? 3 : (nc == 3 ? 1 : 2) + (inside ? 0 : 3));
            }
            ulo_sh[buf][t] = lo;
            kind_sh[buf][t] = kind;
        }
        __syncthreads();
        const int V4 = bwin >> 2;
        float *wb = proj_dyn + buf * NS * qoff;
        for (int e = t; e < NS * kBwdViewChunk * V4; e += kBwdThreads) {
            const int s = (NS == 2 && e >= kBwdViewChunk * V4) ? 1 : 0;
            const int es = e - s * kBwdViewChunk * V4;
            const int vv = es / V4, k4 = es - vv * V4;
            const int v = v0 + vv;
            float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
            const int ub = ulo_sh[buf][vv] + 4 * k4;
            if (v < P.V && ub >= 0 && ub + 3 < Up) {
                val = __ldg(reinterpret_cast<const float4 *>((s ? sino1 : sino0) + (size_t)v * Up + ub));
                const float pl = vsh[buf][vv].P;   // the weights are in units of the view's plateau length
                val.x = __fmul_rn(val.x, pl);
                val.y = __fmul_rn(val.y, pl);
                val.z = __fmul_rn(val.z, pl);
                val.w = __fmul_rn(val.w, pl);
            }
            *reinterpret_cast<float4 *>(wb + s * qoff + vv * bwin + 4 * k4) = val;
        }
    };

    const int per_part = (nchunks + parts - 1) / parts;
    const int c_begin = min(nchunks, vpart * per_part), c_end = min(nchunks, c_begin + per_part);
    if (c_begin < c_end) stage(c_begin);
    __syncthreads();
    int bad = 0;
    for (int c = c_begin; c < c_end; ++c) {
        const int buf = c & 1;
        if (c + 1 < c_end) stage(c + 1);   // other buffer; its previous readers finished at the last barrier
        const int nv = min(kBwdViewChunk, P.V - c * kBwdViewChunk);
        const int wb = buf * NS * qoff;
        // groups of four of this thread group's views, then one Kahan-compensated fold
        for (int g0 = grp; g0 < nv; g0 += 4 * kBwdSplit) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int vv = g0 + q * kBwdSplit;
                if (vv < nv) {
                    const ViewP vp = vsh[buf][vv];
                    const int wr = wb + vv * bwin;
                    const int lo = ulo_sh[buf][vv];
                    const float pb0 = __fmaf_rn(-vp.cu_hi, X, __fmaf_rn(-vp.su_hi, Y[0], -P.uc_hi));
                    // small = uc_lo + cu_lo X + su_lo Y in the view class's order (delta_small), in pairs
                    uint64_t sm2[PX / 2];
                    if (vp.flags & kViewClassB) {
                        const float in = __fmaf_rn(vp.cu_lo, X, P.uc_lo);
                        const uint64_t s2 = pk2(vp.su_lo, vp.su_lo), in2 = pk2(in, in);
#pragma unroll
                        for (int h = 0; h < PX / 2; ++h) sm2[h] = fma2_rn(s2, Y2[h], in2);
                    } else {
                        const uint64_t s2 = pk2(vp.su_lo, vp.su_lo), c2 = pk2(vp.cu_lo, vp.cu_lo),
                                       u2 = pk2(P.uc_lo, P.uc_lo);
#pragma unroll
                        for (int h = 0; h < PX / 2; ++h) sm2[h] = fma2_rn(c2, X2, fma2_rn(s2, Y2[h], u2));
                    }
                    const int kind = kind_sh[buf][vv];
                    if (kind < 3) {
                        if (kind == 1) bwd_view_x2<false, 3, PX, NS>(vp, pb0, sm2, wr, lo, qoff, t2);
                        else bwd_view_x2<false, 2, PX, NS>(vp, pb0, sm2, wr, lo, qoff, t2);
                    } else {   // a window check is needed: the scalar path
                        float sm[PX], t4[NS * PX];
#pragma unroll
                        for (int h = 0; h < PX / 2; ++h) upk2(sm2[h], sm[2 * h], sm[2 * h + 1]);
#pragma unroll
                        for (int h = 0; h < NS * PX / 2; ++h) upk2(t2[h], t4[2 * h], t4[2 * h + 1]);
                        if (kind == 3) bwd_view<true, 2, PX, NS>(vp, pb0, sm, wr, lo, bwin, qoff, t4, &bad);
                        else if (kind == 4) bwd_view<false, 3, PX, NS>(vp, pb0, sm, wr, lo, bwin, qoff, t4, &bad);
                        else bwd_view<false, 2, PX, NS>(vp, pb0, sm, wr, lo, bwin, qoff, t4, &bad);
#pragma unroll
                        for (int h = 0; h < NS * PX / 2; ++h) t2[h] = pk2(t4[2 * h], t4[2 * h + 1]);
                    }
                }
            }
            float t4[NS * PX];
#pragma unroll
            for (int h = 0; h < NS * PX / 2; ++h) {
                upk2(t2[h], t4[2 * h], t4[2 * h + 1]);
                t2[h] = pk2(0.0f, 0.0f);
            }
#pragma unroll
            for (int e = 0; e < NS * PX; ++e) {
                const float y = __fsub_rn(t4[e], comp[e]);
                const float tt = __fadd_rn(part[e], y);
                comp[e] = __fsub_rn(__fsub_rn(tt, part[e]), y);
                part[e] = tt;
            }
        }
        __syncthreads();
    }
    // the Kahan pair as a double-float value part - comp (|comp| <= ulp(part) / 2); the
    // groups' and the parts' sums are added in double-float arithmetic, in a fixed order
    if (bad) atomicExch(&bad_sh, 1);
    __syncthreads();
    if (grp == 1)
#pragma unroll
        for (int e = 0; e < NS * PX; ++e) comb[e * kBwdGroup + tg] = make_float2(part[e], -comp[e]);
    __syncthreads();
    // this part's sums; the tile's last part to finish adds them in part order
    const size_t img = (size_t)P.ny * P.nxp;
    if (grp == 0)
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int e = 0; e < PX; ++e) {
                const int i = i0 + ly + kBwdRowStep * e;
                if (i < P.ny && j < P.nx) {
                    const float2 o2 = comb[(s * PX + e) * kBwdGroup + tg];
                    const df v = df_add(df{part[s * PX + e], -comp[s * PX + e]}, df{o2.x, o2.y});
                    P.bsplit[(size_t)(s * parts + vpart) * img + (size_t)i * P.nxp + j] = make_float2(v.h, v.l);
                }
            }
    if (t == 0 && bad_sh && P.sc) atomicExch(&P.sc->status, (int)SUPCG_ERR_UNSUPPORTED);
    __shared__ int last_sh;
    if (!last_block(&P.tilecnt[tile], parts, &last_sh)) return;
    // output s: the gradient (g from r) or h from q
    const bool is_g[2] = {DUAL || mode != BWD_H, false};
    float *outs[2] = {(!DUAL && mode == BWD_H) ? P.h : P.g, P.h};
    // Bayesian criterion (Eq. (2.3)): g = r^2 R^T r + (x - mu_X), h = r^2 R^T q + p, and
    // ||x - mu_X||^2 for f.  With a reference image, the selective error of Eq. (4.1) of
    // x = x_{k+1/2} over the centred ellipse S (this pass reads x anyway).
    const bool solve = DUAL || mode != BWD_PLAIN;
    const bool bayes = solve && P.r2 > 0.0;
    const bool want_se = (DUAL || mode == BWD_G) && P.se_ref != nullptr && !P.sc->init;
    const double muX = bayes ? P.sc->muX : 0.0;
    double sx = 0.0, sse = 0.0;
    if (grp == 0)
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int e = 0; e < PX; ++e) {
                const int i = i0 + ly + kBwdRowStep * e;
                if (i < P.ny && j < P.nx) {
                    const size_t o = (size_t)i * P.nxp + j;
                    float2 pv[kBwdMaxParts];   // the other blocks' sums: read past L1
#pragma unroll
                    for (int h = 0; h < kBwdMaxParts; ++h)
                        if (h < parts) pv[h] = __ldcg(P.bsplit + (size_t)(s * parts + h) * img + o);
                    df vs = {0.0f, 0.0f};
#pragma unroll
                    for (int h = 0; h < kBwdMaxParts; ++h)
                        if (h < parts) vs = df_add(vs, df{pv[h].x, pv[h].y});
                    if (bayes) {
                        double v = (double)vs.h + (double)vs.l;
                        if (is_g[s]) {
                            const double dx = (double)P.x[o] - muX;
                            v = P.r2 * v + dx;
                            sx += dx * dx;
                        } else {
                            v = P.r2 * v + (double)P.p[o];
                        }
                        const float vh = (float)v;
                        outs[s][o] = vh;
                        if (solve && is_g[s]) P.glo[o] = (float)(v - (double)vh);
                    } else {
                        const float vh = __fadd_rn(vs.h, vs.l);   // the pair rounded to FP32
                        outs[s][o] = vh;
                        if (solve && is_g[s]) P.glo[o] = __fsub_rn(vs.l, __fsub_rn(vh, vs.h));   // its error, exactly
                    }
                    if (want_se && s == 0) {   // pixel centre inside the ellipse (FP64, as the definition)
                        const double ex = ((double)j - 0.5 * (P.nx - 1)) / P.se_ax;
                        const double ey = ((double)i - 0.5 * (P.ny - 1)) / P.se_ay;
                        if (ex * ex + ey * ey <= 1.0) {
                            const double dr = (double)P.x[o] - (double)P.se_ref[(size_t)i * P.nx + j];
                            sse += dr * dr;
                        }
                    }
                }
            }
    if (t == 0) P.tilecnt[tile] = 0;   // ready for the next launch
    if (!(bayes && is_g[0]) && !want_se) return;
    // the tiles' sums, added in tile order by the last tile to finish: f = r^2 ||R x - b||^2 +
    // ||x - mu_X||^2, and SE = sqrt(sum over S)
    const double bs = block_sum<kBwdThreads>(sx, red);
    const double be = block_sum<kBwdThreads>(sse, red);
    const int ntiles = (prefix[pi + 1] - prefix[pi]) / parts;
    if (t == 0) {
        P.partial[tile] = bs;
        P.partial[ntiles + tile] = be;
    }
    if (last_block(&P.counter[4], ntiles, &last_sh)) {
        double tot, tse;
        block_sum_array2<kBwdThreads>(P.partial, P.partial + ntiles, ntiles, red, &tot, &tse);
        if (t == 0) {
            Scal *sc = P.sc;
            if (bayes) {
                sc->f = P.r2 * sc->f_ls + tot;
                if (sc->init) sc->f0 = sc->f;
            }
            if (want_se) P.se_log[sc->k] = sqrt(tse);   // body sc->k + 1 (k counts finished bodies)
            P.counter[4] = 0;
        }
    }
}

// Blocks per problem: `parts` per pixel tile.
int backward_blocks(int nx, int ny, int dual, int parts)
{
    const int ti = dual ? BwdShape<true>::TI : BwdShape<false>::TI;
    return parts * ((ny + ti - 1) / ti) * ((nx + kBwdTileJ - 1) / kBwdTileJ);
}

template <bool DUAL, int FP>
static int launch_bwd(const Launch &L, int mode, int bwin)
{
    const int smem = 2 * (DUAL ? 2 : 1) * kBwdViewChunk * bwin * 4;
    int rc = func_attrs_once((const void *)k_backward<DUAL, FP>, 2 * (DUAL ? 2 : 1) * kBwdViewChunk * 256 * 4);
    if (rc) return rc;
    k_backward<DUAL, FP><<<L.blocks, kBwdThreads, smem, L.st>>>(L.probs, L.prefix, L.count, mode);
    SUPCG_CUDA_TRY(cudaGetLastError());
    return SUPCG_OK;
}

int launch_backward(const Launch &L, int mode, int bwin)
{
    return L.bparts == kBwdViewParts ? launch_bwd<false, kBwdViewParts>(L, mode, bwin)
                                     : launch_bwd<false, 0>(L, mode, bwin);
}

int launch_backward2(const Launch &L, int bwin)
{
    return L.bparts == kBwdViewParts ? launch_bwd<true, kBwdViewParts>(L, BWD_G, bwin)
                                     : launch_bwd<true, 0>(L, BWD_G, bwin);
}

} // namespace supcg
