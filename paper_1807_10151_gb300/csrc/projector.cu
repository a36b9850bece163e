// Forward projection R x (Sec. 2: R x = b + e); its exact transpose R^T y is
// in backprojector.cu.
//
// Forward (ray-driven, gather over pixels).  A warp owns one view and up to 64
// consecutive bins (a warp item), two rays per lane.  The host sorts the warp
// items longest first by the rows their rays can meet, weighted by the cost of
// a row in the item's view, and block b runs items 2b and 2b + 1: a block's
// warps finish together and the grid ends on short items.  Views are split in
// two classes:
// class A (|cos| >= |sin|) walks image rows, class B walks image columns, and
// class B reads the transposed image x^T so that both classes walk contiguous
// rows of the array they read.  Each warp stages chunks of kRowsPerChunk rows
// x BW columns covering its 64 rays in shared memory by 2-D TMA loads (its own
// kFwdBufs boxes, one mbarrier each), and only the rows its rays can meet.
// For every row a ray can only cross the two (three near the diagonal)
// columns nearest to its centre; each is weighted by the shared trapezoid.
#include "internal.cuh"

namespace supcg {

// The kernels' dynamic shared memory, indexed by 32-bit float offsets so that
// operand loads are plain shared-memory loads with 32-bit addresses.
extern __shared__ __align__(128) float proj_dyn[];

static_assert(kRowsPerChunk % 8 == 0, "chunks start at multiples of the fold groups");

constexpr int kFwdBufs = 1;   // forward projector: staged boxes per warp (1: more resident warps hide the copies)

// ============================================================ forward
// Inner loop over the rows [o0, o0 + rows) of one staged box.  A ray meets a
// row in the inner indices within hwq (half-width + margin) of its centre:
// two of them, or three for views within about a degree of the diagonal
// (NC = 3).  Each is weighted by weight(delta) with delta from the exact
// split.  The terms of a group of G rows are summed in FP32 and added to the
// ray's running sum with Kahan compensation (sum, comp), so that the ray sum
// is accurate to about one unit in the last place of FP32 however many rows
// it crosses (groups of G = 8 rows).
// MIR: the staged box is followed (moff floats later) by the same box of the
// left-right mirrored image; each weight is also applied there, giving the ray
// of the same bin in the mirror view (msum, mcomp: its compensated sum).
template <bool CLASS_B, bool AXIS, int NC, bool CHECKED, bool MIR>
__device__ __forceinline__ void fwd_rows(const Prob &P, const ViewP &vp, float tau_hi, float qm, int o0, int rb,
                                         int re, int qs, int pbase, int moff, int *bad,
                                         float &sum, float &comp, float &msum, float &mcomp)
{
    const int BW = P.BW;
    // outer coordinate of row o0 + rb (pixel units) and its change per row
    float Oc = CLASS_B ? __fsub_rn(__int2float_rn(o0 + rb), P.cx) : __fsub_rn(P.cy, __int2float_rn(o0 + rb));
    const float dO = CLASS_B ? 1.0f : -1.0f;
    const float hi_o = CLASS_B ? vp.cu_hi : vp.su_hi;   // coefficient of the outer coordinate
    const float lo_o = CLASS_B ? vp.cu_lo : vp.su_lo;
    const float hi_i = CLASS_B ? vp.su_hi : vp.cu_hi;   // coefficient of the inner coordinate
    const float lo_i = CLASS_B ? vp.su_lo : vp.cu_lo;
    // inner coordinate of inner index q: X = q - cx (class A) or Y = cy - q (class B)
    const float c_in = CLASS_B ? P.cy : P.cx;
    const float dI = CLASS_B ? -1.0f : 1.0f;
    const float E = vp.E, Sn = vp.Sn, ESn = vp.ESn;
    const float qh = __fsub_rn(qm, vp.hwq);
    const int prow = pbase - qs;   // proj_dyn index of inner index 0 of the box's first row
    float rs = 0.0f;   // FP32 sum of the rows of one 8-row group, then folded into (sum, comp)
    float ms = 0.0f;   // the same for the mirror view
    auto row = [&](int r, float rf) {
        const float qc = ceil_magic(__fmaf_rn(rf, vp.b_o, qh));
        int q0 = magic_int(qc);
        if (CHECKED) {
            const int idx = q0 - qs;
            if (idx < 0 || idx > BW - NC) {   // outside the staged box: never for a valid box (host-checked)
                *bad = 1;
                q0 = min(max(idx, 0), BW - NC) + qs;
            }
        }
        const float *pv = proj_dyn + (prow + r * BW + q0);
        const float rbig = __fmaf_rn(-hi_o, Oc, tau_hi);            // exact
        const float rsmall = __fmaf_rn(lo_o, Oc, P.uc_lo);
        Oc = __fadd_rn(Oc, dO);
        const float q0f = CHECKED ? __int2float_rn(q0) : magic_float(qc);   // the clamped index when checked
        const float I0 = CLASS_B ? __fsub_rn(c_in, q0f) : __fsub_rn(q0f, c_in);
        float I = I0;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            if (k) I = __fadd_rn(I, dI);                                // exact half-integer
            const float big = __fmaf_rn(-hi_i, I, rbig);              // exact
            const float ad = fabsf(__fsub_rn(big, __fmaf_rn(lo_i, I, rsmall)));
            const float w = weight_unit(ad, E, Sn, ESn, AXIS);
            rs = __fmaf_rn(w, pv[k], rs);
            if (MIR) ms = __fmaf_rn(w, pv[k + moff], ms);
        }
    };
    // Kahan-compensated fold of a group's sum; a group that summed to exactly 0 is
    // skipped, so rows that only met the zero fill leave the ray's sum untouched
    auto fold = [&]() {
        if (rs != 0.0f) {
            const float y = __fsub_rn(rs, comp);
            const float tt = __fadd_rn(sum, y);
            comp = __fsub_rn(__fsub_rn(tt, sum), y);
            sum = tt;
        }
        rs = 0.0f;
        if (MIR) {
            if (ms != 0.0f) {
                const float y = __fsub_rn(ms, mcomp);
                const float tt = __fadd_rn(msum, y);
                mcomp = __fsub_rn(__fsub_rn(tt, msum), y);
                msum = tt;
            }
            ms = 0.0f;
        }
    };
    // groups of G rows aligned to multiples of G of the outer index (o0 is one), so
    // that a ray's sum does not depend on the rows its warp walks beyond its own
    constexpr int G = 8;
    int r = rb;
    float rf = __int2float_rn(rb);
    while (r < re) {
        const int gend = min(re, (r & ~(G - 1)) + G);
        if (gend - r == G) {
#pragma unroll
            for (int k = 0; k < G; ++k, rf = __fadd_rn(rf, 1.0f)) row(r + k, rf);
        } else {
            for (int q = r; q < gend; ++q, rf = __fadd_rn(rf, 1.0f)) row(q, rf);
        }
        fold();
        r = gend;
    }
}

// Two rays per lane (A, B), every per-ray FP32 step as one f32x2 instruction
// for both: the candidate index, the exact-split coordinates and each
// candidate's weight (lane for lane the scalar IEEE steps of fwd_rows, so
// the weights are the same bits).  Only for boxes that hold every candidate.
template <bool CLASS_B, bool AXIS, int NC, bool MIR>
__device__ __forceinline__ void fwd_rows2(const Prob &P, const ViewP &vp, uint64_t tau2, uint64_t qm2, int o0, int rb,
                                          int re, int qs, int pbase, int moff, const float4 *rtab,
                                          float *sum, float *comp, float *msum, float *mcomp)
{
    const int BW = P.BW;
    const float hi_i = CLASS_B ? vp.su_hi : vp.cu_hi;   // coefficient of the inner coordinate
    const float lo_i = CLASS_B ? vp.su_lo : vp.cu_lo;
    const float c_in = CLASS_B ? P.cy : P.cx;           // inner coordinate = q - cx (A) or cy - q (B)
    const float dI = CLASS_B ? -1.0f : 1.0f;
    const float E = vp.E, Sn = vp.Sn, ESn = vp.ESn;
    const uint64_t hii2 = pk2(-hi_i, -hi_i), loi2 = pk2(lo_i, lo_i), cin2 = pk2(c_in, c_in), dI2 = pk2(dI, dI);
    const uint64_t bo2 = pk2(vp.b_o, vp.b_o), mag2 = pk2(kCeilMagic, kCeilMagic);
    const uint64_t qh2 = sub2_rn(qm2, pk2(vp.hwq, vp.hwq));
    const int prow = pbase - qs;   // proj_dyn index of inner index 0 of the box's first row
    uint64_t acc2 = pk2(0.0f, 0.0f);   // FP32 sums of up to 8 rows of A and B, then folded
    uint64_t macc2 = pk2(0.0f, 0.0f);  // the same for the mirror view
    auto row = [&](int r, uint64_t qp2) {
        const uint64_t qc2 = add2_rp(qp2, mag2);   // first candidates, as magic floats
        float qcA, qcB;
        upk2(qc2, qcA, qcB);
        const int rowi = prow + r * BW;
        const int pA = rowi + magic_int(qcA), pB = rowi + magic_int(qcB);
        const float4 rt = rtab[r];                                   // the row's terms (fwd_row_terms)
        const uint64_t rbig2 = add2_rn(tau2, pk2(rt.x, rt.y));       // exact
        const uint64_t rsmall2 = pk2(rt.z, rt.w);
        const uint64_t q0f2 = sub2_rn(qc2, mag2);
        uint64_t I2 = CLASS_B ? sub2_rn(cin2, q0f2) : sub2_rn(q0f2, cin2);   // exact half-integers
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            if (k) I2 = add2_rn(I2, dI2);
            const uint64_t big2 = fma2_rn(hii2, I2, rbig2);          // exact
            float dA, dB;
            upk2(sub2_rn(big2, fma2_rn(loi2, I2, rsmall2)), dA, dB);
            const uint64_t w2 = pk2(weight_unit(fabsf(dA), E, Sn, ESn, AXIS), weight_unit(fabsf(dB), E, Sn, ESn, AXIS));
            acc2 = fma2_rn(w2, pk2(proj_dyn[pA + k], proj_dyn[pB + k]), acc2);
            if (MIR) macc2 = fma2_rn(w2, pk2(proj_dyn[pA + k + moff], proj_dyn[pB + k + moff]), macc2);
        }
    };
    auto fold = [&]() {   // Kahan-compensated folds of the group's sums, as in fwd_rows
        float g[2];
        upk2(acc2, g[0], g[1]);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (g[q] != 0.0f) {
                const float y = __fsub_rn(g[q], comp[q]);
                const float tt = __fadd_rn(sum[q], y);
                comp[q] = __fsub_rn(__fsub_rn(tt, sum[q]), y);
                sum[q] = tt;
            }
        }
        acc2 = pk2(0.0f, 0.0f);
        if (MIR) {
            upk2(macc2, g[0], g[1]);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (g[q] != 0.0f) {
                    const float y = __fsub_rn(g[q], mcomp[q]);
                    const float tt = __fadd_rn(msum[q], y);
                    mcomp[q] = __fsub_rn(__fsub_rn(tt, msum[q]), y);
                    msum[q] = tt;
                }
            }
            macc2 = pk2(0.0f, 0.0f);
        }
    };
    constexpr int G = 8;   // rows per fold group, as in fwd_rows
    int r = rb;
    while (r < re) {   // groups aligned to multiples of G of the outer index, as in fwd_rows
        const int gend = min(re, (r & ~(G - 1)) + G);
        // the candidates' window start (centre - hwq) of row r, then stepped by b_o per row: it only
        // chooses the candidates (the weights decide), and eight steps stay ~1e-4 pixels from the
        // direct value, far inside the window's margin
        const float rf = __int2float_rn(r);
        uint64_t qp2 = fma2_rn(pk2(rf, rf), bo2, qh2);
        if (gend - r == G) {
#pragma unroll
            for (int k = 0; k < G; ++k, qp2 = add2_rn(qp2, bo2)) row(r + k, qp2);
        } else {
            for (int q = r; q < gend; ++q, qp2 = add2_rn(qp2, bo2)) row(q, qp2);
        }
        fold();
        r = gend;
    }
}

// The outer coordinate's terms of the exact split for the rows of chunk [o0, o0 + RC),
// the same for every ray of the view: rtab[r] = (H, H, s, s) with H = -hi_o O (exact)
// and s = lo_o O + uc_lo (rounded once), O the outer coordinate of row o0 + r, so that
// a ray's row needs big = tau_hi + H (exact, the value of fma(-hi_o, O, tau_hi)) and s.
// Written by lanes 0 .. RC-1 of the warp that reads it.
template <bool CLASS_B, int RC>
__device__ __forceinline__ void fwd_row_terms(const Prob &P, const ViewP &vp, int o0, int lane, float4 *rtab)
{
    if (lane < RC) {
        const float O = CLASS_B ? __fsub_rn(__int2float_rn(o0 + lane), P.cx) : __fsub_rn(P.cy, __int2float_rn(o0 + lane));
        const float H = __fmul_rn(CLASS_B ? -vp.cu_hi : -vp.su_hi, O);
        const float sm = __fmaf_rn(CLASS_B ? vp.cu_lo : vp.su_lo, O, P.uc_lo);
        rtab[lane] = make_float4(H, H, sm, sm);
    }
    __syncwarp();
}

// Lower end (multiple of 4) of the inner range that chunk [o0, o0+RC) of the
// block's rays [u_first, u_last] can touch.
template <int RC>
__device__ __forceinline__ int fwd_box_start(const ViewP &vp, float tf, float tl, int o0)
{
    const float bf = __fmaf_rn(vp.a_tau, tf, vp.g0);
    const float bl = __fmaf_rn(vp.a_tau, tl, vp.g0);
    const float o_a = __int2float_rn(o0), o_b = __int2float_rn(o0 + RC - 1);
    float m = fminf(fminf(__fmaf_rn(vp.b_o, o_a, bf), __fmaf_rn(vp.b_o, o_b, bf)),
                    fminf(__fmaf_rn(vp.b_o, o_a, bl), __fmaf_rn(vp.b_o, o_b, bl)));
    int lo = __float2int_rd(m) - 3;
    return lo & ~3;   // round down to a multiple of 4 floats (16-byte TMA rule)
}

// Two rays per lane (u and u + 32: 64 consecutive bins per warp); each warp
// runs its own pipeline of kFwdBufs kRowsPerChunk-row boxes (BW columns
// covering its 64 rays), so warps never wait for one another.  The warp walks
// only the chunks holding rows that one of its rays can meet, and within them
// only those rows.  Rays past the block's last bin follow the last ray (inside
// the box) and are dropped by the caller.
// MIR: each chunk also stages the same box of the mirrored image (tm_m) right after the
// image's, and acc_m receives the sums of the same bins in the mirror view.
template <bool CLASS_B, bool AXIS, int NC, bool MIR>
__device__ __forceinline__ void fwd_ray2(const Prob &P, const ViewP &vp, const CUtensorMap *tm, const CUtensorMap *tm_m,
                                         int patch0, uint64_t *bars, float4 *rtab, int n_outer, int n_inner, int uA,
                                         int uB, int u_last, float tf, float tl, int *bad, int *timed_out, double *acc,
                                         double *acc_m)
{
    constexpr int RC = kRowsPerChunk;
    const int BW = P.BW;
    const int box_elems = RC * BW;
    // one staged chunk: the image's box, then the mirror's
    const int buf_elems = (MIR ? 2 : 1) * box_elems;
    const int moff = box_elems;
    const int lane = threadIdx.x & 31;
    const int uc[2] = {min(uA, u_last), min(uB, u_last)};
    float tau_hi[2], base[2], sum[2] = {0.0f, 0.0f}, comp[2] = {0.0f, 0.0f};
    float msum[2] = {0.0f, 0.0f}, mcomp[2] = {0.0f, 0.0f};
    // the chunk's boxes, in their order in the buffer
    auto issue = [&](int slot, int qs, int c) {
        float *dst = proj_dyn + patch0 + slot * buf_elems;
        mbar_expect_tx(&bars[slot], buf_elems * 4);
        tma_load_2d(dst, tm, qs, c * RC, &bars[slot]);
        if (MIR) tma_load_2d(dst + moff, tm_m, qs, c * RC, &bars[slot]);
    };
    int r_lo = n_outer, r_hi = -1;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        tau_hi[q] = bin_pos(uc[q], P.uc_hi);                            // exact
        base[q] = __fmaf_rn(vp.a_tau, bin_pos(uc[q], P.uc), vp.g0);     // ray centre at outer index 0
        int lo, hi;
        fwd_row_range(vp, base[q], n_inner, n_outer, &lo, &hi);
        if ((q ? uB : uA) <= u_last) {
            r_lo = min(r_lo, lo);
            r_hi = max(r_hi, hi);
        }
    }
    const uint64_t tau2 = pk2(tau_hi[0], tau_hi[1]);
    const int w_lo = __reduce_min_sync(0xffffffffu, r_lo), w_hi = __reduce_max_sync(0xffffffffu, r_hi);
    const int c_first = w_hi >= w_lo ? w_lo / RC : 0;
    const int nch = w_hi >= w_lo ? w_hi / RC - c_first + 1 : 0;   // chunks with at least one of the warp's rows
    // each box's first inner index, computed once (every lane: the copy and the rows use it)
    int qs_buf[kFwdBufs];
#pragma unroll
    for (int ci = 0; ci < kFwdBufs; ++ci) qs_buf[ci] = fwd_box_start<RC>(vp, tf, tl, (c_first + ci) * RC);
    if (lane == 0) {
        for (int ci = 0; ci < kFwdBufs && ci < nch; ++ci) issue(ci, qs_buf[ci], c_first + ci);
    }
    for (int ci = 0; ci < nch; ++ci) {
        const int buf = ci % kFwdBufs, c = c_first + ci;
        const bool ok = mbar_wait(&bars[buf], (ci / kFwdBufs) & 1);
        const int o0 = c * RC;
        fwd_row_terms<CLASS_B, RC>(P, vp, o0, lane, rtab);
        const int rows = min(RC, n_outer - o0);
        const int rb = max(0, w_lo - o0), re = min(rows, w_hi - o0 + 1);
        if (ok && rb < re) {
            const int qs = qs_buf[buf];
            float qm[2];
            bool inside = true;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                qm[q] = __fmaf_rn(vp.b_o, __int2float_rn(o0), base[q]);   // ray centre at row o0
                // the first candidate is monotone in the row: its end values (with one index
                // of slack for rounding) bound every row of the chunk
                const float qh = __fsub_rn(qm[q], vp.hwq);
                const int qa = __float2int_ru(qh) - qs;
                const int qb = __float2int_ru(__fmaf_rn((float)(rows - 1), vp.b_o, qh)) - qs;
                inside = inside && min(qa, qb) >= 1 && max(qa, qb) <= BW - NC - 1;
            }
            const int pb = patch0 + buf * buf_elems;
            // axis-aligned views too: every ray of theirs crosses every row, so that on the
            // scalar path their items were the longest of a pass (108-118 us against a mean
            // of 47 us at 512^2 / 720 views) and set its length
            if (inside) {
                fwd_rows2<CLASS_B, AXIS, NC, MIR>(P, vp, tau2, pk2(qm[0], qm[1]), o0, rb, re, qs, pb, moff, rtab, sum,
                                                  comp, msum, mcomp);
            } else {
#pragma unroll
                for (int q = 0; q < 2; ++q)
                    fwd_rows<CLASS_B, AXIS, NC, true, MIR>(P, vp, tau_hi[q], qm[q], o0, rb, re, qs, pb, moff, bad, sum[q],
                                                           comp[q], msum[q], mcomp[q]);
            }
        }
        // every lane is done with this buffer; a timeout in any lane ends the warp's loop
        if (__any_sync(0xffffffffu, !ok)) {
            *timed_out = 1;
            if (lane == 0) {   // bounded waits for the copies still in flight: chunk ci's and, if issued, ci + 1's
                for (int cj = ci; cj < ci + kFwdBufs && cj < nch; ++cj)   // this chunk and those issued after it
                    (void)mbar_wait(&bars[cj % kFwdBufs], (cj / kFwdBufs) & 1);
            }
            break;
        }
        __syncwarp();
        if (ci + kFwdBufs < nch) {
            qs_buf[buf] = fwd_box_start<RC>(vp, tf, tl, (c + kFwdBufs) * RC);
            if (lane == 0) issue(buf, qs_buf[buf], c + kFwdBufs);
        }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {   // weights in units of P
        acc[q] = ((double)sum[q] - (double)comp[q]) * (double)vp.P;
        if (MIR) acc_m[q] = ((double)msum[q] - (double)mcomp[q]) * (double)vp.P;
    }
}

constexpr int kFwdThreads = 64;   // two warps of 64 rays: 128 bins per block at most

// MIRK: some problem of the launch has mirror pairs of views.  An item of a pair's first
// view then also sums the second view's rays from the mirrored image's boxes (two boxes
// per chunk, so fewer blocks fit: this variant is compiled for 7 resident blocks, the
// other for 10).  which: the image projected (0 = x, 1 = p, 2 = d); mode: FwdMode.
template <bool MIRK>
__global__ void __launch_bounds__(kFwdThreads, MIRK ? 7 : 10) k_forward(const Prob *__restrict__ probs,
                                                                        const int *__restrict__ prefix, int count,
                                                                        int which, int mode)
{
    // proj_dyn: [warp][kFwdBufs][box: the image, (MIRK) its mirror][kRowsPerChunk][BW]
    __shared__ __align__(8) uint64_t bars[kFwdBufs * (kFwdThreads / 32)];   // one per staged box
    __shared__ float4 rowtab[kFwdThreads / 32][kRowsPerChunk];             // each warp's row terms
    __shared__ __align__(16) double red[40];
    __shared__ int flag;
    __shared__ int bad_sh;

    int local;
    const int pi = find_problem(prefix, count, blockIdx.x, &local);
    const Prob &P = probs[pi];
    if (mode != FWD_PLAIN && P.sc->done) return;

    // the warp's item (longest first; the block's two are of about the same length): the
    // first 64 bins of a (view, bin tile) or the rest of the tile
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int wi = 2 * local + warp;
    // the paired kernel walks the item list without the mirror pairs' second views
    const int nfw = MIRK ? P.nfw : P.nfw_all;
    const bool idle = wi >= nfw;   // the grid's last block may hold one item
    const int item = idle ? 0 : (MIRK ? P.border : P.border_all)[wi];
    const int half = item & 1, tv = item >> 1;
    const int vidx = tv / P.ntu, tile = tv - vidx * P.ntu;
    const bool classB = vidx >= P.nA;
    const int v = P.vlist[vidx];
    const int vm = (MIRK && P.mirror && !idle) ? P.mirror[v] : -1;   // the mirror view, or -1
    const ViewP vp = P.views[v];
    const bool axis = (vp.flags & kViewAxis) != 0;
    const int n_outer = classB ? P.nx : P.ny, n_inner = classB ? P.ny : P.nx;
    const int cb = classB ? 1 : 0;
    const CUtensorMap *tm = &P.tm[which * 2 + cb];
    const CUtensorMap *tm_m = &P.tm[6 + which * 2 + cb];
    // this warp's boxes in proj_dyn
    const int patch0 = warp * kFwdBufs * (MIRK ? 2 : 1) * kRowsPerChunk * P.BW;
    uint64_t *wbars = bars + kFwdBufs * warp;

    const int u_first = tile * P.BU;
    const int u_last = min(P.U, u_first + P.BU) - 1;
    // the warp's rays: uw0 .. uw0 + 63, lane l takes uw0 + l and uw0 + 32 + l
    const int uw0 = u_first + 64 * half, uw1 = min(u_last, uw0 + 63);
    const int uA = uw0 + lane, uB = uw0 + 32 + lane;
    const float tf = bin_pos(min(uw0, u_last), P.uc), tl = bin_pos(uw1, P.uc);

    if (t == 0) bad_sh = 0;
    if (t < kFwdBufs * (kFwdThreads / 32)) mbar_init(&bars[t], 1);
    if (t == 0) fence_mbar_init();
    __syncthreads();

    int bad = 0;
    int timed_out = 0;   // a copy did not arrive (every lane of the warp sees it)
    double acc[2] = {0.0, 0.0}, acc_m[2] = {0.0, 0.0};
    // axis-aligned views meet at most two pixels per row; near-diagonal ones up to three
    const bool three = (vp.flags & kViewFwd3) != 0;
#define SUPCG_FWD(CB, AX, NC, MIR) \
    fwd_ray2<CB, AX, NC, MIR>(P, vp, tm, tm_m, patch0, wbars, rowtab[warp], n_outer, n_inner, uA, uB, u_last, tf, tl, \
                              &bad, &timed_out, acc, acc_m)
    if (idle) {
        // no item for this warp
    } else if (MIRK && vm >= 0) {   // a pair (never axis-aligned: those have no mirror partner)
        if (classB) {
            if (three) SUPCG_FWD(true, false, 3, true); else SUPCG_FWD(true, false, 2, true);
        } else {
            if (three) SUPCG_FWD(false, false, 3, true); else SUPCG_FWD(false, false, 2, true);
        }
    } else if (classB) {
        if (axis) SUPCG_FWD(true, true, 2, false); else if (three) SUPCG_FWD(true, false, 3, false); else SUPCG_FWD(true, false, 2, false);
    } else {
        if (axis) SUPCG_FWD(false, true, 2, false); else if (three) SUPCG_FWD(false, false, 3, false); else SUPCG_FWD(false, false, 2, false);
    }
#undef SUPCG_FWD
    if (__syncthreads_or(timed_out)) {   // a warp's copy did not arrive: the whole block leaves
        if (t == 0 && P.sc) atomicExch(&P.sc->status, (int)SUPCG_ERR_TIMEOUT);
        return;
    }
    if (bad) atomicExch(&bad_sh, 1);

    // epilogue: store, fused residual / norm reduction (exact squares, double-float sums)
    df s = df_make(0.0f);
    const double al = (mode == FWD_RUPD) ? P.sc->alpha : 0.0;   // alpha of the step x just took
    // the item's view, then (a mirror pair) the partner view: the same bins, sums acc_m
    auto emit = [&](int view, double a, int u) {
        if (mode == FWD_PLAIN) {
            const size_t o = (size_t)view * P.U + u;
            if (P.storage == SUPCG_BF16) reinterpret_cast<__nv_bfloat16 *>(P.out_user)[o] = __double2bfloat16(a);
            else reinterpret_cast<float *>(P.out_user)[o] = (float)a;
        } else if (mode == FWD_NORM) {
            const size_t o = (size_t)view * P.Up + u;
            const float qq = (float)a;
            P.q[o] = qq;
            P.qd[o] = a;
            df_acc_prod(s, qq, qq);
        } else {
            // FWD_RESID: r = R x - b, the cancellation taken in FP64; FWD_RUPD: x moved by
            // alpha p (step 7) and then by d (S_TV), so r moves by alpha q + R d
            const size_t o = (size_t)view * P.Up + u;
            const double rn = (mode == FWD_RESID) ? a - (double)P.bpad[o] : fma(al, P.qd[o], P.rd[o]) + a;
            const float rr = (float)rn;
            P.rd[o] = rn;
            P.r[o] = rr;
            df_acc_prod(s, rr, rr);
        }
    };
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int u = q ? uB : uA;
        if (idle || u > uw1) continue;
        emit(v, acc[q], u);
        if (MIRK && vm >= 0) emit(vm, acc_m[q], u);
    }
    __syncthreads();
    if (t == 0 && bad_sh && P.sc) atomicExch(&P.sc->status, (int)SUPCG_ERR_UNSUPPORTED);
    if (mode == FWD_PLAIN) return;

    const double bs = block_sum_df<kFwdThreads>(s, red);
    if (t == 0) P.partial[local] = bs;
    const int nblk = prefix[pi + 1] - prefix[pi];
    if (last_block(&P.counter[0], nblk, &flag)) {
        const double tot = block_sum_array<kFwdThreads>(P.partial, nblk, red);
        if (t == 0) {
            Scal *sc = P.sc;
            if (mode != FWD_NORM) {
                if (P.r2 > 0.0) {
                    sc->f_ls = tot;   // f = r^2 ||r||^2 + ||x - mu_X||^2 is completed by the backprojector
                } else {
                    sc->f = tot;
                    if (sc->init) sc->f0 = tot;
                }
            } else {
                const double pth = (P.r2 > 0.0) ? P.r2 * tot + sc->pp : tot;   // p^T h, h = A p
                sc->pth = pth;
                const double al = -sc->gtp / pth;
                if (!(pth > 0.0) || !isfinite(al)) {
                    atomicExch(&sc->status, (int)SUPCG_ERR_BREAKDOWN);
                    sc->alpha = 0.0;
                    sc->alpha_h = sc->alpha_l = 0.0f;
                } else {
                    sc->alpha = al;
                    sc->alpha_h = (float)al;
                    sc->alpha_l = (float)(al - (double)sc->alpha_h);
                }
                // the end of the pass: after steps 1-9 of Algorithm 3 the loop begins; after a
                // while-body, unless an error stopped it, its log entry and k <- k + 1 (step 14)
                if (sc->init) {
                    sc->init = 0;
                } else if (sc->status != 0) {
                    sc->done = 1;
                } else {
                    if (P.log) {
                        double *Lg = P.log + (size_t)sc->k * SUPCG_LOG_STRIDE;
                        Lg[0] = sc->f;
                        Lg[1] = sc->tv_k;
                        Lg[2] = sc->tv_half;
                        Lg[3] = (double)sc->ell;
                        Lg[4] = sc->alpha;
                        Lg[5] = sc->beta;
                        Lg[6] = sc->snorm2;
                        Lg[7] = (double)sc->trials;
                    }
                    sc->k += 1;
                }
            }
            P.counter[0] = 0;
        }
    }
}

template <bool MIRK>
static int launch_forward_t(const Launch &L, int which, int mode)
{
    // every problem's BW <= 256, so the warps' box buffers never exceed this size; with mirror
    // pairs each chunk holds two boxes
    constexpr int rows = (MIRK ? 2 : 1) * kRowsPerChunk;
    const int per_warp = kFwdBufs * rows;
    const int smem = (kFwdThreads / 32) * per_warp * L.bw_max * 4;
    int rc = func_attrs_once((const void *)k_forward<MIRK>, (kFwdThreads / 32) * per_warp * 256 * 4);
    if (rc) return rc;
    k_forward<MIRK><<<L.blocks, kFwdThreads, smem, L.st>>>(L.probs, L.prefix, L.count, which, mode);
    SUPCG_CUDA_TRY(cudaGetLastError());
    return SUPCG_OK;
}

int launch_forward(const Launch &L, const Launch &La, int which, int mode)
{
    return L.mirror ? launch_forward_t<true>(L, which, mode) : launch_forward_t<false>(La, which, mode);
}

} // namespace supcg
