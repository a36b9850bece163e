// Internal definitions shared by the libsupcg translation units.
//
// Everything here is GPU-path code; none of it is shared with the CPU oracle.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/supcg.h"

namespace supcg {

// ----------------------------------------------------------------- limits
constexpr int kMaxStages = 24;       // FFT stages (radices) per length
constexpr int kMaxRadix = 64;        // largest prime factor handled by the generic butterfly
constexpr int kRowsPerChunk = 16;    // forward projector: image rows staged per TMA box
constexpr int kBwdTileI = 32;        // backprojector pixel tile (rows)
constexpr int kBwdViewParts = 4;     // backprojector: default blocks per tile (view parts), each a share of the view chunks
constexpr int kBwdMaxParts = 8;      // backprojector: most view parts per tile (supcg_set_bwd_parts)
constexpr int kBwdTileJ = 32;        // backprojector pixel tile (columns)
constexpr int kBwdViewChunk = 32;    // backprojector: views staged per shared-memory chunk
constexpr int kRedThreads = 256;     // block size of the reduction / vector kernels
constexpr int kFftSmemTw = 1024;     // preconditioner: twiddle tables up to this length are staged per block
                                     // (longer ones are read through L1: a 2048-point block then needs 64 KB
                                     // instead of 96 KB, and three blocks fit on an SM instead of two)
constexpr long long kSpinLimit = 1ll << 24;  // bounded waits (iterations of a ~100 ns poll); grid barriers: the
                                             // default of supcg_set_wait_limit

// ----------------------------------------------------------------- views
// Per-view constants.  Detector coordinates are in bins.  Pixel (i, j) has
// centre X_j = j - (nx-1)/2, Y_i = (ny-1)/2 - i (pixel units) and ray (v, u)
// sits at signed distance
//   delta = u - uc - cu X_j - su Y_i            (cu = cos d/ds, su = sin d/ds)
// from it.  delta is evaluated as big - small with cu = cu_hi + cu_lo,
// su = su_hi + su_lo, uc = uc_hi + uc_lo, where the _hi parts are multiples
// of 2^-(Q-1) chosen per geometry so that every partial sum of
//   big = u - uc_hi - cu_hi X - su_hi Y
// is a multiple of 2^-Q below 2^(24-Q) in magnitude: big is exact in FP32 in
// any order of evaluation, and only `small` (|small| << 1) and the final
// subtraction round.  Both projector kernels evaluate small in the same order
// (fixed per view class), so they produce identical bits for every
// (ray, pixel) pair: the backprojector applies the exact transpose of the
// forward matrix.  The length is then the trapezoid weight(delta).
struct __align__(16) ViewP {
    float cu, su;   // cos(theta) d/ds, sin(theta) d/ds (approximate uses: candidate centres, boxes)
    float E;        // footprint half-width in bins: (d/ds) (|cos|+|sin|) / 2
    float Sn;       // S / P, S = ds / (|cos| |sin|) the length per bin on the trapezoid's sides
    float P;        // plateau length d / max(|cos|, |sin|)
    float a_tau;    // forward: inner index of the ray centre = a_tau*tau + b_o*outer + g0
    float b_o;
    float g0;
    float cu_hi, su_hi, cu_lo, su_lo;
    int flags;      // kView* bits
    float ESn;      // E * S / P (rounded once): the trapezoid is P * sat(fmaf(-|delta|, Sn, ESn))
    float hwq;      // forward: half-width of a ray's footprint in inner-index units, plus a 0.02 margin
    float hwu;      // backward: half-width of a pixel's footprint in bins, plus a 0.02 margin
};
constexpr int kViewAxis = 1;     // cos or sin exactly 0: box footprint
constexpr int kViewClassB = 2;   // |sin| > |cos|: the forward projector walks columns (reads x^T)
constexpr int kViewFwd3 = 4;     // a ray can meet three pixels of a row within the margin
constexpr int kViewBwd3 = 8;     // a pixel can meet three bins within the margin

// Intersection length for a ray at signed detector distance `delta` (bins)
// from the pixel centre, in units of the view's plateau length P: axis-aligned
// views use the box limit (1 inside, 1/2 exactly on the edge, 0 outside), the
// others the trapezoid clamped to [0, 1] by one saturating FMA.  Both
// projectors evaluate it from the same FP32 operands with pinned rounding, so
// they produce identical bits; the factor P is applied once per ray (forward)
// or to the staged sinogram values (backward).
__device__ __forceinline__ float weight_unit(float ad, float E, float Sn, float ESn, bool axis)
{
    if (axis) return ad < E ? 1.0f : (ad == E ? 0.5f : 0.0f);
    float w;
    asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(w) : "f"(-ad), "f"(Sn), "f"(ESn));
    return w;
}

// Packed pairs of FP32 values (f32x2: one instruction, two IEEE operations with
// the stated rounding, lane by lane identical to the scalar operation).
__device__ __forceinline__ uint64_t pk2(float a, float b)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(uint64_t p, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(p)); }
__device__ __forceinline__ uint64_t add2_rn(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t add2_rp(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("add.rp.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t sub2_rn(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t fma2_rn(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// ceil(x) for |x| < 2^22 by one FP32 addition rounded upward: x + 1.5 * 2^23
// lies where FP32 numbers are the integers, so that sum's bits minus those of
// 1.5 * 2^23 give ceil(x) as an integer, and its value minus 1.5 * 2^23 gives it
// as a float (both exact).  Replaces a float-to-int and an int-to-float conversion.
constexpr float kCeilMagic = 12582912.0f;
constexpr int kCeilMagicBits = 0x4B400000;
__device__ __forceinline__ float ceil_magic(float x) { return __fadd_ru(x, kCeilMagic); }
__device__ __forceinline__ int magic_int(float m) { return __float_as_int(m) - kCeilMagicBits; }
__device__ __forceinline__ float magic_float(float m) { return __fsub_rn(m, kCeilMagic); }

// Approximate detector coordinate of a pixel centre (candidate selection only).
__device__ __forceinline__ float det_coord(const ViewP &vp, float Xj, float Yi)
{
    return __fmaf_rn(vp.cu, Xj, __fmul_rn(vp.su, Yi));
}

// The rounded part of delta: uc_lo + cu_lo X + su_lo Y, in the view class's order.
__device__ __forceinline__ float delta_small(const ViewP &vp, float X, float Y, float uc_lo)
{
    return (vp.flags & kViewClassB) ? __fmaf_rn(vp.su_lo, Y, __fmaf_rn(vp.cu_lo, X, uc_lo))
                                    : __fmaf_rn(vp.cu_lo, X, __fmaf_rn(vp.su_lo, Y, uc_lo));
}

__device__ __forceinline__ float bin_pos(int u, float uc) { return __fsub_rn(__int2float_rn(u), uc); }

// Outer indices [*lo, *hi] at which a ray whose centre sits at inner index
// base + b_o * o can meet the inner range [0, n_inner): the centre within the
// footprint half-width hwq plus one index of slack of either end.  Rows outside
// it contribute nothing (their candidates fall on the zero fill).
__device__ __forceinline__ void fwd_row_range(const ViewP &vp, float base, int n_inner, int n_outer, int *lo, int *hi)
{
    const float L = -vp.hwq - 1.0f, H = __int2float_rn(n_inner) + vp.hwq;
    if (fabsf(vp.b_o) < 1e-20f) {
        const bool in = base >= L && base <= H;
        *lo = in ? 0 : n_outer;
        *hi = in ? n_outer - 1 : -1;
        return;
    }
    const float ra = __fdiv_rn(__fsub_rn(L, base), vp.b_o), rb = __fdiv_rn(__fsub_rn(H, base), vp.b_o);
    const float fo = __int2float_rn(n_outer);
    const float a = fminf(fmaxf(fminf(ra, rb) - 1.0f, -1.0f), fo), b = fminf(fmaxf(fmaxf(ra, rb) + 1.0f, -1.0f), fo);
    *lo = max(0, __float2int_rd(a));
    *hi = min(n_outer - 1, __float2int_ru(b));
}

// ----------------------------------------------------------------- FFT plan
struct FFTPlan {
    int n;
    int nst;
    int radix[kMaxStages];
    const double2 *tw;  // exp(-2 pi i k / n), k = 0 .. n-1 (FP64)
    const float4 *twf;  // the same as double-float pairs (cos h, cos l, sin h, sin l)
};

// ----------------------------------------------------------------- scalars
// Device-resident state of one problem's solve (Algorithm 3).
struct Scal {
    double f;          // f(x_{k+1/2}) of the most recent forward projection of x
    double f0;         // f(x_0)
    double pth;        // p^T h = ||R p||^2 of the current p
    double gtp;        // g^T p
    double zth;        // z^T h_prev
    double alpha, beta;
    double tv_k, tv_half;  // TV(x_k), TV(x_{k+1/2}) of the last S_TV call
    double snorm2;     // ||s_k||^2 of the last S_TV call (accumulated in FP64)
    double eps;
    double f_ls;       // Bayesian criterion: ||R x - b||^2 of the current residual
    double muX;        // Bayesian criterion: the gray level mu_X of Eq. (2.3)
    double pp;         // ||p||^2 of the current p (h = r^2 R^T R p + p for the Bayesian criterion)
    long long ell;     // l of Algorithm 1/3
    long long trials;  // trials of the last S_TV call
    int k;             // executions of the while body
    int done;          // 1: the while condition failed (or an error stopped the loop)
    int status;        // SUPCG_OK or an error code
    int init;          // 1 while running steps 2-7 (beta forced to 0)
    int n_fallback;    // learned perturbation: proposals rejected by the nonascent test
    int n_learned;     // learned perturbation: proposals accepted
    // a^l of Algorithm 1 for l = apow_ell and a = apow_a (valid when apow_ok), advanced by
    // one factor a per S_TV trial, so that a call needs no FP64 pow (slow on the narrow FP64
    // pipe, and on the critical path of every trial) unless l or a changed elsewhere
    double apow, apow_a;
    long long apow_ell;
    int apow_ok;
    // alpha as two FP32 parts (alpha_h + alpha_l to ~2^-48) and beta rounded to FP32, written
    // with alpha and beta, so that the vector kernels read them without FP64 arithmetic
    float alpha_h, alpha_l, beta_f;
};

// ----------------------------------------------------------------- problem
// One problem of a batched launch (device copy lives in global memory).
struct Prob {
    CUtensorMap tm[12];    // TMA maps (FP32, padded pitches) of the projected images: 2 w + c for image w
                           // (0 = x, 1 = p, 2 = d) in layout c (0 = rows, 1 = transposed); 6 + 2 w + c the
                           // same of the mirrored images (only with mirror pairs)
    int nx, ny, V, U;
    int nxp, nyp, Up;      // pitches in elements: image, transposed image, sinogram
    int BU, BW, ntu;       // forward tiling: bins per tile, box width, bin tiles per view
    int nfw;               // forward warp items (a tile's first 64 bins, or the rest)
    int nA, nB;            // number of class-A / class-B views
    float cx, cy, uc;      // uc = (U-1)/2 - off/ds (approximate uses)
    float uc_hi, uc_lo;    // exact split of uc (see ViewP)
    int bwin;              // backprojector: bins staged per view and tile (multiple of 4)
    const ViewP *views;    // [V]
    const int *vlist;      // [nA + nB]: class-A views, then class-B views
    const int *mirror;     // nullable [V]: the partner of a mirror pair's first view, else -1
    const int *border;     // [nfw]: forward warp items ((vidx * ntu + tile) * 2 + half), longest
                           // first; block b's warps take entries 2b and 2b + 1
    const int *border_all; // [nfw_all]: the same with every view's items (border pairs mirror views)
    int nfw_all;
    FFTPlan fx, fy;
    double mu, rho;
    double r2;             // r^2 of the Bayesian criterion (Eq. (2.3)); 0: least squares
    int stv_own;           // 1: S_TV uses stv_K, stv_a, stv_gamma below (a parameter sweep), else its arguments
    int stv_K;
    double stv_a, stv_gamma;
    const float *se_ref;   // nullable: reference image [ny][nx] of the selective error of Eq. (4.1)
    double *se_log;        // SE of x_{k+1/2} of while-body k (1-based) at se_log[k - 1] (with se_ref)
    double se_ax, se_ay;   // semi-axes of the SE ellipse, in pixels (horizontal, vertical)
    double gray_scale;     // ds / (V nx ny d^2): sum of b times this is the gray-level estimate
    int precond;           // 1: M of Eq. (3.2); 0: M = I
    int storage;           // SUPCG_F32 / SUPCG_BF16 element type of in_user / out_user
    int stv_blocks;        // cooperative S_TV: blocks owned by this problem
    int fft_rpb, fft_cw;   // FFT rows per block / columns per block
    // solve buffers (images pitch nxp, transposed pitch nyp, sinograms pitch Up)
    float *x, *xT, *p, *pT, *g, *z, *h, *tbar;
    // low part of the iterate: the solve keeps x as the double-float pair (x, xlo), x = RN(x + xlo)
    // the FP32 image every reader (projector, TV, caller) sees, xlo the rounding error of x,
    // so that the many small updates of S_TV and x <- x + alpha p do not round into x; null:
    // x alone (ART's row actions)
    float *xlo;
    // low part of the gradient of a solve, g + glo = the backprojector's double-float sum:
    // the preconditioner damps g's lowest frequencies by mu, so FP32 rounding of g alone
    // would dominate z = M g there; read by the first transform pass and by g^T p
    float *glo;
    // with mirror pairs: x and p mirrored left-right (xm[i][j] = x[i][nx-1-j]) and their
    // transposes, written with x^T and p^T for the forward projector (else null)
    float *xm, *xmT, *pm, *pmT;
    // the displacement d = x_{k+1/2} - x_k of S_TV (steps 11-12 of Algorithm 3) in the
    // projector's layouts (dm, dmT only with mirror pairs): a while-body projects d, not x
    float *d, *dT, *dm, *dmT;
    // r = R x - b (FP32, read by the backprojector) and q = R p; rd and qd are the same in
    // FP64, where the solve carries the residual from step to step:
    // r_{k+1/2} = r_{k-1/2} + alpha_{k-1} q_{k-1} + R d_k, with the same sums as R x - b
    float *r, *q, *bpad;
    double *rd, *qd;
    double2 *C;            // FFT scratch [ny][nx] (FP64 complex)
    float2 *Dtab;          // h(w_r) / (nx ny) at (min(k1, ny-k1), min(k2, nx-k2)), double-float: [ny/2+1][nx/2+1]
    float2 *bsplit;        // backprojector: each sinogram's and view part's pixel sums, double-float [2][bparts][ny][nxp]
    int bparts;            // backprojector: blocks per pixel tile, each taking a contiguous share of the view chunks
    double *art_u;         // ART: auxiliary value u_i per ray [V][U]
    double *art_rn;        // ART: 1 / (1 + r^2 ||R_i||^2) per ray [V][U]
    unsigned *tilecnt;     // backprojector: parts finished per tile (reset by the last one)
    Scal *sc;
    double *partial;       // reduction partials (>= 2 * max blocks per kernel)
    unsigned *counter;     // last-block tickets [8]
    unsigned *bar;         // cooperative barrier [2]: arrivals, generation
    long long wait_limit;  // polls before a cooperative barrier gives up (supcg_set_wait_limit)
    int bar_extra;         // blocks a cooperative barrier waits for beyond its launch's (test hook, normally 0)
    double *log;           // nullable [max_iter][SUPCG_LOG_STRIDE]
    float *trace;          // nullable [max_iter][ny][nx]: x_k at the start of every while body
    // caller-owned I/O (unpadded): image in / out, sinogram in
    const void *in_user;
    void *out_user;
    const void *in_user2;
};

// Map a block of a batched launch to (problem, block within problem).
__device__ __forceinline__ int find_problem(const int *prefix, int count, int b, int *local)
{
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= b) lo = mid; else hi = mid - 1;
    }
    *local = b - __ldg(prefix + lo);
    return lo;
}

// ----------------------------------------------------------------- double-float arithmetic
// For work that needs more than FP32 but should not run on this part's narrow
// FP64 pipe (the preconditioner's transforms, the projectors' final sums): a
// real value is the unevaluated sum h + l of two FP32 numbers with |l| <=
// ulp(h) / 2, about 48 significant bits.  Sums use Knuth's TwoSum (the
// exact rounding error of a + b for any magnitudes), products the FMA form of
// Dekker's TwoProduct (the exact rounding error of a * b); the low parts are
// then added and the pair renormalised.  Each operation's error is a few units
// of 2^-48 relative to its operands, as a rounded FP64 operation's is of 2^-53.
struct df {
    float h, l;
};

__device__ __forceinline__ df df_make(float v) { return {v, 0.0f}; }
__device__ __forceinline__ df df_neg(df a) { return {-a.h, -a.l}; }
__device__ __forceinline__ df df_half(df a) { return {0.5f * a.h, 0.5f * a.l}; }   // exact

__device__ __forceinline__ df df_add(df a, df b)
{
    const float s = __fadd_rn(a.h, b.h);
    const float bv = __fsub_rn(s, a.h);
    const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bv)), __fsub_rn(b.h, bv));   // TwoSum error
    const float t = __fadd_rn(__fadd_rn(a.l, b.l), e);
    const float h = __fadd_rn(s, t);
    return {h, __fsub_rn(t, __fsub_rn(h, s))};
}
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);                               // TwoProduct error
    e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
    const float h = __fadd_rn(p, e);
    return {h, __fsub_rn(e, __fsub_rn(h, p))};
}

// Per-thread sums of FP32 terms and products for the FP64 reductions of the
// streaming kernels: each term (or the exact product of two FP32 values, a
// TwoProduct pair) is added in double-float arithmetic and the thread's sum is
// converted to FP64 once, so that the narrow FP64 pipe does a few operations
// per thread instead of a conversion and an add per element.
__device__ __forceinline__ df df_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};   // p + e = a b exactly
}
__device__ __forceinline__ void df_acc(df &s, float v) { s = df_add(s, df{v, 0.0f}); }
__device__ __forceinline__ void df_acc_prod(df &s, float a, float b) { s = df_add(s, df_prod(a, b)); }
__device__ __forceinline__ double df_to_double(df a) { return (double)a.h + (double)a.l; }

// ----------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block sum in a fixed order (deterministic); result valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    v = warp_sum(v);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = (l < NT / 32) ? sh[l] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

// Block sum of per-thread double-float values in a fixed order, on the FP32 pipe:
// shuffles of the pairs and double-float adds, one conversion to FP64 at the end
// (this part's FP64 pipe is narrow).  Result valid in thread 0; sh holds >= NT/32
// doubles.
__device__ __forceinline__ df warp_sum_df(df v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const df w = {__shfl_down_sync(0xffffffffu, v.h, o), __shfl_down_sync(0xffffffffu, v.l, o)};
        v = df_add(v, w);
    }
    return v;
}
template <int NT>
__device__ __forceinline__ double block_sum_df(df v, double *sh)
{
    float2 *s2 = reinterpret_cast<float2 *>(sh);
    v = warp_sum_df(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) s2[w] = make_float2(v.h, v.l);
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        df u = (l < NT / 32) ? df{s2[l].x, s2[l].y} : df{0.0f, 0.0f};
        u = warp_sum_df(u);
        if (l == 0) r = df_to_double(u);
    }
    __syncthreads();
    return r;
}

// Two block sums in one pass (one sweep of shuffles, one shared-memory round): the
// same values as two calls of block_sum_df.  Results valid in thread 0; sh holds
// >= NT/16 doubles.
template <int NT>
__device__ __forceinline__ void block_sum_df2(df a, df b, double *sh, double *ra, double *rb)
{
    float4 *s4 = reinterpret_cast<float4 *>(sh);
    a = warp_sum_df(a);
    b = warp_sum_df(b);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) s4[w] = make_float4(a.h, a.l, b.h, b.l);
    __syncthreads();
    *ra = *rb = 0.0;
    if (w == 0) {
        const float4 v = (l < NT / 32) ? s4[l] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        const df ua = warp_sum_df(df{v.x, v.y}), ub = warp_sum_df(df{v.z, v.w});
        if (l == 0) {
            *ra = df_to_double(ua);
            *rb = df_to_double(ub);
        }
    }
    __syncthreads();
}

// Sum partial[0..n) in a fixed order with the whole block; result in all threads.  The
// partials come from other blocks (published by a grid barrier or the last-block ticket,
// both fenced): they are read from L2 (__ldcg, not the non-coherent L1), eight per thread
// in flight, and added in the same order as one by one.
template <int NT>
__device__ __forceinline__ double block_sum_array(const double *partial, int n, double *sh)
{
    double v = 0.0;
    int i = threadIdx.x;
    for (; i + 7 * NT < n; i += 8 * NT) {
        double t[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) t[k] = __ldcg(partial + i + k * NT);
#pragma unroll
        for (int k = 0; k < 8; ++k) v += t[k];
    }
    for (; i < n; i += NT) v += __ldcg(partial + i);
    v = block_sum<NT>(v, sh);
    if (threadIdx.x == 0) sh[32] = v;
    __syncthreads();
    double r = sh[32];
    __syncthreads();
    return r;
}

// Two such sums in one pass (both arrays' loads in flight together, one reduction sweep):
// the same values as two calls of block_sum_array.  Results in all threads; sh holds >= 34
// doubles.
template <int NT>
__device__ __forceinline__ void block_sum_array2(const double *pa, const double *pb, int n, double *sh, double *ra,
                                                 double *rb)
{
    static_assert(NT % 32 == 0 && NT <= 512, "at most 16 warps: their sums sit at sh[0..15] and sh[16..31]");
    double va = 0.0, vb = 0.0;
    int i = threadIdx.x;
    for (; i + 3 * NT < n; i += 4 * NT) {
        double ta[4], tb[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            ta[k] = __ldcg(pa + i + k * NT);
            tb[k] = __ldcg(pb + i + k * NT);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            va += ta[k];
            vb += tb[k];
        }
    }
    for (; i < n; i += NT) {
        va += __ldcg(pa + i);
        vb += __ldcg(pb + i);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        va += __shfl_down_sync(0xffffffffu, va, o);
        vb += __shfl_down_sync(0xffffffffu, vb, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sh[w] = va;
        sh[16 + w] = vb;
    }
    __syncthreads();
    if (w == 0) {
        double a = (l < NT / 32) ? sh[l] : 0.0, b = (l < NT / 32) ? sh[16 + l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
        if (l == 0) {
            sh[32] = a;
            sh[33] = b;
        }
    }
    __syncthreads();
    *ra = sh[32];
    *rb = sh[33];
    __syncthreads();
}

// 1 / sqrt(s) for s > 0: an FP32 seed and two Newton steps in FP64 (multiplies and FMAs
// only; the FP64 square root and division routines are long on the narrow FP64 pipe)
__device__ __forceinline__ double rsqrt_fp64(double s)
{
    if (!(s > 1e-30 && s < 1e30)) return 1.0 / sqrt(s);   // outside the FP32 seed's range
    double y = (double)rsqrtf((float)s);
    y = y * fma(-0.5 * s, y * y, 1.5);
    y = y * fma(-0.5 * s, y * y, 1.5);
    return y;
}

// Last-block-done ticket: true in every thread of the block that finishes last.
__device__ __forceinline__ bool last_block(unsigned *counter, unsigned nblocks, int *sh_flag)
{
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(counter, 1u);
        *sh_flag = (t == nblocks - 1);
    }
    __syncthreads();
    bool last = *sh_flag;
    if (last) __threadfence();
    return last;
}

// Bounded barrier among `nblocks` co-resident blocks (cooperative launch).
// bar[0] counts arrivals, bar[1] is the generation.  Returns false after
// `limit` polls without a release (and raises SUPCG_ERR_TIMEOUT in *status).
__device__ __forceinline__ bool coop_barrier(unsigned *bar, unsigned nblocks, int *status, int *sh_flag,
                                             long long limit)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = bar + 1;
        unsigned gen = *vgen;
        __threadfence();
        unsigned arrived = atomicAdd(bar, 1u);
        int ok = 1;
        if (arrived == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long it = 0;
            while (*vgen == gen) {
                if (++it > limit) { ok = 0; atomicExch(status, (int)SUPCG_ERR_TIMEOUT); break; }
                __nanosleep(64);
            }
        }
        __threadfence();
        *sh_flag = ok && (*(volatile int *)status != (int)SUPCG_ERR_TIMEOUT);
    }
    __syncthreads();
    return *sh_flag;
}

// ----------------------------------------------------------------- TMA / mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Bounded wait for phase `parity` of an mbarrier; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity)
{
    uint32_t a = smem_u32(bar);
    for (long long it = 0; it < kSpinLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 2-D tiled TMA load of box (x0 = innermost coordinate, y0) into shared memory.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tm, int x0, int y0, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x0), "r"(y0), "r"(smem_u32(bar))
        : "memory");
}

// ----------------------------------------------------------------- host side
#define SUPCG_CUDA_TRY(expr)                                   \
    do {                                                       \
        cudaError_t e_ = (expr);                               \
        if (e_ != cudaSuccess) return supcg::cuda_fail(e_, #expr, __FILE__, __LINE__); \
    } while (0)

int cuda_fail(cudaError_t e, const char *what, const char *file, int line);

// Kernel attributes are per device: once per (kernel, current device), raise the
// kernel's dynamic shared-memory limit to max_dyn_smem bytes and, when carveout >= 0,
// set its preferred shared-memory carveout.  Thread-safe.
int func_attrs_once(const void *func, int max_dyn_smem, int carveout = -1);
// Current device (0 .. kMaxDevices-1) for per-device host caches.
constexpr int kMaxDevices = 64;
int current_device(int *dev);

// Launchers (defined in the kernel translation units).  Each enqueues one
// kernel over all `count` problems of `probs` (device array) on `st`.
// FWD_RESID: r = R x - b (steps 1-9); FWD_NORM: q = R p and alpha; FWD_PLAIN: the caller's
// projection; FWD_RUPD: r <- r + alpha q + R d (a while-body with S_TV)
enum FwdMode { FWD_RESID = 0, FWD_NORM = 1, FWD_PLAIN = 2, FWD_RUPD = 3 };
enum BwdMode { BWD_G = 0, BWD_H = 1, BWD_PLAIN = 2 };

struct Launch {
    const Prob *probs;     // device
    int count;
    const int *prefix;     // device: block prefix for this kernel type, count+1 entries
    int blocks;            // total blocks
    int bw_max;            // widest forward box (floats) among the problems
    int bparts;            // backprojector view parts shared by every problem, 0 if they differ
    int mirror;            // 1: some problem has mirror pairs of views (the forward projector's paired variant)
    cudaStream_t st;
};

int launch_forward(const Launch &L, const Launch &La, int which, int mode);   // La: every view's items
int launch_backward(const Launch &L, int mode, int bwin);
int launch_backward2(const Launch &L, int bwin);   // g from r and h from q in one pass
int art_max_blocks(int *out);                                           // co-resident blocks of k_art
int launch_art_init(const Prob *d_prob, double r, int blocks, cudaStream_t st);
int launch_art(const Prob *d_prob, int cycles, double r, double lam, int S, int blocks, cudaStream_t st);
int backward_blocks(int nx, int ny, int dual, int parts);
int encode_tiled(CUtensorMap *m, CUtensorMapDataType type, int rank, void *base, const cuuint64_t *dims,
                 const cuuint64_t *strides_bytes, const cuuint32_t *box);
int launch_stage_in(const Launch &L, int which);           // caller image -> x and x^T (0) or g (1)
int launch_stage_sino(const Launch &L, int which);         // caller sinogram -> r (0, in_user) or bpad (1, in_user2)
int launch_store_out(const Launch &L, int which);          // padded image (0 x, 1 g, 2 z, 3 tbar) -> caller
int launch_fft_rows(const Launch &L, int inverse, int standalone, int smem);
int launch_fft_cols(const Launch &L, int standalone, int smem);
int launch_fft_dtab(const Launch &L);                       // fills Dtab from mu, rho (once per solve or call)
int launch_gray(const Launch &L);                           // sc->muX from bpad (Bayesian criterion)
int launch_pupdate(const Launch &L);
int launch_beta(const Launch &L);
int launch_xupdate(const Launch &L);
int launch_rupdate(const Launch &L);   // r <- r + alpha q and f (a while-body without S_TV)
int launch_gather_xt(const Launch &L, float *xs, float *ts);   // x, tbar of every problem -> [count][ny][nx]
int launch_stv(const Launch &L, int K, double a, double gamma, long long max_trials, int *trials_out,
               int want_snorm, const float *dir = nullptr);
int launch_tv_tbar(const Launch &L);
int stv_max_blocks_per_sm(int *out);
int cnn_forward(struct supcg_cnn_s *net, const float *d_x, const float *d_tbar, int count, cudaStream_t st);
float *cnn_output(struct supcg_cnn_s *net);
int cnn_shape(struct supcg_cnn_s *net, int *ny, int *nx);
int cnn_capacity(struct supcg_cnn_s *net, int *max_batch);

} // namespace supcg
