// Preconditioner z = M g, M = F^-1 D F (Eq. (3.2)), on the ny x nx grid.
//
// Three passes over a complex scratch array S [ny][nx/2 + 1] (FP32 vectors in
// and out; inside, double-float arithmetic: pairs of FP32 numbers carrying
// about 48 bits, on the FP32 pipe, since this part's FP64 pipe is narrow.  The
// operator spans five decades, from h(0) = mu to about pi, and a plain FP32
// transform of a gradient dominated by its low frequencies loses several
// digits of M g).  g and z are real and D is real and even, so every row
// spectrum is Hermitian: only k2 = 0 .. nx/2 is kept, and two real rows share
// one complex transform.
//   rows:  S[i, k2] = FFT(g[i, :])(k2), k2 <= nx/2     (k_fft_rows, forward, row pairs)
//   cols:  S[:, k2] = IFFT(D[:, k2] * FFT(S[:, k2]))   (k_fft_cols)
//   rows:  z[i, :] = IFFT(Hermitian S[i, :])            (k_fft_rows, inverse, row pairs)
// with D = h(w_r) / (nx ny), h(w) = (|w| + mu)(rho + (1-rho) cos w), w_r the
// radial frequency clamped to pi, tabulated once per call or solve in FP64 and
// stored as pairs.  Each length is transformed in shared memory by a
// mixed-radix Stockham (autosort) FFT: radix 4 and 2 butterflies written out,
// any other prime factor by its defining sum.  Twiddles exp(-2 pi i k/n) come
// from FP64 tables built on the host (stored as pairs for the solver's
// transforms; the allocation-free variant at the end of this file keeps FP64).
#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace supcg {

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 twid(const double2 *tw, int e, bool inv)
{
    double2 w = __ldg(tw + e);
    return inv ? make_double2(w.x, -w.y) : w;
}

// Transforms `nvec` contiguous vectors of length pl.n held in a (b is scratch
// of the same size).  Returns the buffer that holds the result.
__device__ double2 *fft_smem(double2 *a, double2 *b, int nvec, const FFTPlan &pl, bool inv)
{
    const int n = pl.n;
    int Ns = 1;
    for (int s = 0; s < pl.nst; ++s) {
        const int R = pl.radix[s];
        const int m = n / R;
        const int stride = n / (Ns * R);
        for (int idx = threadIdx.x; idx < nvec * m; idx += blockDim.x) {
            const int vec = idx / m, j = idx - vec * m;
            const int k = j % Ns;
            const double2 *src = a + vec * n;
            double2 *dst = b + vec * n + (j / Ns) * Ns * R + k;
            if (R == 2) {
                double2 v0 = src[j], v1 = cmul(src[j + m], twid(pl.tw, k * stride, inv));
                dst[0] = cadd(v0, v1);
                dst[Ns] = csub(v0, v1);
            } else if (R == 4) {
                double2 v0 = src[j];
                double2 v1 = cmul(src[j + m], twid(pl.tw, k * stride, inv));
                double2 v2 = cmul(src[j + 2 * m], twid(pl.tw, 2 * k * stride, inv));
                double2 v3 = cmul(src[j + 3 * m], twid(pl.tw, 3 * k * stride, inv));
                double2 t0 = cadd(v0, v2), t1 = csub(v0, v2), t2 = cadd(v1, v3), d = csub(v1, v3);
                // multiply (v1 - v3) by the fourth root of unity -i (forward) or +i (inverse)
                double2 t3 = inv ? make_double2(-d.y, d.x) : make_double2(d.y, -d.x);
                dst[0] = cadd(t0, t2);
                dst[Ns] = cadd(t1, t3);
                dst[2 * Ns] = csub(t0, t2);
                dst[3 * Ns] = csub(t1, t3);
            } else {
                // any radix: V_s = sum_r (src_r w^{rk}) w_R^{rs}
                const int nR = n / R;
                for (int so = 0; so < R; ++so) {
                    double2 acc = make_double2(0.0, 0.0);
                    for (int r = 0; r < R; ++r) {
                        double2 v = cmul(src[j + r * m], twid(pl.tw, r * k * stride, inv));
                        acc = cadd(acc, cmul(v, twid(pl.tw, ((r * so) % R) * nR, inv)));
                    }
                    dst[so * Ns] = acc;
                }
            }
        }
        __syncthreads();
        double2 *t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

// complex double-float, stored as float4 (re.h, re.l, im.h, im.l)
struct dfc {
    df r, i;
};
__device__ __forceinline__ dfc dfc_ld(const float4 &v) { return {{v.x, v.y}, {v.z, v.w}}; }
__device__ __forceinline__ float4 dfc_st(const dfc &a) { return make_float4(a.r.h, a.r.l, a.i.h, a.i.l); }
__device__ __forceinline__ dfc dfc_add(dfc a, dfc b) { return {df_add(a.r, b.r), df_add(a.i, b.i)}; }
__device__ __forceinline__ dfc dfc_sub(dfc a, dfc b) { return {df_sub(a.r, b.r), df_sub(a.i, b.i)}; }
__device__ __forceinline__ dfc dfc_mul(dfc a, dfc b)
{
    return {df_sub(df_mul(a.r, b.r), df_mul(a.i, b.i)), df_add(df_mul(a.r, b.i), df_mul(a.i, b.r))};
}
__device__ __forceinline__ dfc twid_df(const float4 *tw, int e, bool inv)
{
    const float4 w = tw[e];
    return inv ? dfc{{w.x, w.y}, {-w.z, -w.w}} : dfc{{w.x, w.y}, {w.z, w.w}};
}

// The twiddles the block's transforms read: its shared copy (stw, room for
// kFftSmemTw entries) when the length allows, else the global table.  The copy
// is only issued here: the caller's barrier after its own loads completes it, so
// both sets of loads are in flight together.
__device__ __forceinline__ const float4 *stage_twiddles(const FFTPlan &pl, float4 *stw)
{
    if (pl.n > kFftSmemTw) return pl.twf;
    for (int e = threadIdx.x; e < pl.n; e += blockDim.x) stw[e] = __ldg(pl.twf + e);
    return stw;
}

// Elements per thread of a 256-thread pass whose h (rows) or D (columns) is read before
// the transform (nvec x n <= 2048 gives at most 8; the columns keep 4 in registers)
constexpr int kFftPerThread = 8;
constexpr int kFftPerThreadD = 4;

// Transforms `nvec` contiguous vectors of length pl.n held in a (b is scratch
// of the same size), in double-float, with the twiddles tw (shared or global);
// returns the buffer that holds the result.  The same mixed-radix Stockham
// schedule as fft_smem; for power-of-two lengths the index arithmetic is shifts.
__device__ __forceinline__ float4 *fft_smem_df(float4 *a, float4 *b, int nvec, const FFTPlan &pl, const float4 *tw, bool inv)
{
    const int n = pl.n;
    const bool pow2 = (n & (n - 1)) == 0;
    // power-of-two lengths: the host's factorisation is radix 4 while 4 divides, then one
    // radix 2, so the radices follow from the length (no per-stage read of the plan)
    const int lg = __ffs(n) - 1, n4 = lg >> 1;
    const int nst = pow2 ? n4 + (lg & 1) : pl.nst;
    int Ns = 1;
    for (int s = 0; s < nst; ++s) {
        const int R = pow2 ? (s < n4 ? 4 : 2) : pl.radix[s];
        const int m = n / R;
        const int stride = n / (Ns * R);
        const int lm = __ffs(m) - 1, lns = __ffs(Ns) - 1;   // log2 m, log2 Ns (power-of-two lengths)
        for (int idx = threadIdx.x; idx < nvec * m; idx += blockDim.x) {
            int vec, j, k, jq;
            if (pow2) {
                vec = idx >> lm;
                j = idx & (m - 1);
                k = j & (Ns - 1);
                jq = j >> lns;
            } else {
                vec = idx / m;
                j = idx - vec * m;
                jq = j / Ns;
                k = j - jq * Ns;
            }
            const float4 *src = a + vec * n;
            float4 *dst = b + vec * n + jq * Ns * R + k;
            if (R == 2) {
                const dfc v0 = dfc_ld(src[j]), v1 = dfc_mul(dfc_ld(src[j + m]), twid_df(tw, k * stride, inv));
                dst[0] = dfc_st(dfc_add(v0, v1));
                dst[Ns] = dfc_st(dfc_sub(v0, v1));
            } else if (R == 4) {
                const dfc v0 = dfc_ld(src[j]);
                const dfc v1 = dfc_mul(dfc_ld(src[j + m]), twid_df(tw, k * stride, inv));
                const dfc v2 = dfc_mul(dfc_ld(src[j + 2 * m]), twid_df(tw, 2 * k * stride, inv));
                const dfc v3 = dfc_mul(dfc_ld(src[j + 3 * m]), twid_df(tw, 3 * k * stride, inv));
                const dfc t0 = dfc_add(v0, v2), t1 = dfc_sub(v0, v2), t2 = dfc_add(v1, v3), d = dfc_sub(v1, v3);
                // (v1 - v3) times the fourth root of unity -i (forward) or +i (inverse)
                const dfc t3 = inv ? dfc{df_neg(d.i), d.r} : dfc{d.i, df_neg(d.r)};
                dst[0] = dfc_st(dfc_add(t0, t2));
                dst[Ns] = dfc_st(dfc_add(t1, t3));
                dst[2 * Ns] = dfc_st(dfc_sub(t0, t2));
                dst[3 * Ns] = dfc_st(dfc_sub(t1, t3));
            } else {
                // any radix: V_s = sum_r (src_r w^{rk}) w_R^{rs}
                const int nR = n / R;
                for (int so = 0; so < R; ++so) {
                    dfc acc = {{0.0f, 0.0f}, {0.0f, 0.0f}};
                    for (int r = 0; r < R; ++r) {
                        const dfc v = dfc_mul(dfc_ld(src[j + r * m]), twid_df(tw, r * k * stride, inv));
                        acc = dfc_add(acc, dfc_mul(v, twid_df(tw, ((r * so) % R) * nR, inv)));
                    }
                    dst[so * Ns] = dfc_st(acc);
                }
            }
        }
        __syncthreads();
        float4 *t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

// Rows pass on pairs of rows (g and z are real).  Block `local` takes the row
// pairs 2i, 2i+1 for i in [local * rpb, (local + 1) * rpb) (a missing last
// partner is a zero row).
//   inverse = 0:  c = g[2i] + i g[2i+1];  C = FFT(c);  the two rows' spectra
//                 A(k) = (C(k) + conj C(-k)) / 2,  B(k) = (C(k) - conj C(-k)) / (2i)
//                 for k = 0 .. nx/2 (the rest follows by Hermitian symmetry) go to
//                 S[2i][k] and S[2i+1][k], S viewed as [ny][nx/2 + 1].
//   inverse = 1:  c(k) = Y(2i, k) + i Y(2i+1, k) with Y(r, k) = conj Y(r, nx - k)
//                 beyond nx/2 (the filtered rows are real);  z[2i] + i z[2i+1] =
//                 IFFT(c) (the 1 / (nx ny) is folded into D).
__global__ void __launch_bounds__(256) k_fft_rows(const Prob *__restrict__ probs, const int *__restrict__ prefix,
                                                  int count, int inverse, int standalone)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int local;
    const Prob &P = probs[find_problem(prefix, count, blockIdx.x, &local)];
    if (!standalone && P.sc->done) return;
    const int nx = P.nx, ny = P.ny, rpb = P.fft_rpb, hx = nx / 2 + 1;
    const int npairs = (ny + 1) / 2;
    float4 *a = reinterpret_cast<float4 *>(smem_raw);
    float4 *b = a + rpb * nx;
    const float4 *tw = stage_twiddles(P.fx, b + rpb * nx);
    const int p0 = local * rpb;
    const int np = min(rpb, npairs - p0);
    float4 *S = reinterpret_cast<float4 *>(P.C);
    for (int e = threadIdx.x; e < np * nx; e += blockDim.x) {
        const int pr = e / nx, q = e - pr * nx;
        const int ra = 2 * (p0 + pr), rb = ra + 1;
        if (!inverse) {
            // inside a solve the gradient is the double-float pair (g, glo)
            const float *glo = standalone ? nullptr : P.glo;
            const size_t ia = (size_t)ra * P.nxp + q, ib = (size_t)rb * P.nxp + q;
            const float va = P.g[ia];
            const float vb = rb < ny ? P.g[ib] : 0.0f;
            const float la = glo ? glo[ia] : 0.0f;
            const float lb = (glo && rb < ny) ? glo[ib] : 0.0f;
            a[e] = make_float4(va, la, vb, lb);
        } else {
            const bool lo = q <= nx / 2;
            const int kk = lo ? q : nx - q;
            dfc ya = dfc_ld(S[(size_t)ra * hx + kk]);
            dfc yb = rb < ny ? dfc_ld(S[(size_t)rb * hx + kk]) : dfc{{0.0f, 0.0f}, {0.0f, 0.0f}};
            if (!lo) {
                ya.i = df_neg(ya.i);
                yb.i = df_neg(yb.i);
            }
            a[e] = dfc_st(dfc{df_sub(ya.r, yb.i), df_add(ya.i, yb.r)});   // ya + i yb
        }
    }
    // the inverse pass's h (for z^T h), read before the transform so that its loads
    // overlap the butterflies instead of following them
    float hA[kFftPerThread], hB[kFftPerThread];
    const bool want_h = inverse && !standalone;
#pragma unroll
    for (int k = 0; k < kFftPerThread; ++k) {
        const int e = threadIdx.x + k * blockDim.x;
        hA[k] = hB[k] = 0.0f;
        if (want_h && e < np * nx) {
            const int pr = e / nx, q = e - pr * nx;
            const int ra = 2 * (p0 + pr), rb = ra + 1;
            hA[k] = P.h[(size_t)ra * P.nxp + q];
            if (rb < ny) hB[k] = P.h[(size_t)rb * P.nxp + q];
        }
    }
    __syncthreads();
    float4 *res = fft_smem_df(a, b, np, P.fx, tw, inverse != 0);
    if (!inverse) {
        for (int e = threadIdx.x; e < np * hx; e += blockDim.x) {
            const int pr = e / hx, k = e - pr * hx;
            const int ra = 2 * (p0 + pr), rb = ra + 1;
            const dfc c1 = dfc_ld(res[pr * nx + k]), c2 = dfc_ld(res[pr * nx + (k == 0 ? 0 : nx - k)]);
            S[(size_t)ra * hx + k] = dfc_st(dfc{df_half(df_add(c1.r, c2.r)), df_half(df_sub(c1.i, c2.i))});
            if (rb < ny) S[(size_t)rb * hx + k] = dfc_st(dfc{df_half(df_add(c1.i, c2.i)), df_half(df_sub(c2.r, c1.r))});
        }
    } else {
        // z, and inside a solve also z^T h for beta = z^T h / p^T h (Algorithm 2 step 3)
        df s = df_make(0.0f);   // z^T h: exact products, double-float sums
        // element e = threadIdx.x + k blockDim.x; the first kFftPerThread of a thread use the
        // prefetched h (indexed at compile time, so it stays in registers), any further ones
        // read it here
        auto put_z = [&](int e, float ha, float hb) {
            const int pr = e / nx, q = e - pr * nx;
            const int ra = 2 * (p0 + pr), rb = ra + 1;
            const size_t ia = (size_t)ra * P.nxp + q, ib = (size_t)rb * P.nxp + q;
            const float4 v = res[e];
            const float za = __fadd_rn(v.x, v.y);   // the pair rounded to FP32
            P.z[ia] = za;
            if (!standalone) df_acc_prod(s, za, ha);
            if (rb < ny) {
                const float zb = __fadd_rn(v.z, v.w);
                P.z[ib] = zb;
                if (!standalone) df_acc_prod(s, zb, hb);
            }
        };
#pragma unroll
        for (int k = 0; k < kFftPerThread; ++k) {
            const int e = threadIdx.x + k * blockDim.x;
            if (e < np * nx) put_z(e, hA[k], hB[k]);
        }
        for (int e = threadIdx.x + kFftPerThread * blockDim.x; e < np * nx; e += blockDim.x) {
            const int pr = e / nx, q = e - pr * nx;
            const int ra = 2 * (p0 + pr), rb = ra + 1;
            put_z(e, standalone ? 0.0f : P.h[(size_t)ra * P.nxp + q],
                  (standalone || rb >= ny) ? 0.0f : P.h[(size_t)rb * P.nxp + q]);
        }
        if (!standalone) {
            __shared__ __align__(16) double red[40];
            __shared__ int flag;
            const int pi = find_problem(prefix, count, blockIdx.x, &local);
            const double bs = block_sum_df<256>(s, red);
            if (threadIdx.x == 0) P.partial[local] = bs;
            const int nblk = prefix[pi + 1] - prefix[pi];
            if (last_block(&P.counter[2], nblk, &flag)) {
                const double tot_s = block_sum_array<256>(P.partial, nblk, red);
                if (threadIdx.x == 0) {
                    Scal *sc = P.sc;
                    sc->zth = tot_s;
                    if (sc->init) {
                        sc->beta = 0.0;
                    } else {
                        const double b = tot_s / sc->pth;
                        if (!isfinite(b)) atomicExch(&sc->status, (int)SUPCG_ERR_BREAKDOWN);
                        sc->beta = isfinite(b) ? b : 0.0;
                    }
                    sc->beta_f = (float)sc->beta;
                    P.counter[2] = 0;
                }
            }
        }
    }
}

// Columns pass over the nx/2 + 1 stored frequencies k2: forward FFT along
// the columns, multiply by D = h(w_r) / (nx ny), inverse FFT.
__global__ void __launch_bounds__(256) k_fft_cols(const Prob *__restrict__ probs, const int *__restrict__ prefix,
                                                  int count, int standalone)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int local;
    const Prob &P = probs[find_problem(prefix, count, blockIdx.x, &local)];
    if (!standalone && P.sc->done) return;
    const int nx = P.nx, ny = P.ny, cw = P.fft_cw, hx = nx / 2 + 1;
    float4 *a = reinterpret_cast<float4 *>(smem_raw);
    float4 *b = a + cw * ny;
    const float4 *tw = stage_twiddles(P.fy, b + cw * ny);
    const int c0 = local * cw;
    const int nc = min(cw, hx - c0);
    float4 *S = reinterpret_cast<float4 *>(P.C);
    for (int e = threadIdx.x; e < nc * ny; e += blockDim.x) {
        const int k1 = e / nc, c = e - k1 * nc;   // consecutive threads read consecutive columns
        a[c * ny + k1] = S[(size_t)k1 * hx + c0 + c];
    }
    // D for this thread's elements, read before the transform so that its loads overlap it
    float2 dpre[kFftPerThreadD];
#pragma unroll
    for (int k = 0; k < kFftPerThreadD; ++k) {
        const int e = threadIdx.x + k * blockDim.x;
        dpre[k] = make_float2(0.0f, 0.0f);
        if (e < nc * ny) {
            const int c = e / ny, k1 = e - c * ny;
            dpre[k] = __ldg(P.Dtab + (size_t)min(k1, ny - k1) * hx + c0 + c);   // k2 <= nx/2
        }
    }
    __syncthreads();
    float4 *res = fft_smem_df(a, b, nc, P.fy, tw, false);
    float4 *oth = (res == a) ? b : a;
    auto apply_d = [&](int e, float2 hd) {
        const df D = {hd.x, hd.y};
        const dfc v = dfc_ld(res[e]);
        res[e] = dfc_st(dfc{df_mul(v.r, D), df_mul(v.i, D)});
    };
#pragma unroll
    for (int k = 0; k < kFftPerThreadD; ++k) {   // the prefetched D (compile-time index: registers)
        const int e = threadIdx.x + k * blockDim.x;
        if (e < nc * ny) apply_d(e, dpre[k]);
    }
    for (int e = threadIdx.x + kFftPerThreadD * blockDim.x; e < nc * ny; e += blockDim.x) {
        const int c = e / ny, k1 = e - c * ny;
        apply_d(e, __ldg(P.Dtab + (size_t)min(k1, ny - k1) * hx + c0 + c));   // k2 <= nx/2
    }
    __syncthreads();
    float4 *fin = fft_smem_df(res, oth, nc, P.fy, tw, true);
    for (int e = threadIdx.x; e < nc * ny; e += blockDim.x) {
        const int k1 = e / nc, c = e - k1 * nc;
        S[(size_t)k1 * hx + c0 + c] = fin[c * ny + k1];
    }
}

// D = h(w_r) / (nx ny) on the quarter spectrum (D is even in both frequencies),
// as a double-float pair: Dtab[m1][m2], w_i = 2 pi m_i / N_i, w_r = min(sqrt(w1^2 + w2^2), pi).
__global__ void __launch_bounds__(256) k_fft_dtab(const Prob *__restrict__ probs, const int *__restrict__ prefix,
                                                  int count)
{
    int local;
    const Prob &P = probs[find_problem(prefix, count, blockIdx.x, &local)];
    const int nx = P.nx, ny = P.ny, hx = nx / 2 + 1, hy = ny / 2 + 1;
    const double two_pi = 6.28318530717958647692;
    const double pi_d = 3.14159265358979323846;
    const double scale = 1.0 / ((double)nx * (double)ny);
    for (int k = 0; k < 4; ++k) {
        const long long e = (long long)local * 1024 + k * 256 + threadIdx.x;
        if (e >= (long long)hx * hy) break;
        const int m1 = (int)(e / hx), m2 = (int)(e - (long long)m1 * hx);
        const double w1 = two_pi * m1 / ny, w2 = two_pi * m2 / nx;
        const double wr = fmin(sqrt(w1 * w1 + w2 * w2), pi_d);
        const double v = (wr + P.mu) * (P.rho + (1.0 - P.rho) * cos(wr)) * scale;
        const float vh = (float)v;
        P.Dtab[e] = make_float2(vh, (float)(v - (double)vh));
    }
}

int launch_fft_dtab(const Launch &L)
{
    k_fft_dtab<<<L.blocks, 256, 0, L.st>>>(L.probs, L.prefix, L.count);
    SUPCG_CUDA_TRY(cudaGetLastError());
    return SUPCG_OK;
}

int launch_fft_rows(const Launch &L, int inverse, int standalone, int smem)
{
    int rc = func_attrs_once((const void *)k_fft_rows, 200 * 1024);
    if (rc) return rc;
    k_fft_rows<<<L.blocks, 256, smem, L.st>>>(L.probs, L.prefix, L.count, inverse, standalone);
    SUPCG_CUDA_TRY(cudaGetLastError());
    return SUPCG_OK;
}

int launch_fft_cols(const Launch &L, int standalone, int smem)
{
    int rc = func_attrs_once((const void *)k_fft_cols, 200 * 1024);
    if (rc) return rc;
    k_fft_cols<<<L.blocks, 256, smem, L.st>>>(L.probs, L.prefix, L.count, standalone);
    SUPCG_CUDA_TRY(cudaGetLastError());
    return SUPCG_OK;
}

} // namespace supcg

// ====================================================================
// Allocation-free variant of the preconditioner (supcg_precondition_noalloc).
//
// For callers that cannot allocate device memory at all (for example code
// running where cudaMalloc is forbidden or would break a memory budget
// fixed in advance): the FP64 complex scratch and the twiddle tables live
// in one file-scope device array that the library's module reserves when it
// is loaded, on every GPU that loads the library, until the process exits.
// Every call shares that array, so calls whose work overlaps on the GPU
// (for instance on two streams) race; each call overwrites everything it
// reads before reading it, so nothing needs clearing between calls.
// ====================================================================
namespace supcg {
namespace {

constexpr int kNoAllocMaxSide = 512;                                  // nx, ny <= 512
constexpr size_t kNoAllocMaxPixels = (size_t)kNoAllocMaxSide * kNoAllocMaxSide;
constexpr size_t kNoAllocElems = kNoAllocMaxPixels + 2 * kNoAllocMaxSide;   // C, then twiddles (x, y)

// 4 MiB + 16 KiB of FP64 complex scratch.
static __device__ __align__(256) double2 g_noalloc_scratch[kNoAllocElems];

// Twiddles exp(-2 pi i k / n) for the row length and the column length.
__global__ void k_na_twiddles(double2 *tw_x, int nx, double2 *tw_y, int ny)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nx) {
        double s, c;
        sincospi(-2.0 * k / nx, &s, &c);
        tw_x[k] = make_double2(c, s);
    }
    if (k < ny) {
        double s, c;
        sincospi(-2.0 * k / ny, &s, &c);
        tw_y[k] = make_double2(c, s);
    }
}

// Rows pass on caller buffers (pitch nx): forward g -> C, inverse C -> z.
__global__ void __launch_bounds__(256) k_na_rows(FFTPlan fx, int ny, int rpb, const float *g, float *z, double2 *C,
                                                 int inverse)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nx = fx.n;
    double2 *a = reinterpret_cast<double2 *>(smem_raw);
    double2 *b = a + rpb * nx;
    const int i0 = blockIdx.x * rpb;
    const int nr = min(rpb, ny - i0);
    for (int e = threadIdx.x; e < nr * nx; e += blockDim.x) {
        const size_t gi = (size_t)i0 * nx + e;
        a[e] = inverse ? C[gi] : make_double2((double)g[gi], 0.0);
    }
    __syncthreads();
    double2 *res = fft_smem(a, b, nr, fx, inverse != 0);
    const double scale = 1.0 / ((double)nx * (double)ny);
    for (int e = threadIdx.x; e < nr * nx; e += blockDim.x) {
        const size_t gi = (size_t)i0 * nx + e;
        if (inverse) z[gi] = (float)(res[e].x * scale);
        else C[gi] = res[e];
    }
}

// Columns pass: forward FFT, multiply by D = h(w_r), inverse FFT.
__global__ void __launch_bounds__(256) k_na_cols(FFTPlan fy, int nx, int cw, double mu, double rho, double2 *C)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ny = fy.n;
    double2 *a = reinterpret_cast<double2 *>(smem_raw);
    double2 *b = a + cw * ny;
    const int c0 = blockIdx.x * cw;
    const int nc = min(cw, nx - c0);
    for (int e = threadIdx.x; e < nc * ny; e += blockDim.x) {
        const int k1 = e / nc, c = e - k1 * nc;
        a[c * ny + k1] = C[(size_t)k1 * nx + c0 + c];
    }
    __syncthreads();
    double2 *res = fft_smem(a, b, nc, fy, false);
    double2 *oth = (res == a) ? b : a;
    const double two_pi = 6.28318530717958647692;
    const double pi_d = 3.14159265358979323846;
    for (int e = threadIdx.x; e < nc * ny; e += blockDim.x) {
        const int c = e / ny, k1 = e - c * ny;
        const int k2 = c0 + c;
        const int m1 = min(k1, ny - k1), m2 = min(k2, nx - k2);
        const double w1 = two_pi * m1 / ny, w2 = two_pi * m2 / nx;
        const double wr = fmin(sqrt(w1 * w1 + w2 * w2), pi_d);
        const double hD = (wr + mu) * (rho + (1.0 - rho) * cos(wr));
        res[e] = make_double2(res[e].x * hD, res[e].y * hD);
    }
    __syncthreads();
    double2 *fin = fft_smem(res, oth, nc, fy, true);
    for (int e = threadIdx.x; e < nc * ny; e += blockDim.x) {
        const int k1 = e / nc, c = e - k1 * nc;
        C[(size_t)k1 * nx + c0 + c] = fin[c * ny + k1];
    }
}

// Device address of g_noalloc_scratch, looked up once per device and context: the set-up
// runs again when the device's context has changed since (after cudaDeviceReset the module
// is loaded anew and the array has a new address).
std::mutex g_na_mutex;
struct NaSetup {
    unsigned long long ctx_id;   // context the address belongs to
    double2 *ptr;                // nullptr: not set up
};
NaSetup g_na[64] = {};

typedef CUresult (*PfnCtxGetCurrent)(CUcontext *);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long *);

// Unique ID of the calling thread's current context (the device's primary context,
// which cudaSetDevice makes current and initialises).
int current_ctx_id(int dev, unsigned long long *id)
{
    static PfnCtxGetCurrent get_cur = nullptr;
    static PfnCtxGetId get_id = nullptr;
    if (!get_cur || !get_id) {
        void *p1 = nullptr, *p2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        SUPCG_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p1, 12000, cudaEnableDefault, &q1));
        SUPCG_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuCtxGetId", &p2, 12000, cudaEnableDefault, &q2));
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !p1 || !p2)
            return SUPCG_ERR_CUDA;
        get_cur = reinterpret_cast<PfnCtxGetCurrent>(p1);
        get_id = reinterpret_cast<PfnCtxGetId>(p2);
    }
    SUPCG_CUDA_TRY(cudaSetDevice(dev));
    CUcontext ctx = nullptr;
    if (get_cur(&ctx) != CUDA_SUCCESS || !ctx) return SUPCG_ERR_CUDA;
    if (get_id(ctx, id) != CUDA_SUCCESS) return SUPCG_ERR_CUDA;
    return SUPCG_OK;
}

int noalloc_scratch(double2 **out)
{
    int dev = 0;
    SUPCG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return SUPCG_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_na_mutex);
    unsigned long long id = 0;
    int rc = current_ctx_id(dev, &id);
    if (rc) return rc;
    if (!g_na[dev].ptr || g_na[dev].ctx_id != id) {
        void *p = nullptr;
        // the host-side symbol is only a stand-in: the kernels need this device address
        SUPCG_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        SUPCG_CUDA_TRY(cudaFuncSetAttribute(k_na_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024));
        SUPCG_CUDA_TRY(cudaFuncSetAttribute(k_na_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024));
        g_na[dev].ptr = static_cast<double2 *>(p);
        g_na[dev].ctx_id = id;
    }
    *out = g_na[dev].ptr;
    return SUPCG_OK;
}

int na_factor(int n, int *rad)
{
    int k = 0;
    while (n % 4 == 0 && k < kMaxStages) { rad[k++] = 4; n /= 4; }
    while (n % 2 == 0 && k < kMaxStages) { rad[k++] = 2; n /= 2; }
    for (int p = 3; n > 1 && k < kMaxStages; p += 2)
        while (n % p == 0 && k < kMaxStages) { rad[k++] = p; n /= p; }
    return n == 1 ? k : -1;
}

} // namespace

} // namespace supcg

extern "C" int supcg_precondition_noalloc(int ny, int nx, double mu, double rho, const float *d_g, float *d_z,
                                          void *stream)
{
    using namespace supcg;
    if (!d_g || !d_z || nx < 1 || ny < 1) return SUPCG_ERR_ARG;
    if (nx > kNoAllocMaxSide || ny > kNoAllocMaxSide) return SUPCG_ERR_UNSUPPORTED;
    if (!(rho > 0.5) || !(rho <= 1.0) || !(mu >= 0.0) || !isfinite(mu)) return SUPCG_ERR_PRECOND;
    FFTPlan fx = {}, fy = {};
    fx.n = nx;
    fy.n = ny;
    fx.nst = na_factor(nx, fx.radix);
    fy.nst = na_factor(ny, fy.radix);
    if (fx.nst < 0 || fy.nst < 0) return SUPCG_ERR_UNSUPPORTED;
    double2 *base = nullptr;
    int rc = noalloc_scratch(&base);
    if (rc) return rc;
    double2 *C = base;
    double2 *twx = base + kNoAllocMaxPixels, *twy = twx + kNoAllocMaxSide;
    fx.tw = twx;
    fy.tw = twy;
    cudaStream_t st = (cudaStream_t)stream;
    const int rpb = std::max(1, std::min(16, 4096 / nx));
    const int cw = std::max(1, std::min(16, 4096 / ny));
    const int mx = std::max(nx, ny);
    k_na_twiddles<<<(mx + 255) / 256, 256, 0, st>>>(twx, nx, twy, ny);
    k_na_rows<<<(ny + rpb - 1) / rpb, 256, 2 * rpb * nx * 16, st>>>(fx, ny, rpb, d_g, d_z, C, 0);
    k_na_cols<<<(nx + cw - 1) / cw, 256, 2 * cw * ny * 16, st>>>(fy, nx, cw, mu, rho, C);
    k_na_rows<<<(ny + rpb - 1) / rpb, 256, 2 * rpb * nx * 16, st>>>(fx, ny, rpb, d_g, d_z, C, 1);
    SUPCG_CUDA_TRY(cudaGetLastError());
    return SUPCG_OK;
}
