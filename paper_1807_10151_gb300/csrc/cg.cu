// CG vector algebra of U_PCG (Algorithm 2) and the state handling of
// SupPCG (Algorithm 3): axpys with FP64-reduced inner products, the
// termination test, and staging of caller images into the padded / transposed
// layouts the projector reads.
#include "internal.cuh"

namespace supcg {

constexpr int kVecPerThread = 4;
constexpr int kVecPerBlock = kRedThreads * kVecPerThread;   // elements per block of the vector kernels

// ------------------------------------------------------------ layout staging
__device__ __forceinline__ float load_user(const void *p, size_t i, int storage)
{
    return storage == SUPCG_BF16 ? __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(p)[i])
                                 : reinterpret_cast<const float *>(p)[i];
}

// Caller image [ny][nx] -> x [ny][nxp] and x^T [nx][nyp] (zero padding kept).
__global__ void __launch_bounds__(256) k_stage_in(const Prob *__restrict__ probs, const int *__restrict__ prefix,
                                                  int count, int which)
{
    __shared__ float sh[32][33];
    int local;
    const Prob &P = probs[find_problem(prefix, count, blockIdx.x, &local)];
    const int tiles_j = (P.nx + 31) / 32;
    const int ti = local / tiles_j, tj = local - ti * tiles_j;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += 8) {
        const int i = ti * 32 + r, j = tj * 32 + tx;
        float v = 0.0f;
        if (i < P.ny && j < P.nx) {
            v = load_user(P.in_user, (size_t)i * P.nx + j, P.storage);
            (which ? P.g : P.x)[(size_t)i * P.nxp + j] = v;
            if (!which && P.xlo) P.xlo[(size_t)i * P.nxp + j] = 0.0f;   // x_0 is exactly its FP32 value
            if (!which && P.xm) P.xm[(size_t)i * P.nxp + (P.nx - 1 - j)] = v;
        }
        sh[r][tx] = v;
    }
    if (which) return;
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int j = tj * 32 + r, i = ti * 32 + tx;
        if (j < P.nx && i < P.ny) {
            P.xT[(size_t)j * P.nyp + i] = sh[tx][r];
            if (P.xmT) P.xmT[(size_t)(P.nx - 1 - j) * P.nyp + i] = sh[tx][r];
        }
    }
}

int launch_stage_in(const Launch &L, int which)
{
    k_stage_in<<<L.blocks, 256, 0, L.st>>>(L.probs, L.prefix, L.count, which);
    SUPCG_CUDA_TRY(cudaGetLastError());
    return SUPCG_OK;
}

// Caller sinogram [V][U] -> r (which 0) or bpad (which 1), pitch Up, zero padded.
__global__ void __launch_bounds__(256) k_stage_sino(const Prob *__restrict__ probs, const int *__restrict__ prefix,
                                                    int count, int which)
{
    int local;
    const Prob &P = probs[find_problem(prefix, count, blockIdx.x, &local)];
    float *dst = which ? P.bpad : P.r;
    const size_t tot = (size_t)P.V * P.Up;
    for (size_t e = (size_t)local * kVecPerBlock + threadIdx.x; e < tot && e < (size_t)(local + 1) * kVecPerBlock;
         e += kRedThreads) {
        const int v = (int)(e / P.Up), u = (int)(e - (size_t)v * P.Up);
        const void *src = which ? P.in_user2 : P.in_user;
        dst[e] = (u < P.U) ? load_user(src, (size_t)v * P.U + u, which ? SUPCG_F32 : P.storage) : 0.0f;
    }
}

int launch_stage_sino(const Launch &L, int which)
{
    k_stage_sino<<<L.blocks, kRedThreads, 0, L.st>>>(L.probs, L.prefix, L.count, which);
    SUPCG_CUDA_TRY(cudaGetLastError());
    return SUPCG_OK;
}

// The residual of a while-body without S_TV (x_{k+1/2} = x_k): step 7 moved x by
// alpha p, so r = R x - b moves by alpha q (q = R p, kept in FP64 by the norm pass),
// and f = ||r||^2 (r^2 ||r||^2 + ||x - mu_X||^2 with the Bayesian criterion, completed
// by the backprojector).  Sinogram grid (kVecPerBlock entries per block).
__global__ void __launch_bounds__(kRedThreads) k_rupdate(const Prob *__restrict__ probs,
                                                         const int *__restrict__ prefix, int count)
{
    __shared__ __align__(16) double red[40];
    __shared__ int flag;
    int local;
    const int pi = find_problem(prefix, count, blockIdx.x, &local);
    const Prob &P = probs[pi];
    if (P.sc->done) return;
    const double al = P.sc->alpha;
    const size_t tot = (size_t)P.V * P.Up;   // padding bins stay 0: q is 0 there
    df s = df_make(0.0f);
    for (size_t e = (size_t)local * kVecPerBlock + threadIdx.x; e < tot && e < (size_t)(local + 1) * kVecPerBlock;
         e += kRedThreads) {
        const double rn = fma(al, P.qd[e], P.rd[e]);
        const float rr = (float)rn;
        P.rd[e] = rn;
        P.r[e] = rr;
        df_acc_prod(s, rr, rr);
    }
    const double bs = block_sum_df<kRedThreads>(s, red);
    if (threadIdx.x == 0) P.partial[local] = bs;
    const int nblk = prefix[pi + 1] - prefix[pi];
    if (last_block(&P.counter[6], nblk, &flag)) {
        const double tot_s = block_sum_array<kRedThreads>(P.partial, nblk, red);
        if (threadIdx.x == 0) {
            if (P.r2 > 0.0) P.sc->f_ls = tot_s;
            else P.sc->f = tot_s;
            P.counter[6] = 0;
        }
    }
}

int launch_rupdate(const Launch &L)
{
    k_rupdate<<<L.blocks, kRedThreads, 0, L.st>>>(L.probs, L.prefix, L.count);
    SUPCG_CUDA_TRY(cudaGetLastError());
    return SUPCG_OK;
}

// Padded image (which 0: x, 1: g, 2: z, 3: tbar) -> caller image [ny][nx].
__global__ void __launch_bounds__(256) k_store_out(const Prob *__restrict__ probs, const int *__restrict__ prefix,
                                                   int count, int which)
{
    int local;
    const Prob &P = probs[find_problem(prefix, count, blockIdx.x, &local)];
    const float *src = which == 0 ? P.x : (which == 1 ? P.g : (which == 2 ? P.z : P.tbar));
    const size_t tot = (size_t)P.ny * P.nxp;
    for (size_t e = (size_t)local * kVecPerBlock + threadIdx.x; e < tot && e < (size_t)(local + 1) * kVecPerBlock;
         e += kRedThreads) {
        const int i = (int)(e / P.nxp), j = (int)(e - (size_t)i * P.nxp);
        if (j >= P.nx) continue;
        const size_t o = (size_t)i * P.nx + j;
        if (P.storage == SUPCG_BF16) reinterpret_cast<__nv_bfloat16 *>(P.out_user)[o] = __float2bfloat16_rn(src[e]);
        else reinterpret_cast<float *>(P.out_user)[o] = src[e];
    }
}

int launch_store_out(const Launch &L, int which)
{
    k_store_out<<<L.blocks, kRedThreads, 0, L.st>>>(L.probs, L.prefix, L.count, which);
    SUPCG_CUDA_TRY(cudaGetLastError());
    return SUPCG_OK;
}

// ------------------------------------------------------------ Algorithm 2 steps
// Steps 3-4 (beta from z^T h computed earlier) and the g^T p half of step 6:
//   p <- -z + beta p ;  partial g^T p.   In steps 2-7 of Algorithm 3 beta = 0.
// p = -z + beta p (Algorithm 2 step 4; z = g when M = I), g^T p (step 6) and
// ||p||^2 (for h = A p under the Bayesian criterion), on 32 x 32 tiles so that
// the same pass writes p^T for the projector; the last block stores the sums
// and beta.  Launched with the transpose's tile grid.
__global__ void __launch_bounds__(256) k_pupdate(const Prob *__restrict__ probs, const int *__restrict__ prefix,
                                                 int count)
{
    __shared__ float sh[32][33];
    __shared__ __align__(16) double red[40];
    __shared__ int flag;
    int local;
    const int pi = find_problem(prefix, count, blockIdx.x, &local);
    const Prob &P = probs[pi];
    if (P.sc->done) return;
    const float beta = P.sc->init ? 0.0f : P.sc->beta_f;
    const float *z = P.precond ? P.z : P.g;   // M = I: z = g
    const int tiles_j = (P.nx + 31) / 32;
    const int ti = local / tiles_j, tj = local - ti * tiles_j;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    df s = df_make(0.0f), spp = df_make(0.0f);   // g^T p and ||p||^2 (exact products, double-float sums)
    // the thread's four rows: every load issued before the first store
    float pv[4], zv[4], gv[4], glv[4];
    bool in[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = ti * 32 + ty + 8 * q, j = tj * 32 + tx;
        in[q] = i < P.ny && j < P.nx;   // the padding of p stays 0
        const size_t e = in[q] ? (size_t)i * P.nxp + j : 0;
        pv[q] = in[q] ? P.p[e] : 0.0f;
        zv[q] = in[q] ? z[e] : 0.0f;
        gv[q] = in[q] ? P.g[e] : 0.0f;
        glv[q] = in[q] ? P.glo[e] : 0.0f;   // the gradient's low part (written by the backprojector)
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int r = ty + 8 * q;
        float pn = 0.0f;
        if (in[q]) {
            pn = __fmaf_rn(beta, pv[q], -zv[q]);
            P.p[(size_t)(ti * 32 + r) * P.nxp + tj * 32 + tx] = pn;
            if (P.pm) P.pm[(size_t)(ti * 32 + r) * P.nxp + (P.nx - 1 - (tj * 32 + tx))] = pn;
            df_acc_prod(s, gv[q], pn);
            df_acc_prod(s, glv[q], pn);
            df_acc_prod(spp, pn, pn);
        }
        sh[r][tx] = pn;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int j = tj * 32 + r, i = ti * 32 + tx;
        if (j < P.nx && i < P.ny) {
            P.pT[(size_t)j * P.nyp + i] = sh[tx][r];
            if (P.pmT) P.pmT[(size_t)(P.nx - 1 - j) * P.nyp + i] = sh[tx][r];
        }
    }
    double bs, bp;
    block_sum_df2<256>(s, spp, red, &bs, &bp);
    const int nblk = prefix[pi + 1] - prefix[pi];
    if (threadIdx.x == 0) {
        P.partial[local] = bs;
        P.partial[nblk + local] = bp;
    }
    if (last_block(&P.counter[1], nblk, &flag)) {
        double tot_s, tot_p;
        block_sum_array2<256>(P.partial, P.partial + nblk, nblk, red, &tot_s, &tot_p);
        if (threadIdx.x == 0) {
            P.sc->gtp = tot_s;
            P.sc->pp = tot_p;
            if (P.sc->init) {   // steps 2-7 of Algorithm 3: beta = 0
                P.sc->beta = 0.0;
                P.sc->beta_f = 0.0f;
            }
            P.counter[1] = 0;
        }
    }
}

// Gray level mu_X of the Bayesian criterion (Eq. (2.3)) estimated from the data:
// every view's sum_u b ds approximates the image integral, so the mean over views
// divided by the image area is the image average (sc->muX = gray_scale sum b).
__global__ void __launch_bounds__(kRedThreads) k_gray(const Prob *__restrict__ probs, const int *__restrict__ prefix,
                                                      int count)
{
    __shared__ __align__(16) double red[40];
    __shared__ int flag;
    int local;
    const int pi = find_problem(prefix, count, blockIdx.x, &local);
    const Prob &P = probs[pi];
    const size_t tot = (size_t)P.V * P.Up;   // bpad: zero padding beyond U
    double s = 0.0;
    for (size_t e = (size_t)local * kVecPerBlock + threadIdx.x; e < tot && e < (size_t)(local + 1) * kVecPerBlock;
         e += kRedThreads)
        s += (double)P.bpad[e];
    const double bs = block_sum<kRedThreads>(s, red);
    if (threadIdx.x == 0) P.partial[local] = bs;
    const int nblk = prefix[pi + 1] - prefix[pi];
    if (last_block(&P.counter[5], nblk, &flag)) {
        const double sum = block_sum_array<kRedThreads>(P.partial, nblk, red);
        if (threadIdx.x == 0) {
            P.sc->muX = sum * P.gray_scale;
            P.counter[5] = 0;
        }
    }
}

int launch_gray(const Launch &L)
{
    k_gray<<<L.blocks, kRedThreads, 0, L.st>>>(L.probs, L.prefix, L.count);
    SUPCG_CUDA_TRY(cudaGetLastError());
    return SUPCG_OK;
}

int launch_pupdate(const Launch &L)
{
    k_pupdate<<<L.blocks, 256, 0, L.st>>>(L.probs, L.prefix, L.count);
    SUPCG_CUDA_TRY(cudaGetLastError());
    return SUPCG_OK;
}

// Step 3 of Algorithm 2: beta = z^T h / p^T h (p, h of the previous step).
// With M = I, z is g.
__global__ void __launch_bounds__(kRedThreads) k_beta(const Prob *__restrict__ probs,
                                                      const int *__restrict__ prefix, int count)
{
    __shared__ __align__(16) double red[40];
    __shared__ int flag;
    int local;
    const int pi = find_problem(prefix, count, blockIdx.x, &local);
    const Prob &P = probs[pi];
    if (P.sc->done) return;
    const float *z = P.precond ? P.z : P.g;
    const size_t tot = (size_t)P.ny * P.nxp;
    df s = df_make(0.0f);
    for (size_t e = (size_t)local * kVecPerBlock + threadIdx.x; e < tot && e < (size_t)(local + 1) * kVecPerBlock;
         e += kRedThreads)
        df_acc_prod(s, z[e], P.h[e]);
    const double bs = block_sum_df<kRedThreads>(s, red);
    if (threadIdx.x == 0) P.partial[local] = bs;
    const int nblk = prefix[pi + 1] - prefix[pi];
    if (last_block(&P.counter[2], nblk, &flag)) {
        const double tot_s = block_sum_array<kRedThreads>(P.partial, nblk, red);
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

int launch_beta(const Launch &L)
{
    k_beta<<<L.blocks, kRedThreads, 0, L.st>>>(L.probs, L.prefix, L.count);
    SUPCG_CUDA_TRY(cudaGetLastError());
    return SUPCG_OK;
}

// Start of a while-body of Algorithm 3: the condition f(x_{k-1/2}) > eps
// (step 10) and, when it holds, step 7 of the previous U_PCG call
// (x_k = x_{k-1/2} + alpha p_{k-1}), deferred to here so that x holds the
// returned image x_{k-1/2} whenever the loop stops.  With the low part xlo the
// update is x + xlo <- x + xlo + alpha p in double-float arithmetic (alpha split
// into two FP32 parts, the product's rounding error kept), so that the iterate
// does not lose the low bits of alpha p to FP32 rounding at every step.
__global__ void __launch_bounds__(kRedThreads) k_xupdate(const Prob *__restrict__ probs,
                                                         const int *__restrict__ prefix, int count)
{
    int local;
    const Prob &P = probs[find_problem(prefix, count, blockIdx.x, &local)];
    Scal *sc = P.sc;
    if (sc->done) return;
    const bool stop = !(sc->f > sc->eps) || sc->status != 0;
    if (stop) {
        // every block takes the same decision from the same scalars; block 0 records it
        // after all blocks have read it (done is read again only by later launches)
        if (local == 0 && threadIdx.x == 0) sc->done = 2;   // 2: set during this launch
        return;
    }
    const float al = sc->alpha_h, al_lo = sc->alpha_l;   // alpha = al + al_lo to about 2^-48
    const size_t tot = (size_t)P.ny * P.nxp;   // a multiple of 4: rows are padded to 16 bytes
    float *tr = P.trace ? P.trace + (size_t)sc->k * P.ny * P.nx : nullptr;
    // one float4 of x and of p per thread (kVecPerBlock = 4 x kRedThreads elements per block)
    const size_t e4 = (size_t)local * kRedThreads + threadIdx.x;
    if (4 * e4 < tot) {
        const float4 pv = reinterpret_cast<const float4 *>(P.p)[e4];
        float4 xv = reinterpret_cast<const float4 *>(P.x)[e4];
        if (P.xlo) {
            float4 lv = reinterpret_cast<const float4 *>(P.xlo)[e4];
            float *xs = &xv.x, *ls = &lv.x;
            const float *ps = &pv.x;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                df prod = df_prod(al, ps[q]);                  // al p exactly, then + al_lo p
                prod.l = __fmaf_rn(al_lo, ps[q], prod.l);
                const df v = df_add(df{xs[q], ls[q]}, prod);
                xs[q] = v.h;
                ls[q] = v.l;
            }
            reinterpret_cast<float4 *>(P.xlo)[e4] = lv;
        } else {
            xv.x = __fmaf_rn(al, pv.x, xv.x);
            xv.y = __fmaf_rn(al, pv.y, xv.y);
            xv.z = __fmaf_rn(al, pv.z, xv.z);
            xv.w = __fmaf_rn(al, pv.w, xv.w);
        }
        reinterpret_cast<float4 *>(P.x)[e4] = xv;
        if (tr) {
            const float v4[4] = {xv.x, xv.y, xv.z, xv.w};
            for (int q = 0; q < 4; ++q) {
                const size_t e = 4 * e4 + q;
                const int i = (int)(e / P.nxp), j = (int)(e - (size_t)i * P.nxp);
                if (j < P.nx) tr[(size_t)i * P.nx + j] = v4[q];
            }
        }
    }
}

// The iterates and tbar of every problem of a batched learned solve, back to back as
// the network's input batch: xs, ts [count][ny][nx].  Every problem has the network's
// image size and rows padded to nothing (nx a multiple of 4), so a problem's image is
// one contiguous block; one float4 per thread, launched on the vector kernels' grid.
__global__ void __launch_bounds__(kRedThreads) k_gather_xt(const Prob *__restrict__ probs, const int *__restrict__ prefix,
                                                           int count, float *__restrict__ xs, float *__restrict__ ts)
{
    int local;
    const int pi = find_problem(prefix, count, blockIdx.x, &local);
    const Prob &P = probs[pi];
    if (P.sc->done) return;
    const size_t n = (size_t)P.ny * P.nx;
    const size_t e4 = (size_t)local * kRedThreads + threadIdx.x;
    if (4 * e4 < n) {
        reinterpret_cast<float4 *>(xs + pi * n)[e4] = reinterpret_cast<const float4 *>(P.x)[e4];
        reinterpret_cast<float4 *>(ts + pi * n)[e4] = reinterpret_cast<const float4 *>(P.tbar)[e4];
    }
}

int launch_gather_xt(const Launch &L, float *xs, float *ts)
{
    k_gather_xt<<<L.blocks, kRedThreads, 0, L.st>>>(L.probs, L.prefix, L.count, xs, ts);
    SUPCG_CUDA_TRY(cudaGetLastError());
    return SUPCG_OK;
}

int launch_xupdate(const Launch &L)
{
    k_xupdate<<<L.blocks, kRedThreads, 0, L.st>>>(L.probs, L.prefix, L.count);
    SUPCG_CUDA_TRY(cudaGetLastError());
    return SUPCG_OK;
}

} // namespace supcg
