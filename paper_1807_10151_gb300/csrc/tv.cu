// Total variation, its nonascending vector and S_TV (Sec. 3.1, Algorithm 1).
//
//   TV(y) = sum_{i<ny-1, j<nx-1} sqrt((y_ij - y_i+1,j)^2 + (y_ij - y_i,j+1)^2)
//   tbar_p = -dTV/dy_p where the partial exists (every TV term containing y_p
//            has a nonzero root, i.e. not both of its differences are 0), else 0
//   t = tbar / ||tbar||  (0 when tbar = 0)
//
// S_TV runs as one cooperative launch per call: each problem owns a fixed set
// of co-resident blocks that meet at bounded device barriers, so the
// data-dependent backtracking loop (repeat ... until TV(y~) <= TV(y)) runs
// on the device without returning to the host.  Every block sums the
// per-block FP64 partials in the same order, so all blocks take the same
// accept / reject decision.
#include "internal.cuh"

namespace supcg {

constexpr int kTvThreads = 256;

// The seven values of y (pitch ld) that tbar at pixel (i, j) depends on: the pixel,
// its lower and right neighbours, the upper row's pixel and its right neighbour,
// the left pixel and its lower neighbour (0 where the term they belong to does not
// exist).  Loading them apart from the arithmetic lets a thread issue the loads of
// several pixels before it waits for any.
struct Nb7 {
    float c, d, r, u, ur, l, ld;
};
__device__ __forceinline__ Nb7 nb7_load(const float *__restrict__ y, int ld, int ny, int nx, int i, int j)
{
    Nb7 v = {};
    const size_t p = (size_t)i * ld + j;
    v.c = y[p];
    if (i + 1 < ny && j + 1 < nx) {
        v.d = y[p + ld];
        v.r = y[p + 1];
    }
    if (i >= 1 && j + 1 < nx) {
        v.u = y[p - ld];
        v.ur = y[p - ld + 1];
    }
    if (j >= 1 && i + 1 < ny) {
        v.l = y[p - 1];
        v.ld = y[p + ld - 1];
    }
    return v;
}

// tbar at pixel (i, j) from its seven values; *Tb receives the root of the TV term
// whose base is (i, j) (0 if that term does not exist).
__device__ __forceinline__ float tbar_from(const Nb7 &v, int ny, int nx, int i, int j, float *Tb)
{
    float g = 0.0f;
    bool undef = false;
    float tb = 0.0f;
    const float yc = v.c;
    if (i + 1 < ny && j + 1 < nx) {
        const float a = yc - v.d, b = yc - v.r;
        if (a == 0.0f && b == 0.0f) undef = true;
        else {
            const float T = sqrtf(a * a + b * b);
            tb = T;
            g += (a + b) / T;
        }
    }
    if (i >= 1 && j + 1 < nx) {
        const float yu = v.u;
        const float a = yu - yc, b = yu - v.ur;
        if (a == 0.0f && b == 0.0f) undef = true;
        else g -= a / sqrtf(a * a + b * b);
    }
    if (j >= 1 && i + 1 < ny) {
        const float yl = v.l;
        const float a = yl - v.ld, b = yl - yc;
        if (a == 0.0f && b == 0.0f) undef = true;
        else g -= b / sqrtf(a * a + b * b);
    }
    *Tb = tb;
    return undef ? 0.0f : -g;
}

// tbar at pixel (i, j) of y (pitch ld); *Tb as for tbar_from.
__device__ __forceinline__ float tbar_at(const float *__restrict__ y, int ld, int ny, int nx, int i, int j,
                                         float *Tb)
{
    return tbar_from(nb7_load(y, ld, ny, nx, i, j), ny, nx, i, j, Tb);
}

// A thread's pixels e0, e0 + stride, ... of an ny x nx image as (i, j), stepped
// without a division per pixel; S_TV's passes take them kStvGroup at a time, all
// of a group's loads issued before its arithmetic.
constexpr int kStvGroup = 2;
struct PixWalk {
    int i, j, si, sj, nx;
    __device__ PixWalk(int e0, int stride, int nx_) : nx(nx_)
    {
        i = e0 / nx;
        j = e0 - i * nx;
        si = stride / nx;
        sj = stride - si * nx;
    }
    __device__ __forceinline__ void next()
    {
        j += sj;
        i += si;
        if (j >= nx) {
            j -= nx;
            ++i;
        }
    }
};

// Root of the TV term based at (i, j) of y~ = y + c tbar (term must exist).
__device__ __forceinline__ float trial_term(const float *__restrict__ y, const float *__restrict__ t, int ld,
                                            int i, int j, float c)
{
    const size_t p = (size_t)i * ld + j;
    const float yc = __fmaf_rn(c, t[p], y[p]);
    const float yd = __fmaf_rn(c, t[p + ld], y[p + ld]);
    const float yr = __fmaf_rn(c, t[p + 1], y[p + 1]);
    const float a = yc - yd, b = yc - yr;
    return sqrtf(a * a + b * b);
}

// y <- y + c t at element p of the iterate: in double-float arithmetic on the pair
// (x, xlo) when the low part exists (the exact product c t added to it), else one
// FP32 FMA.  Returns the new FP32 image value x = RN(x + xlo).
__device__ __forceinline__ float x_step(float *__restrict__ x, float *__restrict__ xlo, size_t p, float c, float t,
                                        float *lo_out = nullptr)
{
    if (!xlo) {
        const float v = __fmaf_rn(c, t, x[p]);
        x[p] = v;
        if (lo_out) *lo_out = 0.0f;
        return v;
    }
    const df v = df_add(df{x[p], xlo[p]}, df_prod(c, t));
    x[p] = v.h;
    xlo[p] = v.l;
    if (lo_out) *lo_out = v.l;
    return v.h;
}

// Standalone TV and tbar of P.x (one image per problem): writes P.tbar and
// sc->tv_k = TV, sc->snorm2 = ||tbar||^2.
__global__ void __launch_bounds__(kTvThreads) k_tv_tbar(const Prob *__restrict__ probs, const int *__restrict__ prefix,
                                                        int count)
{
    __shared__ __align__(16) double red[40];
    __shared__ int flag;
    int local;
    const int pi = find_problem(prefix, count, blockIdx.x, &local);
    const Prob &P = probs[pi];
    const int nblk = prefix[pi + 1] - prefix[pi];
    const long long n = (long long)P.ny * P.nx;
    df s_tv = df_make(0.0f), s_nn = df_make(0.0f);   // double-float sums, FP64 per thread
    for (long long e = (long long)local * kTvThreads + threadIdx.x; e < n; e += (long long)nblk * kTvThreads) {
        const int i = (int)(e / P.nx), j = (int)(e - (long long)i * P.nx);
        float Tb;
        const float tb = tbar_at(P.x, P.nxp, P.ny, P.nx, i, j, &Tb);
        P.tbar[(size_t)i * P.nxp + j] = tb;
        df_acc(s_tv, Tb);
        df_acc_prod(s_nn, tb, tb);
    }
    double btv, bnn;
    block_sum_df2<kTvThreads>(s_tv, s_nn, red, &btv, &bnn);
    if (threadIdx.x == 0) {
        P.partial[local] = btv;
        P.partial[nblk + local] = bnn;
    }
    if (last_block(&P.counter[3], nblk, &flag)) {
        double tv, nn;
        block_sum_array2<kTvThreads>(P.partial, P.partial + nblk, nblk, red, &tv, &nn);
        if (threadIdx.x == 0) {
            P.sc->tv_k = tv;
            P.sc->snorm2 = nn;
            P.counter[3] = 0;
        }
    }
}

int launch_tv_tbar(const Launch &L)
{
    k_tv_tbar<<<L.blocks, kTvThreads, 0, L.st>>>(L.probs, L.prefix, L.count);
    SUPCG_CUDA_TRY(cudaGetLastError());
    return SUPCG_OK;
}

// Sum of the block partials of one phase, identical in every block (per-thread values
// in FP64 or as double-float pairs).
__device__ __forceinline__ double phase_sum_of(const Prob &P, int nb, int slot, int local, double bs, double *red,
                                               int *flag, bool *ok);
__device__ __forceinline__ double phase_sum(const Prob &P, int nb, int slot, int local, df v, double *red,
                                            int *flag, bool *ok)
{
    return phase_sum_of(P, nb, slot, local, block_sum_df<kTvThreads>(v, red), red, flag, ok);
}
__device__ __forceinline__ double phase_sum(const Prob &P, int nb, int slot, int local, double v, double *red,
                                            int *flag, bool *ok)
{
    return phase_sum_of(P, nb, slot, local, block_sum<kTvThreads>(v, red), red, flag, ok);
}
__device__ __forceinline__ double phase_sum_of(const Prob &P, int nb, int slot, int local, double bs, double *red,
                                               int *flag, bool *ok)
{
    if (threadIdx.x == 0) P.partial[(size_t)slot * nb + local] = bs;
    *ok = coop_barrier(P.bar, nb + P.bar_extra, &P.sc->status, flag, P.wait_limit);
    if (!*ok) return 0.0;
    return block_sum_array<kTvThreads>(P.partial + (size_t)slot * nb, nb, red);
}

// S_TV(x, l, a, gamma, K), Algorithm 1, in place on P.x (one cooperative launch).
// trials_out (nullable): [count][K] trials of every nonascending step.  dir (nullable):
// the learned proposals, [count][ny][nx] (every problem of the launch has the same size).
// Also writes the displacement d = x_{k+1/2} - x_k in the forward projector's layouts
// (P.d, P.dT and, with mirror pairs, P.dm, P.dmT), which a while-body projects to move
// the residual.
__global__ void __launch_bounds__(kTvThreads, 3) k_stv(const Prob *__restrict__ probs, const int *__restrict__ prefix,
                                                    int count, int K_arg, double a_arg, double gamma_arg,
                                                    long long max_trials, int *trials_out, int want_snorm,
                                                    const float *__restrict__ dir_all)
{
    const float *dir = dir_all;
    __shared__ __align__(16) double red[40];
    __shared__ int flag;
    __shared__ double sh_inv;   // grid-uniform FP64 scalars: computed by thread 0, read by all
    __shared__ float sh_c;
    __shared__ float sh_t[32][33];   // tile transposes of d
    bool d_done = false;             // the last step wrote d
    int local;
    const int pi = find_problem(prefix, count, blockIdx.x, &local);
    const Prob &P = probs[pi];
    Scal *sc = P.sc;
    if (sc->done) return;
    // a parameter sweep gives every problem its own K, a, gamma
    const int K = P.stv_own ? P.stv_K : K_arg;
    const double a = P.stv_own ? P.stv_a : a_arg, gamma = P.stv_own ? P.stv_gamma : gamma_arg;
    const int nb = prefix[pi + 1] - prefix[pi];
    const int nx = P.nx, ny = P.ny, ld = P.nxp;
    const int n = ny * nx;   // < 2^31 (each side <= 16384)
    const int stride = nb * kTvThreads;
    const int e0 = local * kTvThreads + threadIdx.x;
    float *x = P.x;
    float *xl = P.xlo;   // low part of the iterate (null: FP32 updates)
    // a batched learned solve passes the proposals of all problems back to back ([count][ny][nx])
    if (dir) dir += (size_t)pi * ny * nx;
    float *tb = P.tbar;
    long long ell = sc->ell;
    // a^ell, carried from trial to trial and from call to call (Scal::apow); thread 0's, kept
    // in shared memory so that it takes no registers through the passes
    __shared__ double sh_apow;
    __shared__ int sh_apow_ok;
    if (threadIdx.x == 0) {
        sh_apow_ok = sc->apow_ok && sc->apow_ell == ell && sc->apow_a == a;
        sh_apow = sh_apow_ok ? sc->apow : 0.0;
    }
    long long total_trials = 0;
    double tv_first = 0.0, tv_last = 0.0;
    int slot = 0;   // partial buffers alternate between two slots (pairs of slots for 2-value phases)
    bool ok = true;
    // x_k is saved before the steps unless one plain step (K = 1) gives d as c tbar itself
    const bool saved = want_snorm || dir || K != 1;
    // d on the 32 x 32 tiles this block owns, in the row layout and transposed (and mirrored
    // with mirror pairs).  step: the last step y <- y + c tbar is taken here, pixel by pixel
    // (no block reads another's pixels after it, so no grid barrier follows); zero: no step
    // moved x.  Otherwise d = x - x_k from the copy saved before the steps, which a grid
    // barrier separates from here.
    auto write_d = [&](bool step, bool zero, float c) {
        const int tiles_j = (nx + 31) / 32, tiles = ((ny + 31) / 32) * tiles_j;
        const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 256 threads: 32 x 8
        for (int tile = local; tile < tiles; tile += nb) {
            const int ti = tile / tiles_j, tj = tile - ti * tiles_j;
            for (int r = ty; r < 32; r += 8) {
                const int i = ti * 32 + r, j = tj * 32 + tx;
                float dv = 0.0f;
                if (i < ny && j < nx) {
                    const size_t p = (size_t)i * ld + j;
                    float v, vl;
                    if (step) {
                        const float t = tb[p];
                        v = x_step(x, xl, p, c, t, &vl);
                        if (!saved) dv = __fmul_rn(c, t);
                    } else {
                        v = x[p];
                        vl = xl ? xl[p] : 0.0f;
                    }
                    if (saved && !zero) dv = __fadd_rn(__fsub_rn(v, P.z[p]), __fsub_rn(vl, P.g[p]));
                    P.d[p] = dv;
                    if (P.dm) P.dm[(size_t)i * ld + (nx - 1 - j)] = dv;
                }
                sh_t[r][tx] = dv;
            }
            __syncthreads();
            for (int r = ty; r < 32; r += 8) {
                const int j = tj * 32 + r, i = ti * 32 + tx;
                if (j < nx && i < ny) {
                    P.dT[(size_t)j * P.nyp + i] = sh_t[tx][r];
                    if (P.dmT) P.dmT[(size_t)(nx - 1 - j) * P.nyp + i] = sh_t[tx][r];
                }
            }
            __syncthreads();
        }
    };

    // the iterate before the steps, high part in z and low part in g (both are recomputed
    // after S_TV in a while-body), for ||s_k||^2 of the log and for d
    if (saved)
        for (int e = e0; e < n; e += stride) {
            const int i = e / nx, j = e - i * nx;
            const size_t p = (size_t)i * ld + j;
            P.z[p] = x[p];
            P.g[p] = xl ? xl[p] : 0.0f;
        }

    // Learned direction (dir != null, pitch nx): accepted only when nonascending for TV,
    // i.e. when the one-sided directional derivative D_TV(x; dir) is negative; then one
    // step of length 2^-j gamma sum_{i<K} a^(l+i) (j = rejected trials so far; halving,
    // since a long step shrinks too slowly by factors of a near 1) replaces the K steps of
    // Algorithm 1, and l advances by K + j, so ||s_k|| <= K gamma a^(l_k) as in Theorem 1.
    // Otherwise the K plain steps run.
    bool plain = true;
    if (dir) {
        double s_nn = 0.0, s_dd = 0.0, s_tv = 0.0;
        for (int e = e0; e < n; e += stride) {
            const int i = e / nx, j = e - i * nx;
            const size_t p = (size_t)i * ld + j;
            const size_t q = (size_t)i * nx + j;
            const float tp = dir[q];
            s_nn += (double)tp * (double)tp;
            if (i + 1 < ny && j + 1 < nx) {
                const float a1 = x[p] - x[p + ld], b1 = x[p] - x[p + 1];
                const float ta = tp - dir[q + nx], tb = tp - dir[q + 1];
                if (a1 == 0.0f && b1 == 0.0f) {
                    s_dd += (double)sqrtf(ta * ta + tb * tb);
                } else {
                    const double T = (double)sqrtf(a1 * a1 + b1 * b1);
                    s_tv += T;
                    s_dd += ((double)a1 * ta + (double)b1 * tb) / T;
                }
            }
        }
        {
            const double v1 = block_sum<kTvThreads>(s_nn, red);
            const double v2 = block_sum<kTvThreads>(s_dd, red);
            const double v3 = block_sum<kTvThreads>(s_tv, red);
            if (threadIdx.x == 0) {
                P.partial[(size_t)8 * nb + local] = v1;
                P.partial[(size_t)9 * nb + local] = v2;
                P.partial[(size_t)10 * nb + local] = v3;
            }
            ok = coop_barrier(P.bar, nb + P.bar_extra, &sc->status, &flag, P.wait_limit);
            if (ok) {
                s_nn = block_sum_array<kTvThreads>(P.partial + (size_t)8 * nb, nb, red);
                s_dd = block_sum_array<kTvThreads>(P.partial + (size_t)9 * nb, nb, red);
                s_tv = block_sum_array<kTvThreads>(P.partial + (size_t)10 * nb, nb, red);
            }
        }
        if (ok && s_dd < 0.0 && s_nn > 0.0) {
            plain = false;
            // the step scalars are the same in every thread: thread 0 evaluates the FP64
            // functions and the block reads the result (the FP64 pipe is narrow)
            if (threadIdx.x == 0) sh_inv = rsqrt_fp64(s_nn);
            long long j = 0;
            float c = 0.0f;
            double tv_t = 0.0;
            for (;;) {
                if (j >= max_trials) {
                    if (local == 0 && threadIdx.x == 0) atomicExch(&sc->status, (int)SUPCG_ERR_BACKTRACK);
                    ok = false;
                    break;
                }
                if (threadIdx.x == 0) {
                    const double geo = (a == 1.0) ? (double)K : (1.0 - pow(a, (double)K)) / (1.0 - a);
                    sh_c = (float)(ldexp(gamma * pow(a, (double)ell) * geo, -(int)min(j, 2000ll)) * sh_inv);
                }
                __syncthreads();
                c = sh_c;
                ++j;
                double sacc = 0.0;
                for (int e = e0; e < n; e += stride) {
                    const int i = e / nx, jj = e - i * nx;
                    if (i + 1 < ny && jj + 1 < nx) {
                        const size_t p = (size_t)i * ld + jj, q = (size_t)i * nx + jj;
                        const float yc = __fmaf_rn(c, dir[q], x[p]);
                        const float yd = __fmaf_rn(c, dir[q + nx], x[p + ld]);
                        const float yr = __fmaf_rn(c, dir[q + 1], x[p + 1]);
                        const float a1 = yc - yd, b1 = yc - yr;
                        sacc += (double)sqrtf(a1 * a1 + b1 * b1);
                    }
                }
                tv_t = phase_sum(P, nb, slot, local, sacc, red, &flag, &ok);
                slot ^= 1;
                if (!ok) break;
                if (tv_t <= s_tv) break;
            }
            if (ok) {
                for (int e = e0; e < n; e += stride) {
                    const int i = e / nx, jj = e - i * nx;
                    (void)x_step(x, xl, (size_t)i * ld + jj, c, dir[(size_t)i * nx + jj]);
                }
                ok = coop_barrier(P.bar, nb + P.bar_extra, &sc->status, &flag, P.wait_limit);
                ell += (long long)K + (j - 1);
                if (threadIdx.x == 0) sh_apow_ok = 0;
                total_trials = j;
                tv_first = s_tv;
                tv_last = tv_t;
                if (local == 0 && threadIdx.x == 0) sc->n_learned += 1;
            }
        } else if (local == 0 && threadIdx.x == 0) {
            sc->n_fallback += 1;
        }
    }

    for (int step = 0; plain && step < K && ok; ++step) {
        // t in the nonascending set at y (Sec. 3.1)
        df d_tv = df_make(0.0f), d_nn = df_make(0.0f);   // double-float sums, FP64 per thread
        for (PixWalk w(e0, stride, nx); w.i < ny;) {
            int gi[kStvGroup], gj[kStvGroup];
            Nb7 v[kStvGroup];
#pragma unroll
            for (int q = 0; q < kStvGroup; ++q) {
                gi[q] = w.i;
                gj[q] = w.j;
                if (w.i < ny) v[q] = nb7_load(x, ld, ny, nx, w.i, w.j);
                w.next();
            }
#pragma unroll
            for (int q = 0; q < kStvGroup; ++q) {
                if (gi[q] < ny) {
                    float Tb;
                    const float t = tbar_from(v[q], ny, nx, gi[q], gj[q], &Tb);
                    tb[(size_t)gi[q] * ld + gj[q]] = t;
                    df_acc(d_tv, Tb);
                    df_acc_prod(d_nn, t, t);
                }
            }
        }
        double s_tv, s_nn;
        // two sums through one barrier: slots 2*slot and 2*slot+1
        {
            double b1, b2;
            block_sum_df2<kTvThreads>(d_tv, d_nn, red, &b1, &b2);
            if (threadIdx.x == 0) {
                P.partial[(size_t)(4 + 2 * slot) * nb + local] = b1;
                P.partial[(size_t)(5 + 2 * slot) * nb + local] = b2;
            }
            ok = coop_barrier(P.bar, nb + P.bar_extra, &sc->status, &flag, P.wait_limit);
            if (!ok) break;
            block_sum_array2<kTvThreads>(P.partial + (size_t)(4 + 2 * slot) * nb, P.partial + (size_t)(5 + 2 * slot) * nb,
                                         nb, red, &s_tv, &s_nn);
            slot ^= 1;
        }
        const double tv_y = s_tv;
        if (step == 0) tv_first = tv_y;
        // the step scalars are the same in every thread: thread 0 evaluates the FP64
        // functions and the block reads the result (the FP64 pipe is narrow)
        if (threadIdx.x == 0) sh_inv = (s_nn > 0.0) ? rsqrt_fp64(s_nn) : 0.0;
        long long trials = 0;
        float c = 0.0f;
        double tv_t = 0.0;
        for (;;) {
            if (trials >= max_trials) {
                if (local == 0 && threadIdx.x == 0) atomicExch(&sc->status, (int)SUPCG_ERR_BACKTRACK);
                ok = false;
                break;
            }
            if (threadIdx.x == 0) {
                const double ap = sh_apow_ok ? sh_apow : pow(a, (double)ell);
                sh_c = (float)(gamma * ap * sh_inv);   // gamma a^l / ||tbar||
                sh_apow = ap * a;                      // a^(l + 1), for the next trial
                sh_apow_ok = 1;
            }
            __syncthreads();
            c = sh_c;                                                                     // y~ = y + c tbar
            ++ell;
            ++trials;
            df s = df_make(0.0f);
            for (PixWalk w(e0, stride, nx); w.i < ny;) {
                float yv[kStvGroup][3], tv[kStvGroup][3];
                bool in[kStvGroup];
#pragma unroll
                for (int q = 0; q < kStvGroup; ++q) {
                    in[q] = w.i + 1 < ny && w.j + 1 < nx;
                    if (in[q]) {
                        const size_t p = (size_t)w.i * ld + w.j;
                        yv[q][0] = x[p];
                        yv[q][1] = x[p + ld];
                        yv[q][2] = x[p + 1];
                        tv[q][0] = tb[p];
                        tv[q][1] = tb[p + ld];
                        tv[q][2] = tb[p + 1];
                    }
                    w.next();
                }
#pragma unroll
                for (int q = 0; q < kStvGroup; ++q) {
                    if (in[q]) {   // the root of the TV term of y~ = y + c tbar based at the pixel
                        const float yc = __fmaf_rn(c, tv[q][0], yv[q][0]);
                        const float yd = __fmaf_rn(c, tv[q][1], yv[q][1]);
                        const float yr = __fmaf_rn(c, tv[q][2], yv[q][2]);
                        const float a1 = yc - yd, b1 = yc - yr;
                        df_acc(s, sqrtf(a1 * a1 + b1 * b1));
                    }
                }
            }
            tv_t = phase_sum(P, nb, slot, local, s, red, &flag, &ok);
            slot ^= 1;
            if (!ok) break;
            if (tv_t <= tv_y) break;   // until TV(y~) <= TV(y)
        }
        total_trials += trials;
        if (!ok) break;
        if (trials_out && local == 0 && threadIdx.x == 0) trials_out[(size_t)pi * K + step] = (int)trials;
        if (step == K - 1 && !want_snorm) {   // the last step, with d
            write_d(true, false, c);
            d_done = true;
        } else {
            for (PixWalk w(e0, stride, nx); w.i < ny;) {   // y <- y~
                size_t gp[kStvGroup];
                float tv[kStvGroup];
#pragma unroll
                for (int q = 0; q < kStvGroup; ++q) {
                    gp[q] = (w.i < ny) ? (size_t)w.i * ld + w.j : ~(size_t)0;
                    if (w.i < ny) tv[q] = tb[gp[q]];
                    w.next();
                }
#pragma unroll
                for (int q = 0; q < kStvGroup; ++q)
                    if (gp[q] != ~(size_t)0) (void)x_step(x, xl, gp[q], c, tv[q]);
            }
            ok = coop_barrier(P.bar, nb + P.bar_extra, &sc->status, &flag, P.wait_limit);
        }
        tv_last = tv_t;
    }
    double sn = 0.0;
    if (ok && want_snorm) {
        double s = 0.0;
        for (int e = e0; e < n; e += stride) {
            const int i = e / nx, j = e - i * nx;
            const size_t p = (size_t)i * ld + j;
            const double dlt = ((double)x[p] - (double)P.z[p]) + ((xl ? (double)xl[p] : 0.0) - (double)P.g[p]);
            s += dlt * dlt;
        }
        sn = phase_sum(P, nb, slot, local, s, red, &flag, &ok);
    }
    if (local == 0 && threadIdx.x == 0) {
        sc->ell = ell;
        sc->apow = sh_apow;
        sc->apow_a = a;
        sc->apow_ell = ell;
        sc->apow_ok = sh_apow_ok;
        sc->trials = total_trials;
        sc->tv_k = tv_first;
        sc->tv_half = (K > 0) ? tv_last : tv_first;
        sc->snorm2 = sn;
    }
    // d, unless the last step wrote it (after the last barrier every block sees the final x);
    // no step ran when the plain loop had none (K = 0), and then no barrier either
    if (ok && !d_done) write_d(false, plain && K == 0, 0.0f);
}

int stv_max_blocks_per_sm(int *out)
{
    SUPCG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_stv, kTvThreads, 0));
    return SUPCG_OK;
}

int launch_stv(const Launch &L, int K, double a, double gamma, long long max_trials, int *trials_out,
               int want_snorm, const float *dir)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(L.blocks);
    cfg.blockDim = dim3(kTvThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = L.st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SUPCG_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_stv, L.probs, L.prefix, L.count, K, a, gamma, max_trials,
                                      trials_out, want_snorm, dir));
    return SUPCG_OK;
}

} // namespace supcg
