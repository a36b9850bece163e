// Learned perturbation network (not part of the paper: a small CNN that
// proposes the TV-nonascending direction of the superiorization step).
//
// Network: five 3x3 convolutions (zero padding), channels
//   16 (x / rms(x), tbar scaled to unit RMS, fourteen zeros) -> 32 -> 32 -> 32 -> 32 -> 1,
// ReLU after the first four; the output is added to the scaled tbar input
// (a residual around the plain direction).  Activations are BF16 NHWC,
// weights BF16, accumulation FP32.
//
// Every convolution (forward, and the input-gradient pass of training, which
// is a convolution with the flipped, transposed kernel) is an implicit GEMM on
// the 5th-generation tensor cores: a CTA stages the three input rows around
// 128 output pixels (M = 128) and the packed weights (N = Cout, K = 9 * Cin)
// in shared memory, one thread issues one tcgen05.mma per tap and 16 channels,
// each reading the staged rows through a descriptor shifted by the tap's
// column offset (no im2col copy), into an FP32 tensor-memory accumulator, and
// the four warps read their 32 lanes back with tcgen05.ld for the epilogue
// (bias, ReLU or ReLU-mask, BF16 store).  The weight gradient is
// a reduction over pixels on the CUDA cores with FP32 accumulation and a
// deterministic two-level sum.  Adam keeps FP32 master weights.
#include <math.h>

#include <algorithm>
#include <vector>

#include "tc.cuh"

namespace supcg {

constexpr int kCnnLayers = 5;
constexpr int kCh = 32;     // hidden channels
constexpr int kInCh = 16;   // stored input channels (2 used; 16 so that one tap fills one K = 16 step)
constexpr int kTile = 128;  // pixels per MMA tile

__host__ __device__ constexpr int kpad(int cin) { return 9 * cin; }   // cin is 16 or 32

// layer l (0-based): storage channels of its input, real input channels, output channels
__host__ __device__ constexpr int l_cin(int l) { return l == 0 ? kInCh : kCh; }
__host__ __device__ constexpr int l_cin_real(int l) { return l == 0 ? 2 : kCh; }
__host__ __device__ constexpr int l_cout(int l) { return l == kCnnLayers - 1 ? 1 : kCh; }
__host__ __device__ constexpr int l_nout(int l) { return l == kCnnLayers - 1 ? 16 : kCh; }   // MMA N

enum { EPI_RELU = 0, EPI_LAST = 1, EPI_MASK = 2 };

struct ConvArgs {
    const __nv_bfloat16 *in;    // NHWC, CIN channels
    const __nv_bfloat16 *w;     // [NOUT][KP] packed, K index = tap * CIN + channel
    const float *bias;          // [>= NOUT] (RELU, LAST)
    __nv_bfloat16 *out_bf;      // NHWC, 32 channels (RELU, MASK)
    float *out_f;               // one channel (LAST)
    const float *resid;         // one channel added to output channel 0 (LAST)
    const __nv_bfloat16 *mask;  // NHWC, 32 channels: keep where mask > 0 (MASK)
    int ny, nx, count;
    int *status;
};

// One CTA: the 128 pixels (i, j0 .. j0+127) of one image row.  Shared memory
// holds the three input rows i-1, i, i+1 over columns j0-1 .. j0+128 (zero
// outside the image), 8-channel chunk by chunk, 16 bytes per pixel, pixels
// contiguous: [dy][chunk][kPixRows].  The A operand of tap (dy, dx) is that
// block started dx pixels in: 8-pixel row groups 128 bytes apart (SBO), channel
// chunks kPixRows * 16 bytes apart (LBO), so the nine taps need no im2col copy.
constexpr int kPixRows = 136;   // staged pixels per row and chunk (>= 130, multiple of 8)

template <int CIN, int NOUT, int EPI>
__global__ void __launch_bounds__(128) k_conv(ConvArgs a)
{
    constexpr int CH8 = CIN / 8;            // 16-byte chunks per pixel
    constexpr int KP = 9 * CIN;             // GEMM K (multiple of 16: CIN is 16 or 32)
    constexpr int KG = KP / 8;
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    __nv_bfloat16 *sa = reinterpret_cast<__nv_bfloat16 *>(sm_raw);   // [3][CH8][kPixRows][8]
    __nv_bfloat16 *sb = sa + 3 * CH8 * kPixRows * 8;                  // NOUT x KP, core-matrix layout
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tbase;
    const int t = threadIdx.x, warp = t >> 5;
    const int tiles_row = (a.nx + kTile - 1) / kTile;
    const long long rowid = blockIdx.x / tiles_row;      // img * ny + i
    const int jb = blockIdx.x - (int)(rowid * tiles_row);
    const int img = (int)(rowid / a.ny), i = (int)(rowid - (long long)img * a.ny);
    const int j0 = jb * kTile;
    const long long n = (long long)a.ny * a.nx;

    // stage: consecutive threads take consecutive chunks of a pixel, then the next pixel
    for (int e = t; e < 3 * 130 * CH8; e += kTile) {
        const int c8 = e % CH8, q = (e / CH8) % 130, dy = e / (CH8 * 130);
        const int ii = i + dy - 1, jj = j0 + q - 1;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (ii >= 0 && ii < a.ny && jj >= 0 && jj < a.nx)
            v = __ldg(reinterpret_cast<const uint4 *>(a.in + (((long long)img * n + (long long)ii * a.nx + jj) * CIN + c8 * 8)));
        *reinterpret_cast<uint4 *>(sa + ((dy * CH8 + c8) * kPixRows + q) * 8) = v;
    }
    for (int e = t; e < NOUT * KG; e += kTile) {   // B: packed weights
        const int row = e / KG, kg = e % KG;
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(a.w + (size_t)row * KP + kg * 8));
        *reinterpret_cast<uint4 *>(sb + ((row >> 3) * KG + kg) * 64 + (row & 7) * 8) = v;
    }
    if (warp == 0) tc_alloc(&tbase, 32);
    if (t == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    fence_proxy_async();   // generic-proxy shared-memory writes -> tensor-core (async proxy) reads
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tbase;
    if (t == 0) {
        constexpr uint32_t idesc = tc_idesc_bf16(128, NOUT);
        const uint32_t sa_u = smem_u32(sa), sb_u = smem_u32(sb);
        int step = 0;
#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
            const int dy = tap / 3, dx = tap % 3;
#pragma unroll
            for (int cp = 0; cp < CH8 / 2; ++cp, ++step) {
                const uint32_t a_addr = sa_u + (uint32_t)(((dy * CH8 + 2 * cp) * kPixRows + dx) * 16);
                const uint32_t b_addr = sb_u + (uint32_t)((tap * CH8 + 2 * cp) * 128);
                tc_mma_bf16(tmem, tc_sdesc(a_addr, kPixRows * 16, 128), tc_sdesc(b_addr, 128, KG * 128), idesc,
                            step > 0);
            }
        }
        tc_commit(&bar);
    }
    bool ok = mbar_wait(&bar, 0);
    tc_fence_after();
    const int r = warp * 32 + (t & 31);
    const int j = j0 + r;
    const long long p = (long long)img * n + (long long)i * a.nx + j;
    if (ok) {
        float acc[32];
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        tc_ld16(lane_addr, acc);
        if (NOUT == 32) tc_ld16(lane_addr + 16, acc + 16);
        if (j < a.nx) {
            if (EPI == EPI_LAST) {
                a.out_f[p] = acc[0] + a.bias[0] + a.resid[p];
            } else {
                __align__(16) __nv_bfloat16 o[32];
                __align__(16) __nv_bfloat16 mk[32];
                if (EPI == EPI_MASK)
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        reinterpret_cast<uint4 *>(mk)[q] = __ldg(reinterpret_cast<const uint4 *>(a.mask + p * 32) + q);
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    float v = acc[c];
                    if (EPI == EPI_RELU) v = fmaxf(0.0f, v + a.bias[c]);
                    else v = (__bfloat162float(mk[c]) > 0.0f) ? v : 0.0f;
                    o[c] = __float2bfloat16_rn(v);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    reinterpret_cast<uint4 *>(a.out_bf + p * 32)[q] = reinterpret_cast<const uint4 *>(o)[q];
            }
        }
    } else {
        if (t == 0) atomicExch(a.status, (int)SUPCG_ERR_TIMEOUT);
        (void)mbar_wait(&bar, 0);   // one more bounded wait for the MMAs before freeing their memory
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, 32);
}

template <int CIN, int NOUT, int EPI>
static int launch_conv(const ConvArgs &a, cudaStream_t st)
{
    constexpr int KP = 9 * CIN;
    constexpr int smem = (3 * (CIN / 8) * kPixRows * 8 + NOUT * KP) * 2;
    static int set = 0;
    if (!set) {
        SUPCG_CUDA_TRY(cudaFuncSetAttribute(k_conv<CIN, NOUT, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        set = 1;
    }
    const long long blocks = (long long)a.count * a.ny * ((a.nx + kTile - 1) / kTile);
    k_conv<CIN, NOUT, EPI><<<(unsigned)blocks, kTile, smem, st>>>(a);
    SUPCG_CUDA_TRY(cudaGetLastError());
    return SUPCG_OK;
}

// ------------------------------------------------------------------ weight gradient
// dW[co][ci][tap] = sum_p G[p][co] * in[p + off(tap)][ci],  db[co] = sum_p G[p][co]
// over a band of kBandRows image rows per block; partial[block][...] is summed by k_reduce.
constexpr int kBandRows = 4;

template <int CIN, int COUT>
__global__ void k_wgrad(const __nv_bfloat16 *in, const __nv_bfloat16 *G, int gch, int cin_real, int ny, int nx,
                        int count, float *partial)
{
    constexpr int COB = COUT >= 4 ? 4 : 1;      // output channels per thread
    constexpr int NCB = COUT / COB;
    const int bands = (ny + kBandRows - 1) / kBandRows;
    const int img = blockIdx.x / bands, band = blockIdx.x - img * bands;
    const int t = threadIdx.x;
    const int cb = t % NCB, rest = t / NCB, tap = rest % 9, c8 = rest / 9;   // c8 < CIN / 8
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const long long n = (long long)ny * nx;
    float acc[COB][8];
    float gsum[COB];
#pragma unroll
    for (int a = 0; a < COB; ++a) {
        gsum[a] = 0.0f;
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;
    }
    if (c8 < CIN / 8) {
        const int i0 = band * kBandRows, i1 = min(ny, i0 + kBandRows);
        for (int i = i0; i < i1; ++i)
            for (int j = 0; j < nx; ++j) {
                const long long p = img * n + (long long)i * nx + j;
                float g[COB];
#pragma unroll
                for (int a = 0; a < COB; ++a) g[a] = __bfloat162float(G[p * gch + cb * COB + a]);
                const int ii = i + dy, jj = j + dx;
                if (ii < 0 || ii >= ny || jj < 0 || jj >= nx) {
                    if (tap == 4)
#pragma unroll
                        for (int a = 0; a < COB; ++a) gsum[a] += g[a];
                    continue;
                }
                __align__(16) __nv_bfloat16 v[8];
                *reinterpret_cast<uint4 *>(v) =
                    __ldg(reinterpret_cast<const uint4 *>(in + (img * n + (long long)ii * nx + jj) * CIN + c8 * 8));
#pragma unroll
                for (int a = 0; a < COB; ++a) {
                    if (tap == 4) gsum[a] += g[a];
#pragma unroll
                    for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(g[a], __bfloat162float(v[b]), acc[a][b]);
                }
            }
        // layout of one block's partial: dW[co][ci][tap] for ci < cin_real, then db[co]
        float *out = partial + (size_t)blockIdx.x * (COUT * cin_real * 9 + COUT);
#pragma unroll
        for (int a = 0; a < COB; ++a) {
            const int co = cb * COB + a;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const int ci = c8 * 8 + b;
                if (ci < cin_real) out[(co * cin_real + ci) * 9 + tap] = acc[a][b];
            }
            if (tap == 4 && c8 == 0) out[COUT * cin_real * 9 + co] = gsum[a];
        }
    }
}

// out[e] = sum_b partial[b][e] in a fixed order.
__global__ void k_reduce(const float *partial, int nb, int len, float *out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= len) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += (double)partial[(size_t)b * len + e];
    out[e] = (float)s;
}

// ------------------------------------------------------------------ input, loss, optimiser
// Per-image sums of squares of x and tbar (one block per image, fixed order).
__global__ void __launch_bounds__(1024) k_norms(const float *x, const float *tb, long long n, double *out)
{
    __shared__ double red[40];
    const int img = blockIdx.x;
    double sx = 0.0, st = 0.0;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) {
        const double a = x[img * n + e], b = tb[img * n + e];
        sx += a * a;
        st += b * b;
    }
    sx = block_sum<1024>(sx, red);
    st = block_sum<1024>(st, red);
    if (threadIdx.x == 0) {
        out[2 * img] = sx;
        out[2 * img + 1] = st;
    }
}

// Input tensor: channel 0 = x / rms(x), channel 1 = tbar scaled to unit RMS,
// channels 2..15 = 0; resid = channel 1 in FP32.
__global__ void k_pack_input(const float *x, const float *tb, const double *norms, long long n, int count,
                             __nv_bfloat16 *act0, float *resid)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n * count) return;
    const long long img = p / n;
    const double sx = norms[2 * img], st = norms[2 * img + 1];
    const float fx = sx > 0.0 ? (float)sqrt((double)n / sx) : 0.0f;
    const float ft = st > 0.0 ? (float)sqrt((double)n / st) : 0.0f;
    const float v0 = x[p] * fx, v1 = tb[p] * ft;
    __align__(16) __nv_bfloat16 o[16];
    o[0] = __float2bfloat16_rn(v0);
    o[1] = __float2bfloat16_rn(v1);
#pragma unroll
    for (int c = 2; c < 16; ++c) o[c] = __float2bfloat16_rn(0.0f);
    reinterpret_cast<uint4 *>(act0)[2 * p] = reinterpret_cast<const uint4 *>(o)[0];
    reinterpret_cast<uint4 *>(act0)[2 * p + 1] = reinterpret_cast<const uint4 *>(o)[1];
    resid[p] = v1;
}

// Loss L = mean (out - target~)^2 with target~ the target scaled per image to unit
// RMS; G5 = dL/dout as a 16-channel BF16 tensor (channel 0).
__global__ void __launch_bounds__(256) k_loss(const float *out, const float *target, const double *tnorms,
                                              long long n, long long total, __nv_bfloat16 *G5, double *partial)
{
    __shared__ double red[40];
    double s = 0.0;
    const float scale = (float)(2.0 / (double)total);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const double tn = tnorms[2 * (p / n)];
        const float ft = tn > 0.0 ? (float)sqrt((double)n / tn) : 0.0f;
        const float d = out[p] - target[p] * ft;
        s += (double)d * (double)d;
        __align__(16) __nv_bfloat16 o[16];
        o[0] = __float2bfloat16_rn(scale * d);
#pragma unroll
        for (int c = 1; c < 16; ++c) o[c] = __float2bfloat16_rn(0.0f);
        reinterpret_cast<uint4 *>(G5)[2 * p] = reinterpret_cast<const uint4 *>(o)[0];
        reinterpret_cast<uint4 *>(G5)[2 * p + 1] = reinterpret_cast<const uint4 *>(o)[1];
    }
    s = block_sum<256>(s, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Adam on the FP32 master parameters.
__global__ void k_adam(float *w, const float *g, float *m, float *v, int len, float lr, float b1, float b2,
                       float c1, float c2, float eps)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= len) return;
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.0f - b1) * gg;
    const float vv = b2 * v[e] + (1.0f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    w[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// Packed BF16 GEMM weights of layer l (forward) and of its input-gradient pass.
//   fwd[co][tap * cin + ci] = W[co][ci][tap]            (co < cout, ci < cin_real; else 0)
//   bwd[ci][tap * gch + co] = W[co][ci][8 - tap]        (flipped kernel, transposed channels)
__global__ void k_pack_weights(const float *W, int cout, int cin, int cin_real, int nout, int kp,
                               __nv_bfloat16 *fwd, int gch, int kpb, __nv_bfloat16 *bwd)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nout * kp) {
        const int co = e / kp, k = e - co * kp;
        const int tap = k / cin, ci = k - tap * cin;
        float v = 0.0f;
        if (co < cout && tap < 9 && ci < cin_real) v = W[(co * cin_real + ci) * 9 + tap];
        fwd[e] = __float2bfloat16_rn(v);
    }
    if (bwd && e < kCh * kpb) {
        const int ci = e / kpb, k = e - ci * kpb;
        const int tap = k / gch, co = k - tap * gch;
        float v = 0.0f;
        if (ci < cin_real && tap < 9 && co < cout) v = W[(co * cin_real + ci) * 9 + (8 - tap)];
        bwd[e] = __float2bfloat16_rn(v);
    }
}

} // namespace supcg

// ------------------------------------------------------------------ network object
using namespace supcg;

struct supcg_cnn_s {
    int ny, nx, cap;             // image size and the largest batch the buffers hold
    int nparam;
    int off_w[kCnnLayers], off_b[kCnnLayers];
    float *params = nullptr, *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
    __nv_bfloat16 *wf[kCnnLayers] = {}, *wb[kCnnLayers] = {};
    __nv_bfloat16 *act[kCnnLayers] = {};   // act[0] input (8 ch), act[1..4] hidden (32 ch)
    __nv_bfloat16 *gbuf[kCnnLayers] = {};  // gbuf[4] = dL/dout (8 ch); gbuf[l] = dL/dz_l (32 ch), l = 1..3; gbuf[0] for layer 1
    float *resid = nullptr, *out = nullptr, *partial = nullptr;
    double *norms = nullptr, *tnorms = nullptr, *lpart = nullptr;
    int *status = nullptr;
    size_t partial_len = 0;
    long long step = 0;
    std::vector<void *> allocs;
};
typedef supcg_cnn_s *supcg_cnn;

static int cnn_alloc(supcg_cnn net, void **p, size_t bytes)
{
    if (cudaMalloc(p, bytes) != cudaSuccess) return SUPCG_ERR_NOMEM;
    net->allocs.push_back(*p);
    if (cudaMemset(*p, 0, bytes) != cudaSuccess) return SUPCG_ERR_CUDA;
    return SUPCG_OK;
}

static int cnn_pack(supcg_cnn net, cudaStream_t st)
{
    for (int l = 0; l < kCnnLayers; ++l) {
        const int kp = kpad(l_cin(l));
        const int gch = (l == kCnnLayers - 1) ? kInCh : kCh;   // channels of dL/dz_l as stored
        const int kpb = kpad(gch);
        const int len = std::max(l_nout(l) * kp, kCh * kpb);
        k_pack_weights<<<(len + 255) / 256, 256, 0, st>>>(net->params + net->off_w[l], l_cout(l), l_cin(l),
                                                          l_cin_real(l), l_nout(l), kp, net->wf[l], gch, kpb,
                                                          l > 0 ? net->wb[l] : nullptr);
    }
    SUPCG_CUDA_TRY(cudaGetLastError());
    return SUPCG_OK;
}

extern "C" int supcg_cnn_create(int ny, int nx, int max_batch, unsigned long long seed, supcg_cnn *out)
{
    if (!out || ny < 1 || nx < 1 || max_batch < 1 || (long long)ny * nx * max_batch > (1ll << 31)) return SUPCG_ERR_ARG;
    *out = nullptr;
    auto *net = new (std::nothrow) supcg_cnn_s();
    if (!net) return SUPCG_ERR_NOMEM;
    net->ny = ny;
    net->nx = nx;
    net->cap = max_batch;
    int off = 0;
    for (int l = 0; l < kCnnLayers; ++l) {
        net->off_w[l] = off;
        off += l_cout(l) * l_cin_real(l) * 9;
        net->off_b[l] = off;
        off += l_cout(l);
    }
    net->nparam = off;
    // He-uniform initial weights from a seeded generator; the last layer starts at zero so that the
    // untrained network returns the plain nonascending direction.
    std::vector<float> h(off, 0.0f);
    unsigned long long s = seed ? seed : 0x9E3779B97F4A7C15ull;
    auto rnd = [&s]() {   // splitmix64
        s += 0x9E3779B97F4A7C15ull;
        unsigned long long z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) / 9007199254740992.0;
    };
    for (int l = 0; l + 1 < kCnnLayers; ++l) {
        const double lim = sqrt(6.0 / (9.0 * l_cin_real(l)));
        for (int e = 0; e < l_cout(l) * l_cin_real(l) * 9; ++e) h[net->off_w[l] + e] = (float)((2.0 * rnd() - 1.0) * lim);
    }
    const long long npix = (long long)ny * nx * max_batch;
    int rc = SUPCG_OK;
    rc = rc ? rc : cnn_alloc(net, (void **)&net->params, sizeof(float) * off);
    rc = rc ? rc : cnn_alloc(net, (void **)&net->grads, sizeof(float) * off);
    rc = rc ? rc : cnn_alloc(net, (void **)&net->adam_m, sizeof(float) * off);
    rc = rc ? rc : cnn_alloc(net, (void **)&net->adam_v, sizeof(float) * off);
    for (int l = 0; l < kCnnLayers && !rc; ++l) {
        rc = cnn_alloc(net, (void **)&net->wf[l], 2 * (size_t)l_nout(l) * kpad(l_cin(l)));
        if (!rc && l > 0) rc = cnn_alloc(net, (void **)&net->wb[l], 2 * (size_t)kCh * kpad(l == kCnnLayers - 1 ? kInCh : kCh));
        if (!rc) rc = cnn_alloc(net, (void **)&net->act[l], 2 * (size_t)npix * (l == 0 ? kInCh : kCh));
        if (!rc) rc = cnn_alloc(net, (void **)&net->gbuf[l], 2 * (size_t)npix * (l == kCnnLayers - 1 ? kInCh : kCh));
    }
    const int bands = (ny + kBandRows - 1) / kBandRows;
    net->partial_len = (size_t)max_batch * bands * (kCh * kCh * 9 + kCh);
    rc = rc ? rc : cnn_alloc(net, (void **)&net->partial, sizeof(float) * net->partial_len);
    rc = rc ? rc : cnn_alloc(net, (void **)&net->resid, sizeof(float) * npix);
    rc = rc ? rc : cnn_alloc(net, (void **)&net->out, sizeof(float) * npix);
    rc = rc ? rc : cnn_alloc(net, (void **)&net->norms, sizeof(double) * 2 * max_batch);
    rc = rc ? rc : cnn_alloc(net, (void **)&net->tnorms, sizeof(double) * 2 * max_batch);
    rc = rc ? rc : cnn_alloc(net, (void **)&net->lpart, sizeof(double) * 1024);
    rc = rc ? rc : cnn_alloc(net, (void **)&net->status, sizeof(int));
    if (!rc && cudaMemcpy(net->params, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = SUPCG_ERR_CUDA;
    if (!rc) rc = cnn_pack(net, 0);
    if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = SUPCG_ERR_CUDA;
    if (rc) {
        for (void *p : net->allocs) cudaFree(p);
        delete net;
        return rc;
    }
    *out = net;
    return SUPCG_OK;
}

extern "C" int supcg_cnn_destroy(supcg_cnn net)
{
    if (!net) return SUPCG_ERR_ARG;
    cudaDeviceSynchronize();
    for (void *p : net->allocs) cudaFree(p);
    delete net;
    return SUPCG_OK;
}

extern "C" int supcg_cnn_num_params(supcg_cnn net) { return net ? net->nparam : SUPCG_ERR_ARG; }

// Host copy of all FP32 parameters: for each layer W[cout][cin][3][3] then b[cout].
extern "C" int supcg_cnn_get_params(supcg_cnn net, float *h_params)
{
    if (!net || !h_params) return SUPCG_ERR_ARG;
    SUPCG_CUDA_TRY(cudaMemcpy(h_params, net->params, sizeof(float) * net->nparam, cudaMemcpyDeviceToHost));
    return SUPCG_OK;
}

extern "C" int supcg_cnn_set_params(supcg_cnn net, const float *h_params)
{
    if (!net || !h_params) return SUPCG_ERR_ARG;
    SUPCG_CUDA_TRY(cudaMemcpy(net->params, h_params, sizeof(float) * net->nparam, cudaMemcpyHostToDevice));
    int rc = cnn_pack(net, 0);
    if (rc) return rc;
    SUPCG_CUDA_TRY(cudaDeviceSynchronize());
    return SUPCG_OK;
}

namespace supcg {

// Forward pass of `count` images: out[count][ny][nx] (FP32, unit-RMS scale).
int cnn_forward(supcg_cnn net, const float *d_x, const float *d_tbar, int count, cudaStream_t st)
{
    const long long n = (long long)net->ny * net->nx;
    k_norms<<<count, 1024, 0, st>>>(d_x, d_tbar, n, net->norms);
    k_pack_input<<<(unsigned)((n * count + 255) / 256), 256, 0, st>>>(d_x, d_tbar, net->norms, n, count, net->act[0],
                                                                     net->resid);
    SUPCG_CUDA_TRY(cudaGetLastError());
    ConvArgs a = {};
    a.ny = net->ny;
    a.nx = net->nx;
    a.count = count;
    a.status = net->status;
    int rc;
    for (int l = 0; l < kCnnLayers; ++l) {
        a.in = net->act[l];
        a.w = net->wf[l];
        a.bias = net->params + net->off_b[l];
        if (l + 1 < kCnnLayers) {
            a.out_bf = net->act[l + 1];
            rc = (l == 0) ? launch_conv<kInCh, kCh, EPI_RELU>(a, st) : launch_conv<kCh, kCh, EPI_RELU>(a, st);
        } else {
            a.out_f = net->out;
            a.resid = net->resid;
            rc = launch_conv<kCh, 16, EPI_LAST>(a, st);
        }
        if (rc) return rc;
    }
    return SUPCG_OK;
}

// Backward pass after cnn_forward with dL/dout in gbuf[4]: gradients into net->grads.
static int cnn_backward(supcg_cnn net, int count, cudaStream_t st)
{
    const int bands = (net->ny + kBandRows - 1) / kBandRows;
    const int nb = count * bands;
    ConvArgs a = {};
    a.ny = net->ny;
    a.nx = net->nx;
    a.count = count;
    a.status = net->status;
    for (int l = kCnnLayers - 1; l >= 0; --l) {
        const int cin_real = l_cin_real(l), cout = l_cout(l);
        const int gch = (l == kCnnLayers - 1) ? kInCh : kCh;
        // weight gradient of layer l: input act[l], output gradient gbuf[l]
        if (l == 0)
            k_wgrad<kInCh, kCh><<<nb, (kCh / 4) * 9 * (kInCh / 8), 0, st>>>(net->act[0], net->gbuf[0], gch, cin_real,
                                                                            net->ny, net->nx, count, net->partial);
        else if (l == kCnnLayers - 1)
            k_wgrad<kCh, 1><<<nb, 1 * 9 * (kCh / 8), 0, st>>>(net->act[l], net->gbuf[l], gch, cin_real, net->ny,
                                                              net->nx, count, net->partial);
        else
            k_wgrad<kCh, kCh><<<nb, (kCh / 4) * 9 * (kCh / 8), 0, st>>>(net->act[l], net->gbuf[l], gch, cin_real,
                                                                        net->ny, net->nx, count, net->partial);
        const int len = cout * cin_real * 9 + cout;
        k_reduce<<<(len + 255) / 256, 256, 0, st>>>(net->partial, nb, len, net->grads + net->off_w[l]);
        SUPCG_CUDA_TRY(cudaGetLastError());
        if (l == 0) break;
        // input gradient: dL/dz_{l-1} = conv(gbuf[l], flipped W_l) masked by act[l] > 0
        a.in = net->gbuf[l];
        a.w = net->wb[l];
        a.mask = net->act[l];
        a.out_bf = net->gbuf[l - 1];
        int rc = (l == kCnnLayers - 1) ? launch_conv<kInCh, kCh, EPI_MASK>(a, st) : launch_conv<kCh, kCh, EPI_MASK>(a, st);
        if (rc) return rc;
    }
    return SUPCG_OK;
}

static int cnn_loss(supcg_cnn net, const float *d_target, int count, cudaStream_t st, double *h_loss)
{
    const long long n = (long long)net->ny * net->nx;
    const long long total = n * count;
    const int blocks = (int)std::min<long long>(1024, (total + 255) / 256);
    k_norms<<<count, 1024, 0, st>>>(d_target, d_target, n, net->tnorms);
    k_loss<<<blocks, 256, 0, st>>>(net->out, d_target, net->tnorms, n, total, net->gbuf[kCnnLayers - 1], net->lpart);
    SUPCG_CUDA_TRY(cudaGetLastError());
    if (h_loss) {
        std::vector<double> hp(blocks);
        SUPCG_CUDA_TRY(cudaMemcpyAsync(hp.data(), net->lpart, sizeof(double) * blocks, cudaMemcpyDeviceToHost, st));
        SUPCG_CUDA_TRY(cudaStreamSynchronize(st));
        double s = 0.0;
        for (double v : hp) s += v;
        *h_loss = s / (double)total;
    }
    return SUPCG_OK;
}

} // namespace supcg

namespace supcg {
float *cnn_output(supcg_cnn net) { return net->out; }
int cnn_shape(supcg_cnn net, int *ny, int *nx)
{
    *ny = net->ny;
    *nx = net->nx;
    return SUPCG_OK;
}
} // namespace supcg

static int cnn_check(supcg_cnn net, int count)
{
    return (!net || count < 1 || count > net->cap) ? SUPCG_ERR_ARG : SUPCG_OK;
}

static int cnn_status(supcg_cnn net, cudaStream_t st)
{
    int s = 0;
    SUPCG_CUDA_TRY(cudaMemcpyAsync(&s, net->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    SUPCG_CUDA_TRY(cudaStreamSynchronize(st));
    return s;
}

extern "C" int supcg_cnn_forward(supcg_cnn net, const float *d_x, const float *d_tbar, int count, float *d_out,
                                 void *stream)
{
    int rc = cnn_check(net, count);
    if (rc || !d_x || !d_tbar || !d_out) return rc ? rc : SUPCG_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = cnn_forward(net, d_x, d_tbar, count, st))) return rc;
    SUPCG_CUDA_TRY(cudaMemcpyAsync(d_out, net->out, sizeof(float) * (size_t)net->ny * net->nx * count,
                                   cudaMemcpyDeviceToDevice, st));
    return cnn_status(net, st);
}

extern "C" int supcg_cnn_gradients(supcg_cnn net, const float *d_x, const float *d_tbar, const float *d_target,
                                   int count, float *h_grads, double *h_loss, void *stream)
{
    int rc = cnn_check(net, count);
    if (rc || !d_x || !d_tbar || !d_target || !h_grads) return rc ? rc : SUPCG_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = cnn_forward(net, d_x, d_tbar, count, st))) return rc;
    if ((rc = cnn_loss(net, d_target, count, st, h_loss))) return rc;
    if ((rc = cnn_backward(net, count, st))) return rc;
    SUPCG_CUDA_TRY(cudaMemcpyAsync(h_grads, net->grads, sizeof(float) * net->nparam, cudaMemcpyDeviceToHost, st));
    return cnn_status(net, st);
}

extern "C" int supcg_cnn_train_step(supcg_cnn net, const float *d_x, const float *d_tbar, const float *d_target,
                                    int count, double lr, double *h_loss, void *stream)
{
    int rc = cnn_check(net, count);
    if (rc || !d_x || !d_tbar || !d_target || !(lr > 0.0)) return rc ? rc : SUPCG_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = cnn_forward(net, d_x, d_tbar, count, st))) return rc;
    if ((rc = cnn_loss(net, d_target, count, st, h_loss))) return rc;
    if ((rc = cnn_backward(net, count, st))) return rc;
    net->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 - pow(0.9, (double)net->step)), c2 = (float)(1.0 - pow(0.999, (double)net->step));
    k_adam<<<(net->nparam + 255) / 256, 256, 0, st>>>(net->params, net->grads, net->adam_m, net->adam_v, net->nparam,
                                                      (float)lr, b1, b2, c1, c2, 1e-8f);
    SUPCG_CUDA_TRY(cudaGetLastError());
    if ((rc = cnn_pack(net, st))) return rc;
    return h_loss ? cnn_status(net, st) : SUPCG_OK;
}
