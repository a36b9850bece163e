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
// (bias, ReLU or ReLU-mask, BF16 store).  The weight gradient is a
// contraction over pixels on the same tensor cores (both operands MN-major from
// the staged rows), accumulated per CTA in tensor memory and summed over CTAs
// in a fixed order.  Adam keeps FP32 master weights.
#include <math.h>

#include <algorithm>
#include <mutex>
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
    const __nv_bfloat16 *w;     // [NOUT][KP] packed in core-matrix order, K index = tap * CIN + channel
    const float *bias;          // [>= NOUT] (RELU, LAST)
    __nv_bfloat16 *out_bf;      // NHWC, 32 channels (RELU, MASK)
    float *out_f;               // one channel (LAST)
    const float *resid;         // one channel added to output channel 0 (LAST)
    const __nv_bfloat16 *mask;  // NHWC, 32 channels: keep where mask > 0 (MASK)
    int ny, nx, count;
    int *status;
};

// A tile is the 128 pixels (i, j0 .. j0+127) of one image row.  Shared memory
// holds the three input rows i-1, i, i+1 over columns j0-1 .. j0+128, 8-channel
// chunk by chunk, 16 bytes per pixel, pixels contiguous: [dy][chunk][kPixRows].
// Each (row, chunk) is one 4-D TMA load (channels, columns, rows, images) whose
// out-of-image part the TMA fills with zeros.  The A operand of tap (dy, dx) is
// that block started dx pixels in: 8-pixel row groups 128 bytes apart (SBO),
// channel chunks kPixRows * 16 bytes apart (LBO), so the nine taps need no
// im2col copy.  CTAs are persistent and software-pipelined over their tiles
// q = 0, 1, ...: the packed weights arrive once by one bulk copy; tile q's rows
// sit in stage buffer q & 1 and its accumulator in tensor-memory columns
// 32 * (q & 1), so while the four warps run the epilogue of tile q, tile q+1's
// MMAs and tile q+2's row loads are already in flight.
constexpr int kPixRows = 136;                        // staged pixels per row and chunk (>= 130, multiple of 8)
constexpr int kChunkBytes = kPixRows * 16;           // 2176 = 17 x 128: every TMA destination 128-byte aligned
constexpr int kBoxPix = 130;                         // columns j0-1 .. j0+128

template <int CIN, int NOUT, int EPI>
__global__ void __launch_bounds__(128) k_conv(ConvArgs a, const __grid_constant__ CUtensorMap tm)
{
    constexpr int CH8 = CIN / 8;            // 16-byte chunks per pixel
    constexpr int KP = 9 * CIN;             // GEMM K (multiple of 16: CIN is 16 or 32)
    constexpr int KG = KP / 8;
    constexpr int ABYTES = 3 * CH8 * kChunkBytes;
    constexpr unsigned WBYTES = NOUT * KP * 2;
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    unsigned char *sb = sm_raw + 2 * ABYTES;   // NOUT x KP, core-matrix layout (as packed in global memory)
    __shared__ __align__(8) uint64_t bar_tma[2], bar_mma[2], bar_w;
    __shared__ uint32_t tbase;
    __shared__ float s_bias[32];
    const int t = threadIdx.x, warp = t >> 5;
    const int tiles_row = (a.nx + kTile - 1) / kTile;
    const long long ntiles = (long long)a.count * a.ny * tiles_row;
    const long long n = (long long)a.ny * a.nx;
    const long long first = blockIdx.x, stride = gridDim.x;
    const int nq = first < ntiles ? (int)((ntiles - 1 - first) / stride) + 1 : 0;   // this CTA's tiles

    if (warp == 0) tc_alloc(&tbase, 64);
    if (t < 32) s_bias[t] = (EPI == EPI_RELU || (EPI == EPI_LAST && t == 0)) ? a.bias[t] : 0.0f;   // LAST: one bias
    if (t == 0) {
        mbar_init(&bar_tma[0], 1);
        mbar_init(&bar_tma[1], 1);
        mbar_init(&bar_mma[0], 1);
        mbar_init(&bar_mma[1], 1);
        mbar_init(&bar_w, 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tbase;

    auto tile_pos = [&](int q, int &img, int &i, int &jb) {
        const long long tile = first + (long long)q * stride;
        const long long rowid = tile / tiles_row;
        jb = (int)(tile - rowid * tiles_row);
        img = (int)(rowid / a.ny);
        i = (int)(rowid - (long long)img * a.ny);
    };
    // thread 0: the 3 x CH8 row loads of tile q into stage buffer q & 1
    auto issue_rows = [&](int q) {
        int img, i, jb;
        tile_pos(q, img, i, jb);
        const int buf = q & 1;
        const uint32_t bar = smem_u32(&bar_tma[buf]);
        mbar_expect_tx(&bar_tma[buf], 3 * CH8 * kBoxPix * 16);
        for (int dy = 0; dy < 3; ++dy)
            for (int c8 = 0; c8 < CH8; ++c8) {
                const uint32_t dst = smem_u32(sm_raw + buf * ABYTES + (dy * CH8 + c8) * kChunkBytes);
                asm volatile(
                    "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                    " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
                    "l"(reinterpret_cast<uint64_t>(&tm)), "r"(c8 * 8), "r"(jb * kTile - 1), "r"(i + dy - 1),
                    "r"(img), "r"(bar)
                    : "memory");
            }
    };
    // thread 0: the 9 * CH8 / 2 MMAs of tile q into accumulator q & 1
    auto issue_mma = [&](int q) {
        constexpr uint32_t idesc = tc_idesc_bf16(128, NOUT);
        const uint32_t sa_u = smem_u32(sm_raw + (q & 1) * ABYTES), sb_u = smem_u32(sb);
        const uint32_t acc = tmem + 32u * (uint32_t)(q & 1);
        int step = 0;
#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
            const int dy = tap / 3, dx = tap % 3;
#pragma unroll
            for (int cp = 0; cp < CH8 / 2; ++cp, ++step) {
                const uint32_t a_addr = sa_u + (uint32_t)((dy * CH8 + 2 * cp) * kChunkBytes + dx * 16);
                const uint32_t b_addr = sb_u + (uint32_t)((tap * CH8 + 2 * cp) * 128);
                tc_mma_bf16(acc, tc_sdesc(a_addr, kChunkBytes, 128), tc_sdesc(b_addr, 128, KG * 128), idesc, step > 0);
            }
        }
        tc_commit(&bar_mma[q & 1]);
    };

    // thread 0's record of what is in flight, for the cleanup after a timeout (-1: nothing)
    int tma_q0 = -1, tma_q1 = -1, mma_q0 = -1, mma_q1 = -1;
    auto tma_q = [&](int k) -> int & { return k ? tma_q1 : tma_q0; };
    auto mma_q = [&](int k) -> int & { return k ? mma_q1 : mma_q0; };
    bool ok = true;
    if (t == 0 && nq > 0) {
        mbar_expect_tx(&bar_w, WBYTES);
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_u32(sb)),
                     "l"(a.w), "r"(WBYTES), "r"(smem_u32(&bar_w))
                     : "memory");
        issue_rows(0);
        tma_q(0) = 0;
        if (nq > 1) {
            issue_rows(1);
            tma_q(1) = 1;
        }
        ok = mbar_wait(&bar_w, 0) && mbar_wait(&bar_tma[0], 0);
        if (ok) {
            tma_q(0) = -1;
            tc_fence_after();
            issue_mma(0);
            mma_q(0) = 0;
        }
    }
    int q = 0;
    for (; q < nq; ++q) {
        const int b = q & 1;
        if (t == 0 && ok && q + 1 < nq) {   // tile q+1: rows landed -> MMAs into the other accumulator
            ok = mbar_wait(&bar_tma[b ^ 1], ((q + 1) >> 1) & 1);
            if (ok) {
                tma_q(b ^ 1) = -1;
                tc_fence_after();
                issue_mma(q + 1);
                mma_q(b ^ 1) = q + 1;
            }
        }
        int img, i, jb;
        tile_pos(q, img, i, jb);
        const int j = jb * kTile + warp * 32 + (t & 31);
        const long long p = (long long)img * n + (long long)i * a.nx + j;
        __align__(16) __nv_bfloat16 mk[32];
        float res = 0.0f;
        if (j < a.nx) {   // epilogue operands, fetched while the MMAs run
            if (EPI == EPI_MASK)
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    reinterpret_cast<uint4 *>(mk)[c] = __ldg(reinterpret_cast<const uint4 *>(a.mask + p * 32) + c);
            if (EPI == EPI_LAST) res = a.resid[p];
        }
        const bool got = mbar_wait(&bar_mma[b], (q >> 1) & 1);
        tc_fence_after();
        if (t == 0 && got) {
            mma_q(b) = -1;
            if (ok && q + 2 < nq) {   // stage buffer b is free again: tile q+2's rows
                issue_rows(q + 2);
                tma_q(b) = q + 2;
            }
        }
        if (got) {
            float acc[32];
            const uint32_t lane_addr = tmem + 32u * (uint32_t)b + ((uint32_t)(warp * 32) << 16);
            tc_ld16(lane_addr, acc);
            if (NOUT == 32) tc_ld16(lane_addr + 16, acc + 16);
            if (j < a.nx) {
                if (EPI == EPI_LAST) {
                    a.out_f[p] = acc[0] + s_bias[0] + res;
                } else {
                    __align__(16) __nv_bfloat16 o[32];
#pragma unroll
                    for (int c = 0; c < 32; ++c) {
                        float v = acc[c];
                        if (EPI == EPI_RELU) v = fmaxf(0.0f, v + s_bias[c]);
                        else v = (__bfloat162float(mk[c]) > 0.0f) ? v : 0.0f;
                        o[c] = __float2bfloat16_rn(v);
                    }
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        reinterpret_cast<uint4 *>(a.out_bf + p * 32)[c] = reinterpret_cast<const uint4 *>(o)[c];
                }
            }
        }
        tc_fence_before();
        // accumulator b read by every warp before tile q+2's MMAs overwrite it; uniform exit on a timeout
        if (!__syncthreads_and(ok && got)) {
            ok = false;
            break;
        }
        tc_fence_after();
    }
    if (!ok && t == 0) {
        atomicExch(a.status, (int)SUPCG_ERR_TIMEOUT);
        // bounded waits for the copies and MMAs still in flight before their memory is released
        for (int k = 0; k < 2; ++k) {
            if (mma_q(k) >= 0) (void)mbar_wait(&bar_mma[k], (mma_q(k) >> 1) & 1);
            if (tma_q(k) >= 0) (void)mbar_wait(&bar_tma[k], (tma_q(k) >> 1) & 1);
        }
        (void)mbar_wait(&bar_w, 0);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, 64);
}

// 4-D map of an NHWC BF16 tensor with a box of 8 channels x `pix` columns.
static int nhwc_map(CUtensorMap *m, const __nv_bfloat16 *base, int ch, int ny, int nx, int count, int pix)
{
    const cuuint64_t dims[4] = {(cuuint64_t)ch, (cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)count};
    const cuuint64_t strides[3] = {(cuuint64_t)ch * 2, (cuuint64_t)nx * ch * 2, (cuuint64_t)ny * nx * ch * 2};
    const cuuint32_t box[4] = {8, (cuuint32_t)pix, 1, 1};
    return encode_tiled(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16 *>(base), dims, strides, box);
}

template <int CIN, int NOUT, int EPI>
static int launch_conv(const ConvArgs &a, cudaStream_t st)
{
    constexpr int KP = 9 * CIN;
    constexpr int smem = 2 * 3 * (CIN / 8) * kChunkBytes + NOUT * KP * 2;
    // attributes and the persistent grid size are per device
    static std::mutex mu;
    static int ctas_dev[kMaxDevices] = {};
    int dev = 0;
    int rc0 = current_device(&dev);
    if (rc0) return rc0;
    rc0 = func_attrs_once((const void *)k_conv<CIN, NOUT, EPI>, smem, (int)cudaSharedmemCarveoutMaxShared);
    if (rc0) return rc0;
    int ctas;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!ctas_dev[dev]) {
            int per_sm = 1, nsm = 1;
            SUPCG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv<CIN, NOUT, EPI>, kTile, smem));
            SUPCG_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
            int smem_sm = 0;
            SUPCG_CUDA_TRY(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
            const int by_smem = smem_sm / (smem + 2048);   // dynamic + static shared memory and the per-CTA reserve
            per_sm = std::max(per_sm, std::min(by_smem, 512 / 64));   // 64 tensor-memory columns per CTA
            ctas_dev[dev] = nsm * std::max(1, per_sm);
        }
        ctas = ctas_dev[dev];
    }
    CUtensorMap tm;
    int rc = nhwc_map(&tm, a.in, CIN, a.ny, a.nx, a.count, kBoxPix);
    if (rc) return rc;
    const long long tiles = (long long)a.count * a.ny * ((a.nx + kTile - 1) / kTile);
    const unsigned grid = (unsigned)std::min<long long>(tiles, ctas);
    k_conv<CIN, NOUT, EPI><<<grid, kTile, smem, st>>>(a, tm);
    SUPCG_CUDA_TRY(cudaGetLastError());
    return SUPCG_OK;
}

// ------------------------------------------------------------------ weight gradient
// dW[co][ci][dy][dx] = sum_p G[p][co] * in[p + (dy-1, dx-1)][ci],  db[co] = sum_p G[p][co].
// A contraction over pixels, on the tensor cores: per 128-pixel tile and per
// column offset dx, D_dx[m][co] += sum_k A_dx[m][k] G[k][co] with
//   m = (dy * CIN + ci) (the staged rows, chunk by chunk) and k the tile's pixels,
//   A_dx[m][k] = in[i + dy - 1][j0 + k + dx - 1][ci],
// both operands read MN-major from the same [chunk][pixel][8 channels] stage
// layout as the convolution (A's start shifted dx pixels in; core matrices
// 128 bytes apart along the pixels (LBO), chunks kChunkBytes apart (SBO)).  M is
// 128 = 16 chunks: the 3 * CIN / 8 input chunks, then a chunk of ones whose rows
// give db, then padding.  Each persistent CTA accumulates its tiles in tensor
// memory (one FP32 accumulator per dx) and writes one partial; k_reduce sums the
// partials in CTA order, so the result is deterministic.
constexpr int kWgChunks = 16;                                 // M = 128 rows of 8 channels
constexpr int kWgStageBytes = kWgChunks * kChunkBytes;        // 34816

template <int CIN, int GCH>
__global__ void __launch_bounds__(128) k_wgrad(int ny, int nx, int count, int cin_real, int cout, float *partial,
                                               int *status, const __grid_constant__ CUtensorMap tin,
                                               const __grid_constant__ CUtensorMap tg)
{
    constexpr int CH8 = CIN / 8, GH8 = GCH / 8;
    constexpr int ONES = 3 * CH8;                       // chunk index of the ones
    constexpr int GBYTES = GH8 * kChunkBytes;
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    unsigned char *sg0 = sm_raw + 2 * kWgStageBytes;   // two G stages follow the two A stages
    __shared__ __align__(8) uint64_t bar_tma[2], bar_mma[2];
    __shared__ uint32_t tbase;
    const int t = threadIdx.x, warp = t >> 5;
    const int tiles_row = (nx + kTile - 1) / kTile;
    const long long ntiles = (long long)count * ny * tiles_row;
    const long long first = blockIdx.x, stride = gridDim.x;
    const int nq = first < ntiles ? (int)((ntiles - 1 - first) / stride) + 1 : 0;

    // constant chunks of both A stages: ones at chunk ONES, zeros after it
    for (int e = t; e < 2 * (kWgChunks - ONES) * kChunkBytes / 16; e += 128) {
        const int per = (kWgChunks - ONES) * kChunkBytes / 16;
        const int sbuf = e / per, r = e - sbuf * per;
        const uint32_t one2 = 0x3F803F80u;   // two BF16 ones
        const uint4 v = r < kChunkBytes / 16 ? make_uint4(one2, one2, one2, one2) : make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4 *>(sm_raw + sbuf * kWgStageBytes + ONES * kChunkBytes + r * 16) = v;
    }
    if (warp == 0) tc_alloc(&tbase, 128);
    if (t == 0) {
        for (int k = 0; k < 2; ++k) {
            mbar_init(&bar_tma[k], 1);
            mbar_init(&bar_mma[k], 1);
        }
        fence_mbar_init();
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tbase;

    auto issue_rows = [&](int q) {   // thread 0: input rows and G row of tile q into stage q & 1
        const long long tile = first + (long long)q * stride;
        const long long rowid = tile / tiles_row;
        const int jb = (int)(tile - rowid * tiles_row);
        const int img = (int)(rowid / ny), i = (int)(rowid - (long long)img * ny);
        const int buf = q & 1;
        const uint32_t bar = smem_u32(&bar_tma[buf]);
        mbar_expect_tx(&bar_tma[buf], (3 * CH8 * kBoxPix + GH8 * kTile) * 16);
        for (int dy = 0; dy < 3; ++dy)
            for (int c8 = 0; c8 < CH8; ++c8) {
                const uint32_t dst = smem_u32(sm_raw + buf * kWgStageBytes + (dy * CH8 + c8) * kChunkBytes);
                asm volatile(
                    "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                    " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
                    "l"(reinterpret_cast<uint64_t>(&tin)), "r"(c8 * 8), "r"(jb * kTile - 1), "r"(i + dy - 1),
                    "r"(img), "r"(bar)
                    : "memory");
            }
        for (int c8 = 0; c8 < GH8; ++c8) {
            const uint32_t dst = smem_u32(sg0 + buf * GBYTES + c8 * kChunkBytes);
            asm volatile(
                "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
                "l"(reinterpret_cast<uint64_t>(&tg)), "r"(c8 * 8), "r"(jb * kTile), "r"(i), "r"(img), "r"(bar)
                : "memory");
        }
    };

    int tma_q0 = -1, tma_q1 = -1, mma_q0 = -1, mma_q1 = -1;   // thread 0: in flight (-1: nothing)
    auto tma_q = [&](int k) -> int & { return k ? tma_q1 : tma_q0; };
    auto mma_q = [&](int k) -> int & { return k ? mma_q1 : mma_q0; };
    bool ok = true;
    if (t == 0) {
        if (nq > 0) { issue_rows(0); tma_q(0) = 0; }
        if (nq > 1) { issue_rows(1); tma_q(1) = 1; }
        constexpr uint32_t idesc = tc_idesc_bf16(128, GCH) | (1u << 15) | (1u << 16);   // A and B MN-major
        for (int q = 0; q < nq && ok; ++q) {
            const int b = q & 1;
            ok = mbar_wait(&bar_tma[b], (q >> 1) & 1);
            if (!ok) break;
            tma_q(b) = -1;
            tc_fence_after();
            const uint32_t sa_u = smem_u32(sm_raw + b * kWgStageBytes), sg_u = smem_u32(sg0 + b * GBYTES);
#pragma unroll 1
            for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                for (int ks = 0; ks < kTile / 16; ++ks)
                    tc_mma_bf16(tmem + (uint32_t)(dx * GCH), tc_sdesc(sa_u + dx * 16 + ks * 256, 128, kChunkBytes),
                                tc_sdesc(sg_u + ks * 256, 128, kChunkBytes), idesc, (q > 0 || ks > 0) ? 1u : 0u);
            tc_commit(&bar_mma[b]);
            mma_q(b) = q;
            if (q + 1 < nq && q >= 1) {   // stage b ^ 1 is free once tile q-1's MMAs are done: tile q+1
                ok = mbar_wait(&bar_mma[b ^ 1], ((q - 1) >> 1) & 1);
                if (!ok) break;
                mma_q(b ^ 1) = -1;
                issue_rows(q + 1);
                tma_q(b ^ 1) = q + 1;
            }
        }
        if (ok && nq > 0) {   // the last tile's MMAs complete after all earlier ones (commit order)
            ok = mbar_wait(&bar_mma[(nq - 1) & 1], ((nq - 1) >> 1) & 1);
            if (ok) mma_q0 = mma_q1 = -1;
        }
        if (!ok) {
            atomicExch(status, (int)SUPCG_ERR_TIMEOUT);
            for (int k = 0; k < 2; ++k) {
                if (mma_q(k) >= 0) (void)mbar_wait(&bar_mma[k], (mma_q(k) >> 1) & 1);
                if (tma_q(k) >= 0) (void)mbar_wait(&bar_tma[k], (tma_q(k) >> 1) & 1);
            }
        }
    }
    ok = __syncthreads_and(ok);
    tc_fence_after();
    if (ok && nq > 0) {
        // lane m = warp * 32 + lane: chunk m / 8 (dy = chunk / CH8, ci = (chunk % CH8) * 8 + m % 8) or the ones
        const int m = warp * 32 + (t & 31), chunk = m >> 3;
        const int len = cout * cin_real * 9 + cout;
        float *out = partial + (size_t)blockIdx.x * len;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        for (int dx = 0; dx < 3; ++dx) {
            float acc[GCH];
#pragma unroll
            for (int c = 0; c < GCH; c += 16) tc_ld16(lane_addr + (uint32_t)(dx * GCH + c), acc + c);
            if (chunk < ONES) {
                const int dy = chunk / CH8, ci = (chunk % CH8) * 8 + (m & 7);
                if (ci < cin_real)
#pragma unroll
                    for (int co = 0; co < GCH; ++co)
                        if (co < cout) out[(co * cin_real + ci) * 9 + dy * 3 + dx] = acc[co];
            } else if (chunk == ONES && (m & 7) == 0 && dx == 0) {
#pragma unroll
                for (int co = 0; co < GCH; ++co)
                    if (co < cout) out[cout * cin_real * 9 + co] = acc[co];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, 128);
}

constexpr int kWgradCtasPerSm = 2;

// Weight gradient of one layer into partial[grid][len]; returns the grid (the partial count) or an error (< 0).
template <int CIN, int GCH>
static int launch_wgrad(const __nv_bfloat16 *in, const __nv_bfloat16 *G, int cin_real, int cout, int ny, int nx,
                        int count, int max_ctas, float *partial, int *status, cudaStream_t st)
{
    constexpr int smem = 2 * kWgStageBytes + 2 * (GCH / 8) * kChunkBytes;
    const int rc0 = func_attrs_once((const void *)k_wgrad<CIN, GCH>, smem, (int)cudaSharedmemCarveoutMaxShared);
    if (rc0) return rc0;
    CUtensorMap tin, tg;
    int rc = nhwc_map(&tin, in, CIN, ny, nx, count, kBoxPix);
    if (!rc) rc = nhwc_map(&tg, G, GCH, ny, nx, count, kTile);
    if (rc) return rc;
    const long long tiles = (long long)count * ny * ((nx + kTile - 1) / kTile);
    const int grid = (int)std::min<long long>(tiles, max_ctas);
    k_wgrad<CIN, GCH><<<grid, 128, smem, st>>>(ny, nx, count, cin_real, cout, partial, status, tin, tg);
    SUPCG_CUDA_TRY(cudaGetLastError());
    return grid;
}

// out[e] = sum_b partial[b][e] in a fixed order: warp w of a block adds the
// partials b = w, w + 8, ... for 32 consecutive e (lane = e), then warp 0 adds
// the eight warp sums in warp order.
__global__ void __launch_bounds__(256) k_reduce(const float *partial, int nb, int len, float *out)
{
    __shared__ double sh[8][33];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int e = blockIdx.x * 32 + l;
    double s = 0.0;
    if (e < len)
        for (int b = w; b < nb; b += 8) s += (double)partial[(size_t)b * len + e];
    sh[w][l] = s;
    __syncthreads();
    if (w == 0 && e < len) {
        double tot = 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k) tot += sh[k][l];
        out[e] = (float)tot;
    }
}

// ------------------------------------------------------------------ input, loss, optimiser
// Per-image unit-RMS scale factors sqrt(n / sum x^2) and sqrt(n / sum tbar^2)
// (0 for an all-zero image).  Grid (nblk, count), nblk = norm_blocks(n) <= kNormBlocks:
// each block sums a contiguous part of one image in FP64; the image's last block
// adds the partials in block order (deterministic) and writes the two FP32 factors.
constexpr int kNormBlocks = 64;

static int norm_blocks(long long n) { return (int)std::max(1ll, std::min<long long>(kNormBlocks, n / 4096)); }

__global__ void __launch_bounds__(256) k_norms(const float *x, const float *tb, long long n, double *part,
                                               unsigned *counter, float *scale)
{
    __shared__ __align__(16) double red[40];
    __shared__ int sh_last;
    const int img = blockIdx.y, blk = blockIdx.x, nblk = gridDim.x;
    const long long per = (n + nblk - 1) / nblk;
    const long long e0 = blk * per, e1 = e0 + per < n ? e0 + per : n;
    const float *xi = x + img * n, *ti = tb + img * n;
    double sx = 0.0, st = 0.0;
    for (long long e = e0 + threadIdx.x; e < e1; e += 256) {
        const double u = xi[e], v = ti[e];
        sx += u * u;
        st += v * v;
    }
    sx = block_sum<256>(sx, red);
    st = block_sum<256>(st, red);
    if (threadIdx.x == 0) {
        part[(2 * img) * kNormBlocks + blk] = sx;
        part[(2 * img + 1) * kNormBlocks + blk] = st;
    }
    if (!last_block(&counter[img], nblk, &sh_last)) return;
    if (threadIdx.x < 2) {
        const volatile double *pp = part + (2 * img + threadIdx.x) * kNormBlocks;
        double s = 0.0;
        for (int k = 0; k < nblk; ++k) s += pp[k];
        scale[2 * img + threadIdx.x] = s > 0.0 ? (float)sqrt((double)n / s) : 0.0f;
    }
    if (threadIdx.x == 0) counter[img] = 0;   // ready for the next launch
}

// Input tensor: channel 0 = x / rms(x), channel 1 = tbar scaled to unit RMS,
// channels 2..15 = 0; resid = channel 1 in FP32.
__global__ void k_pack_input(const float *x, const float *tb, const float *scale, long long n, int count,
                             __nv_bfloat16 *act0, float *resid)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n * count) return;
    const long long img = p / n;
    const float v0 = x[p] * scale[2 * img], v1 = tb[p] * scale[2 * img + 1];
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
__global__ void __launch_bounds__(256) k_loss(const float *out, const float *target, const float *tscale,
                                              long long n, long long total, __nv_bfloat16 *G5, double *partial)
{
    __shared__ __align__(16) double red[40];
    double s = 0.0;
    const float scale = (float)(2.0 / (double)total);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const float ft = tscale[2 * (p / n)];
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

// Packed BF16 GEMM weights of layer l (forward) and of its input-gradient pass,
// as GEMM B operands B[row][k] (row = output channel, k = tap * channels + channel):
//   fwd: B[co][tap * cin + ci] = W[co][ci][tap]          (co < cout, ci < cin_real; else 0)
//   bwd: B[ci][tap * gch + co] = W[co][ci][8 - tap]      (flipped kernel, transposed channels)
// stored in the tensor cores' K-major core-matrix order (8 rows x 16 bytes per
// 128-byte block, blocks K-contiguous): element (row, k) at
// ((row / 8) * (K / 8) + k / 8) * 64 + (row % 8) * 8 + k % 8, so that one bulk
// copy puts it in shared memory ready for the MMA descriptors.
__device__ __forceinline__ int core_matrix_index(int row, int k, int K)
{
    return ((row >> 3) * (K >> 3) + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}

__global__ void k_pack_weights(const float *W, int cout, int cin, int cin_real, int nout, int kp,
                               __nv_bfloat16 *fwd, int gch, int kpb, __nv_bfloat16 *bwd)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nout * kp) {
        const int co = e / kp, k = e - co * kp;
        const int tap = k / cin, ci = k - tap * cin;
        float v = 0.0f;
        if (co < cout && tap < 9 && ci < cin_real) v = W[(co * cin_real + ci) * 9 + tap];
        fwd[core_matrix_index(co, k, kp)] = __float2bfloat16_rn(v);
    }
    if (bwd && e < kCh * kpb) {
        const int ci = e / kpb, k = e - ci * kpb;
        const int tap = k / gch, co = k - tap * gch;
        float v = 0.0f;
        if (ci < cin_real && tap < 9 && co < cout) v = W[(co * cin_real + ci) * 9 + (8 - tap)];
        bwd[core_matrix_index(ci, k, kpb)] = __float2bfloat16_rn(v);
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
    float *scales = nullptr, *tscales = nullptr;   // per image: factors of x and tbar (target) to unit RMS
    double *npart = nullptr, *lpart = nullptr;
    unsigned *ncount = nullptr;
    int *status = nullptr;
    size_t partial_len = 0;
    int wg_ctas = 1;              // weight-gradient CTAs (partials) per layer
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
    if (!out || ny < 1 || nx < 1 || max_batch < 1 || max_batch > 65535 || (long long)ny * nx * max_batch > (1ll << 31))
        return SUPCG_ERR_ARG;
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
    int dev = 0, nsm = 1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        rc = SUPCG_ERR_CUDA;
    net->wg_ctas = nsm * kWgradCtasPerSm;
    net->partial_len = (size_t)net->wg_ctas * (kCh * kCh * 9 + kCh);
    rc = rc ? rc : cnn_alloc(net, (void **)&net->partial, sizeof(float) * net->partial_len);
    rc = rc ? rc : cnn_alloc(net, (void **)&net->resid, sizeof(float) * npix);
    rc = rc ? rc : cnn_alloc(net, (void **)&net->out, sizeof(float) * npix);
    rc = rc ? rc : cnn_alloc(net, (void **)&net->scales, sizeof(float) * 2 * max_batch);
    rc = rc ? rc : cnn_alloc(net, (void **)&net->tscales, sizeof(float) * 2 * max_batch);
    rc = rc ? rc : cnn_alloc(net, (void **)&net->npart, sizeof(double) * 2 * kNormBlocks * max_batch);
    rc = rc ? rc : cnn_alloc(net, (void **)&net->ncount, sizeof(unsigned) * max_batch);
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
    k_norms<<<dim3(norm_blocks(n), count), 256, 0, st>>>(d_x, d_tbar, n, net->npart, net->ncount, net->scales);
    k_pack_input<<<(unsigned)((n * count + 255) / 256), 256, 0, st>>>(d_x, d_tbar, net->scales, n, count, net->act[0],
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
    ConvArgs a = {};
    a.ny = net->ny;
    a.nx = net->nx;
    a.count = count;
    a.status = net->status;
    for (int l = kCnnLayers - 1; l >= 0; --l) {
        const int cin_real = l_cin_real(l), cout = l_cout(l);
        // weight gradient of layer l: input act[l], output gradient gbuf[l]
        int nb;
        if (l == 0)
            nb = launch_wgrad<kInCh, kCh>(net->act[0], net->gbuf[0], cin_real, cout, net->ny, net->nx, count,
                                          net->wg_ctas, net->partial, net->status, st);
        else if (l == kCnnLayers - 1)
            nb = launch_wgrad<kCh, kInCh>(net->act[l], net->gbuf[l], cin_real, cout, net->ny, net->nx, count,
                                          net->wg_ctas, net->partial, net->status, st);
        else
            nb = launch_wgrad<kCh, kCh>(net->act[l], net->gbuf[l], cin_real, cout, net->ny, net->nx, count,
                                        net->wg_ctas, net->partial, net->status, st);
        if (nb < 0) return nb;
        const int len = cout * cin_real * 9 + cout;
        k_reduce<<<(len + 31) / 32, 256, 0, st>>>(net->partial, nb, len, net->grads + net->off_w[l]);
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
    k_norms<<<dim3(norm_blocks(n), count), 256, 0, st>>>(d_target, d_target, n, net->npart, net->ncount, net->tscales);
    k_loss<<<blocks, 256, 0, st>>>(net->out, d_target, net->tscales, n, total, net->gbuf[kCnnLayers - 1], net->lpart);
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
int cnn_capacity(supcg_cnn net, int *max_batch)
{
    *max_batch = net->cap;
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
