// bfloat16 tcgen05 tensor-core kernels of libdeepinv (sm_103a).
//
//  * tc_gemm   -- y = Phi x (Sec. 1) and the FC layer x~ = Phi^T y (Sec. 4);
//                 one or two 128-row tiles per CTA, optional split-K.
//  * conv1_tc  -- Eq. (1), layer 1 (1 -> 64 filters of 11 x 11): per kernel
//                 row one GEMM with M = 128 positions, N = 64 filters, K = 16
//                 columns, the A operand read straight from an expanded window.
//  * conv2_tc  -- layer 2 (64 -> 32), 95 % of the network's flops, as a
//                 tap-stacked implicit GEMM (below); the same kernel, as
//                 template variants, computes the e4m3 forward, conv2's input
//                 gradient and the hidden 32 -> 32 layers of deeper networks
//                 (forward and input gradient).
//  * conv3_tc  -- layer 3 (32 -> 1): per-row partial sums by GEMM (N = kernel
//                 row x column phase), summed over the 11 kernel rows in a
//                 shared-memory ring in the same kernel.
//
// Operands are K-major without swizzle (see tc.cuh; conv1's A is MN-major),
// moved by the TMA engine with 1-D bulk copies; accumulators live in TMEM.
#include <algorithm>
#include <climits>
#include <cstdlib>

#include <cuda_fp8.h>

#include "kernels.cuh"
#include "tc.cuh"

namespace di {

using namespace tc;

namespace {

__device__ __forceinline__ uint4 pack8_bf16(const float* v)
{
    uint4 r;
    uint32_t* u = reinterpret_cast<uint32_t*>(&r);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __nv_bfloat162 p = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        u[i] = *reinterpret_cast<uint32_t*>(&p);
    }
    return r;
}

// 16 floats scaled by `scale` -> 16 e4m3 bytes (round to nearest, saturating to +-448).
__device__ __forceinline__ uint4 pack16_e4m3(const float* v, float scale)
{
    uint4 r;
    uint32_t* u = reinterpret_cast<uint32_t*>(&r);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(v[4 * i] * scale, v[4 * i + 1] * scale),
                                                     __NV_SATFINITE, __NV_E4M3);
        const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(v[4 * i + 2] * scale, v[4 * i + 3] * scale),
                                                     __NV_SATFINITE, __NV_E4M3);
        u[i] = (lo & 0xFFFFu) | (hi << 16);
    }
    return r;
}


// ---------------------------------------------------------------- packing
__global__ void pack_kmajor_kernel(const float* __restrict__ src, long long rs, long long cs, int R,
                                   int K, int TR, int Kp, long long nchunks, bf16* __restrict__ dst)
{
    pdl_wait();
    pdl_trigger();
    const int kcs = Kp / 8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nchunks;
         i += (long long)gridDim.x * blockDim.x) {
        const int rr = (int)(i % TR);
        const int kc = (int)((i / TR) % kcs);
        const long long rt = i / ((long long)TR * kcs);
        const long long r = rt * TR + rr;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = kc * 8 + e;
            v[e] = (r < R && k < K) ? src[r * rs + (long long)k * cs] : 0.f;
        }
        reinterpret_cast<uint4*>(dst)[i] = pack8_bf16(v);
    }
}

// conv1 B operand: block (dy, h) holds rows n = filter co, K = columns
//   dx = 8 h .. 8 h + 7, weight W1[co][0][dy][dx] (zero for dx >= 11).
// conv2 A operand: block (dy, s, kk) holds rows m = 32 g + co (g = tap slot),
//   K = input channels 16 kk .. 16 kk + 15, weight W2[co][ci][dy][4 s + g]
//   (zero when 4 s + g = 11).
// conv3 B operand: block (x, kk) holds rows n = 4 dy + e, K = channels
//   16 kk .. 16 kk + 15, weight W3[0][ci][dy][4 x + e] (zero for dy >= 11 or
//   4 x + e >= 11).
__global__ void pack_conv_weights_kernel(const float* __restrict__ w1, const float* __restrict__ w2,
                                         const float* __restrict__ w3, bf16* __restrict__ w1p,
                                         bf16* __restrict__ w2p, bf16* __restrict__ w3p)
{
    const long long n1 = kW1PackElems, n2 = kW2PackElems, n3 = kW3PackElems;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n1 + n2 + n3;
         i += (long long)gridDim.x * blockDim.x) {
        if (i < n1) {
            const int e = (int)(i % 8), co = (int)((i / 8) % 64), blk = (int)(i / (8 * 64));
            const int dy = blk / 2, dx = (blk % 2) * 8 + e;
            const float v = dx < 11 ? w1[co * 121 + dy * 11 + dx] : 0.f;
            w1p[i] = __float2bfloat16_rn(v);
        } else if (i < n1 + n2) {
            const long long j = i - n1;
            const int e = (int)(j % 8);
            const int m = (int)((j / 8) % 128);
            const int half = (int)((j / (8 * 128)) % 2);
            const int kk = (int)((j / (8 * 128 * 2)) % 4);
            const int s = (int)((j / (8 * 128 * 2 * 4)) % 3);
            const int dy = (int)(j / (8 * 128 * 2 * 4 * 3));
            const int co = m % 32, g = m / 32, dx = 4 * s + g, ci = kk * 16 + half * 8 + e;
            const float v = dx < 11 ? w2[((co * 64 + ci) * 11 + dy) * 11 + dx] : 0.f;
            w2p[j] = __float2bfloat16_rn(v);
        } else {
            const long long j = i - n1 - n2;
            const int e8 = (int)(j % 8), n = (int)((j / 8) % 64), half = (int)((j / 512) % 2);
            const int kk = (int)((j / 1024) % 2), x = (int)(j / 2048);
            const int ci = kk * 16 + half * 8 + e8, dy = n / 4, dx = 4 * x + n % 4;
            const float v = (dy < 11 && dx < 11) ? w3[(ci * 11 + dy) * 11 + dx] : 0.f;
            w3p[j] = __float2bfloat16_rn(v);
        }
    }
}

// Hidden layer (32 -> 32) operands, conv2's layout with 2 chunk pairs: block
// (dy, s, kk) holds rows m = 32 g + r (tap slot g, row channel r), K =
// channels c = 16 kk .. 16 kk + 15; with dx = 4 s + g (zero for dx = 11)
//   forward (whp):        Wh[r][c][dy][dx]            (r = filter, c = input)
//   input gradient (wht): Wh[c][r][10 - dy][10 - dx]  (r = input, c = filter).
__global__ void pack_hidden_weights_kernel(const float* __restrict__ w, bf16* __restrict__ whp,
                                           bf16* __restrict__ wht)
{
    const long long n = kWhPackElems;
    const long long total = wht ? 2 * n : n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const bool dgrad = i >= n;
        const long long j = dgrad ? i - n : i;
        const int e = (int)(j % 8);
        const int m = (int)((j / 8) % 128);
        const int half = (int)((j / (8 * 128)) % 2);
        const int kk = (int)((j / (8 * 128 * 2)) % 2);
        const int s = (int)((j / (8 * 128 * 2 * 2)) % 3);
        const int dy = (int)(j / (8 * 128 * 2 * 2 * 3));
        const int r = m % 32, g = m / 32, dx = 4 * s + g, c = kk * 16 + half * 8 + e;
        float v = 0.f;
        if (dx < 11)
            v = dgrad ? w[((c * 32 + r) * 11 + (10 - dy)) * 11 + (10 - dx)] : w[((r * 32 + c) * 11 + dy) * 11 + dx];
        (dgrad ? wht : whp)[j] = __float2bfloat16_rn(v);
    }
}

// Per-filter absolute maximum of the conv2 weights: amax[co] = max |W2[co][.][.][.]|.
__global__ void conv2_absmax_kernel(const float* __restrict__ w2, float* __restrict__ amax)
{
    const int co = blockIdx.x;
    float m = 0.f;
    for (int i = threadIdx.x; i < 64 * 121; i += blockDim.x) m = fmaxf(m, fabsf(w2[(size_t)co * 64 * 121 + i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
        amax[co] = t;
    }
}

// conv2 A operand in e4m3 with a scale per filter, sw[co] = amax[co] / 448:
// block (dy, s, kk) holds rows m = 32 g + co, K = channels 32 kk .. 32 kk + 31
// as two 16-byte chunks, value W2[co][ci][dy][4 s + g] / sw[co] (zero for 4 s + g = 11).
__global__ void pack_w2_e4m3_kernel(const float* __restrict__ w2, const float* __restrict__ amax,
                                    uint8_t* __restrict__ w2q, float* __restrict__ sw)
{
    const long long n = (long long)kW2E4M3Bytes;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(j % 16);
        const int m = (int)((j / 16) % 128);
        const int half = (int)((j / (16 * 128)) % 2);
        const int kk = (int)((j / (16 * 128 * 2)) % 2);
        const int s = (int)((j / (16 * 128 * 2 * 2)) % 3);
        const int dy = (int)(j / (16 * 128 * 2 * 2 * 3));
        const int co = m % 32, g = m / 32, dx = 4 * s + g, ci = kk * 32 + half * 16 + e;
        const float scale = amax[co] > 0.f ? amax[co] / 448.f : 1.f;
        if (j < 32) sw[j] = amax[j] > 0.f ? amax[j] / 448.f : 1.f;
        const float v = dx < 11 ? w2[((co * 64 + ci) * 11 + dy) * 11 + dx] / scale : 0.f;
        w2q[j] = (uint8_t)(__nv_cvt_float2_to_fp8x2(make_float2(v, 0.f), __NV_SATFINITE, __NV_E4M3) & 0xFFu);
    }
}

// Activation scale of the e4m3 path from the calibrated maximum of a1:
// sa = amax / 448, inv_sa = 1 / sa, oscale[co] = sw[co] * sa.
__global__ void e4m3_scales_kernel(const float* __restrict__ amax_a1, const float* __restrict__ sw,
                                   float* __restrict__ inv_sa, float* __restrict__ oscale)
{
    const float a = *amax_a1;
    const float sa = a > 0.f ? a / 448.f : 1.f;
    if (threadIdx.x == 0) *inv_sa = 1.f / sa;
    if (threadIdx.x < 32) oscale[threadIdx.x] = sw[threadIdx.x] * sa;
}

// ---------------------------------------------------------------- GEMM
// One 128 x NB output tile per CTA; K in stages of kGemmKS MMA steps (16 each).
// Warp 0 lane 0: producer (bulk copies).  Warp 1: TMEM owner and MMA issuer.
// Warps 2..5: epilogue (TMEM lane quarter = warp % 4).
constexpr int kGemmKS = 4;
constexpr int kGemmNS = 3;

struct GemmSmem {
    uint64_t full[kGemmNS], empty[kGemmNS], acc_full, drain;
    uint32_t tmem_base;
    int abort_flag;
};

__device__ __forceinline__ int plane_index(int j, int W, int P) { return (j / W) * P + (j % W) + kPad * P + kPad; }

// MT = 128-row tiles of A per CTA: with MT = 2 each B stage feeds two MMAs
// (two TMEM accumulators), so B is read once per 256 rows of A.
template <int MODE, int MT>
__global__ void __launch_bounds__(192, 1) tc_gemm_kernel(const bf16* __restrict__ A, const bf16* __restrict__ Bm,
                                                         int Kp, int Mr, int Nc, int NB, uint32_t tmem_cols,
                                                         float* __restrict__ out_f32, long long ldo,
                                                         bf16* __restrict__ plane, int H, int W, int P,
                                                         int plane_len, int* status)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = smem_raw;
    const uint32_t a_tile = kGemmKS * 4096;                // one row tile's share of a stage
    const uint32_t a_stage = MT * a_tile;
    const uint32_t b_stage = (uint32_t)kGemmKS * NB * 32;
    uint8_t* sA = smem;
    uint8_t* sB = smem + kGemmNS * a_stage;
    GemmSmem* ss = reinterpret_cast<GemmSmem*>(sB + kGemmNS * b_stage);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int mt = blockIdx.x, nt = blockIdx.y;
    const int mtiles = min(MT, (Mr + 127) / 128 - mt * MT);   // row tiles of this CTA (the last may have one)
    // split-K: this CTA sums MMA steps [s0, s1) of the Kp / 16 and writes slice z
    const int ksplit = gridDim.z, z = blockIdx.z;
    const int nsteps_all = Kp / 16;
    const int s0 = nsteps_all * z / ksplit, s1 = nsteps_all * (z + 1) / ksplit;
    const int nsteps = s1 - s0;
    const int nstages = (nsteps + kGemmKS - 1) / kGemmKS;
    if (ksplit > 1) out_f32 += (size_t)z * Mr * ldo;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kGemmNS; ++s) {
            mbar_init(smem_u32(&ss->full[s]), 1);
            mbar_init(smem_u32(&ss->empty[s]), 1);
        }
        mbar_init(smem_u32(&ss->acc_full), 1);
        mbar_init(smem_u32(&ss->drain), 1);
        ss->abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(&ss->tmem_base), tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = ss->tmem_base;
    pdl_wait();
    pdl_trigger();

    if (warp == 0 && lane == 0) {
        // producer
        const bf16* Ablk = A + (size_t)mt * MT * (Kp / 8) * 128 * 8;
        const bf16* Bblk = Bm + (size_t)nt * (Kp / 8) * NB * 8;
        int armed_parity[kGemmNS];
        for (int s = 0; s < kGemmNS; ++s) armed_parity[s] = -1;
        for (int st = 0; st < nstages; ++st) {
            const int slot = st % kGemmNS, n = st / kGemmNS;
            if (!mbar_wait(smem_u32(&ss->empty[slot]), (n & 1) ^ 1, status, &ss->abort_flag)) break;
            const int k0 = s0 + st * kGemmKS;
            const int ks = min(kGemmKS, s1 - k0);
            const uint32_t abytes = ks * 4096, bbytes = ks * NB * 32;
            mbar_arrive_expect_tx(smem_u32(&ss->full[slot]), mtiles * abytes + bbytes);
            armed_parity[slot] = n & 1;
            for (int r = 0; r < mtiles; ++r)
                bulk_g2s(smem_u32(sA + slot * a_stage + r * a_tile),
                         Ablk + ((size_t)r * (Kp / 8) * 128 + (size_t)k0 * 2 * 128) * 8, abytes,
                         smem_u32(&ss->full[slot]));
            bulk_g2s(smem_u32(sB + slot * b_stage), Bblk + (size_t)k0 * 2 * NB * 8, bbytes,
                     smem_u32(&ss->full[slot]));
        }
        for (int s = 0; s < kGemmNS; ++s)
            if (armed_parity[s] >= 0) mbar_wait_drain(smem_u32(&ss->full[s]), armed_parity[s]);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = idesc_bf16(128, NB);
        bool ok = true;
        for (int st = 0; st < nstages && ok; ++st) {
            const int slot = st % kGemmNS, n = st / kGemmNS;
            if (!mbar_wait(smem_u32(&ss->full[slot]), n & 1, status, &ss->abort_flag)) { ok = false; break; }
            tc_fence_after();
            const int k0 = s0 + st * kGemmKS;
            const int ks = min(kGemmKS, s1 - k0);
            for (int j = 0; j < ks; ++j) {
                const uint64_t bd = sdesc(smem_u32(sB + slot * b_stage + j * NB * 32), NB * 16, 128);
                for (int r = 0; r < mtiles; ++r) {
                    const uint64_t ad = sdesc(smem_u32(sA + slot * a_stage + r * a_tile + j * 4096), 2048, 128);
                    mma_bf16(tbase + (uint32_t)(r * NB), ad, bd, idesc, (k0 + j) > s0 ? 1u : 0u);
                }
            }
            mma_commit(smem_u32(&ss->empty[slot]));
        }
        mma_commit(smem_u32(&ss->acc_full));
        mma_commit(smem_u32(&ss->drain));
        mbar_wait_drain(smem_u32(&ss->drain), 0);
    } else if (warp >= 2) {
        // epilogue
        const int q = warp % 4;
        bool ok = mbar_wait(smem_u32(&ss->acc_full), 0, status, &ss->abort_flag);
        ok = __all_sync(0xffffffffu, ok);
        tc_fence_after();
        for (int r = 0; r < mtiles && ok; ++r) {
            const int m = (mt * MT + r) * 128 + q * 32 + lane;
            for (int c0 = 0; c0 < NB; c0 += 16) {
                float v[16];
                if (nsteps > 0) {
                    tmem_ld16(tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(r * NB + c0), v);
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = 0.f;
                }
                if (m >= Mr) continue;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int n = nt * NB + c0 + i;
                    if (n >= Nc) break;
                    if (MODE == GEMM_OUT_F32) {
                        out_f32[(long long)m * ldo + n] = v[i];
                    } else {
                        plane[(size_t)n * plane_len + plane_index(m, W, P)] = __float2bfloat16_rn(v[i]);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tbase, tmem_cols);
    }
}

// Named barrier of the 128 epilogue threads (warps of one role).
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// ---------------------------------------------------------------- conv1
// Correlating one input channel with 11 x 11 kernels is, per kernel row dy, a
// GEMM with K = the 11 columns dx (padded to 16, weights of dx >= 11 zero).
// Its A operand (position m, column dx) = x~[q0 + m + dy P + dx] is read by
// the tensor core straight from an expanded window: row i of the window holds
// the 8 consecutive plane values x~[base + i .. base + i + 7], so the MN-major
// core matrix (K group h, M group mg) of kernel row dy is the 8 rows starting
// at dy P + 8 h + 8 mg; both core-matrix strides are 128 bytes and no im2col
// is built.  One piece of kC1Rows window rows per kernel row.
//
// Persistent CTAs over tiles of 128 positions, 13 warps: warps 8..11 expand
// the window of the next tile into a 2-stage ring; warp 12 owns TMEM (2
// accumulators) and one of its threads issues the 11 MMAs per tile; warps
// 0..7 drain an accumulator, warp w reading TMEM lane quarter w % 4 (32
// positions) and half w / 4 of the channels.  Each epilogue warp applies
// bias/ReLU (or the mode's transform) and stores its 32 positions straight to
// the output planes (one 512-byte run per channel chunk and warp), so the
// epilogue warps never wait on one another.
constexpr int kC1Rows = 144;                 // 8-value rows per piece (136 read + alignment)
constexpr int kC1Stride = kC1Rows + 1;       // piece stride in 16-byte rows (staggers banks)
constexpr int kC1Groups = kC1Rows / 8;       // 8-row groups per piece
constexpr int kC1Items = 11 * kC1Groups;     // groups per tile window
constexpr int kC1PerThread = (kC1Items + 127) / 128;
constexpr uint32_t kC1XBytes = 11 * kC1Stride * 16;
constexpr int kC1Threads = 416;

struct Conv1Smem {
    alignas(16) float bias[64];   // read as float4
    uint64_t wbar;
    uint64_t xfull[2], xempty[2];
    uint64_t afull[2], aempty[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort_flag;
};

__host__ __device__ constexpr uint32_t conv1_wbytes(int cout) { return 11u * 2u * cout * 16u; }
// 16-byte output chunks per position
__host__ __device__ constexpr int conv1_out_chunks(int cout, int mode)
{
    return mode == kConv1OutE4M3 ? cout / 16 : (mode == kConv1AmaxOnly ? 0 : cout / 8);
}

// Ring mode: one expanded window per CTA, row e = x~[e .. e + 7] of the image at
// ring row e mod RS (RS a power of two), its first kC1ETail rows repeated past
// the end so that no operand wraps.  Successive tiles share all but their last
// 128 rows, so each tile writes 16 groups instead of rebuilding 11 pieces.  A
// tile's window is 10 P + 136 rows; the producer of tile n may overwrite rows
// of tile n - 2 only, so RS >= 10 P + 272.
// The first tile of every image rebuilds the whole window and waits for the tile
// before it, so the ring pays only where images have many tiles (measured at
// batch 1024 / 256: 256 x 256, 536 tiles per image: 0.574 -> 0.551 ms; 64 x 64,
// 35 tiles: 0.1576 -> 0.1591 ms): images of fewer than 64 tiles keep the pieces.
constexpr int kC1ETail = 144;
constexpr int kC1ERingMax = 4096;
constexpr int kC1ERingMinTiles = 64;
static inline int conv1_ering(int P, int t1)
{
    if (t1 < kC1ERingMinTiles) return 0;
    const int need = 10 * P + 272;
    int rs = 1024;
    while (rs < need) rs *= 2;
    return rs <= kC1ERingMax ? rs : 0;
}
static inline size_t conv1_xbytes(int ering) { return ering ? (size_t)(ering + kC1ETail) * 16 : 2 * (size_t)kC1XBytes; }

// Window of tile (b, q0): piece dy starts at the 8-aligned plane index
// a = (q0 + dy P) & ~7, group j of it (rows 8 j .. 8 j + 7) comes from the 16
// values x~[a + 8 j .. a + 8 j + 15] (two aligned 16-byte loads; the plane
// holds at least t1 * 128 + 10 P + 24 values); row k of the group is values
// k .. k + 7 of those 16.  Items run dy-fastest so that the 8 lanes of one
// store phase mostly hit different banks.
__device__ __forceinline__ void conv1_load(const bf16* __restrict__ img, int q0, int P, int pt, uint4* lo, uint4* hi)
{
#pragma unroll
    for (int r = 0; r < kC1PerThread; ++r) {
        const int it = pt + r * 128;
        if (it < kC1Items) {
            const int dy = it % 11, j = it / 11;
            const uint4* src = reinterpret_cast<const uint4*>(img + ((q0 + dy * P) & ~7) + 8 * j);
            lo[r] = __ldg(src);
            hi[r] = __ldg(src + 1);
        }
    }
}

__device__ __forceinline__ void conv1_expand(uint4* sx, int pt, const uint4* lo, const uint4* hi)
{
#pragma unroll
    for (int r = 0; r < kC1PerThread; ++r) {
        const int it = pt + r * 128;
        if (it < kC1Items) {
            const int dy = it % 11, j = it / 11;
            const uint32_t w[8] = {lo[r].x, lo[r].y, lo[r].z, lo[r].w, hi[r].x, hi[r].y, hi[r].z, hi[r].w};
            uint4* dst = sx + dy * kC1Stride + 8 * j;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                uint32_t o[4];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    o[e] = (k & 1) ? __byte_perm(w[k / 2 + e], w[k / 2 + e + 1], 0x5432) : w[k / 2 + e];
                dst[k] = make_uint4(o[0], o[1], o[2], o[3]);
            }
        }
    }
}

// Tiles [lo, hi) of CTA `cta` out of `ncta`: contiguous, so that the image and
// tile index of successive tiles advance without divisions.
struct TileRange {
    int lo, hi;
};
__device__ __forceinline__ TileRange tile_range(int ntiles, int cta, int ncta)
{
    return {(int)((long long)ntiles * cta / ncta), (int)((long long)ntiles * (cta + 1) / ncta)};
}

// COUT = 64: conv1 itself.  COUT = 32 with mode kConv1GradMask: the input
// gradient of conv3 (one input channel, the gradient plane of x^, correlated
// with conv3's flipped kernels), times the ReLU mask of a2.
template <int COUT>
__global__ void __launch_bounds__(kC1Threads, 2) conv1_kernel(const bf16* __restrict__ xt, int B, int H, int W,
                                                              int P, int plane_len, int t1,
                                                              const bf16* __restrict__ w1p,
                                                              const float* __restrict__ b1, void* __restrict__ a1,
                                                              int mode, const float* __restrict__ inv_sa,
                                                              float* __restrict__ amax,
                                                              const bf16* __restrict__ mask_src, int ering,
                                                              int* status)
{
    constexpr uint32_t BBYTES = conv1_wbytes(COUT);
    constexpr int CPW = COUT / 2;                             // channels per epilogue warp
    constexpr uint32_t TCOLS = 2 * COUT < 32 ? 32 : 2 * COUT;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* sB = smem_raw;
    uint4* sX = reinterpret_cast<uint4*>(smem_raw + BBYTES);   // pieces [2][11][kC1Stride], or the ring
    const uint32_t xbytes = ering ? (uint32_t)(ering + kC1ETail) * 16u : 2u * kC1XBytes;
    Conv1Smem* ss = reinterpret_cast<Conv1Smem*>(smem_raw + BBYTES + xbytes);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int HP = H * P;
    const int ntiles = B * t1;

    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&ss->wbar), 1);
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&ss->xfull[s]), 128);
            mbar_init(smem_u32(&ss->xempty[s]), 1);
            mbar_init(smem_u32(&ss->afull[s]), 1);
            mbar_init(smem_u32(&ss->aempty[s]), 8);
        }
        mbar_init(smem_u32(&ss->drain), 1);
        ss->abort_flag = 0;
        fence_mbar_init();
    }
    if (threadIdx.x < 64) ss->bias[threadIdx.x] = (b1 && threadIdx.x < COUT) ? __ldg(&b1[threadIdx.x]) : 0.f;
    if (warp == 12) {
        tmem_alloc(smem_u32(&ss->tmem_base), TCOLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = ss->tmem_base;
    pdl_wait();
    pdl_trigger();

    if (warp >= 8 && warp < 12 && ering) {
        // ------------------------------------------------ window ring producers
        const int pt = threadIdx.x - 256;
        const TileRange tr = tile_range(ntiles, blockIdx.x, gridDim.x);
        const uint32_t rmask = (uint32_t)ering - 1u;
        auto put_group = [&](int G, uint4 lo, uint4 hi) {
            const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
            const uint32_t r0 = (uint32_t)(8 * G) & rmask;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                uint32_t o[4];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    o[e] = (k & 1) ? __byte_perm(w[k / 2 + e], w[k / 2 + e + 1], 0x5432) : w[k / 2 + e];
                const uint4 row = make_uint4(o[0], o[1], o[2], o[3]);
                sX[r0 + k] = row;
                if (r0 < (uint32_t)kC1ETail) sX[r0 + k + ering] = row;
            }
        };
        int b = tr.lo / t1, tt = tr.lo % t1, gnext = 0;
        // a tile after the first of an image adds 16 groups: threads pt < 16 load theirs
        // into registers before waiting for the slot, so that the load's latency overlaps
        // the wait
        int pG = -1;
        uint4 plo = make_uint4(0, 0, 0, 0), phi = plo;
        for (int tile = tr.lo, it = 0; tile < tr.hi; ++tile, ++it) {
            const int s = it & 1, use = it >> 1;
            // the rows written overwrite those of tile it - 2; a new image rewrites the
            // whole window, so tile it - 1 must be done too
            const bool fresh = tile == tr.lo || tt == 0;
            bool ok = mbar_wait(smem_u32(&ss->xempty[s]), (use & 1) ^ 1, status, &ss->abort_flag);
            if (ok && fresh && it > 0)
                ok = mbar_wait(smem_u32(&ss->xempty[(it - 1) & 1]), ((it - 1) >> 1) & 1, status, &ss->abort_flag);
            if (!ok) break;
            const int q0 = tt * 128;
            const int g1 = (q0 + 10 * P + 135) >> 3;
            const bf16* img = xt + (size_t)b * plane_len;
            if (fresh) {
                for (int G = (q0 >> 3) + pt; G <= g1; G += 128) {
                    const uint4* src = reinterpret_cast<const uint4*>(img + 8 * G);
                    put_group(G, __ldg(src), __ldg(src + 1));
                }
            } else if (pG >= 0) {
                put_group(pG, plo, phi);
            }
            gnext = g1 + 1;
            fence_proxy_async();
            mbar_arrive(smem_u32(&ss->xfull[s]));
            if (++tt == t1) {
                tt = 0;
                ++b;
            }
            pG = -1;
            if (tile + 1 < tr.hi && tt != 0 && pt < 16) {
                pG = gnext + pt;
                const uint4* src = reinterpret_cast<const uint4*>(img + 8 * pG);
                plo = __ldg(src);
                phi = __ldg(src + 1);
            }
        }
    } else if (warp >= 8 && warp < 12) {
        // ------------------------------------------------ window producers
        const int pt = threadIdx.x - 256;
        const TileRange tr = tile_range(ntiles, blockIdx.x, gridDim.x);
        uint4 lo[kC1PerThread], hi[kC1PerThread];
        int b = tr.lo / t1, tt = tr.lo % t1;
        if (tr.lo < tr.hi) conv1_load(xt + (size_t)b * plane_len, tt * 128, P, pt, lo, hi);
        for (int tile = tr.lo, it = 0; tile < tr.hi; ++tile, ++it) {
            const int s = it & 1, use = it >> 1;
            if (!mbar_wait(smem_u32(&ss->xempty[s]), (use & 1) ^ 1, status, &ss->abort_flag)) break;
            conv1_expand(sX + s * (11 * kC1Stride), pt, lo, hi);
            fence_proxy_async();
            mbar_arrive(smem_u32(&ss->xfull[s]));
            if (++tt == t1) {
                tt = 0;
                ++b;
            }
            if (tile + 1 < tr.hi) conv1_load(xt + (size_t)b * plane_len, tt * 128, P, pt, lo, hi);
        }
    } else if (warp == 12) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            bool ok = true;
            if (blockIdx.x < ntiles) {
                mbar_arrive_expect_tx(smem_u32(&ss->wbar), BBYTES);
                bulk_g2s(smem_u32(sB), w1p, BBYTES, smem_u32(&ss->wbar));
                ok = mbar_wait(smem_u32(&ss->wbar), 0, status, &ss->abort_flag);
                if (!ok) mbar_wait_drain(smem_u32(&ss->wbar), 0);
            }
            // A MN-major (bit 15), B K-major
            const uint32_t idesc = idesc_bf16(128, COUT) | (1u << 15);
            const TileRange tr = tile_range(ntiles, blockIdx.x, gridDim.x);
            int tt = tr.lo % t1;
            for (int tile = tr.lo, it = 0; tile < tr.hi && ok; ++tile, ++it, tt = tt + 1 == t1 ? 0 : tt + 1) {
                const int s = it & 1, use = it >> 1;
                if (!mbar_wait(smem_u32(&ss->aempty[s]), (use & 1) ^ 1, status, &ss->abort_flag)) break;
                if (!mbar_wait(smem_u32(&ss->xfull[s]), use & 1, status, &ss->abort_flag)) break;
                tc_fence_after();
                const int q0 = tt * 128;
                const uint32_t d = tbase + (uint32_t)(s * COUT);
                const uint4* sx = sX + s * (11 * kC1Stride);
#pragma unroll
                for (int dy = 0; dy < 11; ++dy) {
                    const int row = ering ? (int)((uint32_t)(q0 + dy * P) & (uint32_t)(ering - 1))
                                          : dy * kC1Stride + ((q0 + dy * P) & 7);
                    const uint64_t ad = sdesc(smem_u32((ering ? sX : sx) + row), 128, 128);
                    const uint64_t bd = sdesc(smem_u32(sB + dy * 2 * COUT * 16), COUT * 16, 128);
                    mma_bf16(d, ad, bd, idesc, dy > 0 ? 1u : 0u);
                }
                mma_commit(smem_u32(&ss->xempty[s]));
                mma_commit(smem_u32(&ss->afull[s]));
            }
            mma_commit(smem_u32(&ss->drain));
            mbar_wait_drain(smem_u32(&ss->drain), 0);
        }
    } else {
        // ------------------------------------------------ epilogue (warps 0..7)
        const int quarter = warp & 3, half = warp >> 2;
        const int c_lo = half * CPW;                          // first channel of this warp
        const int m = quarter * 32 + lane;                    // position within the tile = TMEM lane
        const float isa = mode == kConv1OutE4M3 ? __ldg(inv_sa) : 1.f;
        const int nch = conv1_out_chunks(COUT, mode);         // 16-byte chunks per position
        const int wch = nch / 2;                              // chunks of this warp
        float vmax = 0.f;
        const TileRange tr = tile_range(ntiles, blockIdx.x, gridDim.x);
        const int r128 = 128 % P;
        int b = tr.lo / t1, tt = tr.lo % t1;
        int col = (tt * 128 + m) % P;                         // column of this lane's position
        for (int tile = tr.lo, it = 0; tile < tr.hi; ++tile, ++it) {
            if (tile > tr.lo) {
                if (++tt == t1) {
                    tt = 0;
                    ++b;
                    col = m % P;
                } else {
                    col += r128;
                    if (col >= P) col -= P;
                }
            }
            const int s = it & 1, use = it >> 1;
            const bool ok = mbar_wait(smem_u32(&ss->afull[s]), use & 1, status, &ss->abort_flag);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc_fence_after();
            float v[CPW];
            if (CPW == 32) tmem_ld32(tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(s * COUT + c_lo), v);
            else tmem_ld16(tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(s * COUT + c_lo), v);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&ss->aempty[s]));
            const int q0 = tt * 128;
            const int qq = q0 + m;
            const bool valid = qq < HP;
            const bool data = valid && col < W;
            // chunk c of this warp: 16 bytes at plane position qq + 5 P + 5 of output chunk half * wch + c
            uint8_t* so = reinterpret_cast<uint8_t*>(a1) +
                          (((size_t)b * nch + half * wch) * plane_len + (size_t)(qq + kPad * P + kPad)) * 16;
            const size_t cstride = (size_t)plane_len * 16;
            if (mode == kConv1GradMask) {
                const size_t pos = (size_t)(qq + kPad * P + kPad);
#pragma unroll
                for (int c = 0; c < CPW / 8; ++c) {
                    uint4 mk = make_uint4(0, 0, 0, 0);
                    if (data)
                        mk = *reinterpret_cast<const uint4*>(
                            mask_src + (((size_t)b * (COUT / 8) + c_lo / 8 + c) * plane_len + pos) * 8);
                    const bf16* mv = reinterpret_cast<const bf16*>(&mk);
                    float o[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) o[i] = __bfloat162float(mv[i]) > 0.f ? v[8 * c + i] : 0.f;
                    if (valid) *reinterpret_cast<uint4*>(so + c * cstride) = pack8_bf16(o);
                }
            } else {
#pragma unroll
                for (int i = 0; i < CPW; i += 4) {
                    const float4 bb = *reinterpret_cast<const float4*>(&ss->bias[c_lo + i]);
                    v[i] = fmaxf(v[i] + bb.x, 0.f);
                    v[i + 1] = fmaxf(v[i + 1] + bb.y, 0.f);
                    v[i + 2] = fmaxf(v[i + 2] + bb.z, 0.f);
                    v[i + 3] = fmaxf(v[i + 3] + bb.w, 0.f);
                }
                // positions outside the image (pad columns, past the last row) store zeros
                const uint32_t keep = data ? 0xFFFFFFFFu : 0u;
                if (mode == kConv1OutBF16) {
#pragma unroll
                    for (int c = 0; c < CPW / 8; ++c) {
                        uint4 u = pack8_bf16(v + 8 * c);
                        u.x &= keep; u.y &= keep; u.z &= keep; u.w &= keep;
                        if (valid) *reinterpret_cast<uint4*>(so + c * cstride) = u;
                    }
                } else if (mode == kConv1OutE4M3) {
#pragma unroll
                    for (int c = 0; c < CPW / 16; ++c) {
                        uint4 u = pack16_e4m3(v + 16 * c, isa);
                        u.x &= keep; u.y &= keep; u.z &= keep; u.w &= keep;
                        if (valid) *reinterpret_cast<uint4*>(so + c * cstride) = u;
                    }
                } else if (data) {
#pragma unroll
                    for (int i = 0; i < CPW; ++i) vmax = fmaxf(vmax, v[i]);
                }
            }
        }
        if (mode == kConv1AmaxOnly) {
            for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
            if (lane == 0) atomicMax(reinterpret_cast<int*>(amax), __float_as_int(vmax));   // vmax >= 0
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 12) {
        tc_fence_after();
        tmem_dealloc(tbase, TCOLS);
    }
}

// ---------------------------------------------------------------- conv1, row tiles
// The same 11 MMAs per tile as conv1_kernel (kernel row dy: M = 128 positions,
// N = 64 filters, K = 16 columns dx, weights of dx >= 11 zero, issued in the
// same order), with the A operand in tensor memory and tiles aligned to image
// rows so that one A operand serves several tiles.  The image's columns are cut
// into nseg segments of Sw <= 128; a tile is R = 128 / Sw rows (at most
// kC1RMaxRows) of one segment, position m = i Sw + c (row i, column c) in TMEM
// lane m.  Kernel row dy of the tile whose first row is h0 reads the window
//   A_s(m, k) = x~[(s + i) P + c0 + c + k],   s = h0 + dy,
// which depends on s alone: the tile R rows further down reads the same window
// at dy - R.  A CTA walks its tiles in runs down a column of tiles (one image
// segment); a run of tiles rb0..rb1 reads windows s = R rb0 .. R rb1 + 10, each
// built once into a ring of kC1RSlots TMEM slots of 8 columns (16 bf16 of K per
// lane) and handed back once the last tile that reads it has its MMAs completed.
// Only image positions are computed; each tile's epilogue writes the zeros of
// the pad columns right of its rows.  Shared memory holds the weights and a ring
// of x~ row pieces, so the tensor core's shared-memory reads per tile are the 11
// B operands alone.
//
// Warp 13 copies the plane row pieces a run reads (Sw + 15 values from column
// c0, widened to 16-byte bounds) into a ring of kC1RRows slots with bulk copies.
// Warps 8..11 build windows: warp 8 + q owns TMEM lane quarter q; each thread
// reads the three 16-byte pieces around its 16 values from its row's slot (8
// neighbouring lanes read the same piece), shifts them into place and stores
// them with tcgen05.st.  Warp 12 owns TMEM (2 accumulators of 64 columns, then
// the window slots) and one of its threads issues the MMAs, committing each
// tile to its accumulator's barrier and to a tile-done barrier the builders
// wait on before reusing a slot.  Warps 0..7 drain an accumulator as in
// conv1_kernel (bias, ReLU, bf16 or scaled e4m3, 16-byte stores).
constexpr int kC1RThreads = 448;
constexpr int kC1RSlots = 16;
constexpr int kC1RMaxRows = kC1RSlots - 11;   // 11 windows in use + R being built
constexpr uint32_t kC1RCols = 256;            // 2 x 64 accumulator columns + 16 x 8 slot columns
constexpr int kC1RRows = 32;                  // x~ row piece slots
constexpr int kC1RRowElems = 160;             // >= 7 + 127 + 24 values a slot is read at
constexpr uint32_t kC1RRowBytes = kC1RRows * kC1RRowElems * 2;
constexpr int kC1RDone = 8;                   // tile-done barriers
constexpr int kC1RChunk = 3;                  // windows a builder pass produces

// Tiles of an image: nseg column segments of Sw columns (the last may be
// narrower) x nrb row blocks of R rows.
struct Conv1RGeo {
    int R, Sw, nseg, nrb;
};
// Row tiles are built where they fill at least 96 of the 128 TMEM lanes.
static inline bool conv1_rows_geo(const Geo& g, Conv1RGeo& r)
{
    r.nseg = cdiv(g.W, 128);
    r.Sw = cdiv(g.W, r.nseg);
    r.R = std::min(128 / r.Sw, kC1RMaxRows);
    r.nrb = cdiv(g.H, r.R);
    return r.R * r.Sw >= 96;
}

struct Conv1RSmem {
    alignas(16) float bias[64];
    uint64_t wbar;
    uint64_t rfull[kC1RRows], rempty[kC1RRows];
    uint64_t wfull[kC1RSlots];
    uint64_t tdone[kC1RDone];
    uint64_t afull[2], aempty[2];
    uint64_t drain;
    int rel[4][kC1RSlots];                    // per builder warp: tile that hands back each slot's window
    uint32_t tmem_base;
    int abort_flag;
};

// A run: tiles rb0..rb1 of column col (image b, segment starting at column c0).
struct Conv1RRun {
    int rb0, rb1, b, c0;
};
__device__ __forceinline__ Conv1RRun c1r_run(int tile, int hi, int nrb, int nseg, int Sw)
{
    const int col = tile / nrb, rb0 = tile - col * nrb;
    const int b = col / nseg;
    return {rb0, min(nrb - 1, rb0 + (hi - 1 - tile)), b, (col - b * nseg) * Sw};
}

// 16 consecutive bf16 starting at element o (0..7) of the 24 held in a, b, c,
// as 8 words (element 2 j in the low half of word j).
__device__ __forceinline__ void c1r_shift16(const uint4& a, const uint4& b, const uint4& c, int o, uint32_t* r)
{
    const uint32_t w[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
    uint32_t v[10], u[9];
#pragma unroll
    for (int j = 0; j < 10; ++j) v[j] = (o & 4) ? w[j + 2] : w[j];
#pragma unroll
    for (int j = 0; j < 9; ++j) u[j] = (o & 2) ? v[j + 1] : v[j];
    const uint32_t sel = (o & 1) ? 0x5432u : 0x3210u;
#pragma unroll
    for (int j = 0; j < 8; ++j) r[j] = __byte_perm(u[j], u[j + 1], sel);
}

__global__ void __launch_bounds__(kC1RThreads, 2) conv1_rows_kernel(const bf16* __restrict__ xt, int B, int H,
                                                                    int W, int P, int plane_len, Conv1RGeo rg,
                                                                    const bf16* __restrict__ w1p,
                                                                    const float* __restrict__ b1,
                                                                    void* __restrict__ a1, int mode,
                                                                    const float* __restrict__ inv_sa, int* status)
{
    constexpr uint32_t BBYTES = conv1_wbytes(64);
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* sB = smem_raw;
    uint8_t* sRow = smem_raw + BBYTES;                         // [kC1RRows][kC1RRowElems] bf16
    Conv1RSmem* ss = reinterpret_cast<Conv1RSmem*>(sRow + kC1RRowBytes);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int R = rg.R, Sw = rg.Sw, nrb = rg.nrb, nseg = rg.nseg;
    const int ntiles = B * nseg * nrb;

    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&ss->wbar), 1);
        for (int j = 0; j < kC1RRows; ++j) {
            mbar_init(smem_u32(&ss->rfull[j]), 1);
            mbar_init(smem_u32(&ss->rempty[j]), 4);
        }
        for (int j = 0; j < kC1RSlots; ++j) mbar_init(smem_u32(&ss->wfull[j]), 4);
        for (int j = 0; j < kC1RDone; ++j) mbar_init(smem_u32(&ss->tdone[j]), 1);
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&ss->afull[s]), 1);
            mbar_init(smem_u32(&ss->aempty[s]), 8);
        }
        mbar_init(smem_u32(&ss->drain), 1);
        ss->abort_flag = 0;
        fence_mbar_init();
    }
    if (threadIdx.x < 64) ss->bias[threadIdx.x] = b1 ? __ldg(&b1[threadIdx.x]) : 0.f;
    if (warp == 12) {
        tmem_alloc(smem_u32(&ss->tmem_base), kC1RCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = ss->tmem_base;
    pdl_wait();
    pdl_trigger();
    const TileRange tr = tile_range(ntiles, blockIdx.x, gridDim.x);

    if (warp == 13) {
        // ------------------------------------------------ x~ row pieces
        if (lane == 0) {
            uint32_t k = 0;
            bool ok = true;
            for (int tile = tr.lo; tile < tr.hi && ok;) {
                const Conv1RRun run = c1r_run(tile, tr.hi, nrb, nseg, Sw);
                const bf16* img = xt + (size_t)run.b * plane_len;
                const int r1 = R * run.rb1 + 10 + R - 1;
                for (int r = R * run.rb0; r <= r1; ++r, ++k) {
                    const uint32_t slot = k % kC1RRows;
                    ok = mbar_wait(smem_u32(&ss->rempty[slot]), ((k / kC1RRows) & 1) ^ 1, status, &ss->abort_flag);
                    if (!ok) break;
                    const int e0 = r * P + run.c0, ea = e0 & ~7;
                    const int ee = min((e0 + Sw + 15 + 7) & ~7, plane_len);
                    if (ee > ea) {
                        mbar_arrive_expect_tx(smem_u32(&ss->rfull[slot]), (uint32_t)(ee - ea) * 2u);
                        bulk_g2s(smem_u32(sRow + slot * (kC1RRowElems * 2)), img + ea, (uint32_t)(ee - ea) * 2u,
                                 smem_u32(&ss->rfull[slot]));
                    } else {
                        mbar_arrive(smem_u32(&ss->rfull[slot]));   // past the plane: only discarded lanes read it
                    }
                }
                tile += run.rb1 - run.rb0 + 1;
            }
            // let copies in flight land before the CTA ends
            for (uint32_t kk = k > (uint32_t)kC1RRows ? k - kC1RRows : 0; kk < k; ++kk)
                mbar_wait_drain(smem_u32(&ss->rfull[kk % kC1RRows]), (kk / kC1RRows) & 1);
        }
    } else if (warp >= 8 && warp < 12) {
        // ------------------------------------------------ window builders
        // Windows go in chunks of up to kC1RChunk consecutive windows of a run: one
        // wait for their rows, their pieces read and shifted, one wait for their
        // slots, their TMEM stores issued back to back and completed together.
        const int q = warp - 8;
        const int m = threadIdx.x - 256;                      // TMEM lane = 32 q + lane
        const int mi = m / Sw, mc = m - (m / Sw) * Sw;        // row and column in the tile
        const bool live = mi < R;
        const uint32_t tlane = tbase + ((uint32_t)(32 * q) << 16) + 128u;
        int* rel = ss->rel[q];
        uint32_t n = 0, k0 = 0, rwaited = 0, rfreed = 0;
        int it0 = 0;                                          // CTA tile index of the run's first tile
        bool ok = true;
        for (int tile = tr.lo; tile < tr.hi && ok;) {
            const Conv1RRun run = c1r_run(tile, tr.hi, nrb, nseg, Sw);
            const int s0 = R * run.rb0, s1 = R * run.rb1 + 10;
            for (int sa = s0; sa <= s1; sa += kC1RChunk) {
                const int g = min(kC1RChunk, s1 - sa + 1);
                // rows sa .. sa + g - 1 + R - 1 of the run: row numbers k0 + (row - s0)
                const uint32_t kmax = k0 + (uint32_t)(sa + g - 1 - s0 + R - 1);
                for (; rwaited <= kmax && ok; ++rwaited)
                    ok = mbar_wait(smem_u32(&ss->rfull[rwaited % kC1RRows]), (rwaited / kC1RRows) & 1, status,
                                   &ss->abort_flag);
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                uint32_t r[kC1RChunk][8];
#pragma unroll
                for (int j = 0; j < kC1RChunk; ++j) {
                    if (j < g) {
                        uint4 x0 = make_uint4(0, 0, 0, 0), x1 = x0, x2 = x0;
                        int o = 0;
                        if (live) {
                            const int e0 = (sa + j + mi) * P + run.c0;
                            const int off = (e0 & 7) + mc;
                            const uint32_t a = smem_u32(sRow) +
                                               ((k0 + (uint32_t)(sa + j - s0 + mi)) % kC1RRows) * (kC1RRowElems * 2) +
                                               (uint32_t)(off & ~7) * 2u;
                            x0 = lds128(a);
                            x1 = lds128(a + 16);
                            x2 = lds128(a + 32);
                            o = off & 7;
                        }
                        c1r_shift16(x0, x1, x2, o, r[j]);
                    }
                }
                // rows no later window of the run reads go back to the copier
                __syncwarp();
                const int slast = sa + g - 1;
                const uint32_t kfree = slast < s1 ? k0 + (uint32_t)(slast - s0) : kmax;
                if (lane == 0)
                    for (uint32_t kk = rfreed; kk <= kfree; ++kk) mbar_arrive(smem_u32(&ss->rempty[kk % kC1RRows]));
                rfreed = kfree + 1;
                // the chunk's slots: free once the tile that read the last of their previous
                // windows is done (tiles complete in order)
                const uint32_t nlast = n + (uint32_t)g - 1u;
                if (nlast >= (uint32_t)kC1RSlots) {
                    const int itr = rel[nlast % kC1RSlots];
                    ok = mbar_wait(smem_u32(&ss->tdone[itr % kC1RDone]), (itr / kC1RDone) & 1, status,
                                   &ss->abort_flag);
                }
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                __syncwarp();
                if (lane == 0)
                    for (int j = 0; j < g; ++j) rel[(n + (uint32_t)j) % kC1RSlots] = it0 + min((sa + j) / R, run.rb1) - run.rb0;
                tc_fence_after();
#pragma unroll
                for (int j = 0; j < kC1RChunk; ++j)
                    if (j < g) tmem_st8_async(tlane + 8u * ((n + (uint32_t)j) % kC1RSlots), r[j]);
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0)
                    for (int j = 0; j < g; ++j) mbar_arrive(smem_u32(&ss->wfull[(n + (uint32_t)j) % kC1RSlots]));
                n += (uint32_t)g;
            }
            k0 += (uint32_t)(s1 - s0 + R);
            it0 += run.rb1 - run.rb0 + 1;
            tile += run.rb1 - run.rb0 + 1;
        }
    } else if (warp == 12) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            bool ok = true;
            if (tr.lo < tr.hi) {
                mbar_arrive_expect_tx(smem_u32(&ss->wbar), BBYTES);
                bulk_g2s(smem_u32(sB), w1p, BBYTES, smem_u32(&ss->wbar));
                ok = mbar_wait(smem_u32(&ss->wbar), 0, status, &ss->abort_flag);
                if (!ok) mbar_wait_drain(smem_u32(&ss->wbar), 0);
            }
            const uint32_t idesc = idesc_bf16(128, 64);      // A from TMEM, B K-major
            uint64_t bd[11];
#pragma unroll
            for (int dy = 0; dy < 11; ++dy) bd[dy] = sdesc(smem_u32(sB + dy * 2 * 64 * 16), 64 * 16, 128);
            uint32_t waited = 0, nrun = 0;
            int it = 0;
            for (int tile = tr.lo; tile < tr.hi && ok;) {
                const Conv1RRun run = c1r_run(tile, tr.hi, nrb, nseg, Sw);
                for (int rb = run.rb0; rb <= run.rb1; ++rb, ++it) {
                    const uint32_t n0 = nrun + (uint32_t)(R * (rb - run.rb0));   // window of kernel row 0
                    for (; waited <= n0 + 10u && ok; ++waited)
                        ok = mbar_wait(smem_u32(&ss->wfull[waited % kC1RSlots]), (waited / kC1RSlots) & 1, status,
                                       &ss->abort_flag);
                    if (!ok) break;
                    const int a = it & 1, ause = it >> 1;
                    if (!mbar_wait(smem_u32(&ss->aempty[a]), (ause & 1) ^ 1, status, &ss->abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tbase + (uint32_t)(64 * a);
#pragma unroll
                    for (int dy = 0; dy < 11; ++dy)
                        mma_bf16_ta(d, tbase + 128u + 8u * ((n0 + (uint32_t)dy) % kC1RSlots), bd[dy], idesc,
                                    dy > 0 ? 1u : 0u);
                    mma_commit(smem_u32(&ss->afull[a]));
                    mma_commit(smem_u32(&ss->tdone[it % kC1RDone]));
                }
                nrun += (uint32_t)(R * (run.rb1 - run.rb0) + 11);
                tile += run.rb1 - run.rb0 + 1;
            }
            mma_commit(smem_u32(&ss->drain));
            mbar_wait_drain(smem_u32(&ss->drain), 0);
        }
    } else {
        // ------------------------------------------------ epilogue (warps 0..7)
        const int quarter = warp & 3, half = warp >> 2;
        const int m = quarter * 32 + lane;
        const int mi = m / Sw, mc = m - (m / Sw) * Sw;
        const float isa = mode == kConv1OutE4M3 ? __ldg(inv_sa) : 1.f;
        const int nch = conv1_out_chunks(64, mode);
        const int wch = nch / 2;
        const size_t cstride = (size_t)plane_len * 16;
        int col = tr.lo / nrb, rb = tr.lo % nrb;
        for (int tile = tr.lo, it = 0; tile < tr.hi; ++tile, ++it) {
            if (tile > tr.lo && ++rb == nrb) {
                rb = 0;
                ++col;
            }
            const int b = col / nseg, sg = col - b * nseg;
            uint8_t* img = reinterpret_cast<uint8_t*>(a1) + (size_t)b * nch * cstride;
            // the 5 pad positions right of each row of the last segment hold zeros
            // (R * 5 * nch <= 200 16-byte chunks: one per thread at most)
            if (sg == nseg - 1) {
                const int per_row = kPad * nch, e = half * 128 + m;
                const int i = e / per_row, rem = e - i * per_row;
                const int j = rem / nch, ch = rem - j * nch;
                const int hh = R * rb + i;
                if (i < R && hh < H)
                    *reinterpret_cast<uint4*>(img + ch * cstride + ((size_t)(hh + kPad + 1) * P + j) * 16) =
                        make_uint4(0, 0, 0, 0);
            }
            const int a = it & 1, ause = it >> 1;
            const bool ok = mbar_wait(smem_u32(&ss->afull[a]), ause & 1, status, &ss->abort_flag);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc_fence_after();
            float v[32];
            tmem_ld32(tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(64 * a + 32 * half), v);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&ss->aempty[a]));
            const int h = R * rb + mi, w = sg * Sw + mc;
            const bool valid = mi < R && h < H && w < W;
#pragma unroll
            for (int i = 0; i < 32; i += 4) {
                const float4 bb = *reinterpret_cast<const float4*>(&ss->bias[32 * half + i]);
                v[i] = fmaxf(v[i] + bb.x, 0.f);
                v[i + 1] = fmaxf(v[i + 1] + bb.y, 0.f);
                v[i + 2] = fmaxf(v[i + 2] + bb.z, 0.f);
                v[i + 3] = fmaxf(v[i + 3] + bb.w, 0.f);
            }
            if (valid) {
                uint8_t* so = img + half * wch * cstride + ((size_t)(h + kPad) * P + kPad + w) * 16;
                if (mode == kConv1OutBF16) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) *reinterpret_cast<uint4*>(so + c * cstride) = pack8_bf16(v + 8 * c);
                } else {
#pragma unroll
                    for (int c = 0; c < 2; ++c)
                        *reinterpret_cast<uint4*>(so + c * cstride) = pack16_e4m3(v + 16 * c, isa);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 12) {
        tc_fence_after();
        tmem_dealloc(tbase, kC1RCols);
    }
}

// ---------------------------------------------------------------- conv2
// Tap-stacked implicit GEMM.  For kernel row dy and column group s (taps
// dx = 4 s + g, g = 0..3), one MMA with M = 128 rows (row 32 g + co: tap slot
// g, filter co), N = 256 positions and K = 16 channels computes
//   D_g[co][n] += sum_ci W2[co][ci][dy][4 s + g] a1[q0 + n + dy P + 4 s][ci],
// so that output q0 + j = sum_g D_g[co][j + g].  Slot g is TMEM lane quarter
// g, i.e. epilogue warp g: each warp reads its slot shifted by g columns, the
// four slots are added through a small shared-memory exchange, and each
// thread then stores 8 channels of one position as one 16-byte vector.
// 33 (dy, s) pairs x 4 channel chunks = 132 MMAs per tile, 253 valid outputs
// per tile (the last 3 columns lack their slot-3 partner).
//
// Persistent CTAs, 7 warps: warp 6 streams the input and (row mode) the
// weights, warp 0 streams the weights in window mode; warp 1 owns TMEM (2
// accumulators x 256 columns) and issues MMAs; warps 2..5 drain the
// accumulator of the previous tile.
//
// Row mode (the default): for every kernel row dy one ring stage holds the
// 272 positions that row's MMAs read and the row's stacked weights (all its
// column groups), filled by one producer on one barrier; the ring is as deep
// as shared memory allows (conv2_row_slots: 2 stages of 82 KB for the bf16
// forward, 3 for the input gradient, 4 for the 4-chunk variants).  The MMA
// thread then waits and commits once per kernel row instead of once per
// (dy, s) weight block: both cost it about as long as an MMA issue, so this
// took conv2 from 1.27 to 1.20 ms at 64 x 64 and the 66-MMA variants (e4m3,
// hidden layers) 1.5x faster.
// Window mode (DEEPINV_CONV2_WINDOW=1, narrow images only) keeps the whole
// window of 10 P + 272 positions of a tile as slabs, freed as soon as the last
// kernel row reading them has been multiplied, with the weights in a separate
// ring of (dy, s) blocks; it streams fewer bytes but runs slower.
enum Conv2Variant {
    kC2Fwd = 0,       // conv2 forward, bf16: 64 -> 32 channels, bias + ReLU
    kC2FwdE4M3 = 1,   // conv2 forward, e4m3 input and weights
    kC2Dgrad = 2,     // conv2 input gradient: 32 -> 64 channels, 2 tap slots, mask of a1
    kHidFwd = 3,      // hidden layer forward: 32 -> 32 channels, bias + ReLU
    kHidDgrad = 4,    // hidden layer input gradient: 32 -> 32 channels, mask of its input
};
constexpr int kW2Stages = 4;
constexpr int kConv2Threads = 224;
constexpr int kMaxSlabs = 10;

constexpr int kPiecePx = 16 + kConv2N; // positions one kernel row's MMAs read (row mode; shift <= 10)
constexpr int kMaxRowSlots = 4;        // row-mode ring depth limit
constexpr int kXStride = 36;          // floats per row of the slot exchange (32 + 4 pad)
constexpr int kXBytes = 4 * 32 * kXStride * 4;

struct Conv2Smem {
    uint64_t full[kMaxSlabs], empty[kMaxSlabs];
    uint64_t wfull[kW2Stages], wempty[kW2Stages];
    uint64_t acc_full[2], acc_empty[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort_flag;
    int vote[2][4];
};

// Row of the slot exchange: x[j] = v[j + G] (the slot-G contribution to column j).
template <int G>
__device__ __forceinline__ void put_shifted(float* x, const float* v)
{
#pragma unroll
    for (int j = 0; j < 32; j += 4)
        *reinterpret_cast<float4*>(x + j) = make_float4(v[j + G], v[j + G + 1], v[j + G + 2], v[j + G + 3]);
}

// Row mode: kernel row dy of the tile starting at output q0 reads input positions
// q0 + dy P .. q0 + dy P + kPiecePx - 1; when they all lie in the zero rows above
// (below plane index 5 P + 5) or below the image (from (H + 5) P on) the row's
// products are zero, and its load and MMAs are skipped.
__device__ __forceinline__ bool conv2_row_zero(int q0, int dy, int P, int H)
{
    const int a = q0 + dy * P;
    return a + kPiecePx <= kPad * P + kPad || a >= (H + kPad) * P;
}

__host__ __device__ inline int conv2_dylast(int j, int P)
{
    const int d = (j * kSlabPx + kSlabPx - 1) / P;
    return d < 10 ? d : 10;
}

template <bool ROWS, int V>
__global__ void __launch_bounds__(kConv2Threads, 1) conv2_kernel(const void* __restrict__ a1, int B, int H, int W, int P,
                                                       int plane_len, int t2, int nslab,
                                                       const void* __restrict__ w2p,
                                                       const float* __restrict__ b2,
                                                       const float* __restrict__ oscale,
                                                       const bf16* __restrict__ mask_src, bf16* __restrict__ a2,
                                                       int* status)
{
    // Forward: 4 tap slots x 32 filters, input 64 channels.  bf16: 8 chunks of
    // 8 channels per position, K = 16 per MMA (4 MMAs per (dy, s)); e4m3: 4
    // chunks of 16 channels, K = 32 per MMA (2 MMAs per (dy, s)).
    // DGRAD (input gradient of conv2, a correlation of the 32-channel output
    // gradient with the flipped, transposed weights): 2 tap slots x 64 input
    // channels, taps dx = 2 s + g for s = 0..5, input 32 channels (4 chunks,
    // 2 MMAs per (dy, s)); the epilogue applies the ReLU mask of a1.
    // Hidden layers (32 -> 32, bf16): 4 tap slots x 32 filters like the
    // forward, input 32 channels (4 chunks, 2 MMAs per (dy, s)); kHidFwd adds
    // bias and ReLU, kHidDgrad (flipped, transposed weights) applies the ReLU
    // mask of the layer's input instead.
    constexpr bool FP8 = V == kC2FwdE4M3;
    constexpr bool DGRAD = V == kC2Dgrad;                     // 2 tap slots x 64 outputs
    constexpr bool MASK = V == kC2Dgrad || V == kHidDgrad;     // ReLU-mask epilogue, no bias
    constexpr int NCH = V == kC2Fwd ? 8 : 4;
    constexpr int KK = V == kC2Fwd ? 4 : 2;
    constexpr int GROUPS = DGRAD ? 6 : 3;      // column groups s per kernel row
    constexpr int SSTEP = DGRAD ? 2 : 4;       // taps per group (= position shift between groups)
    constexpr int MAXSHIFT = SSTEP * (GROUPS - 1);
    constexpr uint32_t WSTAGE = KK * 4096;
    constexpr bool FUSEDW = ROWS;                  // a kernel row's weights share its input piece's stage
    // zero border rows skipped (conv2_row_zero) in the 8-chunk forward and the input
    // gradient; the 66-MMA variants ran 8 % slower with the same skip and keep every row
    constexpr bool SKIPZ = ROWS && (V == kC2Fwd || V == kC2Dgrad);
    const int WRING = FUSEDW ? nslab * GROUPS : kW2Stages;   // weight blocks resident in shared memory
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // window mode: [NCH][nslab * 128][16 B]; row mode: [nslab pieces][NCH][kPiecePx][16 B]
    const uint32_t CH = ROWS ? (uint32_t)kPiecePx * 16 : (uint32_t)nslab * kSlabPx * 16;
    const uint32_t win_bytes = ROWS ? (uint32_t)nslab * NCH * CH : NCH * CH;
    uint8_t* sWin = smem_raw;
    uint8_t* sW = smem_raw + win_bytes;             // [WRING][WSTAGE]: row mode [nslab][GROUPS], window mode a ring
    float* sX = reinterpret_cast<float*>(sW + WRING * WSTAGE);   // [4 slots][32 filters][kXStride]
    Conv2Smem* ss = reinterpret_cast<Conv2Smem*>(sW + WRING * WSTAGE + kXBytes);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int HP = H * P;
    const int ntiles = B * t2;

    if (threadIdx.x == 0) {
        for (int j = 0; j < nslab; ++j) {
            mbar_init(smem_u32(&ss->full[j]), 1);
            mbar_init(smem_u32(&ss->empty[j]), 1);
        }
        for (int s = 0; s < kW2Stages; ++s) {
            mbar_init(smem_u32(&ss->wfull[s]), 1);
            mbar_init(smem_u32(&ss->wempty[s]), 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&ss->acc_full[s]), 1);
            mbar_init(smem_u32(&ss->acc_empty[s]), 4);
        }
        mbar_init(smem_u32(&ss->drain), 1);
        ss->abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(&ss->tmem_base), 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = ss->tmem_base;
    pdl_wait();
    pdl_trigger();

    if (warp == 6 && lane == 0) {
        // ------------------------------------------------ window producer
        // Runs ahead on its own: the slabs of the next tile are loaded as soon as the
        // kernel rows that read the previous tile's slabs have been multiplied, not in
        // step with the weight stream.
        int slab_parity[kMaxSlabs];
        for (int j = 0; j < kMaxSlabs; ++j) slab_parity[j] = -1;
        int it = 0, pc = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it) {
            const int b = tile / t2, q0 = (tile % t2) * kConv2Valid;
            const uint8_t* src_img = reinterpret_cast<const uint8_t*>(a1) + (size_t)b * NCH * plane_len * 16;
            int next_slab = 0;
            for (int dy = 0; dy < 11 && ok; ++dy) {
                if (SKIPZ && conv2_row_zero(q0, dy, P, H)) continue;
                if (ROWS) {
                    const int slot = pc % nslab, n = pc / nslab;
                    ++pc;
                    if (!mbar_wait(smem_u32(&ss->empty[slot]), (n & 1) ^ 1, status, &ss->abort_flag)) { ok = false; break; }
                    mbar_arrive_expect_tx(smem_u32(&ss->full[slot]), NCH * kPiecePx * 16 + (FUSEDW ? GROUPS * WSTAGE : 0));
                    slab_parity[slot] = n & 1;
                    for (int c = 0; c < NCH; ++c)
                        bulk_g2s(smem_u32(sWin + (slot * NCH + c) * CH),
                                 src_img + ((size_t)c * plane_len + q0 + dy * P) * 16, kPiecePx * 16,
                                 smem_u32(&ss->full[slot]));
                    if (FUSEDW)
                        bulk_g2s(smem_u32(sW + slot * GROUPS * WSTAGE),
                                 reinterpret_cast<const uint8_t*>(w2p) + (size_t)dy * GROUPS * WSTAGE, GROUPS * WSTAGE,
                                 smem_u32(&ss->full[slot]));
                }
                const int last = ROWS ? -1 : (dy * P + MAXSHIFT + kConv2N - 1) / kSlabPx;
                while (next_slab <= last) {
                    const int j = next_slab++;
                    if (!mbar_wait(smem_u32(&ss->empty[j]), (it & 1) ^ 1, status, &ss->abort_flag)) { ok = false; break; }
                    mbar_arrive_expect_tx(smem_u32(&ss->full[j]), NCH * kSlabPx * 16);
                    slab_parity[j] = it & 1;
                    for (int c = 0; c < NCH; ++c)
                        bulk_g2s(smem_u32(sWin + c * CH + j * kSlabPx * 16),
                                 src_img + ((size_t)c * plane_len + q0 + j * kSlabPx) * 16, kSlabPx * 16,
                                 smem_u32(&ss->full[j]));
                }
            }
        }
        for (int j = 0; j < nslab; ++j)
            if (slab_parity[j] >= 0) mbar_wait_drain(smem_u32(&ss->full[j]), slab_parity[j]);
    } else if (warp == 0 && lane == 0 && !FUSEDW) {
        // ------------------------------------------------ weight producer
        int w_parity[kW2Stages];
        for (int s = 0; s < kW2Stages; ++s) w_parity[s] = -1;
        int wst = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            for (int dy = 0; dy < 11 && ok; ++dy) {
                for (int s = 0; s < GROUPS && ok; ++s, ++wst) {
                    const int slot = wst % kW2Stages, n = wst / kW2Stages;
                    if (!mbar_wait(smem_u32(&ss->wempty[slot]), (n & 1) ^ 1, status, &ss->abort_flag)) { ok = false; break; }
                    mbar_arrive_expect_tx(smem_u32(&ss->wfull[slot]), WSTAGE);
                    w_parity[slot] = n & 1;
                    bulk_g2s(smem_u32(sW + slot * WSTAGE),
                             reinterpret_cast<const uint8_t*>(w2p) + (size_t)(dy * GROUPS + s) * WSTAGE, WSTAGE,
                             smem_u32(&ss->wfull[slot]));
                }
            }
        }
        for (int s = 0; s < kW2Stages; ++s)
            if (w_parity[s] >= 0) mbar_wait_drain(smem_u32(&ss->wfull[s]), w_parity[s]);
    } else if (warp == 1 && lane == 0) {
        // ------------------------------------------------ MMA issuer
        const uint32_t idesc = FP8 ? idesc_e4m3(128, kConv2N) : idesc_bf16(128, kConv2N);
        int it = 0, wst = 0, pc = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it) {
            const int buf = it & 1, use = it >> 1;
            if (!mbar_wait(smem_u32(&ss->acc_empty[buf]), (use & 1) ^ 1, status, &ss->abort_flag)) { ok = false; break; }
            tc_fence_after();
            const uint32_t d = tbase + (uint32_t)buf * kConv2N;
            const int q0 = SKIPZ ? (tile % t2) * kConv2Valid : 0;
            int next_wait = 0, next_free = 0;
            bool first = true;                          // no MMA of this tile issued yet
            for (int dy = 0; dy < 11 && ok; ++dy) {
                if (SKIPZ && conv2_row_zero(q0, dy, P, H)) continue;
                int slot = 0;
                uint32_t bbase, off;
                if (ROWS) {
                    slot = pc % nslab;
                    const int n = pc / nslab;
                    ++pc;
                    if (!mbar_wait(smem_u32(&ss->full[slot]), n & 1, status, &ss->abort_flag)) { ok = false; break; }
                    bbase = smem_u32(sWin + slot * NCH * CH);
                    off = 0;
                } else {
                    const int last = (dy * P + MAXSHIFT + kConv2N - 1) / kSlabPx;
                    while (next_wait <= last) {
                        if (!mbar_wait(smem_u32(&ss->full[next_wait]), it & 1, status, &ss->abort_flag)) { ok = false; break; }
                        ++next_wait;
                    }
                    bbase = smem_u32(sWin);
                    off = (uint32_t)(dy * P) * 16;
                }
                if (!ok) break;
                tc_fence_after();
                for (int s = 0; s < GROUPS; ++s, ++wst) {
                    const int wslot = FUSEDW ? slot * GROUPS + s : wst % kW2Stages, n = wst / kW2Stages;
                    if (!FUSEDW) {
                        if (!mbar_wait(smem_u32(&ss->wfull[wslot]), n & 1, status, &ss->abort_flag)) { ok = false; break; }
                        tc_fence_after();
                    }
                    const uint32_t boff = off + (uint32_t)(SSTEP * s) * 16;
#pragma unroll
                    for (int kk = 0; kk < KK; ++kk) {
                        const uint64_t ad = sdesc(smem_u32(sW + wslot * WSTAGE + kk * 4096), 2048, 128);
                        const uint64_t bd = sdesc(bbase + (2 * kk) * CH + boff, CH, 128);
                        const uint32_t acc = SKIPZ ? ((!first || s || kk) ? 1u : 0u) : ((dy | s | kk) ? 1u : 0u);
                        if (FP8) mma_e4m3(d, ad, bd, idesc, acc);
                        else mma_bf16(d, ad, bd, idesc, acc);
                    }
                    if (!FUSEDW) mma_commit(smem_u32(&ss->wempty[wslot]));
                }
                if (!ok) break;
                if (SKIPZ) first = false;
                if (ROWS) mma_commit(smem_u32(&ss->empty[slot]));
                while (!ROWS && next_free < nslab && conv2_dylast(next_free, P) == dy) {
                    mma_commit(smem_u32(&ss->empty[next_free]));
                    ++next_free;
                }
            }
            if (!ok) break;
            mma_commit(smem_u32(&ss->acc_full[buf]));
        }
        mma_commit(smem_u32(&ss->drain));
        mbar_wait_drain(smem_u32(&ss->drain), 0);
    } else if (warp >= 2 && warp < 6) {
        // ------------------------------------------------ epilogue
        const int quarter = warp % 4;                         // TMEM lane quarter
        const int g = DGRAD ? quarter / 2 : quarter;          // tap slot of this warp's rows
        const int le = threadIdx.x - 64;                      // 0..127
        const int jl = le % 32;                               // sum phase: column jl of the chunk
        constexpr int ITEMS = DGRAD ? 2 : 1;                  // 8-channel groups per thread in the sum phase
        float bias8[8], scale8[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            bias8[e] = MASK ? 0.f : __ldg(&b2[(le / 32) * 8 + e]);
            scale8[e] = FP8 ? __ldg(&oscale[(le / 32) * 8 + e]) : 1.f;
        }
        float* xrow = sX + (quarter * 32 + lane) * kXStride;  // exchange row = TMEM lane (32 g + co or 64 g + co)
        int it = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const int buf = it & 1, use = it >> 1;
            bool ok = mbar_wait(smem_u32(&ss->acc_full[buf]), use & 1, status, &ss->abort_flag);
            ok = __all_sync(0xffffffffu, ok);
            if (lane == 0) ss->vote[buf][quarter] = ok ? 1 : 0;
            epi_bar();
            ok = ss->vote[buf][0] && ss->vote[buf][1] && ss->vote[buf][2] && ss->vote[buf][3];
            if (!ok) break;
            tc_fence_after();
            const int b = tile / t2, q0 = (tile % t2) * kConv2Valid;
            const uint32_t lane_addr = tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)buf * kConv2N;
            for (int cc = 0; cc < kConv2N; cc += 32) {
                const int jcol = cc + jl, qq = q0 + jcol;
                const bool store = jcol < kConv2Valid && qq < HP;
                const bool data = store && (qq % P) < W;
                const size_t pos = (size_t)(qq + kPad * P + kPad);
                constexpr int OUTCH = DGRAD ? 8 : 4;
                // ReLU masks of this thread's outputs, loaded before the TMEM read and
                // the slot exchange so that their latency overlaps them
                uint4 mk[ITEMS];
#pragma unroll
                for (int item = 0; item < ITEMS; ++item) {
                    mk[item] = make_uint4(0, 0, 0, 0);
                    if (MASK && data)
                        mk[item] = *reinterpret_cast<const uint4*>(
                            mask_src + (((size_t)b * OUTCH + le / 32 + 4 * item) * plane_len + pos) * 8);
                }
                float v[36];
                tmem_ld32(lane_addr + cc, v);
                if (cc + 32 < kConv2N) {
                    tmem_ld4(lane_addr + cc + 32, v + 32);
                } else {
                    v[32] = v[33] = v[34] = v[35] = 0.f;
                }
                switch (g) {
                    case 0: put_shifted<0>(xrow, v); break;
                    case 1: put_shifted<1>(xrow, v); break;
                    case 2: put_shifted<2>(xrow, v); break;
                    default: put_shifted<3>(xrow, v); break;
                }
                epi_bar();
#pragma unroll
                for (int item = 0; item < ITEMS; ++item) {
                    const int c8 = le / 32 + 4 * item;                // 8-channel group of the output
                    float acc[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        float t = 0.f;
                        if (DGRAD) {
                            t = sX[(c8 * 8 + e) * kXStride + jl] + sX[(64 + c8 * 8 + e) * kXStride + jl];
                        } else {
#pragma unroll
                            for (int gg = 0; gg < 4; ++gg) t += sX[(gg * 32 + c8 * 8 + e) * kXStride + jl];
                        }
                        acc[e] = FP8 ? fmaf(t, scale8[e], bias8[e]) : t + bias8[e];
                    }
                    if (store) {
                        bf16* dst = a2 + (((size_t)b * OUTCH + c8) * plane_len + pos) * 8;
                        if (MASK) {
                            // input gradient times the ReLU mask [input > 0]; zero outside the image
                            const bf16* mv = reinterpret_cast<const bf16*>(&mk[item]);
#pragma unroll
                            for (int e = 0; e < 8; ++e) acc[e] = (data && __bfloat162float(mv[e]) > 0.f) ? acc[e] : 0.f;
                        } else {
#pragma unroll
                            for (int e = 0; e < 8; ++e) acc[e] = data ? fmaxf(acc[e], 0.f) : 0.f;
                        }
                        *reinterpret_cast<uint4*>(dst) = pack8_bf16(acc);
                    }
                }
                epi_bar();
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&ss->acc_empty[buf]));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tbase, 512);
    }
}

// ---------------------------------------------------------------- conv3
// conv3 (one output channel) as row partial sums
//   T[p][dy] = sum_{dx, ci} W3[ci][dy][dx] a2[p + dx][ci],
// then xhat[q] = b3 + sum_dy T[q + dy P][dy].  With column groups x = 0..2
// (dx0 = 4 x) and column phases e = 0..3 (dx = 4 x + e), one tile of 128
// positions pstart + m accumulates
//   D[m][4 dy + e] = sum_x sum_ci W3[ci][dy][4 x + e] a2[pstart + m + 4 x][ci]
// (A = the input window shifted by 4 x rows, K = channels; B = 64 rows
// (dy, e), zero for dy >= 11 or dx >= 11): 3 x CIN / 16 MMAs with M = 128,
// N = 64.  The product of tap dx taken at input pstart + m + 4 x belongs to
// output pstart + m - e, so T[pstart + m][dy] = sum_e D[m + e][4 dy + e]; the
// epilogue adds the phases with warp shuffles and takes the 3 rows past a
// warp from the next warp through shared memory.  Tiles advance by
// kConv3Valid = 125 positions (the last 3 rows of a tile lack their e > 0
// partners).
//
// Fused modes: each CTA owns a contiguous range of output tiles (125
// positions) and walks, per image it touches, the row-sum tiles from its
// first output q_a to its last output + 10 P.  kConv3RingT (pitch P < 125)
// keeps the last R >= 10 P + 125 positions of T in a shared-memory ring and
// after tile k completes the outputs q = pstart - 10 P + m, whose 11 row sums
// are then all in the ring.  kConv3RingAcc (P >= 125) keeps one partial sum
// per pending output instead: T[p][dy] is added to acc[p - dy P] (dy = 0
// sets it, dy = 10 completes the output), which no two threads of a tile can
// share because their positions differ by less than P; every output still
// adds its kernel rows in the order dy = 0..10.  kConv3Global writes T to
// global memory and conv3_sum_kernel adds the kernel rows (images too wide
// for the ring).
//
// Persistent CTAs, 6 warps: warp 4 streams the input windows (136 rows per
// channel chunk) through a kC3Stages ring, warp 5 owns TMEM (2 accumulators
// of 64 columns) and issues the MMAs, warps 0..3 (TMEM lane quarters) drain
// an accumulator.
constexpr int kC3Rows = 136;            // window rows per channel chunk (128 + 8)
constexpr int kC3Stages = 2;
constexpr int kC3Threads = 192;

struct Conv3Smem {
    uint64_t wbar;
    uint64_t xfull[kC3Stages], xempty[kC3Stages];
    uint64_t afull[2], aempty[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort_flag;
    alignas(16) float halo[2][4][3][12];   // [tile parity][warp][target lane 29 + i][dy] halo sums
};

__host__ __device__ constexpr uint32_t conv3_wbytes(int cin) { return 3u * (cin / 16) * 2048u; }
__host__ __device__ constexpr uint32_t conv3_stage_bytes(int cin) { return (cin / 8) * kC3Rows * 16u; }
__host__ __device__ constexpr size_t conv3_base_smem(int cin)
{
    return conv3_wbytes(cin) + kC3Stages * (size_t)conv3_stage_bytes(cin) + sizeof(Conv3Smem) + 16;
}
// ring positions of the fused kernel
__host__ __device__ inline int conv3_ring(int P) { return (10 * P + 128 + 31) / 32 * 32; }

enum { kConv3Global = 0, kConv3RingT = 1, kConv3RingAcc = 2 };

// Row sums T[p][dy] read input positions p .. p + 10 only, so a tile whose
// positions all read the input's zero border rows (the 5 rows above the image,
// or the rows below it) has T = 0: the fused modes skip its loads and MMAs and
// take the zeros as its row sums.
__device__ __forceinline__ bool conv3_zero_tile(int pstart, int H, int P)
{
    return pstart + kConv3Valid + 10 <= kPad * P || pstart >= (H + kPad) * P;
}

// Named barrier of the 128 epilogue threads that also returns the OR of `v`
// over them (the same value in every thread).
__device__ __forceinline__ bool epi_bar_or3(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)(v ? 1 : 0))
        : "memory");
    return r != 0;
}

// Calls f(it, b, pstart, qa, qb) for the row-sum tiles of output tiles [lo, hi)
// in order until f returns false.  FUSED: per image, tiles pstart = qa + 125 k
// covering [qa, qb + 10 P); otherwise tiles u of [0, t3) with pstart = 125 u.
template <bool FUSED, typename F>
__device__ __forceinline__ void conv3_walk(int lo, int hi, int tper, int HP, int P, F f)
{
    int it = 0;
    if (FUSED) {
        for (int b = lo / tper; b * tper < hi; ++b) {
            const int ua = lo - b * tper > 0 ? lo - b * tper : 0;
            const int ub = hi - b * tper < tper ? hi - b * tper : tper;
            if (ua >= ub) continue;
            const int qa = ua * kConv3Valid, qb = ub * kConv3Valid < HP ? ub * kConv3Valid : HP;
            const int K = (qb + kConv2Reach * P - qa + kConv3Valid - 1) / kConv3Valid;
            for (int k = 0; k < K; ++k, ++it)
                if (!f(it, b, qa + k * kConv3Valid, qa, qb)) return;
        }
    } else {
        int b = lo / tper, u = lo % tper;
        for (int tile = lo; tile < hi; ++tile, ++it) {
            if (!f(it, b, u * kConv3Valid, 0, 0)) return;
            if (++u == tper) {
                u = 0;
                ++b;
            }
        }
    }
}

// CIN = 32: conv3 (input a2, [B][4][plane][8]).  CIN = 64: the input gradient
// of conv1 (input the gradient plane of z1, [B][8][plane][8], conv1's kernels
// flipped), needed to train the FC layer.  tper = output tiles per image
// (fused modes: cdiv(H P, 125)) or row-sum tiles per image (t3).
template <int CIN, int MODE>
__global__ void __launch_bounds__(kC3Threads) conv3_kernel(const bf16* __restrict__ a2, int B, int H, int W, int P,
                                                           int plane_len, int tper, int tlen,
                                                           const bf16* __restrict__ w3p, float* __restrict__ T,
                                                           const float* __restrict__ b3, int final_relu,
                                                           float* __restrict__ xhat, int R, int* status)
{
    constexpr int NCH = CIN / 8, KK = CIN / 16;
    constexpr bool FUSED = MODE != kConv3Global;
    constexpr uint32_t WB = conv3_wbytes(CIN), SB = conv3_stage_bytes(CIN), CHB = kC3Rows * 16;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* sW = smem_raw;                                    // [x][kk][2][64][8]
    uint8_t* sX = smem_raw + WB;                               // [stage][NCH][kC3Rows][8]
    Conv3Smem* ss = reinterpret_cast<Conv3Smem*>(sX + kC3Stages * SB);
    // kConv3RingT: [11][R] row sums; kConv3RingAcc: [R] partial outputs
    float* ring = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(ss) + sizeof(Conv3Smem));

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int HP = H * P;
    const TileRange tr = tile_range(B * tper, blockIdx.x, gridDim.x);

    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&ss->wbar), 1);
        for (int s = 0; s < kC3Stages; ++s) {
            mbar_init(smem_u32(&ss->xfull[s]), 1);
            mbar_init(smem_u32(&ss->xempty[s]), 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&ss->afull[s]), 1);
            mbar_init(smem_u32(&ss->aempty[s]), 4);
        }
        mbar_init(smem_u32(&ss->drain), 1);
        ss->abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 5) {
        tmem_alloc(smem_u32(&ss->tmem_base), 128);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = ss->tmem_base;
    pdl_wait();
    pdl_trigger();

    if (warp == 4) {
        // ------------------------------------------------ producer
        if (lane == 0) {
            int parity[kC3Stages];
            for (int s = 0; s < kC3Stages; ++s) parity[s] = -1;
            int li = 0;                                         // loaded tiles
            conv3_walk<FUSED>(tr.lo, tr.hi, tper, HP, P, [&](int, int b, int pstart, int, int) {
                if (FUSED && conv3_zero_tile(pstart, H, P)) return true;
                const int it = li++;
                const int st = it % kC3Stages, n = it / kC3Stages;
                if (!mbar_wait(smem_u32(&ss->xempty[st]), (n & 1) ^ 1, status, &ss->abort_flag)) return false;
                mbar_arrive_expect_tx(smem_u32(&ss->xfull[st]), SB);
                parity[st] = n & 1;
                const uint8_t* src = reinterpret_cast<const uint8_t*>(a2) + (size_t)b * NCH * plane_len * 16;
                for (int c = 0; c < NCH; ++c)
                    bulk_g2s(smem_u32(sX + st * SB + c * CHB), src + ((size_t)c * plane_len + pstart) * 16, CHB,
                             smem_u32(&ss->xfull[st]));
                return true;
            });
            for (int s = 0; s < kC3Stages; ++s)
                if (parity[s] >= 0) mbar_wait_drain(smem_u32(&ss->xfull[s]), parity[s]);
        }
    } else if (warp == 5) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            bool ok = true;
            if (tr.lo < tr.hi) {
                mbar_arrive_expect_tx(smem_u32(&ss->wbar), WB);
                bulk_g2s(smem_u32(sW), w3p, WB, smem_u32(&ss->wbar));
                ok = mbar_wait(smem_u32(&ss->wbar), 0, status, &ss->abort_flag);
                if (!ok) mbar_wait_drain(smem_u32(&ss->wbar), 0);
            }
            // N = 48: the 44 columns (dy, e) and 4 of zero weights
            const uint32_t idesc = idesc_bf16(128, 48);
            int li = 0;
            if (ok)
                conv3_walk<FUSED>(tr.lo, tr.hi, tper, HP, P, [&](int, int, int pstart, int, int) {
                    if (FUSED && conv3_zero_tile(pstart, H, P)) return true;
                    const int it = li++;
                    const int s = it & 1, use = it >> 1;
                    const int st = it % kC3Stages, n = it / kC3Stages;
                    if (!mbar_wait(smem_u32(&ss->aempty[s]), (use & 1) ^ 1, status, &ss->abort_flag)) return false;
                    if (!mbar_wait(smem_u32(&ss->xfull[st]), n & 1, status, &ss->abort_flag)) return false;
                    tc_fence_after();
                    const uint32_t d = tbase + (uint32_t)(s * 64);
                    const uint32_t x0 = smem_u32(sX + st * SB);
#pragma unroll
                    for (int x = 0; x < 3; ++x)
#pragma unroll
                        for (int kk = 0; kk < KK; ++kk) {
                            const uint64_t ad = sdesc(x0 + (2 * kk) * CHB + (4 * x) * 16, CHB, 128);
                            const uint64_t bd = sdesc(smem_u32(sW + (x * KK + kk) * 2048), 1024, 128);
                            mma_bf16(d, ad, bd, idesc, (x | kk) ? 1u : 0u);
                        }
                    mma_commit(smem_u32(&ss->xempty[st]));
                    mma_commit(smem_u32(&ss->afull[s]));
                    return true;
                });
            mma_commit(smem_u32(&ss->drain));
            mbar_wait_drain(smem_u32(&ss->drain), 0);
        }
    } else {
        // ------------------------------------------------ epilogue (warps 0..3)
        const int m = warp * 32 + lane;                         // row of this thread
        const bool row_ok = m < kConv3Valid;
        const float bias = (FUSED && b3) ? __ldg(b3) : 0.f;
        const int RP = kConv2Reach * P;
        // fused bookkeeping: ring slot of pstart, and (row, column) of output q = pstart - 10 P + m
        int base = 0, orow = 0, ocol = 0, cur_b = -1, cur_qa = -1;
        const int step_r = kConv3Valid / P, step_c = kConv3Valid % P;
        int li = 0;                                             // tiles with MMAs
        conv3_walk<FUSED>(tr.lo, tr.hi, tper, HP, P, [&](int, int b, int pstart, int qa, int qb) {
            float tv[11];
            if (FUSED && conv3_zero_tile(pstart, H, P)) {
#pragma unroll
                for (int dy = 0; dy < 11; ++dy) tv[dy] = 0.f;
                // the barrier every tile passes before its ring updates: it orders them
                // after the previous tile's (another warp may hold the same ring slot)
                epi_bar();
            } else {
            const int it = li++;
            const int s = it & 1, use = it >> 1;
            bool ok = mbar_wait(smem_u32(&ss->afull[s]), use & 1, status, &ss->abort_flag);
            ok = __all_sync(0xffffffffu, ok);
            float v[48];                                        // v[4 dy + e] = D[m][4 dy + e]
            if (ok) {
                tc_fence_after();
                const uint32_t ta = tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(s * 64);
                tmem_ld48(ta, v);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&ss->aempty[s]));
                // the previous warp's lane 29 + i needs, for each dy, the terms
                // D[j][4 dy + j + 3 - i] of this warp's rows j = max(0, i - 2) .. i:
                // lane i sums them (own e = 3 term, lane i - 1's e = 2, lane i - 2's e = 1)
                float hs[12];
#pragma unroll
                for (int dy = 0; dy < 11; ++dy) {
                    const float e2 = __shfl_up_sync(0xffffffffu, v[4 * dy + 2], 1);
                    const float e1 = __shfl_up_sync(0xffffffffu, v[4 * dy + 1], 2);
                    hs[dy] = v[4 * dy + 3] + (lane >= 1 ? e2 : 0.f) + (lane >= 2 ? e1 : 0.f);
                }
                hs[11] = 0.f;
                if (lane < 3) {
                    float4* hd = reinterpret_cast<float4*>(ss->halo[s][warp][lane]);
#pragma unroll
                    for (int q4 = 0; q4 < 3; ++q4)
                        hd[q4] = make_float4(hs[4 * q4], hs[4 * q4 + 1], hs[4 * q4 + 2], hs[4 * q4 + 3]);
                }
            }
            // also the per-tile barrier that orders this tile's ring updates after the
            // previous tile's
            if (epi_bar_or3(!ok)) return false;
            // rows past this warp come from the next warp's halo sums (never needed by
            // warp 3's valid rows; the index is clamped so that the read stays in bounds)
            float hv[12];
            if (lane >= 29) {
                const float4* hsrc = reinterpret_cast<const float4*>(ss->halo[s][warp < 3 ? warp + 1 : 3][lane - 29]);
#pragma unroll
                for (int q4 = 0; q4 < 3; ++q4) {
                    const float4 h4 = hsrc[q4];
                    hv[4 * q4] = h4.x;
                    hv[4 * q4 + 1] = h4.y;
                    hv[4 * q4 + 2] = h4.z;
                    hv[4 * q4 + 3] = h4.w;
                }
            } else {
#pragma unroll
                for (int i = 0; i < 12; ++i) hv[i] = 0.f;
            }
#pragma unroll
            for (int dy = 0; dy < 11; ++dy) {
                float t = v[4 * dy];
#pragma unroll
                for (int e = 1; e < 4; ++e) {
                    const float nb = __shfl_down_sync(0xffffffffu, v[4 * dy + e], e);
                    if (lane + e < 32) t += nb;
                }
                tv[dy] = t + hv[dy];
            }
            }
            if (!FUSED) {
                if (row_ok) {
                    float* dst = T + (size_t)b * 11 * tlen + pstart + m;
#pragma unroll
                    for (int dy = 0; dy < 11; ++dy) dst[(size_t)dy * tlen] = tv[dy];
                }
                return true;
            }
            if (b != cur_b || qa != cur_qa) {
                // new segment: ring slot of pstart = qa is 0; output q = qa - 10 P + m
                cur_b = b;
                cur_qa = qa;
                base = 0;
                const int q = qa - RP + m;
                orow = q >= 0 ? q / P : -((-q + P - 1) / P);
                ocol = q - orow * P;
            } else {
                base += kConv3Valid;
                if (base >= R) base -= R;
                orow += step_r;
                ocol += step_c;
                if (ocol >= P) {
                    ocol -= P;
                    ++orow;
                }
            }
            if (MODE == kConv3RingAcc) {
                // contribution dy of position p goes to output p - dy P (slot r), in the order dy = 0..10
                const int p = pstart + m;
                int r = base + m;
                if (r >= R) r -= R;
#pragma unroll
                for (int dy = 0; dy < 11; ++dy) {
                    const int q = p - dy * P;
                    if (row_ok && q >= qa && q < qb) {
                        if (dy == 0) {
                            ring[r] = tv[0];
                        } else if (dy < 10) {
                            ring[r] += tv[dy];
                        } else if (ocol < W) {
                            const float x = ring[r] + tv[10] + bias;
                            xhat[((size_t)b * H + orow) * W + ocol] = final_relu ? fmaxf(x, 0.f) : x;
                        }
                    }
                    r -= P;
                    if (r < 0) r += R;
                }
                return true;
            }
            if (row_ok) {
                int w = base + m;
                if (w >= R) w -= R;
#pragma unroll
                for (int dy = 0; dy < 11; ++dy) ring[dy * R + w] = tv[dy];
            }
            epi_bar();
            const int q = pstart - RP + m;
            if (row_ok && q >= qa && q < qb && ocol < W) {
                int r = base + m - RP;
                if (r < 0) r += R;
                float x = bias;
#pragma unroll
                for (int dy = 0; dy < 11; ++dy) {
                    x += ring[dy * R + r];
                    r += P;
                    if (r >= R) r -= R;
                }
                xhat[((size_t)b * H + orow) * W + ocol] = final_relu ? fmaxf(x, 0.f) : x;
            }
            return true;
        });
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 5) {
        tc_fence_after();
        tmem_dealloc(tbase, 128);
    }
}

__global__ void conv3_sum_kernel(const float* __restrict__ T, int B, int H, int W, int P, int tlen,
                                 const float* __restrict__ b3, int final_relu, float* __restrict__ xhat)
{
    const long long n = (long long)B * H * W;
    const float bias = b3 ? __ldg(b3) : 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % W);
        const int r = (int)((i / W) % H);
        const long long b = i / ((long long)W * H);
        const float* t = T + (size_t)b * 11 * tlen + (size_t)r * P + c;
        float s = bias;
#pragma unroll
        for (int dy = 0; dy < 11; ++dy) s += t[(size_t)dy * tlen + (size_t)dy * P];
        xhat[i] = final_relu ? fmaxf(s, 0.f) : s;
    }
}

// y[m][n] = sum_z part[z][m][n] (fixed order) for the split-K GEMM.
__global__ void splitk_reduce_kernel(const float* __restrict__ part, int ksplit, long long n, float* __restrict__ y)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < ksplit; ++z) s += part[(size_t)z * n + i];
        y[i] = s;
    }
}

inline int grid1d(long long n, int threads = 256)
{
    long long b = (n + threads - 1) / threads;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

// ================================================================ launchers
size_t packed_elems(int R, int TR, int Kp) { return (size_t)cdiv(R, TR) * TR * Kp; }

int pack_kmajor(const float* src, long long rs, long long cs, int R, int K, int TR, int Kp, bf16* dst,
                cudaStream_t st)
{
    const long long nchunks = (long long)cdiv(R, TR) * TR * (Kp / 8);
    if (nchunks <= 0) return DEEPINV_OK;
    DI_CUDA(launch_pdl(pack_kmajor_kernel, dim3(grid1d(nchunks)), dim3(256), 0, st, src, rs, cs, R, K, TR, Kp,
                       nchunks, dst));
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

int pack_hidden_weights(const float* w, bf16* whp, bf16* wht, cudaStream_t st)
{
    const long long n = (long long)kWhPackElems * (wht ? 2 : 1);
    pack_hidden_weights_kernel<<<grid1d(n), 256, 0, st>>>(w, whp, wht);
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

int pack_conv_weights(const float* w1, const float* w2, const float* w3, bf16* w1p, bf16* w2p, bf16* w3p,
                      cudaStream_t st)
{
    const long long n = (long long)(kW1PackElems + kW2PackElems + kW3PackElems);
    pack_conv_weights_kernel<<<grid1d(n), 256, 0, st>>>(w1, w2, w3, w1p, w2p, w3p);
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

int tc_gemm_splitk(const bf16* A, const bf16* B, int Kp, int Mr, int Nc, int NB, float* out, float* part, int ksplit,
                   int* status, cudaStream_t st)
{
    if (Mr <= 0 || Nc <= 0) return DEEPINV_OK;
    if (ksplit <= 1 || !part) return tc_gemm(A, B, Kp, Mr, Nc, NB, GEMM_OUT_F32, out, Nc, nullptr, Geo{}, status, st);
    if (NB < 16 || NB > 256 || NB % 16 || Kp % 16 || Kp <= 0) {
        set_error("tc_gemm_splitk: bad tile N=%d or K=%d", NB, Kp);
        return DEEPINV_EINVAL;
    }
    // two row tiles per CTA when B is too large to stay in L2 (it is then read once)
    const int mt = (Mr > 128 && (size_t)Nc * Kp * 2 > ((size_t)64 << 20)) ? 2 : 1;
    if (mt == 2) {
        // about one wave of CTAs over the halved tile count (the partials buffer holds 16 slices)
        int nsm = 152, dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaGetLastError();
        const int tiles = cdiv(Mr, 256) * cdiv(Nc, NB), kmax = Kp / 16 / 16;
        ksplit = nsm / (tiles > 0 ? tiles : 1);
        if (ksplit > kmax) ksplit = kmax;
        if (ksplit > 16) ksplit = 16;
        if (ksplit < 1) ksplit = 1;
    }
    uint32_t cols = 32;
    while (cols < (uint32_t)(mt * NB)) cols <<= 1;
    const size_t smem = (size_t)kGemmNS * (mt * kGemmKS * 4096 + (size_t)kGemmKS * NB * 32) + sizeof(GemmSmem);
    dim3 grid(cdiv(Mr, 128 * mt), cdiv(Nc, NB), ksplit);
    if (mt == 2) {
        DI_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<GEMM_OUT_F32, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        tc_gemm_kernel<GEMM_OUT_F32, 2><<<grid, 192, smem, st>>>(A, B, Kp, Mr, Nc, NB, cols, part, Nc, nullptr, 0, 0,
                                                                 0, 0, status);
    } else {
        DI_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<GEMM_OUT_F32, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        tc_gemm_kernel<GEMM_OUT_F32, 1><<<grid, 192, smem, st>>>(A, B, Kp, Mr, Nc, NB, cols, part, Nc, nullptr, 0, 0,
                                                                 0, 0, status);
    }
    DI_LAUNCH_CHECK();
    const long long n = (long long)Mr * Nc;
    splitk_reduce_kernel<<<grid1d(n), 256, 0, st>>>(part, ksplit, n, out);
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

int tc_gemm(const bf16* A, const bf16* B, int Kp, int Mr, int Nc, int NB, int mode, float* out_f32,
            long long ldo, bf16* plane, const Geo& geo, int* status, cudaStream_t st)
{
    if (Mr <= 0 || Nc <= 0) return DEEPINV_OK;
    if (NB < 16 || NB > 256 || NB % 16 || Kp % 16 || Kp <= 0) {
        set_error("tc_gemm: bad tile N=%d or K=%d", NB, Kp);
        return DEEPINV_EINVAL;
    }
    // two row tiles per CTA (B read half as often) when there are at least two per SM
    int nsm = 152;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaGetLastError();
    }
    const int mt = cdiv(Mr, 128) >= 2 * nsm * cdiv(Nc, NB) ? 2 : 1;
    uint32_t cols = 32;
    while (cols < (uint32_t)(mt * NB)) cols <<= 1;
    const size_t smem = (size_t)kGemmNS * (mt * kGemmKS * 4096 + (size_t)kGemmKS * NB * 32) + sizeof(GemmSmem);
    dim3 grid(cdiv(Mr, 128 * mt), cdiv(Nc, NB));
#define DI_GEMM_LAUNCH(MODE_, MT_)                                                                                     \
    do {                                                                                                               \
        DI_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<MODE_, MT_>, cudaFuncAttributeMaxDynamicSharedMemorySize,           \
                                     (int)smem));                                                                      \
        DI_CUDA(launch_pdl(tc_gemm_kernel<MODE_, MT_>, grid, dim3(192), smem, st, A, B, Kp, Mr, Nc, NB, cols, out_f32, \
                           ldo, plane, geo.H, geo.W, geo.P, geo.plane, status));                                       \
    } while (0)
    if (mode == GEMM_OUT_F32) {
        if (mt == 2) DI_GEMM_LAUNCH(GEMM_OUT_F32, 2);
        else DI_GEMM_LAUNCH(GEMM_OUT_F32, 1);
    } else {
        if (mt == 2) DI_GEMM_LAUNCH(GEMM_OUT_PLANE, 2);
        else DI_GEMM_LAUNCH(GEMM_OUT_PLANE, 1);
    }
#undef DI_GEMM_LAUNCH
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

int conv1_tc(const bf16* xt, int B, const Geo& g, const bf16* w1p, const float* b1, void* a1, int mode,
             const float* inv_sa, float* amax, int* status, cudaStream_t st)
{
    if (B <= 0) return DEEPINV_OK;
    const int ering = conv1_ering(g.P, g.t1);
    const size_t smem = conv1_wbytes(64) + conv1_xbytes(ering) + sizeof(Conv1Smem) + 16;
    int dev = 0, sms = 0;
    DI_CUDA(cudaGetDevice(&dev));
    DI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int ntiles = B * g.t1;
    const int grid = ntiles < 2 * sms ? ntiles : 2 * sms;
    DI_CUDA(cudaFuncSetAttribute(conv1_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    DI_CUDA(launch_pdl(conv1_kernel<64>, dim3(grid), dim3(kC1Threads), smem, st, xt, B, g.H, g.W, g.P, g.plane, g.t1,
                       w1p, b1, a1, mode, inv_sa, amax, (const bf16*)nullptr, ering, status));
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

int conv1_rows_fit(const Geo& g)
{
    Conv1RGeo r;
    if (!conv1_rows_geo(g, r)) return 0;
    // measured (GB300, bf16): one row of >= 120 columns per tile is faster than the
    // consecutive-position tiles (256 x 256: 0.51-0.53 against 0.56-0.57 ms at batch
    // 256; 128 x 128: 0.288 against 0.296 ms at batch 512); several rows per tile
    // (64 x 64: 0.196 against 0.157 ms) or partly filled tiles (100 x 100: 0.22
    // against 0.19 ms) are slower
    return r.R == 1 && r.Sw >= 120 ? 2 : 1;
}

int conv1_rows_tc(const bf16* xt, int B, const Geo& g, const bf16* w1p, const float* b1, void* a1, int mode,
                  const float* inv_sa, int* status, cudaStream_t st)
{
    if (B <= 0) return DEEPINV_OK;
    DI_REQUIRE(mode == kConv1OutBF16 || mode == kConv1OutE4M3, "conv1 row tiles: bf16 or e4m3 output only");
    Conv1RGeo r;
    DI_REQUIRE(conv1_rows_geo(g, r), "conv1 row tiles: fewer than 96 positions per tile");
    const long long ntiles = (long long)B * r.nseg * r.nrb;
    DI_REQUIRE(ntiles < INT_MAX, "conv1 row tiles: too many tiles");
    const size_t smem = conv1_wbytes(64) + kC1RRowBytes + sizeof(Conv1RSmem) + 16;
    int dev = 0, sms = 0;
    DI_CUDA(cudaGetDevice(&dev));
    DI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = (int)std::min<long long>(ntiles, 2LL * sms);
    DI_CUDA(cudaFuncSetAttribute(conv1_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    DI_CUDA(launch_pdl(conv1_rows_kernel, dim3(grid), dim3(kC1RThreads), smem, st, xt, B, g.H, g.W, g.P, g.plane, r,
                       w1p, b1, a1, mode, inv_sa, status));
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

int conv3_dgrad_tc(const bf16* g3p, int B, const Geo& g, const bf16* w3t, const bf16* a2, bf16* g2, int* status,
                   cudaStream_t st)
{
    if (B <= 0) return DEEPINV_OK;
    const int ering = conv1_ering(g.P, g.t1);
    const size_t smem = conv1_wbytes(32) + conv1_xbytes(ering) + sizeof(Conv1Smem) + 16;
    int dev = 0, sms = 0;
    DI_CUDA(cudaGetDevice(&dev));
    DI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int ntiles = B * g.t1;
    const int grid = ntiles < 2 * sms ? ntiles : 2 * sms;
    DI_CUDA(cudaFuncSetAttribute(conv1_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    DI_CUDA(launch_pdl(conv1_kernel<32>, dim3(grid), dim3(kC1Threads), smem, st, g3p, B, g.H, g.W, g.P, g.plane,
                       g.t1, w3t, (const float*)nullptr, (void*)g2, (int)kConv1GradMask, (const float*)nullptr,
                       (float*)nullptr, a2, ering, status));
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

int pack_w2_e4m3(const float* w2, float* amax_scratch, uint8_t* w2q, float* sw, cudaStream_t st)
{
    conv2_absmax_kernel<<<32, 256, 0, st>>>(w2, amax_scratch);
    DI_LAUNCH_CHECK();
    pack_w2_e4m3_kernel<<<grid1d(kW2E4M3Bytes), 256, 0, st>>>(w2, amax_scratch, w2q, sw);
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

int e4m3_scales(const float* amax_a1, const float* sw, float* inv_sa, float* oscale, cudaStream_t st)
{
    e4m3_scales_kernel<<<1, 32, 0, st>>>(amax_a1, sw, inv_sa, oscale);
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

// narrow: 4 input chunks per position (e4m3 input, or a 32-channel bf16 input)
// and 8 KB weight blocks; otherwise 8 chunks and 16 KB blocks.
// Row mode: ring stages of one kernel row's input piece and weights; as many
// as fit next to the slot exchange (at most kMaxRowSlots).
static size_t conv2_fixed_bytes() { return kXBytes + sizeof(Conv2Smem); }
static int conv2_row_slots(bool narrow, int groups)
{
    const size_t stage = (size_t)(narrow ? 4 : 8) * kPiecePx * 16 + (size_t)groups * (narrow ? 8192 : 16384);
    const size_t n = (227 * 1024 - conv2_fixed_bytes()) / stage;
    return (int)(n > kMaxRowSlots ? kMaxRowSlots : n);
}
static size_t conv2_smem_bytes(const Geo& g, bool rows, bool narrow, int groups = 3)
{
    const int nch = narrow ? 4 : 8;
    const size_t wstage = narrow ? 8192 : 16384;
    if (rows) {
        const int slots = conv2_row_slots(narrow, groups);
        return (size_t)slots * (nch * kPiecePx * 16 + groups * wstage) + conv2_fixed_bytes();
    }
    const size_t win = (size_t)nch * g.nslab * kSlabPx * 16;
    return win + (size_t)kW2Stages * wstage + kXBytes + sizeof(Conv2Smem);
}

// Row mode by default (64 x 64, batch 1024: 1.20 ms against 1.42 ms in window
// mode; wider images fit only row mode).  DEEPINV_CONV2_WINDOW=1 in
// the environment selects window mode where the window fits in shared memory
// (both modes give bit-identical results; the tests compare them).
static bool conv2_window_mode(const Geo& g, bool narrow)
{
    static const bool window = [] {
        const char* e = getenv("DEEPINV_CONV2_WINDOW");
        return e && e[0] == '1';
    }();
    return window && g.nslab <= kMaxSlabs && conv2_smem_bytes(g, false, narrow) <= 227 * 1024;
}

bool conv2_tc_supported(const Geo& g)
{
    return conv2_window_mode(g, false) || conv2_smem_bytes(g, true, false) <= 227 * 1024;
}

template <bool ROWS, int V>
static int launch_conv2_mode(const void* in, int B, const Geo& g, const void* wp, const float* bias,
                             const float* oscale, const bf16* mask_src, bf16* out, int grid, size_t smem, int nslab,
                             int* status, cudaStream_t st)
{
    DI_CUDA(cudaFuncSetAttribute(conv2_kernel<ROWS, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    DI_CUDA(launch_pdl(conv2_kernel<ROWS, V>, dim3(grid), dim3(kConv2Threads), smem, st, in, B, g.H, g.W, g.P,
                       g.plane, g.t2, nslab, wp, bias, oscale, mask_src, out, status));
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

// One persistent CTA per SM (at most one per tile), row or window mode.
template <int V>
static int launch_conv2(const void* in, int B, const Geo& g, const void* wp, const float* bias, const float* oscale,
                        const bf16* mask_src, bf16* out, int num_sms, int* status, cudaStream_t st)
{
    if (B <= 0) return DEEPINV_OK;
    if (!conv2_tc_supported(g)) {
        set_error("conv2_tc: no kernel configuration for image width %d", g.W);
        return DEEPINV_EUNSUPPORTED;
    }
    constexpr bool narrow = V != kC2Fwd;
    const bool rows = !conv2_window_mode(g, narrow);
    constexpr int groups = V == kC2Dgrad ? 6 : 3;
    const size_t smem = conv2_smem_bytes(g, rows, narrow, groups);
    const int ntiles = B * g.t2;
    const int grid = ntiles < num_sms ? ntiles : num_sms;
    const int nslab = rows ? conv2_row_slots(narrow, groups) : g.nslab;
    if (rows)
        return launch_conv2_mode<true, V>(in, B, g, wp, bias, oscale, mask_src, out, grid, smem, nslab, status, st);
    return launch_conv2_mode<false, V>(in, B, g, wp, bias, oscale, mask_src, out, grid, smem, nslab, status, st);
}

int conv2_tc(const void* a1, int B, const Geo& g, const void* w2p, const float* b2, const float* oscale,
             bool fp8, bf16* a2, int num_sms, int* status, cudaStream_t st)
{
    return fp8 ? launch_conv2<kC2FwdE4M3>(a1, B, g, w2p, b2, oscale, nullptr, a2, num_sms, status, st)
               : launch_conv2<kC2Fwd>(a1, B, g, w2p, b2, nullptr, nullptr, a2, num_sms, status, st);
}

int conv2_dgrad_tc(const bf16* g2, int B, const Geo& g, const bf16* w2t, const bf16* a1, bf16* g1, int num_sms,
                   int* status, cudaStream_t st)
{
    return launch_conv2<kC2Dgrad>(g2, B, g, w2t, nullptr, nullptr, a1, g1, num_sms, status, st);
}

int hidden_tc(const bf16* in, int B, const Geo& g, const bf16* whp, const float* bias, bf16* out, int num_sms,
              int* status, cudaStream_t st)
{
    return launch_conv2<kHidFwd>(in, B, g, whp, bias, nullptr, nullptr, out, num_sms, status, st);
}

int hidden_dgrad_tc(const bf16* gout, int B, const Geo& g, const bf16* wht, const bf16* act_in, bf16* gin,
                    int num_sms, int* status, cudaStream_t st)
{
    return launch_conv2<kHidDgrad>(gout, B, g, wht, nullptr, nullptr, act_in, gin, num_sms, status, st);
}


// Failure-path check: one thread waits, with the bounded wait every pipeline
// uses, for an mbarrier phase that nothing completes.  After the wait's time
// limit it records DEV_TIMEOUT in the status word and the kernel returns; no
// copy, MMA or TMEM is involved, so nothing is left in flight.
__global__ void bounded_wait_probe_kernel(int* status)
{
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait(smem_u32(&bar), 0, status, &abort_flag);
}

int bounded_wait_probe(int* status, cudaStream_t st)
{
    bounded_wait_probe_kernel<<<1, 32, 0, st>>>(status);
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

size_t conv3_chunk(const Geo& g, int B)
{
    // images per unfused conv3 pass: the row sums T of one pass stay within ~48 MB of L2
    const size_t per = (size_t)11 * g.tlen * sizeof(float);
    size_t c = ((size_t)48 << 20) / per;
    if (c < 1) c = 1;
    return c < (size_t)B ? c : (size_t)B;
}

static int conv3_mode(const Geo& g) { return g.P < kConv3Valid ? kConv3RingT : kConv3RingAcc; }

static size_t conv3_fused_smem(const Geo& g, int cin)
{
    const size_t per = conv3_mode(g) == kConv3RingT ? 11 : 1;
    return conv3_base_smem(cin) + per * conv3_ring(g.P) * sizeof(float);
}

bool conv3_fused(const Geo& g, int cin) { return conv3_fused_smem(g, cin) <= 227 * 1024; }

size_t conv3_scratch_elems(const Geo& g, int B, int cin)
{
    return (B > 0 && !conv3_fused(g, cin)) ? conv3_chunk(g, B) * 11 * g.tlen : 0;
}

// One pass over B images of `in` ([B][CIN / 8][plane][8]): fused (xhat written)
// or, for images too wide for the ring, row sums into T.
template <int CIN>
static int launch_conv3(const bf16* in, int B, const Geo& g, const bf16* w, float* T, const float* b3,
                        int final_relu, float* xhat, bool fused, int* status, cudaStream_t st)
{
    int dev = 0, sms = 0;
    DI_CUDA(cudaGetDevice(&dev));
    DI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = fused ? conv3_fused_smem(g, CIN) : conv3_base_smem(CIN);
    const int tper = fused ? cdiv(g.HP, kConv3Valid) : g.t3;
    int occ = (int)((228 * 1024) / (smem + 1024));
    const int occ_max = CIN == 32 ? 3 : 2;
    if (occ > occ_max) occ = occ_max;
    if (occ < 1) occ = 1;
    const long long ntiles = (long long)B * tper;
    const int grid = ntiles < (long long)occ * sms ? (int)ntiles : occ * sms;
    const int R = conv3_ring(g.P);
    const int mode = fused ? conv3_mode(g) : kConv3Global;
    auto go = [&](auto kern) -> int {
        DI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        DI_CUDA(launch_pdl(kern, dim3(grid), dim3(kC3Threads), smem, st, in, B, g.H, g.W, g.P, g.plane, tper, g.tlen,
                           w, T, b3, final_relu, xhat, R, status));
        return DEEPINV_OK;
    };
    if (mode == kConv3RingT) DI_TRY(go(conv3_kernel<CIN, kConv3RingT>));
    else if (mode == kConv3RingAcc) DI_TRY(go(conv3_kernel<CIN, kConv3RingAcc>));
    else DI_TRY(go(conv3_kernel<CIN, kConv3Global>));
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

template <int CIN>
static int conv3_all(const bf16* in, int B, const Geo& g, const bf16* w, const float* b3, float* T, float* out,
                     int final_relu, int* status, cudaStream_t st)
{
    if (B <= 0) return DEEPINV_OK;
    if (conv3_fused(g, CIN)) return launch_conv3<CIN>(in, B, g, w, nullptr, b3, final_relu, out, true, status, st);
    const int chunk = (int)conv3_chunk(g, B);
    for (int b0 = 0; b0 < B; b0 += chunk) {
        const int nb = B - b0 < chunk ? B - b0 : chunk;
        DI_TRY(launch_conv3<CIN>(in + (size_t)b0 * (CIN / 8) * g.plane * 8, nb, g, w, T, nullptr, 0, nullptr, false,
                                 status, st));
        const long long n = (long long)nb * g.H * g.W;
        conv3_sum_kernel<<<grid1d(n), 256, 0, st>>>(T, nb, g.H, g.W, g.P, g.tlen, b3, final_relu,
                                                    out + (size_t)b0 * g.H * g.W);
        DI_LAUNCH_CHECK();
    }
    return DEEPINV_OK;
}

int conv3_tc(const bf16* a2, int B, const Geo& g, const bf16* w3p, const float* b3, float* T, float* xhat,
             int final_relu, int* status, cudaStream_t st)
{
    return conv3_all<32>(a2, B, g, w3p, b3, T, xhat, final_relu, status, st);
}

int conv1_dgrad_tc(const bf16* g1, int B, const Geo& g, const bf16* w1t, float* T, float* dxt, int* status,
                   cudaStream_t st)
{
    return conv3_all<64>(g1, B, g, w1t, nullptr, T, dxt, 0, status, st);
}

}  // namespace di
