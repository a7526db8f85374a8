// Backward pass of the bfloat16 path (the MSE objective of Sec. 4 by
// backpropagation), on the padded planes of the forward pass.
//
// In plane coordinates the forward convolution reads input position
// q + dy P + dx for output q (data at plane index q + 5 P + 5).  Hence
//   input gradient:  dA[q] = sum_{dy',dx'} W[10-dy'][10-dx']^T G[q + dy' P + dx']
//                    -- the same correlation with flipped, transposed kernels,
//                       run by the forward kernels (conv1<32>, conv2 DGRAD);
//   weight gradient: dW[dy][dx] = sum_u G[u] A[u + (dy-5) P + (dx-5)]^T over
//                    plane positions u (G is zero off the data positions).
#include <algorithm>

#include "kernels.cuh"
#include "tc.cuh"

namespace di {
namespace {

using namespace tc;

inline int grid_for(long long n, int threads = 256)
{
    long long b = (n + threads - 1) / threads;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    return (int)b;
}

// conv2 input-gradient weights: block (dy', s) holds rows m = 64 g + ci
// (g = tap slot, dx' = 2 s + g), K = the 32 output channels in two chunks of
// 16, value W2[co][ci][10 - dy'][10 - dx'] (zero for dx' = 11).
// conv3 input-gradient weights (conv1<32> layout): block (dy', h) holds rows
// n = ci, K = columns dx' = 8 h .. 8 h + 7 (zero for dx' >= 11), value
// W3[0][ci][10 - dy'][10 - dx'].
// conv1 input-gradient weights (conv3<64> layout): block (x, kk) holds rows
// n = 4 dy' + e, K = filters 16 kk .. 16 kk + 15, value
// W1[co][0][10 - dy'][10 - dx'] with dx' = 4 x + e (zero for dy' >= 11 or
// dx' >= 11).
__global__ void pack_dgrad_weights_kernel(const float* __restrict__ w1, const float* __restrict__ w2,
                                          const float* __restrict__ w3, bf16* __restrict__ w1t,
                                          bf16* __restrict__ w2t, bf16* __restrict__ w3t)
{
    const long long n2 = kW2PackElems, n3 = kW3tPackElems, n1 = kW1tPackElems;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2 + n3 + n1;
         i += (long long)gridDim.x * blockDim.x) {
        if (i >= n2 + n3) {
            const long long j = i - n2 - n3;
            const int e8 = (int)(j % 8), n = (int)((j / 8) % 64), half = (int)((j / 512) % 2);
            const int kk = (int)((j / 1024) % 4), x = (int)(j / 4096);
            const int co = kk * 16 + half * 8 + e8, dy = n / 4, dx = 4 * x + n % 4;
            const float v = (dy < 11 && dx < 11) ? w1[(co * 11 + (10 - dy)) * 11 + (10 - dx)] : 0.f;
            w1t[j] = __float2bfloat16_rn(v);
        } else if (i < n2) {
            const int e = (int)(i % 8);
            const int m = (int)((i / 8) % 128);
            const int half = (int)((i / (8 * 128)) % 2);
            const int kk = (int)((i / (8 * 128 * 2)) % 2);
            const int s = (int)((i / (8 * 128 * 2 * 2)) % 6);
            const int dy = (int)(i / (8 * 128 * 2 * 2 * 6));
            const int ci = m % 64, g = m / 64, dx = 2 * s + g, co = kk * 16 + half * 8 + e;
            const float v = dx < 11 ? w2[((co * 64 + ci) * 11 + (10 - dy)) * 11 + (10 - dx)] : 0.f;
            w2t[i] = __float2bfloat16_rn(v);
        } else {
            const long long j = i - n2;
            const int e = (int)(j % 8), ci = (int)((j / 8) % 32), blk = (int)(j / (8 * 32));
            const int dy = blk / 2, dx = (blk % 2) * 8 + e;
            const float v = dx < 11 ? w3[(ci * 11 + (10 - dy)) * 11 + (10 - dx)] : 0.f;
            w3t[j] = __float2bfloat16_rn(v);
        }
    }
}

// Gradient plane of x^: gp[b][q + 5 P + 5] = g[b][r n2 + c], q = r P + c (other entries untouched).
// Images over grid.y (striding past 65535), pixels over grid.x: 32-bit index
// arithmetic within an image.
__global__ void grad_plane_kernel(const float* __restrict__ g, int B, int H, int W, int P, int plane_len,
                                  bf16* __restrict__ gp)
{
    const int N = H * W;
    for (int b = blockIdx.y; b < B; b += gridDim.y) {
        const float* gi = g + (size_t)b * N;
        bf16* pi = gp + (size_t)b * plane_len + kPad * P + kPad;
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
            const int r = j / W, c = j - r * W;
            pi[r * P + c] = __float2bfloat16_rn(gi[j]);
        }
    }
}

// Channel sums of a chunked bf16 plane [B][C/8][plane][8] (C % 8 == 0) or of a
// one-channel plane (C == 1), per image and segment of the plane:
// part[b nseg + seg][c] in float64.  One block per (image, 8-channel chunk,
// segment); each thread loads 16 bytes at a time (8 channels of a position, or
// 8 positions of the one-channel plane), four loads in flight before they are
// added (the same order of additions as one at a time); float32 per thread and
// across a warp, float64 across warps and blocks.
__global__ void plane_sum_kernel(const bf16* __restrict__ src, int C, int plane_len, int nseg,
                                 double* __restrict__ part)
{
    const int b = blockIdx.x, ch = blockIdx.y, seg = blockIdx.z;
    const int nch = C == 1 ? 1 : C / 8;
    // 16-byte units of this (image, chunk) plane and this block's segment of them
    const int units = C == 1 ? plane_len / 8 : plane_len;
    const int u_lo = (int)((long long)units * seg / nseg), u_hi = (int)((long long)units * (seg + 1) / nseg);
    const uint4* s4 = reinterpret_cast<const uint4*>(src + ((size_t)b * nch + ch) * plane_len * (C == 1 ? 1 : 8));
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int bd = blockDim.x;
    for (int p = u_lo + threadIdx.x; p < u_hi; p += 4 * bd) {
        uint4 u[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) u[k] = p + k * bd < u_hi ? s4[p + k * bd] : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (p + k * bd >= u_hi) break;
            const bf16* v = reinterpret_cast<const bf16*>(&u[k]);
#pragma unroll
            for (int e = 0; e < 8; ++e) acc[e] += __bfloat162float(v[e]);
        }
    }
    // a fixed butterfly over the warp in float32 (float64 arithmetic is slow on this
    // GPU), then the warps' sums in float64
    const int nc = C == 1 ? 1 : 8;
    if (C == 1) {
#pragma unroll
        for (int e = 1; e < 8; ++e) acc[0] += acc[e];
    }
    __shared__ double red[8][8];
    const int w = threadIdx.x / 32;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        if (e >= nc) break;
        float t = acc[e];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if ((threadIdx.x & 31) == 0) red[w][e] = (double)t;
    }
    __syncthreads();
    if (threadIdx.x < (C == 1 ? 1 : 8)) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x / 32); ++k) t += red[k][threadIdx.x];
        part[((size_t)b * nseg + seg) * C + (C == 1 ? 0 : ch * 8 + threadIdx.x)] = t;
    }
}

// out[c] = sum_b part[b][c] in a fixed order: one warp per channel, lane l adds
// b = l, l + 32, ... in turn, then a fixed butterfly over the lanes.
__global__ void sum_parts_kernel(const double* __restrict__ part, int B, int C, float* __restrict__ out)
{
    const int c = blockIdx.x, lane = threadIdx.x;
    double s = 0.0;
    for (int b = lane; b < B; b += 32) s += part[(size_t)b * C + c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[c] = (float)s;
}


// ---------------------------------------------------------------- cp.async (16 bytes, L2 only)
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

// Arrive on `bar` once all of this thread's earlier cp.async copies have
// completed (the barrier's expected count includes this arrival).
__device__ __forceinline__ void cp_async_arrive(uint32_t bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Instruction descriptor of tcgen05.mma.kind::f16 with both operands MN-major
// (bits 15 and 16), bf16 in, float32 out.
__device__ __forceinline__ uint32_t idesc_bf16_mn(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// ---------------------------------------------------------------- conv1 / conv3 weight gradients
// D[t][j] = sum_u S[u + sgn off(t)] C[u][j], off(t) = (dy - 5) P + (dx - 5) for
// tap t = 11 dy + dx, over the data positions u of every image:
//   conv1: S = x~ plane, sgn = +1, C = g1 plane (64 ch):  dW1[j][0][t] = D[t][j]
//   conv3: S = x^ gradient plane, sgn = -1, C = a2 plane (32 ch): dW3[0][j][t] = D[t][j]
// MMAs with M = 128 taps (rows >= 121 zero; with sgn = +1 row 127 is all ones,
// giving sum_u C[u][j], conv1's bias gradient), N = CJ channels, K = 16
// positions.  A is an im2col of S built in shared memory (K-major); B is the C
// plane itself (MN-major, bulk-copied).  Each CTA covers a run of 128-position
// blocks, keeps its sum in TMEM and leaves a float32 partial.
//
// Warps 0..3: thread t builds im2col row t of each block from aligned 16-byte
// reads of the block's window of S, shifted into place (the shift is the same
// for every chunk of the row), into one of two A buffers.  Warp 4 runs the
// block pipeline: its lanes issue the bulk copies of a block's window and C
// planes (one copy per lane) into one of two load stages as soon as the MMAs of
// the block that last used the stage are done, and its lane 0 issues each
// block's MMAs once the im2col warps have built its A.  With two stages (nst;
// images too wide for two windows in shared memory take one) block n's MMAs
// overlap block n + 1's im2col and block n + 2's copies.
constexpr int kTwKB = 128;
constexpr int kTwStages = 2;          // at most: load stages and A buffers
constexpr int kTwCtas = 304;          // 2 per SM
constexpr int kTwThreads = 160;

struct TwSmem {
    uint64_t lfull[kTwStages], afull[kTwStages], mdone[kTwStages];
    uint32_t tmem_base;
    int abort_flag;
};

// Window elements a stage holds: a block's 128 positions, the 10 P + 10 of its
// taps' reach, rounded up to 16 bytes, and 8 more that the last aligned read of
// a row may touch (never used).
__host__ __device__ inline int tw_wlen(int P) { return (kTwKB + 10 * P + 10 + 7) / 8 * 8 + 8; }

// 8 consecutive bf16 starting at element o (0..7) of the 16 held in a, b, as 4
// words (element 2 j in the low half of word j).
__device__ __forceinline__ uint4 tw_shift8(const uint4& a, const uint4& b, int o)
{
    const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    uint32_t v[6], u[5];
#pragma unroll
    for (int j = 0; j < 6; ++j) v[j] = (o & 4) ? w[j + 2] : w[j];
#pragma unroll
    for (int j = 0; j < 5; ++j) u[j] = (o & 2) ? v[j + 1] : v[j];
    const uint32_t sel = (o & 1) ? 0x5432u : 0x3210u;
    return make_uint4(__byte_perm(u[0], u[1], sel), __byte_perm(u[1], u[2], sel), __byte_perm(u[2], u[3], sel),
                      __byte_perm(u[3], u[4], sel));
}

template <int CJ, int SGN>
__global__ void __launch_bounds__(kTwThreads) tapwgrad_kernel(const bf16* __restrict__ S, const bf16* __restrict__ C,
                                                              int B, int P, int HP16, int plane_len, int nst,
                                                              float* __restrict__ part, int* status)
{
    constexpr uint32_t ABYTES = (kTwKB / 8) * 128 * 16;   // [16 chunks][128 rows][8]
    constexpr uint32_t BBYTES = (CJ / 8) * kTwKB * 16;    // [CJ/8 groups][128 positions][8]
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* sA = smem_raw;                               // [stage][ABYTES]
    uint8_t* sB = sA + nst * ABYTES;                      // [stage][BBYTES]
    const int wlen = tw_wlen(P);
    uint8_t* sS = sB + nst * BBYTES;                      // [stage][wlen] bf16
    TwSmem* ss = reinterpret_cast<TwSmem*>(sS + nst * wlen * 2);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int nb_img = (HP16 + kTwKB - 1) / kTwKB;
    const long long total = (long long)B * nb_img;
    const long long blk0 = total * blockIdx.x / gridDim.x, blk1 = total * (blockIdx.x + 1) / gridDim.x;
    const int nblk = (int)(blk1 - blk0);
    const int u_begin = kPad * P + kPad;

    if (threadIdx.x == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(smem_u32(&ss->lfull[s]), 1);
            mbar_init(smem_u32(&ss->afull[s]), 128);
            mbar_init(smem_u32(&ss->mdone[s]), 1);
        }
        ss->abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 4) {
        tmem_alloc(smem_u32(&ss->tmem_base), CJ < 32 ? 32 : CJ);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = ss->tmem_base;
    auto block_pos = [&](int n, int& b, int& u0, int& npos) {
        const long long k = blk0 + n;
        b = (int)(k / nb_img);
        u0 = u_begin + (int)(k % nb_img) * kTwKB;
        npos = min(kTwKB, u_begin + HP16 - u0);
    };
    bool ok = true;
    if (warp == 4) {
        // ------------------------------------------------ copies and MMAs
        // block n's window and C planes into stage n % nst: lane 0 the window, lane
        // 1 + c the C plane c (lane 0 first sets the stage's byte count)
        auto issue = [&](int n) {
            int b, u0, npos;
            block_pos(n, b, u0, npos);
            const int st = n % nst;
            const uint32_t bar = smem_u32(&ss->lfull[st]);
            const int wcopy = (npos + 10 * P + 10 + 7) / 8 * 8;   // stays inside the plane for the last block
            if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)wcopy * 2 + (CJ / 8) * npos * 16);
            __syncwarp();
            if (lane == 0)
                bulk_g2s(smem_u32(sS + st * wlen * 2), S + (size_t)b * plane_len + u0 - 5 * P - 5,
                         (uint32_t)wcopy * 2, bar);
            else if (lane <= CJ / 8)
                bulk_g2s(smem_u32(sB + st * BBYTES + (lane - 1) * kTwKB * 16),
                         reinterpret_cast<const uint8_t*>(C) +
                             (((size_t)b * (CJ / 8) + (lane - 1)) * plane_len + u0) * 16,
                         npos * 16, bar);
        };
        for (int n = 0; n < nblk && n < nst; ++n) issue(n);
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((uint32_t)(CJ >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);
        for (int n = 0; n < nblk && ok; ++n) {
            const int st = n % nst, use = n / nst;
            int b, u0, npos;
            block_pos(n, b, u0, npos);
            ok = mbar_wait(smem_u32(&ss->afull[st]), use & 1, status, &ss->abort_flag);
            if (!__all_sync(0xffffffffu, ok)) {
                ok = false;
                break;
            }
            if (lane == 0) {
                tc_fence_after();
                for (int ks = 0; ks < npos / 16; ++ks) {
                    const uint64_t ad = sdesc(smem_u32(sA + st * ABYTES + ks * 2 * 2048), 2048, 128);
                    const uint64_t bd = sdesc(smem_u32(sB + st * BBYTES + ks * 256), 128, kTwKB * 16);
                    mma_bf16(tbase, ad, bd, idesc, (n == 0 && ks == 0) ? 0u : 1u);
                }
                mma_commit(smem_u32(&ss->mdone[st]));
            }
            // stage st is free again once these MMAs are done: fill it with block n + nst
            if (n + nst < nblk) {
                ok = mbar_wait(smem_u32(&ss->mdone[st]), use & 1, status, &ss->abort_flag);
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                issue(n + nst);
            }
        }
        // the last MMAs, and copies in flight after an abort
        if (lane == 0) {
            for (int n = max(0, nblk - nst); n < nblk; ++n)
                mbar_wait_drain(smem_u32(&ss->mdone[n % nst]), (n / nst) & 1);
            for (int n = max(0, nblk - nst); n < nblk; ++n)
                mbar_wait_drain(smem_u32(&ss->lfull[n % nst]), (n / nst) & 1);
        }
    } else {
        // ------------------------------------------------ im2col (warps 0..3)
        const int t = threadIdx.x;                              // im2col row = tap
        const int dy = t / 11, dx = t % 11;
        const int base_t = SGN * ((dy - 5) * P + (dx - 5)) + 5 * P + 5;   // window index of position 0
        const int o = base_t & 7;
        for (int n = 0; n < nblk && ok; ++n) {
            const int st = n % nst, use = n / nst;
            int b, u0, npos;
            block_pos(n, b, u0, npos);
            ok = mbar_wait(smem_u32(&ss->lfull[st]), use & 1, status, &ss->abort_flag);
            // A buffer st was read by block n - nst's MMAs
            if (ok && n >= nst)
                ok = mbar_wait(smem_u32(&ss->mdone[st]), (use - 1) & 1, status, &ss->abort_flag);
            if (!__all_sync(0xffffffffu, ok)) {
                ok = false;
                break;
            }
            uint4* dA = reinterpret_cast<uint4*>(sA + st * ABYTES);
            if (t < 121) {
                const uint32_t a0 = smem_u32(sS + st * wlen * 2) + (uint32_t)(base_t & ~7) * 2u;
                uint4 cur = lds128(a0);
                for (int kc = 0; kc < npos / 8; ++kc) {
                    const uint4 nxt = lds128(a0 + 16u * (uint32_t)(kc + 1));
                    dA[kc * 128 + t] = tw_shift8(cur, nxt, o);
                    cur = nxt;
                }
            } else {
                const uint32_t fill = (SGN > 0 && t == 127) ? 0x3F803F80u : 0u;   // bf16 1.0 (bias row) or 0
                for (int kc = 0; kc < npos / 8; ++kc) dA[kc * 128 + t] = make_uint4(fill, fill, fill, fill);
            }
            fence_proxy_async();
            mbar_arrive(smem_u32(&ss->afull[st]));
        }
    }
    // this CTA's partial
    __syncthreads();
    tc_fence_after();
    ok = !ss->abort_flag;
    if (warp < 4) {
        float* dst = part + ((size_t)blockIdx.x * 128 + warp * 32 + lane) * CJ;
        for (int c0 = 0; c0 < CJ; c0 += 16) {
            float v[16];
            if (ok && nblk > 0) tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + c0, v);
            else
                for (int i = 0; i < 16; ++i) v[i] = 0.f;
#pragma unroll
            for (int i = 0; i < 16; i += 4)
                *reinterpret_cast<float4*>(dst + c0 + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 4) {
        tc_fence_after();
        tmem_dealloc(tbase, CJ < 32 ? 32 : CJ);
    }
}

// conv1: dw[j][t] (= [64][1][11][11]) and db[j] from row 127; conv3: dw[j][t] (= [1][32][11][11]).
// One block per tap row r (row 127 for the bias); thread (grp, j) adds the
// partials of CTAs grp, grp + kTwGroups, ... (contiguous over j), then thread
// (0, j) adds the kTwGroups sums in order: a fixed summation order.
constexpr int kTwGroups = 8;
template <int CJ>
__global__ void tapwgrad_reduce_kernel(const float* __restrict__ part, int nctas, float* __restrict__ dw,
                                       float* __restrict__ db)
{
    const int r = blockIdx.x;
    if (r == 121 && !db) return;
    const int row = r < 121 ? r : 127;
    const int j = threadIdx.x % CJ, grp = threadIdx.x / CJ;
    double acc = 0.0;
    for (int c = grp; c < nctas; c += kTwGroups) acc += (double)part[((size_t)c * 128 + row) * CJ + j];
    __shared__ double red[kTwGroups][CJ];
    red[grp][j] = acc;
    __syncthreads();
    if (grp == 0) {
        double t = 0.0;
        for (int k = 0; k < kTwGroups; ++k) t += red[k][j];
        if (r < 121) dw[j * 121 + r] = (float)t;
        else db[j] = (float)t;
    }
}

}  // namespace

int pack_dgrad_weights(const float* w1, const float* w2, const float* w3, bf16* w1t, bf16* w2t, bf16* w3t,
                       cudaStream_t st)
{
    pack_dgrad_weights_kernel<<<grid_for((long long)(kW2PackElems + kW3tPackElems + kW1tPackElems)), 256, 0, st>>>(
        w1, w2, w3, w1t, w2t, w3t);
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

int grad_plane(const float* g, int B, const Geo& geo, bf16* gp, cudaStream_t st)
{
    if (B <= 0) return DEEPINV_OK;
    const int N = geo.H * geo.W;
    dim3 grid((unsigned)std::min((N + 255) / 256, 64), (unsigned)std::min(B, 65535));
    grad_plane_kernel<<<grid, 256, 0, st>>>(g, B, geo.H, geo.W, geo.P, geo.plane, gp);
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

int plane_channel_sums(const bf16* src, int B, int C, const Geo& geo, double* part, float* out, cudaStream_t st)
{
    // segments per plane (the partials fill part's B x 64 entries at most); the
    // one-channel plane's partials are all added by one warp, so it takes fewer
    const int nseg = C == 1 ? 4 : 64 / C;
    plane_sum_kernel<<<dim3(B, C == 1 ? 1 : C / 8, nseg), 256, 0, st>>>(src, C, geo.plane, nseg, part);
    DI_LAUNCH_CHECK();
    sum_parts_kernel<<<C, 32, 0, st>>>(part, B * nseg, C, out);
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

// ---------------------------------------------------------------- conv2 / hidden-layer weight gradients
// dW2[co][ci][dy][4 s + g] = sum_u G[u - g][co] A1[u + (dy - 5) P + 4 s - 5][ci]
// over plane positions u (G is zero off the data positions), as MMAs with
// K = 16 positions whose operands are shifted windows of the two planes: the
// tap phase g shifts G, the kernel row and column group (dy, s) shift A1.
// Every shifted window is read straight out of ONE window per plane instead of
// one copy per shift.  The windows are stored channel-contiguous per position, with the
// tensor core's swizzles: the a1 window as 128-byte rows (64 channels, 16-byte
// chunk c of row r at chunk c ^ (r % 8)), the g2 window as 64-byte rows (32
// channels, chunk c at c ^ ((r / 2) % 4)).  Both are MN-major operands whose
// swizzle follows the shared-memory address, so an operand may start at any
// row: the A operand (M = 128: slots j = 0..3 x 32 filters, slot j = tap phase
// g = 3 - j, i.e. the g2 rows one position apart) is the g2 window from row
// 16 k + 5 with LBO = 64 bytes (next slot) and SBO = 512 (next 8 positions);
// the B operand (N = 192: column groups s = 0..2 x 64 channels, 4 positions
// apart) is the a1 window from row 16 k + r P (kernel row dy0 + r) with
// LBO = 512 and SBO = 1024.  One MMA covers the 12 taps (dy, 4 s + g) of a
// kernel row (tap 11 unused) for 16 positions.
//
// Each CTA takes ROWS consecutive kernel rows (its column; ROWS = 2 for conv2
// and 4 for a hidden layer when three stages of the window fit, one TMEM
// accumulator per row) and a run of 128-position blocks (its split).  Per block
// the four epilogue warps load the two windows with 16-byte cp.async, each
// chunk placed at its swizzled address (the g2 window serves every row of the
// CTA): for conv2 at 64 x 64, 35 KB per block for 16 MMAs M128 N192 K16.  A
// copy of every shifted window (one 1-D bulk copy or cp.async run per window)
// had taken 72 KB for 6 MMAs M128 N256 K16, paced by the copies.
constexpr int kWsKB = 128;                         // positions per block
constexpr int kWsRows = kWsKB + 8;                 // g2 window rows; the a1 window adds (ROWS - 1) P
constexpr int kWsMaxStages = 6;
constexpr uint32_t kWsGBytes = 9 * 1024;           // g2 window: 136 x 64 B, rounded up to 1024

// CIN = 64: conv2 (a1 window rows of 128 bytes, 128-byte swizzle, N = 192).
// CIN = 32: a hidden layer (its input plane as 64-byte rows, 64-byte swizzle,
// N = 96; up to four kernel rows per CTA).
template <int CIN, int ROWS>
struct WsCfg {
    static constexpr int N = 3 * CIN;                    // column groups s = 0..2 x CIN channels
    static constexpr int RB = 2 * CIN;                   // bytes per window row of the input plane
    static constexpr int CPG = CIN / 8;                  // 16-byte chunks per row
    static constexpr uint32_t SWZ = CIN == 64 ? 2 : 4;   // 128- or 64-byte swizzle
    static constexpr int TCOLS = N <= 128 ? 128 : 256;   // TMEM columns per kernel row
    static constexpr int COLS = (11 + ROWS - 1) / ROWS;
    static constexpr int SPLIT = 144 / COLS;             // 143 or 144 CTAs
};

// input-window bytes (a whole number of 1024-byte swizzle patterns)
__host__ __device__ inline uint32_t ws_abytes(int rows, int P, int rb)
{
    return ((uint32_t)(kWsRows + (rows - 1) * P) * (uint32_t)rb + 1023u) / 1024u * 1024u;
}

struct WsSmem {
    uint64_t full[kWsMaxStages], empty[kWsMaxStages], acc_full, drain;
    uint32_t tmem_base;
    int abort_flag;
};

// MN-major shared-memory descriptor with a swizzle mode (2 = 128-byte, 4 = 64-byte).
__device__ __forceinline__ uint64_t sdesc_sw(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t swz)
{
    return sdesc(saddr, lbo, sbo) | ((uint64_t)swz << 61);
}

template <int CIN, int ROWS>
__global__ void __launch_bounds__(192, 1) wgrad2sw_kernel(const bf16* __restrict__ G2, const bf16* __restrict__ A1,
                                                          int B, int P, int HP16, int plane_len, int nst,
                                                          float* __restrict__ part, int* status)
{
    using C = WsCfg<CIN, ROWS>;
    extern __shared__ uint8_t smem_dyn[];
    uint8_t* smem = smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
    const uint32_t abytes = ws_abytes(ROWS, P, C::RB), stage = abytes + kWsGBytes;
    WsSmem* ss = reinterpret_cast<WsSmem*>(smem + nst * stage);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int col = blockIdx.x % C::COLS, split = blockIdx.x / C::COLS;
    const int dy0 = col * ROWS, nrows = min(ROWS, 11 - dy0);
    const int arows = kWsRows + (nrows - 1) * P;       // a1 window rows of this CTA
    const int nb_img = (HP16 + kWsKB - 1) / kWsKB;
    const long long total = (long long)B * nb_img;
    const long long blk0 = total * split / C::SPLIT, blk1 = total * (split + 1) / C::SPLIT;
    const int u_begin = kPad * P + kPad;
    const int off0 = (dy0 - 5) * P - 5;                // a1 offset of kernel row dy0, column group s = 0

    if (threadIdx.x == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(smem_u32(&ss->full[s]), 128);    // one cp.async arrival per loader thread
            mbar_init(smem_u32(&ss->empty[s]), 1);
        }
        mbar_init(smem_u32(&ss->acc_full), 1);
        mbar_init(smem_u32(&ss->drain), 1);
        ss->abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(&ss->tmem_base), ROWS * C::TCOLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = ss->tmem_base;

    if (warp >= 2) {
        // ------------------------------------------------ loaders (then the epilogue)
        const int t = threadIdx.x - 64;
        for (long long k = blk0; k < blk1; ++k) {
            const int st = (int)((k - blk0) % nst), n = (int)((k - blk0) / nst);
            bool ok = true;
            if (lane == 0) ok = mbar_wait(smem_u32(&ss->empty[st]), (n & 1) ^ 1, status, &ss->abort_flag);
            if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) break;
            const int b = (int)(k / nb_img);
            const int u0 = u_begin + (int)(k % nb_img) * kWsKB;
            const uint8_t* a1b =
                reinterpret_cast<const uint8_t*>(A1) + ((size_t)b * C::CPG * plane_len + (size_t)(u0 + off0)) * 16;
            const uint8_t* g2b = reinterpret_cast<const uint8_t*>(G2) + ((size_t)b * 4 * plane_len + (size_t)(u0 - 8)) * 16;
            const uint32_t dA = smem_u32(smem + st * stage), dG = dA + abytes;
            // input: row r = position u0 + off0 + r, chunk c (CPG per row); g2: row r = position
            // u0 - 8 + r, chunk c (4 per row)
            for (int i = t; i < arows * C::CPG; i += 128) {
                const int r = i / C::CPG, c = i % C::CPG;
                const int pc = CIN == 64 ? (c ^ (r & 7)) : (c ^ ((r >> 1) & 3));
                cp_async16(dA + r * C::RB + (pc << 4), a1b + ((size_t)c * plane_len + r) * 16);
            }
            for (int i = t; i < kWsRows * 4; i += 128) {
                const int r = i >> 2, c = i & 3;
                cp_async16(dG + r * 64 + ((c ^ ((r >> 1) & 3)) << 4), g2b + ((size_t)c * plane_len + r) * 16);
            }
            cp_async_arrive(smem_u32(&ss->full[st]));
        }
        cp_async_wait_all();
    } else if (warp == 1 && lane == 0) {
        // ------------------------------------------------ MMA issuer
        const uint32_t idesc = idesc_bf16_mn(128, C::N);
        bool first = true;
        for (long long k = blk0; k < blk1; ++k) {
            const int st = (int)((k - blk0) % nst), n = (int)((k - blk0) / nst);
            if (!mbar_wait(smem_u32(&ss->full[st]), n & 1, status, &ss->abort_flag)) break;
            fence_proxy_async();   // the windows were written by cp.async (generic proxy)
            tc_fence_after();
            const int u0 = u_begin + (int)(k % nb_img) * kWsKB;
            const int nsteps = min(kWsKB, u_begin + HP16 - u0) / 16;
            const uint32_t a0 = smem_u32(smem + st * stage), g0 = a0 + abytes;
            for (int j = 0; j < nsteps; ++j) {
                const uint64_t ad = sdesc_sw(g0 + (16 * j + 5) * 64, 64, 512, 4);
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    if (r < nrows) {
                        const uint64_t bd = sdesc_sw(a0 + (16 * j + r * P) * C::RB, 4 * C::RB, 8 * C::RB, C::SWZ);
                        mma_bf16(tbase + (uint32_t)(r * C::TCOLS), ad, bd, idesc, first ? 0u : 1u);
                    }
                }
                first = false;
            }
            mma_commit(smem_u32(&ss->empty[st]));
        }
        // an empty range still produces a (zero) partial
        mma_commit(smem_u32(&ss->acc_full));
        mma_commit(smem_u32(&ss->drain));
        mbar_wait_drain(smem_u32(&ss->drain), 0);
    }
    if (warp >= 2) {
        const int q = warp % 4;
        bool ok = mbar_wait(smem_u32(&ss->acc_full), 0, status, &ss->abort_flag);
        ok = __all_sync(0xffffffffu, ok);
        tc_fence_after();
        const bool empty = blk1 <= blk0;
        for (int r = 0; r < nrows; ++r) {
            float* dst = part + (((size_t)blockIdx.x * ROWS + r) * 128 + q * 32 + lane) * C::N;
            for (int c0 = 0; c0 < C::N; c0 += 16) {
                float v[16];
                if (ok && !empty) tmem_ld16(tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(r * C::TCOLS + c0), v);
                else
                    for (int i = 0; i < 16; ++i) v[i] = 0.f;
#pragma unroll
                for (int i = 0; i < 16; i += 4)
                    *reinterpret_cast<float4*>(dst + c0 + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tbase, ROWS * C::TCOLS);
    }
}

// dW[co][ci][dy][dx] = sum over splits of part[col + COLS split][row][32 (3 - g) + co][CIN s + ci],
// col = dy / ROWS, row = dy % ROWS, dx = 4 s + g, in float64 in split order.
// Consecutive threads take consecutive ci (contiguous partials).
template <int CIN, int ROWS>
__global__ void wgrad2sw_reduce_kernel(const float* __restrict__ part, float* __restrict__ dw)
{
    using C = WsCfg<CIN, ROWS>;
    const int n = 32 * CIN * 121;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int ci = i % CIN, dx = (i / CIN) % 11, dy = (i / (CIN * 11)) % 11, co = i / (CIN * 121);
        const int s = dx / 4, g = dx % 4, col = dy / ROWS, row = dy % ROWS;
        double acc = 0.0;
        for (int k = 0; k < C::SPLIT; ++k)
            acc += (double)part[((((size_t)(col + C::COLS * k) * ROWS + row) * 128) + 32 * (3 - g) + co) * C::N +
                                CIN * s + ci];
        dw[((co * CIN + ci) * 11 + dy) * 11 + dx] = (float)acc;
    }
}

// Positions u that can carry a nonzero gradient: the data rows [5P+5, 5P+5+HP).
size_t wgrad2_scratch_floats()
{
    size_t sw = 0;
    auto upd = [&](size_t v) { if (v > sw) sw = v; };
    upd((size_t)WsCfg<64, 1>::COLS * WsCfg<64, 1>::SPLIT * 1 * 128 * WsCfg<64, 1>::N);
    upd((size_t)WsCfg<64, 2>::COLS * WsCfg<64, 2>::SPLIT * 2 * 128 * WsCfg<64, 2>::N);
    upd((size_t)WsCfg<32, 1>::COLS * WsCfg<32, 1>::SPLIT * 1 * 128 * WsCfg<32, 1>::N);
    upd((size_t)WsCfg<32, 4>::COLS * WsCfg<32, 4>::SPLIT * 4 * 128 * WsCfg<32, 4>::N);
    return sw;
}


template <int CIN, int ROWS>
static int wgrad2sw_launch(const bf16* G2, const bf16* A1, int B, const Geo& g, int nst, float* part, float* dw,
                           int* status, cudaStream_t st)
{
    using C = WsCfg<CIN, ROWS>;
    const int HP16 = (g.HP + 15) / 16 * 16;
    const size_t smem = 1024 + (size_t)nst * (ws_abytes(ROWS, g.P, C::RB) + kWsGBytes) + sizeof(WsSmem);
    DI_CUDA(cudaFuncSetAttribute(wgrad2sw_kernel<CIN, ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    wgrad2sw_kernel<CIN, ROWS><<<C::COLS * C::SPLIT, 192, smem, st>>>(G2, A1, B, g.P, HP16, g.plane, nst, part,
                                                                      status);
    DI_LAUNCH_CHECK();
    wgrad2sw_reduce_kernel<CIN, ROWS><<<grid_for(32 * CIN * 121), 256, 0, st>>>(part, dw);
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

// Stages of the swizzled-window kernel that fit in shared memory (0: none).
static int ws_stages(int rows, int P, int rb)
{
    const size_t per = (size_t)ws_abytes(rows, P, rb) + kWsGBytes;
    const size_t avail = 227 * 1024 - 1024 - sizeof(WsSmem);
    const size_t n = avail / per;
    return (int)(n > (size_t)kWsMaxStages ? kWsMaxStages : n);
}

int wgrad2_tc(const bf16* G2, const bf16* A1, int B, const Geo& g, float* part, float* dw, int* status,
              cudaStream_t st)
{
    // two kernel rows per CTA while three stages of their window fit, else one
    // row per CTA (its window does not depend on the image width)
    const int n2 = ws_stages(2, g.P, 128);
    if (n2 >= 3) return wgrad2sw_launch<64, 2>(G2, A1, B, g, n2, part, dw, status, st);
    return wgrad2sw_launch<64, 1>(G2, A1, B, g, ws_stages(1, g.P, 128), part, dw, status, st);
}

int wgrad_hidden_tc(const bf16* G, const bf16* A, int B, const Geo& g, float* part, float* dw, int* status,
                    cudaStream_t st)
{
    // four kernel rows per CTA (TMEM: 4 x 128 columns) while three stages fit,
    // else one
    const int n4 = ws_stages(4, g.P, 64);
    if (n4 >= 3) return wgrad2sw_launch<32, 4>(G, A, B, g, n4, part, dw, status, st);
    return wgrad2sw_launch<32, 1>(G, A, B, g, ws_stages(1, g.P, 64), part, dw, status, st);
}

size_t tapwgrad_scratch_floats() { return (size_t)kTwCtas * 128 * 64; }

int tap_wgrad_tc(bool conv1, const bf16* S, const bf16* C, int B, const Geo& g, float* part, float* dw, float* db,
                 int* status, cudaStream_t st)
{
    const int HP16 = (g.HP + 15) / 16 * 16;
    const int wlen = tw_wlen(g.P);
    const int CJ = conv1 ? 64 : 32;
    auto smem_for = [&](int k) {
        return k * ((size_t)(kTwKB / 8) * 128 * 16 + (size_t)(CJ / 8) * kTwKB * 16 + (size_t)wlen * 2) +
               sizeof(TwSmem) + 16;
    };
    const int nst = smem_for(kTwStages) <= 227 * 1024 ? kTwStages : 1;
    const size_t smem = smem_for(nst);
    if (smem > 227 * 1024) {
        set_error("weight gradient: image width %d too large for the shared-memory window", g.W);
        return DEEPINV_EUNSUPPORTED;
    }
    if (conv1) {
        DI_CUDA(cudaFuncSetAttribute(tapwgrad_kernel<64, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        tapwgrad_kernel<64, 1><<<kTwCtas, kTwThreads, smem, st>>>(S, C, B, g.P, HP16, g.plane, nst, part, status);
        DI_LAUNCH_CHECK();
        tapwgrad_reduce_kernel<64><<<122, 64 * kTwGroups, 0, st>>>(part, kTwCtas, dw, db);
    } else {
        DI_CUDA(cudaFuncSetAttribute(tapwgrad_kernel<32, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        tapwgrad_kernel<32, -1><<<kTwCtas, kTwThreads, smem, st>>>(S, C, B, g.P, HP16, g.plane, nst, part, status);
        DI_LAUNCH_CHECK();
        tapwgrad_reduce_kernel<32><<<122, 32 * kTwGroups, 0, st>>>(part, kTwCtas, dw, nullptr);
    }
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

}  // namespace di
