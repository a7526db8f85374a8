// conv1 and conv2 of the bfloat16 path in one kernel (Sec. 4, Eq. 1: the first
// two layers, 1 -> 64 -> 32 channels, bias and ReLU after each), so that a1
// never travels through HBM.
//
// Each persistent CTA walks a contiguous run of conv2 tiles of one image
// plane after another.  conv1's output for the positions the next kernel rows
// will read is produced into a shared-memory ring of a1 (8 blocks of 128
// positions x 64 channels, bf16, the conv2 operand layout: 8 chunks of 8
// channels, 16 bytes per position), so every a1 value is computed once per
// walk; a block's slot is handed back as soon as no later kernel row of the
// walk reads it.  The live window of a walk is 10 rows of the plane plus a
// tile, so the ring holds planes whose pitch is at most 75 positions; wider
// images are cut into column strips of at most 55 columns, each walked as its
// own plane (pitch = strip width + 20: a 5-column halo of a1 on each side and
// another 5 of x~ for conv1), their x~ first gathered into strip planes.
//
// conv1 per block of 128 a1 positions: per kernel row dy one MMA M = 128
// positions, N = 64 filters, K = 16 (the 11 columns dx, zero weights for
// dx >= 11), the A operand read MN-major from an expanded x~ ring whose row e
// holds x~[e .. e + 7] (core matrices overlap, both strides 128 bytes); the
// ring keeps the 10 plane rows + 136 positions a block reads, its first 144
// rows repeated past its end so that no operand wraps.
// conv2 per tile of 221 outputs: conv2's tap stacking (4 tap slots x 32
// filters as M = 128, N = 224 positions, K = 16 channels; 33 (dy, s) pairs x 4
// chunks), B read straight from the a1 ring; an operand that would run past
// the ring's end is issued as two MMAs split at a multiple of 16 columns, the
// second starting in a 16-position copy of the ring's end kept before its
// start.
//
// TMEM: two conv2 accumulators of 224 columns and one conv1 accumulator of 64.
// Warps: 0 expands x~ into its ring; 1 owns TMEM, one thread issues every MMA
// (conv1 blocks ahead of need, whenever their inputs are ready, between conv2
// kernel rows); 2..5 drain conv2 tiles (conv2's epilogue: slot exchange, bias,
// ReLU, 16-byte stores); 6 streams conv1's weights once and conv2's stacked
// weights as a 2-deep ring of (dy, s) blocks; 7..10 drain conv1 blocks (bias,
// ReLU, zero outside the image) into the a1 ring.  Every wait is bounded.
#include "kernels.cuh"
#include "tc.cuh"

#include <climits>

namespace di {

using namespace tc;

namespace {

constexpr int kFN = 224;                            // conv2 MMA N: positions per tile
constexpr int kFValid = kFN - 3;                    // outputs a tile completes
constexpr int kFRead = kFN + 8;                     // a1 positions one kernel row's MMAs read
constexpr int kFBlocks = 8;                         // a1 ring blocks of 128 positions
constexpr int kFRing = kFBlocks * 128;
constexpr int kFPre = 16;                           // copy of the ring's last 16 positions
constexpr uint32_t kFChunk = (kFPre + kFRing) * 16; // bytes per 8-channel chunk of the ring
constexpr int kFERows = 1024;                       // expanded-x~ ring rows
constexpr int kFETail = 144;                        // rows [0, 144) repeated past its end
constexpr uint32_t kFEOff = 1u << 24;               // keeps (negative) x~ indices positive before the modulo
constexpr uint32_t kFWBlock = 16384;                // one (dy, s) block of stacked conv2 weights
constexpr uint32_t kFW1Bytes = 11 * 2 * 64 * 16;    // conv1 weights [dy][K half][64][8]
constexpr int kFXStride = 36;                       // floats per row of the slot exchange
constexpr uint32_t kFXBytes = 4 * 32 * kFXStride * 4;
constexpr int kFThreads = 352;
constexpr uint32_t kFC1Col = 2 * kFN;               // TMEM column of the conv1 accumulator
constexpr int kFMaxPitch = 75;                      // widest plane the rings hold
constexpr int kFMaxStrip = kFMaxPitch - 20;         // widest column strip

struct FusedSmem {
    alignas(16) float bias1[64];
    uint64_t a1_full[kFBlocks], slot_free[kFBlocks];
    uint64_t wfull[2], wempty[2];
    uint64_t efull[2], efree[2];
    uint64_t c1_full, c1_empty;
    uint64_t w1bar;
    uint64_t acc_full[2], acc_empty[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort_flag;
    int vote[2][4];
};

constexpr size_t kFOffW2 = (size_t)8 * kFChunk;
constexpr size_t kFOffW1 = kFOffW2 + 2 * (size_t)kFWBlock;
constexpr size_t kFOffE = kFOffW1 + kFW1Bytes;
constexpr size_t kFOffX = kFOffE + (size_t)(kFERows + kFETail) * 16;
constexpr size_t kFOffS = kFOffX + kFXBytes;
constexpr size_t kFSmem = kFOffS + sizeof(FusedSmem);
static_assert(kFSmem <= 232448, "fused conv1/conv2 shared memory");
static_assert(kFOffW2 % 1024 == 0 && kFOffW1 % 16 == 0 && kFOffE % 16 == 0 && kFOffX % 16 == 0, "alignment");

// The planes the kernel walks.  Whole width (strips == 0): the real x~ plane
// (pitch P), a1 position p = (r + 5) P + c + 5 for pixel (r, c).  Strips: the
// gathered x~ strip plane of pitch PV, x~ position (R, C) = pixel (R - 5,
// c0 + C - 10), and a1 position (R, C) = pixel (R - 5, c0 + C - 5) for
// C < PV - 10.  conv2's output index q = r PV + C' is pixel (r, c0 + C').
struct FusedGeo {
    int H, W, P;      // image rows, columns, pitch of the real planes
    int PV;           // pitch of the planes walked
    int nstrip, SW;   // column strips and their width (1 and W: the whole width)
    int strips;       // 1: walked planes are gathered strip planes
    int HV;           // H * PV output indices per walked plane
    int t2;           // tiles per walked plane
    int xplane;       // elements per x~ plane read
    int aplane;       // positions per real a2 plane
};

struct Walked {
    const bf16* x;    // its x~ plane
    int b;            // image
    int c0, sw;       // first column, columns
    bool last;        // rightmost strip: also writes the pad columns
    int acol;         // pixel column of a1 column C is C + acol
    int ca;           // a1 columns computed from in-row x~ (C < ca)
    int xoff;         // x~ index of a1 position p, tap (dy, dx): p + (dy - 5) PV + dx + xoff
};

__device__ __forceinline__ Walked walked(const FusedGeo& g, const bf16* xt, int v)
{
    Walked w;
    w.b = v / g.nstrip;
    const int s = v - w.b * g.nstrip;
    w.c0 = s * g.SW;
    w.sw = min(g.SW, g.W - w.c0);
    w.last = s == g.nstrip - 1;
    if (g.strips) {
        w.x = xt + (size_t)v * g.xplane;
        w.acol = w.c0 - 5;
        w.ca = g.PV - 10;
        w.xoff = 0;
    } else {
        w.x = xt + (size_t)w.b * g.xplane;
        w.acol = -5;
        w.ca = g.PV;
        w.xoff = -5;
    }
    return w;
}

// a1 blocks [k0, k1] a run of tiles [tlo, thi) of one plane reads
__device__ __forceinline__ void run_blocks(int tlo, int thi, int PV, int& k0, int& k1)
{
    k0 = (tlo * kFValid) >> 7;
    k1 = ((thi - 1) * kFValid + 10 * PV + kFRead - 1) >> 7;
}

__device__ __forceinline__ uint4 f12_pack8(const float* v)
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

__device__ __forceinline__ void f12_epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

template <int G>
__device__ __forceinline__ void f12_put_shifted(float* x, const float* v)
{
#pragma unroll
    for (int j = 0; j < 32; j += 4)
        *reinterpret_cast<float4*>(x + j) = make_float4(v[j + G], v[j + G + 1], v[j + G + 2], v[j + G + 3]);
}

__global__ void __launch_bounds__(kFThreads, 1)
    conv12_kernel(const bf16* __restrict__ xt, int V, FusedGeo g, const bf16* __restrict__ w1p,
                  const float* __restrict__ b1, const bf16* __restrict__ w2p, const float* __restrict__ b2,
                  bf16* __restrict__ a2, int* status)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* sRing = smem_raw;                                        // [8 chunks][16 + 1024 positions][16 B]
    uint8_t* sW2 = smem_raw + kFOffW2;                                // [2][16 KB]
    uint8_t* sW1 = smem_raw + kFOffW1;
    uint4* sE = reinterpret_cast<uint4*>(smem_raw + kFOffE);          // [1024 + 144] rows
    float* sX = reinterpret_cast<float*>(smem_raw + kFOffX);          // [4 slots][32 filters][kFXStride]
    FusedSmem* ss = reinterpret_cast<FusedSmem*>(smem_raw + kFOffS);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int PV = g.PV;
    const int ntiles = V * g.t2;
    const int tlo_all = (int)((long long)ntiles * blockIdx.x / gridDim.x);
    const int thi_all = (int)((long long)ntiles * (blockIdx.x + 1) / gridDim.x);

    if (threadIdx.x == 0) {
        for (int j = 0; j < kFBlocks; ++j) {
            mbar_init(smem_u32(&ss->a1_full[j]), 128);
            mbar_init(smem_u32(&ss->slot_free[j]), 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&ss->wfull[s]), 1);
            mbar_init(smem_u32(&ss->wempty[s]), 1);
            mbar_init(smem_u32(&ss->efull[s]), 32);
            mbar_init(smem_u32(&ss->efree[s]), 1);
            mbar_init(smem_u32(&ss->acc_full[s]), 1);
            mbar_init(smem_u32(&ss->acc_empty[s]), 4);
        }
        mbar_init(smem_u32(&ss->c1_full), 1);
        mbar_init(smem_u32(&ss->c1_empty), 4);
        mbar_init(smem_u32(&ss->w1bar), 1);
        mbar_init(smem_u32(&ss->drain), 1);
        ss->abort_flag = 0;
        fence_mbar_init();
    }
    if (threadIdx.x < 64) ss->bias1[threadIdx.x] = __ldg(&b1[threadIdx.x]);
    if (warp == 1) {
        tmem_alloc(smem_u32(&ss->tmem_base), 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = ss->tmem_base;
    volatile int* abort_flag = &ss->abort_flag;

    if (warp == 0) {
        // ------------------------------------------------ x~ expansion into the E ring
        int n = 0;
        bool ok = true;
        for (int tile = tlo_all; tile < thi_all && ok;) {
            const int v = tile / g.t2, tlo = tile - v * g.t2, thi = min(g.t2, tlo + (thi_all - tile));
            tile += thi - tlo;
            const Walked w = walked(g, xt, v);
            int k0, k1;
            run_blocks(tlo, thi, PV, k0, k1);
            int gnext = 0;
            for (int k = k0; k <= k1; ++k, ++n) {
                // rows of block n - 2 are overwritten; a run's first block rewrites
                // the whole ring, so block n - 1 must be done too
                ok = mbar_wait(smem_u32(&ss->efree[n & 1]), ((n >> 1) & 1) ^ 1, status, abort_flag);
                if (ok && k == k0 && n > 0)
                    ok = mbar_wait(smem_u32(&ss->efree[(n - 1) & 1]), ((n - 1) >> 1) & 1, status, abort_flag);
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                const int eb = 128 * k - 5 * PV + w.xoff;
                const int g0 = k == k0 ? (eb >> 3) : gnext;
                const int g1 = (eb + 10 * PV + 135) >> 3;
                for (int G = g0 + lane; G <= g1; G += 32) {
                    const int e0 = 8 * G;
                    uint4 lo = make_uint4(0, 0, 0, 0), hi = lo;
                    if (e0 >= 0 && e0 + 8 <= g.xplane) lo = __ldg(reinterpret_cast<const uint4*>(w.x + e0));
                    if (e0 + 8 >= 0 && e0 + 16 <= g.xplane) hi = __ldg(reinterpret_cast<const uint4*>(w.x + e0 + 8));
                    const uint32_t wv[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
                    const uint32_t r0 = ((uint32_t)e0 + kFEOff) & (kFERows - 1);
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        uint32_t o[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            o[e] = (kk & 1) ? __byte_perm(wv[kk / 2 + e], wv[kk / 2 + e + 1], 0x5432) : wv[kk / 2 + e];
                        const uint4 row = make_uint4(o[0], o[1], o[2], o[3]);
                        sE[r0 + kk] = row;
                        if (r0 < kFETail) sE[r0 + kk + kFERows] = row;
                    }
                }
                gnext = g1 + 1;
                fence_proxy_async();
                mbar_arrive(smem_u32(&ss->efull[n & 1]));
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0 && tlo_all < thi_all) {
            bool ok = mbar_wait(smem_u32(&ss->w1bar), 0, status, abort_flag);
            const uint32_t idesc1 = idesc_bf16(128, 64) | (1u << 15);   // A MN-major
            int n_iss = 0, n_ready = 0, n_free = 0, it = 0, ws = 0;
            for (int tile = tlo_all; tile < thi_all && ok;) {
                const int v = tile / g.t2, tlo = tile - v * g.t2, thi = min(g.t2, tlo + (thi_all - tile));
                tile += thi - tlo;
                const int xoff = g.strips ? 0 : -5;
                int k0, k1;
                run_blocks(tlo, thi, PV, k0, k1);
                const int nseg = n_iss;                // every earlier block is issued, ready and released
                const int nlast = nseg + k1 - k0;
                // conv1 MMAs of block n (blocking: wait for its inputs; else only if ready)
                auto issue = [&](int n, bool blocking) -> bool {
                    const uint32_t ef = smem_u32(&ss->efull[n & 1]), ce = smem_u32(&ss->c1_empty);
                    const uint32_t ep = (n >> 1) & 1, cp = (n & 1) ^ 1;
                    if (blocking) {
                        if (!mbar_wait(ef, ep, status, abort_flag) || !mbar_wait(ce, cp, status, abort_flag)) {
                            ok = false;
                            return false;
                        }
                    } else if (!mbar_test(ef, ep) || !mbar_test(ce, cp)) {
                        return false;
                    }
                    tc_fence_after();
                    const int eb = 128 * (k0 + n - nseg) - 5 * PV + xoff;
#pragma unroll
                    for (int dy = 0; dy < 11; ++dy) {
                        const uint32_t idx = ((uint32_t)(eb + dy * PV) + kFEOff) & (kFERows - 1);
                        const uint64_t ad = sdesc(smem_u32(sE + idx), 128, 128);
                        const uint64_t bd = sdesc(smem_u32(sW1 + dy * 2048), 1024, 128);
                        mma_bf16(tbase + kFC1Col, ad, bd, idesc1, dy > 0 ? 1u : 0u);
                    }
                    mma_commit(smem_u32(&ss->efree[n & 1]));
                    mma_commit(smem_u32(&ss->c1_full));
                    return true;
                };
                for (int tt = tlo; tt < thi && ok; ++tt, ++it) {
                    const int buf = it & 1;
                    if (!mbar_wait(smem_u32(&ss->acc_empty[buf]), ((it >> 1) & 1) ^ 1, status, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tbase + (uint32_t)(buf * kFN);
                    const int q0 = tt * kFValid;
                    for (int dy = 0; dy < 11 && ok; ++dy) {
                        const int lo = q0 + dy * PV;
                        const int nneed = nseg + ((lo + kFRead - 1) >> 7) - k0;
                        while (ok && n_iss <= nneed)
                            if (issue(n_iss, true)) ++n_iss;
                        while (ok && n_iss <= nlast && n_iss < n_free + kFBlocks && issue(n_iss, false)) ++n_iss;
                        while (ok && n_ready <= nneed) {
                            ok = mbar_wait(smem_u32(&ss->a1_full[n_ready % kFBlocks]), (n_ready / kFBlocks) & 1,
                                           status, abort_flag);
                            ++n_ready;
                        }
                        if (!ok) break;
                        tc_fence_after();
                        for (int s = 0; s < 3; ++s, ++ws) {
                            const int wslot = ws & 1;
                            if (!mbar_wait(smem_u32(&ss->wfull[wslot]), (ws >> 1) & 1, status, abort_flag)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const int p = lo + 4 * s;
                            const int R = ((nseg + (p >> 7) - k0) & (kFBlocks - 1)) * 128 + (p & 127);
                            const int n1 = R + kFN <= kFRing ? kFN : ((kFRing - R) & ~15);
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint64_t ad = sdesc(smem_u32(sW2 + wslot * kFWBlock + kk * 4096), 2048, 128);
                                const uint32_t cb = smem_u32(sRing + (2 * kk) * kFChunk);
                                const uint32_t acc = (dy | s | kk) ? 1u : 0u;
                                if (n1 > 0)
                                    mma_bf16(d, ad, sdesc(cb + (uint32_t)(kFPre + R) * 16, kFChunk, 128),
                                             idesc_bf16(128, n1), acc);
                                if (n1 < kFN)
                                    mma_bf16(d + (uint32_t)n1, ad,
                                             sdesc(cb + (uint32_t)(kFPre + R + n1 - kFRing) * 16, kFChunk, 128),
                                             idesc_bf16(128, kFN - n1), acc);
                            }
                            mma_commit(smem_u32(&ss->wempty[wslot]));
                        }
                        if (!ok) break;
                        // hand back the blocks that no later kernel row of this run reads
                        int lowest = dy < 10 ? lo + PV : INT_MAX;
                        if (tt + 1 < thi && q0 + kFValid < lowest) lowest = q0 + kFValid;
                        while (n_free < n_iss && ((long long)(k0 + n_free - nseg + 1) << 7) <= (long long)lowest) {
                            mma_commit(smem_u32(&ss->slot_free[n_free % kFBlocks]));
                            ++n_free;
                        }
                    }
                    if (!ok) break;
                    mma_commit(smem_u32(&ss->acc_full[buf]));
                }
            }
            mma_commit(smem_u32(&ss->drain));
            mbar_wait_drain(smem_u32(&ss->drain), 0);
        }
    } else if (warp < 6) {
        // ------------------------------------------------ conv2 epilogue
        const int quarter = warp % 4;                         // TMEM lane quarter = tap slot
        const int le = threadIdx.x - 64;                      // 0..127
        const int jl = le % 32;
        const int c8 = le / 32;                               // 8-channel group of this thread's outputs
        float bias8[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) bias8[e] = __ldg(&b2[c8 * 8 + e]);
        float* xrow = sX + (quarter * 32 + lane) * kFXStride;
        int it = 0;
        for (int tile = tlo_all; tile < thi_all; ++tile, ++it) {
            const int buf = it & 1, use = it >> 1;
            bool ok = mbar_wait(smem_u32(&ss->acc_full[buf]), use & 1, status, abort_flag);
            ok = __all_sync(0xffffffffu, ok);
            if (lane == 0) ss->vote[buf][quarter] = ok ? 1 : 0;
            f12_epi_bar();
            ok = ss->vote[buf][0] && ss->vote[buf][1] && ss->vote[buf][2] && ss->vote[buf][3];
            if (!ok) break;
            tc_fence_after();
            const int v = tile / g.t2;
            const int q0 = (tile - v * g.t2) * kFValid;
            const Walked w = walked(g, xt, v);
            const uint32_t lane_addr = tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * kFN);
            for (int cc = 0; cc < kFN; cc += 32) {
                const int jcol = cc + jl, qq = q0 + jcol;
                const int r = qq / PV, cv = qq - r * PV;
                const bool store = jcol < kFValid && qq < g.HV && (cv < w.sw || (w.last && cv < w.sw + 5));
                const bool data = store && cv < w.sw;
                float vv[36];
                tmem_ld32(lane_addr + cc, vv);
                if (cc + 32 < kFN) {
                    tmem_ld4(lane_addr + cc + 32, vv + 32);
                } else {
                    vv[32] = vv[33] = vv[34] = vv[35] = 0.f;
                }
                switch (quarter) {
                    case 0: f12_put_shifted<0>(xrow, vv); break;
                    case 1: f12_put_shifted<1>(xrow, vv); break;
                    case 2: f12_put_shifted<2>(xrow, vv); break;
                    default: f12_put_shifted<3>(xrow, vv); break;
                }
                f12_epi_bar();
                float acc[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    float t = 0.f;
#pragma unroll
                    for (int gg = 0; gg < 4; ++gg) t += sX[(gg * 32 + c8 * 8 + e) * kFXStride + jl];
                    acc[e] = data ? fmaxf(t + bias8[e], 0.f) : 0.f;
                }
                if (store) {
                    const size_t pos = (size_t)(r + kPad) * g.P + w.c0 + cv + kPad;
                    *reinterpret_cast<uint4*>(a2 + (((size_t)w.b * 4 + c8) * g.aplane + pos) * 8) = f12_pack8(acc);
                }
                f12_epi_bar();
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&ss->acc_empty[buf]));
        }
    } else if (warp == 6) {
        // ------------------------------------------------ weight streams
        if (lane == 0 && tlo_all < thi_all) {
            mbar_arrive_expect_tx(smem_u32(&ss->w1bar), kFW1Bytes);
            bulk_g2s(smem_u32(sW1), w1p, kFW1Bytes, smem_u32(&ss->w1bar));
            int wpar[2] = {-1, -1};
            int ws = 0;
            bool ok = true;
            for (int tile = tlo_all; tile < thi_all && ok; ++tile) {
                for (int j = 0; j < 33; ++j, ++ws) {
                    const int slot = ws & 1, use = ws >> 1;
                    if (!mbar_wait(smem_u32(&ss->wempty[slot]), (use & 1) ^ 1, status, abort_flag)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(smem_u32(&ss->wfull[slot]), kFWBlock);
                    wpar[slot] = use & 1;
                    bulk_g2s(smem_u32(sW2 + slot * kFWBlock), reinterpret_cast<const uint8_t*>(w2p) + (size_t)j * kFWBlock,
                             kFWBlock, smem_u32(&ss->wfull[slot]));
                }
            }
            mbar_wait_drain(smem_u32(&ss->w1bar), 0);
            for (int s = 0; s < 2; ++s)
                if (wpar[s] >= 0) mbar_wait_drain(smem_u32(&ss->wfull[s]), wpar[s]);
        }
    } else {
        // ------------------------------------------------ conv1 epilogue (warps 7..10)
        const int quarter = warp & 3;
        const int m = quarter * 32 + lane;                    // position in the block = TMEM lane
        int n = 0;
        bool ok = true;
        for (int tile = tlo_all; tile < thi_all && ok;) {
            const int v = tile / g.t2, tlo = tile - v * g.t2, thi = min(g.t2, tlo + (thi_all - tile));
            tile += thi - tlo;
            const Walked w = walked(g, xt, v);
            int k0, k1;
            run_blocks(tlo, thi, PV, k0, k1);
            for (int k = k0; k <= k1; ++k, ++n) {
                ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&ss->c1_full), n & 1, status, abort_flag));
                if (!ok) break;
                tc_fence_after();
                float vv[64];
                tmem_ld32(tbase + ((uint32_t)(quarter * 32) << 16) + kFC1Col, vv);
                tmem_ld32(tbase + ((uint32_t)(quarter * 32) << 16) + kFC1Col + 32, vv + 32);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&ss->c1_empty));
                const int p = 128 * k + m;
                const int R = p / PV, C = p - R * PV;
                const int row = R - kPad, col = C + w.acol;
                const bool data = row >= 0 && row < g.H && col >= 0 && col < g.W && C < w.ca;
                uint4 u[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    float o[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) o[e] = data ? fmaxf(vv[8 * c + e] + ss->bias1[8 * c + e], 0.f) : 0.f;
                    u[c] = f12_pack8(o);
                }
                const int slot = n % kFBlocks;
                ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&ss->slot_free[slot]), ((n / kFBlocks) & 1) ^ 1,
                                                       status, abort_flag));
                if (!ok) break;
                const int rr = slot * 128 + m;
#pragma unroll
                for (int c = 0; c < 8; ++c) *reinterpret_cast<uint4*>(sRing + c * kFChunk + (kFPre + rr) * 16) = u[c];
                if (rr >= kFRing - kFPre) {
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        *reinterpret_cast<uint4*>(sRing + c * kFChunk + (kFPre + rr - kFRing) * 16) = u[c];
                }
                fence_proxy_async();
                mbar_arrive(smem_u32(&ss->a1_full[slot]));
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tbase, 512);
    }
}

// x~ strip planes: plane v = (image b, strip s), position (R, C) = pixel
// (R - 5, s SW + C - 10) of x~, zero outside the image.
__global__ void gather_strips_kernel(const bf16* __restrict__ xt, int V, FusedGeo g, int plane, bf16* __restrict__ xs)
{
    const long long total = (long long)V * g.xplane;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int v = (int)(i / g.xplane), e = (int)(i - (long long)v * g.xplane);
        const int b = v / g.nstrip, s = v - b * g.nstrip;
        const int R = e / g.PV, C = e - R * g.PV;
        const int r = R - kPad, c = s * g.SW + C - 10;
        bf16 val = __float2bfloat16(0.f);
        if (r >= 0 && r < g.H && c >= 0 && c < g.W) val = xt[(size_t)b * plane + (size_t)(r + kPad) * g.P + c + kPad];
        xs[i] = val;
    }
}

FusedGeo fused_geo(const Geo& g)
{
    FusedGeo f;
    f.H = g.H;
    f.W = g.W;
    f.P = g.P;
    f.aplane = g.plane;
    if (g.P <= kFMaxPitch) {
        f.PV = g.P;
        f.nstrip = 1;
        f.SW = g.W;
        f.strips = 0;
        f.xplane = g.plane;
    } else {
        f.nstrip = cdiv(g.W, kFMaxStrip);
        f.SW = cdiv(g.W, f.nstrip);
        f.PV = f.SW + 20;
        f.strips = 1;
        f.xplane = (int)align_up((size_t)(g.H + 2 * kPad) * f.PV, 8);
    }
    f.HV = g.H * f.PV;
    f.t2 = cdiv(f.HV, kFValid);
    return f;
}

}  // namespace

size_t conv12_scratch_bytes(int B, const Geo& g)
{
    const FusedGeo f = fused_geo(g);
    return f.strips ? (size_t)B * f.nstrip * f.xplane * sizeof(bf16) : 0;
}

int conv12_tc(const bf16* xt, int B, const Geo& g, const bf16* w1p, const float* b1, const bf16* w2p,
              const float* b2, bf16* a2, bf16* xs, int num_sms, int* status, cudaStream_t st)
{
    if (B <= 0) return DEEPINV_OK;
    const FusedGeo f = fused_geo(g);
    const int V = B * f.nstrip;
    const bf16* src = xt;
    if (f.strips) {
        DI_REQUIRE(xs, "fused conv1/conv2: strip planes need scratch");
        const long long total = (long long)V * f.xplane;
        const int blocks = (int)std::min<long long>((total + 255) / 256, 16LL * num_sms);
        gather_strips_kernel<<<blocks, 256, 0, st>>>(xt, V, f, g.plane, xs);
        DI_LAUNCH_CHECK();
        src = xs;
    }
    DI_CUDA(cudaFuncSetAttribute(conv12_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFSmem));
    const long long ntiles = (long long)V * f.t2;
    DI_REQUIRE(ntiles < INT_MAX, "fused conv1/conv2: too many tiles");
    const int grid = (int)std::min<long long>(ntiles, num_sms);
    conv12_kernel<<<grid, kFThreads, kFSmem, st>>>(src, V, f, w1p, b1, w2p, b2, a2, status);
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

}  // namespace di
