// The measurement y = Phi x (Sec. 1) as one GEMM fed straight from the caller's
// float32 signals: Y [B][M] = X [B][N] Phi^T.
//
// X arrives by TMA (a 2-D tensor map over the float32 rows, boxes of 128 rows x
// 32 values, 128-byte swizzle) into a staging ring; the four warps that later
// run the epilogue round each box to bfloat16 (nearest even) into the K-major
// core-matrix layout the tensor core reads, so no separate packing pass writes
// and re-reads x.  Phi (packed once when the network is created) arrives by
// bulk copy.
//
// There are few output tiles (B / 128 x M / NB: 16 at 64 x 64, batch 1024)
// and a long K (the N = 4096 pixels), so K is split over the CTAs of a
// thread-block cluster along z.  Each CTA leaves its 128 x NB float32 partial in
// its own shared memory; after a cluster handshake every CTA sums one slice of
// the tile over the cluster's partials through distributed shared memory, in
// the fixed order of the cluster ranks, so the result is deterministic and no
// partial sums travel through global memory.
//
// Warp roles (192 threads): warp 0 lane 0 bulk-copies Phi; warp 1 owns TMEM and
// one of its threads issues the MMAs; warps 2..5 convert the staged float32
// boxes (one of their threads keeps kFiRawNS stages of x loads in flight), then
// drain the accumulator.  Every wait is bounded.
#include <mutex>

#include "kernels.cuh"
#include "tc.cuh"
#include "tma.cuh"

namespace di {
namespace {

using namespace tc;

constexpr int kFiKS = 4;       // MMA steps (K = 16 each) per stage: two 32-column boxes of x
constexpr int kFiRawNS = 4;    // stages of staged float32 x in flight (the HBM stream)
constexpr int kFiNS = 2;       // stages of bf16 A and of Phi
constexpr int kFiMaxCluster = 8;
constexpr uint32_t kFiBox = 128 * 128;            // one box: 128 rows x 32 float32
constexpr uint32_t kFiRaw = 2 * kFiBox;           // staged float32 of one stage
constexpr uint32_t kFiA = kFiKS * 4096;           // bf16 A of one stage

struct FiSmem {
    uint64_t raw_full[kFiRawNS], full[kFiNS], empty[kFiNS];
    uint64_t acc_full, drain, ready, done;
    uint32_t tmem_base;
    int abort_flag;
};

// ---------------------------------------------------------------- cluster helpers
__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Address in the cluster window of CTA `rank`'s copy of the local shared address `a`.
__device__ __forceinline__ uint32_t mapa(uint32_t a, uint32_t rank)
{
    uint32_t d;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(rank));
    return d;
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t remote_bar)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote_bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait (acquire at cluster scope) for a barrier that peers arrive on.
// With `honour_abort`, a CTA that has already given up stops waiting at once.
__device__ __forceinline__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity, int* status, volatile int* abort_flag,
                                                  bool honour_abort)
{
    const unsigned long long t0 = globaltimer();
    while (!mbar_try_wait_cluster(bar, parity)) {
        if (honour_abort && *abort_flag) return false;
        if (globaltimer() - t0 > kWaitLimitNs) {
            atomicExch(status, DEV_TIMEOUT);
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ float4 ld_cluster_f4(uint32_t addr)
{
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}

// Every thread of every CTA of the cluster: the cluster's barriers are
// initialised before any peer arrives on them.
__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// ---------------------------------------------------------------- conversion
// One stage: the two staged boxes (rows 0..127, columns 32 b .. 32 b + 31 at
// b * kFiBox + r * 128, 16-byte chunk j stored at chunk j ^ (r % 8) by the
// 128-byte swizzle) -> bfloat16 A in the layout [step][8-row group][K chunk]
// [8 rows][16 B]: chunk c of row r at (c / 2) 4096 + (r / 8) 256 + (c % 2) 128 +
// (r % 8) 16, so that the descriptor of step j starts at j 4096 with LBO = 128
// (next K chunk) and SBO = 256 (next 8 rows).  A warp handles 8 rows x 4 chunks
// at a time; each 8-lane phase touches 8 different rows, one 16-byte bank group
// each, on both the staged reads and the stores.
__device__ __forceinline__ void convert_stage(uint8_t* dst, const uint8_t* raw, int ks, int t)
{
    const int l = t & 31, w = t >> 5;
    const int nchunks = 2 * ks;
    const int nit = 16 * ((nchunks + 3) / 4);           // 16 row groups x chunk quads
#pragma unroll 2
    for (int it = w; it < nit; it += 4) {
        const int g = it & 15, c = (it >> 4) * 4 + (l >> 3), r = g * 8 + (l & 7);
        if (c < nchunks) {
            const uint8_t* row = raw + (c >> 2) * kFiBox + r * 128;
            const int j = 2 * (c & 3), sw = r & 7;
            const float4 a = *reinterpret_cast<const float4*>(row + ((j ^ sw) << 4));
            const float4 b = *reinterpret_cast<const float4*>(row + (((j + 1) ^ sw) << 4));
            __nv_bfloat162 p0 = __floats2bfloat162_rn(a.x, a.y), p1 = __floats2bfloat162_rn(a.z, a.w);
            __nv_bfloat162 p2 = __floats2bfloat162_rn(b.x, b.y), p3 = __floats2bfloat162_rn(b.z, b.w);
            uint4 o;
            o.x = *reinterpret_cast<uint32_t*>(&p0);
            o.y = *reinterpret_cast<uint32_t*>(&p1);
            o.z = *reinterpret_cast<uint32_t*>(&p2);
            o.w = *reinterpret_cast<uint32_t*>(&p3);
            *reinterpret_cast<uint4*>(dst + (c >> 1) * 4096 + g * 256 + (c & 1) * 128 + (r & 7) * 16) = o;
        }
    }
}

// Named barrier of the 128 converter / epilogue threads.
__device__ __forceinline__ void epi_bar_fi() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// The same barrier, returning the OR of `v` over the 128 threads (the same
// value in every thread, so that they leave a loop together).
__device__ __forceinline__ bool epi_bar_or(bool v)
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

// Issue the TMA loads of x for stage st (columns of MMA steps k0 .. k0 + ks)
// into staging slot st % kFiRawNS.
__device__ __forceinline__ void fi_load_x(const CUtensorMap* tmx, uint8_t* sRaw, FiSmem* ss, int st, int s0, int s1,
                                          int row0)
{
    const int slot = st % kFiRawNS;
    const int k0 = s0 + st * kFiKS, ks = min(kFiKS, s1 - k0);
    const int nbox = (ks * 16 + 31) / 32;
    mbar_arrive_expect_tx(smem_u32(&ss->raw_full[slot]), (uint32_t)nbox * kFiBox);
    for (int b = 0; b < nbox; ++b)
        tma_load_2d(smem_u32(sRaw + slot * kFiRaw + b * kFiBox), tmx, k0 * 16 + 32 * b, row0,
                    smem_u32(&ss->raw_full[slot]));
}

__global__ void __launch_bounds__(192, 1) measure_f32in_kernel(const __grid_constant__ CUtensorMap tmx,
                                                               const bf16* __restrict__ Bpk, int Kp, int Mr, int Nc,
                                                               int NB, uint32_t tmem_cols, float* __restrict__ out,
                                                               long long ldo, int* status)
{
    extern __shared__ uint8_t smem_dyn[];
    // 1024-byte alignment for the swizzled TMA destinations
    uint8_t* smem = smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
    const uint32_t b_stage = (uint32_t)kFiKS * NB * 32;
    uint8_t* sRaw = smem;                                  // [kFiRawNS][2 boxes]
    uint8_t* sA = sRaw + kFiRawNS * kFiRaw;                // [kFiNS][kFiA]
    uint8_t* sB = sA + kFiNS * kFiA;                       // [kFiNS][b_stage]
    FiSmem* ss = reinterpret_cast<FiSmem*>(sB + kFiNS * b_stage);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int mt = blockIdx.x, nt = blockIdx.y;
    const int ksplit = gridDim.z, z = blockIdx.z;
    const int nsteps_all = Kp / 16;
    const int s0 = nsteps_all * z / ksplit, s1 = nsteps_all * (z + 1) / ksplit;
    const int nstages = (s1 - s0 + kFiKS - 1) / kFiKS;
    const bool cluster = ksplit > 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kFiRawNS; ++s) mbar_init(smem_u32(&ss->raw_full[s]), 1);
        for (int s = 0; s < kFiNS; ++s) {
            mbar_init(smem_u32(&ss->full[s]), 1 + 4);      // Phi bytes + 4 converter warps
            mbar_init(smem_u32(&ss->empty[s]), 1);
        }
        mbar_init(smem_u32(&ss->acc_full), 1);
        mbar_init(smem_u32(&ss->drain), 1);
        mbar_init(smem_u32(&ss->ready), ksplit);
        mbar_init(smem_u32(&ss->done), ksplit);
        ss->abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(&ss->tmem_base), tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    if (cluster) cluster_sync_all();
    tc_fence_after();
    const uint32_t tbase = ss->tmem_base;

    if (warp == 0 && lane == 0) {
        // ------------------------------------------------ producer of Phi (bulk copies)
        int armed[kFiNS];
        for (int s = 0; s < kFiNS; ++s) armed[s] = -1;
        for (int st = 0; st < nstages; ++st) {
            const int slot = st % kFiNS, n = st / kFiNS;
            const int k0 = s0 + st * kFiKS, ks = min(kFiKS, s1 - k0);
            if (!mbar_wait(smem_u32(&ss->empty[slot]), (n & 1) ^ 1, status, &ss->abort_flag)) break;
            const uint32_t bytes = (uint32_t)ks * NB * 32;
            mbar_arrive_expect_tx(smem_u32(&ss->full[slot]), bytes);
            armed[slot] = n & 1;
            bulk_g2s(smem_u32(sB + slot * b_stage), Bpk + (size_t)nt * (Kp / 8) * NB * 8 + (size_t)k0 * 2 * NB * 8,
                     bytes, smem_u32(&ss->full[slot]));
        }
        for (int s = 0; s < kFiNS; ++s)
            if (armed[s] >= 0) mbar_wait_drain(smem_u32(&ss->full[s]), armed[s]);
    } else if (warp == 1 && lane == 0) {
        // ------------------------------------------------ MMA issuer
        const uint32_t idesc = idesc_bf16(128, NB);
        for (int st = 0; st < nstages; ++st) {
            const int slot = st % kFiNS, n = st / kFiNS;
            if (!mbar_wait(smem_u32(&ss->full[slot]), n & 1, status, &ss->abort_flag)) break;
            tc_fence_after();
            const int k0 = s0 + st * kFiKS, ks = min(kFiKS, s1 - k0);
            for (int j = 0; j < ks; ++j) {
                // converted A: LBO 128, SBO 256; packed Phi: LBO = NB x 16, SBO 128
                const uint64_t ad = sdesc(smem_u32(sA + slot * kFiA + j * 4096), 128, 256);
                const uint64_t bd = sdesc(smem_u32(sB + slot * b_stage + j * NB * 32), NB * 16, 128);
                mma_bf16(tbase, ad, bd, idesc, (k0 + j) > s0 ? 1u : 0u);
            }
            mma_commit(smem_u32(&ss->empty[slot]));
        }
        mma_commit(smem_u32(&ss->acc_full));
        mma_commit(smem_u32(&ss->drain));
        mbar_wait_drain(smem_u32(&ss->drain), 0);
    } else if (warp >= 2) {
        // ------------------------------------------------ converters (thread 64 also streams x)
        const int t = threadIdx.x - 64;                     // 0..127
        int issued = min(kFiRawNS, nstages);                // x stages whose loads are out
        if (t == 0)
            for (int st = 0; st < issued; ++st) fi_load_x(&tmx, sRaw, ss, st, s0, s1, mt * 128);
        bool ok = true;
        int st = 0;
        for (; st < nstages && ok; ++st) {
            const int slot = st % kFiNS, n = st / kFiNS;
            if (lane == 0)
                ok = mbar_wait(smem_u32(&ss->raw_full[st % kFiRawNS]), (st / kFiRawNS) & 1, status, &ss->abort_flag) &&
                     mbar_wait(smem_u32(&ss->empty[slot]), (n & 1) ^ 1, status, &ss->abort_flag);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            const int k0 = s0 + st * kFiKS, ks = min(kFiKS, s1 - k0);
            if (ok) {
                convert_stage(sA + slot * kFiA, sRaw + (st % kFiRawNS) * kFiRaw, ks, t);
                fence_proxy_async();          // generic-proxy stores -> tensor-core reads
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&ss->full[slot]));
            }
            // every converter warp is done with this staging slot: refill it (all 128
            // threads leave together if any of them, or another role, gave up)
            ok = !epi_bar_or(!ok || ss->abort_flag != 0);
            if (t == 0 && ok && issued < nstages) fi_load_x(&tmx, sRaw, ss, issued++, s0, s1, mt * 128);
        }
        // loads still in flight after an abort land before the CTA leaves
        if (t == 0)
            for (int k = st; k < issued; ++k) mbar_wait_drain(smem_u32(&ss->raw_full[k % kFiRawNS]), (k / kFiRawNS) & 1);
        // ------------------------------------------------ epilogue
        const int q = warp % 4;
        ok = ok && mbar_wait(smem_u32(&ss->acc_full), 0, status, &ss->abort_flag);
        ok = __all_sync(0xffffffffu, ok);
        tc_fence_after();
        const int m_row = q * 32 + lane;                    // TMEM lane = tile row
        if (!cluster) {
            const int m = mt * 128 + m_row;
            for (int c0 = 0; c0 < NB && ok; c0 += 16) {
                float v[16];
                tmem_ld16(tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
                if (m >= Mr) continue;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int nn = nt * NB + c0 + i;
                    if (nn >= Nc) break;
                    out[(long long)m * ldo + nn] = v[i];
                }
            }
        } else {
            // partial of this CTA -> its shared memory, over the staging and A rings (both
            // free: every MMA has completed and every copy has landed), row stride RS floats
            const int RS = NB + 4;
            float* part = reinterpret_cast<float*>(smem);
            if (ok) {
                for (int c0 = 0; c0 < NB; c0 += 16) {
                    float v[16];
                    tmem_ld16(tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
                    float4* d = reinterpret_cast<float4*>(part + (size_t)m_row * RS + c0);
#pragma unroll
                    for (int i = 0; i < 4; ++i) d[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                }
            }
            // handshake 1: this CTA's partial is in place (every peer is told, itself included)
            epi_bar_fi();
            const uint32_t rank = cluster_rank();
            if (threadIdx.x == 64)
                for (int p = 0; p < ksplit; ++p) mbar_arrive_cluster(mapa(smem_u32(&ss->ready), (uint32_t)p));
            const bool peers = mbar_wait_cluster(smem_u32(&ss->ready), 0, status, &ss->abort_flag, true);
            if (peers) {
                // slice `rank` of the tile's elements, in float4 groups, summed over the
                // cluster's partials in rank order
                const int groups = 128 * (NB / 4);
                const int g0 = (int)((long long)groups * rank / ksplit), g1 = (int)((long long)groups * (rank + 1) / ksplit);
                uint32_t pb[kFiMaxCluster];
#pragma unroll
                for (int p = 0; p < kFiMaxCluster; ++p) pb[p] = mapa(smem_u32(part), (uint32_t)(p < ksplit ? p : 0));
                for (int gi = g0 + t; gi < g1; gi += 128) {
                    const int r = gi / (NB / 4), c = (gi % (NB / 4)) * 4;
                    const uint32_t off = (uint32_t)((r * RS + c) * 4);
                    float4 s = ld_cluster_f4(pb[0] + off);
#pragma unroll
                    for (int p = 1; p < kFiMaxCluster; ++p) {
                        if (p < ksplit) {
                            const float4 v = ld_cluster_f4(pb[p] + off);
                            s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
                        }
                    }
                    const int m = mt * 128 + r, nn = nt * NB + c;
                    if (m < Mr) {
                        float* o = out + (long long)m * ldo + nn;
                        if (nn < Nc) o[0] = s.x;
                        if (nn + 1 < Nc) o[1] = s.y;
                        if (nn + 2 < Nc) o[2] = s.z;
                        if (nn + 3 < Nc) o[3] = s.w;
                    }
                }
            }
            // handshake 2: no CTA leaves while a peer may still read its partial
            epi_bar_fi();
            if (threadIdx.x == 64)
                for (int p = 0; p < ksplit; ++p) mbar_arrive_cluster(mapa(smem_u32(&ss->done), (uint32_t)p));
            // (waits out its time limit even after an abort: a peer may still be reading)
            mbar_wait_cluster(smem_u32(&ss->done), 0, status, &ss->abort_flag, false);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tbase, tmem_cols);
    }
}

size_t fi_smem(int NB)
{
    return 1024 + (size_t)kFiRawNS * kFiRaw + (size_t)kFiNS * (kFiA + (size_t)kFiKS * NB * 32) + sizeof(FiSmem);
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    });
    return fn;
}

// ================================================================ launcher
bool measure_f32in_supported(const float* X, long long ldx, int NB)
{
    return tensor_map_encoder() != nullptr && (reinterpret_cast<uintptr_t>(X) & 15) == 0 && (ldx * 4) % 16 == 0 &&
           NB >= 16 && NB <= 256 && NB % 16 == 0 && fi_smem(NB) <= 227 * 1024;
}

int gemm_measure_f32in(const float* X, long long ldx, int K, const bf16* Bpk, int Kp, int Mr, int Nc, int NB,
                       float* out, long long ldo, int num_sms, int* status, cudaStream_t st)
{
    if (Mr <= 0 || Nc <= 0) return DEEPINV_OK;
    if (!measure_f32in_supported(X, ldx, NB) || Kp % 16 || Kp <= 0 || K > Kp || K < 1) {
        set_error("gemm_measure_f32in: unsupported operands (N tile %d, K %d / %d, row stride %lld)", NB, K, Kp, ldx);
        return DEEPINV_EUNSUPPORTED;
    }
    // the x tensor map: columns (K) innermost, then rows; boxes of 32 x 128, zero
    // fill past the last row and column
    CUtensorMap tm;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)Mr};
    const cuuint64_t strides[1] = {(cuuint64_t)ldx * 4};
    const cuuint32_t box[2] = {32, 128};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult cr = tensor_map_encoder()(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(X), dims, strides, box,
                                       estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) {
        set_error("gemm_measure_f32in: cuTensorMapEncodeTiled failed (%d)", (int)cr);
        return DEEPINV_ECUDA;
    }
    const size_t smem = fi_smem(NB);
    // the reduction reuses the staging and A rings (contiguous) for the
    // 128 x (NB + 4) float32 partial
    if ((size_t)128 * (NB + 4) * 4 > (size_t)kFiRawNS * kFiRaw + (size_t)kFiNS * kFiA) {
        set_error("gemm_measure_f32in: partial does not fit");
        return DEEPINV_EINVAL;
    }
    uint32_t cols = 32;
    while (cols < (uint32_t)NB) cols <<= 1;
    DI_CUDA(cudaFuncSetAttribute(measure_f32in_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(192, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // split K over a cluster of up to 8 CTAs, at least 4 MMA steps each: the
    // largest split whose clusters all fit on the GPU at once (one wave)
    const int tiles = cdiv(Mr, 128) * cdiv(Nc, NB);
    int ks = num_sms / (tiles > 0 ? tiles : 1);
    if (ks > kFiMaxCluster) ks = kFiMaxCluster;
    if (ks > Kp / 16 / 4) ks = Kp / 16 / 4;
    for (; ks > 1; --ks) {
        cfg.gridDim = dim3(cdiv(Mr, 128), cdiv(Nc, NB), ks);
        attr[0].val.clusterDim.z = (unsigned)ks;
        int active = 0;
        if (cudaOccupancyMaxActiveClusters(&active, measure_f32in_kernel, &cfg) != cudaSuccess) {
            cudaGetLastError();
            active = 0;
        }
        if (active >= tiles) break;
    }
    if (ks < 1) ks = 1;
    cfg.gridDim = dim3(cdiv(Mr, 128), cdiv(Nc, NB), ks);
    attr[0].val.clusterDim.z = (unsigned)ks;
    DI_CUDA(cudaLaunchKernelEx(&cfg, measure_f32in_kernel, tm, Bpk, Kp, Mr, Nc, NB, cols, out, ldo, status));
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

}  // namespace di
