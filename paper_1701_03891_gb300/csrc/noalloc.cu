// deepinv_measure_noalloc: y = Phi x on the bfloat16 tensor cores without
// any device allocation.
//
// deepinv_measure(..., DEEPINV_BF16) repacks Phi and x into bfloat16 operand
// tiles in memory it takes from the stream-ordered allocator.  Some callers
// cannot let a library allocate: processes whose device memory is carved up
// once at start-up (a fixed budget per model or per sensor stream), real-time
// loops that must not hit the allocator after initialisation, and hosts that
// install their own allocator and forbid any other.  For them this file keeps
// the operand tiles in one static device array instead.
#include <mutex>

#include "kernels.cuh"

namespace di {
namespace {

// Scratch for the packed operands: a 256-byte header (word 0 is the status
// word of the bounded waits in the GEMM kernel, read and reset by
// deepinv_device_status) followed by the packed Phi and the packed x.  Every
// device that loads the library holds these 32 MiB until the process exits.
constexpr size_t kScratchBytes = 32u << 20;
constexpr size_t kHeaderBytes = 256;
static __device__ __align__(256) unsigned char g_measure_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_addr[kMaxDevices];   // device address per device, as last looked up

inline int up16(int x) { return (x + 15) / 16 * 16; }
inline int nb_for(int n)
{
    const int tiles = cdiv(n, 256);
    return up16(cdiv(n, tiles));
}

// Device address of the static array on `dev` (which must be current).  The
// address is looked up on every call; when it differs from the one recorded
// for the device (the first call, or a new context after a device reset), the
// header is cleared before the array is used.
int scratch_on(int dev, unsigned char** out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_measure_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        set_error("deepinv_measure_noalloc: cudaGetSymbolAddress failed on device %d: %s", dev,
                  cudaGetErrorString(e));
        return DEEPINV_ECUDA;
    }
    if (g_scratch_addr[dev] != p) {
        e = cudaMemset(p, 0, kHeaderBytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("deepinv_measure_noalloc: clearing the scratch header failed: %s", cudaGetErrorString(e));
            return DEEPINV_ECUDA;
        }
        g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_addr[dev];
    return DEEPINV_OK;
}

}  // namespace

int* noalloc_status_word(int dev)
{
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    return reinterpret_cast<int*>(g_scratch_addr[dev]);
}

}  // namespace di

using namespace di;

extern "C" int deepinv_measure_noalloc(const float* phi, int M, int N, const float* x, int B, float* y,
                                       void* stream)
{
    // (sizes up to 2^30, so that padded extents stay within int)
    DI_REQUIRE(M >= 1 && N >= 1 && B >= 0 && M <= (1 << 30) && N <= (1 << 30) && B <= (1 << 30),
               "bad sizes M=%d N=%d B=%d", M, N, B);
    DI_REQUIRE(B == 0 || (phi && x && y), "null pointer");
    if (B == 0) return DEEPINV_OK;
    const int Kp = up16(N), NB = nb_for(M);
    const size_t phi_bytes = align_up(packed_elems(M, NB, Kp) * sizeof(bf16), 256);
    const size_t x_bytes = packed_elems(B, 128, Kp) * sizeof(bf16);
    if (kHeaderBytes + phi_bytes + x_bytes > kScratchBytes) {
        set_error("deepinv_measure_noalloc: M=%d, N=%d, B=%d needs %zu bytes of packed operands, "
                  "more than the %zu-byte static scratch",
                  M, N, B, phi_bytes + x_bytes, kScratchBytes - kHeaderBytes);
        return DEEPINV_EINVAL;
    }
    const int dev = device_of(phi);
    DI_REQUIRE(dev >= 0, "deepinv_measure_noalloc: phi is not device or managed memory");
    DI_REQUIRE(dev < kMaxDevices, "device %d out of range", dev);
    int prev = -1;
    DI_CUDA(cudaGetDevice(&prev));
    if (prev != dev) DI_CUDA(cudaSetDevice(dev));
    unsigned char* base = nullptr;
    int rc = scratch_on(dev, &base);
    if (rc == DEEPINV_OK) {
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        int* status = reinterpret_cast<int*>(base);
        bf16* phiB = reinterpret_cast<bf16*>(base + kHeaderBytes);
        bf16* xpk = reinterpret_cast<bf16*>(base + kHeaderBytes + phi_bytes);
        // Both packs overwrite every element they cover (zero padding included),
        // so nothing left over from an earlier call is read.
        rc = pack_kmajor(phi, N, 1, M, N, NB, Kp, phiB, st);
        if (rc == DEEPINV_OK) rc = pack_kmajor(x, N, 1, B, N, 128, Kp, xpk, st);
        if (rc == DEEPINV_OK) {
            Geo none{};
            rc = tc_gemm(xpk, phiB, Kp, B, M, NB, GEMM_OUT_F32, y, M, nullptr, none, status, st);
        }
    }
    if (prev != dev) cudaSetDevice(prev);
    return rc;
}
