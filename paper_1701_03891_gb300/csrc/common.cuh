// Shared host/device helpers of libdeepinv: status reporting, checks, and the
// padded-plane geometry that the bfloat16 tensor-core path lays images out in.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include "deepinv.h"

namespace di {

// Thread-local message for deepinv_last_error().
void set_error(const char* fmt, ...);

// Per-device sticky status word that kernels with bounded waits write into.
int* device_status_word();

// Status word of deepinv_measure_noalloc's static scratch on `dev` (NULL
// until that entry point has run on the device); deepinv_device_status reads
// and resets it beside the per-device word above.
int* noalloc_status_word(int dev);

// Device that owns `p` (device or managed memory), else -1.
int device_of(const void* p);

// Counts one kernel launch of the library (deepinv_launch_count).
void count_launch();

#define DI_REQUIRE(cond, ...)                 \
    do {                                      \
        if (!(cond)) {                        \
            ::di::set_error(__VA_ARGS__);     \
            return DEEPINV_EINVAL;            \
        }                                     \
    } while (0)

#define DI_CUDA(call)                                                               \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            ::di::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                            __FILE__, __LINE__);                                    \
            return DEEPINV_ECUDA;                                                   \
        }                                                                           \
    } while (0)

// After every kernel launch: checks the launch and counts it.
#define DI_LAUNCH_CHECK()                 \
    do {                                  \
        DI_CUDA(cudaGetLastError());      \
        ::di::count_launch();             \
    } while (0)

// Launch that lets the kernel start while the stream's previous kernel finishes
// (programmatic dependent launch); the kernel calls pdl_wait before it touches
// memory that kernel may still read or write.
template <typename... KArgs, typename... Args>
static inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                     Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

#define DI_TRY(expr)                  \
    do {                              \
        int rc_ = (expr);             \
        if (rc_ != DEEPINV_OK) return rc_; \
    } while (0)

// Device-side status codes written to the status word.
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1 };

// Time limit of one bounded wait inside a kernel, in nanoseconds.
constexpr unsigned long long kWaitLimitNs = 1000ull * 1000ull * 1000ull;  // 1 s

static inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
static inline int cdiv(int a, int b) { return (a + b - 1) / b; }

// Geometry of the padded image planes used by the bfloat16 path.
//
// An n1 x n2 image is stored with a row pitch P = n2 + 5: every row carries
// its n2 pixels followed by five zeros.  With a half-width of five (11 x 11
// kernels) those five zeros serve both as the right border of a row and the
// left border of the next one, so that every tap (dy, dx) of output position
// q = r * P + c reads input position q + dy * P + dx of the plane (the crop S
// of Eq. 1 is then the 'same' zero padding).  Pixel (r, c) lives at plane
// index q + 5 P + 5; the first 5 P + 5 entries and everything after the last
// row are zero.  Output positions with c >= n2 are computed and discarded.
struct Geo {
    int H, W, P;   // rows, columns, pitch
    int HP;        // H * P output positions per image
    int t1;        // conv1 tiles (128 positions) per image
    int t2;        // conv2 tiles (kConv2Valid positions) per image
    int t3;        // conv3 row-sum tiles (kConv3Valid positions) per image
    int tlen;      // row sums per image and kernel row (>= t3 * kConv3Valid)
    int nslab;     // conv2 window slabs of kSlabPx positions
    int plane;     // positions per image plane (multiple of 8)
};

constexpr int kPad = 5;            // (k - 1) / 2 for k = 11
constexpr int kConv2N = 256;       // MMA N of conv2 (positions per tile)
constexpr int kConv2Valid = 253;   // outputs a conv2 tile completes (256 - 3)
constexpr int kSlabPx = 128;       // conv2 window slab
constexpr int kConv2Reach = 10;    // rows of halo below an output row (k - 1)
constexpr int kConv3Valid = 125;   // row sums a conv3 tile completes (128 - 3)

static inline Geo make_geo(int H, int W)
{
    Geo g;
    g.H = H;
    g.W = W;
    g.P = W + kPad;
    g.HP = H * g.P;
    g.t1 = cdiv(g.HP, 128);
    g.t2 = cdiv(g.HP, kConv2Valid);
    // conv3 computes row partial sums T[p] for p in [0, (H + 10) P).
    g.t3 = cdiv((H + kConv2Reach) * g.P, kConv3Valid);
    g.tlen = (int)align_up((size_t)g.t3 * kConv3Valid, 32);
    const int win2 = kConv2Reach * g.P + 16 + kConv2N;   // positions one conv2 tile reads (shift <= 10)
    g.nslab = cdiv(win2, kSlabPx);
    size_t need = 0;
    auto upd = [&](size_t v) { if (v > need) need = v; };
    upd((size_t)(g.t2 - 1) * kConv2Valid + (size_t)g.nslab * kSlabPx);     // conv2 window
    upd((size_t)g.t1 * 128 + (size_t)kConv2Reach * g.P + 24);              // conv1 expanded window
    upd((size_t)g.t3 * kConv3Valid + 16);                                  // conv3 window (136 rows per tile)
    upd((size_t)(H + 2 * kPad) * g.P + 2 * kPad);                          // data + borders
    upd((size_t)g.HP + (size_t)kConv2Reach * g.P + 136);                    // conv2 weight-gradient / fused conv3 windows
    g.plane = (int)align_up(need, 8);
    return g;
}

}  // namespace di
