// C ABI of libdeepinv (declared in include/deepinv.h): argument checks,
// network objects (weights in float32 masters plus kernel layouts), workspace
// management and the dispatch of the forward, backward and update passes.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <atomic>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "kernels.cuh"

namespace di {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

static std::mutex g_status_mu;
static std::vector<int*> g_status_words;

int* device_status_word()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_status_mu);
    if ((int)g_status_words.size() <= dev) g_status_words.resize(dev + 1, nullptr);
    if (!g_status_words[dev]) {
        int* p = nullptr;
        if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
        if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return nullptr;
        g_status_words[dev] = p;
    }
    return g_status_words[dev];
}

int device_of(const void* p)
{
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged ? a.device : -1;
}

static std::atomic<unsigned long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static int num_sms_current()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

// Largest batch a call accepts (padded batch extents stay within int).
constexpr int kMaxBatch = 1 << 30;

// Round up to a multiple of 16 (the K granularity of one bf16 MMA).
static inline int up16(int x) { return (x + 15) / 16 * 16; }

// N tile of a GEMM whose N extent is n (16 .. 256, multiple of 16).
static inline int gemm_nb(int n)
{
    const int tiles = cdiv(n, 256);
    return up16(cdiv(n, tiles));
}

// Batch tile of the FC GEMM for batch B.
static inline int fc_nb(int B) { return B >= 256 ? 256 : up16(B > 0 ? B : 1); }

}  // namespace di

using namespace di;

struct deepinv_net {
    deepinv_net_desc d;
    int dev = 0;       // CUDA device the network lives on
    int N = 0;
    int num_sms = 1;
    Geo geo{};
    bool tc = false;   // tensor-core path (bf16, or e4m3 conv2)
    bool fp8 = false;  // conv2 in e4m3
    // float32 masters of the L = 3 + hidden conv layers, in network order
    // (conv1, conv2, hidden 1..hidden, conv3)
    static constexpr int kMaxLayers = 3 + DEEPINV_MAX_HIDDEN;
    int L = 3;
    float* phi = nullptr;
    float* w[kMaxLayers] = {};
    float* b[kMaxLayers] = {};
    float* wfc = nullptr;
    float* vw[kMaxLayers] = {};
    float* vb[kMaxLayers] = {};
    float* vfc = nullptr;
    // bf16 kernel layouts
    bf16* fcA = nullptr;    // FC: rows = pixel j, K = measurement i
    int Kfc = 0;
    bf16* msB = nullptr;    // measurement: rows = i, K = pixel j
    int Kms = 0, NBms = 0;
    bf16* w1p = nullptr;
    bf16* w2p = nullptr;
    bf16* w3p = nullptr;
    bf16* w2t = nullptr;        // conv2 input-gradient weights (flipped, transposed)
    bf16* w3t = nullptr;        // conv3 input-gradient weights
    bf16* w1t = nullptr;        // conv1 input-gradient weights
    bf16* whp = nullptr;        // hidden layers' operands, kWhPackElems each
    bf16* wht = nullptr;        // hidden layers' input-gradient operands (trainable networks)
    // e4m3 conv2: weights, per-filter scales, calibrated activation scale
    uint8_t* w2q = nullptr;
    float* sw = nullptr;        // [32] weight scales
    float* oscale = nullptr;    // [32] sw * sa
    float* inv_sa = nullptr;    // 1 / sa
    float* amax_a1 = nullptr;   // calibrated max of a1
    float* amax_w = nullptr;    // [32] scratch
    bool calibrated = false;
    bool fused12 = false;       // conv1 + conv2 as one kernel in inference passes
    int conv1_rows = 1;         // conv1 in row tiles: 0 never, 1 where faster, 2 where they fit
    // forward workspace
    char* ws = nullptr;
    size_t ws_bytes = 0;
    int ws_B = 0;
    // backward workspace
    char* bws = nullptr;
    size_t bws_bytes = 0;
    int bws_B = 0;
    // activation recomputation: budget for the activations of one chunk, the
    // chunk's saved-activation buffer and the gradient scratch of later chunks
    size_t act_budget = 0;
    char* rsaved = nullptr;
    size_t rsaved_bytes = 0;
    char* gacc = nullptr;
    size_t gacc_bytes = 0;
    // profiler: event pool and (stage, start event, end event) spans
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<int> spans;
    // host-memory entry points: two staging slots (input and x^), copy streams
    // and per-slot events, so that a batch's copies overlap its neighbours' compute
    cudaStream_t cs_in = nullptr, cs_out = nullptr;
    float* hin[2] = {nullptr, nullptr};
    float* hout[2] = {nullptr, nullptr};
    size_t hin_elems = 0, hout_elems = 0;
    cudaEvent_t ev_h2d[2] = {}, ev_read[2] = {}, ev_comp[2] = {}, ev_d2h[2] = {};
    uint64_t hnext = 0;    // ticket of the next submission
};

namespace {

// Makes `dev` current for this library's runtime for the duration of a call
// (the library's CUDA runtime state is separate from the caller's).
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (dev >= 0 && dev != prev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Record an event from the pool on `st`; returns its index or -1.
int prof_event(deepinv_net* n, cudaStream_t st)
{
    if (n->ev_used == n->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return -1; }
        n->ev_pool.push_back(e);
    }
    const int i = (int)n->ev_used++;
    if (cudaEventRecord(n->ev_pool[i], st) != cudaSuccess) { cudaGetLastError(); return -1; }
    return i;
}

// NVTX range for the duration of a host call (visible to profilers; nearly free otherwise).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

const char* stage_name(int stage)
{
    static const char* names[DEEPINV_NSTAGES] = {"deepinv measure", "deepinv fc", "deepinv conv1", "deepinv conv2",
                                                "deepinv conv3", "deepinv hidden"};
    return stage >= 0 && stage < DEEPINV_NSTAGES ? names[stage] : "deepinv";
}

// Marks a stage: an NVTX range, and with the profiler on, CUDA events whose span
// the destructor records.
struct StageTimer {
    deepinv_net* n;
    cudaStream_t st;
    int stage, e0;
    NvtxRange range;
    StageTimer(deepinv_net* n_, cudaStream_t st_, int stage_)
        : n(n_), st(st_), stage(stage_), e0(-1), range(stage_name(stage_))
    {
        if (n->prof) e0 = prof_event(n, st);
    }
    ~StageTimer()
    {
        if (!n->prof || e0 < 0) return;
        const int e1 = prof_event(n, st);
        if (e1 < 0) return;
        n->spans.push_back(stage);
        n->spans.push_back(e0);
        n->spans.push_back(e1);
    }
};

struct Arena {
    char* base;
    size_t off;
    template <typename T>
    T* take(size_t n)
    {
        off = align_up(off, 256);
        T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
        off += n * sizeof(T);
        return p;
    }
};

// Forward workspace carve-up for batch B (base == nullptr: size only).
struct FwdWs {
    bf16 *ypk, *xpk, *xt, *a1, *a2;
    bf16* h;                // hidden layers: second 32-channel plane (ping-pong with a2)
    float *T;
    float *fxt, *fa1, *fa2, *fh;
    float *yd, *xhd;        // y of the host-memory entry points; x^ staging (serving, recomputation)
    float* mpart;           // split-K partials of the measurement GEMM
    size_t bytes;
};

FwdWs carve_fwd(const deepinv_net* n, int B, char* base)
{
    Arena a{base, 0};
    FwdWs w{};
    const int N = n->N, M = n->d.M;
    if (n->tc) {
        const Geo& g = n->geo;
        w.ypk = a.take<bf16>((align_up((size_t)B, 256) + 256) * n->Kfc);
        w.xpk = a.take<bf16>(packed_elems(B, 128, n->Kms));
        // zero-bordered planes: everything from here to `T` is cleared at allocation
        w.xt = a.take<bf16>((size_t)B * g.plane);
        w.a1 = a.take<bf16>((size_t)B * 8 * g.plane * 8);
        w.a2 = a.take<bf16>((size_t)B * 4 * g.plane * 8);
        if (n->d.hidden > 0) w.h = a.take<bf16>((size_t)B * 4 * g.plane * 8);
        w.T = a.take<float>(conv3_scratch_elems(g, B, 32));
    } else {
        w.fxt = a.take<float>((size_t)B * N);
        w.fa1 = a.take<float>((size_t)B * n->d.l1 * N);
        w.fa2 = a.take<float>((size_t)B * n->d.l2 * N);
        if (n->d.hidden > 0) w.fh = a.take<float>((size_t)B * n->d.l2 * N);
    }
    if (n->tc) w.mpart = a.take<float>((size_t)16 * B * M);   // split-K partials of y = Phi x
    w.yd = a.take<float>((size_t)B * M);
    w.xhd = a.take<float>((size_t)B * N);
    w.bytes = align_up(a.off, 256);
    return w;
}

// Layout of the caller's `saved` buffer at batch B.
struct Saved {
    bf16 *xt, *a1, *a2;      // bf16 path planes
    bf16* h;                 // hidden layers' output planes, hstride elements apart
    float *fxt, *fa1, *fa2;  // float32 path NCHW
    float* fh;               // hidden layers' outputs (float32 path), hstride apart
    size_t hstride;
    float* xhat;
    size_t bytes;
    // Activation a_l (the input of layer l, 0-based): a_0 = x~, a_1 = conv1's
    // output, a_2 = conv2's, a_{2+j} = hidden layer j's (j = 1..hidden).
    bf16* plane(int l) const { return l == 0 ? xt : l == 1 ? a1 : l == 2 ? a2 : h + (size_t)(l - 3) * hstride; }
    float* f32(int l) const { return l == 0 ? fxt : l == 1 ? fa1 : l == 2 ? fa2 : fh + (size_t)(l - 3) * hstride; }
};

Saved carve_saved(const deepinv_net* n, int B, char* base)
{
    Arena a{base, 0};
    Saved s{};
    const int N = n->N;
    if (n->tc) {
        const Geo& g = n->geo;
        s.xt = a.take<bf16>((size_t)B * g.plane);
        s.a1 = a.take<bf16>((size_t)B * 8 * g.plane * 8);
        s.a2 = a.take<bf16>((size_t)B * 4 * g.plane * 8);
        s.hstride = (size_t)B * 4 * g.plane * 8;
        if (n->d.hidden > 0) s.h = a.take<bf16>(s.hstride * n->d.hidden);
    } else {
        s.fxt = a.take<float>((size_t)B * N);
        s.fa1 = a.take<float>((size_t)B * n->d.l1 * N);
        s.fa2 = a.take<float>((size_t)B * n->d.l2 * N);
        s.hstride = (size_t)B * n->d.l2 * N;
        if (n->d.hidden > 0) s.fh = a.take<float>(s.hstride * n->d.hidden);
    }
    s.xhat = a.take<float>((size_t)B * N);
    s.bytes = align_up(a.off, 256);
    return s;
}

// Zero what the forward kernels never write in a caller's saved buffer: the
// whole one-channel x~ plane (the FC layer writes its pixels only, not the pad
// columns) and, of every multi-channel plane, the positions before its first
// pixel row and after its last (conv1, conv2 and the hidden layers write every
// position in between, pad columns included).
int clear_saved_borders(const deepinv_net* n, const Saved& sv, int B, cudaStream_t st)
{
    const Geo& g = n->geo;
    const size_t head = (size_t)kPad * g.P + kPad, tail0 = (size_t)g.HP + head, tail = (size_t)g.plane - tail0;
    const size_t pitch = (size_t)g.plane * 16;
    DI_CUDA(cudaMemsetAsync(sv.xt, 0, (size_t)B * g.plane * sizeof(bf16), st));
    auto borders = [&](bf16* base, size_t nplanes) -> int {
        DI_CUDA(cudaMemset2DAsync(base, pitch, 0, head * 16, nplanes, st));
        DI_CUDA(cudaMemset2DAsync(reinterpret_cast<char*>(base) + tail0 * 16, pitch, 0, tail * 16, nplanes, st));
        return DEEPINV_OK;
    };
    DI_TRY(borders(sv.a1, (size_t)B * 8));
    DI_TRY(borders(sv.a2, (size_t)B * 4));
    if (n->d.hidden > 0) DI_TRY(borders(sv.h, (size_t)B * 4 * n->d.hidden));
    return DEEPINV_OK;
}

int ensure_ws(deepinv_net* n, int B, cudaStream_t st)
{
    if (B <= n->ws_B && n->ws) return DEEPINV_OK;
    const FwdWs need = carve_fwd(n, B, nullptr);
    DI_CUDA(cudaStreamSynchronize(st));
    if (n->ws) {
        DI_CUDA(cudaFree(n->ws));
        n->ws = nullptr;
        n->ws_B = 0;
        n->ws_bytes = 0;
    }
    char* p = nullptr;
    if (cudaMalloc(&p, need.bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("workspace of %zu bytes for batch %d: out of device memory", need.bytes, B);
        return DEEPINV_ENOMEM;
    }
    DI_CUDA(cudaMemset(p, 0, need.bytes));
    n->ws = p;
    n->ws_bytes = need.bytes;
    n->ws_B = B;
    return DEEPINV_OK;
}

int check_desc(const deepinv_net_desc* d)
{
    DI_REQUIRE(d, "desc is NULL");
    DI_REQUIRE(d->n1 >= 1 && d->n2 >= 1 && (long long)d->n1 * d->n2 <= (1 << 24),
               "bad image size %d x %d", d->n1, d->n2);
    DI_REQUIRE(d->M >= 1 && d->M <= d->n1 * d->n2, "bad M = %d for N = %d", d->M, d->n1 * d->n2);
    DI_REQUIRE(d->l1 >= 1 && d->l2 >= 1 && d->l3 == 1, "filters (%d, %d, %d): need l1, l2 >= 1, l3 = 1",
               d->l1, d->l2, d->l3);
    DI_REQUIRE(d->k >= 1 && d->k <= 15 && d->k % 2 == 1, "kernel size %d must be odd and <= 15", d->k);
    DI_REQUIRE(d->hidden >= 0 && d->hidden <= DEEPINV_MAX_HIDDEN, "hidden layers %d: need 0..%d", d->hidden,
               DEEPINV_MAX_HIDDEN);
    DI_REQUIRE(d->prec == DEEPINV_F32 || d->prec == DEEPINV_BF16 || d->prec == DEEPINV_FP8_E4M3,
               "unknown precision %d", d->prec);
    if (d->prec != DEEPINV_F32) {
        if (d->l1 != 64 || d->l2 != 32 || d->k != 11) {
            set_error("bf16 path is built for the paper network (64, 32, 1 filters of 11 x 11)");
            return DEEPINV_EUNSUPPORTED;
        }
        if (!conv2_tc_supported(make_geo(d->n1, d->n2))) {
            set_error("bf16 path: image width %d not supported yet", d->n2);
            return DEEPINV_EUNSUPPORTED;
        }
    }
    return DEEPINV_OK;
}

int repack(deepinv_net* n, cudaStream_t st)
{
    if (!n->tc) return DEEPINV_OK;
    const int N = n->N, M = n->d.M;
    const int last = n->L - 1;
    DI_TRY(pack_conv_weights(n->w[0], n->w[1], n->w[last], n->w1p, n->w2p, n->w3p, st));
    if (n->w2t) DI_TRY(pack_dgrad_weights(n->w[0], n->w[1], n->w[last], n->w1t, n->w2t, n->w3t, st));
    for (int j = 0; j < n->d.hidden; ++j)
        DI_TRY(pack_hidden_weights(n->w[2 + j], n->whp + (size_t)j * kWhPackElems,
                                   n->wht ? n->wht + (size_t)j * kWhPackElems : nullptr, st));
    if (n->fp8) {
        DI_TRY(pack_w2_e4m3(n->w[1], n->amax_w, n->w2q, n->sw, st));
        if (n->calibrated) DI_TRY(e4m3_scales(n->amax_a1, n->sw, n->inv_sa, n->oscale, st));
    }
    // FC operand (rows = pixel j, K = measurement i): Phi^T or the trained copy.
    if (n->wfc) DI_TRY(pack_kmajor(n->wfc, M, 1, N, M, 128, n->Kfc, n->fcA, st));
    else DI_TRY(pack_kmajor(n->phi, 1, N, N, M, 128, n->Kfc, n->fcA, st));
    return DEEPINV_OK;
}

void free_net(deepinv_net* n)
{
    if (!n) return;
    cudaFree(n->phi);
    for (int l = 0; l < deepinv_net::kMaxLayers; ++l) {
        cudaFree(n->w[l]);
        cudaFree(n->b[l]);
        cudaFree(n->vw[l]);
        cudaFree(n->vb[l]);
    }
    cudaFree(n->wfc);
    cudaFree(n->vfc);
    cudaFree(n->fcA);
    cudaFree(n->msB);
    cudaFree(n->w1p);
    cudaFree(n->w2p);
    cudaFree(n->w3p);
    cudaFree(n->w2q);
    cudaFree(n->sw);
    cudaFree(n->w2t);
    cudaFree(n->w3t);
    cudaFree(n->w1t);
    cudaFree(n->whp);
    cudaFree(n->wht);
    cudaFree(n->ws);
    cudaFree(n->bws);
    cudaFree(n->rsaved);
    cudaFree(n->gacc);
    for (cudaEvent_t e : n->ev_pool) cudaEventDestroy(e);
    for (int k = 0; k < 2; ++k) {
        cudaFree(n->hin[k]);
        cudaFree(n->hout[k]);
        for (cudaEvent_t e : {n->ev_h2d[k], n->ev_read[k], n->ev_comp[k], n->ev_d2h[k]})
            if (e) cudaEventDestroy(e);
    }
    if (n->cs_in) cudaStreamDestroy(n->cs_in);
    if (n->cs_out) cudaStreamDestroy(n->cs_out);
    delete n;
}

// Channels into and out of layer l (network order: conv1, conv2, hidden layers, conv3).
int layer_cin(const deepinv_net* n, int l) { return l == 0 ? 1 : (l == 1 ? n->d.l1 : n->d.l2); }
int layer_cout(const deepinv_net* n, int l) { return l == 0 ? n->d.l1 : (l == n->L - 1 ? n->d.l3 : n->d.l2); }

size_t wsize(const deepinv_net* n, int l)
{
    return (size_t)layer_cout(n, l) * layer_cin(n, l) * n->d.k * n->d.k;
}

size_t bsize(const deepinv_net* n, int l) { return (size_t)layer_cout(n, l); }

template <typename T>
int dev_alloc(T** p, size_t n)
{
    if (n == 0) n = 1;
    if (cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        set_error("device allocation of %zu bytes failed", n * sizeof(T));
        return DEEPINV_ENOMEM;
    }
    return DEEPINV_OK;
}

int measure_bf16_packed(const bf16* phiB, int Kp, int NB, const float* x, int N, int M, int B, float* y,
                        bf16* xpk, cudaStream_t st)
{
    int* status = device_status_word();
    DI_REQUIRE(status, "no device status word");
    DI_TRY(pack_kmajor(x, N, 1, B, N, 128, Kp, xpk, st));
    Geo dummy{};
    return tc_gemm(xpk, phiB, Kp, B, M, NB, GEMM_OUT_F32, y, M, nullptr, dummy, status, st);
}

// The forward pass in a given workspace `w` (carved for at least B images).
int forward_core(deepinv_net* n, const FwdWs& w, const float* y, int B, float* xhat, void* saved, cudaStream_t st)
{
    if (n->fp8 && !n->calibrated) {
        set_error("e4m3 network: call deepinv_net_calibrate before the first forward pass");
        return DEEPINV_EINVAL;
    }
    if (n->fp8 && saved) {
        set_error("e4m3 networks are inference only (train in bf16 or f32)");
        return DEEPINV_EUNSUPPORTED;
    }
    const int N = n->N, M = n->d.M, H = n->d.n1, W = n->d.n2, k = n->d.k;
    Saved sv{};
    if (saved) {
        sv = carve_saved(n, B, static_cast<char*>(saved));
        if (n->tc) DI_TRY(clear_saved_borders(n, sv, B, st));   // float32 arrays are written in full
    }
    if (n->tc) {
        const Geo& g = n->geo;
        int* status = device_status_word();
        DI_REQUIRE(status, "no device status word");
        bf16* xt = saved ? sv.xt : w.xt;
        bf16* a1 = saved ? sv.a1 : w.a1;
        bf16* a2 = saved ? sv.a2 : w.a2;
        const int nb = fc_nb(B);
        {
            StageTimer t(n, st, DEEPINV_STAGE_FC);
            DI_TRY(pack_kmajor(y, M, 1, B, M, nb, n->Kfc, w.ypk, st));
            DI_TRY(tc_gemm(n->fcA, w.ypk, n->Kfc, N, B, nb, GEMM_OUT_PLANE, nullptr, 0, xt, g, status, st));
        }
        if (n->fused12 && !saved && !n->fp8) {
            // a1 never leaves the kernel; its workspace holds the x~ strip planes of wide images
            StageTimer t(n, st, DEEPINV_STAGE_CONV2);
            DI_REQUIRE(conv12_scratch_bytes(B, g) <= (size_t)B * 8 * g.plane * 8 * sizeof(bf16),
                       "fused conv1/conv2: strip planes exceed the a1 workspace");
            DI_TRY(conv12_tc(xt, B, g, n->w1p, n->b[0], n->w2p, n->b[1], a2, a1, n->num_sms, status, st));
        } else {
            {
                StageTimer t(n, st, DEEPINV_STAGE_CONV1);
                const int mode = n->fp8 ? kConv1OutE4M3 : kConv1OutBF16;
                const int fit = conv1_rows_fit(g);
                if ((n->conv1_rows == 1 && fit == 2) || (n->conv1_rows == 2 && fit >= 1))
                    DI_TRY(conv1_rows_tc(xt, B, g, n->w1p, n->b[0], a1, mode, n->inv_sa, status, st));
                else
                    DI_TRY(conv1_tc(xt, B, g, n->w1p, n->b[0], a1, mode, n->inv_sa, nullptr, status, st));
            }
            {
                StageTimer t(n, st, DEEPINV_STAGE_CONV2);
                if (n->fp8) DI_TRY(conv2_tc(a1, B, g, n->w2q, n->b[1], n->oscale, true, a2, n->num_sms, status, st));
                else DI_TRY(conv2_tc(a1, B, g, n->w2p, n->b[1], nullptr, false, a2, n->num_sms, status, st));
            }
        }
        bf16* last = a2;
        if (n->d.hidden > 0) {
            // hidden layers: into the saved planes, or alternating between the
            // workspace's two 32-channel planes
            StageTimer t(n, st, DEEPINV_STAGE_HIDDEN);
            for (int j = 0; j < n->d.hidden; ++j) {
                bf16* out = saved ? sv.plane(3 + j) : (j % 2 == 0 ? w.h : w.a2);
                DI_TRY(hidden_tc(last, B, g, n->whp + (size_t)j * kWhPackElems, n->b[2 + j], out, n->num_sms,
                                 status, st));
                last = out;
            }
        }
        {
            StageTimer t(n, st, DEEPINV_STAGE_CONV3);
            DI_TRY(conv3_tc(last, B, g, n->w3p, n->b[n->L - 1], w.T, xhat, n->d.final_relu, status, st));
        }
    } else {
        float* xt = saved ? sv.fxt : w.fxt;
        float* a1 = saved ? sv.fa1 : w.fa1;
        float* a2 = saved ? sv.fa2 : w.fa2;
        {
            StageTimer t(n, st, DEEPINV_STAGE_FC);
            if (n->wfc) DI_TRY(sgemm(B, N, M, y, M, 1, n->wfc, 1, M, xt, N, st));
            else DI_TRY(sgemm(B, N, M, y, M, 1, n->phi, N, 1, xt, N, st));
        }
        {
            StageTimer t(n, st, DEEPINV_STAGE_CONV1);
            DI_TRY(conv_f32(xt, B, 1, H, W, n->w[0], n->b[0], n->d.l1, k, a1, 1, st));
        }
        {
            StageTimer t(n, st, DEEPINV_STAGE_CONV2);
            DI_TRY(conv_f32(a1, B, n->d.l1, H, W, n->w[1], n->b[1], n->d.l2, k, a2, 1, st));
        }
        float* last = a2;
        if (n->d.hidden > 0) {
            StageTimer t(n, st, DEEPINV_STAGE_HIDDEN);
            for (int j = 0; j < n->d.hidden; ++j) {
                float* out = saved ? sv.f32(3 + j) : (j % 2 == 0 ? w.fh : w.fa2);
                DI_TRY(conv_f32(last, B, n->d.l2, H, W, n->w[2 + j], n->b[2 + j], n->d.l2, k, out, 1, st));
                last = out;
            }
        }
        {
            StageTimer t(n, st, DEEPINV_STAGE_CONV3);
            DI_TRY(conv_f32(last, B, n->d.l2, H, W, n->w[n->L - 1], n->b[n->L - 1], n->d.l3, k, xhat,
                            n->d.final_relu, st));
        }
    }
    if (saved) DI_CUDA(cudaMemcpyAsync(sv.xhat, xhat, (size_t)B * N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    return DEEPINV_OK;
}

int forward_impl(deepinv_net* n, const float* y, int B, float* xhat, void* saved, cudaStream_t st)
{
    if (B == 0) return DEEPINV_OK;
    DI_TRY(ensure_ws(n, B, st));
    // carve at the allocated batch so that plane offsets never move
    const FwdWs w = carve_fwd(n, n->ws_B, n->ws);
    return forward_core(n, w, y, B, xhat, saved, st);
}


// Backward of the bf16 path on the forward pass's planes (tensor cores for the
// conv2 and conv3 input gradients and the conv2 weight gradient).
struct BwdWs {
    float* g3;            // dL/dz3 [B][N]
    bf16 *g3p, *g2, *g1;  // gradient planes (zero borders)
    bf16* g2b;            // hidden layers: second 32-channel gradient plane
    float* part2;         // conv2 weight-gradient partials
    double *acc, *bpart, *lpart;
    float *T, *dxt;         // train_fc: conv1 input gradient (row sums, result)
    bf16 *dxp, *ypk;        // train_fc: packed operands of the FC weight gradient
    size_t bytes;
};

BwdWs carve_bwd_tc(const deepinv_net* n, int B, char* base)
{
    Arena a{base, 0};
    BwdWs w{};
    const Geo& g = n->geo;
    const int N = n->N;
    w.g3p = a.take<bf16>((size_t)B * g.plane);
    w.g2 = a.take<bf16>((size_t)B * 4 * g.plane * 8);
    w.g1 = a.take<bf16>((size_t)B * 8 * g.plane * 8);
    if (n->d.hidden > 0) w.g2b = a.take<bf16>((size_t)B * 4 * g.plane * 8);
    w.g3 = a.take<float>((size_t)B * N);
    w.part2 = a.take<float>(wgrad2_scratch_floats() > tapwgrad_scratch_floats() ? wgrad2_scratch_floats()
                                                                                 : tapwgrad_scratch_floats());
    w.acc = a.take<double>(64 * 121);
    w.bpart = a.take<double>((size_t)B * 64);
    w.lpart = a.take<double>(kLossBlocks);
    if (n->d.train_fc) {
        const int Kb = (B + 15) / 16 * 16, M = n->d.M;
        w.T = a.take<float>(conv3_scratch_elems(g, B, 64));
        w.dxt = a.take<float>((size_t)B * N);
        w.dxp = a.take<bf16>(packed_elems(N, 128, Kb));
        w.ypk = a.take<bf16>(packed_elems(M, gemm_nb(M), Kb));
    }
    w.bytes = align_up(a.off, 256);
    return w;
}

// Bnorm: the batch the loss is normalised by, (1 / Bnorm) sum_b ||x^_b - x_b||^2
// (B itself, or the whole batch when these B images are one chunk of it).
int backward_tc(deepinv_net* n, const float* y, const float* x, int B, int Bnorm, const Saved& sv,
                float* const dW[], float* const db[], float* dWfc, double* loss, cudaStream_t st)
{
    const Geo& g = n->geo;
    const int N = n->N, M = n->d.M;
    if (B > n->bws_B || !n->bws) {
        const size_t need = carve_bwd_tc(n, B, nullptr).bytes;
        DI_CUDA(cudaStreamSynchronize(st));
        cudaFree(n->bws);
        n->bws = nullptr;
        n->bws_bytes = 0;
        n->bws_B = 0;
        if (cudaMalloc(&n->bws, need) != cudaSuccess) {
            cudaGetLastError();
            n->bws = nullptr;
            set_error("backward workspace of %zu bytes: out of device memory", need);
            return DEEPINV_ENOMEM;
        }
        DI_CUDA(cudaMemset(n->bws, 0, need));   // gradient planes need zero borders
        n->bws_bytes = need;
        n->bws_B = B;
    }
    const BwdWs w = carve_bwd_tc(n, n->bws_B, n->bws);
    int* status = device_status_word();
    DI_REQUIRE(status, "no device status word");
    // dL/dz3 = 2 (x^ - x) / B (times [x^ > 0] with final_relu) and the loss in float64
    DI_TRY(mse_loss_grad(sv.xhat, x, (long long)B * N, Bnorm, n->d.final_relu, w.g3, w.lpart, loss, st));
    DI_TRY(grad_plane(w.g3, B, g, w.g3p, st));
    // conv3 (layer L-1, input a_{L-1}): bias and weight gradients, input
    // gradient times [a_{L-1} > 0] -> the gradient plane of layer L-2
    const int last = n->L - 1;
    DI_TRY(plane_channel_sums(w.g3p, B, 1, g, w.bpart, db[last], st));
    DI_TRY(tap_wgrad_tc(false, w.g3p, sv.plane(last), B, g, w.part2, dW[last], nullptr, status, st));
    DI_TRY(conv3_dgrad_tc(w.g3p, B, g, n->w3t, sv.plane(last), w.g2, status, st));
    // hidden layers l = L-2 .. 2 (input a_l): gradients, then the input gradient
    // times [a_l > 0], alternating between the two 32-channel gradient planes
    bf16* gcur = w.g2;
    bf16* gnext = w.g2b;
    for (int l = last - 1; l >= 2; --l) {
        const size_t j = (size_t)(l - 2);
        DI_TRY(plane_channel_sums(gcur, B, 32, g, w.bpart, db[l], st));
        DI_TRY(wgrad_hidden_tc(gcur, sv.plane(l), B, g, w.part2, dW[l], status, st));
        DI_TRY(hidden_dgrad_tc(gcur, B, g, n->wht + j * kWhPackElems, sv.plane(l), gnext, n->num_sms, status, st));
        bf16* t = gcur;
        gcur = gnext;
        gnext = t;
    }
    // conv2
    DI_TRY(plane_channel_sums(gcur, B, 32, g, w.bpart, db[1], st));
    DI_TRY(wgrad2_tc(gcur, sv.a1, B, g, w.part2, dW[1], status, st));
    DI_TRY(conv2_dgrad_tc(gcur, B, g, n->w2t, sv.a1, w.g1, n->num_sms, status, st));
    // conv1
    DI_TRY(tap_wgrad_tc(true, sv.xt, w.g1, B, g, w.part2, dW[0], db[0], status, st));
    if (n->d.train_fc) {
        // dx~ = conv1's input gradient, then dWfc[j][i] = sum_b dx~[b][j] y[b][i]
        // on the tensor cores with K = the batch
        DI_TRY(conv1_dgrad_tc(w.g1, B, g, n->w1t, w.T, w.dxt, status, st));
        const int Kb = (B + 15) / 16 * 16, NB = gemm_nb(M);
        DI_TRY(pack_kmajor(w.dxt, 1, N, N, B, 128, Kb, w.dxp, st));
        DI_TRY(pack_kmajor(y, 1, M, M, B, NB, Kb, w.ypk, st));
        DI_TRY(tc_gemm(w.dxp, w.ypk, Kb, N, M, NB, GEMM_OUT_F32, dWfc, M, nullptr, g, status, st));
    }
    return DEEPINV_OK;
}

int net_measure_impl(deepinv_net* n, const float* x, int B, float* y, cudaStream_t st)
{
    if (B == 0) return DEEPINV_OK;
    const int N = n->N, M = n->d.M;
    DI_TRY(ensure_ws(n, B, st));
    StageTimer t(n, st, DEEPINV_STAGE_MEASURE);
    if (n->tc) {
        const FwdWs w = carve_fwd(n, n->ws_B, n->ws);
        int* status = device_status_word();
        DI_REQUIRE(status, "no device status word");
        if ((size_t)n->Kms * cdiv(M, n->NBms) * n->NBms * sizeof(bf16) <= ((size_t)64 << 20) &&
            measure_f32in_supported(x, N, n->NBms)) {
            // x read by TMA and rounded to bf16 inside the GEMM, K split over a
            // cluster (Phi stays in L2)
            return gemm_measure_f32in(x, N, N, n->msB, n->Kms, B, M, n->NBms, y, M, n->num_sms, status, st);
        }
        // Phi too large for L2: x packed once, two row tiles per CTA read Phi once per 256 signals
        DI_TRY(pack_kmajor(x, N, 1, B, N, 128, n->Kms, w.xpk, st));
        const int ks = gemm_ksplit(B, M, n->NBms, n->Kms, n->num_sms);
        return tc_gemm_splitk(w.xpk, n->msB, n->Kms, B, M, n->NBms, y, w.mpart, ks, status, st);
    }
    return sgemm(B, M, N, x, N, 1, n->phi, 1, N, y, M, st);
}

}  // namespace

// ================================================================ internal interface (serving)
namespace di {

int net_device(const deepinv_net* n) { return n->dev; }
int net_M(const deepinv_net* n) { return n->d.M; }
int net_N(const deepinv_net* n) { return n->N; }

// Bytes of a private forward workspace for batches up to max_B (the staging
// buffers for y and x^ included); it must be zeroed once before first use.
size_t net_ws_bytes(const deepinv_net* n, int max_B) { return carve_fwd(n, max_B, nullptr).bytes; }

// x^ = M(y) for B <= max_B images with a private workspace `ws` (carved for
// max_B).  y_dev / xhat_dev may be NULL to use the workspace's own staging
// buffers, whose device addresses net_ws_staging returns.
int net_forward_ws(deepinv_net* n, char* ws, int max_B, const float* y, int B, float* xhat, cudaStream_t st)
{
    if (B == 0) return DEEPINV_OK;
    const FwdWs w = carve_fwd(n, max_B, ws);
    return forward_core(n, w, y, B, xhat, nullptr, st);
}

void net_ws_staging(const deepinv_net* n, char* ws, int max_B, float** y_dev, float** xhat_dev)
{
    const FwdWs w = carve_fwd(n, max_B, ws);
    *y_dev = w.yd;
    *xhat_dev = w.xhd;
}

}  // namespace di

// ================================================================ C ABI
namespace {

// Backward of the float32 path (NCHW activations in `sv`); Bnorm as in backward_tc.
int backward_f32(deepinv_net* net, const float* y, const float* x, int B, int Bnorm, const Saved& sv,
                 float* const dW[], float* const db[], float* dWfc, double* loss, cudaStream_t st)
{
    const int N = net->N, M = net->d.M, H = net->d.n1, W = net->d.n2, k = net->d.k;
    const int l1 = net->d.l1, l2 = net->d.l2, last = net->L - 1;
    size_t maxw = 0;
    for (int l = 0; l < net->L; ++l) maxw = wsize(net, l) > maxw ? wsize(net, l) : maxw;
    auto carve_bwd = [&](char* base, float** g3, float** gA, float** gC, float** gB, float** dxt, float** wt,
                         double** wpart, double** lpart) {
        Arena a{base, 0};
        *g3 = a.take<float>((size_t)B * N);
        *gA = a.take<float>((size_t)B * l2 * N);
        *gC = net->d.hidden > 0 ? a.take<float>((size_t)B * l2 * N) : nullptr;
        *gB = a.take<float>((size_t)B * l1 * N);
        *dxt = a.take<float>((size_t)B * N);
        *wt = a.take<float>(maxw);
        *wpart = a.take<double>((size_t)kWgradChunks * maxw);
        *lpart = a.take<double>(kLossBlocks);
        return align_up(a.off, 256);
    };
    float *g3, *gA, *gC, *gB, *dxt, *wt;
    double *wpart, *lpart;
    const size_t need = carve_bwd(nullptr, &g3, &gA, &gC, &gB, &dxt, &wt, &wpart, &lpart);
    if (need > net->bws_bytes) {
        DI_CUDA(cudaStreamSynchronize(st));
        cudaFree(net->bws);
        net->bws = nullptr;
        net->bws_bytes = 0;
        if (cudaMalloc(&net->bws, need) != cudaSuccess) {
            cudaGetLastError();
            net->bws = nullptr;
            set_error("backward workspace of %zu bytes: out of device memory", need);
            return DEEPINV_ENOMEM;
        }
        net->bws_bytes = need;
    }
    carve_bwd(net->bws, &g3, &gA, &gC, &gB, &dxt, &wt, &wpart, &lpart);

    // dL/dz_L = 2 (x^ - x) / B, and the loss in float64
    DI_TRY(mse_loss_grad(sv.xhat, x, (long long)B * N, Bnorm, net->d.final_relu, g3, lpart, loss, st));
    // conv3 (layer L-1, input a_{L-1})
    DI_TRY(conv_wgrad_f32(sv.f32(last), g3, B, l2, H, W, net->d.l3, k, wpart, dW[last], db[last], st));
    DI_TRY(conv_dgrad_f32(g3, B, net->d.l3, H, W, net->w[last], l2, k, wt, gA, st));
    DI_TRY(relu_mask_f32(gA, sv.f32(last), (long long)B * l2 * N, st));
    // hidden layers l = L-2 .. 2 (input a_l), alternating gA / gC
    float* gcur = gA;
    float* gnext = gC;
    for (int l = last - 1; l >= 2; --l) {
        DI_TRY(conv_wgrad_f32(sv.f32(l), gcur, B, l2, H, W, l2, k, wpart, dW[l], db[l], st));
        DI_TRY(conv_dgrad_f32(gcur, B, l2, H, W, net->w[l], l2, k, wt, gnext, st));
        DI_TRY(relu_mask_f32(gnext, sv.f32(l), (long long)B * l2 * N, st));
        float* t = gcur;
        gcur = gnext;
        gnext = t;
    }
    // conv2
    DI_TRY(conv_wgrad_f32(sv.fa1, gcur, B, l1, H, W, l2, k, wpart, dW[1], db[1], st));
    DI_TRY(conv_dgrad_f32(gcur, B, l2, H, W, net->w[1], l1, k, wt, gB, st));
    DI_TRY(relu_mask_f32(gB, sv.fa1, (long long)B * l1 * N, st));
    // conv1
    DI_TRY(conv_wgrad_f32(sv.fxt, gB, B, 1, H, W, l1, k, wpart, dW[0], db[0], st));
    if (net->d.train_fc) {
        DI_TRY(conv_dgrad_f32(gB, B, l1, H, W, net->w[0], 1, k, wt, dxt, st));
        // dWfc[j][i] = sum_b dx~[b][j] y[b][i]
        DI_TRY(sgemm(N, M, B, dxt, 1, N, y, M, 1, dWfc, M, st));
    }
    return DEEPINV_OK;
}

int backward_run(deepinv_net* net, const float* y, const float* x, int B, int Bnorm, const Saved& sv,
                 float* const dW[], float* const db[], float* dWfc, double* loss, cudaStream_t st)
{
    if (net->tc) return backward_tc(net, y, x, B, Bnorm, sv, dW, db, dWfc, loss, st);
    return backward_f32(net, y, x, B, Bnorm, sv, dW, db, dWfc, loss, st);
}

// Grow a library-owned device buffer to at least `need` bytes (synchronises when it grows).
int grow(char** buf, size_t* bytes, size_t need, const char* what, cudaStream_t st)
{
    if (need <= *bytes && *buf) return DEEPINV_OK;
    DI_CUDA(cudaStreamSynchronize(st));
    cudaFree(*buf);
    *buf = nullptr;
    *bytes = 0;
    if (cudaMalloc(buf, need) != cudaSuccess) {
        cudaGetLastError();
        *buf = nullptr;
        set_error("%s of %zu bytes: out of device memory", what, need);
        return DEEPINV_ENOMEM;
    }
    *bytes = need;
    return DEEPINV_OK;
}

// Backward without a saved buffer: the forward activations are recomputed in
// chunks of images whose activations fit the network's activation budget (one
// chunk when the budget is 0), each chunk's gradients added to the first
// chunk's in chunk order (deterministic).  The loss and its gradient stay
// normalised by the whole batch.
int backward_recompute(deepinv_net* net, const float* y, const float* x, int B, float* const dW[],
                       float* const db[], float* dWfc, double* loss, cudaStream_t st)
{
    const int N = net->N, M = net->d.M;
    int Bc = B;
    if (net->act_budget) {
        const size_t per = carve_saved(net, 1, nullptr).bytes;
        Bc = (int)(net->act_budget / per < (size_t)B ? net->act_budget / per : (size_t)B);
        if (Bc < 1) Bc = 1;
        while (Bc > 1 && carve_saved(net, Bc, nullptr).bytes > net->act_budget) --Bc;
    }
    DI_TRY(grow(&net->rsaved, &net->rsaved_bytes, carve_saved(net, Bc, nullptr).bytes, "recomputation buffer", st));
    DI_TRY(ensure_ws(net, Bc, st));
    const FwdWs fw = carve_fwd(net, net->ws_B, net->ws);
    // gradient scratch of the chunks after the first: dW[L], db[L], dWfc, loss
    float* gW[deepinv_net::kMaxLayers];
    float* gB[deepinv_net::kMaxLayers];
    float* gFc = nullptr;
    double* gL = nullptr;
    if (Bc < B) {
        Arena a{nullptr, 0};
        for (int l = 0; l < net->L; ++l) a.take<float>(wsize(net, l));
        for (int l = 0; l < net->L; ++l) a.take<float>(bsize(net, l));
        if (net->d.train_fc) a.take<float>((size_t)N * M);
        a.take<double>(1);
        DI_TRY(grow(&net->gacc, &net->gacc_bytes, align_up(a.off, 256), "gradient scratch", st));
        Arena g{net->gacc, 0};
        for (int l = 0; l < net->L; ++l) gW[l] = g.take<float>(wsize(net, l));
        for (int l = 0; l < net->L; ++l) gB[l] = g.take<float>(bsize(net, l));
        if (net->d.train_fc) gFc = g.take<float>((size_t)N * M);
        gL = g.take<double>(1);
    }
    for (int b0 = 0; b0 < B; b0 += Bc) {
        const int nb = B - b0 < Bc ? B - b0 : Bc;
        const float* yc = y + (size_t)b0 * M;
        const float* xc = x + (size_t)b0 * N;
        DI_TRY(forward_impl(net, yc, nb, fw.xhd, net->rsaved, st));
        const Saved sv = carve_saved(net, nb, net->rsaved);
        if (b0 == 0) {
            DI_TRY(backward_run(net, yc, xc, nb, B, sv, dW, db, dWfc, loss, st));
            continue;
        }
        DI_TRY(backward_run(net, yc, xc, nb, B, sv, gW, gB, gFc, gL, st));
        for (int l = 0; l < net->L; ++l) {
            DI_TRY(accumulate_f32(dW[l], gW[l], (long long)wsize(net, l), st));
            DI_TRY(accumulate_f32(db[l], gB[l], (long long)bsize(net, l), st));
        }
        if (net->d.train_fc) DI_TRY(accumulate_f32(dWfc, gFc, (long long)N * M, st));
        DI_TRY(accumulate_f64(loss, gL, 1, st));
    }
    return DEEPINV_OK;
}

// Host-memory entry points: submit one batch (input from host memory, x^ to
// host memory) without waiting.  Slot t % 2 of the staging buffers serves
// ticket t: its input copy (stream cs_in) waits until batch t - 2 has read the
// slot's input, its compute (the caller's stream `st`) waits for the copy and
// for the device -> host copy of batch t - 2 out of the slot's x^ buffer, and
// its x^ copy (stream cs_out) follows the compute.  So batch t + 1's input and
// batch t - 1's result move while batch t computes.  in_host is x [B][N]
// (measure first) or y [B][M].
int host_submit(deepinv_net* net, const float* in_host, bool measure, int B, float* xhat_host, cudaStream_t st,
                uint64_t* ticket)
{
    const int N = net->N, M = net->d.M;
    const size_t in_elems = (size_t)B * (measure ? N : M), out_elems = (size_t)B * N;
    // copy streams and slot events, created on first use (each one that is
    // still missing, so that a failed creation is retried by the next call)
    if (!net->cs_in) DI_CUDA(cudaStreamCreateWithFlags(&net->cs_in, cudaStreamNonBlocking));
    if (!net->cs_out) DI_CUDA(cudaStreamCreateWithFlags(&net->cs_out, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k)
        for (cudaEvent_t* e : {&net->ev_h2d[k], &net->ev_read[k], &net->ev_comp[k], &net->ev_d2h[k]})
            if (!*e) DI_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    if (in_elems > net->hin_elems || out_elems > net->hout_elems) {
        // grow the staging slots once nothing in flight uses them
        DI_CUDA(cudaStreamSynchronize(net->cs_in));
        DI_CUDA(cudaStreamSynchronize(st));
        DI_CUDA(cudaStreamSynchronize(net->cs_out));
        // (a size is recorded only once both slots hold it, so that a failed
        // allocation leaves no null slot behind a nonzero size)
        if (in_elems > net->hin_elems) {
            net->hin_elems = 0;
            for (int k = 0; k < 2; ++k) {
                cudaFree(net->hin[k]);
                net->hin[k] = nullptr;
            }
            for (int k = 0; k < 2; ++k) DI_TRY(dev_alloc(&net->hin[k], in_elems));
            net->hin_elems = in_elems;
        }
        if (out_elems > net->hout_elems) {
            net->hout_elems = 0;
            for (int k = 0; k < 2; ++k) {
                cudaFree(net->hout[k]);
                net->hout[k] = nullptr;
            }
            for (int k = 0; k < 2; ++k) DI_TRY(dev_alloc(&net->hout[k], out_elems));
            net->hout_elems = out_elems;
        }
    }
    DI_TRY(ensure_ws(net, B, st));
    const FwdWs w = carve_fwd(net, net->ws_B, net->ws);
    const uint64_t t = net->hnext++;
    const int k = (int)(t & 1);
    DI_CUDA(cudaStreamWaitEvent(net->cs_in, net->ev_read[k], 0));
    DI_CUDA(cudaMemcpyAsync(net->hin[k], in_host, in_elems * sizeof(float), cudaMemcpyHostToDevice, net->cs_in));
    DI_CUDA(cudaEventRecord(net->ev_h2d[k], net->cs_in));
    DI_CUDA(cudaStreamWaitEvent(st, net->ev_h2d[k], 0));
    DI_CUDA(cudaStreamWaitEvent(st, net->ev_d2h[k], 0));
    const float* y = net->hin[k];
    if (measure) {
        DI_TRY(net_measure_impl(net, net->hin[k], B, w.yd, st));
        y = w.yd;
        DI_CUDA(cudaEventRecord(net->ev_read[k], st));
    }
    DI_TRY(forward_impl(net, y, B, net->hout[k], nullptr, st));
    if (!measure) DI_CUDA(cudaEventRecord(net->ev_read[k], st));
    DI_CUDA(cudaEventRecord(net->ev_comp[k], st));
    DI_CUDA(cudaStreamWaitEvent(net->cs_out, net->ev_comp[k], 0));
    DI_CUDA(cudaMemcpyAsync(xhat_host, net->hout[k], out_elems * sizeof(float), cudaMemcpyDeviceToHost, net->cs_out));
    DI_CUDA(cudaEventRecord(net->ev_d2h[k], net->cs_out));
    if (ticket) *ticket = t;
    return DEEPINV_OK;
}

// Wait until the x^ of `ticket` is in host memory (or a later batch's, which
// implies it).
int host_wait(deepinv_net* net, uint64_t ticket)
{
    if (!net->cs_out || ticket >= net->hnext) return DEEPINV_OK;
    DI_CUDA(cudaEventSynchronize(net->ev_d2h[ticket & 1]));
    return DEEPINV_OK;
}

// Training state file: "DINVSTAT", uint32 version, the network's deepinv_net_desc,
// then per layer (network order) w, its momentum, b, its momentum, then with
// train_fc the FC weights and their momentum; every array float32, preceded by
// its element count (uint64).
const char kStateMagic[8] = {'D', 'I', 'N', 'V', 'S', 'T', 'A', 'T'};
const uint32_t kStateVersion = 1;

int state_io(deepinv_net* net, FILE* f, bool save)
{
    std::vector<float> host;
    auto one = [&](float* dev, size_t n) -> int {
        uint64_t cnt = n;
        if (save) {
            host.resize(n);
            DI_CUDA(cudaMemcpy(host.data(), dev, n * 4, cudaMemcpyDeviceToHost));
            if (fwrite(&cnt, 8, 1, f) != 1 || fwrite(host.data(), 4, n, f) != n) {
                set_error("state file: write failed");
                return DEEPINV_EINVAL;
            }
        } else {
            if (fread(&cnt, 8, 1, f) != 1 || cnt != n) {
                set_error("state file: array of %llu elements where the network has %zu",
                          (unsigned long long)cnt, n);
                return DEEPINV_EINVAL;
            }
            host.resize(n);
            if (fread(host.data(), 4, n, f) != n) {
                set_error("state file: truncated");
                return DEEPINV_EINVAL;
            }
            DI_CUDA(cudaMemcpy(dev, host.data(), n * 4, cudaMemcpyHostToDevice));
        }
        return DEEPINV_OK;
    };
    for (int l = 0; l < net->L; ++l) {
        DI_TRY(one(net->w[l], wsize(net, l)));
        DI_TRY(one(net->vw[l], wsize(net, l)));
        DI_TRY(one(net->b[l], bsize(net, l)));
        DI_TRY(one(net->vb[l], bsize(net, l)));
    }
    if (net->d.train_fc) {
        DI_TRY(one(net->wfc, (size_t)net->N * net->d.M));
        DI_TRY(one(net->vfc, (size_t)net->N * net->d.M));
    }
    return DEEPINV_OK;
}
}  // namespace

extern "C" {

const char* deepinv_last_error(void) { return di::g_err; }

int deepinv_version(void) { return 201; }

unsigned long long deepinv_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int deepinv_device_status(int reset)
{
    std::vector<int*> words;
    {
        std::lock_guard<std::mutex> lk(g_status_mu);
        words = g_status_words;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        ndev = 0;
    }
    if ((int)words.size() > ndev) ndev = (int)words.size();
    int v = 0;
    for (int dev = 0; dev < ndev; ++dev) {
        // the library's status word and the allocation-free measurement's one
        int* w2[2] = {dev < (int)words.size() ? words[dev] : nullptr, noalloc_status_word(dev)};
        if (!w2[0] && !w2[1]) continue;
        DeviceGuard g(dev);
        DI_CUDA(cudaDeviceSynchronize());
        for (int* p : w2) {
            if (!p) continue;
            int w = 0;
            DI_CUDA(cudaMemcpy(&w, p, sizeof(int), cudaMemcpyDeviceToHost));
            if (reset) DI_CUDA(cudaMemset(p, 0, sizeof(int)));
            if (w) v = w;
        }
    }
    if (v == DEV_TIMEOUT) {
        set_error("a bounded wait inside a kernel ran out");
        return DEEPINV_ETIMEOUT;
    }
    return DEEPINV_OK;
}

int deepinv_selftest_bounded_wait(void* stream)
{
    int* status = device_status_word();
    DI_REQUIRE(status, "no device status word");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DI_TRY(bounded_wait_probe(status, st));
    DI_CUDA(cudaStreamSynchronize(st));
    return DEEPINV_OK;
}

int deepinv_measure(const float* phi, int M, int N, const float* x, int B, float* y, int prec, void* stream)
{
    // (sizes up to 2^30, so that padded extents stay within int)
    DI_REQUIRE(M >= 1 && N >= 1 && B >= 0 && M <= (1 << 30) && N <= (1 << 30) && B <= (1 << 30),
               "bad sizes M=%d N=%d B=%d", M, N, B);
    DI_REQUIRE(B == 0 || (phi && x && y), "null pointer");
    DI_REQUIRE(prec == DEEPINV_F32 || prec == DEEPINV_BF16, "unknown precision %d", prec);
    if (B == 0) return DEEPINV_OK;
    DeviceGuard dg(device_of(phi));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (prec == DEEPINV_F32) return sgemm(B, M, N, x, N, 1, phi, 1, N, y, M, st);
    const int Kp = up16(N), NB = gemm_nb(M);
    bf16* phiB = nullptr;
    bf16* xpk = nullptr;
    const size_t nphi = packed_elems(M, NB, Kp), nx = packed_elems(B, 128, Kp);
    if (cudaMallocAsync(reinterpret_cast<void**>(&phiB), nphi * sizeof(bf16), st) != cudaSuccess ||
        cudaMallocAsync(reinterpret_cast<void**>(&xpk), nx * sizeof(bf16), st) != cudaSuccess) {
        cudaGetLastError();
        if (phiB) cudaFreeAsync(phiB, st);
        set_error("deepinv_measure: out of device memory");
        return DEEPINV_ENOMEM;
    }
    int rc = pack_kmajor(phi, N, 1, M, N, NB, Kp, phiB, st);
    if (rc == DEEPINV_OK) rc = measure_bf16_packed(phiB, Kp, NB, x, N, M, B, y, xpk, st);
    cudaFreeAsync(phiB, st);
    cudaFreeAsync(xpk, st);
    return rc;
}

int deepinv_net_create(const deepinv_net_desc* desc, const float* phi, const float* const w[],
                       const float* const b[], void* stream, deepinv_net** out)
{
    DI_REQUIRE(out, "out is NULL");
    DI_TRY(check_desc(desc));
    DI_REQUIRE(phi && w && b, "null pointer");
    for (int l = 0; l < 3 + desc->hidden; ++l) DI_REQUIRE(w[l] && b[l], "null weight pointer for layer %d", l + 1);
    const int dev = device_of(phi);
    DI_REQUIRE(dev >= 0, "phi is not device memory");
    DeviceGuard dg(dev);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    deepinv_net* n = new (std::nothrow) deepinv_net();
    DI_REQUIRE(n, "host allocation failed");
    n->d = *desc;
    n->L = 3 + desc->hidden;
    n->dev = dev;
    n->N = desc->n1 * desc->n2;
    n->tc = desc->prec != DEEPINV_F32;
    n->fp8 = desc->prec == DEEPINV_FP8_E4M3;
    n->num_sms = num_sms_current();
    const int N = n->N, M = desc->M;
    int rc = DEEPINV_OK;
#define DI_STEP(x) do { rc = (x); if (rc != DEEPINV_OK) { free_net(n); return rc; } } while (0)
    DI_STEP(dev_alloc(&n->phi, (size_t)M * N));
    DI_STEP(cudaMemcpyAsync(n->phi, phi, (size_t)M * N * sizeof(float), cudaMemcpyDeviceToDevice, st) == cudaSuccess
                ? DEEPINV_OK : DEEPINV_ECUDA);
    for (int l = 0; l < n->L; ++l) {
        DI_STEP(dev_alloc(&n->w[l], wsize(n, l)));
        DI_STEP(dev_alloc(&n->b[l], bsize(n, l)));
        DI_STEP(dev_alloc(&n->vw[l], wsize(n, l)));
        DI_STEP(dev_alloc(&n->vb[l], bsize(n, l)));
        DI_STEP(cudaMemcpyAsync(n->w[l], w[l], wsize(n, l) * 4, cudaMemcpyDeviceToDevice, st) == cudaSuccess
                    ? DEEPINV_OK : DEEPINV_ECUDA);
        DI_STEP(cudaMemcpyAsync(n->b[l], b[l], bsize(n, l) * 4, cudaMemcpyDeviceToDevice, st) == cudaSuccess
                    ? DEEPINV_OK : DEEPINV_ECUDA);
        DI_STEP(cudaMemsetAsync(n->vw[l], 0, wsize(n, l) * 4, st) == cudaSuccess ? DEEPINV_OK : DEEPINV_ECUDA);
        DI_STEP(cudaMemsetAsync(n->vb[l], 0, bsize(n, l) * 4, st) == cudaSuccess ? DEEPINV_OK : DEEPINV_ECUDA);
    }
    if (desc->train_fc) {
        DI_STEP(dev_alloc(&n->wfc, (size_t)N * M));
        DI_STEP(dev_alloc(&n->vfc, (size_t)N * M));
        DI_STEP(cudaMemsetAsync(n->vfc, 0, (size_t)N * M * 4, st) == cudaSuccess ? DEEPINV_OK : DEEPINV_ECUDA);
    }
    if (n->tc) {
        n->geo = make_geo(desc->n1, desc->n2);
        n->Kfc = up16(M);
        n->Kms = up16(N);
        n->NBms = gemm_nb(M);
        DI_STEP(dev_alloc(&n->fcA, packed_elems(N, 128, n->Kfc)));
        DI_STEP(dev_alloc(&n->msB, packed_elems(M, n->NBms, n->Kms)));
        DI_STEP(dev_alloc(&n->w1p, kW1PackElems));
        DI_STEP(dev_alloc(&n->w2p, kW2PackElems));
        DI_STEP(dev_alloc(&n->w3p, kW3PackElems));
        if (!n->fp8) {
            DI_STEP(dev_alloc(&n->w2t, kW2PackElems));
            DI_STEP(dev_alloc(&n->w3t, kW3tPackElems));
            DI_STEP(dev_alloc(&n->w1t, kW1tPackElems));
        }
        if (desc->hidden > 0) {
            DI_STEP(dev_alloc(&n->whp, kWhPackElems * desc->hidden));
            if (!n->fp8) DI_STEP(dev_alloc(&n->wht, kWhPackElems * desc->hidden));
        }
        if (n->fp8) {
            DI_STEP(dev_alloc(&n->w2q, kW2E4M3Bytes));
            DI_STEP(dev_alloc(&n->sw, 32 + 32 + 1 + 1 + 32));   // sw | oscale | inv_sa | amax_a1 | amax_w
            n->oscale = n->sw + 32;
            n->inv_sa = n->sw + 64;
            n->amax_a1 = n->sw + 65;
            n->amax_w = n->sw + 66;
        }
        DI_STEP(pack_kmajor(n->phi, N, 1, M, N, n->NBms, n->Kms, n->msB, st));
    }
    if (desc->train_fc) DI_STEP(transpose_f32(n->phi, M, N, n->wfc, st));
    DI_STEP(repack(n, st));
    DI_STEP(cudaStreamSynchronize(st) == cudaSuccess ? DEEPINV_OK : DEEPINV_ECUDA);
#undef DI_STEP
    *out = n;
    return DEEPINV_OK;
}

int deepinv_net_destroy(deepinv_net* net)
{
    if (!net) return DEEPINV_OK;
    DeviceGuard dg(net->dev);
    cudaDeviceSynchronize();
    free_net(net);
    return DEEPINV_OK;
}

int deepinv_net_get_desc(const deepinv_net* net, deepinv_net_desc* desc)
{
    DI_REQUIRE(net && desc, "null pointer");
    *desc = net->d;
    return DEEPINV_OK;
}

int deepinv_net_reserve(deepinv_net* net, int max_B, void* stream)
{
    DI_REQUIRE(net, "net is NULL");
    DeviceGuard dg(net->dev);
    DI_REQUIRE(max_B >= 0 && max_B <= kMaxBatch, "bad batch %d", max_B);
    if (max_B == 0) return DEEPINV_OK;
    return ensure_ws(net, max_B, static_cast<cudaStream_t>(stream));
}

int deepinv_net_measure(deepinv_net* net, const float* x, int B, float* y, void* stream)
{
    DI_REQUIRE(net, "net is NULL");
    DeviceGuard dg(net->dev);
    DI_REQUIRE(B >= 0 && B <= kMaxBatch, "bad batch %d", B);
    DI_REQUIRE(B == 0 || (x && y), "null pointer");
    return net_measure_impl(net, x, B, y, static_cast<cudaStream_t>(stream));
}

size_t deepinv_saved_bytes(const deepinv_net* net, int B)
{
    if (!net || B <= 0) return 0;
    return carve_saved(net, B, nullptr).bytes;
}

int deepinv_forward(deepinv_net* net, const float* y, int B, float* xhat, void* saved, void* stream)
{
    DI_REQUIRE(net, "net is NULL");
    DeviceGuard dg(net->dev);
    DI_REQUIRE(B >= 0 && B <= kMaxBatch, "bad batch %d", B);
    DI_REQUIRE(B == 0 || (y && xhat), "null pointer");
    return forward_impl(net, y, B, xhat, saved, static_cast<cudaStream_t>(stream));
}

int deepinv_forward_host(deepinv_net* net, const float* y_host, int B, float* xhat_host, void* stream)
{
    DI_REQUIRE(net, "net is NULL");
    DeviceGuard dg(net->dev);
    DI_REQUIRE(B >= 0 && B <= kMaxBatch, "bad batch %d", B);
    DI_REQUIRE(B == 0 || (y_host && xhat_host), "null pointer");
    if (B == 0) return DEEPINV_OK;
    uint64_t t = 0;
    DI_TRY(host_submit(net, y_host, false, B, xhat_host, static_cast<cudaStream_t>(stream), &t));
    return host_wait(net, t);
}

int deepinv_sense_recover_host(deepinv_net* net, const float* x_host, int B, float* xhat_host, void* stream)
{
    DI_REQUIRE(net, "net is NULL");
    DeviceGuard dg(net->dev);
    DI_REQUIRE(B >= 0 && B <= kMaxBatch, "bad batch %d", B);
    DI_REQUIRE(B == 0 || (x_host && xhat_host), "null pointer");
    if (B == 0) return DEEPINV_OK;
    uint64_t t = 0;
    DI_TRY(host_submit(net, x_host, true, B, xhat_host, static_cast<cudaStream_t>(stream), &t));
    return host_wait(net, t);
}

int deepinv_sense_recover_host_submit(deepinv_net* net, const float* x_host, int B, float* xhat_host, void* stream,
                                      uint64_t* ticket)
{
    DI_REQUIRE(net, "net is NULL");
    DeviceGuard dg(net->dev);
    DI_REQUIRE(B >= 1 && B <= kMaxBatch && x_host && xhat_host && ticket, "bad batch %d or null pointer", B);
    return host_submit(net, x_host, true, B, xhat_host, static_cast<cudaStream_t>(stream), ticket);
}

int deepinv_host_wait(deepinv_net* net, uint64_t ticket)
{
    DI_REQUIRE(net, "net is NULL");
    DeviceGuard dg(net->dev);
    return host_wait(net, ticket);
}

int deepinv_net_set_act_budget(deepinv_net* net, size_t bytes)
{
    DI_REQUIRE(net, "net is NULL");
    net->act_budget = bytes;
    return DEEPINV_OK;
}

int deepinv_net_set_fused(deepinv_net* net, int enable)
{
    DI_REQUIRE(net, "net is NULL");
    net->fused12 = enable != 0;
    return DEEPINV_OK;
}

int deepinv_net_set_conv1_rows(deepinv_net* net, int mode)
{
    DI_REQUIRE(net, "net is NULL");
    DI_REQUIRE(mode >= 0 && mode <= 2, "conv1 row-tile mode %d (0, 1 or 2)", mode);
    net->conv1_rows = mode;
    return DEEPINV_OK;
}

int deepinv_backward(deepinv_net* net, const float* y, const float* x, int B, const void* saved,
                     float* const dW[], float* const db[], float* dWfc, double* loss, void* stream)
{
    DI_REQUIRE(net, "net is NULL");
    DeviceGuard dg(net->dev);
    DI_REQUIRE(B >= 1 && B <= kMaxBatch, "bad batch %d", B);
    DI_REQUIRE(y && x && dW && db && loss, "null pointer");
    for (int l = 0; l < net->L; ++l) DI_REQUIRE(dW[l] && db[l], "null gradient pointer for layer %d", l + 1);
    DI_REQUIRE(!net->d.train_fc || dWfc, "train_fc network needs dWfc");
    if (net->fp8) {
        set_error("e4m3 networks are inference only (train in bf16 or f32)");
        return DEEPINV_EUNSUPPORTED;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    NvtxRange range("deepinv backward");
    if (!saved) return backward_recompute(net, y, x, B, dW, db, dWfc, loss, st);
    const Saved sv = carve_saved(net, B, static_cast<char*>(const_cast<void*>(saved)));
    return backward_run(net, y, x, B, B, sv, dW, db, dWfc, loss, st);
}

int deepinv_sgd_momentum(deepinv_net* net, const float* const dW[], const float* const db[], const float* dWfc,
                         float lr, float mu, void* stream)
{
    DI_REQUIRE(net, "net is NULL");
    DeviceGuard dg(net->dev);
    DI_REQUIRE(dW && db, "null pointer");
    for (int l = 0; l < net->L; ++l) DI_REQUIRE(dW[l] && db[l], "null gradient pointer for layer %d", l + 1);
    DI_REQUIRE(!net->d.train_fc || dWfc, "train_fc network needs dWfc");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    NvtxRange range("deepinv sgd_momentum");
    // every tensor in one launch (2 L + 1 <= kSgdMaxTensors)
    SgdTensors t{};
    for (int l = 0; l < net->L; ++l) {
        t.w[t.count] = net->w[l], t.v[t.count] = net->vw[l], t.g[t.count] = dW[l], t.n[t.count++] = (long long)wsize(net, l);
        t.w[t.count] = net->b[l], t.v[t.count] = net->vb[l], t.g[t.count] = db[l], t.n[t.count++] = (long long)bsize(net, l);
    }
    if (net->d.train_fc)
        t.w[t.count] = net->wfc, t.v[t.count] = net->vfc, t.g[t.count] = dWfc, t.n[t.count++] = (long long)net->N * net->d.M;
    DI_TRY(sgd_momentum_multi(t, lr, mu, st));
    return repack(net, st);
}

int deepinv_net_save_state(deepinv_net* net, const char* path)
{
    DI_REQUIRE(net && path, "null pointer");
    DeviceGuard dg(net->dev);
    DI_CUDA(cudaDeviceSynchronize());
    FILE* f = fopen(path, "wb");
    DI_REQUIRE(f, "cannot open %s for writing", path);
    int rc = DEEPINV_OK;
    if (fwrite(kStateMagic, 1, 8, f) != 8 || fwrite(&kStateVersion, 4, 1, f) != 1 ||
        fwrite(&net->d, sizeof(net->d), 1, f) != 1) {
        set_error("state file: write failed");
        rc = DEEPINV_EINVAL;
    }
    if (rc == DEEPINV_OK) rc = state_io(net, f, true);
    if (fclose(f) != 0 && rc == DEEPINV_OK) {
        set_error("state file: close failed");
        rc = DEEPINV_EINVAL;
    }
    return rc;
}

int deepinv_net_load_state(deepinv_net* net, const char* path, void* stream)
{
    DI_REQUIRE(net && path, "null pointer");
    DeviceGuard dg(net->dev);
    FILE* f = fopen(path, "rb");
    DI_REQUIRE(f, "cannot open %s", path);
    char magic[8];
    uint32_t version = 0;
    deepinv_net_desc d{};
    int rc = DEEPINV_OK;
    if (fread(magic, 1, 8, f) != 8 || memcmp(magic, kStateMagic, 8) != 0 || fread(&version, 4, 1, f) != 1 ||
        version != kStateVersion || fread(&d, sizeof(d), 1, f) != 1) {
        set_error("%s is not a version-%u state file", path, kStateVersion);
        rc = DEEPINV_EINVAL;
    } else if (d.n1 != net->d.n1 || d.n2 != net->d.n2 || d.M != net->d.M || d.l1 != net->d.l1 ||
               d.l2 != net->d.l2 || d.l3 != net->d.l3 || d.k != net->d.k || d.hidden != net->d.hidden ||
               d.train_fc != net->d.train_fc || d.final_relu != net->d.final_relu) {
        set_error("state file %s was saved from a different network", path);
        rc = DEEPINV_EINVAL;
    }
    if (rc == DEEPINV_OK) {
        DI_CUDA(cudaDeviceSynchronize());
        rc = state_io(net, f, false);
    }
    fclose(f);
    if (rc != DEEPINV_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DI_TRY(repack(net, st));
    DI_CUDA(cudaStreamSynchronize(st));
    return DEEPINV_OK;
}

int deepinv_get_params(const deepinv_net* net, float* const w[], float* const b[], float* wfc, void* stream)
{
    DI_REQUIRE(net, "net is NULL");
    DeviceGuard dg(net->dev);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int l = 0; l < net->L; ++l) {
        if (w && w[l]) DI_CUDA(cudaMemcpyAsync(w[l], net->w[l], wsize(net, l) * 4, cudaMemcpyDeviceToDevice, st));
        if (b && b[l]) DI_CUDA(cudaMemcpyAsync(b[l], net->b[l], bsize(net, l) * 4, cudaMemcpyDeviceToDevice, st));
    }
    if (wfc) {
        DI_REQUIRE(net->wfc, "network has no trainable FC weights");
        DI_CUDA(cudaMemcpyAsync(wfc, net->wfc, (size_t)net->N * net->d.M * 4, cudaMemcpyDeviceToDevice, st));
    }
    return DEEPINV_OK;
}

int deepinv_profile_enable(deepinv_net* net, int enable)
{
    DI_REQUIRE(net, "net is NULL");
    net->prof = enable != 0;
    net->spans.clear();
    net->ev_used = 0;
    return DEEPINV_OK;
}

int deepinv_profile_read(deepinv_net* net, float stage_ms[DEEPINV_NSTAGES], int stage_count[DEEPINV_NSTAGES])
{
    DI_REQUIRE(net, "net is NULL");
    DeviceGuard dg(net->dev);
    float ms[DEEPINV_NSTAGES] = {0};
    int cnt[DEEPINV_NSTAGES] = {0};
    for (size_t i = 0; i + 2 < net->spans.size(); i += 3) {
        const int stg = net->spans[i];
        cudaEvent_t e0 = net->ev_pool[net->spans[i + 1]], e1 = net->ev_pool[net->spans[i + 2]];
        DI_CUDA(cudaEventSynchronize(e1));
        float t = 0.f;
        DI_CUDA(cudaEventElapsedTime(&t, e0, e1));
        if (stg >= 0 && stg < DEEPINV_NSTAGES) {
            ms[stg] += t;
            cnt[stg] += 1;
        }
    }
    net->spans.clear();
    net->ev_used = 0;
    for (int s = 0; s < DEEPINV_NSTAGES; ++s) {
        if (stage_ms) stage_ms[s] = ms[s];
        if (stage_count) stage_count[s] = cnt[s];
    }
    return DEEPINV_OK;
}

int deepinv_net_calibrate(deepinv_net* net, const float* y, int B, void* stream)
{
    DI_REQUIRE(net, "net is NULL");
    DeviceGuard dg(net->dev);
    DI_REQUIRE(B >= 1 && B <= kMaxBatch && y, "calibration needs a batch (1 <= B <= 2^30) of measurements");
    if (!net->fp8) return DEEPINV_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DI_TRY(ensure_ws(net, B, st));
    const FwdWs w = carve_fwd(net, net->ws_B, net->ws);
    const Geo& g = net->geo;
    int* status = device_status_word();
    DI_REQUIRE(status, "no device status word");
    const int N = net->N, M = net->d.M;
    const int nb = fc_nb(B);
    DI_TRY(pack_kmajor(y, M, 1, B, M, nb, net->Kfc, w.ypk, st));
    DI_TRY(tc_gemm(net->fcA, w.ypk, net->Kfc, N, B, nb, GEMM_OUT_PLANE, nullptr, 0, w.xt, g, status, st));
    DI_CUDA(cudaMemsetAsync(net->amax_a1, 0, sizeof(float), st));
    DI_TRY(conv1_tc(w.xt, B, g, net->w1p, net->b[0], nullptr, kConv1AmaxOnly, nullptr, net->amax_a1, status, st));
    DI_TRY(e4m3_scales(net->amax_a1, net->sw, net->inv_sa, net->oscale, st));
    DI_CUDA(cudaStreamSynchronize(st));
    net->calibrated = true;
    return DEEPINV_OK;
}

}  // extern "C"
