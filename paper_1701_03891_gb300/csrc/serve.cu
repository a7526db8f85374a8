// Continuous-batching server of libdeepinv (deepinv_serve_*).
//
// The paper motivates DeepInverse by low-latency recovery (Sec. 5).  Here a
// host scheduler thread turns a stream of single recoveries for several
// networks (image sizes and M/N ratios) into batches: per-network FIFO queues,
// up to max_streams batches in flight on separate CUDA streams, each batch in
// a private workspace leased under an HBM budget, results copied back to the
// requests' host buffers as soon as their batch's event completes.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "kernels.cuh"

namespace di {
int net_device(const deepinv_net* n);
int net_M(const deepinv_net* n);
int net_N(const deepinv_net* n);
size_t net_ws_bytes(const deepinv_net* n, int max_B);
int net_forward_ws(deepinv_net* n, char* ws, int max_B, const float* y, int B, float* xhat, cudaStream_t st);
void net_ws_staging(const deepinv_net* n, char* ws, int max_B, float** y_dev, float** xhat_dev);
}  // namespace di

using namespace di;
using Clock = std::chrono::steady_clock;

namespace {

struct Req {
    int net;
    uint64_t tag;
    float* xhat;
    std::vector<float> y;   // copy of the caller's measurement
    Clock::time_point t_submit;
};

struct Lease {
    int net;
    char* ws;
    size_t bytes;
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    float* y_pin = nullptr;   // [max_batch][maxM] page-locked staging
    float* x_pin = nullptr;   // [max_batch][maxN]
    bool busy = false;
    int net = -1;
    std::vector<Req> reqs;
    Lease* lease = nullptr;
    Clock::time_point t_launch;
};

double us_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::micro>(b - a).count();
}

// Helper threads that share a batch's per-request host copies (staging the
// measurements, handing back the results) with the scheduler thread: at a few
// hundred thousand requests per second those copies are several GB/s, more
// than one thread moves.  run(n, f) calls f(i) once for every i < n, on the
// calling thread and on the helpers, and returns when all calls have returned.
struct CopyPool {
    std::vector<std::thread> th;
    std::mutex mu;
    std::condition_variable cv, cv_done;
    const std::function<void(int)>* job = nullptr;
    int n = 0, next = 0, active = 0;
    uint64_t gen = 0;
    bool stop = false;

    void worker()
    {
        uint64_t seen = 0;
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            cv.wait(lk, [&] { return stop || gen != seen; });
            if (stop) return;
            seen = gen;
            ++active;
            while (next < n) {
                const int i = next++;
                const std::function<void(int)>* f = job;
                lk.unlock();
                (*f)(i);
                lk.lock();
            }
            if (--active == 0) cv_done.notify_all();
        }
    }
    void start(int helpers)
    {
        for (int k = 0; k < helpers; ++k) th.emplace_back([this] { worker(); });
    }
    void run(int count, const std::function<void(int)>& f)
    {
        if (th.empty() || count < 2) {
            for (int i = 0; i < count; ++i) f(i);
            return;
        }
        std::unique_lock<std::mutex> lk(mu);
        job = &f;
        n = count;
        next = 0;
        ++gen;
        cv.notify_all();
        while (next < n) {
            const int i = next++;
            lk.unlock();
            f(i);
            lk.lock();
        }
        cv_done.wait(lk, [&] { return active == 0; });
        job = nullptr;
        n = next = 0;
    }
    void shutdown()
    {
        {
            std::lock_guard<std::mutex> lk(mu);
            stop = true;
        }
        cv.notify_all();
        for (std::thread& t : th) t.join();
        th.clear();
    }
};

// Batches whose copies are smaller than this stay on the scheduler thread.
constexpr size_t kParallelCopyBytes = 256 << 10;

}  // namespace

struct deepinv_server {
    size_t budget = 0;
    int max_streams = 1, max_batch = 1;
    int dev = -1;
    int maxM = 0, maxN = 0;
    std::vector<deepinv_net*> nets;
    std::vector<size_t> lease_bytes;
    std::vector<std::deque<Req>> pending;
    std::vector<std::vector<Lease*>> cache;
    std::vector<Slot> slots;
    size_t held = 0;
    std::deque<deepinv_result> done;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread thr;
    bool stop = false, started = false, waiting_admission = false;
    uint64_t outstanding = 0;   // submitted and not yet finished
    deepinv_serve_stats stats{};
    CopyPool copies;            // used by the scheduler thread only
};

namespace {

void fail_request(deepinv_server* s, const Req& r, int status)
{
    deepinv_result res{};
    res.tag = r.tag;
    res.status = status;
    res.net_id = r.net;
    res.batch = 0;
    const auto now = Clock::now();
    res.queue_us = us_between(r.t_submit, now);
    res.latency_us = res.queue_us;
    s->done.push_back(res);
    s->stats.failed++;
    s->outstanding--;
}

// A workspace for network `net`: reuse an idle one, else allocate after
// releasing idle workspaces of other networks while the budget demands.
// Returns nullptr if it does not fit now.
Lease* acquire(deepinv_server* s, int net, cudaStream_t st)
{
    if (!s->cache[net].empty()) {
        Lease* l = s->cache[net].back();
        s->cache[net].pop_back();
        return l;
    }
    const size_t need = s->lease_bytes[net];
    for (size_t other = 0; other < s->cache.size() && s->held + need > s->budget; ++other) {
        while (!s->cache[other].empty() && s->held + need > s->budget) {
            Lease* l = s->cache[other].back();
            s->cache[other].pop_back();
            cudaFreeAsync(l->ws, st);
            s->held -= l->bytes;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                s->stats.evictions++;
                s->stats.workspace_bytes = s->held;
            }
            delete l;
        }
    }
    if (s->held + need > s->budget) return nullptr;
    char* p = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void**>(&p), need, st) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    // zero once: the planes' borders must be zero and are never written
    if (cudaMemsetAsync(p, 0, need, st) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeAsync(p, st);
        return nullptr;
    }
    s->held += need;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stats.workspace_bytes = s->held;
        s->stats.peak_workspace_bytes = std::max(s->stats.peak_workspace_bytes, s->held);
    }
    Lease* l = new Lease{net, p, need};
    return l;
}

// Copies a finished batch's results into the requests' host buffers and builds
// their result records, without the server lock (the slot and its requests
// belong to the scheduler thread; a caller does not touch a request's buffer
// before its result is handed back).
void collect_slot(deepinv_server* s, Slot& sl, int status, std::vector<deepinv_result>& out)
{
    const int N = net_N(s->nets[sl.net]);
    const auto now = Clock::now();
    if (status == DEEPINV_OK) {
        const std::function<void(int)> copy = [&](int i) {
            std::memcpy(sl.reqs[i].xhat, sl.x_pin + (size_t)i * N, (size_t)N * sizeof(float));
        };
        const int b = (int)sl.reqs.size();
        if ((size_t)b * N * sizeof(float) >= kParallelCopyBytes) s->copies.run(b, copy);
        else
            for (int i = 0; i < b; ++i) copy(i);
    }
    for (size_t i = 0; i < sl.reqs.size(); ++i) {
        Req& r = sl.reqs[i];
        deepinv_result res{};
        res.tag = r.tag;
        res.status = status;
        res.net_id = r.net;
        res.batch = (int)sl.reqs.size();
        res.queue_us = us_between(r.t_submit, sl.t_launch);
        res.latency_us = us_between(r.t_submit, status == DEEPINV_OK ? Clock::now() : now);
        out.push_back(res);
    }
    sl.reqs.clear();
    if (sl.lease) s->cache[sl.net].push_back(sl.lease);
    sl.lease = nullptr;
    sl.busy = false;
    sl.net = -1;
}

// Hands finished results to the callers (lock held).
void publish(deepinv_server* s, std::vector<deepinv_result>& res)
{
    for (const deepinv_result& r : res) {
        s->done.push_back(r);
        if (r.status == DEEPINV_OK) s->stats.completed++;
        else s->stats.failed++;
        s->outstanding--;
    }
    res.clear();
}

// Launches the batch already moved into sl.reqs (network `net`, workspace
// `lease`) on slot `sl`, without the server lock: staging copy, input copy,
// forward pass, output copy and the slot's completion event.  On failure the
// batch's failed results are appended to `failed`.
int launch(deepinv_server* s, Slot& sl, int net, Lease* lease, std::vector<deepinv_result>& failed)
{
    deepinv_net* n = s->nets[net];
    const int M = net_M(n), N = net_N(n);
    const int b = (int)sl.reqs.size();
    const std::function<void(int)> stage = [&](int i) {
        std::memcpy(sl.y_pin + (size_t)i * M, sl.reqs[i].y.data(), (size_t)M * sizeof(float));
    };
    if ((size_t)b * M * sizeof(float) >= kParallelCopyBytes) s->copies.run(b, stage);
    else
        for (int i = 0; i < b; ++i) stage(i);
    sl.net = net;
    sl.lease = lease;
    sl.t_launch = Clock::now();
    float *yd = nullptr, *xd = nullptr;
    net_ws_staging(n, lease->ws, s->max_batch, &yd, &xd);
    int rc = DEEPINV_OK;
    if (cudaMemcpyAsync(yd, sl.y_pin, (size_t)b * M * sizeof(float), cudaMemcpyHostToDevice, sl.st) != cudaSuccess)
        rc = DEEPINV_ECUDA;
    if (rc == DEEPINV_OK) rc = net_forward_ws(n, lease->ws, s->max_batch, yd, b, xd, sl.st);
    if (rc == DEEPINV_OK &&
        cudaMemcpyAsync(sl.x_pin, xd, (size_t)b * N * sizeof(float), cudaMemcpyDeviceToHost, sl.st) != cudaSuccess)
        rc = DEEPINV_ECUDA;
    if (rc == DEEPINV_OK && cudaEventRecord(sl.ev, sl.st) != cudaSuccess) rc = DEEPINV_ECUDA;
    if (rc != DEEPINV_OK) {
        cudaGetLastError();
        collect_slot(s, sl, rc, failed);
        return rc;
    }
    sl.busy = true;
    return DEEPINV_OK;
}

// The scheduler thread.  It owns the slots, the workspace cache and the
// budget accounting; the server lock guards only what callers share with it
// (the pending queues, the finished results, the counters), so that copying
// results, staging inputs, allocating a workspace and enqueueing a batch never
// keep a caller's submit or harvest waiting.
void scheduler(deepinv_server* s)
{
    cudaSetDevice(s->dev);
    {
        const unsigned hw = std::thread::hardware_concurrency();
        s->copies.start(hw >= 8 ? 3 : (hw >= 4 ? 1 : 0));
    }
    std::vector<deepinv_result> ready;
    auto last_progress = std::chrono::steady_clock::now();
    while (true) {
        bool progressed = false;
        // 1. collect finished batches (results copied out without the lock)
        for (Slot& sl : s->slots) {
            if (!sl.busy) continue;
            const cudaError_t e = cudaEventQuery(sl.ev);
            if (e == cudaErrorNotReady) continue;
            if (e != cudaSuccess) cudaGetLastError();
            collect_slot(s, sl, e == cudaSuccess ? DEEPINV_OK : DEEPINV_ECUDA, ready);
            progressed = true;
        }
        // 2. start batches on free streams, oldest waiting network first
        bool blocked = false;
        for (Slot& sl : s->slots) {
            if (sl.busy || blocked) continue;
            int best = -1;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                if (!ready.empty()) {
                    publish(s, ready);
                    s->cv_done.notify_all();
                }
                for (size_t k = 0; k < s->pending.size(); ++k)
                    if (!s->pending[k].empty() &&
                        (best < 0 || s->pending[k].front().t_submit < s->pending[best].front().t_submit))
                        best = (int)k;
                if (best < 0) break;
                if (s->lease_bytes[best] > s->budget) {
                    // can never fit: fail this network's waiting requests
                    while (!s->pending[best].empty()) {
                        fail_request(s, s->pending[best].front(), DEEPINV_ENOMEM);
                        s->pending[best].pop_front();
                    }
                    s->cv_done.notify_all();
                    progressed = true;
                    continue;
                }
            }
            // workspace lease (may allocate) outside the lock
            Lease* l = acquire(s, best, sl.st);
            if (!l) {
                std::lock_guard<std::mutex> lk(s->mu);
                if (!s->waiting_admission) s->stats.admission_waits++;
                s->waiting_admission = true;
                blocked = true;
                continue;
            }
            {
                std::lock_guard<std::mutex> lk(s->mu);
                s->waiting_admission = false;
                std::deque<Req>& q = s->pending[best];
                const size_t b = std::min<size_t>(q.size(), (size_t)s->max_batch);
                sl.reqs.clear();
                for (size_t i = 0; i < b; ++i) {
                    sl.reqs.push_back(std::move(q.front()));
                    q.pop_front();
                }
                s->stats.batches++;
            }
            if (launch(s, sl, best, l, ready) == DEEPINV_OK) {
                int inflight = 0;
                for (const Slot& o : s->slots) inflight += o.busy ? 1 : 0;
                std::lock_guard<std::mutex> lk(s->mu);
                s->stats.max_in_flight = std::max(s->stats.max_in_flight, inflight);
            }
            progressed = true;
        }
        bool any_busy = false, any_pending = false;
        for (const Slot& sl : s->slots) any_busy |= sl.busy;
        std::unique_lock<std::mutex> lk(s->mu);
        if (!ready.empty()) {
            publish(s, ready);
            s->cv_done.notify_all();
        }
        for (const auto& q : s->pending) any_pending |= !q.empty();
        if (s->stop && !any_busy && !any_pending) break;
        if (progressed) {
            last_progress = std::chrono::steady_clock::now();
            continue;
        }
        if (any_busy) {
            lk.unlock();
            // batches in flight: poll their events by yielding (a sleep of a few
            // microseconds lasts tens of them on a loaded host) for up to 2 ms after
            // the last progress, then sleep between polls
            if (std::chrono::steady_clock::now() - last_progress < std::chrono::milliseconds(2))
                std::this_thread::yield();
            else
                std::this_thread::sleep_for(std::chrono::microseconds(10));
        } else {
            s->cv_work.wait_for(lk, std::chrono::milliseconds(20));
        }
    }
    s->copies.shutdown();
    std::lock_guard<std::mutex> lk(s->mu);
    s->cv_done.notify_all();
}

int ensure_slots(deepinv_server* s)
{
    for (Slot& sl : s->slots) {
        if (!sl.st) {
            DI_CUDA(cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking));
            DI_CUDA(cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming));
        }
        if (sl.y_pin) cudaFreeHost(sl.y_pin);
        if (sl.x_pin) cudaFreeHost(sl.x_pin);
        sl.y_pin = sl.x_pin = nullptr;
        if (cudaMallocHost(&sl.y_pin, (size_t)s->max_batch * s->maxM * sizeof(float)) != cudaSuccess ||
            cudaMallocHost(&sl.x_pin, (size_t)s->max_batch * s->maxN * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            set_error("serve: page-locked staging allocation failed");
            return DEEPINV_ENOMEM;
        }
    }
    return DEEPINV_OK;
}

}  // namespace

extern "C" {

int deepinv_serve_open(size_t hbm_budget_bytes, int max_streams, int max_batch, deepinv_server** out)
{
    DI_REQUIRE(out, "out is NULL");
    DI_REQUIRE(max_streams >= 1 && max_streams <= 16, "max_streams %d not in 1..16", max_streams);
    DI_REQUIRE(max_batch >= 1 && max_batch <= 1024, "max_batch %d not in 1..1024", max_batch);
    deepinv_server* s = new (std::nothrow) deepinv_server();
    DI_REQUIRE(s, "host allocation failed");
    s->budget = hbm_budget_bytes;
    s->max_streams = max_streams;
    s->max_batch = max_batch;
    s->slots.resize(max_streams);
    *out = s;
    return DEEPINV_OK;
}

int deepinv_serve_add_net(deepinv_server* s, deepinv_net* net, int* net_id)
{
    DI_REQUIRE(s && net && net_id, "null pointer");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->outstanding > 0) {
        set_error("serve_add_net: requests are in flight");
        return DEEPINV_EBUSY;
    }
    const int dev = net_device(net);
    DI_REQUIRE(s->dev < 0 || s->dev == dev, "network on device %d, server on device %d", dev, s->dev);
    s->dev = dev;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(dev);
    s->nets.push_back(net);
    s->lease_bytes.push_back(net_ws_bytes(net, s->max_batch));
    s->pending.emplace_back();
    s->cache.emplace_back();
    s->maxM = std::max(s->maxM, net_M(net));
    s->maxN = std::max(s->maxN, net_N(net));
    int rc = ensure_slots(s);
    if (prev >= 0) cudaSetDevice(prev);
    if (rc != DEEPINV_OK) {
        s->nets.pop_back();
        s->lease_bytes.pop_back();
        s->pending.pop_back();
        s->cache.pop_back();
        return rc;
    }
    *net_id = (int)s->nets.size() - 1;
    // Workspaces for this network's batches, one per stream while the budget
    // allows, are allocated here rather than when a batch first needs them: a
    // fresh allocation can take milliseconds (the stream-ordered pool growing),
    // and the scheduler would hold back every network's batches meanwhile.  The
    // pool keeps released memory, so that a workspace evicted and leased again
    // under a tight budget is quick to get back.
    {
        cudaSetDevice(dev);
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
        const int id = *net_id;
        const size_t need = s->lease_bytes[id];
        cudaStream_t st0 = s->slots[0].st;
        for (int k = 0; k < s->max_streams && s->held + need <= s->budget; ++k) {
            char* p = nullptr;
            if (cudaMallocAsync(reinterpret_cast<void**>(&p), need, st0) != cudaSuccess) {
                cudaGetLastError();
                break;
            }
            if (cudaMemsetAsync(p, 0, need, st0) != cudaSuccess) {   // zero borders, written once
                cudaGetLastError();
                cudaFreeAsync(p, st0);
                break;
            }
            s->cache[id].push_back(new Lease{id, p, need});
            s->held += need;
        }
        cudaStreamSynchronize(st0);
        cudaGetLastError();
        s->stats.workspace_bytes = s->held;
        s->stats.peak_workspace_bytes = std::max(s->stats.peak_workspace_bytes, s->held);
        if (prev >= 0) cudaSetDevice(prev);
    }
    if (!s->started) {
        s->started = true;
        s->thr = std::thread(scheduler, s);
    }
    return DEEPINV_OK;
}

int deepinv_serve(deepinv_server* s, const deepinv_request* in, int n_in, deepinv_result* out, int max_out,
                  int* n_out, int timeout_us)
{
    DI_REQUIRE(s && n_out, "null pointer");
    DI_REQUIRE(n_in >= 0 && max_out >= 0 && timeout_us >= 0, "negative count or timeout");
    DI_REQUIRE(n_in == 0 || in, "requests pointer is NULL");
    DI_REQUIRE(max_out == 0 || out, "results pointer is NULL");
    *n_out = 0;
    // the requests' measurements are copied between two short holds of the lock
    // (the first reads each request's measurement count)
    std::vector<Req> reqs;
    if (n_in > 0) {
        std::vector<int> m(n_in);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            const int nnets = (int)s->nets.size();
            for (int i = 0; i < n_in; ++i) {
                const deepinv_request& r = in[i];
                DI_REQUIRE(r.net_id >= 0 && r.net_id < nnets, "request %d: unknown net_id %d", i, r.net_id);
                DI_REQUIRE(r.y && r.xhat, "request %d: null y or xhat", i);
                m[i] = net_M(s->nets[r.net_id]);
            }
        }
        reqs.resize(n_in);
        const auto now = Clock::now();
        for (int i = 0; i < n_in; ++i) {
            const deepinv_request& r = in[i];
            Req& q = reqs[i];
            q.net = r.net_id;
            q.tag = r.tag;
            q.xhat = r.xhat;
            q.y.assign(r.y, r.y + m[i]);
            q.t_submit = now;
        }
    }
    std::unique_lock<std::mutex> lk(s->mu);
    for (Req& q : reqs) {
        const int net = q.net;
        s->pending[net].push_back(std::move(q));
        s->stats.submitted++;
        s->outstanding++;
    }
    if (n_in > 0) s->cv_work.notify_one();
    if (max_out == 0) return DEEPINV_OK;
    if (s->done.empty() && timeout_us > 0 && s->outstanding > 0)
        s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [s] { return !s->done.empty(); });
    int n = 0;
    while (n < max_out && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    *n_out = n;
    if (n == 0 && timeout_us > 0 && s->outstanding > 0) {
        set_error("serve: no request finished within %d us", timeout_us);
        return DEEPINV_ETIMEOUT;
    }
    return DEEPINV_OK;
}

int deepinv_serve_get_stats(deepinv_server* s, deepinv_serve_stats* st)
{
    DI_REQUIRE(s && st, "null pointer");
    std::lock_guard<std::mutex> lk(s->mu);
    *st = s->stats;
    return DEEPINV_OK;
}

int deepinv_serve_close(deepinv_server* s)
{
    if (!s) return DEEPINV_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->thr.joinable()) s->thr.join();
    if (s->dev >= 0) cudaSetDevice(s->dev);
    for (Slot& sl : s->slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
    }
    cudaStream_t fs = s->slots.empty() ? nullptr : s->slots[0].st;
    for (auto& c : s->cache)
        for (Lease* l : c) {
            cudaFreeAsync(l->ws, fs);
            delete l;
        }
    for (Slot& sl : s->slots) {
        if (sl.lease) {
            cudaFreeAsync(sl.lease->ws, fs);
            delete sl.lease;
        }
    }
    if (fs) cudaStreamSynchronize(fs);
    for (Slot& sl : s->slots) {
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.st) cudaStreamDestroy(sl.st);
        if (sl.y_pin) cudaFreeHost(sl.y_pin);
        if (sl.x_pin) cudaFreeHost(sl.x_pin);
    }
    delete s;
    return DEEPINV_OK;
}

}  // extern "C"
