/*
 * deepinv.h -- C ABI of libdeepinv.so, the GB300 (sm_103a) hot path of
 * DeepInverse (Mousavi & Baraniuk, "Learning to Invert: Signal Recovery via
 * Deep Convolutional Networks", arXiv 1701.03891).
 *
 * The library recovers signals x in R^N from undersampled linear measurements
 * y = Phi x in R^M (Sec. 1) with the network of Sec. 4: a fully connected
 * layer fixed to Phi^T (x~ = Phi^T y, reshaped to n1 x n2), then three
 * convolutional layers, Eq. (1), with 64, 32 and 1 filters of 11 x 11
 * (Sec. 5), optionally with more 32-filter layers before the last (the
 * deeper networks Sec. 5 leaves to future work).  It also trains that network
 * on the MSE loss of Sec. 4.
 *
 * Conventions shared by every call:
 *  - Tensor arguments are DEVICE pointers owned by the caller, contiguous,
 *    row-major float32 unless stated otherwise.  Images are stored row-major,
 *    pixel j = r * n2 + c (the reshape of Sec. 4).  The library never frees
 *    caller memory and keeps no caller pointer after a call returns, except
 *    deepinv_sense_recover_host_submit's host buffers until their ticket
 *    completes.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Every
 *    call is asynchronous on that stream unless its comment says otherwise.
 *  - Arguments are checked before any launch; a batch B is at most 2^30
 *    images.  A negative return value is a
 *    deepinv_status and deepinv_last_error() returns a message for the calling
 *    thread; after DEEPINV_EINVAL or DEEPINV_EUNSUPPORTED the outputs are
 *    untouched, after DEEPINV_ECUDA their contents are undefined.
 *  - No call aborts the process or traps the GPU.  Waits inside kernels are
 *    bounded; a wait that runs out makes the call report DEEPINV_ETIMEOUT
 *    through deepinv_device_status().
 *  - Precision: DEEPINV_F32 runs every product in float32 on CUDA cores;
 *    DEEPINV_BF16 runs the FC layer and the convolutions on the tcgen05 tensor
 *    cores with bfloat16 operands (round to nearest even) and float32
 *    accumulation; DEEPINV_FP8_E4M3 is the bf16 path with conv2 (95 % of the
 *    flops) on e4m3 operands: weights scaled per filter (max |w| -> 448), the
 *    conv1 output scaled by one static factor found by deepinv_net_calibrate,
 *    float32 accumulation; it is inference only.
 */
#ifndef DEEPINV_H
#define DEEPINV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DEEPINV_OK = 0,
    DEEPINV_EINVAL = -1,       /* bad argument: null pointer, bad size, bad shape */
    DEEPINV_ENOMEM = -2,       /* device allocation failed */
    DEEPINV_ECUDA = -3,        /* a CUDA runtime call failed (message in deepinv_last_error) */
    DEEPINV_EUNSUPPORTED = -4, /* valid request the library has no kernel for */
    DEEPINV_ETIMEOUT = -5,     /* a bounded wait ran out (in a kernel or in the server) */
    DEEPINV_EBUSY = -6         /* the server has requests in flight (deepinv_serve_add_net) */
} deepinv_status;

typedef enum {
    DEEPINV_F32 = 0,
    DEEPINV_BF16 = 1,
    DEEPINV_FP8_E4M3 = 2   /* bf16 path with conv2 in e4m3 (see deepinv_net_calibrate) */
} deepinv_precision;

/* Network shape (Sec. 4 and Sec. 5).  The paper's network is
 * l1 = 64, l2 = 32, l3 = 1, k = 11; the BF16 path requires exactly that,
 * the F32 path accepts any l1, l2 >= 1 and odd k <= 15 (l3 = 1 always: the
 * output is the one-channel image). */
typedef struct {
    int n1, n2;      /* image rows and columns, N = n1 * n2 */
    int M;           /* number of measurements, 1 <= M <= N */
    int l1, l2, l3;  /* filters of conv1, conv2, conv3 */
    int k;           /* square kernel size, odd */
    int final_relu;  /* 1: ReLU after conv3 as well (the paper's "each layer") */
    int train_fc;    /* 1: the FC weights are a trainable copy initialised to Phi^T */
    int prec;        /* deepinv_precision */
    int hidden;      /* extra l2 -> l2 conv layers (k x k, ReLU) between conv2 and
                        conv3, 0..DEEPINV_MAX_HIDDEN; 0 is the paper's network.
                        The network then has L = 3 + hidden conv layers, and every
                        per-layer array below has L entries in network order:
                        conv1, conv2, hidden 1..hidden, conv3 (the deeper networks
                        of larger capacity that Sec. 5 leaves to future work). */
} deepinv_net_desc;

#define DEEPINV_MAX_HIDDEN 16

typedef struct deepinv_net deepinv_net;       /* opaque; owns weights and workspace */

/* Message for the last non-OK status returned on the calling thread. */
const char* deepinv_last_error(void);

/* Library ABI version (major * 100 + minor). */
int deepinv_version(void);

/* Sticky device-side status of the library: DEEPINV_OK, or DEEPINV_ETIMEOUT
 * if a bounded wait in a kernel ran out since the last reset, on any device
 * the library has used (the status words of the network and measurement
 * calls and of deepinv_measure_noalloc).  Synchronises those devices.
 * `reset` != 0 clears the words. */
int deepinv_device_status(int reset);

/* Number of kernels the library has launched in this process so far (every
 * launch of every entry point, counted on the host as it is issued); a
 * caller takes the difference around a region to count its launches.  No
 * counterpart in the paper. */
unsigned long long deepinv_launch_count(void);

/* Failure-path check of the device status word (no counterpart in the paper):
 * launches one kernel on the current device whose bounded wait is never
 * satisfied; after the wait's time limit (about 1 s) it records a timeout and
 * returns without a fault, so the context stays usable.  Waits for it.
 * deepinv_device_status() then reports DEEPINV_ETIMEOUT until reset. */
int deepinv_selftest_bounded_wait(void* stream);

/* y = Phi x for B signals (Sec. 1).
 * phi [M][N], x [B][N] -> y [B][M], all float32 device memory.
 * prec selects float32 CUDA-core products or bfloat16 tensor-core products
 * with float32 accumulation.  1 <= M, N <= 2^30 and 0 <= B <= 2^30 (B == 0 is
 * a no-op); other sizes return DEEPINV_EINVAL. */
int deepinv_measure(const float* phi, int M, int N, const float* x, int B, float* y,
                    int prec, void* stream);

/* y = Phi x on the bfloat16 tensor cores, like deepinv_measure(..., DEEPINV_BF16),
 * but without any device allocation (the paper has no counterpart; this is a
 * service to callers).  It is meant for callers that cannot let a library
 * allocate device memory: processes that split their device memory once at
 * start-up into fixed budgets, real-time loops that must not reach the
 * allocator after initialisation, and hosts that install their own allocator.
 *
 * phi [M][N], x [B][N] -> y [B][M], float32 device memory owned by the caller,
 * as in deepinv_measure; the result is the same as deepinv_measure with
 * DEEPINV_BF16.  The bfloat16 operand tiles live in one static device array of
 * 32 MiB (minus a 256-byte header) that every device which loads the library
 * holds until the process exits; requests whose packed operands,
 * 2 (ceil(M / NB) NB + ceil(B / 128) 128) ceil16(N) bytes with
 * NB = ceil16(M / ceil(M / 256)), do not fit are rejected with DEEPINV_EINVAL
 * before anything is launched (M = 410, N = 4096 fits up to B = 3584).
 *
 * phi may also be managed memory; its device is the one the call runs on.
 *
 * Every call looks the array's device address up (cudaGetSymbolAddress); the
 * first call on a device (and the first after a device reset gave the array a
 * new address) also clears its header, synchronously, so make that first call
 * before any stream capture.  All calls on a device share the array and it
 * keeps the last call's contents, so calls whose work overlaps on the GPU
 * (different streams without ordering) race and may return wrong results.  A
 * bounded wait that runs out inside this call is recorded in the array's
 * header, and deepinv_device_status() reports it (DEEPINV_ETIMEOUT) like any
 * other; its reset clears it. */
int deepinv_measure_noalloc(const float* phi, int M, int N, const float* x, int B, float* y,
                            void* stream);

/* Create a network (Sec. 4).  phi [M][N] is copied (it defines the FC layer,
 * x~ = Phi^T y); w[l] is [c_out][c_in][k][k] and b[l] is [c_out] for the
 * L = 3 + desc->hidden layers l = 0 .. L-1 in network order (conv1: 1 -> l1,
 * conv2: l1 -> l2, each hidden layer: l2 -> l2, conv3: l2 -> l3), all device
 * float32, copied into float32 master weights plus the kernel layouts of
 * desc->prec.  Synchronises `stream`.  On success *out owns device memory
 * until deepinv_net_destroy. */
int deepinv_net_create(const deepinv_net_desc* desc, const float* phi,
                       const float* const w[], const float* const b[],
                       void* stream, deepinv_net** out);

/* Fix the activation scale of a DEEPINV_FP8_E4M3 network: run the FC layer
 * and conv1 on the calibration batch y [B][M] (device float32) and map the
 * largest conv1 output to the largest finite e4m3 value (448); later values
 * above it saturate.  Required once before the first forward pass of such a
 * network (weight updates keep it).  Synchronises `stream`.  A no-op for the
 * other precisions. */
int deepinv_net_calibrate(deepinv_net* net, const float* y, int B, void* stream);

/* Free everything the network owns.  Synchronises the device.  NULL is a no-op. */
int deepinv_net_destroy(deepinv_net* net);

/* Copy out the description the network was created with. */
int deepinv_net_get_desc(const deepinv_net* net, deepinv_net_desc* desc);

/* Make the network's workspace large enough for batches up to max_B so that
 * later calls with B <= max_B allocate nothing.  Synchronises `stream`. */
int deepinv_net_reserve(deepinv_net* net, int max_B, void* stream);

/* y = Phi x with the network's own Phi (kept in the layout of its precision).
 * x [B][N] -> y [B][M]. */
int deepinv_net_measure(deepinv_net* net, const float* x, int B, float* y, void* stream);

/* Bytes of the buffer deepinv_forward fills for deepinv_backward at batch B. */
size_t deepinv_saved_bytes(const deepinv_net* net, int B);

/* Activation budget, in bytes, of a deepinv_backward called without a saved
 * buffer: it recomputes the forward pass in chunks of as many images as have
 * activations (deepinv_saved_bytes) within `bytes` (at least one image per
 * chunk; 0, the default, means the whole batch at once).  The library keeps
 * one chunk's activations and, with more than one chunk, scratch for one set
 * of gradients.  Trades one extra forward pass for memory when B x image size
 * would not fit. */
int deepinv_net_set_act_budget(deepinv_net* net, size_t bytes);

/* Runs the first two layers of Eq. (1) (conv1 + ReLU, conv2 + ReLU) as one
 * fused kernel in the inference forward pass of a bfloat16 network (enable =
 * 1) instead of two (0, the default).  The fused kernel keeps conv1's output
 * in shared memory instead of writing it to HBM and reading it back: each CTA
 * walks a run of conv2 tiles and produces conv1's output for the rows ahead
 * of it once.  Images up to 70 columns are walked whole; wider ones as column
 * strips of at most 55 columns, whose halos cost extra conv2 work.  The
 * result is bit-identical to the two-kernel path.  Forward passes that save
 * activations for deepinv_backward, e4m3 and float32 networks keep the
 * two-kernel path.  With the profiler on, the fused kernel is timed as
 * DEEPINV_STAGE_CONV2 (DEEPINV_STAGE_CONV1 then counts nothing).  Returns
 * DEEPINV_EINVAL for a NULL net. */
int deepinv_net_set_fused(deepinv_net* net, int enable);

/* Chooses between two kernels for conv1 (the first layer of Eq. (1), 1 -> 64
 * filters of 11 x 11, bias and ReLU) in bfloat16 and e4m3 networks.  Row tiles
 * keep conv1's shifted input windows in tensor memory, where each serves the
 * tiles of several rows (segments of at most 128 image columns, at most 5 rows
 * per tile); the other kernel takes tiles of 128 consecutive plane positions.
 * mode 0: never row tiles; 1 (the default): row tiles where they are faster
 * (one row of at least 120 columns per tile, e.g. 128 or 256 columns); 2: row
 * tiles wherever they fill at least 96 of a tile's 128 positions.  Both kernels
 * issue the same products in the same order and give bit-identical results.
 * Returns DEEPINV_EINVAL for a NULL net or a mode outside 0..2. */
int deepinv_net_set_conv1_rows(deepinv_net* net, int mode);

/* x^ = M(y, Omega) (Sec. 4): FC layer, reshape to n1 x n2, conv1 + ReLU,
 * conv2 + ReLU, each hidden layer + ReLU, conv3 (+ ReLU when final_relu).
 * y [B][M] -> xhat [B][N].  `saved` is NULL for inference, or a device buffer
 * of deepinv_saved_bytes(net, B) bytes that receives the activations the
 * backward pass needs.  Uses the network's workspace (grown if B exceeds the
 * reserved batch, which synchronises); calls on one network must not overlap
 * on different streams. */
int deepinv_forward(deepinv_net* net, const float* y, int B, float* xhat, void* saved,
                    void* stream);

/* End to end on HOST memory: copy y_host [B][M] to the device, run
 * deepinv_forward, copy x^ back to xhat_host [B][N], and wait for the copy.
 * Host buffers should be page-locked for asynchronous copies. */
int deepinv_forward_host(deepinv_net* net, const float* y_host, int B, float* xhat_host,
                         void* stream);

/* Sense and recover on HOST memory: x_host [B][N] -> y = Phi x on the device
 * -> x^ -> xhat_host [B][N]; waits for the result. */
int deepinv_sense_recover_host(deepinv_net* net, const float* x_host, int B, float* xhat_host,
                               void* stream);

/* Asynchronous form of deepinv_sense_recover_host for a stream of batches:
 * queues the copy of x_host [B][N] to the device, y = Phi x, x^ and the copy of
 * x^ to xhat_host [B][N], and returns at once with *ticket.  The network keeps
 * two device staging slots, so a batch's copies overlap the compute of the
 * batches before and after it; the compute runs on `stream`, the copies on
 * the network's own streams.  Host buffers must be page-locked and stay
 * untouched until the ticket completes; all submissions and other calls on
 * one network must use the same stream.  Errors found while queueing are
 * returned; a bounded wait that runs out in a kernel shows in
 * deepinv_device_status(). */
int deepinv_sense_recover_host_submit(deepinv_net* net, const float* x_host, int B, float* xhat_host,
                                      void* stream, uint64_t* ticket);

/* Wait until the batch of `ticket` has its x^ in host memory. */
int deepinv_host_wait(deepinv_net* net, uint64_t ticket);

/* Gradient of L(Omega) = (1/B) sum_b ||x^_b - x_b||^2 (Sec. 4) by
 * backpropagation.  y [B][M] and x [B][N] are the batch; `saved` is the
 * buffer a deepinv_forward of this same y filled, or NULL: then the forward
 * activations are recomputed here, in chunks of images whose activations fit
 * the network's activation budget (deepinv_net_set_act_budget; one chunk when
 * it is 0), the chunks' gradients added in chunk order.  Writes dW[l] (shape
 * of w[l]), db[l] (shape of b[l]), dWfc [N][M] (only when train_fc; else pass
 * NULL) and *loss (one device double).  All outputs are overwritten. */
int deepinv_backward(deepinv_net* net, const float* y, const float* x, int B, const void* saved,
                     float* const dW[], float* const db[], float* dWfc, double* loss,
                     void* stream);

/* One SGD-with-momentum step on the float32 master weights:
 * v <- mu v + g ; w <- w - lr v (momentum buffers live in the network, zero at
 * creation), then refresh the kernel-layout copies.  dWfc is used only when
 * train_fc. */
int deepinv_sgd_momentum(deepinv_net* net, const float* const dW[], const float* const db[],
                         const float* dWfc, float lr, float mu, void* stream);

/* Checkpoint / resume of training.  save_state writes the float32 master
 * weights, their SGD momentum buffers and (with train_fc) the FC weights and
 * momentum to a binary file under `path` (a header with the network's
 * description, then the arrays); it synchronises the device.  load_state reads
 * such a file into a network created with the same description (the precision
 * may differ), refreshes the kernel layouts and synchronises `stream`; a file
 * of another network or a truncated file returns DEEPINV_EINVAL and may leave
 * the network partly updated.  Training resumed from a saved state continues
 * bit for bit as if it had not stopped. */
int deepinv_net_save_state(deepinv_net* net, const char* path);
int deepinv_net_load_state(deepinv_net* net, const char* path, void* stream);

/* Copy the float32 master weights out (any pointer may be NULL to skip it);
 * wfc is [N][M] and is only available when train_fc. */
int deepinv_get_params(const deepinv_net* net, float* const w[], float* const b[], float* wfc,
                       void* stream);

/* ------------------------------------------------------------------ serving
 * Low-latency recovery (Sec. 5: DeepInverse suits applications that need
 * low-latency recovery) as a continuous-batching server inside the library.
 * A scheduler thread keeps requests in one queue per network; whenever one of
 * the server's CUDA streams is free it takes up to max_batch waiting requests
 * of the network whose oldest request has waited longest, and runs them as one
 * batch on that stream, so batches of different networks (image sizes, M/N)
 * overlap on the device and requests that arrive while others run join the
 * next batch.  The scheduler never holds the lock that submission and
 * harvest take while it copies data, allocates or enqueues work.  Each batch
 * needs a workspace of that network for max_batch
 * images; workspaces are kept for reuse and count against the HBM budget,
 * idle ones of other networks are released when a new one does not fit, and
 * a batch waits while its workspace does not fit; requests of a network whose
 * workspace exceeds the whole budget finish with status DEEPINV_ENOMEM.
 * Results do not depend on the batch a request ran in. */
typedef struct deepinv_server deepinv_server;  /* opaque */

typedef struct {
    int net_id;         /* from deepinv_serve_add_net */
    const float* y;     /* HOST [M] measurement of that network; read before deepinv_serve returns */
    float* xhat;        /* HOST [N] result; written before the request's result is returned */
    uint64_t tag;       /* caller's identifier, echoed in the result */
} deepinv_request;

typedef struct {
    uint64_t tag;
    int status;         /* DEEPINV_OK, or the error that failed the request */
    int net_id;
    int batch;          /* number of requests in the batch it ran in */
    double queue_us;    /* submission -> batch launch */
    double latency_us;  /* submission -> result written to xhat */
} deepinv_result;

/* Create a server; it runs on the device of the first network added.
 * hbm_budget_bytes bounds the device memory its workspaces may hold;
 * max_streams (1..16) batches may be in flight at once; max_batch (1..1024)
 * requests per batch.  No device work happens until a network is added. */
int deepinv_serve_open(size_t hbm_budget_bytes, int max_streams, int max_batch, deepinv_server** out);

/* Register a network (not owned; it must outlive the server and must not be
 * used by the caller while the server runs).  All networks of a server live
 * on one device.  Add networks before the first request; returns
 * DEEPINV_EBUSY while requests are in flight.  Synchronously allocates (and
 * zeroes) up to max_streams workspaces for the network while they fit in the
 * budget, so that batches do not wait on allocations later; the device's
 * default stream-ordered memory pool is set to keep released memory. */
int deepinv_serve_add_net(deepinv_server* s, deepinv_net* net, int* net_id);

/* Submit n_in requests (copied; n_in may be 0), then return up to max_out
 * finished results (in completion order), waiting up to timeout_us for at
 * least one when none is ready (timeout_us = 0: do not wait).  *n_out is the
 * number returned.  Returns DEEPINV_ETIMEOUT if the wait ran out with nothing
 * finished while requests were pending, DEEPINV_EINVAL for a bad request
 * (nothing of this call is submitted). */
int deepinv_serve(deepinv_server* s, const deepinv_request* in, int n_in,
                  deepinv_result* out, int max_out, int* n_out, int timeout_us);

typedef struct {
    uint64_t submitted, completed, failed;
    uint64_t batches;
    int max_in_flight;        /* largest number of concurrent batches seen */
    size_t workspace_bytes;   /* device memory held for workspaces now */
    size_t peak_workspace_bytes;
    uint64_t evictions;       /* idle workspaces released to make room */
    uint64_t admission_waits; /* times a batch waited for its workspace to fit */
} deepinv_serve_stats;

int deepinv_serve_get_stats(deepinv_server* s, deepinv_serve_stats* st);

/* Finish every submitted request, stop the scheduler and free the server's
 * memory.  Results not yet harvested are dropped.  NULL is a no-op. */
int deepinv_serve_close(deepinv_server* s);

/* Stages of the forward pass timed by the profiler. */
#define DEEPINV_NSTAGES 6
enum {
    DEEPINV_STAGE_MEASURE = 0, /* y = Phi x (deepinv_net_measure) */
    DEEPINV_STAGE_FC = 1,      /* x~ = Phi^T y, written in the conv1 input layout */
    DEEPINV_STAGE_CONV1 = 2,
    DEEPINV_STAGE_CONV2 = 3,
    DEEPINV_STAGE_CONV3 = 4,
    DEEPINV_STAGE_HIDDEN = 5   /* all hidden layers of a deeper network */
};

/* Profiling of the network's calls by CUDA events.  While enabled,
 * deepinv_net_measure and deepinv_forward record an event before and after
 * each stage on the caller's stream (no synchronisation).  Enabling or
 * disabling clears what was recorded. */
int deepinv_profile_enable(deepinv_net* net, int enable);

/* Wait for the recorded events and return, per stage, the summed device
 * milliseconds and the number of recorded executions (either array may be
 * NULL); then clear the record. */
int deepinv_profile_read(deepinv_net* net, float stage_ms[DEEPINV_NSTAGES],
                         int stage_count[DEEPINV_NSTAGES]);

#ifdef __cplusplus
}
#endif

#endif /* DEEPINV_H */
