// float32 CUDA-core kernels of libdeepinv: the DEEPINV_F32 path of the
// measurement (Sec. 1), the FC layer and the convolutions of Eq. (1), and the
// backward pass of the MSE loss of Sec. 4 (used by both precisions).
//
// Layout: planar NCHW float32, images row-major (pixel j = r * n2 + c).
#include "kernels.cuh"

namespace di {

// ---------------------------------------------------------------- GEMM
// C[m][n] = sum_k A(m, k) B(k, n), with A(m, k) = A[m * sam + k * sak] and
// B(k, n) = B[k * sbk + n * sbn]; C row stride ldc.  64 x 64 tiles, 4 x 4 per
// thread, 256 threads.  Sequential float32 FMA accumulation along k.
namespace {
constexpr int GBM = 64, GBN = 64, GBK = 16;

__global__ void __launch_bounds__(256) sgemm_kernel(int Mr, int Nc, int K, const float* __restrict__ A,
                                                    long long sam, long long sak,
                                                    const float* __restrict__ Bm, long long sbk,
                                                    long long sbn, float* __restrict__ C, long long ldc)
{
    __shared__ float As[GBK][GBM + 4];
    __shared__ float Bs[GBK][GBN + 4];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    for (int k0 = 0; k0 < K; k0 += GBK) {
        for (int i = tid; i < GBM * GBK; i += 256) {
            int mm, kk;
            if (sak == 1) { kk = i % GBK; mm = i / GBK; } else { mm = i % GBM; kk = i / GBM; }
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < Mr && k < K) ? A[(long long)m * sam + (long long)k * sak] : 0.f;
        }
        for (int i = tid; i < GBN * GBK; i += 256) {
            int nn, kk;
            if (sbk == 1) { kk = i % GBK; nn = i / GBK; } else { nn = i % GBN; kk = i / GBN; }
            const int n = n0 + nn, k = k0 + kk;
            Bs[kk][nn] = (n < Nc && k < K) ? Bm[(long long)k * sbk + (long long)n * sbn] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= Mr) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n < Nc) C[(long long)m * ldc + n] = acc[i][j];
        }
    }
}
}  // namespace

int sgemm(int Mr, int Nc, int K, const float* A, long long sam, long long sak, const float* B,
          long long sbk, long long sbn, float* C, long long ldc, cudaStream_t st)
{
    if (Mr <= 0 || Nc <= 0) return DEEPINV_OK;
    // gridDim.y is at most 65535 row tiles: taller problems run in row chunks
    constexpr int kRowsPerLaunch = 65535 * GBM;
    for (long long r0 = 0; r0 < Mr; r0 += kRowsPerLaunch) {
        const int mr = (int)(Mr - r0 < kRowsPerLaunch ? Mr - r0 : kRowsPerLaunch);
        dim3 grid(cdiv(Nc, GBN), cdiv(mr, GBM));
        sgemm_kernel<<<grid, 256, 0, st>>>(mr, Nc, K, A + r0 * sam, sam, sak, B, sbk, sbn, C + r0 * ldc, ldc);
        DI_LAUNCH_CHECK();
    }
    return DEEPINV_OK;
}

// ---------------------------------------------------------------- convolution
// Eq. (1) with 'same' zero padding, cross-correlation:
// out[b][co][r][c] = act(bias[co] + sum_{ci,u,v} w[co][ci][u][v] in[b][ci][r+u-h][c+v-h]).
// Block: 8 rows x 64 columns x 16 output channels; each thread 4 adjacent
// pixels x 16 channels, sliding a register window along the row.
namespace {
constexpr int CTR = 8, CTC = 64, CCO = 16;

template <int KS>
__global__ void __launch_bounds__(128) conv_f32_kernel(const float* __restrict__ in, int Cin, int H,
                                                       int W, const float* __restrict__ w,
                                                       const float* __restrict__ bias, int Cout,
                                                       float* __restrict__ out, int relu)
{
    constexpr int HALF = KS / 2;
    constexpr int SR = CTR + KS - 1, SC = CTC + KS - 1;
    __shared__ float s_in[SR][SC + 1];
    __shared__ __align__(16) float s_w[KS * KS][CCO];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int tiles_w = (W + CTC - 1) / CTC;
    const int r0 = (blockIdx.x / tiles_w) * CTR, c0 = (blockIdx.x % tiles_w) * CTC;
    const int co0 = blockIdx.y * CCO;
    const int b = blockIdx.z;

    float acc[CCO][4];
#pragma unroll
    for (int co = 0; co < CCO; ++co) {
        const float bv = (bias && co0 + co < Cout) ? bias[co0 + co] : 0.f;
#pragma unroll
        for (int p = 0; p < 4; ++p) acc[co][p] = bv;
    }

    for (int ci = 0; ci < Cin; ++ci) {
        __syncthreads();
        const float* src = in + ((size_t)b * Cin + ci) * H * W;
        for (int i = tid; i < SR * SC; i += 128) {
            const int rr = i / SC, cc = i % SC;
            const int r = r0 - HALF + rr, c = c0 - HALF + cc;
            s_in[rr][cc] = (r >= 0 && r < H && c >= 0 && c < W) ? src[(size_t)r * W + c] : 0.f;
        }
        for (int i = tid; i < KS * KS * CCO; i += 128) {
            const int co = i / (KS * KS), t = i % (KS * KS);
            s_w[t][co] = (co0 + co < Cout) ? w[(((size_t)(co0 + co)) * Cin + ci) * KS * KS + t] : 0.f;
        }
        __syncthreads();
#pragma unroll 1
        for (int u = 0; u < KS; ++u) {
            float seg[4 + KS - 1];
#pragma unroll
            for (int j = 0; j < 4 + KS - 1; ++j) seg[j] = s_in[ty + u][tx * 4 + j];
#pragma unroll
            for (int v = 0; v < KS; ++v) {
#pragma unroll
                for (int cq = 0; cq < CCO / 4; ++cq) {
                    const float4 wv = *reinterpret_cast<const float4*>(&s_w[u * KS + v][cq * 4]);
                    const float wa[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e)
#pragma unroll
                        for (int p = 0; p < 4; ++p)
                            acc[cq * 4 + e][p] = fmaf(wa[e], seg[v + p], acc[cq * 4 + e][p]);
                }
            }
        }
    }
    const int r = r0 + ty;
    if (r >= H) return;
#pragma unroll
    for (int co = 0; co < CCO; ++co) {
        if (co0 + co >= Cout) break;
        float* dst = out + (((size_t)b * Cout + co0 + co) * H + r) * W;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int c = c0 + tx * 4 + p;
            if (c < W) {
                float v = acc[co][p];
                dst[c] = relu ? fmaxf(v, 0.f) : v;
            }
        }
    }
}
}  // namespace

int conv_f32(const float* in, int B, int Cin, int H, int W, const float* w, const float* bias,
             int Cout, int k, float* out, int relu, cudaStream_t st)
{
    if (B <= 0) return DEEPINV_OK;
    if (k < 1 || k > 15 || k % 2 == 0) {
        set_error("conv_f32: unsupported kernel size %d", k);
        return DEEPINV_EUNSUPPORTED;
    }
    // gridDim.z (one image per z) is at most 65535: larger batches run in chunks
    constexpr int kImagesPerLaunch = 65535;
    for (long long b0 = 0; b0 < B; b0 += kImagesPerLaunch) {
        const int nb = (int)(B - b0 < kImagesPerLaunch ? B - b0 : kImagesPerLaunch);
        const float* inb = in + (size_t)b0 * Cin * H * W;
        float* outb = out + (size_t)b0 * Cout * H * W;
        dim3 grid(cdiv(H, CTR) * cdiv(W, CTC), cdiv(Cout, CCO), nb);
        switch (k) {
#define DI_CONV_CASE(KS) \
    case KS: conv_f32_kernel<KS><<<grid, 128, 0, st>>>(inb, Cin, H, W, w, bias, Cout, outb, relu); break;
        DI_CONV_CASE(1)
        DI_CONV_CASE(3)
        DI_CONV_CASE(5)
        DI_CONV_CASE(7)
        DI_CONV_CASE(9)
        DI_CONV_CASE(11)
        DI_CONV_CASE(13)
        DI_CONV_CASE(15)
#undef DI_CONV_CASE
        }
        DI_LAUNCH_CHECK();
    }
    return DEEPINV_OK;
}

// ---------------------------------------------------------------- backward helpers
namespace {
// wt[ci][co][u'][v'] = w[co][ci][k-1-u'][k-1-v']: the input-gradient of a
// 'same' correlation is the 'same' correlation of the output gradient with
// this flipped, channel-transposed kernel.
__global__ void flip_transpose_kernel(const float* __restrict__ w, int Cout, int Cin, int k,
                                      float* __restrict__ wt)
{
    const int n = Cout * Cin * k * k;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int v = i % k, u = (i / k) % k, ci = (i / (k * k)) % Cin, co = i / (k * k * Cin);
        wt[(((size_t)ci * Cout + co) * k + (k - 1 - u)) * k + (k - 1 - v)] = w[i];
    }
}

// dw[co][ci][u][v] = sum_{b,r,c} g[b][co][r][c] in[b][ci][r+u-h][c+v-h]
// One block per (co, ci) and per pixel chunk; a thread per tap; float64
// partial sums, combined in a fixed order by wgrad_reduce_kernel.
__global__ void wgrad_partial_kernel(const float* __restrict__ in, const float* __restrict__ g, int B,
                                     int Cin, int H, int W, int Cout, int k, int nchunk,
                                     double* __restrict__ part)
{
    const int co = blockIdx.x / Cin, ci = blockIdx.x % Cin;
    const int chunk = blockIdx.y;
    const int h = k / 2;
    const long long total = (long long)B * H * W;
    const long long per = (total + nchunk - 1) / nchunk;
    const long long p0 = chunk * per, p1 = min(total, p0 + per);
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
        const int u = t / k, v = t % k;
        double s = 0.0;
        for (long long p = p0; p < p1; ++p) {
            const int c = (int)(p % W), r = (int)((p / W) % H), b = (int)(p / ((long long)W * H));
            const int rr = r + u - h, cc = c + v - h;
            if (rr < 0 || rr >= H || cc < 0 || cc >= W) continue;
            s += (double)g[(((size_t)b * Cout + co) * H + r) * W + c] *
                 (double)in[(((size_t)b * Cin + ci) * H + rr) * W + cc];
        }
        part[((size_t)chunk * Cout * Cin + (size_t)co * Cin + ci) * k * k + t] = s;
    }
}

__global__ void wgrad_reduce_kernel(const double* __restrict__ part, int nchunk, int n,
                                    float* __restrict__ dw)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < nchunk; ++c) s += part[(size_t)c * n + i];
        dw[i] = (float)s;
    }
}

// db[co] = sum over batch and pixels of g[b][co][.][.], float64, one block per co.
__global__ void bias_grad_kernel(const float* __restrict__ g, int B, int C, int HW,
                                 float* __restrict__ db)
{
    const int co = blockIdx.x;
    double s = 0.0;
    for (long long i = threadIdx.x; i < (long long)B * HW; i += blockDim.x) {
        const long long b = i / HW, p = i % HW;
        s += (double)g[((size_t)b * C + co) * HW + p];
    }
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[co] = (float)red[0];
}

// g <- g * [a > 0] (ReLU derivative, 0 at the kink; a is the ReLU output).
__global__ void relu_mask_kernel(float* __restrict__ g, const float* __restrict__ a, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        if (!(a[i] > 0.f)) g[i] = 0.f;
}

// Loss partials: part[blk] = sum over this block's slice of (xhat - x)^2 in
// float64, and g = 2 (xhat - x) / B (masked by [xhat > 0] when final_relu).
__global__ void mse_partial_kernel(const float* __restrict__ xhat, const float* __restrict__ x,
                                   long long n, int B, int final_relu, float* __restrict__ g,
                                   double* __restrict__ part)
{
    double s = 0.0;
    const float scale = 2.0f / (float)B;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float d = xhat[i] - x[i];
        s += (double)d * (double)d;
        if (g) g[i] = (final_relu && !(xhat[i] > 0.f)) ? 0.f : scale * d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
}

// Loss = (sum of the block partials) / B: lane l adds partials l, l + 32, ...
// in turn, then a fixed butterfly over the lanes (one warp).
__global__ void mse_final_kernel(const double* __restrict__ part, int nb, int B, double* __restrict__ loss)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += 32) s += part[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *loss = s / (double)B;
}

// dst[i] += src[i] (gradients of later recomputation chunks, added in chunk order).
template <typename T>
__global__ void accumulate_kernel(T* __restrict__ dst, const T* __restrict__ src, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] += src[i];
}

// The same step for several tensors in one launch: tensor k owns blocks
// [t.boff[k], t.boff[k + 1]) of the grid.
__global__ void sgd_momentum_multi_kernel(SgdTensors t, float lr, float mu)
{
    int k = 0;
    while (k + 1 < t.count && (int)blockIdx.x >= t.boff[k + 1]) ++k;
    float* __restrict__ w = t.w[k];
    float* __restrict__ v = t.v[k];
    const float* __restrict__ g = t.g[k];
    const long long n = t.n[k];
    const long long nb = t.boff[k + 1] - t.boff[k];
    for (long long i = ((long long)blockIdx.x - t.boff[k]) * blockDim.x + threadIdx.x; i < n; i += nb * blockDim.x) {
        const float vn = mu * v[i] + g[i];
        v[i] = vn;
        w[i] = w[i] - lr * vn;
    }
}

inline int grid_for(long long n, int threads = 256)
{
    long long b = (n + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}
}  // namespace

int conv_dgrad_f32(const float* g, int B, int Cout, int H, int W, const float* w, int Cin, int k,
                   float* wt_scratch, float* din, cudaStream_t st)
{
    const int n = Cout * Cin * k * k;
    flip_transpose_kernel<<<grid_for(n), 256, 0, st>>>(w, Cout, Cin, k, wt_scratch);
    DI_LAUNCH_CHECK();
    return conv_f32(g, B, Cout, H, W, wt_scratch, nullptr, Cin, k, din, 0, st);
}

size_t wgrad_scratch_bytes(int Cout, int Cin, int k) { return (size_t)kWgradChunks * Cout * Cin * k * k * sizeof(double); }

int conv_wgrad_f32(const float* in, const float* g, int B, int Cin, int H, int W, int Cout, int k,
                   double* scratch, float* dw, float* db, cudaStream_t st)
{
    dim3 grid(Cout * Cin, kWgradChunks);
    wgrad_partial_kernel<<<grid, 128, 0, st>>>(in, g, B, Cin, H, W, Cout, k, kWgradChunks, scratch);
    DI_LAUNCH_CHECK();
    const int n = Cout * Cin * k * k;
    wgrad_reduce_kernel<<<grid_for(n), 256, 0, st>>>(scratch, kWgradChunks, n, dw);
    DI_LAUNCH_CHECK();
    if (db) {
        bias_grad_kernel<<<Cout, 256, 0, st>>>(g, B, Cout, H * W, db);
        DI_LAUNCH_CHECK();
    }
    return DEEPINV_OK;
}

int relu_mask_f32(float* g, const float* a, long long n, cudaStream_t st)
{
    relu_mask_kernel<<<grid_for(n), 256, 0, st>>>(g, a, n);
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

int mse_loss_grad(const float* xhat, const float* x, long long n, int B, int final_relu, float* g,
                  double* part, double* loss, cudaStream_t st)
{
    mse_partial_kernel<<<kLossBlocks, 256, 0, st>>>(xhat, x, n, B, final_relu, g, part);
    DI_LAUNCH_CHECK();
    mse_final_kernel<<<1, 32, 0, st>>>(part, kLossBlocks, B, loss);
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

int accumulate_f32(float* dst, const float* src, long long n, cudaStream_t st)
{
    if (n <= 0) return DEEPINV_OK;
    accumulate_kernel<float><<<grid_for(n), 256, 0, st>>>(dst, src, n);
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

int accumulate_f64(double* dst, const double* src, long long n, cudaStream_t st)
{
    if (n <= 0) return DEEPINV_OK;
    accumulate_kernel<double><<<grid_for(n), 256, 0, st>>>(dst, src, n);
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

int sgd_momentum_multi(SgdTensors t, float lr, float mu, cudaStream_t st)
{
    if (t.count <= 0) return DEEPINV_OK;
    // blocks per tensor: about 4 elements per thread, at most 2432
    int total = 0;
    for (int k = 0; k < t.count; ++k) {
        t.boff[k] = total;
        long long nb = (t.n[k] + 1023) / 1024;
        if (nb < 1) nb = 1;
        if (nb > 2432) nb = 2432;
        total += (int)nb;
    }
    t.boff[t.count] = total;
    sgd_momentum_multi_kernel<<<total, 256, 0, st>>>(t, lr, mu);
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}

}  // namespace di

namespace di {
namespace {
// dst[c][r] = src[r][c] for an R x C matrix.
__global__ void transpose_kernel(const float* __restrict__ src, int R, int C, float* __restrict__ dst)
{
    __shared__ float t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        if (r < R && c < C) t[i][threadIdx.x] = src[(size_t)r * C + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (r < R && c < C) dst[(size_t)c * R + r] = t[threadIdx.x][i];
    }
}
}  // namespace

int transpose_f32(const float* src, int R, int C, float* dst, cudaStream_t st)
{
    dim3 grid(cdiv(C, 32), cdiv(R, 32));
    transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(src, R, C, dst);
    DI_LAUNCH_CHECK();
    return DEEPINV_OK;
}
}  // namespace di
