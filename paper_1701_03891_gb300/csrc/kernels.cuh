// Host-side launchers of the libdeepinv kernels (declarations).
#pragma once

#include "common.cuh"

namespace di {

typedef __nv_bfloat16 bf16;

// ---------------------------------------------------------------- float32 path (f32_kernels.cu)
constexpr int kWgradChunks = 64;   // pixel chunks of the float32 weight-gradient reduction
constexpr int kLossBlocks = 256;   // partial sums of the loss reduction

int sgemm(int Mr, int Nc, int K, const float* A, long long sam, long long sak, const float* B,
          long long sbk, long long sbn, float* C, long long ldc, cudaStream_t st);
int conv_f32(const float* in, int B, int Cin, int H, int W, const float* w, const float* bias,
             int Cout, int k, float* out, int relu, cudaStream_t st);
int conv_dgrad_f32(const float* g, int B, int Cout, int H, int W, const float* w, int Cin, int k,
                   float* wt_scratch, float* din, cudaStream_t st);
size_t wgrad_scratch_bytes(int Cout, int Cin, int k);
int conv_wgrad_f32(const float* in, const float* g, int B, int Cin, int H, int W, int Cout, int k,
                   double* scratch, float* dw, float* db, cudaStream_t st);
int relu_mask_f32(float* g, const float* a, long long n, cudaStream_t st);
int mse_loss_grad(const float* xhat, const float* x, long long n, int B, int final_relu, float* g,
                  double* part, double* loss, cudaStream_t st);
int transpose_f32(const float* src, int R, int C, float* dst, cudaStream_t st);
// dst += src, element-wise.
int accumulate_f32(float* dst, const float* src, long long n, cudaStream_t st);
int accumulate_f64(double* dst, const double* src, long long n, cudaStream_t st);
// SGD with momentum, v <- mu v + g; w <- w - lr v, over up to kSgdMaxTensors
// tensors in one launch (passed by value).
constexpr int kSgdMaxTensors = 40;
struct SgdTensors {
    float* w[kSgdMaxTensors];
    float* v[kSgdMaxTensors];
    const float* g[kSgdMaxTensors];
    long long n[kSgdMaxTensors];
    int boff[kSgdMaxTensors + 1];   // first grid block of each tensor (set by the launcher)
    int count;
};
int sgd_momentum_multi(SgdTensors t, float lr, float mu, cudaStream_t st);

// ---------------------------------------------------------------- bfloat16 tensor-core path (tc_kernels.cu)
// Packed K-major operand: dst holds ceil(R / TR) row tiles, each Kp / 8
// chunks of TR rows x 8 bf16 (16 bytes per row), i.e. element (r, k) at
// ((r / TR * (Kp / 8) + k / 8) * TR + r % TR) * 8 + k % 8.  Source element
// (r, k) = src[r * rs + k * cs]; zero outside R x K.
size_t packed_elems(int R, int TR, int Kp);
int pack_kmajor(const float* src, long long rs, long long cs, int R, int K, int TR, int Kp,
                bf16* dst, cudaStream_t st);

// Weight layouts of the paper network (l1 = 64, l2 = 32, l3 = 1, k = 11).
constexpr size_t kW1PackElems = 11 * 2 * 64 * 8;         // [dy][h][64 rows][8]
constexpr size_t kW2PackElems = 11 * 3 * 4 * 2 * 128 * 8;  // [dy][s][kk][2][128][8]
constexpr size_t kW3PackElems = 3 * 2 * 2 * 64 * 8;      // [x][kk][2][64][8]
int pack_conv_weights(const float* w1, const float* w2, const float* w3, bf16* w1p, bf16* w2p,
                      bf16* w3p, cudaStream_t st);

// Hidden 32 -> 32 layers: forward and input-gradient operands of one layer
// (conv2's A layout with 2 chunk pairs, [dy][s][kk][2][128][8]); wht may be
// NULL (inference-only networks).
constexpr size_t kWhPackElems = 11 * 3 * 2 * 2 * 128 * 8;
int pack_hidden_weights(const float* w, bf16* whp, bf16* wht, cudaStream_t st);

enum GemmOut { GEMM_OUT_F32 = 0, GEMM_OUT_PLANE = 1 };

// D[m][n] = sum_k A[m][k] B[n][k] over packed operands (A: TR = 128, B: TR =
// NB).  GEMM_OUT_F32 writes out_f32[m * ldo + n] for m < Mr, n < Nc;
// GEMM_OUT_PLANE treats m as pixel j of an n1 x n2 image and n as the image
// index, writing bf16 to plane[n * geo.plane + L(j)].
int tc_gemm(const bf16* A, const bf16* B, int Kp, int Mr, int Nc, int NB, int mode, float* out_f32,
            long long ldo, bf16* plane, const Geo& geo, int* status, cudaStream_t st);

// out [Mr][Nc] float32 = A B^T with the K steps split over `ksplit` CTAs per
// tile; part holds ksplit * Mr * Nc floats of partial sums (summed in order).
int tc_gemm_splitk(const bf16* A, const bf16* B, int Kp, int Mr, int Nc, int NB, float* out, float* part, int ksplit,
                   int* status, cudaStream_t st);
// The measurement fed straight from the float32 signals (gemm_f32in.cu):
// out [Mr][Nc] float32 = X B^T, X float32 [Mr][K] (row stride ldx) read by TMA
// and rounded to bfloat16 inside the kernel, B packed (TR = NB, Kp); K split
// over a thread-block cluster, summed through distributed shared memory in a
// fixed order.  Supported when X is 16-byte aligned with a row stride of a
// multiple of 4 floats (the tensor map's rules) and NB <= 256; otherwise the
// call returns DEEPINV_EUNSUPPORTED.
bool measure_f32in_supported(const float* X, long long ldx, int NB);
int gemm_measure_f32in(const float* X, long long ldx, int K, const bf16* Bpk, int Kp, int Mr, int Nc, int NB,
                       float* out, long long ldo, int num_sms, int* status, cudaStream_t st);
// Split that keeps about one wave of CTAs busy for a GEMM with the given tiles.
inline int gemm_ksplit(int Mr, int Nc, int NB, int Kp, int num_sms)
{
    const int tiles = ((Mr + 127) / 128) * ((Nc + NB - 1) / NB);
    int k = num_sms / (tiles > 0 ? tiles : 1);
    const int kmax = Kp / 16 / 16;               // at least 16 MMA steps per split
    if (k > kmax) k = kmax;
    if (k > 16) k = 16;
    return k < 1 ? 1 : k;
}
// conv1: x~ plane [B][plane] -> a1 (bias, ReLU, zero pad columns), as
//   kConv1OutBF16: bf16 [B][8][plane][8];
//   kConv1OutE4M3: e4m3 [B][4][plane][16], values times *inv_sa;
//   kConv1AmaxOnly: no output, atomically raises *amax to the largest a1 value.
//   kConv1GradMask: (backward, 32 filters) result times [mask > 0] as a bf16 gradient plane.
enum { kConv1OutBF16 = 0, kConv1OutE4M3 = 1, kConv1AmaxOnly = 2, kConv1GradMask = 3 };
int conv1_tc(const bf16* xt, int B, const Geo& g, const bf16* w1p, const float* b1, void* a1, int mode,
             const float* inv_sa, float* amax, int* status, cudaStream_t st);
// conv1 in row tiles with its A operands kept in TMEM (kConv1OutBF16 or
// kConv1OutE4M3 only; same output, bit for bit, as conv1_tc).  conv1_rows_fit:
// 0 where row tiles would fill fewer than 96 of 128 positions, 1 where they fit,
// 2 where they also measured faster than conv1_tc.
int conv1_rows_fit(const Geo& g);
int conv1_rows_tc(const bf16* xt, int B, const Geo& g, const bf16* w1p, const float* b1, void* a1, int mode,
                  const float* inv_sa, int* status, cudaStream_t st);
// conv2: a1 (bf16, or e4m3 when fp8) -> a2 bf16 [B][4][plane][8] (bias, ReLU,
// zero pad columns); the e4m3 path multiplies the accumulators by oscale[co].
int conv2_tc(const void* a1, int B, const Geo& g, const void* w2p, const float* b2, const float* oscale,
             bool fp8, bf16* a2, int num_sms, int* status, cudaStream_t st);
// ---------------------------------------------------------------- backward (bf16 path)
// Input gradients as correlations with flipped kernels, ReLU masks fused:
// conv3: gradient plane of x^ [B][plane] -> g2 = dL/dz2 [B][4][plane][8] (mask a2 > 0);
// conv2: g2 -> g1 = dL/dz1 [B][8][plane][8] (mask a1 > 0).
int conv3_dgrad_tc(const bf16* g3p, int B, const Geo& g, const bf16* w3t, const bf16* a2, bf16* g2, int* status,
                   cudaStream_t st);
int conv2_dgrad_tc(const bf16* g2, int B, const Geo& g, const bf16* w2t, const bf16* a1, bf16* g1, int num_sms,
                   int* status, cudaStream_t st);
// Hidden layer (32 -> 32 channels, planes [B][4][plane][8]): forward with
// bias and ReLU (zero pad columns), and the input gradient from the output
// gradient times the ReLU mask [act_in > 0] of the layer's input.
int hidden_tc(const bf16* in, int B, const Geo& g, const bf16* whp, const float* bias, bf16* out, int num_sms,
              int* status, cudaStream_t st);
int hidden_dgrad_tc(const bf16* gout, int B, const Geo& g, const bf16* wht, const bf16* act_in, bf16* gin,
                    int num_sms, int* status, cudaStream_t st);
constexpr size_t kW3tPackElems = 11 * 2 * 32 * 8;      // conv3 input-gradient weights [dy'][h][32][8]
constexpr size_t kW1tPackElems = 3 * 4 * 2 * 64 * 8;   // conv1 input-gradient weights [x][4][2][64][8]
// w1t, w2t ([dy'][6][2][2][128][8], kW2PackElems) and w3t from the float32 masters.
int pack_dgrad_weights(const float* w1, const float* w2, const float* w3, bf16* w1t, bf16* w2t, bf16* w3t,
                       cudaStream_t st);
// Input gradient of conv1 (for training the FC layer): g1 plane -> row sums T
// (scratch, conv3_scratch_elems) -> dxt [B][N] float32.
int conv1_dgrad_tc(const bf16* g1, int B, const Geo& g, const bf16* w1t, float* T, float* dxt, int* status,
                   cudaStream_t st);
// g [B][N] float32 -> data positions of the one-channel plane gp (pads untouched).
int grad_plane(const float* g, int B, const Geo& geo, bf16* gp, cudaStream_t st);
// Channel sums of a bf16 plane (bias gradients): part [B][C] float64 scratch, out [C].
int plane_channel_sums(const bf16* src, int B, int C, const Geo& geo, double* part, float* out, cudaStream_t st);
// conv1 (conv1 = true: S = x~ plane, C = g1 plane; also db = conv1's bias
// gradient) or conv3 (S = x^ gradient plane, C = a2 plane; db unused) weight
// gradient on the tensor cores; part is float32 scratch of tapwgrad_scratch_floats().
size_t tapwgrad_scratch_floats();
int tap_wgrad_tc(bool conv1, const bf16* S, const bf16* C, int B, const Geo& g, float* part, float* dw, float* db,
                 int* status, cudaStream_t st);
// conv2 weight gradient on the tensor cores: g2 plane [B][4][plane][8] and a1
// plane [B][8][plane][8] -> dw [32][64][11][11]; part is float32 scratch of
// wgrad2_scratch_floats().
size_t wgrad2_scratch_floats();
int wgrad2_tc(const bf16* G2, const bf16* A1, int B, const Geo& g, float* part, float* dw, int* status,
              cudaStream_t st);
// Hidden layer weight gradient: output gradient plane [B][4][plane][8] and the
// layer's input plane [B][4][plane][8] -> dw [32][32][11][11] (same scratch).
int wgrad_hidden_tc(const bf16* G, const bf16* A, int B, const Geo& g, float* part, float* dw, int* status,
                    cudaStream_t st);
// e4m3 conv2 weights: [dy][s][kk][2][128][16] bytes with per-filter scales sw[32].
constexpr size_t kW2E4M3Bytes = 11 * 3 * 2 * 2 * 128 * 16;
int pack_w2_e4m3(const float* w2, float* amax_scratch, uint8_t* w2q, float* sw, cudaStream_t st);
int e4m3_scales(const float* amax_a1, const float* sw, float* inv_sa, float* oscale, cudaStream_t st);
bool conv2_tc_supported(const Geo& g);
// conv1 + conv2 fused (fused12.cu): x~ plane [B][plane] -> a2 bf16
// [B][4][plane][8] (bias and ReLU after each layer, zero pad columns), a1 kept
// in shared memory.  Images wider than 70 columns are walked as column strips
// whose x~ planes are gathered into `xs` (conv12_scratch_bytes; 0 otherwise).
size_t conv12_scratch_bytes(int B, const Geo& g);
int conv12_tc(const bf16* xt, int B, const Geo& g, const bf16* w1p, const float* b1, const bf16* w2p,
              const float* b2, bf16* a2, bf16* xs, int num_sms, int* status, cudaStream_t st);
// conv3: a2 -> row partial sums T [images of one pass][11][tlen] -> xhat [B][n1 * n2] float32.
// conv3 keeps its row sums (or, for pitches >= 125, its partial outputs) in a
// shared-memory ring and needs no scratch, up to about 4000 columns; wider
// images use a float scratch of row sums, conv3_scratch_elems floats for a
// batch of B, filled conv3_chunk images at a time.
bool conv3_fused(const Geo& g, int cin);
size_t conv3_chunk(const Geo& g, int B);
size_t conv3_scratch_elems(const Geo& g, int B, int cin);
int conv3_tc(const bf16* a2, int B, const Geo& g, const bf16* w3p, const float* b3, float* T,
             float* xhat, int final_relu, int* status, cudaStream_t st);

// One kernel whose bounded wait never completes: records DEV_TIMEOUT in `status`.
int bounded_wait_probe(int* status, cudaStream_t st);


}  // namespace di
