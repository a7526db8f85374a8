/*
 * FP64 CPU oracle for the DeepInverse forward and backward pass.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check of the
 * package entry point and the CPU-baseline leg of the benchmark may load this
 * code.  It shares nothing with the CUDA path: no headers, no layouts, no
 * helpers.  Every routine is the plain definition from the paper written out
 * as direct loops in double precision, one output element at a time.
 *
 * Notation (paper, Sec. 1 and Sec. 4): Phi is M x N, x in R^N, y = Phi x in
 * R^M; the proxy is x~ = Phi^T y reshaped to n1 x n2; each convolutional layer
 * computes Eq. (1).  Layout here is planar NCHW, row-major, double.
 *
 * Readings of the paper used here (each one also listed in the design notes):
 *  - the "*" of Eq. (1) is cross-correlation (no kernel flip);
 *  - the crop S of Eq. (1) applied to a full (n+k-1) convolution equals a
 *    'same' convolution with (k-1)/2 zeros on each side (oracle_conv_full
 *    exists so that a test can check this identity);
 *  - the bias of Eq. (1) is one scalar per filter.
 */
#include <stddef.h>

#define IDX4(a, b, c, d, B_, C_, D_) ((((size_t)(a) * (B_) + (b)) * (C_) + (c)) * (D_) + (d))

/* Sec. 1: y = Phi x for each of B signals.
 * phi [M][N], x [B][N]  ->  y [B][M]. */
void oracle_measure(const double* phi, int M, int N, const double* x, int B, double* y)
{
    #pragma omp parallel for collapse(2) schedule(static)
    for (int b = 0; b < B; ++b)
        for (int i = 0; i < M; ++i) {
            double s = 0.0;
            for (int j = 0; j < N; ++j)
                s += phi[(size_t)i * N + j] * x[(size_t)b * N + j];
            y[(size_t)b * M + i] = s;
        }
}

/* Sec. 4: the fully connected layer that lifts R^M to R^N.
 * w [N][M] holds the weight of measurement i for proxy pixel j at w[j][i];
 * with w = Phi^T (w[j][i] = Phi[i][j]) this is the adjoint x~ = Phi^T y.
 * y [B][M] -> xt [B][N]. */
void oracle_fc(const double* w, int N, int M, const double* y, int B, double* xt)
{
    #pragma omp parallel for collapse(2) schedule(static)
    for (int b = 0; b < B; ++b)
        for (int j = 0; j < N; ++j) {
            double s = 0.0;
            for (int i = 0; i < M; ++i)
                s += w[(size_t)j * M + i] * y[(size_t)b * M + i];
            xt[(size_t)b * N + j] = s;
        }
}

/* Eq. (1) before the ReLU, 'same' size:
 * z[b][co][r][c] = bias[co] + sum_{ci,u,v} w[co][ci][u][v] * in[b][ci][r+u-h][c+v-h],
 * h = (k-1)/2, input taken as zero outside [0,H) x [0,W).
 * in [B][Cin][H][W], w [Cout][Cin][k][k], bias [Cout] (may be NULL) -> z [B][Cout][H][W]. */
void oracle_conv_same(const double* in, int B, int Cin, int H, int W,
                      const double* w, const double* bias, int Cout, int k, double* z)
{
    const int h = (k - 1) / 2;
    #pragma omp parallel for collapse(2) schedule(dynamic, 1)
    for (int b = 0; b < B; ++b)
        for (int co = 0; co < Cout; ++co)
            for (int r = 0; r < H; ++r)
                for (int c = 0; c < W; ++c) {
                    double s = bias ? bias[co] : 0.0;
                    for (int ci = 0; ci < Cin; ++ci)
                        for (int u = 0; u < k; ++u) {
                            const int rr = r + u - h;
                            if (rr < 0 || rr >= H) continue;
                            for (int v = 0; v < k; ++v) {
                                const int cc = c + v - h;
                                if (cc < 0 || cc >= W) continue;
                                s += w[IDX4(co, ci, u, v, Cin, k, k)] *
                                     in[IDX4(b, ci, rr, cc, Cin, H, W)];
                            }
                        }
                    z[IDX4(b, co, r, c, Cout, H, W)] = s;
                }
}

/* Eq. (1) read literally: the full correlation of the input zero-padded by
 * k-1 on every side, size (H+k-1) x (W+k-1), before the crop S.
 * zf[b][co][R][C] = bias[co] + sum w[co][ci][u][v] * in[b][ci][R-(k-1)+u][C-(k-1)+v]. */
void oracle_conv_full(const double* in, int B, int Cin, int H, int W,
                      const double* w, const double* bias, int Cout, int k, double* zf)
{
    const int HF = H + k - 1, WF = W + k - 1;
    #pragma omp parallel for collapse(2) schedule(dynamic, 1)
    for (int b = 0; b < B; ++b)
        for (int co = 0; co < Cout; ++co)
            for (int R = 0; R < HF; ++R)
                for (int C = 0; C < WF; ++C) {
                    double s = bias ? bias[co] : 0.0;
                    for (int ci = 0; ci < Cin; ++ci)
                        for (int u = 0; u < k; ++u) {
                            const int rr = R - (k - 1) + u;
                            if (rr < 0 || rr >= H) continue;
                            for (int v = 0; v < k; ++v) {
                                const int cc = C - (k - 1) + v;
                                if (cc < 0 || cc >= W) continue;
                                s += w[IDX4(co, ci, u, v, Cin, k, k)] *
                                     in[IDX4(b, ci, rr, cc, Cin, H, W)];
                            }
                        }
                    zf[IDX4(b, co, R, C, Cout, HF, WF)] = s;
                }
}

/* Backpropagation (Sec. 4, the MSE objective) through one 'same' layer,
 * weight side.  g = dL/dz [B][Cout][H][W], in = layer input [B][Cin][H][W]:
 * dw[co][ci][u][v] = sum_{b,r,c} g[b][co][r][c] * in[b][ci][r+u-h][c+v-h],
 * db[co] = sum_{b,r,c} g[b][co][r][c]   (db may be NULL). */
void oracle_conv_same_wgrad(const double* in, const double* g, int B, int Cin, int H, int W,
                            int Cout, int k, double* dw, double* db)
{
    const int h = (k - 1) / 2;
    #pragma omp parallel for collapse(2) schedule(dynamic, 1)
    for (int co = 0; co < Cout; ++co)
        for (int ci = 0; ci < Cin; ++ci)
            for (int u = 0; u < k; ++u)
                for (int v = 0; v < k; ++v) {
                    double s = 0.0;
                    for (int b = 0; b < B; ++b)
                        for (int r = 0; r < H; ++r) {
                            const int rr = r + u - h;
                            if (rr < 0 || rr >= H) continue;
                            for (int c = 0; c < W; ++c) {
                                const int cc = c + v - h;
                                if (cc < 0 || cc >= W) continue;
                                s += g[IDX4(b, co, r, c, Cout, H, W)] *
                                     in[IDX4(b, ci, rr, cc, Cin, H, W)];
                            }
                        }
                    dw[IDX4(co, ci, u, v, Cin, k, k)] = s;
                }
    if (db) {
        for (int co = 0; co < Cout; ++co) {
            double s = 0.0;
            for (int b = 0; b < B; ++b)
                for (int r = 0; r < H; ++r)
                    for (int c = 0; c < W; ++c)
                        s += g[IDX4(b, co, r, c, Cout, H, W)];
            db[co] = s;
        }
    }
}

/* Backpropagation through one 'same' layer, input side:
 * din[b][ci][p][q] = sum_{co,u,v} w[co][ci][u][v] * g[b][co][p-u+h][q-v+h]
 * (the output position (r,c) that read input (p,q) through tap (u,v) is
 * r = p-u+h, c = q-v+h; terms with (r,c) outside the image vanish). */
void oracle_conv_same_dgrad(const double* g, const double* w, int B, int Cin, int H, int W,
                            int Cout, int k, double* din)
{
    const int h = (k - 1) / 2;
    #pragma omp parallel for collapse(2) schedule(dynamic, 1)
    for (int b = 0; b < B; ++b)
        for (int ci = 0; ci < Cin; ++ci)
            for (int p = 0; p < H; ++p)
                for (int q = 0; q < W; ++q) {
                    double s = 0.0;
                    for (int co = 0; co < Cout; ++co)
                        for (int u = 0; u < k; ++u) {
                            const int r = p - u + h;
                            if (r < 0 || r >= H) continue;
                            for (int v = 0; v < k; ++v) {
                                const int c = q - v + h;
                                if (c < 0 || c >= W) continue;
                                s += w[IDX4(co, ci, u, v, Cin, k, k)] *
                                     g[IDX4(b, co, r, c, Cout, H, W)];
                            }
                        }
                    din[IDX4(b, ci, p, q, Cin, H, W)] = s;
                }
}

/* Backpropagation through the fully connected layer (weight side):
 * dw[j][i] = sum_b dxt[b][j] * y[b][i]. */
void oracle_fc_wgrad(const double* dxt, const double* y, int B, int N, int M, double* dw)
{
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < M; ++i) {
            double s = 0.0;
            for (int b = 0; b < B; ++b)
                s += dxt[(size_t)b * N + j] * y[(size_t)b * M + i];
            dw[(size_t)j * M + i] = s;
        }
}

/* Threads of later parallel loops (the timed baselines use every host core;
 * a launcher may have set OMP_NUM_THREADS=1 for its workers). */
void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Number of threads the OpenMP runtime will use (reported by the baseline). */
int oracle_num_threads(void)
{
    int n = 1;
    #pragma omp parallel
    {
        #pragma omp single
        {
#ifdef _OPENMP
            extern int omp_get_num_threads(void);
            n = omp_get_num_threads();
#endif
        }
    }
    return n;
}
