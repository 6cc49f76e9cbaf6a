/*
 * FP64 CPU oracle for the CNN forward pass (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use
 * this file.  It shares no code, header, table or helper with the CUDA
 * library; it is compiled on its own with gcc.
 *
 * What it computes is the plain definition of each layer of the Darknet
 * network the paper offloads to the GPU (Sec. 5.1.1: the detection /
 * image-processing sample apps of Darknet; Sec. 3.2: the loops whose data
 * stays on the GPU).  The paper itself prints no layer formulas, so each
 * function states the textbook definition it implements:
 *
 *   conv:   y[n,o,i,j] = sum_{c,kh,kw} x[n,c,i+kh-p,j+kw-p] * w[o,c,kh,kw],
 *           p = (k-1)/2, stride 1, x outside the image = 0.
 *   bn:     z = gamma*(y - mean)/sqrt(var + eps) + beta   (applied unfolded)
 *   leaky:  z > 0 ? z : 0.1*z
 *   pool:   2x2 stride 2 max; or 2x2 stride 1 "same" max whose window is
 *           anchored at the top-left and clipped at the bottom/right edge.
 *
 * The accumulation in oracle_conv2d walks the terms of every output in
 * (c, kh, kw) lexicographic order, exactly as the sum is written; the loop
 * over output positions sits inside only so that memory is read
 * contiguously.  OpenMP splits the independent (n, o) planes.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>

int oracle_version(void) { return 1; }

int oracle_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads used by later calls (the CPU baseline times 1 and all cores). */
void oracle_set_threads(int n) {
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* 2-D convolution, NCHW in / OIHW weights / NCHW out, zero pad p=(k-1)/2. */
void oracle_conv2d(const double* x, int N, int C, int H, int W,
                   const double* w, int O, int k, double* y) {
    const int p = (k - 1) / 2;
    const long HW = (long)H * W;
    long planes = (long)N * O;
#pragma omp parallel for schedule(dynamic, 1)
    for (long no = 0; no < planes; ++no) {
        const int n = (int)(no / O), o = (int)(no % O);
        double* yp = y + no * HW;
        for (long t = 0; t < HW; ++t) yp[t] = 0.0;
        for (int c = 0; c < C; ++c) {
            const double* xp = x + ((long)n * C + c) * HW;
            for (int kh = 0; kh < k; ++kh) {
                for (int kw = 0; kw < k; ++kw) {
                    const double wv = w[(((long)o * C + c) * k + kh) * k + kw];
                    for (int i = 0; i < H; ++i) {
                        const int ii = i + kh - p;
                        if (ii < 0 || ii >= H) continue;
                        for (int j = 0; j < W; ++j) {
                            const int jj = j + kw - p;
                            if (jj < 0 || jj >= W) continue;
                            yp[(long)i * W + j] += xp[(long)ii * W + jj] * wv;
                        }
                    }
                }
            }
        }
    }
}

/* Gradient of a conv layer's input (the "nightmare" backward pass):
 *   dx[n,c,i,j] = sum_{o,kh,kw} dy[n,o,i-kh+p,j-kw+p] * w[o,c,kh,kw],
 * over the (i-kh+p, j-kw+p) inside the map: the derivative of
 * y[n,o,a,b] = sum x[n,c,a+kh-p,b+kw-p] w[o,c,kh,kw] with respect to
 * x[n,c,i,j] (a = i-kh+p, b = j-kw+p).  dy: N,O,H,W; w: O,C,k,k; dx: N,C,H,W. */
void oracle_conv2d_bwd_data(const double* dy, int N, int O, int H, int W,
                            const double* w, int C, int k, double* dx) {
    const int p = (k - 1) / 2;
    const long HW = (long)H * W;
    long planes = (long)N * C;
#pragma omp parallel for schedule(dynamic, 1)
    for (long nc = 0; nc < planes; ++nc) {
        const int n = (int)(nc / C), c = (int)(nc % C);
        double* xp = dx + nc * HW;
        for (long t = 0; t < HW; ++t) xp[t] = 0.0;
        for (int o = 0; o < O; ++o) {
            const double* yp = dy + ((long)n * O + o) * HW;
            for (int kh = 0; kh < k; ++kh) {
                for (int kw = 0; kw < k; ++kw) {
                    const double wv = w[(((long)o * C + c) * k + kh) * k + kw];
                    for (int i = 0; i < H; ++i) {
                        const int a = i - kh + p;
                        if (a < 0 || a >= H) continue;
                        for (int j = 0; j < W; ++j) {
                            const int b = j - kw + p;
                            if (b < 0 || b >= W) continue;
                            xp[(long)i * W + j] += yp[(long)a * W + b] * wv;
                        }
                    }
                }
            }
        }
    }
}

/* Batchnorm with running statistics, unfolded, per channel o. */
void oracle_batchnorm(double* y, int N, int O, long HW, const double* gamma,
                      const double* beta, const double* mean, const double* var,
                      double eps) {
    for (int n = 0; n < N; ++n)
        for (int o = 0; o < O; ++o) {
            double* yp = y + ((long)n * O + o) * HW;
            const double inv = 1.0 / sqrt(var[o] + eps);
            for (long t = 0; t < HW; ++t)
                yp[t] = gamma[o] * (yp[t] - mean[o]) * inv + beta[o];
        }
}

void oracle_bias(double* y, int N, int O, long HW, const double* bias) {
    for (int n = 0; n < N; ++n)
        for (int o = 0; o < O; ++o) {
            double* yp = y + ((long)n * O + o) * HW;
            for (long t = 0; t < HW; ++t) yp[t] += bias[o];
        }
}

/* Leaky rectifier with slope `slope` for non-positive inputs. */
void oracle_leaky(double* y, long n, double slope) {
    for (long t = 0; t < n; ++t)
        if (!(y[t] > 0.0)) y[t] = slope * y[t];
}

/* 2x2 max pool, stride 2 (H, W even): out is N x C x H/2 x W/2. */
void oracle_maxpool2_s2(const double* x, int N, int C, int H, int W, double* y) {
    const int Ho = H / 2, Wo = W / 2;
    for (long nc = 0; nc < (long)N * C; ++nc) {
        const double* xp = x + nc * H * W;
        double* yp = y + nc * Ho * Wo;
        for (int i = 0; i < Ho; ++i)
            for (int j = 0; j < Wo; ++j) {
                double m = xp[(2 * i) * W + 2 * j];
                for (int di = 0; di < 2; ++di)
                    for (int dj = 0; dj < 2; ++dj) {
                        double v = xp[(2 * i + di) * W + 2 * j + dj];
                        if (v > m) m = v;
                    }
                yp[i * Wo + j] = m;
            }
    }
}

/* 2x2 max pool, stride 1, output H x W: the window at (i, j) covers rows
 * i..i+1 and columns j..j+1, clipped to the image (bottom/right edge
 * windows shrink). */
void oracle_maxpool2_s1_same(const double* x, int N, int C, int H, int W, double* y) {
    for (long nc = 0; nc < (long)N * C; ++nc) {
        const double* xp = x + nc * H * W;
        double* yp = y + nc * H * W;
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < W; ++j) {
                double m = xp[i * W + j];
                for (int di = 0; di < 2; ++di)
                    for (int dj = 0; dj < 2; ++dj) {
                        if (i + di >= H || j + dj >= W) continue;
                        double v = xp[(i + di) * W + j + dj];
                        if (v > m) m = v;
                    }
                yp[i * W + j] = m;
            }
    }
}

/* ---- rounding to the storage formats, for the quantisation-aware oracle --
 * Both are round-to-nearest, ties to even, from the exact double value.
 * bfloat16: 8 significant bits, exponent range of binary32.
 * E4M3 (OCP FP8): 4 significant bits, normals down to 2^-6, subnormals
 * spaced 2^-9, largest finite 448; "satfinite" clamps to +-448. */
static double round_sig(double v, int sig_bits, int min_exp) {
    /* v = f * 2^e with 0.5 <= |f| < 1: the leading bit has weight 2^(e-1),
     * the last kept bit 2^(e-sig_bits); below 2^min_exp the spacing stays
     * at 2^(min_exp-sig_bits+1) (subnormals). */
    if (v == 0.0 || !isfinite(v)) return v;
    int e;
    frexp(v, &e);
    int lead = e - 1;
    if (lead < min_exp) lead = min_exp;
    double q = ldexp(1.0, lead - (sig_bits - 1));
    return nearbyint(v / q) * q; /* default rounding mode: ties to even */
}

void oracle_round_bf16(double* v, long n) {
    for (long t = 0; t < n; ++t) v[t] = round_sig(v[t], 8, -126);
}

void oracle_round_e4m3_sat(double* v, long n) {
    for (long t = 0; t < n; ++t) {
        double r = round_sig(v[t], 4, -6);
        if (r > 448.0) r = 448.0;
        if (r < -448.0) r = -448.0;
        v[t] = r;
    }
}
