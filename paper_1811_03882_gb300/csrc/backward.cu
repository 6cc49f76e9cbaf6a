// backward.cu — the "nightmare" pass: the gradient, with respect to the input
// frames, of the energy 1/2 * sum(output of layer L)^2 of one layer, and a
// gradient-ascent step on the frames.
//
// Paper Sec. 5.1.1: the offloaded Darknet benchmark runs the "nightmare"
// sample app, which changes an image so that it excites a chosen layer more.
// Everything stays on the device (Sec. 3.2): a forward pass that keeps each
// layer's activation before its pool, then the layers in reverse:
//   * max pool backward: each pooled output's gradient goes to the first
//     maximum of its window (scan (0,0), (0,1), (1,0), (1,1)); for the
//     stride-1 "same" pool a position sums the gradients of the windows it
//     wins (a gather, so no atomics and a fixed summation order);
//   * leaky backward: times 1 where the activation (same sign as the
//     pre-activation) is positive, 0.1 elsewhere — fused with the pool step;
//   * conv backward-data: dx[c](i,j) = sum_{o,kh,kw} dy[o](i-kh+p, j-kw+p)
//     W'[o,kh,kw,c] is a forward conv of dy with the weights transposed
//     (c <-> o) and flipped (kh, kw -> k-1-kh, k-1-kw), stride 1, pad p, so it
//     runs on the same CUDA-core conv kernel (and split-K reduction) as the
//     forward pass.  The batchnorm scale is folded into W', so its backward
//     comes with the weights; the bias has no input gradient.
// The pass runs on the FP32 path (handles created with NET_FP32 for every
// layer): gradients are accumulated in FP32.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/net.h"
#include "common.cuh"
#include "kernels.h"
#include "net_internal.h"

using namespace dn;

namespace dn {

struct NightState {
    int max_batch = 0, max_side = 0, nl = 0;
    std::vector<float*> h;      // per layer: activation before its pool, NHWC, channel stride rup(cout, 4)
    std::vector<float*> wt;     // per layer: transposed, flipped weights [rup(cin, 256)][k*k][rup(cout, 4)]
    float* a[2] = {nullptr, nullptr};   // forward inputs (pooled), NHWC
    float* g[2] = {nullptr, nullptr};   // gradients, NHWC
    float* zero_bias = nullptr;
    float* ws = nullptr;
    size_t ws_bytes = 0;
    float* grad = nullptr;      // net_nightmare_step: the frames' gradient, NCHW
    double* d_red = nullptr;    // per-frame reductions
    double* d_part = nullptr;   // their per-block parts
    double* h_red = nullptr;    // pinned host copy
};

void night_free(net* n) {
    NightState* S = n->night;
    if (!S) return;
    for (float* p : S->h) dn::dfree(p);
    for (float* p : S->wt) dn::dfree(p);
    dn::dfree(S->a[0]);
    dn::dfree(S->a[1]);
    dn::dfree(S->g[0]);
    dn::dfree(S->g[1]);
    dn::dfree(S->zero_bias);
    dn::dfree(S->ws);
    dn::dfree(S->grad);
    dn::dfree(S->d_red);
    dn::dfree(S->d_part);
    if (S->h_red) cudaFreeHost(S->h_red);
    delete S;
    n->night = nullptr;
}

}  // namespace dn

namespace {

// W_T[c][KK-1-t][o] = W'[o][t][c] (flip of both kernel indices = reversal of
// the tap index t = kh*k + kw); zero beyond cout / cin.
__global__ void transpose_flip_kernel(const float* __restrict__ w, int cin, int cout, int KK, int Cp,
                                      float* __restrict__ wt, int rows_t, int Cp_t) {
    const long long total = (long long)rows_t * KK * Cp_t;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int o = (int)(i % Cp_t);
        const long long r = i / Cp_t;
        const int tp = (int)(r % KK);
        const int c = (int)(r / KK);
        float v = 0.f;
        if (c < cin && o < cout) v = w[((long long)o * KK + (KK - 1 - tp)) * Cp + c];
        wt[i] = v;
    }
}

// 2x2 stride-2 max pool, NHWC float32 (the saving forward pass keeps the
// unpooled activation, so this pool runs on its own).
__global__ void maxpool_s2_kernel(const float* __restrict__ x, float* __restrict__ y, int n, int H, int W, int cs) {
    const int Ho = H / 2, Wo = W / 2;
    const long long total = (long long)n * Ho * Wo * cs;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % cs);
        long long r = i / cs;
        const int xo = (int)(r % Wo);
        r /= Wo;
        const int yo = (int)(r % Ho);
        const int img = (int)(r / Ho);
        const float* p = x + (((long long)img * H + 2 * yo) * W + 2 * xo) * cs + c;
        y[i] = fmaxf(fmaxf(p[0], p[cs]), fmaxf(p[(long long)W * cs], p[(long long)W * cs + cs]));
    }
}

enum { PB_NONE = 0, PB_S2 = 1, PB_S1 = 2 };

// First maximum of the 2x2 window at (wy, wx) of h (clipped at H, W), as a
// (dy, dx) code 0..3 in scan order.
__device__ __forceinline__ int first_max(const float* h, int H, int W, int cs, int wy, int wx) {
    float best = h[((long long)wy * W + wx) * cs];
    int arg = 0;
#pragma unroll
    for (int q = 1; q < 4; ++q) {
        const int yy = wy + (q >> 1), xx = wx + (q & 1);
        if (yy < H && xx < W) {
            const float v = h[((long long)yy * W + xx) * cs];
            if (v > best) {
                best = v;
                arg = q;
            }
        }
    }
    return arg;
}

// Gradient of one layer's activation (before its pool) from the gradient of
// its output, times the leaky slope: g_h (n, H, W, cs) from g_out.
template <int MODE>
__global__ void pool_leaky_bwd_kernel(const float* __restrict__ gout, const float* __restrict__ h,
                                      float* __restrict__ gh, int n, int H, int W, int cs, int cout, int leaky) {
    const long long total = (long long)n * H * W * cs;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % cs);
        long long r = i / cs;
        const int x = (int)(r % W);
        r /= W;
        const int y = (int)(r % H);
        const int img = (int)(r / H);
        float g = 0.f;
        if (c < cout) {
            const float* hp = h + (long long)img * H * W * cs + c;   // this image and channel
            if (MODE == PB_NONE) {
                g = gout[i];
            } else if (MODE == PB_S2) {
                const int wy = y & ~1, wx = x & ~1;
                const int q = ((y - wy) << 1) | (x - wx);
                if (first_max(hp, H, W, cs, wy, wx) == q)
                    g = gout[(((long long)img * (H / 2) + (y >> 1)) * (W / 2) + (x >> 1)) * cs + c];
            } else {
                // windows anchored at (y, x), (y, x-1), (y-1, x), (y-1, x-1) that
                // contain (y, x); each sends its gradient if (y, x) is its first max
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int wy = y - (q >> 1), wx = x - (q & 1);
                    if (wy >= 0 && wx >= 0 && first_max(hp, H, W, cs, wy, wx) == q)
                        g += gout[(((long long)img * H + wy) * W + wx) * cs + c];
                }
            }
            if (leaky && !(hp[((long long)y * W + x) * cs] > 0.f)) g *= kLeakySlope;
        }
        gh[i] = g;
    }
}

// Per-frame sum of v^2 (kind 0) or |v| (kind 1) over `count` floats at
// stride `fstride`, in FP64, in two passes with a fixed summation order (so
// deterministic): kRedParts blocks per frame each sum a contiguous part
// into part[frame][block] (grid kRedParts x frames), then one thread per
// frame adds the parts in order.
constexpr int kRedParts = 64;
__global__ void frame_reduce_parts_kernel(const float* __restrict__ v, long long count, long long fstride, int kind,
                                          double* part) {
    const float* p = v + blockIdx.y * fstride;
    const long long per = (count + kRedParts - 1) / kRedParts;
    const long long b = blockIdx.x * per, e = min(count, b + per);
    double s = 0.0;
    for (long long i = b + threadIdx.x; i < e; i += blockDim.x) {
        const double t = p[i];
        s += kind == 0 ? t * t : fabs(t);
    }
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.y * kRedParts + blockIdx.x] = red[0];
}

__global__ void frame_reduce_sum_kernel(const double* __restrict__ part, int frames, double* out) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= frames) return;
    double s = 0.0;
    for (int b = 0; b < kRedParts; ++b) s += part[f * kRedParts + b];
    out[f] = s;
}

// x += rate * g / mean|g| per frame (mean from frame_reduce_kernel's sums).
__global__ void ascent_kernel(float* x, const float* __restrict__ g, long long per_frame, int n,
                              const double* __restrict__ sum_abs, float rate) {
    const long long total = per_frame * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(i / per_frame);
        const double m = sum_abs[f] / (double)per_frame;
        x[i] += (float)((double)rate * g[i] / (m > 1e-30 ? m : 1e-30));
    }
}

cudaError_t frame_reduce(const float* v, long long count, long long fstride, int kind, int frames, double* part,
                         double* out, cudaStream_t st) {
    frame_reduce_parts_kernel<<<dim3(kRedParts, frames), 256, 0, st>>>(v, count, fstride, kind, part);
    frame_reduce_sum_kernel<<<(frames + 127) / 128, 128, 0, st>>>(part, frames, out);
    return cudaGetLastError();
}

unsigned grid_for(long long total, int threads) {
    return (unsigned)std::min<long long>((total + threads - 1) / threads, 152LL * 16);
}

}  // namespace

#define NK(call)                                                                                      \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return fail(e_ == cudaErrorMemoryAllocation ? NET_E_OOM : NET_E_CUDA, "%s: %s", #call,   \
                        cudaGetErrorString(e_));                                                      \
    } while (0)

static net_status night_setup(net* n) {
    if (n->night) return NET_OK;
    for (auto& L : n->L)
        if (L.engine != ENG_SIMT || L.in_dt != DT_F32)
            return fail(NET_E_UNSUPPORTED, "the nightmare pass runs on FP32 handles (every layer NET_FP32)");
    NightState* S = new NightState();
    n->night = S;
    S->max_batch = n->max_batch;
    S->max_side = n->max_side;
    S->nl = (int)n->L.size();
    std::vector<int> H, W;
    layer_dims(n, n->max_side, n->max_side, H, W);
    size_t amax = 0, gmax = 0;
    int rows_max = 0;
    for (int l = 0; l < S->nl; ++l) {
        const Layer& L = n->L[l];
        const int cs = rup(L.d.cout, 4);
        // the conv's output size is its input size (the pool follows)
        const size_t hb = (size_t)n->max_batch * H[l] * W[l] * cs * sizeof(float);
        float* p = nullptr;
        NK(dn::dalloc(&p, hb));
        S->h.push_back(p);
        amax = std::max(amax, (size_t)n->max_batch * H[l] * W[l] * std::max(cs, L.in_cs) * sizeof(float));
        gmax = std::max(gmax, (size_t)n->max_batch * H[l] * W[l] * std::max(cs, L.in_cs) * sizeof(float));
        const int KK = L.d.k * L.d.k, rows_t = rup(L.cin, 256);
        rows_max = std::max(rows_max, rows_t);
        float* w = nullptr;
        NK(dn::dalloc(&w, (size_t)rows_t * KK * cs * sizeof(float)));
        S->wt.push_back(w);
    }
    for (int b = 0; b < 2; ++b) {
        NK(dn::dalloc(&S->a[b], amax));
        NK(dn::dalloc(&S->g[b], gmax));
    }
    NK(dn::dalloc(&S->zero_bias, rows_max * sizeof(float)));
    NK(cudaMemsetAsync(S->zero_bias, 0, rows_max * sizeof(float), n->stream));
    NK(dn::dalloc(&S->grad, (size_t)n->max_batch * n->in_c * n->max_side * n->max_side * sizeof(float)));
    NK(dn::dalloc(&S->d_red, sizeof(double) * n->max_batch));
    NK(dn::dalloc(&S->d_part, sizeof(double) * n->max_batch * kRedParts));
    NK(cudaHostAlloc(&S->h_red, sizeof(double) * n->max_batch, cudaHostAllocDefault));
    return NET_OK;
}

// Weights of the backward convs, from the handle's folded FP32 weights.
static net_status night_weights(net* n) {
    NightState* S = n->night;
    for (int l = 0; l < S->nl; ++l) {
        const Layer& L = n->L[l];
        const int KK = L.d.k * L.d.k, cs = rup(L.d.cout, 4), rows_t = rup(L.cin, 256);
        const long long total = (long long)rows_t * KK * cs;
        transpose_flip_kernel<<<grid_for(total, 256), 256, 0, n->stream>>>(
            reinterpret_cast<const float*>(L.w), L.cin, L.d.cout, KK, L.in_cs, S->wt[l], rows_t, cs);
        NK(cudaGetLastError());
        ++n->launches;
    }
    return NET_OK;
}

// One CUDA-core conv (+ split-K reduction) of the nightmare pass.
static net_status night_conv(net* n, const void* x, const void* w, int w_rows, void* y, int batch, int H, int W,
                             int Cp, int k, const Epilogue& ep) {
    NightState* S = n->night;
    const int nc = ep.out_layout == LAYOUT_NCHW ? ep.cout : std::max(ep.out_cs, ep.cout);
    const SimtGeom g = simt_geom(nc, ep.pool == POOL_S2, batch, H, W, false);
    const int bn = g.bn;
    const int m_tiles = g.m_tiles, n_tiles = cdiv(nc, bn);
    const int grid = m_tiles * n_tiles, nall = k * k * cdiv(Cp, 8);
    int ks = 1;
    if (grid < 2 * n->num_sms && nall >= 32) ks = std::max(1, std::min({cdiv(4 * n->num_sms, grid), nall / 16, 32}));
    if (ks > 1) {
        const size_t need = (size_t)ks * m_tiles * g.px * n_tiles * bn * sizeof(float);
        if (need > S->ws_bytes) {
            NK(cudaStreamSynchronize(n->stream));
            dn::dfree(S->ws);
            S->ws = nullptr;
            S->ws_bytes = 0;
            NK(dn::dalloc(&S->ws, need));
            S->ws_bytes = need;
        }
    }
    ConvLaunch c{};
    c.x = x;
    c.w = w;
    c.y = y;
    c.n = batch;
    c.H = H;
    c.W = W;
    c.Cp = Cp;
    c.k = k;
    c.w_rows = w_rows;
    c.ep = ep;
    c.ksplit = ks;
    c.ws = S->ws;
    NK(conv_simt(c, n->stream));
    ++n->launches;
    if (ks > 1) {
        SplitReduce sr{S->ws, ks, m_tiles * g.px, n_tiles * bn, g.red_tw, g.red_th, g.red_tx, g.red_ty, batch, H, W,
                       y, ep};
        NK(splitk_reduce(sr, n->stream));
        ++n->launches;
    }
    return NET_OK;
}

// Forward through `layer` keeping activations, then the gradient back to the
// frames (NCHW float32 into d_grad); J = 1/2 sum(output of layer)^2 per frame
// into S->d_red.
static net_status night_grad(net* n, const float* d_in, int batch, int h, int w, int layer, float* d_grad,
                             float* const* t_act = nullptr, float* const* t_gout = nullptr) {
    NightState* S = n->night;
    cudaStream_t st = n->stream;
    std::vector<int> H, W;
    layer_dims(n, h, w, H, W);
    // ---- forward, keeping each layer's activation before its pool
    NK(pack_frames(d_in, S->a[0], batch, n->in_c, h, w, n->L[0].in_cs, DT_F32, 1.f, st));
    ++n->launches;
    const float* x = S->a[0];
    int ab = 0;
    for (int l = 0; l <= layer; ++l) {
        const Layer& L = n->L[l];
        const int cs = rup(L.d.cout, 4);
        Epilogue ep{};
        ep.bias = L.bias;
        ep.act = L.d.act;
        ep.pool = POOL_NONE;
        ep.out_dt = DT_F32;
        ep.out_layout = LAYOUT_NHWC;
        ep.out_cs = cs;
        ep.out_inv_scale = 1.f;
        ep.cout = L.d.cout;
        net_status s = night_conv(n, x, L.w, L.w_rows, S->h[l], batch, H[l], W[l], L.in_cs, L.d.k, ep);
        if (s != NET_OK) return s;
        if (t_act && t_act[l]) {
            NK(unpack_nchw(S->h[l], t_act[l], batch, L.d.cout, H[l], W[l], cs, DT_F32, 1.f, st));
            ++n->launches;
        }
        if (L.d.pool == NET_POOL_2X2S2) {
            ab ^= 1;
            const long long tot = (long long)batch * H[l + 1] * W[l + 1] * cs;
            maxpool_s2_kernel<<<grid_for(tot, 256), 256, 0, st>>>(S->h[l], S->a[ab], batch, H[l], W[l], cs);
            NK(cudaGetLastError());
            ++n->launches;
            x = S->a[ab];
        } else if (L.d.pool == NET_POOL_2X2S1_SAME) {
            ab ^= 1;
            NK(maxpool_s1_same(S->h[l], S->a[ab], batch, H[l], W[l], cs, DT_F32, st));
            ++n->launches;
            x = S->a[ab];
        } else {
            x = S->h[l];
        }
    }
    // objective per frame: the output of `layer` (padded channels are zero)
    const int csL = rup(n->L[layer].d.cout, 4);
    const long long per_frame = (long long)H[layer + 1] * W[layer + 1] * csL;
    NK(frame_reduce(x, per_frame, per_frame, 0, batch, S->d_part, S->d_red, st));
    n->launches += 2;
    // ---- backward: dJ/d(output of layer) = that output.  g[1] holds the
    // gradient before a layer's pool and leaky, g[0] the one after its conv
    // (the next layer down's output gradient): no kernel reads the buffer it
    // writes.
    const float* gout = x;
    for (int l = layer; l >= 0; --l) {
        const Layer& L = n->L[l];
        const int cs = rup(L.d.cout, 4);
        const long long tot = (long long)batch * H[l] * W[l] * cs;
        float* gh = S->g[1];
        if (t_gout && t_gout[l]) {
            NK(unpack_nchw(gout, t_gout[l], batch, L.d.cout, H[l + 1], W[l + 1], cs, DT_F32, 1.f, st));
            ++n->launches;
        }
        const int leaky = L.d.act == NET_ACT_LEAKY ? 1 : 0;
        if (L.d.pool == NET_POOL_2X2S2)
            pool_leaky_bwd_kernel<PB_S2><<<grid_for(tot, 256), 256, 0, st>>>(gout, S->h[l], gh, batch, H[l], W[l], cs,
                                                                              L.d.cout, leaky);
        else if (L.d.pool == NET_POOL_2X2S1_SAME)
            pool_leaky_bwd_kernel<PB_S1><<<grid_for(tot, 256), 256, 0, st>>>(gout, S->h[l], gh, batch, H[l], W[l], cs,
                                                                              L.d.cout, leaky);
        else
            pool_leaky_bwd_kernel<PB_NONE><<<grid_for(tot, 256), 256, 0, st>>>(gout, S->h[l], gh, batch, H[l], W[l],
                                                                                cs, L.d.cout, leaky);
        NK(cudaGetLastError());
        ++n->launches;
        // conv backward-data: a conv of gh (cs channels) with the transposed,
        // flipped weights to cin channels
        Epilogue ep{};
        ep.bias = S->zero_bias;
        ep.act = ACT_LINEAR;
        ep.pool = POOL_NONE;
        ep.out_dt = DT_F32;
        ep.out_inv_scale = 1.f;
        ep.cout = L.cin;
        void* y;
        if (l == 0) {
            ep.out_layout = LAYOUT_NCHW;
            ep.out_cs = L.cin;
            y = d_grad;
        } else {
            ep.out_layout = LAYOUT_NHWC;
            ep.out_cs = L.in_cs;
            y = S->g[0];
        }
        net_status s = night_conv(n, gh, S->wt[l], rup(L.cin, 256), y, batch, H[l], W[l], cs, L.d.k, ep);
        if (s != NET_OK) return s;
        gout = S->g[0];
    }
    return NET_OK;
}

static net_status night_check(net* n, const void* p, int batch, int h, int w, int layer) {
    if (!n || !p) return fail(NET_E_INVAL, "NULL argument");
    if (!n->weights_loaded) return fail(NET_E_WEIGHTS, "weights not loaded");
    if (layer < 0 || layer >= (int)n->L.size()) return fail(NET_E_INVAL, "layer %d out of range", layer);
    net_status s = check_shape(n, batch, h, w);
    if (s != NET_OK) return s;
    NK(cudaSetDevice(n->device));
    const bool fresh = n->night == nullptr;
    s = night_setup(n);
    if (s != NET_OK) {
        night_free(n);
        return s;
    }
    if (fresh || n->night_weights_stale) {
        s = night_weights(n);
        if (s != NET_OK) return s;
        n->night_weights_stale = false;
    }
    return NET_OK;
}

extern "C" net_status net_nightmare_grad(net_t* n, const float* d_in, int batch, int h, int w, int layer,
                                         float* d_grad, double* objective) {
    if (!d_grad) return fail(NET_E_INVAL, "NULL argument");
    net_status s = night_check(n, d_in, batch, h, w, layer);
    if (s != NET_OK) return s;
    s = night_grad(n, d_in, batch, h, w, layer, d_grad);
    if (s != NET_OK) return s;
    NK(cudaMemcpyAsync(n->night->h_red, n->night->d_red, sizeof(double) * batch, cudaMemcpyDeviceToHost, n->stream));
    NK(cudaStreamSynchronize(n->stream));
    if (objective)
        for (int f = 0; f < batch; ++f) objective[f] = 0.5 * n->night->h_red[f];
    return check_device_error(n);
}

extern "C" net_status net_nightmare_trace(net_t* n, const float* d_in, int batch, int h, int w, int layer,
                                          float* d_grad, float* const* d_act, float* const* d_gout) {
    if (!d_grad || !d_act || !d_gout) return fail(NET_E_INVAL, "NULL argument");
    net_status s = night_check(n, d_in, batch, h, w, layer);
    if (s != NET_OK) return s;
    s = night_grad(n, d_in, batch, h, w, layer, d_grad, d_act, d_gout);
    if (s != NET_OK) return s;
    NK(cudaStreamSynchronize(n->stream));
    return check_device_error(n);
}

extern "C" net_status net_nightmare_step(net_t* n, float* d_frames, int batch, int h, int w, int layer, float rate,
                                         double* objective) {
    if (!std::isfinite(rate)) return fail(NET_E_INVAL, "rate %g", (double)rate);
    net_status s = night_check(n, d_frames, batch, h, w, layer);
    if (s != NET_OK) return s;
    NightState* S = n->night;
    s = night_grad(n, d_frames, batch, h, w, layer, S->grad);
    if (s != NET_OK) return s;
    NK(cudaMemcpyAsync(S->h_red, S->d_red, sizeof(double) * batch, cudaMemcpyDeviceToHost, n->stream));
    const long long per = (long long)n->in_c * h * w;
    NK(frame_reduce(S->grad, per, per, 1, batch, S->d_part, S->d_red, n->stream));
    ascent_kernel<<<grid_for(per * batch, 256), 256, 0, n->stream>>>(d_frames, S->grad, per, batch, S->d_red, rate);
    NK(cudaGetLastError());
    n->launches += 3;
    NK(cudaStreamSynchronize(n->stream));
    if (objective)
        for (int f = 0; f < batch; ++f) objective[f] = 0.5 * S->h_red[f];
    return check_device_error(n);
}
