// noalloc.cu — one FP32 conv layer that allocates no device memory.
//
// Everything else in this library owns device memory it allocates itself
// (net_create's activation arena, the split-K workspace a plan grows).
// Some callers cannot allocate at call time: code that runs while a CUDA
// graph is being captured, real-time loops that forbid allocation after
// start-up, or hosts that hand the GPU to the library with a fixed memory
// budget.  net_conv2d_f32_noalloc serves them: the same split-K FP32
// implicit-GEMM conv kernels as the network path, with every intermediate
// (packed input, reordered weights, split-K partial sums) placed in one
// file-scope __device__ array of NET_NOALLOC_SCRATCH_BYTES.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/net.h"
#include "common.cuh"
#include "kernels.h"
#include "net_internal.h"

using namespace dn;

// Loaded into every device that loads the library, kept until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NET_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_addr[kMaxDevices];   // device address of the array, per device

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" net_status net_conv2d_f32_noalloc(const float* d_x, int n, int cin, int h, int w,
                                             const float* d_weight, const float* d_bias, int cout, int k,
                                             int act, int pool, float* d_y, void* cuda_stream) {
    if (!d_x || !d_weight || !d_bias || !d_y) return fail(NET_E_INVAL, "NULL argument");
    if (n < 1 || cin < 1 || h < 1 || w < 1 || cout < 1 || (k != 1 && k != 3) || act < 0 || act > 1 ||
        (pool != NET_POOL_NONE && pool != NET_POOL_2X2S2))
        return fail(NET_E_INVAL, "unsupported layer (n=%d cin=%d %dx%d cout=%d k=%d act=%d pool=%d)", n, cin, h,
                    w, cout, k, act, pool);
    if (pool == NET_POOL_2X2S2 && ((h & 1) || (w & 1)))
        return fail(NET_E_SHAPE, "2x2/s2 pool needs even size, got %dx%d", h, w);

    // ---- scratch plan (host arithmetic only)
    const int Cp = rup(cin, 4);
    const int KK = k * k;
    const int w_rows = rup(cout, 256);
    int bn, th, tw;
    simt_tile(cout, &bn, &th, &tw);
    const int tiles_x = cdiv(w, tw), tiles_y = cdiv(h, th);
    const int m_tiles = n * tiles_x * tiles_y;
    const int n_tiles = cdiv(cout, bn);
    const int nall = KK * cdiv(Cp, 8);
    int dev = 0, sms = 148;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(NET_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 148;
    int ksplit = 1;
    const int grid = m_tiles * n_tiles;
    if (grid < 2 * sms && nall >= 32) ksplit = std::max(1, std::min({cdiv(4 * sms, grid), nall / 16, 32}));
    const size_t b_s = up256(sizeof(double) * cout), b_amax = b_s, b_bias = up256(sizeof(float) * cout);
    const size_t b_x = up256((size_t)n * h * w * Cp * sizeof(float));
    const size_t b_w = up256((size_t)w_rows * KK * Cp * sizeof(float));
    const size_t b_ws = ksplit > 1 ? up256((size_t)ksplit * m_tiles * th * tw * n_tiles * bn * sizeof(float)) : 0;
    const size_t need = b_s + b_amax + b_bias + b_x + b_w + b_ws;
    if (need > (size_t)NET_NOALLOC_SCRATCH_BYTES)
        return fail(NET_E_INVAL, "layer needs %zu bytes of scratch, the static array holds %zu", need,
                    (size_t)NET_NOALLOC_SCRATCH_BYTES);

    // ---- per-device set-up: the array's device address (no allocation)
    if (dev < 0 || dev >= kMaxDevices) return fail(NET_E_INVAL, "device %d beyond %d", dev, kMaxDevices);
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return fail(NET_E_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            g_scratch_addr[dev] = static_cast<unsigned char*>(p);
        }
        base = g_scratch_addr[dev];
    }
    double* s_tmp = reinterpret_cast<double*>(base);
    double* s_amax = reinterpret_cast<double*>(base + b_s);
    float* s_bias = reinterpret_cast<float*>(base + b_s + b_amax);
    float* s_x = reinterpret_cast<float*>(base + b_s + b_amax + b_bias);
    float* s_w = reinterpret_cast<float*>(base + b_s + b_amax + b_bias + b_x);
    float* s_ws = reinterpret_cast<float*>(base + b_s + b_amax + b_bias + b_x + b_w);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    // ---- weights: reorder OIHW -> [w_rows][kh][kw][Cp] (rows and channels
    // beyond the layer are written as zeros, so no clearing is needed)
    FoldArgs fa{};
    fa.raw_w = d_weight;
    fa.bias = d_bias;
    fa.cout = cout;
    fa.cin = cin;
    fa.k = k;
    fa.Cp = Cp;
    fa.w_rows = w_rows;
    fa.dt = DT_F32;
    fa.out_w = s_w;
    fa.out_bias = s_bias;
    fa.tmp_s = s_tmp;
    fa.tmp_amax = s_amax;
    e = fold_layer(fa, st);
    // ---- input: NCHW -> NHWC with zero channel padding
    if (e == cudaSuccess) e = pack_frames(d_x, s_x, n, cin, h, w, Cp, DT_F32, 1.f, st);
    // ---- conv (+ split-K reduction), epilogue writes NCHW float32
    ConvLaunch c{};
    c.x = s_x;
    c.w = s_w;
    c.y = d_y;
    c.n = n;
    c.H = h;
    c.W = w;
    c.Cp = Cp;
    c.k = k;
    c.w_rows = w_rows;
    c.ep.bias = s_bias;
    c.ep.alpha = nullptr;
    c.ep.act = act;
    c.ep.pool = pool == NET_POOL_2X2S2 ? POOL_S2 : POOL_NONE;
    c.ep.out_dt = DT_F32;
    c.ep.out_layout = LAYOUT_NCHW;
    c.ep.out_cs = cout;
    c.ep.cout = cout;
    c.ksplit = ksplit;
    c.quads = 1;   // the scratch bound above assumes quad tiles
    c.ws = s_ws;
    if (e == cudaSuccess) e = conv_simt(c, st);
    if (e == cudaSuccess && ksplit > 1) {
        SplitReduce sr{s_ws, ksplit, m_tiles * th * tw, n_tiles * bn, tw, th, tiles_x, tiles_y, n, h, w, d_y, c.ep};
        e = splitk_reduce(sr, st);
    }
    if (e != cudaSuccess) return fail(NET_E_CUDA, "noalloc conv: %s", cudaGetErrorString(e));
    return NET_OK;
}
