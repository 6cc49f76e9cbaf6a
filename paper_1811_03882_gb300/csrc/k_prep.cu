// k_prep.cu — memory-bound helper kernels: frame pack, result unpack,
// stride-1 "same" max pool, one-time FP64 batchnorm fold and FP8 weight
// quantisation, FP8 scale helpers.
#include "common.cuh"
#include "kernels.h"

namespace dn {

static inline unsigned grid_for(size_t n, int threads) {
    size_t b = (n + threads - 1) / threads;
    if (b > 152u * 32u) b = 152u * 32u;   // grid-stride beyond 32 CTAs per SM
    return (unsigned)(b ? b : 1);
}

// ---------------------------------------------------------------- pack
// The frame pack opens a forward pass, so it also clears the pass's
// row-band counters (zero[0 .. nzero - 1], spread over the grid): the conv
// layers after it count from zero.
__device__ __forceinline__ void clear_counters(int* zero, int nzero) {
    // the first conv layer may start its prologue now (it waits for this
    // kernel's completion before it reads the frames): 0.3658 -> 0.3626 ms
    // per 19-conv 448^2 b8 pass
    pdl_trigger();
    const int b = blockIdx.y * gridDim.x + blockIdx.x;
    for (int i = b * blockDim.x + threadIdx.x; i < nzero; i += gridDim.x * gridDim.y * blockDim.x) zero[i] = 0;
}

// One grid row (blockIdx.y) per frame; a thread per (pixel, group of 16
// bytes); 32-bit indices within a frame (the host checks the size).
template <int DT>
__global__ void pack_kernel(const float* __restrict__ x, void* __restrict__ y, int C, int HW, int Cp,
                            FastDiv fd_groups, float inv_scale, int* zero, int nzero) {
    clear_counters(zero, nzero);
    constexpr int V = DT == DT_F32 ? 4 : DT == DT_BF16 ? 8 : 16;   // elements per 16 B
    const int groups = Cp / V;
    const int nn = blockIdx.y;
    const int total = HW * groups;
    const float* xf = x + (size_t)nn * C * HW;
    uint8_t* yf = reinterpret_cast<uint8_t*>(y) + (size_t)nn * HW * Cp * dt_size(DT);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int yx = groups == 1 ? i : fdiv(i, fd_groups);
        const int g = i - yx * groups;
        float v[V];
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const int c = g * V + j;
            v[j] = c < C ? xf[(size_t)c * HW + yx] : 0.f;
        }
        uint8_t* dst = yf + ((size_t)yx * Cp + (size_t)g * V) * dt_size(DT);
        if (DT == DT_F32) {
            *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
        } else if (DT == DT_BF16) {
            uint4 pk;
            uint32_t* p = reinterpret_cast<uint32_t*>(&pk);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                p[j] = *reinterpret_cast<uint32_t*>(&b);
            }
            *reinterpret_cast<uint4*>(dst) = pk;
        } else {
            uint4 pk;
            uint8_t* p = reinterpret_cast<uint8_t*>(&pk);
#pragma unroll
            for (int j = 0; j < 16; ++j) p[j] = f32_to_e4m3_sat(v[j] * inv_scale);
            *reinterpret_cast<uint4*>(dst) = pk;
        }
    }
}

// BF16, at most 8 channels padded to 8 (one 16-byte group per pixel), the
// frame's pixel count a multiple of 4: a thread packs four adjacent pixels
// from one float4 load per channel and stores their 64 contiguous bytes.
__global__ void pack_bf16_c8_px4_kernel(const float* __restrict__ x, void* __restrict__ y, int C, int HW4, int* zero,
                                        int nzero) {
    clear_counters(zero, nzero);
    const int nn = blockIdx.y;
    const int HW = HW4 * 4;
    const float4* xf = reinterpret_cast<const float4*>(x + (size_t)nn * C * HW);
    uint4* yf = reinterpret_cast<uint4*>(y) + (size_t)nn * HW;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < HW4; i += gridDim.x * blockDim.x) {
        float v[8][4];   // [channel][pixel]
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float4 t = c < C ? xf[(size_t)c * HW4 + i] : make_float4(0.f, 0.f, 0.f, 0.f);
            v[c][0] = t.x;
            v[c][1] = t.y;
            v[c][2] = t.z;
            v[c][3] = t.w;
        }
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            uint4 pk;
            uint32_t* w = reinterpret_cast<uint32_t*>(&pk);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * j][p], v[2 * j + 1][p]);
                w[j] = *reinterpret_cast<uint32_t*>(&b);
            }
            yf[(size_t)4 * i + p] = pk;
        }
    }
}

cudaError_t pack_frames(const float* x, void* y, int n, int C, int H, int W, int Cp, int dt,
                        float inv_scale, cudaStream_t st, int* zero, int nzero) {
    if (nzero > 0 && (n <= 0 || (size_t)H * W == 0)) {
        const cudaError_t e = cudaMemsetAsync(zero, 0, (size_t)nzero * sizeof(int), st);
        if (e != cudaSuccess) return e;
        nzero = 0;
    }
    if (dt == DT_BF16 && Cp == 8 && C <= 8 && n > 0 && n <= 65535 && ((size_t)H * W) % 4 == 0 &&
        (size_t)H * W < (size_t)INT32_MAX && ((uintptr_t)x & 15) == 0 && ((uintptr_t)y & 15) == 0) {
        const int HW4 = H * W / 4;
        unsigned bx = (unsigned)((HW4 + 255) / 256);
        const unsigned cap = (152u * 32u + (unsigned)n - 1) / (unsigned)n;
        if (bx > cap) bx = cap;
        pack_bf16_c8_px4_kernel<<<dim3(bx ? bx : 1, (unsigned)n), 256, 0, st>>>(x, y, C, HW4, zero, nzero);
        return cudaGetLastError();
    }
    const int V = dt == DT_F32 ? 4 : dt == DT_BF16 ? 8 : 16;
    const size_t per = (size_t)H * W * (Cp / V);
    if (n <= 0 || per == 0) return cudaSuccess;
    if (per >= (size_t)INT32_MAX || n > 65535 || Cp % V != 0) return cudaErrorInvalidValue;
    unsigned bx = (unsigned)((per + 255) / 256);
    const unsigned cap = (152u * 32u + (unsigned)n - 1) / (unsigned)n;   // grid-stride beyond ~32 CTAs per SM
    if (bx > cap) bx = cap;
    const dim3 g(bx ? bx : 1, (unsigned)n);
    const FastDiv fg = make_fast_div(Cp / V);
    const int HW = H * W;
    if (dt == DT_F32) pack_kernel<DT_F32><<<g, 256, 0, st>>>(x, y, C, HW, Cp, fg, inv_scale, zero, nzero);
    else if (dt == DT_BF16) pack_kernel<DT_BF16><<<g, 256, 0, st>>>(x, y, C, HW, Cp, fg, inv_scale, zero, nzero);
    else pack_kernel<DT_FP8><<<g, 256, 0, st>>>(x, y, C, HW, Cp, fg, inv_scale, zero, nzero);
    return cudaGetLastError();
}

template <int DT>
__device__ __forceinline__ void store_vec(uint8_t* dst, const float* v, float inv_scale) {
    if (DT == DT_F32) {
        *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
    } else if (DT == DT_BF16) {
        uint4 pk;
        uint32_t* p = reinterpret_cast<uint32_t*>(&pk);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
            p[j] = *reinterpret_cast<uint32_t*>(&b);
        }
        *reinterpret_cast<uint4*>(dst) = pk;
    } else {
        uint4 pk;
        uint8_t* p = reinterpret_cast<uint8_t*>(&pk);
#pragma unroll
        for (int j = 0; j < 16; ++j) p[j] = f32_to_e4m3_sat(v[j] * inv_scale);
        *reinterpret_cast<uint4*>(dst) = pk;
    }
}

// One thread per output pixel: the C*K*K taps are read with neighbouring
// threads on neighbouring pixels (coalesced), and the pixel's 32 channels
// are written as whole 16-byte vectors.  C and K are compile-time so the
// 32 values stay in registers.
template <int DT, int C, int K>
__device__ __forceinline__ void im2col_pixel(const float* __restrict__ x, int H, int W, int yy, int xx,
                                             uint8_t* dst, float inv_scale) {
    constexpr int V = DT == DT_F32 ? 4 : DT == DT_BF16 ? 8 : 16;
    constexpr int CP = 32;
    static_assert(C * K * K <= CP, "im2col layout holds 32 channels");
    float v[CP];
#pragma unroll
    for (int j = 0; j < CP; ++j) v[j] = 0.f;
#pragma unroll
    for (int tap = 0; tap < K * K; ++tap) {
        const int iy = yy + tap / K - K / 2, ix = xx + tap % K - K / 2;
        if (iy >= 0 && iy < H && ix >= 0 && ix < W) {
#pragma unroll
            for (int c = 0; c < C; ++c) v[tap * C + c] = __ldg(x + ((size_t)c * H + iy) * W + ix);
        }
    }
#pragma unroll
    for (int g = 0; g < CP / V; ++g) store_vec<DT>(dst + (size_t)g * V * dt_size(DT), v + g * V, inv_scale);
}

template <int DT>
__device__ __forceinline__ void im2col_dispatch(const float* x, int C, int H, int W, int yy, int xx, uint8_t* dst,
                                                float inv_scale) {
    if (C == 3) im2col_pixel<DT, 3, 3>(x, H, W, yy, xx, dst, inv_scale);
    else if (C == 2) im2col_pixel<DT, 2, 3>(x, H, W, yy, xx, dst, inv_scale);
    else im2col_pixel<DT, 1, 3>(x, H, W, yy, xx, dst, inv_scale);
}

template <int DT>
__global__ void pack_im2col_kernel(const float* __restrict__ x, void* __restrict__ y, int n, int C, int H, int W,
                                   int Cp, int k, float inv_scale) {
    const size_t HW = (size_t)H * W;
    const size_t total = (size_t)n * HW;
    for (size_t pix = blockIdx.x * (size_t)blockDim.x + threadIdx.x; pix < total;
         pix += (size_t)gridDim.x * blockDim.x) {
        const size_t nn = pix / HW, yx = pix % HW;
        uint8_t* dst = reinterpret_cast<uint8_t*>(y) + pix * Cp * dt_size(DT);
        im2col_dispatch<DT>(x + nn * C * HW, C, H, W, (int)(yx / W), (int)(yx % W), dst, inv_scale);
    }
}

cudaError_t pack_frames_im2col(const float* x, void* y, int n, int C, int H, int W, int Cp, int k, int dt,
                               float inv_scale, cudaStream_t st) {
    // the first-layer im2col layout: 32 channels, a 3x3 kernel over <= 3 channels
    if (Cp != 32 || k != 3 || C < 1 || C > 3) return cudaErrorInvalidValue;
    const size_t total = (size_t)n * H * W;
    const unsigned g = grid_for(total, 256);
    if (dt == DT_F32) pack_im2col_kernel<DT_F32><<<g, 256, 0, st>>>(x, y, n, C, H, W, Cp, k, inv_scale);
    else if (dt == DT_BF16) pack_im2col_kernel<DT_BF16><<<g, 256, 0, st>>>(x, y, n, C, H, W, Cp, k, inv_scale);
    else pack_im2col_kernel<DT_FP8><<<g, 256, 0, st>>>(x, y, n, C, H, W, Cp, k, inv_scale);
    return cudaGetLastError();
}

template <typename J>
__device__ __forceinline__ int find_job(const J* jobs, int njobs, long long i) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].begin <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int DT>
__global__ void pack_grouped_kernel(const PackJob* __restrict__ jobs, int njobs, long long total,
                                    float inv_scale) {
    constexpr int V = DT == DT_F32 ? 4 : DT == DT_BF16 ? 8 : 16;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const PackJob& J = jobs[find_job(jobs, njobs, i)];
        const long long li = i - J.begin;
        if (J.im2col_k) {   // one work item per pixel (the job counts pixels)
            uint8_t* dst = reinterpret_cast<uint8_t*>(J.dst) + li * J.Cp * dt_size(DT);
            im2col_dispatch<DT>(J.src, J.C, J.H, J.W, (int)(li / J.W), (int)(li % J.W), dst, inv_scale);
            continue;
        }
        const int groups = J.Cp / V;
        const int g = (int)(li % groups);
        const long long yx = li / groups;
        const long long HW = (long long)J.H * J.W;
        float v[V];
        {
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const int c = g * V + j;
                v[j] = c < J.C ? J.src[c * HW + yx] : 0.f;
            }
        }
        store_vec<DT>(reinterpret_cast<uint8_t*>(J.dst) + (yx * J.Cp + (long long)g * V) * dt_size(DT), v, inv_scale);
    }
}

cudaError_t pack_frames_grouped(const PackJob* jobs, int njobs, long long total, int dt, float inv_scale,
                                cudaStream_t st) {
    const unsigned g = grid_for((size_t)total, 256);
    if (dt == DT_F32) pack_grouped_kernel<DT_F32><<<g, 256, 0, st>>>(jobs, njobs, total, inv_scale);
    else if (dt == DT_BF16) pack_grouped_kernel<DT_BF16><<<g, 256, 0, st>>>(jobs, njobs, total, inv_scale);
    else pack_grouped_kernel<DT_FP8><<<g, 256, 0, st>>>(jobs, njobs, total, inv_scale);
    return cudaGetLastError();
}

// -------------------------------------------------------------- unpack
__device__ __forceinline__ float load_as_f32(const void* base, size_t i, int dt, float scale) {
    if (dt == DT_F32) return reinterpret_cast<const float*>(base)[i];
    if (dt == DT_BF16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(base)[i]);
    return e4m3_to_f32(reinterpret_cast<const uint8_t*>(base)[i]) * scale;
}

__global__ void unpack_kernel(const void* __restrict__ x, float* __restrict__ y, int n, int C, int H,
                              int W, int cs, int dt, float scale) {
    const size_t HW = (size_t)H * W, total = (size_t)n * C * HW;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t yx = i % HW, nc = i / HW;
        const int c = (int)(nc % C);
        const size_t nn = nc / C;
        y[i] = load_as_f32(x, (nn * HW + yx) * cs + c, dt, scale);
    }
}

cudaError_t unpack_nchw(const void* x, float* y, int n, int C, int H, int W, int cs, int dt,
                        float scale, cudaStream_t st) {
    const size_t total = (size_t)n * C * H * W;
    unpack_kernel<<<grid_for(total, 256), 256, 0, st>>>(x, y, n, C, H, W, cs, dt, scale);
    return cudaGetLastError();
}

// ------------------------------------------------------- s1 "same" pool
// out(i,j) = max over rows i..i+1, cols j..j+1 inside the image.  Max of
// values in one storage format is one of them, so no re-rounding happens.
__device__ __forceinline__ float dec(const uint8_t* p, int j, int dt) {
    if (dt == DT_F32) return reinterpret_cast<const float*>(p)[j];
    if (dt == DT_BF16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[j]);
    return e4m3_to_f32(p[j]);
}

__global__ void pool_s1_kernel(const uint8_t* __restrict__ x, uint8_t* __restrict__ y, int n, int H,
                               int W, int cs, int dt) {
    pdl_trigger();
    pdl_wait();
    const int esz = dt == DT_F32 ? 4 : dt == DT_BF16 ? 2 : 1;
    const int V = 16 / esz;
    const int groups = cs / V;
    const size_t total = (size_t)n * H * W * groups;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int g = (int)(i % groups);
        size_t pix = i / groups;
        const int xx = (int)(pix % W);
        const int yy = (int)((pix / W) % H);
        const size_t rowb = (size_t)cs * esz;
        const uint8_t* p00 = x + pix * rowb + (size_t)g * 16;
        uint4 best = *reinterpret_cast<const uint4*>(p00);
        for (int d = 1; d < 4; ++d) {
            const int dy = d >> 1, dx = d & 1;
            if (yy + dy >= H || xx + dx >= W) continue;
            const uint8_t* q = p00 + ((size_t)dy * W + dx) * rowb;
            uint4 cand = *reinterpret_cast<const uint4*>(q);
            uint8_t* bb = reinterpret_cast<uint8_t*>(&best);
            const uint8_t* cb = reinterpret_cast<const uint8_t*>(&cand);
            for (int j = 0; j < V; ++j)
                if (dec(cb, j, dt) > dec(bb, j, dt))
                    for (int b = 0; b < esz; ++b) bb[j * esz + b] = cb[j * esz + b];
        }
        *reinterpret_cast<uint4*>(y + pix * rowb + (size_t)g * 16) = best;
    }
}

__global__ void pool_s1_grouped_kernel(const PoolJob* __restrict__ jobs, int njobs, long long total, int cs,
                                       int dt) {
    pdl_trigger();
    pdl_wait();
    const int esz = dt == DT_F32 ? 4 : dt == DT_BF16 ? 2 : 1;
    const int V = 16 / esz;
    const int groups = cs / V;
    const size_t rowb = (size_t)cs * esz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const PoolJob& J = jobs[find_job(jobs, njobs, i)];
        const long long li = i - J.begin;
        const int g = (int)(li % groups);
        const long long pix = li / groups;
        const int xx = (int)(pix % J.W), yy = (int)(pix / J.W);
        const uint8_t* x = reinterpret_cast<const uint8_t*>(J.x);
        const uint8_t* p00 = x + pix * rowb + (size_t)g * 16;
        uint4 best = *reinterpret_cast<const uint4*>(p00);
        for (int d = 1; d < 4; ++d) {
            const int dy = d >> 1, dx = d & 1;
            if (yy + dy >= J.H || xx + dx >= J.W) continue;
            uint4 cand = *reinterpret_cast<const uint4*>(p00 + ((size_t)dy * J.W + dx) * rowb);
            uint8_t* bb = reinterpret_cast<uint8_t*>(&best);
            const uint8_t* cb = reinterpret_cast<const uint8_t*>(&cand);
            for (int j = 0; j < V; ++j)
                if (dec(cb, j, dt) > dec(bb, j, dt))
                    for (int b = 0; b < esz; ++b) bb[j * esz + b] = cb[j * esz + b];
        }
        *reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(J.y) + pix * rowb + (size_t)g * 16) = best;
    }
}

cudaError_t maxpool_s1_grouped(const PoolJob* jobs, int njobs, long long total, int cs, int dt,
                               cudaStream_t st) {
    return launch_pdl(pool_s1_grouped_kernel, dim3(grid_for((size_t)total, 256)), dim3(256), 0, st, jobs, njobs, total,
                      cs, dt);
}

cudaError_t maxpool_s1_same(const void* x, void* y, int n, int H, int W, int cs, int dt,
                            cudaStream_t st) {
    const int V = 16 / (int)dt_size(dt);
    const size_t total = (size_t)n * H * W * (cs / V);
    return launch_pdl(pool_s1_kernel, dim3(grid_for(total, 256)), dim3(256), 0, st,
                      reinterpret_cast<const uint8_t*>(x), reinterpret_cast<uint8_t*>(y), n, H, W, cs, dt);
}

// ---------------------------------------------------------------- fold
// One block per output channel: s_o, b'_o and max|W'_o| in FP64.
__global__ void fold_scale_kernel(FoldArgs a) {
    const int o = blockIdx.x;
    const bool bn = a.gamma != nullptr;
    const double s = bn ? (double)a.gamma[o] / sqrt((double)a.var[o] + kBnEps) : 1.0;
    const int fan = a.cin * a.k * a.k;
    const float* wr = a.raw_w + (size_t)o * fan;
    double m = 0.0;
    for (int i = threadIdx.x; i < fan; i += blockDim.x) m = fmax(m, fabs((double)wr[i] * s));
    __shared__ double red[32];
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, red[i]);
        m = fmax(m, red[0]);
        a.tmp_s[o] = s;
        a.tmp_amax[o] = m;
        const double b = bn ? (double)a.beta[o] - (double)a.mean[o] * s : (double)a.bias[o];
        a.out_bias[o] = (float)b;
        if (a.out_wscale) a.out_wscale[o] = (float)(fmax(m, 1e-30) / (double)kFp8Max);
    }
}

// One thread per element of the [w_rows][k*k][Cp] output: reorder + cast.
__global__ void fold_write_kernel(FoldArgs a) {
    const int KK = a.im2col ? 1 : a.k * a.k;
    const size_t total = (size_t)a.w_rows * KK * a.Cp;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        int c = (int)(i % a.Cp);
        int tap = (int)((i / a.Cp) % KK);
        const int o = (int)(i / ((size_t)a.Cp * KK));
        bool real = o < a.cout && c < a.cin;
        if (a.im2col) {   // one row of Cp = taps x cin (+ zero padding)
            real = o < a.cout && c < a.cin * a.k * a.k;
            tap = c / a.cin;
            c = c % a.cin;
        }
        double v = 0.0;
        if (real) {
            const int kh = tap / a.k, kw = tap % a.k;
            v = (double)a.raw_w[(((size_t)o * a.cin + c) * a.k + kh) * a.k + kw] * a.tmp_s[o];
        }
        if (a.dt == DT_F32) {
            reinterpret_cast<float*>(a.out_w)[i] = (float)v;
        } else if (a.dt == DT_BF16) {
            reinterpret_cast<__nv_bfloat16*>(a.out_w)[i] = __double2bfloat16(v);
        } else {
            const double sw = (o < a.cout) ? fmax(a.tmp_amax[o], 1e-30) / (double)kFp8Max : 1.0;
            reinterpret_cast<uint8_t*>(a.out_w)[i] =
                (uint8_t)__nv_cvt_double_to_fp8(v / sw, __NV_SATFINITE, __NV_E4M3);
        }
        if (a.out_w32 && c < a.Cp32)
            a.out_w32[((size_t)o * KK + tap) * a.Cp32 + c] = (float)v;
    }
    // channels [Cp, Cp32) of the FP32 copy (when it is wider) stay zero:
    // the caller zero-fills it.
}

cudaError_t fold_layer(const FoldArgs& a, cudaStream_t st) {
    fold_scale_kernel<<<a.cout, 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t total = (size_t)a.w_rows * (a.im2col ? 1 : a.k * a.k) * a.Cp;
    fold_write_kernel<<<grid_for(total, 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

__global__ void alpha_kernel(const float* wscale, double act_scale, float* alpha, int cout) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o < cout) alpha[o] = (float)((double)wscale[o] * act_scale);
}

cudaError_t make_alpha(const float* wscale, double act_scale, float* alpha, int cout,
                       cudaStream_t st) {
    alpha_kernel<<<cdiv(cout, 256), 256, 0, st>>>(wscale, act_scale, alpha, cout);
    return cudaGetLastError();
}

__global__ void absmax_kernel(const float* __restrict__ x, size_t count, float* out) {
    float m = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(x[i]));
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int*>(out), __float_as_int(m));
}

cudaError_t absmax_f32(const float* x, size_t count, float* out, cudaStream_t st) {
    absmax_kernel<<<grid_for(count, 256), 256, 0, st>>>(x, count, out);
    return cudaGetLastError();
}

}  // namespace dn
