// k_splitk.cu — split-K reduction with the fused conv epilogue.
//
// Layers with few output tiles (small maps at batch 1, e.g. 13 x 13 x 1024)
// split K = k*k*Cin over several CTAs; each writes raw FP32 partial sums
// to a workspace and this kernel adds them in a fixed order (z = 0, 1, ...),
// so the result is deterministic, then applies alpha/bias, leaky, the
// optional 2x2/s2 max and the store of the conv epilogue.
#include "common.cuh"
#include "kernels.h"

namespace dn {

// One thread per (output pixel, group of V = 4 or 8 channels); all index
// arithmetic in 32 bits (the host checks the sizes).
template <int V>
__global__ void splitk_reduce_kernel(SplitReduce r) {
    pdl_trigger();
    pdl_wait();   // the partial sums come from the conv launch before this one
    const bool pool = r.ep.pool == POOL_S2;
    const int Ho = pool ? r.H / 2 : r.H, Wo = pool ? r.W / 2 : r.W;
    const bool nchw = r.ep.out_layout == LAYOUT_NCHW;
    const int ncols = nchw ? r.ep.cout : r.ep.out_cs;   // columns written
    const int groups = (ncols + V - 1) / V;
    const int npix = r.n * Ho * Wo;
    const int total = npix * groups;
    const int PX = r.TW * r.TH;
    const size_t zstride = (size_t)r.m_rows * r.ncols_pad;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        // NCHW output: pixel fastest (coalesced stores); NHWC: channels fastest
        int pix, g;
        if (nchw) {
            g = i / npix;
            pix = i - g * npix;
        } else {
            pix = i / groups;
            g = i - pix * groups;
        }
        const int row = pix / Wo;
        const int xo = pix - row * Wo;
        const int img = row / Ho;
        const int yo = row - img * Ho;
        const int o = g * V;
        float a[V], b[V], best[V];
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const bool real = o + j < r.ep.cout;
            b[j] = real ? r.ep.bias[o + j] : 0.f;
            a[j] = (real && r.ep.alpha) ? r.ep.alpha[o + j] : 1.f;
            best[j] = -INFINITY;
        }
        const int np = pool ? 4 : 1;
        for (int p = 0; p < np; ++p) {
            const int yy = pool ? 2 * yo + (p >> 1) : yo;
            const int xx = pool ? 2 * xo + (p & 1) : xo;
            const int ty = yy / r.TH, tx = xx / r.TW;
            const int m = ((img * r.tiles_y + ty) * r.tiles_x + tx) * PX + (yy - ty * r.TH) * r.TW + (xx - tx * r.TW);
            const float* src = r.ws + (size_t)m * r.ncols_pad + o;
            float sv[V];
#pragma unroll
            for (int q = 0; q < V / 4; ++q) {
                float4 acc = *reinterpret_cast<const float4*>(src + 4 * q);
                for (int z = 1; z < r.ksplit; ++z) {   // fixed order: deterministic
                    const float4 t = *reinterpret_cast<const float4*>(src + z * zstride + 4 * q);
                    acc.x += t.x;
                    acc.y += t.y;
                    acc.z += t.z;
                    acc.w += t.w;
                }
                sv[4 * q] = acc.x;
                sv[4 * q + 1] = acc.y;
                sv[4 * q + 2] = acc.z;
                sv[4 * q + 3] = acc.w;
            }
#pragma unroll
            for (int j = 0; j < V; ++j) best[j] = fmaxf(best[j], act_apply(fmaf(sv[j], a[j], b[j]), r.ep.act));
        }
        if (nchw) {
            float* yf = reinterpret_cast<float*>(r.y);
#pragma unroll
            for (int j = 0; j < V; ++j)
                if (o + j < r.ep.cout) yf[(((size_t)img * r.ep.cout + o + j) * Ho + yo) * Wo + xo] = best[j];
            continue;
        }
#pragma unroll
        for (int j = 0; j < V; ++j)
            if (o + j >= r.ep.cout) best[j] = 0.f;
        const size_t off = (size_t)pix * r.ep.out_cs + o;
#pragma unroll
        for (int q = 0; q < V / 4; ++q) {
            const float* bq = best + 4 * q;
            if (r.ep.out_dt == DT_F32) {
                *reinterpret_cast<float4*>(reinterpret_cast<float*>(r.y) + off + 4 * q) =
                    make_float4(bq[0], bq[1], bq[2], bq[3]);
            } else if (r.ep.out_dt == DT_BF16) {
                __nv_bfloat162 lo = __floats2bfloat162_rn(bq[0], bq[1]);
                __nv_bfloat162 hi = __floats2bfloat162_rn(bq[2], bq[3]);
                uint2 pk;
                pk.x = *reinterpret_cast<uint32_t*>(&lo);
                pk.y = *reinterpret_cast<uint32_t*>(&hi);
                *reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(r.y) + off + 4 * q) = pk;
            } else {
                uint32_t pk = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j) pk |= (uint32_t)f32_to_e4m3_sat(bq[j] * r.ep.out_inv_scale) << (8 * j);
                *reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(r.y) + off + 4 * q) = pk;
            }
        }
    }
}

// Tile-major workspace (tensor-core launches): one block per (128-row M
// tile, 64 columns).  The block first sums the ksplit partials of its
// 128 x 64 slab in the fixed order z = 0, 1, ... with coalesced float4 loads
// (a warp reads 512 contiguous bytes) into shared memory, then applies the
// epilogue from there with threads laid out along the output's contiguous
// dimension: four channels of one pixel (NHWC) or one pixel of one channel
// (NCHW).  Same arithmetic, in the same order, as splitk_reduce_kernel.
constexpr int kRedCols = 64;
__global__ void __launch_bounds__(256) splitk_tile_reduce_kernel(SplitReduce r) {
    pdl_trigger();
    __shared__ float s[128][kRedCols + 1];   // +1: rows and columns both conflict-free
    __shared__ float s_b[kRedCols], s_a[kRedCols];   // bias / alpha of the block's columns
    const int tile = blockIdx.x, col0 = blockIdx.y * kRedCols;
    const int ncg = r.ncols_pad >> 2;
    const size_t zstride = (size_t)r.m_rows * r.ncols_pad;
    if (threadIdx.x < kRedCols) {
        // bias and alpha are padded with zeros to the weight rows, which cover
        // the workspace's columns
        const int c = col0 + threadIdx.x;
        const bool in = c < r.ncols_pad;
        s_b[threadIdx.x] = in ? r.ep.bias[c] : 0.f;
        s_a[threadIdx.x] = in && r.ep.alpha ? r.ep.alpha[c] : 1.f;
    }
    pdl_wait();   // (a no-op under an ordinary launch)
    {
        // thread -> row rr of the tile and column groups q0, q0 + 2, ..., all
        // eight loads of a plane issued before any is used (memory-level
        // parallelism: one block per SM or two hold the whole launch)
        constexpr int NQ = kRedCols / 4 / 2;
        const int rr = threadIdx.x & 127, q0 = threadIdx.x >> 7;
        const float* base = r.ws + ((size_t)tile * ncg + (col0 >> 2)) * 512 + rr * 4;
        float4 acc[NQ];
#pragma unroll
        for (int u = 0; u < NQ; ++u) {
            const int q = q0 + 2 * u;
            acc[u] = (col0 >> 2) + q < ncg ? *reinterpret_cast<const float4*>(base + q * 512)
                                           : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int z = 1; z < r.ksplit; ++z) {   // fixed order: deterministic
            float4 t[NQ];
#pragma unroll
            for (int u = 0; u < NQ; ++u) {
                const int q = q0 + 2 * u;
                t[u] = (col0 >> 2) + q < ncg ? *reinterpret_cast<const float4*>(base + z * zstride + q * 512)
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < NQ; ++u) {
                acc[u].x += t[u].x;
                acc[u].y += t[u].y;
                acc[u].z += t[u].z;
                acc[u].w += t[u].w;
            }
        }
#pragma unroll
        for (int u = 0; u < NQ; ++u) {
            const int q = q0 + 2 * u;
            s[rr][4 * q] = acc[u].x;
            s[rr][4 * q + 1] = acc[u].y;
            s[rr][4 * q + 2] = acc[u].z;
            s[rr][4 * q + 3] = acc[u].w;
        }
    }
    __syncthreads();
    const bool pool = r.ep.pool == POOL_S2;
    const bool nchw = r.ep.out_layout == LAYOUT_NCHW;
    const int ncols = nchw ? r.ep.cout : r.ep.out_cs;   // columns written
    const int Ho = pool ? r.H / 2 : r.H, Wo = pool ? r.W / 2 : r.W;
    const int tpi = r.tiles_x * r.tiles_y;
    const int img = tile / tpi, txy = tile - img * tpi;
    const int ty = txy / r.tiles_x, tx = txy - ty * r.tiles_x;
    // output pixels of the tile: TH x TW, or (TH / 2) x (TW / 2) after the
    // pool; TW and TH = 128 / TW are powers of two
    const int twl = 31 - __clz(r.TW), owl = pool ? twl - 1 : twl;
    const int OW = 1 << owl, OH = pool ? r.TH / 2 : r.TH;
    const int npx = OW * OH;
    const int y0 = ty * OH, x0 = tx * OW;
    // epilogue of block column cl at output pixel (oy, ox), from the sums
    auto value = [&](int oy, int ox, int cl) {
        const float b = s_b[cl], a = s_a[cl];
        if (!pool) {
            return act_apply(fmaf(s[(oy << twl) + ox][cl], a, b), r.ep.act);
        }
        float best = -INFINITY;
#pragma unroll
        for (int p = 0; p < 4; ++p) {   // (0,0), (0,1), (1,0), (1,1): the unfused order
            const float v = fmaf(s[((2 * oy + (p >> 1)) << twl) + 2 * ox + (p & 1)][cl], a, b);
            best = fmaxf(best, act_apply(v, r.ep.act));
        }
        return best;
    };
    if (nchw) {
        // thread -> (column, pixel), pixels fastest: runs along x in the output
        const int ncl = min(kRedCols, ncols - col0);
        float* yf = reinterpret_cast<float*>(r.y);
        for (int i = threadIdx.x; i < ncl * 128; i += blockDim.x) {
            const int cl = i >> 7, opx = i & 127;
            if (opx >= npx) continue;
            const int oy = opx >> owl, ox = opx & (OW - 1);
            const int yo = y0 + oy, xo = x0 + ox;
            if (yo >= Ho || xo >= Wo) continue;
            yf[(((size_t)img * r.ep.cout + col0 + cl) * Ho + yo) * Wo + xo] = value(oy, ox, cl);
        }
        return;
    }
    // NHWC: thread -> (pixel, group of four columns), sixteen groups per pixel
    const int g = threadIdx.x & 15;
    const int o = col0 + 4 * g;
    if (o >= min(col0 + kRedCols, ncols)) return;
    for (int opx = threadIdx.x >> 4; opx < npx; opx += blockDim.x >> 4) {
        const int oy = opx >> owl, ox = opx & (OW - 1);
        const int yo = y0 + oy, xo = x0 + ox;
        if (yo >= Ho || xo >= Wo) continue;
        float bq[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) bq[j] = o + j < r.ep.cout ? value(oy, ox, 4 * g + j) : 0.f;
        const size_t off = (((size_t)img * Ho + yo) * Wo + xo) * r.ep.out_cs + o;
        if (r.ep.out_dt == DT_F32) {
            *reinterpret_cast<float4*>(reinterpret_cast<float*>(r.y) + off) = make_float4(bq[0], bq[1], bq[2], bq[3]);
        } else if (r.ep.out_dt == DT_BF16) {
            __nv_bfloat162 lo = __floats2bfloat162_rn(bq[0], bq[1]);
            __nv_bfloat162 hi = __floats2bfloat162_rn(bq[2], bq[3]);
            uint2 pk;
            pk.x = *reinterpret_cast<uint32_t*>(&lo);
            pk.y = *reinterpret_cast<uint32_t*>(&hi);
            *reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(r.y) + off) = pk;
        } else {
            uint32_t pk = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) pk |= (uint32_t)f32_to_e4m3_sat(bq[j] * r.ep.out_inv_scale) << (8 * j);
            *reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(r.y) + off) = pk;
        }
    }
}

cudaError_t splitk_reduce(const SplitReduce& r, cudaStream_t st) {
    if (r.tile_major) {
        const bool nchw = r.ep.out_layout == LAYOUT_NCHW;
        const int ncols = nchw ? r.ep.cout : r.ep.out_cs;
        // whole 128-row tiles, whole column groups (NHWC stores four columns
        // at a time), pool windows inside a tile, every column written
        // present in the workspace
        const bool pow2 = r.TW > 0 && (r.TW & (r.TW - 1)) == 0;   // TW x TH = 128: both powers of two
        if (!pow2 || r.TW * r.TH != 128 || r.m_rows % 128 != 0 || r.ncols_pad % 4 != 0 || (!nchw && ncols % 4 != 0) ||
            ncols > r.ncols_pad || (r.ep.pool == POOL_S2 && ((r.TW | r.TH) & 1)) ||
            r.m_rows / 128 != r.n * r.tiles_x * r.tiles_y ||
            (size_t)r.m_rows * r.ncols_pad * r.ksplit >= ((size_t)1 << 40))
            return cudaErrorInvalidValue;
        const dim3 grid((unsigned)(r.m_rows / 128), (unsigned)((ncols + kRedCols - 1) / kRedCols));
        static bool carve = false;
        if (!carve) {
            // the conv launches around this one run with the largest shared
            // memory carveout; keeping it avoids an SM reconfiguration (which
            // waits for the SM to drain) at every switch between the two
            const cudaError_t e = cudaFuncSetAttribute(splitk_tile_reduce_kernel,
                                                       cudaFuncAttributePreferredSharedMemoryCarveout,
                                                       (int)cudaSharedmemCarveoutMaxShared);
            if (e != cudaSuccess) return e;
            carve = true;
        }
        // an ordinary launch: under programmatic launch the blocks become
        // resident early on the few SMs the conv grid leaves free, several per
        // SM, and all start there when the conv ends (measured slower)
        splitk_tile_reduce_kernel<<<grid, 256, 0, st>>>(r);
        return cudaGetLastError();
    }
    const bool pool = r.ep.pool == POOL_S2;
    const size_t npix = (size_t)r.n * (pool ? r.H / 2 : r.H) * (pool ? r.W / 2 : r.W);
    const int ncols = r.ep.out_layout == LAYOUT_NCHW ? r.ep.cout : r.ep.out_cs;
    // eight channels a thread when every group of eight is whole (NHWC
    // channel strides are multiples of 16 bytes; NCHW counts real channels)
    const bool v8 = ncols % 8 == 0;
    const size_t total = npix * (size_t)((ncols + (v8 ? 7 : 3)) / (v8 ? 8 : 4));
    if (total >= (size_t)INT32_MAX || (size_t)r.m_rows * r.ncols_pad * r.ksplit >= ((size_t)1 << 40))
        return cudaErrorInvalidValue;
    size_t blocks = (total + 255) / 256;
    if (blocks > 152u * 16u) blocks = 152u * 16u;
    const dim3 grid((unsigned)(blocks ? blocks : 1));
    return v8 ? launch_pdl(splitk_reduce_kernel<8>, grid, dim3(256), 0, st, r)
              : launch_pdl(splitk_reduce_kernel<4>, grid, dim3(256), 0, st, r);
}

}  // namespace dn
