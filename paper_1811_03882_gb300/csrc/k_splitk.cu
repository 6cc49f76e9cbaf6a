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

cudaError_t splitk_reduce(const SplitReduce& r, cudaStream_t st) {
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
