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

__global__ void splitk_reduce_kernel(SplitReduce r) {
    pdl_trigger();
    pdl_wait();   // the partial sums come from the conv launch before this one
    const bool pool = r.ep.pool == POOL_S2;
    const int Ho = pool ? r.H / 2 : r.H, Wo = pool ? r.W / 2 : r.W;
    const bool nchw = r.ep.out_layout == LAYOUT_NCHW;
    const int ncols = nchw ? r.ep.cout : r.ep.out_cs;   // columns written
    const int groups = (ncols + 3) / 4;
    const size_t npix = (size_t)r.n * Ho * Wo;
    const size_t total = npix * groups;
    const int PX = r.TW * r.TH;
    const size_t zstride = (size_t)r.m_rows * r.ncols_pad;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        // NCHW output: pixel fastest (coalesced stores); NHWC: channels fastest
        size_t pix;
        int g;
        if (nchw) {
            pix = i % npix;
            g = (int)(i / npix);
        } else {
            g = (int)(i % groups);
            pix = i / groups;
        }
        const int xo = (int)(pix % Wo);
        const int yo = (int)((pix / Wo) % Ho);
        const int img = (int)(pix / ((size_t)Wo * Ho));
        const int o = g * 4;
        float a4[4], b4[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool real = o + j < r.ep.cout;
            b4[j] = real ? r.ep.bias[o + j] : 0.f;
            a4[j] = (real && r.ep.alpha) ? r.ep.alpha[o + j] : 1.f;
        }
        float best[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
        const int np = pool ? 4 : 1;
        for (int p = 0; p < np; ++p) {
            const int yy = pool ? 2 * yo + (p >> 1) : yo;
            const int xx = pool ? 2 * xo + (p & 1) : xo;
            const int ty = yy / r.TH, tx = xx / r.TW;
            const size_t m = (((size_t)img * r.tiles_y + ty) * r.tiles_x + tx) * PX + (yy % r.TH) * r.TW + (xx % r.TW);
            const float* src = r.ws + m * r.ncols_pad + o;
            float4 s = *reinterpret_cast<const float4*>(src);
            for (int z = 1; z < r.ksplit; ++z) {
                const float4 t = *reinterpret_cast<const float4*>(src + z * zstride);
                s.x += t.x;
                s.y += t.y;
                s.z += t.z;
                s.w += t.w;
            }
            const float sv[4] = {s.x, s.y, s.z, s.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) best[j] = fmaxf(best[j], act_apply(fmaf(sv[j], a4[j], b4[j]), r.ep.act));
        }
        if (nchw) {
            float* yf = reinterpret_cast<float*>(r.y);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (o + j < r.ep.cout) yf[(((size_t)img * r.ep.cout + o + j) * Ho + yo) * Wo + xo] = best[j];
            continue;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (o + j >= r.ep.cout) best[j] = 0.f;
        const size_t off = pix * r.ep.out_cs + o;
        if (r.ep.out_dt == DT_F32) {
            *reinterpret_cast<float4*>(reinterpret_cast<float*>(r.y) + off) =
                make_float4(best[0], best[1], best[2], best[3]);
        } else if (r.ep.out_dt == DT_BF16) {
            __nv_bfloat162 lo = __floats2bfloat162_rn(best[0], best[1]);
            __nv_bfloat162 hi = __floats2bfloat162_rn(best[2], best[3]);
            uint2 pk;
            pk.x = *reinterpret_cast<uint32_t*>(&lo);
            pk.y = *reinterpret_cast<uint32_t*>(&hi);
            *reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(r.y) + off) = pk;
        } else {
            uint32_t pk = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) pk |= (uint32_t)f32_to_e4m3_sat(best[j] * r.ep.out_inv_scale) << (8 * j);
            *reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(r.y) + off) = pk;
        }
    }
}

cudaError_t splitk_reduce(const SplitReduce& r, cudaStream_t st) {
    const bool pool = r.ep.pool == POOL_S2;
    const size_t npix = (size_t)r.n * (pool ? r.H / 2 : r.H) * (pool ? r.W / 2 : r.W);
    const int ncols = r.ep.out_layout == LAYOUT_NCHW ? r.ep.cout : r.ep.out_cs;
    const size_t total = npix * ((ncols + 3) / 4);
    size_t blocks = (total + 255) / 256;
    if (blocks > 152u * 16u) blocks = 152u * 16u;
    return launch_pdl(splitk_reduce_kernel, dim3((unsigned)(blocks ? blocks : 1)), dim3(256), 0, st, r);
}

}  // namespace dn
