// k_conv_simt.cu — FP32 implicit-GEMM convolution on the CUDA cores.
//
// y[n,i,j,o] = sum_{kh,kw,c} x[n, i+kh-p, j+kw-p, c] * W'[o, kh, kw, c]
// (stride 1, zero pad p = k/2), i.e. a GEMM with M = N*H*W output pixels,
// N = Cout and K = k*k*Cin whose A operand is gathered from the NHWC
// activation on the fly.  This is the FP32 path: true FP32 FFMA, no TF32,
// so its error against the FP64 oracle stays at FP32 rounding level.
//
// Tile: a TH x TW rectangle of output pixels of one frame times BN output
// channels; 256 threads.  Pixels are ordered by 2x2 quads inside the tile
// and every thread owns whole quads, so the fused 2x2/s2 max pool of the
// epilogue is a register-local max.  Layers without that pool may instead
// take PXF consecutive output pixels in (frame, row, column) order (flat
// tiles): no rectangle to round up to, so a 13 x 13 map computes 192
// pixels instead of the 256 of two 8 x 16 rectangles.
#include "common.cuh"
#include "kernels.h"

namespace dn {

template <int BN, int TH, int TW, int PXF>
struct SimtCfg {
    static constexpr int THREADS = 256;
    static constexpr int PX = PXF ? PXF : TH * TW;   // pixels per tile
    static constexpr int CG = BN / 4;           // channel groups (4 ch each)
    static constexpr int PG = THREADS / CG;     // pixel groups
    static constexpr int PPT = PX / PG;         // pixels per thread
    static constexpr int QX = TW / 2;           // quads per tile row
    static constexpr int BK = 8;                // channels per K step
    static constexpr int A_SLOTS = PX * BK / 4;              // float4 loads (A)
    static constexpr int A_VEC = (A_SLOTS + THREADS - 1) / THREADS;   // per thread
    static constexpr int B_VEC_TOTAL = BN * BK / 4;      // float4 loads (B)
    static_assert(PPT % 4 == 0 && PX == PG * PPT, "threads own four-pixel groups (2x2 quads)");
    static_assert(PXF ? true : A_SLOTS % THREADS == 0, "A tile split");
    static_assert(B_VEC_TOTAL <= THREADS, "B tile split");
};

// PXF > 0: flat tiles of PXF pixels (no 2x2/s2 pool); nfr frames.  Flat
// tiles are held to two CTAs an SM's registers.
template <int BN, int TH, int TW, int PXF>
__global__ void __launch_bounds__(256, PXF ? 2 : 1)
conv_simt_kernel(const float* __restrict__ x, const float* __restrict__ w,
                 void* __restrict__ y, int H, int W, int Cp, int k, int kw_rows,
                 int tiles_x, int tiles_y, Epilogue ep, int ksplit, float* __restrict__ ws,
                 int ws_cols, int nfr) {
    using C = SimtCfg<BN, TH, TW, PXF>;
    constexpr bool FLAT = PXF > 0;
    __shared__ __align__(16) float As[2][C::BK][C::PX];
    __shared__ __align__(16) float Bs[2][C::BK][BN];

    const int tid = threadIdx.x;
    int t = blockIdx.x;
    const int tx = FLAT ? 0 : t % tiles_x;
    if (!FLAT) t /= tiles_x;
    const int ty = FLAT ? 0 : t % tiles_y;
    const int n = FLAT ? 0 : t / tiles_y;
    const int y0 = ty * TH, x0 = tx * TW;
    // flat tiles: first pixel of the tile and pixels in the layer
    const int m0 = blockIdx.x * C::PX, mtot = nfr * H * W;
    // flat tiles: each A load slot's pixel, decoded once (frame, row, column;
    // frame -1 past the layer's last pixel)
    int sn[C::A_VEC], sy[C::A_VEC], sx[C::A_VEC];
    if (FLAT) {
#pragma unroll
        for (int v = 0; v < C::A_VEC; ++v) {
            const int m = m0 + ((tid + v * C::THREADS) >> 1);
            const int row = m / W;
            sx[v] = m - row * W;
            sn[v] = row / H;
            sy[v] = row - sn[v] * H;
            if (m >= mtot || tid + v * C::THREADS >= C::A_SLOTS) sn[v] = -1;
        }
    }
    const int n0 = blockIdx.y * BN;
    const int pad = k / 2;
    const int KK = k * k;
    const int csteps = (Cp + C::BK - 1) / C::BK;
    const int nall = KK * csteps;
    const int z = blockIdx.z;
    const int s_begin = (int)((long)nall * z / ksplit), s_end = (int)((long)nall * (z + 1) / ksplit);
    const int nsteps = s_end - s_begin;
    const size_t wrow = (size_t)KK * Cp;

    float4 ra[C::A_VEC];
    float4 rb;

    auto load = [&](int lstep) {
        const int step = s_begin + lstep;
        const int tap = step / csteps;
        const int c0 = (step % csteps) * C::BK;
        const int kh = tap / k, kwi = tap % k;
#pragma unroll
        for (int v = 0; v < C::A_VEC; ++v) {
            const int f = tid + v * C::THREADS;
            const int pos = f >> 1, half = f & 1;
            int iy, ix, nn;
            if (FLAT) {
                nn = sn[v];
                iy = sy[v] + kh - pad;
                ix = sx[v] + kwi - pad;
            } else {
                const int q = pos >> 2, dy = (pos >> 1) & 1, dx = pos & 1;
                const int py = 2 * (q / C::QX) + dy, px = 2 * (q % C::QX) + dx;
                nn = n;
                iy = y0 + py + kh - pad;
                ix = x0 + px + kwi - pad;
            }
            const int c = c0 + half * 4;
            float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
            if (nn >= 0 && iy >= 0 && iy < H && ix >= 0 && ix < W && c < Cp)
                val = *reinterpret_cast<const float4*>(x + (((size_t)nn * H + iy) * W + ix) * Cp + c);
            ra[v] = val;
        }
        if (tid < C::B_VEC_TOTAL) {
            const int o = tid >> 1, half = tid & 1;
            const int c = c0 + half * 4;
            float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
            if (c < Cp && n0 + o < kw_rows)
                val = *reinterpret_cast<const float4*>(w + (size_t)(n0 + o) * wrow + (size_t)tap * Cp + c);
            rb = val;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int v = 0; v < C::A_VEC; ++v) {
            const int f = tid + v * C::THREADS;
            if (FLAT && f >= C::A_SLOTS) continue;
            const int pos = f >> 1, kb = (f & 1) * 4;
            As[buf][kb + 0][pos] = ra[v].x;
            As[buf][kb + 1][pos] = ra[v].y;
            As[buf][kb + 2][pos] = ra[v].z;
            As[buf][kb + 3][pos] = ra[v].w;
        }
        if (tid < C::B_VEC_TOTAL) {
            const int o = tid >> 1, kb = (tid & 1) * 4;
            Bs[buf][kb + 0][o] = rb.x;
            Bs[buf][kb + 1][o] = rb.y;
            Bs[buf][kb + 2][o] = rb.z;
            Bs[buf][kb + 3][o] = rb.w;
        }
    };

    float acc[C::PPT][4];
#pragma unroll
    for (int i = 0; i < C::PPT; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    const int cg = tid % C::CG, pg = tid / C::CG;
    if (nsteps > 0) {
        load(0);
        store(0);
    }
    __syncthreads();
    for (int s = 0; s < nsteps; ++s) {
        const int buf = s & 1;
        if (s + 1 < nsteps) load(s + 1);
#pragma unroll
        for (int kk = 0; kk < C::BK; ++kk) {
            float a[C::PPT];
#pragma unroll
            for (int i = 0; i < C::PPT; i += 4) {
                float4 v = *reinterpret_cast<const float4*>(&As[buf][kk][pg * C::PPT + i]);
                a[i] = v.x; a[i + 1] = v.y; a[i + 2] = v.z; a[i + 3] = v.w;
            }
            float4 b = *reinterpret_cast<const float4*>(&Bs[buf][kk][cg * 4]);
#pragma unroll
            for (int i = 0; i < C::PPT; ++i) {
                acc[i][0] = fmaf(a[i], b.x, acc[i][0]);
                acc[i][1] = fmaf(a[i], b.y, acc[i][1]);
                acc[i][2] = fmaf(a[i], b.z, acc[i][2]);
                acc[i][3] = fmaf(a[i], b.w, acc[i][3]);
            }
        }
        if (s + 1 < nsteps) {
            store(buf ^ 1);
            __syncthreads();
        }
    }

    const int obase = n0 + cg * 4;
    if (ksplit > 1) {
        // raw partial sums; the reduction kernel applies the epilogue
        const size_t mbase = (size_t)blockIdx.x * C::PX;
        float* wz = ws + (size_t)z * gridDim.x * C::PX * ws_cols;
#pragma unroll
        for (int i = 0; i < C::PPT; ++i) {
            const int pos = pg * C::PPT + i;
            const int q = pos >> 2;
            const int py = 2 * (q / C::QX) + ((pos >> 1) & 1), px = 2 * (q % C::QX) + (pos & 1);
            // flat tiles: row = pixel index; rows past the layer are never read
            *reinterpret_cast<float4*>(wz + (mbase + (FLAT ? pos : py * TW + px)) * ws_cols + obase) =
                make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        }
        return;
    }

    // ---- epilogue: alpha/bias, activation, optional 2x2/s2 max, store ----
    float bia[4], alp[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int o = obase + j;
        bia[j] = (o < ep.cout) ? ep.bias[o] : 0.f;
        alp[j] = (o < ep.cout && ep.alpha) ? ep.alpha[o] : 1.f;
    }
    const bool pool = ep.pool == POOL_S2;
    const int Ho = pool ? H / 2 : H, Wo = pool ? W / 2 : W;
    if constexpr (FLAT) {
        // no pool: each of the thread's pixels on its own
#pragma unroll
        for (int i = 0; i < C::PPT; ++i) {
            const int m = m0 + pg * C::PPT + i;
            if (m >= mtot) continue;
            float o4[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) o4[j] = act_apply(fmaf(acc[i][j], alp[j], bia[j]), ep.act);
            if (ep.out_layout == LAYOUT_NCHW) {
                const int row = m / W, xo = m - row * W, img = row / H, yo = row - img * H;
                float* yf = reinterpret_cast<float*>(y);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int o = obase + j;
                    if (o < ep.cout) yf[(((size_t)img * ep.cout + o) * H + yo) * W + xo] = o4[j];
                }
                continue;
            }
            if (obase >= ep.out_cs) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (obase + j >= ep.cout) o4[j] = 0.f;
            const size_t off = (size_t)m * ep.out_cs + obase;   // NHWC: pixel m's row
            if (ep.out_dt == DT_F32) {
                *reinterpret_cast<float4*>(reinterpret_cast<float*>(y) + off) =
                    make_float4(o4[0], o4[1], o4[2], o4[3]);
            } else if (ep.out_dt == DT_BF16) {
                __nv_bfloat162 lo = __floats2bfloat162_rn(o4[0], o4[1]);
                __nv_bfloat162 hi = __floats2bfloat162_rn(o4[2], o4[3]);
                uint2 pk;
                pk.x = *reinterpret_cast<uint32_t*>(&lo);
                pk.y = *reinterpret_cast<uint32_t*>(&hi);
                *reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(y) + off) = pk;
            } else {
                uint32_t pk = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    pk |= (uint32_t)f32_to_e4m3_sat(o4[j] * ep.out_inv_scale) << (8 * j);
                *reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(y) + off) = pk;
            }
        }
        return;
    }
#pragma unroll
    for (int qi = 0; qi < C::PPT / 4; ++qi) {
        const int q = (pg * C::PPT) / 4 + qi;
        const int qy = q / C::QX, qx = q % C::QX;
        float v[4][4];  // [pixel in quad][channel]
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                v[p][j] = act_apply(fmaf(acc[qi * 4 + p][j], alp[j], bia[j]), ep.act);
        const int npix = pool ? 1 : 4;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            if (p >= npix) break;
            float o4[4];
            int yo, xo;
            if (pool) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    o4[j] = fmaxf(fmaxf(v[0][j], v[1][j]), fmaxf(v[2][j], v[3][j]));
                yo = (y0 >> 1) + qy;
                xo = (x0 >> 1) + qx;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) o4[j] = v[p][j];
                yo = y0 + 2 * qy + (p >> 1);
                xo = x0 + 2 * qx + (p & 1);
            }
            if (yo >= Ho || xo >= Wo) continue;
            if (ep.out_layout == LAYOUT_NCHW) {
                float* yf = reinterpret_cast<float*>(y);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int o = obase + j;
                    if (o < ep.cout) yf[(((size_t)n * ep.cout + o) * Ho + yo) * Wo + xo] = o4[j];
                }
                continue;
            }
            if (obase >= ep.out_cs) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (obase + j >= ep.cout) o4[j] = 0.f;
            const size_t off = (((size_t)n * Ho + yo) * Wo + xo) * ep.out_cs + obase;
            if (ep.out_dt == DT_F32) {
                *reinterpret_cast<float4*>(reinterpret_cast<float*>(y) + off) =
                    make_float4(o4[0], o4[1], o4[2], o4[3]);
            } else if (ep.out_dt == DT_BF16) {
                __nv_bfloat162 lo = __floats2bfloat162_rn(o4[0], o4[1]);
                __nv_bfloat162 hi = __floats2bfloat162_rn(o4[2], o4[3]);
                uint2 pk;
                pk.x = *reinterpret_cast<uint32_t*>(&lo);
                pk.y = *reinterpret_cast<uint32_t*>(&hi);
                *reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(y) + off) = pk;
            } else {
                uint32_t pk = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    pk |= (uint32_t)f32_to_e4m3_sat(o4[j] * ep.out_inv_scale) << (8 * j);
                *reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(y) + off) = pk;
            }
        }
    }
}

template <int BN, int TH, int TW, int PXF>
static cudaError_t launch_simt(const ConvLaunch& L, int ncols, int m_tiles, cudaStream_t st) {
    const int tiles_x = cdiv(L.W, TW), tiles_y = cdiv(L.H, TH);
    const int ks = L.ksplit > 1 ? L.ksplit : 1;
    const int n_tiles = cdiv(ncols, BN);
    dim3 grid((unsigned)m_tiles, (unsigned)n_tiles, (unsigned)ks);
    conv_simt_kernel<BN, TH, TW, PXF><<<grid, 256, 0, st>>>(
        reinterpret_cast<const float*>(L.x), reinterpret_cast<const float*>(L.w), L.y, L.H, L.W,
        L.Cp, L.k, L.w_rows, tiles_x, tiles_y, L.ep, ks, L.ws, n_tiles * BN, L.n);
    return cudaGetLastError();
}

void simt_tile(int ncols, int* bn, int* th, int* tw) {
    if (ncols <= 16) { *bn = 16; *th = 16; *tw = 16; }
    else if (ncols <= 32) { *bn = 32; *th = 8; *tw = 16; }
    else { *bn = 64; *th = 8; *tw = 16; }
}

constexpr int kFlatPx = 192;   // flat tile pixels (64-column tiles: 12 pixels a thread)

SimtGeom simt_geom(int ncols, bool pool, int n, int H, int W, bool quads) {
    SimtGeom g;
    simt_tile(ncols, &g.bn, &g.th, &g.tw);
    const long quad_px = (long)n * cdiv(H, g.th) * g.th * cdiv(W, g.tw) * g.tw;
    const long flat_tiles = cdiv((long)n * H * W, (long)kFlatPx);
    // flat tiles where they compute fewer pixels (64-column tiles, no pool)
    g.flat = (!pool && !quads && g.bn == 64 && flat_tiles * kFlatPx < quad_px) ? 1 : 0;
    g.px = g.flat ? kFlatPx : g.th * g.tw;
    g.m_tiles = g.flat ? (int)flat_tiles : n * cdiv(H, g.th) * cdiv(W, g.tw);
    // split-K reduction geometry: flat rows are pixel indices, i.e. one
    // H x W "tile" per frame
    g.red_tw = g.flat ? W : g.tw;
    g.red_th = g.flat ? H : g.th;
    g.red_tx = g.flat ? 1 : cdiv(W, g.tw);
    g.red_ty = g.flat ? 1 : cdiv(H, g.th);
    return g;
}

cudaError_t conv_simt(const ConvLaunch& L, cudaStream_t st) {
    const int ncols = L.ep.out_layout == LAYOUT_NCHW ? L.ep.cout
                                                      : (L.ep.out_cs > L.ep.cout ? L.ep.out_cs : L.ep.cout);
    const SimtGeom g = simt_geom(ncols, L.ep.pool == POOL_S2, L.n, L.H, L.W, L.quads != 0);
    if (g.bn == 16) return launch_simt<16, 16, 16, 0>(L, ncols, g.m_tiles, st);
    if (g.bn == 32) return launch_simt<32, 8, 16, 0>(L, ncols, g.m_tiles, st);
    if (g.flat) return launch_simt<64, 8, 16, kFlatPx>(L, ncols, g.m_tiles, st);
    return launch_simt<64, 8, 16, 0>(L, ncols, g.m_tiles, st);
}

}  // namespace dn
