// net.cu — C ABI, layer-graph executor and device buffer planner.
//
// Data-transfer rule (paper, Sec. 3.2) taken to its limit: weights are
// uploaded and folded once, a forward pass copies the frames to the device
// once and the result back once, and every activation in between lives in
// a ping-pong pair of device buffers planned at net_create for the largest
// batch and frame side.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <memory>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/net.h"
#include "common.cuh"
#include "kernels.h"
#include "net_internal.h"

using namespace dn;

static thread_local std::string g_err;

net_status dn::fail(net_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define CK(call)                                                                            \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(e_ == cudaErrorMemoryAllocation ? NET_E_OOM : NET_E_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                 \
    } while (0)

// ------------------------------------------------------------- planning
static int layer_engine(int prec) { return prec == NET_FP32 ? ENG_SIMT : ENG_TC; }

// A layer reading fewer than 16 channels (the raw 3-channel frame) keeps its
// operands in BF16 even in an FP8 network: its K chunk is padded to 32 bytes
// either way, and E4M3 would round the frame itself to 4 significant bits.
static int effective_prec(int prec, int cin) { return (prec == NET_FP8 && cin < 16) ? NET_BF16 : prec; }

static int prec_dt(int prec) { return prec == NET_FP32 ? DT_F32 : prec == NET_BF16 ? DT_BF16 : DT_FP8; }

// Spatial size of the input of every layer (and the final output) for h x w.
void dn::layer_dims(const net* n, int h, int w, std::vector<int>& H, std::vector<int>& W) {
    H.assign(n->L.size() + 1, 0);
    W.assign(n->L.size() + 1, 0);
    H[0] = h;
    W[0] = w;
    for (size_t l = 0; l < n->L.size(); ++l) {
        const bool s2 = n->L[l].d.pool == NET_POOL_2X2S2;
        H[l + 1] = s2 ? H[l] / 2 : H[l];
        W[l + 1] = s2 ? W[l] / 2 : W[l];
    }
}

net_status dn::check_shape(const net* n, int batch, int h, int w) {
    if (batch < 1 || batch > n->max_batch)
        return fail(NET_E_SHAPE, "batch %d outside [1, %d]", batch, n->max_batch);
    if (h < 1 || w < 1 || h > n->max_side || w > n->max_side)
        return fail(NET_E_SHAPE, "frame %dx%d outside [1, %d]", h, w, n->max_side);
    int hh = h, ww = w;
    for (size_t l = 0; l < n->L.size(); ++l) {
        if (n->L[l].d.pool == NET_POOL_2X2S2) {
            if ((hh & 1) || (ww & 1))
                return fail(NET_E_SHAPE, "layer %zu: 2x2/s2 pool needs even size, got %dx%d", l, hh, ww);
            hh /= 2;
            ww /= 2;
        }
    }
    return NET_OK;
}

size_t dn::act_bytes_for(const net* n, int batch, int h, int w) {
    std::vector<int> H, W;
    layer_dims(n, h, w, H, W);
    size_t mx = 0;
    for (size_t l = 0; l < n->L.size(); ++l) {
        const Layer& L = n->L[l];
        // input of layer l
        mx = std::max(mx, (size_t)batch * H[l] * W[l] * L.in_cs * dt_size(L.in_dt));
        // un-pooled output kept for the standalone stride-1 pool
        if (L.d.pool == NET_POOL_2X2S1_SAME) {
            const bool last = l + 1 == n->L.size();
            const int cs = last ? rup(L.d.cout, 4) : n->L[l + 1].in_cs;
            const int dt = last ? DT_F32 : n->L[l + 1].in_dt;
            mx = std::max(mx, (size_t)batch * H[l + 1] * W[l + 1] * cs * dt_size(dt));
        }
    }
    // the last layer's NHWC float32 output (trace / standalone pool paths)
    const size_t nl = n->L.size();
    mx = std::max(mx, (size_t)batch * H[nl] * W[nl] * rup(n->L.back().d.cout, 4) * 4);
    return std::max((size_t)256, ((mx + 255) / 256) * 256);
}

extern "C" net_status net_create(const net_desc* d, net_t** out) {
    if (!d || !out) return fail(NET_E_INVAL, "NULL argument");
    *out = nullptr;
    if (d->n_layers < 1 || !d->layers) return fail(NET_E_INVAL, "no layers");
    if (d->in_c < 1 || d->in_c > 4096) return fail(NET_E_INVAL, "in_c %d", d->in_c);
    if (d->max_batch < 1 || d->max_side < 1 || d->max_side > 8192)
        return fail(NET_E_INVAL, "max_batch %d / max_side %d", d->max_batch, d->max_side);
    if (d->prec < NET_FP32 || d->prec > NET_FP8) return fail(NET_E_INVAL, "precision %d", d->prec);
    for (int l = 0; l < d->n_layers; ++l) {
        const net_layer& s = d->layers[l];
        const int p = d->layer_prec ? d->layer_prec[l] : d->prec;
        if ((s.k != 1 && s.k != 3) || s.cout < 1 || s.cout > 16384 || s.act < 0 || s.act > 1 ||
            s.pool < 0 || s.pool > 2 || s.bn < 0 || s.bn > 1)
            return fail(NET_E_INVAL, "layer %d: unsupported (k=%d cout=%d bn=%d act=%d pool=%d)", l,
                        s.k, s.cout, s.bn, s.act, s.pool);
        if (p < NET_FP32 || p > NET_FP8) return fail(NET_E_INVAL, "layer %d precision %d", l, p);
    }
    std::unique_ptr<net> n(new net());
    n->device = d->device;
    CK(cudaSetDevice(n->device));
    n->in_c = d->in_c;
    n->max_batch = d->max_batch;
    n->max_side = d->max_side;
    n->budget = d->hbm_budget_bytes ? d->hbm_budget_bytes : (size_t)40 << 30;
    int cin = d->in_c;
    for (int l = 0; l < d->n_layers; ++l) {
        const net_layer& s = d->layers[l];
        Layer L;
        L.d = s;
        L.cin = cin;
        L.prec = effective_prec(d->layer_prec ? d->layer_prec[l] : d->prec, cin);
        L.engine = layer_engine(L.prec);
        L.in_dt = L.engine == ENG_SIMT ? DT_F32 : prec_dt(L.prec);
        L.in_cs = pad_channels(cin, L.in_dt, L.engine == ENG_TC);
        L.kx = s.k;
        static const bool pair_on = [] {
            const char* e = getenv("NET_L0_PAIR");
            return !(e && atoi(e) == 0);
        }();
        if (l == 0 && L.engine == ENG_TC && L.in_dt == DT_BF16 && s.k == 3 && cin <= 8 && s.cout <= 256 &&
            pair_on) {
            // first layer on few channels: channels padded to 8 (16 bytes a
            // pixel), nine taps as five MMAs of two taps each (K = 16); one
            // N tile of at most 256 columns keeps its weights resident
            L.pair = true;
            L.in_cs = 8;
        } else if (l == 0 && L.engine == ENG_TC && L.in_dt == DT_BF16 && s.k == 3 && cin * 9 <= 32) {
            // first layer on few channels: fold its 9 taps into 32 channels at
            // pack time and run it as a 1x1 conv (one 64-byte K chunk per tile
            // instead of nine 32-byte ones)
            L.im2col_k = 3;
            L.kx = 1;
            L.in_cs = 32;
        }
        L.w_rows = rup(std::max(s.cout, rup(s.cout, 128)), 256);
        L.act_scale = 1.0;
        n->L.push_back(L);
        cin = s.cout;
    }
    for (auto& L : n->L)
        if (L.prec == NET_FP8) {
            n->has_fp8 = true;
            L.fp8_capable = true;
            L.cs_var[0] = pad_channels(L.cin, DT_BF16, true);
            L.cs_var[1] = pad_channels(L.cin, DT_FP8, true);
        }
    if (d->cuda_stream) {
        n->stream = (cudaStream_t)d->cuda_stream;
    } else {
        CK(cudaStreamCreate(&n->stream));   // blocking: ordered with the legacy default stream
        n->own_stream = true;
    }
    CK(cudaDeviceGetAttribute(&n->num_sms, cudaDevAttrMultiProcessorCount, n->device));
    CK(cudaHostAlloc((void**)&n->err_host, sizeof(int), cudaHostAllocMapped));
    *n->err_host = 0;
    CK(cudaHostGetDevicePointer((void**)&n->err_dev, n->err_host, 0));
    n->act_bytes = act_bytes_for(n.get(), n->max_batch, n->max_side, n->max_side);
    if (n->has_fp8) {
        // room for every FP8-capable layer switched to BF16 (the wider format)
        std::vector<Layer> keep = n->L;
        for (auto& L : n->L)
            if (L.fp8_capable) {
                L.in_dt = DT_BF16;
                L.in_cs = L.cs_var[0];
            }
        n->act_bytes = std::max(n->act_bytes, act_bytes_for(n.get(), n->max_batch, n->max_side, n->max_side));
        n->L = keep;
    }
    for (int i = 0; i < 3; ++i) {
        CK(dn::dalloc(&n->act[i], n->act_bytes));
        CK(cudaMemsetAsync(n->act[i], 0, n->act_bytes, n->stream));
    }
    int co, ho, wo;
    net_output_shape(n.get(), n->max_side, n->max_side, &co, &ho, &wo);
    n->in_stage_bytes = (size_t)n->max_batch * n->in_c * n->max_side * n->max_side * sizeof(float);
    n->out_stage_bytes = (size_t)n->max_batch * co * ho * wo * sizeof(float);
    CK(dn::dalloc(&n->d_in_stage, n->in_stage_bytes));
    CK(dn::dalloc(&n->d_out_stage, n->out_stage_bytes));
    CK(cudaStreamSynchronize(n->stream));
    *out = n.release();
    return NET_OK;
}

extern "C" net_status net_output_shape(const net_t* n, int h, int w, int* c, int* ho, int* wo) {
    if (!n || !c || !ho || !wo) return fail(NET_E_INVAL, "NULL argument");
    std::vector<int> H, W;
    layer_dims(n, h, w, H, W);
    *c = n->L.back().d.cout;
    *ho = H.back();
    *wo = W.back();
    return NET_OK;
}

// ------------------------------------------------------------- weights
static const int bns_all[3] = {64, 128, 256};

void dn::set_layer_format(Layer& L, int prec) {
    if (!L.fp8_capable) return;
    const int v = prec == NET_FP8 ? 1 : 0;
    L.prec = v ? NET_FP8 : NET_BF16;
    L.in_dt = v ? DT_FP8 : DT_BF16;
    L.in_cs = L.cs_var[v];
    if (L.w_var[v]) {
        L.w = L.w_var[v];
        std::memcpy(L.tmB, L.tmB_var[v], sizeof(L.tmB));
    }
}

extern "C" net_status net_load_weights(net_t* n, const float* blob, size_t n_floats) {
    if (!n || !blob) return fail(NET_E_INVAL, "NULL argument");
    size_t need = 0;
    for (auto& L : n->L)
        need += (size_t)L.d.cout * (L.d.bn ? 4 : 1) + (size_t)L.d.cout * L.cin * L.d.k * L.d.k;
    if (n_floats != need)
        return fail(NET_E_WEIGHTS, "weight blob has %zu floats, layers need %zu", n_floats, need);
    CK(cudaSetDevice(n->device));
    CK(cudaStreamSynchronize(n->stream));
    float* d_blob = nullptr;
    CK(dn::dalloc(&d_blob, need * sizeof(float)));
    cudaError_t e = cudaMemcpyAsync(d_blob, blob, need * sizeof(float), cudaMemcpyHostToDevice, n->stream);
    int maxc = 0;
    for (auto& L : n->L) maxc = std::max(maxc, L.d.cout);
    double* tmp = nullptr;
    if (e == cudaSuccess) e = dn::dalloc(&tmp, 2 * (size_t)maxc * sizeof(double));
    size_t off = 0;
    for (size_t l = 0; l < n->L.size() && e == cudaSuccess; ++l) {
        Layer& L = n->L[l];
        const int KK = L.d.k * L.d.k;
        FoldArgs a{};
        if (L.d.bn) {
            a.beta = d_blob + off;
            a.gamma = d_blob + off + L.d.cout;
            a.mean = d_blob + off + 2 * L.d.cout;
            a.var = d_blob + off + 3 * L.d.cout;
            off += 4 * (size_t)L.d.cout;
        } else {
            a.bias = d_blob + off;
            off += L.d.cout;
        }
        a.raw_w = d_blob + off;
        off += (size_t)L.d.cout * L.cin * KK;
        const int dt = L.in_dt;
        const int KKx = L.kx * L.kx;   // taps of the stored layout (1 when im2col-packed)
        const size_t wbytes = (size_t)L.w_rows * KKx * L.in_cs * dt_size(dt);
        if (!L.w) e = dn::dalloc(&L.w, wbytes);
        // bias and alpha are padded with zeros to w_rows: the tensor-core
        // epilogue reads them four at a time without bounds checks
        if (e == cudaSuccess && !L.bias) e = dn::dalloc(&L.bias, L.w_rows * sizeof(float));
        if (e == cudaSuccess) e = cudaMemsetAsync(L.bias, 0, L.w_rows * sizeof(float), n->stream);
        const bool fp8w = dt == DT_FP8 || L.fp8_capable;
        if (e == cudaSuccess && fp8w && !L.wscale) e = dn::dalloc(&L.wscale, L.d.cout * sizeof(float));
        if (e == cudaSuccess && fp8w && !L.alpha) {
            e = dn::dalloc(&L.alpha, L.w_rows * sizeof(float));
            if (e == cudaSuccess) e = cudaMemsetAsync(L.alpha, 0, L.w_rows * sizeof(float), n->stream);
        }
        L.cs32 = rup(L.cin, 4);
        const bool want32 = n->has_fp8 && dt != DT_F32;
        if (e == cudaSuccess && want32 && !L.w32) {
            e = dn::dalloc(&L.w32, (size_t)L.w_rows * KK * L.cs32 * sizeof(float));
            if (e == cudaSuccess)
                e = cudaMemsetAsync(L.w32, 0, (size_t)L.w_rows * KK * L.cs32 * sizeof(float), n->stream);
        }
        if (e != cudaSuccess) break;
        a.cout = L.d.cout;
        a.cin = L.cin;
        a.k = L.d.k;
        a.Cp = L.in_cs;
        a.w_rows = L.w_rows;
        a.dt = dt;
        a.out_w = L.w;
        a.out_bias = L.bias;
        a.out_wscale = L.wscale;
        a.tmp_s = tmp;
        a.tmp_amax = tmp + maxc;
        a.out_w32 = (want32 && !L.im2col_k) ? L.w32 : nullptr;
        a.Cp32 = L.cs32;
        a.im2col = L.im2col_k ? 1 : 0;
        e = fold_layer(a, n->stream);
        if (e == cudaSuccess && want32 && L.im2col_k) {
            // the FP32 reference copy keeps the plain [kh][kw][cin] layout
            FoldArgs b = a;
            b.im2col = 0;
            b.dt = DT_F32;
            b.Cp = L.cs32;
            b.out_w = L.w32;
            b.out_w32 = nullptr;
            b.out_wscale = nullptr;
            e = fold_layer(b, n->stream);
        }
        if (e == cudaSuccess && L.engine == ENG_TC) {
            const int bns[3] = {64, 128, 256};
            for (int i = 0; i < 3 && e == cudaSuccess; ++i)
                e = tc_encode_weights(&L.tmB[i], L.w, dt, L.w_rows, KKx, L.in_cs, bns[i]);
        }
        if (e == cudaSuccess && L.fp8_capable) {
            // both formats, whichever is active now: FP8 [1] and BF16 [0]
            for (int v = 0; v < 2 && e == cudaSuccess; ++v) {
                const int vdt = v ? DT_FP8 : DT_BF16;
                if (vdt == dt) {
                    L.w_var[v] = L.w;
                    std::memcpy(L.tmB_var[v], L.tmB, sizeof(L.tmB));
                    continue;
                }
                const size_t vb = (size_t)L.w_rows * KK * L.cs_var[v] * dt_size(vdt);
                if (!L.w_var[v]) e = dn::dalloc(&L.w_var[v], vb);
                if (e != cudaSuccess) break;
                FoldArgs b = a;
                b.Cp = L.cs_var[v];
                b.dt = vdt;
                b.out_w = L.w_var[v];
                b.out_w32 = nullptr;
                b.out_wscale = v ? L.wscale : nullptr;
                e = fold_layer(b, n->stream);
                for (int i = 0; i < 3 && e == cudaSuccess; ++i)
                    e = tc_encode_weights(&L.tmB_var[v][i], L.w_var[v], vdt, L.w_rows, KK, L.cs_var[v], bns_all[i]);
            }
        }
        if (e == cudaSuccess && fp8w) e = make_alpha(L.wscale, L.act_scale, L.alpha, L.d.cout, n->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    dn::dfree(d_blob);
    dn::dfree(tmp);
    if (e != cudaSuccess) return fail(NET_E_CUDA, "weight fold: %s", cudaGetErrorString(e));
    n->weights_loaded = true;
    n->night_weights_stale = true;
    n->graphs_clear();
    return NET_OK;
}

extern "C" net_status net_set_act_scales(net_t* n, const float* scales, int cnt) {
    if (!n || !scales) return fail(NET_E_INVAL, "NULL argument");
    if (cnt != (int)n->L.size()) return fail(NET_E_INVAL, "need %zu scales, got %d", n->L.size(), cnt);
    for (int l = 0; l < cnt; ++l)
        if (!(scales[l] > 0.f) || !std::isfinite(scales[l]))
            return fail(NET_E_INVAL, "scale %d = %g not positive finite", l, (double)scales[l]);
    CK(cudaSetDevice(n->device));
    for (int l = 0; l < cnt; ++l) {
        Layer& L = n->L[l];
        L.act_scale = scales[l];
        if ((L.in_dt == DT_FP8 || L.fp8_capable) && L.alpha && L.wscale) {
            cudaError_t e = make_alpha(L.wscale, L.act_scale, L.alpha, L.d.cout, n->stream);
            if (e != cudaSuccess) return fail(NET_E_CUDA, "alpha: %s", cudaGetErrorString(e));
        }
    }
    CK(cudaStreamSynchronize(n->stream));
    n->graphs_clear();
    return NET_OK;
}

// ------------------------------------------------------------ executor
// Input scale of layer l's storage for the FP8 format (1 otherwise).
static float in_scale(const Layer& L) { return L.in_dt == DT_FP8 ? (float)L.act_scale : 1.f; }

Plan::~Plan() {
    for (auto& r : runs)
        if (r.d_prob) dn::dfree(r.d_prob);
    if (flags) dn::dfree(flags);
}

bool dn::tc_flow_on() {
    static const bool on = [] {
        const char* e = getenv("NET_TC_FLOW");
        return !(e && atoi(e) == 0);
    }();
    return on;
}

// Analytic tile/split choice for the tensor-core kernel.  The mainloop is
// bound by the operand traffic from L2 (about 10 TB/s over the chip): per
// K step of a 128-byte chunk an SM moves the A box (16 KB, once per tap and
// N tile) plus BN x 128 B of B.  Measured K-step times with every SM busy:
// ~900, ~1020, ~1450 cycles for BN = 64, 128, 256 (so 256 does 1.4x the
// work per byte of 128).  Rounds of ceil(items / SMs) persistent tiles,
// plus the cost of a K split: reduced inside clusters (BF16, one wave), the
// partial tile's round trip through distributed shared memory (128 x BN x 4
// bytes at ~64 bytes a cycle) and ~1500 cycles per doubling of the cluster
// (calibrated on the 14 x 14 layers at batch 8, where a split of 4 instead
// of 2 measured no faster); otherwise the
// workspace written and read back by a reduction launch whose blocks (one
// per 128-row tile and 64 columns) fill the SMs only on large layers, plus
// that launch's fixed cost (~3 us).
static double tc_cost(long m_tiles, int ncols, int BN, int ks, int nk, int num_sms, bool xred) {
    static const double kstep_clk[3] = {900.0, 1020.0, 1450.0};   // BN = 64, 128, 256
    const int bi = BN == 64 ? 0 : BN == 128 ? 1 : 2;
    const long items = m_tiles * cdiv(ncols, BN) * ks;
    const long rounds = (items + num_sms - 1) / num_sms;
    double t = (double)rounds * ((double)nk / ks) * kstep_clk[bi] + rounds * 1500.0;   // + epilogue tail
    if (ks > 1) {
        if (xred && items <= num_sms && items <= tc_xred_capacity(BN, ks)) {
            t += 1500.0 * (1.0 + std::log2((double)ks)) + 128.0 * BN * 4.0 / 64.0;
        } else {
            const double blocks = (double)m_tiles * cdiv(ncols, 64);
            const double bw = 3450.0 * std::min(1.0, blocks / num_sms);   // bytes a cycle
            t += 6000.0 + (double)ks * m_tiles * 128 * cdiv(ncols, BN) * BN * 4.0 * 2.0 / bw;
        }
    }
    return t;
}

void dn::tc_choose(int batch, int H, int W, bool pool, int ncols, int num_sms, int* TW, int* TH, int* BN) {
    static const int tws[5] = {16, 8, 32, 64, 128};
    long best = -1;
    for (int i = 0; i < 5; ++i) {
        const int tw = tws[i], th = 128 / tw;
        if (pool && tw > 16) continue;
        const long cover = (long)cdiv(H, th) * th * cdiv(W, tw) * tw;
        if (best < 0 || cover < best) {
            best = cover;
            *TW = tw;
            *TH = th;
        }
    }
    (void)batch;
    (void)num_sms;
    *BN = ncols > 128 ? 256 : ncols > 64 ? 128 : 64;   // refined by tc_choose_split
}

// CTAs per SM, persistent worker count and resident-weight mode of a
// tensor-core launch.  Two CTAs an SM (mb_req = 0: chosen here; 1 or 2:
// forced) double the epilogue warps, which bound launches of many short
// tiles, but halve each CTA's shared memory: only for N tiles of at most 128
// columns, at least one tile an SM, and weights that stay resident (A-only
// stages) or at most two K steps per work item (a halved ring of A + B
// stages would starve a longer mainloop).
void dn::tc_workers(int m_tiles, int n_tiles, int ks, int BN, int nk, int chb, int num_sms, int mb_req, int* workers,
                    int* bres, int* mb) {
    const int items = m_tiles * n_tiles * ks;
    const bool res2 = BN <= 128 && tc_b_resident(BN, n_tiles, ks, nk, chb, 2);
    int m = 1;
    if (mb_req == 2 && BN <= 128) m = 2;
    else if (mb_req == 0 && BN <= 128 && items >= num_sms && (res2 || nk / ks <= 2)) m = 2;
    *mb = m;
    *bres = tc_b_resident(BN, n_tiles, ks, nk, chb, m) ? 1 : 0;
    *workers = std::max(1, std::min(items, num_sms * m));
    // resident weights with several N tiles: each CTA serves one N tile, so
    // the grid must be a multiple of the N tile count (the round-robin items
    // of a CTA then share it); drop residency where that rounds too far
    if (*bres && n_tiles > 1) {
        const int w = (*workers / n_tiles) * n_tiles;
        if (w < n_tiles || w * 8 < *workers * 7) *bres = 0;
        else *workers = w;
    }
}

// split-K reduced inside clusters where it can be (NET_TC_XRED=0: never)
bool dn::tc_xred_on() {
    static const bool on = [] {
        const char* e = getenv("NET_TC_XRED");
        return !(e && atoi(e) == 0);
    }();
    return on;
}

int dn::tc_mb_forced() {
    static const int v = [] {
        const char* e = getenv("NET_TC_MB");
        return e ? atoi(e) : 0;
    }();
    return v == 1 || v == 2 ? v : 0;
}

// CTA pairs for the layers that can take them (NET_TC_PAIR=0: never)
bool dn::tc_pair_enabled() {
    static const bool on = [] {
        const char* e = getenv("NET_TC_PAIR");
        return e && atoi(e) == 1;
    }();
    return on;
}

bool dn::pdl_enabled() {
    static const bool on = [] {
        const char* e = getenv("NET_PDL");
        return !(e && atoi(e) == 0);
    }();
    return on;
}

int dn::tmb_index(int BN) { return BN == 64 ? 0 : BN == 128 ? 1 : 2; }

void dn::tc_choose_split(long m_tiles, int ncols, int nk, int num_sms, int* BN, int* ksplit, int max_ks, bool xred) {
    double best = -1.0;
    for (int bn : {64, 128, 256}) {
        if (bn > rup(ncols, 64)) continue;
        for (int ks = 1; ks <= max_ks && (ks == 1 || ks * 4 <= nk); ks = ks < 2 ? ks + 1 : ks * 2) {
            const double t = tc_cost(m_tiles, ncols, bn, ks, nk, num_sms, xred);
            if (best < 0 || t < best) {
                best = t;
                *BN = bn;
                *ksplit = ks;
            }
        }
    }
    if (best < 0) {
        *BN = 64;
        *ksplit = 1;
    }
}

void dn::tc_tile_options(const net* n, int l, std::vector<TileOpt>* opts) {
    opts->clear();
    const Layer& L = n->L[l];
    if (L.engine != ENG_TC) return;
    const bool last = l + 1 == (int)n->L.size();
    const int out_cs = last ? rup(L.d.cout, 4) : n->L[l + 1].in_cs;
    const int ncols = std::max(L.d.cout, out_cs);
    const int nk = L.kx * L.kx * (L.in_cs / (tc_chunk_bytes(L.in_cs, L.in_dt) / (int)dt_size(L.in_dt)));
    for (int bn : {64, 128, 256}) {
        if (bn > rup(ncols, 64)) continue;
        if (L.pair && bn < ncols) continue;   // pair mode: one N tile
        for (int ks : {1, 2, 4, 8, 16})
            if (ks == 1 || (ks * 4 <= nk && !L.pair))
                for (int mb = 1; mb <= (bn <= 128 ? 2 : 1); ++mb) opts->push_back({bn, ks, mb});
    }
}

// Buffer sequence and TC launch tables for one (batch, h, w).
net_status dn::get_plan(net* n, int batch, int h, int w, Plan** out) {
    auto key = std::make_tuple(batch, h, w);
    auto it = n->plans.find(key);
    if (it != n->plans.end()) {
        *out = it->second;
        return NET_OK;
    }
    std::unique_ptr<Plan> P(new Plan());
    std::vector<int> H, W;
    layer_dims(n, h, w, H, W);
    const int nl = (int)n->L.size();
    int cur = 0;
    for (int l = 0; l < nl; ++l) {
        const Layer& L = n->L[l];
        const bool last = l + 1 == nl;
        LayerRun r;
        r.in_buf = cur;
        r.out_buf = (cur + 1) % 3;
        r.H = H[l];
        r.W = W[l];
        const int out_cs = last ? rup(L.d.cout, 4) : n->L[l + 1].in_cs;
        const int ncols = std::max(L.d.cout, out_cs);
        const int KK = L.kx * L.kx;
        if (L.engine == ENG_SIMT) {
            simt_tile(ncols, &r.sbn, &r.sth, &r.stw);
            const SimtGeom g = simt_geom(ncols, L.d.pool == NET_POOL_2X2S2, batch, r.H, r.W, false);
            r.m_tiles = g.m_tiles;
            r.n_tiles = cdiv(ncols, r.sbn);
            const int grid = r.m_tiles * r.n_tiles;
            const int nall = KK * cdiv(L.in_cs, 8);
            if (grid < 2 * n->num_sms && nall >= 32)
                r.ksplit = std::max(1, std::min({cdiv(4 * n->num_sms, grid), nall / 16, 32}));
            if (r.ksplit > 1)
                P->ws_bytes = std::max(P->ws_bytes, (size_t)r.ksplit * r.m_tiles * g.px *
                                                        r.n_tiles * r.sbn * sizeof(float));
        }
        if (L.engine == ENG_TC) {
            tc_choose(batch, r.H, r.W, L.d.pool == NET_POOL_2X2S2, ncols, n->num_sms, &r.TW, &r.TH, &r.BN);
            if (L.pair && !((r.TW == 16 && r.TH == 8) || (r.TW == 8 && r.TH == 16))) {
                r.TW = 16;   // pair mode runs on tap-merged 16 x 8 stages
                r.TH = 8;
            }
            // pair mode on 8 x 16 tiles: one TMA box a stage (NET_L0_BOX1=0: three)
            static const bool box1_on = [] {
                const char* e = getenv("NET_L0_BOX1");
                return !(e && atoi(e) == 0);
            }();
            if (L.pair && box1_on) {
                r.TW = 8;
                r.TH = 16;
            }
            r.m_tiles = batch * cdiv(r.H, r.TH) * cdiv(r.W, r.TW);
            const int nk = KK * (L.in_cs / (tc_chunk_bytes(L.in_cs, L.in_dt) / (int)dt_size(L.in_dt)));
            tc_choose_split(r.m_tiles, ncols, nk, n->num_sms, &r.BN, &r.ksplit, 16,
                            L.in_dt == DT_BF16 && tc_xred_on());
            // overrides (net_set_layer_tiles / net_tune_tiles), if still valid
            // for the layer's current format
            if (L.tile_bn > 0 && L.tile_bn <= rup(ncols, 64)) r.BN = L.tile_bn;
            if (L.tile_ks == 1 || (L.tile_ks > 1 && L.tile_ks * 4 <= nk)) r.ksplit = L.tile_ks;
            if (L.pair) {   // one N tile, no K split: the weights stay resident
                r.ksplit = 1;
                while (r.BN < ncols && r.BN < 256) r.BN *= 2;
            }
            r.n_tiles = cdiv(ncols, r.BN);
            const int tiles = r.m_tiles * r.n_tiles;
            if (r.ksplit > 1)
                P->ws_bytes = std::max(P->ws_bytes, (size_t)r.ksplit * r.m_tiles * 128 * r.n_tiles * r.BN *
                                                        sizeof(float));
            // the tap-pair first layer (32 live columns) measured slower with
            // two CTAs an SM (its 16-column epilogue chunks double the fixed
            // cost per chunk): one, unless forced or overridden
            int mb_req = (L.tile_mb == 1 || (L.tile_mb == 2 && r.BN <= 128)) ? L.tile_mb : tc_mb_forced();
            if (mb_req == 0 && L.pair) mb_req = 1;
            tc_workers(r.m_tiles, r.n_tiles, r.ksplit, r.BN, nk, tc_chunk_bytes(L.in_cs, L.in_dt), n->num_sms, mb_req,
                       &r.grid, &r.bres, &r.mb);
            {
                // one work item per CTA: the two MMA issuers share
                // each tile's K steps instead of idling one of them.  Fixed-batch
                // plans only: grouped launches keep one summation order for a
                // frame whatever else is in the batch.
                static const bool kalt_on = [] {
                    const char* e = getenv("NET_TC_KALT");
                    return !(e && atoi(e) == 0);
                }();
                // 3x3 layers with resident weights: one ring stage per channel
                // chunk of all nine taps (three boxes of TH + 2 rows)
                static const bool tapm_on = [] {
                    const char* e = getenv("NET_TC_TAPM");
                    return !(e && atoi(e) == 0);
                }();
                r.tapm = (tapm_on && r.bres && L.kx == 3 && r.ksplit == 1 &&
                          ((r.TW == 16 && r.TH == 8) || (r.TW == 8 && r.TH == 16)))
                             ? 1
                             : 0;
                if (L.pair) {
                    if (!r.bres) return fail(NET_E_UNSUPPORTED, "layer %d: pair mode needs resident weights", l);
                    r.tapm = 1;
                }
                const int steps = r.tapm ? nk / 9 : nk;   // pipeline steps per tile
                const int items = r.m_tiles * r.n_tiles * r.ksplit;
                r.kalt = (kalt_on && items <= r.grid && steps / r.ksplit >= 2) ? 1 : 0;
                // CTA pairs: layers that stream wide weight tiles (N tile of 128
                // or 256, not resident, one CTA an SM): an M = 256 tile a pair
                if (tc_pair_enabled() && r.mb == 1 && !r.bres && !r.tapm && !L.pair && r.BN >= 128) {
                    const int units = cdiv(r.m_tiles, 2) * r.n_tiles * r.ksplit;
                    r.cg = 2;
                    r.kalt = 0;
                    r.grid = 2 * std::max(1, std::min(units, n->num_sms / 2));
                }
                // BF16 split-K with one work item a CTA that all fit at once:
                // the ksplit CTAs of a tile form a cluster and add their partial
                // sums through distributed shared memory (no workspace round
                // trip, no reduction launch)
                r.xred = (tc_xred_on() && L.in_dt == DT_BF16 && r.ksplit > 1 && r.mb == 1 && r.cg == 1 && !r.bres &&
                          !r.tapm && !L.pair && items == r.grid && items <= tc_xred_capacity(r.BN, r.ksplit))
                             ? 1
                             : 0;
            }
            (void)tiles;
            ConvProblem hp;
            std::memset(&hp, 0, sizeof hp);
            const bool box1 = L.pair && r.TW == 8;   // one box of (TH + 2) x (TW + 2) pixels a stage
            cudaError_t e = tc_encode_act(&hp.tmA, n->act[r.in_buf], L.in_dt, batch, r.H, r.W, L.in_cs,
                                          box1 ? r.TW + 2 : r.TW, r.tapm ? r.TH + 2 : r.TH);
            if (e != cudaSuccess) return fail(NET_E_CUDA, "layer %d: activation tensor map: %s", l, cudaGetErrorString(e));
            hp.x = n->act[r.in_buf];
            hp.y = n->act[r.out_buf];
            hp.n = batch;
            hp.H = r.H;
            hp.W = r.W;
            hp.tiles_x = cdiv(r.W, r.TW);
            hp.tiles_y = cdiv(r.H, r.TH);
            tc_problem_divisors(hp);
            hp.tile_begin = 0;
            // row-band counters: one per (frame, tile row) of the output, and
            // the input-read counter
            if (r.cg == 1) {
                r.sig_off = P->nflags;
                P->nflags += batch * hp.tiles_y;
                r.rd_off = P->nflags++;
                r.done_off = P->nflags++;
            }
            // the table is complete on the device before any launch reads it
            // (kernels read it ahead of their dependency wait)
            CK(dn::dalloc(&r.d_prob, sizeof(ConvProblem)));
            CK(cudaMemcpyAsync(r.d_prob, &hp, sizeof hp, cudaMemcpyHostToDevice, n->stream));
            CK(cudaStreamSynchronize(n->stream));
            static const bool dump = getenv("NET_PLAN_DUMP") != nullptr;   // diagnostics: one line per layer
            if (dump)
                fprintf(stderr,
                        "plan b%d %dx%d layer %d: tile %dx%d BN %d m_tiles %d n_tiles %d ksplit %d grid %d mb %d "
                        "bres %d kalt %d tapm %d pair %d cg %d xred %d (cluster capacity %d)\n",
                        batch, h, w, l, r.TW, r.TH, r.BN, r.m_tiles, r.n_tiles, r.ksplit, r.grid, r.mb, r.bres,
                        r.kalt, r.tapm, L.pair ? 1 : 0, r.cg, r.xred,
                        r.ksplit > 1 && L.in_dt == DT_BF16 ? tc_xred_capacity(r.BN, r.ksplit) : 0);
        }
        P->runs.push_back(r);
        if (L.d.pool != NET_POOL_2X2S1_SAME) cur = (cur + 1) % 3;
    }
    if (P->nflags > 0) {
        CK(dn::dalloc(&P->flags, (size_t)P->nflags * sizeof(int)));
        CK(cudaMemsetAsync(P->flags, 0, (size_t)P->nflags * sizeof(int), n->stream));
        CK(cudaStreamSynchronize(n->stream));
    }
    if (P->ws_bytes > n->ws_bytes) {
        // grow the split-K workspace; graphs captured on the old one are dropped
        n->graphs_clear();
        if (n->ws) dn::dfree(n->ws);
        n->ws = nullptr;
        n->ws_bytes = 0;
        CK(dn::dalloc(&n->ws, P->ws_bytes));
        n->ws_bytes = P->ws_bytes;
    }
    *out = P.get();
    n->plans[key] = P.release();
    return NET_OK;
}

net_status dn::check_device_error(net* n) {
    if (n->err_host && *(volatile int*)n->err_host) {
        const int code = *(volatile int*)n->err_host;
        *(volatile int*)n->err_host = 0;
        return fail(NET_E_DEVICE_WAIT, "a bounded device-side wait expired (code %d)", code);
    }
    return NET_OK;
}

// Row-band dataflow of a fixed-batch plan: layer l runs without the
// dependency wait on the whole previous kernel (dep[l] = 1) when layers l - 1
// and l are tensor-core launches whose epilogues write their final outputs
// (no K split through the workspace, no reduction launch), no stride-1 pool
// sits among layers l - 2 .. l - 1, and layer l - 2 (whose input buffer
// layer l overwrites) is a tensor-core launch that counts its finished reads,
// or the pack.  Every tile a layer l - 1 epilogue warp drains costs it a
// release fence (about a round trip to L2), so only layers whose epilogue
// warps drain at most four tiles each signal their bands (at 19-conv 448^2
// b8 the first layer's 41 tiles a warp cost it 24 us of fences; a limit of
// two or eight tiles measured slower than four).  wpt[l]: the epilogue
// warps that add to a band per tile of layer l.  False (and nothing set)
// when the dataflow is off.
static bool flow_layers(const net* n, const Plan* plan, std::vector<char>& dep, std::vector<int>& wpt) {
    const int nl = (int)n->L.size();
    dep.assign(nl, 0);
    wpt.assign(nl, 0);
    if (!plan || !plan->flags || !pdl_enabled() || !tc_flow_on()) return false;
    std::vector<char> own(nl, 0), cheap(nl, 0);
    auto s1 = [&](int l) { return n->L[l].d.pool == NET_POOL_2X2S1_SAME; };
    for (int l = 0; l < nl; ++l) {
        const LayerRun& r = plan->runs[l];
        if (n->L[l].engine != ENG_TC || r.cg != 1 || r.sig_off < 0) continue;
        const bool last = l + 1 == nl;
        // the cluster reduction's epilogue writes BF16 NHWC (inner layers)
        const bool xr = r.xred && !last && !s1(l) && n->L[l + 1].in_dt == DT_BF16;
        if (r.ksplit == 1 || xr) {
            own[l] = 1;
            const int items = r.m_tiles * r.n_tiles * r.ksplit;
            const int per_cta = cdiv(items, std::max(1, r.grid));
            const int per_warp = r.kalt || xr ? per_cta : cdiv(per_cta, 2);
            cheap[l] = per_warp <= 4;
            wpt[l] = xr ? 8 * r.ksplit : r.kalt ? 8 : 4;
        }
    }
    for (int l = 1; l < nl; ++l)
        dep[l] = own[l] && own[l - 1] && cheap[l - 1] && !s1(l - 1) &&
                 (l < 2 || (n->L[l - 2].engine == ENG_TC && plan->runs[l - 2].cg == 1 && !s1(l - 2)));
    return true;
}

net_status dn::enqueue_forward(net* n, const float* d_in, int batch, int h, int w, float* d_out,
                               float* const* trace, bool fp32_copy, float* amax) {
    std::vector<int> H, W;
    layer_dims(n, h, w, H, W);
    cudaStream_t st = n->stream;
    const int nl = (int)n->L.size();
    Plan* plan = nullptr;
    if (!fp32_copy) {
        net_status ps = get_plan(n, batch, h, w, &plan);
        if (ps != NET_OK) return ps;
    }
    auto in_dt = [&](int l) { return fp32_copy ? DT_F32 : n->L[l].in_dt; };
    auto in_cs = [&](int l) { return fp32_copy ? n->L[l].cs32 : n->L[l].in_cs; };
    // the FP32 calibration copy alternates between two buffers; the pass
    // proper runs on the ring of three
    void* buf[3] = {fp32_copy ? n->cal[0] : n->act[0], fp32_copy ? n->cal[1] : n->act[1],
                    fp32_copy ? nullptr : n->act[2]};
    auto nxt = [&](int c) { return fp32_copy ? c ^ 1 : (c + 1) % 3; };
    int cur = 0;
    // Row-band dataflow (flow_layers): not with per-layer copies out (trace),
    // calibration or fault injection
    std::vector<char> dep(nl, 0);
    std::vector<int> wpt(nl, 0);
    const bool flow_ok = !fp32_copy && !amax && !trace && plan && n->fault_layer < 0 && flow_layers(n, plan, dep, wpt);
    int* zero = flow_ok ? plan->flags : nullptr;
    const int nzero = flow_ok ? plan->nflags : 0;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cap);
    auto mark = [&](cudaEvent_t ev) {
        return cap == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal)
                                                    : cudaEventRecord(ev, st);
    };
    const bool prof = n->prof && !fp32_copy && (int)n->prof_ev.size() == 2 * nl;
    n->pending = 1;
    cudaError_t e = cudaSuccess;
    if (!fp32_copy && n->L[0].im2col_k) {
        e = pack_frames_im2col(d_in, buf[cur], batch, n->in_c, h, w, in_cs(0), n->L[0].im2col_k, in_dt(0),
                               1.f / in_scale(n->L[0]), st);
    } else {
        e = pack_frames(d_in, buf[cur], batch, n->in_c, h, w, in_cs(0), in_dt(0), 1.f / in_scale(n->L[0]), st, zero,
                        nzero);
        zero = nullptr;
    }
    if (e == cudaSuccess && zero) e = cudaMemsetAsync(zero, 0, (size_t)nzero * sizeof(int), st);   // (im2col pack)
    if (e != cudaSuccess) return fail(NET_E_CUDA, "pack: %s", cudaGetErrorString(e));
    for (int l = 0; l < nl; ++l) {
        const Layer& L = n->L[l];
        const bool last = l + 1 == nl;
        if (amax && e == cudaSuccess) {
            ++n->pending;
            e = absmax_f32(reinterpret_cast<const float*>(buf[cur]),
                           (size_t)batch * H[l] * W[l] * in_cs(l), amax + l, st);
        }
        Epilogue ep{};
        ep.bias = L.bias;
        ep.alpha = (!fp32_copy && L.in_dt == DT_FP8) ? L.alpha : nullptr;
        ep.act = L.d.act;
        ep.pool = L.d.pool == NET_POOL_2X2S2 ? POOL_S2 : POOL_NONE;
        ep.cout = L.d.cout;
        const bool s1 = L.d.pool == NET_POOL_2X2S1_SAME;
        const bool direct_nchw = last && !s1 && !trace;
        void* y = nullptr;
        if (direct_nchw) {
            y = d_out;
            ep.out_layout = LAYOUT_NCHW;
            ep.out_dt = DT_F32;
            ep.out_cs = L.d.cout;
        } else {
            y = buf[nxt(cur)];
            ep.out_layout = LAYOUT_NHWC;
            ep.out_dt = last ? DT_F32 : in_dt(l + 1);
            ep.out_cs = last ? rup(L.d.cout, 4) : in_cs(l + 1);
            ep.out_inv_scale = (!last && ep.out_dt == DT_FP8) ? 1.f / in_scale(n->L[l + 1]) : 1.f;
        }
        if (e == cudaSuccess && prof) e = mark(n->prof_ev[2 * l]);
        if (e == cudaSuccess) {
            ++n->pending;
            if (!fp32_copy && L.engine == ENG_TC) {
                const LayerRun& r = plan->runs[l];
                TcArgs a{};
                a.probs = r.d_prob;
                a.nprob = 1;
                a.m_tiles = r.m_tiles;
                a.n_tiles = r.n_tiles;
                a.Cp = L.in_cs;
                a.k = L.kx;
                a.TW = r.TW;
                a.TH = r.TH;
                a.chb = tc_chunk_bytes(L.in_cs, L.in_dt);
                a.cpc = a.chb / (int)dt_size(L.in_dt);
                a.chunks = L.in_cs / a.cpc;
                a.y_override = y;
                a.ksplit = r.ksplit;
                a.ws = n->ws;
                a.bres = r.bres;
                a.kalt = r.kalt;
                a.tapm = r.tapm;
                a.pair = L.pair ? (r.TW == 8 ? 2 : 1) : 0;
                a.ep = ep;
                a.err = n->err_dev;
                int grid = r.grid, cg = r.cg;
                a.trace = (n->trace_on && n->trace_dev && grid <= kTraceCtas)
                              ? n->trace_dev + (size_t)l * kTraceCtas * kTraceEvents
                              : nullptr;
                // the cluster reduction's epilogue writes BF16 NHWC or FP32 NCHW
                a.xred = (r.xred && ((ep.out_layout == LAYOUT_NHWC && ep.out_dt == DT_BF16) ||
                                     (ep.out_layout == LAYOUT_NCHW && ep.out_dt == DT_F32)))
                             ? 1
                             : 0;
                // the frame pack lets this launch start early; the layers after
                // it must not start before the pack (which clears the counters)
                // has completed
                if (flow_ok && l == 0) a.late_trigger = 1;
                if (flow_ok && n->L[l].engine == ENG_TC && r.cg == 1 && r.rd_off >= 0) {
                    a.rd_sig = plan->flags + r.rd_off;   // read by layer l + 2, if it waits on it
                    if (l + 1 < nl && dep[l + 1]) {
                        a.sig = plan->flags + r.sig_off;
                        a.done_sig = plan->flags + r.done_off;
                    }
                    if (dep[l]) {
                        const LayerRun& rp = plan->runs[l - 1];
                        const bool pooled = n->L[l - 1].d.pool == NET_POOL_2X2S2;
                        const int band = pooled ? rp.TH / 2 : rp.TH;   // output rows of a tile row
                        int sh = 0;
                        while ((1 << sh) < band) ++sh;
                        if ((1 << sh) != band) return fail(NET_E_UNSUPPORTED, "layer %d: band of %d rows", l, band);
                        a.dep = plan->flags + rp.sig_off;
                        a.dep_shift = sh;
                        a.dep_nb = cdiv(rp.H, rp.TH);
                        a.dep_target = cdiv(rp.W, rp.TW) * rp.n_tiles * wpt[l - 1];
                        a.dep_done = plan->flags + rp.done_off;
                        a.dep_done_target = 8 * rp.grid;   // eight epilogue warps a CTA
                        if (l >= 2) {
                            const LayerRun& r2 = plan->runs[l - 2];
                            a.rd_dep = plan->flags + r2.rd_off;
                            a.rd_target = 2 * r2.grid;   // two producer warps a CTA
                        }
                    }
                }
                if (flow_ok && l == n->flow_fault_layer && dep[l]) {
                    // net_inject_flow_fault: a band count the previous layer never
                    // reaches, no whole-layer shortcut and a ~1 ms bound, once
                    a.dep_target += 1 << 28;
                    a.dep_done = nullptr;
                    a.wait_limit = 2000000;
                    n->flow_fault_layer = -1;
                }
                if (l == n->fault_layer) {
                    // net_inject_device_fault: a ~1 ms bound (clock64 cycles at
                    // ~2 GHz) and one K step withheld by a producer, once (a
                    // pair layer runs single-CTA for it: same tiles, one issuer)
                    a.wait_limit = 2000000;
                    a.withhold = 1;
                    a.xred = 0;   // the withheld step's layer reduces through the workspace
                    n->fault_layer = -1;
                    if (cg == 2) {
                        cg = 1;
                        grid = std::max(1, std::min(r.m_tiles * r.n_tiles * r.ksplit, n->num_sms));
                    }
                }
                e = conv_tc_launch(L.tmB[tmb_index(cg == 2 ? r.BN / 2 : r.BN)], a, r.BN, L.in_dt, grid, r.mb, cg,
                                   st);
                if (e == cudaSuccess && r.ksplit > 1 && !a.xred) {
                    ++n->pending;
                    SplitReduce sr{n->ws, r.ksplit, r.m_tiles * 128, r.n_tiles * r.BN, r.TW, r.TH,
                                   cdiv(r.W, r.TW), cdiv(r.H, r.TH), batch, r.H, r.W, y, ep, 1};
                    e = splitk_reduce(sr, st);
                }
            } else {
                ConvLaunch c{};
                c.x = buf[cur];
                c.w = fp32_copy ? (const void*)L.w32 : L.w;
                c.y = y;
                c.n = batch;
                c.H = H[l];
                c.W = W[l];
                c.Cp = in_cs(l);
                c.k = L.d.k;
                c.w_rows = L.w_rows;
                c.ep = ep;
                const LayerRun* r = plan ? &plan->runs[l] : nullptr;
                c.ksplit = r ? r->ksplit : 1;
                c.ws = n->ws;
                e = conv_simt(c, st);
                if (e == cudaSuccess && c.ksplit > 1) {
                    ++n->pending;
                    const int nc = ep.out_layout == LAYOUT_NCHW ? ep.cout : std::max(ep.out_cs, ep.cout);
                    const SimtGeom g = simt_geom(nc, ep.pool == POOL_S2, batch, H[l], W[l], false);
                    SplitReduce sr{n->ws, c.ksplit, g.m_tiles * g.px, cdiv(nc, g.bn) * g.bn, g.red_tw, g.red_th,
                                   g.red_tx, g.red_ty, batch, H[l], W[l], y, ep};
                    e = splitk_reduce(sr, st);
                }
            }
        }
        if (e == cudaSuccess && prof) e = mark(n->prof_ev[2 * l + 1]);
        if (e != cudaSuccess) return fail(NET_E_CUDA, "layer %d conv: %s", l, cudaGetErrorString(e));
        if (direct_nchw) break;
        const float osc = (last || ep.out_dt != DT_FP8) ? 1.f : in_scale(n->L[l + 1]);
        if (s1) {
            ++n->pending;
            e = maxpool_s1_same(buf[nxt(cur)], buf[cur], batch, H[l + 1], W[l + 1], ep.out_cs, ep.out_dt, st);
            // pooled result is back in buf[cur]
        } else {
            cur = nxt(cur);
        }
        if (e == cudaSuccess && (trace && trace[l]) && ++n->pending)
            e = unpack_nchw(buf[cur], trace[l], batch, L.d.cout, H[l + 1], W[l + 1], ep.out_cs, ep.out_dt, osc, st);
        if (e == cudaSuccess && last && ++n->pending)
            e = unpack_nchw(buf[cur], d_out, batch, L.d.cout, H[l + 1], W[l + 1], ep.out_cs, ep.out_dt, osc, st);
        if (e != cudaSuccess) return fail(NET_E_CUDA, "layer %d: %s", l, cudaGetErrorString(e));
    }
    return NET_OK;
}

void net::graphs_clear() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
    graph_kernels.clear();
    uneven_graphs_clear(this);   // uneven-batch graphs bake epilogue scales and weight maps too
}

net_status dn::run_forward(net* n, const float* d_in, int batch, int h, int w, float* d_out) {
    if (!n->use_graphs || n->fault_layer >= 0 || n->flow_fault_layer >= 0) {   // an injected fault is not baked into a graph
        net_status s = enqueue_forward(n, d_in, batch, h, w, d_out, nullptr, false, nullptr);
        if (s == NET_OK) n->launches += n->pending;
        return s;
    }
    auto key = std::make_tuple(batch, h, w, (const void*)d_in, (const void*)d_out);
    auto it = n->graphs.find(key);
    if (it == n->graphs.end()) {
        Plan* plan = nullptr;
        net_status ps = get_plan(n, batch, h, w, &plan);   // allocations happen outside capture
        if (ps != NET_OK) return ps;
        if (n->graphs.size() >= 64) n->graphs_clear();
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(n->stream, cudaStreamCaptureModeThreadLocal));
        net_status s = enqueue_forward(n, d_in, batch, h, w, d_out, nullptr, false, nullptr);
        cudaError_t e = cudaStreamEndCapture(n->stream, &g);
        if (s != NET_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) return fail(NET_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(NET_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
        it = n->graphs.emplace(key, ex).first;
        n->graph_kernels[key] = n->pending;
    }
    CK(cudaGraphLaunch(it->second, n->stream));
    n->launches += n->graph_kernels[key];
    return NET_OK;
}

extern "C" net_status net_forward_device(net_t* n, const float* d_in, int batch, int h, int w,
                                         float* d_out) {
    if (!n || !d_in || !d_out) return fail(NET_E_INVAL, "NULL argument");
    if (!n->weights_loaded) return fail(NET_E_WEIGHTS, "weights not loaded");
    net_status s = check_shape(n, batch, h, w);
    if (s != NET_OK) return s;
    s = check_device_error(n);   // a failure recorded by an earlier stream-ordered call
    if (s != NET_OK) return s;
    CK(cudaSetDevice(n->device));
    return run_forward(n, d_in, batch, h, w, d_out);
}

extern "C" net_status net_forward(net_t* n, const float* in, int batch, int h, int w, float* out,
                                  size_t cap) {
    if (!n || !in || !out) return fail(NET_E_INVAL, "NULL argument");
    if (!n->weights_loaded) return fail(NET_E_WEIGHTS, "weights not loaded");
    net_status s = check_shape(n, batch, h, w);
    if (s != NET_OK) return s;
    int c, ho, wo;
    net_output_shape(n, h, w, &c, &ho, &wo);
    const size_t nout = (size_t)batch * c * ho * wo;
    if (cap < nout) return fail(NET_E_INVAL, "output capacity %zu < %zu floats", cap, nout);
    CK(cudaSetDevice(n->device));
    const size_t nin = (size_t)batch * n->in_c * h * w;
    CK(cudaMemcpyAsync(n->d_in_stage, in, nin * sizeof(float), cudaMemcpyHostToDevice, n->stream));
    s = run_forward(n, n->d_in_stage, batch, h, w, n->d_out_stage);
    if (s != NET_OK) return s;
    CK(cudaMemcpyAsync(out, n->d_out_stage, nout * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    CK(cudaStreamSynchronize(n->stream));
    return check_device_error(n);
}

extern "C" net_status net_inject_device_fault(net_t* n, int layer) {
    if (!n) return fail(NET_E_INVAL, "NULL argument");
    if (layer < 0 || layer >= (int)n->L.size()) return fail(NET_E_INVAL, "layer %d out of range", layer);
    if (n->L[layer].engine != ENG_TC) return fail(NET_E_INVAL, "layer %d runs on CUDA cores", layer);
    n->fault_layer = layer;
    return NET_OK;
}

extern "C" net_status net_inject_flow_fault(net_t* n, int layer, int batch, int h, int w) {
    if (!n) return fail(NET_E_INVAL, "NULL argument");
    if (layer < 0 || layer >= (int)n->L.size()) return fail(NET_E_INVAL, "layer %d out of range", layer);
    net_status s = check_shape(n, batch, h, w);
    if (s != NET_OK) return s;
    CK(cudaSetDevice(n->device));
    Plan* P = nullptr;
    s = get_plan(n, batch, h, w, &P);
    if (s != NET_OK) return s;
    std::vector<char> d;
    std::vector<int> wpt;
    if (!flow_layers(n, P, d, wpt) || !d[layer])
        return fail(NET_E_INVAL, "layer %d does not wait on row bands in a %d x %d x %d pass", layer, batch, h, w);
    n->flow_fault_layer = layer;
    return NET_OK;
}

extern "C" net_status net_set_layer_tiles(net_t* n, int layer, int bn, int ksplit) {
    if (!n) return fail(NET_E_INVAL, "NULL argument");
    if (layer < 0 || layer >= (int)n->L.size()) return fail(NET_E_INVAL, "layer %d out of range", layer);
    if ((bn != 0 && bn != 64 && bn != 128 && bn != 256) ||
        (ksplit != 0 && ksplit != 1 && ksplit != 2 && ksplit != 4 && ksplit != 8 && ksplit != 16))
        return fail(NET_E_INVAL, "tile bn %d / ksplit %d not in {0,64,128,256} / {0,1,2,4,8,16}", bn, ksplit);
    Layer& L = n->L[layer];
    if (L.engine != ENG_TC && (bn || ksplit)) return fail(NET_E_INVAL, "layer %d runs on CUDA cores", layer);
    std::vector<TileOpt> opts;
    tc_tile_options(n, layer, &opts);
    bool bn_ok = bn == 0, ks_ok = ksplit == 0;
    for (auto& o : opts) {
        bn_ok |= o.bn == bn;
        ks_ok |= o.ks == ksplit;
    }
    if (!bn_ok || !ks_ok) return fail(NET_E_INVAL, "layer %d cannot take bn %d / ksplit %d", layer, bn, ksplit);
    if (L.tile_bn != bn || L.tile_ks != ksplit) {
        L.tile_bn = bn;
        L.tile_ks = ksplit;
        invalidate_plans(n);
    }
    return NET_OK;
}

extern "C" net_status net_set_layer_ctas(net_t* n, int layer, int mb) {
    if (!n) return fail(NET_E_INVAL, "NULL argument");
    if (layer < 0 || layer >= (int)n->L.size()) return fail(NET_E_INVAL, "layer %d out of range", layer);
    if (mb < 0 || mb > 2) return fail(NET_E_INVAL, "CTAs per SM %d not in {0, 1, 2}", mb);
    Layer& L = n->L[layer];
    if (L.engine != ENG_TC && mb) return fail(NET_E_INVAL, "layer %d runs on CUDA cores", layer);
    if (L.tile_mb != mb) {
        L.tile_mb = mb;
        invalidate_plans(n);
    }
    return NET_OK;
}

extern "C" net_status net_plan_ctas(net_t* n, int batch, int h, int w, int* mb, int nn) {
    if (!n || !mb) return fail(NET_E_INVAL, "NULL argument");
    if (nn < (int)n->L.size()) return fail(NET_E_INVAL, "need %d entries", (int)n->L.size());
    net_status s = check_shape(n, batch, h, w);
    if (s != NET_OK) return s;
    CK(cudaSetDevice(n->device));
    Plan* P = nullptr;
    s = get_plan(n, batch, h, w, &P);
    if (s != NET_OK) return s;
    for (size_t l = 0; l < n->L.size(); ++l) mb[l] = n->L[l].engine == ENG_TC ? P->runs[l].mb : 0;
    return NET_OK;
}

extern "C" net_status net_plan_flow(net_t* n, int batch, int h, int w, int* dep, int nn) {
    if (!n || !dep) return fail(NET_E_INVAL, "NULL argument");
    if (nn < (int)n->L.size()) return fail(NET_E_INVAL, "need %d entries", (int)n->L.size());
    net_status s = check_shape(n, batch, h, w);
    if (s != NET_OK) return s;
    CK(cudaSetDevice(n->device));
    Plan* P = nullptr;
    s = get_plan(n, batch, h, w, &P);
    if (s != NET_OK) return s;
    std::vector<char> d;
    std::vector<int> wpt;
    flow_layers(n, P, d, wpt);
    for (size_t l = 0; l < n->L.size(); ++l) dep[l] = d[l];
    return NET_OK;
}

extern "C" net_status net_plan_tiles(net_t* n, int batch, int h, int w, int* bn, int* ks, int nn) {
    if (!n || !bn || !ks) return fail(NET_E_INVAL, "NULL argument");
    if (nn < (int)n->L.size()) return fail(NET_E_INVAL, "need %d entries", (int)n->L.size());
    net_status s = check_shape(n, batch, h, w);
    if (s != NET_OK) return s;
    CK(cudaSetDevice(n->device));
    Plan* P = nullptr;
    s = get_plan(n, batch, h, w, &P);
    if (s != NET_OK) return s;
    for (size_t l = 0; l < n->L.size(); ++l) {
        const bool tc = n->L[l].engine == ENG_TC;
        bn[l] = tc ? P->runs[l].BN : 0;
        ks[l] = tc ? P->runs[l].ksplit : 0;
    }
    return NET_OK;
}

static net_status async_start(net* n) {
    if (n->async) return NET_OK;
    std::unique_ptr<net::AsyncState> A(new net::AsyncState());
    // own staging for both slots: a synchronous net_forward may run between
    // asynchronous calls without touching their buffers
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = dn::dalloc(&A->d_in[k], n->in_stage_bytes);
        if (e == cudaSuccess) e = dn::dalloc(&A->d_out[k], n->out_stage_bytes);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&A->s_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&A->s_out, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaEventCreateWithFlags(&A->ev_in[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&A->ev_comp[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&A->ev_free[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        for (int k = 0; k < 2; ++k) {
            dn::dfree(A->d_in[k]);
            dn::dfree(A->d_out[k]);
        }
        if (A->s_in) cudaStreamDestroy(A->s_in);
        if (A->s_out) cudaStreamDestroy(A->s_out);
        for (int k = 0; k < 2; ++k) {
            if (A->ev_in[k]) cudaEventDestroy(A->ev_in[k]);
            if (A->ev_comp[k]) cudaEventDestroy(A->ev_comp[k]);
            if (A->ev_free[k]) cudaEventDestroy(A->ev_free[k]);
        }
        return fail(NET_E_OOM, "async staging: %s", cudaGetErrorString(e));
    }
    n->async = A.release();
    return NET_OK;
}

static void async_free(net* n) {
    net::AsyncState* A = n->async;
    if (!A) return;
    cudaStreamSynchronize(A->s_in);
    cudaStreamSynchronize(n->stream);
    cudaStreamSynchronize(A->s_out);
    for (int k = 0; k < 2; ++k) {
        dn::dfree(A->d_in[k]);
        dn::dfree(A->d_out[k]);
    }
    cudaStreamDestroy(A->s_in);
    cudaStreamDestroy(A->s_out);
    for (int k = 0; k < 2; ++k) {
        cudaEventDestroy(A->ev_in[k]);
        cudaEventDestroy(A->ev_comp[k]);
        cudaEventDestroy(A->ev_free[k]);
    }
    delete A;
    n->async = nullptr;
}

extern "C" net_status net_forward_async(net_t* n, const float* in, int batch, int h, int w, float* out,
                                        size_t cap) {
    if (!n || !in || !out) return fail(NET_E_INVAL, "NULL argument");
    if (!n->weights_loaded) return fail(NET_E_WEIGHTS, "weights not loaded");
    net_status s = check_shape(n, batch, h, w);
    if (s != NET_OK) return s;
    int c, ho, wo;
    net_output_shape(n, h, w, &c, &ho, &wo);
    const size_t nout = (size_t)batch * c * ho * wo;
    if (cap < nout) return fail(NET_E_INVAL, "output capacity %zu < %zu floats", cap, nout);
    CK(cudaSetDevice(n->device));
    s = async_start(n);
    if (s != NET_OK) return s;
    net::AsyncState* A = n->async;
    const int k = A->next;
    A->next ^= 1;
    // the slot's previous batch: its download done means its pass and upload are too
    if (A->used[k]) CK(cudaEventSynchronize(A->ev_free[k]));
    A->used[k] = true;
    const size_t nin = (size_t)batch * n->in_c * h * w;
    CK(cudaMemcpyAsync(A->d_in[k], in, nin * sizeof(float), cudaMemcpyHostToDevice, A->s_in));
    CK(cudaEventRecord(A->ev_in[k], A->s_in));
    CK(cudaStreamWaitEvent(n->stream, A->ev_in[k], 0));
    s = run_forward(n, A->d_in[k], batch, h, w, A->d_out[k]);
    if (s != NET_OK) {
        if (A->first_err == NET_OK) A->first_err = s;
        return s;
    }
    CK(cudaEventRecord(A->ev_comp[k], n->stream));
    CK(cudaStreamWaitEvent(A->s_out, A->ev_comp[k], 0));
    CK(cudaMemcpyAsync(out, A->d_out[k], nout * sizeof(float), cudaMemcpyDeviceToHost, A->s_out));
    CK(cudaEventRecord(A->ev_free[k], A->s_out));
    return NET_OK;
}

extern "C" net_status net_forward_wait(net_t* n) {
    if (!n) return fail(NET_E_INVAL, "NULL argument");
    net::AsyncState* A = n->async;
    if (!A) return NET_OK;
    CK(cudaSetDevice(n->device));
    CK(cudaStreamSynchronize(A->s_in));
    CK(cudaStreamSynchronize(n->stream));
    CK(cudaStreamSynchronize(A->s_out));
    net_status s = A->first_err;
    A->first_err = NET_OK;
    A->used[0] = A->used[1] = false;
    if (s != NET_OK) return s;
    return check_device_error(n);
}

extern "C" net_status net_forward_trace(net_t* n, const float* d_in, int batch, int h, int w,
                                        float* const* d_layer_out) {
    if (!n || !d_in || !d_layer_out) return fail(NET_E_INVAL, "NULL argument");
    if (!n->weights_loaded) return fail(NET_E_WEIGHTS, "weights not loaded");
    net_status s = check_shape(n, batch, h, w);
    if (s != NET_OK) return s;
    CK(cudaSetDevice(n->device));
    net_status s2 = enqueue_forward(n, d_in, batch, h, w, d_layer_out[n->L.size() - 1], d_layer_out,
                                    false, nullptr);
    if (s2 == NET_OK) n->launches += n->pending;
    return s2;
}

extern "C" net_status net_profile(net_t* n, int enable) {
    if (!n) return fail(NET_E_INVAL, "NULL argument");
    CK(cudaSetDevice(n->device));
    CK(cudaStreamSynchronize(n->stream));
    if (enable && n->prof_ev.empty()) {
        n->prof_ev.resize(2 * n->L.size());
        for (auto& ev : n->prof_ev) CK(cudaEventCreate(&ev));
    }
    n->prof = enable != 0;
    n->graphs_clear();
    return NET_OK;
}

extern "C" net_status net_layer_times(net_t* n, double* ms, int cnt) {
    if (!n || !ms) return fail(NET_E_INVAL, "NULL argument");
    if (cnt != (int)n->L.size()) return fail(NET_E_INVAL, "need %zu entries", n->L.size());
    if (!n->prof) return fail(NET_E_STATE, "profiling not enabled");
    CK(cudaStreamSynchronize(n->stream));
    for (int l = 0; l < cnt; ++l) {
        float t = 0.f;
        cudaError_t e = cudaEventElapsedTime(&t, n->prof_ev[2 * l], n->prof_ev[2 * l + 1]);
        if (e != cudaSuccess) return fail(NET_E_STATE, "layer %d has no timing yet: %s", l, cudaGetErrorString(e));
        ms[l] = t;
    }
    return NET_OK;
}

extern "C" net_status net_trace(net_t* n, int enable) {
    if (!n) return fail(NET_E_INVAL, "NULL argument");
    CK(cudaSetDevice(n->device));
    CK(cudaStreamSynchronize(n->stream));
    const size_t bytes = n->L.size() * (size_t)kTraceCtas * kTraceEvents * sizeof(unsigned long long);
    if (enable && !n->trace_dev) CK(dn::dalloc(&n->trace_dev, bytes));
    if (enable) CK(cudaMemset(n->trace_dev, 0, bytes));
    n->trace_on = enable != 0;
    n->graphs_clear();   // captured launches hold the trace pointer (or none)
    return NET_OK;
}

extern "C" net_status net_trace_read(net_t* n, uint64_t* out, size_t cap) {
    if (!n || !out) return fail(NET_E_INVAL, "NULL argument");
    const size_t words = n->L.size() * (size_t)kTraceCtas * kTraceEvents;
    if (cap < words) return fail(NET_E_INVAL, "need %zu entries", words);
    if (!n->trace_dev) return fail(NET_E_STATE, "tracing never enabled");
    CK(cudaSetDevice(n->device));
    CK(cudaStreamSynchronize(n->stream));
    CK(cudaMemcpy(out, n->trace_dev, words * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    return NET_OK;
}

extern "C" net_status net_launches(const net_t* n, uint64_t* total) {
    if (!n || !total) return fail(NET_E_INVAL, "NULL argument");
    *total = n->launches;
    return NET_OK;
}

net_status dn::run_fp32_reference(net* n, const float* d_frames, int batch, int h, int w, float* d_out,
                                  float* amax) {
    // FP32 buffers for the pass over the FP32 copy of the folded weights
    std::vector<int> H, W;
    layer_dims(n, h, w, H, W);
    size_t mx = 0;
    for (size_t l = 0; l < n->L.size(); ++l) {
        mx = std::max(mx, (size_t)batch * H[l] * W[l] * n->L[l].cs32 * 4);
        mx = std::max(mx, (size_t)batch * H[l + 1] * W[l + 1] * rup(n->L[l].d.cout, 4) * 4);
    }
    CK(dn::dalloc(&n->cal[0], mx));
    cudaError_t e = dn::dalloc(&n->cal[1], mx);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->cal[0], 0, mx, n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->cal[1], 0, mx, n->stream);
    // layers whose own weights are FP32 use them directly
    std::vector<float*> saved(n->L.size());
    for (size_t l = 0; l < n->L.size(); ++l) {
        saved[l] = n->L[l].w32;
        if (!n->L[l].w32) n->L[l].w32 = reinterpret_cast<float*>(n->L[l].w);
    }
    net_status s = e == cudaSuccess ? enqueue_forward(n, d_frames, batch, h, w, d_out, nullptr, true, amax)
                                    : fail(NET_E_OOM, "reference buffers: %s", cudaGetErrorString(e));
    if (s == NET_OK) {
        e = cudaStreamSynchronize(n->stream);
        if (e != cudaSuccess) s = fail(NET_E_CUDA, "reference pass: %s", cudaGetErrorString(e));
    }
    for (size_t l = 0; l < n->L.size(); ++l) n->L[l].w32 = saved[l];
    dn::dfree(n->cal[0]);
    dn::dfree(n->cal[1]);
    n->cal[0] = n->cal[1] = nullptr;
    return s;
}

extern "C" net_status net_calibrate(net_t* n, const float* d_frames, int batch, int h, int w,
                                    float* scales_out) {
    if (!n || !d_frames) return fail(NET_E_INVAL, "NULL argument");
    if (!n->weights_loaded) return fail(NET_E_WEIGHTS, "weights not loaded");
    if (!n->has_fp8) return fail(NET_E_STATE, "no FP8 layer to calibrate");
    net_status s = check_shape(n, batch, h, w);
    if (s != NET_OK) return s;
    CK(cudaSetDevice(n->device));
    float *amax = nullptr, *dout = nullptr;
    int c, ho, wo;
    net_output_shape(n, h, w, &c, &ho, &wo);
    CK(dn::dalloc(&amax, n->L.size() * sizeof(float)));
    CK(dn::dalloc(&dout, (size_t)batch * c * ho * wo * sizeof(float)));
    CK(cudaMemsetAsync(amax, 0, n->L.size() * sizeof(float), n->stream));
    s = run_fp32_reference(n, d_frames, batch, h, w, dout, amax);
    std::vector<float> hm(n->L.size());
    // the handle's stream may be non-blocking: finish it before a plain copy
    cudaError_t e = cudaStreamSynchronize(n->stream);
    if (e == cudaSuccess) e = cudaMemcpy(hm.data(), amax, hm.size() * sizeof(float), cudaMemcpyDeviceToHost);
    dn::dfree(amax);
    dn::dfree(dout);
    if (s != NET_OK) return s;
    if (e != cudaSuccess) return fail(NET_E_CUDA, "calibrate: %s", cudaGetErrorString(e));
    std::vector<float> sc(n->L.size());
    for (size_t l = 0; l < n->L.size(); ++l) sc[l] = std::max(hm[l], 1e-30f) / kFp8Max;
    if (scales_out) std::memcpy(scales_out, sc.data(), sc.size() * sizeof(float));
    return net_set_act_scales(n, sc.data(), (int)sc.size());
}

void dn::invalidate_plans(net* n) {
    n->graphs_clear();
    for (auto& kv : n->plans) delete kv.second;
    n->plans.clear();
    uneven_free(n);
}

extern "C" net_status net_set_layer_prec(net_t* n, const int* prec, int cnt) {
    if (!n || !prec) return fail(NET_E_INVAL, "NULL argument");
    if (cnt != (int)n->L.size()) return fail(NET_E_INVAL, "need %zu entries", n->L.size());
    for (int l = 0; l < cnt; ++l) {
        const Layer& L = n->L[l];
        const bool ok = L.fp8_capable ? (prec[l] == NET_FP8 || prec[l] == NET_BF16) : prec[l] == L.prec;
        if (!ok)
            return fail(NET_E_INVAL, "layer %d: precision %d not available (created as %d%s)", l, prec[l], L.prec,
                        L.fp8_capable ? ", FP8/BF16 switchable" : "");
    }
    CK(cudaSetDevice(n->device));
    CK(cudaStreamSynchronize(n->stream));
    for (int l = 0; l < cnt; ++l) set_layer_format(n->L[l], prec[l]);
    invalidate_plans(n);
    return NET_OK;
}

extern "C" net_status net_get_layer_prec(const net_t* n, int* prec, int cnt) {
    if (!n || !prec) return fail(NET_E_INVAL, "NULL argument");
    if (cnt != (int)n->L.size()) return fail(NET_E_INVAL, "need %zu entries", n->L.size());
    for (int l = 0; l < cnt; ++l) prec[l] = n->L[l].prec;
    return NET_OK;
}

extern "C" net_status net_forward_uneven(net_t* n, const float* const* d_in, const int* side, int cnt,
                                         float* const* d_out) {
    if (!n || !d_in || !side || !d_out || cnt < 1) return fail(NET_E_INVAL, "bad argument");
    if (!n->weights_loaded) return fail(NET_E_WEIGHTS, "weights not loaded");
    for (int i = 0; i < cnt; ++i) {
        net_status s = check_shape(n, 1, side[i], side[i]);
        if (s != NET_OK) return s;
        if (!d_in[i] || !d_out[i]) return fail(NET_E_INVAL, "NULL frame pointer %d", i);
    }
    CK(cudaSetDevice(n->device));
    return enqueue_uneven(n, d_in, side, cnt, d_out);
}

extern "C" net_status net_free(net_t* n) {
    if (!n) return NET_OK;
    cudaSetDevice(n->device);
    serve_stop(n);
    if (n->stream) cudaStreamSynchronize(n->stream);
    n->graphs_clear();
    for (auto ev : n->prof_ev) cudaEventDestroy(ev);
    if (n->trace_dev) dn::dfree(n->trace_dev);
    for (auto& L : n->L) {
        for (int v = 0; v < 2; ++v)
            if (L.w_var[v] && L.w_var[v] != L.w) dn::dfree(L.w_var[v]);
        dn::dfree(L.w);
        dn::dfree(L.bias);
        dn::dfree(L.wscale);
        dn::dfree(L.alpha);
        dn::dfree(L.w32);
    }
    for (auto& kv : n->plans) delete kv.second;
    n->plans.clear();
    if (n->ws) dn::dfree(n->ws);
    if (n->err_host) cudaFreeHost(n->err_host);
    dn::dfree(n->act[0]);
    dn::dfree(n->act[1]);
    dn::dfree(n->act[2]);
    async_free(n);
    dn::dfree(n->d_in_stage);
    dn::dfree(n->d_out_stage);
    uneven_free(n);
    region_free(n);
    night_free(n);
    if (n->own_stream) cudaStreamDestroy(n->stream);
    delete n;
    return NET_OK;
}

extern "C" const char* net_last_error(void) { return g_err.c_str(); }

extern "C" const char* net_version(void) { return "gb300-darknet-resident 0.1 (sm_103a)"; }
