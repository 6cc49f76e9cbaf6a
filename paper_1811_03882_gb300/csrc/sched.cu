// sched.cu — uneven-batch execution and the serving request queue.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <vector>

#include "../../include/net.h"
#include "net_internal.h"

using namespace dn;

// ------------------------------------------------------------ uneven batch
// All frames of an uneven batch go through each layer in ONE grouped launch:
// the tensor-core kernel takes a device table of problems (one per frame,
// each with its own activation tensor map, size and output), and the pack
// and stride-1 pool kernels take job tables.  Frames share no reduction, so
// a frame's result does not depend on the other frames in the batch.
namespace dn {

struct UPlan {
    std::vector<LayerRun> runs;        // d_prob: table of `frames` problems
    PackJob* d_pack = nullptr;
    long long pack_total = 0;
    std::vector<PoolJob*> d_pool;      // per layer (stride-1 pool layers only)
    std::vector<long long> pool_total;
    std::vector<int> cur;              // buffer holding the input of layer l
    cudaGraphExec_t graph = nullptr;
    int kernels = 0;
    ~UPlan() {
        for (auto& r : runs)
            if (r.d_prob) dn::dfree(r.d_prob);
        if (d_pack) dn::dfree(d_pack);
        for (auto* p : d_pool)
            if (p) dn::dfree(p);
        if (graph) cudaGraphExecDestroy(graph);
    }
};

struct UnevenState {
    void* buf[2] = {nullptr, nullptr};
    size_t cap = 0;
    std::map<std::vector<uintptr_t>, UPlan*> plans;
};

}  // namespace dn

static size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

static net_status build_uplan(net* n, const float* const* d_in, const int* side, int cnt,
                              float* const* d_out, UPlan** out) {
    UnevenState* U = n->uneven;
    const int nl = (int)n->L.size();
    // per-frame sizes at every layer input
    std::vector<std::vector<int>> H(cnt), W(cnt);
    for (int f = 0; f < cnt; ++f) layer_dims(n, side[f], side[f], H[f], W[f]);
    // offsets of each frame's tensor at each layer boundary t (input of layer t)
    std::vector<std::vector<size_t>> off(nl, std::vector<size_t>(cnt));
    size_t need = 256;
    for (int t = 0; t < nl; ++t) {
        size_t o = 0;
        for (int f = 0; f < cnt; ++f) {
            off[t][f] = o;
            o += up256((size_t)H[f][t] * W[f][t] * n->L[t].in_cs * dt_size(n->L[t].in_dt));
        }
        need = std::max(need, o);
    }
    if (need > U->cap) {
        for (auto& kv : U->plans) delete kv.second;   // plans point into the old arena
        U->plans.clear();
        for (int i = 0; i < 2; ++i) {
            if (U->buf[i]) dn::dfree(U->buf[i]);
            U->buf[i] = nullptr;
        }
        U->cap = 0;
        for (int i = 0; i < 2; ++i) {
            cudaError_t e = dn::dalloc(&U->buf[i], need);
            if (e != cudaSuccess) return fail(NET_E_OOM, "uneven arena %zu bytes: %s", need, cudaGetErrorString(e));
            cudaMemset(U->buf[i], 0, need);
        }
        U->cap = need;
    }
    std::unique_ptr<UPlan> P(new UPlan());
    P->d_pool.assign(nl, nullptr);
    P->pool_total.assign(nl, 0);
    P->cur.assign(nl, 0);
    auto bufp = [&](int b, size_t o) { return (void*)((char*)U->buf[b] + o); };
    // pack jobs
    {
        std::vector<PackJob> jobs(cnt);
        const int V = 16 / (int)dt_size(n->L[0].in_dt);
        long long b = 0;
        for (int f = 0; f < cnt; ++f) {
            jobs[f] = PackJob{d_in[f], bufp(0, off[0][f]), n->in_c, side[f], side[f], n->L[0].in_cs,
                              n->L[0].im2col_k, b};
            b += (long long)side[f] * side[f] * (n->L[0].im2col_k ? 1 : n->L[0].in_cs / V);
        }
        P->pack_total = b;
        cudaError_t e = dn::dalloc(&P->d_pack, sizeof(PackJob) * cnt);
        if (e == cudaSuccess) e = cudaMemcpy(P->d_pack, jobs.data(), sizeof(PackJob) * cnt, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(NET_E_CUDA, "pack table: %s", cudaGetErrorString(e));
    }
    int cur = 0;
    for (int l = 0; l < nl; ++l) {
        const Layer& L = n->L[l];
        const bool last = l + 1 == nl;
        P->cur[l] = cur;
        LayerRun r;
        r.in_buf = cur;
        r.out_buf = cur ^ 1;
        const bool pool2 = L.d.pool == NET_POOL_2X2S2;
        const int out_cs = last ? L.d.cout : n->L[l + 1].in_cs;
        const int ncols = std::max(L.d.cout, out_cs);
        // one tile shape for all frames: least padded area over the batch
        static const int tws[5] = {16, 8, 32, 64, 128};
        long best = -1;
        for (int i = 0; i < 5; ++i) {
            const int tw = tws[i], th = 128 / tw;
            if (pool2 && tw > 16) continue;
            long cover = 0;
            for (int f = 0; f < cnt; ++f) cover += (long)cdiv(H[f][l], th) * th * cdiv(W[f][l], tw) * tw;
            if (best < 0 || cover < best) {
                best = cover;
                r.TW = tw;
                r.TH = th;
            }
        }
        if (L.pair) {   // pair mode: tap-merged 16 x 8 stages
            r.TW = 16;
            r.TH = 8;
        }
        std::vector<ConvProblem> probs(cnt);
        int mt = 0;
        for (int f = 0; f < cnt; ++f) {
            ConvProblem& q = probs[f];
            std::memset(&q, 0, sizeof q);
            cudaError_t e = tc_encode_act(&q.tmA, bufp(cur, off[l][f]), L.in_dt, 1, H[f][l], W[f][l], L.in_cs,
                                          r.TW, L.pair ? r.TH + 2 : r.TH);
            if (e != cudaSuccess) return fail(NET_E_CUDA, "layer %d frame %d tensor map", l, f);
            q.x = bufp(cur, off[l][f]);
            q.y = last ? (void*)d_out[f] : bufp(cur ^ 1, off[l + 1][f]);
            q.n = 1;
            q.H = H[f][l];
            q.W = W[f][l];
            q.tiles_x = cdiv(q.W, r.TW);
            q.tiles_y = cdiv(q.H, r.TH);
            tc_problem_divisors(q);
            q.tile_begin = mt;
            mt += q.tiles_x * q.tiles_y;
        }
        r.m_tiles = mt;
        int ks_unused = 1;
        const int nk = L.kx * L.kx * (L.in_cs / (tc_chunk_bytes(L.in_cs, L.in_dt) / (int)dt_size(L.in_dt)));
        // grouped launches do not split K; pick the N tile for ks = 1
        tc_choose_split(mt, ncols, nk, n->num_sms, &r.BN, &ks_unused, 1);
        int mb_req = 1;
        grouped_tiles(L, ncols, &r.BN, &mb_req, &r.nst_cap);
        r.n_tiles = cdiv(ncols, r.BN);
        tc_workers(r.m_tiles, r.n_tiles, 1, r.BN, nk, tc_chunk_bytes(L.in_cs, L.in_dt), n->num_sms, mb_req, &r.grid,
                   &r.bres, &r.mb);
        if (L.pair && !r.bres) return fail(NET_E_UNSUPPORTED, "layer %d: pair mode needs resident weights", l);
        r.tapm = L.pair ? 1 : 0;
        cudaError_t e = dn::dalloc(&r.d_prob, sizeof(ConvProblem) * cnt);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(r.d_prob, probs.data(), sizeof(ConvProblem) * cnt, cudaMemcpyHostToDevice, n->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
        if (e != cudaSuccess) return fail(NET_E_CUDA, "layer %d problem table: %s", l, cudaGetErrorString(e));
        if (L.d.pool == NET_POOL_2X2S1_SAME) {
            if (last) return fail(NET_E_UNSUPPORTED, "stride-1 pool on the last layer of an uneven batch");
            std::vector<PoolJob> jobs(cnt);
            const int V = 16 / (int)dt_size(n->L[l + 1].in_dt);
            long long b = 0;
            for (int f = 0; f < cnt; ++f) {
                jobs[f] = PoolJob{bufp(cur ^ 1, off[l + 1][f]), bufp(cur, off[l + 1][f]), H[f][l + 1], W[f][l + 1], b};
                b += (long long)H[f][l + 1] * W[f][l + 1] * (n->L[l + 1].in_cs / V);
            }
            P->pool_total[l] = b;
            e = dn::dalloc(&P->d_pool[l], sizeof(PoolJob) * cnt);
            if (e == cudaSuccess) e = cudaMemcpy(P->d_pool[l], jobs.data(), sizeof(PoolJob) * cnt, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return fail(NET_E_CUDA, "pool table: %s", cudaGetErrorString(e));
        } else {
            cur ^= 1;
        }
        P->runs.push_back(r);
    }
    *out = P.release();
    return NET_OK;
}

static float in_scale_of(const Layer& L) { return L.in_dt == DT_FP8 ? (float)L.act_scale : 1.f; }

static net_status enqueue_uplan(net* n, UPlan* P, int cnt, int* kernels) {
    cudaStream_t st = n->stream;
    const int nl = (int)n->L.size();
    int k = 1;
    cudaError_t e = pack_frames_grouped(P->d_pack, cnt, P->pack_total, n->L[0].in_dt, 1.f / in_scale_of(n->L[0]), st);
    for (int l = 0; l < nl && e == cudaSuccess; ++l) {
        const Layer& L = n->L[l];
        const LayerRun& r = P->runs[l];
        const bool last = l + 1 == nl;
        TcArgs a{};
        a.probs = r.d_prob;
        a.nprob = cnt;
        a.m_tiles = r.m_tiles;
        a.n_tiles = r.n_tiles;
        a.Cp = L.in_cs;
        a.k = L.kx;
        a.TW = r.TW;
        a.TH = r.TH;
        a.chb = tc_chunk_bytes(L.in_cs, L.in_dt);
        a.cpc = a.chb / (int)dt_size(L.in_dt);
        a.chunks = L.in_cs / a.cpc;
        a.y_override = nullptr;
        a.ksplit = 1;
        a.ws = nullptr;
        a.bres = r.bres;
        a.nst_cap = r.nst_cap;
        a.tapm = r.tapm;
        a.pair = L.pair ? 1 : 0;
        a.err = n->err_dev;
        a.ep.bias = L.bias;
        a.ep.alpha = L.in_dt == DT_FP8 ? L.alpha : nullptr;
        a.ep.act = L.d.act;
        a.ep.pool = L.d.pool == NET_POOL_2X2S2 ? POOL_S2 : POOL_NONE;
        a.ep.cout = L.d.cout;
        if (last) {
            a.ep.out_layout = LAYOUT_NCHW;
            a.ep.out_dt = DT_F32;
            a.ep.out_cs = L.d.cout;
        } else {
            a.ep.out_layout = LAYOUT_NHWC;
            a.ep.out_dt = n->L[l + 1].in_dt;
            a.ep.out_cs = n->L[l + 1].in_cs;
            a.ep.out_inv_scale = a.ep.out_dt == DT_FP8 ? 1.f / in_scale_of(n->L[l + 1]) : 1.f;
        }
        const bool prof = n->prof && (int)n->prof_ev.size() == 2 * nl;
        if (prof) e = cudaEventRecordWithFlags(n->prof_ev[2 * l], st, cudaEventRecordExternal);
        if (e == cudaSuccess) e = conv_tc_launch(L.tmB[tmb_index(r.BN)], a, r.BN, L.in_dt, r.grid, r.mb, 1, st);
        if (e == cudaSuccess && prof) e = cudaEventRecordWithFlags(n->prof_ev[2 * l + 1], st, cudaEventRecordExternal);
        ++k;
        if (e == cudaSuccess && P->d_pool[l]) {
            e = maxpool_s1_grouped(P->d_pool[l], cnt, P->pool_total[l], n->L[l + 1].in_cs, n->L[l + 1].in_dt, st);
            ++k;
        }
    }
    if (e != cudaSuccess) return fail(NET_E_CUDA, "uneven batch: %s", cudaGetErrorString(e));
    *kernels = k;
    return NET_OK;
}

static net_status enqueue_uplan_graph(net* n, UPlan* P, int cnt) {
    if (!P->graph) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(n->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return fail(NET_E_CUDA, "capture: %s", cudaGetErrorString(e));
        net_status s = enqueue_uplan(n, P, cnt, &P->kernels);
        e = cudaStreamEndCapture(n->stream, &g);
        if (s != NET_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) return fail(NET_E_CUDA, "capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&P->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(NET_E_CUDA, "instantiate: %s", cudaGetErrorString(e));
    }
    cudaError_t e = cudaGraphLaunch(P->graph, n->stream);
    if (e != cudaSuccess) return fail(NET_E_CUDA, "graph launch: %s", cudaGetErrorString(e));
    n->launches += P->kernels;
    return NET_OK;
}

net_status dn::enqueue_uneven(net* n, const float* const* d_in, const int* side, int cnt,
                              float* const* d_out) {
    bool all_tc = true;
    for (auto& L : n->L) all_tc = all_tc && L.engine == ENG_TC;
    if (!all_tc) {
        // CUDA-core (FP32) layers have no grouped kernel: frame by frame
        for (int i = 0; i < cnt; ++i) {
            net_status s = run_forward(n, d_in[i], 1, side[i], side[i], d_out[i]);
            if (s != NET_OK) return s;
        }
        return NET_OK;
    }
    if (!n->uneven) n->uneven = new UnevenState();
    std::vector<uintptr_t> key;
    for (int i = 0; i < cnt; ++i) {
        key.push_back((uintptr_t)side[i]);
        key.push_back((uintptr_t)d_in[i]);
        key.push_back((uintptr_t)d_out[i]);
    }
    auto it = n->uneven->plans.find(key);
    UPlan* P = nullptr;
    if (it == n->uneven->plans.end()) {
        net_status s = build_uplan(n, d_in, side, cnt, d_out, &P);
        if (s != NET_OK) return s;
        if (n->uneven->plans.size() >= 16) {
            for (auto& kv : n->uneven->plans) delete kv.second;
            n->uneven->plans.clear();
        }
        n->uneven->plans[key] = P;
    } else {
        P = it->second;
    }
    return enqueue_uplan_graph(n, P, cnt);
}

void dn::grouped_tiles(const Layer& L, int ncols, int* BN, int* mb, int* nst_cap) {
    if (L.grp_bn > 0 && L.grp_bn <= rup(ncols, 64)) *BN = L.grp_bn;
    if (L.pair)   // one N tile: the weights stay resident
        while (*BN < ncols && *BN < 256) *BN *= 2;
    *mb = (L.grp_mb == 2 && *BN <= 128) ? 2 : 1;
    *nst_cap = L.grp_nst;
}

void dn::uneven_plans_clear(net* n) {
    if (!n->uneven) return;
    for (auto& kv : n->uneven->plans) delete kv.second;
    n->uneven->plans.clear();
}

void dn::uneven_graphs_clear(net* n) {
    if (!n->uneven) return;
    for (auto& kv : n->uneven->plans)
        if (kv.second->graph) {
            cudaGraphExecDestroy(kv.second->graph);
            kv.second->graph = nullptr;
        }
}

void dn::uneven_free(net* n) {
    if (!n->uneven) return;
    for (auto& kv : n->uneven->plans) delete kv.second;
    for (int i = 0; i < 2; ++i)
        if (n->uneven->buf[i]) dn::dfree(n->uneven->buf[i]);
    delete n->uneven;
    n->uneven = nullptr;
}
