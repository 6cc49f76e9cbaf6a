// serve.cu — request queue with continuous (layer-step) batching.
//
// Frames arrive from many cameras through net_submit at any time.  A
// scheduler thread admits queued requests while the HBM activation budget
// allows (first come, first served), then repeats one step: every admitted
// request advances by one layer, and all requests that stand at the same
// layer share one grouped launch (one problem per request: its own
// activations, size and output).  A request that arrives while others are
// on the GPU joins at the next step; a request that finished its last layer
// is copied back and its memory returns to the budget.  The weights are the
// handle's resident weights; nothing is re-uploaded per request.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/net.h"
#include "common.cuh"
#include "kernels.h"
#include "net_internal.h"

using namespace dn;

namespace dn {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    int h = 0, w = 0;
    std::vector<float> frame;        // host copy of the submitted frame
    std::vector<float> result;       // host result once done
    int layer = -1;                  // next layer to run (-1: not admitted)
    size_t block = 0, block_bytes = 0;   // offset / size in the device arena
    std::vector<int> H, W;           // per-layer input size
    int cur = 0;                     // which half of the block holds the current input
    net_status status = NET_OK;
    bool done = false;
    Clock::time_point t_submit, t_done;
};

// First-fit allocator over one device arena (offsets only).
struct Arena {
    size_t size = 0;
    std::map<size_t, size_t> free_;  // offset -> bytes
    void init(size_t bytes) {
        size = bytes;
        free_.clear();
        free_[0] = bytes;
    }
    bool alloc(size_t bytes, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t o = it->first + bytes;
                free_.erase(it);
                if (rest) free_[o] = rest;
                return true;
            }
        return false;
    }
    void release(size_t off, size_t bytes) {
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct ServeState {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread th;
    bool stop = false;
    uint64_t next_id = 1;
    std::deque<std::shared_ptr<Request>> queue;            // submitted, not admitted
    std::vector<std::shared_ptr<Request>> active;          // on the device
    std::map<uint64_t, std::shared_ptr<Request>> all;      // until the result is taken
    // device
    void* arena = nullptr;
    Arena alloc;
    ConvProblem* d_tab = nullptr;     // per-step problem tables (device)
    ConvProblem* h_tab = nullptr;     // pinned staging
    int tab_cap = 0;
    PackJob* d_pack = nullptr;
    PackJob* h_pack = nullptr;
    PoolJob* d_pool = nullptr;
    PoolJob* h_pool = nullptr;
    float* h_out = nullptr;           // pinned result staging
    size_t h_out_floats = 0;
    float* h_in = nullptr;            // pinned frame staging
    size_t h_in_floats = 0;
    // statistics
    std::vector<double> lat_ms;
    Clock::time_point t_first, t_last;
    uint64_t completed = 0;
};

static size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device bytes one request needs: its float32 frame, then two halves that
// hold the input and output activation of the running layer.
static size_t request_bytes(const net* n, int h, int w, std::vector<int>& H, std::vector<int>& W,
                            size_t* half) {
    layer_dims(n, h, w, H, W);
    size_t mx = 0;
    for (size_t l = 0; l < n->L.size(); ++l)
        mx = std::max(mx, (size_t)H[l] * W[l] * n->L[l].in_cs * dt_size(n->L[l].in_dt));
    const size_t nl = n->L.size();   // the final NCHW float32 map lands in one half too
    mx = std::max(mx, (size_t)H[nl] * W[nl] * rup(n->L.back().d.cout, 4) * sizeof(float));
    *half = up256(mx);
    return up256((size_t)n->in_c * h * w * sizeof(float)) + 2 * *half;
}

static float in_scale_of(const Layer& L) { return L.in_dt == DT_FP8 ? (float)L.act_scale : 1.f; }

// One step: admitted-but-unpacked requests are packed, then every active
// request runs its current layer; requests at the same layer share a launch.
static net_status serve_step(net* n, ServeState* S, std::vector<std::shared_ptr<Request>>& act) {
    cudaStream_t st = n->stream;
    const int nl = (int)n->L.size();
    char* base = static_cast<char*>(S->arena);
    cudaError_t e = cudaSuccess;
    // pack the frames of newly admitted requests (grouped)
    int np = 0;
    long long ptotal = 0;
    const int V0 = 16 / (int)dt_size(n->L[0].in_dt);
    for (auto& r : act)
        if (r->layer == 0 && r->cur == -1) {
            const size_t fb = up256((size_t)n->in_c * r->h * r->w * sizeof(float));
            S->h_pack[np] = PackJob{reinterpret_cast<const float*>(base + r->block), base + r->block + fb, n->in_c,
                                    r->h, r->w, n->L[0].in_cs, n->L[0].im2col_k, ptotal};
            ptotal += (long long)r->h * r->w * (n->L[0].in_cs / V0);
            r->cur = 0;
            ++np;
        }
    if (np) {
        e = cudaMemcpyAsync(S->d_pack, S->h_pack, sizeof(PackJob) * np, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = pack_frames_grouped(S->d_pack, np, ptotal, n->L[0].in_dt, 1.f / in_scale_of(n->L[0]), st);
        if (e == cudaSuccess) ++n->launches;
    }
    // group by layer; every group gets its own slice of the staging tables
    int tab_used = 0, pool_used = 0;
    for (int l = 0; l < nl && e == cudaSuccess; ++l) {
        std::vector<Request*> grp;
        for (auto& r : act)
            if (r->layer == l) grp.push_back(r.get());
        if (grp.empty()) continue;
        const Layer& L = n->L[l];
        const bool last = l + 1 == nl;
        const bool pool2 = L.d.pool == NET_POOL_2X2S2;
        const int out_cs = last ? L.d.cout : n->L[l + 1].in_cs;
        const int ncols = std::max(L.d.cout, out_cs);
        Epilogue ep{};
        ep.bias = L.bias;
        ep.alpha = L.in_dt == DT_FP8 ? L.alpha : nullptr;
        ep.act = L.d.act;
        ep.pool = pool2 ? POOL_S2 : POOL_NONE;
        ep.cout = L.d.cout;
        ep.out_layout = last ? LAYOUT_NCHW : LAYOUT_NHWC;
        ep.out_dt = last ? DT_F32 : n->L[l + 1].in_dt;
        ep.out_cs = out_cs;
        ep.out_inv_scale = (!last && ep.out_dt == DT_FP8) ? 1.f / in_scale_of(n->L[l + 1]) : 1.f;
        auto half_ptr = [&](Request* r, int which) {
            const size_t fb = up256((size_t)n->in_c * r->h * r->w * sizeof(float));
            return base + r->block + fb + (size_t)which * ((r->block_bytes - fb) / 2);
        };
        // the last layer writes NCHW float32 into the first half's space
        if (L.engine == ENG_SIMT) {
            for (Request* r : grp) {
                ConvLaunch c{};
                c.x = half_ptr(r, r->cur);
                c.w = L.w;
                c.y = half_ptr(r, r->cur ^ 1);
                c.n = 1;
                c.H = r->H[l];
                c.W = r->W[l];
                c.Cp = L.in_cs;
                c.k = L.d.k;
                c.w_rows = L.w_rows;
                c.ep = ep;
                c.ksplit = 1;
                e = conv_simt(c, st);
                ++n->launches;
                if (e != cudaSuccess) break;
            }
        } else {
            int TW = 16, TH = 8, BN = 128, ks = 1;
            {
                static const int tws[5] = {16, 8, 32, 64, 128};
                long best = -1;
                for (int i = 0; i < 5; ++i) {
                    const int tw = tws[i], th = 128 / tw;
                    if (pool2 && tw > 16) continue;
                    long cover = 0;
                    for (Request* r : grp) cover += (long)cdiv(r->H[l], th) * th * cdiv(r->W[l], tw) * tw;
                    if (best < 0 || cover < best) {
                        best = cover;
                        TW = tw;
                        TH = th;
                    }
                }
            }
            if (tab_used + (int)grp.size() > S->tab_cap) return fail(NET_E_STATE, "problem table full");
            ConvProblem* ht = S->h_tab + tab_used;
            int mt = 0;
            for (size_t i = 0; i < grp.size(); ++i) {
                Request* r = grp[i];
                ConvProblem& q = ht[i];
                std::memset(&q, 0, sizeof q);
                e = tc_encode_act(&q.tmA, half_ptr(r, r->cur), L.in_dt, 1, r->H[l], r->W[l], L.in_cs, TW, TH);
                if (e != cudaSuccess) return fail(NET_E_CUDA, "serve: tensor map");
                q.y = half_ptr(r, r->cur ^ 1);
                q.n = 1;
                q.H = r->H[l];
                q.W = r->W[l];
                q.tiles_x = cdiv(q.W, TW);
                q.tiles_y = cdiv(q.H, TH);
                q.tile_begin = mt;
                mt += q.tiles_x * q.tiles_y;
            }
            const int nk = L.kx * L.kx * (L.in_cs / (tc_chunk_bytes(L.in_cs, L.in_dt) / (int)dt_size(L.in_dt)));
            tc_choose_split(mt, ncols, nk, n->num_sms, &BN, &ks, 1);
            e = cudaMemcpyAsync(S->d_tab + tab_used, ht, sizeof(ConvProblem) * grp.size(), cudaMemcpyHostToDevice, st);
            TcArgs a{};
            a.probs = S->d_tab + tab_used;
            a.nprob = (int)grp.size();
            a.m_tiles = mt;
            a.n_tiles = cdiv(ncols, BN);
            a.Cp = L.in_cs;
            a.k = L.kx;
            a.TW = TW;
            a.TH = TH;
            a.chb = tc_chunk_bytes(L.in_cs, L.in_dt);
            a.cpc = a.chb / (int)dt_size(L.in_dt);
            a.chunks = L.in_cs / a.cpc;
            a.ksplit = 1;
            a.ep = ep;
            a.err = n->err_dev;
            int cs = 1, workers = 1;
            tc_workers(mt, a.n_tiles, 1, BN, n->num_sms, &cs, &workers);
            if (e == cudaSuccess) e = conv_tc_launch(L.tmB[tmb_index(BN, cs)], a, BN, L.in_dt, workers, cs, st);
            ++n->launches;
            tab_used += (int)grp.size();
        }
        if (e != cudaSuccess) break;
        if (L.d.pool == NET_POOL_2X2S1_SAME && !last) {
            // staging slots of this step are not reused before the step's
            // closing synchronisation
            if (pool_used + (int)grp.size() > S->tab_cap) return fail(NET_E_STATE, "pool table full");
            PoolJob* hp = S->h_pool + pool_used;
            int npl = 0;
            long long total = 0;
            const int V = 16 / (int)dt_size(n->L[l + 1].in_dt);
            for (Request* r : grp) {
                hp[npl++] = PoolJob{half_ptr(r, r->cur ^ 1), half_ptr(r, r->cur), r->H[l + 1], r->W[l + 1], total};
                total += (long long)r->H[l + 1] * r->W[l + 1] * (n->L[l + 1].in_cs / V);
            }
            e = cudaMemcpyAsync(S->d_pool + pool_used, hp, sizeof(PoolJob) * npl, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess)
                e = maxpool_s1_grouped(S->d_pool + pool_used, npl, total, n->L[l + 1].in_cs, n->L[l + 1].in_dt, st);
            pool_used += npl;
            ++n->launches;
            // the pooled activation is back in the current half
        } else {
            for (Request* r : grp) r->cur ^= 1;
        }
        if (e != cudaSuccess) break;
        for (Request* r : grp) r->layer = l + 1;
    }
    if (e != cudaSuccess) return fail(NET_E_CUDA, "serve step: %s", cudaGetErrorString(e));
    return NET_OK;
}

static void serve_loop(net* n) {
    ServeState* S = n->serve;
    cudaSetDevice(n->device);
    // Host-side fault injection for tests: a slow step (microseconds).
    const char* slow = getenv("NET_SERVE_STEP_DELAY_US");
    const long delay_us = slow ? atol(slow) : 0;
    while (true) {
        std::vector<std::shared_ptr<Request>> act;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty() || !S->active.empty(); });
            if (S->stop) return;
            // admission: FIFO while the activation budget has room
            while (!S->queue.empty()) {
                auto r = S->queue.front();
                size_t off;
                if (!S->alloc.alloc(r->block_bytes, &off)) break;
                r->block = off;
                r->layer = 0;
                r->cur = -1;   // frame not packed yet
                S->queue.pop_front();
                S->active.push_back(r);
            }
            act = S->active;
        }
        net_status s = NET_OK;
        // upload the frames of newly admitted requests
        for (auto& r : act)
            if (r->cur == -1 && s == NET_OK) {
                const size_t fl = r->frame.size();
                std::memcpy(S->h_in, r->frame.data(), fl * sizeof(float));
                cudaError_t e = cudaMemcpyAsync(static_cast<char*>(S->arena) + r->block, S->h_in, fl * sizeof(float),
                                                cudaMemcpyHostToDevice, n->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);   // staging is reused
                if (e != cudaSuccess) s = fail(NET_E_CUDA, "serve H2D: %s", cudaGetErrorString(e));
            }
        if (delay_us > 0) std::this_thread::sleep_for(std::chrono::microseconds(delay_us));
        if (s == NET_OK) s = serve_step(n, S, act);
        if (s == NET_OK && cudaStreamSynchronize(n->stream) != cudaSuccess) s = NET_E_CUDA;
        if (s == NET_OK && n->err_host && *(volatile int*)n->err_host) s = NET_E_DEVICE_WAIT;
        // completions: results back to the host, memory back to the budget
        std::vector<std::shared_ptr<Request>> fin;
        for (auto& r : act)
            if (r->layer == (int)n->L.size() || s != NET_OK) fin.push_back(r);
        for (auto& r : fin) {
            if (s == NET_OK) {
                int c, ho, wo;
                net_output_shape(n, r->h, r->w, &c, &ho, &wo);
                const size_t fl = (size_t)c * ho * wo;
                const size_t fb = up256((size_t)n->in_c * r->h * r->w * sizeof(float));
                const size_t halfb = (r->block_bytes - fb) / 2;
                const char* src = static_cast<char*>(S->arena) + r->block + fb + (size_t)r->cur * halfb;
                cudaError_t e = cudaMemcpy(S->h_out, src, fl * sizeof(float), cudaMemcpyDeviceToHost);
                r->result.assign(S->h_out, S->h_out + fl);
                r->status = e == cudaSuccess ? NET_OK : NET_E_CUDA;
            } else {
                r->status = s;
            }
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            const auto now = Clock::now();
            for (auto& r : fin) {
                r->done = true;
                r->t_done = now;
                r->frame.clear();
                r->frame.shrink_to_fit();
                S->alloc.release(r->block, r->block_bytes);
                S->active.erase(std::find(S->active.begin(), S->active.end(), r));
                if (r->status == NET_OK) {
                    S->lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
                    if (S->completed == 0) S->t_first = r->t_submit;
                    S->t_last = now;
                    ++S->completed;
                }
            }
        }
        if (!fin.empty()) S->cv_done.notify_all();
    }
}

static net_status serve_start(net* n) {
    if (n->serve) return NET_OK;
    if (!n->weights_loaded) return fail(NET_E_WEIGHTS, "weights not loaded");
    std::unique_ptr<ServeState> S(new ServeState());
    cudaError_t e = cudaSetDevice(n->device);
    size_t freeb = 0, totalb = 0;
    if (e == cudaSuccess) e = cudaMemGetInfo(&freeb, &totalb);
    if (e != cudaSuccess) return fail(NET_E_CUDA, "serve start: %s", cudaGetErrorString(e));
    const size_t arena = std::min(n->budget, freeb / 2);
    if ((e = cudaMalloc(&S->arena, arena)) != cudaSuccess)
        return fail(NET_E_OOM, "serving arena %zu bytes: %s", arena, cudaGetErrorString(e));
    S->alloc.init(arena);
    S->tab_cap = 1024;
    std::vector<int> H, W;
    int c, ho, wo;
    net_output_shape(n, n->max_side, n->max_side, &c, &ho, &wo);
    S->h_out_floats = (size_t)c * ho * wo;
    S->h_in_floats = (size_t)n->in_c * n->max_side * n->max_side;
    if ((e = cudaMalloc(&S->d_tab, sizeof(ConvProblem) * S->tab_cap)) == cudaSuccess &&
        (e = cudaMallocHost(&S->h_tab, sizeof(ConvProblem) * S->tab_cap)) == cudaSuccess &&
        (e = cudaMalloc(&S->d_pack, sizeof(PackJob) * S->tab_cap)) == cudaSuccess &&
        (e = cudaMallocHost(&S->h_pack, sizeof(PackJob) * S->tab_cap)) == cudaSuccess &&
        (e = cudaMalloc(&S->d_pool, sizeof(PoolJob) * S->tab_cap)) == cudaSuccess &&
        (e = cudaMallocHost(&S->h_pool, sizeof(PoolJob) * S->tab_cap)) == cudaSuccess &&
        (e = cudaMallocHost(&S->h_out, S->h_out_floats * sizeof(float))) == cudaSuccess &&
        (e = cudaMallocHost(&S->h_in, S->h_in_floats * sizeof(float))) == cudaSuccess) {
    }
    if (e != cudaSuccess) return fail(NET_E_OOM, "serving staging: %s", cudaGetErrorString(e));
    n->serve = S.release();
    n->serve->th = std::thread(serve_loop, n);
    return NET_OK;
}

void serve_stop(net* n) {
    ServeState* S = n->serve;
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    cudaFree(S->arena);
    cudaFree(S->d_tab);
    cudaFreeHost(S->h_tab);
    cudaFree(S->d_pack);
    cudaFreeHost(S->h_pack);
    cudaFree(S->d_pool);
    cudaFreeHost(S->h_pool);
    cudaFreeHost(S->h_out);
    cudaFreeHost(S->h_in);
    delete S;
    n->serve = nullptr;
}

}  // namespace dn

extern "C" net_status net_submit(net_t* n, const float* frame, int h, int w, uint64_t* req_id) {
    if (!n || !frame || !req_id) return fail(NET_E_INVAL, "NULL argument");
    net_status s = check_shape(n, 1, h, w);
    if (s != NET_OK) return s;
    if (!n->serve) {
        s = serve_start(n);
        if (s != NET_OK) return s;
    }
    ServeState* S = n->serve;
    auto r = std::make_shared<Request>();
    r->h = h;
    r->w = w;
    size_t half;
    r->block_bytes = request_bytes(n, h, w, r->H, r->W, &half);
    if (r->block_bytes > S->alloc.size)
        return fail(NET_E_BUDGET, "frame %dx%d needs %zu bytes, budget %zu", h, w, r->block_bytes, S->alloc.size);
    r->frame.assign(frame, frame + (size_t)n->in_c * h * w);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r->id = S->next_id++;
        S->all[r->id] = r;
        S->queue.push_back(r);
    }
    S->cv_work.notify_one();
    *req_id = r->id;
    return NET_OK;
}

static net_status take_result(ServeState* S, uint64_t id, float* out, size_t cap, bool* done) {
    auto it = S->all.find(id);
    if (it == S->all.end()) return fail(NET_E_INVAL, "unknown request %llu", (unsigned long long)id);
    auto r = it->second;
    *done = r->done;
    if (!r->done) return NET_OK;
    if (r->status != NET_OK) {
        S->all.erase(it);
        return fail(r->status, "request %llu failed", (unsigned long long)id);
    }
    if (cap < r->result.size()) return fail(NET_E_INVAL, "output capacity %zu < %zu", cap, r->result.size());
    std::memcpy(out, r->result.data(), r->result.size() * sizeof(float));
    S->all.erase(it);
    return NET_OK;
}

extern "C" net_status net_poll(net_t* n, uint64_t id, float* out, size_t cap, int* done) {
    if (!n || !out || !done) return fail(NET_E_INVAL, "NULL argument");
    if (!n->serve) return fail(NET_E_STATE, "no request submitted");
    std::lock_guard<std::mutex> lk(n->serve->mu);
    bool d = false;
    net_status s = take_result(n->serve, id, out, cap, &d);
    *done = d ? 1 : 0;
    return s;
}

extern "C" net_status net_wait(net_t* n, uint64_t id, float* out, size_t cap, int timeout_ms) {
    if (!n || !out) return fail(NET_E_INVAL, "NULL argument");
    if (!n->serve) return fail(NET_E_STATE, "no request submitted");
    ServeState* S = n->serve;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return fail(NET_E_INVAL, "unknown request %llu", (unsigned long long)id);
    auto r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_ms < 0) S->cv_done.wait(lk, ready);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return fail(NET_E_TIMEOUT, "request %llu not done after %d ms", (unsigned long long)id, timeout_ms);
    bool d = false;
    return take_result(S, id, out, cap, &d);
}

extern "C" net_status net_stats(net_t* n, double* fps, double* p50, double* p99) {
    if (!n || !fps || !p50 || !p99) return fail(NET_E_INVAL, "NULL argument");
    *fps = *p50 = *p99 = 0.0;
    if (!n->serve) return NET_OK;
    std::lock_guard<std::mutex> lk(n->serve->mu);
    ServeState* S = n->serve;
    if (S->completed == 0) return NET_OK;
    const double span = std::chrono::duration<double>(S->t_last - S->t_first).count();
    *fps = span > 0 ? S->completed / span : 0.0;
    std::vector<double> v = S->lat_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
    *p50 = pct(0.50);
    *p99 = pct(0.99);
    return NET_OK;
}

extern "C" net_status net_stats_reset(net_t* n) {
    if (!n) return fail(NET_E_INVAL, "NULL argument");
    if (!n->serve) return NET_OK;
    std::lock_guard<std::mutex> lk(n->serve->mu);
    n->serve->lat_ms.clear();
    n->serve->completed = 0;
    return NET_OK;
}
