// serve.cu — request queue with continuous batching.
//
// Frames arrive from many cameras through net_submit at any time.  A
// scheduler thread admits queued requests while the in-flight cap and the
// HBM activation budget allow (first come, first served) and enqueues them
// as one step: every layer runs as one grouped launch over all the step's
// requests (one problem per request: its own activations, size and output).
// Steps are pipelined two deep on three streams (upload, compute, download):
// requests that arrive while a step is on the GPU are admitted into the next
// step, whose frames upload while the first step computes, and whose kernels
// start as soon as the first step's last kernel ends.  A finished request's
// result is copied back and its memory returns to the budget.  The weights
// are the handle's resident weights; nothing is re-uploaded per request.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <string>
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

// Host copies of frames and results split over a few persistent threads.
// A request's frame is copied into the pinned arena inside net_submit, on
// the request's latency path: one thread copies a 416 x 416 frame (2.1 MB)
// in ~0.13 ms and a 608 x 608 one (4.4 MB) in ~0.3 ms, a third to half of a
// lone request's latency.  Copies below kMinSplit bytes stay on the calling
// thread; larger ones are cut into chunks of at least kMinChunk bytes, the
// caller copying one and then helping with any queued chunk until its own
// are done.  Several callers may copy at once.
class CopyPool {
public:
    void start(int workers) {
        for (int i = 0; i < workers; ++i) th_.emplace_back([this] { run(); });
    }
    void stop() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            quit_ = true;
        }
        cv_.notify_all();
        for (auto& t : th_) t.join();
        th_.clear();
    }
    void copy(void* dst, const void* src, size_t bytes) {
        const size_t parts = th_.empty() || bytes < kMinSplit
                                 ? 1
                                 : std::min<size_t>(th_.size() + 1, bytes / kMinChunk);
        if (parts <= 1) {
            std::memcpy(dst, src, bytes);
            return;
        }
        const size_t step = ((bytes + parts - 1) / parts + 63) & ~(size_t)63;
        std::atomic<int> left{0};
        {
            std::lock_guard<std::mutex> lk(mu_);
            for (size_t o = step; o < bytes; o += step) {
                q_.push_back(Task{static_cast<char*>(dst) + o, static_cast<const char*>(src) + o,
                                  std::min(step, bytes - o), &left});
                left.fetch_add(1, std::memory_order_relaxed);
            }
        }
        cv_.notify_all();
        std::memcpy(dst, src, std::min(step, bytes));
        while (left.load(std::memory_order_acquire) > 0) {
            Task t;
            if (pop(&t)) do_task(t);
            else std::this_thread::yield();
        }
    }

private:
    static constexpr size_t kMinSplit = 512 << 10, kMinChunk = 256 << 10;
    struct Task {
        char* d;
        const char* s;
        size_t n;
        std::atomic<int>* left;
    };
    bool pop(Task* t) {
        std::lock_guard<std::mutex> lk(mu_);
        if (q_.empty()) return false;
        *t = q_.front();
        q_.pop_front();
        return true;
    }
    static void do_task(const Task& t) {
        std::memcpy(t.d, t.s, t.n);
        t.left->fetch_sub(1, std::memory_order_acq_rel);
    }
    void run() {
        while (true) {
            Task t;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [this] { return quit_ || !q_.empty(); });
                if (q_.empty()) return;   // quit with nothing queued
                t = q_.front();
                q_.pop_front();
            }
            do_task(t);
        }
    }
    std::mutex mu_;
    std::condition_variable cv_;
    std::deque<Task> q_;
    std::vector<std::thread> th_;
    bool quit_ = false;
};

struct Request {
    uint64_t id = 0;
    int h = 0, w = 0;
    std::vector<float> frame;        // host copy of the submitted frame
    std::vector<float> result;       // host result once done
    int layer = -1;                  // next layer to run (-1: not admitted)
    size_t block = 0, block_bytes = 0;   // offset / size in the device arena
    std::vector<int> H, W;           // per-layer input size
    int cur = 0;                     // which half of the block holds the current input
    std::vector<ConvProblem> probs;  // per layer: tensor map and output of this request (built at admission)
    size_t stage_off = 0;            // pinned staging offset of the frame (admission step)
    // pinned host arena chunks: the submitted frame (copied by net_submit)
    // and the result (copied out by net_poll / net_wait); npos = not used
    size_t pin_off = std::string::npos, pin_bytes = 0;
    size_t res_off = std::string::npos, res_bytes = 0, res_floats = 0;
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

// Steps in flight: the host admits and enqueues one step while the GPU runs
// the one before it.
constexpr int kSlots = 2;

// The staging of one step, reused only after that step has finished.
struct StepSlot {
    char* h_stage = nullptr;          // pinned: the step's pack jobs, problem tables and pool jobs
    char* d_stage = nullptr;          // their device copy (one copy per step)
    float* h_in = nullptr;            // pinned frame staging for admissions without a pinned chunk
    float* h_out = nullptr;           // pinned result staging for completions without one
    cudaEvent_t ev_in = nullptr, ev_comp = nullptr, ev_done = nullptr;
    bool busy = false;
    net_status status = NET_OK;
    std::vector<std::shared_ptr<Request>> reqs;   // admitted by the step; all finish in it
    std::vector<size_t> out_off;                  // per request: h_out offset, npos = pinned chunk
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
    cudaStream_t s_in = nullptr, s_out = nullptr;   // uploads / downloads beside the compute stream
    StepSlot slot[kSlots];
    size_t stage_bytes = 0;
    size_t h_out_floats = 0, h_in_floats = 0;   // per slot
    int max_active = 128;             // requests on the device at once
    char* hpin = nullptr;             // pinned host arena for frames and results
    Arena hpin_alloc;
    // statistics
    std::vector<double> lat_ms;
    Clock::time_point t_first, t_last;
    uint64_t completed = 0;
    uint64_t steps = 0;
    CopyPool copies;                  // frame copy-in (net_submit) and result copy-out
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

// Serving tile: one shape for every layer of every request (pooled layers
// need TW = 16 or 8), so a request's tensor maps are built once.
constexpr int kServeTW = 16, kServeTH = 8;

static size_t frame_bytes(const net* n, const Request* r) {
    return up256((size_t)n->in_c * r->h * r->w * sizeof(float));
}

static char* half_ptr(const net* n, ServeState* S, const Request* r, int which) {
    const size_t fb = frame_bytes(n, r);
    return static_cast<char*>(S->arena) + r->block + fb + (size_t)which * ((r->block_bytes - fb) / 2);
}

// Builds the per-layer problems of an admitted request (its buffers are fixed
// for its lifetime).  The ping-pong half that holds each layer's input
// follows the same rule as the step: it flips after every layer except a
// stride-1 pool layer.
static net_status build_request_problems(net* n, ServeState* S, Request* r) {
    const int nl = (int)n->L.size();
    r->probs.assign(nl, ConvProblem{});
    int cur = 0;
    for (int l = 0; l < nl; ++l) {
        const Layer& L = n->L[l];
        ConvProblem& q = r->probs[l];
        std::memset(&q, 0, sizeof q);
        if (L.engine == ENG_TC) {
            // pair mode (tap-merged stages): boxes of TH + 2 rows
            cudaError_t e = tc_encode_act(&q.tmA, half_ptr(n, S, r, cur), L.in_dt, 1, r->H[l], r->W[l], L.in_cs,
                                          kServeTW, L.pair ? kServeTH + 2 : kServeTH);
            if (e != cudaSuccess) return fail(NET_E_CUDA, "serve: tensor map");
        }
        q.x = half_ptr(n, S, r, cur);
        q.y = half_ptr(n, S, r, cur ^ 1);
        q.n = 1;
        q.H = r->H[l];
        q.W = r->W[l];
        q.tiles_x = cdiv(q.W, kServeTW);
        q.tiles_y = cdiv(q.H, kServeTH);
        tc_problem_divisors(q);
        if (L.d.pool != NET_POOL_2X2S1_SAME) cur ^= 1;
    }
    return NET_OK;
}

// Releases what serve_start allocated (any part may be missing).
static void serve_free(ServeState* S) {
    S->copies.stop();
    if (S->arena) dn::dfree(S->arena);
    for (StepSlot& sl : S->slot) {
        if (sl.h_stage) cudaFreeHost(sl.h_stage);
        if (sl.d_stage) dn::dfree(sl.d_stage);
        if (sl.h_in) cudaFreeHost(sl.h_in);
        if (sl.h_out) cudaFreeHost(sl.h_out);
        if (sl.ev_in) cudaEventDestroy(sl.ev_in);
        if (sl.ev_comp) cudaEventDestroy(sl.ev_comp);
        if (sl.ev_done) cudaEventDestroy(sl.ev_done);
        sl = StepSlot{};
    }
    if (S->s_in) cudaStreamDestroy(S->s_in);
    if (S->s_out) cudaStreamDestroy(S->s_out);
    if (S->hpin) cudaFreeHost(S->hpin);
    S->arena = nullptr;
    S->s_in = S->s_out = nullptr;
    S->hpin = nullptr;
}

// Enqueues one step without waiting for it.  The upload stream carries the
// admitted frames and the step's tables (one copy); the compute stream packs
// the frames and runs every layer as one grouped launch over all the step's
// requests (one problem per request: its own activations and size); the
// download stream copies each result back.  ev_done closes the step.
static net_status enqueue_step(net* n, ServeState* S, StepSlot& sl) {
    cudaStream_t st = n->stream;
    const int nl = (int)n->L.size();
    char* base = static_cast<char*>(S->arena);
    const auto& reqs = sl.reqs;
    const int na = (int)reqs.size();
    cudaError_t e = cudaSuccess;
#define SERVE_CK(x, what)                                                         \
    do {                                                                          \
        if ((e = (x)) != cudaSuccess)                                             \
            return fail(NET_E_CUDA, "serve %s: %s", what, cudaGetErrorString(e)); \
    } while (0)
    // frames: from the pinned chunk net_submit filled, else via the slot's staging
    size_t staged = 0;
    for (const auto& r : reqs) {
        net_status s = build_request_problems(n, S, r.get());
        if (s != NET_OK) return s;
        const size_t fbytes = (size_t)n->in_c * r->h * r->w * sizeof(float);
        const void* src = nullptr;
        if (r->pin_off != std::string::npos) {
            src = S->hpin + r->pin_off;
        } else {
            std::memcpy(sl.h_in + staged, r->frame.data(), fbytes);
            src = sl.h_in + staged;
            staged += r->frame.size();
        }
        SERVE_CK(cudaMemcpyAsync(base + r->block, src, fbytes, cudaMemcpyHostToDevice, S->s_in), "H2D");
    }
    // tables, packed into one block: pack jobs | problems (layer-major) | pool jobs
    int ntc = 0;
    for (const Layer& L : n->L) ntc += L.engine == ENG_TC;
    const size_t off_tab = up256((size_t)na * sizeof(PackJob));
    const size_t off_pool = off_tab + (size_t)na * ntc * sizeof(ConvProblem);
    PackJob* hk = reinterpret_cast<PackJob*>(sl.h_stage);
    ConvProblem* ht = reinterpret_cast<ConvProblem*>(sl.h_stage + off_tab);
    PoolJob* hpj = reinterpret_cast<PoolJob*>(sl.h_stage + off_pool);
    ConvProblem* dt = reinterpret_cast<ConvProblem*>(sl.d_stage + off_tab);
    PoolJob* dpj = reinterpret_cast<PoolJob*>(sl.d_stage + off_pool);
    long long ptotal = 0;
    const int V0 = 16 / (int)dt_size(n->L[0].in_dt);
    for (int i = 0; i < na; ++i) {
        Request* r = reqs[i].get();
        const size_t fb = up256((size_t)n->in_c * r->h * r->w * sizeof(float));
        hk[i] = PackJob{reinterpret_cast<const float*>(base + r->block), base + r->block + fb, n->in_c, r->h, r->w,
                        n->L[0].in_cs, n->L[0].im2col_k, ptotal};
        ptotal += (long long)r->h * r->w * (n->L[0].im2col_k ? 1 : n->L[0].in_cs / V0);
        r->cur = 0;
    }
    struct LayerStep {
        int l = 0;
        TcArgs a{};
        int BN = 0, workers = 1, mb = 1;
        size_t simt_begin = 0, simt_end = 0;
        int pool_begin = 0, npool = 0;
        long long pool_total = 0;
    };
    std::vector<LayerStep> plan(nl);
    std::vector<ConvLaunch> simt;
    int ntab = 0, npool = 0;
    auto hp = [&](Request* r, int which) { return half_ptr(n, S, r, which); };
    for (int l = 0; l < nl; ++l) {
        const Layer& L = n->L[l];
        LayerStep& P = plan[l];
        P.l = l;
        const bool last = l + 1 == nl;
        const int out_cs = last ? L.d.cout : n->L[l + 1].in_cs;
        const int ncols = std::max(L.d.cout, out_cs);
        Epilogue ep{};
        ep.bias = L.bias;
        ep.alpha = L.in_dt == DT_FP8 ? L.alpha : nullptr;
        ep.act = L.d.act;
        ep.pool = L.d.pool == NET_POOL_2X2S2 ? POOL_S2 : POOL_NONE;
        ep.cout = L.d.cout;
        ep.out_layout = last ? LAYOUT_NCHW : LAYOUT_NHWC;   // the last layer writes NCHW float32
        ep.out_dt = last ? DT_F32 : n->L[l + 1].in_dt;
        ep.out_cs = out_cs;
        ep.out_inv_scale = (!last && ep.out_dt == DT_FP8) ? 1.f / in_scale_of(n->L[l + 1]) : 1.f;
        if (L.engine == ENG_SIMT) {
            P.simt_begin = simt.size();
            for (const auto& rp : reqs) {
                Request* r = rp.get();
                ConvLaunch c{};
                c.x = hp(r, r->cur);
                c.w = L.w;
                c.y = hp(r, r->cur ^ 1);
                c.n = 1;
                c.H = r->H[l];
                c.W = r->W[l];
                c.Cp = L.in_cs;
                c.k = L.d.k;
                c.w_rows = L.w_rows;
                c.ep = ep;
                c.ksplit = 1;
                simt.push_back(c);
            }
            P.simt_end = simt.size();
        } else {
            // each request's tensor maps for this layer were built with the
            // serving tile (16 x 8 pixels) when it was admitted
            int mt = 0;
            for (int i = 0; i < na; ++i) {
                ConvProblem& q = ht[ntab + i];
                q = reqs[i]->probs[l];
                q.tile_begin = mt;
                mt += q.tiles_x * q.tiles_y;
            }
            const int nk = L.kx * L.kx * (L.in_cs / (tc_chunk_bytes(L.in_cs, L.in_dt) / (int)dt_size(L.in_dt)));
            int BN = 128, ks = 1;
            tc_choose_split(mt, ncols, nk, n->num_sms, &BN, &ks, 1);
            int mb_req = 1, nst_cap = 0;
            grouped_tiles(L, ncols, &BN, &mb_req, &nst_cap);
            TcArgs& a = P.a;
            a.probs = dt + ntab;
            a.nprob = na;
            a.m_tiles = mt;
            a.n_tiles = cdiv(ncols, BN);
            a.Cp = L.in_cs;
            a.k = L.kx;
            a.TW = kServeTW;
            a.TH = kServeTH;
            a.chb = tc_chunk_bytes(L.in_cs, L.in_dt);
            a.cpc = a.chb / (int)dt_size(L.in_dt);
            a.chunks = L.in_cs / a.cpc;
            a.ksplit = 1;
            a.ep = ep;
            a.err = n->err_dev;
            P.BN = BN;
            a.nst_cap = nst_cap;
            tc_workers(mt, a.n_tiles, 1, BN, nk, a.chb, n->num_sms, mb_req, &P.workers, &a.bres, &P.mb);
            // pair mode needs resident weights (the launch refuses it otherwise)
            a.tapm = L.pair ? 1 : 0;
            a.pair = L.pair ? 1 : 0;
            ntab += na;
        }
        if (L.d.pool == NET_POOL_2X2S1_SAME && !last) {
            // the pooled activation goes back into the layer's input half
            const int V = 16 / (int)dt_size(n->L[l + 1].in_dt);
            P.pool_begin = npool;
            for (const auto& rp : reqs) {
                Request* r = rp.get();
                hpj[npool++] = PoolJob{hp(r, r->cur ^ 1), hp(r, r->cur), r->H[l + 1], r->W[l + 1], P.pool_total};
                P.pool_total += (long long)r->H[l + 1] * r->W[l + 1] * (n->L[l + 1].in_cs / V);
            }
            P.npool = npool - P.pool_begin;
        } else {
            for (const auto& rp : reqs) rp->cur ^= 1;
        }
        for (const auto& rp : reqs) rp->layer = l + 1;
    }
    SERVE_CK(cudaMemcpyAsync(sl.d_stage, sl.h_stage, off_pool + (size_t)npool * sizeof(PoolJob), cudaMemcpyHostToDevice,
                             S->s_in),
             "tables");
    SERVE_CK(cudaEventRecord(sl.ev_in, S->s_in), "event");
    SERVE_CK(cudaStreamWaitEvent(st, sl.ev_in, 0), "event wait");
    SERVE_CK(pack_frames_grouped(reinterpret_cast<const PackJob*>(sl.d_stage), na, ptotal, n->L[0].in_dt,
                                 1.f / in_scale_of(n->L[0]), st),
             "pack");
    ++n->launches;
    for (const LayerStep& P : plan) {
        const Layer& L = n->L[P.l];
        if (L.engine == ENG_SIMT) {
            for (size_t j = P.simt_begin; j < P.simt_end; ++j) {
                SERVE_CK(conv_simt(simt[j], st), "conv");
                ++n->launches;
            }
        } else {
            SERVE_CK(conv_tc_launch(L.tmB[tmb_index(P.BN)], P.a, P.BN, L.in_dt, P.workers, P.mb, 1, st), "conv");
            ++n->launches;
        }
        if (P.npool) {
            SERVE_CK(maxpool_s1_grouped(dpj + P.pool_begin, P.npool, P.pool_total, n->L[P.l + 1].in_cs,
                                        n->L[P.l + 1].in_dt, st),
                     "pool");
            ++n->launches;
        }
    }
    SERVE_CK(cudaEventRecord(sl.ev_comp, st), "event");
    SERVE_CK(cudaStreamWaitEvent(S->s_out, sl.ev_comp, 0), "event wait");
    for (int i = 0; i < na; ++i) {
        Request* r = reqs[i].get();
        float* dst = r->res_off != std::string::npos ? reinterpret_cast<float*>(S->hpin + r->res_off)
                                                      : sl.h_out + sl.out_off[i];
        SERVE_CK(cudaMemcpyAsync(dst, hp(r, r->cur), r->res_floats * sizeof(float), cudaMemcpyDeviceToHost, S->s_out),
                 "D2H");
    }
    SERVE_CK(cudaEventRecord(sl.ev_done, S->s_out), "event");
#undef SERVE_CK
    return NET_OK;
}

// Waits for a step and hands its results over: the requests are marked done
// (failed with the step's status if it failed) and their device memory and
// frame chunks go back to the pools.
static void complete_step(net* n, ServeState* S, StepSlot& sl) {
    net_status s = sl.status;
    if (s == NET_OK) {
        const cudaError_t e = cudaEventSynchronize(sl.ev_done);
        if (e != cudaSuccess) s = fail(NET_E_CUDA, "serve step: %s", cudaGetErrorString(e));
    } else {
        // a step that failed while being enqueued: let what was enqueued drain
        cudaStreamSynchronize(S->s_in);
        cudaStreamSynchronize(n->stream);
        cudaStreamSynchronize(S->s_out);
    }
    if (s == NET_OK) s = check_device_error(n);
    for (size_t i = 0; i < sl.reqs.size(); ++i) {
        Request* r = sl.reqs[i].get();
        r->status = s;
        if (s == NET_OK && r->res_off == std::string::npos)
            r->result.assign(sl.h_out + sl.out_off[i], sl.h_out + sl.out_off[i] + r->res_floats);
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        const auto now = Clock::now();
        for (auto& r : sl.reqs) {
            if (r->pin_off != std::string::npos) {
                S->hpin_alloc.release(r->pin_off, r->pin_bytes);
                r->pin_off = std::string::npos;
            }
            if (r->status != NET_OK && r->res_off != std::string::npos) {
                S->hpin_alloc.release(r->res_off, r->res_bytes);
                r->res_off = std::string::npos;
            }
            r->done = true;
            r->t_done = now;
            r->frame.clear();
            r->frame.shrink_to_fit();
            r->probs.clear();
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
    sl.reqs.clear();
    sl.out_off.clear();
    sl.busy = false;
    sl.status = NET_OK;
    S->cv_done.notify_all();
}

// Admits queued requests into a free slot, first come first served, while
// the in-flight cap, the slot's pinned staging, the result space and the
// activation budget all have room.  Called with S->mu held.
static void admit(net* n, ServeState* S, StepSlot& sl) {
    size_t staged = 0, outs = 0;
    while (!S->queue.empty() && (int)S->active.size() < S->max_active) {
        auto r = S->queue.front();
        const size_t fl = r->pin_off != std::string::npos ? 0 : r->frame.size();
        if (staged + fl > S->h_in_floats) break;
        int c, ho, wo;
        net_output_shape(n, r->h, r->w, &c, &ho, &wo);
        const size_t rf = (size_t)c * ho * wo;
        size_t roff = std::string::npos, ooff = std::string::npos;
        if (S->hpin && S->hpin_alloc.alloc(up256(rf * sizeof(float)), &roff)) {
        } else if (outs + rf <= S->h_out_floats) {
            ooff = outs;
        } else {
            break;
        }
        size_t off;
        if (!S->alloc.alloc(r->block_bytes, &off)) {
            if (roff != std::string::npos) S->hpin_alloc.release(roff, up256(rf * sizeof(float)));
            break;
        }
        r->res_off = roff;
        r->res_bytes = roff != std::string::npos ? up256(rf * sizeof(float)) : 0;
        r->res_floats = rf;
        if (ooff != std::string::npos) outs += rf;
        r->block = off;
        r->layer = 0;
        r->cur = -1;   // frame not packed yet
        r->stage_off = staged;
        staged += fl;
        S->queue.pop_front();
        S->active.push_back(r);
        sl.reqs.push_back(r);
        sl.out_off.push_back(ooff);
    }
}

static void serve_loop(net* n, ServeState* S) {
    cudaSetDevice(n->device);
    // Host-side fault injection for tests: a slow step (microseconds).
    const char* slow = getenv("NET_SERVE_STEP_DELAY_US");
    const long delay_us = slow ? atol(slow) : 0;
    int next = 0, oldest = 0;   // slots are used round robin; the busy ones start at oldest
    auto retire_oldest = [&] {
        complete_step(n, S, S->slot[oldest]);
        oldest = (oldest + 1) % kSlots;
    };
    while (true) {
        // results of finished steps, oldest first, without blocking
        while (S->slot[oldest].busy && (S->slot[oldest].status != NET_OK ||
                                        cudaEventQuery(S->slot[oldest].ev_done) != cudaErrorNotReady))
            retire_oldest();
        StepSlot& sl = S->slot[next];
        if (sl.busy) {   // every slot in flight: wait for the oldest step
            retire_oldest();
            continue;
        }
        const bool inflight = S->slot[oldest].busy;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            auto ready = [&] { return S->stop || !S->queue.empty(); };
            if (!inflight) {
                S->cv_work.wait(lk, ready);
            } else if (!ready()) {
                // a step is on the GPU: look again shortly for arrivals or its end
                S->cv_work.wait_for(lk, std::chrono::microseconds(20), ready);
                if (!ready()) continue;
            }
            if (S->stop) break;
            admit(n, S, sl);
        }
        if (sl.reqs.empty()) {   // the head of the queue waits for memory a step will free
            if (inflight) retire_oldest();
            else std::this_thread::sleep_for(std::chrono::microseconds(100));
            continue;
        }
        if (delay_us > 0) std::this_thread::sleep_for(std::chrono::microseconds(delay_us));
        sl.busy = true;
        sl.status = enqueue_step(n, S, sl);
        ++S->steps;
        next = (next + 1) % kSlots;
    }
    while (S->slot[oldest].busy) retire_oldest();
}

static net_status serve_start(net* n) {
    if (n->serve.load()) return NET_OK;
    if (!n->weights_loaded) return fail(NET_E_WEIGHTS, "weights not loaded");
    std::unique_ptr<ServeState> S(new ServeState());
    cudaError_t e = cudaSetDevice(n->device);
    size_t freeb = 0, totalb = 0;
    if (e == cudaSuccess) e = cudaMemGetInfo(&freeb, &totalb);
    if (e != cudaSuccess) return fail(NET_E_CUDA, "serve start: %s", cudaGetErrorString(e));
    auto cleanup = [&] { serve_free(S.get()); };
    const size_t arena = std::min(n->budget, freeb / 2);
    if ((e = dn::dalloc(&S->arena, arena)) != cudaSuccess) {
        cleanup();
        return fail(NET_E_OOM, "serving arena %zu bytes: %s", arena, cudaGetErrorString(e));
    }
    S->alloc.init(arena);
    if (const char* m = getenv("NET_SERVE_MAX_ACTIVE")) S->max_active = std::max(1, atoi(m));
    const int nl = (int)n->L.size();
    S->stage_bytes = up256((size_t)S->max_active * sizeof(PackJob)) +
                     (size_t)S->max_active * nl * (sizeof(ConvProblem) + sizeof(PoolJob));
    int c, ho, wo;
    net_output_shape(n, n->max_side, n->max_side, &c, &ho, &wo);
    // per-slot pinned staging, used only by requests that got no chunk of the
    // pinned arena: room for at least the largest frame and result
    S->h_out_floats = std::max((size_t)c * ho * wo, (size_t)4 << 20);
    S->h_in_floats = std::max((size_t)n->in_c * n->max_side * n->max_side, (size_t)4 << 20);
    {
        // pinned host arena: net_submit copies frames into it and results
        // land in it, so uploads and downloads run at pinned speed
        size_t mb = 1024;
        if (const char* v = getenv("NET_SERVE_PINNED_MB")) mb = (size_t)std::max(0, atoi(v));
        if (mb > 0 && cudaHostAlloc((void**)&S->hpin, mb << 20, cudaHostAllocDefault) == cudaSuccess)
            S->hpin_alloc.init(mb << 20);
        else
            S->hpin = nullptr;
    }
    e = cudaStreamCreateWithFlags(&S->s_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->s_out, cudaStreamNonBlocking);
    for (StepSlot& sl : S->slot) {
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_stage, S->stage_bytes);
        if (e == cudaSuccess) e = dn::dalloc(&sl.d_stage, S->stage_bytes);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_in, S->h_in_floats * sizeof(float));
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_out, S->h_out_floats * sizeof(float));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev_in, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev_comp, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev_done, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        cleanup();
        return fail(NET_E_OOM, "serving staging: %s", cudaGetErrorString(e));
    }
    {
        // copy threads: three beside the caller (NET_SERVE_COPY_THREADS
        // overrides; 0 keeps every copy on the calling thread)
        const unsigned hc = std::thread::hardware_concurrency();
        int nt = hc >= 8 ? 3 : hc >= 4 ? 1 : 0;
        if (const char* v = getenv("NET_SERVE_COPY_THREADS")) nt = std::max(0, std::min(16, atoi(v)));
        S->copies.start(nt);
    }
    S->th = std::thread(serve_loop, n, S.get());
    n->serve.store(S.release());
    return NET_OK;
}

void serve_stop(net* n) {
    ServeState* S = n->serve.load();
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    serve_free(S);
    delete S;
    n->serve.store(nullptr);
}

}  // namespace dn

extern "C" net_status net_submit(net_t* n, const float* frame, int h, int w, uint64_t* req_id) {
    if (!n || !frame || !req_id) return fail(NET_E_INVAL, "NULL argument");
    net_status s = check_shape(n, 1, h, w);
    if (s != NET_OK) return s;
    if (!n->serve.load()) {
        std::lock_guard<std::mutex> lk(n->serve_mu);
        s = serve_start(n);   // no-op when another submitter started it first
        if (s != NET_OK) return s;
    }
    ServeState* S = n->serve.load();
    auto r = std::make_shared<Request>();
    r->h = h;
    r->w = w;
    size_t half;
    r->block_bytes = request_bytes(n, h, w, r->H, r->W, &half);
    if (r->block_bytes > S->alloc.size)
        return fail(NET_E_BUDGET, "frame %dx%d needs %zu bytes, budget %zu", h, w, r->block_bytes, S->alloc.size);
    r->t_submit = Clock::now();
    const size_t fbytes = (size_t)n->in_c * h * w * sizeof(float);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        size_t off;
        if (S->hpin && S->hpin_alloc.alloc(up256(fbytes), &off)) {
            r->pin_off = off;
            r->pin_bytes = up256(fbytes);
        }
    }
    if (r->pin_off != std::string::npos) S->copies.copy(S->hpin + r->pin_off, frame, fbytes);
    else r->frame.assign(frame, frame + (size_t)n->in_c * h * w);
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
    const size_t nres = r->res_off != std::string::npos ? r->res_floats : r->result.size();
    if (cap < nres) return fail(NET_E_INVAL, "output capacity %zu < %zu", cap, nres);
    if (r->res_off != std::string::npos) {
        S->copies.copy(out, S->hpin + r->res_off, nres * sizeof(float));
        S->hpin_alloc.release(r->res_off, r->res_bytes);
        r->res_off = std::string::npos;
    } else {
        std::memcpy(out, r->result.data(), nres * sizeof(float));
    }
    S->all.erase(it);
    return NET_OK;
}

extern "C" net_status net_poll(net_t* n, uint64_t id, float* out, size_t cap, int* done) {
    if (!n || !out || !done) return fail(NET_E_INVAL, "NULL argument");
    ServeState* S = n->serve.load();
    if (!S) return fail(NET_E_STATE, "no request submitted");
    std::lock_guard<std::mutex> lk(S->mu);
    bool d = false;
    net_status s = take_result(S, id, out, cap, &d);
    *done = d ? 1 : 0;
    return s;
}

extern "C" net_status net_wait(net_t* n, uint64_t id, float* out, size_t cap, int timeout_ms) {
    if (!n || !out) return fail(NET_E_INVAL, "NULL argument");
    ServeState* S = n->serve.load();
    if (!S) return fail(NET_E_STATE, "no request submitted");
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
    ServeState* S = n->serve.load();
    if (!S) return NET_OK;
    std::lock_guard<std::mutex> lk(S->mu);
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
    ServeState* S = n->serve.load();
    if (!S) return NET_OK;
    std::lock_guard<std::mutex> lk(S->mu);
    S->lat_ms.clear();
    S->completed = 0;
    return NET_OK;
}
