// net_internal.h — the handle and the executor's internal entry points.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/net.h"
#include "kernels.h"

namespace dn {

enum { ENG_SIMT = 0, ENG_TC = 1 };

struct Layer {
    net_layer d{};
    int cin = 0;
    int prec = 0;        // net_precision of the operands
    int engine = 0;      // ENG_SIMT or ENG_TC
    int kx = 0;          // kernel size the conv kernel runs (1 for an im2col-packed layer)
    int im2col_k = 0;    // k > 0: the input is packed im2col-style (taps folded into channels)
    bool pair = false;   // BF16 3x3 first layer over 8 channels, two taps per MMA (TcArgs::pair)
    int in_dt = 0;       // storage dtype of this layer's input activation
    int in_cs = 0;       // its channel stride (padded channels)
    int w_rows = 0;      // allocated weight rows (zero beyond cout)
    int cs32 = 0;        // channel stride of the FP32 calibration copy
    void* w = nullptr;   // [w_rows][k*k][in_cs], dtype in_dt
    float* bias = nullptr;
    float* wscale = nullptr;  // FP8 per-channel weight scale
    float* alpha = nullptr;   // FP8: wscale * act_scale
    float* w32 = nullptr;     // FP32 copy of W' for calibration (FP8 nets)
    double act_scale = 1.0;   // FP8 scale of this layer's input
    int tile_bn = 0, tile_ks = 0;   // fixed-batch plan overrides: N tile, split-K (0: analytic choice)
    int tile_mb = 0;                // ... and CTAs per SM (0: chosen per launch)
    // grouped launches (uneven batches, serving): N tile, CTAs per SM, ring
    // stage cap (0: the analytic choice, one CTA an SM, as many as fit)
    int grp_bn = 0, grp_mb = 0, grp_nst = 0;
    CUtensorMap tmB[3];       // TC weights, box rows BN = 64, 128, 256
    // Layers created as FP8 tensor-core layers also keep a BF16 copy, so the
    // precision of each can be switched after loading (precision search).
    bool fp8_capable = false;
    void* w_var[2] = {nullptr, nullptr};   // [0] BF16, [1] FP8 weights
    CUtensorMap tmB_var[2][3];
    int cs_var[2] = {0, 0};                // channel stride of each format
};

// Switches an FP8-capable layer between its BF16 and FP8 operands.
void set_layer_format(Layer& L, int prec);
// Drops every plan and graph that baked a layer format in.
void invalidate_plans(net* n);
// Runs the FP32 copy of the folded weights over d_frames into d_out
// (NCHW float32) and, if amax is not null, the per-layer input max|x|.
net_status run_fp32_reference(net* n, const float* d_frames, int batch, int h, int w, float* d_out,
                              float* amax);

// Launch plan of one layer for one input shape.
struct LayerRun {
    int in_buf = 0, out_buf = 1;   // activation buffers read / written by the conv
    int H = 0, W = 0;              // conv input (= pre-pool output) size
    int TW = 16, TH = 8, BN = 128; // TC tile: TH x TW pixels x BN channels
    int m_tiles = 0, n_tiles = 0, grid = 0;
    int ksplit = 1;                // split-K factor (partial sums in the workspace)
    int bres = 0;                  // TC: weights resident in shared memory
    int kalt = 0;                  // TC: both MMA issuers on each tile (one work item per CTA)
    int mb = 1;                    // TC: CTAs per SM (2: short tiles, epilogue-bound)
    int cg = 1;                    // TC: 2 = CTA pairs (one M = 256 tile across two SMs)
    int nst_cap = 0;               // TC: ring stages at most (0: as many as fit)
    int tapm = 0;                  // TC: ring stages of all nine taps (3x3, resident weights)
    int xred = 0;                  // TC: split-K reduced inside clusters of ksplit CTAs (BF16)
    int sig_off = -1, rd_off = -1, done_off = -1; // TC: row-band counters (batch x tile rows), input-read and
                                                  // finished-warp counters in Plan::flags
    int sbn = 64, sth = 8, stw = 16; // CUDA-core tile
    ConvProblem* d_prob = nullptr; // TC: device problem table (one entry)
};

struct Plan {
    std::vector<LayerRun> runs;
    size_t ws_bytes = 0;           // split-K workspace this plan needs
    int* flags = nullptr;          // row-band dataflow counters of every TC layer (cleared by each pass's pack)
    int nflags = 0;
    ~Plan();
};
// NET_TC_FLOW=0 in the environment keeps every tensor-core launch behind the
// dependency wait on the whole previous kernel (no row-band dataflow); read
// once per process.
bool tc_flow_on();

// TC tile choice for an H x W map (pooled layers need whole 2x2 windows in
// one warp: TW = 8 or 16).
void tc_choose(int batch, int H, int W, bool pool, int ncols, int num_sms, int* TW, int* TH, int* BN);
// xred: the layer's K split may be reduced inside clusters (BF16 operands)
void tc_choose_split(long m_tiles, int ncols, int nk, int num_sms, int* BN, int* ksplit, int max_ks = 16,
                     bool xred = false);
// NET_TC_XRED=0 in the environment keeps every K split on the workspace
// reduction; read once per process.
bool tc_xred_on();
// (N tile, split-K, CTAs per SM) a tensor-core layer can take in its current
// format (two CTAs an SM for N tiles of at most 128 columns).
struct TileOpt {
    int bn, ks, mb;
};
void tc_tile_options(const net* n, int l, std::vector<TileOpt>* opts);
// CTAs per SM, persistent worker count and resident-weight mode of a
// tensor-core launch (nk K steps of chb bytes per tile; mb_req 0: chosen).
void tc_workers(int m_tiles, int n_tiles, int ks, int BN, int nk, int chb, int num_sms, int mb_req, int* workers,
                int* bres, int* mb);
// NET_TC_MB=1 or 2 in the environment forces the CTAs per SM of fixed-batch
// launches (0: chosen per launch); read once per process.
int tc_mb_forced();
// NET_TC_PAIR=1: fixed-batch layers that can take CTA pairs use them; read once.
bool tc_pair_enabled();
// Index into Layer::tmB of the weight map whose box has BN rows.
int tmb_index(int BN);

struct UnevenState;
struct ServeState;
struct RegionState;
struct NightState;

}  // namespace dn

struct net {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int in_c = 0;
    std::vector<dn::Layer> L;
    int max_batch = 1, max_side = 1;
    size_t budget = 0;
    bool has_fp8 = false;
    bool weights_loaded = false;
    bool use_graphs = true;
    // activation buffers, a ring of three: layer l reads act[l % 3] and
    // writes act[(l + 1) % 3] (the stride-1 pool writes back into its conv's
    // input), so a layer that starts before the one two back has finished
    // reading overwrites nothing it still reads
    void* act[3] = {nullptr, nullptr, nullptr};
    size_t act_bytes = 0;
    void* cal[2] = {nullptr, nullptr};
    float* d_in_stage = nullptr;
    float* d_out_stage = nullptr;
    size_t in_stage_bytes = 0, out_stage_bytes = 0;
    // net_forward_async: two staging slots of its own,
    // upload and download streams, per slot: upload done, pass done, slot free
    struct AsyncState {
        float* d_in[2] = {nullptr, nullptr};
        float* d_out[2] = {nullptr, nullptr};
        cudaStream_t s_in = nullptr, s_out = nullptr;
        cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_comp[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
        bool used[2] = {false, false};
        int next = 0;
        net_status first_err = NET_OK;
    };
    AsyncState* async = nullptr;
    std::map<std::tuple<int, int, int, const void*, const void*>, cudaGraphExec_t> graphs;
    bool prof = false;
    std::vector<cudaEvent_t> prof_ev;   // 2 per layer
    // phase trace (net_trace): [layer][kTraceCtas][kTraceEvents] globaltimer stamps
    unsigned long long* trace_dev = nullptr;
    bool trace_on = false;
    uint64_t launches = 0;              // kernels launched so far
    int pending = 0;                    // kernels enqueued by the current forward
    std::map<std::tuple<int, int, int, const void*, const void*>, int> graph_kernels;
    std::map<std::tuple<int, int, int>, dn::Plan*> plans;
    int num_sms = 148;
    float* ws = nullptr;       // split-K workspace (grown by plans, before any capture)
    size_t ws_bytes = 0;
    int* err_host = nullptr;   // mapped pinned: bounded device waits that expired
    int* err_dev = nullptr;
    int fault_layer = -1;      // net_inject_device_fault: layer of the next pass to fault (tests)
    int flow_fault_layer = -1; // net_inject_flow_fault: layer of the next pass whose band wait expires (tests)
    dn::UnevenState* uneven = nullptr;
    dn::RegionState* region = nullptr;   // detection post-processing (net_set_region)
    dn::NightState* night = nullptr;     // nightmare pass buffers (first net_nightmare_* call)
    bool night_weights_stale = false;    // weights reloaded since the backward weights were built
    // request queue, started by the first net_submit; serve_mu serialises
    // concurrent first submits so exactly one queue is created
    std::atomic<dn::ServeState*> serve{nullptr};
    std::mutex serve_mu;
    void graphs_clear();
};

namespace dn {

net_status fail(net_status s, const char* fmt, ...);
// Device buffers of the library: cudaMalloc, with canary guard regions
// around each buffer when NET_GUARD=1 (guard.cu, net_guard_check); freed
// with dfree (which frees a plain cudaMalloc'd pointer too).
cudaError_t dalloc_raw(void** p, size_t bytes);
cudaError_t dfree(void* p);
template <class T>
inline cudaError_t dalloc(T** p, size_t bytes) {
    return dalloc_raw(reinterpret_cast<void**>(p), bytes);
}
void layer_dims(const net* n, int h, int w, std::vector<int>& H, std::vector<int>& W);
net_status check_shape(const net* n, int batch, int h, int w);
size_t act_bytes_for(const net* n, int batch, int h, int w);
net_status enqueue_forward(net* n, const float* d_in, int batch, int h, int w, float* d_out,
                           float* const* trace, bool fp32_copy, float* amax);
net_status get_plan(net* n, int batch, int h, int w, Plan** out);
net_status check_device_error(net* n);
net_status run_forward(net* n, const float* d_in, int batch, int h, int w, float* d_out);
net_status enqueue_uneven(net* n, const float* const* d_in, const int* side, int cnt,
                          float* const* d_out);
void uneven_free(net* n);
void uneven_graphs_clear(net* n);
void uneven_plans_clear(net* n);
// The grouped-launch tile choice of a layer, after the grp_* overrides: N
// tile (given the analytic one), CTAs per SM and stage cap.
void grouped_tiles(const Layer& L, int ncols, int* BN, int* mb, int* nst_cap);
void serve_stop(net* n);
void region_free(net* n);
void night_free(net* n);

}  // namespace dn
