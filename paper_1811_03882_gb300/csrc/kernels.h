// kernels.h — internal launchers (C++), called by the executor in net.cu.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include "common.cuh"

namespace dn {

// One conv layer over a batch of n equal frames, NHWC in / out.
struct ConvLaunch {
    const void* x;   // input activation, NHWC, channel stride Cp, dtype of the layer
    const void* w;   // folded weights [w_rows][k*k][Cp], dtype of the layer
    void* y;         // output (layout/dtype per ep)
    int n, H, W;     // batch and (pre-pool) spatial size
    int Cp;          // padded input channels
    int k;           // 1 or 3
    int w_rows;      // allocated weight rows (>= every column a tile touches)
    Epilogue ep;
    int bn, th, tw;  // unused by the CUDA-core conv (simt_geom chooses the tile)
    int quads;       // 1: 2x2-quad tiles even without a pool (0: flat tiles where they save work)
    int ksplit;      // > 1: K split over grid.z, raw sums to ws
    float* ws;       // split-K partial sums [ksplit][m_tiles*th*tw][n_tiles*bn]
};

// CUDA-core tile choice for a layer with `ncols` output columns.
void simt_tile(int ncols, int* bn, int* th, int* tw);
// Geometry of a CUDA-core conv launch: N tile bn; th x tw quad tiles, or
// (flat = 1: 64-column tiles without a 2x2/s2 pool, where that computes
// fewer pixels; never when `quads`) runs of px consecutive output pixels;
// m_tiles tiles of px pixels (the split-K workspace has m_tiles * px rows);
// red_*: the SplitReduce tile fields for that workspace.
struct SimtGeom {
    int bn, th, tw, flat, px, m_tiles;
    int red_tw, red_th, red_tx, red_ty;
};
SimtGeom simt_geom(int ncols, bool pool, int n, int H, int W, bool quads);
cudaError_t conv_simt(const ConvLaunch& L, cudaStream_t st);

// Split-K reduction + epilogue: y = epilogue(sum_z ws[z]) in fixed z order.
struct SplitReduce {
    const float* ws;
    int ksplit, m_rows, ncols_pad;   // ws geometry: [ksplit][m_rows][ncols_pad]
    int TW, TH, tiles_x, tiles_y;    // tile geometry (row m = tile*TW*TH + py*TW + px)
    int n, H, W;                     // frames and pre-pool size
    void* y;
    Epilogue ep;
    // 0: each z plane row-major [m_rows][ncols_pad].  1 (tensor-core
    // launches, 128-row tiles): [m_rows / 128][ncols_pad / 4][128][4], so a
    // warp that holds one column group of 32 rows writes 512 contiguous bytes.
    int tile_major;
};
cudaError_t splitk_reduce(const SplitReduce& r, cudaStream_t st);

// Frame NCHW float32 -> NHWC (channel stride Cp, zero padded) in dtype dt;
// FP8 codes are value * inv_scale.  zero[0 .. nzero - 1] (a forward pass's
// row-band counters) are cleared by the same launch.
cudaError_t pack_frames(const float* x, void* y, int n, int C, int H, int W, int Cp, int dt,
                        float inv_scale, cudaStream_t st, int* zero = nullptr, int nzero = 0);

// Frame NCHW float32 -> "im2col" NHWC for a k x k first layer with few
// channels: channel j = (kh*k + kw)*C + c of pixel (i, j) holds
// x[c, i+kh-k/2, j+kw-k/2] (zero outside), zero beyond C*k*k; the layer then
// runs as a 1x1 conv over Cp channels.
cudaError_t pack_frames_im2col(const float* x, void* y, int n, int C, int H, int W, int Cp, int k, int dt,
                               float inv_scale, cudaStream_t st);

// NHWC (dtype dt, channel stride cs, value = code*scale for FP8) -> NCHW f32.
cudaError_t unpack_nchw(const void* x, float* y, int n, int C, int H, int W, int cs, int dt,
                        float scale, cudaStream_t st);

// 2x2 stride-1 max pool, window clipped at the bottom/right edge, NHWC.
cudaError_t maxpool_s1_same(const void* x, void* y, int n, int H, int W, int cs, int dt,
                            cudaStream_t st);

// Batchnorm fold and cast of one layer, FP64 on the device.
//  raw_w: [cout][cin][k][k] f32; bn arrays (or bias) f32, device.
//  out_w: [w_rows][k*k][Cp] in dt (zero padded); out_bias[cout] f32;
//  out_wscale[cout] (FP8 per-channel weight scale, may be null otherwise);
//  out_w32: optional FP32 copy of W' in the same layout (Cp32 channels).
struct FoldArgs {
    const float* raw_w;
    const float *beta, *gamma, *mean, *var, *bias;  // bn: first four; else bias
    int cout, cin, k, Cp, w_rows, dt;
    void* out_w;
    float* out_bias;
    float* out_wscale;
    double* tmp_s;      // [cout] scratch: per-channel BN scale
    double* tmp_amax;   // [cout] scratch: per-channel max |W'|
    float* out_w32;
    int Cp32;
    int im2col;         // 1: write [w_rows][Cp] with channel j = (kh*k + kw)*cin + c
};
cudaError_t fold_layer(const FoldArgs& a, cudaStream_t st);

// alpha[o] = (float)((double)wscale[o] * act_scale), FP8 layers.
cudaError_t make_alpha(const float* wscale, double act_scale, float* alpha, int cout,
                       cudaStream_t st);

// max |x| over count floats, atomically folded into *out (out >= 0 floats).
cudaError_t absmax_f32(const float* x, size_t count, float* out, cudaStream_t st);

}  // namespace dn

namespace dn {
// n / d for 0 <= n < 2^31 and 1 <= d < 2^31 by one multiply-high, an add and
// a shift (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, n / d = (mulhi(n, m) + n) >> l.  The
// tensor-core kernel's tile and K-step decodes divide by launch constants
// once per tile; a runtime integer division there costs a dependent chain of
// some twenty instructions on a warp with nothing else to issue.
struct FastDiv {
    uint32_t mul = 1u, shift = 0u;   // d = 1
};
inline FastDiv make_fast_div(int d) {
    FastDiv f;
    uint32_t l = 0;
    while ((1ull << l) < (unsigned long long)d) ++l;
    f.mul = (uint32_t)(((1ull << 32) * ((1ull << l) - (unsigned long long)d)) / (unsigned long long)d + 1ull);
    f.shift = l;
    return f;
}
#ifdef __CUDACC__
__device__ __forceinline__ int fdiv(int n, FastDiv f) {
    return (int)((__umulhi((uint32_t)n, f.mul) + (uint32_t)n) >> f.shift);
}
#endif

// One group member of a tensor-core conv launch: a batch of n equal frames
// with its own activation tensor map and output.  The device-side table of
// problems lets one launch cover frames of different sizes.
struct alignas(128) ConvProblem {
    CUtensorMap tmA;    // NHWC activation, box (chunk, TW, TH, 1)
    const void* x;      // activation base (CUDA-core kernels)
    void* y;            // output base
    int n, H, W;        // frames, pre-pool size
    int tiles_x, tiles_y;
    int tile_begin;     // first M tile of this problem in the launch
    FastDiv fd_tx, fd_ty;   // division by tiles_x, tiles_y (set by tc_problem_divisors)
};
// Fills a problem's division constants from its tiles_x / tiles_y.
inline void tc_problem_divisors(ConvProblem& p) {
    p.fd_tx = make_fast_div(p.tiles_x);
    p.fd_ty = make_fast_div(p.tiles_y);
}

struct TcArgs {
    const ConvProblem* probs;  // device table, nprob entries
    int nprob, m_tiles, n_tiles;
    int Cp, k, TW, TH;
    int chb;      // bytes of one K chunk (32, 64 or 128): the swizzle width
    int cpc;      // channels per chunk
    int chunks;   // chunks per tap (Cp / cpc)
    void* y_override;  // if not null, output base for every problem
    int ksplit;        // K split factor (tiles x ksplit work items)
    float* ws;         // ksplit > 1: raw sums [ksplit][m_tiles*128][n_tiles*BN]
    int bres;          // 1: the whole weight slice stays in shared memory (tc_b_resident)
    // shared-memory geometry, filled by conv_tc_launch: ring stages, stage
    // bytes, resident-weight offset, control-block offset
    int nst, st_bytes, bres_off, ctrl_off;
    int plane;    // producer lanes per producer warp (2 * plane divides nst)
    int kalt;     // 1: the two MMA issuers take alternate K steps of each tile
                  //    (needs at least two K steps per work item)
    // tapm = 1 (3 x 3 layers with resident weights, 16 x 8 or 8 x 16 tiles):
    // a ring stage is one channel chunk of all nine taps, three TMA boxes of
    // TH + 2 rows (one per tap column; the activation map's box is TH + 2
    // rows high), and each tap's A operand starts dy * TW rows into its box.
    int tapm;
    // pair = 1 (a BF16 3 x 3 first layer over 8 channels: 16-byte K chunks,
    // tap-merged stages without swizzle, resident weights): each K = 16 MMA
    // covers two taps, its A descriptor's leading-dimension offset pointing
    // from the first tap's core matrices to the second's
    int pair;     // (2: the same with one box of (TH + 2) x (TW + 2) pixels a stage, TW = 8, TH = 16)
    Epilogue ep;
    int* err;     // bounded-wait failure code (0 = none)
    long long wait_limit;   // bound of each pipeline wait, clock64 cycles (<= 0: ~2 s)
    int nst_cap;            // ring stages at most (even, >= 2; 0: as many as fit)
    int withhold;           // fault injection (tests): one producer skips one K step
    // xred = 1 (K split, one work item per CTA): the ksplit CTAs of a tile form
    // one thread-block cluster and add their partial sums through distributed
    // shared memory, each applying the epilogue to 1 / ksplit of the columns;
    // no workspace and no reduction launch
    int xred;
    // phase trace (net_trace): if not null, CTA b writes globaltimer stamps
    // to trace[b * kTraceEvents + e] (kTraceEvents per CTA; the host passes
    // null when the grid exceeds kTraceCtas)
    unsigned long long* trace;
    // division by ksplit, n_tiles, chunks, k and nst (filled by conv_tc_launch)
    FastDiv fd_ksplit, fd_ntiles, fd_chunks, fd_k, fd_nst;
    // Row-band dataflow between consecutive layers of a fixed-batch pass (all
    // null: the dependency wait orders the launch after the whole previous
    // kernel).  sig: this launch's output bands, one counter per (frame, tile
    // row), to which every epilogue warp that drains a tile adds 1 once its
    // stores are done.  dep: the previous layer's sig; instead of the
    // dependency wait, a producer waits for the bands under a tile's input
    // rows (a band is 2^dep_shift input rows, dep_nb bands a frame, complete
    // at dep_target) before it loads them.  rd_sig: this launch's input-read
    // counter (each producer warp adds 1 once its last copy has landed);
    // rd_dep: the counter of the layer whose input buffer this launch
    // overwrites, which the epilogue waits for (rd_target) before its first
    // store.  done_sig: this launch's finished-warp counter (each epilogue
    // warp adds 1 after its last tile); dep_done: the previous layer's, at
    // dep_done_target the whole layer is out and a producer stops waiting
    // for bands.  The counters are cleared by the pass's frame pack.
    int* sig;
    const int* dep;
    int dep_shift, dep_nb, dep_target;
    int* rd_sig;
    const int* rd_dep;
    int rd_target;
    int* done_sig;
    const int* dep_done;
    int dep_done_target;
    // 1: let the next kernel launch only once this one is past its
    // dependency wait (the first layer of a pass on the row-band dataflow)
    int late_trigger;
};

// Grouped memory-bound helpers: one launch over several frames of
// different sizes.  Jobs are a device table; `begin` is each job's first
// work item (16-byte vector) in the launch's flat index space.
struct PackJob {
    const float* src;   // NCHW float32 frame
    void* dst;          // NHWC, channel stride Cp
    int C, H, W, Cp;
    int im2col_k;       // 0: plain pack; k: im2col pack for a k x k layer
    long long begin;
};
cudaError_t pack_frames_grouped(const PackJob* jobs, int njobs, long long total, int dt, float inv_scale,
                                cudaStream_t st);
struct PoolJob {
    const void* x;
    void* y;
    int H, W;
    long long begin;
};
cudaError_t maxpool_s1_grouped(const PoolJob* jobs, int njobs, long long total, int cs, int dt,
                               cudaStream_t st);

// Phase trace of a tensor-core launch: per CTA, globaltimer stamps (ns) at
// 0 kernel start, 1 end of the prologue (barriers, tensor memory), 2 the
// first producer past the dependency wait, 3 the first MMA issuer's first
// K step ready, 4 its last MMA issued, 5 epilogue warp 2 started (after the
// bias staging), 6 epilogue warp 2 done, 7 epilogue warp 6 done, 8 the
// kernel's closing barrier passed (before tensor memory is freed), 9 warp
// 2's last accumulator ready.
constexpr int kTraceEvents = 10;
constexpr int kTraceCtas = 512;
int tc_chunk_bytes(int Cp, int dt);
// Whether a launch keeps its weights resident in shared memory: no K split,
// and nk boxes of BN x chunk bytes (one N tile's weights; with several N
// tiles each CTA serves one, the grid a multiple of n_tiles) fit beside the
// A stages (of a CTA's share of the SM: mb CTAs an SM).
bool tc_b_resident(int BN, int n_tiles, int ksplit, int nk, int chb, int mb);
cudaError_t tc_encode_act(CUtensorMap* tm, const void* base, int dt, int n, int H, int W, int Cp, int TW,
                          int TH);
cudaError_t tc_encode_weights(CUtensorMap* tm, const void* w, int dt, int rows, int KK, int Cp, int BN);
// CTAs of one cluster-reduced launch (xred) that can be resident at once
// with N tile BN and ksplit CTAs a cluster (0 if such clusters cannot run)
int tc_xred_capacity(int BN, int ksplit);
// workers = persistent CTAs; tmB has box rows BN (cg = 2: BN / 2); mb =
// CTAs per SM (1, or 2 for BN <= 128: half the shared memory and TMEM, 80
// registers a thread); cg = 2: CTA pairs (2-CTA clusters, workers even, one
// M = 256 tile a pair; BN 128 or 256, mb 1, streamed weights, no tap
// merging and one MMA issuer).  a.xred = 1: clusters of a.ksplit CTAs,
// workers = m_tiles * n_tiles * ksplit (one work item a CTA), BF16 operands,
// BF16 NHWC or FP32 NCHW output.
cudaError_t conv_tc_launch(const CUtensorMap& tmB, const TcArgs& a, int BN, int dt, int workers, int mb, int cg,
                           cudaStream_t st);
}  // namespace dn
