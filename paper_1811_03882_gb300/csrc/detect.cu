// detect.cu — detection post-processing after the last conv layer: region
// (anchor-box) decode and per-class non-maximum suppression, on the device.
//
// The paper offloads Darknet's "detection" sample app (Sec. 5.1.1); the
// network's final map is decoded where it was computed, so that only the
// detections cross back to the host (the transfer rule of Sec. 3.2).  Region
// output of a detection network, as this library reads it: anchor a owns map
// channels a*(5+C) .. a*(5+C)+4+C (tx, ty, tw, th, objectness logit, C class
// logits); cell (i, j) and anchor a form box id (i*GW + j)*A + a with
//   x = (j + sigmoid(tx)) / GW, y = (i + sigmoid(ty)) / GH,
//   w = exp(tw) * pw / GW,      h = exp(th) * ph / GH,
// class-c score = sigmoid(to) * softmax(logits)_c.  Boxes whose class-c score
// exceeds the threshold are candidates of class c; greedy NMS per class takes
// them by score (descending, equal scores by id) and drops a box whose IoU
// with a kept box of its class exceeds the IoU threshold.  A frame's
// detections are its kept boxes class by class, each class in that order.
//
// Two kernels, all FP32.  Decode: one thread per box, threads along grid
// columns so that each channel is read contiguously, up to 32 class logits
// in registers; candidates are appended to per-(frame, class) lists, one
// atomic per warp and class reserving the slots of its lanes.  NMS: one CTA
// per (frame, class) sorts its list by a 64-bit key (inverted score bits,
// id; bitonic, keys in registers), so the result does not depend on the
// order the atomics appended in, and suppresses in blocks of 32 candidates:
// the overlaps inside each block are found in parallel first, then a warp
// settles a block by bit operations and the CTA drops what its kept boxes
// overlap (the decisions of one-at-a-time greedy NMS).  The last CTA of a
// frame to finish concatenates the frame's classes into its detection rows.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "../../include/net.h"
#include "common.cuh"
#include "kernels.h"
#include "net_internal.h"

using namespace dn;

namespace dn {

struct RegionCand {   // 32 bytes
    float score;
    int id;
    float x, y, w, h;
    int pad0, pad1;
};

struct RegionState {
    net_region r{};
    int maxc = 0;               // candidate slots per (frame, class): grid cells x anchors
    int max_batch = 0;
    int* d_cnt = nullptr;       // [max_batch][C + 1]: per class candidates, then kept; classes done
    RegionCand* d_cand = nullptr;   // [max_batch][C][maxc]
    float* d_anchor = nullptr;  // [2A]
    void* d_out = nullptr;      // forward_detect: [counts (max_batch ints, 256-byte block)][dets]
    void* h_out = nullptr;      // pinned host copy of d_out
    size_t out_bytes = 0;
};

void region_free(net* n) {
    RegionState* R = n->region;
    if (!R) return;
    dn::dfree(R->d_cnt);
    dn::dfree(R->d_cand);
    dn::dfree(R->d_anchor);
    dn::dfree(R->d_out);
    cudaFreeHost(R->h_out);
    delete R;
    n->region = nullptr;
}

}  // namespace dn

namespace {

constexpr int kMaxCand = 4096;   // candidate slots per (frame, class): the NMS sort's register/shared bound

__device__ __forceinline__ float sigm(float v) { return 1.f / (1.f + expf(-v)); }

// Counters, per frame f: cnt[f*(C+1) + c] the candidates (after NMS: the
// kept boxes) of class c, cnt[f*(C+1) + C] the classes of f done with NMS.
__global__ void region_decode_kernel(const float* __restrict__ map, int batch, int A, int C, int GH, int GW,
                                     const float* __restrict__ anchor, float thresh, int maxc, int* cnt,
                                     RegionCand* cand) {
    // boxes of a launch: batch * A * GH * GW < 2^31 (the set-up's bounds)
    const int t = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int total = batch * A * GH * GW;
    const bool valid = t < total;
    const int lane = threadIdx.x & 31;
    // thread order (frame, anchor, row, column): consecutive threads read
    // consecutive columns of each channel
    const int tt = valid ? t : total - 1;
    const int r1 = tt / GW, j = tt - r1 * GW;
    const int r2 = r1 / GH, i = r1 - r2 * GH;
    const int f = r2 / A, a = r2 - f * A;
    const long long plane = (long long)GH * GW;
    const float* p = map + ((long long)f * A * (5 + C) + (long long)a * (5 + C)) * plane + (long long)i * GW + j;
    const float x = ((float)j + sigm(p[0])) / (float)GW;
    const float y = ((float)i + sigm(p[plane])) / (float)GH;
    const float w = expf(p[2 * plane]) * anchor[2 * a] / (float)GW;
    const float h = expf(p[3 * plane]) * anchor[2 * a + 1] / (float)GH;
    const float obj = sigm(p[4 * plane]);
    const float* lg = p + 5 * plane;
    const int id = (i * GW + j) * A + a;
    // the lanes of one frame share its counters: one atomic per (warp, frame,
    // class) reserves their slots, each lane's slot follows from the ballot
    const unsigned peers = __match_any_sync(0xffffffffu, valid ? f : -1);
    int* fcnt = cnt + (long long)f * (C + 1);
    RegionCand* fcand = cand + (long long)f * C * maxc;
    auto put = [&](int c, int slot, float s) {
        if (slot < maxc) {
            RegionCand q;
            q.score = s;
            q.id = id;
            q.x = x;
            q.y = y;
            q.w = w;
            q.h = h;
            q.pad0 = q.pad1 = 0;
            fcand[(long long)c * maxc + slot] = q;
        }
    };
    auto append = [&](int c, float s) {   // called by all 32 lanes, c uniform
        const bool pass = valid && s > thresh;
        const unsigned m = __ballot_sync(0xffffffffu, pass) & peers;
        if (pass) {
            const int leader = __ffs(m) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(&fcnt[c], __popc(m));
            base = __shfl_sync(m, base, leader);
            put(c, base + __popc(m & ((1u << lane) - 1u)), s);
        }
    };
    if (C <= 32) {
        // up to 32 classes: all logits in registers, their loads issued together
        float e[32];
        float m = -INFINITY;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            e[c] = c < C ? lg[c * plane] : -INFINITY;
            m = fmaxf(m, e[c]);
        }
        float sum = 0.f;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            e[c] = c < C ? expf(e[c] - m) : 0.f;
            sum += e[c];
        }
        const float os = obj / sum;   // class-c score = obj * e_c / sum
#pragma unroll
        for (int c = 0; c < 32; ++c) e[c] *= os;
        // lane c reserves class c's slots for the lanes of one frame, all
        // classes' atomics in flight together; a warp that straddles frames
        // does this once per frame
        const unsigned vmask = __ballot_sync(0xffffffffu, valid);
        unsigned rem = vmask;
        while (rem) {   // warp-uniform
            const int leader = __ffs(rem) - 1;
            const unsigned grp = __shfl_sync(0xffffffffu, peers, leader) & vmask;   // the leader's frame
            const bool in = (grp >> lane) & 1u;
            unsigned mine = 0;
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                if (c < C) {
                    const unsigned b = __ballot_sync(0xffffffffu, in && e[c] > thresh);
                    if (lane == c) mine = b;
                }
            }
            int* gcnt = cnt + (long long)__shfl_sync(0xffffffffu, f, leader) * (C + 1);
            int base = 0;
            if (mine) base = atomicAdd(&gcnt[lane], __popc(mine));
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                if (c < C) {
                    const unsigned b = __shfl_sync(0xffffffffu, mine, c);
                    const int bc = __shfl_sync(0xffffffffu, base, c);
                    if ((b >> lane) & 1u) put(c, bc + __popc(b & ((1u << lane) - 1u)), e[c]);
                }
            }
            rem &= ~grp;
        }
    } else {
        float m = lg[0];
        for (int c = 1; c < C; ++c) m = fmaxf(m, lg[c * plane]);
        float sum = 0.f;
        for (int c = 0; c < C; ++c) sum += expf(lg[c * plane] - m);
        const float os = obj / sum;
        for (int c = 0; c < C; ++c) append(c, expf(lg[c * plane] - m) * os);
    }
}

// Box edges (left, top, right, bottom) and area, from centre and size.
__device__ __forceinline__ float4 edges_of(float x, float y, float w, float h) {
    return make_float4(x - w * 0.5f, y - h * 0.5f, x + w * 0.5f, y + h * 0.5f);
}

// Whether IoU(a, b) exceeds thr, as inter > thr * union (no division); a
// union of zero has IoU 0.
__device__ __forceinline__ bool overlaps(float4 a, float area_a, float4 b, float area_b, float thr) {
    const float iw = fminf(a.z, b.z) - fmaxf(a.x, b.x);
    const float ih = fminf(a.w, b.w) - fmaxf(a.y, b.y);
    const float inter = fmaxf(iw, 0.f) * fmaxf(ih, 0.f);
    const float uni = area_a + area_b - inter;
    return uni > 0.f ? inter > thr * uni : 0.f > thr;
}

__device__ __forceinline__ unsigned long long shfl_xor_u64(unsigned long long v, int m) {
    const unsigned lo = __shfl_xor_sync(0xffffffffu, (unsigned)v, m);
    const unsigned hi = __shfl_xor_sync(0xffffffffu, (unsigned)(v >> 32), m);
    return ((unsigned long long)hi << 32) | lo;
}

// Shared memory of the NMS kernel for P = 2^LOGP sort slots and C classes.
struct NmsSmem {
    size_t keys, edge, box, sc, ids, area, pre, supp, prefix, total;
};
__host__ __device__ inline NmsSmem nms_layout(int P, int C) {
    NmsSmem s;
    s.keys = 0;                              // 2 x P u64: the sort's exchange buffers ...
    s.edge = 0;                              // ... then P float4 edges, in rank order
    s.box = s.keys + 16 * (size_t)P;         // P float4 (x, y, w, h)
    s.sc = s.box + 16 * (size_t)P;           // P float score
    s.ids = s.sc + 4 * (size_t)P;            // P int box id
    s.area = s.ids + 4 * (size_t)P;          // P float area
    s.pre = s.area + 4 * (size_t)P;          // P u32: overlaps with later candidates of the same 32-block
    s.supp = s.pre + 4 * (size_t)P;          // P u8: suppressed
    s.prefix = (s.supp + (size_t)P + 15) & ~(size_t)15;   // C + 1 int: the frame's class offsets
    s.total = s.prefix + 4 * ((size_t)C + 1);
    return s;
}

__host__ __device__ constexpr int nms_threads(int logp) { return (1 << logp) < 1024 ? (1 << logp) : 1024; }

// One CTA per (frame, class): sort the class's candidates by (score
// descending, id ascending), suppress greedily, write the kept ones back to
// the front of the list in rank order and their count to the counter.  The
// last CTA of a frame to finish (a counter per frame) concatenates the
// frame's classes into its detection rows.
//
// Sort: bitonic over P = 2^LOGP slots with T = min(P, 1024) threads, keys in
// registers (slot m*T + tid in register m); partners within a warp by
// shuffles, in the same thread by register pairs, across warps through
// shared memory (two buffers, so one barrier per such stage).  Suppression
// in blocks of 32 in rank order: first, for every candidate, the bits of the
// later candidates of its block that it overlaps (all threads); then per
// block warp 0 settles who is kept (the first alive candidate is kept and
// drops the later ones it overlaps, and so on), and the CTA drops every
// later candidate that a kept one overlaps.  These are the decisions of
// greedy NMS taken one candidate at a time.
template <int LOGP>
__global__ void __launch_bounds__(nms_threads(LOGP)) region_nms_kernel(int C, int maxc, float iou_thr,
                                                                       int max_det, int* cnt, RegionCand* cand,
                                                                       int* counts, net_detection* det) {
    constexpr int P = 1 << LOGP;
    constexpr int T = nms_threads(LOGP);
    constexpr int KPT = P / T;   // keys per thread
    static_assert(KPT >= 1 && T % 32 == 0 && P <= kMaxCand, "sort slots");
    extern __shared__ __align__(16) unsigned char sm[];
    const NmsSmem lay = nms_layout(P, C);
    unsigned long long* kbuf = reinterpret_cast<unsigned long long*>(sm + lay.keys);
    float4* edge = reinterpret_cast<float4*>(sm + lay.edge);
    float4* box = reinterpret_cast<float4*>(sm + lay.box);
    float* sc = reinterpret_cast<float*>(sm + lay.sc);
    int* ids = reinterpret_cast<int*>(sm + lay.ids);
    float* area = reinterpret_cast<float*>(sm + lay.area);
    unsigned* pre = reinterpret_cast<unsigned*>(sm + lay.pre);
    unsigned char* supp = sm + lay.supp;
    int* prefix = reinterpret_cast<int*>(sm + lay.prefix);
    __shared__ unsigned s_kept;
    __shared__ int s_r0, s_last;

    const int tid = threadIdx.x, lane = tid & 31;
    const int f = blockIdx.x / C, c = blockIdx.x - f * C;
    int* fcnt = cnt + (long long)f * (C + 1);
    const int n = min(fcnt[c], maxc);
    RegionCand* L = cand + ((long long)f * C + c) * maxc;

    // key: inverted score bits (scores are positive, so larger scores have
    // larger bits), then the id (unique within a class, 12 bits), then the
    // slot (12 bits, carried along); empty slots sort last
    unsigned long long v[KPT];
#pragma unroll
    for (int m = 0; m < KPT; ++m) {
        const int q = m * T + tid;
        if (q < n) {
            const unsigned s = __float_as_uint(L[q].score);
            v[m] = ((unsigned long long)(0xFFFFFFFFu - s) << 32) | ((unsigned long long)L[q].id << 12) | (unsigned)q;
        } else {
            v[m] = ~0ull;
        }
    }
    // the network's merges of width k sort each k-slot block on its own:
    // stopping at the first k >= n leaves slots [0, k) sorted ascending
    // (empty slots hold the largest key); n is uniform, so is the stop
    int buf = 0;
#pragma unroll
    for (int lk = 1; lk <= LOGP; ++lk) {
        if (lk > 5 && (1 << (lk - 1)) >= n) break;
#pragma unroll
        for (int lj = lk - 1; lj >= 0; --lj) {
            const int k = 1 << lk, jj = 1 << lj;
            if (jj >= T) {                      // partner in the same thread
                const int s = jj / T;
#pragma unroll
                for (int m = 0; m < KPT; ++m) {
                    if (m & s) continue;
                    const int q = m * T + tid;
                    const bool up = (q & k) == 0;
                    const unsigned long long lo = v[m], hi = v[m | s];
                    if ((lo > hi) == up) {
                        v[m] = hi;
                        v[m | s] = lo;
                    }
                }
            } else if (jj >= 32) {              // partner in another warp
                unsigned long long* kb = kbuf + buf * P;
#pragma unroll
                for (int m = 0; m < KPT; ++m) kb[m * T + tid] = v[m];
                __syncthreads();
#pragma unroll
                for (int m = 0; m < KPT; ++m) {
                    const int q = m * T + tid;
                    const unsigned long long o = kb[q ^ jj];
                    const bool keep_min = ((q & jj) == 0) == ((q & k) == 0);
                    v[m] = keep_min ? (o < v[m] ? o : v[m]) : (o > v[m] ? o : v[m]);
                }
                buf ^= 1;
            } else {                            // partner in the same warp
#pragma unroll
                for (int m = 0; m < KPT; ++m) {
                    const int q = m * T + tid;
                    const unsigned long long o = shfl_xor_u64(v[m], jj);
                    const bool keep_min = ((q & jj) == 0) == ((q & k) == 0);
                    v[m] = keep_min ? (o < v[m] ? o : v[m]) : (o > v[m] ? o : v[m]);
                }
            }
        }
    }
    __syncthreads();   // the exchange buffers become the edges
    // gather in rank order
#pragma unroll
    for (int m = 0; m < KPT; ++m) {
        const int r = m * T + tid;
        if (r < n) {
            const RegionCand& e = L[(int)(v[m] & 0xFFFu)];
            box[r] = make_float4(e.x, e.y, e.w, e.h);
            edge[r] = edges_of(e.x, e.y, e.w, e.h);
            area[r] = e.w * e.h;
            sc[r] = e.score;
            ids[r] = e.id;
            supp[r] = 0;
        }
    }
    __syncthreads();
    // overlaps within each block of 32: bit q of post[r] = candidate r
    // overlaps the later candidate r0 + q of its block (earlier box first, as
    // greedy NMS compares a kept box with a later one)
    for (int r = tid; r < n; r += T) {
        const int l = r & 31, r0 = r - l;
        const float4 mine = edge[r];
        const float am = area[r];
        unsigned bits = 0;
#pragma unroll 8
        for (int q = 1; q < 32; ++q)
            if (q > l && r0 + q < n && overlaps(mine, am, edge[r0 + q], area[r0 + q], iou_thr)) bits |= 1u << q;
        pre[r] = bits;
    }
    __syncthreads();
    int r0 = 0;
    for (;;) {
        if (tid < 32) {
            // settle blocks until one keeps a box (or the list ends): the
            // first alive candidate is kept and drops the later ones of the
            // block it overlaps, then the next alive one, and so on (one step
            // per kept candidate)
            unsigned kept = 0;
            while (r0 < n) {
                const int r = r0 + lane;
                const bool alive = r < n && !supp[r];
                unsigned live = __ballot_sync(0xffffffffu, alive);
                const unsigned post = r < n ? pre[r] : 0u;
                kept = 0;
                while (live) {
                    const int q = __ffs(live) - 1;
                    kept |= 1u << q;
                    live &= ~(1u << q);
                    live &= ~__shfl_sync(0xffffffffu, post, q);
                }
                if (r < n) supp[r] = ((kept >> lane) & 1u) ? 0 : 1;
                if (kept) break;
                r0 += 32;
            }
            if (lane == 0) {
                s_kept = kept;
                s_r0 = r0;
            }
        }
        __syncthreads();
        const unsigned kept = s_kept;
        r0 = s_r0;
        if (r0 >= n) break;
        for (int q = r0 + 32 + tid; q < n; q += T) {
            if (supp[q]) continue;
            const float4 eq = edge[q];
            const float aq = area[q];
            bool drop = false;
            for (unsigned mm = kept; mm; mm &= mm - 1) {
                const int b = r0 + __ffs(mm) - 1;
                drop |= overlaps(edge[b], area[b], eq, aq, iou_thr);
            }
            if (drop) supp[q] = 1;
        }
        r0 += 32;
        __syncthreads();
    }
    // kept ones to the front of the list, in rank order (warp 0, ballots)
    if (tid < 32) {
        int out = 0;
        for (int b0 = 0; b0 < n; b0 += 32) {
            const int r = b0 + lane;
            const bool keep = r < n && !supp[r];
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int pos = out + __popc(m & ((1u << lane) - 1u));
                RegionCand e;
                e.score = sc[r];
                e.id = ids[r];
                e.x = box[r].x;
                e.y = box[r].y;
                e.w = box[r].z;
                e.h = box[r].w;
                e.pad0 = e.pad1 = 0;
                L[pos] = e;
            }
            out += __popc(m);
        }
        if (lane == 0) fcnt[c] = out;
        __threadfence();   // the list and count before this class is counted done
    }
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(&fcnt[C], 1) == C - 1;
    __syncthreads();
    if (!s_last) return;
    // the frame's last class: its detections are the classes' kept boxes,
    // class by class, cut at max_det; its count is the number before the cut
    __threadfence();
    if (tid < 32) {
        int base = 0;
        for (int c0 = 0; c0 < C; c0 += 32) {
            const int k = c0 + lane < C ? __ldcg(&fcnt[c0 + lane]) : 0;
            int incl = k;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            if (c0 + lane < C) prefix[c0 + lane] = base + incl - k;
            base += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) {
            prefix[C] = base;
            counts[f] = base;
        }
    }
    __syncthreads();
    const int ncut = min(prefix[C], max_det);
    const RegionCand* F = cand + (long long)f * C * maxc;
    for (int o = tid; o < ncut; o += T) {
        int lo = 0, hi = C - 1;   // the class c with prefix[c] <= o < prefix[c + 1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= o) lo = mid;
            else hi = mid - 1;
        }
        const RegionCand* e = F + (long long)lo * maxc + (o - prefix[lo]);
        net_detection d;
        d.x = __ldcg(&e->x);
        d.y = __ldcg(&e->y);
        d.w = __ldcg(&e->w);
        d.h = __ldcg(&e->h);
        d.score = __ldcg(&e->score);
        d.cls = lo;
        d.id = __ldcg(&e->id);
        d.pad = 0;
        det[(long long)f * max_det + o] = d;
    }
}

int nms_logp(int maxc) {
    int lp = 8;
    while ((1 << lp) < maxc) ++lp;
    return lp;
}

template <int LOGP>
cudaError_t launch_nms(int batch, int C, int maxc, float iou_thr, int max_det, int* cnt, RegionCand* cand,
                       int* counts, net_detection* det, cudaStream_t st) {
    const size_t smem = nms_layout(1 << LOGP, C).total;
    cudaError_t e = cudaFuncSetAttribute(region_nms_kernel<LOGP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    region_nms_kernel<LOGP><<<batch * C, nms_threads(LOGP), smem, st>>>(C, maxc, iou_thr, max_det, cnt, cand,
                                                                         counts, det);
    return cudaSuccess;
}

cudaError_t enqueue_region(const RegionState& R, const float* d_map, int batch, int GH, int GW, int* d_counts,
                           net_detection* d_det, cudaStream_t st, uint64_t* launches) {
    const int A = R.r.n_anchors, C = R.r.n_classes;
    cudaError_t e = cudaMemsetAsync(R.d_cnt, 0, sizeof(int) * (size_t)batch * (C + 1), st);
    if (e != cudaSuccess) return e;
    // 64-thread blocks: a batch's few thousand boxes spread over ~100 SMs
    const long long total = (long long)batch * A * GH * GW;
    region_decode_kernel<<<(unsigned)((total + 63) / 64), 64, 0, st>>>(
        d_map, batch, A, C, GH, GW, R.d_anchor, R.r.score_thresh, R.maxc, R.d_cnt, R.d_cand);
    switch (nms_logp(R.maxc)) {
        case 8: e = launch_nms<8>(batch, C, R.maxc, R.r.nms_iou, R.r.max_det, R.d_cnt, R.d_cand, d_counts, d_det, st); break;
        case 9: e = launch_nms<9>(batch, C, R.maxc, R.r.nms_iou, R.r.max_det, R.d_cnt, R.d_cand, d_counts, d_det, st); break;
        case 10: e = launch_nms<10>(batch, C, R.maxc, R.r.nms_iou, R.r.max_det, R.d_cnt, R.d_cand, d_counts, d_det, st); break;
        case 11: e = launch_nms<11>(batch, C, R.maxc, R.r.nms_iou, R.r.max_det, R.d_cnt, R.d_cand, d_counts, d_det, st); break;
        default: e = launch_nms<12>(batch, C, R.maxc, R.r.nms_iou, R.r.max_det, R.d_cnt, R.d_cand, d_counts, d_det, st); break;
    }
    if (e != cudaSuccess) return e;
    *launches += 2;
    return cudaGetLastError();
}

size_t counts_block(int max_batch) { return ((size_t)max_batch * sizeof(int) + 255) & ~(size_t)255; }

}  // namespace

#define CK(call)                                                                                      \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return fail(e_ == cudaErrorMemoryAllocation ? NET_E_OOM : NET_E_CUDA, "%s: %s", #call,   \
                        cudaGetErrorString(e_));                                                      \
    } while (0)

extern "C" net_status net_set_region(net_t* n, const net_region* r) {
    if (!n || !r) return fail(NET_E_INVAL, "NULL argument");
    const int A = r->n_anchors, C = r->n_classes;
    if (A < 1 || A > NET_REGION_MAX_ANCHORS || C < 1 || C > 4096)
        return fail(NET_E_INVAL, "anchors %d / classes %d out of range", A, C);
    if (A * (5 + C) != n->L.back().d.cout)
        return fail(NET_E_INVAL, "%d anchors x (5 + %d classes) != %d output channels", A, C, n->L.back().d.cout);
    for (int a = 0; a < 2 * A; ++a)
        if (!(r->anchors[a] > 0.f) || !std::isfinite(r->anchors[a]))
            return fail(NET_E_INVAL, "anchor prior %d = %g not positive finite", a, (double)r->anchors[a]);
    if (!std::isfinite(r->score_thresh) || r->score_thresh < 0.f || !std::isfinite(r->nms_iou) || r->max_det < 1)
        return fail(NET_E_INVAL, "score threshold %g / IoU threshold %g / max_det %d", (double)r->score_thresh,
                    (double)r->nms_iou, r->max_det);
    std::vector<int> H, W;
    layer_dims(n, n->max_side, n->max_side, H, W);
    const long long maxc = (long long)H.back() * W.back() * A;
    if (maxc > kMaxCand)
        return fail(NET_E_UNSUPPORTED, "grid %dx%d x %d anchors = %lld boxes, more than %d", H.back(), W.back(), A,
                    maxc, kMaxCand);
    CK(cudaSetDevice(n->device));
    CK(cudaStreamSynchronize(n->stream));
    region_free(n);
    RegionState* R = new RegionState();
    n->region = R;
    R->r = *r;
    R->maxc = (int)maxc;
    R->max_batch = n->max_batch;
    R->out_bytes = counts_block(n->max_batch) + (size_t)n->max_batch * r->max_det * sizeof(net_detection);
    CK(dn::dalloc(&R->d_cnt, sizeof(int) * (size_t)n->max_batch * (C + 1)));
    CK(dn::dalloc(&R->d_cand, sizeof(RegionCand) * (size_t)n->max_batch * C * R->maxc));
    CK(dn::dalloc(&R->d_anchor, sizeof(float) * 2 * A));
    CK(dn::dalloc(&R->d_out, R->out_bytes));
    CK(cudaHostAlloc(&R->h_out, R->out_bytes, cudaHostAllocDefault));
    CK(cudaMemcpy(R->d_anchor, r->anchors, sizeof(float) * 2 * A, cudaMemcpyHostToDevice));
    return NET_OK;
}

extern "C" net_status net_detect_device(net_t* n, const float* d_map, int batch, int gh, int gw, int* d_counts,
                                        net_detection* d_det) {
    if (!n || !d_map || !d_counts || !d_det) return fail(NET_E_INVAL, "NULL argument");
    if (!n->region) return fail(NET_E_STATE, "no region set (net_set_region)");
    const RegionState& R = *n->region;
    if (batch < 1 || batch > R.max_batch) return fail(NET_E_SHAPE, "batch %d outside [1, %d]", batch, R.max_batch);
    if (gh < 1 || gw < 1 || (long long)gh * gw * R.r.n_anchors > R.maxc)
        return fail(NET_E_SHAPE, "grid %dx%d beyond the %d boxes set up for", gh, gw, R.maxc);
    CK(cudaSetDevice(n->device));
    CK(enqueue_region(R, d_map, batch, gh, gw, d_counts, d_det, n->stream, &n->launches));
    return NET_OK;
}

extern "C" net_status net_forward_detect(net_t* n, const float* in, int batch, int h, int w, int* counts,
                                         net_detection* det) {
    if (!n || !in || !counts || !det) return fail(NET_E_INVAL, "NULL argument");
    if (!n->weights_loaded) return fail(NET_E_WEIGHTS, "weights not loaded");
    if (!n->region) return fail(NET_E_STATE, "no region set (net_set_region)");
    net_status s = check_shape(n, batch, h, w);
    if (s != NET_OK) return s;
    const RegionState& R = *n->region;
    int c, gh, gw;
    net_output_shape(n, h, w, &c, &gh, &gw);
    CK(cudaSetDevice(n->device));
    const size_t nin = (size_t)batch * n->in_c * h * w;
    CK(cudaMemcpyAsync(n->d_in_stage, in, nin * sizeof(float), cudaMemcpyHostToDevice, n->stream));
    s = run_forward(n, n->d_in_stage, batch, h, w, n->d_out_stage);
    if (s != NET_OK) return s;
    int* d_counts = static_cast<int*>(R.d_out);
    net_detection* d_det =
        reinterpret_cast<net_detection*>(static_cast<unsigned char*>(R.d_out) + counts_block(R.max_batch));
    CK(enqueue_region(R, n->d_out_stage, batch, gh, gw, d_counts, d_det, n->stream, &n->launches));
    // one device->host copy: the counts block and the frames' detection rows
    const size_t bytes = counts_block(R.max_batch) + (size_t)batch * R.r.max_det * sizeof(net_detection);
    CK(cudaMemcpyAsync(R.h_out, R.d_out, bytes, cudaMemcpyDeviceToHost, n->stream));
    CK(cudaStreamSynchronize(n->stream));
    std::memcpy(counts, R.h_out, sizeof(int) * batch);
    std::memcpy(det, static_cast<unsigned char*>(R.h_out) + counts_block(R.max_batch),
                (size_t)batch * R.r.max_det * sizeof(net_detection));
    return check_device_error(n);
}
