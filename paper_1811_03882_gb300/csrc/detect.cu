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
// Three kernels, all FP32: decode (one thread per box, threads along grid
// columns so that each channel is read contiguously; up to 32 class logits
// in registers) appends candidates to per-(frame, class) lists; NMS (one CTA
// per (frame, class)) sorts its list in shared memory by a 64-bit key
// (inverted score bits, id), so the result does not depend on the order the
// atomics appended in, and suppresses in blocks of 32 candidates (a warp
// settles a block, the CTA applies its kept boxes to the rest: one barrier
// per block, the decisions of one-at-a-time greedy NMS); compaction (one
// warp per frame) concatenates the classes' kept boxes.
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
    int* d_cnt = nullptr;       // [max_batch][C] candidates, then kept, per (frame, class)
    RegionCand* d_cand = nullptr;   // [max_batch][C][maxc]
    float* d_anchor = nullptr;  // [2A]
    void* d_out = nullptr;      // forward_detect: [counts (max_batch ints, 256-byte block)][dets]
    void* h_out = nullptr;      // pinned host copy of d_out
    size_t out_bytes = 0;
};

void region_free(net* n) {
    RegionState* R = n->region;
    if (!R) return;
    cudaFree(R->d_cnt);
    cudaFree(R->d_cand);
    cudaFree(R->d_anchor);
    cudaFree(R->d_out);
    cudaFreeHost(R->h_out);
    delete R;
    n->region = nullptr;
}

}  // namespace dn

namespace {

constexpr int kMaxCand = 4096;   // candidate slots per (frame, class): the NMS sort's shared-memory bound
constexpr int kNmsThreads = 256;

__device__ __forceinline__ float sigm(float v) { return 1.f / (1.f + expf(-v)); }

__global__ void region_decode_kernel(const float* __restrict__ map, int batch, int A, int C, int GH, int GW,
                                     const float* __restrict__ anchor, float thresh, int maxc, int* cnt,
                                     RegionCand* cand) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)batch * A * GH * GW;
    if (t >= total) return;
    // thread order (frame, anchor, row, column): consecutive threads read
    // consecutive columns of each channel
    const int j = (int)(t % GW);
    long long r = t / GW;
    const int i = (int)(r % GH);
    r /= GH;
    const int a = (int)(r % A);
    const int f = (int)(r / A);
    const long long plane = (long long)GH * GW;
    const float* p = map + ((long long)f * A * (5 + C) + (long long)a * (5 + C)) * plane + (long long)i * GW + j;
    const float x = ((float)j + sigm(p[0])) / (float)GW;
    const float y = ((float)i + sigm(p[plane])) / (float)GH;
    const float w = expf(p[2 * plane]) * anchor[2 * a] / (float)GW;
    const float h = expf(p[3 * plane]) * anchor[2 * a + 1] / (float)GH;
    const float obj = sigm(p[4 * plane]);
    const float* lg = p + 5 * plane;
    const int id = (i * GW + j) * A + a;
    auto append = [&](int c, float s) {
        if (s > thresh) {
            const int slot = atomicAdd(&cnt[f * C + c], 1);
            if (slot < maxc) {
                RegionCand q;
                q.score = s;
                q.id = id;
                q.x = x;
                q.y = y;
                q.w = w;
                q.h = h;
                q.pad0 = q.pad1 = 0;
                cand[((long long)f * C + c) * maxc + slot] = q;
            }
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
#pragma unroll
        for (int c = 0; c < 32; ++c)
            if (c < C) append(c, obj * (e[c] / sum));
    } else {
        float m = lg[0];
        for (int c = 1; c < C; ++c) m = fmaxf(m, lg[c * plane]);
        float sum = 0.f;
        for (int c = 0; c < C; ++c) sum += expf(lg[c * plane] - m);
        for (int c = 0; c < C; ++c) append(c, obj * (expf(lg[c * plane] - m) / sum));
    }
}

__device__ __forceinline__ float iou_f(float4 a, float4 b) {
    const float al = a.x - a.z * 0.5f, ar = a.x + a.z * 0.5f, at = a.y - a.w * 0.5f, ab = a.y + a.w * 0.5f;
    const float bl = b.x - b.z * 0.5f, br = b.x + b.z * 0.5f, bt = b.y - b.w * 0.5f, bb = b.y + b.w * 0.5f;
    const float iw = fminf(ar, br) - fmaxf(al, bl);
    const float ih = fminf(ab, bb) - fmaxf(at, bt);
    const float inter = fmaxf(iw, 0.f) * fmaxf(ih, 0.f);
    const float uni = a.z * a.w + b.z * b.w - inter;
    return uni > 0.f ? inter / uni : 0.f;
}

// One CTA per (frame, class): sort the class's candidates by (score
// descending, id ascending), suppress greedily, write the kept ones back to
// the front of the list in rank order and their count to cnt.
__global__ void __launch_bounds__(kNmsThreads) region_nms_kernel(int C, int maxc, float iou_thr, int* cnt,
                                                                 RegionCand* cand) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int fc = blockIdx.x;
    const int n = min(cnt[fc], maxc);
    RegionCand* L = cand + (long long)fc * maxc;
    int np2 = 1;
    while (np2 < n) np2 <<= 1;
    unsigned long long* key = reinterpret_cast<unsigned long long*>(sm);
    float4* box = reinterpret_cast<float4*>(sm + (size_t)kMaxCand * 8);
    float* sc = reinterpret_cast<float*>(sm + (size_t)kMaxCand * 24);
    int* ids = reinterpret_cast<int*>(sm + (size_t)kMaxCand * 28);
    unsigned char* supp = sm + (size_t)kMaxCand * 32;
    // key: inverted score bits (scores are positive, so larger scores have
    // larger bits), then the id (unique within a class, 12 bits), then the
    // slot (12 bits, carried along)
    for (int q = threadIdx.x; q < np2; q += blockDim.x) {
        if (q < n) {
            const unsigned s = __float_as_uint(L[q].score);
            key[q] = ((unsigned long long)(0xFFFFFFFFu - s) << 32) | ((unsigned long long)L[q].id << 12) | (unsigned)q;
        } else {
            key[q] = ~0ull;
        }
    }
    __syncthreads();
    for (int k = 2; k <= np2; k <<= 1) {   // bitonic sort, ascending
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int q = threadIdx.x; q < np2; q += blockDim.x) {
                const int o = q ^ jj;
                if (o > q) {
                    const bool up = (q & k) == 0;
                    const unsigned long long kq = key[q], ko = key[o];
                    if ((kq > ko) == up) {
                        key[q] = ko;
                        key[o] = kq;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int r = threadIdx.x; r < n; r += blockDim.x) {   // gather in rank order
        const RegionCand& e = L[(int)(key[r] & 0xFFFu)];
        box[r] = make_float4(e.x, e.y, e.w, e.h);
        sc[r] = e.score;
        ids[r] = e.id;
        supp[r] = 0;
    }
    __syncthreads();
    // greedy suppression in blocks of 32 candidates: warp 0 settles a block
    // among itself (lane l = candidate r0 + l; in rank order each candidate
    // still alive is kept and drops the later ones it overlaps), then the
    // whole CTA drops every later candidate a kept one of the block overlaps.
    // The same decisions as one candidate at a time, one barrier per block.
    __shared__ unsigned kept_mask;
    for (int r0 = 0; r0 < n; r0 += 32) {
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x, r = r0 + lane;
            bool alive = r < n && !supp[r];
            const float4 mine = r < n ? box[r] : make_float4(0.f, 0.f, 0.f, 0.f);
            for (int i = 0; i < 32; ++i) {
                const bool ai = __shfl_sync(0xffffffffu, alive, i);
                if (!ai) continue;   // uniform across the warp
                const float4 bi = make_float4(__shfl_sync(0xffffffffu, mine.x, i), __shfl_sync(0xffffffffu, mine.y, i),
                                              __shfl_sync(0xffffffffu, mine.z, i), __shfl_sync(0xffffffffu, mine.w, i));
                if (lane > i && alive && iou_f(bi, mine) > iou_thr) alive = false;
            }
            const unsigned m = __ballot_sync(0xffffffffu, alive);
            if (r < n) supp[r] = alive ? 0 : 1;
            if (lane == 0) kept_mask = m;
        }
        __syncthreads();
        const unsigned m = kept_mask;
        for (int q = r0 + 32 + threadIdx.x; q < n; q += blockDim.x) {
            if (supp[q]) continue;
            const float4 bq = box[q];
            for (unsigned mm = m; mm; mm &= mm - 1) {
                if (iou_f(box[r0 + __ffs(mm) - 1], bq) > iou_thr) {
                    supp[q] = 1;
                    break;
                }
            }
        }
        __syncthreads();
    }
    // kept ones to the front of the list, in rank order (warp 0, ballots)
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int out = 0;
        for (int r0 = 0; r0 < n; r0 += 32) {
            const int r = r0 + lane;
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
        if (lane == 0) cnt[fc] = out;
    }
}

// One warp per frame: the classes' kept boxes, class by class, cut at max_det.
__global__ void region_compact_kernel(int batch, int C, int maxc, int max_det, const int* __restrict__ cnt,
                                      const RegionCand* __restrict__ cand, int* counts, net_detection* det) {
    const int f = blockIdx.x;
    if (f >= batch) return;
    const int lane = threadIdx.x;
    int base = 0;
    for (int c = 0; c < C; ++c) {
        const int k = cnt[f * C + c];
        const RegionCand* L = cand + ((long long)f * C + c) * maxc;
        for (int q = lane; q < k && base + q < max_det; q += 32) {
            net_detection d;
            d.x = L[q].x;
            d.y = L[q].y;
            d.w = L[q].w;
            d.h = L[q].h;
            d.score = L[q].score;
            d.cls = c;
            d.id = L[q].id;
            d.pad = 0;
            det[(long long)f * max_det + base + q] = d;
        }
        base += k;
    }
    if (lane == 0) counts[f] = base;
}

size_t nms_smem() { return (size_t)kMaxCand * 33; }

cudaError_t enqueue_region(const RegionState& R, const float* d_map, int batch, int GH, int GW, int* d_counts,
                           net_detection* d_det, cudaStream_t st, uint64_t* launches) {
    const int A = R.r.n_anchors, C = R.r.n_classes;
    cudaError_t e = cudaMemsetAsync(R.d_cnt, 0, sizeof(int) * (size_t)batch * C, st);
    if (e != cudaSuccess) return e;
    const long long total = (long long)batch * A * GH * GW;
    region_decode_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
        d_map, batch, A, C, GH, GW, R.d_anchor, R.r.score_thresh, R.maxc, R.d_cnt, R.d_cand);
    static bool attr = false;
    if (!attr) {
        e = cudaFuncSetAttribute(region_nms_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)nms_smem());
        if (e != cudaSuccess) return e;
        attr = true;
    }
    region_nms_kernel<<<batch * C, kNmsThreads, nms_smem(), st>>>(C, R.maxc, R.r.nms_iou, R.d_cnt, R.d_cand);
    region_compact_kernel<<<batch, 32, 0, st>>>(batch, C, R.maxc, R.r.max_det, R.d_cnt, R.d_cand, d_counts, d_det);
    *launches += 3;
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
    CK(cudaMalloc(&R->d_cnt, sizeof(int) * (size_t)n->max_batch * C));
    CK(cudaMalloc(&R->d_cand, sizeof(RegionCand) * (size_t)n->max_batch * C * R->maxc));
    CK(cudaMalloc(&R->d_anchor, sizeof(float) * 2 * A));
    CK(cudaMalloc(&R->d_out, R->out_bytes));
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
