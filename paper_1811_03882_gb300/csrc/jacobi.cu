// jacobi.cu — Jacobi solver of the Laplace equation, device-resident.
//
// Paper Sec. 4 reports a 13.5x speed-up of a sample application that solves
// the Laplace equation by the Jacobi method; its data-transfer rule
// (Sec. 3.2) is applied in full: the grid crosses to the device once, every
// sweep reads and writes device memory only, and the result crosses back
// once.  One sweep replaces each interior point of the ny x nx grid by the
// mean of its four neighbours in the previous iterate (the first and last
// rows and columns are fixed boundary values); sweeps repeat while the
// largest change of an interior point exceeds tol and fewer than iter_max
// sweeps have run.
//
// Device side, FP32, memory-bound (8 bytes of DRAM traffic per point and
// sweep at best: one read, one write):
//  * jacobi_sweep_kernel: persistent grid (a multiple of the SM count), each
//    work tile a strip of R rows x 4*blockDim columns; a thread owns four
//    adjacent columns and walks down the strip keeping the rows above, at
//    and below in registers (each input row is read once per strip) and the
//    next six rows in flight by cp.async into a per-thread shared-memory ring
//    (bytes in flight, not instructions, bound a streaming kernel; the ring
//    takes no registers), the left and right neighbours coming from the
//    adjacent lanes by shuffles; sixteen 128-thread blocks per SM.
//    Each block writes its largest change to a partial slot; the last block
//    to finish (an arrival counter) reduces the partials and applies the
//    stopping rule on the device: sweeps += 1, done when the change is at or
//    below tol or sweeps reached iter_max.  The kernel returns at once when
//    done is set, so the host can queue sweeps ahead and poll the 16-byte
//    state only every few of them.
//  * Strips of 64 rows (fewer halo rows re-read than shorter strips; measured
//    faster at 8192 x 8192 than strips sized to give every resident block
//    exactly one tile).
//  * jacobi_sweep2_kernel: two sweeps in one pass (temporal blocking), the
//    default: the grid is read and written once per pair, eight blocks an
//    SM, strips of 128 rows; a pair whose first sweep meets the stopping
//    rule is discarded and redone by the single-sweep kernel (the fix-up
//    launch at the end of each graph).  Both give the same bits.
//  * The state records which buffer holds the current iterate.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <utility>

#include "../../include/net.h"
#include "common.cuh"
#include "net_internal.h"

using namespace dn;

namespace {

struct JState {
    int sweeps;
    int done;
    float change;
    unsigned arrived;   // blocks of the running launch that are done (the last resets it)
    int cur;            // buffer holding the current iterate
    int fix;            // a fused pair stopped after its first sweep: the fix-up sweep redoes it
};

constexpr int kThreads = 128;   // 512 columns per tile row
constexpr int kAhead = 6;       // rows in flight ahead of the one being computed (per thread, cp.async ring)
constexpr int kChunk = 16;      // sweeps per captured graph (even: buffer parity is kept per chunk)

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* src, bool in) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
                 "l"(src), "r"(in ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// 16 blocks of 128 threads an SM.  The rows below the one being computed
// stream into a per-thread ring of kAhead 16-byte slots in shared memory by
// cp.async (zero-filled past the strip), so the bytes in flight (~196 KB an
// SM) take no registers; each thread reads only its own slots, so no block
// barrier is needed, only the wait for its own oldest copy group.
__global__ void __launch_bounds__(kThreads, 16) jacobi_sweep_kernel(float* b0, float* b1, int ny, int nx, int P,
                                                                     JState* st, float* partial, float tol,
                                                                     int iter_max, int col_blocks, int strips,
                                                                     int rows, int fixup) {
    __shared__ float4 ring[kAhead][kThreads];
    // fixup = 1: runs only after a fused pair whose first sweep met the
    // stopping rule (the pair's second sweep is discarded)
    if (fixup ? !st->fix : st->done) return;
    const int k = st->sweeps;
    const float* src = st->cur ? b1 : b0;
    float* dst = st->cur ? b0 : b1;
    const int lane = threadIdx.x & 31;
    float best = 0.f;
    const int tiles = col_blocks * strips;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int cb = tile % col_blocks, sb = tile / col_blocks;
        const int x0 = (cb * kThreads + threadIdx.x) * 4;   // first of this thread's four columns
        const bool inb = x0 < P;                             // inside the pitched row
        const int y0 = 1 + sb * rows, y1 = min(y0 + rows, ny - 1);
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 up = inb ? ld4(src + (size_t)(y0 - 1) * P + x0) : z4;
        float4 cur = inb ? ld4(src + (size_t)y0 * P + x0) : z4;
        // slot q holds row y0 + 1 + q, then every kAhead rows further down
#pragma unroll
        for (int q = 0; q < kAhead; ++q) {
            const int yy = y0 + 1 + q;
            const bool ok = inb && yy <= y1;
            cp_async16(&ring[q][threadIdx.x], src + (size_t)(ok ? yy : 0) * P + (ok ? x0 : 0), ok);
            cp_async_commit();
        }
        int slot = 0;
        for (int y = y0; y < y1; ++y) {   // uniform over the block
            cp_async_wait<kAhead - 1>();   // the oldest group: row y + 1
            const float4 dn = ring[slot][threadIdx.x];
            float left = __shfl_up_sync(0xffffffffu, cur.w, 1);
            float right = __shfl_down_sync(0xffffffffu, cur.x, 1);
            if (lane == 0) left = (inb && x0 > 0) ? src[(size_t)y * P + x0 - 1] : 0.f;
            if (lane == 31) right = (x0 + 4 < P) ? src[(size_t)y * P + x0 + 4] : 0.f;
            float4 nw;
            nw.x = 0.25f * ((up.x + dn.x) + (left + cur.y));
            nw.y = 0.25f * ((up.y + dn.y) + (cur.x + cur.z));
            nw.z = 0.25f * ((up.z + dn.z) + (cur.y + cur.w));
            nw.w = 0.25f * ((up.w + dn.w) + (cur.z + right));
            // interior columns 1 .. nx - 2 take the new value; the boundary and
            // the pitch padding keep theirs
            const float c4[4] = {cur.x, cur.y, cur.z, cur.w};
            float n4[4] = {nw.x, nw.y, nw.z, nw.w};
#pragma unroll
            for (int k4 = 0; k4 < 4; ++k4) {
                const int x = x0 + k4;
                if (x >= 1 && x <= nx - 2) best = fmaxf(best, fabsf(n4[k4] - c4[k4]));
                else n4[k4] = c4[k4];
            }
            if (inb) *reinterpret_cast<float4*>(dst + (size_t)y * P + x0) = make_float4(n4[0], n4[1], n4[2], n4[3]);
            {
                // refill the slot (its row is consumed: nw depends on it) with the
                // row kAhead further down
                const int yy = y + 1 + kAhead;
                const bool ok = inb && yy <= y1;
                cp_async16(&ring[slot][threadIdx.x], src + (size_t)(ok ? yy : 0) * P + (ok ? x0 : 0), ok);
                cp_async_commit();
            }
            slot = slot + 1 == kAhead ? 0 : slot + 1;
            up = cur;
            cur = dn;
        }
        cp_async_wait<0>();   // no copy of this strip outlives it (slots are reused by the next)
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
    __shared__ float wmax[kThreads / 32];
    __shared__ int last;
    if (lane == 0) wmax[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = wmax[0];
        for (int w = 1; w < kThreads / 32; ++w) m = fmaxf(m, wmax[w]);
        partial[blockIdx.x] = m;
        __threadfence();   // the partial before the arrival
        // every other block read the state at its start before arriving, so
        // the last one may update it
        last = atomicAdd(&st->arrived, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    float m = 0.f;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kThreads) m = fmaxf(m, __ldcg(&partial[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __syncthreads();
    if (lane == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 0; w < kThreads / 32; ++w) m = fmaxf(m, wmax[w]);
        st->change = m;
        st->sweeps = k + 1;
        st->cur ^= 1;
        st->arrived = 0;
        if (m <= tol || k + 1 >= iter_max || fixup) st->done = 1;
        st->fix = 0;
    }
}

// Two sweeps in one pass over the grid (temporal blocking): each thread
// walks down its strip computing the first sweep's values A for rows y0 - 1
// .. y1 (one halo row each side, recomputed by the neighbouring strips too)
// from the source rows streamed in, and from three consecutive A rows the
// second sweep's values B for rows y0 .. y1 - 1, which it stores.  A's
// left and right neighbours come from the adjacent lanes; the warp's edge
// lanes compute the A value one column beyond their warp themselves (two
// extra loads a row).  Every value is the expression the single sweep
// computes, so the pair gives the two sweeps' bits.  Both sweeps' largest
// changes are reduced; the last block applies the stopping rule to the
// first, then the second: if the first sweep already meets it, the pair's
// result is discarded (the current buffer is untouched) and the fix-up sweep
// redoes that one sweep.  Eight blocks of 128 threads an SM, twelve rows in
// flight a thread.
constexpr int kAhead2 = 12;
__global__ void __launch_bounds__(kThreads, 8) jacobi_sweep2_kernel(float* b0, float* b1, int ny, int nx, int P,
                                                                    JState* st, float* partial, float tol,
                                                                    int iter_max, int col_blocks, int strips,
                                                                    int rows) {
    __shared__ float4 ring[kAhead2][kThreads];
    // the 16 bytes beyond each warp's columns (left of lane 0, right of lane
    // 31), streamed with the rows: [slot][warp][side]
    __shared__ float4 halo[kAhead2][kThreads / 32][2];
    if (st->done) return;
    const int k = st->sweeps;
    const float* src = st->cur ? b1 : b0;
    float* dst = st->cur ? b0 : b1;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float best1 = 0.f, best2 = 0.f;
    const int tiles = col_blocks * strips;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    auto interior_x = [&](int x) { return x >= 1 && x <= nx - 2; };
    const bool edge_lane = lane == 0 || lane == 31;
    const int side = lane == 0 ? 0 : 1;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int cb = tile % col_blocks, sb = tile / col_blocks;
        const int x0 = (cb * kThreads + threadIdx.x) * 4;   // first of this thread's four columns
        const bool inb = x0 < P;
        const int y0 = 1 + sb * rows, y1 = min(y0 + rows, ny - 1);   // B rows [y0, y1)
        // the edge lanes' halo chunk: columns x0 - 4 .. x0 - 1 (lane 0) or
        // x0 + 4 .. x0 + 7 (lane 31), zero outside the pitched row
        const int xh = lane == 0 ? x0 - 4 : x0 + 4;
        const bool hin = edge_lane && inb && xh >= 0 && xh < P;
        auto ldh = [&](int y) { return (hin && y >= 0) ? ld4(src + (size_t)y * P + xh) : z4; };
        // source rows a - 1, a, a + 1 around A row a = y0 - 1 (row -1 is never read)
        float4 sup = (inb && y0 >= 2) ? ld4(src + (size_t)(y0 - 2) * P + x0) : z4;
        float4 scur = inb ? ld4(src + (size_t)(y0 - 1) * P + x0) : z4;
        float4 sdn = inb ? ld4(src + (size_t)y0 * P + x0) : z4;
        float4 hup = ldh(y0 - 2), hcur = ldh(y0 - 1), hdn = ldh(y0);
        // ring slot q holds source row y0 + 1 + q, then every kAhead2 rows
        // further down, up to row y1 + 1 (the last A row's lower neighbour)
        const int ylast = min(y1 + 1, ny - 1);
        // row pointers advanced one row per copy (out-of-range copies read
        // nothing: zero fill from the row's own start)
        const float* rp = src + (size_t)(y0 + 1) * P + (inb ? x0 : 0);
        const float* hp = src + (size_t)(y0 + 1) * P + (hin ? xh : 0);
        int yy = y0 + 1;
        auto issue = [&](int q) {
            const bool ok = inb && yy <= ylast;
            cp_async16(&ring[q][threadIdx.x], ok ? rp : src, ok);
            if (edge_lane) cp_async16(&halo[q][wid][side], (hin && yy <= ylast) ? hp : src, hin && yy <= ylast);
            cp_async_commit();
            rp += P;
            hp += P;
            ++yy;
        };
#pragma unroll
        for (int q = 0; q < kAhead2; ++q) issue(q);
        // interior columns of this thread's four and of the edge column
        bool cin[4];
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4) cin[k4] = interior_x(x0 + k4);
        const bool ein = edge_lane && interior_x(lane == 0 ? x0 - 1 : x0 + 4);
        float4 a2 = z4, a1 = z4;        // A rows a - 2, a - 1
        float e1 = 0.f;                 // A row a - 1 at the edge column
        int slot = 0;
        for (int a = y0 - 1; a <= y1; ++a) {   // uniform over the block
            // the edge column and the one beyond it, rows a - 1, a, a + 1
            const float eup = lane == 0 ? hup.w : hup.x, ecur = lane == 0 ? hcur.w : hcur.x;
            const float edn = lane == 0 ? hdn.w : hdn.x, far = lane == 0 ? hcur.z : hcur.y;
            // ---- A row a (the first sweep): boundary rows and columns keep theirs
            float4 av;
            float ae;
            {
                float left = __shfl_up_sync(0xffffffffu, scur.w, 1);
                float right = __shfl_down_sync(0xffffffffu, scur.x, 1);
                if (lane == 0) left = ecur;
                if (lane == 31) right = ecur;
                const bool row_in = a >= 1 && a <= ny - 2;
                float4 nw;
                nw.x = 0.25f * ((sup.x + sdn.x) + (left + scur.y));
                nw.y = 0.25f * ((sup.y + sdn.y) + (scur.x + scur.z));
                nw.z = 0.25f * ((sup.z + sdn.z) + (scur.y + scur.w));
                nw.w = 0.25f * ((sup.w + sdn.w) + (scur.z + right));
                const float c4[4] = {scur.x, scur.y, scur.z, scur.w};
                float n4[4] = {nw.x, nw.y, nw.z, nw.w};
#pragma unroll
                for (int k4 = 0; k4 < 4; ++k4) {
                    if (row_in && cin[k4]) best1 = fmaxf(best1, fabsf(n4[k4] - c4[k4]));
                    else n4[k4] = c4[k4];
                }
                av = make_float4(n4[0], n4[1], n4[2], n4[3]);
                // the edge column's A value, as its owner (the neighbouring
                // warp's edge lane) computes it: its outer source neighbour is
                // `far`, its inner one this thread's first or last column
                ae = ecur;
                if (row_in && ein) {
                    const float near = lane == 0 ? scur.x : scur.w;
                    ae = lane == 0 ? 0.25f * ((eup + edn) + (far + near)) : 0.25f * ((eup + edn) + (near + far));
                }
            }
            // ---- B row a - 1 (the second sweep) from A rows a - 2, a - 1, a
            if (a >= y0 + 1) {
                const int y = a - 1;
                float left = __shfl_up_sync(0xffffffffu, a1.w, 1);
                float right = __shfl_down_sync(0xffffffffu, a1.x, 1);
                if (lane == 0) left = e1;
                if (lane == 31) right = e1;
                float4 nw;
                nw.x = 0.25f * ((a2.x + av.x) + (left + a1.y));
                nw.y = 0.25f * ((a2.y + av.y) + (a1.x + a1.z));
                nw.z = 0.25f * ((a2.z + av.z) + (a1.y + a1.w));
                nw.w = 0.25f * ((a2.w + av.w) + (a1.z + right));
                const float c4[4] = {a1.x, a1.y, a1.z, a1.w};
                float n4[4] = {nw.x, nw.y, nw.z, nw.w};
#pragma unroll
                for (int k4 = 0; k4 < 4; ++k4) {
                    if (cin[k4]) best2 = fmaxf(best2, fabsf(n4[k4] - c4[k4]));
                    else n4[k4] = c4[k4];
                }
                if (inb) *reinterpret_cast<float4*>(dst + (size_t)y * P + x0) = make_float4(n4[0], n4[1], n4[2], n4[3]);
            }
            a2 = a1;
            a1 = av;
            e1 = ae;
            if (a == y1) break;
            // ---- the next source row (a + 2) from the ring, which gets row a + 2 + kAhead2
            cp_async_wait<kAhead2 - 1>();
            const float4 nx4 = ring[slot][threadIdx.x];
            const float4 nh4 = edge_lane ? halo[slot][wid][side] : z4;
            issue(slot);   // row a + 2 + kAhead2
            slot = slot + 1 == kAhead2 ? 0 : slot + 1;
            sup = scur;
            scur = sdn;
            sdn = nx4;
            hup = hcur;
            hcur = hdn;
            hdn = nh4;
        }
        cp_async_wait<0>();   // no copy of this strip outlives it (slots are reused by the next)
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        best1 = fmaxf(best1, __shfl_xor_sync(0xffffffffu, best1, o));
        best2 = fmaxf(best2, __shfl_xor_sync(0xffffffffu, best2, o));
    }
    __shared__ float wmax[2][kThreads / 32];
    __shared__ int last;
    if (lane == 0) {
        wmax[0][threadIdx.x >> 5] = best1;
        wmax[1][threadIdx.x >> 5] = best2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float m1 = wmax[0][0], m2 = wmax[1][0];
        for (int w = 1; w < kThreads / 32; ++w) {
            m1 = fmaxf(m1, wmax[0][w]);
            m2 = fmaxf(m2, wmax[1][w]);
        }
        partial[2 * blockIdx.x] = m1;
        partial[2 * blockIdx.x + 1] = m2;
        __threadfence();   // the partials before the arrival
        last = atomicAdd(&st->arrived, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    float m1 = 0.f, m2 = 0.f;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kThreads) {
        m1 = fmaxf(m1, __ldcg(&partial[2 * i]));
        m2 = fmaxf(m2, __ldcg(&partial[2 * i + 1]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        m2 = fmaxf(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    }
    __syncthreads();
    if (lane == 0) {
        wmax[0][threadIdx.x >> 5] = m1;
        wmax[1][threadIdx.x >> 5] = m2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 0; w < kThreads / 32; ++w) {
            m1 = fmaxf(m1, wmax[0][w]);
            m2 = fmaxf(m2, wmax[1][w]);
        }
        st->arrived = 0;
        if (m1 <= tol || k + 1 >= iter_max) {
            // stop after the pair's first sweep: the fix-up sweep recomputes it
            st->change = m1;
            st->fix = 1;
            st->done = 1;
        } else {
            st->change = m2;
            st->sweeps = k + 2;
            st->cur ^= 1;
            if (m2 <= tol || k + 2 >= iter_max) st->done = 1;
        }
    }
}

}  // namespace

struct net_jacobi {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int ny = 0, nx = 0, P = 0;        // grid and row pitch (floats, multiple of 4)
    float* buf[2] = {nullptr, nullptr};
    float* partial = nullptr;
    JState* d_state = nullptr;
    JState* h_state = nullptr;        // pinned, two slots (chunks in flight)
    int grid = 0, col_blocks = 0, strips = 0, rows = 0;
    int grid2 = 0, strips2 = 0, rows2 = 0;   // the two-sweep kernel: blocks (eight an SM), strips
    bool fuse = true;                 // sweeps in fused pairs (NET_JACOBI_FUSE=0: one a launch)
    std::map<std::pair<float, int>, cudaGraphExec_t> graphs;   // per (tol, iter_max)
    uint64_t launches = 0;
};

#define JK(call)                                                                                      \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return fail(e_ == cudaErrorMemoryAllocation ? NET_E_OOM : NET_E_CUDA, "%s: %s", #call,   \
                        cudaGetErrorString(e_));                                                      \
    } while (0)

static net_status jacobi_graph(net_jacobi* j, float tol, int iter_max, cudaGraphExec_t* out) {
    auto key = std::make_pair(tol, iter_max);
    auto it = j->graphs.find(key);
    if (it != j->graphs.end()) {
        *out = it->second;
        return NET_OK;
    }
    cudaGraph_t g = nullptr;
    JK(cudaStreamBeginCapture(j->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    if (j->fuse) {
        // kChunk sweeps: kChunk / 2 fused pairs, then the fix-up sweep (it
        // returns at once unless a pair stopped after its first sweep)
        for (int s = 0; s < kChunk / 2 && e == cudaSuccess; ++s) {
            jacobi_sweep2_kernel<<<j->grid2, kThreads, 0, j->stream>>>(j->buf[0], j->buf[1], j->ny, j->nx, j->P,
                                                                       j->d_state, j->partial, tol, iter_max,
                                                                       j->col_blocks, j->strips2, j->rows2);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            jacobi_sweep_kernel<<<j->grid, kThreads, 0, j->stream>>>(j->buf[0], j->buf[1], j->ny, j->nx, j->P,
                                                                     j->d_state, j->partial, tol, iter_max,
                                                                     j->col_blocks, j->strips, j->rows, 1);
            e = cudaGetLastError();
        }
    } else {
        for (int s = 0; s < kChunk && e == cudaSuccess; ++s) {
            jacobi_sweep_kernel<<<j->grid, kThreads, 0, j->stream>>>(j->buf[0], j->buf[1], j->ny, j->nx, j->P,
                                                                     j->d_state, j->partial, tol, iter_max,
                                                                     j->col_blocks, j->strips, j->rows, 0);
            e = cudaGetLastError();
        }
    }
    cudaError_t e2 = cudaStreamEndCapture(j->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(NET_E_CUDA, "jacobi capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(NET_E_CUDA, "jacobi graph: %s", cudaGetErrorString(e));
    if (j->graphs.size() >= 16) {
        for (auto& kv : j->graphs) cudaGraphExecDestroy(kv.second);
        j->graphs.clear();
    }
    j->graphs[key] = ex;
    *out = ex;
    return NET_OK;
}

extern "C" net_status net_jacobi_create(int ny, int nx, int device, void* cuda_stream, net_jacobi_t** out) {
    if (!out) return fail(NET_E_INVAL, "NULL argument");
    *out = nullptr;
    if (ny < 3 || nx < 3 || ny > 65536 || nx > 65536)
        return fail(NET_E_INVAL, "grid %d x %d: each side must be in [3, 65536] (a grid needs an interior)", ny, nx);
    net_jacobi* j = new net_jacobi();
    j->device = device;
    j->ny = ny;
    j->nx = nx;
    j->P = rup(nx, 4);
    auto bail = [&](net_status s) {
        net_jacobi_free(j);
        return s;
    };
    if (cudaSetDevice(device) != cudaSuccess) return bail(fail(NET_E_CUDA, "cudaSetDevice(%d)", device));
    if (cuda_stream) {
        j->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreate(&j->stream) != cudaSuccess) return bail(fail(NET_E_CUDA, "stream"));
        j->own_stream = true;
    }
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    // persistent: sixteen 128-thread blocks per SM (all resident: 32 registers
    // a thread, 12 KB of shared memory a block) taking strips of 64 rows
    // round robin (NET_JACOBI_ROWS overrides the strip height)
    j->col_blocks = cdiv(j->P, 4 * kThreads);
    j->rows = 64;
    if (const char* v = getenv("NET_JACOBI_ROWS"))
        if (atoi(v) > 0) j->rows = atoi(v);
    j->strips = cdiv(ny - 2, j->rows);
    j->grid = std::max(1, std::min(j->col_blocks * j->strips, 16 * sms));
    // the two-sweep kernel: strips of 128 rows (measured at 8192 x 8192: 0.0613
    // ms a sweep against 0.0656 with 64 rows and 0.0651 with 32)
    j->rows2 = 128;
    if (const char* v = getenv("NET_JACOBI_ROWS"))
        if (atoi(v) > 0) j->rows2 = atoi(v);
    j->strips2 = cdiv(ny - 2, j->rows2);
    j->grid2 = std::max(1, std::min(j->col_blocks * j->strips2, 8 * sms));
    if (const char* v = getenv("NET_JACOBI_FUSE"))
        if (atoi(v) == 0) j->fuse = false;
    const size_t bytes = (size_t)ny * j->P * sizeof(float);
    for (int b = 0; b < 2; ++b) {
        cudaError_t e = dn::dalloc(&j->buf[b], bytes);
        if (e != cudaSuccess) return bail(fail(e == cudaErrorMemoryAllocation ? NET_E_OOM : NET_E_CUDA, "grid buffer"));
        cudaMemsetAsync(j->buf[b], 0, bytes, j->stream);
    }
    if (dn::dalloc(&j->partial, 2 * sizeof(float) * std::max(j->grid, j->grid2)) != cudaSuccess ||
        dn::dalloc(&j->d_state, sizeof(JState)) != cudaSuccess ||
        cudaHostAlloc(&j->h_state, 2 * sizeof(JState), cudaHostAllocDefault) != cudaSuccess)
        return bail(fail(NET_E_OOM, "jacobi state"));
    if (cudaStreamSynchronize(j->stream) != cudaSuccess) return bail(fail(NET_E_CUDA, "jacobi set-up"));
    *out = j;
    return NET_OK;
}

// Runs the sweeps on the handle's buffers after buf[0] and buf[1] hold the
// initial grid; result in buf[*cur].
static net_status jacobi_run(net_jacobi* j, float tol, int iter_max, int* sweeps, float* change, int* cur) {
    JState s0{0, iter_max <= 0 ? 1 : 0, 0.f, 0, 0, 0};
    JK(cudaMemcpyAsync(j->d_state, &s0, sizeof s0, cudaMemcpyHostToDevice, j->stream));
    if (iter_max > 0) {
        cudaGraphExec_t ex = nullptr;
        net_status s = jacobi_graph(j, tol, iter_max, &ex);
        if (s != NET_OK) return s;
        // two chunks in flight: the state of chunk c is read while chunk c + 1
        // runs (sweeps past convergence return at once)
        cudaEvent_t ev[2];
        JK(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
        JK(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
        const int chunks = cdiv(iter_max, kChunk);
        net_status st = NET_OK;
        for (int c = 0; c < chunks; ++c) {
            cudaError_t e = cudaGraphLaunch(ex, j->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&j->h_state[c & 1], j->d_state, sizeof(JState),
                                                      cudaMemcpyDeviceToHost, j->stream);
            if (e == cudaSuccess) e = cudaEventRecord(ev[c & 1], j->stream);
            if (e != cudaSuccess) {
                st = fail(NET_E_CUDA, "jacobi chunk: %s", cudaGetErrorString(e));
                break;
            }
            j->launches += j->fuse ? kChunk / 2 + 1 : kChunk;
            if (c > 0) {
                e = cudaEventSynchronize(ev[(c - 1) & 1]);
                if (e != cudaSuccess) {
                    st = fail(NET_E_CUDA, "jacobi: %s", cudaGetErrorString(e));
                    break;
                }
                if (j->h_state[(c - 1) & 1].done) break;
            }
        }
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        if (st != NET_OK) return st;
    }
    JK(cudaMemcpyAsync(&j->h_state[0], j->d_state, sizeof(JState), cudaMemcpyDeviceToHost, j->stream));
    JK(cudaStreamSynchronize(j->stream));
    if (sweeps) *sweeps = j->h_state[0].sweeps;
    if (change) *change = j->h_state[0].change;
    *cur = j->h_state[0].cur;
    return NET_OK;
}

extern "C" net_status net_jacobi_solve(net_jacobi_t* j, const float* grid_in, float tol, int iter_max,
                                       float* grid_out, int* sweeps, float* change) {
    if (!j || !grid_in || !grid_out) return fail(NET_E_INVAL, "NULL argument");
    if (!(tol >= 0.f) || iter_max < 0) return fail(NET_E_INVAL, "tol %g / iter_max %d", (double)tol, iter_max);
    JK(cudaSetDevice(j->device));
    const size_t row = (size_t)j->nx * sizeof(float), pitch = (size_t)j->P * sizeof(float);
    // one host->device copy; the second buffer takes the boundary by a device copy
    if (pitch == row)
        JK(cudaMemcpyAsync(j->buf[0], grid_in, row * j->ny, cudaMemcpyHostToDevice, j->stream));
    else
        JK(cudaMemcpy2DAsync(j->buf[0], pitch, grid_in, row, row, j->ny, cudaMemcpyHostToDevice, j->stream));
    JK(cudaMemcpyAsync(j->buf[1], j->buf[0], pitch * j->ny, cudaMemcpyDeviceToDevice, j->stream));
    int k = 0, cur = 0;
    net_status s = jacobi_run(j, tol, iter_max, &k, change, &cur);
    if (s != NET_OK) return s;
    if (sweeps) *sweeps = k;
    if (pitch == row)
        JK(cudaMemcpyAsync(grid_out, j->buf[cur], row * j->ny, cudaMemcpyDeviceToHost, j->stream));
    else
        JK(cudaMemcpy2DAsync(grid_out, row, j->buf[cur], pitch, row, j->ny, cudaMemcpyDeviceToHost, j->stream));
    JK(cudaStreamSynchronize(j->stream));
    return NET_OK;
}

extern "C" net_status net_jacobi_solve_device(net_jacobi_t* j, const float* d_in, float tol, int iter_max,
                                              float* d_out, int* sweeps, float* change) {
    if (!j || !d_in || !d_out) return fail(NET_E_INVAL, "NULL argument");
    if (!(tol >= 0.f) || iter_max < 0) return fail(NET_E_INVAL, "tol %g / iter_max %d", (double)tol, iter_max);
    JK(cudaSetDevice(j->device));
    const size_t row = (size_t)j->nx * sizeof(float), pitch = (size_t)j->P * sizeof(float);
    JK(cudaMemcpy2DAsync(j->buf[0], pitch, d_in, row, row, j->ny, cudaMemcpyDeviceToDevice, j->stream));
    JK(cudaMemcpyAsync(j->buf[1], j->buf[0], pitch * j->ny, cudaMemcpyDeviceToDevice, j->stream));
    int k = 0, cur = 0;
    net_status s = jacobi_run(j, tol, iter_max, &k, change, &cur);
    if (s != NET_OK) return s;
    if (sweeps) *sweeps = k;
    JK(cudaMemcpy2DAsync(d_out, row, j->buf[cur], pitch, row, j->ny, cudaMemcpyDeviceToDevice, j->stream));
    JK(cudaStreamSynchronize(j->stream));
    return NET_OK;
}

extern "C" net_status net_jacobi_launches(const net_jacobi_t* j, uint64_t* total) {
    if (!j || !total) return fail(NET_E_INVAL, "NULL argument");
    *total = j->launches;
    return NET_OK;
}

extern "C" net_status net_jacobi_free(net_jacobi_t* j) {
    if (!j) return NET_OK;
    cudaSetDevice(j->device);
    if (j->stream) cudaStreamSynchronize(j->stream);
    for (auto& kv : j->graphs) cudaGraphExecDestroy(kv.second);
    dn::dfree(j->buf[0]);
    dn::dfree(j->buf[1]);
    dn::dfree(j->partial);
    dn::dfree(j->d_state);
    if (j->h_state) cudaFreeHost(j->h_state);
    if (j->own_stream && j->stream) cudaStreamDestroy(j->stream);
    delete j;
    return NET_OK;
}
