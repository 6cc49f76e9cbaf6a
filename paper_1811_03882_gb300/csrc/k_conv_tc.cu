// k_conv_tc.cu — tensor-core implicit-GEMM convolution for sm_103a.
//
// y[n,i,j,o] = sum_{kh,kw,c} x[n, i+kh-p, j+kw-p, c] * W'[o, kh, kw, c]
// as a GEMM with M = output pixels, N = Cout, K = k*k*Cin: tcgen05.mma
// (BF16: kind::f16, FP8 E4M3: kind::f8f6f4) with FP32 accumulators in
// tensor memory, operands staged in shared memory by TMA.
//
// The A operand of one K step is one box of the NHWC activation: a TH x TW
// rectangle of pixels (TH*TW = 128 = the MMA's M) shifted by the tap
// (kh, kw), times one chunk of channels (32, 64 or 128 bytes, the swizzle
// width).  TMA's out-of-bounds zero fill supplies the convolution's zero
// padding, so no im2col buffer exists.  B is the matching [BN x chunk]
// box of the K-major weights [Cout][kh][kw][Cin].
//
// Persistent, warp-specialised CTA (one per SM, 384 threads):
//   warps 0,10 TMA producers (one lane each, alternate K steps) into a
//              shared-memory ring of nst stages (nst even).  A stage holds one
//              K step's A box and B box (A only when the weights are
//              resident); the ring is sized from the actual box bytes, since
//              a box takes ~2000 cycles to land under load and throughput is
//              stages in flight over that latency
//   warps 1,11 MMA issuers (one lane each, alternate tiles); warp 1 owns TMEM
//   warps 2-9  epilogue: two warpgroups, one per issuer's tiles:
//              tcgen05.ld, alpha/bias, leaky, 2x2 max via warp shuffles,
//              downcast, 16-byte stores
// Several TMEM accumulators (four up to BN = 128, else two) let the
// epilogue of one tile overlap the mainloop of the next; an accumulator is
// handed back as soon as its last live column is in registers.  Every
// mbarrier wait is bounded: on expiry the kernel records an error code,
// drains its TMA copies, frees TMEM and returns.
#include <cuda.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace dn {

namespace tc {

constexpr int THREADS = 384;   // producer, MMA issuer, 8 epilogue warps, second producer, second MMA issuer
constexpr int NUM_WARPS = THREADS / 32;
constexpr int kMaxStages = 32;                // ring stages (bit masks below are 32 bits)
constexpr int kEpiCols = 1024;                // bias / alpha columns kept in shared memory
constexpr long long WAIT_LIMIT = 4000000000LL;  // clock64 cycles (~2 s): bound of the drains, default of the waits

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// A waiting thread is suspended until the phase completes or the hint
// (1 ms) runs out, so waiters take no issue slots from the warps that share
// their SM sub-partition; the bounded waits below still re-check their
// clocks between suspensions.
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "n"(1000000)
        : "memory");
    return ok != 0;
}

// As mbar_try, acquiring at cluster scope: for barriers that threads of the
// peer CTA of a pair arrive on.
__device__ __forceinline__ bool mbar_try_cl(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "n"(1000000)
        : "memory");
    return ok != 0;
}

// Bounded wait; false (and the error code recorded) when `lim` clock64
// cycles passed or another role already aborted.  CL: cluster scope.
template <bool CL = false>
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          int* err, int code, long long lim) {
    auto tryw = [&] { return CL ? mbar_try_cl(bar, parity) : mbar_try(bar, parity); };
    if (tryw()) return true;
    const long long t0 = clock64();
    while (true) {
        if (tryw()) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > lim) {
            *abort_flag = 1;
            atomicExch(err, code);
            return false;
        }
    }
}

// Row-band dataflow between the layers of a pass: counters written by
// another kernel, polled with relaxed gpu-scope loads (several in flight; an
// acquire load would hold back the ones after it), then one acquire fence.
__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded wait until the whole previous kernel is done (*done >= done_target:
// *all_done is set, and later tiles need no wait) or the counters p[0 .. n -
// 1] all reach `target`, then the fences that order this thread's later
// reads, the TMA copies included, after what the counters announced.  False
// (and the code recorded) when `lim` clock64 cycles passed or another role
// already aborted.  done may be null.
__device__ __forceinline__ bool flags_wait(const int* p, int n, int target, const int* done, int done_target,
                                           bool* all_done, volatile int* abort_flag, int* err, int code,
                                           long long lim) {
    long long t0 = 0;
    bool timing = false;
    for (int i0 = 0; i0 < n;) {
        const int d = done ? ld_relaxed_gpu(done) : 0;
        int v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = i0 + j < n ? ld_relaxed_gpu(p + i0 + j) : target;
        if (done && d >= done_target) {
            *all_done = true;
            break;
        }
        int ready = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) ready += v[j] >= target ? 1 : 0;
        if (ready == 4) {
            i0 += 4;
            continue;
        }
        if (*abort_flag) return false;
        const long long now = clock64();
        if (!timing) {
            t0 = now;
            timing = true;
        } else if (now - t0 > lim) {
            *abort_flag = 1;
            atomicExch(err, code);
            return false;
        }
        __nanosleep(128);
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");
    return true;
}

// One increment of a counter (or of two) for the calling warp, after all of
// its lanes' global stores: each lane's fence orders its stores before the
// warp barrier, and lane 0 adds 1 after it.  All 32 lanes call it.  A fence
// costs the warp about a round trip to L2, so callers issue as few as they
// can and late.
// Coalesced BF16 stores of an unpooled epilogue chunk.  Lane i of a warp
// holds NV 16-byte pieces of one pixel's channels, and lanes 4k .. 4k + 3
// (NV = 4) or 2k, 2k + 1 (NV = 2) are horizontally adjacent pixels of one
// tile row.  A transpose by xor shuffles (one round per factor of two) leaves
// lane 4k + j holding piece j of each of its group's pixels, so one store
// instruction writes whole 16 NV-byte runs instead of one 16-byte piece of
// 32 pixels.
template <int NV>
__device__ __forceinline__ void group_transpose(uint4 (&v)[NV], int lane) {
#pragma unroll
    for (int s = 1; s < NV; s <<= 1) {
        const bool hi = (lane & s) != 0;
#pragma unroll
        for (int a = 0; a < NV; ++a) {
            if (a & s) continue;
            uint4 t = hi ? v[a] : v[a + s];
            t.x = __shfl_xor_sync(0xffffffffu, t.x, s);
            t.y = __shfl_xor_sync(0xffffffffu, t.y, s);
            t.z = __shfl_xor_sync(0xffffffffu, t.z, s);
            t.w = __shfl_xor_sync(0xffffffffu, t.w, s);
            if (hi) v[a] = t;
            else v[a + s] = t;
        }
    }
}

__device__ __forceinline__ void warp_signal(int* p, int* q = nullptr) {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        if (p) asm volatile("red.relaxed.gpu.global.add.s32 [%0], 1;" ::"l"(p) : "memory");
        if (q) asm volatile("red.relaxed.gpu.global.add.s32 [%0], 1;" ::"l"(q) : "memory");
    }
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const void* tmap, int c0, int c1, int c2,
                                            int c3, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int c0, int c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(tmap), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

// ---- CTA pairs (cta_group::2).  A 2-CTA cluster computes an M = 256 tile:
// the even CTA issues each MMA once for both, every CTA supplying its own
// 128 A rows and half of the B columns from its own shared memory, at the
// same offsets, and receiving its 128 accumulator rows in its own tensor
// memory.  Each CTA loads only its own shared memory; a load's completion is
// counted on the even CTA's barrier, an address in the cluster window.
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// cluster-window address of the shared variable at `local` in CTA `rank`
__device__ __forceinline__ uint32_t cl_addr(uint32_t local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}
__device__ __forceinline__ void mbar_arrive_cl(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
// loads into this CTA's shared memory whose completion counts on the barrier
// at cluster address `bar` (this CTA's or its peer's)
__device__ __forceinline__ void tma_load_4d_pair(uint32_t dst, const void* tmap, int c0, int c1, int c2, int c3,
                                                 uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.cta_group::2"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const void* tmap, int c0, int c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.cta_group::2"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(tmap), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

// 16-byte store to this CTA's shared memory; 16-byte load from any CTA's
// shared memory of the cluster (a cluster-window address)
__device__ __forceinline__ void st_shared_v4(uint32_t addr, float x, float y, float z, float w) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(x), "f"(y), "f"(z), "f"(w) : "memory");
}
__device__ __forceinline__ float4 ld_cluster_v4(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}

// phase trace: globaltimer (ns) of event e for this CTA
__device__ __forceinline__ void trace_stamp(unsigned long long* tr, int e) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    tr[blockIdx.x * kTraceEvents + e] = t;
}

// Shared-memory matrix descriptor (tcgen05), K-major operand with 32/64/128
// byte swizzle: start >> 4, leading offset (unused for swizzled K-major) 16,
// stride offset = 8 rows * row bytes, fixed version bits 46..48 = 0b001.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, int chb) {
    const uint64_t swz = chb == 128 ? 2 : chb == 64 ? 4 : 6;
    const uint64_t sbo = (uint64_t)(8 * chb) >> 4;
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | (sbo << 32) | ((uint64_t)1 << 46) |
           (swz << 61);
}

// Non-swizzled K-major operand: core matrices of 8 rows x 16 bytes, each
// 128 contiguous bytes; lbo = byte distance between the two core matrices
// of one 16-element K step, sbo = distance between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc_plain(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Tap pairs of a pair-mode layer (BF16, 8-channel K chunks, 16 bytes): the
// nine taps in the order of their A operands' offsets in a tap-merged stage
// (tap column dx major, tap row dy minor; slot s holds tap (dy, dx) =
// (s % 3, s / 3)), plus a tenth, all-zero weight slot; MMA j (K = 16) takes
// slots 2j and 2j + 1.
constexpr int kPairSlots = 10;

// Instruction descriptor: D = F32, A/B = BF16 (kind::f16) or E4M3
// (kind::f8f6f4), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
template <int DT>
__device__ __forceinline__ uint32_t instr_desc(int n, int m = 128) {
    const uint32_t ab = DT == DT_BF16 ? 1u : 0u;
    return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// CG = 1: one CTA; CG = 2: the CTA pair (issued by its even CTA)
template <int DT, int CG = 1>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                    uint32_t accumulate) {
    if (DT == DT_BF16 && CG == 1) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else if (DT == DT_BF16) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else if (CG == 1) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}

// Arrives on `bar` once every MMA this thread issued has completed.  CG = 2:
// `bar` is a cluster-window address (this CTA's barrier or its peer's).
template <int CG = 1>
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    if (CG == 1)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                     : "memory");
    else
        asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                     : "memory");
}

__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
        " [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// A TMEM load split in two: issue now, wait later, so that independent work
// runs in between.  The wait names the destination registers as read-write
// operands, so no use of them can be scheduled before it.
template <int CW>
__device__ __forceinline__ void tmem_ld_issue(uint32_t taddr, uint32_t* r) {
    if constexpr (CW == 32) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
              "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
              "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
    } else {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
            " [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15])
            : "r"(taddr));
    }
}
template <int CW>
__device__ __forceinline__ void tmem_ld_wait(uint32_t* r) {
    if constexpr (CW == 32) {
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                       "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                       "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]),
                       "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]),
                       "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                     :
                     : "memory");
    } else {
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                       "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                       "+r"(r[14]), "+r"(r[15])
                     :
                     : "memory");
    }
}

template <int CW>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float* v) {
    if constexpr (CW == 32) tmem_ld32(taddr, v);
    else tmem_ld16(taddr, v);
}

// Problem whose M tiles contain tile mt (tile_begin is increasing).
__device__ __forceinline__ int find_problem(const ConvProblem* probs, int nprob, int mt) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (probs[mid].tile_begin <= mt) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct Smem {
    // full[m][s]: stage s holds data for a tile of MMA issuer m.  One barrier
    // per (issuer, stage) keeps every barrier's phases consumed in order by a
    // single waiter, which a parity wait needs: with one barrier per stage the
    // second issuer could test a stage two phases ahead and pass on old data.
    uint64_t full[2][kMaxStages], empty[kMaxStages], accf[4], acce[4], done, bres;
    // cluster split-K: every epilogue warp of every CTA of the cluster has
    // written its partial sums (8 x ksplit arrivals)
    uint64_t xfull;
    uint32_t tmem;
    int abort;
};

}  // namespace tc

// MB = CTAs per SM: 1, or 2 for launches of many short tiles (few K steps
// each), whose time goes to the epilogue warps' dependent instruction chains:
// two CTAs give each SM sub-partition four epilogue warps instead of two.
// With MB = 2 a CTA has at most 80 registers a thread (the epilogue drains
// 16 columns at a time), half the shared memory and at most 256 TMEM
// columns, so that two CTAs always fit on an SM at once.
//
// CG = 2: CTA pairs (2-CTA clusters, one CTA an SM).  A work item is an M =
// 256 tile: M tiles 2u and 2u + 1 of pair item u, one a CTA (the second
// absent when the M tile count is odd: that CTA loads a duplicate and stores
// nothing).  Each CTA streams its A box and its half of the N tile's B box
// (BN / 2 rows) into its own ring; the even CTA's single MMA issuer waits
// for both halves on its own full barrier, issues cta_group::2 MMAs and
// commits to the stage's empty barrier and the accumulator barrier of both
// CTAs; each CTA's epilogue drains its own 128 accumulator rows and hands
// the buffer back on the even CTA's barrier.  Per SM a K step then moves
// 128 rows of A and BN / 2 of B instead of 128 + BN, so more stages fit and
// each byte in flight feeds twice the MMA work.  No resident weights, tap
// merging, tap pairs or K-alternating issuers in this mode.
template <int BN, int DT, int MB, int CG, int SP>
__global__ void __launch_bounds__(tc::THREADS, MB)
conv_tc_kernel(const __grid_constant__ CUtensorMap tmB, const TcArgs a) {
    using namespace tc;
    // Specialisations, their modes fixed at compile time so that the epilogue
    // (which bounds the short-tile layers) carries no code for other cases:
    // SP = 1, the tap-pair first layer (tap pairs on tap-merged stages,
    // resident weights, one issuer a tile); SP = 2, any other BF16 layer; both
    // with no K split and BF16 NHWC output without alpha.  SP = 3, a BF16
    // layer with a K split: its epilogue writes raw partial sums only.  SP =
    // 4, a BF16 last layer: no K split, FP32 NCHW output without alpha.
    // SP = 5, a BF16 layer with a K split reduced inside its cluster (a.xred):
    // streamed weights, one work item a CTA, BF16 NHWC or FP32 NCHW output.
    static_assert(SP == 0 || (SP >= 1 && SP <= 5 && DT == DT_BF16 && CG == 1), "specialisations");
    // (read where used, as the generic variant reads its launch arguments)
#define kKalt (SP == 1 ? 0 : a.kalt)
#define kTapm (SP == 1 ? 1 : SP == 5 ? 0 : a.tapm)
#define kPair (SP == 1 ? 1 : (SP == 2 || SP == 4 || SP == 5) ? 0 : a.pair)
#define kBres (SP == 1 ? 1 : SP == 5 ? 0 : a.bres)
#define kKsplit ((SP == 1 || SP == 2 || SP == 4) ? 1 : a.ksplit)
#define kAlpha ((SP == 1 || SP == 2 || SP == 4 || SP == 5) ? (const float*)nullptr : a.ep.alpha)
#define kOutLayout ((SP == 1 || SP == 2) ? (int)LAYOUT_NHWC : SP == 4 ? (int)LAYOUT_NCHW : (int)a.ep.out_layout)
#define kOutDt ((SP == 1 || SP == 2) ? (int)DT_BF16 : SP == 4 ? (int)DT_F32 : (int)a.ep.out_dt)
    static_assert(MB == 1 || (MB == 2 && BN <= 128), "two CTAs per SM: N tiles of at most 128 columns");
    static_assert(CG == 1 || (CG == 2 && MB == 1 && BN >= 128), "CTA pairs: one CTA an SM, N tiles of 128 or 256");
    constexpr bool C2 = CG == 2;
    // accumulator buffers in TMEM (512 columns an SM): four up to BN = 128,
    // so the MMAs of the next tiles never wait for an epilogue's round trip;
    // with two CTAs an SM, 256 columns each; CTA pairs allocate 256 columns
    constexpr int NBUF = C2 ? 256 / BN : MB == 2 ? 256 / BN : (BN <= 128 ? 4 : 2);
    constexpr int NBUF_LOG = NBUF == 4 ? 2 : NBUF == 2 ? 1 : 0;
    constexpr int TMEM_COLS = NBUF * BN;
    constexpr int CW = MB == 2 ? 16 : 32;   // epilogue columns per TMEM load
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // ring stages of st_bytes at smem (A box, then B box), resident weights at
    // bres_off, then the control block (host-computed geometry: tc_geometry)
    uint8_t* sRing = smem;
    uint8_t* sBres = smem + a.bres_off;
    Smem* sm = reinterpret_cast<Smem*>(smem + a.ctrl_off);
    const int nst = a.nst;
    const uint32_t st_bytes = (uint32_t)a.st_bytes;
    // epilogue copies of bias / alpha (launches with at most kEpiCols columns)
    float* s_bias = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(sm) + ((sizeof(Smem) + 15) & ~(size_t)15));
    float* s_alpha = s_bias + kEpiCols;

    // the next kernel may start its prologue as SMs free up (the first layer
    // of a pass on the row-band dataflow triggers only after its dependency
    // wait: the layers after it read counters the frame pack clears)
    if (!a.late_trigger) pdl_trigger();
#define TRACE(e) \
    do {                                   \
        if (a.trace) tc::trace_stamp(a.trace, e); \
    } while (0)
    if (threadIdx.x == 0) TRACE(0);
    const long long lim = a.wait_limit;   // bound of every pipeline wait (clock64 cycles)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int KK = a.k * a.k;
    const int nkb = KK * a.chunks;                // weight boxes (tap, chunk) per tile
    const int nk = kTapm ? a.chunks : nkb;       // pipeline steps per tile
    // CTA pairs: this CTA's rank (0 issues the MMAs); cluster split-K: the
    // CTA's K slice (blockIdx.x modulo ksplit)
    constexpr bool XR = SP == 5;
    const uint32_t rank = (C2 || XR) ? cluster_rank() : 0u;
    // work items: (m unit, n-tile, K slice), taken round robin by the CTAs
    // (CTA pairs: by the pairs; an m unit is then two M tiles)
    const int worker = C2 ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
    const int nworkers = C2 ? (int)(gridDim.x >> 1) : (int)gridDim.x;
    const int m_units = C2 ? (a.m_tiles + 1) >> 1 : a.m_tiles;
    const int total = m_units * a.n_tiles * kKsplit;
    const int pad = a.k >> 1;
    // A bytes per stage: one 128-row box, or three (TH + 2)-row boxes (tapm);
    // B: the N tile's box, or (CTA pairs) this CTA's half of it
    // (pair = 2: the tap-pair layer's stage is one box of (TH + 2) x (TW + 2)
    // pixels, TW = 8, holding all nine taps' rows)
    const bool box1 = kPair && a.pair == 2;
    const uint32_t a_box = box1   ? (uint32_t)(a.TH + 2) * (a.TW + 2) * a.chb
                           : kTapm ? (uint32_t)(a.TH + 2) * a.TW * a.chb
                                   : 128u * a.chb;
    const uint32_t a_bytes = (kTapm && !box1) ? 3u * a_box : a_box, b_bytes = (uint32_t)(C2 ? BN / 2 : BN) * a.chb;

    if (threadIdx.x == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
        for (int s = 0; s < nst; ++s) {
            tc::mbar_init(smem_u32(&sm->full[0][s]), 1);
            tc::mbar_init(smem_u32(&sm->full[1][s]), 1);
            tc::mbar_init(smem_u32(&sm->empty[s]), 1);
        }
        for (int b = 0; b < NBUF; ++b) {
            tc::mbar_init(smem_u32(&sm->accf[b]), 1);
            // the 4 warps of the warpgroup that drains buffer b; in K-alternating
            // mode both warpgroups drain every tile (half of its columns each);
            // CTA pairs: the 8 epilogue warps of both CTAs (on the even CTA's)
            tc::mbar_init(smem_u32(&sm->acce[b]), C2 ? 16 : kKalt ? 8 : 4);
        }
        // one commit from each MMA issuer (CTA pairs: the even CTA's issuer)
        tc::mbar_init(smem_u32(&sm->done), C2 ? 1 : 2);
        tc::mbar_init(smem_u32(&sm->bres), 1);
        if (XR) tc::mbar_init(smem_u32(&sm->xfull), 8u * (uint32_t)a.ksplit);
        sm->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        // CTA pairs: one warp of each CTA allocates, collectively, the same
        // columns in both CTAs' tensor memory
        if constexpr (C2) {
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&sm->tmem)),
                         "r"(TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&sm->tmem)),
                         "r"(TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    tc::fence_before();
    __syncthreads();
    // CTA pairs: both CTAs' barriers are initialised before either arrives on
    // or loads toward the other's (cluster split-K: before any CTA arrives on
    // another's xfull)
    if constexpr (C2 || XR) cluster_sync();
    tc::fence_after();
    if (threadIdx.x == 0) TRACE(1);
    const uint32_t tmem_base = sm->tmem;
    volatile int* abort_flag = &sm->abort;
    if (kBres && warp == 0 && lane == 0) {
        // resident weights: every K step's [BN x chunk] box of this CTA's N
        // tile, once, side by side.  The launch has no K split and a grid
        // that is a multiple of the N tile count, so the round-robin work
        // items (m-tile-major, N tile fastest) of a CTA all have the N tile
        // worker % n_tiles.  Weights are written only by the fold at load
        // time, which the host waits for, so these loads may overlap the
        // previous kernel's tail.
        const uint32_t rb = smem_u32(&sm->bres);
        const int nt_res = (worker - fdiv(worker, a.fd_ntiles) * a.n_tiles) * BN;   // first weight row
        if (kPair) {
            // pair mode: slots in tap-pair order; slot 9 starts at K column
            // 9 * Cp, past the weights' last column, so TMA fills it with zeros
            tc::mbar_expect_tx(rb, (uint32_t)kPairSlots * b_bytes);
            for (int s = 0; s < kPairSlots; ++s) {
                const int tap = s < 9 ? (box1 ? s : (s % 3) * 3 + s / 3) : 9;
                tc::tma_load_2d(smem_u32(sBres + (size_t)s * b_bytes), &tmB, tap * a.Cp, nt_res, rb);
            }
        } else {
            tc::mbar_expect_tx(rb, (uint32_t)nkb * b_bytes);
            int ch = 0, tap = 0;
            for (int ks = 0; ks < nkb; ++ks) {
                tc::tma_load_2d(smem_u32(sBres + (size_t)ks * b_bytes), &tmB, tap * a.Cp + ch * a.cpc, nt_res, rb);
                if (++ch == a.chunks) {
                    ch = 0;
                    ++tap;
                }
            }
        }
    }
    __syncwarp();
    // the prologue above may overlap the previous kernel; activations and
    // split-K workspace are touched only after it ended.  The TMA producers
    // wait further down, after the weight box of their first K step is on its
    // way (weights and problem tables are complete before the forward pass
    // starts).
    const bool lane_producer = warp == 0 || warp == NUM_WARPS - 2;
    // row-band dataflow (a.dep): no wait for the whole previous kernel; the
    // producers wait for the bands each tile reads, and the epilogue for the
    // layer whose input buffer it overwrites
    const bool flow = a.dep != nullptr;
    if (!lane_producer && !flow) {
        pdl_wait();
        if (a.late_trigger) pdl_trigger();
    }

    if (warp == 0 || warp == NUM_WARPS - 2) {
        // ------------------------------------------------ TMA producers
        // A warp issues one cp.async.bulk.tensor instruction per ~500 cycles
        // whatever its size, but lanes of one instruction are nearly free:
        // each of the two producer warps runs G lanes, lane j filling the K
        // steps it = pid + 2j (mod 2G) of this CTA's sequence.  2G divides
        // the stage count, so every stage is always filled by the same lane
        // and sees its uses in order (its empty phases are waited in order).
        const int pid = warp == 0 ? 0 : 1;
        const int G = a.plane;
        const int S2 = 2 * G;
        if (a.late_trigger && lane >= G && !flow) {   // lanes without a producer role
            pdl_wait();
            pdl_trigger();
        }
        if (lane < G) {
            const unsigned gmask = (1u << G) - 1u;
            // a single-problem launch keeps the problem's fields in registers
            const ConvProblem* P1 = a.nprob == 1 ? a.probs : nullptr;
            int tiles_x = 1, tiles_y = 1, tbeg = 0;
            FastDiv fd_tx, fd_ty;
            if (P1) {
                tiles_x = P1->tiles_x;
                tiles_y = P1->tiles_y;
                tbeg = P1->tile_begin;
                fd_tx = P1->fd_tx;
                fd_ty = P1->fd_ty;
            }
            // this lane's position: tile sequence index t (tile = worker + t *
            // nworkers), K step ks of that tile's slice [ks0, ks1), and `it`
            int t = 0, tile = worker, ks0 = 0, ks1 = 0, ks = 0;
            int ch = 0, kw = 0, kh = 0;   // chunk, tap column, tap row of ks
            int towner = 0, nt = 0, img = 0, x0 = 0, y0 = 0;
            const ConvProblem* P = P1;
            // row-band dataflow: the previous layer's bands under the current
            // tile's input rows, waited for before the tile's first A box
            const int Hin = P1 ? P1->H : 0;
            const int* dep_p = nullptr;
            int dep_n = 0;
            bool dep_need = false, prev_done = false;
            auto slice = [&] {
                if (kKsplit > 1) {
                    const int z = tile - fdiv(tile, a.fd_ksplit) * kKsplit;
                    ks0 = fdiv(nk * z, a.fd_ksplit);
                    ks1 = fdiv(nk * (z + 1), a.fd_ksplit);
                } else {
                    ks0 = 0;
                    ks1 = nk;
                }
            };
            auto setup = [&] {   // coordinates of the lane's current tile
                const int mn = kKsplit > 1 ? fdiv(tile, a.fd_ksplit) : tile;
                const int mq = fdiv(mn, a.fd_ntiles);
                // CTA pairs: M tile 2 mq + rank (an absent second tile loads a
                // duplicate of the last one, which its epilogue does not store)
                const int mt = C2 ? min(2 * mq + (int)rank, a.m_tiles - 1) : mq;
                nt = mn - mq * a.n_tiles;
                towner = t & 1;
                if (!P1) {
                    P = a.probs + tc::find_problem(a.probs, a.nprob, mt);
                    tiles_x = P->tiles_x;
                    tiles_y = P->tiles_y;
                    tbeg = P->tile_begin;
                    fd_tx = P->fd_tx;
                    fd_ty = P->fd_ty;
                }
                const int local = mt - tbeg;
                const int txy = fdiv(local, fd_tx);
                const int tx = local - txy * tiles_x;
                img = fdiv(txy, fd_ty);
                const int ty = txy - img * tiles_y;
                x0 = tx * a.TW - pad;
                y0 = ty * a.TH - pad;
                if (flow) {   // (single-problem launches)
                    const int r0 = max(y0, 0), r1 = min(y0 + a.TH - 1 + 2 * pad, Hin - 1);
                    const int b0 = r0 >> a.dep_shift;
                    dep_p = a.dep + img * a.dep_nb + b0;
                    dep_n = (r1 >> a.dep_shift) - b0 + 1;
                    dep_need = true;
                }
            };
            auto decompose = [&] {   // (ch, kw, kh) of ks, by division (tile changes only)
                const int tap = fdiv(ks, a.fd_chunks);
                ch = ks - tap * a.chunks;
                kh = fdiv(tap, a.fd_k);
                kw = tap - kh * a.k;
            };
            // moves the position forward by d K steps (across tiles)
            auto advance = [&](int d) {
                ks += d;
                if (ks < ks1) {   // same tile: step the chunk / tap counters
                    ch += d;
                    while (ch >= a.chunks) {
                        ch -= a.chunks;
                        if (++kw == a.k) {
                            kw = 0;
                            ++kh;
                        }
                    }
                    return;
                }
                while (tile < total && ks >= ks1) {
                    const int over = ks - ks1;
                    ++t;
                    tile += nworkers;
                    if (tile >= total) return;
                    slice();
                    ks = ks0 + over;
                }
                setup();
                decompose();
            };
            if (tile < total) {
                slice();
                ks = ks0;
                setup();
                decompose();
                advance(pid + 2 * lane);
            }
            int it = pid + 2 * lane;
            int ps = it;                 // stage of `it` (S2 divides nst: stepped by S2)
            uint32_t eph = 0u;           // parity of that stage's next empty phase
            bool ok = true;
            // the first K step's weight box does not depend on the previous
            // kernel: its stage is free, so it is armed for the whole step and
            // the box is issued before the dependency wait
            bool pre_b = false;
            // CTA pairs: stages are armed on the even CTA only (for both CTAs'
            // bytes), and every load completes on the even CTA's barrier
            const int b_row0 = C2 ? (int)rank * (BN / 2) : 0;   // this CTA's first row of the B box
            const uint32_t st_tx = C2 ? 2u * (a_bytes + b_bytes) : a_bytes + b_bytes;
            if (!kBres && tile < total) {
                const int owner = C2 ? 0 : kKalt ? ((ks - ks0) & 1) : towner;
                const uint32_t fb = smem_u32(&sm->full[owner][ps]);
                if constexpr (C2) {
                    if (rank == 0) tc::mbar_expect_tx(fb, st_tx);
                    tc::tma_load_2d_pair(smem_u32(sRing + (size_t)ps * st_bytes + a_bytes), &tmB,
                                         (kh * a.k + kw) * a.Cp + ch * a.cpc, nt * BN + b_row0, cl_addr(fb, 0));
                } else {
                    tc::mbar_expect_tx(fb, st_tx);
                    tc::tma_load_2d(smem_u32(sRing + (size_t)ps * st_bytes + a_bytes), &tmB,
                                    (kh * a.k + kw) * a.Cp + ch * a.cpc, nt * BN, fb);
                }
                pre_b = true;
            }
            if (!flow) {
                pdl_wait();
                if (a.late_trigger) pdl_trigger();
            }
            if (warp == 0 && lane == 0) TRACE(2);
            // per issuer: bit s = phase parity of the next use of full[m][s];
            // per stage this lane fills: the issuer of its last use
            uint32_t pph0 = 0u, pph1 = 0u, last_owner = 0u, issued = 0u;
            while (true) {
                const bool act = ok && tile < total;
                if (!__any_sync(gmask, act) || __any_sync(gmask, !ok)) break;
                if (act && !tc::mbar_wait(smem_u32(&sm->empty[ps]), eph ^ 1u, abort_flag, a.err, 1, lim)) ok = false;
                if (act && ok && dep_need && !prev_done) {
                    // the input rows of a new tile: the previous layer's bands
                    // complete (or the whole layer), the copies ordered after
                    if (!tc::flags_wait(dep_p, dep_n, a.dep_target, a.dep_done, a.dep_done_target, &prev_done,
                                        abort_flag, a.err, 8, lim))
                        ok = false;
                }
                if (act && ok) dep_need = false;
                __syncwarp(gmask);
                if (act && ok && a.withhold && it == S2) {
                    // fault injection (tests only): the second K step of producer
                    // 0's first lane is never loaded, so the wait of the issuer that
                    // consumes it runs out; nothing is armed, issued or recorded
                    it += S2;
                    ps += S2;
                    if (ps >= nst) {
                        ps -= nst;
                        eph ^= 1u;
                    }
                    advance(S2);
                    continue;
                }
                if (act && ok) {
                    const int s = ps;
                    // the issuer that consumes this K step: the tile's, or in
                    // K-alternating mode the K step's parity within the tile
                    const int owner = C2 ? 0 : kKalt ? ((ks - ks0) & 1) : towner;
                    const uint32_t fb = smem_u32(&sm->full[owner][s]);
                    if (owner) pph1 ^= 1u << s;
                    else pph0 ^= 1u << s;
                    last_owner = (last_owner & ~(1u << s)) | ((uint32_t)owner << s);
                    issued |= 1u << s;
                    const int c0 = ch * a.cpc;
                    const int kcol = (kh * a.k + kw) * a.Cp + c0;   // K column of the weights
                    uint8_t* stg = sRing + (size_t)s * st_bytes;
                    if constexpr (C2) {
                        if (!pre_b && rank == 0) tc::mbar_expect_tx(fb, st_tx);
                        const uint32_t fbc = cl_addr(fb, 0);
                        tc::tma_load_4d_pair(smem_u32(stg), &P->tmA, c0, x0 + kw, y0 + kh, img, fbc);
                        if (pre_b) pre_b = false;
                        else tc::tma_load_2d_pair(smem_u32(stg + a_bytes), &tmB, kcol, nt * BN + b_row0, fbc);
                    } else {
                        if (!pre_b) tc::mbar_expect_tx(fb, kBres ? a_bytes : st_tx);
                        if (box1) {   // all nine taps' rows in one box
                            tc::tma_load_4d(smem_u32(stg), &P->tmA, ks * a.cpc, x0, y0, img, fb);
                        } else if (kTapm) {   // step = chunk ks of all nine taps: one box per tap column
                            for (int dx = 0; dx < 3; ++dx)
                                tc::tma_load_4d(smem_u32(stg + dx * a_box), &P->tmA, ks * a.cpc, x0 + dx, y0, img,
                                                fb);
                        } else {
                            tc::tma_load_4d(smem_u32(stg), &P->tmA, c0, x0 + kw, y0 + kh, img, fb);
                        }
                        if (kBres || pre_b) {
                            pre_b = false;
                        } else {
                            tc::tma_load_2d(smem_u32(stg + a_bytes), &tmB, kcol, nt * BN, fb);
                        }
                    }
                    it += S2;
                    ps += S2;
                    if (ps >= nst) {
                        ps -= nst;
                        eph ^= 1u;
                    }
                    advance(S2);
                }
            }
            if (kBres && pid == 0 && lane == 0 &&
                !tc::mbar_wait(smem_u32(&sm->bres), 0u, abort_flag, a.err, 5, lim)) {
                const long long t0 = clock64();
                while (!tc::mbar_try(smem_u32(&sm->bres), 0u) && clock64() - t0 < WAIT_LIMIT) {
                }
            }
            // drain: every copy issued must have landed before smem goes away.
            // Earlier uses of a stage were consumed before it was refilled, so
            // only the last use of each stage can still be in flight.  CTA
            // pairs: the even CTA's barriers count both CTAs' copies, so the odd
            // CTA leaves the drain to it (the kernel's last cluster barrier
            // orders its exit after the even CTA's drain).
            for (int st = 0; st < nst && !(C2 && rank != 0); ++st) {
                if (!((issued >> st) & 1u)) continue;
                const int o = (int)((last_owner >> st) & 1u);
                const uint32_t bar = smem_u32(&sm->full[o][st]);
                const uint32_t lph = (((o ? pph1 : pph0) >> st) & 1u) ^ 1u;   // parity of the last use
                if (!tc::mbar_wait(bar, lph, abort_flag, a.err, 5, lim)) {
                    // abort already flagged: give the copies a bounded grace period
                    const long long t0 = clock64();
                    while (!tc::mbar_try(bar, lph) && clock64() - t0 < WAIT_LIMIT) {
                    }
                }
            }
            if (a.rd_sig) {
                // every copy of this warp's lanes has landed: its reads of the
                // input buffer are over
                __syncwarp(gmask);
                if (lane == 0) {
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                    asm volatile("fence.acq_rel.gpu;" ::: "memory");
                    asm volatile("red.relaxed.gpu.global.add.s32 [%0], 1;" ::"l"(a.rd_sig) : "memory");
                }
            }
        }
    } else if (warp == 1 || warp == NUM_WARPS - 1) {
        // ------------------------------------------------ MMA issuers
        // One thread pays ~150 cycles to issue each tcgen05 instruction, more
        // than a small MMA keeps the tensor pipe busy: two issuer warps take
        // alternate tiles (and so alternate accumulator buffers) and their
        // issue latencies overlap.  When a CTA has a single work item they
        // take alternate K steps of it instead (K-alternating mode), each into
        // its own accumulator of the tile's pair; the epilogue adds the two.
        const int mid = warp == 1 ? 0 : 1;
        // CTA pairs: the even CTA's first issuer alone issues for both CTAs;
        // it commits to a barrier of both (this CTA's, then the odd one's)
        auto commit = [&](uint64_t* bar) {
            if constexpr (C2) {
                tc::mma_commit<2>(cl_addr(smem_u32(bar), 0));
                tc::mma_commit<2>(cl_addr(smem_u32(bar), 1));
            } else {
                tc::mma_commit(smem_u32(bar));
            }
        };
        if (C2 && lane == 0 && mid == 0 && rank != 0) {
            // the odd CTA: its tensor memory and shared memory stay allocated
            // until every MMA of the even CTA's issuer has completed
            const long long t0 = clock64();
            while (!tc::mbar_try(smem_u32(&sm->done), 0) && clock64() - t0 < WAIT_LIMIT) {
            }
        } else if (lane == 0 && !(C2 && mid != 0)) {
            const uint32_t idesc = tc::instr_desc<DT>(BN, C2 ? 256 : 128);
            int it = 0, tcount = 0;
            uint32_t fph = 0u;   // bit s = phase parity of this issuer's next use of stage s
            bool ok = true;
            if (kBres) {
                ok = tc::mbar_wait(smem_u32(&sm->bres), 0u, abort_flag, a.err, 6, lim);
                tc::fence_after();
            }
            for (int tile = worker; tile < total && ok; tile += nworkers, ++tcount) {
                int ks0 = 0, ks1 = nk;
                if (kKsplit > 1) {
                    const int z = tile - fdiv(tile, a.fd_ksplit) * kKsplit;
                    ks0 = fdiv(nk * z, a.fd_ksplit);
                    ks1 = fdiv(nk * (z + 1), a.fd_ksplit);
                }
                if (!C2 && !kKalt && (tcount & 1) != mid) {   // the other issuer's tile: its stages are skipped
                    it += ks1 - ks0;
                    continue;
                }
                // accumulator slots: NBUF, or NBUF / 2 pairs (both powers of two)
                const int nsl_log = kKalt ? NBUF_LOG - 1 : NBUF_LOG;
                const int slot = tcount & ((1 << nsl_log) - 1);
                const int b = kKalt ? 2 * slot + mid : slot;
                const uint32_t aph = (uint32_t)(tcount >> nsl_log) & 1u;
                if (!tc::mbar_wait<C2>(smem_u32(&sm->acce[b]), aph ^ 1u, abort_flag, a.err, 2, lim)) break;
                tc::fence_after();
                const uint32_t dtm = tmem_base + (uint32_t)(b * BN);
                int ms = it - fdiv(it, a.fd_nst) * nst;   // stage of this tile's first K step
                bool first = true;   // the issuer's first K step of the tile overwrites its accumulator
                for (int ks = ks0; ks < ks1; ++ks, ++it) {
                    const int s = ms;
                    if (++ms == nst) ms = 0;
                    if (kKalt && ((ks - ks0) & 1) != mid) continue;   // the other issuer's K step
                    const uint32_t ph = (fph >> s) & 1u;
                    if (!tc::mbar_wait(smem_u32(&sm->full[mid][s]), ph, abort_flag, a.err, 3, lim)) {
                        ok = false;
                        break;
                    }
                    fph ^= 1u << s;
                    if (mid == 0 && it == 0) TRACE(3);
                    tc::fence_after();
                    uint8_t* stg = sRing + (size_t)s * st_bytes;
                    const int nmma = a.chb / 32;   // 32 bytes of K per MMA
                    if (kPair) {
                        // five MMAs of K = 16, each over two taps: the A core
                        // matrices of the second tap lie lbo bytes after the
                        // first's (for the tenth, zero-weight slot lbo is 0:
                        // the ninth tap's rows are read twice)
                        // (one box: slot s holds tap (dy, dx) = (s / 3, s % 3) at
                        // pixel dy * (TW + 2) + dx, a pixel row of the tile (8
                        // pixels, one core matrix) every TW + 2 pixels)
                        const uint32_t row_b = (uint32_t)a.TW * 16u, rowp = (uint32_t)(a.TW + 2) * 16u;
                        for (int j = 0; j < 5; ++j) {
                            const int s0 = 2 * j, s1 = 2 * j + 1;
                            const uint32_t o0 = box1 ? (uint32_t)(s0 / 3) * rowp + (uint32_t)(s0 % 3) * 16u
                                                     : (uint32_t)(s0 / 3) * a_box + (uint32_t)(s0 % 3) * row_b;
                            const uint32_t o1 = s1 >= 9 ? o0
                                                : box1  ? (uint32_t)(s1 / 3) * rowp + (uint32_t)(s1 % 3) * 16u
                                                        : (uint32_t)(s1 / 3) * a_box + (uint32_t)(s1 % 3) * row_b;
                            const uint64_t ad = tc::smem_desc_plain(smem_u32(stg + o0), o1 - o0, box1 ? rowp : 128u);
                            const uint64_t bd =
                                tc::smem_desc_plain(smem_u32(sBres + (size_t)s0 * b_bytes), b_bytes, 128u);
                            tc::mma<DT, CG>(dtm, ad, bd, idesc, (!first || j != 0) ? 1u : 0u);
                        }
                        first = false;
                    } else if (kTapm) {
                        // nine taps of chunk ks: tap (dy, dx) reads box dx from row dy * TW
                        for (int dx = 0; dx < 3; ++dx)
                            for (int dy = 0; dy < 3; ++dy) {
                                const uint64_t ad =
                                    tc::smem_desc(smem_u32(stg + dx * a_box + dy * a.TW * a.chb), a.chb);
                                const uint64_t bd = tc::smem_desc(
                                    smem_u32(sBres + (size_t)((dy * 3 + dx) * a.chunks + ks) * b_bytes), a.chb);
                                for (int j = 0; j < nmma; ++j)
                                    tc::mma<DT, CG>(dtm, ad + (uint64_t)(2 * j), bd + (uint64_t)(2 * j), idesc,
                                                (!first || j != 0) ? 1u : 0u);
                                first = false;
                            }
                    } else {
                        const uint64_t ad = tc::smem_desc(smem_u32(stg), a.chb);
                        const uint64_t bd =
                            tc::smem_desc(smem_u32(kBres ? sBres + (size_t)ks * b_bytes : stg + a_bytes), a.chb);
                        for (int j = 0; j < nmma; ++j)
                            tc::mma<DT, CG>(dtm, ad + (uint64_t)(2 * j), bd + (uint64_t)(2 * j), idesc,
                                            (!first || j != 0) ? 1u : 0u);
                        first = false;
                    }
                    commit(&sm->empty[s]);
                }
                if (ok) commit(&sm->accf[b]);
            }
            if (mid == 0) TRACE(4);
            // every MMA issued has finished before TMEM and smem are released
            commit(&sm->done);
            const long long t0 = clock64();
            while (!tc::mbar_try(smem_u32(&sm->done), 0) && clock64() - t0 < WAIT_LIMIT) {
            }
        }
    } else {
        // ------------------------------------------------ epilogue (warps 2..9)
        // Two warpgroups: warpgroup g drains the tiles of MMA issuer g (every
        // other tile), all their columns, so both groups stay busy even when a
        // layer has only a few live output channels.  Each SM sub-partition
        // runs one warp of each.
        const int q = warp & 3;                 // TMEM lane quarter of this warp
        const int grp = (warp - 2) >> 2;        // warpgroup = MMA issuer whose tiles it drains
        // columns of a tile this warp drains: all, or in K-alternating mode
        // (one tile per CTA) half of them, so the last tile's epilogue, which
        // nothing overlaps, runs on both warpgroups
        // (CTA pairs: both warpgroups on every tile too; one issuer, one buffer
        // sequence)
        const int half = (kKalt || C2) ? grp : 0;
        const int HC = (kKalt || C2) ? BN / 2 : BN;
        const int row = q * 32 + lane;          // pixel index in the tile
        const int py = row / a.TW, px = row % a.TW;
        const bool pool = a.ep.pool == POOL_S2;
        // bias / alpha of the launch's columns into shared memory once (they are
        // padded with zeros to the weight rows, which cover every N tile)
        const int ncol_all = a.n_tiles * BN;
        const bool epi_smem = ncol_all <= kEpiCols;
        if (epi_smem) {
            for (int i = threadIdx.x - 64; i < ncol_all; i += 256) {
                s_bias[i] = a.ep.bias[i];
                if (kAlpha) s_alpha[i] = kAlpha[i];
            }
            asm volatile("bar.sync 1, 256;" ::: "memory");   // the 8 epilogue warps
        }
        if (lane == 0 && warp == 2) TRACE(5);
        if (a.rd_dep) {
            // row-band dataflow: the output buffer was the input of the layer
            // two back, whose copies must all have landed before it is
            // overwritten (on expiry the abort flag stops the pipeline)
            bool unused = false;
            if (lane == 0)
                (void)tc::flags_wait(a.rd_dep, 1, a.rd_target, nullptr, 0, &unused, abort_flag, a.err, 9, lim);
            __syncwarp();
        }
        const float* e_bias = epi_smem ? s_bias : a.ep.bias;
        const float* e_alpha = epi_smem ? s_alpha : kAlpha;
        const int ymask = a.TW == 16 ? 16 : 8;  // lane distance of the pixel below (pool tiles)
        // columns at or beyond `live` are padding nobody reads: skipped
        const int live = kOutLayout == LAYOUT_NCHW ? a.ep.cout : max(a.ep.out_cs, a.ep.cout);
        void* pY = nullptr;
        int pH = 0, pW = 0, pTX = 1, pTY = 1, pBegin = 0;
        FastDiv fTX, fTY;
        int tcount = 0;
        bool have_p = false;   // problem fields loaded (single-problem launches read them once)
        bool pairs_done = false;
        // row-band dataflow: the band counter of this warp's last tile, whose
        // increment waits until the next tile's arithmetic is done (the
        // increment's fence then finds the tile's stores already performed)
        int* pend = nullptr;
        if constexpr (SP == 1) {
            // The tap-pair first layer, one problem, one N tile, at most CW
            // live columns: a warpgroup drains its next two tiles (tcount t and
            // t + 2, accumulator buffers t & 3 and (t + 2) & 3) in one pass, so
            // that their two dependent chains (TMEM load, tile decode,
            // arithmetic, pool shuffles, stores) overlap.  The MMA issuer needs
            // those buffers back only for tiles t + 4 and t + 6.  Same
            // operations per element as the loop below.
            static_assert(SP != 1 || NBUF == 4, "two tiles a pass take four accumulator buffers");
            if (a.nprob == 1 && a.n_tiles == 1 && live <= CW) {
                pairs_done = true;
                const ConvProblem& P0 = a.probs[0];
                void* ybase = a.y_override ? a.y_override : P0.y;
                const int H0 = P0.H, W0 = P0.W, TX0 = P0.tiles_x, TY0 = P0.tiles_y, B0 = P0.tile_begin;
                const FastDiv fx = P0.fd_tx, fy = P0.fd_ty;
                const int Ho = pool ? H0 / 2 : H0, Wo = pool ? W0 / 2 : W0;
                float bb[CW];   // the live columns' bias, once
#pragma unroll
                for (int j = 0; j < CW / 4; ++j) {
                    const float4 t = reinterpret_cast<const float4*>(e_bias)[j];
                    bb[4 * j] = t.x;
                    bb[4 * j + 1] = t.y;
                    bb[4 * j + 2] = t.z;
                    bb[4 * j + 3] = t.w;
                }
                const uint32_t tlane = tmem_base + ((uint32_t)(q * 32) << 16);
                auto finish = [&](int mt, const uint32_t* r) {
                    const int local = mt - B0;
                    const int txy = fdiv(local, fx);
                    const int tx = local - txy * TX0;
                    const int img = fdiv(txy, fy);
                    const int ty = txy - img * TY0;
                    const int gy = ty * a.TH + py, gx = tx * a.TW + px;
                    const bool valid = gy < H0 && gx < W0;
                    const int yo = pool ? gy / 2 : gy, xo = pool ? gx / 2 : gx;
                    const bool writer = valid && (!pool || ((lane & 1) == 0 && (lane & ymask) == 0));
                    const size_t pix = ((size_t)img * Ho + yo) * Wo + xo;
                    float v[CW];
#pragma unroll
                    for (int j = 0; j < CW / 2; ++j) {
                        const float2 s = __fadd2_rn(make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1])),
                                                    make_float2(bb[2 * j], bb[2 * j + 1]));
                        v[2 * j] = s.x;
                        v[2 * j + 1] = s.y;
                    }
                    if (a.ep.act == ACT_LEAKY) {
                        const float2 slope = make_float2(kLeakySlope, kLeakySlope);
#pragma unroll
                        for (int j = 0; j < CW / 2; ++j) {
                            const float2 s2 = __fmul2_rn(make_float2(v[2 * j], v[2 * j + 1]), slope);
                            v[2 * j] = fmaxf(v[2 * j], s2.x);
                            v[2 * j + 1] = fmaxf(v[2 * j + 1], s2.y);
                        }
                    }
                    uint32_t w[CW / 2];
#pragma unroll
                    for (int j = 0; j < CW / 2; ++j) {
                        __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                        w[j] = *reinterpret_cast<uint32_t*>(&h2);
                    }
                    if (pool) {
#pragma unroll
                        for (int j = 0; j < CW / 2; ++j) {
                            uint32_t o = __shfl_xor_sync(0xffffffffu, w[j], 1);
                            __nv_bfloat162 m = __hmax2(*reinterpret_cast<__nv_bfloat162*>(&w[j]),
                                                       *reinterpret_cast<__nv_bfloat162*>(&o));
                            w[j] = *reinterpret_cast<uint32_t*>(&m);
                            o = __shfl_xor_sync(0xffffffffu, w[j], ymask);
                            m = __hmax2(*reinterpret_cast<__nv_bfloat162*>(&w[j]),
                                        *reinterpret_cast<__nv_bfloat162*>(&o));
                            w[j] = *reinterpret_cast<uint32_t*>(&m);
                        }
                    }
                    // the previous tile's band, now that its stores have had
                    // this tile's loads and arithmetic to drain
                    if (pend) {
                        tc::warp_signal(pend);
                        pend = nullptr;
                    }
                    if (writer) {
                        uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(ybase) +
                                                              pix * a.ep.out_cs);
                        const int nvec = a.ep.out_cs >= CW ? CW / 8 : 2;
#pragma unroll
                        for (int i = 0; i < CW / 8; ++i)
                            if (i < nvec) dst[i] = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
                    }
                    if (a.sig) pend = a.sig + img * TY0 + ty;   // signalled after the next tile's arithmetic
                };
                for (int tc = grp;; tc += 4) {
                    const int tile0 = worker + tc * nworkers;
                    if (tile0 >= total) break;
                    const int tile1 = tile0 + 2 * nworkers;
                    const bool has1 = tile1 < total;   // warp-uniform
                    const int b0 = tc & 3, b1 = (tc + 2) & 3;
                    if (!tc::mbar_wait(smem_u32(&sm->accf[b0]), (uint32_t)(tc >> 2) & 1u, abort_flag, a.err, 4, lim))
                        break;
                    if (has1 &&
                        !tc::mbar_wait(smem_u32(&sm->accf[b1]), (uint32_t)((tc + 2) >> 2) & 1u, abort_flag, a.err, 4, lim))
                        break;
                    tc::fence_after();
                    uint32_t r0[CW], r1[CW];
                    __syncwarp();
                    tc::tmem_ld_issue<CW>(tlane + (uint32_t)(b0 * BN), r0);
                    if (has1) tc::tmem_ld_issue<CW>(tlane + (uint32_t)(b1 * BN), r1);
                    tc::tmem_ld_wait<CW>(r0);
                    if (has1) tc::tmem_ld_wait<CW>(r1);
                    // both buffers back to the MMA issuer
                    tc::fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        tc::mbar_arrive(smem_u32(&sm->acce[b0]));
                        if (has1) tc::mbar_arrive(smem_u32(&sm->acce[b1]));
                    }
                    finish(tile0, r0);
                    if (has1) finish(tile1, r1);
                }
            }
        }
        if constexpr (XR) {
            // Cluster split-K.  The cluster's ksplit CTAs computed K slices 0 ..
            // ksplit - 1 (their ranks) of one tile.  Phase 1: the two
            // warpgroups drain half of this CTA's accumulator columns each (the
            // K-alternating pair added) into the ring, idle now that every MMA
            // has completed, as [BN / 4][128 rows][4] floats: a warp's float4
            // stores cover 512 contiguous bytes.  Phase 2: once every CTA's
            // partial sums are in place, CTA r takes columns r * BN / ksplit ..
            // (r + 1) * BN / ksplit - 1 (half of them a warpgroup), adds the
            // slices from the CTAs' shared memory in the order 0, 1, ... (the
            // workspace reduction's order), applies the epilogue and stores.
            // The kernel's closing cluster barrier keeps every CTA's shared
            // memory alive until all reads of it are done.
            const int S = a.ksplit;
            const int mn = fdiv(worker, a.fd_ksplit);   // one work item a CTA: the cluster's tile
            const int mq = fdiv(mn, a.fd_ntiles);
            const int mt = mq, nt = mn - mq * a.n_tiles;
            const uint32_t xs = smem_u32(sRing);
            bool ok = worker < total;
            if (ok) ok = tc::mbar_wait(smem_u32(&sm->accf[0]), 0u, abort_flag, a.err, 4, lim);
            if (ok && kKalt) ok = tc::mbar_wait(smem_u32(&sm->accf[1]), 0u, abort_flag, a.err, 4, lim);
            if (ok && lane == 0 && warp == 2) TRACE(9);
            if (ok) {
                tc::fence_after();
                // the ring was last written by TMA (the async proxy)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                const uint32_t trow = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(grp * (BN / 2));
#pragma unroll 1
                for (int c0 = 0; c0 < BN / 2; c0 += CW) {
                    const int c = grp * (BN / 2) + c0;   // tile column
                    if (nt * BN + c >= live) break;
                    float v[CW];
                    __syncwarp();
                    {   // both accumulators' loads issued before one wait
                        uint32_t r0[CW], r1[CW];
                        tc::tmem_ld_issue<CW>(trow + (uint32_t)c0, r0);
                        if (kKalt) tc::tmem_ld_issue<CW>(trow + (uint32_t)(BN + c0), r1);
                        tc::tmem_ld_wait<CW>(r0);
                        if (kKalt) {
                            tc::tmem_ld_wait<CW>(r1);   // (nothing left to wait for: names r1)
#pragma unroll
                            for (int j = 0; j < CW / 2; ++j) {
                                const float2 r2 =
                                    __fadd2_rn(make_float2(__uint_as_float(r0[2 * j]), __uint_as_float(r0[2 * j + 1])),
                                               make_float2(__uint_as_float(r1[2 * j]), __uint_as_float(r1[2 * j + 1])));
                                v[2 * j] = r2.x;
                                v[2 * j + 1] = r2.y;
                            }
                        } else {
#pragma unroll
                            for (int j = 0; j < CW; ++j) v[j] = __uint_as_float(r0[j]);
                        }
                    }
#pragma unroll
                    for (int j = 0; j < CW / 4; ++j)
                        tc::st_shared_v4(xs + (uint32_t)((((c >> 2) + j) * 128 + row) * 16), v[4 * j], v[4 * j + 1],
                                         v[4 * j + 2], v[4 * j + 3]);
                }
                // the warp's stores are ordered before lane 0's release
                __syncwarp();
                if (lane == 0)
                    for (int r = 0; r < S; ++r) tc::mbar_arrive_cl(cl_addr(smem_u32(&sm->xfull), (uint32_t)r));
            }
            if (ok) ok = tc::mbar_wait<true>(smem_u32(&sm->xfull), 0u, abort_flag, a.err, 7, lim);
            // phase 2 for a cluster of SC CTAs (a compile-time count, so that the
            // batch of remote loads below lives in registers)
            auto reduce = [&](auto SC) {
                constexpr int S2 = decltype(SC)::value;
                constexpr int CPO = BN / S2;                // columns this CTA reduces (a multiple of 8)
                constexpr int WG = CPO >= 16 ? 2 : 1;       // warpgroups sharing them
                constexpr int NCW = CPO / WG;               // this warpgroup's columns
                static_assert(NCW % 8 == 0, "columns a warpgroup reduces: whole chunks of 8");
                if (grp >= WG) return;
                // remote loads are issued in batches of 16 float4 a thread: G
                // chunks of 8 columns times SB slices; the additions still run
                // in slice order 0, 1, ... for every column
                constexpr int SB = S2 < 8 ? S2 : 8;
                constexpr int G = 8 / SB < NCW / 8 ? 8 / SB : NCW / 8;
                const int cb = (int)rank * CPO + grp * NCW;   // this warpgroup's first tile column
                uint32_t peer[S2];
#pragma unroll
                for (int r = 0; r < S2; ++r) peer[r] = cl_addr(xs, (uint32_t)r);
                const ConvProblem& P = a.probs[0];
                void* ybase = a.y_override ? a.y_override : P.y;
                const int local = mt - P.tile_begin;
                const int txy = fdiv(local, P.fd_tx);
                const int tx = local - txy * P.tiles_x;
                const int img = fdiv(txy, P.fd_ty);
                const int ty = txy - img * P.tiles_y;
                const int gy = ty * a.TH + py, gx = tx * a.TW + px;
                const bool valid = gy < P.H && gx < P.W;
                const int Ho = pool ? P.H / 2 : P.H, Wo = pool ? P.W / 2 : P.W;
                const int yo = pool ? gy / 2 : gy, xo = pool ? gx / 2 : gx;
                const bool writer = valid && (!pool || ((lane & 1) == 0 && (lane & ymask) == 0));
                const size_t pix = ((size_t)img * Ho + yo) * Wo + xo;
                const bool nchw = a.ep.out_layout == LAYOUT_NCHW;
#pragma unroll 1
                for (int cg0 = 0; cg0 < NCW; cg0 += 8 * G) {
                    if (nt * BN + cb + cg0 >= live) break;
                    float acc[G][8];
#pragma unroll
                    for (int sb0 = 0; sb0 < S2; sb0 += SB) {
                        float4 t[G][SB][2];
#pragma unroll
                        for (int g = 0; g < G; ++g)
#pragma unroll
                            for (int r = 0; r < SB; ++r)
#pragma unroll
                                for (int h = 0; h < 2; ++h)
                                    t[g][r][h] = tc::ld_cluster_v4(
                                        peer[sb0 + r] + (uint32_t)(((((cb + cg0 + 8 * g) >> 2) + h) * 128 + row) * 16));
#pragma unroll
                        for (int g = 0; g < G; ++g)
#pragma unroll
                            for (int r = 0; r < SB; ++r) {
                                const float u[8] = {t[g][r][0].x, t[g][r][0].y, t[g][r][0].z, t[g][r][0].w,
                                                    t[g][r][1].x, t[g][r][1].y, t[g][r][1].z, t[g][r][1].w};
#pragma unroll
                                for (int j = 0; j < 8; ++j) acc[g][j] = (sb0 + r == 0) ? u[j] : acc[g][j] + u[j];
                            }
                    }
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        const int o0 = nt * BN + cb + cg0 + 8 * g;   // first output channel of the chunk
                        if (o0 >= live) break;
                        float v[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) v[j] = acc[g][j];
                        // bias (padded with zeros to the weight rows), leaky
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const float2 r2 = __fadd2_rn(make_float2(v[2 * j], v[2 * j + 1]),
                                                         make_float2(e_bias[o0 + 2 * j], e_bias[o0 + 2 * j + 1]));
                            v[2 * j] = r2.x;
                            v[2 * j + 1] = r2.y;
                        }
                        if (a.ep.act == ACT_LEAKY) {
                            const float2 slope = make_float2(kLeakySlope, kLeakySlope);
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const float2 s2 = __fmul2_rn(make_float2(v[2 * j], v[2 * j + 1]), slope);
                                v[2 * j] = fmaxf(v[2 * j], s2.x);
                                v[2 * j + 1] = fmaxf(v[2 * j + 1], s2.y);
                            }
                        }
                        if (nchw) {   // FP32 NCHW (a last layer)
                            if (pool) {
#pragma unroll
                                for (int j = 0; j < 8; ++j) {
                                    v[j] = fmaxf(v[j], __shfl_xor_sync(0xffffffffu, v[j], 1));
                                    v[j] = fmaxf(v[j], __shfl_xor_sync(0xffffffffu, v[j], ymask));
                                }
                            }
                            if (writer) {
                                float* yf = reinterpret_cast<float*>(ybase);
#pragma unroll
                                for (int j = 0; j < 8; ++j)
                                    if (o0 + j < a.ep.cout)
                                        yf[(((size_t)img * a.ep.cout + o0 + j) * Ho + yo) * Wo + xo] = v[j];
                            }
                            continue;
                        }
                        // BF16 NHWC: round, then pool on packed pairs (as the other epilogues)
                        uint32_t w[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                            w[j] = *reinterpret_cast<uint32_t*>(&h2);
                        }
                        if (pool) {
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                uint32_t o = __shfl_xor_sync(0xffffffffu, w[j], 1);
                                __nv_bfloat162 m = __hmax2(*reinterpret_cast<__nv_bfloat162*>(&w[j]),
                                                           *reinterpret_cast<__nv_bfloat162*>(&o));
                                w[j] = *reinterpret_cast<uint32_t*>(&m);
                                o = __shfl_xor_sync(0xffffffffu, w[j], ymask);
                                m = __hmax2(*reinterpret_cast<__nv_bfloat162*>(&w[j]),
                                            *reinterpret_cast<__nv_bfloat162*>(&o));
                                w[j] = *reinterpret_cast<uint32_t*>(&m);
                            }
                        }
                        if (writer && o0 < a.ep.out_cs)
                            *reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(ybase) + pix * a.ep.out_cs +
                                                      o0) = make_uint4(w[0], w[1], w[2], w[3]);
                    }
                }
            };
            if (ok) {
                if (S == 2) reduce(std::integral_constant<int, 2>{});
                if (S == 4) reduce(std::integral_constant<int, 4>{});
                if (S == 8) reduce(std::integral_constant<int, 8>{});
                if constexpr (BN >= 128) {
                    if (S == 16) reduce(std::integral_constant<int, 16>{});
                }
                if (a.sig) {   // every epilogue warp of every CTA of the cluster, once (at the end)
                    const ConvProblem& P = a.probs[0];
                    const int txy = fdiv(mt - P.tile_begin, P.fd_tx);
                    const int img = fdiv(txy, P.fd_ty);
                    pend = a.sig + img * P.tiles_y + (txy - img * P.tiles_y);
                }
            }
        }
        for (int tile = (XR || pairs_done) ? total : worker; tile < total; tile += nworkers, ++tcount) {
            if (!C2 && !kKalt && (tcount & 1) != grp) continue;
            // the tile's accumulator (or pair of them in K-alternating mode)
            const int nsl_log = kKalt ? NBUF_LOG - 1 : NBUF_LOG;
            const int slot = tcount & ((1 << nsl_log) - 1);
            const int b = kKalt ? 2 * slot : slot;
            const uint32_t aph = (uint32_t)(tcount >> nsl_log) & 1u;
            if (!tc::mbar_wait<C2>(smem_u32(&sm->accf[b]), aph, abort_flag, a.err, 4, lim)) break;
            if (kKalt && !tc::mbar_wait(smem_u32(&sm->accf[b + 1]), aph, abort_flag, a.err, 4, lim)) break;
            if (lane == 0 && warp == 2) TRACE(9);
            tc::fence_after();
            const int mn = kKsplit > 1 ? fdiv(tile, a.fd_ksplit) : tile;
            const int z = tile - mn * kKsplit;
            const int mq = fdiv(mn, a.fd_ntiles);
            const int mt = C2 ? 2 * mq + (int)rank : mq, nt = mn - mq * a.n_tiles;
            const uint32_t trow = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + half * HC);
            // the buffer goes back to the MMA issuer right after its last live
            // column is in registers; the math and stores of that chunk follow
            // a chunk of the tile's accumulator: in K-alternating mode both
            // accumulators' loads are issued before one wait, and added
            auto ld_acc = [&](uint32_t taddr, float* v) {
                uint32_t r0[CW];
                tc::tmem_ld_issue<CW>(taddr, r0);
                if (kKalt) {
                    uint32_t r1[CW];
                    tc::tmem_ld_issue<CW>(taddr + (uint32_t)BN, r1);
                    tc::tmem_ld_wait<CW>(r0);
                    tc::tmem_ld_wait<CW>(r1);   // (nothing left to wait for: names r1)
#pragma unroll
                    for (int j = 0; j < CW / 2; ++j) {
                        const float2 r = __fadd2_rn(make_float2(__uint_as_float(r0[2 * j]), __uint_as_float(r0[2 * j + 1])),
                                                    make_float2(__uint_as_float(r1[2 * j]), __uint_as_float(r1[2 * j + 1])));
                        v[2 * j] = r.x;
                        v[2 * j + 1] = r.y;
                    }
                } else {
                    tc::tmem_ld_wait<CW>(r0);
#pragma unroll
                    for (int j = 0; j < CW; ++j) v[j] = __uint_as_float(r0[j]);
                }
            };
            bool released = false;
            auto release = [&] {
                tc::fence_before();
                __syncwarp();
                if (lane == 0) {
                    if constexpr (C2) {
                        tc::mbar_arrive_cl(cl_addr(smem_u32(&sm->acce[b]), 0));   // the even CTA's
                    } else {
                        tc::mbar_arrive(smem_u32(&sm->acce[b]));
                        if (kKalt) tc::mbar_arrive(smem_u32(&sm->acce[b + 1]));
                    }
                }
                released = true;
            };
            if (C2 && mt >= a.m_tiles) {   // the absent second tile of an odd count
                release();
                continue;
            }
            if (SP == 3 || kKsplit > 1) {   // (SP = 3: always)
                // raw partial sums of this K slice; the reduction applies the
                // epilogue.  Workspace plane z is tile-major in groups of four
                // columns ([m_tiles][ncp / 4][128 rows][4]): the 32 rows of a warp
                // write one contiguous 512-byte run per float4 store.
                const int ncp = a.n_tiles * BN;
                float* wr = a.ws + (size_t)z * a.m_tiles * 128 * ncp +
                            ((size_t)mt * (ncp >> 2) + ((nt * BN + half * HC) >> 2)) * 512 + row * 4;
#pragma unroll 1
                for (int c0 = 0; c0 < HC; c0 += CW) {
                    if (nt * BN + half * HC + c0 >= live) break;
                    float v[CW];
                    __syncwarp();
                    ld_acc(trow + (uint32_t)c0, v);
                    if (c0 + CW >= HC || nt * BN + half * HC + c0 + CW >= live) release();
#pragma unroll
                    for (int j = 0; j < CW; j += 4)
                        *reinterpret_cast<float4*>(wr + (size_t)((c0 + j) >> 2) * 512) =
                            make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                }
            } else {
                // the single-problem case keeps its fields in registers (read once)
                if (a.nprob > 1 || !have_p) {
                    have_p = true;
                    const ConvProblem& P = a.probs[a.nprob > 1 ? tc::find_problem(a.probs, a.nprob, mt) : 0];
                    pY = P.y;
                    pH = P.H;
                    pW = P.W;
                    pTX = P.tiles_x;
                    pTY = P.tiles_y;
                    pBegin = P.tile_begin;
                    fTX = P.fd_tx;
                    fTY = P.fd_ty;
                }
                void* ybase = a.y_override ? a.y_override : pY;
                const int local = mt - pBegin;
                const int txy = fdiv(local, fTX);
                const int tx = local - txy * pTX;
                const int img = fdiv(txy, fTY);
                const int ty = txy - img * pTY;
                const int gy = ty * a.TH + py, gx = tx * a.TW + px;
                const bool valid = gy < pH && gx < pW;
                const int Ho = pool ? pH / 2 : pH, Wo = pool ? pW / 2 : pW;
                const int yo = pool ? gy / 2 : gy, xo = pool ? gx / 2 : gx;
                const bool writer = valid && (!pool || ((lane & 1) == 0 && (lane & ymask) == 0));
                const size_t pix = ((size_t)img * Ho + yo) * Wo + xo;
#pragma unroll 1
                for (int c0 = 0; c0 < HC; c0 += CW) {
                    const int o0 = nt * BN + half * HC + c0;   // first output channel of the chunk
                    if (o0 >= live) break;
                    // bias / alpha are padded with zeros to the weight rows: no bounds
                    // checks; loaded before the TMEM read so the two latencies overlap
                    float bb[CW];
#pragma unroll
                    for (int j = 0; j < CW / 4; ++j) {
                        const float4 t = reinterpret_cast<const float4*>(e_bias + o0)[j];
                        bb[4 * j] = t.x;
                        bb[4 * j + 1] = t.y;
                        bb[4 * j + 2] = t.z;
                        bb[4 * j + 3] = t.w;
                    }
                    float v[CW];
                    __syncwarp();
                    ld_acc(trow + (uint32_t)c0, v);
                    if (c0 + CW >= HC || o0 + CW >= live) release();
                    // warp-uniform branches: each variant is one straight-line loop.
                    // Paired FP32 operations (one instruction on a register
                    // pair) round exactly as the scalar ones.
                    if (kAlpha) {
#pragma unroll
                        for (int j = 0; j < CW / 4; ++j) {
                            const float4 t = reinterpret_cast<const float4*>(e_alpha + o0)[j];
                            const float2 lo = __ffma2_rn(make_float2(v[4 * j], v[4 * j + 1]), make_float2(t.x, t.y),
                                                         make_float2(bb[4 * j], bb[4 * j + 1]));
                            const float2 hi = __ffma2_rn(make_float2(v[4 * j + 2], v[4 * j + 3]), make_float2(t.z, t.w),
                                                         make_float2(bb[4 * j + 2], bb[4 * j + 3]));
                            v[4 * j] = lo.x;
                            v[4 * j + 1] = lo.y;
                            v[4 * j + 2] = hi.x;
                            v[4 * j + 3] = hi.y;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < CW / 2; ++j) {
                            const float2 r = __fadd2_rn(make_float2(v[2 * j], v[2 * j + 1]),
                                                        make_float2(bb[2 * j], bb[2 * j + 1]));
                            v[2 * j] = r.x;
                            v[2 * j + 1] = r.y;
                        }
                    }
                    if (a.ep.act == ACT_LEAKY) {
                        // leaky(v) = max(v, 0.1 v): v for v > 0, 0.1 v otherwise
                        const float2 slope = make_float2(kLeakySlope, kLeakySlope);
#pragma unroll
                        for (int j = 0; j < CW / 2; ++j) {
                            const float2 s2 = __fmul2_rn(make_float2(v[2 * j], v[2 * j + 1]), slope);
                            v[2 * j] = fmaxf(v[2 * j], s2.x);
                            v[2 * j + 1] = fmaxf(v[2 * j + 1], s2.y);
                        }
                    }
                    if (pend) {   // the previous tile's band (its stores had this chunk's loads to drain)
                        tc::warp_signal(pend);
                        pend = nullptr;
                    }
                    if (kOutLayout == LAYOUT_NCHW) {
                        if (pool) {
#pragma unroll
                            for (int j = 0; j < CW; ++j) {
                                v[j] = fmaxf(v[j], __shfl_xor_sync(0xffffffffu, v[j], 1));
                                v[j] = fmaxf(v[j], __shfl_xor_sync(0xffffffffu, v[j], ymask));
                            }
                        }
                        if (writer) {
                            float* yf = reinterpret_cast<float*>(ybase);
#pragma unroll
                            for (int j = 0; j < CW; ++j)
                                if (o0 + j < a.ep.cout)
                                    yf[(((size_t)img * a.ep.cout + o0 + j) * Ho + yo) * Wo + xo] = v[j];
                        }
                        continue;
                    }
                    if (kOutDt == DT_BF16) {
                        // round first, then pool on packed pairs: RNE is monotone,
                        // so max(rn(a), rn(b)) == rn(max(a, b)) and half the shuffles go
                        uint32_t w[CW / 2];
#pragma unroll
                        for (int j = 0; j < CW / 2; ++j) {
                            __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                            w[j] = *reinterpret_cast<uint32_t*>(&h2);
                        }
                        if (pool) {
#pragma unroll
                            for (int j = 0; j < CW / 2; ++j) {
                                uint32_t o = __shfl_xor_sync(0xffffffffu, w[j], 1);
                                __nv_bfloat162 m = __hmax2(*reinterpret_cast<__nv_bfloat162*>(&w[j]),
                                                           *reinterpret_cast<__nv_bfloat162*>(&o));
                                w[j] = *reinterpret_cast<uint32_t*>(&m);
                                o = __shfl_xor_sync(0xffffffffu, w[j], ymask);
                                m = __hmax2(*reinterpret_cast<__nv_bfloat162*>(&w[j]),
                                            *reinterpret_cast<__nv_bfloat162*>(&o));
                                w[j] = *reinterpret_cast<uint32_t*>(&m);
                            }
                        }
                        if (MB == 1 && SP != 1 && !pool && a.ep.out_cs - o0 >= CW) {
                            // whole chunk: stored through the lane-group transpose
                            // (one CTA an SM: the 80-register variant would spill;
                            // the tap-pair first layer always pools)
                            constexpr int NV = CW / 8;
                            uint4 pc[NV];
#pragma unroll
                            for (int i = 0; i < NV; ++i) pc[i] = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
                            tc::group_transpose<NV>(pc, lane);
                            const int jj = lane & (NV - 1), gx0 = gx - jj;   // piece jj of pixels gx0 ..
                            __nv_bfloat16* row0 = reinterpret_cast<__nv_bfloat16*>(ybase) +
                                                  (((size_t)img * pH + gy) * pW + gx0) * a.ep.out_cs + o0 + 8 * jj;
#pragma unroll
                            for (int i = 0; i < NV; ++i)
                                if (gy < pH && gx0 + i < pW)
                                    *reinterpret_cast<uint4*>(row0 + (size_t)i * a.ep.out_cs) = pc[i];
                            continue;
                        }
                        if (writer && o0 < a.ep.out_cs) {
                            uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(ybase) +
                                                                  pix * a.ep.out_cs + o0);
                            // out_cs is 16, 32 or a multiple of 64: a 32-channel chunk
                            // may be half outside, a 16-channel one is not
                            const int nvec = (a.ep.out_cs - o0) >= CW ? CW / 8 : 2;
#pragma unroll
                            for (int i = 0; i < CW / 8; ++i)
                                if (i < nvec) dst[i] = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
                        }
                        continue;
                    }
                    if (pool) {
#pragma unroll
                        for (int j = 0; j < CW; ++j) {
                            v[j] = fmaxf(v[j], __shfl_xor_sync(0xffffffffu, v[j], 1));
                            v[j] = fmaxf(v[j], __shfl_xor_sync(0xffffffffu, v[j], ymask));
                        }
                    }
                    if (!writer || o0 >= a.ep.out_cs) continue;
                    if (kOutDt == DT_FP8) {
                        uint4 pk[CW / 16];
                        uint8_t* w8 = reinterpret_cast<uint8_t*>(pk);
#pragma unroll
                        for (int j = 0; j < CW; ++j) w8[j] = f32_to_e4m3_sat(v[j] * a.ep.out_inv_scale);
                        uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(ybase) + pix * a.ep.out_cs + o0);
                        // out_cs is 32, 64 or a multiple of 128 here
#pragma unroll
                        for (int i = 0; i < CW / 16; ++i) dst[i] = pk[i];
                    } else {
                        float* dst = reinterpret_cast<float*>(ybase) + pix * a.ep.out_cs + o0;
#pragma unroll
                        for (int j = 0; j < CW; j += 4)
                            if (o0 + j < a.ep.out_cs)
                                *reinterpret_cast<float4*>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                    }
                }
                if (a.sig) {   // this warp's share of the tile is out: signalled during the next tile
                    if (pend) tc::warp_signal(pend);
                    pend = a.sig + img * pTY + ty;
                }
            }
            if (!released) release();   // a tile without live columns (not produced by the planner)
        }
        // the last tile's band and, every tile of this warp being out, one
        // count toward the kernel's end: one fence for both
        if (pend || a.done_sig) tc::warp_signal(pend, a.done_sig);
        if (lane == 0 && warp == 2) TRACE(6);
        if (lane == 0 && warp == 6) TRACE(7);
    }

    tc::fence_before();
    __syncthreads();
    // CTA pairs: neither CTA leaves while the other may still arrive on its
    // barriers, load into its ring or read its shared memory (cluster
    // split-K: read its partial sums)
    if constexpr (C2 || XR) cluster_sync();
    tc::fence_after();
    if (threadIdx.x == 0) TRACE(8);
#undef TRACE
    __syncwarp();
    if (warp == 1) {
        if constexpr (C2)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                         : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                         : "memory");
    }
}

#undef kKalt
#undef kTapm
#undef kPair
#undef kBres
#undef kKsplit
#undef kAlpha
#undef kOutLayout
#undef kOutDt

// ----------------------------------------------------------------- host
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encode_fn() {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

static CUtensorMapSwizzle swz_of(int chb) {
    return chb == 128  ? CU_TENSOR_MAP_SWIZZLE_128B
           : chb == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
           : chb == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                       : CU_TENSOR_MAP_SWIZZLE_NONE;   // 16-byte chunks (pair mode): plain core matrices
}

int tc_chunk_bytes(int Cp, int dt) {
    const int bytes = Cp * (int)dt_size(dt);
    return bytes >= 128 ? 128 : bytes;   // Cp is 16 (pair mode), 32 or 64 bytes or a multiple of 128
}

cudaError_t tc_encode_act(CUtensorMap* tm, const void* base, int dt, int n, int H, int W, int Cp, int TW,
                          int TH) {
    EncodeTiled enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const int es = (int)dt_size(dt);
    const int chb = tc_chunk_bytes(Cp, dt);
    cuuint64_t dims[4] = {(cuuint64_t)Cp, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)n};
    cuuint64_t strides[3] = {(cuuint64_t)Cp * es, (cuuint64_t)W * Cp * es, (cuuint64_t)H * W * Cp * es};
    cuuint32_t box[4] = {(cuuint32_t)(chb / es), (cuuint32_t)TW, (cuuint32_t)TH, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(tm, dt == DT_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 4,
                     const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz_of(chb),
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t tc_encode_weights(CUtensorMap* tm, const void* w, int dt, int rows, int KK, int Cp, int BN) {
    EncodeTiled enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const int es = (int)dt_size(dt);
    const int chb = tc_chunk_bytes(Cp, dt);
    cuuint64_t dims[2] = {(cuuint64_t)KK * Cp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)KK * Cp * es};
    cuuint32_t box[2] = {(cuuint32_t)(chb / es), (cuuint32_t)BN};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(tm, dt == DT_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                     const_cast<void*>(w), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz_of(chb),
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

constexpr size_t kSmemLimit = 232448;   // opt-in dynamic shared memory per block (227 KB)
constexpr size_t kSmemLimit2 = 115712;  // per block with two blocks an SM (228 KB - 2 x 1 KB reserved, halved)

static size_t tc_ctrl_bytes() {
    return ((sizeof(tc::Smem) + 15) & ~(size_t)15) + 2 * tc::kEpiCols * sizeof(float);
}
static size_t tc_avail(int mb) { return (mb == 2 ? kSmemLimit2 : kSmemLimit) - 1024 - tc_ctrl_bytes(); }

// Ring geometry: as many stages of (A box + B box, or A only with resident
// weights) as fit beside the resident weights and the control block.  CTA
// pairs (cg = 2): a stage holds half of the B box.
static bool tc_geometry(int BN, int chb, int bres, int nk, int mb, int cg, TcArgs* g) {
    // (pair = 2: one box of (TH + 2) x (TW + 2) pixels, the stage rounded to
    // 128 bytes for the copy's destination)
    const size_t a_bytes = g->pair == 2 ? ((size_t)(g->TH + 2) * (g->TW + 2) * chb + 127) / 128 * 128
                           : g->tapm    ? 3 * (size_t)(g->TH + 2) * g->TW * chb
                                        : 128 * (size_t)chb;
    const size_t b_bytes = (size_t)(cg == 2 ? BN / 2 : BN) * chb;
    const size_t st = a_bytes + (bres ? 0 : b_bytes);
    const size_t bres_bytes = bres ? (size_t)(g->pair ? tc::kPairSlots : nk) * b_bytes : 0;
    if (tc_avail(mb) < bres_bytes + 2 * st) return false;
    int nst = (int)std::min<size_t>(tc::kMaxStages, (tc_avail(mb) - bres_bytes) / st) & ~1;
    if (g->nst_cap >= 2) nst = std::min(nst, g->nst_cap & ~1);   // a tuned ring depth
    // producer lanes: four per warp on deep rings (stage count cut to a
    // multiple of eight).  The lanes of a warp issue in lockstep, so on a
    // shallow ring one lane per warp keeps stages refilling one by one.
    int plane = 1;
    if (nst >= 16) {
        plane = 4;
        nst -= nst % 8;
    }
    g->plane = plane;
    g->nst = nst;
    g->st_bytes = (int)st;
    g->bres_off = (int)(nst * st);
    g->ctrl_off = (int)(nst * st + bres_bytes);
    return true;
}

bool tc_b_resident(int BN, int n_tiles, int ksplit, int nk, int chb, int mb) {
    // resident weights must leave room for at least 8 A-only stages (4 with
    // two CTAs an SM)
    const size_t a_st = (mb == 2 ? 4 : 8) * 128 * (size_t)chb;
    (void)n_tiles;   // several N tiles: each CTA keeps its own tile's weights (launch grid a multiple of n_tiles)
    return ksplit == 1 && (size_t)nk * BN * chb + a_st <= tc_avail(mb);
}

template <int BN, int DT, int MB, int CG, int SP = 0>
static cudaError_t launch_tc_bn(const CUtensorMap& tmB, const TcArgs& a0, int workers, cudaStream_t st) {
    TcArgs a = a0;
    // CTA pairs: streamed weights (half a box each), plain stages, one MMA
    // issuer, an even grid of 2-CTA clusters; no fault injection
    if (CG == 2 && (a.bres || a.tapm || a.pair || a.kalt || a.withhold || workers % 2 != 0))
        return cudaErrorInvalidValue;
    // 16-byte chunks (K = 8) only in pair mode, and pair mode only in its one shape
    if ((a.chb == 16) != (a.pair != 0)) return cudaErrorInvalidValue;
    // resident weights: one N tile per CTA, which needs a grid that is a
    // multiple of the N tile count and no K split
    if (a.bres && (a.ksplit != 1 || workers % a.n_tiles != 0)) return cudaErrorInvalidValue;
    if (a.pair && (DT != DT_BF16 || !a.tapm || !a.bres || a.ksplit != 1 || a.k != 3 || a.chunks != 1 || a.kalt))
        return cudaErrorInvalidValue;
    if (a.pair == 2 && (a.TW != 8 || a.TH != 16 || a.chb != 16)) return cudaErrorInvalidValue;   // one box a stage
    if (!tc_geometry(BN, a.chb, a.bres, a.k * a.k * a.chunks, MB, CG, &a)) return cudaErrorInvalidValue;
    if (a.ksplit < 1 || a.n_tiles < 1 || a.chunks < 1 || a.k < 1) return cudaErrorInvalidValue;
    // cluster split-K: clusters of ksplit CTAs (2, 4, 8 or 16, the last a
    // non-portable cluster size; each CTA's share of the columns a multiple
    // of 8), one work item a CTA, one
    // problem, streamed weights, and a ring that holds the 128 x BN FP32
    // partial tile (a tuned ring depth gives way to that)
    if ((SP == 5) != (a.xred != 0)) return cudaErrorInvalidValue;
    // row-band dataflow: single-CTA launches over one problem; a signalling
    // launch writes its final output itself (no workspace reduction after
    // it), and a waiting one touches no workspace either
    if ((a.sig || a.dep || a.rd_sig || a.rd_dep) && (CG != 1 || a.nprob != 1)) return cudaErrorInvalidValue;
    if ((a.sig || a.dep) && a.ksplit > 1 && !a.xred) return cudaErrorInvalidValue;
    if (a.dep && (a.dep_shift < 0 || a.dep_shift > 12 || a.dep_nb < 1 || a.dep_target < 1)) return cudaErrorInvalidValue;
    if (SP == 5) {
        const int S = a.ksplit;
        if ((S != 2 && S != 4 && S != 8 && S != 16) || BN % (8 * S) != 0 || a.nprob != 1 || a.bres || a.tapm || a.pair ||
            a.withhold || workers != a.m_tiles * a.n_tiles * S)
            return cudaErrorInvalidValue;
        if ((size_t)a.nst * a.st_bytes < (size_t)128 * BN * sizeof(float)) {
            a.nst_cap = 0;
            if (!tc_geometry(BN, a.chb, 0, a.k * a.k * a.chunks, MB, CG, &a) ||
                (size_t)a.nst * a.st_bytes < (size_t)128 * BN * sizeof(float))
                return cudaErrorInvalidValue;
        }
    }
    a.fd_ksplit = make_fast_div(a.ksplit);
    a.fd_ntiles = make_fast_div(a.n_tiles);
    a.fd_chunks = make_fast_div(a.chunks);
    a.fd_k = make_fast_div(a.k);
    a.fd_nst = make_fast_div(a.nst);
    if (a.wait_limit <= 0) a.wait_limit = tc::WAIT_LIMIT;
    const size_t smem = 1024 + (size_t)a.ctrl_off + tc_ctrl_bytes();
    if (smem > (MB == 2 ? kSmemLimit2 : kSmemLimit)) return cudaErrorInvalidValue;
    auto kern = conv_tc_kernel<BN, DT, MB, CG, SP>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(MB == 2 ? kSmemLimit2 : kSmemLimit));
        if (e != cudaSuccess) return e;
        if (SP == 5) {   // clusters of 16 CTAs
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
        }
        attr = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)workers);
    cfg.blockDim = dim3(tc::THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    int na = 0;
    if (pdl_enabled()) {
        at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[na].val.programmaticStreamSerializationAllowed = 1;
        ++na;
    }
    if (CG == 2 || SP == 5) {
        at[na].id = cudaLaunchAttributeClusterDimension;
        at[na].val.clusterDim.x = CG == 2 ? 2 : (unsigned)a.ksplit;
        at[na].val.clusterDim.y = 1;
        at[na].val.clusterDim.z = 1;
        ++na;
    }
    cfg.attrs = at;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, kern, tmB, a);
}

template <int BN>
static int xred_capacity_bn(int S) {
    auto kern = conv_tc_kernel<BN, DT_BF16, 1, 1, 5>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(S * 64));
    cfg.blockDim = dim3(tc::THREADS);
    cfg.dynamicSmemBytes = kSmemLimit;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)S;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return clusters * S;
}

int tc_xred_capacity(int BN, int ksplit) {
    if (ksplit != 2 && ksplit != 4 && ksplit != 8 && ksplit != 16) return 0;
    if (BN % (8 * ksplit) != 0) return 0;
    static int cache[3][17] = {};   // (BN 64 / 128 / 256, ksplit); -1: queried, none
    int& c = cache[BN == 64 ? 0 : BN == 128 ? 1 : 2][ksplit];
    if (c == 0) {
        const int v = BN == 64 ? xred_capacity_bn<64>(ksplit)
                    : BN == 128 ? xred_capacity_bn<128>(ksplit)
                    : BN == 256 ? xred_capacity_bn<256>(ksplit) : 0;
        c = v > 0 ? v : -1;
    }
    return c > 0 ? c : 0;
}

cudaError_t conv_tc_launch(const CUtensorMap& tmB, const TcArgs& a, int BN, int dt, int workers, int mb, int cg,
                           cudaStream_t st) {
    if (a.xred) {   // cluster split-K (BF16)
        if (dt != DT_BF16 || mb != 1 || cg != 1) return cudaErrorInvalidValue;
        if (BN == 64) return launch_tc_bn<64, DT_BF16, 1, 1, 5>(tmB, a, workers, st);
        if (BN == 128) return launch_tc_bn<128, DT_BF16, 1, 1, 5>(tmB, a, workers, st);
        if (BN == 256) return launch_tc_bn<256, DT_BF16, 1, 1, 5>(tmB, a, workers, st);
        return cudaErrorInvalidValue;
    }
    if (cg == 2) {
        if (mb != 1) return cudaErrorInvalidValue;
        if (dt == DT_BF16 && BN == 128) return launch_tc_bn<128, DT_BF16, 1, 2>(tmB, a, workers, st);
        if (dt == DT_BF16 && BN == 256) return launch_tc_bn<256, DT_BF16, 1, 2>(tmB, a, workers, st);
        if (dt == DT_FP8 && BN == 128) return launch_tc_bn<128, DT_FP8, 1, 2>(tmB, a, workers, st);
        if (dt == DT_FP8 && BN == 256) return launch_tc_bn<256, DT_FP8, 1, 2>(tmB, a, workers, st);
        return cudaErrorInvalidValue;
    }
    if (cg != 1) return cudaErrorInvalidValue;
    // BF16 layers run specialised variants: with a K split SP = 3; without
    // one and with BF16 NHWC output, the tap-pair first layer SP = 1 and the
    // others SP = 2; a last layer with FP32 NCHW output SP = 4 (NET_TC_SPEC=0:
    // the generic kernel)
    static const bool spec_on = [] {
        const char* e = getenv("NET_TC_SPEC");
        return !(e && atoi(e) == 0);
    }();
    if (spec_on && dt == DT_BF16 && a.ksplit > 1 && !a.pair) {   // split-K partial sums
        if (mb == 1) {
            if (BN == 64) return launch_tc_bn<64, DT_BF16, 1, 1, 3>(tmB, a, workers, st);
            if (BN == 128) return launch_tc_bn<128, DT_BF16, 1, 1, 3>(tmB, a, workers, st);
            if (BN == 256) return launch_tc_bn<256, DT_BF16, 1, 1, 3>(tmB, a, workers, st);
        }
    }
    if (spec_on && dt == DT_BF16 && a.ksplit == 1 && !a.pair && a.ep.out_layout == LAYOUT_NCHW &&
        a.ep.out_dt == DT_F32 && !a.ep.alpha && mb == 1) {   // the last layer
        if (BN == 64) return launch_tc_bn<64, DT_BF16, 1, 1, 4>(tmB, a, workers, st);
        if (BN == 128) return launch_tc_bn<128, DT_BF16, 1, 1, 4>(tmB, a, workers, st);
        if (BN == 256) return launch_tc_bn<256, DT_BF16, 1, 1, 4>(tmB, a, workers, st);
    }
    if (spec_on && dt == DT_BF16 && a.ksplit == 1 && a.ep.out_layout == LAYOUT_NHWC && a.ep.out_dt == DT_BF16 &&
        !a.ep.alpha) {
        if (a.pair && a.tapm && a.bres && !a.kalt) {
            if (BN == 64 && mb == 1) return launch_tc_bn<64, DT_BF16, 1, 1, 1>(tmB, a, workers, st);
            if (BN == 128 && mb == 1) return launch_tc_bn<128, DT_BF16, 1, 1, 1>(tmB, a, workers, st);
        } else if (!a.pair) {
            if (mb == 1) {
                if (BN == 64) return launch_tc_bn<64, DT_BF16, 1, 1, 2>(tmB, a, workers, st);
                if (BN == 128) return launch_tc_bn<128, DT_BF16, 1, 1, 2>(tmB, a, workers, st);
                if (BN == 256) return launch_tc_bn<256, DT_BF16, 1, 1, 2>(tmB, a, workers, st);
            } else if (mb == 2) {
                if (BN == 64) return launch_tc_bn<64, DT_BF16, 2, 1, 2>(tmB, a, workers, st);
                if (BN == 128) return launch_tc_bn<128, DT_BF16, 2, 1, 2>(tmB, a, workers, st);
            }
        }
    }
    if (mb == 2) {
        if (dt == DT_BF16 && BN == 64) return launch_tc_bn<64, DT_BF16, 2, 1>(tmB, a, workers, st);
        if (dt == DT_BF16 && BN == 128) return launch_tc_bn<128, DT_BF16, 2, 1>(tmB, a, workers, st);
        if (dt == DT_FP8 && BN == 64) return launch_tc_bn<64, DT_FP8, 2, 1>(tmB, a, workers, st);
        if (dt == DT_FP8 && BN == 128) return launch_tc_bn<128, DT_FP8, 2, 1>(tmB, a, workers, st);
        return cudaErrorInvalidValue;
    }
    if (mb != 1) return cudaErrorInvalidValue;
    if (dt == DT_BF16) {
        if (BN == 64) return launch_tc_bn<64, DT_BF16, 1, 1>(tmB, a, workers, st);
        if (BN == 128) return launch_tc_bn<128, DT_BF16, 1, 1>(tmB, a, workers, st);
        if (BN == 256) return launch_tc_bn<256, DT_BF16, 1, 1>(tmB, a, workers, st);
    } else if (dt == DT_FP8) {
        if (BN == 64) return launch_tc_bn<64, DT_FP8, 1, 1>(tmB, a, workers, st);
        if (BN == 128) return launch_tc_bn<128, DT_FP8, 1, 1>(tmB, a, workers, st);
        if (BN == 256) return launch_tc_bn<256, DT_FP8, 1, 1>(tmB, a, workers, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dn
