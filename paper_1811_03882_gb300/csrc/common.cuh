// common.cuh — shared device/host definitions of the CUDA library.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include <utility>

namespace dn {

enum { ACT_LINEAR = 0, ACT_LEAKY = 1 };
enum { POOL_NONE = 0, POOL_S2 = 1, POOL_S1SAME = 2 };
enum { DT_F32 = 0, DT_BF16 = 1, DT_FP8 = 2 };
enum { LAYOUT_NHWC = 0, LAYOUT_NCHW = 1 };

constexpr float kLeakySlope = 0.1f;
constexpr double kBnEps = 1e-5;
constexpr float kFp8Max = 448.f;

__host__ __device__ static inline int cdiv(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ static inline int rup(int a, int b) { return cdiv(a, b) * b; }
__host__ __device__ static inline size_t dt_size(int dt) { return dt == DT_F32 ? 4 : dt == DT_BF16 ? 2 : 1; }

// Channel padding of an NHWC activation stored in dtype `dt`: rows of whole
// 16-byte vectors; tensor-core operands additionally need 32/64/128-byte
// K chunks (16/32/multiple-of-64 BF16 channels, 32/64/multiple-of-128 FP8).
static inline int pad_channels(int c, int dt, bool tensor_core) {
    if (dt == DT_F32) return rup(c, 4);
    int v = dt == DT_BF16 ? 8 : 16;           // elements per 16 bytes
    if (!tensor_core) return rup(c, v);
    int row = 128 / (int)dt_size(dt);         // elements per 128-byte row
    if (c <= row / 4) return row / 4;
    if (c <= row / 2) return row / 2;
    return rup(c, row);
}

// Epilogue of a conv tile: acc * alpha[o] + bias[o] -> activation ->
// optional 2x2/s2 max -> store in the output dtype/layout.
struct Epilogue {
    const float* bias;    // [cout]
    const float* alpha;   // [cout] multiplier of the accumulator, or nullptr
    int act;              // ACT_*
    int pool;             // POOL_NONE or POOL_S2 (fused); S1SAME runs separately
    int out_dt;           // DT_*
    int out_layout;       // LAYOUT_NHWC (channel stride out_cs) or LAYOUT_NCHW (float)
    int out_cs;           // NHWC channel stride (padded count)
    float out_inv_scale;  // FP8 output: code = value * out_inv_scale
    int cout;             // real output channels
};

__device__ __forceinline__ float act_apply(float v, int act) {
    return (act == ACT_LEAKY) ? (v > 0.f ? v : kLeakySlope * v) : v;
}

__device__ __forceinline__ uint8_t f32_to_e4m3_sat(float v) {
    return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

__device__ __forceinline__ float e4m3_to_f32(uint8_t b) {
    __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)b, __NV_E4M3);
    return __half2float(__half(h));
}

// Programmatic dependent launch.  A kernel launched with launch_pdl may be
// scheduled while the previous kernel in its stream is still finishing:
// pdl_trigger lets the next kernel start its own prologue early, and
// pdl_wait blocks until every earlier kernel of the stream has completed and
// its writes are visible, so it must come before the first global access.
// Both are no-ops for a kernel launched the ordinary way.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Whether launches use the programmatic-serialisation attribute (on unless
// NET_PDL=0 in the environment).
bool pdl_enabled();

template <typename... KArgs, typename... Args>
static inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                     Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace dn
