// guard.cu — canary guard regions around the library's device buffers.
//
// A debug aid for out-of-bounds writes (compute-sanitizer is not used):
// with NET_GUARD=1 in the environment (read once, at the process's first
// allocation), every device buffer the library allocates gets a 4 KB region
// of 0xA5 bytes directly before and directly after it.  A buffer's regions
// are compared with the pattern when it is freed, and those of every live
// buffer when net_guard_check runs (copied back to the host after a device
// synchronisation); net_guard_check reports both.  A kernel that writes past
// either end of a buffer, even by one byte, changes a region.  Without the
// variable, allocation is a plain cudaMalloc.
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/net.h"
#include "common.cuh"
#include "net_internal.h"

namespace {

constexpr size_t kGuard = 4096;            // bytes before and after each buffer
constexpr unsigned char kPattern = 0xA5;

struct Region {
    unsigned char* base;   // the cudaMalloc'd block: guard, buffer, guard
    size_t bytes;          // the buffer's size
    int device;
};

std::mutex g_mu;
uint64_t g_freed = 0, g_freed_bad = 0;   // buffers checked at their free, and changed ones
std::map<const void*, Region>& regions() {   // by buffer address, in address order
    static std::map<const void*, Region> m;
    return m;
}

bool guards_enabled() {
    static const bool on = [] {
        const char* e = getenv("NET_GUARD");
        return e && atoi(e) == 1;
    }();
    return on;
}

// Whether either region of r still holds the pattern everywhere (false and
// *err set when a copy fails).  The device is synchronised first.
bool regions_intact(const Region& r, cudaError_t* err) {
    std::vector<unsigned char> h(kGuard);
    *err = cudaSetDevice(r.device);
    if (*err == cudaSuccess) *err = cudaDeviceSynchronize();
    for (int side = 0; side < 2 && *err == cudaSuccess; ++side) {
        const unsigned char* g = side ? r.base + kGuard + r.bytes : r.base;
        *err = cudaMemcpy(h.data(), g, kGuard, cudaMemcpyDeviceToHost);
        if (*err != cudaSuccess) break;
        for (size_t i = 0; i < kGuard; ++i)
            if (h[i] != kPattern) return false;
    }
    return true;
}

}  // namespace

namespace dn {

cudaError_t dalloc_raw(void** p, size_t bytes) {
    if (!guards_enabled()) return cudaMalloc(p, bytes);
    *p = nullptr;
    unsigned char* base = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&base), bytes + 2 * kGuard);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemset(base, kPattern, kGuard)) != cudaSuccess ||
        (e = cudaMemset(base + kGuard + bytes, kPattern, kGuard)) != cudaSuccess) {
        cudaFree(base);
        return e;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    *p = base + kGuard;
    std::lock_guard<std::mutex> lk(g_mu);
    regions()[*p] = Region{base, bytes, dev};
    return cudaSuccess;
}

cudaError_t dfree(void* p) {
    if (!p) return cudaSuccess;
    if (guards_enabled()) {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = regions().find(p);
        if (it != regions().end()) {
            const Region r = it->second;
            regions().erase(it);
            int cur = 0;
            cudaGetDevice(&cur);
            cudaError_t e = cudaSuccess;
            const bool ok = regions_intact(r, &e);
            ++g_freed;
            if (!ok && e == cudaSuccess) ++g_freed_bad;
            cudaSetDevice(cur);
            return cudaFree(r.base);
        }
    }
    return cudaFree(p);
}

}  // namespace dn

extern "C" net_status net_guard_check(uint64_t* buffers, uint64_t* corrupted) {
    if (!buffers || !corrupted) return dn::fail(NET_E_INVAL, "NULL argument");
    *buffers = 0;
    *corrupted = 0;
    if (!guards_enabled()) return NET_OK;
    std::lock_guard<std::mutex> lk(g_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    uint64_t n = g_freed, bad = g_freed_bad;
    for (auto& kv : regions()) {
        cudaError_t e = cudaSuccess;
        const bool ok = regions_intact(kv.second, &e);
        if (e != cudaSuccess) {
            cudaSetDevice(cur);
            return dn::fail(NET_E_CUDA, "guard check: %s", cudaGetErrorString(e));
        }
        ++n;
        if (!ok) ++bad;
    }
    cudaSetDevice(cur);
    *buffers = n;
    *corrupted = bad;
    return NET_OK;
}

extern "C" net_status net_guard_poke(uint64_t index) {
    if (!guards_enabled()) return dn::fail(NET_E_STATE, "guard regions are off (NET_GUARD=1 enables them)");
    std::lock_guard<std::mutex> lk(g_mu);
    if (index >= regions().size()) return dn::fail(NET_E_INVAL, "buffer %llu of %zu", (unsigned long long)index,
                                                   regions().size());
    auto it = regions().begin();
    std::advance(it, (long)index);
    const Region& r = it->second;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(r.device);
    // the first byte after the buffer: what a one-element overrun writes
    const cudaError_t e = cudaMemset(r.base + kGuard + r.bytes, 0, 1);
    cudaSetDevice(cur);
    if (e != cudaSuccess) return dn::fail(NET_E_CUDA, "guard poke: %s", cudaGetErrorString(e));
    return NET_OK;
}
