// Host check of make_fast_div (the tensor-core kernel's tile decode): for
// every divisor d used by a launch, n / d == (mulhi(n, m) + n) >> l with the
// constants it computes, for 0 <= n < 2^31.  Prints "OK" or the first
// failing (d, n).
#include <cstdio>
#include <cstdint>
#include "kernels.h"

static int q_of(uint32_t n, dn::FastDiv f) {
    const uint32_t hi = (uint32_t)(((uint64_t)n * f.mul) >> 32);
    return (int)((hi + n) >> f.shift);
}

int main() {
    uint64_t state = 0x9E3779B97F4A7C15ull;
    auto next = [&]() {   // SplitMix64
        uint64_t z = (state += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    const int big[] = {12544, 3136, 784, 65535, 65536, 1 << 20, 999999, 2147483647};
    for (int t = 0; t < 4096 + 8; ++t) {
        const int d = t < 4096 ? t + 1 : big[t - 4096];
        const dn::FastDiv f = dn::make_fast_div(d);
        for (int k = 0; k < 3000; ++k) {
            uint32_t n;
            if (k < 1000) n = (uint32_t)k;                                // small numerators
            else if (k < 2000) n = (uint32_t)((uint64_t)(k - 999) * d - (k & 1));   // around multiples of d
            else n = (uint32_t)(next() & 0x7FFFFFFFu);                    // random below 2^31
            if (n > 0x7FFFFFFFu) continue;
            if (q_of(n, f) != (int)(n / (uint32_t)d)) {
                printf("FAIL d=%d n=%u\n", d, n);
                return 1;
            }
        }
        const uint32_t top = 0x7FFFFFFFu;
        if (q_of(top, f) != (int)(top / (uint32_t)d)) {
            printf("FAIL d=%d n=%u\n", d, top);
            return 1;
        }
    }
    printf("OK\n");
    return 0;
}
