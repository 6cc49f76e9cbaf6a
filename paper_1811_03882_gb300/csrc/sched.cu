// sched.cu — uneven-batch execution and the serving request queue.
#include <cuda_runtime.h>

#include "../../include/net.h"
#include "net_internal.h"

using namespace dn;

net_status dn::enqueue_uneven(net* n, const float* const* d_in, const int* side, int cnt,
                              float* const* d_out) {
    for (int i = 0; i < cnt; ++i) {
        net_status s = enqueue_forward(n, d_in[i], 1, side[i], side[i], d_out[i], nullptr, false, nullptr);
        if (s != NET_OK) return s;
    }
    return NET_OK;
}

void dn::uneven_free(net*) {}
void dn::serve_stop(net*) {}

extern "C" net_status net_submit(net_t*, const float*, int, int, uint64_t*) {
    return fail(NET_E_UNSUPPORTED, "request queue not built yet");
}
extern "C" net_status net_poll(net_t*, uint64_t, float*, size_t, int*) {
    return fail(NET_E_UNSUPPORTED, "request queue not built yet");
}
extern "C" net_status net_wait(net_t*, uint64_t, float*, size_t, int) {
    return fail(NET_E_UNSUPPORTED, "request queue not built yet");
}
extern "C" net_status net_stats(net_t*, double*, double*, double*) {
    return fail(NET_E_UNSUPPORTED, "request queue not built yet");
}
