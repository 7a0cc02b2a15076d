// Host side of the multi-feature run (fcm_run_multi).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>

#include "fcm.h"
#include "fcm_multi.h"
#include "fcm_runtime.h"

namespace fcm {

struct MultiWorkspace {
    MultiState* d_st = nullptr;
    MultiState* h_st = nullptr;  // pinned
    float* partials = nullptr;
    int64_t partial_floats = 0;
    std::map<const void*, int> occupancy;
};

}  // namespace fcm

using namespace fcm;

namespace {

MultiTable g_multi;
std::once_flag g_multi_once;

const MultiTable& multi_table() {
    std::call_once(g_multi_once, [] {
        std::memset(&g_multi, 0, sizeof(g_multi));
        register_multi_d1(g_multi);
        register_multi_d2(g_multi);
        register_multi_d3(g_multi);
        register_multi_d4(g_multi);
    });
    return g_multi;
}

bool dev_ptr(const void* p) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return ctx_fail(h, e_, #call); \
    } while (0)

void fcm_release_multi(fcm_ctx* h) {
    if (!h || !h->multi) return;
    MultiWorkspace* w = h->multi;
    cudaFree(w->d_st);
    cudaFree(w->partials);
    cudaFreeHost(w->h_st);
    delete w;
    h->multi = nullptr;
}

extern "C" int fcm_run_multi(fcm_handle h, const float* x, int64_t n, int D, int C, float m, float eps,
                             int max_iter, int init_mode, const float* U0, float* U, float* V, double* V64,
                             fcm_report* rep) {
    NvtxRange nvtx_range("fcm_run_multi");
    if (!h) return FCM_ERR_INVALID_ARG;
    if (!x || !U || !V) return ctx_invalid(h, "null x, U or V");
    if (n < 1 || n > ((int64_t)1 << 40)) return ctx_invalid(h, "n must be in [1, 2^40]");
    if (D < 1 || D > MULTI_MAX_D) return ctx_invalid(h, "D must be in [1, 4]");
    if (C < 1 || C > FCM_MAX_CLUSTERS) return ctx_invalid(h, "C must be in [1, 8]");
    if (!(m > 1.0f) || !std::isfinite(m)) return ctx_invalid(h, "m must be a finite number > 1");
    if (!(eps >= 0.0f) || !std::isfinite(eps)) return ctx_invalid(h, "eps must be finite and >= 0");
    if (max_iter < 1) return ctx_invalid(h, "max_iter must be >= 1");
    if (init_mode != FCM_INIT_U && init_mode != FCM_INIT_V) return ctx_invalid(h, "bad init_mode");
    const bool from_u = init_mode == FCM_INIT_U;
    if (from_u && !U0) U0 = U;
    if (!dev_ptr(x) || !dev_ptr(U) || (from_u && !dev_ptr(U0)))
        return ctx_invalid(h, "x, U and U0 must be device memory");
    if (!h->coop) return ctx_invalid(h, "the multi-feature run needs cooperative launch support");
    const bool V_dev = dev_ptr(V);
    DeviceGuard g(h->device);
    if (!h->multi) h->multi = new MultiWorkspace();
    MultiWorkspace* w = h->multi;
    if (!w->d_st) CK(dev_malloc(h, &w->d_st, sizeof(MultiState)));
    if (!w->h_st) CK(host_malloc(h, &w->h_st, sizeof(MultiState)));
    const MultiTable& t = multi_table();
    const MultiFn fn = t.run[D][C][m == 2.0f ? 0 : 1][from_u ? 0 : 1];
    int per_sm = 0;
    auto it = w->occupancy.find((const void*)fn);
    if (it != w->occupancy.end()) {
        per_sm = it->second;
    } else {
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)fn, 256, 0));
        w->occupancy[(const void*)fn] = per_sm;
    }
    if (per_sm < 1) return ctx_invalid(h, "the multi-feature kernel does not fit on this device");
    const int64_t want = (n + 256 * 4 - 1) / (256 * 4);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)per_sm * h->num_sms));
    const int64_t S = (int64_t)C * D + C + 1 + 3;
    const int64_t need = 2 * 2 * S * blocks;
    if (w->partial_floats < need) {
        cudaFree(w->partials);
        w->partials = nullptr;
        w->partial_floats = 0;
        CK(dev_malloc(h, &w->partials, sizeof(float) * need));
        w->partial_floats = need;
    }
    MultiState* hs = w->h_st;
    std::memset(hs, 0, sizeof(MultiState));
    hs->x = x;
    hs->U0 = from_u ? U0 : nullptr;
    hs->U = U;
    hs->n = n;
    hs->m = m;
    hs->inv_m1 = (float)(1.0 / ((double)m - 1.0));
    hs->eps = eps;
    hs->max_iter = max_iter;
    hs->status = FCM_ERR_TIMEOUT;
    hs->lim = h->limits;
    if (!from_u && !V_dev) std::memcpy(hs->V0, V, sizeof(float) * C * D);
    CK(cudaMemcpyAsync(w->d_st, hs, sizeof(MultiState), cudaMemcpyHostToDevice, h->stream));
    if (!from_u && V_dev)
        CK(cudaMemcpyAsync(&w->d_st->V0, V, sizeof(float) * C * D, cudaMemcpyDeviceToDevice, h->stream));
    MultiState* dst = w->d_st;
    float* part = w->partials;
    void* args[2] = {&dst, &part};
    CK(cudaLaunchCooperativeKernel((const void*)fn, dim3(blocks), dim3(256), args, 0, h->stream));
    CK(cudaMemcpyAsync(hs, w->d_st, sizeof(MultiState), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(V, &w->d_st->V, sizeof(float) * C * D,
                       V_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (V64) std::memcpy(V64, hs->V64, sizeof(double) * C * D);
    if (rep) {
        std::memset(rep, 0, sizeof(*rep));
        rep->iters = hs->iters;
        rep->status = hs->status;
        rep->flags = hs->flags;
        rep->C = C;
        rep->delta = hs->delta;
        rep->J = hs->J;
        for (int j = 0; j < std::min(C * D, FCM_MAX_CLUSTERS); ++j) rep->V64[j] = hs->V64[j];
        rep->launches = 1;
    }
    return hs->status;
}
