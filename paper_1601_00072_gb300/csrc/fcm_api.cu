// Host runtime and C ABI of the single-image FCM path.
//
// A handle owns a device workspace (run state, per-block partials, optional
// trace, staging buffers for host inputs) and one instantiated CUDA graph per
// launch shape. A graph is
//
//     first pass (P_ACCUM0 or P_INITV)  ->  WHILE(cond) { P_ITER pass }
//
// where the last block of every pass sets `cond` with
// cudaGraphSetConditional, so the whole of Algorithm 1 (arXiv:1601.00072,
// Sec. 2.1) runs on the device after one graph launch. The paper copies U to
// the host every iteration to test convergence (Sec. 4.3); here the only
// host-device traffic of a run is the 200-byte state upload, the state
// read-back and, for host buffers, the input/output copies.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "fcm.h"
#include "fcm_device.cuh"
#include "fcm_internal.h"
#include "fcm_recompute.h"
#include "fcm_runtime.h"

using namespace fcm;

namespace {

SingleTable g_table;
std::once_flag g_table_once;
RcTable g_rc;

void init_table() {
    std::memset(&g_table, 0, sizeof(g_table));
    std::memset(&g_rc, 0, sizeof(g_rc));
    register_rc_c1(g_rc);
    register_rc_c2(g_rc);
    register_rc_c3(g_rc);
    register_rc_c4(g_rc);
    register_rc_c5(g_rc);
    register_rc_c6(g_rc);
    register_rc_c7(g_rc);
    register_rc_c8(g_rc);
    register_single_c1(g_table);
    register_single_c2(g_table);
    register_single_c3(g_table);
    register_single_c4(g_table);
    register_single_c5(g_table);
    register_single_c6(g_table);
    register_single_c7(g_table);
    register_single_c8(g_table);
}

// Default wait bounds of a handle; FCM_TIMEOUT_SPINS overrides the grid
// barrier's.
WaitLimits default_limits() {
    WaitLimits w{DEFAULT_GRID_SPINS, DEFAULT_TMA_POLLS, 0u, 0u};
    if (const char* e = std::getenv("FCM_TIMEOUT_SPINS")) {
        const long long v = std::atoll(e);
        if (v > 0 && v <= 0xffffffffll) w.grid_spins = (uint32_t)v;
    }
    return w;
}

// Percent of a pass's tiles the whole-run kernel deals in fixed warp shares;
// FCM_RUN_STATIC_PCT overrides the default (100: fixed shares only).
int default_static_pct() {
    if (const char* e = std::getenv("FCM_RUN_STATIC_PCT")) {
        const long v = std::atol(e);
        if (v >= 1 && v <= 100) return (int)v;
    }
    return DEFAULT_STATIC_PCT;
}

// Grid of a whole-run kernel for n pixels when at most max_blocks blocks are
// co-resident: the fewest blocks that keep the largest number of 128-pixel
// tiles per warp that max_blocks would give, so every warp holds about the
// same number of tiles (8,192 tiles on 304 blocks would leave a third of the
// warps one tile more than the rest; 256 blocks give each warp 4).
int run_grid(int64_t n, int64_t max_blocks) {
    if (max_blocks < 1) return 0;
    const int64_t ntiles = (n + WARP_TILE - 1) / WARP_TILE;
    const int64_t per_warp = (ntiles + max_blocks * NWARP - 1) / (max_blocks * NWARP);
    return (int)std::max<int64_t>(1, (ntiles + per_warp * NWARP - 1) / (per_warp * NWARP));
}

bool is_device_pointer(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

namespace fcm {

const SingleTable& single_table() {
    std::call_once(g_table_once, init_table);
    return g_table;
}

int ctx_fail(fcm_ctx* h, cudaError_t e, const char* what) {
    cudaGetLastError();  // a failed call leaves its error as the last one: clear it for the next check
    if (h) {
        char buf[256];
        std::snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
        h->last_error = buf;
    }
    return e == cudaErrorMemoryAllocation ? FCM_ERR_OOM : FCM_ERR_CUDA;
}

int ctx_invalid(fcm_ctx* h, const char* what) {
    if (h) h->last_error = what;
    return FCM_ERR_INVALID_ARG;
}

// Counts down the injected failure of fcm_set_limits: true when this
// allocation is the one to fail.
static bool injected_failure(fcm_ctx* h) {
    if (!h || h->alloc_fail_in <= 0) return false;
    return --h->alloc_fail_in == 0;
}

cudaError_t dev_malloc_raw(fcm_ctx* h, void** p, size_t bytes) {
    if (injected_failure(h)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t host_malloc_raw(fcm_ctx* h, void** p, size_t bytes) {
    if (injected_failure(h)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocHost(p, bytes);
}

int ctx_grow(fcm_ctx* h, void** p, size_t* cap, size_t bytes, const char* what) {
    if (*cap >= bytes) return 0;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = dev_malloc_raw(h, p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return ctx_fail(h, e, what);
    }
    *cap = bytes;
    return 0;
}

}  // namespace fcm

#define CK(call)                                                  \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return ctx_fail(h, e_, #call);     \
    } while (0)

namespace {

// Each buffer is allocated when missing, so a call after a failed allocation
// completes the workspace.
int ensure_single_workspace(fcm_ctx* h) {
    if (!h->d_st) {
        CK(dev_malloc(h, &h->d_st, sizeof(RunState)));
        CK(cudaMemset(h->d_st, 0, sizeof(RunState)));
    }
    if (!h->h_st) CK(host_malloc(h, &h->h_st, sizeof(RunState)));
    if (!h->d_partials) {
        h->partial_blocks = h->num_sms * 32;
        CK(dev_malloc(h, &h->d_partials, sizeof(double) * SLOTS_MAX * h->partial_blocks));
    }
    return 0;
}

// Blocks per SM of a pass kernel with `smem` bytes of dynamic shared memory;
// the first call also raises the kernel's dynamic shared memory limit.
int blocks_per_sm(fcm_ctx* h, const void* k, int smem) {
    auto it = h->occupancy.find(k);
    if (it != h->occupancy.end()) return it->second;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NT, smem) != cudaSuccess) {
        cudaGetLastError();
        nb = 0;
    }
    h->occupancy[k] = nb;
    return nb;
}

struct Launch {
    PassFn kfirst, kiter;
    int smem_first, smem_iter, var, nblocks;
};

// Kernel variant and grid of a run. The TMA ring needs n % 4 == 0 and 16-byte
// aligned rows (every bulk copy starts and ends on a 16-byte boundary).
int choose_launch(fcm_ctx* h, int64_t n, int C, int mk, int pass0, const void* x, const void* U,
                  const void* Uprev, int options, Launch* L) {
    const bool aligned = (n % 4 == 0) && ((uintptr_t)x % 16 == 0) && ((uintptr_t)U % 16 == 0) &&
                         ((uintptr_t)Uprev % 16 == 0);
    int var = aligned && !(options & FCM_OPT_NO_TMA) ? 1 : 0;
    int bps = 0, bps0 = 0;
    for (; var >= 0; --var) {
        bps = blocks_per_sm(h, (const void*)g_table.k[C][mk][P_ITER][var], g_table.smem[C][mk][P_ITER][var]);
        bps0 = blocks_per_sm(h, (const void*)g_table.k[C][mk][pass0][var], g_table.smem[C][mk][pass0][var]);
        if (bps > 0 && bps0 > 0) break;
    }
    if (var < 0) {
        h->last_error = "no pass kernel fits on this device";
        return FCM_ERR_CUDA;
    }
    L->var = var;
    L->kfirst = g_table.k[C][mk][pass0][var];
    L->kiter = g_table.k[C][mk][P_ITER][var];
    L->smem_first = g_table.smem[C][mk][pass0][var];
    L->smem_iter = g_table.smem[C][mk][P_ITER][var];
    const int64_t per_block = var == 1 ? 4 * NT : NT;  // pixels one block covers per step
    const int64_t want = (n + per_block - 1) / per_block;
    L->nblocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)h->num_sms * std::min(bps, bps0)));
    return 0;
}

int build_graph(fcm_ctx* h, PassFn kfirst, int smem_first, PassFn kiter, int smem_iter, int nblocks,
                GraphEntry* out) {
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle cond;
    cudaError_t e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return ctx_fail(h, e, "cudaGraphConditionalHandleCreate");
    }
    int use_cond = 1;
    void* args[4] = {&h->d_st, &h->d_partials, &cond, &use_cond};
    cudaKernelNodeParams kp;
    std::memset(&kp, 0, sizeof(kp));
    kp.func = (void*)kfirst;
    kp.gridDim = dim3(nblocks);
    kp.blockDim = dim3(NT);
    kp.sharedMemBytes = smem_first;
    kp.kernelParams = args;
    cudaGraphNode_t n1, n2, n3;
    e = cudaGraphAddKernelNode(&n1, g, nullptr, 0, &kp);
    // cudaGraphNodeParams holds a union without a default constructor:
    // zero-initialised raw storage stands in for it.
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
    std::memset(cp_raw, 0, sizeof(cp_raw));
    cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (e == cudaSuccess) e = cudaGraphAddNode(&n2, g, &n1, nullptr, 1, &cp);
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        kp.func = (void*)kiter;
        kp.sharedMemBytes = smem_iter;
        e = cudaGraphAddKernelNode(&n3, body, nullptr, 0, &kp);
    }
    cudaGraphExec_t ex = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return ctx_fail(h, e, "building the FCM graph");
    }
    out->graph = g;
    out->exec = ex;
    return 0;
}

int run_host_loop(fcm_ctx* h, PassFn kfirst, int smem_first, PassFn kiter, int smem_iter, int nblocks) {
    const cudaGraphConditionalHandle none = 0;
    kfirst<<<nblocks, NT, smem_first, h->stream>>>(h->d_st, h->d_partials, none, 0);
    CK(cudaGetLastError());
    int chunk = 4;
    int launched = 0;
    const int max_iter = h->h_st->max_iter;
    int* done_host = &h->h_done;
    while (true) {
        const int todo = std::min(chunk, max_iter - launched);
        for (int t = 0; t < todo; ++t)
            kiter<<<nblocks, NT, smem_iter, h->stream>>>(h->d_st, h->d_partials, none, 0);
        CK(cudaGetLastError());
        launched += todo;
        h->last_launches = 1 + launched;
        CK(cudaMemcpyAsync(done_host, &h->d_st->done, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        if (*done_host || launched >= max_iter) break;
        chunk = std::min(chunk * 2, 64);
    }
    return 0;
}

}  // namespace

extern "C" {

int fcm_create(fcm_handle* out, int device, void* cuda_stream) {
    if (!out) return FCM_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return FCM_ERR_CUDA;
    }
    std::call_once(g_table_once, init_table);
    fcm_ctx* h = new fcm_ctx();
    h->device = device;
    h->stream = (cudaStream_t)cuda_stream;
    DeviceGuard g(device);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete h;
        return FCM_ERR_CUDA;
    }
    h->num_sms = prop.multiProcessorCount;
    int coop = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess) coop = 0;
    h->coop = coop != 0;
    h->max_smem_optin = (int)prop.sharedMemPerBlockOptin;
    h->device_name = prop.name;
    h->limits = default_limits();
    h->static_pct = default_static_pct();
    *out = h;
    return FCM_OK;
}

int fcm_set_limits(fcm_handle h, const fcm_limits* lim) {
    if (!h) return FCM_ERR_INVALID_ARG;
    const WaitLimits dflt = default_limits();
    if (!lim) {
        h->limits = dflt;
        h->alloc_fail_in = 0;
        return FCM_OK;
    }
    if (lim->barrier_phantoms > 1024u || lim->fail_alloc_in < 0)
        return ctx_invalid(h, "limits: barrier_phantoms <= 1024 and fail_alloc_in >= 0");
    h->limits.grid_spins = lim->grid_wait_spins ? lim->grid_wait_spins : dflt.grid_spins;
    h->limits.tma_polls = lim->tma_wait_polls ? lim->tma_wait_polls : DEFAULT_TMA_POLLS;
    h->limits.phantoms = lim->barrier_phantoms;
    h->alloc_fail_in = lim->fail_alloc_in;
    return FCM_OK;
}

int fcm_get_limits(fcm_handle h, fcm_limits* lim) {
    if (!h || !lim) return FCM_ERR_INVALID_ARG;
    std::memset(lim, 0, sizeof(*lim));
    lim->grid_wait_spins = h->limits.grid_spins;
    lim->tma_wait_polls = h->limits.tma_polls;
    lim->barrier_phantoms = h->limits.phantoms;
    lim->fail_alloc_in = h->alloc_fail_in;
    return FCM_OK;
}

int fcm_set_stream(fcm_handle h, void* cuda_stream) {
    if (!h) return FCM_ERR_INVALID_ARG;
    h->stream = (cudaStream_t)cuda_stream;
    return FCM_OK;
}

void fcm_destroy(fcm_handle h) {
    if (!h) return;
    {
        DeviceGuard g(h->device);
        cudaStreamSynchronize(h->stream);
        for (auto& kv : h->graphs) {
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
            if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
        }
        if (h->d_st) cudaFree(h->d_st);
        if (h->h_st) cudaFreeHost(h->h_st);
        if (h->d_partials) cudaFree(h->d_partials);
        if (h->d_trace) cudaFree(h->d_trace);
        if (h->d_stage_x) cudaFree(h->d_stage_x);
        if (h->d_stage_U) cudaFree(h->d_stage_U);
        if (h->pipe_in) cudaStreamSynchronize(h->pipe_in);
        if (h->pipe_out) cudaStreamSynchronize(h->pipe_out);
        for (int b = 0; b < fcm_ctx::PIPE_SETS; ++b) {
            if (h->d_pipe_x[b]) cudaFree(h->d_pipe_x[b]);
            if (h->d_pipe_U[b]) cudaFree(h->d_pipe_U[b]);
        }
        if (h->h_pipe_st) cudaFreeHost(h->h_pipe_st);
        for (cudaEvent_t ev : h->pipe_ev)
            if (ev) cudaEventDestroy(ev);
        if (h->pipe_in) cudaStreamDestroy(h->pipe_in);
        if (h->pipe_out) cudaStreamDestroy(h->pipe_out);
        fcm_release_batched(h);
        fcm_release_mlp(h);
        fcm_release_hist(h);
        fcm_release_multi(h);
        release_bins(h);
    }
    delete h;
}

const char* fcm_status_string(int s) {
    switch (s) {
        case FCM_OK: return "FCM_OK";
        case FCM_NOT_CONVERGED: return "FCM_NOT_CONVERGED";
        case FCM_ERR_INVALID_ARG: return "FCM_ERR_INVALID_ARG";
        case FCM_ERR_CUDA: return "FCM_ERR_CUDA";
        case FCM_ERR_OOM: return "FCM_ERR_OOM";
        case FCM_ERR_BAD_INPUT: return "FCM_ERR_BAD_INPUT";
        case FCM_ERR_TIMEOUT: return "FCM_ERR_TIMEOUT";
        case FCM_ERR_TOO_LARGE: return "FCM_ERR_TOO_LARGE";
        default: return "FCM_UNKNOWN_STATUS";
    }
}

const char* fcm_version(void) { return "0.1.0"; }

const char* fcm_last_error(fcm_handle h) {
    return h ? h->last_error.c_str() : "null handle";
}

int fcm_run(fcm_handle h, const float* x, int64_t n, int C, float m, float eps, int max_iter,
            int init_mode, const float* U0, float* U, float* V, int options, fcm_report* rep) {
    NvtxRange nvtx_range("fcm_run");
    if (!h) return FCM_ERR_INVALID_ARG;
    if (!x || !U || !V) return ctx_invalid(h, "null x, U or V");
    if (n < 1) return ctx_invalid(h, "n must be >= 1");
    if (C < 1 || C > FCM_MAX_CLUSTERS) return ctx_invalid(h, "C must be in [1, 8]");
    if (!(m > 1.0f) || !std::isfinite(m)) return ctx_invalid(h, "m must be a finite number > 1");
    if (!(eps >= 0.0f) || !std::isfinite(eps)) return ctx_invalid(h, "eps must be finite and >= 0");
    if (max_iter < 1) return ctx_invalid(h, "max_iter must be >= 1");
    if (init_mode != FCM_INIT_U && init_mode != FCM_INIT_V) return ctx_invalid(h, "bad init_mode");
    if (n > (int64_t)1 << 40) return ctx_invalid(h, "n too large");

    DeviceGuard g(h->device);
    int rc = ensure_single_workspace(h);
    if (rc) return rc;

    // Host buffers are staged through the workspace.
    if (init_mode == FCM_INIT_U && !U0) U0 = U;
    const bool x_dev = is_device_pointer(x);
    const bool U_dev = is_device_pointer(U);
    const bool V_dev = is_device_pointer(V);
    const bool U0_dev = init_mode == FCM_INIT_U && is_device_pointer(U0);
    const size_t xb = sizeof(float) * (size_t)n, Ub = sizeof(float) * (size_t)n * C;
    const float* dx = x;
    float* dU = U;
    const float* dU0 = init_mode == FCM_INIT_U ? U0 : nullptr;
    if (!x_dev) {
        if ((rc = ctx_grow(h, (void**)&h->d_stage_x, &h->stage_x_cap, xb, "staging x"))) return rc;
        CK(cudaMemcpyAsync(h->d_stage_x, x, xb, cudaMemcpyHostToDevice, h->stream));
        dx = h->d_stage_x;
    }
    if (!U_dev) {
        if ((rc = ctx_grow(h, (void**)&h->d_stage_U, &h->stage_U_cap, Ub, "staging U"))) return rc;
        dU = h->d_stage_U;
    }
    if (init_mode == FCM_INIT_U && !U0_dev) {
        // a host U^0 is staged into the U buffer and updated in place there
        CK(cudaMemcpyAsync(dU, U0, Ub, cudaMemcpyHostToDevice, h->stream));
        dU0 = dU;
    }

    const bool trace = (options & FCM_OPT_TRACE) != 0;
    if (trace) {
        if ((rc = ctx_grow(h, (void**)&h->d_trace, &h->trace_cap,
                           sizeof(double) * (size_t)max_iter * (2 + C), "trace buffer")))
            return rc;
    }

    RunState* hs = h->h_st;
    std::memset(hs, 0, sizeof(RunState));
    hs->x = dx;
    hs->Uprev = init_mode == FCM_INIT_U ? dU0 : dU;
    hs->U = dU;
    hs->trace = trace ? h->d_trace : nullptr;
    hs->n = n;
    hs->m = m;
    hs->inv_m1 = (float)(1.0 / ((double)m - 1.0));
    hs->eps = eps;
    hs->max_iter = max_iter;
    hs->C = C;
    hs->status = STATUS_RUNNING;
    hs->lim = h->limits;
    hs->static_pct = (options & FCM_OPT_DETERMINISTIC) ? 100 : h->static_pct;
    if (init_mode == FCM_INIT_V && !V_dev) std::memcpy(hs->V0, V, sizeof(float) * C);
    CK(cudaMemcpyAsync(h->d_st, hs, sizeof(RunState), cudaMemcpyHostToDevice, h->stream));
    if (init_mode == FCM_INIT_V && V_dev)
        CK(cudaMemcpyAsync(&h->d_st->V0, V, sizeof(float) * C, cudaMemcpyDeviceToDevice, h->stream));

    const int mk = mkind_of(m);
    const int pass0 = init_mode == FCM_INIT_U ? P_ACCUM0 : P_INITV;
    const bool aligned = (n % 4 == 0) && ((uintptr_t)dx % 16 == 0) && ((uintptr_t)dU % 16 == 0) &&
                         ((uintptr_t)hs->Uprev % 16 == 0);
    int run_blocks = 0;
    const bool recompute = (options & FCM_OPT_RECOMPUTE) != 0;
    const int iu = init_mode == FCM_INIT_U ? 0 : 1;
    const void* krun = recompute ? (const void*)g_rc.run[C][mk][iu] : (const void*)g_table.run[C][mk][iu];
    const int run_smem = recompute ? g_rc.smem[C][iu] : g_table.run_smem[C];
    if (recompute && !(aligned && h->coop))
        return ctx_invalid(h, "FCM_OPT_RECOMPUTE needs n % 4 == 0, 16-byte-aligned rows and cooperative launch");
    if (recompute ||
        (aligned && h->coop && !(options & (FCM_OPT_NO_TMA | FCM_OPT_NO_PERSISTENT | FCM_OPT_NO_GRAPH)))) {
        run_blocks = run_grid(n, (int64_t)h->num_sms * blocks_per_sm(h, krun, run_smem));
    }
    if (run_blocks > 0) {
        // the whole run: one cooperative launch (all blocks co-resident)
        void* args[2] = {&h->d_st, &h->d_partials};
        CK(cudaLaunchCooperativeKernel(krun, dim3(run_blocks), dim3(NT), args, run_smem, h->stream));
        h->last_blocks = run_blocks;
        h->last_path = 2;
    } else {
    Launch L;
    if ((rc = choose_launch(h, n, C, mk, pass0, dx, dU, hs->Uprev, options, &L))) return rc;
    PassFn kfirst = L.kfirst, kiter = L.kiter;
    const int smem_first = L.smem_first, smem_iter = L.smem_iter, var = L.var, nblocks = L.nblocks;
    h->last_blocks = nblocks;
    h->last_path = (options & FCM_OPT_NO_GRAPH) ? 0 : 1;

    if (options & FCM_OPT_NO_GRAPH) {
        if ((rc = run_host_loop(h, kfirst, smem_first, kiter, smem_iter, nblocks))) return rc;
    } else {
        const GraphKey key{C, mk, pass0, var, nblocks};
        auto it = h->graphs.find(key);
        if (it == h->graphs.end()) {
            GraphEntry ge;
            if ((rc = build_graph(h, kfirst, smem_first, kiter, smem_iter, nblocks, &ge))) return rc;
            it = h->graphs.emplace(key, ge).first;
        }
        CK(cudaGraphLaunch(it->second.exec, h->stream));
    }
    }

    CK(cudaMemcpyAsync(hs, h->d_st, sizeof(RunState), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(V, &h->d_st->V, sizeof(float) * C,
                       V_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    if (!U_dev) CK(cudaMemcpyAsync(U, h->d_stage_U, Ub, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));

    h->last_trace_iters = trace ? hs->iters : 0;
    h->last_C = C;
    if (rep) {
        std::memset(rep, 0, sizeof(*rep));
        rep->iters = hs->iters;
        rep->status = hs->status;
        rep->flags = hs->flags | (int)hs->bounds;
        rep->C = C;
        rep->delta = hs->delta;
        rep->J = hs->J;
        for (int j = 0; j < C; ++j) rep->V64[j] = hs->V64[j];
        rep->launches = h->last_path == 2 ? 1 : h->last_path == 1 ? 1 + hs->iters : h->last_launches;
    }
    if (hs->status == STATUS_RUNNING) {
        h->last_error = "run ended without a status";
        return FCM_ERR_CUDA;
    }
    return hs->status;
}

int fcm_run_stream(fcm_handle h, int n_images, const float* const* x, int64_t n, int C, float m, float eps,
                   int max_iter, const float* const* U0, float* const* U, float* V, int options,
                   fcm_report* reps) {
    NvtxRange nvtx_range("fcm_run_stream");
    if (!h) return FCM_ERR_INVALID_ARG;
    if (n_images < 1 || !x || !U || !V) return ctx_invalid(h, "n_images >= 1 and non-null x, U and V");
    for (int i = 0; i < n_images; ++i)
        if (!x[i] || !U[i]) return ctx_invalid(h, "null x[i] or U[i]");
    if (n < 1) return ctx_invalid(h, "n must be >= 1");
    if (C < 1 || C > FCM_MAX_CLUSTERS) return ctx_invalid(h, "C must be in [1, 8]");
    if (!(m > 1.0f) || !std::isfinite(m)) return ctx_invalid(h, "m must be a finite number > 1");
    if (!(eps >= 0.0f) || !std::isfinite(eps)) return ctx_invalid(h, "eps must be finite and >= 0");
    if (max_iter < 1) return ctx_invalid(h, "max_iter must be >= 1");
    if (n > (int64_t)1 << 40) return ctx_invalid(h, "n too large");
    if (n % 4 != 0) return ctx_invalid(h, "fcm_run_stream needs n % 4 == 0");
    if (options & ~(FCM_OPT_RECOMPUTE | FCM_OPT_DETERMINISTIC))
        return ctx_invalid(h, "fcm_run_stream takes no option but FCM_OPT_RECOMPUTE and FCM_OPT_DETERMINISTIC");

    DeviceGuard g(h->device);
    int rc = ensure_single_workspace(h);
    if (rc) return rc;
    if (!h->coop) return ctx_invalid(h, "fcm_run_stream needs cooperative launch");
    const size_t xb = sizeof(float) * (size_t)n, Ub = sizeof(float) * (size_t)n * C;
    constexpr int NS = fcm_ctx::PIPE_SETS;
    for (int b = 0; b < NS; ++b) {
        if ((rc = ctx_grow(h, (void**)&h->d_pipe_x[b], &h->pipe_x_cap[b], xb, "stream staging x"))) return rc;
        if ((rc = ctx_grow(h, (void**)&h->d_pipe_U[b], &h->pipe_U_cap[b], Ub, "stream staging U"))) return rc;
    }
    if (h->pipe_st_cap < n_images) {
        if (h->h_pipe_st) cudaFreeHost(h->h_pipe_st);
        h->h_pipe_st = nullptr;
        h->pipe_st_cap = 0;
        CK(host_malloc(h, &h->h_pipe_st, sizeof(RunState) * (size_t)n_images));
        h->pipe_st_cap = n_images;
    }
    if (!h->pipe_in) {
        CK(cudaStreamCreateWithFlags(&h->pipe_in, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&h->pipe_out, cudaStreamNonBlocking));
        for (cudaEvent_t& ev : h->pipe_ev) CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
    cudaEvent_t* in_done = h->pipe_ev;
    cudaEvent_t* run_done = h->pipe_ev + NS;
    cudaEvent_t* out_done = h->pipe_ev + 2 * NS;
    cudaEvent_t ev_start = h->pipe_ev[3 * NS], ev_end = h->pipe_ev[3 * NS + 1];

    const int mk = mkind_of(m);
    const bool recompute = (options & FCM_OPT_RECOMPUTE) != 0;
    const void* krun = recompute ? (const void*)g_rc.run[C][mk][0] : (const void*)g_table.run[C][mk][0];
    const int run_smem = recompute ? g_rc.smem[C][0] : g_table.run_smem[C];
    const int run_blocks = run_grid(n, (int64_t)h->num_sms * blocks_per_sm(h, krun, run_smem));
    if (run_blocks < 1) return ctx_invalid(h, "the whole-run kernel does not fit on this device");

    // the copy streams start behind the work already queued on the handle's stream
    CK(cudaEventRecord(ev_start, h->stream));
    CK(cudaStreamWaitEvent(h->pipe_in, ev_start, 0));
    CK(cudaStreamWaitEvent(h->pipe_out, ev_start, 0));
    cudaError_t e = cudaSuccess;
    const char* what = "queueing the image sequence";
    for (int i = 0; i < n_images && e == cudaSuccess; ++i) {
        const int b = i % NS;
        float* dx = h->d_pipe_x[b];
        float* dU = h->d_pipe_U[b];
        RunState* hs = h->h_pipe_st + i;
        std::memset(hs, 0, sizeof(RunState));
        hs->x = dx;
        hs->Uprev = dU;  // U^0 is staged into the U set and updated in place
        hs->U = dU;
        hs->n = n;
        hs->m = m;
        hs->inv_m1 = (float)(1.0 / ((double)m - 1.0));
        hs->eps = eps;
        hs->max_iter = max_iter;
        hs->C = C;
        hs->status = STATUS_RUNNING;
        hs->lim = h->limits;
        hs->static_pct = (options & FCM_OPT_DETERMINISTIC) ? 100 : h->static_pct;
        const float* u0 = (U0 && U0[i]) ? U0[i] : U[i];
        // upload, once the download of image i - NS has drained this set
        if (i >= NS) e = cudaStreamWaitEvent(h->pipe_in, out_done[b], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dx, x[i], xb, cudaMemcpyDefault, h->pipe_in);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dU, u0, Ub, cudaMemcpyDefault, h->pipe_in);
        if (e == cudaSuccess) e = cudaEventRecord(in_done[b], h->pipe_in);
        // the run, with its state uploaded before and read back after
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, in_done[b], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_st, hs, sizeof(RunState), cudaMemcpyHostToDevice, h->stream);
        void* args[2] = {&h->d_st, &h->d_partials};
        if (e == cudaSuccess)
            e = cudaLaunchCooperativeKernel(krun, dim3(run_blocks), dim3(NT), args, run_smem, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hs, h->d_st, sizeof(RunState), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(run_done[b], h->stream);
        // download
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->pipe_out, run_done[b], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(U[i], dU, Ub, cudaMemcpyDefault, h->pipe_out);
        if (e == cudaSuccess) e = cudaEventRecord(out_done[b], h->pipe_out);
    }
    // later work on the handle's stream follows the last download
    if (e == cudaSuccess) e = cudaEventRecord(ev_end, h->pipe_out);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, ev_end, 0);
    // drain all three streams, also after an error, so no copy into a caller's
    // buffer is still pending when the call returns
    const cudaError_t s_in = cudaStreamSynchronize(h->pipe_in);
    const cudaError_t s_run = cudaStreamSynchronize(h->stream);
    const cudaError_t s_out = cudaStreamSynchronize(h->pipe_out);
    if (e == cudaSuccess) {
        e = s_in != cudaSuccess ? s_in : s_run != cudaSuccess ? s_run : s_out;
        what = "running the image sequence";
    }
    if (e != cudaSuccess) return ctx_fail(h, e, what);

    h->last_blocks = run_blocks;
    h->last_path = 2;
    h->last_C = C;
    h->last_trace_iters = 0;
    int worst = FCM_OK;
    for (int i = 0; i < n_images; ++i) {
        RunState* hs = h->h_pipe_st + i;
        if (hs->status == STATUS_RUNNING) {
            hs->status = FCM_ERR_CUDA;
            h->last_error = "a run of the sequence ended without a status";
        }
        for (int j = 0; j < C; ++j) V[(size_t)i * C + j] = hs->V[j];
        if (reps) {
            fcm_report* rep = reps + i;
            std::memset(rep, 0, sizeof(*rep));
            rep->iters = hs->iters;
            rep->status = hs->status;
            rep->flags = hs->flags | (int)hs->bounds;
            rep->C = C;
            rep->delta = hs->delta;
            rep->J = hs->J;
            for (int j = 0; j < C; ++j) rep->V64[j] = hs->V64[j];
            rep->launches = 1;
        }
        if (hs->status < 0 && worst >= 0) worst = hs->status;
        if (hs->status == FCM_NOT_CONVERGED && worst == FCM_OK) worst = FCM_NOT_CONVERGED;
    }
    return worst;
}

int fcm_time_pass(fcm_handle h, const float* x, int64_t n, int C, float m, float* U, const float* V,
                  int launches, int options, float* ms_per_launch) {
    NvtxRange nvtx_range("fcm_time_pass");
    if (!h) return FCM_ERR_INVALID_ARG;
    if (!x || !U || !V || !ms_per_launch) return ctx_invalid(h, "null argument");
    if (n < 1 || C < 1 || C > FCM_MAX_CLUSTERS || !(m > 1.0f) || launches < 1)
        return ctx_invalid(h, "bad size, C, m or launch count");
    if (!is_device_pointer(x) || !is_device_pointer(U)) return ctx_invalid(h, "x and U must be device memory");
    DeviceGuard g(h->device);
    int rc = ensure_single_workspace(h);
    if (rc) return rc;
    RunState* hs = h->h_st;
    std::memset(hs, 0, sizeof(RunState));
    hs->x = x;
    hs->Uprev = U;
    hs->U = U;
    hs->n = n;
    hs->m = m;
    hs->inv_m1 = (float)(1.0 / ((double)m - 1.0));
    hs->eps = 0.0f;                 // delta < 0 never holds: no stop
    hs->max_iter = launches + 2;    // nor does the iteration bound
    hs->C = C;
    hs->k = 1;
    hs->status = STATUS_RUNNING;
    hs->lim = h->limits;
    hs->static_pct = (options & FCM_OPT_DETERMINISTIC) ? 100 : h->static_pct;
    const bool V_dev = is_device_pointer(V);
    if (!V_dev)
        for (int j = 0; j < C; ++j) {
            hs->V[j] = V[j];
            hs->V64[j] = V[j];
        }
    CK(cudaMemcpyAsync(h->d_st, hs, sizeof(RunState), cudaMemcpyHostToDevice, h->stream));
    if (V_dev) CK(cudaMemcpyAsync(&h->d_st->V, V, sizeof(float) * C, cudaMemcpyDeviceToDevice, h->stream));
    Launch L;
    if ((rc = choose_launch(h, n, C, mkind_of(m), P_ACCUM0, x, U, U, options, &L))) return rc;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const cudaGraphConditionalHandle none = 0;
    cudaEventRecord(e0, h->stream);
    for (int t = 0; t < launches; ++t)
        L.kiter<<<L.nblocks, NT, L.smem_iter, h->stream>>>(h->d_st, h->d_partials, none, 0);
    cudaEventRecord(e1, h->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return ctx_fail(h, e, "timing the pass");
    *ms_per_launch = ms / launches;
    return FCM_OK;
}

int fcm_get_trace(fcm_handle h, double* delta, double* J, double* V, int cap) {
    if (!h || cap < 0) return FCM_ERR_INVALID_ARG;
    const int k = std::min(cap, h->last_trace_iters);
    if (k == 0) return 0;
    const int C = h->last_C, row = 2 + C;
    DeviceGuard g(h->device);
    double* tmp = new double[(size_t)k * row];
    cudaError_t e = cudaMemcpy(tmp, h->d_trace, sizeof(double) * (size_t)k * row, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        delete[] tmp;
        return ctx_fail(h, e, "reading the trace");
    }
    for (int t = 0; t < k; ++t) {
        if (delta) delta[t] = tmp[(size_t)t * row];
        if (J) J[t] = tmp[(size_t)t * row + 1];
        if (V)
            for (int j = 0; j < C; ++j) V[(size_t)t * C + j] = tmp[(size_t)t * row + 2 + j];
    }
    delete[] tmp;
    return k;
}

}  // extern "C"
