// fcm_run_noalloc: a whole FCM run that allocates no memory.
//
// Who needs this: code that may not allocate device memory when it runs —
// for example a host application whose device memory is reserved up front
// by a pool it does not control, a plugin inside a framework that owns the
// allocator, or a latency-critical service where a cudaMalloc (which can
// synchronise the device and can fail under memory pressure) is not
// acceptable. fcm_run keeps its scratch in a handle that allocates on first
// use; this entry point instead keeps it in one fixed array of device memory
// that is part of the library image and exists on every GPU that loads the
// library until the process exits.
//
// The scratch holds the device-side run state and the per-block partial sums
// of the cooperative whole-run kernel (the same kernel fcm_run launches for
// aligned inputs). Its size is fixed: partial sums for at most
// FCM_NOALLOC_MAX_BLOCKS thread blocks. Every call shares it, so calls whose
// work overlaps on the GPU (from several host threads, or on several streams
// without ordering between them) race and give wrong results.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "fcm.h"
#include "fcm_device.cuh"
#include "fcm_internal.h"

using namespace fcm;

namespace {

constexpr size_t kStateBytes = (sizeof(RunState) + 255) / 256 * 256;
constexpr size_t kPartialBytes = sizeof(float) * 2 * SLOTS_MAX * FCM_NOALLOC_MAX_BLOCKS;

// The scratch: run state, then two buffers of per-block partial sums.
// In host code this name is only a stand-in for the device array; its device
// address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kStateBytes + kPartialBytes];

constexpr int kMaxDevices = 64;

struct DeviceSetup {
    bool done = false;
    int status = FCM_OK;
    unsigned char* scratch = nullptr;  // device address of g_noalloc_scratch
    int num_sms = 0;
    // blocks per SM of the whole-run kernel: [C][m kind][from U^0 / from V^0]
    int bps[FCM_MAX_CLUSTERS + 1][4][2] = {};
};

std::mutex g_mu;
DeviceSetup g_dev[kMaxDevices];

// First call on a device: resolve the scratch address and the launch limits
// of every whole-run kernel, with that device current.
int setup_device(int dev) {
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceSetup& d = g_dev[dev];
    if (d.done) return d.status;
    d.done = true;
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return d.status = FCM_ERR_CUDA;
    }
    d.scratch = static_cast<unsigned char*>(ptr);
    int coop = 0;
    if (cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) {
        cudaGetLastError();
        return d.status = FCM_ERR_CUDA;
    }
    const SingleTable& t = single_table();
    for (int C = 1; C <= FCM_MAX_CLUSTERS; ++C)
        for (int mk = 0; mk < 4; ++mk)
            for (int init = 0; init < 2; ++init) {
                const void* k = (const void*)t.run[C][mk][init];
                const int smem = t.run_smem[C];
                int nb = 0;
                if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NT, smem) != cudaSuccess) {
                    cudaGetLastError();
                    nb = 0;
                }
                d.bps[C][mk][init] = nb;
            }
    return d.status = FCM_OK;
}

bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int fcm_run_noalloc(const float* x, int64_t n, int C, float m, float eps, int max_iter,
                               int init_mode, const float* U0, float* U, float* V, void* cuda_stream,
                               fcm_report* rep) {
    if (!x || !U || !V) return FCM_ERR_INVALID_ARG;
    if (n < 1 || n > ((int64_t)1 << 40) || n % 4 != 0) return FCM_ERR_INVALID_ARG;
    if (C < 1 || C > FCM_MAX_CLUSTERS) return FCM_ERR_INVALID_ARG;
    if (!(m > 1.0f) || !std::isfinite(m) || !(eps >= 0.0f) || !std::isfinite(eps) || max_iter < 1)
        return FCM_ERR_INVALID_ARG;
    if (init_mode != FCM_INIT_U && init_mode != FCM_INIT_V) return FCM_ERR_INVALID_ARG;
    // the call copies through host memory and synchronises its stream, which a
    // stream under capture cannot do: refuse such a stream before any other
    // runtime call
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)cuda_stream, &cap) != cudaSuccess) {
        cudaGetLastError();
        return FCM_ERR_INVALID_ARG;
    }
    if (cap != cudaStreamCaptureStatusNone) return FCM_ERR_INVALID_ARG;
    if (init_mode == FCM_INIT_U && !U0) U0 = U;
    const float* Uin = init_mode == FCM_INIT_U ? U0 : U;
    if (!on_device(x) || !on_device(U) || !on_device(Uin)) return FCM_ERR_INVALID_ARG;
    if ((uintptr_t)x % 16 || (uintptr_t)U % 16 || (uintptr_t)Uin % 16) return FCM_ERR_INVALID_ARG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return FCM_ERR_CUDA;
    }
    int rc = setup_device(dev);
    if (rc) return rc;
    const DeviceSetup& d = g_dev[dev];
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    const int mk = mkind_of(m);
    const int init = init_mode == FCM_INIT_U ? 0 : 1;
    const int bps = d.bps[C][mk][init];
    if (bps < 1) return FCM_ERR_CUDA;
    const int64_t want = (n + (int64_t)WARP_TILE * NWARP - 1) / ((int64_t)WARP_TILE * NWARP);
    const int64_t blocks = std::min<int64_t>(want, (int64_t)d.num_sms * bps);
    if (blocks > FCM_NOALLOC_MAX_BLOCKS) return FCM_ERR_TOO_LARGE;

    RunState* st = reinterpret_cast<RunState*>(d.scratch);
    double* partials = reinterpret_cast<double*>(d.scratch + kStateBytes);

    // A fresh state for every call: the grid-barrier counter and the status
    // must start at zero; the partial sums are always written before read.
    RunState hs;
    std::memset(&hs, 0, sizeof(hs));
    hs.x = x;
    hs.Uprev = Uin;
    hs.U = U;
    hs.n = n;
    hs.m = m;
    hs.inv_m1 = (float)(1.0 / ((double)m - 1.0));
    hs.eps = eps;
    hs.max_iter = max_iter;
    hs.C = C;
    hs.status = STATUS_RUNNING;
    hs.lim = WaitLimits{DEFAULT_GRID_SPINS, DEFAULT_TMA_POLLS, 0u, 0u};
    hs.static_pct = DEFAULT_STATIC_PCT;
    const bool V_dev = on_device(V);
    if (init_mode == FCM_INIT_V && !V_dev) std::memcpy(hs.V0, V, sizeof(float) * C);

    cudaError_t e = cudaMemcpyAsync(st, &hs, sizeof(RunState), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess && init_mode == FCM_INIT_V && V_dev)
        e = cudaMemcpyAsync(&st->V0, V, sizeof(float) * C, cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess) {
        void* args[2] = {&st, &partials};
        e = cudaLaunchCooperativeKernel((const void*)single_table().run[C][mk][init], dim3((unsigned)blocks),
                                        dim3(NT), args, single_table().run_smem[C], stream);
    }
    RunState out;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&out, st, sizeof(RunState), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(V, &st->V, sizeof(float) * C, V_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FCM_ERR_CUDA;
    }
    if (rep) {
        std::memset(rep, 0, sizeof(*rep));
        rep->iters = out.iters;
        rep->status = out.status;
        rep->flags = out.flags;
        rep->C = C;
        rep->delta = out.delta;
        rep->J = out.J;
        for (int j = 0; j < C; ++j) rep->V64[j] = out.V64[j];
        rep->launches = 1;
    }
    return out.status == STATUS_RUNNING ? FCM_ERR_CUDA : out.status;
}
