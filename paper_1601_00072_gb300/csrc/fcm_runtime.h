// The handle behind fcm_handle, shared by the host modules of the library.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <tuple>

#include <nvtx3/nvToolsExt.h>

#include "fcm.h"
#include "fcm_internal.h"

namespace fcm {

struct GraphKey {
    int C, mk, pass0, vec, nblocks;
    bool operator<(const GraphKey& o) const {
        return std::tie(C, mk, pass0, vec, nblocks) < std::tie(o.C, o.mk, o.pass0, o.vec, o.nblocks);
    }
};

struct GraphEntry {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

struct BatchedWorkspace;  // fcm_batched.cu
struct MlpWorkspace;      // fcm_mlp.cu
struct HistWorkspace;     // fcm_hist.cu
struct MultiWorkspace;    // fcm_multi.cu
struct BinWorkspace;      // fcm_bins.cu
struct SliceDesc;         // fcm_batched.h
struct SliceResult;
struct BinRun;

}  // namespace fcm


// An NVTX range around one entry-point call, named after it, so the library's
// work shows up by call in Nsight timelines (a no-op without a tool attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct fcm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    bool coop = false;        // cooperative launch supported
    int last_blocks = 0;      // grid of the last run
    int last_path = 0;        // 0 host loop, 1 graph WHILE loop, 2 one cooperative launch
    int last_launches = 0;    // kernel launches of the last host-loop run
    int max_smem_optin = 0;
    std::string device_name;
    std::string last_error;

    // bounds of the device-side waits (fcm_set_limits), copied into every
    // run's state; alloc_fail_in > 0 makes the allocation that many calls
    // from now fail once (fault injection for tests, 0 = off)
    fcm::WaitLimits limits{fcm::DEFAULT_GRID_SPINS, fcm::DEFAULT_TMA_POLLS, 0u, 0u};
    // whole-run kernel: percent of a pass's tiles dealt in fixed warp shares
    // (FCM_RUN_STATIC_PCT in the environment overrides it, 1..100)
    int static_pct = fcm::DEFAULT_STATIC_PCT;
    int alloc_fail_in = 0;

    // single-image path
    fcm::RunState* d_st = nullptr;
    fcm::RunState* h_st = nullptr;   // pinned
    int h_done = 0;
    double* d_partials = nullptr;
    int partial_blocks = 0;
    double* d_trace = nullptr;
    size_t trace_cap = 0;
    int last_trace_iters = 0;
    int last_C = 0;
    float* d_stage_x = nullptr;
    size_t stage_x_cap = 0;
    float* d_stage_U = nullptr;
    size_t stage_U_cap = 0;
    std::map<fcm::GraphKey, fcm::GraphEntry> graphs;
    std::map<const void*, int> occupancy;   // blocks per SM of each kernel (smem attribute set)

    // pipelined image sequences (fcm_run_stream): PIPE_SETS staging sets, a
    // pinned run state per image, an upload and a download stream, and per
    // set the events upload done, run done and download done, then start/end
    static constexpr int PIPE_SETS = 3;
    float* d_pipe_x[PIPE_SETS] = {};
    float* d_pipe_U[PIPE_SETS] = {};
    size_t pipe_x_cap[PIPE_SETS] = {};
    size_t pipe_U_cap[PIPE_SETS] = {};
    fcm::RunState* h_pipe_st = nullptr;
    int pipe_st_cap = 0;
    cudaStream_t pipe_in = nullptr;
    cudaStream_t pipe_out = nullptr;
    cudaEvent_t pipe_ev[3 * PIPE_SETS + 2] = {};

    // other paths
    fcm::BatchedWorkspace* batched = nullptr;
    fcm::MlpWorkspace* mlp = nullptr;
    fcm::HistWorkspace* hist = nullptr;
    fcm::MultiWorkspace* multi = nullptr;
    fcm::BinWorkspace* bins = nullptr;
};

namespace fcm {

// Makes a device current for a scope and restores the caller's afterwards.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Every device and pinned-host allocation of a handle goes through these, so
// that a test can make one fail (fcm_set_limits) without a real shortage.
cudaError_t dev_malloc_raw(fcm_ctx* h, void** p, size_t bytes);
cudaError_t host_malloc_raw(fcm_ctx* h, void** p, size_t bytes);
template <typename T>
cudaError_t dev_malloc(fcm_ctx* h, T** p, size_t bytes) {
    return dev_malloc_raw(h, reinterpret_cast<void**>(p), bytes);
}
template <typename T>
cudaError_t host_malloc(fcm_ctx* h, T** p, size_t bytes) {
    return host_malloc_raw(h, reinterpret_cast<void**>(p), bytes);
}

int ctx_fail(fcm_ctx* h, cudaError_t e, const char* what);
int ctx_invalid(fcm_ctx* h, const char* what);
int ctx_grow(fcm_ctx* h, void** p, size_t* cap, size_t bytes, const char* what);

// Histogram-domain runs (fcm_bins.cu) of the ns slices whose descriptors are
// at h_desc (host) and d_desc (device, already uploaded): queues the uploads
// and kernels on the handle's stream, and the download of the nr results into
// h_results (pinned host memory; nullable). Does not synchronise.
int bins_run(fcm_ctx* h, const SliceDesc* h_desc, const SliceDesc* d_desc, int ns, const BinRun* runs, int nr,
             const float* v0_dev, int v0_stride, SliceResult* h_results);
void release_bins(fcm_ctx* h);

// Checks a batch (n < n_limit per slice), fills its device descriptors in the
// batched workspace's pinned array and queues their upload on the handle's
// stream. The arrays stay valid until the next batched call on the handle.
int batch_descs(fcm_ctx* h, const fcm_slice* slices, int n_slices, int64_t n_limit, SliceDesc** h_desc,
                SliceDesc** d_desc);
}  // namespace fcm

void fcm_release_batched(fcm_ctx* h);
void fcm_release_mlp(fcm_ctx* h);
void fcm_release_hist(fcm_ctx* h);
void fcm_release_multi(fcm_ctx* h);
