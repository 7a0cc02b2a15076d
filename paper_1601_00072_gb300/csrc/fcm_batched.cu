// Host runtime of the batched FCM path: argument checks, LPT work order, the
// tiling of the round schedule, the launch-shape autotuner with its cache, and
// the CUDA graph of a batch.
//
// A batch is one persistent kernel launch. Its graph holds, in order: the
// upload of the slice descriptors and of the work order or tiling (from pinned
// host buffers the handle refills before each launch), the reset of the
// kernel's control state, the kernel (a thread-block-cluster launch, or a
// cooperative launch for the round schedule), and the download of the
// per-slice results. The graph is instantiated once per (slice count, plan).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <tuple>
#include <unordered_set>
#include <vector>

#include "fcm.h"
#include "fcm_batched.h"
#include "fcm_device.cuh"
#include "fcm_runtime.h"

using namespace fcm;

namespace fcm {

struct BatchedWorkspace {
    int cap = 0;
    SliceDesc* d_desc = nullptr;
    SliceResult* d_res = nullptr;
    int* d_order = nullptr;
    BatchCtl* d_ctl = nullptr;
    SliceDesc* h_desc = nullptr;   // pinned
    SliceResult* h_res = nullptr;  // pinned
    int* h_order = nullptr;        // pinned
    cudaStream_t cap_stream = nullptr;
    // round schedule: per-slice state, control block, batch sizes, first slot
    // of each slice, and the slot partials (capacity in slots)
    RoundSlice* d_rstate = nullptr;
    RoundCtl* d_rctl = nullptr;
    RoundsHdr* d_rhdr = nullptr;
    RoundsHdr* h_rhdr = nullptr;  // pinned
    int* d_slot_base = nullptr;
    int* h_slot_base = nullptr;   // pinned, cap + 1
    int64_t slot_cap = 0;
    double* d_rpart = nullptr;
    std::map<std::tuple<int, int, int, int64_t, int, int>, GraphEntry> graphs;
    std::map<std::string, fcm_batch_plan> plans;
    bool cache_loaded = false;
    bool forced = false;
    fcm_batch_plan forced_plan{};
    fcm_batch_plan last{};
    std::map<std::pair<int, int>, int> grid;  // (block, cluster) -> CTAs of a full persistent grid
    // device pointers already checked by this handle (the check is a driver
    // call per pointer; repeated batches reuse their buffers)
    std::unordered_set<const void*> known_device;
    std::map<std::pair<int, int>, int> rgrid;  // (block, shared bytes) -> CTAs of a cooperative round grid
    std::vector<int64_t> size, cost;          // per slice of the current batch: n, and its queue cost
    // team schedule: the seat queue (fixed length cap * TEAM_MAX, so a captured
    // graph serves every batch of a slice count), rank slots and barrier counters
    int4* d_items = nullptr;
    int4* h_items = nullptr;  // pinned
    float2* d_tslots = nullptr;
    unsigned* d_tctr = nullptr;
    int team_cap = 0;
    std::map<int, int> tgrid;  // block -> CTAs of a full cooperative team grid
};

}  // namespace fcm

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return ctx_fail(h, e_, #call); \
    } while (0)

namespace {

// The work order of the slice queue for a plan (LPT): first the slices a
// whole cluster shares (n >= big), then the rest, each group costliest first
// (ties by index, so the order is stable). A cluster takes slices of the
// first group together and splits up at the first slice of the second.
void order_for(BatchedWorkspace* w, int n, int64_t big) {
    std::iota(w->h_order, w->h_order + n, 0);
    std::stable_sort(w->h_order, w->h_order + n, [&](int a, int b) {
        const bool ba = w->size[a] >= big, bb = w->size[b] >= big;
        if (ba != bb) return ba;
        return w->cost[a] > w->cost[b];
    });
}

BatchKernel kernel_for(int block) { return block == 256 ? batched_kernel_256() : batched_kernel_512(); }
RoundsKernel rounds_for(int block) { return block == 256 ? rounds_kernel_256() : rounds_kernel_512(); }

bool plan_valid(const fcm_batch_plan& p) {
    if (p.block != 256 && p.block != 512) return false;
    if (p.schedule == FCM_SCHED_ROUNDS) return p.tile >= 1024 && p.tile <= 65536 && p.tile % 1024 == 0;
    if (p.schedule == FCM_SCHED_TEAMS) return p.tile >= 10 && p.tile <= 10000;
    if (p.schedule != FCM_SCHED_SLICES) return false;
    return (p.cluster == 1 || p.cluster == 2 || p.cluster == 4 || p.cluster == 8) && p.big >= 1 && p.tile >= 0;
}

void free_graphs(BatchedWorkspace* w) {
    for (auto& kv : w->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    w->graphs.clear();
}

int ensure_batched(fcm_ctx* h, int n) {
    if (!h->batched) h->batched = new BatchedWorkspace();
    BatchedWorkspace* w = h->batched;
    if (!w->cap_stream) CK(cudaStreamCreateWithFlags(&w->cap_stream, cudaStreamNonBlocking));
    if (!w->d_ctl) CK(dev_malloc(h, &w->d_ctl, sizeof(BatchCtl)));
    if (!w->d_rctl) CK(dev_malloc(h, &w->d_rctl, sizeof(RoundCtl)));
    if (!w->d_rhdr) CK(dev_malloc(h, &w->d_rhdr, sizeof(RoundsHdr)));
    if (!w->h_rhdr) CK(host_malloc(h, &w->h_rhdr, sizeof(RoundsHdr)));
    if (w->cap >= n) return 0;
    free_graphs(w);  // graphs point at the old buffers
    void* dev[] = {w->d_desc, w->d_res, w->d_order, w->d_rstate, w->d_slot_base};
    for (void* p : dev) cudaFree(p);
    void* host[] = {w->h_desc, w->h_res, w->h_order, w->h_slot_base};
    for (void* p : host) cudaFreeHost(p);
    w->d_desc = nullptr;
    w->d_res = nullptr;
    w->d_order = nullptr;
    w->d_rstate = nullptr;
    w->d_slot_base = nullptr;
    w->h_desc = nullptr;
    w->h_res = nullptr;
    w->h_order = nullptr;
    w->h_slot_base = nullptr;
    w->cap = 0;
    const int cap = std::max(n, 64);
    CK(dev_malloc(h, &w->d_desc, sizeof(SliceDesc) * cap));
    CK(dev_malloc(h, &w->d_res, sizeof(SliceResult) * cap));
    CK(dev_malloc(h, &w->d_order, sizeof(int) * cap));
    CK(dev_malloc(h, &w->d_rstate, sizeof(RoundSlice) * cap));
    CK(dev_malloc(h, &w->d_slot_base, sizeof(int) * (cap + 1)));
    CK(host_malloc(h, &w->h_desc, sizeof(SliceDesc) * cap));
    CK(host_malloc(h, &w->h_res, sizeof(SliceResult) * cap));
    CK(host_malloc(h, &w->h_order, sizeof(int) * cap));
    CK(host_malloc(h, &w->h_slot_base, sizeof(int) * (cap + 1)));
    w->cap = cap;
    return 0;
}

// First slot of every slice for a plan's minimum chunk, and the round bound,
// into the pinned buffers; grows the slot partials when needed.
int fill_slots(fcm_ctx* h, const fcm_slice* slices, int n, int min_chunk) {
    BatchedWorkspace* w = h->batched;
    if (n > ROUND_MAX_SLICES) return ctx_invalid(h, "the round schedule takes at most 8192 slices");
    int64_t total = 0;
    int max_iter = 1;
    for (int i = 0; i < n; ++i) {
        w->h_slot_base[i] = (int)total;
        total += round_slots(slices[i].n, min_chunk);
        if (total >= ((int64_t)1 << 31) / ROUND_SUMS) return ctx_invalid(h, "batch too large for the round schedule");
        max_iter = std::max(max_iter, slices[i].max_iter);
    }
    w->h_slot_base[n] = (int)total;
    w->h_rhdr->n_slices = n;
    w->h_rhdr->max_rounds = max_iter + 1;
    // in the header, which every replay of the batch graph uploads afresh
    w->h_rhdr->wait_spins = h->limits.grid_spins;
    w->h_rhdr->phantoms = h->limits.phantoms;
    if (w->slot_cap < total) {
        free_graphs(w);  // graphs point at the old buffer
        cudaFree(w->d_rpart);
        w->d_rpart = nullptr;
        w->slot_cap = 0;
        const int64_t cap = std::max<int64_t>(total + total / 4, 4096);
        CK(dev_malloc(h, &w->d_rpart, sizeof(double) * ROUND_SUMS * cap));
        w->slot_cap = cap;
    }
    return 0;
}

// CTAs of a full persistent grid for this shape (0 if it cannot run).
int grid_ctas(fcm_ctx* h, int block, int cluster) {
    BatchedWorkspace* w = h->batched;
    auto it = w->grid.find({block, cluster});
    if (it != w->grid.end()) return it->second;
    const BatchKernel k = kernel_for(block);
    int ctas = 0;
    if (cudaFuncSetAttribute((const void*)k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, k.smem) ==
        cudaSuccess) {
        if (cluster == 1) {
            int nb = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)k.fn, block, k.smem) == cudaSuccess)
                ctas = nb * h->num_sms;
        } else {
            cudaLaunchConfig_t cfg;
            std::memset(&cfg, 0, sizeof(cfg));
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = cluster;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(cluster * h->num_sms);
            cfg.blockDim = dim3(block);
            cfg.dynamicSmemBytes = k.smem;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int nc = 0;
            if (cudaOccupancyMaxActiveClusters(&nc, (const void*)k.fn, &cfg) == cudaSuccess) ctas = nc * cluster;
        }
    }
    cudaGetLastError();
    w->grid[{block, cluster}] = ctas;
    return ctas;
}

int round_smem(int n_slices) { return (int)sizeof(int64_t) * (n_slices + 1); }

// CTAs of a full cooperative grid of the round kernel (0 if it cannot run).
int round_ctas(fcm_ctx* h, int block, int smem) {
    BatchedWorkspace* w = h->batched;
    auto it = w->rgrid.find({block, smem});
    if (it != w->rgrid.end()) return it->second;
    const void* fn = (const void*)rounds_for(block).fn;
    int nb = 0;
    if (!h->coop || cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, smem) != cudaSuccess)
        nb = 0;
    cudaGetLastError();
    w->rgrid[{block, smem}] = nb * h->num_sms;
    return nb * h->num_sms;
}

int launch_rounds(fcm_ctx* h, cudaStream_t s, const fcm_batch_plan& p, int n_slices) {
    BatchedWorkspace* w = h->batched;
    const RoundsKernel k = rounds_for(p.block);
    const int smem = round_smem(n_slices);
    const int ctas = round_ctas(h, p.block, smem);
    if (ctas < 1) {
        h->last_error = "the round schedule needs cooperative launch support";
        return FCM_ERR_CUDA;
    }
    k.init<<<(n_slices + 255) / 256, 256, 0, s>>>(w->d_rstate, w->d_res, w->d_rctl, n_slices);
    CK(cudaGetLastError());
    RoundsArgs a;
    std::memset(&a, 0, sizeof(a));
    a.descs = w->d_desc;
    a.results = w->d_res;
    a.state = w->d_rstate;
    a.ctl = w->d_rctl;
    a.hdr = w->d_rhdr;
    a.slot_base = w->d_slot_base;
    a.partials = w->d_rpart;
    a.min_chunk = p.tile;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(p.block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, k.fn, a));
    return 0;
}

// CTAs of a full cooperative grid of the team kernel (0 if it cannot run).
int team_ctas(fcm_ctx* h, int block) {
    BatchedWorkspace* w = h->batched;
    auto it = w->tgrid.find(block);
    if (it != w->tgrid.end()) return it->second;
    const BatchKernel k = kernel_for(block);
    int nb = 0;
    if (!h->coop ||
        cudaFuncSetAttribute((const void*)k.teams, cudaFuncAttributeMaxDynamicSharedMemorySize, k.smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)k.teams, block, k.smem) != cudaSuccess)
        nb = 0;
    cudaGetLastError();
    w->tgrid[block] = nb * h->num_sms;
    return nb * h->num_sms;
}

// The seat queue of the team schedule. A slice whose cost (n times its
// expected passes, or n without hints) is large next to the mean cost per CTA
// gets a team: the smallest power of two T with cost / T <= (tile / 100) *
// (total cost / CTAs), at most TEAM_MAX, the grid, and one CTA per 4,096
// pixels (so a rank's pixels outweigh its barrier). Items are ordered by team
// time, cost / T, longest first; a slice's T seats are consecutive.
int fill_teams(fcm_ctx* h, int n, const fcm_batch_plan& p) {
    BatchedWorkspace* w = h->batched;
    const int ctas = team_ctas(h, p.block);
    if (ctas < 1) {
        h->last_error = "the team schedule needs cooperative launch support";
        return FCM_ERR_CUDA;
    }
    if (w->team_cap < n) {
        free_graphs(w);  // graphs point at the old buffers
        cudaFree(w->d_items);
        cudaFree(w->d_tslots);
        cudaFree(w->d_tctr);
        cudaFreeHost(w->h_items);
        w->d_items = nullptr;
        w->d_tslots = nullptr;
        w->d_tctr = nullptr;
        w->h_items = nullptr;
        w->team_cap = 0;
        const int cap = std::max(n, 64);
        CK(dev_malloc(h, &w->d_items, sizeof(int4) * (size_t)cap * TEAM_MAX));
        CK(host_malloc(h, &w->h_items, sizeof(int4) * (size_t)cap * TEAM_MAX));
        CK(dev_malloc(h, &w->d_tslots, sizeof(float2) * (size_t)cap * TEAM_MAX * 2 * TEAM_SLOT));
        CK(dev_malloc(h, &w->d_tctr, sizeof(unsigned) * cap));
        w->team_cap = cap;
    }
    double total = 0.0;
    for (int i = 0; i < n; ++i) total += (double)w->cost[i];
    const double target = std::max(1.0, (p.tile / 100.0) * total / ctas);
    const int tmax = std::min(TEAM_MAX, ctas);
    std::vector<int> T(n);
    for (int i = 0; i < n; ++i) {
        int t = 1;
        const int64_t by_size = std::max<int64_t>(1, w->size[i] / 4096);
        while (t < tmax && 2 * t <= by_size && (double)w->cost[i] / t > target) t *= 2;
        T[i] = t;
    }
    std::vector<int> ord(n);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(),
                     [&](int a, int b) { return (double)w->cost[a] / T[a] > (double)w->cost[b] / T[b]; });
    int base = 0, k = 0;
    for (int i = 0; i < n; ++i) {
        w->h_slot_base[i] = base;
        base += T[i];
    }
    for (int i : ord)
        for (int r = 0; r < T[i]; ++r) w->h_items[k++] = make_int4(i, r, T[i], 0);
    w->h_rhdr->n_slices = n;
    w->h_rhdr->max_rounds = k;  // the team schedule: number of items
    w->h_rhdr->wait_spins = h->limits.grid_spins;
    w->h_rhdr->phantoms = h->limits.phantoms;
    return 0;
}

int launch_teams(fcm_ctx* h, cudaStream_t s, const fcm_batch_plan& p, int n_slices) {
    BatchedWorkspace* w = h->batched;
    const BatchKernel k = kernel_for(p.block);
    const int ctas = team_ctas(h, p.block);
    if (ctas < 1) {
        h->last_error = "the team schedule needs cooperative launch support";
        return FCM_ERR_CUDA;
    }
    CK(cudaMemsetAsync(w->d_ctl, 0, sizeof(BatchCtl), s));
    CK(cudaMemsetAsync(w->d_tctr, 0, sizeof(unsigned) * n_slices, s));
    TeamArgs a;
    std::memset(&a, 0, sizeof(a));
    a.descs = w->d_desc;
    a.results = w->d_res;
    a.ctl = w->d_ctl;
    a.items = w->d_items;
    a.hdr = w->d_rhdr;
    a.slot_base = w->d_slot_base;
    a.slots = w->d_tslots;
    a.counters = w->d_tctr;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(p.block);
    cfg.dynamicSmemBytes = k.smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, k.teams, a));
    return 0;
}

// Uploads of one batch's work description (descriptors, order or tiling).
int upload_batch(fcm_ctx* h, cudaStream_t s, const fcm_batch_plan& p, int n) {
    BatchedWorkspace* w = h->batched;
    CK(cudaMemcpyAsync(w->d_desc, w->h_desc, sizeof(SliceDesc) * n, cudaMemcpyHostToDevice, s));
    if (p.schedule == FCM_SCHED_ROUNDS) {
        CK(cudaMemcpyAsync(w->d_rhdr, w->h_rhdr, sizeof(RoundsHdr), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(w->d_slot_base, w->h_slot_base, sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s));
    } else if (p.schedule == FCM_SCHED_TEAMS) {
        CK(cudaMemcpyAsync(w->d_rhdr, w->h_rhdr, sizeof(RoundsHdr), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(w->d_slot_base, w->h_slot_base, sizeof(int) * n, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(w->d_items, w->h_items, sizeof(int4) * (size_t)n * TEAM_MAX, cudaMemcpyHostToDevice, s));
    } else {
        CK(cudaMemcpyAsync(w->d_order, w->h_order, sizeof(int) * n, cudaMemcpyHostToDevice, s));
    }
    return 0;
}

// One launch of the slice-queue kernel over the whole order: phase 0 runs
// every slice (parking those not stopped after `cap` iterations), phase 1
// finishes the parked ones.
int launch_slices(fcm_ctx* h, cudaStream_t s, int block, int cluster, int64_t big, int n_slices, int phase,
                  int cap) {
    BatchedWorkspace* w = h->batched;
    const BatchKernel k = kernel_for(block);
    const int ctas = grid_ctas(h, block, cluster);
    if (ctas < cluster) {
        h->last_error = "batched launch shape does not fit on this device";
        return FCM_ERR_CUDA;
    }
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = k.smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CK(cudaMemsetAsync(w->d_ctl, 0, sizeof(BatchCtl), s));
    const SliceDesc* d = w->d_desc;
    const int* o = w->d_order;
    SliceResult* r = w->d_res;
    BatchCtl* c = w->d_ctl;
    CK(cudaLaunchKernelEx(&cfg, k.fn, d, o, n_slices, r, c, big, phase, cap));
    return 0;
}

int launch_kernel(fcm_ctx* h, cudaStream_t s, const fcm_batch_plan& p, int n_slices) {
    if (p.schedule == FCM_SCHED_ROUNDS) return launch_rounds(h, s, p, n_slices);
    if (p.schedule == FCM_SCHED_TEAMS) return launch_teams(h, s, p, n_slices);
    if (p.tile <= 0) return launch_slices(h, s, p.block, p.cluster, p.big, n_slices, 0, 0x7fffffff);
    // two phases: the slices that have not stopped after p.tile iterations
    // are finished by a second launch that gives big slices clusters of 8
    int rc = launch_slices(h, s, p.block, p.cluster, p.big, n_slices, 0, p.tile);
    if (rc) return rc;
    if (grid_ctas(h, 512, 8) >= 8) return launch_slices(h, s, 512, 8, 32768, n_slices, 1, 0x7fffffff);
    return launch_slices(h, s, 256, 4, 16384, n_slices, 1, 0x7fffffff);
}

// ---- autotune cache ------------------------------------------------------

std::string cache_path() {
    const char* p = std::getenv("FCM_AUTOTUNE_CACHE");
    return p ? std::string(p) : std::string();
}

void load_cache(BatchedWorkspace* w) {
    w->cache_loaded = true;
    const std::string path = cache_path();
    if (path.empty()) return;
    FILE* f = std::fopen(path.c_str(), "r");
    if (!f) return;
    // One entry per line:
    // "<key>": {"block": B, "cluster": K, "big": G, "ms": T, "schedule": S, "tile": L},
    char line[1024];
    while (std::fgets(line, sizeof(line), f)) {
        char key[512];
        int block = 0, cluster = 0, schedule = 0, tile = 0;
        long long big = 0;
        double ms = 0;
        if (std::sscanf(line,
                        " \"%511[^\"]\": {\"block\": %d, \"cluster\": %d, \"big\": %lld, \"ms\": %lf, "
                        "\"schedule\": %d, \"tile\": %d",
                        key, &block, &cluster, &big, &ms, &schedule, &tile) == 7) {
            const fcm_batch_plan p{block, cluster, (int64_t)big, ms, schedule, tile};
            if (plan_valid(p)) w->plans[key] = p;
        }
    }
    std::fclose(f);
}

void save_cache(BatchedWorkspace* w) {
    const std::string path = cache_path();
    if (path.empty()) return;
    const std::string tmp = path + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    std::fprintf(f, "{\n");
    size_t i = 0;
    for (auto& kv : w->plans) {
        std::fprintf(f,
                     "  \"%s\": {\"block\": %d, \"cluster\": %d, \"big\": %lld, \"ms\": %.4f, "
                     "\"schedule\": %d, \"tile\": %d}%s\n",
                     kv.first.c_str(), kv.second.block, kv.second.cluster, (long long)kv.second.big, kv.second.ms,
                     kv.second.schedule, kv.second.tile, ++i < w->plans.size() ? "," : "");
    }
    std::fprintf(f, "}\n");
    std::fclose(f);
    std::rename(tmp.c_str(), path.c_str());
}

int ilog2(int64_t v) {
    int l = 0;
    while (v > 1) {
        v >>= 1;
        ++l;
    }
    return l;
}

std::string bucket_key(fcm_ctx* h, const fcm_slice* s, int n, bool presolved) {
    int64_t total = 0, largest = 0;
    unsigned cset = 0;
    bool hinted = true;
    for (int i = 0; i < n; ++i) {
        total += s[i].n;
        largest = std::max(largest, s[i].n);
        cset |= 1u << s[i].C;
        hinted &= s[i].iters_hint > 0;
    }
    hinted |= presolved;
    char buf[512];
    std::snprintf(buf, sizeof(buf), "%s|C%x|s%d|p%d|l%d%s", h->device_name.c_str(), cset, ilog2(n), ilog2(total),
                  ilog2(largest), hinted ? "|hinted" : "");
    return buf;
}

fcm_batch_plan default_plan() { return fcm_batch_plan{512, 4, 65536, 0.0, FCM_SCHED_SLICES, 0}; }

}  // namespace

void fcm_release_batched(fcm_ctx* h) {
    if (!h || !h->batched) return;
    BatchedWorkspace* w = h->batched;
    free_graphs(w);
    cudaFree(w->d_desc);
    cudaFree(w->d_res);
    cudaFree(w->d_order);
    cudaFree(w->d_ctl);
    void* dev[] = {w->d_rstate, w->d_rctl, w->d_rhdr, w->d_slot_base, w->d_rpart, w->d_items, w->d_tslots, w->d_tctr};
    for (void* p : dev) cudaFree(p);
    cudaFreeHost(w->h_items);
    cudaFreeHost(w->h_desc);
    cudaFreeHost(w->h_res);
    cudaFreeHost(w->h_order);
    void* host[] = {w->h_rhdr, w->h_slot_base};
    for (void* p : host) cudaFreeHost(p);
    if (w->cap_stream) cudaStreamDestroy(w->cap_stream);
    delete w;
    h->batched = nullptr;
}

namespace {

bool device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// One batch, synchronously: descriptors and order are already in the pinned
// host buffers; results land in w->h_res.
int run_once(fcm_ctx* h, const fcm_batch_plan& p, int n, bool use_graph) {
    BatchedWorkspace* w = h->batched;
    int rc;
    if (!use_graph) {
        if ((rc = upload_batch(h, h->stream, p, n))) return rc;
        if ((rc = launch_kernel(h, h->stream, p, n))) return rc;
        CK(cudaMemcpyAsync(w->h_res, w->d_res, sizeof(SliceResult) * n, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        return 0;
    }
    const auto key = std::make_tuple(n, p.block, p.cluster, p.big, p.schedule, p.tile);
    auto it = w->graphs.find(key);
    if (it == w->graphs.end()) {
        cudaStream_t s = w->cap_stream;
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        int lrc = upload_batch(h, s, p, n);
        if (lrc == 0) lrc = launch_kernel(h, s, p, n);
        if (e == cudaSuccess && lrc == 0)
            e = cudaMemcpyAsync(w->h_res, w->d_res, sizeof(SliceResult) * n, cudaMemcpyDeviceToHost, s);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(s, &g);
        if (e != cudaSuccess || lrc != 0 || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return lrc ? lrc : ctx_fail(h, e != cudaSuccess ? e : e2, "capturing the batch graph");
        }
        GraphEntry ge;
        ge.graph = g;
        e = cudaGraphInstantiate(&ge.exec, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            return ctx_fail(h, e, "instantiating the batch graph");
        }
        it = w->graphs.emplace(key, ge).first;
    }
    CK(cudaGraphLaunch(it->second.exec, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return 0;
}

// Time one plan on the batch: best of `reps` launches after one warm-up.
int time_plan(fcm_ctx* h, const fcm_slice* slices, const fcm_batch_plan& p, int n, int reps, double* ms_out) {
    int rc = 0;
    if (p.schedule == FCM_SCHED_ROUNDS && (rc = fill_slots(h, slices, n, p.tile))) return rc;
    if (p.schedule == FCM_SCHED_TEAMS && (rc = fill_teams(h, n, p))) return rc;
    if (p.schedule == FCM_SCHED_SLICES) order_for(h->batched, n, p.big);
    if ((rc = upload_batch(h, h->stream, p, n))) return rc;
    rc = launch_kernel(h, h->stream, p, n);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double best = 1e30;
    for (int r = 0; r < reps && rc == 0; ++r) {
        cudaEventRecord(e0, h->stream);
        rc = launch_kernel(h, h->stream, p, n);
        cudaEventRecord(e1, h->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = FCM_ERR_CUDA;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, (double)ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_out = best;
    return rc;
}

}  // namespace

namespace {

// Argument checks shared by the batch entry points: sizes below n_limit,
// x 16-byte aligned. in_place: some slice updates its U^0 in place.
int check_slices(fcm_ctx* h, const fcm_slice* slices, int n_slices, int64_t n_limit, bool* in_place) {
    if (!slices || n_slices < 1) return ctx_invalid(h, "no slices");
    *in_place = false;
    for (int i = 0; i < n_slices; ++i) {
        const fcm_slice& s = slices[i];
        const bool ok = s.n >= 1 && s.n < n_limit && s.C >= 1 && s.C <= FCM_MAX_CLUSTERS && s.m > 1.0f &&
                        std::isfinite(s.m) && s.eps >= 0.0f && std::isfinite(s.eps) && s.max_iter >= 1 &&
                        (s.init_mode == FCM_INIT_U || s.init_mode == FCM_INIT_V) && s.x && s.U && s.V &&
                        ((uintptr_t)s.x % 16 == 0);
        if (!ok) {
            char buf[96];
            std::snprintf(buf, sizeof(buf), "slice %d: bad size, C, m, eps, max_iter, mode or pointer", i);
            return ctx_invalid(h, buf);
        }
        if (s.init_mode == FCM_INIT_U && (!s.U0 || s.U0 == s.U)) *in_place = true;
    }
    return FCM_OK;
}

// The device descriptors of a batch in the pinned host array, and its work
// order.
int fill_descs(fcm_ctx* h, const fcm_slice* slices, int n_slices, const int* hints = nullptr) {
    int rc = ensure_batched(h, n_slices);
    if (rc) return rc;
    BatchedWorkspace* w = h->batched;
    for (int i = 0; i < n_slices; ++i) {
        const fcm_slice& s = slices[i];
        const float* U0 = s.init_mode == FCM_INIT_U ? (s.U0 ? s.U0 : s.U) : s.U;
        const void* ptrs[4] = {s.x, s.U, s.V, U0};
        bool dev = true;
        for (const void* q : ptrs) {
            if (w->known_device.count(q)) continue;
            if (!device_ptr(q)) {
                dev = false;
                break;
            }
            if (w->known_device.size() > (1u << 16)) w->known_device.clear();
            w->known_device.insert(q);
        }
        if (!dev) {
            char buf[96];
            std::snprintf(buf, sizeof(buf), "slice %d: x, U, U0 and V must be device memory", i);
            return ctx_invalid(h, buf);
        }
        SliceDesc& d = w->h_desc[i];
        std::memset(&d, 0, sizeof(d));
        d.x = s.x;
        d.U0 = U0;
        d.U = s.U;
        d.V = s.V;
        d.n = s.n;
        d.C = s.C;
        d.mk = mkind_of(s.m);
        d.m = s.m;
        d.inv_m1 = (float)(1.0 / ((double)s.m - 1.0));
        d.eps = s.eps;
        d.max_iter = s.max_iter;
        d.init = s.init_mode;
        for (int j = 0; j < s.C; ++j) d.V0[j] = s.init_mode == FCM_INIT_V ? s.V0[j] : 0.0f;
    }
    // the cost of each slice for the work order: its pixels, times its
    // expected passes when every slice carries an iteration hint (its own,
    // or the pre-solve's in hints)
    auto hint = [&](int i) { return hints ? hints[i] : slices[i].iters_hint; };
    bool hinted = true;
    for (int i = 0; i < n_slices && hinted; ++i) hinted = hint(i) > 0;
    w->cost.resize(n_slices);
    w->size.resize(n_slices);
    for (int i = 0; i < n_slices; ++i) {
        w->size[i] = slices[i].n;
        w->cost[i] = hinted ? slices[i].n * (int64_t)(hint(i) + 3) : slices[i].n;
    }
    order_for(w, n_slices, (int64_t)1 << 62);
    return FCM_OK;
}

// Each slice's results from the pinned result array; the aggregate status.
int collect_results(fcm_ctx* h, fcm_slice* slices, int n_slices) {
    BatchedWorkspace* w = h->batched;
    int worst = FCM_OK;
    for (int i = 0; i < n_slices; ++i) {
        const SliceResult& r = w->h_res[i];
        fcm_slice& s = slices[i];
        s.iters = r.iters;
        s.status = r.status;
        s.flags = r.flags;
        s.delta = r.delta;
        s.J = r.J;
        for (int j = 0; j < FCM_MAX_CLUSTERS; ++j) s.V64[j] = j < s.C ? r.V64[j] : 0.0;
        if (r.status < 0 && worst >= 0) worst = r.status;
        if (r.status == FCM_NOT_CONVERGED && worst == FCM_OK) worst = FCM_NOT_CONVERGED;
    }
    return worst;
}

}  // namespace

namespace fcm {

int batch_descs(fcm_ctx* h, const fcm_slice* slices, int n_slices, int64_t n_limit, SliceDesc** h_desc,
                SliceDesc** d_desc) {
    bool in_place = false;
    int rc = check_slices(h, slices, n_slices, n_limit, &in_place);
    if (rc) return rc;
    if ((rc = fill_descs(h, slices, n_slices))) return rc;
    BatchedWorkspace* w = h->batched;
    CK(cudaMemcpyAsync(w->d_desc, w->h_desc, sizeof(SliceDesc) * n_slices, cudaMemcpyHostToDevice, h->stream));
    *h_desc = w->h_desc;
    *d_desc = w->d_desc;
    return FCM_OK;
}

}  // namespace fcm

namespace {

// FCM_BATCH_PRESOLVE: every slice's iteration count from its own start, run
// to convergence on its grey-level histogram (the runs give the per-pixel
// iterates up to rounding, so the counts agree within about one), into
// hints (the caller's structs are not touched). A slice that is not all grey
// levels gets the mean of the others.
int presolve_hints(fcm_ctx* h, const fcm_slice* slices, int n, std::vector<int>* hints) {
    for (int i = 0; i < n; ++i)
        if (slices[i].n >= ((int64_t)1 << 31)) return FCM_OK;  // beyond the bin counters: no hints
    SliceDesc *hd = nullptr, *dd = nullptr;
    int rc = batch_descs(h, slices, n, (int64_t)1 << 31, &hd, &dd);
    if (rc) return rc;
    std::vector<BinRun> runs(n);
    for (int i = 0; i < n; ++i) runs[i] = BinRun{i, slices[i].init_mode == FCM_INIT_U ? BIN_FROM_U : BIN_FROM_V, 0, 0};
    BatchedWorkspace* w = h->batched;
    if ((rc = bins_run(h, hd, dd, n, runs.data(), n, nullptr, 0, w->h_res))) return rc;
    CK(cudaStreamSynchronize(h->stream));
    int64_t sum = 0, cnt = 0;
    for (int i = 0; i < n; ++i)
        if (w->h_res[i].status >= 0 && w->h_res[i].iters > 0) {
            sum += w->h_res[i].iters;
            ++cnt;
        }
    hints->resize(n);
    for (int i = 0; i < n; ++i)
        (*hints)[i] = (w->h_res[i].status >= 0 && w->h_res[i].iters > 0) ? w->h_res[i].iters
                                                                        : (cnt ? (int)(sum / cnt) : 1);
    return FCM_OK;
}

}  // namespace

extern "C" {

int fcm_run_batched(fcm_handle h, fcm_slice* slices, int n_slices, int options) {
    NvtxRange nvtx_range("fcm_run_batched");
    if (!h) return FCM_ERR_INVALID_ARG;
    bool in_place = false;
    int rc = check_slices(h, slices, n_slices, (int64_t)1 << 40, &in_place);
    if (rc) return rc;
    DeviceGuard g(h->device);
    std::vector<int> hints;  // the pre-solve's iteration counts, or empty
    if (options & FCM_BATCH_PRESOLVE) {
        bool hinted = true;
        for (int i = 0; i < n_slices && hinted; ++i) hinted = slices[i].iters_hint > 0;
        if (!hinted && (rc = presolve_hints(h, slices, n_slices, &hints))) return rc;
    }
    rc = fill_descs(h, slices, n_slices, hints.empty() ? nullptr : hints.data());
    if (rc) return rc;
    BatchedWorkspace* w = h->batched;

    fcm_batch_plan plan;
    if (w->forced) {
        plan = w->forced_plan;
    } else {
        if (!w->cache_loaded) load_cache(w);
        const std::string key = bucket_key(h, slices, n_slices, !hints.empty());
        auto it = w->plans.find(key);
        const bool may_tune = !(options & FCM_BATCH_NO_TUNE) && !in_place;
        if (it != w->plans.end() && !(options & FCM_BATCH_RETUNE)) {
            plan = it->second;
        } else if (may_tune) {
            // time every candidate shape of both schedules on the batch itself
            std::vector<fcm_batch_plan> cands;
            const int blocks[2] = {256, 512};
            const int clusters[4] = {1, 2, 4, 8};
            const int64_t bigs[6] = {4096, 8192, 16384, 49152, 98304, 196608};
            const int tiles[3] = {2048, 8192, 32768};
            const int team_targets[3] = {50, 100, 200};
            for (int b : blocks) {
                for (int k : clusters)
                    for (int gi = 0; gi < (k == 1 ? 1 : 6); ++gi)
                        if (grid_ctas(h, b, k) >= k)
                            cands.push_back({b, k, k == 1 ? ((int64_t)1 << 62) : bigs[gi], 0.0, FCM_SCHED_SLICES, 0});
                if (n_slices <= ROUND_MAX_SLICES && round_ctas(h, b, round_smem(n_slices)) > 0)
                    for (int t : tiles) cands.push_back({b, 1, 0, 0.0, FCM_SCHED_ROUNDS, t});
                if (team_ctas(h, b) > 0)
                    for (int t : team_targets) cands.push_back({b, 1, 0, 0.0, FCM_SCHED_TEAMS, t});
            }
            fcm_batch_plan best = default_plan();
            best.ms = 1e30;
            fcm_batch_plan best_slices = default_plan();
            best_slices.ms = 1e30;
            for (const fcm_batch_plan& p : cands) {
                double ms = 0;
                if ((rc = time_plan(h, slices, p, n_slices, 2, &ms))) return rc;
                if (ms < best.ms) {
                    best = p;
                    best.ms = ms;
                }
                if (p.schedule == FCM_SCHED_SLICES && ms < best_slices.ms) {
                    best_slices = p;
                    best_slices.ms = ms;
                }
            }
            // then the best slice-queue shape split in two phases at a few caps
            const int caps[3] = {24, 40, 64};
            for (int cap : caps) {
                fcm_batch_plan p = best_slices;
                p.tile = cap;
                p.ms = 0.0;
                double ms = 0;
                if ((rc = time_plan(h, slices, p, n_slices, 2, &ms))) return rc;
                if (ms < best.ms) {
                    best = p;
                    best.ms = ms;
                }
            }
            plan = best;
            w->plans[key] = best;
            save_cache(w);
        } else {
            plan = default_plan();
        }
    }
    if (plan.schedule == FCM_SCHED_ROUNDS && (rc = fill_slots(h, slices, n_slices, plan.tile))) return rc;
    if (plan.schedule == FCM_SCHED_TEAMS && (rc = fill_teams(h, n_slices, plan))) return rc;
    if (plan.schedule == FCM_SCHED_SLICES) order_for(w, n_slices, plan.big);
    const bool use_graph = !(options & FCM_BATCH_NO_GRAPH);
    rc = run_once(h, plan, n_slices, use_graph);
    // a runtime that cannot capture a cooperative launch runs it directly
    if (rc && use_graph && plan.schedule != FCM_SCHED_SLICES) rc = run_once(h, plan, n_slices, false);
    if (rc) return rc;
    w->last = plan;

    return collect_results(h, slices, n_slices);
}

int fcm_run_batched_hist(fcm_handle h, fcm_slice* slices, int n_slices) {
    NvtxRange nvtx_range("fcm_run_batched_hist");
    if (!h) return FCM_ERR_INVALID_ARG;
    bool in_place = false;
    // 32-bit bin counters per slice
    int rc = check_slices(h, slices, n_slices, (int64_t)1 << 31, &in_place);
    if (rc) return rc;
    DeviceGuard g(h->device);
    rc = fill_descs(h, slices, n_slices);
    if (rc) return rc;
    BatchedWorkspace* w = h->batched;
    CK(cudaMemcpyAsync(w->d_desc, w->h_desc, sizeof(SliceDesc) * n_slices, cudaMemcpyHostToDevice, h->stream));
    // one run per slice, from its own start, writing its U and V
    std::vector<BinRun> runs(n_slices);
    for (int i = 0; i < n_slices; ++i)
        runs[i] = BinRun{i, slices[i].init_mode == FCM_INIT_U ? BIN_FROM_U : BIN_FROM_V, 1, 0};
    if ((rc = bins_run(h, w->h_desc, w->d_desc, n_slices, runs.data(), n_slices, nullptr, 0, w->h_res))) return rc;
    CK(cudaStreamSynchronize(h->stream));
    return collect_results(h, slices, n_slices);
}

int fcm_batched_plan(fcm_handle h, fcm_batch_plan* plan) {
    if (!h || !plan) return FCM_ERR_INVALID_ARG;
    if (!h->batched) return ctx_invalid(h, "no batched run yet");
    *plan = h->batched->last;
    return FCM_OK;
}

int fcm_batched_set_plan(fcm_handle h, const fcm_batch_plan* plan) {
    if (!h) return FCM_ERR_INVALID_ARG;
    if (!h->batched) h->batched = new BatchedWorkspace();
    if (!plan) {
        h->batched->forced = false;
        return FCM_OK;
    }
    if (!plan_valid(*plan))
        return ctx_invalid(h,
                           "plan: block 256|512; slices schedule: cluster 1|2|4|8, big >= 1, tile (first-phase "
                           "iteration cap) >= 0; rounds schedule: tile 1024..65536, a multiple of 1024");
    h->batched->forced = true;
    h->batched->forced_plan = *plan;
    return FCM_OK;
}

}  // extern "C"
