// Shared definitions of the batched FCM path (host runtime and kernels).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fcm.h"

namespace fcm {

// Device-side copy of one slice's arguments.
struct alignas(16) SliceDesc {
    const float* x;
    const float* U0;  // initial memberships (FCM_INIT_U); may equal U
    float* U;         // final memberships, written once at the end
    float* V;         // final centers (device)
    int64_t n;
    int C;
    int mk;           // fuzzifier kind (MKind)
    float m, inv_m1, eps;
    int max_iter;
    int init;         // FCM_INIT_U or FCM_INIT_V
    int pad;
    float V0[FCM_MAX_CLUSTERS];  // initial centers (FCM_INIT_V), copied before the run
};

// Status of a slice parked by the first phase of a two-phase batch (never
// returned to the caller: the second phase finishes every parked slice).
constexpr int SLICE_PARKED = 3;

struct alignas(16) SliceResult {
    int iters;
    int status;
    int flags;
    int pad;
    double delta;
    double J;
    double V64[FCM_MAX_CLUSTERS];
    // state of a parked slice: V^k and V^{k-1} for iteration k = iters + 1
    float vcur[FCM_MAX_CLUSTERS];
    float vprev[FCM_MAX_CLUSTERS];
};

struct alignas(128) BatchCtl {
    unsigned int next;  // work-queue head (index into the LPT order)
    unsigned int pad[31];
};

// Launch shape of the batched kernel.
struct BatchPlan {
    int block;      // threads per CTA: 256 or 512
    int cluster;    // CTAs per cluster: 1, 2, 4 or 8
    int64_t big;    // slices with n >= big are shared by a whole cluster
};

// phase 0: every slice from its start, parked before iteration cap + 1 when it
// has not stopped by then; phase 1: only the parked slices, resumed from their
// saved state.
typedef void (*BatchFn)(const SliceDesc*, const int*, int, SliceResult*, BatchCtl*, int64_t, int, int);

// Kernel of each block size, and its dynamic shared memory (x staging).
struct BatchKernel {
    BatchFn fn;
    int smem;
    int xcap;  // pixels of x one CTA keeps in shared memory
};

BatchKernel batched_kernel_256();
BatchKernel batched_kernel_512();

// Histogram-domain runs of 8-bit slices, one CTA per slice in the given order
// (fcm_bhist.cu).
cudaError_t launch_bhist(const SliceDesc* descs, const int* order, int n_slices, SliceResult* results,
                         cudaStream_t s);

// ---- round-synchronous schedule (every slice steps in every round) ----

constexpr int ROUND_SUMS = 2 * FCM_MAX_CLUSTERS + 3;  // values per slot: num[C], den[C], J, max|dU|, bad
constexpr int ROUND_MAX_SLICES = 8192;                 // the per-round prefix lives in shared memory

// Mutable per-slice state, written by the slice's finaliser.
struct alignas(16) RoundSlice {
    double v64[FCM_MAX_CLUSTERS];   // FP64 quotients behind vcur
    float vcur[FCM_MAX_CLUSTERS];   // V^k
    float vprev[FCM_MAX_CLUSTERS];  // V^{k-1}
    unsigned ticket;                // segments of this round finished (reset by the finaliser)
    int end_round;                  // open (INT_MAX), round of the U write, or -1 (bad input)
    int flags;
    int pad;
};

struct alignas(128) RoundCtl {
    unsigned bar;        // grid barrier arrivals
    unsigned undecided;  // slices without a stop decision
    int last_round;      // latest round in which some slice writes its U
    unsigned timeout;    // set when a grid barrier wait gave up
    unsigned pad[28];
};

// Sizes of one batch, uploaded with the descriptors (so one captured graph
// serves every batch of the same slice count and plan).
struct alignas(16) RoundsHdr {
    int n_slices;
    int max_rounds;  // largest max_iter + 1
    int pad[2];
};

struct RoundsArgs {
    const SliceDesc* descs;
    SliceResult* results;
    RoundSlice* state;
    RoundCtl* ctl;
    const RoundsHdr* hdr;
    const int* slot_base;  // [n_slices + 1] first slot of each slice
    double* partials;      // [slots * ROUND_SUMS], sum-major within a slice
    int min_chunk;         // fewest pixels a CTA takes in a round (even)
    int pad;
    uint32_t wait_spins;   // polls of the round barrier before it gives up
    uint32_t phantoms;     // extra arrivals the barrier waits for (fault injection; 0 normally)
};

// Slots a slice needs: at most ceil(n / min_chunk) + 1 CTAs share it in a round.
inline int64_t round_slots(int64_t n, int min_chunk) { return (n + 1 + min_chunk - 1) / min_chunk + 2; }

struct RoundsKernel {
    void (*fn)(RoundsArgs);
    void (*init)(RoundSlice*, SliceResult*, RoundCtl*, int);
};

RoundsKernel rounds_kernel_256();
RoundsKernel rounds_kernel_512();

}  // namespace fcm
