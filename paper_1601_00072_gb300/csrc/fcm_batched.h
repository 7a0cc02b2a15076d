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


struct TeamArgs;
typedef void (*TeamFn)(TeamArgs);

// Kernel of each block size, and its dynamic shared memory (x staging).
struct BatchKernel {
    BatchFn fn;
    int smem;
    int xcap;  // pixels of x one CTA keeps in shared memory
    TeamFn teams;  // the team schedule's cooperative kernel (same shared memory)
};

BatchKernel batched_kernel_256();
BatchKernel batched_kernel_512();

// ---- histogram-domain runs of 8-bit slices (fcm_bins.cu) ----
//
// Pixel passes are spread over the whole grid in chunks of BIN_CHUNK pixels
// (one CTA each, any number per slice); the iterations of Algorithm 1 run on
// each slice's 256 grey levels, one CTA per run. A "run" is one start of one
// slice: from its U^0 (the center sums of pass A) or from centers V^0. Several
// runs may share a slice's histogram (the warm-start judge solves each slice
// from its U^0 and from the predicted centers); at most one run per slice
// starts from U^0 and at most one writes the slice's U and V.
constexpr int BIN_CHUNK = 8192;

enum BinInit : int {
    BIN_FROM_U = 0,      // U^0 of the slice descriptor
    BIN_FROM_V = 1,      // V^0 of the slice descriptor
    BIN_FROM_V_DEV = 2,  // V^0 in device memory: row `slice` of BinArgs::v0_dev
};

struct alignas(8) BinChunk {
    int slice;
    int lo;  // first pixel; the chunk is [lo, min(lo + BIN_CHUNK, n))
};

struct alignas(16) BinRun {
    int slice;
    int init;     // BinInit
    int write_u;  // pass C writes the slice's U, and the solve its V
    int pad;
};

struct BinArgs {
    const SliceDesc* descs;  // [n_slices]
    const BinChunk* chunks;  // [n_chunks], slice-major
    const int* chunk_base;   // [n_slices + 1] first chunk of each slice
    const BinRun* runs;      // [n_runs]
    const int* slice_urun;   // [n_slices] the run from U^0 of each slice, or -1
    const int* slice_wrun;   // [n_slices] the run that writes each slice's U, or -1
    const float* v0_dev;     // BIN_FROM_V_DEV centers, row stride v0_stride
    int v0_stride;
    int n_slices, n_chunks, n_runs;
    int phase;               // solve: 0 first attempt, 1 the runs that needed pass B
    unsigned* hist;          // [n_slices][256] pixel counts
    int* rep;                // [n_slices][256] some pixel of each grey level, or -1
    unsigned* bad;           // [n_slices] bit 0: not all grey levels; bit 1: a bad U^0;
                             // bit 2: a FCM_DEBUG_BOUNDS guard skipped an access
    float2* part;            // [n_chunks][2 * FCM_MAX_CLUSTERS] (hi, lo) sums of V^1
    float* table;            // [n_runs][256][FCM_MAX_CLUSTERS] U^1, then U^k, per grey level
    unsigned* d1;            // [n_runs] first stopping quantity from pass B (float bits)
    int* need_b;             // [n_runs] the lower bound could not decide the first stop
    SliceResult* results;    // [n_runs]
};

// The kernels of one bin-domain batch, in stream order: the caller has
// zeroed hist, bad, d1 and need_b and set rep to -1.
cudaError_t launch_bins(const BinArgs& a, bool write_any, cudaStream_t s);

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
    int max_rounds;       // largest max_iter + 1
    uint32_t wait_spins;  // polls of the round barrier before it gives up
    uint32_t phantoms;    // extra arrivals the barrier waits for (fault injection; 0 normally)
};

// ---- team schedule (a slice shared by any number of CTAs of the grid) ----

constexpr int TEAM_MAX = 32;                        // largest team
constexpr int TEAM_SLOT = 2 * FCM_MAX_CLUSTERS + 3;  // values a rank publishes per pass

struct TeamArgs {
    const SliceDesc* descs;
    SliceResult* results;
    BatchCtl* ctl;          // queue head
    const int4* items;      // (slice, seat, team size, 0), seats of a slice in a row
    const RoundsHdr* hdr;   // n_slices; max_rounds = number of items; wait_spins, phantoms
    const int* slot_base;   // [n_slices]: first rank slot of each slice
    float2* slots;          // [sum of team sizes][2][TEAM_SLOT]
    unsigned* counters;     // [n_slices] barrier arrivals (zero before the batch)
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
