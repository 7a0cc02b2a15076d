// Host/device shared definitions of the single-image FCM path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fcm.h"

namespace fcm {

constexpr int NT = 256;                                  // threads per block of the pass
constexpr int NWARP = NT / 32;
constexpr int WARP_TILE = 128;                           // pixels per warp tile of the TMA kernels
constexpr int DCHUNK = 4;  // tiles per grab from the shared part of a pass (stored-U whole-run kernel)
// Issue-side state of one warp's TMA ring in the stored-U whole-run kernel
// (lane 0 only, kept in shared memory): copies issued, next tile of the chunk being
// issued, pass, index in the fixed share, ring slot, tiles left in the chunk,
// and the counter value grabbed for the next chunk.
struct IssueState {
    int64_t issued, cb;
    int ip, ik, is, cl;
    unsigned grab;
};
constexpr int SLOTS_MAX = 2 * FCM_MAX_CLUSTERS + 4;      // num[C], den[C], J, delta, 2 flags
constexpr int STATUS_RUNNING = 2;

// Bounds of the device-side waits of one run, set per handle from the host
// (fcm_set_limits). Every spin or suspension loop counts against one of them
// and, when it runs out, the kernel records FCM_ERR_TIMEOUT and returns.
struct WaitLimits {
    uint32_t grid_spins;  // polls, about 128 ns apart, of a grid-wide barrier
    uint32_t tma_polls;   // suspensions, up to about 1 ms each, of a wait for TMA bytes
    uint32_t phantoms;    // arrivals every grid-wide barrier waits for beyond the
                          // grid's own: 0 in normal use; a test sets 1 to make
                          // every barrier give up (fault injection on the host side)
    uint32_t pad;
};
constexpr uint32_t DEFAULT_GRID_SPINS = 1u << 23;  // about 1 s
constexpr uint32_t DEFAULT_TMA_POLLS = 2048;       // about 2 s

// Which half-step a launch of the pass performs.
enum Pass : int {
    P_ACCUM0 = 0,  // V^1 from a given U^0 (Eq. 3); validates x and U^0
    P_INITV = 1,   // U^0 = membership(V^0) (Eq. 4), written to U; V^1 from it
    P_ITER = 2,    // U^k from V^k in place, delta_k, J_k, V^{k+1} (Eqs. 4, 1, 3)
    P_COUNT = 3
};

// Device-resident state of one run. The host writes the whole struct before a
// run; the passes read their inputs from it and the last block of each pass
// writes the evolving part. Kernels and graphs therefore never need new
// parameters when the caller's buffers change.
struct alignas(128) RunState {
    // per-run inputs
    const float* x;
    const float* Uprev;  // U^{k-1}: the caller's U^0 for the first pass, then U
    float* U;            // U^k, written in place
    double* trace;   // nullable: (max_iter) rows of (delta, J, V^k[C])
    int64_t n;
    float m;
    float inv_m1;    // 1 / (m - 1)
    float eps;
    int max_iter;
    int C;
    int pad0;
    float V0[FCM_MAX_CLUSTERS];
    // evolving
    float V[FCM_MAX_CLUSTERS];      // V^k used by the next pass
    double V64[FCM_MAX_CLUSTERS];   // the FP64 quotients V rounds
    double delta;
    double J;
    int k;          // index of the next iteration
    int status;
    int done;
    int flags;
    int iters;
    unsigned int ticket;  // last-block-done counter of the current pass
    int launches;         // passes started in this run (loop guard)
    WaitLimits lim;
    // stored-U whole-run kernel: percent of each pass's tiles dealt to the
    // warps in fixed shares (100: all of them); the rest is taken in chunks from
    // dyn[pass & 1] (zeroed by the upload of this state, re-zeroed on the
    // device two passes before each reuse)
    int static_pct;
    unsigned int dyn[2];
    unsigned int bounds;  // FCM_FLAG_BOUNDS from a FCM_DEBUG_BOUNDS build's guards
};
constexpr int DEFAULT_STATIC_PCT = 60;

typedef void (*PassFn)(RunState*, double*, cudaGraphConditionalHandle, int);

// Kernel table: [C][m kind][pass][variant], variant 0 = grid-stride scalar
// loads (any n), 1 = TMA ring (n % 4 == 0, 16-byte aligned rows); smem holds
// each kernel's dynamic shared memory in bytes.
typedef void (*RunFn)(RunState*, double*);

struct SingleTable {
    PassFn k[FCM_MAX_CLUSTERS + 1][4][P_COUNT][2];
    int smem[FCM_MAX_CLUSTERS + 1][4][P_COUNT][2];
    // the whole run in one cooperative launch: [C][m kind][0 = from U^0, 1 = from V^0]
    RunFn run[FCM_MAX_CLUSTERS + 1][4][2];
    int run_smem[FCM_MAX_CLUSTERS + 1];
};

// The kernel table, filled on first use.
const SingleTable& single_table();

void register_single_c1(SingleTable&);
void register_single_c2(SingleTable&);
void register_single_c3(SingleTable&);
void register_single_c4(SingleTable&);
void register_single_c5(SingleTable&);
void register_single_c6(SingleTable&);
void register_single_c7(SingleTable&);
void register_single_c8(SingleTable&);

}  // namespace fcm
