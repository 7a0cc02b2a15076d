/*
 * fcm.h — C ABI of the GB300 Fuzzy C-Means library (libfcm_gb300.so).
 *
 * The library runs the per-iteration pixel pass of Fuzzy C-Means image
 * segmentation (arXiv:1601.00072, "GPU-Based Fuzzy C-Means Clustering
 * Algorithm for Image Segmentation") on one CUDA device:
 *
 *   membership (Eq. 4)  u_ij = 1 / sum_k (d_ij / d_ik)^(2/(m-1)),
 *                       d_ij = |x_i - v_j|   (Sec. 2.1; grey level feature)
 *   centers    (Eq. 3)  v_j  = sum_i u_ij^m x_i / sum_i u_ij^m
 *   objective  (Eq. 1)  J_m  = sum_i sum_j u_ij^m d_ij^2
 *   loop (Algorithm 1)  V from U, then U from V, until the change of U
 *                       between iterations falls below eps.
 *
 * Conventions shared by every entry point:
 *   - Pixels x: n floats (grey levels; the paper's data is uint8 cast to
 *     float). Memberships U: C*n floats, cluster-major, U[j*n + i] (the
 *     paper's 1-D layout of the 3-D membership array, Sec. 5.1).
 *     Centers V: C floats.
 *   - 1 <= C <= FCM_MAX_CLUSTERS; m > 1 (Eq. 4's exponent 2/(m-1) needs it);
 *     eps >= 0; max_iter >= 1; n >= 1.
 *   - Zero distance (a pixel exactly equal to one or more centers): those
 *     clusters share the membership equally, every other cluster gets 0
 *     (Bezdek's rule; the paper does not define the case).
 *   - Stopping test: iteration k computes U^k from V^k and
 *     delta_k = max_{i,j} |u^k_ij - u^{k-1}_ij| (L-infinity, Algorithm 1
 *     step 3); the run stops with (U^k, V^k) when delta_k < eps (strict),
 *     else V^{k+1} = centers(U^k). V^1 comes from the initial U^0, or from
 *     U^0 = membership(V^0) when initial centers are given.
 *   - Arithmetic: memberships and per-thread sums in FP32; the sums across
 *     threads and blocks (center numerators/denominators and J) in
 *     compensated FP32 (double-float, about 44 bits) or FP64, in a fixed
 *     order. A run is deterministic, with one exception: on images large
 *     enough that every warp of the default whole-run kernel (stored U)
 *     holds more than a ring of tiles (about 4 million pixels), 40% of each
 *     pass's tiles go to whichever warps ask first, so SMs that stream
 *     faster take more of them (about 11% faster on a 256^3 volume). Which
 *     block sums which tile then depends on timing, and so does the FP32
 *     rounding of the block sums: results agree to rounding, and the
 *     iteration count can differ by one when delta_k lands at eps.
 *     FCM_OPT_DETERMINISTIC keeps fixed shares for bit-reproducible runs.
 *     The histogram-domain entry points form V^1 the same way from the
 *     pixels; their loop over the 256 bins sums non-negative terms in FP32
 *     within each warp (a fixed tree, at most five roundings) and combines
 *     the warp totals in double-float.
 *   - Ownership: the caller owns x, U, V and every output array; the library
 *     never frees them. A handle owns its device workspace, CUDA graphs and
 *     autotuning cache, and frees them in fcm_destroy.
 *   - Streams: work is issued on the handle's stream. Entry points that fill
 *     host-side results (iters, reports, statuses) synchronise that stream
 *     before returning. fcm_run_stream also uses an upload and a download
 *     stream of the handle's own, ordered after the work already queued on
 *     the handle's stream, and returns after all three have drained.
 *   - Errors: every entry point returns an int status (FCM_OK or
 *     FCM_NOT_CONVERGED on success, a negative FCM_ERR_* otherwise);
 *     fcm_status_string names it. A handle is not thread-safe.
 */
#ifndef FCM_GB300_H
#define FCM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FCM_MAX_CLUSTERS 8

/* Status codes. */
#define FCM_OK 0                 /* converged: delta_k < eps                 */
#define FCM_NOT_CONVERGED 1      /* stopped at max_iter; results are valid   */
#define FCM_ERR_INVALID_ARG (-1) /* bad size, m <= 1, null pointer, ...      */
#define FCM_ERR_CUDA (-2)        /* a CUDA runtime call failed               */
#define FCM_ERR_OOM (-3)         /* workspace allocation failed              */
#define FCM_ERR_BAD_INPUT (-4)   /* NaN/Inf in x or V0, or NaN/Inf/negative U0 */
#define FCM_ERR_NONFINITE FCM_ERR_BAD_INPUT /* the same code, named after its commonest cause */
#define FCM_ERR_TIMEOUT (-5)     /* a bounded device-side wait gave up       */
#define FCM_ERR_TOO_LARGE (-6)   /* beyond a fixed limit of fcm_run_noalloc  */

/* Report flags. */
#define FCM_FLAG_EMPTY_CLUSTER 1 /* some sum_i u_ij^m underflowed to 0: v_j kept */
#define FCM_FLAG_BOUNDS 2 /* a FCM_DEBUG_BOUNDS build skipped an out-of-range access
                             (a library bug; never set by the normal build) */

/* Initialisation modes (Algorithm 1 step 2). */
#define FCM_INIT_U 0 /* U holds the initial membership U^0 on entry         */
#define FCM_INIT_V 1 /* V holds initial centers V^0; U^0 = membership(V^0)  */

/* Run options (bit flags). */
#define FCM_OPT_TRACE 1    /* record delta_k, J_k and V^k of every iteration */
#define FCM_OPT_NO_GRAPH 2 /* host-driven loop instead of a CUDA graph WHILE node */
#define FCM_OPT_NO_TMA 4   /* plain-load pass kernel instead of the TMA-fed one */
#define FCM_OPT_NO_PERSISTENT 8 /* one launch per pass (graph or host loop) instead of
                                    one cooperative launch for the whole run */
#define FCM_OPT_RECOMPUTE 16 /* do not store U between iterations: recompute U^{k-1}
                                 from V^{k-1}, so an iteration reads only x; U^k is
                                 written once at the end (one cooperative launch;
                                 needs n % 4 == 0 and 16-byte-aligned rows) */
#define FCM_OPT_DETERMINISTIC 32 /* whole-run kernel: every tile in fixed warp
                                     shares, so the result does not depend on
                                     timing (see the arithmetic note above) */

typedef struct fcm_ctx* fcm_handle;

/* Result of one run. V64 holds the final centers as the quotients of the
 * combined sums, to about 44 bits or better, in FP64 (V holds the same values
 * rounded to float). */
typedef struct {
    int iters;      /* k of the returned (U^k, V^k)                         */
    int status;     /* FCM_OK, FCM_NOT_CONVERGED or a negative FCM_ERR_*     */
    int flags;      /* FCM_FLAG_* bits                                       */
    int C;
    double delta;   /* delta_k of the last iteration (L-infinity)            */
    double J;       /* J_m(U^k, V^k), Eq. 1                                  */
    double V64[FCM_MAX_CLUSTERS];
    int launches;   /* kernel launches the run used                          */
    int reserved;
} fcm_report;

/* Create a handle on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream). Allocates nothing on
 * the device until the first run. Returns FCM_ERR_CUDA for a bad device. */
int fcm_create(fcm_handle* out, int device, void* cuda_stream);

/* Rebind the handle to another stream of the same device. */
int fcm_set_stream(fcm_handle h, void* cuda_stream);

/* Free the handle's workspace and graphs (never caller buffers). NULL is a
 * no-op. */
void fcm_destroy(fcm_handle h);

/*
 * Bounds of the device-side waits, and fault injection for tests. Not in the
 * paper: its kernels never wait on one another (Sec. 4); here a whole run is
 * one cooperative launch whose blocks meet at a grid-wide barrier after every
 * pass, and passes wait for TMA copies. Every such wait polls a bounded number
 * of times and then gives up: the run ends with FCM_ERR_TIMEOUT (U and V
 * unspecified) and the handle stays usable.
 *
 *   grid_wait_spins   polls, about 128 ns apart, of a grid-wide barrier
 *                     (whole-run, U-free, multi-feature and round-schedule
 *                     kernels). 0 = the default 2^23 (about 1 s). The
 *                     environment variable FCM_TIMEOUT_SPINS sets the default
 *                     of new handles.
 *   tma_wait_polls    suspensions, up to about 1 ms each, of a wait for a TMA
 *                     copy to land. 0 = the default 2048.
 *   barrier_phantoms  for tests: every grid-wide barrier also waits for this
 *                     many arrivals that never come, so it gives up after
 *                     grid_wait_spins polls. 0 (normal use) to 1024.
 *   fail_alloc_in     for tests: when > 0, the handle's allocation that many
 *                     calls from now (1 = the next) fails as if the device
 *                     were out of memory, once: the entry point that made it
 *                     returns FCM_ERR_OOM and a later call completes the
 *                     workspace. 0 = off.
 */
typedef struct {
    uint32_t grid_wait_spins;
    uint32_t tma_wait_polls;
    uint32_t barrier_phantoms;
    int32_t fail_alloc_in;
} fcm_limits;

/* Set the limits (NULL restores every default and turns injection off). */
int fcm_set_limits(fcm_handle h, const fcm_limits* lim);
/* The limits in force (defaults filled in). */
int fcm_get_limits(fcm_handle h, fcm_limits* lim);

/*
 * fcm_run — Algorithm 1 on one image (Sec. 2.1, Eqs. 1, 3, 4; the paper's
 * center kernels of Sec. 4.2 and membership kernel of Sec. 4.3 are one fused
 * pass here, and its host-side convergence check of Sec. 4.3 runs on the
 * device).
 *
 *   x         n floats, device or host memory (host memory is staged through
 *             the handle's workspace; pinned host memory copies fastest).
 *   n         number of pixels, >= 1.
 *   C, m, eps, max_iter   as above.
 *   init_mode FCM_INIT_U or FCM_INIT_V.
 *   U0        nullable; C*n floats, cluster-major, device or host, read only.
 *             With FCM_INIT_U and U0 != NULL the initial membership is read
 *             from U0 and left unchanged; with U0 == NULL (or U0 == U) it is
 *             read from U. Ignored with FCM_INIT_V.
 *   U         C*n floats, cluster-major, device or host. Out: U^k (the run
 *             updates it in place from the first iteration on).
 *   V         C floats, device or host. In: V^0 when init_mode == FCM_INIT_V.
 *             Out: V^k.
 *   options   FCM_OPT_* bits. By default, when n % 4 == 0 and the buffers are
 *             16-byte aligned, the whole run is one cooperative kernel launch
 *             (grid-wide exchange of the per-block sums after each pass);
 *             otherwise, or with FCM_OPT_NO_PERSISTENT, one launch per pass
 *             inside a CUDA graph WHILE loop (or a host loop with
 *             FCM_OPT_NO_GRAPH).
 *   rep       nullable; filled on return.
 *
 * Returns FCM_OK, FCM_NOT_CONVERGED, or an error. On FCM_ERR_BAD_INPUT the
 * contents of U and V are unspecified.
 */
int fcm_run(fcm_handle h, const float* x, int64_t n, int C, float m,
            float eps, int max_iter, int init_mode, const float* U0, float* U,
            float* V, int options, fcm_report* rep);

/*
 * fcm_init_dirichlet — the random initial membership of Algorithm 1 step 2
 * ("initialize U randomly", Sec. 2.1), drawn on the device: each pixel's
 * column of U^0 is a uniform Dirichlet(1, ..., 1) draw, C standard
 * exponentials E_j = -ln r_j normalised to sum 1. The uniforms r_j come from
 * the counter-based generator Philox4x32-10 (Salmon et al., SC'11): pixel i
 * uses counter (i mod 2^32, i div 2^32, j div 4, 0) under key
 * (seed mod 2^32, seed div 2^32), word j mod 4; a word w gives
 * r = (2 floor(w / 512) + 1) / 2^24. A pixel's draw depends only on its index
 * and the seed. Exponentials and the normalisation are FP32.
 *
 *   n, C     pixels (>= 1) and clusters (1..8).
 *   U        C*n floats, device memory, cluster-major; receives U^0.
 *
 * Queued on the handle's stream; returns FCM_OK or FCM_ERR_INVALID_ARG.
 */
int fcm_init_dirichlet(fcm_handle h, int64_t n, int C, uint64_t seed, float* U);

/*
 * fcm_run_seeded — fcm_run from the seeded random start: fcm_init_dirichlet
 * into U, then fcm_run with FCM_INIT_U and U^0 read from U (updated in place).
 * Arguments as fcm_run; U must be device memory.
 */
int fcm_run_seeded(fcm_handle h, const float* x, int64_t n, int C, float m, float eps, int max_iter,
                   uint64_t seed, float* U, float* V, int options, fcm_report* rep);

/*
 * fcm_run_stream — fcm_run over a sequence of images of one shape (n pixels,
 * C clusters, the same m, eps and max_iter), each read from and written back
 * to host memory, with the host-device copies overlapped with the runs:
 * while image i runs on the handle's stream, the upload of image i+1 and the
 * download of image i-1 proceed on two copy streams of the handle, through
 * three device staging sets it owns (3 x (4 + 4C) x n bytes). Each image is one run of Algorithm 1
 * (Sec. 2.1) from its own U^0, computed by the same whole-run kernel as
 * fcm_run with FCM_INIT_U, so each result equals that call's on the image.
 *
 *   n_images  >= 1.
 *   x         n_images pointers to n floats each. Host memory (pinned memory
 *             lets the copies overlap the runs; pageable memory works but the
 *             driver stages it) or device memory.
 *   U0        nullable array of n_images pointers to C*n floats, cluster-
 *             major, read only. A NULL array, or a NULL entry, reads image
 *             i's U^0 from U[i].
 *   U         n_images pointers to C*n floats. Out: each image's U^k.
 *   V         n_images*C floats, host memory. Out: row i = image i's V^k.
 *   options   0, or FCM_OPT_RECOMPUTE and/or FCM_OPT_DETERMINISTIC.
 *   reps      nullable; n_images reports.
 *
 * Needs n % 4 == 0 and a device with cooperative launch; returns
 * FCM_ERR_INVALID_ARG otherwise. Returns after every image is done and every
 * copy has landed: FCM_OK when all converged, FCM_NOT_CONVERGED when some
 * image hit max_iter, else the first image's error status (reps[i].status
 * holds each image's own; the other images' results are valid). A CUDA
 * error ends the call with FCM_ERR_CUDA after the handle's streams drain.
 */
int fcm_run_stream(fcm_handle h, int n_images, const float* const* x, int64_t n, int C, float m,
                   float eps, int max_iter, const float* const* U0, float* const* U, float* V,
                   int options, fcm_report* reps);

/*
 * fcm_run_hist — Algorithm 1 (Sec. 2.1) for images whose intensities are
 * integer grey levels 0..255, run on the 256-bin histogram (the grey-level
 * reduction of brFCM, cited in Sec. 3). Under Eq. 4 a pixel's memberships
 * depend only on its grey level, so after pass 0 every center update (Eq. 3),
 * J (Eq. 1) and stopping quantity is a sum or maximum over the grey levels
 * present, weighted by their pixel counts. The iterates equal fcm_run's up to
 * the order of rounding: same U^0, V^1, stopping rule and outputs. With
 * FCM_INIT_U the first stopping quantity compares U^1 with every pixel's U^0.
 *
 * Arguments as fcm_run, except: x, U and U0 must be device memory (V may be
 * host or device), and there are no options. Passes over the pixels: one
 * (histogram, and with FCM_INIT_U the sums of V^1), one more with FCM_INIT_U
 * (first stopping quantity), and one that writes U^k; the iterations run in
 * one CTA on the bins.
 *
 * Returns as fcm_run; FCM_ERR_BAD_INPUT when some x_i is not an integer in
 * [0, 255] (or not finite), or U^0 holds a negative or non-finite value, or V^0
 * a non-finite one. U is not written then.
 */
int fcm_run_hist(fcm_handle h, const float* x, int64_t n, int C, float m, float eps, int max_iter,
                 int init_mode, const float* U0, float* U, float* V, fcm_report* rep);

/*
 * fcm_dsc — defuzzify a result and score it against ground truth with the
 * Dice similarity coefficient per class (Sec. 5.2, Eq. 5):
 * DSC_c = 2 |PR_c n GT_c| / (|PR_c| + |GT_c|).
 *
 *   U                 C*n floats, cluster-major, device memory (a run's U^k).
 *                     Pixel i's label is argmax_j U[j*n + i], ties to the
 *                     lowest j (Sec. 2.1).
 *   truth             n bytes, device memory: the true class of each pixel, in
 *                     [0, n_classes).
 *   class_of_cluster  C ints, host memory: the class each cluster stands for.
 *   n_classes         1..16.
 *   counts            nullable, host, 3*n_classes: |PR_c|, |GT_c|, |PR_c n GT_c|.
 *   dsc               host, n_classes doubles. A class absent from both the
 *                     segmentation and the truth scores 1.
 *
 * The counts are exact integers. Returns FCM_OK, or FCM_ERR_INVALID_ARG (also
 * for a truth label outside [0, n_classes)).
 */
int fcm_dsc(fcm_handle h, const float* U, int64_t n, int C, const uint8_t* truth, const int* class_of_cluster,
            int n_classes, int64_t* counts, double* dsc);

/*
 * fcm_run_multi — Algorithm 1 on pixels with D channels (colour, or
 * co-registered MR sequences). Sec. 2.1 defines d_ij as a norm of x_i - v_j;
 * here it is the Euclidean norm over the channels, so Eq. 4 uses
 * d_ij^2 = sum_d (x_id - v_jd)^2, Eq. 3 gives each center channel by channel
 * and Eq. 1 sums u_ij^m d_ij^2. Readings as fcm_run (zero distance, L-infinity
 * stopping test, empty clusters). One cooperative launch per run; U^{k-1} is
 * recomputed from V^{k-1}, so an iteration reads only x and U^k is written
 * once at the end.
 *
 *   x        D*n floats, channel-major (x[d*n + i]), device memory.
 *   D        1..4 channels.  C, m, eps, max_iter, init_mode as fcm_run.
 *   U0       nullable; C*n floats, device, read only (FCM_INIT_U; NULL means
 *            U holds U^0).
 *   U        C*n floats, device. Out: U^k.
 *   V        C*D floats, cluster-major (V[j*D + d]), device or host. In: V^0
 *            with FCM_INIT_V. Out: V^k.
 *   V64      nullable, host, C*D doubles: the FP64 quotients behind V^k.
 *   rep      nullable; its V64 holds the first min(C*D, 8) of them.
 *
 * Returns as fcm_run.
 */
int fcm_run_multi(fcm_handle h, const float* x, int64_t n, int D, int C, float m, float eps, int max_iter,
                  int init_mode, const float* U0, float* U, float* V, double* V64, fcm_report* rep);

/*
 * Batched runs: many independent images ("slices") of different sizes, cluster
 * counts and fuzzifiers in one persistent launch (not in the paper, which
 * segments one image at a time; each slice follows Algorithm 1 exactly as
 * fcm_run does).
 *
 * fcm_slice — one slice. Pointers are device memory.
 *   x         n floats, 16-byte aligned.
 *   n, C, m, eps, max_iter   as for fcm_run.
 *   init_mode FCM_INIT_U (U^0 in U0, or in U when U0 is NULL) or FCM_INIT_V
 *             (initial centers in V0[], host values inside the struct).
 *   iters_hint  0, or the iterations the slice is expected to take. When
 *             every slice of a batch has one, the slice-queue schedule takes
 *             slices in order of decreasing cost n * (iters_hint + 3) instead
 *             of decreasing n (fcm_run_batched_warm sets them from its
 *             histogram-domain runs).
 *   U0        C*n floats, cluster-major, read only; nullable.
 *   U         C*n floats, cluster-major: receives U^k.
 *   V         C floats: receives V^k.
 *   iters, status, flags, delta, J, V64: outputs, written on return.
 */
typedef struct {
    const float* x;
    int64_t n;
    int C;
    float m;
    float eps;
    int max_iter;
    int init_mode;
    int iters_hint;
    const float* U0;
    float* U;
    float* V;
    float V0[FCM_MAX_CLUSTERS];
    int iters;
    int status;
    int flags;
    int reserved1;
    double delta;
    double J;
    double V64[FCM_MAX_CLUSTERS];
} fcm_slice;

/* Launch shape of the batched kernels (see fcm_run_batched). */
#define FCM_SCHED_SLICES 0 /* slices from a queue, one CTA or one cluster each     */
#define FCM_SCHED_ROUNDS 1 /* every slice steps each round; pixels tiled over the grid */
#define FCM_SCHED_TEAMS 2  /* slices from a queue, each on a team of 1..32 CTAs sized by its cost */
typedef struct {
    int block;      /* threads per CTA: 256 or 512                                   */
    int cluster;    /* FCM_SCHED_SLICES: CTAs per thread-block cluster, 1, 2, 4 or 8; */
                    /* FCM_SCHED_ROUNDS: 1                                            */
    int64_t big;    /* FCM_SCHED_SLICES: slices with n >= big are shared by a whole  */
                    /* cluster; FCM_SCHED_ROUNDS: unused (0)                          */
    double ms;      /* measured batch time when the autotuner chose it, or 0          */
    int schedule;   /* FCM_SCHED_SLICES, FCM_SCHED_ROUNDS or FCM_SCHED_TEAMS          */
    int tile;       /* FCM_SCHED_ROUNDS: fewest pixels one CTA takes in a round,      */
                    /* 1024 to 65536, a multiple of 1024. FCM_SCHED_SLICES: 0 for one */
                    /* launch, or an iteration cap: slices not stopped after `tile`  */
                    /* iterations are parked and finished by a second launch that    */
                    /* gives big slices clusters of 8 (in the same graph).           */
                    /* FCM_SCHED_TEAMS: 10..10000, the team-size target in percent   */
                    /* of the mean cost per CTA (see fcm_run_batched)                */
} fcm_batch_plan;

/* Batch options (bit flags). */
#define FCM_BATCH_RETUNE 16  /* run the autotuner even if a plan is cached        */
#define FCM_BATCH_NO_TUNE 32 /* use the cached or default plan, never tune        */
#define FCM_BATCH_NO_GRAPH 64 /* launch directly instead of replaying a CUDA graph */
#define FCM_BATCH_PRESOLVE 128 /* unless every slice has an iters_hint: first run each slice
                                  on its grey-level histogram from its own start and order
                                  the queue (and size teams) by the iterations that took,
                                  within the call (the structs' iters_hint are not
                                  written); the pixel runs and their results are the same */

/*
 * fcm_run_batched — Algorithm 1 on each of n_slices slices, in one persistent
 * launch captured in a CUDA graph. Memberships U^{k-1} are recomputed from
 * V^{k-1} rather than stored, so each iteration reads only x; U^k is written
 * once, after the last iteration. Two schedules:
 *
 *   FCM_SCHED_SLICES  slices are taken from a work queue in order of
 *                     decreasing size; slices with n >= plan.big are shared by
 *                     the CTAs of a thread-block cluster (per-iteration sums
 *                     exchanged through distributed shared memory), smaller
 *                     ones run one per CTA. With plan.tile > 0 the batch runs
 *                     in two phases: slices still running after plan.tile
 *                     iterations are parked and resumed by a second launch
 *                     with bigger clusters, so the few slowly converging
 *                     slices do not hold a few SMs while the rest idle.
 *   FCM_SCHED_TEAMS   a cooperative launch without clusters; a slice's cost
 *                     is n * (iters_hint + 3) when every slice has a hint,
 *                     else n. A slice gets a team of T CTAs, T the smallest
 *                     power of two with cost / T <= (plan.tile / 100) * (total
 *                     cost / CTAs), at most 32 and at most one CTA per 4,096
 *                     pixels; the T seats of a slice sit together in a queue
 *                     ordered by cost / T, longest first. A team exchanges
 *                     its sums after every pass through global memory, behind
 *                     a bounded barrier of its own. So the costliest slices,
 *                     which otherwise hold a few SMs while the rest idle,
 *                     spread over as many SMs as their cost asks for.
 *   FCM_SCHED_ROUNDS  a cooperative launch; round k is iteration k of every
 *                     slice still running, the pixels of those slices cut
 *                     into one equal contiguous chunk per CTA (at least
 *                     plan.tile pixels), with a grid barrier between rounds.
 *                     Slices that need many iterations then use the whole GPU
 *                     instead of a few SMs. At most 8192 slices.
 *
 * The launch shape comes from an autotuner: on the first batch of a new
 * "bucket" (device, set of C values, and the powers of two of the slice
 * count, total pixels and largest slice), it times each candidate shape of
 * both schedules on the batch itself and keeps the fastest, in memory and,
 * when the environment variable FCM_AUTOTUNE_CACHE names a file, in that JSON
 * file. Tuning runs the batch several times, so it is skipped (default plan)
 * when a slice updates its initial memberships in place (FCM_INIT_U with U0
 * NULL or equal to U).
 *
 * Returns FCM_OK if every slice converged, FCM_NOT_CONVERGED if some slice
 * stopped at max_iter, the first negative status of a failed slice, or an
 * error of the whole call (FCM_ERR_INVALID_ARG names no slice then). Per-slice
 * results are in the structs. A slice whose run was cut short by a bounded
 * wait of the round schedule giving up reports FCM_ERR_TIMEOUT.
 */
int fcm_run_batched(fcm_handle h, fcm_slice* slices, int n_slices, int options);

/*
 * fcm_run_batched_hist — the histogram-domain run (as fcm_run_hist: the
 * grey-level reduction of brFCM, cited in Sec. 3) for each slice of a batch
 * of 8-bit slices. The pixel passes are cut into chunks of 8,192 pixels,
 * one CTA each, over the whole GPU; the iterations run on each slice's 256
 * bins, one CTA per slice. A first pass builds every slice's histogram (and
 * from U^0 the sums of V^1); the first stopping quantity max_i |f(x_i, V^1)
 * - U^0_i| is bounded from below by one recorded pixel per grey level, and a
 * second pass over the pixels takes it exactly only when that bound does not
 * already exceed eps (or max_iter is 1); Algorithm 1 then iterates on the
 * bins, and a last pass writes U^k by table lookup. The iterates equal
 * fcm_run_batched's up to the order of rounding.
 *
 * Slices as for fcm_run_batched (device x, U0, U and V; x 16-byte aligned),
 * with n < 2^31. A slice whose x holds anything but integer grey levels
 * 0..255, or whose U^0 has a negative or non-finite value, or whose V^0 a
 * non-finite one, gets FCM_ERR_BAD_INPUT and V = V^0 (0 from a U^0); its U
 * is not written. Returns as fcm_run_batched.
 */
int fcm_run_batched_hist(fcm_handle h, fcm_slice* slices, int n_slices);

/* The plan the last batched run used. */
int fcm_batched_plan(fcm_handle h, fcm_batch_plan* plan);

/* Force a plan for later batched runs (NULL returns to the autotuner). */
int fcm_batched_set_plan(fcm_handle h, const fcm_batch_plan* plan);

/*
 * Learned warm start (not in the paper, which starts from random memberships,
 * Algorithm 1 step 2). A small network maps a slice's grey-level histogram to
 * initial centers V^0:
 *   f  = [histogram / n over 256 bins of round(clip(x, 0, 255)), onehot(C)]
 *                                                     (264 values, FP32)
 *   a1 = GELU(W1 f + b1) (128), a2 = GELU(W2 a1 + b2) (128), y = W3 a2 + b3 (8)
 *   V^0 = sort(255 * y[0..C-1])
 * Weights are W[out, in], kept as FP32 master copies and used in BF16;
 * accumulation, activations, gradients and Adam state are FP32. Training
 * minimises the masked mean squared error sum_{b, j<C_b} (y_bj - t_bj)^2 /
 * sum_b C_b against t = (sorted converged centers of plain FCM) / 255.
 * Parameters, as one FP32 vector, in the order W1, b1, W2, b2, W3, b3.
 * Device arrays: features [B, 264] row-major, targets [B, 8], C [B] (int).
 */
#define FCM_MODEL_PARAMS 51464

/* Initialise the network (He-normal weights from a splitmix64 stream seeded
 * with `seed`, zero hidden biases, output biases (j+1)/9). */
int fcm_model_init(fcm_handle h, uint64_t seed);
/* Set / read the FP32 parameters (host arrays of FCM_MODEL_PARAMS floats);
 * setting resets the optimiser state. */
int fcm_model_set_params(fcm_handle h, const float* params, int64_t count);
int fcm_model_get_params(fcm_handle h, float* params, int64_t count);
/* Save / load the parameters as a small binary file. */
int fcm_model_save(fcm_handle h, const char* path);
int fcm_model_load(fcm_handle h, const char* path);
/* Network input of each slice (x and C of the structs are used) into device
 * features [n, 264]. */
int fcm_features(fcm_handle h, const fcm_slice* slices, int n, float* feats);
/* Outputs y [B, 8] (device) of B feature rows (device). */
int fcm_model_forward(fcm_handle h, const float* feats, int B, float* out);
/* Loss and gradient (host arrays: loss[1], grad[FCM_MODEL_PARAMS]) of B rows,
 * without updating the parameters. */
int fcm_model_loss_grad(fcm_handle h, const float* feats, const float* targets, const int* C, int B,
                        float* grad, float* loss);
/* Adam (lr, beta 0.9 / 0.999, eps 1e-8) over `epochs` passes of shuffled
 * full mini-batches of `batch` rows of the n training rows (device arrays),
 * all on the GPU; *last_loss (nullable) receives the last epoch's mean loss. */
int fcm_model_train(fcm_handle h, const float* feats, const float* targets, const int* C, int n,
                    int epochs, int batch, float lr, uint64_t seed, float* last_loss);
/* Predicted V^0 of every slice into slices[i].V0, with init_mode set to
 * FCM_INIT_V. */
int fcm_predict_centers(fcm_handle h, fcm_slice* slices, int n);
/*
 * fcm_run_batched_warm — a batch in which plain cold-start FCM (Algorithm 1
 * from the slice's own U^0, Sec. 2.1) is both the judge and the fallback of
 * the learned warm start. Every slice must give its own U0 (not NULL, not U).
 *
 *   1. The network predicts V^0 of every slice.
 *   2. The judge runs every 8-bit slice twice on its grey-level histogram
 *      (the brFCM reduction cited in Sec. 3, which gives the per-pixel
 *      iterates up to rounding): from U^0, and from the predicted V^0.
 *   3. A slice starts from V^0 when the prediction is usable (finite, no two
 *      centers within 1e-3) and the warm fixed point passes the acceptance
 *      rule against the cold one: sorted centers within 1e-4 relative
 *      (to max(|v|, 1)), or a final J no larger (relative slack 1e-5). Every
 *      other slice, and every slice that is not all grey levels 0..255, starts
 *      from its U^0. Each slice's iters_hint is set to the iterations its
 *      start took on the histogram, so the batch is ordered by cost.
 *   4. fcm_run_batched runs the batch.
 *   5. Each warm result is checked against the judge's cold fixed point by
 *      the same rule (and must have converged without emptying a cluster);
 *      a slice that fails is run again from its U^0 within the call.
 *
 * On return slices[i].init_mode is FCM_INIT_V for a slice whose result came
 * from the warm start and FCM_INIT_U for one that ran cold; *n_cold
 * (nullable) counts the latter. Returns as fcm_run_batched.
 */
int fcm_run_batched_warm(fcm_handle h, fcm_slice* slices, int n, int options, int* n_cold);

/*
 * fcm_time_pass — profiling aid: time `launches` back-to-back launches of the
 * iteration pass (one Algorithm 1 iteration each: Eq. 4, Eq. 1, Eq. 3) on the
 * handle's stream with CUDA events, starting from centers V (device or host,
 * C floats) and updating U (device, C*n floats, cluster-major) in place; the
 * stopping test is disabled. x is n device floats. Writes the average
 * milliseconds per launch and returns FCM_OK or an error. The same launch
 * configuration as fcm_run is used (options: FCM_OPT_NO_TMA).
 */
int fcm_time_pass(fcm_handle h, const float* x, int64_t n, int C, float m, float* U,
                  const float* V, int launches, int options, float* ms_per_launch);

/*
 * fcm_run_noalloc — the same run as fcm_run for aligned inputs, for callers
 * that must not allocate memory while they run. The paper has no counterpart;
 * this is a deployment variant of the library's own whole-run kernel.
 *
 * Some callers cannot call cudaMalloc: code whose device memory is owned by a
 * pool or framework allocator it may not bypass, plugins that receive only
 * pre-allocated buffers, and latency-critical services where an allocation
 * (which may synchronise the device or fail under memory pressure) is not
 * acceptable. fcm_run keeps its scratch in a handle that allocates on first
 * use; this entry point needs no handle and allocates nothing (no cudaMalloc,
 * cudaFree or allocating library call). Its scratch — the device-side run
 * state and the per-block partial sums — lives in one fixed array inside the
 * library image (about 80 KB plus the state) that every GPU which loads the
 * library holds until the process exits.
 *
 *   x, n, C, m, eps, max_iter, init_mode, U0, U, V: as for fcm_run, except
 *             that x, U and U0 must be device memory, 16-byte aligned, and
 *             n % 4 == 0 (host memory cannot be staged without allocating).
 *             V may be device or host memory.
 *   cuda_stream  the cudaStream_t to run on (NULL = legacy default stream),
 *             on the current device. The call synchronises that stream.
 *   rep       nullable; filled on return.
 *
 * Limit: the scratch holds partial sums for at most FCM_NOALLOC_MAX_BLOCKS
 * thread blocks; a device that would need more (more SMs than any current
 * GPU) gets FCM_ERR_TOO_LARGE. Other bad arguments give FCM_ERR_INVALID_ARG.
 *
 * The first call on each device looks up the scratch address and the kernels'
 * launch limits on that device; make that first call before capturing any
 * stream into a CUDA graph. Every call copies its run state through host
 * memory and synchronises its stream, so a stream that is being captured is
 * refused with FCM_ERR_INVALID_ARG. Every call shares the one scratch array
 * and resets it as needed, so calls must not overlap on the GPU: calls from
 * several host threads, or on streams not ordered with one another, race.
 */
#define FCM_NOALLOC_MAX_BLOCKS 512
int fcm_run_noalloc(const float* x, int64_t n, int C, float m, float eps, int max_iter,
                    int init_mode, const float* U0, float* U, float* V, void* cuda_stream,
                    fcm_report* rep);

/* Copy the trace of the last run made with FCM_OPT_TRACE into host arrays
 * (each nullable): delta[k-1], J[k-1] and V[(k-1)*C + j] for k = 1..iters.
 * `cap` is the number of iterations the arrays hold. Returns the number of
 * iterations copied, or a negative error. */
int fcm_get_trace(fcm_handle h, double* delta, double* J, double* V, int cap);

/* Text of the last error recorded on the handle ("" if none). */
const char* fcm_last_error(fcm_handle h);

/* Name of a status code (static string). */
const char* fcm_status_string(int status);

/* Library version as "major.minor.patch" (static string). */
const char* fcm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FCM_GB300_H */
