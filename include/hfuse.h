/*
 * hfuse.h -- C ABI of the GB300 horizontal-fusion runtime.
 *
 * Horizontal fusion (Sec. 1.1, Sec. 2.2 of "Automatic Horizontal Fusion for
 * GPU Kernels", Li, Zheng, Pekhimenko, Long, arXiv 2007.01277) runs two or
 * more independent kernels as ONE launch: each thread block of d0 threads is
 * cut into warp-aligned thread intervals, a thread-index branch sends every
 * interval to one original kernel's body (Algorithm 1, Sec. 3.1), each body's
 * block barrier becomes a named barrier "bar.sync id, d_k" over its own
 * interval only, and the fused kernel's shared memory is the sum of the
 * bodies' (Sec. 2.3).  The thread split and a register bound are chosen by
 * profiling (Algorithm 2, Sec. 3.2).
 *
 * The built-in kernels are hand-written "bodies" that already address
 * threads through an interval context, so one body serves a standalone
 * launch and any fused interval.  A fused instance is a compiled kernel per
 * (body A, body B, register cap); split, block size, grid and barrier ids
 * are launch-time values.  Separately, the hf_src_* entry points apply
 * Algorithm 1 to CUDA source text and compile the result at run time.
 *
 * Conventions for every entry point:
 *   - Pointers named d_* or held in argument blocks are DEVICE pointers the
 *     caller allocates and owns; the library never frees them.  Handles
 *     (hf_kernel, hf_fused) are owned by the library until destroyed.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy stream).
 *     Launches are asynchronous; argument blocks are copied at launch, so
 *     the caller may reuse them as soon as the call returns.
 *   - Every function returns an hf_status; no exception or abort crosses the
 *     boundary.  On error nothing is launched and hf_last_error() gives a
 *     one-line reason.  All validation happens on the host before a launch.
 *   - One device: the device current on the calling thread when a handle is
 *     created is the device it launches on.
 */
#ifndef HFUSE_H
#define HFUSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HF_ABI_VERSION 1
#define HF_MAX_INTERVALS 15   /* named barrier ids 1..15; id 0 stays the block barrier */
#define HF_MAX_SCHEDULE 16    /* kernels per N-way fused launch                     */
#define HF_POLY_NCOEF 33      /* degree-32 polynomial                                */

typedef enum {
    HF_OK = 0,
    HF_ERR_INVALID = -1,      /* bad argument, null pointer, bad size or alignment  */
    HF_ERR_SPLIT = -2,        /* thread split not warp aligned / out of range       */
    HF_ERR_BARRIER = -3,      /* more intervals with barriers than named ids        */
    HF_ERR_SMEM = -4,         /* combined shared memory above the per-block limit   */
    HF_ERR_REGS = -5,         /* block too large for the instance's register use    */
    HF_ERR_UNSUPPORTED = -6,  /* register cap or body combination not compiled      */
    HF_ERR_CUDA = -7,         /* a CUDA runtime call failed (message has the name)  */
    HF_ERR_TIMEOUT = -8       /* a bounded wait expired                             */
} hf_status;

/* Built-in constituent bodies. */
typedef enum {
    HF_BODY_BN_STATS = 0,     /* batch-norm mean / biased variance (Sec. 2.3)        */
    HF_BODY_UPSAMPLE2X = 1,   /* bilinear x2, half-pixel centres (Sec. 4.1)          */
    HF_BODY_MAXPOOL3S2 = 2,   /* 3x3 max pool, stride 2, pad 1 (Sec. 4.1)            */
    HF_BODY_IM2COL3 = 3,      /* 3x3 im2col, stride 1, pad 1 (Sec. 4.1)              */
    HF_BODY_HIST256 = 4,      /* 256-bin byte histogram, shared atomics (Sec. 2.3)   */
    HF_BODY_PHILOX = 5,       /* Philox4x32-10 stream                                */
    HF_BODY_POLY = 6,         /* repeated degree-32 Horner chain                     */
    HF_BODY_BF16_AXPY = 7,    /* out = bf16(alpha*x + y)                             */
    HF_BODY_STREAM_TMPL = 8,  /* parametric stream kernel (cost-model corpus)        */
    HF_BODY_SHA256D = 9,      /* double SHA-256 nonce scan (Sec. 4.1 "SHA256")       */
    HF_BODY_BLAKE256 = 10,    /* BLAKE-256, 14 rounds, nonce scan ("Blake256")       */
    HF_BODY_BLAKE2B = 11,     /* BLAKE2b-256 nonce scan ("Blake2B")                  */
    HF_BODY_COUNT = 12
} hf_body_id;

/* ------------------------------------------------------------------ */
/* Argument blocks, one per body.  All tensors are dense, row-major.   */

/* Per-channel statistics of x[N][C][HW] (float32): mean[c] and the biased
 * variance var[c] over the N*HW values of channel c.  `workspace` is
 * device scratch of hf_workspace_size() bytes (16-byte aligned): C tile
 * counters, then one partial-sum pair per 2048-value tile.  Zero-fill it
 * once before its first use; every completed launch leaves the counters at
 * zero again (the partial sums are written before they are read), so one
 * workspace serves any number of launches on one stream (launches that
 * overlap in time need separate workspaces).  Requires HW % 4 == 0 and x
 * 16-byte aligned for the vector path; other shapes use a scalar path. */
typedef struct {
    const float *x;
    float *mean;
    float *var;
    int N, C, HW;
    void *workspace;
} hf_bn_stats_args;

/* y[P][2H][2W] = bilinear x2 upsampling of x[P][H][W], align_corners=false
 * (source coordinate max(0, (o + 0.5)/2 - 0.5), clamped neighbours). */
typedef struct {
    const float *x;
    float *y;
    int P, H, W;
} hf_upsample2x_args;

/* y[P][Ho][Wo] = 3x3 max over the in-bounds window at (2*oy-1, 2*ox-1),
 * Ho = (H-1)/2 + 1, Wo = (W-1)/2 + 1. */
typedef struct {
    const float *x;
    float *y;
    int P, H, W;
} hf_maxpool3s2_args;

/* col[n][c*9 + ky*3 + kx][oy*W + ox] = x[n][c][oy+ky-1][ox+kx-1] or 0. */
typedef struct {
    const float *x;
    float *col;
    int N, C, H, W;
} hf_im2col3_args;

/* bins[v] += number of bytes equal to v in x[0..n).  The body ADDS into
 * bins (as the paper's histogram kernel does into a zeroed output): the
 * caller zero-fills bins before the launch. */
typedef struct {
    const uint8_t *x;
    uint32_t *bins;
    int64_t n;
} hf_hist256_args;

/* out[i][0..3] = Philox4x32-10 block for counter (lo32(first+i),
 * hi32(first+i), 0, 0) under key (lo32(seed), hi32(seed)), i < n. */
typedef struct {
    uint32_t *out;
    int64_t n;
    uint64_t seed;
    uint64_t first;
} hf_philox_args;

/* y[i] = acc_iters(x[i]) with acc_0 = 0 and, per step,
 * h = acc; for k = 32..0: h = fma(h, x, coef[k]); acc = h.
 * Coefficients travel by value in the argument block. */
typedef struct {
    const float *x;
    float *y;
    int64_t n;
    int iters;
    float coef[HF_POLY_NCOEF];
} hf_poly_args;

/* out[i] = bf16_rne(alpha * x[i] + y[i]); x, y, out hold bfloat16 bits. */
typedef struct {
    const uint16_t *x;
    const uint16_t *y;
    uint16_t *out;
    int64_t n;
    float alpha;
} hf_bf16_axpy_args;

/* Parametric stream kernel: for each 16-byte group of x (n floats, n % 4 ==
 * 0, 16-byte aligned) apply k multiply-adds v = v*a + b, the j-th to
 * component j % 4, and store the group to y.  Each tile of the loop stages
 * through `smem_bytes` of shared memory (0..49152, multiple of 16) and
 * passes `n_barriers` (0..4) interval barriers; neither changes the values. */
typedef struct {
    const float *x;
    float *y;
    int64_t n;
    int k;
    int n_barriers;
    int smem_bytes;
    float a, b;
} hf_stream_tmpl_args;

/* Nonce scan of an 80-byte block header, the work of the compute-bound hash
 * kernels of Sec. 4.1 (a miner hashes one header again and again with a
 * different nonce).  Item i (0 <= i < n) hashes `header` with bytes 76..79
 * replaced by the nonce (first + i) mod 2^32 as a little-endian uint32:
 *   HF_BODY_SHA256D   SHA-256(SHA-256(header))          (FIPS 180-4)
 *   HF_BODY_BLAKE256  BLAKE-256, 14 rounds, salt 0      (the SHA-3 finalist)
 *   HF_BODY_BLAKE2B   unkeyed BLAKE2b, 32-byte digest   (RFC 7693)
 * each giving a 32-byte digest in the function's own byte order.
 * digests: NULL, or [n][32] bytes (16-byte aligned) that receive every
 * digest.  An item hits when digest bytes 28..31, read as a little-endian
 * uint32, are <= target; each hit increments *hit_count (if hit_count is
 * not NULL) and, while the old count is below hit_cap, stores its nonce at
 * hits[old count] -- so the stored hits are in no particular order, and
 * *hit_count ends as the total number of hits even past hit_cap.  The
 * caller zeroes *hit_count.  HF_ERR_INVALID: n < 0 or n > 2^32, unaligned
 * digests, hit_cap < 0, or hit_cap > 0 without hits and hit_count. */
typedef struct {
    uint8_t header[80];
    uint32_t first;
    uint32_t target;
    int64_t n;
    uint8_t *digests;
    uint32_t *hits;
    uint32_t *hit_count;
    int32_t hit_cap;
} hf_hash_scan_args;

/* ------------------------------------------------------------------ */
/* Kernels and fused kernels.                                          */

typedef struct hf_kernel_t *hf_kernel;
typedef struct hf_fused_t *hf_fused;

/* A registered kernel: one built-in body plus the interval sizes it may run
 * with (the tunable block dimension of Sec. 2.1).  0 selects the default:
 * min 32, max 1024, granularity 32.  Sizes must be multiples of 32. */
typedef struct {
    const char *name;
    int body_id;
    int min_threads;
    int max_threads;
    int thread_granularity;
} hf_kernel_desc;

/* Register a kernel.  HF_ERR_INVALID for an unknown body or sizes that are
 * not multiples of 32 / not ordered. */
hf_status hf_register_kernel(const hf_kernel_desc *desc, hf_kernel *out);
void hf_destroy_kernel(hf_kernel k);

/* Fuse two kernels (Algorithm 1, Sec. 3.1): a block of d0 threads whose
 * threads [0, split) run kernel a with "bar.sync 1, split" and threads
 * [split, d0) run kernel b with "bar.sync 2, d0 - split".  regcap = 0 for no
 * register bound, else one of hf_regcaps().  Errors: HF_ERR_SPLIT when split
 * is not a multiple of 32 with 0 < split < d0 <= 1024 or violates a kernel's
 * thread range; HF_ERR_UNSUPPORTED for an uncompiled register cap. */
hf_status hf_fuse(hf_kernel a, hf_kernel b, int split, int d0, int regcap,
                  hf_fused *out);

/* hf_fuse without a register bound, from the checked build: the same two
 * bodies in the same block layout, but every interval barrier (the
 * "bar.sync id, d_k" that Sec. 3.1 puts in place of __syncthreads) is a
 * software barrier over the interval's warps whose wait gives up after one
 * second, setting bit 2 (value 2, a software barrier gave up) of the device
 * error word (hf_check_device_error) instead of stalling the warps for good.  Use it to
 * check a barrier schedule on the device without the risk of a hang; the
 * results equal hf_fuse's.  Compiled for the pairs whose bodies have
 * barriers: histogram + Philox, batch-norm + histogram, batch-norm +
 * polynomial and stream template + stream template (either order);
 * HF_ERR_UNSUPPORTED for any other pair.  Launch, query and destroy as any
 * fused handle. */
hf_status hf_fuse_checked(hf_kernel a, hf_kernel b, int split, int d0, hf_fused *out);

/* N-way fusion into one persistent kernel.  n kernels ks[0..n) are placed on
 * n_intervals intervals of interval_threads[i] threads each (block size =
 * their sum); kernel j runs on interval interval_of[j], and kernels sharing
 * an interval run one after another in index order.  Interval i uses named
 * barrier i + 1.  n <= HF_MAX_SCHEDULE, n_intervals <= HF_MAX_INTERVALS. */
hf_status hf_fuse_n(const hf_kernel *ks, int n, const int *interval_of,
                    const int *interval_threads, int n_intervals, int regcap,
                    hf_fused *out);
void hf_destroy_fused(hf_fused f);

/* Launch a fused kernel: args[j] points to the argument block of kernel j
 * (the type its body id names).  grid = number of blocks; 0 picks
 * blocks_per_sm * SM count, where blocks_per_sm is the occupancy limit of
 * the instance at this block size and shared memory.  The bodies stride over
 * the grid, so any grid >= 1 computes the full result. */
hf_status hf_launch(hf_fused f, const void *const *args, int grid, void *stream);

/* hf_launch of an N-way fused kernel that also records, per interval i,
 * the earliest start and latest end (global nanosecond timer) over all its
 * warps: trace (device, 2 * n_intervals unsigned 64-bit values) must hold
 * (UINT64_MAX, 0) per interval before the launch.  Used to balance interval
 * sizes; HF_ERR_UNSUPPORTED for a 2-way pair instance. */
hf_status hf_launch_traced(hf_fused f, const void *const *args, int grid, void *stream,
                           unsigned long long *trace);

/* Launch one kernel alone with `threads` threads per block (the unfused
 * baseline, Sec. 4.1).  Same argument block as in a fused launch; a body run
 * alone on d threads and grid g computes bit-identical results to the same
 * body on a d-thread interval of a fused launch with grid g. */
hf_status hf_launch_single(hf_kernel k, const void *args, int threads, int grid,
                           void *stream);

/* Resource use of a fused instance at its block size (Sec. 2.1, Sec. 4.3):
 * registers per thread, spill bytes (local memory per thread), combined
 * dynamic shared memory for `args`, and resident blocks per SM. */
typedef struct {
    int regs;
    int spill_bytes;
    int smem_bytes;
    int block_threads;
    int blocks_per_sm;
    int max_threads_per_block;
    int n_intervals;
} hf_fused_info;

hf_status hf_query(hf_fused f, const void *const *args, hf_fused_info *info);

/* The same figures for a kernel launched alone with `threads` threads. */
hf_status hf_query_single(hf_kernel k, const void *args, int threads,
                          hf_fused_info *info);

/* Scratch bytes a body needs for this argument block (0 for most bodies). */
hf_status hf_workspace_size(int body_id, const void *args, size_t *bytes);

/* The register caps that have compiled fused instances (ascending; the list
 * excludes 0, which is always available).  Writes at most cap entries and
 * returns the count. */
int hf_regcaps(int *caps, int cap);

/* Device limits used by the occupancy rule of Sec. 2.1 and the register
 * bound of Algorithm 2: registers, shared memory and threads per SM, SM
 * count, per-block opt-in shared memory and L2 bytes of the current device. */
typedef struct {
    int sm_count;
    int regs_per_sm;
    int smem_per_sm;
    int threads_per_sm;
    int smem_per_block_optin;
    int l2_bytes;
    int cc_major, cc_minor;
} hf_device_limits;

hf_status hf_device_info(hf_device_limits *lim);

/* Register bound r0 of Algorithm 2 (Sec. 3.2) for a split d1 / d2 given the
 * standalone kernels' registers per thread and the fused shared memory,
 * using the limits in lim.  Writes 0 when the fused block cannot be
 * resident.  Host arithmetic only. */
hf_status hf_register_bound(const hf_device_limits *lim, int d1, int nregs1,
                            int d2, int nregs2, int smem_fused, int *r0);

/* ------------------------------------------------------------------ */
/* Profiling search (Sec. 3.2).                                         */

/* One timed configuration.  status is HF_OK when time_us is valid. */
typedef struct {
    int split;          /* threads of the first kernel (d1)            */
    int regcap;         /* register bound, 0 = none                    */
    int blocks_per_sm;  /* grid = blocks_per_sm * SM count             */
    int grid;
    float time_us;      /* median over reps                            */
    float p10_us, p90_us;
    int regs, spill_bytes;
    int status;
} hf_tune_point;

/* Time a fused (or a single) launch on `stream` with CUDA events: two
 * warm-up launches, then `reps` timed launches, each preceded by a write of
 * a buffer twice the L2 size when flush_l2 != 0 (the buffer is allocated by
 * the library on first use and kept).  Median and 10th/90th percentile in
 * microseconds; outputs may be NULL.  Synchronises the stream. */
hf_status hf_time_fused(hf_fused f, const void *const *args, int grid, int reps, int flush_l2,
                        void *stream, float *median_us, float *p10_us, float *p90_us);
hf_status hf_time_single(hf_kernel k, const void *args, int threads, int grid, int reps,
                         int flush_l2, void *stream, float *median_us, float *p10_us,
                         float *p90_us);

/* Exhaustive profile of kernels a and b fused in a d0-thread block over
 * every (split, regcap, blocks_per_sm) of the given lists; table receives
 * n_splits * n_regcaps * n_bps points in that nesting order.  Points that
 * cannot be built or are not resident carry a non-OK status and time -1.
 * Note: kernels that accumulate into their outputs (the histogram) run
 * (reps + 2) times per point. */
hf_status hf_profile_pair(hf_kernel a, hf_kernel b, const void *const *args, int d0,
                          const int *splits, int n_splits, const int *regcaps, int n_regcaps,
                          const int *bps, int n_bps, int reps, int flush_l2, void *stream,
                          hf_tune_point *table);

/* Algorithm 2 (Sec. 3.2): for d1 = step, 2*step, ... < d0 profile the fused
 * kernel without a register bound and with the bound r0 of
 * hf_register_bound (NRegs from the kernels compiled alone at d1 and
 * d0 - d1, ShMem from the fused instance), r0 snapped down to the nearest
 * compiled cap; keep the first strictly fastest.  Grid = resident blocks per
 * SM * SM count.  The visited points go to trace (up to trace_cap). */
hf_status hf_search_alg2(hf_kernel a, hf_kernel b, const void *const *args, int d0, int step,
                         int reps, int flush_l2, void *stream, hf_tune_point *best,
                         hf_tune_point *trace, int trace_cap, int *n_trace);

/* One call that tunes a pair for a d0-thread block and returns the point
 * to launch: mode HF_TUNE_EXHAUSTIVE profiles every split in warp steps
 * (32 .. d0 - 32, within both kernels' thread ranges) x every compiled
 * register cap and "none" x 1..4 blocks per SM and takes the fastest;
 * mode HF_TUNE_ALG2 runs hf_search_alg2 with step 128 (64 for d0 < 512);
 * mode HF_TUNE_MODEL replaces Algorithm 2's profiling loop with the learned
 * cost model installed by hf_cost_model_set: the same candidates as the
 * exhaustive mode are built and queried (no launch), their features
 * (hf_pair_features) scored in one hf_mlp_forward launch, and only the
 * model's best at each blocks/SM and its `confirm` best with distinct
 * (split, blocks/SM) are timed, then
 * the untimed neighbours of the fastest so far (its split with another
 * blocks/SM or register cap, the splits one warp either side), again while
 * that finds a faster one (at most three rounds); the fastest measured
 * point is returned (HF_ERR_INVALID when no model is installed).
 * Timing as hf_time_fused (reps launches, L2 flushed when flush_l2).
 * HF_ERR_INVALID for an unknown mode or when no point can be launched. */
enum { HF_TUNE_EXHAUSTIVE = 0, HF_TUNE_ALG2 = 1, HF_TUNE_MODEL = 2 };
hf_status hf_autotune(hf_kernel a, hf_kernel b, const void *const *args, int d0, int mode, int reps,
                      int flush_l2, void *stream, hf_tune_point *best);

/* hf_autotune in HF_TUNE_MODEL mode that also reports how many candidates
 * it timed (*n_timed, may be NULL): the model's `confirm` best plus the
 * neighbour steps -- against every candidate for the exhaustive search. */
hf_status hf_autotune_model(hf_kernel a, hf_kernel b, const void *const *args, int d0, int reps,
                            int flush_l2, void *stream, hf_tune_point *best, int *n_timed);

/* ------------------------------------------------------------------ */
/* Allocation-free batch-norm statistics.                               */

/* Size of the fixed device scratch array behind hf_bn_stats_noalloc: room
 * for the per-channel counters (4 bytes each, rounded up to 256 bytes) and
 * one 8-byte partial sum per 2048-value tile of every channel, i.e. up to
 * about 129,000 tiles (264 million input values) at C <= 4096. */
#define HF_BN_NOALLOC_SCRATCH_BYTES (1 << 20)

/* Batch-norm statistics (same result as HF_BODY_BN_STATS launched alone with
 * the same threads and grid) that allocates no device memory.  It is meant
 * for callers that must not call cudaMalloc: hosts whose device memory is
 * fully reserved up front, or latency-bound loops where an allocation would
 * stall every stream.  It has no counterpart in the paper.
 *
 * Instead of a caller workspace it uses one file-scope device array of
 * HF_BN_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library holds
 * until the process exits.  The first call on a device looks up that
 * array's device address (once, with the device current); make that first
 * call before any stream capture.  The address is kept for the life of the
 * process, so the library must not be used across a reset of the device's
 * context (cudaDeviceReset): later calls would use a stale address.  (The
 * device error word of hf_check_device_error is looked up the same way.)
 * Every call clears the counters at the
 * start of the array on `stream` and then launches; calls share the one
 * array, so calls whose work overlaps on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  Shapes whose scratch
 * would exceed the array are rejected with HF_ERR_INVALID before anything
 * is queued.  grid = 0 picks resident blocks per SM times the SM count.
 * x is float32 [N][C][HW]; mean and var receive C floats. */
hf_status hf_bn_stats_noalloc(const float *x, float *mean, float *var, int N, int C, int HW,
                              int threads, int grid, void *stream);

/* A schedule for N-way fusion: kernel j runs on interval interval_of[j];
 * interval i has interval_threads[i] threads; plus the register cap, the
 * grid and the measured time of the plan. */
typedef struct {
    int n_intervals;
    int interval_of[HF_MAX_SCHEDULE];
    int interval_threads[HF_MAX_INTERVALS];
    int regcap;
    int grid;
    float time_us;
    int evals;
} hf_nway_plan;

/* Autotuner for N-way fusion (an extension: the paper fuses pairs and
 * searches their split and register bound with Algorithm 2, Sec. 3.2; the
 * plan here also assigns several kernels to an interval).  Times every
 * kernel alone (256 threads), then
 * packs kernels onto intervals longest-first (LPT: each goes to the least
 * loaded interval), gives each interval warps in proportion to its load, and
 * times these plans for block sizes 512, 768 and 1024, register caps
 * none/40/48/64/96, and one interval per kernel or about two kernels per
 * interval; the packed plans also once more with warps in proportion to each
 * interval's busiest-pipe time (from hf_body_work_of).  Each of
 * the twelve fastest is rebalanced up to six times from a traced launch
 * (hf_launch_traced), giving interval i warps in proportion to its warps
 * times its finishing time while that helps; from each of the five
 * fastest plans seen it then searches locally -- move one or two warps
 * between two intervals, move one kernel to another interval, swap two
 * kernels of different intervals, change the register cap -- taking the
 * best neighbour while the measured time drops by more than 0.5%; the
 * budget left after that goes to restarts (at most 512), each from a few
 * random moves (or three or four warps shifted) away from, in turn, one of
 * the three fastest plans so far, the fastest plan of one block size and
 * register cap (the families in turn, so that one that started behind is
 * still refined), or one of the packing seeds, and each followed by a
 * first-improvement local search over the same moves in random order (a
 * fixed-seed generator, so the search depends only on the measured
 * times).  Finally the ten fastest distinct plans are timed
 * again with 3 * reps launches and the fastest of those is returned.  The
 * seeds (at most 45) and the final timings are always done; max_evals
 * bounds the total including the seeds for the phases between.
 * standalone_us (n entries, may be NULL) receives the single-kernel times. */
hf_status hf_autotune_nway(const hf_kernel *ks, int n, const void *const *args, int max_evals,
                           int reps, int flush_l2, void *stream, hf_nway_plan *best,
                           float *standalone_us);

/* A plan's cost for hf_nway_search_sim: the time of `plan` (> 0; 0 or less
 * when the plan cannot run), and each interval's finishing time (relative
 * to the earliest start, any unit) in interval_finish[0 .. n_intervals). */
typedef float (*hf_plan_cost_fn)(const hf_nway_plan *plan, float *interval_finish, void *user);

/* The search of hf_autotune_nway (phases after the standalone timings) run
 * against a cost function instead of the GPU, so that the search itself can
 * be tested on the host: standalone_us[0..n) stand in for the kernels'
 * standalone times and issue_us[0..n) (may be NULL: no issue-weighted
 * seeds; else values >= 0) for their busiest-pipe times, and `cost` is
 * asked wherever hf_autotune_nway would time a plan, trace a launch or time
 * a finalist again.  best->evals counts the
 * plans asked for; best->grid is 0.  The library keeps nothing of `user`.
 * Returns HF_ERR_INVALID for bad arguments or when no plan has a cost.  No
 * counterpart in the paper: a test hook of the N-way extension above. */
hf_status hf_nway_search_sim(int n, const float *standalone_us, const float *issue_us, hf_plan_cost_fn cost,
                             void *user, int max_evals, hf_nway_plan *best);

/* ------------------------------------------------------------------ */
/* Source-level front-end: Algorithm 1 (Sec. 3.1) as a transformation of
 * CUDA source text (the paper's automatic tool, Sec. 3.3), compiled at run
 * time with NVRTC for the current device.  Kernels are 1-D: in each
 * kernel's body threadIdx.x becomes the interval's thread index, blockDim.x
 * its size, __syncthreads() "bar.sync id, d" (id 1 for kernel a, 2 for b),
 * and "extern __shared__ T name[]" a pointer to the kernel's slice of the
 * combined dynamic shared memory; blockIdx and gridDim are unchanged.
 * HF_ERR_UNSUPPORTED: threadIdx/blockDim .y/.z, __syncthreads_count/and/or,
 * kernel templates, these builtins in a __device__ helper, other forms of
 * extern __shared__; HF_ERR_INVALID: no such kernel, or NVRTC rejected the
 * source (hf_last_error() has the start of its log) or is not installed. */
typedef struct hf_src_module_t *hf_src_module;

/* The fused source: kernel name_a of src_a on threads [0, split), kernel
 * name_b of src_b (NULL: the same source) on [split, d0), as one
 * extern "C" __global__ kernel "hf_src_fused" whose parameters are a's, then
 * b's, then the byte offset of b's dynamic shared memory.  Written to
 * out[0..cap) NUL-terminated; *len = bytes needed including the NUL
 * (out may be NULL to query it).  Two different sources are concatenated,
 * so their file-scope names must not collide.  HF_ERR_SPLIT as hf_fuse. */
hf_status hf_src_fuse(const char *src_a, const char *name_a, const char *src_b, const char *name_b,
                      int split, int d0, char *out, size_t cap, size_t *len);

/* Compile a source with NVRTC (no GPU needed) and check that it defines
 * kernel `name`; the compiler log goes to log[0..cap) when log != NULL. */
hf_status hf_src_compile_check(const char *src, const char *name, int regcap, char *log, size_t cap);

/* Compile and load: one kernel of a source as it is (the standalone
 * launch), or the fused kernel of two (regcap = register bound, 0 none). */
hf_status hf_src_load(const char *src, const char *name, int regcap, hf_src_module *out);
hf_status hf_src_fuse_load(const char *src_a, const char *name_a, const char *src_b, const char *name_b,
                           int split, int d0, int regcap, hf_src_module *out);

/* Launch a single kernel: params[i] points at the value of parameter i
 * (the cuLaunchKernel convention); asynchronous on `stream`. */
hf_status hf_src_launch(hf_src_module m, void **params, int grid, int block, size_t dyn_smem,
                        void *stream);

/* Launch a fused module on `grid` blocks of d0 threads: params_a / params_b
 * as above for each kernel; each kernel gets its own dynamic shared memory
 * of the given size (b's slice starts 128-byte aligned after a's). */
hf_status hf_src_launch_fused(hf_src_module m, void **params_a, void **params_b, size_t dyn_smem_a,
                              size_t dyn_smem_b, int grid, void *stream);

/* Registers per thread, local (spill) bytes per thread, static shared
 * memory and the largest block of the loaded kernel. */
hf_status hf_src_query(hf_src_module m, int *regs, int *local_bytes, int *static_smem, int *max_threads);
void hf_src_unload(hf_src_module m);

/* The bulk-copy ring geometry the launch planner gives a block of n
 * intervals (warps[i] warps) at blocks_per_sm resident blocks.  ring[i] is
 * the kind of ring interval i's kernel takes: 0 none; 1 a stream ring --
 * whole tiles of a flat array, wanting at least min_bytes[i] in flight per
 * warp; 2 an item ring -- one work item (min_bytes[i] bytes) per stage.
 * Item rings get two stages of min_bytes[i] (rounded up to 128) per warp.
 * Stream rings share about 40 KB in flight per SM over their warps, in
 * stages of 1, 2 or 4 KB, 2 to 4 per warp; intervals whose minimum the
 * share misses fall back to register loads.  Per interval: stage[i] bytes,
 * stages[i] (0 when no ring) and uses[i].  When they do not fit in shared
 * memory the launch drops item rings, the largest first, before it lowers
 * the blocks per SM.  Host arithmetic only. */
hf_status hf_ring_plan(int n, const int *warps, const int *ring, const unsigned *min_bytes,
                       int blocks_per_sm, unsigned *stage, int *stages, int *uses);

/* Device-side failure detection.  Bodies that stage their input through
 * bulk asynchronous copies wait on them with a time limit (about 2 s); on
 * expiry the kernel sets a bit in a per-device error word (1 = a bounded
 * wait on bulk copies expired, 2 = a bounded software barrier expired),
 * waits (bounded) for its copies in flight and stops consuming, so the
 * context stays usable and the host can detect it.
 * hf_check_device_error reads the word after the launches have finished
 * (synchronize the streams first) and clears it when `clear` is set. */
hf_status hf_check_device_error(unsigned *flags, int clear);

/* Launches one warp that waits on a barrier nothing will complete, with a
 * limit of limit_us microseconds (1 .. 10^7): it must give up and set bit
 * 1 of the error word.  Tests the timeout path without any fault. */
hf_status hf_selftest_wait_timeout(int limit_us, void *stream);

/* Barrier-schedule check without the risk of a hang (Sec. 3.1's partial
 * barriers wait for a count of threads; a count that is never reached would
 * stall a hardware barrier for good).  Launches one block of `warps` warps
 * (1..32) that run `rounds` (1..1000) rounds of a software barrier over all
 * of them with a wait bounded by limit_us microseconds (1 .. 10^7); warp
 * `missing` (or none when -1) skips the barrier.  Each warp adds the rounds
 * it completed to *d_completed (device pointer, may be NULL).  With every
 * warp present all rounds complete; with one missing the others give up,
 * set bit 2 of the error word and leave the context usable. */
hf_status hf_selftest_barrier(int warps, int missing, int rounds, int limit_us,
                              unsigned *d_completed, void *stream);

/* Measured throughput of one execution pipe on the current device, for
 * the compute terms of the ideal-overlap bound: what = 0 FP32 fused
 * multiply-adds per second, 1 32-bit integer multiplies (high or low half)
 * per second as the Philox4x32 round issues them (four per round, with its
 * XORs), 2 shared-memory atomic adds per second (conflict-free),
 * 3 32-bit integer ALU operations per second in the add / XOR / rotate mix
 * of the hash rounds.
 * Runs a few milliseconds of calibration kernels on `stream`. */
hf_status hf_calibrate(int what, void *stream, double *ops_per_s);

/* ------------------------------------------------------------------ */
/* Learned cost model (replaces profiling every configuration of the    */
/* search of Algorithm 2, Sec. 3.2, by a prediction).                  */

#define HF_MLP_NPARAMS 5825   /* 24-64-64-1 perceptron, see hf_mlp_forward */
#define HF_MLP_FEATURES 24

/* The 24 features of two stream-template kernels fused in one d0-thread
 * block (split threads for a) at a register cap, blocks per SM and the
 * fused instance's registers and spill bytes; hbm_gbs and ffma_per_s are
 * the device's measured bandwidth and FP32 FMA rate.  Host arithmetic; out
 * receives HF_MLP_FEATURES floats scaled to about [0, 1]. */
hf_status hf_tmpl_features(const hf_stream_tmpl_args *a, const hf_stream_tmpl_args *b, int split,
                           int d0, int regcap, int blocks_per_sm, int fused_regs, int spill_bytes,
                           double hbm_gbs, double ffma_per_s, float *out);

/* Algorithmic work of one launch of a body on its arguments, the quantities
 * of the ideal-overlap bound: the HBM bytes its definition moves (every
 * input read once, every output written once) and its operations per
 * pipe -- FP32 multiply-adds or FP32 operations, 32-bit integer
 * multiplies, shared-memory atomics, 32-bit add/XOR/rotate operations --
 * plus its barriers per tile.  Host arithmetic. */
typedef struct {
    double bytes;
    double ffma;
    double imul;
    double smem_atomic;
    double ialu;
    int barriers;
    int reserved;
} hf_body_work;
hf_status hf_body_work_of(int body_id, const void *args, hf_body_work *out);

/* Measured pipe rates (hf_calibrate) and HBM bandwidth of the device. */
typedef struct {
    double hbm_gbs;
    double ffma_per_s;
    double imul_per_s;
    double smem_atomic_per_s;
    double ialu_per_s;
} hf_pipe_peaks;

/* The HF_MLP_FEATURES features of any two registered kernels fused in one
 * d0-thread block (split threads for a, args[0] and args[1] their argument
 * blocks), generalising hf_tmpl_features to every body: per kernel, its
 * size (HBM bytes / 8), its operations per 32 bytes in FP32-FMA time
 * (the busiest pipe's time over the FMA rate), barriers, the shared memory
 * of its interval (with the bulk-copy ring the launch gives it at that
 * occupancy), its roofline time alone max(bytes / HBM, busiest pipe),
 * how compute-bound that is, its share of the block's threads, its warps
 * per SM and its share of the pair's roofline time; then the configuration
 * (register cap, blocks per SM, threads per SM, the fused instance's
 * registers and spill bytes, shared memory per SM).  For two stream
 * templates the result equals hf_tmpl_features.  Host arithmetic. */
hf_status hf_pair_features(hf_kernel a, hf_kernel b, const void *const *args, int split, int d0,
                           int regcap, int blocks_per_sm, int fused_regs, int spill_bytes,
                           const hf_pipe_peaks *peaks, float *out);

/* Installs the learned cost model used by hf_autotune(HF_TUNE_MODEL): an
 * ensemble of n_models (1..16) perceptrons, params (host) holding their
 * n_models * HF_MLP_NPARAMS floats back to back in the layout of
 * hf_mlp_forward.  Each predicts (log(time) - log(t_ideal) - mu) / sd from
 * hf_pair_features under `peaks`, t_ideal being the pair's ideal-overlap
 * time (the same for every candidate of a pair, so only the ranking
 * matters); candidates are ranked by the ensemble's mean prediction and the
 * `confirm` (>= 1) best are timed.  The library keeps a copy; a later call
 * replaces it, params = NULL removes it. */
hf_status hf_cost_model_set(const float *params, int n_models, float mu, float sd,
                            const hf_pipe_peaks *peaks, int confirm);

/* FP32 perceptron 24 -> 64 -> ReLU -> 64 -> ReLU -> 1 over n rows of
 * X[n][24] (device), writing y[n] (device).  params (device) is the flat
 * row-major array W1[64][24], b1[64], W2[64][64], b2[64], w3[64], b3. */
hf_status hf_mlp_forward(const float *params, const float *X, int n, float *y, void *stream);

/* Trains params in place with Adam on the mean squared error, all `steps`
 * steps in one kernel launch (one thread block): step s uses the batch rows
 * idx[s*batch .. s*batch + batch) of X[.][24] / Y[.] (batch <= 64); adam_m
 * and adam_v are the first and second moment arrays (device, HF_MLP_NPARAMS
 * each, zero for a fresh run); t0 is the number of Adam steps already taken.
 * loss_out[steps] (may be NULL) receives each step's batch loss; grad_out
 * (may be NULL) receives the first step's gradient.  Deterministic. */
hf_status hf_mlp_train(float *params, float *adam_m, float *adam_v, const float *X, const float *Y,
                       const int *idx, int steps, int batch, float lr, float beta1, float beta2,
                       float eps, int t0, float *loss_out, float *grad_out, void *stream);
int hf_mlp_nparams(void);

/* ------------------------------------------------------------------ */
/* CUDA graphs.                                                        */

typedef struct hf_graph_t *hf_graph;

/* Start recording the work issued to `stream` (relaxed capture mode): every
 * hf_launch / hf_launch_single on it, and on streams joined to it through
 * events, becomes part of the graph instead of running.  Launch each
 * configuration once before capturing it so that its resource queries are
 * cached.  hf_graph_end stops recording and instantiates the graph. */
hf_status hf_graph_begin(void *stream);
hf_status hf_graph_end(void *stream, hf_graph *out);
/* Replays the recorded work on `stream` as one submission. */
hf_status hf_graph_launch(hf_graph g, void *stream);
void hf_graph_destroy(hf_graph g);

/* Waits until all work queued on `stream` has finished, polling for at most
 * timeout_ms milliseconds: HF_ERR_TIMEOUT if it has not finished by then
 * (the work keeps running; nothing is cancelled), HF_ERR_CUDA if the stream
 * reports an error.  The launch-timeout check of the failure-detection
 * path; it never blocks longer than the limit. */
hf_status hf_stream_wait(void *stream, int timeout_ms);

const char *hf_status_string(hf_status s);
/* One-line description of the most recent error on this thread. */
const char *hf_last_error(void);
/* Size of the argument block of a body (for binding checks). */
size_t hf_args_size(int body_id);

#ifdef __cplusplus
}
#endif
#endif /* HFUSE_H */
