/*
 * zsort.h -- C ABI of a GB300 (sm_103a) stable distribution sort of 64-bit
 * keys with a 32-bit payload, after zSort (Jain et al., "zSort: Stable
 * Distribution Sort using Z-Score Partitioning", arXiv 2605.14419).
 *
 * The operation (section "Proposed Work", problem statement and stability
 * paragraph): sort n (key, payload) pairs in place, ascending by key; among
 * equal keys the input order is kept.  The result is the unique permutation
 * that orders the tuples (key, input position) lexicographically, so it is
 * bit-for-bit reproducible and independent of every tuning choice.
 *
 * The method (Alg. 1 and zsortRec): per (sub)array the mean and population
 * standard deviation of the keys, the z-score map of Eq. 1 from a key to one
 * of k buckets, a histogram and an exclusive scan for the bucket offsets, a
 * stable scatter; oversized buckets repeat the same steps, small ones are
 * finished in on-chip shared memory.  A learned monotone piecewise-linear
 * CDF map may replace Eq. 1 (not in the paper; see ZSORT_MAP_LEARNED).
 *
 * Conventions for every entry point below
 *   - keys, vals and seg_offsets are CUDA DEVICE pointers of the current
 *     device, 16-byte aligned is recommended (8 required for keys, 4 for
 *     vals); the caller owns them.  The library owns its scratch workspace
 *     (about 12 bytes per element plus bookkeeping), cached per (device,
 *     stream) and grown on demand; zsort_reserve() sizes it up front so
 *     that later calls do not allocate.
 *   - Calls are stream ordered and asynchronous: they return once the work
 *     is enqueued on `stream` (NULL = the legacy default stream).  Calls on
 *     different streams use different workspaces and may overlap; calls on
 *     one stream come from one host thread at a time.
 *   - Host-detectable errors (bad arguments, allocation failure, launch
 *     failure) are returned at once and nothing is enqueued.  Errors found
 *     on the device (a wait that timed out, decreasing segment offsets, a
 *     full internal queue) are written to a device status word that
 *     zsort_sync_status() returns; the contents of keys/vals are then
 *     unspecified, but no kernel traps, faults or hangs.
 */
#ifndef ZSORT_H
#define ZSORT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t, spelled without the CUDA headers. */
typedef struct CUstream_st *zsort_stream_t;

/* Status codes. */
enum {
    ZSORT_OK = 0,
    ZSORT_ERR_INVALID = -1,     /* bad argument (null pointer, n too large) */
    ZSORT_ERR_NOMEM = -2,       /* device allocation of the workspace failed */
    ZSORT_ERR_CUDA = -3,        /* a CUDA runtime call or a launch failed    */
    ZSORT_ERR_TIMEOUT = -4,     /* a bounded device-side wait expired        */
    ZSORT_ERR_BAD_OFFSETS = -5, /* segment offsets decrease or exceed n      */
    ZSORT_ERR_CAPACITY = -6,    /* an internal device queue overflowed       */
    ZSORT_ERR_INTERNAL = -7     /* a device-side consistency check failed    */
};

/* Largest n accepted by zsort_pairs* (look-back status words carry 30-bit
 * counts); zsort_segmented* accept arrays up to ZSORT_MAX_SEG_TOTAL with
 * every segment at most ZSORT_MAX_N long. */
#define ZSORT_MAX_N ((uint64_t)1 << 30)
#define ZSORT_MAX_SEG_TOTAL ((uint64_t)1 << 34)

/* Bucket maps (zsort_opts.mapper). */
enum {
    ZSORT_MAP_ZSCORE = 0,  /* Eq. 1: floor(((x - mean)/sd + |z_min|) * k/4)   */
    ZSORT_MAP_LEARNED = 1, /* piecewise-linear CDF, 256 pieces, FP32, trained
                              on a sample of keys normalised to binary32;
                              when it fails the load test, the same CDF with
                              exact-key breakpoints (ZSORT_MAPINFO_SPLIT),
                              then Eq. 1                                     */
    ZSORT_MAP_MLP = 2      /* 2-layer MLP with positive weights and 32
                              clamp(., 0, 1) hidden units, FP32, fitted to
                              the same sample's 257 quantiles: f(u) =
                              sum_h a_h clamp(w_h u + b_h, 0, 1), a, w >= 0,
                              bucket = trunc(k (f(u) - f(0)) / (f(u_max) -
                              f(0))); monotone by construction; when it
                              fails the load test, the exact-key CDF
                              (ZSORT_MAPINFO_SPLIT), then Eq. 1              */
};

/* Map actually used at the top level (zsort_map_info.map). */
enum {
    ZSORT_MAPINFO_ZSCORE = 0,
    ZSORT_MAPINFO_LEARNED = 1,
    ZSORT_MAPINFO_RANGE = 2,  /* the progress guard's exact range map */
    ZSORT_MAPINFO_MLP = 3,
    ZSORT_MAPINFO_SPLIT = 4   /* the learned CDF with exact-key breakpoints (the
                                 sample's 256-quantile keys) and binary32
                                 interpolation inside each piece, relative to
                                 its lower key; tried when the normalised map
                                 fails the load test */
};

/* Key types for zsort_pairs_ex. */
enum {
    ZSORT_KEY_U64 = 0,
    ZSORT_KEY_I64 = 1, /* two's complement order                           */
    ZSORT_KEY_F64 = 2  /* IEEE-754 totalOrder: -NaN < -inf < ... < -0.0 <
                          +0.0 < ... < +inf < +NaN                           */
};

/* Tuning options.  Fill with zsort_default_opts() and change fields. */
typedef struct {
    uint32_t struct_size;    /* sizeof(zsort_opts)                            */
    uint32_t mapper;         /* ZSORT_MAP_ZSCORE or ZSORT_MAP_LEARNED          */
    uint32_t kmax;           /* most buckets per partition, power of 2, 16..512 */
    uint32_t leaf_target;    /* k = clamp(pow2ceil(len / leaf_target), 16, kmax) */
    uint32_t large_min;      /* longer (sub)arrays are partitioned by all SMs
                                with a decoupled look-back; shorter ones by
                                one CTA                                      */
    uint32_t learn_min;      /* arrays at least this long train a learned map */
    uint32_t sample;         /* learned-map training sample, 256..65536       */
    float fallback_ratio;    /* learned map rejected if its sampled largest
                                bucket exceeds fallback_ratio * sample / k   */
    uint64_t seed;           /* seed of the sample positions                  */
    uint32_t guard_level;    /* from this depth on, the exact range map is used */
    uint32_t ctas_per_sm;    /* persistent CTAs per SM, 0 = from occupancy     */
    uint32_t wait_limit_ms;  /* bound of every device-side wait (no progress)  */
    uint32_t flags;          /* ZSORT_FLAG_*                                    */
    uint32_t leaf_cap;       /* small-bucket cutoff: buckets (and groups of
                                consecutive buckets) of at most this many
                                pairs are finished in shared memory,
                                256..4096 (the CTA's 256 threads hold
                                leaf_cap / 256 items each)                    */
    uint32_t chunks_per_cta; /* look-back chunk tasks per CTA over one level
                                of large partitions, 1..64                    */
    uint32_t ipt;            /* items per thread of a streamed tile: 12 (tiles
                                of 3072 pairs) or 8 (2048); the statistics,
                                histogram and scatter passes all use it       */
} zsort_opts;

/* flags: capture the call's launch sequence (control-block reset, two set-up
 * kernels, the persistent kernel) in a CUDA graph on first use and replay it
 * with one cudaGraphLaunch while the workspace, pointers, sizes and options
 * stay the same.  Needs a non-default stream (else ignored). */
#define ZSORT_FLAG_GRAPH 1u
/* Test of the bounded waits: the call publishes no work but counts one
 * pending entry, so every CTA of the persistent kernel waits at the empty
 * queue -- for a ready word that nothing sets -- until wait_limit_ms pass
 * without progress; the kernel then records ZSORT_ERR_TIMEOUT and returns.
 * keys/vals are not touched and the next call on the stream works as usual.
 * Not a sort: it exists to check the failure path without any GPU fault. */
#define ZSORT_FLAG_TEST_STALL 2u

/* Fault injection for failure-path tests, without any GPU fault: the
 * environment variable ZSORT_FAULT, read at every sorting call.
 *   "alloc"       the workspace allocation fails: the call returns
 *                 ZSORT_ERR_NOMEM and enqueues nothing;
 *   "timeout"     as ZSORT_FLAG_TEST_STALL with a 50 ms wait limit:
 *                 zsort_sync_status returns ZSORT_ERR_TIMEOUT;
 *   "badoffsets"  the segment check reports malformed offsets:
 *                 zsort_sync_status returns ZSORT_ERR_BAD_OFFSETS.
 * In every case keys and payloads are untouched and the next call without
 * the variable works as usual. */
/* Task trace: the persistent kernel records every task it runs (one record
 * per dequeued task: start and end time, CTA, task type, partition depth),
 * read back with zsort_last_trace.  The first traced call on a stream
 * allocates the workspace's trace buffer of ZSORT_TRACE_CAP records (32 MB);
 * tasks past it are counted, not recorded.  Costs one global atomic and one
 * 32-byte store per task. */
#define ZSORT_FLAG_TRACE 4u
#define ZSORT_TRACE_CAP (1u << 20)
/* Exact statistics at every level.  By default a large sub-array below the
 * top level (one that a partition pass produced) takes its Eq. 1 statistics
 * from ZSORT_SUB_SAMPLE keys at stratified positions instead of a pass over
 * all its keys: the sub-problems of zsortRec (section "Proposed Work") keep
 * the top level's map form and estimate its inputs, and the map only has to
 * be monotone for the sort to be exact.  The top level, sub-arrays that use
 * the range map (progress guard) or a learned map, and sub-arrays whose
 * sample keys are all equal always take the exact pass.  This flag makes
 * every level take it. */
#define ZSORT_FLAG_EXACT_SUBSTATS 8u
#define ZSORT_SUB_SAMPLE 4096u

/* One record of the task trace.  type is the task type of zsort_stats.task_ns
 * (1 statistics chunk, 2 learned-map sample run, 3 histogram chunk, 4
 * scatter chunk, 5 single-CTA partition, 6 finish, 7 copy, 8 map inspection,
 * 9 learned-map fit, 10 sampled statistics), or ZSORT_TRACE_HANDLER + t for the phase-completion
 * work that the last task of a phase of type t ran right after it (the
 * bucket scan after a histogram, the classification of the children after
 * a scatter; count 0).  Times are the device's globaltimer in ns.  A CTA's
 * idle time is the gap between its consecutive records. */
#define ZSORT_TRACE_HANDLER 16u
typedef struct {
    uint64_t t_start_ns;
    uint64_t t_end_ns;
    uint32_t cta;     /* block index in the persistent launch                 */
    uint16_t type;    /* task type (above)                                    */
    uint16_t level;   /* partition depth of the task's (sub)array              */
    uint32_t arg;     /* (sub)array descriptor, or item index for types 5 and 6 */
    uint32_t count;   /* chunks / items the task covered                       */
} zsort_trace_rec;

/* Counters of the last completed call on a (device, stream) workspace. */
typedef struct {
    uint64_t n;                 /* elements of the call                         */
    uint64_t partitions_large;  /* multi-CTA partition passes                   */
    uint64_t partitions_small;  /* single-CTA partition passes                  */
    uint64_t leaves;            /* shared-memory finish tasks                   */
    uint64_t leaf_fallbacks;    /* finish tasks that took the bitonic fallback  */
    uint64_t copies;            /* all-equal (sub)arrays copied back            */
    uint64_t learned_accepted;  /* learned maps accepted by the load test       */
    uint64_t learned_rejected;  /* learned maps rejected (Eq. 1 used)           */
    uint64_t guard_levels;      /* partitions that used the range map           */
    uint64_t max_level;         /* deepest partition level                      */
    uint64_t bytes_algorithmic; /* bytes read + written by the method's passes  */
    uint64_t tasks;             /* tasks executed by the persistent kernel      */
    uint64_t persistent_ctas;   /* CTAs of the persistent launch                */
    double top_mean_d;          /* top level: mean of key - min (segment 0)     */
    double top_sd;              /* top level: population standard deviation     */
    uint64_t top_min, top_max;  /* top level: exact min and max                 */
    uint32_t top_k;             /* top level: buckets                           */
    uint32_t top_map;           /* top level: map used (ZSORT_MAPINFO_*)           */
    /* device time of the persistent kernel's tasks, summed over CTAs (ns);
       index = task type: 1 statistics tile or sample, 2 learned-map training, 3
       histogram tile, 4 look-back scatter tile, 5 single-CTA partition,
       6 shared-memory finish, 7 copy */
    uint64_t task_ns[8];
    uint64_t task_count[8];
    uint64_t handler_ns;        /* phase-completion work, after its last task     */
    uint64_t idle_ns;           /* time CTAs spent waiting for work               */
    uint64_t busy_window_ns;    /* first task start to last task end              */
    uint64_t sampled_stats;     /* sub-arrays whose statistics came from a sample */
} zsort_stats;

/* Fills *o with the defaults (z-score map, kmax 512, leaf target 2048, ...). */
void zsort_default_opts(zsort_opts *o);

/* Sorts n (uint64 key, uint32 payload) pairs in place, stably (see above).
 * n <= ZSORT_MAX_N.  Uses the default options.  vals may be NULL: then the
 * keys are sorted alone (key-only mode, the paper's own workload; each pass
 * moves 8 bytes per element instead of 12).  Every entry point below that
 * takes vals accepts NULL the same way. */
int zsort_pairs(uint64_t *keys, uint32_t *vals, uint64_t n, zsort_stream_t stream);

/* Key-only sort of n uint64 keys in place: zsort_pairs(keys, NULL, n, stream). */
int zsort_keys(uint64_t *keys, uint64_t n, zsort_stream_t stream);

/* 128-bit keys (UUIDs, hashes; the paper's motivation, section
 * "Introduction": zSort's pass count does not grow with the key width):
 * key i is the pair of words keys[2i] (low 64 bits) and keys[2i+1] (high 64
 * bits), compared as an unsigned 128-bit number; sorted in place with vals
 * (may be NULL), stably.  With d = key - min (exact, 128 bits) and s =
 * max(0, bitlen(max - min) - 64), the window d >> s fits 64 bits and,
 * with the s bits below it, orders like the key.  One stable zSort of
 * (window, input index); then only the keys in runs of equal windows (none
 * when the keys' top 64 significant bits differ, as for hashes) are sorted
 * by the bits below the window, run by run, in segmented zSorts of those
 * keys alone (2^20 runs a launch); then one gather of keys and payloads.  Keys that share
 * windows in bulk (a few distinct high words over a 2^128 range) make the
 * second sort as long as the first.  The call waits for the stream once,
 * to read the size of the tied runs.  Scratch: 44 bytes per key (28 without
 * payloads) kept with the stream's workspace (grown on demand, freed by
 * zsort_release), plus 20 bytes per tied key of stream-ordered scratch
 * (cudaMallocAsync).
 * n <= ZSORT_MAX_N; opts may be NULL. */
int zsort_pairs_u128(uint64_t *keys, uint32_t *vals, uint64_t n, const zsort_opts *opts, zsort_stream_t stream);

/* The same for int64 keys (two's complement order) and float64 keys (IEEE
 * totalOrder, so -0.0 sorts before +0.0).  The keys are encoded to uint64 in
 * place on the device, sorted, and decoded. */
int zsort_pairs_i64(int64_t *keys, uint32_t *vals, uint64_t n, zsort_stream_t stream);
int zsort_pairs_f64(double *keys, uint32_t *vals, uint64_t n, zsort_stream_t stream);

/* General form: key_type is ZSORT_KEY_*, opts may be NULL (defaults). */
int zsort_pairs_ex(void *keys, uint32_t key_type, uint32_t *vals, uint64_t n,
                   const zsort_opts *opts, zsort_stream_t stream);

/* Batched sort: keys/vals hold n elements; segment i is
 * [seg_offsets[i], seg_offsets[i+1]) and is sorted on its own, stably.
 * seg_offsets is a device array of nseg + 1 non-decreasing values <= n, and no
 * segment may be longer than ZSORT_MAX_N;
 * empty segments are allowed and elements outside
 * [seg_offsets[0], seg_offsets[nseg]) are untouched.  The whole batch runs
 * as one persistent kernel over a device work queue.  A violation of the
 * offsets contract is reported as ZSORT_ERR_BAD_OFFSETS by
 * zsort_sync_status() and leaves keys/vals untouched. */
int zsort_segmented(uint64_t *keys, uint32_t *vals, uint64_t n, const uint64_t *seg_offsets,
                    uint64_t nseg, zsort_stream_t stream);
int zsort_segmented_ex(uint64_t *keys, uint32_t *vals, uint64_t n, const uint64_t *seg_offsets,
                       uint64_t nseg, const zsort_opts *opts, zsort_stream_t stream);

/* Sizes the (device, stream) workspace for calls of up to n elements and
 * nseg segments (n <= ZSORT_MAX_SEG_TOTAL), so that those calls allocate
 * nothing. */
int zsort_reserve(uint64_t n, uint64_t nseg, zsort_stream_t stream);

/* Frees every workspace of the current device.  No call may be in flight. */
int zsort_release(void);

/* Waits for `stream`, then returns the device status word of its workspace
 * (ZSORT_OK or a negative code) and clears it. */
int zsort_sync_status(zsort_stream_t stream);

/* Waits for `stream` and copies the counters of its last call to *out. */
int zsort_last_stats(zsort_stream_t stream, zsort_stats *out);

/* Waits for `stream` and copies the task trace of its last call (made with
 * ZSORT_FLAG_TRACE) to out[0 .. min(cap, recorded, ZSORT_TRACE_CAP)), in the
 * order the tasks finished.  *count = tasks of that call (more than were
 * recorded if the buffer overflowed; 0 if the call was not traced).  out may
 * be NULL when cap is 0.  ZSORT_ERR_INVALID if count is NULL. */
int zsort_last_trace(zsort_stream_t stream, zsort_trace_rec *out, uint64_t cap, uint64_t *count);

/* Top-level partition plan of one array (zsort_map_buckets). */
typedef struct {
    uint32_t map;               /* ZSORT_MAPINFO_*                                     */
    uint32_t k;                 /* buckets                                            */
    uint64_t min, max;          /* exact min / max of the keys                        */
    double mean_d, sd;          /* mean of key - min, population sd (exact sums)      */
    float zc;                   /* Eq. 1 multiplier: bucket = min(k-1, trunc(fl32(u32((key - min) >> zsh)) * zc)) */
    uint32_t zsh;
    float escale;               /* learned map: u = fl32(key - min) * escale           */
    uint32_t trained;           /* 1 if a learned map was trained (q, r valid)         */
    float q[257];               /* learned map breakpoints                             */
    float r[256];               /* learned map reciprocal piece widths                 */
    uint32_t learned_max_load;  /* load test: largest learned bucket on the sample     */
    uint32_t zscore_max_load;   /* load test: largest Eq. 1 bucket on the sample       */
    float mlp[98];              /* MLP map (mapper ZSORT_MAP_MLP): w[32], b[32], a[32],
                                   f0, inv                                             */
} zsort_map_info;

/* Inspection: runs the statistics step and the bucket-map choice (Eq. 1 of
 * section "Proposed Work", or the learned map with its load test) that
 * zsort_pairs_ex would run at the top level of keys[0..n), and writes every
 * key's top-level bucket to the device array buckets[0..n) instead of
 * sorting.  keys are not modified.  Synchronous: waits for `stream` and fills
 * *info.  2 <= n <= ZSORT_MAX_N. */
int zsort_map_buckets(const uint64_t *keys, uint64_t n, const zsort_opts *opts, uint32_t *buckets,
                      zsort_map_info *info, zsort_stream_t stream);

/* Pairs per streamed tile at the default zsort_opts.ipt (12 per thread): the
 * unit in which a large (sub)array is cut into chunk tasks (each chunk is at
 * least four tiles); 256 * ipt in general. */
#define ZSORT_TILE_PAIRS 3072u

/* Largest n accepted by zsort_pairs_noalloc. */
#define ZSORT_NOALLOC_MAX_N ((uint64_t)1 << 20)

/* zsort_pairs_noalloc -- the sort of zsort_pairs (default options, uint64
 * keys) for callers that cannot allocate device memory: real-time or
 * embedded hosts that forbid device allocation once they have started, and
 * processes that must stay inside a fixed memory pool they may not grow.
 * The paper has no counterpart; it is a deployment variant.
 *   - Allocates nothing: no cudaMalloc/cudaFree and no allocating library
 *     call.  Its scratch is a static __device__ array of about 24 MB for up
 *     to ZSORT_NOALLOC_MAX_N (2^20) elements that every GPU which loads this
 *     library holds until the process exits.  n > ZSORT_NOALLOC_MAX_N is
 *     rejected with ZSORT_ERR_INVALID before anything is enqueued.
 *   - The first call on a device does its set-up (looks up the array's device
 *     address and sets a kernel attribute), so make that first call before
 *     any stream capture.
 *   - Every call, on every stream, shares the one array and leaves its
 *     contents behind; calls that overlap on the GPU race and corrupt each
 *     other's results, so order them (one stream, or events).
 *   - status: optional caller-owned DEVICE int32 that receives the call's
 *     device status (ZSORT_OK or a negative code) in stream order; NULL
 *     skips it.  zsort_sync_status() and zsort_last_stats() do not cover
 *     this entry point.
 * keys/vals as for zsort_pairs; returns host-detected errors at once. */
int zsort_pairs_noalloc(uint64_t *keys, uint32_t *vals, uint64_t n, int32_t *status,
                        zsort_stream_t stream);

/* Human-readable text of a status code (static storage). */
const char *zsort_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* ZSORT_H */
