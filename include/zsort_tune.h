/*
 * zsort_tune.h -- autotuner of the runtime parameters of zsort (C ABI).
 *
 * The paper fixes its constants for one CPU thread (k = 0.6 sqrt(n) buckets,
 * scale k/4, insertion sort below 96 elements; Alg. 1 and section "Proposed
 * Work"); the GPU executor has its own tiling knobs instead, and this tuner
 * chooses them by measurement.  It is not part of the method: every choice
 * gives the same, uniquely defined sorted output.
 *
 * Knobs searched (fields of zsort_opts):
 *   kmax            bucket count per partition pass   {128, 256, 512}
 *   leaf_target     elements per bucket aimed at       {1024, 2048, 4096}
 *   leaf_cap        small-bucket cutoff (items per thread = leaf_cap / 256)
 *                                                      {2048, 3072, 4096}
 *   large_min       single-CTA / multi-CTA partition threshold
 *                                                      {32768, 65536, 131072, 262144}
 *   chunks_per_cta  look-back chunks per CTA and level {4, 8, 16}
 *   ipt             items per thread of a streamed tile {8, 12}
 * by coordinate descent from the caller's base options (each knob in turn,
 * every candidate value timed on a device copy of the caller's data, the
 * fastest kept; passes repeat until nothing changes or the budget is spent).
 *
 * Call classes.  Results are cached per class, a string
 *   "sm<SMs>/n<round(log2 n)>/s<round(log2 nseg), 0 for one array>/<dist>"
 * where <dist> comes from a strided sample of min(n, 4096) keys:
 *   "dup"       fewer than half of the sampled keys are distinct
 *   "sorted"    at least 90% of adjacent sample pairs ascend (non-strictly)
 *   "reversed"  at least 90% of adjacent sample pairs descend (strictly)
 *   "flat"      the Eq. 1 map (k = 512, scale k/4, sample statistics) puts at
 *               most 4x the mean load into its largest bucket
 *   "skew"      otherwise
 *
 * Cache file.  A JSON object, one entry per line, written by this library:
 *   {
 *   "sm152/n28/s0/flat": {"kmax": 512, "leaf_target": 2048, "leaf_cap": 4096,
 *                         "large_min": 65536, "chunks_per_cta": 8, "ipt": 12, "ms": 14.3},
 *   ...
 *   }
 * (each entry on a single line).  Writes replace the whole file through a
 * temporary file and a rename; concurrent writers are not coordinated (the
 * last rename wins).  A NULL cache_path means the path in the environment
 * variable ZSORT_TUNE_CACHE, and no caching when that is unset.
 */
#ifndef ZSORT_TUNE_H
#define ZSORT_TUNE_H

#include "zsort.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Returned when the cache holds no entry for a class (not an error). */
#define ZSORT_NOT_TUNED 1
/* Longest class string including its terminating zero. */
#define ZSORT_TUNE_CLASS_MAX 64

/* Class of a call from a HOST sample of m keys taken at positions
 * floor(i * n / m), i = 0..m-1, of an array of n keys in nseg segments (0 or
 * 1 = one array), on a GPU with sms SMs.  Writes the class string to
 * cls[0..cls_len) (cls_len >= ZSORT_TUNE_CLASS_MAX).  Pure host code. */
int zsort_tune_class_host(const uint64_t *sample, uint64_t m, uint64_t n, uint64_t nseg, int sms, char *cls,
                          size_t cls_len);

/* The same for DEVICE keys[0..n): copies the strided sample to the host
 * (synchronous on `stream`) and uses the current device's SM count. */
int zsort_tune_class(const uint64_t *keys, uint64_t n, uint64_t nseg, char *cls, size_t cls_len,
                     zsort_stream_t stream);

/* Cache lookup: on ZSORT_OK, copies the five tuned fields of the entry `cls`
 * into *out (other fields untouched) and its time into *ms (may be NULL).
 * ZSORT_NOT_TUNED if the file or the entry does not exist; ZSORT_ERR_INVALID
 * for a NULL argument or an entry that does not parse.  Pure host code. */
int zsort_tune_cache_get(const char *path, const char *cls, zsort_opts *out, double *ms);

/* Cache update: adds or replaces the entry `cls` with the five tuned fields
 * of *o and time ms.  ZSORT_ERR_INVALID if a field is out of range (see
 * zsort_opts) or the file cannot be written.  Pure host code. */
int zsort_tune_cache_put(const char *path, const char *cls, const zsort_opts *o, double ms);

/* Tuned options for a call like (keys, n, nseg): *out = *base (defaults when
 * base is NULL) with the cached fields of the call's class.  ZSORT_OK if an
 * entry was found, ZSORT_NOT_TUNED if not (then *out is the base).
 * Synchronous on `stream` (it samples the keys). */
int zsort_tuned_opts(const uint64_t *keys, uint64_t n, uint64_t nseg, const zsort_opts *base,
                     const char *cache_path, zsort_opts *out, zsort_stream_t stream);

/* Tunes the knobs for sorting (keys, vals) -- one array when seg_offsets is
 * NULL (then nseg is ignored, n <= ZSORT_MAX_N), else the batch of
 * zsort_segmented -- and returns the fastest options in *out.  keys, vals
 * and seg_offsets (DEVICE pointers) are read, never modified: every trial
 * sorts a device copy, so the call allocates 12 * n bytes for its duration.
 * With a cache, an existing entry of the call's class is returned without
 * any trial unless (flags & ZSORT_TUNE_FORCE); the result is stored.  Each
 * candidate is timed with CUDA events as the median of `reps` runs (0 = 3);
 * the search stops when budget_ms of wall time are spent (0 = no limit).
 * Synchronous.  Candidates whose sort reports a device error are skipped. */
#define ZSORT_TUNE_FORCE 1u
int zsort_autotune(const uint64_t *keys, const uint32_t *vals, uint64_t n, const uint64_t *seg_offsets,
                   uint64_t nseg, const zsort_opts *base, const char *cache_path, uint32_t budget_ms,
                   uint32_t reps, uint32_t flags, zsort_opts *out, zsort_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* ZSORT_TUNE_H */
