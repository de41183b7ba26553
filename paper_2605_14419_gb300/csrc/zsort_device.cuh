// zsort_device.cuh -- device-side building blocks of the GB300 zSort.
//
// Data layout in HBM (all arrays structure-of-arrays, 64-bit keys, 32-bit
// payloads):  the caller's keys/vals, a scratch pair of the same length
// (scratch[i] mirrors user[i]; a bucket keeps its index range in both), and
// the bookkeeping pools of the persistent executor (queue entries, large
// segment descriptors, work items, bucket starts, look-back status rows,
// learned-map tables and training buffers).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <cstddef>

namespace zs {

// ---------------------------------------------------------------- constants
constexpr int BLOCK = 256;                // threads per CTA
constexpr int WARPS = BLOCK / 32;
constexpr int IPT = 12;                   // items per thread of a streamed tile (default, largest)
constexpr int IPT_SMALL = 8;              // the other choice of zsort_opts.ipt
constexpr int TILE = BLOCK * IPT;         // 3072 pairs: the largest streamed tile (buffer size)
constexpr int TILE_MIN = BLOCK * IPT_SMALL;  // 2048 pairs: the smallest
constexpr int WARP_SPAN = 32 * IPT;       // contiguous elements per warp and tile of IPT items
constexpr int LEAF_IPT = 16;              // items per thread of a leaf
constexpr int LEAF_CAP = BLOCK * LEAF_IPT;  // 4096: a bucket (group) this small is finished in smem
constexpr int LEAF_SPAN = 32 * LEAF_IPT;
constexpr int PAD = 8;                    // smem slack for 16-byte aligned bulk copies
constexpr int NB_MAX = 512;               // buckets per partition pass
constexpr int RANK_SMALL = BLOCK;         // leaves this small are ranked by counting
constexpr int SC_STAGES = 2;              // streamed (key, payload) tile buffers per CTA
static_assert(8 * WARP_SPAN >= 16 + 4 * NB_MAX, "a warp's peer table fits its span of the tile's keys");
constexpr uint32_t LEAF_M2_MAX = 2048;    // sub-buckets of the fast leaf path
constexpr int LEAF_RANK_U = 4;            // staged pairs per thread and round of the leaf's rank count
constexpr int PWL_P = 256;                // pieces of the learned map
constexpr int SAMPLE_MAX = 65536;         // largest training sample
constexpr int SAMPLE_RUNS = 8;            // the sample is sorted as this many runs, one CTA each
constexpr int MIN_K = 16;                 // fewest buckets of a partition pass
constexpr int MAX_LEVEL = 48;             // hard bound on the partition depth
constexpr uint32_t INVALID = 0xFFFFFFFFu;
constexpr uint32_t FLAG_A = 1u << 30;     // look-back: chunk aggregate only
constexpr uint32_t FLAG_P = 2u << 30;     // look-back: inclusive prefix
constexpr uint32_t VAL_MASK = (1u << 30) - 1;

// Status codes (mirror zsort.h).
constexpr int ST_TIMEOUT = -4;
constexpr int ST_BAD_OFFSETS = -5;
constexpr int ST_CAPACITY = -6;
constexpr int ST_INTERNAL = -7;

enum MapKind : uint32_t { MAP_Z = 0, MAP_PWL = 1, MAP_RANGE = 2, MAP_MLP = 3, MAP_SPLIT = 4 };
constexpr int MLP_H = 32;                 // hidden units of the MLP map
constexpr int MLP_ITERS = 128;            // its training iterations
constexpr int MLP_TABLE = 3 * MLP_H + 2;  // w[H], b[H], a[H], f0, inv
enum TaskType : uint32_t {
    T_NONE = 0,
    T_LSTATS = 1,    // large segment: statistics tile
    T_LSAMPLE = 2,   // large segment: learned-map sample, drawn and sorted as
                     // SAMPLE_RUNS runs (one CTA each, beside the statistics tiles)
    T_LHIST = 3,     // large segment: histogram tile
    T_LSCATTER = 4,  // large segment: look-back stable scatter tile
    T_MPART = 5,     // medium segment: whole partition pass by one CTA
    T_FINISH = 6,    // leaf (group of small buckets): shared-memory sort
    T_COPY = 7,      // all-equal large segment living in scratch: copy back
    T_DUMP = 8,      // map inspection: bucket of every key of a chunk
    T_LFIT = 9,      // large segment: learned-map breakpoints and load test (one CTA,
                     // after both the statistics and the sample)
    T_SSTATS = 10    // large sub-array: statistics and Eq. 1 map from a sample (one CTA)
};
constexpr int WARP_DISTINCT_MAX = 32;  // stable leaf path: distinct keys a warp's counting sort takes
constexpr uint32_t LEAF_INSERT_MAX = 16;  // stable leaf path: sub-buckets this short sorted by insertion
constexpr uint32_t LOCAL_CLAIM = 8;  // stashed leaves taken per task (the next one is prefetched)
constexpr uint32_t SUB_SAMPLE = 4096;     // keys of a sub-array's statistics sample

// ---------------------------------------------------------------- records
// A large segment: partitioned by many CTAs, phase by phase.
struct Seg {
    unsigned long long off;      // first element (absolute index)
    unsigned long long mn, mx;   // exact min / max (atomics)
    unsigned long long s1[2];    // exact sum of keys, 128-bit (atomics)
    unsigned long long s2[3];    // exact sum of squared keys, 192-bit
    unsigned long long status_base;  // first look-back word
    double mean_d, sd;           // mean of key - min, population sd
    float zc;                    // z-score map multiplier: (k/4) / sd * 2^zsh
    float escale;                // learned map: 2^-bitlen(max - min)
    uint32_t zsh;                // z-score map: keys - min are shifted right by zsh
    uint32_t len, k, tiles, level, buf;
    uint32_t kind;               // MapKind
    uint32_t rshift, rmult;      // range map
    uint32_t train_slot;         // learned map training buffer, INVALID if none
    uint32_t max_learned, max_z; // load test: largest sample bucket per map
    uint32_t chunk_tiles;        // tiles per chunk task (the first chunks_big chunks)
    uint32_t chunks;             // chunk tasks per phase
    uint32_t chunks_big;         // chunks of chunk_tiles tiles; the rest have chunk_tiles_small
    uint32_t chunk_tiles_small;
    uint32_t join;               // learned map: statistics + sample selection still running
    uint32_t runs_left;          // learned map: sample runs not yet sorted
    uint32_t next_type, next_nt; // learned map: the task the last of the two publishes
    uint32_t range_map;          // the parent's partition left it more than half: exact range map
};

// Bit 15 of Item.level: partition this medium (sub)array with the range map.
constexpr uint32_t ITEM_RANGE_MAP = 0x8000u;

// A leaf group or a medium segment.
struct Item {
    unsigned long long off;
    uint32_t len;
    uint16_t buf;
    uint16_t level;
};

struct Entry {
    uint32_t type, arg, ntiles, pad;
};

// Two work queues, each an append-only array of entries: 0 = partition work
// (statistics, samples, histograms, scatters, fits, single-CTA partitions,
// copies), 1 = leaves.  A CTA takes partition work first: it creates the
// later work, so the deep chains of skewed inputs start early, and leaves,
// which depend on nothing, fill the gaps.
constexpr int QUEUES = 2;

struct Ctl {
    unsigned int q_head[QUEUES], q_alloc[QUEUES];
    unsigned int pending, error, seg_alloc, item_alloc;
    unsigned int train_alloc, init_leaf, init_med, pad0;
    unsigned long long status_alloc;
    unsigned long long progress;
    // counters reported through zsort_stats
    unsigned long long n_large, n_small, n_leaves, n_leaf_fb, n_copies;
    unsigned long long n_learn_ok, n_learn_rej, n_guard, max_level, bytes, tasks;
    double top_mean_d, top_sd;
    unsigned long long top_min, top_max;
    unsigned int top_k, top_map;
    unsigned int epoch, pad3;      // this call's queue epoch (from the persistent counter)
    // device time per task type (ns, summed over CTAs), handler and idle time
    unsigned long long task_ns[8], task_cnt[8], handler_ns, idle_ns;
    unsigned long long t_first, t_last;
    unsigned long long trace_n;    // task records written (or attempted) to the trace
    unsigned long long n_sampled;  // sub-arrays whose statistics came from a sample
};

// Trace type of the phase-completion work a task triggered (type | this).
constexpr uint32_t TRACE_HANDLER = 16u;
// One task of the persistent kernel in the optional trace (zsort_trace_rec).
struct TraceRec {
    unsigned long long t_start, t_end;
    uint32_t cta;
    uint16_t type, level;
    uint32_t arg, count;
};
static_assert(sizeof(TraceRec) == 32, "trace record layout");

struct Params {
    uint64_t *ukeys;
    uint32_t *uvals;
    uint64_t *skeys;
    uint32_t *svals;
    unsigned long long n;
    Ctl *ctl;
    Entry *entries;
    uint32_t *ready, *tnext, *tdone;
    uint32_t qcap;               // entries per queue (entries, ready, tnext, tdone hold QUEUES * qcap)
    uint32_t epoch_unused;
    uint32_t *epoch_ctr;         // persistent call counter (not cleared between calls)
    Seg *segs;
    uint32_t segcap;
    Item *items;
    uint32_t itemcap;
    uint32_t *bstart;   // segcap * NB_MAX
    uint16_t *ids;      // n: a learned map's bucket of every key, from histogram to scatter
    uint32_t *status;            // look-back words and chunk offsets: 2 * chunks * k per segment
    unsigned long long statuscap;
    uint32_t nctas;              // CTAs of the persistent launch
    uint32_t *plan_out;          // map inspection: bucket of every key (else null)
    uint32_t user_aligned;       // caller's keys and vals 16-byte aligned: bulk copies allowed
    uint32_t kv;                 // 1: (key, payload) pairs; 0: keys only (vals == null)
    uint32_t test_stall;         // publish nothing, one entry pending: every wait runs out
    uint32_t test_badoff;        // fault injection: the segment check reports bad offsets
    TraceRec *trace;             // task trace (null: not traced)
    uint32_t trace_cap;          // records trace can hold
    float *pwl;         // segcap * PWL_STRIDE: breakpoints q[0..P], reciprocals r[0..P), MLP table
    unsigned long long *trainbuf; // traincap * 2 * SAMPLE_MAX sampled keys (ping-pong)
    uint32_t traincap;
    // options
    uint32_t kmax, leaf_target, large_min, learn_min, sample, mapper, guard_level;
    uint32_t leaf_cap, chunks_per_cta;
    uint32_t ipt, tile;          // items per thread of a streamed tile, pairs per tile (256 ipt)
    uint32_t sub_sample;         // 1: large sub-arrays below the top take sampled statistics
    float fallback_ratio;
    unsigned long long seed;
    unsigned long long wait_ns;
};

// ---------------------------------------------------------------- memory ops
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void set_error(const Params &P, int code)
{
    atomicCAS(&P.ctl->error, 0u, (unsigned int)code);
}
__device__ __forceinline__ bool has_error(const Params &P)
{
    return ld_relaxed(&P.ctl->error) != 0;
}

__device__ __forceinline__ uint32_t bitlen64(unsigned long long x)
{
    return x ? 64u - (uint32_t)__clzll((long long)x) : 0u;
}
__device__ __forceinline__ uint32_t pow2ceil32(uint32_t x)
{
    return x <= 1 ? 1u : 1u << (32 - __clz((int)(x - 1)));
}

// ------------------------------------------------------- exact moments
// Exact running sums of a set of keys: count is implicit, S1 = sum x
// (128-bit), S2 = sum x^2 (192-bit), exact min / max.  Integer sums are
// associative, so the result does not depend on the reduction order.
struct Acc {
    unsigned long long mn, mx;
    unsigned __int128 s1;
    unsigned __int128 s2lo;
    unsigned long long s2hi;
};

__device__ __forceinline__ void acc_merge(Acc &a, const Acc &b)
{
    a.mn = b.mn < a.mn ? b.mn : a.mn;
    a.mx = b.mx > a.mx ? b.mx : a.mx;
    a.s1 += b.s1;
    unsigned __int128 t = a.s2lo + b.s2lo;
    a.s2hi += b.s2hi + ((t < b.s2lo) ? 1ull : 0ull);
    a.s2lo = t;
}
// The per-thread form of the streamed sums, in 32-bit pieces: with x = h 2^32
// + l, S1 = 2^32 sum h + sum l and S2 = 2^64 sum h^2 + 2^33 sum h l +
// sum l^2.  Each product is one 32 x 32 -> 64-bit multiply, added into a
// 96-bit sum by one carry chain (no 128-bit multiply or compare per key).
// A thread adds at most 2^30 keys, so no sum overflows its width.
struct LAcc {
    unsigned long long mn, mx;
    unsigned long long sl, sh;       // sum l, sum h
    uint32_t a0, a1, a2;             // sum l^2
    uint32_t b0, b1, b2;             // sum h l
    uint32_t c0, c1, c2;             // sum h^2
};
__device__ __forceinline__ void lacc_init(LAcc &a)
{
    a.mn = ~0ull;
    a.mx = 0ull;
    a.sl = a.sh = 0ull;
    a.a0 = a.a1 = a.a2 = a.b0 = a.b1 = a.b2 = a.c0 = a.c1 = a.c2 = 0u;
}
__device__ __forceinline__ void add96(uint32_t &x0, uint32_t &x1, uint32_t &x2, unsigned long long p)
{
    asm("add.cc.u32 %0, %0, %3;\n\taddc.cc.u32 %1, %1, %4;\n\taddc.u32 %2, %2, 0;"
        : "+r"(x0), "+r"(x1), "+r"(x2)
        : "r"((uint32_t)p), "r"((uint32_t)(p >> 32)));
}
__device__ __forceinline__ void lacc_key(LAcc &a, unsigned long long x)
{
    a.mn = x < a.mn ? x : a.mn;
    a.mx = x > a.mx ? x : a.mx;
    const uint32_t l = (uint32_t)x, h = (uint32_t)(x >> 32);
    a.sl += l;
    a.sh += h;
    add96(a.a0, a.a1, a.a2, (unsigned long long)l * l);
    add96(a.b0, a.b1, a.b2, (unsigned long long)h * l);
    add96(a.c0, a.c1, a.c2, (unsigned long long)h * h);
}
// The canonical sums of a piecewise accumulator.
__device__ __forceinline__ Acc lacc_sums(const LAcc &a)
{
    Acc r;
    r.mn = a.mn;
    r.mx = a.mx;
    r.s1 = ((unsigned __int128)a.sh << 32) + a.sl;
    const unsigned __int128 A = ((unsigned __int128)a.a2 << 64) | ((unsigned long long)a.a1 << 32) | a.a0;
    const unsigned __int128 B = ((unsigned __int128)a.b2 << 64) | ((unsigned long long)a.b1 << 32) | a.b0;
    const unsigned __int128 C = ((unsigned __int128)a.c2 << 64) | ((unsigned long long)a.c1 << 32) | a.c0;
    unsigned __int128 lo = A;
    unsigned long long hi = 0;
    unsigned __int128 t = B << 33;  // 2^33 B: low 128 bits, then the bits above
    unsigned __int128 u = lo + t;
    hi += (unsigned long long)(B >> 95) + (u < t ? 1ull : 0ull);
    lo = u;
    t = C << 64;  // 2^64 C
    u = lo + t;
    hi += (unsigned long long)(C >> 64) + (u < t ? 1ull : 0ull);
    r.s2lo = u;
    r.s2hi = hi;
    return r;
}
__device__ __forceinline__ unsigned long long shfl_down64(unsigned long long v, int o)
{
    return __shfl_down_sync(0xffffffffu, v, o);
}
__device__ __forceinline__ unsigned __int128 shfl_down128(unsigned __int128 v, int o)
{
    unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
    lo = __shfl_down_sync(0xffffffffu, lo, o);
    hi = __shfl_down_sync(0xffffffffu, hi, o);
    return ((unsigned __int128)hi << 64) | lo;
}

// Block reduction; the result is valid in thread 0.  `sh` holds WARPS Accs.
__device__ void acc_block_reduce(Acc &a, Acc *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        Acc b;
        b.mn = shfl_down64(a.mn, o);
        b.mx = shfl_down64(a.mx, o);
        b.s1 = shfl_down128(a.s1, o);
        b.s2lo = shfl_down128(a.s2lo, o);
        b.s2hi = shfl_down64(a.s2hi, o);
        acc_merge(a, b);
    }
    if (lane == 0) sh[warp] = a;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < WARPS; w++) acc_merge(a, sh[w]);
    __syncthreads();
}

// Exact multiword atomic accumulation: each limb is added atomically and
// the carry out of a limb is added to the next one, so the final value is
// the exact sum whatever the order of the contributions.
__device__ void atomic_add_wide(unsigned long long *w, const unsigned long long *v, int nw)
{
    unsigned long long carry = 0;
    for (int i = 0; i < nw; i++) {
        unsigned long long add = v[i] + carry;
        unsigned long long c = (add < v[i]) ? 1ull : 0ull;
        if (add) {
            unsigned long long old = atomicAdd(&w[i], add);
            c += (old + add < old) ? 1ull : 0ull;
        }
        carry = c;
    }
}

// Rounds a 256-bit unsigned integer (4 limbs, little endian) to double.
__device__ double u256_to_double(const unsigned long long *x)
{
    int top = 3;
    while (top > 0 && x[top] == 0) top--;
    if (top == 0) return __ull2double_rn(x[0]);
    int lz = __clzll((long long)x[top]);
    unsigned long long hi = x[top], lo = x[top - 1];
    unsigned long long m = lz ? (hi << lz) | (lo >> (64 - lz)) : hi;
    unsigned long long rest = lz ? (lo << lz) : lo;
    for (int i = top - 2; i >= 0; i--) rest |= x[i];
    m |= rest ? 1ull : 0ull;  // sticky bit: 64 > 53 + 2 bits keeps the rounding exact
    return ldexp(__ull2double_rn(m), 64 * top - lz);
}

// mean of (key - min) and population variance from exact sums (Alg. 1's
// statistics, evaluated exactly and rounded once to double).
__device__ void moments_from_sums(unsigned long long n, unsigned long long mn,
                                  const unsigned long long s1w[2], const unsigned long long s2w[3],
                                  double *mean_d, double *var)
{
    unsigned __int128 s1 = ((unsigned __int128)s1w[1] << 64) | s1w[0];
    unsigned __int128 sum_d = s1 - (unsigned __int128)n * mn;  // exact, >= 0
    unsigned long long sd4[4] = {(unsigned long long)sum_d, (unsigned long long)(sum_d >> 64), 0, 0};
    *mean_d = u256_to_double(sd4) / (double)n;
    // n * S2 (S2 < 2^192, n < 2^32)
    unsigned long long a[4];
    unsigned __int128 c = 0;
    for (int i = 0; i < 3; i++) {
        c += (unsigned __int128)s2w[i] * n;
        a[i] = (unsigned long long)c;
        c >>= 64;
    }
    a[3] = (unsigned long long)c;
    // S1^2 (S1 < 2^128)
    unsigned long long p[4] = {0, 0, 0, 0};
    unsigned long long s1l[2] = {s1w[0], s1w[1]};
    for (int i = 0; i < 2; i++) {
        unsigned __int128 cc = 0;
        for (int j = 0; j < 2; j++) {
            cc += (unsigned __int128)s1l[i] * s1l[j] + p[i + j];
            p[i + j] = (unsigned long long)cc;
            cc >>= 64;
        }
        int q = i + 2;
        while (cc && q < 4) {
            cc += p[q];
            p[q] = (unsigned long long)cc;
            cc >>= 64;
            q++;
        }
    }
    // n * S2 - S1^2 >= 0 (Cauchy-Schwarz)
    unsigned long long r[4];
    unsigned long long borrow = 0;
    for (int i = 0; i < 4; i++) {
        unsigned long long t = a[i] - p[i];
        unsigned long long b1 = a[i] < p[i];
        unsigned long long t2 = t - borrow;
        unsigned long long b2 = t < borrow;
        r[i] = t2;
        borrow = b1 | b2;
    }
    double dn = (double)n;
    *var = borrow ? 0.0 : u256_to_double(r) / (dn * dn);
}

// ------------------------------------------------------------ bucket maps
// One definition serves the histogram and the scatter, so both passes
// compute bit-identical buckets.  Every map is monotone non-decreasing in
// the key, which is all the sort's exactness needs.
constexpr int PWL_BINS = 4096;  // learned map: bins of the normalised key's float bits
constexpr int PWL_MLP_OFF = 2 * PWL_P + 1;            // per-segment table: q[0..P], r[0..P), MLP table
constexpr int PWL_STRIDE = PWL_MLP_OFF + MLP_TABLE;
struct MapSm {
    unsigned long long mn;
    uint32_t kind, k, K, rshift, rmult, zsh;
    float zc, escale;
    float q[PWL_P + 1];          // learned map: breakpoints
    float r[PWL_P];              // learned map: 1 / (q[s+1] - q[s]), 0 for an empty piece
    uint8_t lo8[PWL_BINS];       // learned map: piece holding the lower edge of each bin
    uint32_t bin_lo, bin_sh;     // learned map: bin of u = (bits(u) - bin_lo) >> bin_sh, clamped
    uint32_t steps;              // learned map: 2^steps > most pieces a bin touches, minus one
    float mlp[MLP_TABLE];        // MLP map: w = omega^2, b, a = alpha^2 per unit, f0, inv
    unsigned long long bq[PWL_P + 1];  // exact-key map: breakpoint keys (slopes in r)
};

// fl32(d), round to nearest even, without the 64-bit conversion instruction:
// the top 32 significant bits with the lost bits OR-ed into the lowest one
// (a sticky bit below the guard bit keeps the rounding exact), converted,
// then scaled back by a power of two (exact).
__device__ __forceinline__ float u64_to_f32_rn(unsigned long long d)
{
    const uint32_t hi = (uint32_t)(d >> 32);
    const uint32_t s = hi ? 32u - (uint32_t)__clz((int)hi) : 0u;
    const unsigned long long lost = d & ((1ull << s) - 1ull);
    const uint32_t m = (uint32_t)(d >> s) | (lost ? 1u : 0u);
    return __fmul_rn(__uint2float_rn(m), __int_as_float((int)(127u + s) << 23));
}

// Learned map on the normalised key u = fl32(key - min) * 2^-E in [0, 1]:
// piece s = the last breakpoint q[s] <= u, linear interpolation inside the
// piece.  The piece is found from a bin table over the float bits of u
// (bins spread over [q[1], 1], the range the breakpoints occupy) that gives
// the piece at the bin's lower edge, then by binary lifting: steps
// strides 2^(steps-1), ..., 1, each taken if its breakpoint is still <= u
// (indices clamped to the last piece).  A bin touches at most 2^steps
// pieces, so the lifting always ends on the piece, with no data-dependent
// branch: the tile loops interleave the searches of all their keys.
__device__ __forceinline__ uint32_t pwl_bin(const MapSm &m, float u)
{
    const int c = ((int)__float_as_uint(u) - (int)m.bin_lo) >> m.bin_sh;
    return (uint32_t)min(max(c, 0), PWL_BINS - 1);
}
__device__ __forceinline__ uint32_t pwl_lift(const MapSm &m, float u, uint32_t lo, uint32_t st)
{
    const uint32_t j = min(lo + st, (uint32_t)PWL_P - 1u);
    return m.q[j] <= u ? j : lo;
}
__device__ __forceinline__ uint32_t pwl_finish(const MapSm &m, float u, uint32_t lo)
{
    float frac = __fmul_rn(__fsub_rn(u, m.q[lo]), m.r[lo]);
    frac = fminf(fmaxf(frac, 0.0f), 0x1.fffffep-1f);
    uint32_t w = __float2uint_rz(__fmul_rn(frac, (float)m.K));
    w = w < m.K ? w : m.K - 1;
    return lo * m.K + w;
}
__device__ __forceinline__ uint32_t pwl_bucket_u(const MapSm &m, float u)
{
    uint32_t lo = m.lo8[pwl_bin(m, u)];
    for (uint32_t st = m.steps ? 1u << (m.steps - 1) : 0u; st; st >>= 1) lo = pwl_lift(m, u, lo, st);
    return pwl_finish(m, u, lo);
}

// Exact-key learned map (MAP_SPLIT): piece s = the last breakpoint key
// bq[s] <= key (binary lifting over bq[1..P-1]); inside it the binary32
// interpolation relative to the piece's own lower key, frac = fl32(key -
// bq[s]) * r[s], clipped to [0, 1 - 2^-24]; bucket = s * K + floor(frac * K).
__device__ __forceinline__ uint32_t split_lift(const MapSm &m, unsigned long long key, uint32_t lo, uint32_t st)
{
    const uint32_t j = lo + st;  // <= P - 1: the strides sum to P - 1
    return m.bq[j] <= key ? j : lo;
}
__device__ __forceinline__ uint32_t split_finish(const MapSm &m, unsigned long long key, uint32_t s)
{
    const unsigned long long b = m.bq[s];
    float frac = __fmul_rn(u64_to_f32_rn(key > b ? key - b : 0ull), m.r[s]);
    frac = fminf(fmaxf(frac, 0.0f), 0x1.fffffep-1f);
    uint32_t w = __float2uint_rz(__fmul_rn(frac, (float)m.K));
    w = w < m.K ? w : m.K - 1;
    return s * m.K + w;
}
__device__ __forceinline__ uint32_t split_bucket(const MapSm &m, unsigned long long key)
{
    uint32_t lo = 0;
    for (uint32_t st = PWL_P / 2; st; st >>= 1) lo = split_lift(m, key, lo, st);
    return split_finish(m, key, lo);
}

// The scalar part of a map, held in registers by the tile loops (the tables
// of the learned map stay in shared memory).
struct MapK {
    unsigned long long mn;
    uint32_t kind, k, rshift, rmult, zsh;
    float zc, escale;
};

__device__ __forceinline__ MapK map_regs(const MapSm &m)
{
    MapK r;
    r.mn = m.mn;
    r.kind = m.kind;
    r.k = m.k;
    r.rshift = m.rshift;
    r.rmult = m.rmult;
    r.zsh = m.zsh;
    r.zc = m.zc;
    r.escale = m.escale;
    return r;
}

// MLP map: f(u) = sum_h a_h * clamp(w_h * u + b_h, 0, 1) with a_h, w_h >= 0
// (summed in unit order), g = (f(u) - f0) * inv clipped to [0, 1 - 2^-24],
// bucket = min(k - 1, trunc(g * k)).  Every step is a monotone binary32
// rounding of a monotone function, so the map is non-decreasing in u.
__device__ __forceinline__ float mlp_f(const float *t, float u)
{
    float f = 0.0f;
#pragma unroll 8
    for (int h = 0; h < MLP_H; h++) {
        const float c = fminf(fmaxf(__fadd_rn(__fmul_rn(t[h], u), t[MLP_H + h]), 0.0f), 1.0f);
        f = __fadd_rn(f, __fmul_rn(t[2 * MLP_H + h], c));
    }
    return f;
}
__device__ __forceinline__ uint32_t mlp_bucket_u(const float *t, float u, uint32_t k)
{
    const float g = __fmul_rn(__fsub_rn(mlp_f(t, u), t[3 * MLP_H]), t[3 * MLP_H + 1]);
    const float gc = fminf(fmaxf(g, 0.0f), 0x1.fffffep-1f);
    const uint32_t b = __float2uint_rz(__fmul_rn(gc, (float)k));
    return b < k ? b : k - 1;
}

// Eq. 1, the range map or the piecewise-linear map (not the MLP map).
__device__ __forceinline__ uint32_t map_key(const MapK &r, const MapSm &m, unsigned long long key)
{
    const unsigned long long d = key - r.mn;
    if (r.kind == MAP_Z) {
        // Eq. 1 with |z_min| = (mean - min)/sd: h = (key - min) * (k/4) / sd,
        // on d >> zsh (a 32-bit value; zc carries the 2^zsh back).  Keys
        // below mn go to bucket 0 and shifted values above 32 bits saturate
        // (statistics from a sample need not bound every key); both clamps
        // keep the map monotone, and neither acts when mn and the shift come
        // from the exact min and max.
        const unsigned long long e = key > r.mn ? d >> r.zsh : 0ull;
        const uint32_t e32 = e > 0xffffffffull ? 0xffffffffu : (uint32_t)e;
        const float f = __fmul_rn(__uint2float_rz(e32), r.zc);
        const uint32_t b = __float2uint_rz(f);
        return b < r.k ? b : r.k - 1;
    }
    if (r.kind == MAP_RANGE) {
        if (r.rmult == 0) return (uint32_t)d;  // range < k: counting map
        return __umulhi((uint32_t)(d >> r.rshift), r.rmult);
    }
    if (r.kind == MAP_SPLIT) return split_bucket(m, key);
    return pwl_bucket_u(m, __fmul_rn(u64_to_f32_rn(d), r.escale));
}

// The MLP map of a key (its own instantiation of the tile loops, so that the
// other maps' code keeps its registers).
__device__ __forceinline__ uint32_t map_key_mlp(const MapK &r, const MapSm &m, unsigned long long key)
{
    return mlp_bucket_u(m.mlp, __fmul_rn(u64_to_f32_rn(key - r.mn), r.escale), r.k);
}

// Any map, MLP included (inspection only).
__device__ __noinline__ uint32_t map_key_any(const MapSm &m, unsigned long long key)
{
    const MapK r = map_regs(m);
    return r.kind == MAP_MLP ? map_key_mlp(r, m, key) : map_key(r, m, key);
}

__device__ __forceinline__ uint32_t map_key(const MapSm &m, unsigned long long key)
{
    return map_key(map_regs(m), m, key);
}

// The buckets of NI keys of a tile loop (the MLP map when MLP, else the
// segment's map).  The learned map runs phase by phase over all NI keys --
// normalise and look up the bin, each lifting step, interpolate -- so the
// keys' shared-memory lookups overlap.  Same function as map_key.
template <int NI, bool MLP>
__device__ __forceinline__ void map_tile(const MapK &mk, const MapSm &m, const unsigned long long (&x)[NI],
                                         uint32_t (&b)[NI])
{
    if (MLP) {
#pragma unroll
        for (int i = 0; i < NI; i++) b[i] = map_key_mlp(mk, m, x[i]);
    } else if (mk.kind == MAP_PWL) {
        float u[NI];
#pragma unroll
        for (int i = 0; i < NI; i++) {
            u[i] = __fmul_rn(u64_to_f32_rn(x[i] - mk.mn), mk.escale);
            b[i] = m.lo8[pwl_bin(m, u[i])];
        }
        for (uint32_t st = m.steps ? 1u << (m.steps - 1) : 0u; st; st >>= 1) {
#pragma unroll
            for (int i = 0; i < NI; i++) b[i] = pwl_lift(m, u[i], b[i], st);
        }
#pragma unroll
        for (int i = 0; i < NI; i++) b[i] = pwl_finish(m, u[i], b[i]);
    } else if (mk.kind == MAP_SPLIT) {  // phase by phase over the NI keys, as above
#pragma unroll
        for (int i = 0; i < NI; i++) b[i] = 0;
        for (uint32_t st = PWL_P / 2; st; st >>= 1) {
#pragma unroll
            for (int i = 0; i < NI; i++) b[i] = split_lift(m, x[i], b[i], st);
        }
#pragma unroll
        for (int i = 0; i < NI; i++) b[i] = split_finish(m, x[i], b[i]);
    } else {
#pragma unroll
        for (int i = 0; i < NI; i++) b[i] = map_key(mk, m, x[i]);
    }
}

// Range map parameters: floor-like (d >> shift) * mult / 2^32, monotone,
// bucket(0) = 0, bucket(range) >= 1 for k >= 16, never above k - 1.
__device__ __forceinline__ void range_params(unsigned long long range, uint32_t k, uint32_t *rshift,
                                             uint32_t *rmult)
{
    if (range < k) {
        *rshift = 0;
        *rmult = 0;
        return;
    }
    uint32_t e = bitlen64(range);
    uint32_t sh = e > 32 ? e - 32 : 0;
    unsigned long long rr = range >> sh;
    *rshift = sh;
    *rmult = (uint32_t)((((unsigned long long)k) << 32) / (rr + 1));
}

// --------------------------------------------------------------- smem
// Lists built when a partition's children are classified; alias the tiles.
struct ChildList {
    uint32_t leaf_off[NB_MAX], leaf_len[NB_MAX];
    uint32_t med_off[NB_MAX], med_len[NB_MAX];
    uint32_t lg_off[NB_MAX], lg_len[NB_MAX], lg_need[NB_MAX], lg_slot[NB_MAX];
    uint32_t lg_chunks[NB_MAX], lg_k[NB_MAX];  // chunks, buckets
    uint32_t lg_sampled[NB_MAX];               // statistics from a sample
};

struct TileBuf {
    unsigned long long key[TILE + PAD];
    uint32_t val[TILE + PAD];
};
struct LeafBuf {
    unsigned long long key[LEAF_CAP + 2 * PAD];
    uint32_t val[LEAF_CAP + 2 * PAD];
};
// A leaf: its pairs, the leaf position of each staged pair (also the index
// array of the sorting network), and the sub-bucket counters.
struct LeafArea {
    LeafBuf leaf;
    uint16_t sidx[LEAF_CAP];
    __align__(16) uint32_t cnt[LEAF_M2_MAX + 1];
};

constexpr int KEY_STAGES = 3;  // key-only streams: tiles in flight per CTA
struct KeyRing {
    unsigned long long key[KEY_STAGES][TILE + PAD];
};

struct SmemTile {
    union {
        TileBuf buf[SC_STAGES];  // ring of streamed tiles (bulk-copy targets)
        KeyRing ring;     // key-only streams: three stages of keys
        LeafArea la;      // one leaf of up to LEAF_CAP pairs
        ChildList children;
    } u;
    uint16_t bkt[TILE];              // bucket of each staged element
    __align__(16) uint16_t wcnt[WARPS * NB_MAX];  // [warp][bucket] counts, then warp prefixes
    uint32_t tcount[NB_MAX];         // tile count per bucket
    uint32_t tstart[NB_MAX];         // tile-local exclusive start per bucket
    uint32_t gdelta[NB_MAX];         // global position - tile position (mod 2^32)
    uint32_t hist[NB_MAX];           // histogram
    uint32_t cursor[NB_MAX];         // running bucket cursor
    uint32_t bs[NB_MAX];             // bucket starts
    uint32_t wsum[WARPS + 1];
    Acc acc[WARPS];
    MapSm map;
    unsigned long long bar[KEY_STAGES];  // mbarriers of the tile buffers / key stages
    uint32_t task[8];
    uint32_t flag, flag2, n_leaf, n_med, n_large, n_large_ok, item_base, e_base, span_max;
    uint32_t drain;  // scatter: warps done with the current tile's buffer (0 between tiles)
    uint32_t local_base, local_n;  // leaves a medium partition kept for this CTA: items [base, base + n)
    unsigned long long red64[WARPS * 2];
};
static_assert(SC_STAGES <= KEY_STAGES, "one mbarrier per streamed tile buffer");
static_assert(sizeof(LeafArea) <= sizeof(TileBuf) * SC_STAGES, "a leaf fits the tile buffers");
static_assert(WARPS * (WARP_DISTINCT_MAX + 16) * 8 <= sizeof(LeafArea::cnt) && WARP_DISTINCT_MAX <= 32,
              "the warps' distinct-key tables fit the leaf's sub-bucket counters");
static_assert(offsetof(LeafArea, cnt) == offsetof(LeafArea, sidx) + sizeof(LeafArea::sidx) &&
                  WARPS * NB_MAX * 4 <= sizeof(LeafArea::sidx) + sizeof(LeafArea::cnt),
              "the stable leaf path's per-warp peer tables fit the contiguous sidx + cnt arrays");
static_assert(sizeof(KeyRing) <= sizeof(TileBuf) * SC_STAGES, "the key stages fit the tile buffers");
static_assert(sizeof(ChildList) <= sizeof(TileBuf) * SC_STAGES, "child lists fit the tile buffers");
static_assert(sizeof(SmemTile) <= 112 * 1024, "two CTAs per SM");
static_assert(IPT % 2 == 0, "the statistics loop takes the slots in pairs");
static_assert(LEAF_M2_MAX <= 8 * BLOCK && LEAF_M2_MAX % 8 == 0, "the leaf's sub-bucket scan: 8 counters a thread");

// ------------------------------------------------------------ block scan
// Exclusive scan of in[0..nb) into out (may alias); returns the total.
// nb <= BLOCK * MAXPER.
template <int MAXPER = NB_MAX / BLOCK>
__device__ uint32_t block_exclusive_scan(const uint32_t *in, uint32_t *out, uint32_t nb, uint32_t *wsum)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t per = (nb + BLOCK - 1) / BLOCK;
    const uint32_t base = threadIdx.x * per;
    uint32_t loc[MAXPER];
    uint32_t sum = 0;
#pragma unroll
    for (uint32_t j = 0; j < (uint32_t)MAXPER; j++) {
        if (j < per) {
            uint32_t idx = base + j;
            uint32_t v = idx < nb ? in[idx] : 0u;
            loc[j] = sum;
            sum += v;
        }
    }
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t wofs = 0, total = 0;
#pragma unroll
    for (int w = 0; w < WARPS; w++) {
        const uint32_t ws = wsum[w];
        wofs += w < warp ? ws : 0u;
        total += ws;
    }
    const uint32_t excl = wofs + x - sum;
#pragma unroll
    for (uint32_t j = 0; j < (uint32_t)MAXPER; j++) {
        if (j < per) {
            uint32_t idx = base + j;
            if (idx < nb) out[idx] = excl + loc[j];
        }
    }
    __syncthreads();
    return total;
}

// In-place exclusive scan of a[0..nb) (nb a multiple of 8, at most
// 8 * BLOCK; a 16-byte aligned): thread t owns a[8t, 8t + 8), read and
// written as two 16-byte vectors (a warp's vector accesses meet each bank
// once per 128 bytes), then one warp scan of the threads' sums and one
// barrier for the warps' totals.  a[nb] receives the total, which is also
// returned.
__device__ uint32_t block_exclusive_scan_vec8(uint32_t *a, uint32_t nb, uint32_t *wsum)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t b = threadIdx.x * 8u;
    uint4 x0 = make_uint4(0u, 0u, 0u, 0u), x1 = x0;
    if (b < nb) {
        x0 = reinterpret_cast<const uint4 *>(a + b)[0];
        x1 = reinterpret_cast<const uint4 *>(a + b)[1];
    }
    const uint32_t sum = x0.x + x0.y + x0.z + x0.w + x1.x + x1.y + x1.z + x1.w;
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t run = incl - sum, total = 0;
#pragma unroll
    for (int w = 0; w < WARPS; w++) {
        const uint32_t ws = wsum[w];
        run += w < warp ? ws : 0u;
        total += ws;
    }
    if (b < nb) {
        uint4 y0, y1;
        y0.x = run; run += x0.x;
        y0.y = run; run += x0.y;
        y0.z = run; run += x0.z;
        y0.w = run; run += x0.w;
        y1.x = run; run += x1.x;
        y1.y = run; run += x1.y;
        y1.z = run; run += x1.z;
        y1.w = run;
        reinterpret_cast<uint4 *>(a + b)[0] = y0;
        reinterpret_cast<uint4 *>(a + b)[1] = y1;
    }
    if (threadIdx.x == 0) a[nb] = total;
    __syncthreads();
    return total;
}

// Warp-wide min and max of 64-bit values by 32-bit reductions: the high
// words first, then the low words of the lanes that hold the extreme high
// word.  Every lane gets the result.
__device__ __forceinline__ void warp_minmax64(unsigned long long &mn, unsigned long long &mx)
{
    const uint32_t full = 0xffffffffu;
    const uint32_t hmin = __reduce_min_sync(full, (uint32_t)(mn >> 32));
    const uint32_t lmin = __reduce_min_sync(full, (uint32_t)(mn >> 32) == hmin ? (uint32_t)mn : 0xffffffffu);
    const uint32_t hmax = __reduce_max_sync(full, (uint32_t)(mx >> 32));
    const uint32_t lmax = __reduce_max_sync(full, (uint32_t)(mx >> 32) == hmax ? (uint32_t)mx : 0u);
    mn = ((unsigned long long)hmin << 32) | lmin;
    mx = ((unsigned long long)hmax << 32) | lmax;
}

// ------------------------------------------------------------ tile ranking
// Stable multisplit of one tile of N = BLOCK * NI elements, cnt of them
// valid.  Element (warp w, slot i, lane l) is the tile's element
// w*32*NI + i*32 + l, so (w, i, l) order is input order.  In each slot the
// warp's lanes with equal buckets are found from a per-warp shared-memory OR
// table of the buckets (rank_peers_tbl), or, where no room for the table
// exists, from NBITS ballots, one per bit of the bucket id (rank_peers);
// their rank is the count of earlier equal lanes plus the warp's running
// count for that bucket.  Warp prefixes per bucket and a block scan over
// buckets then give each element its position in the tile ordered by
// (bucket, input position).  Lanes past cnt are ignored (their bucket value
// does not matter).  The ranking in steps, so that a tile loop can place its
// own barriers:
//   rank_peers    (registers)  lanes of the warp with an equal bucket, per slot
//   rank_leaders  (smem)       the group leader reads and advances the warp's
//                              counter of the bucket (row warp of wcnt, so the
//                              leaders of one slot spread over the banks);
//                              wcnt must start at zero
//   -- barrier --
//   rank_scan                  per bucket: exclusive prefix over the warps
//                              (written back into wcnt), tile count, and the
//                              tile start by a block scan over the buckets;
//                              ends with a barrier
//   rank_place                 position = tile start + warp prefix + rank
// Bucket q's counters and prefixes belong to thread q / per (contiguous).
template <int NI, int NBITS>
__device__ __forceinline__ void rank_peers(const uint32_t (&b)[NI], uint32_t cnt, uint32_t (&peers)[NI])
{
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NI; i++) {
        const uint32_t bi = b[i];
        uint32_t p = 0xffffffffu;
#pragma unroll
        for (int bit = 0; bit < NBITS; bit++) {
            const uint32_t f = (bi >> bit) & 1u;
            const uint32_t bal = __ballot_sync(0xffffffffu, f);
            p &= f ? bal : ~bal;
        }
        // valid lanes of this slot, from the tile count
        const int first = warp * 32 * NI + i * 32;
        const int nv = (int)cnt - first;
        const uint32_t vmask = nv >= 32 ? 0xffffffffu : (nv <= 0 ? 0u : (1u << nv) - 1u);
        peers[i] = p & vmask;
    }
}

// rank_peers by a shared-memory table instead of ballots: each valid lane
// ORs its bit into the word of its bucket in the warp's own table of nb
// words (nb a multiple of 4, tbl 16-byte aligned, private to the warp), and
// reads the word back: the mask of the lanes with its bucket.  The lowest
// of them clears the word for the next slot.  A slot whose valid lanes all
// share one bucket (a run of equal keys) skips the table, so that its lanes
// do not serialise on one word.  The table is zeroed first; the warp's lanes
// must be done with whatever the table's memory held.
template <int NI>
__device__ __forceinline__ void rank_peers_tbl(const uint32_t (&b)[NI], uint32_t cnt, uint32_t *tbl, uint32_t nb,
                                               uint32_t (&peers)[NI])
{
    const uint32_t full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint4 *t4 = reinterpret_cast<uint4 *>(tbl);
    __syncwarp();
    for (uint32_t q = lane; q < nb / 4; q += 32) t4[q] = make_uint4(0u, 0u, 0u, 0u);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < NI; i++) {
        const int first = warp * 32 * NI + i * 32;
        const int nv = (int)cnt - first;
        const uint32_t vmask = nv >= 32 ? full : (nv <= 0 ? 0u : (1u << nv) - 1u);
        const bool valid = (vmask >> lane) & 1u;
        const uint32_t bi = b[i];
        const uint32_t b0 = __shfl_sync(full, bi, 0);
        if (__all_sync(full, !valid || bi == b0)) {  // one bucket (or no valid lane)
            peers[i] = vmask;
            continue;
        }
        if (valid) atomicOr(tbl + bi, 1u << lane);
        __syncwarp();
        const uint32_t pe = valid ? tbl[bi] : 0u;
        __syncwarp();
        if (valid && (pe & ((1u << lane) - 1u)) == 0u) tbl[bi] = 0u;
        __syncwarp();
        peers[i] = pe;
    }
}

template <int NI>
__device__ __forceinline__ void rank_leaders(const uint32_t (&b)[NI], const uint32_t (&peers)[NI],
                                             uint32_t (&pos)[NI], SmemTile &s)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < NI; i++) {
        const bool valid = (peers[i] >> lane) & 1u;
        const int leader = valid ? __ffs(peers[i]) - 1 : lane;
        uint32_t before = 0;
        if (valid && lane == leader) {
            uint16_t *c = s.wcnt + warp * NB_MAX + b[i];
            before = *c;
            *c = (uint16_t)(before + __popc(peers[i]));
        }
        before = __shfl_sync(0xffffffffu, before, leader);
        pos[i] = valid ? before + __popc(peers[i] & lt) : INVALID;
    }
}

// SCATTER: also advance the running cursors (gdelta = cursor - tile start,
// cursor += count); else store the counts in s.tcount.
template <bool SCATTER>
__device__ __forceinline__ void rank_scan(uint32_t nb, SmemTile &s)
{
    constexpr int MAXPER = NB_MAX / BLOCK;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t per = nb >= (uint32_t)BLOCK ? nb / BLOCK : 1u;
    const uint32_t q0 = threadIdx.x * per;
    uint32_t tot[MAXPER], loc[MAXPER];
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < MAXPER; j++) {
        tot[j] = 0;
        loc[j] = sum;
        if ((uint32_t)j < per && q0 + j < nb) {
            // column q of the [warp][bucket] counters: the warps' counts,
            // replaced by their exclusive prefix over the warps
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < WARPS; w++) {
                uint16_t *c = s.wcnt + w * NB_MAX + q0 + j;
                const uint32_t v = *c;
                *c = (uint16_t)run;
                run += v;
            }
            tot[j] = run;
            sum += run;
        }
    }
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s.wsum[warp] = x;
    __syncthreads();
    uint32_t wofs = 0;
#pragma unroll
    for (int w = 0; w < WARPS; w++) wofs += w < warp ? s.wsum[w] : 0u;
    const uint32_t excl = wofs + x - sum;
#pragma unroll
    for (int j = 0; j < MAXPER; j++) {
        if ((uint32_t)j < per && q0 + j < nb) {
            const uint32_t q = q0 + j, st = excl + loc[j];
            s.tstart[q] = st;
            if (SCATTER) {
                const uint32_t c = s.cursor[q];
                s.gdelta[q] = c - st;
                s.cursor[q] = c + tot[j];
            } else {
                s.tcount[q] = tot[j];
            }
        }
    }
    __syncthreads();
}

template <int NI>
__device__ __forceinline__ void rank_place(const uint32_t (&b)[NI], uint32_t (&pos)[NI], SmemTile &s)
{
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NI; i++)
        if (pos[i] != INVALID) pos[i] += s.tstart[b[i]] + s.wcnt[warp * NB_MAX + b[i]];
}

// Zeroes this warp's counter of every bucket (its own row of wcnt, eight
// counters per 16-byte store; nb is a multiple of 8).
__device__ __forceinline__ void rank_zero_warp(uint32_t nb, SmemTile &s)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint4 *row = reinterpret_cast<uint4 *>(s.wcnt + warp * NB_MAX);
    __syncwarp();
    for (uint32_t q = lane; q < nb / 8; q += 32) row[q] = make_uint4(0u, 0u, 0u, 0u);
    __syncwarp();
}

// ------------------------------------------------------------ bulk copies
// Tiles are staged in shared memory by the Blackwell bulk-copy engine
// (cp.async.bulk, completion counted on an mbarrier), double-buffered so
// that the next tile streams in while the current one is processed.
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
// Hint: bring the u16 entries [e0, e1) of arr into L2 with one bulk
// prefetch, trimmed to whole 16-byte pieces inside that range (the bulk
// prefetch wants a 16-byte aligned address and size; arr is 16-byte aligned).
__device__ __forceinline__ void bulk_prefetch_l2_inside(const uint16_t *arr, unsigned long long e0,
                                                        unsigned long long e1)
{
    const unsigned long long b0 = (e0 * 2ull + 15ull) & ~15ull, b1 = (e1 * 2ull) & ~15ull;
    if (b1 > b0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<const char *>(arr) + b0),
                     "r"((uint32_t)(b1 - b0))
                     : "memory");
}
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_arrive(unsigned long long *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// L2 policy for data read once (streamed tiles, leaves): evicted first, so
// that the stream does not push out the partly written output lines (the
// write fronts of the scatter), which would then be written to HBM in parts.
__device__ __forceinline__ unsigned long long policy_evict_first()
{
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ unsigned long long policy_evict_last()
{
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy_evict_first())
        : "memory");
}
// Scatter stores with an L2 policy (the write fronts).
__device__ __forceinline__ void st_front(uint64_t *p, unsigned long long v, unsigned long long pol)
{
    asm volatile("st.global.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_front(uint32_t *p, uint32_t v, unsigned long long pol)
{
    asm volatile("st.global.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}
// Hint: bring [src, src + bytes) into L2 (16-byte aligned address and size).
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
// Waits for the given phase parity of an mbarrier; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, unsigned long long limit_ns)
{
    const uint32_t a = smem_u32(bar);
    unsigned long long t0 = 0;
    for (uint32_t it = 0;; it++) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 15u) == 15u) {
            unsigned long long now = globaltimer();
            if (t0 == 0)
                t0 = now;
            else if (now - t0 > limit_ns)
                return false;
        }
    }
}

// ------------------------------------------------------------ sampling
// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) output for state x + 1 step.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x)
{
    unsigned long long z = x + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Position of sample i of m drawn from [0, len): one per stratum.
__device__ __forceinline__ unsigned long long sample_pos(unsigned long long seed, unsigned long long len,
                                                         unsigned long long m, unsigned long long i)
{
    unsigned long long lo = (i * len) / m;
    unsigned long long hi = ((i + 1) * len) / m;
    unsigned long long w = hi - lo;
    return lo + (w ? splitmix64(seed + i) % w : 0ull);
}

}  // namespace zs
