// zsort_tasks.cuh -- the tasks of the persistent zSort executor.
//
// Every (sub)array goes through the steps of Alg. 1: statistics (exact
// min, max, mean and population sd), the bucket map (Eq. 1, or the learned
// map, or the range map of the progress guard), a histogram, an exclusive
// scan for the bucket offsets, and a stable scatter; its buckets become the
// next level's (sub)arrays, or leaves finished in shared memory.
//   large (sub)arrays  -> per phase, one task per chunk of consecutive tiles;
//                         the histogram phase finds each chunk's offsets with
//                         a decoupled look-back across chunks, so the scatter
//                         phase streams its chunk with plain running cursors
//   medium (sub)arrays -> one task that runs every phase in one CTA
//   leaves             -> one task that sorts a group of small buckets in smem
// Tiles reach shared memory through double-buffered bulk copies (TMA).
#pragma once
#include "zsort_device.cuh"

namespace zs {

// ------------------------------------------------------------ queue
// Queue of a task type: leaves go to the leaf queue, all else to the
// partition queue.
__device__ __forceinline__ uint32_t queue_of(uint32_t type)
{
    return type == T_FINISH ? 1u : 0u;
}

// Reserves `count` consecutive entries of queue q (thread 0 only) and counts
// them as pending; returns their absolute index, INVALID when the queue is
// full (error recorded).
__device__ uint32_t q_reserve(const Params &P, uint32_t count, uint32_t q = 0)
{
    if (count == 0) return 0;
    uint32_t e = atomicAdd(&P.ctl->q_alloc[q], count);
    if (e + count > P.qcap) {
        set_error(P, ST_CAPACITY);
        return INVALID;
    }
    atomicAdd(&P.ctl->pending, count);
    return q * P.qcap + e;
}

// Writes an entry; it becomes visible once q_release_all() ran.
__device__ void q_write(const Params &P, uint32_t e, uint32_t type, uint32_t arg, uint32_t ntiles)
{
    Entry en;
    en.type = type;
    en.arg = arg;
    en.ntiles = ntiles;
    en.pad = 0;
    P.entries[e] = en;
    P.tnext[e] = 0;
    P.tdone[e] = 0;
}

// This call's queue epoch: ready words equal to it mark published entries.
__device__ __forceinline__ uint32_t call_epoch(const Params &P)
{
    return __ldcg(&P.ctl->epoch);
}

// Publishes entries [e, e+count): one fence, then the ready flags.
__device__ void q_release_all(const Params &P, uint32_t e, uint32_t count)
{
    __threadfence();
    const uint32_t ep = call_epoch(P);
    for (uint32_t i = 0; i < count; i++) st_relaxed(&P.ready[e + i], ep);
}

// Warp 0 of a CTA (all 32 lanes): claims the next tiles of a published entry,
// partition queue first, else the leaf queue.  One round trip reads the
// error word and every queue's head (one lane each); then the lanes look at
// 32 entries from a queue's head at once: lane i reads entry head + i's
// ready word (against this call's epoch `ep`) and claim counter, the first
// entry with tiles left is claimed with one atomic, and the head jumps over
// the leading run of published entries whose tiles are all claimed (one
// compare-and-swap).  Lane 0 writes out = {type, arg, first tile, entry,
// ntiles, count}; type T_NONE when all work is done or an error was
// recorded.  A wait without any progress anywhere for longer than P.wait_ns
// records ST_TIMEOUT.
__device__ void dequeue(const Params &P, uint32_t ep, uint32_t *out)
{
    const uint32_t full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    Ctl *C = P.ctl;
    const uint32_t qcap = P.qcap, nctas = P.nctas;
    unsigned long long last = 0, t0 = 0;
    bool waited = false;
    if (lane == 0) out[0] = T_NONE;
    for (;;) {
        uint32_t w = 0;
        if (lane == 0)
            w = ld_relaxed(&C->error);
        else if (lane <= QUEUES)
            w = ld_relaxed(&C->q_head[lane - 1]);
        if (__shfl_sync(full, w, 0)) return;
        for (uint32_t q = 0; q < (uint32_t)QUEUES; q++) {
            const uint32_t h = __shfl_sync(full, w, (int)q + 1);
            uint32_t next_head = h;
            for (uint32_t base = h; base < qcap; base += 32) {
                const uint32_t i = base + lane;
                const uint32_t e = q * qcap + i;
                const bool rdy = i < qcap && ld_acquire(&P.ready[e]) == ep;
                uint32_t type = 0, arg = 0, nt = 0, tn = 0;
                if (rdy) {
                    const uint4 en = __ldcg(reinterpret_cast<const uint4 *>(P.entries + e));
                    type = en.x;
                    arg = en.y;
                    nt = en.z;
                    tn = ld_relaxed(&P.tnext[e]);
                }
                const uint32_t mr = __ballot_sync(full, rdy);
                // the head may pass the leading run of published entries
                // whose tiles are all claimed (seen here, even if this window
                // still has tiles to give)
                const uint32_t spent = __ballot_sync(full, rdy && tn >= nt);
                if (next_head == base) next_head = base + (spent == full ? 32u : (uint32_t)(__ffs(~spent) - 1));
                uint32_t m = __ballot_sync(full, rdy && tn < nt);
                // CTAs start at different entries of the window (by block
                // index), so that they do not all race for the first one; the
                // tiles of one entry are still handed out in order
                const uint32_t rot = blockIdx.x & 31u;
                m = rot ? (m >> rot) | (m << (32u - rot)) : m;
                while (m) {
                    const int f = (int)((__ffs(m) - 1 + rot) & 31u);
                    uint32_t got = 0;
                    if (lane == f) {
                        // leaves a few at a time, so that each can be
                        // prefetched while its predecessor is sorted (about a
                        // quarter of what the entry has left, at most 8); the
                        // statistics and scatter chunks (which wait on no
                        // other chunk) two at a time while many remain.  Never
                        // histogram chunks: the look-back needs every
                        // predecessor chunk running or done.
                        uint32_t claim = 1u;
                        if (type == T_FINISH)
                            claim = min(8u, max(1u, (nt - tn + 3u) / 4u));
                        else if ((type == T_LSTATS || type == T_LSCATTER) && nt - tn >= 4u * nctas)
                            claim = 2u;
                        const uint32_t t = atomicAdd(&P.tnext[e], claim);
                        if (t < nt) {
                            out[0] = type;
                            out[1] = arg;
                            out[2] = t;
                            out[3] = e;
                            out[4] = nt;
                            out[5] = min(claim, nt - t);
                            got = 1;
                        }
                    }
                    if (__shfl_sync(full, got, f)) {
                        if (lane == 0 && next_head > h) atomicCAS(&C->q_head[q], h, next_head);
                        return;
                    }
                    m &= m - 1;
                }
                // every published entry of this window is now fully claimed
                if (mr != full) break;  // an unpublished entry: look again later
            }
            if (lane == 0 && next_head > h) atomicCAS(&C->q_head[q], h, next_head);
        }
        // nothing to claim: all work done, or wait for more
        uint32_t stop = 0;
        if (lane == 0) {
            if (ld_acquire(&C->pending) == 0) {
                stop = 1;
            } else {
                const unsigned long long pr = ld_relaxed64(&C->progress), now = globaltimer();
                if (!waited || pr != last) {
                    waited = true;
                    last = pr;
                    t0 = now;
                } else if (now - t0 > P.wait_ns) {
                    set_error(P, ST_TIMEOUT);
                    stop = 1;
                }
            }
        }
        if (__shfl_sync(full, stop, 0)) return;
        __nanosleep(128);
    }
}

// Work items and segment fields are written by other CTAs during the call:
// read them at L2 (ld.global.cg), never from a possibly stale L1 line.
__device__ __forceinline__ Item load_item(const Params &P, uint32_t idx)
{
    const Item *p = P.items + idx;
    Item it;
    it.off = __ldcg(&p->off);
    it.len = __ldcg(&p->len);
    uint32_t bl = __ldcg(reinterpret_cast<const uint32_t *>(&p->buf));
    it.buf = (uint16_t)(bl & 0xffffu);
    it.level = (uint16_t)(bl >> 16);
    return it;
}

// Bytes of one element: key and payload, or the key alone.
__device__ __forceinline__ unsigned long long elem_bytes(const Params &P)
{
    return P.kv ? 12ull : 8ull;
}

__device__ __forceinline__ uint64_t *keys_of(const Params &P, uint32_t buf)
{
    return buf ? P.skeys : P.ukeys;
}
__device__ __forceinline__ uint32_t *vals_of(const Params &P, uint32_t buf)
{
    return buf ? P.svals : P.uvals;
}
// Bulk copies need 16-byte aligned bases: always true of the scratch arrays.
__device__ __forceinline__ bool bulk_ok(const Params &P, uint32_t buf)
{
    return buf || P.user_aligned;
}

// Buckets of one partition pass: enough for leaf_target elements per bucket.
__device__ __forceinline__ uint32_t choose_k(const Params &P, uint32_t len)
{
    uint32_t k = pow2ceil32((len + P.leaf_target - 1) / P.leaf_target);
    k = k < (uint32_t)MIN_K ? (uint32_t)MIN_K : k;
    return k > P.kmax ? P.kmax : k;
}

// A large (sub)array of len elements with k buckets at depth level learns
// its map (the statistics decide later whether Eq. 1 applies at all).
__device__ __forceinline__ bool wants_learned_map(const Params &P, uint32_t len, uint32_t k, uint32_t level)
{
    return P.mapper >= 1 && len >= P.learn_min && P.sample <= len && k >= (uint32_t)PWL_P && level < P.guard_level;
}

// Takes a training slot for a new large (sub)array (any thread): INVALID if
// none is left, then the (sub)array keeps Eq. 1.
__device__ __forceinline__ uint32_t take_train_slot(const Params &P, uint32_t len, uint32_t k, uint32_t level)
{
    if (!wants_learned_map(P, len, k, level)) return INVALID;
    const uint32_t slot = atomicAdd(&P.ctl->train_alloc, 1u);
    return slot < P.traincap ? slot : INVALID;
}

// Tiles per chunk task of a large (sub)array of len elements: chunks in
// proportion to its share of the call's n, about chunks_per_cta (default 8)
// per CTA of the grid over a whole level (so one level needs about
// chunks_per_cta * nctas look-back rows in all; more chunks shorten the tail
// of a phase), at least four tiles each.
__device__ __forceinline__ uint32_t choose_chunk_tiles(const Params &P, uint32_t tiles, uint32_t len)
{
    const unsigned long long want =
        ((unsigned long long)P.chunks_per_cta * P.nctas * len + P.n - 1) / P.n;
    const uint32_t target = (uint32_t)(want < 1 ? 1 : want);
    const uint32_t ct = (tiles + target - 1) / target;
    return ct < 4u ? 4u : ct;
}

// Chunk geometry of a large (sub)array of `tiles` tiles: chunks of ct tiles,
// except that a (sub)array spanning more than two rounds of chunks over the
// grid has its last round's worth of tiles (nctas x ct) cut into chunks of
// a quarter of that size, so that its phases end with short tasks and the
// CTAs finish them close together.
struct ChunkPlan {
    uint32_t ct, ct_small, big, chunks;
};
__device__ __forceinline__ ChunkPlan chunk_plan(const Params &P, uint32_t tiles, uint32_t len)
{
    ChunkPlan c;
    c.ct = choose_chunk_tiles(P, tiles, len);
    const uint32_t whole = (tiles + c.ct - 1) / c.ct;
    c.ct_small = c.ct;
    c.big = whole;
    c.chunks = whole;
    const uint32_t small = max(4u, c.ct / 4u);
    if (whole > 2u * P.nctas && small < c.ct) {
        const uint32_t tail = P.nctas * c.ct;  // below tiles, as whole > 2 nctas
        c.big = (tiles - tail) / c.ct;
        const uint32_t rest = tiles - c.big * c.ct;
        c.ct_small = small;
        c.chunks = c.big + (rest + small - 1) / small;
    }
    return c;
}

// Fills the map for a (sub)array from its exact sums: Eq. 1 (z-score) unless
// the depth reached the guard level or the parent's partition made poor
// progress (force_range), in which cases the exact range map.
__device__ void map_from_sums(const Params &P, unsigned long long n, unsigned long long mn,
                              unsigned long long mx, const unsigned long long s1[2],
                              const unsigned long long s2[3], uint32_t k, uint32_t level, bool force_range,
                              MapSm &m, double *mean_d, double *sd)
{
    double var;
    moments_from_sums(n, mn, s1, s2, mean_d, &var);
    *sd = sqrt(var);
    m.mn = mn;
    m.k = k;
    m.K = k >= PWL_P ? k / PWL_P : 1;
    unsigned long long range = mx - mn;
    m.escale = __int_as_float((127 - (int)bitlen64(range)) << 23);  // 2^-bitlen(range)
    m.zc = 0.0f;
    m.zsh = 0;
    m.rshift = 0;
    m.rmult = 0;
    if (level >= P.guard_level || force_range || !(*sd > 0.0)) {
        m.kind = MAP_RANGE;
        range_params(range, k, &m.rshift, &m.rmult);
        atomicAdd(&P.ctl->n_guard, 1ull);
    } else {
        // scale = k/4 (Alg. 1); |z_min| = (mean - min)/sd cancels the mean.
        const uint32_t e = bitlen64(range);
        m.kind = MAP_Z;
        m.zsh = e > 32 ? e - 32 : 0;
        m.zc = (float)(((double)k / 4.0) / *sd * (double)(1ull << m.zsh));
    }
}

__device__ void record_top(const Params &P, const MapSm &m, unsigned long long mn, unsigned long long mx,
                           double mean_d, double sd)
{
    Ctl *C = P.ctl;
    C->top_mean_d = mean_d;
    C->top_sd = sd;
    C->top_min = mn;
    C->top_max = mx;
    C->top_k = m.k;
    C->top_map = m.kind;
}

__device__ void note_level(const Params &P, uint32_t level)
{
    atomicMax(&P.ctl->max_level, (unsigned long long)level);
}

// Bin table of the learned map (all threads; q[0..P] in place): bins of
// equal width in the float bits of u between q[1] and 1 (below q[1] every
// key is in piece 0), lo8[c] = the last piece s whose breakpoint q[s] lies
// at or below the lower edge of bin c, and the lifting steps for the most
// pieces one bin touches (its upper edge is the next bin's lower edge, or 1).
__device__ uint32_t pwl_piece_at(const MapSm &m, float edge)
{
    uint32_t lo = 0, hi = PWL_P - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (m.q[mid] <= edge)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}
__device__ void build_pwl_bins(MapSm &m, uint32_t *scratch)
{
    const uint32_t top = __float_as_uint(1.0f);
    const uint32_t lo_bits = min(__float_as_uint(m.q[1]), top);
    uint32_t sh = 0;
    while (((top - lo_bits) >> sh) >= (uint32_t)PWL_BINS) sh++;
    if (threadIdx.x == 0) {
        m.bin_lo = lo_bits;
        m.bin_sh = sh;
        *scratch = 0;
    }
    __syncthreads();
    uint32_t span = 0;
    for (uint32_t c = threadIdx.x; c < (uint32_t)PWL_BINS; c += BLOCK) {
        const float lo_edge = c == 0 ? 0.0f : __uint_as_float(min(lo_bits + (c << sh), top));
        const unsigned long long up = (unsigned long long)lo_bits + ((unsigned long long)(c + 1) << sh);
        const float hi_edge = c + 1 == (uint32_t)PWL_BINS || up >= top ? 1.0f : __uint_as_float((uint32_t)up);
        const uint32_t a = pwl_piece_at(m, lo_edge);
        m.lo8[c] = (uint8_t)a;
        span = max(span, pwl_piece_at(m, hi_edge) - a);
    }
    span = __reduce_max_sync(0xffffffffu, span);
    if ((threadIdx.x & 31) == 0) atomicMax(scratch, span);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t st = 0;
        while ((1u << st) <= *scratch) st++;
        m.steps = st;
    }
}

// Loads a large segment's map into shared memory (all threads).
__device__ void load_seg_map(const Params &P, uint32_t sid, SmemTile &s)
{
    const Seg *S = &P.segs[sid];
    const uint32_t kind = __ldcg(&S->kind);
    if (threadIdx.x == 0) {
        s.map.mn = __ldcg(&S->mn);
        s.map.kind = kind;
        s.map.k = __ldcg(&S->k);
        s.map.K = s.map.k >= PWL_P ? s.map.k / PWL_P : 1;
        s.map.zc = __ldcg(&S->zc);
        s.map.zsh = __ldcg(&S->zsh);
        s.map.escale = __ldcg(&S->escale);
        s.map.rshift = __ldcg(&S->rshift);
        s.map.rmult = __ldcg(&S->rmult);
    }
    if (kind == MAP_MLP) {
        const float *t = P.pwl + (size_t)sid * PWL_STRIDE + PWL_MLP_OFF;
        for (int j = threadIdx.x; j < MLP_TABLE; j += BLOCK) s.map.mlp[j] = __ldcg(t + j);
    }
    if (kind == MAP_PWL) {
        const float *t = P.pwl + (size_t)sid * PWL_STRIDE;
        for (int j = threadIdx.x; j <= PWL_P; j += BLOCK) s.map.q[j] = __ldcg(t + j);
        for (int j = threadIdx.x; j < PWL_P; j += BLOCK) s.map.r[j] = __ldcg(t + PWL_P + 1 + j);
        __syncthreads();
        build_pwl_bins(s.map, &s.span_max);
    }
    if (kind == MAP_SPLIT) {  // breakpoint keys in the training slot's selection area, slopes in the table
        const unsigned long long *bq =
            P.trainbuf + (size_t)__ldcg(&S->train_slot) * 2 * SAMPLE_MAX + SAMPLE_MAX;
        const float *t = P.pwl + (size_t)sid * PWL_STRIDE;
        for (int j = threadIdx.x; j <= PWL_P; j += BLOCK) s.map.bq[j] = __ldcg(bq + j);
        for (int j = threadIdx.x; j < PWL_P; j += BLOCK) s.map.r[j] = __ldcg(t + PWL_P + 1 + j);
    }
    __syncthreads();
}

// ------------------------------------------------------------ tile streaming
// Per-thread copy (identical in every thread) of how often each tile
// mbarrier has completed, which gives the parity to wait for.
struct Pipe {
    uint32_t uses[KEY_STAGES];
};

// Thread 0: bulk copies of elements [a, a+cnt) of keys (and vals) into
// tile buffer w.  Copies start and end on 16-byte boundaries inside the
// arrays ([0, n) rounded down), so the element a sits at index a & 1 of the
// key buffer and a & 3 of the value buffer; up to 3 trailing elements past
// the last full 16 bytes of the array are left to stream_fix_tail().
template <bool VALS>
__device__ void stream_issue(const Params &P, SmemTile &s, int w, const uint64_t *keys, const uint32_t *vals,
                             unsigned long long a, uint32_t cnt)
{
    const unsigned long long a0 = a & ~1ull;
    const unsigned long long a1 = min((a + cnt + 1) & ~1ull, P.n & ~1ull);
    const uint32_t bk = a1 > a0 ? (uint32_t)(a1 - a0) * 8u : 0u;
    uint32_t bv = 0;
    unsigned long long b0 = 0;
    if (VALS && P.kv) {
        b0 = a & ~3ull;
        const unsigned long long b1 = min((a + cnt + 3) & ~3ull, P.n & ~3ull);
        bv = b1 > b0 ? (uint32_t)(b1 - b0) * 4u : 0u;
    }
    mbar_expect_arrive(&s.bar[w], bk + bv);
    if (bk) bulk_g2s(s.u.buf[w].key, keys + a0, bk, &s.bar[w]);
    if (VALS && bv) bulk_g2s(s.u.buf[w].val, vals + b0, bv, &s.bar[w]);
}

template <bool VALS>
__device__ void stream_fix_tail(const Params &P, unsigned long long *sk, uint32_t *sv, const uint64_t *keys,
                                const uint32_t *vals, unsigned long long a, uint32_t cnt)
{
    const unsigned long long end = a + cnt;
    const unsigned long long ka = max(a, P.n & ~1ull);
    for (unsigned long long e = ka + threadIdx.x; e < end; e += BLOCK) sk[e - a] = __ldcg(keys + e);
    if (VALS && P.kv) {
        const unsigned long long va = max(a, P.n & ~3ull);
        for (unsigned long long e = va + threadIdx.x; e < end; e += BLOCK) sv[e - a] = __ldcg(vals + e);
    }
}

// Thread 0: bulk copy of keys [a, a+cnt) into key stage w (16-byte aligned
// span inside the array, as stream_issue; the tail is left to plain loads).
__device__ void stream_issue_keys(const Params &P, SmemTile &s, int w, const uint64_t *keys, unsigned long long a,
                                  uint32_t cnt)
{
    const unsigned long long a0 = a & ~1ull;
    const unsigned long long a1 = min((a + cnt + 1) & ~1ull, P.n & ~1ull);
    const uint32_t bk = a1 > a0 ? (uint32_t)(a1 - a0) * 8u : 0u;
    mbar_expect_arrive(&s.bar[w], bk);
    if (bk) bulk_g2s(s.u.ring.key[w], keys + a0, bk, &s.bar[w]);
}

// Streams the keys [start, start+len) through a ring of KEY_STAGES stages
// (two tiles in flight while one is processed) and calls body(tile, cnt,
// keys_smem, nullptr) for each tile, in order, with all threads; the body
// must not need a barrier of its own.  One barrier a tile: once every thread
// is past it, every thread has left the previous tile, whose stage then
// takes the copy of the tile after next.  Returns false (error recorded) if
// a bulk copy did not complete.
template <bool VALS, class Body>
__device__ bool stream_tiles(const Params &P, SmemTile &s, Pipe &pp, const uint64_t *keys, const uint32_t *,
                             bool bulk, unsigned long long start, unsigned long long len, Body body)
{
    static_assert(!VALS, "streams of payloads go through the scatter's own loop");
    const uint32_t tile = P.tile;  // 256 * ipt keys, at most TILE
    const uint32_t nt = (uint32_t)((len + tile - 1) / tile);
    if (nt == 0) return true;
    auto tile_len = [&](uint32_t t) {
        return (uint32_t)min((unsigned long long)tile, len - (unsigned long long)t * tile);
    };
    if (bulk && threadIdx.x == 0)
        for (uint32_t t = 0; t < KEY_STAGES - 1 && t < nt; t++)
            stream_issue_keys(P, s, (int)t, keys, start + (unsigned long long)t * tile, tile_len(t));
    for (uint32_t t = 0; t < nt; t++) {
        const int w = (int)(t % KEY_STAGES);
        const unsigned long long a = start + (unsigned long long)t * tile;
        const uint32_t cnt = tile_len(t);
        unsigned long long *sk;
        if (bulk) {
            sk = s.u.ring.key[w] + (a & 1ull);
            const bool ok = mbar_wait(&s.bar[w], pp.uses[w] & 1u, P.wait_ns);
            pp.uses[w]++;
            if (__syncthreads_or(!ok)) {  // CTA-uniform: every thread leaves together
                // one more bounded wait for every copy that may be in flight
                mbar_wait(&s.bar[w], (pp.uses[w] - 1u) & 1u, P.wait_ns);
                for (uint32_t tn = t + 1; tn < nt && tn < t + KEY_STAGES - 1; tn++) {
                    const int wn = (int)(tn % KEY_STAGES);
                    mbar_wait(&s.bar[wn], pp.uses[wn] & 1u, P.wait_ns);
                }
                set_error(P, ST_TIMEOUT);
                return false;
            }
            // every thread has left tile t - 1: its stage takes tile t + 2
            if (t + KEY_STAGES - 1 < nt && threadIdx.x == 0) {
                const uint32_t tn = t + KEY_STAGES - 1;
                stream_issue_keys(P, s, (int)(tn % KEY_STAGES), keys, start + (unsigned long long)tn * tile,
                                  tile_len(tn));
            }
            if (a + cnt > (P.n & ~1ull)) {  // the array's last key: a plain load (uniform branch)
                for (unsigned long long e = max(a, P.n & ~1ull) + threadIdx.x; e < a + cnt; e += BLOCK)
                    sk[e - a] = __ldcg(keys + e);
                __syncthreads();
            }
        } else {
            // the stage last held tile t - 3; every thread left it before the
            // previous tile's barrier
            sk = s.u.ring.key[w];
            for (uint32_t i = threadIdx.x; i < cnt; i += BLOCK) sk[i] = __ldcg(keys + a + i);
            __syncthreads();
        }
        body(t, cnt, sk, (uint32_t *)nullptr);
        fence_proxy_async();  // this thread's smem accesses before the stage's next bulk write
    }
    __syncthreads();  // the last tile's body is complete for the caller
    return true;
}

// Element of slot i of this thread in a tile of NI items per thread: warp w
// holds the 32 * NI consecutive elements from w * 32 * NI on.
template <int NI = IPT>
__device__ __forceinline__ uint32_t slot_index(int i)
{
    return (threadIdx.x >> 5) * (32 * NI) + i * 32 + (threadIdx.x & 31);
}
__device__ __forceinline__ uint32_t leaf_slot(int i)
{
    return (threadIdx.x >> 5) * LEAF_SPAN + i * 32 + (threadIdx.x & 31);
}

// ------------------------------------------------------------ tile bodies
// Exact sums of the tile's keys into a per-thread accumulator.
template <int NI>
__device__ __forceinline__ void body_stats(LAcc &a, LAcc &b, uint32_t cnt, const unsigned long long *sk)
{
    static_assert(NI % 2 == 0, "the slots are taken in pairs");
    // two accumulators: the even and the odd slots form independent chains
#pragma unroll
    for (int i = 0; i < NI; i += 2) {
        const uint32_t p = slot_index<NI>(i), p1 = slot_index<NI>(i + 1);
        if (p < cnt) lacc_key(a, sk[p]);
        if (p1 < cnt) lacc_key(b, sk[p1]);
    }
}

// Histogram of the tile's buckets into s.hist: one shared-memory atomic per
// key, except when a whole warp slot shares one bucket (duplicate runs).
template <int NI, bool MLP, bool IDS = false>
__device__ __forceinline__ void body_hist(SmemTile &s, const MapK &mk, uint32_t cnt, const unsigned long long *sk,
                                          uint16_t *ids = nullptr)
{
    const int lane = threadIdx.x & 31;
    unsigned long long x[NI];
    uint32_t bb[NI];
#pragma unroll
    for (int i = 0; i < NI; i++) {
        const uint32_t p = slot_index<NI>(i);
        x[i] = p < cnt ? sk[p] : mk.mn;
    }
    map_tile<NI, MLP>(mk, s.map, x, bb);
    if (IDS) {  // a learned map's buckets, for the scatter to read back
#pragma unroll
        for (int i = 0; i < NI; i++)
            if (slot_index<NI>(i) < cnt) __stcg(ids + slot_index<NI>(i), (unsigned short)bb[i]);
    }
#pragma unroll
    for (int i = 0; i < NI; i++) {
        const uint32_t b = slot_index<NI>(i) >= cnt ? INVALID : bb[i];
        const uint32_t b0 = __shfl_sync(0xffffffffu, b, 0);
        if (__all_sync(0xffffffffu, b == b0)) {
            if (lane == 0 && b0 != INVALID) atomicAdd(&s.hist[b0], 32u);
        } else if (b != INVALID) {
            atomicAdd(&s.hist[b], 1u);
        }
    }
}

// Histogram of [start, start+len) into s.hist (its own instantiation per map
// family, so that each keeps its registers).
// A learned map (piecewise-linear or MLP) also writes every key's bucket to
// ids[start, start+len): the scatter of the same chunk reads them back
// instead of evaluating the map a second time.
template <int NI, bool MLP>
__device__ __noinline__ void hist_stream(const Params &P, SmemTile &s, Pipe &pp, const uint64_t *src, bool bulk,
                                         unsigned long long start, unsigned long long len, const MapK mk)
{
    stream_tiles<false>(P, s, pp, src, nullptr, bulk, start, len,
                        [&](uint32_t t, uint32_t cnt, unsigned long long *sk, uint32_t *) {
                            body_hist<NI, MLP, true>(s, mk, cnt, sk, P.ids + start + (unsigned long long)t * P.tile);
                        });
}

// The Eq. 1 or range-map histogram of a stream (no bucket ids written),
// inlined into its task at each items-per-thread choice.
#define ZS_HIST_PLAIN(NI, src, bulk, start, len)                                                        \
    stream_tiles<false>(P, s, pp, src, nullptr, bulk, start, len,                                       \
                        [&](uint32_t, uint32_t cnt, unsigned long long *sk, uint32_t *) {               \
                            body_hist<NI, false>(s, mk, cnt, sk);                                       \
                        })
// The exact sums of a stream into the task's two accumulators la, la2 (kept
// in registers: the loop is inlined into the task).
#define ZS_STATS(NI, src, bulk, start, len)                                                             \
    stream_tiles<false>(P, s, pp, src, nullptr, bulk, start, len,                                       \
                        [&](uint32_t, uint32_t cnt, unsigned long long *sk, uint32_t *) {               \
                            body_stats<NI>(la, la2, cnt, sk);                                           \
                        })

// Stable scatter of [start, start+len) of a (sub)array whose map is in s.map
// and whose running bucket cursors are in s.cursor.  Per tile: rank the
// pairs by (bucket, position) with the warps' peer tables (ballots where a
// table does not fit), stage them in that order in the
// tile's own buffer with their buckets, then write each bucket's run at its
// cursor (coalesced within runs; a staged bucket is cheaper to read back
// than any map is to recompute).  Tiles stream through a ring of SC_STAGES
// buffers: the last warp to finish writing tile t out (a counter in shared
// memory, no CTA barrier) refills its buffer with the bulk copy of tile
// t + SC_STAGES, which then has the whole of tile t + 1 to arrive.  Where
// the buckets come from the histogram pass (IDS), the same warp also
// prefetches that tile's bucket ids into L2, since their loads at the top
// of the tile no longer wait behind a copy.  Each warp clears its own
// bucket counters.
template <int NI, bool IDS, bool KV>
__device__ __noinline__ void scatter_stream(const Params &P, SmemTile &s, Pipe &pp, const uint64_t *srck,
                                            const uint32_t *srcv, bool bulk, unsigned long long start,
                                            unsigned long long len, uint64_t *dstk, uint32_t *dstv, uint32_t seglen)
{
    constexpr uint32_t TL = (uint32_t)(BLOCK * NI);  // pairs per tile
    const uint32_t nt = (uint32_t)((len + TL - 1) / TL);
    if (nt == 0) return;
    const MapK mk = map_regs(s.map);
    const uint32_t k = mk.k;
    constexpr bool kv = KV;  // payloads move with the keys
    // the runs written per tile end inside lines that the next tile (or the
    // neighbouring chunk) completes: keep those lines in L2 until then
    const unsigned long long pol_front = policy_evict_last();
    auto tile_cnt = [&](uint32_t t) {
        return (uint32_t)min((unsigned long long)TL, len - (unsigned long long)t * TL);
    };
    // a warp's peer table (k words, 16 bytes in) must fit its span of the
    // tile's keys: always at 12 items per thread, for k <= 256 at 8
    const bool table = 8u * 32u * NI >= 16u + 4u * k;
    rank_zero_warp(k, s);
    if (bulk && threadIdx.x == 0)
        for (uint32_t t = 0; t < SC_STAGES && t < nt; t++)
            stream_issue<KV>(P, s, (int)t, srck, srcv, start + (unsigned long long)t * TL, tile_cnt(t));
    bool err = false;
    for (uint32_t t = 0; t < nt; t++) {
        const int w = (int)(t % SC_STAGES);
        const unsigned long long a = start + (unsigned long long)t * TL;
        const uint32_t cnt = tile_cnt(t);
        unsigned long long *sk;
        uint32_t *sv;
        bool ok = true;
        uint32_t b[NI];
        if (IDS) {  // the histogram pass's buckets: loads in flight during the tile's wait
#pragma unroll
            for (int i = 0; i < NI; i++) {
                const uint32_t p = slot_index<NI>(i);
                b[i] = p < cnt ? (uint32_t)__ldcg(reinterpret_cast<const unsigned short *>(P.ids) + a + p) : 0u;
            }
        }
        if (bulk) {
            sk = s.u.buf[w].key + (a & 1ull);
            sv = s.u.buf[w].val + (a & 3ull);
            ok = mbar_wait(&s.bar[w], pp.uses[w] & 1u, P.wait_ns);
            pp.uses[w]++;
            if (a + cnt > (P.n & ~3ull)) {  // the array's last elements: plain loads (uniform branch)
                stream_fix_tail<KV>(P, sk, sv, srck, srcv, a, cnt);
                __syncthreads();
            }
        } else {
            sk = s.u.buf[w].key;
            sv = s.u.buf[w].val;
            for (uint32_t i = threadIdx.x; i < cnt; i += BLOCK) {
                sk[i] = __ldcg(srck + a + i);
                if (kv) sv[i] = __ldcg(srcv + a + i);
            }
            __syncthreads();
        }
        unsigned long long x[NI];
        uint32_t v[NI], pos[NI], peers[NI];
#pragma unroll
        for (int i = 0; i < NI; i++) {
            const uint32_t p = slot_index<NI>(i);
            const bool in = p < cnt;
            x[i] = in ? sk[p] : mk.mn;
            v[i] = in && kv ? sv[p] : 0u;
        }
        if (!IDS) map_tile<NI, false>(mk, s.map, x, b);  // lanes past cnt: ignored by the ranking
        // the peer table lies inside this warp's own span of the tile's keys
        // (16 bytes in: past the alignment offset, so clear of the previous
        // warp's last key), which the warp has just loaded into registers;
        // the tile is staged there only after the scan's barriers
        if (table)
            rank_peers_tbl<NI>(b, cnt, reinterpret_cast<uint32_t *>(s.u.buf[w].key + (threadIdx.x >> 5) * (32 * NI) + 2),
                               k, peers);
        else
            rank_peers<NI, 9>(b, cnt, peers);
        rank_leaders<NI>(b, peers, pos, s);
        // every thread has left the previous tile: its buffer may be refilled
        if (__syncthreads_or(!ok)) {
            // a copy did not complete in time: give every copy that may still
            // be in flight (this tile's and the next ones') one more bounded
            // wait before leaving, so that no copy lands in a reused buffer
            if (bulk) {
                mbar_wait(&s.bar[w], (pp.uses[w] - 1u) & 1u, P.wait_ns);
                for (uint32_t tn = t + 1; tn < nt && tn < t + SC_STAGES; tn++) {  // issued in earlier tiles
                    const int wn = (int)(tn % SC_STAGES);
                    mbar_wait(&s.bar[wn], pp.uses[wn] & 1u, P.wait_ns);
                }
            }
            err = true;
            break;
        }
        rank_scan<true>(k, s);
        rank_place<NI>(b, pos, s);
        rank_zero_warp(k, s);
#pragma unroll
        for (int i = 0; i < NI; i++) {
            if (pos[i] != INVALID) {
                sk[pos[i]] = x[i];
                if (kv) sv[pos[i]] = v[i];
                s.bkt[pos[i]] = (uint16_t)b[i];
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < NI; i++) {
            const uint32_t p = threadIdx.x + i * BLOCK;
            if (p < cnt) {
                const unsigned long long key = sk[p];
                const uint32_t rel = s.gdelta[s.bkt[p]] + p;
                if (rel < seglen) {
                    st_front(dstk + rel, key, pol_front);
                    if (kv) st_front(dstv + rel, sv[p], pol_front);
                } else {
                    set_error(P, ST_INTERNAL);
                }
            }
        }
        fence_proxy_async();  // this thread's smem accesses before the buffer's next bulk write
        // the last warp out of this tile's buffer refills it with tile
        // t + SC_STAGES (the branch is uniform over the CTA: every warp
        // arrives, and the counter is back at 0 for the next tile)
        if (bulk && t + SC_STAGES < nt) {
            __syncwarp();
            if ((threadIdx.x & 31) == 0) {
                __threadfence_block();
                if (atomicAdd(&s.drain, 1u) == (uint32_t)WARPS - 1u) {
                    s.drain = 0u;
                    __threadfence_block();
                    const uint32_t tn = t + SC_STAGES;
                    const unsigned long long e0 = start + (unsigned long long)tn * TL;
                    stream_issue<KV>(P, s, w, srck, srcv, e0, tile_cnt(tn));
                    if (IDS) bulk_prefetch_l2_inside(P.ids, e0, e0 + tile_cnt(tn));
                }
            }
        }
    }
    if (err) set_error(P, ST_TIMEOUT);
    __syncthreads();
}

// One instantiation per payload mode and bucket source, so that each keeps
// its own registers.
template <bool KV>
__device__ __forceinline__ void scatter_pick(const Params &P, SmemTile &s, Pipe &pp, const uint64_t *srck,
                                             const uint32_t *srcv, bool bulk, unsigned long long start,
                                             unsigned long long len, uint64_t *dstk, uint32_t *dstv, uint32_t seglen,
                                             uint32_t k, bool ids)
{
    const bool learned = s.map.kind == MAP_MLP || s.map.kind == MAP_PWL || s.map.kind == MAP_SPLIT;
    if (learned != ids) {  // only chunked partitions learn maps, and their histograms write ids
        set_error(P, ST_INTERNAL);
        return;
    }
    const bool small = P.ipt == (uint32_t)IPT_SMALL;
    if (ids && small)  // learned: buckets from the histogram pass
        scatter_stream<IPT_SMALL, true, KV>(P, s, pp, srck, srcv, bulk, start, len, dstk, dstv, seglen);
    else if (ids)
        scatter_stream<IPT, true, KV>(P, s, pp, srck, srcv, bulk, start, len, dstk, dstv, seglen);
    else if (small)
        scatter_stream<IPT_SMALL, false, KV>(P, s, pp, srck, srcv, bulk, start, len, dstk, dstv, seglen);
    else
        scatter_stream<IPT, false, KV>(P, s, pp, srck, srcv, bulk, start, len, dstk, dstv, seglen);
}

// ids: the buckets of a learned map come from the histogram pass (chunked
// partitions); otherwise the scatter evaluates the (z-score or range) map.
__device__ void scatter_dispatch(const Params &P, SmemTile &s, Pipe &pp, const uint64_t *srck, const uint32_t *srcv,
                                 bool bulk, unsigned long long start, unsigned long long len, uint64_t *dstk,
                                 uint32_t *dstv, uint32_t seglen, uint32_t k, bool ids)
{
    if (P.kv)
        scatter_pick<true>(P, s, pp, srck, srcv, bulk, start, len, dstk, dstv, seglen, k, ids);
    else
        scatter_pick<false>(P, s, pp, srck, srcv, bulk, start, len, dstk, dstv, seglen, k, ids);
}

// ------------------------------------------------------------ children
// After a partition of the (sub)array at absolute offset poff: bucket counts
// in s.hist[0..k), starts (relative) in s.bs[0..k).  Consecutive small
// buckets are grouped into leaves of at most leaf_cap (<= LEAF_CAP) elements (sorting a
// group of whole, ordered buckets gives the same result as sorting each);
// larger buckets become medium or large (sub)arrays of the next level.
// A child holding more than half of its parent (plen elements) -- typically a
// value that dominates a skewed, duplicate-heavy input, which Eq. 1 keeps
// lumped with its neighbours level after level -- is partitioned with the
// exact range map, which separates the other values from it at once.
__device__ __noinline__ void classify_children(const Params &P, unsigned long long poff, uint32_t k,
                                  uint32_t child_buf, uint32_t child_level, uint32_t plen, SmemTile &s,
                                  bool keep_leaves = false)
{
    ChildList &L = s.u.children;
    // 1. thread 0 walks the buckets in order: leaf groups, medium and large
    //    children (shared memory only)
    if (threadIdx.x == 0) {
        // in registers: the loop's shared-memory stores would otherwise make
        // the compiler reload the launch parameters on every bucket
        const uint32_t leaf_cap = P.leaf_cap, large_min = P.large_min;
        uint32_t nl = 0, nm = 0, ng = 0, glen = 0, gstart = 0;
        for (uint32_t b8 = 0; b8 < k; b8 += 8) {  // k: a power of two >= 16
          uint32_t cc[8], ss[8];
#pragma unroll
          for (int j = 0; j < 8; j++) {  // eight independent loads, then the walk
              cc[j] = s.hist[b8 + j];
              ss[j] = s.bs[b8 + j];
          }
#pragma unroll
          for (int j = 0; j < 8; j++) {
            const uint32_t c = cc[j];
            if (c == 0) continue;
            if (c > leaf_cap) {
                if (glen) {
                    L.leaf_off[nl] = gstart;
                    L.leaf_len[nl++] = glen;
                    glen = 0;
                }
                if (c <= large_min) {
                    L.med_off[nm] = ss[j];
                    L.med_len[nm++] = c;
                } else {
                    L.lg_off[ng] = ss[j];
                    L.lg_len[ng++] = c;
                }
            } else {
                if (glen + c > leaf_cap) {
                    L.leaf_off[nl] = gstart;
                    L.leaf_len[nl++] = glen;
                    glen = 0;
                }
                if (glen == 0) gstart = ss[j];
                glen += c;
            }
          }
        }
        if (glen) {
            L.leaf_off[nl] = gstart;
            L.leaf_len[nl++] = glen;
        }
        if (child_level > (uint32_t)MAX_LEVEL && (nm + ng) > 0) set_error(P, ST_INTERNAL);
        s.n_leaf = nl;
        s.n_med = nm;
        s.n_large = ng;
        s.red64[0] = 0;
    }
    __syncthreads();
    const uint32_t ng = s.n_large;
    // 2. every thread a share of the large children: chunk geometry and
    //    look-back rows (2 x chunks x k words each), then their offsets
    unsigned long long part = 0;
    for (uint32_t g = threadIdx.x; g < ng; g += BLOCK) {
        const uint32_t len = L.lg_len[g];
        const uint32_t tiles = (len + P.tile - 1) / P.tile;
        const uint32_t chunks = chunk_plan(P, tiles, len).chunks;
        const uint32_t kk = choose_k(P, len);
        L.lg_chunks[g] = chunks;
        L.lg_k[g] = kk;
        L.lg_need[g] = 2u * chunks * kk;
        part += 2ull * chunks * kk;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0 && part) atomicAdd(&s.red64[0], part);
    __syncthreads();
    const unsigned long long need = s.red64[0];
    if (need < (1ull << 32)) block_exclusive_scan(L.lg_need, L.lg_need, ng, s.wsum);  // ends with a barrier
    // 3. thread 0: one allocation of descriptors, look-back rows and items
    if (threadIdx.x == 0) {
        uint32_t nl = s.n_leaf, nm = s.n_med;
        uint32_t sid0 = 0;
        unsigned long long sb0 = 0;
        bool ok = ng > 0 && need < (1ull << 32);
        if (ok) {
            sid0 = atomicAdd(&P.ctl->seg_alloc, ng);
            ok = sid0 + (unsigned long long)ng <= P.segcap;
        }
        if (ok) {
            sb0 = atomicAdd(&P.ctl->status_alloc, need);
            ok = sb0 + need <= P.statuscap;
        }
        uint32_t nok = ng;
        if (!ok && ng > 0) {  // no room: all medium
            for (uint32_t g = 0; g < ng; g++) {
                L.med_off[nm] = L.lg_off[g];
                L.med_len[nm++] = L.lg_len[g];
            }
            nok = 0;
        }
        uint32_t base = atomicAdd(&P.ctl->item_alloc, nl + nm);
        if (base + nl + nm > P.itemcap) {
            set_error(P, ST_CAPACITY);
            nl = nm = nok = 0;
        }
        s.n_leaf = nl;
        s.n_med = nm;
        s.n_large_ok = nok;
        s.item_base = base;
        s.e_base = sid0;
        s.red64[1] = sb0;
    }
    __syncthreads();
    const uint32_t nl = s.n_leaf, nm = s.n_med, nok = s.n_large_ok, base = s.item_base, sid0 = s.e_base;
    const unsigned long long sb0 = s.red64[1];
    // 4. items, descriptors and cleared counters, every thread a share
    for (uint32_t i = threadIdx.x; i < nl + nm; i += BLOCK) {
        Item it;
        const bool leaf = i < nl;
        it.off = poff + (leaf ? L.leaf_off[i] : L.med_off[i - nl]);
        it.len = leaf ? L.leaf_len[i] : L.med_len[i - nl];
        it.buf = (uint16_t)child_buf;
        const bool poor = !leaf && 2ull * it.len > plen;  // medium child: range-map flag in bit 15
        it.level = (uint16_t)(child_level | (poor ? ITEM_RANGE_MAP : 0u));
        P.items[base + i] = it;
    }
    for (uint32_t g = threadIdx.x; g < nok; g += BLOCK) {
        const uint32_t len = L.lg_len[g];
        Seg *S = &P.segs[sid0 + g];
        S->off = poff + L.lg_off[g];
        S->mn = ~0ull;
        S->mx = 0ull;
        S->s1[0] = S->s1[1] = 0ull;
        S->s2[0] = S->s2[1] = S->s2[2] = 0ull;
        S->status_base = sb0 + L.lg_need[g];
        S->len = len;
        S->k = L.lg_k[g];
        S->tiles = (len + P.tile - 1) / P.tile;
        const ChunkPlan cp = chunk_plan(P, S->tiles, len);
        S->chunk_tiles = cp.ct;
        S->chunk_tiles_small = cp.ct_small;
        S->chunks_big = cp.big;
        S->chunks = cp.chunks;
        S->level = child_level;
        S->buf = child_buf;
        S->kind = MAP_Z;
        S->range_map = 2ull * len > plen;
        const uint32_t slot = S->range_map ? INVALID : take_train_slot(P, len, S->k, child_level);
        S->train_slot = slot;
        // Eq. 1 sub-arrays take their statistics from a sample (the range
        // map and the learned map keep the exact pass)
        L.lg_sampled[g] = P.sub_sample && !S->range_map && slot == INVALID && child_level < P.guard_level;
        S->join = 2;
        S->runs_left = SAMPLE_RUNS;
        S->max_learned = S->max_z = 0;
        L.lg_slot[g] = slot;
    }
    __threadfence();  // descriptors and items before the entries are published
    __syncthreads();
    // 5. queue entries: thread 0 reserves them and writes the learned-map
    //    samples (few: one per training slot) first -- each is one CTA's long
    //    task that runs beside its (sub)array's statistics tiles; every
    //    thread then writes a share of the statistics entries, and the ready
    //    words follow one fence later
    if (threadIdx.x == 0) {
        uint32_t nsample = 0;
        for (uint32_t g = 0; g < nok; g++) nsample += L.lg_slot[g] != INVALID;
        const uint32_t cnt = (nm > 0) + nok + nsample;
        uint32_t e = cnt ? q_reserve(P, cnt, 0) : INVALID;
        if (e != INVALID) {
            uint32_t j = e;
            for (uint32_t g = 0; g < nok && j < e + nsample; g++)
                if (L.lg_slot[g] != INVALID) q_write(P, j++, T_LSAMPLE, sid0 + g, SAMPLE_RUNS);
            if (nm) q_write(P, e + nsample + nok, T_MPART, base + nl, nm);
        }
        s.red64[2] = e;
        s.red64[3] = ((unsigned long long)cnt << 32) | nsample;
        if (nl && keep_leaves) {  // finished by this CTA next, from its stash
            s.local_base = base;
            s.local_n = nl;
        } else if (nl) {
            const uint32_t el = q_reserve(P, 1, queue_of(T_FINISH));
            if (el != INVALID) {
                q_write(P, el, T_FINISH, base, nl);
                q_release_all(P, el, 1);
            }
        }
    }
    __syncthreads();
    const uint32_t e = (uint32_t)s.red64[2], nsample = (uint32_t)s.red64[3], cnt = (uint32_t)(s.red64[3] >> 32);
    if (e != INVALID) {
        for (uint32_t g = threadIdx.x; g < nok; g += BLOCK) {
            if (L.lg_sampled[g])
                q_write(P, e + nsample + g, T_SSTATS, sid0 + g, 1);
            else
                q_write(P, e + nsample + g, T_LSTATS, sid0 + g, L.lg_chunks[g]);
        }
        __threadfence();
        __syncthreads();
        const uint32_t ep = call_epoch(P);
        for (uint32_t i = threadIdx.x; i < cnt; i += BLOCK) st_relaxed(&P.ready[e + i], ep);
    }
    __syncthreads();
}

// ------------------------------------------------------------ chunk geometry
struct Chunk {
    unsigned long long off, start, len;  // segment offset; chunk start; chunk length
    unsigned long long sbase;
    uint32_t seglen, buf, k, chunks;
};

__device__ __forceinline__ Chunk chunk_of(const Params &P, uint32_t sid, uint32_t c)
{
    const Seg *S = &P.segs[sid];
    Chunk ch;
    ch.off = __ldcg(&S->off);
    ch.seglen = __ldcg(&S->len);
    ch.buf = __ldcg(&S->buf);
    ch.k = __ldcg(&S->k);
    ch.chunks = __ldcg(&S->chunks);
    ch.sbase = __ldcg(&S->status_base);
    const unsigned long long big_span = (unsigned long long)__ldcg(&S->chunk_tiles) * P.tile;
    const uint32_t big = __ldcg(&S->chunks_big);
    unsigned long long span = big_span, rel = (unsigned long long)c * big_span;
    if (c >= big) {  // the short chunks at the end
        span = (unsigned long long)__ldcg(&S->chunk_tiles_small) * P.tile;
        rel = (unsigned long long)big * big_span + (unsigned long long)(c - big) * span;
    }
    ch.start = ch.off + rel;
    ch.len = min(span, (unsigned long long)ch.seglen - rel);
    return ch;
}

// ------------------------------------------------------------ LSTATS
__device__ __noinline__ void task_lstats(const Params &P, uint32_t sid, uint32_t c, SmemTile &s, Pipe &pp)
{
    const Chunk ch = chunk_of(P, sid, c);
    // this chunk's look-back row must read zero before the histogram phase
    uint32_t *row = P.status + ch.sbase + (size_t)c * ch.k;
    for (uint32_t q = threadIdx.x; q < ch.k; q += BLOCK) __stcg(row + q, 0u);
    LAcc la, la2;
    lacc_init(la);
    lacc_init(la2);
    const uint64_t *src = keys_of(P, ch.buf);
    if (P.ipt == (uint32_t)IPT_SMALL)
        ZS_STATS(IPT_SMALL, src, bulk_ok(P, ch.buf), ch.start, ch.len);
    else
        ZS_STATS(IPT, src, bulk_ok(P, ch.buf), ch.start, ch.len);
    Acc a = lacc_sums(la);
    acc_merge(a, lacc_sums(la2));
    acc_block_reduce(a, s.acc);
    if (threadIdx.x == 0) {
        Seg *W = &P.segs[sid];
        atomicMin(&W->mn, a.mn);
        atomicMax(&W->mx, a.mx);
        unsigned long long v1[2] = {(unsigned long long)a.s1, (unsigned long long)(a.s1 >> 64)};
        unsigned long long v2[3] = {(unsigned long long)a.s2lo, (unsigned long long)(a.s2lo >> 64), a.s2hi};
        atomic_add_wide(W->s1, v1, 2);
        atomic_add_wide(W->s2, v2, 3);
        atomicAdd(&P.ctl->bytes, 8ull * ch.len);
    }
}

// Thread 0: publishes one entry (nothing for type T_NONE).
__device__ void publish1(const Params &P, uint32_t type, uint32_t arg, uint32_t nt)
{
    if (type == T_NONE) return;
    const uint32_t e = q_reserve(P, 1, queue_of(type));
    if (e != INVALID) {
        q_write(P, e, type, arg, nt);
        q_release_all(P, e, 1);
    }
}

// Thread 0, for a (sub)array with a training slot: the statistics and each
// sample run call this once when done; the last one publishes the successor
// that the statistics chose (written before their call).
__device__ void learned_join(const Params &P, uint32_t sid)
{
    Seg *S = &P.segs[sid];
    __threadfence();
    if (atomicSub(&S->join, 1u) == 1u) {
        __threadfence();
        publish1(P, __ldcg(&S->next_type), sid, __ldcg(&S->next_nt));
    }
}

__device__ __noinline__ void lstats_done(const Params &P, uint32_t sid, SmemTile &s)
{
    if (threadIdx.x == 0) {
        Seg *S = &P.segs[sid];
        const unsigned long long mn = __ldcg(&S->mn), mx = __ldcg(&S->mx);
        const uint32_t len = __ldcg(&S->len), level = __ldcg(&S->level);
        const uint32_t sbuf = __ldcg(&S->buf), sk = __ldcg(&S->k), chunks = __ldcg(&S->chunks);
        const uint32_t slot = __ldcg(&S->train_slot);
        uint32_t next = T_NONE, nt = 0;
        if (mn == mx && P.plan_out) {  // inspection of identical keys: all in bucket 0
            S->kind = MAP_RANGE;
            S->rshift = 0;
            S->rmult = 0;
            if (level == 0 && sid == 0) {
                MapSm m0;
                m0.k = sk;
                m0.kind = MAP_RANGE;
                record_top(P, m0, mn, mx, 0.0, 0.0);
            }
            next = T_DUMP;
            nt = chunks;
        } else if (mn == mx) {  // a set of identical keys is sorted (Alg. 1 early exit)
            if (sbuf) {
                next = T_COPY;
                nt = (len + LEAF_CAP - 1) / LEAF_CAP;
                atomicAdd(&P.ctl->n_copies, 1ull);
            }
        } else {
            unsigned long long s1[2] = {__ldcg(&S->s1[0]), __ldcg(&S->s1[1])};
            unsigned long long s2[3] = {__ldcg(&S->s2[0]), __ldcg(&S->s2[1]), __ldcg(&S->s2[2])};
            MapSm m;
            double mean_d, sd;
            map_from_sums(P, len, mn, mx, s1, s2, sk, level, __ldcg(&S->range_map) != 0, m, &mean_d, &sd);
            S->mean_d = mean_d;
            S->sd = sd;
            S->kind = m.kind;
            S->zc = m.zc;
            S->zsh = m.zsh;
            S->escale = m.escale;
            S->rshift = m.rshift;
            S->rmult = m.rmult;
            if (level == 0 && sid == 0) record_top(P, m, mn, mx, mean_d, sd);
            next = P.plan_out ? T_DUMP : T_LHIST;
            nt = chunks;
            if (m.kind == MAP_Z && slot != INVALID) {
                next = T_LFIT;
                nt = 1;
            }
        }
        if (slot != INVALID) {
            S->next_type = next;
            S->next_nt = nt;
            learned_join(P, sid);
        } else {
            publish1(P, next, sid, nt);
        }
    }
}

// ------------------------------------------------------------ SSTATS
// Statistics of a large sub-array from a sample.  zsortRec (section
// "Proposed Work") keeps the top level's map form on every sub-problem and
// estimates its inputs (meanEst) instead of computing them; here a sub-array
// below the top takes min, max, mean and sd from SUB_SAMPLE keys at
// stratified positions (exact sums of the sample, as the statistics pass
// computes them), which replaces its whole statistics pass.  Eq. 1 then
// clamps keys outside the sampled [min, max] (map_key), so the map stays
// monotone on every key and the sort stays exact; the sampled min is below
// the sampled max, so the map still splits the sub-array.  A sample whose
// keys are all equal says nothing about the others: then the exact
// statistics pass runs after all.  Also clears the look-back rows, which the
// statistics chunks clear otherwise.
__device__ __noinline__ void task_sstats(const Params &P, uint32_t sid, SmemTile &s)
{
    Seg *S = &P.segs[sid];
    const unsigned long long off = __ldcg(&S->off), sbase = __ldcg(&S->status_base);
    const uint32_t len = __ldcg(&S->len), buf = __ldcg(&S->buf), k = __ldcg(&S->k);
    const uint32_t chunks = __ldcg(&S->chunks), level = __ldcg(&S->level);
    for (uint32_t q = threadIdx.x; q < chunks * k; q += BLOCK) __stcg(P.status + sbase + q, 0u);
    const uint32_t m = min(SUB_SAMPLE, len);
    const unsigned long long seed = P.seed + ((unsigned long long)sid << 32);
    const uint64_t *src = keys_of(P, buf) + off;
    constexpr int U = (SUB_SAMPLE + BLOCK - 1) / BLOCK;  // independent loads in flight per thread
    unsigned long long x[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
        const uint32_t i = threadIdx.x + u * BLOCK;
        x[u] = i < m ? __ldcg(src + sample_pos(seed, len, m, i)) : 0ull;
    }
    LAcc la;
    lacc_init(la);
#pragma unroll
    for (int u = 0; u < U; u++)
        if (threadIdx.x + u * BLOCK < m) lacc_key(la, x[u]);
    Acc a = lacc_sums(la);
    acc_block_reduce(a, s.acc);
    if (threadIdx.x == 0) {
        atomicAdd(&P.ctl->bytes, 8ull * m);
        if (a.mn == a.mx) {  // no spread in the sample: the exact pass decides
            publish1(P, T_LSTATS, sid, chunks);
            return;
        }
        unsigned long long s1[2] = {(unsigned long long)a.s1, (unsigned long long)(a.s1 >> 64)};
        unsigned long long s2[3] = {(unsigned long long)a.s2lo, (unsigned long long)(a.s2lo >> 64), a.s2hi};
        MapSm mp;
        double mean_d, sd;
        map_from_sums(P, m, a.mn, a.mx, s1, s2, k, level, false, mp, &mean_d, &sd);
        S->mn = a.mn;
        S->mx = a.mx;
        S->mean_d = mean_d;
        S->sd = sd;
        S->kind = mp.kind;
        S->zc = mp.zc;
        S->zsh = mp.zsh;
        S->escale = mp.escale;
        S->rshift = mp.rshift;
        S->rmult = mp.rmult;
        atomicAdd(&P.ctl->n_sampled, 1ull);
        __threadfence();  // the map before the histogram tasks are published
        publish1(P, T_LHIST, sid, chunks);
    }
}

// ------------------------------------------------------------ LSAMPLE / LFIT
// Exact LSD radix sort of m 64-bit keys by key - base (8-bit digits, `passes`
// of them) by one CTA, A and B ping-pong in global memory (L2 resident);
// returns 1 if the result is in B.  One read pass builds the histograms of
// all digits; a digit that every key shares is skipped (its pass would be
// the identity).  Each pass streams tiles of 2048 keys in input order, the
// next tile's loads in flight while the current one is ranked (ballots,
// stable), and every key goes straight to its bucket's running cursor.
__device__ uint32_t cta_lsd_sort64(unsigned long long *A, unsigned long long *B, uint32_t m,
                                   unsigned long long base, uint32_t passes, SmemTile &s)
{
    uint32_t *h8 = reinterpret_cast<uint32_t *>(&s.u);  // [8][256] digit histograms
    for (uint32_t q = threadIdx.x; q < 8 * 256; q += BLOCK) h8[q] = 0;
    __syncthreads();
    for (uint32_t i0 = 0; i0 < m; i0 += TILE) {
        unsigned long long x[IPT];
#pragma unroll
        for (int i = 0; i < IPT; i++) {
            const uint32_t p = i0 + threadIdx.x + i * BLOCK;
            x[i] = p < m ? __ldcg(A + p) - base : 0ull;
        }
#pragma unroll
        for (int i = 0; i < IPT; i++)
            if (i0 + threadIdx.x + i * BLOCK < m)
                for (uint32_t d = 0; d < passes; d++) atomicAdd(&h8[d * 256 + ((x[i] >> (8 * d)) & 255u)], 1u);
    }
    __syncthreads();
    uint32_t sel = 0;
    const unsigned long long *src = A;
    unsigned long long *dst = B;
    for (uint32_t d = 0; d < passes; d++) {
        // skip a digit shared by every key
        const uint32_t c = h8[d * 256 + threadIdx.x];
        if (__syncthreads_or(c == m)) continue;
        block_exclusive_scan(h8 + d * 256, s.cursor, 256, s.wsum);
        rank_zero_warp(256, s);
        const uint32_t nt = (m + TILE - 1) / TILE;
        unsigned long long nx[IPT];
#pragma unroll
        for (int i = 0; i < IPT; i++) {
            const uint32_t p = slot_index(i);
            nx[i] = p < m ? __ldcg(src + p) : 0ull;
        }
        for (uint32_t t = 0; t < nt; t++) {
            const uint32_t t0 = t * TILE, cnt = min((uint32_t)TILE, m - t0);
            unsigned long long v[IPT];
            uint32_t b[IPT], pos[IPT], peers[IPT];
#pragma unroll
            for (int i = 0; i < IPT; i++) {
                v[i] = nx[i];
                b[i] = (uint32_t)((v[i] - base) >> (8 * d)) & 255u;
            }
            if (t + 1 < nt) {
#pragma unroll
                for (int i = 0; i < IPT; i++) {
                    const uint32_t p = t0 + TILE + slot_index<IPT>(i);
                    nx[i] = p < m ? __ldcg(src + p) : 0ull;
                }
            }
            rank_peers<IPT, 8>(b, cnt, peers);
            rank_leaders<IPT>(b, peers, pos, s);
            __syncthreads();
            rank_scan<true>(256, s);
            rank_place<IPT>(b, pos, s);
            rank_zero_warp(256, s);
#pragma unroll
            for (int i = 0; i < IPT; i++)
                if (pos[i] != INVALID) __stcg(dst + s.gdelta[b[i]] + pos[i], v[i]);
        }
        __syncthreads();
        sel ^= 1u;
        const unsigned long long *t2 = dst;
        dst = const_cast<unsigned long long *>(src);
        src = t2;
    }
    return sel;
}

// The r-th smallest (0-based) of the sample held as SAMPLE_RUNS sorted runs
// in X: the smallest value v with at least r + 1 sample keys <= v, by a
// binary search over values between the sample's min and max.  Each run
// keeps the index window that holds the count of its keys <= v for every v
// still in the search interval, so its searches shrink as the interval does;
// the runs' searches advance in lockstep (their loads are independent).
__device__ unsigned long long sample_select(const unsigned long long *X, uint32_t m, uint32_t r)
{
    uint32_t wl[SAMPLE_RUNS], wh[SAMPLE_RUNS];
    unsigned long long lo = ~0ull, hi = 0ull;
#pragma unroll
    for (int t = 0; t < SAMPLE_RUNS; t++) {
        wl[t] = (uint32_t)((unsigned long long)t * m / SAMPLE_RUNS);
        wh[t] = (uint32_t)((unsigned long long)(t + 1) * m / SAMPLE_RUNS);
        if (wh[t] > wl[t]) {
            lo = min(lo, __ldcg(X + wl[t]));
            hi = max(hi, __ldcg(X + wh[t] - 1));
        }
    }
    while (lo < hi) {
        const unsigned long long mid = lo + ((hi - lo) >> 1);
        // per run: the first index in [wl, wh) whose key is > mid (wh if none)
        uint32_t a[SAMPLE_RUNS], b[SAMPLE_RUNS];
        bool active = false;
#pragma unroll
        for (int t = 0; t < SAMPLE_RUNS; t++) {
            a[t] = wl[t];
            b[t] = wh[t];
            active = active || a[t] < b[t];
        }
        while (active) {
            unsigned long long v[SAMPLE_RUNS];
#pragma unroll
            for (int t = 0; t < SAMPLE_RUNS; t++) v[t] = a[t] < b[t] ? __ldcg(X + ((a[t] + b[t]) >> 1)) : 0ull;
            active = false;
#pragma unroll
            for (int t = 0; t < SAMPLE_RUNS; t++) {
                if (a[t] < b[t]) {
                    const uint32_t h = (a[t] + b[t]) >> 1;
                    if (v[t] <= mid)
                        a[t] = h + 1;
                    else
                        b[t] = h;
                }
                active = active || a[t] < b[t];
            }
        }
        uint32_t c = 0;
#pragma unroll
        for (int t = 0; t < SAMPLE_RUNS; t++) c += a[t] - (uint32_t)((unsigned long long)t * m / SAMPLE_RUNS);
        if (c >= r + 1) {
            hi = mid;
#pragma unroll
            for (int t = 0; t < SAMPLE_RUNS; t++) wh[t] = a[t];
        } else {
            lo = mid + 1;
#pragma unroll
            for (int t = 0; t < SAMPLE_RUNS; t++) wl[t] = a[t];
        }
    }
    return lo;
}

// Learned map, first half (beside the statistics tiles): run `run` of the
// sample, i.e. sample indices [run * m / R, (run + 1) * m / R) at the
// stratified positions, drawn and sorted exactly by one CTA (in place in
// buffer A of the slot).  The keys are sorted as they are: the
// normalisation u = fl32(key - min) * 2^-E is monotone, so the sorted keys
// give the sorted normalised sample once min and max are known.
__device__ __noinline__ void task_lsample(const Params &P, uint32_t sid, uint32_t run, SmemTile &s)
{
    Seg *S = &P.segs[sid];
    const unsigned long long off = __ldcg(&S->off);
    const uint32_t len = __ldcg(&S->len), buf = __ldcg(&S->buf), slot = __ldcg(&S->train_slot);
    const uint32_t m = P.sample;
    const uint32_t lo = (uint32_t)((unsigned long long)run * m / SAMPLE_RUNS);
    const uint32_t hi = (uint32_t)((unsigned long long)(run + 1) * m / SAMPLE_RUNS);
    const uint32_t mr = hi - lo;
    unsigned long long *A = P.trainbuf + (size_t)slot * 2 * SAMPLE_MAX + lo;
    unsigned long long *B = A + SAMPLE_MAX;
    const uint64_t *src = keys_of(P, buf) + off;
    unsigned long long mn = ~0ull, mx = 0ull;
    constexpr int U = 8;  // independent loads in flight per thread
    for (uint32_t i0 = 0; i0 < mr; i0 += BLOCK * U) {
        unsigned long long x[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint32_t i = i0 + threadIdx.x + u * BLOCK;
            x[u] = i < mr ? __ldcg(src + sample_pos(P.seed, len, m, lo + i)) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint32_t i = i0 + threadIdx.x + u * BLOCK;
            if (i < mr) {
                __stcg(A + i, x[u]);
                mn = x[u] < mn ? x[u] : mn;
                mx = x[u] > mx ? x[u] : mx;
            }
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long a = shfl_down64(mn, o), b2 = shfl_down64(mx, o);
        mn = a < mn ? a : mn;
        mx = b2 > mx ? b2 : mx;
    }
    if ((threadIdx.x & 31) == 0) {
        s.red64[threadIdx.x >> 5] = mn;
        s.red64[WARPS + (threadIdx.x >> 5)] = mx;
    }
    __syncthreads();
    mn = s.red64[0];
    mx = s.red64[WARPS];
    for (int w = 1; w < WARPS; w++) {
        mn = s.red64[w] < mn ? s.red64[w] : mn;
        mx = s.red64[WARPS + w] > mx ? s.red64[WARPS + w] : mx;
    }
    __syncthreads();
    if (mr > 0 && cta_lsd_sort64(A, B, mr, mn, (bitlen64(mx - mn) + 7) / 8, s))
        for (uint32_t i = threadIdx.x; i < mr; i += BLOCK) __stcg(A + i, __ldcg(B + i));
    __threadfence();  // the sorted run before the last run's selection reads it
    __syncthreads();
    if (threadIdx.x == 0) s.flag = atomicSub(&S->runs_left, 1u) == 1u ? 1u : 0u;
    __syncthreads();
    if (!s.flag) return;
    // the last run to finish selects the breakpoint keys from all runs (it
    // needs no statistics, so it runs beside the statistics pass): key of
    // rank floor(j m / P) for j = 1..P-1, into the free half of the buffer
    __threadfence();
    const unsigned long long *X = P.trainbuf + (size_t)slot * 2 * SAMPLE_MAX;
    unsigned long long *sel = P.trainbuf + (size_t)slot * 2 * SAMPLE_MAX + SAMPLE_MAX;
    for (int j = 1 + threadIdx.x; j < PWL_P; j += BLOCK)
        __stcg(sel + j, sample_select(X, m, (uint32_t)((size_t)j * m / PWL_P)));
    __threadfence();  // the selected keys before the join publishes the fit
    __syncthreads();
    if (threadIdx.x == 0) learned_join(P, sid);
}

// MLP map training state (aliases the tile buffers during the fit).
struct MlpTrain {
    float om[MLP_H], be[MLP_H], al[MLP_H];  // w = om^2, b = be, a = al^2
    float so[MLP_H], sb[MLP_H], sa[MLP_H];  // step of each parameter
    int po[MLP_H], pb[MLP_H], pa[MLP_H];    // sign of its last gradient
    float r[PWL_P + 1];                     // residual at each knot
};
static_assert(sizeof(MlpTrain) <= sizeof(TileBuf) * 2, "MLP training state fits the tile buffers");

__device__ __forceinline__ float mlp_forward_train(const MlpTrain &T, float u)
{
    float f = 0.0f;
    for (int h = 0; h < MLP_H; h++) {
        const float w = __fmul_rn(T.om[h], T.om[h]);
        const float c = fminf(fmaxf(__fadd_rn(__fmul_rn(w, u), T.be[h]), 0.0f), 1.0f);
        f = __fadd_rn(f, __fmul_rn(__fmul_rn(T.al[h], T.al[h]), c));
    }
    return f;
}

__device__ __forceinline__ void rprop_step(float &p, float &step, int &sprev, float g)
{
    const int sg = (g > 0.0f) - (g < 0.0f);
    if (sg * sprev < 0) {
        step = __fmul_rn(step, 0.5f);
        sprev = 0;
        return;
    }
    if (sg * sprev > 0) step = __fmul_rn(step, 1.2f);
    if (sg > 0) p = __fsub_rn(p, step);
    if (sg < 0) p = __fadd_rn(p, step);
    sprev = sg;
}

// The MLP map fitted to the knots (q[j], j / P) of the piecewise-linear map
// in s.map.q: a 2-layer MLP with positive weights (w = omega^2, a = alpha^2)
// and clamp(., 0, 1) hidden units, f(u) = sum_h a_h clamp(w_h u + b_h, 0, 1),
// started as the MLP_H-piece interpolation of the knots and trained by
// full-batch resilient gradient descent on the squared error, MLP_ITERS
// iterations; one thread per knot for the residuals, one per unit for its
// gradients (each sum in a fixed order, so the result is reproducible).
// Writes w, b, a, f0 = f(0), inv = 1 / (f(q[P]) - f0) to s.map.mlp and t.
__device__ void mlp_train(SmemTile &s, float *t)
{
    MlpTrain &T = *reinterpret_cast<MlpTrain *>(&s.u);
    const float *q = s.map.q;
    const int h = threadIdx.x;
    if (h < MLP_H) {
        const float lo = q[h * PWL_P / MLP_H], hi = q[(h + 1) * PWL_P / MLP_H];
        const float w = hi > lo ? __fdiv_rn(1.0f, __fsub_rn(hi, lo)) : 1048576.0f;
        T.om[h] = __fsqrt_rn(w);
        T.be[h] = -__fmul_rn(lo, w);
        T.al[h] = __fsqrt_rn(__fdiv_rn(1.0f, (float)MLP_H));
        T.so[h] = __fmul_rn(0.001f, T.om[h]);
        T.sb[h] = 0.001f;
        T.sa[h] = __fmul_rn(0.001f, T.al[h]);
        T.po[h] = T.pb[h] = T.pa[h] = 0;
    }
    __syncthreads();
    for (int it = 0; it < MLP_ITERS; it++) {
        for (int j = threadIdx.x; j <= PWL_P; j += BLOCK)
            T.r[j] = __fsub_rn(mlp_forward_train(T, q[j]), __fdiv_rn((float)j, (float)PWL_P));
        __syncthreads();
        if (h < MLP_H) {
            const float w = __fmul_rn(T.om[h], T.om[h]), a = __fmul_rn(T.al[h], T.al[h]);
            float ga = 0.0f, gw = 0.0f, gb = 0.0f;
            for (int j = 0; j <= PWL_P; j++) {
                const float t2 = __fadd_rn(__fmul_rn(w, q[j]), T.be[h]);
                const float c = fminf(fmaxf(t2, 0.0f), 1.0f);
                ga = __fadd_rn(ga, __fmul_rn(T.r[j], c));
                if (t2 > 0.0f && t2 < 1.0f) {
                    gw = __fadd_rn(gw, __fmul_rn(T.r[j], q[j]));
                    gb = __fadd_rn(gb, T.r[j]);
                }
            }
            if (!(a > 0.0f)) gw = gb = 0.0f;
            rprop_step(T.om[h], T.so[h], T.po[h], __fmul_rn(gw, T.om[h]));
            rprop_step(T.be[h], T.sb[h], T.pb[h], gb);
            rprop_step(T.al[h], T.sa[h], T.pa[h], __fmul_rn(ga, T.al[h]));
        }
        __syncthreads();
    }
    if (h < MLP_H) {
        s.map.mlp[h] = __fmul_rn(T.om[h], T.om[h]);
        s.map.mlp[MLP_H + h] = T.be[h];
        s.map.mlp[2 * MLP_H + h] = __fmul_rn(T.al[h], T.al[h]);
    }
    if (h == 0) {
        const float f0 = mlp_forward_train(T, 0.0f), f1 = mlp_forward_train(T, q[PWL_P]);
        s.map.mlp[3 * MLP_H] = f0;
        s.map.mlp[3 * MLP_H + 1] = f1 > f0 ? __fdiv_rn(1.0f, __fsub_rn(f1, f0)) : 0.0f;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < MLP_TABLE; j += BLOCK) t[j] = s.map.mlp[j];
}

// Learned map, second half (after the statistics and the sample): breakpoints
// at the 1/256 quantiles of the normalised sample and their reciprocal
// widths, then the load test that keeps Eq. 1 as the fallback.
__device__ __noinline__ void task_lfit(const Params &P, uint32_t sid, SmemTile &s)
{
    Seg *S = &P.segs[sid];
    const unsigned long long mn = __ldcg(&S->mn), mx = __ldcg(&S->mx);
    const uint32_t k = __ldcg(&S->k), slot = __ldcg(&S->train_slot), chunks = __ldcg(&S->chunks);
    const float escale = __ldcg(&S->escale), zc = __ldcg(&S->zc);
    const uint32_t zsh = __ldcg(&S->zsh);
    const uint32_t m = P.sample;
    const unsigned long long *X = P.trainbuf + (size_t)slot * 2 * SAMPLE_MAX;  // sorted runs
    if (threadIdx.x == 0) {
        s.map.mn = mn;
        s.map.kind = MAP_PWL;
        s.map.k = k;
        s.map.K = k / PWL_P;
        s.map.escale = escale;
        s.map.zc = zc;
        s.map.zsh = zsh;
    }
    float *t = P.pwl + (size_t)sid * PWL_STRIDE;
    for (int j = threadIdx.x; j <= PWL_P; j += BLOCK) {
        float q;
        if (j == 0)
            q = 0.0f;
        else if (j == PWL_P)
            q = __fmul_rn(u64_to_f32_rn(mx - mn), escale);
        else
            q = __fmul_rn(u64_to_f32_rn(__ldcg(X + SAMPLE_MAX + j) - mn), escale);  // selected by the last run
        s.map.q[j] = q;
        t[j] = q;
    }
    for (uint32_t q = threadIdx.x; q < k; q += BLOCK) {
        s.hist[q] = 0;
        s.cursor[q] = 0;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < PWL_P; j += BLOCK) {
        const float lo = s.map.q[j], hi = s.map.q[j + 1];
        const float r = hi > lo ? __fdiv_rn(1.0f, __fsub_rn(hi, lo)) : 0.0f;
        s.map.r[j] = r;
        t[PWL_P + 1 + j] = r;
    }
    build_pwl_bins(s.map, &s.span_max);
    __syncthreads();
    const bool mlp = P.mapper == 2;
    if (mlp) mlp_train(s, t + PWL_MLP_OFF);  // the MLP map replaces the piecewise-linear one
    // load test on the sample: largest learned bucket vs largest Eq. 1 bucket
    for (uint32_t i0 = 0; i0 < m; i0 += BLOCK * IPT) {
        unsigned long long x[IPT];
#pragma unroll
        for (int u = 0; u < IPT; u++) {
            const uint32_t i = i0 + threadIdx.x + u * BLOCK;
            x[u] = i < m ? __ldcg(X + i) : mn;
        }
#pragma unroll
        for (int u = 0; u < IPT; u++) {
            if (i0 + threadIdx.x + u * BLOCK < m) {
                const unsigned long long d = x[u] - mn;
                const float u = __fmul_rn(u64_to_f32_rn(d), escale);
                atomicAdd(&s.hist[mlp ? mlp_bucket_u(s.map.mlp, u, k) : pwl_bucket_u(s.map, u)], 1u);
                const uint32_t bz = __float2uint_rz(__fmul_rn(__uint2float_rz((uint32_t)(d >> zsh)), zc));
                atomicAdd(&s.cursor[bz < k ? bz : k - 1], 1u);
            }
        }
    }
    __syncthreads();
    uint32_t ml = 0, mz = 0;
    for (uint32_t q = threadIdx.x; q < k; q += BLOCK) {
        ml = max(ml, s.hist[q]);
        mz = max(mz, s.cursor[q]);
    }
    ml = __reduce_max_sync(0xffffffffu, ml);
    mz = __reduce_max_sync(0xffffffffu, mz);
    if ((threadIdx.x & 31) == 0) {
        s.red64[threadIdx.x >> 5] = ml;
        s.red64[WARPS + (threadIdx.x >> 5)] = mz;
    }
    __threadfence();  // the map tables before the histogram tasks are published
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < WARPS; w++) {
            ml = max(ml, (uint32_t)s.red64[w]);
            mz = max(mz, (uint32_t)s.red64[WARPS + w]);
        }
        const bool ok = (float)ml <= P.fallback_ratio * (float)m / (float)k && ml <= mz;
        S->max_learned = ml;
        S->max_z = mz;
        s.flag = ok ? 1u : 0u;
        s.red64[0] = mz;
    }
    __syncthreads();
    uint32_t kind = s.flag ? (mlp ? (uint32_t)MAP_MLP : (uint32_t)MAP_PWL) : (uint32_t)MAP_Z;
    if (!s.flag) {
        // Second try, when binary32 normalisation collapsed the sample (a
        // dense interval far from the minimum becomes one u): the same CDF
        // with exact-key breakpoints -- the selected sample keys, the exact
        // min and max -- and binary32 interpolation inside each piece,
        // relative to its own lower key.  The breakpoint keys stay in the
        // training slot's selection area, the slopes replace r in the table.
        const uint32_t mz0 = (uint32_t)s.red64[0];
        unsigned long long *sel = P.trainbuf + (size_t)slot * 2 * SAMPLE_MAX + SAMPLE_MAX;
        for (int j = threadIdx.x; j <= PWL_P; j += BLOCK) {
            const unsigned long long b = j == 0 ? mn : (j == PWL_P ? mx : __ldcg(sel + j));
            s.map.bq[j] = b;
            if (j == 0 || j == PWL_P) __stcg(sel + j, b);
        }
        for (uint32_t q = threadIdx.x; q < k; q += BLOCK) s.hist[q] = 0;
        __syncthreads();
        for (int j = threadIdx.x; j < PWL_P; j += BLOCK) {
            const unsigned long long lo = s.map.bq[j], hi = s.map.bq[j + 1];
            const float r = hi > lo ? __fdiv_rn(1.0f, u64_to_f32_rn(hi - lo)) : 0.0f;
            s.map.r[j] = r;
            t[PWL_P + 1 + j] = r;
        }
        __syncthreads();
        for (uint32_t i0 = 0; i0 < m; i0 += BLOCK * IPT) {
            unsigned long long x[IPT];
#pragma unroll
            for (int u = 0; u < IPT; u++) {
                const uint32_t i = i0 + threadIdx.x + u * BLOCK;
                x[u] = i < m ? __ldcg(X + i) : mn;
            }
#pragma unroll
            for (int u = 0; u < IPT; u++)
                if (i0 + threadIdx.x + u * BLOCK < m) atomicAdd(&s.hist[split_bucket(s.map, x[u])], 1u);
        }
        __syncthreads();
        uint32_t ms = 0;
        for (uint32_t q = threadIdx.x; q < k; q += BLOCK) ms = max(ms, s.hist[q]);
        ms = __reduce_max_sync(0xffffffffu, ms);
        if ((threadIdx.x & 31) == 0) s.red64[1 + (threadIdx.x >> 5)] = ms;
        __threadfence();  // the slopes and the breakpoint keys before the histogram tasks are published
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < WARPS; w++) ms = max(ms, (uint32_t)s.red64[1 + w]);
            if ((float)ms <= P.fallback_ratio * (float)m / (float)k && ms <= mz0) kind = MAP_SPLIT;
        }
    }
    if (threadIdx.x == 0) {
        S->kind = kind;
        atomicAdd(kind != MAP_Z ? &P.ctl->n_learn_ok : &P.ctl->n_learn_rej, 1ull);
        if (__ldcg(&S->level) == 0 && sid == 0) P.ctl->top_map = kind;
        publish1(P, P.plan_out ? T_DUMP : T_LHIST, sid, chunks);
    }
}

// ------------------------------------------------------------ DUMP
// Map inspection: the bucket the histogram and scatter would compute for
// every key of one chunk (same map_key, same shared-memory map).
__device__ __noinline__ void task_dump(const Params &P, uint32_t sid, uint32_t c, SmemTile &s, Pipe &pp)
{
    load_seg_map(P, sid, s);
    const Chunk ch = chunk_of(P, sid, c);
    uint32_t *out = P.plan_out;
    stream_tiles<false>(P, s, pp, keys_of(P, ch.buf), nullptr, bulk_ok(P, ch.buf), ch.start, ch.len,
                        [&](uint32_t t, uint32_t cnt, unsigned long long *sk, uint32_t *) {
                            const unsigned long long a = ch.start + (unsigned long long)t * P.tile;
                            for (uint32_t p = threadIdx.x; p < cnt; p += BLOCK) __stcg(out + a + p, map_key_any(s.map, sk[p]));
                        });
}

// ------------------------------------------------------------ LHIST
// Histogram of one chunk, then its bucket offsets over the preceding chunks
// by a decoupled look-back: the chunk publishes, per bucket, its count
// (FLAG_A) and then its inclusive prefix over chunks 0..c (FLAG_P), walking
// back over predecessors until one has FLAG_P.  Chunks are handed out in
// increasing order, so a predecessor is always running or done.
__device__ __noinline__ void task_lhist(const Params &P, uint32_t sid, uint32_t c, SmemTile &s, Pipe &pp)
{
    load_seg_map(P, sid, s);
    const Chunk ch = chunk_of(P, sid, c);
    const uint32_t k = ch.k;
    const MapK mk = map_regs(s.map);
    for (uint32_t q = threadIdx.x; q < k; q += BLOCK) s.hist[q] = 0;
    __syncthreads();
    const uint64_t *src = keys_of(P, ch.buf);
    const bool small = P.ipt == (uint32_t)IPT_SMALL, bulk = bulk_ok(P, ch.buf);
    if (mk.kind == MAP_MLP && small)
        hist_stream<IPT_SMALL, true>(P, s, pp, src, bulk, ch.start, ch.len, mk);
    else if (mk.kind == MAP_MLP)
        hist_stream<IPT, true>(P, s, pp, src, bulk, ch.start, ch.len, mk);
    else if ((mk.kind == MAP_PWL || mk.kind == MAP_SPLIT) && small)
        hist_stream<IPT_SMALL, false>(P, s, pp, src, bulk, ch.start, ch.len, mk);
    else if (mk.kind == MAP_PWL || mk.kind == MAP_SPLIT)
        hist_stream<IPT, false>(P, s, pp, src, bulk, ch.start, ch.len, mk);
    else if (small)
        ZS_HIST_PLAIN(IPT_SMALL, src, bulk, ch.start, ch.len);
    else
        ZS_HIST_PLAIN(IPT, src, bulk, ch.start, ch.len);
    uint32_t *status = P.status + ch.sbase;
    uint32_t *row = status + (size_t)c * k;
    uint32_t *offs = status + (size_t)ch.chunks * k + (size_t)c * k;
    for (uint32_t q = threadIdx.x; q < k; q += BLOCK) {
        const uint32_t h = s.hist[q];
        st_relaxed(row + q, (c == 0 ? FLAG_P : FLAG_A) | h);
    }
    constexpr int PER = NB_MAX / BLOCK;
    uint32_t excl[PER], j[PER];
    bool done[PER];
#pragma unroll
    for (int r = 0; r < PER; r++) {
        excl[r] = 0;
        j[r] = c;
        done[r] = (threadIdx.x + r * BLOCK >= k) || c == 0;
    }
    unsigned long long t0 = 0;
    uint32_t spins = 0;
    bool failed = false;
    for (;;) {
        bool all = true, moved = false;
#pragma unroll
        for (int r = 0; r < PER; r++) {
            if (done[r]) continue;
            const uint32_t q = threadIdx.x + r * BLOCK;
            const uint32_t w = ld_relaxed(status + (size_t)(j[r] - 1) * k + q);
            const uint32_t f = w & ~VAL_MASK;
            if (f == FLAG_P) {
                excl[r] += w & VAL_MASK;
                done[r] = true;
                st_relaxed(row + q, FLAG_P | (excl[r] + s.hist[q]));
                moved = true;
            } else if (f == FLAG_A && j[r] > 1) {
                excl[r] += w & VAL_MASK;
                j[r]--;
                moved = true;
            } else if (f == FLAG_A || f == (FLAG_A | FLAG_P)) {
                set_error(P, ST_INTERNAL);  // chunk 0 always publishes FLAG_P
                done[r] = true;
            } else {
                all = false;
            }
        }
#pragma unroll
        for (int r = 0; r < PER; r++) all = all && done[r];
        if (all) break;
        if (moved) {  // the limit counts from the last progress, not from the first stall
            t0 = 0;
            spins = 0;
        } else if ((++spins & 31u) == 0) {
            const unsigned long long now = globaltimer();
            if (t0 == 0)
                t0 = now;
            else if (now - t0 > P.wait_ns || has_error(P)) {
                failed = true;
                break;
            }
        }
    }
    if (failed) set_error(P, ST_TIMEOUT);
#pragma unroll
    for (int r = 0; r < PER; r++) {
        const uint32_t q = threadIdx.x + r * BLOCK;
        if (q < k) __stcg(offs + q, excl[r]);
    }
    if (threadIdx.x == 0) atomicAdd(&P.ctl->bytes, 8ull * ch.len);
}

// Bucket totals of a large (sub)array once all its chunks are through the
// look-back: the inclusive prefix that its last chunk published.
__device__ __forceinline__ void load_bucket_totals(const Params &P, const Seg *S, uint32_t k, uint32_t chunks,
                                                   uint32_t *out)
{
    const uint32_t *last = P.status + __ldcg(&S->status_base) + (size_t)(chunks - 1) * k;
    for (uint32_t q = threadIdx.x; q < k; q += BLOCK) out[q] = __ldcg(last + q) & VAL_MASK;
}

__device__ __noinline__ void lhist_done(const Params &P, uint32_t sid, SmemTile &s)
{
    const Seg *S = &P.segs[sid];
    const uint32_t k = __ldcg(&S->k), chunks = __ldcg(&S->chunks);
    load_bucket_totals(P, S, k, chunks, s.hist);
    __syncthreads();
    block_exclusive_scan(s.hist, s.bs, k, s.wsum);
    for (uint32_t q = threadIdx.x; q < k; q += BLOCK) P.bstart[(size_t)sid * NB_MAX + q] = s.bs[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t e = q_reserve(P, 1);
        if (e != INVALID) {
            q_write(P, e, T_LSCATTER, sid, chunks);
            q_release_all(P, e, 1);
        }
    }
}

// ------------------------------------------------------------ LSCATTER
// Stable scatter of one chunk: its cursors start at the bucket start plus the
// chunk's look-back offset, and its tiles are streamed in input order.
__device__ __noinline__ void task_lscatter(const Params &P, uint32_t sid, uint32_t c, SmemTile &s, Pipe &pp)
{
    load_seg_map(P, sid, s);
    const Chunk ch = chunk_of(P, sid, c);
    const uint32_t k = ch.k;
    const uint32_t *offs = P.status + ch.sbase + (size_t)ch.chunks * k + (size_t)c * k;
    for (uint32_t q = threadIdx.x; q < k; q += BLOCK)
        s.cursor[q] = __ldcg(&P.bstart[(size_t)sid * NB_MAX + q]) + __ldcg(offs + q);
    __syncthreads();
    uint64_t *dstk = keys_of(P, ch.buf ^ 1u) + ch.off;
    uint32_t *dstv = vals_of(P, ch.buf ^ 1u) + ch.off;
    scatter_dispatch(P, s, pp, keys_of(P, ch.buf), vals_of(P, ch.buf), bulk_ok(P, ch.buf), ch.start, ch.len, dstk,
                     dstv, ch.seglen, k, s.map.kind == MAP_MLP || s.map.kind == MAP_PWL || s.map.kind == MAP_SPLIT);
    if (threadIdx.x == 0) atomicAdd(&P.ctl->bytes, 2ull * elem_bytes(P) * ch.len);
}

__device__ __noinline__ void lscatter_done(const Params &P, uint32_t sid, SmemTile &s)
{
    const Seg *S = &P.segs[sid];
    const uint32_t k = __ldcg(&S->k), buf = __ldcg(&S->buf), level = __ldcg(&S->level);
    const unsigned long long off = __ldcg(&S->off);
    load_bucket_totals(P, S, k, __ldcg(&S->chunks), s.hist);
    for (uint32_t q = threadIdx.x; q < k; q += BLOCK) s.bs[q] = __ldcg(&P.bstart[(size_t)sid * NB_MAX + q]);
    if (threadIdx.x == 0) {
        atomicAdd(&P.ctl->n_large, 1ull);
        note_level(P, level);
    }
    __syncthreads();
    classify_children(P, off, k, buf ^ 1u, level + 1, __ldcg(&S->len), s);
}

// ------------------------------------------------------------ MPART
// A medium (sub)array: every step of Alg. 1 by one CTA, three streamed
// passes in input order, so the scatter is stable with running cursors.
__device__ __noinline__ void task_mpart(const Params &P, const Item it, SmemTile &s, Pipe &pp)
{
    const unsigned long long off = it.off;
    const uint32_t len = it.len, buf = it.buf, level = it.level & (ITEM_RANGE_MAP - 1u);
    const bool force_range = (it.level & ITEM_RANGE_MAP) != 0;
    const uint64_t *srck = keys_of(P, buf);
    const uint32_t *srcv = vals_of(P, buf);
    const bool bulk = bulk_ok(P, buf);
    LAcc la, la2;
    lacc_init(la);
    lacc_init(la2);
    const bool small = P.ipt == (uint32_t)IPT_SMALL;
    if (small)
        ZS_STATS(IPT_SMALL, srck, bulk, off, len);
    else
        ZS_STATS(IPT, srck, bulk, off, len);
    Acc a = lacc_sums(la);
    acc_merge(a, lacc_sums(la2));
    acc_block_reduce(a, s.acc);
    if (threadIdx.x == 0) {
        if (a.mn == a.mx) {
            s.flag = 1;
        } else {
            s.flag = 0;
            unsigned long long s1[2] = {(unsigned long long)a.s1, (unsigned long long)(a.s1 >> 64)};
            unsigned long long s2[3] = {(unsigned long long)a.s2lo, (unsigned long long)(a.s2lo >> 64), a.s2hi};
            double mean_d, sd;
            map_from_sums(P, len, a.mn, a.mx, s1, s2, choose_k(P, len), level, force_range, s.map, &mean_d, &sd);
            if (level == 0 && off == 0) record_top(P, s.map, a.mn, a.mx, mean_d, sd);
        }
    }
    __syncthreads();
    if (s.flag) {  // identical keys: already sorted
        if (buf) {
            for (uint32_t p = threadIdx.x; p < len; p += BLOCK) {
                __stcg(P.ukeys + off + p, __ldcg(srck + off + p));
                if (P.kv) __stcg(P.uvals + off + p, __ldcg(srcv + off + p));
            }
            if (threadIdx.x == 0) {
                atomicAdd(&P.ctl->n_copies, 1ull);
                atomicAdd(&P.ctl->bytes, (8ull + 2ull * elem_bytes(P)) * len);
            }
        } else if (threadIdx.x == 0) {
            atomicAdd(&P.ctl->bytes, 8ull * len);
        }
        return;
    }
    const uint32_t k = s.map.k;
    const MapK mk = map_regs(s.map);
    for (uint32_t q = threadIdx.x; q < k; q += BLOCK) s.hist[q] = 0;
    __syncthreads();
    if (small)
        ZS_HIST_PLAIN(IPT_SMALL, srck, bulk, off, len);
    else
        ZS_HIST_PLAIN(IPT, srck, bulk, off, len);
    block_exclusive_scan(s.hist, s.bs, k, s.wsum);
    for (uint32_t q = threadIdx.x; q < k; q += BLOCK) s.cursor[q] = s.bs[q];
    __syncthreads();
    uint64_t *dstk = keys_of(P, buf ^ 1u) + off;
    uint32_t *dstv = vals_of(P, buf ^ 1u) + off;
    scatter_dispatch(P, s, pp, srck, srcv, bulk, off, len, dstk, dstv, len, k, false);
    if (threadIdx.x == 0) {
        atomicAdd(&P.ctl->n_small, 1ull);
        atomicAdd(&P.ctl->bytes, (16ull + 2ull * elem_bytes(P)) * len);
        note_level(P, level);
    }
    // the leaves stay with this CTA (still in L2) when the medium is small
    // against a CTA's share of the whole call: there are then many mediums,
    // and one small queue entry each made the leaf phase's claims contend.
    // In a small call a medium's leaves go to the queue, where other CTAs
    // can take them at once.
    const bool keep = (unsigned long long)len * P.nctas * 4ull <= P.n;
    classify_children(P, off, k, buf ^ 1u, level + 1, len, s, keep);
}

// ------------------------------------------------------------ FINISH
// Thread 0: L2 prefetch of a leaf's pairs (the span its bulk copies read).
__device__ void prefetch_item_l2(const Params &P, const Item it)
{
    if (!bulk_ok(P, it.buf)) return;
    const unsigned long long off = it.off, len = it.len;
    const unsigned long long a0 = off & ~1ull, a1 = min((off + len + 1) & ~1ull, P.n & ~1ull);
    const unsigned long long b0 = off & ~3ull, b1 = min((off + len + 3) & ~3ull, P.n & ~3ull);
    if (a1 > a0) bulk_prefetch_l2(keys_of(P, it.buf) + a0, (uint32_t)(a1 - a0) * 8u);
    if (P.kv && b1 > b0) bulk_prefetch_l2(vals_of(P, it.buf) + b0, (uint32_t)(b1 - b0) * 4u);
}

__device__ bool insertion_sort_budget(unsigned long long *k, uint32_t *v, uint32_t n, uint32_t budget)
{
    uint32_t moves = 0;
    for (uint32_t i = 1; i < n; i++) {
        if (moves > budget) return false;
        unsigned long long ck = k[i];
        uint32_t cv = v[i];
        uint32_t j = i;
        while (j > 0 && k[j - 1] > ck) {  // strict: equal keys keep their order
            k[j] = k[j - 1];
            v[j] = v[j - 1];
            j--;
            moves++;
        }
        k[j] = ck;
        v[j] = cv;
    }
    return true;
}

// Sorting network on key/val[a, a+c) by (key, current position), so stable:
// the bitonic merge in the form whose comparators all put the smaller item
// first (each merge starts by pairing i with the mirror index), so the
// implicit +infinity items past c never move and need no storage.
__device__ void bitonic_range(SmemTile &s, unsigned long long *key, uint32_t *val, uint32_t a, uint32_t c)
{
    const uint32_t L = pow2ceil32(c);
    uint16_t *ix = s.u.la.sidx;  // current position of each item (the tie-break)
    for (uint32_t i = threadIdx.x; i < c; i += BLOCK) ix[a + i] = (uint16_t)i;
    __syncthreads();
    auto cmpswap = [&](uint32_t i, uint32_t j) {
        const unsigned long long ki = key[a + i], kj = key[a + j];
        const uint16_t ii = ix[a + i], ij = ix[a + j];
        if (ki > kj || (ki == kj && ii > ij)) {
            key[a + i] = kj;
            key[a + j] = ki;
            ix[a + i] = ij;
            ix[a + j] = ii;
            const uint32_t tv = val[a + i];
            val[a + i] = val[a + j];
            val[a + j] = tv;
        }
    };
    for (uint32_t size = 2; size <= L; size <<= 1) {
        const uint32_t half = size >> 1;
        for (uint32_t t = threadIdx.x; t < L / 2; t += BLOCK) {
            const uint32_t blk = t / half, o = t % half;
            const uint32_t i = blk * size + o, j = blk * size + size - 1 - o;
            if (j < c) cmpswap(i, j);
        }
        __syncthreads();
        for (uint32_t stride = half >> 1; stride > 0; stride >>= 1) {
            for (uint32_t t = threadIdx.x; t < L / 2; t += BLOCK) {
                const uint32_t i = 2 * stride * (t / stride) + (t % stride), j = i + stride;
                if (j < c) cmpswap(i, j);
            }
            __syncthreads();
        }
    }
}


// Sub-bucket of a leaf key: range map (the counting map when rm == 0).
__device__ __forceinline__ uint32_t leaf_sub(unsigned long long key, unsigned long long mn, uint32_t rs,
                                             uint32_t rm)
{
    const unsigned long long d = key - mn;
    return rm == 0 ? (uint32_t)d : __umulhi((uint32_t)(d >> rs), rm);
}

constexpr uint32_t LEAF_FAST_MAX = 32;  // largest sub-bucket the fast path ranks by counting

// Fast leaf path.  Every thread holds its pairs (leaf positions threadIdx.x +
// j * BLOCK) in registers and already took, with a shared-memory atomic on the
// counter of its sub-bucket, an arrival slot a[j] inside it; cnt[0..M2) holds
// the sub-bucket counts.  The pairs are staged by sub-bucket (arrival order,
// not yet stable) with their leaf positions; then each staged pair counts its
// rank inside its sub-bucket on (key, leaf position) -- a total order whose
// sorted sequence is the stable sort -- and goes straight to that rank of the
// output (consecutive staged pairs have nearly consecutive ranks).
template <bool KV>
__device__ __forceinline__ void finish_fast(SmemTile &s, unsigned long long *key, uint32_t *val, uint32_t len,
                                         unsigned long long mn, uint32_t rs, uint32_t rm, uint32_t M2,
                                         const unsigned long long (&kk)[LEAF_IPT], const uint32_t (&vv)[LEAF_IPT],
                                         const uint32_t (&a)[LEAF_IPT], uint64_t *dk, uint32_t *dv)
{
    uint32_t *cnt = s.u.la.cnt;
    uint16_t *sidx = s.u.la.sidx;  // leaf position of each staged pair
    block_exclusive_scan_vec8(cnt, M2, s.wsum);  // and cnt[M2] = len: the end of the last sub-bucket
#pragma unroll
    for (int j = 0; j < LEAF_IPT; j++) {
        const uint32_t p = threadIdx.x + j * BLOCK;
        if (p < len) {
            const uint32_t q = cnt[leaf_sub(kk[j], mn, rs, rm)] + a[j];
            key[q] = kk[j];
            val[q] = vv[j];
            sidx[q] = (uint16_t)p;
        }
    }
    __syncthreads();
    // the warp's lanes walk their sub-buckets in lockstep (warp-uniform trip
    // count, clamped reads): no divergence in the counting loop.  Each thread
    // takes LEAF_RANK_U staged pairs per round, so that their loads and
    // compares overlap.
    constexpr int U = LEAF_RANK_U;
    for (uint32_t p0 = 0; p0 < len; p0 += U * BLOCK) {
        unsigned long long xk[U];
        uint32_t me[U], lo[U], hi[U], r[U];
        uint32_t widest = 0;
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint32_t p = p0 + u * BLOCK + threadIdx.x;
            const uint32_t pc = p < len ? p : len - 1;
            xk[u] = key[pc];
            me[u] = sidx[pc];
            const uint32_t q = leaf_sub(xk[u], mn, rs, rm);
            lo[u] = cnt[q];
            hi[u] = cnt[q + 1];
            r[u] = lo[u];
            widest = max(widest, hi[u] - lo[u]);
        }
        const uint32_t m = __reduce_max_sync(0xffffffffu, widest);
        for (uint32_t t = 0; t < m; t++) {
#pragma unroll
            for (int u = 0; u < U; u++) {
                const uint32_t j = min(lo[u] + t, hi[u] - 1);
                const unsigned long long kj = key[j];
                const uint32_t sj = sidx[j];
                r[u] += (uint32_t)(lo[u] + t < hi[u]) &
                        ((uint32_t)(kj < xk[u]) | ((uint32_t)(kj == xk[u]) & (uint32_t)(sj < me[u])));
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint32_t p = p0 + u * BLOCK + threadIdx.x;
            if (p < len) {
                __stcg(dk + r[u], xk[u]);
                if (KV) __stcg(dv + r[u], val[p]);
            }
        }
    }
}

// Stable order of the sub-bucket key/val[a, a+c) (staged in input order) by
// one warp, when it holds at most WARP_DISTINCT_MAX distinct keys: the
// distinct keys in ascending order (one warp minimum above the last, per
// key), their counts and starts, then every pair placed in input order at
// its key's running cursor -- a stable counting sort -- and written straight
// to dk/dv at the same leaf positions.  Returns false, having written
// nothing, when the sub-bucket holds more distinct keys.  dtab / dcur: the
// warp's own shared memory (WARP_DISTINCT_MAX keys, as many cursors).
template <bool KV>
__device__ bool warp_distinct_sort(const unsigned long long *key, const uint32_t *val, uint32_t a, uint32_t c,
                                   unsigned long long *dtab, uint32_t *dcur, uint64_t *dk, uint32_t *dv)
{
    const uint32_t full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    uint32_t D = 0;
    unsigned long long last = 0;
    for (;;) {
        unsigned long long m = ~0ull;
        bool any = false;
        for (uint32_t j = lane; j < c; j += 32) {
            const unsigned long long x = key[a + j];
            if ((D == 0 || x > last) && (!any || x < m)) {
                m = x;
                any = true;
            }
        }
        if (!__any_sync(full, any)) break;
        if (D == (uint32_t)WARP_DISTINCT_MAX) return false;
        unsigned long long mx = 0;
        warp_minmax64(m, mx);  // lanes without a key offer ~0, never below a real one
        if (lane == 0) dtab[D] = m;
        last = m;
        D++;
    }
    __syncwarp();
    auto index_of = [&](unsigned long long x) {  // position of x among the D sorted keys
        uint32_t lo = 0, hi = D - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (dtab[mid] < x)
                lo = mid + 1;
            else
                hi = mid;
        }
        return lo;
    };
    if (lane < (int)D) dcur[lane] = 0u;
    __syncwarp();
    for (uint32_t j = lane; j < c; j += 32) atomicAdd(&dcur[index_of(key[a + j])], 1u);
    __syncwarp();
    const uint32_t cnt = lane < (int)D ? dcur[lane] : 0u;
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += y;
    }
    __syncwarp();
    if (lane < (int)D) dcur[lane] = incl - cnt;  // start of each key's run
    __syncwarp();
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t j0 = 0; j0 < c; j0 += 32) {
        const uint32_t j = j0 + lane;
        const bool valid = j < c;
        const unsigned long long x = valid ? key[a + j] : 0ull;
        const uint32_t d = valid ? index_of(x) : 0xffffu;
        const uint32_t peers = __match_any_sync(full, d) & __ballot_sync(full, valid);
        const uint32_t base = valid ? dcur[d] : 0u;
        __syncwarp();
        if (valid && (peers & lt) == 0u) dcur[d] = base + __popc(peers);  // the lowest lane of the key advances it
        __syncwarp();
        if (valid) {
            const uint32_t p = a + base + __popc(peers & lt);
            __stcg(dk + p, x);
            if (KV) __stcg(dv + p, val[a + j]);
        }
    }
    return true;
}

// Stable leaf path, for leaves with a large sub-bucket (typically many equal
// keys): sub-buckets by the range map, placed in input order by the
// multisplit; then every sub-bucket with an out-of-order neighbour pair is
// sorted by one warp -- insertion when short, else a stable counting sort
// over its distinct keys -- and only one with more than WARP_DISTINCT_MAX
// distinct keys by a bitonic network on (key, position).
template <bool KV>
__device__ __noinline__ void finish_stable(const Params &P, SmemTile &s, unsigned long long *key, uint32_t *val,
                                           uint32_t len, unsigned long long mn, unsigned long long mx,
                                           uint64_t *dk, uint32_t *dv)
{
    const uint32_t M = min((uint32_t)NB_MAX, pow2ceil32(len) / 4);
    uint32_t rshift, rmult;
    range_params(mx - mn, M, &rshift, &rmult);
    unsigned long long x[LEAF_IPT];
    uint32_t v[LEAF_IPT], b[LEAF_IPT], pos[LEAF_IPT];
#pragma unroll
    for (int i = 0; i < LEAF_IPT; i++) {
        const uint32_t p = leaf_slot(i);
        x[i] = p < len ? key[p] : 0ull;
        v[i] = p < len ? val[p] : 0u;
        b[i] = p < len ? leaf_sub(x[i], mn, rshift, rmult) : 0u;
    }
    // stable multisplit of the leaf into its M sub-buckets: peers from a
    // per-warp OR table (M words) in the leaf's position and counter arrays,
    // which this path does not use until its network
    rank_zero_warp(M, s);
    __syncthreads();
    {
        uint32_t peers[LEAF_IPT];
        uint32_t *tbl = reinterpret_cast<uint32_t *>(s.u.la.sidx) + (threadIdx.x >> 5) * NB_MAX;
        rank_peers_tbl<LEAF_IPT>(b, len, tbl, M, peers);
        rank_leaders<LEAF_IPT>(b, peers, pos, s);
    }
    __syncthreads();
    rank_scan<false>(M, s);
    rank_place<LEAF_IPT>(b, pos, s);
#pragma unroll
    for (int i = 0; i < LEAF_IPT; i++) {
        if (pos[i] != INVALID) {
            key[pos[i]] = x[i];
            val[pos[i]] = v[i];
        }
    }
    if (threadIdx.x == 0) {
        s.flag = 0;
        s.flag2 = 0;
    }
    for (uint32_t q = threadIdx.x; q < M; q += BLOCK) s.hist[q] = 0;
    __syncthreads();
    // a sub-bucket is in order (stably: equal keys are in input order) unless
    // two neighbours in it are inverted; only those are sorted -- one thread
    // walking a long run of equal keys would hold up the whole CTA
    for (uint32_t p = threadIdx.x + 1; p < len; p += BLOCK) {
        const unsigned long long kp = key[p], kq = key[p - 1];
        if (kq > kp) {
            const uint32_t q = leaf_sub(kp, mn, rshift, rmult);
            if (q == leaf_sub(kq, mn, rshift, rmult)) s.hist[q] = 1u;
        }
    }
    __syncthreads();
    uint32_t *inv = s.bs;       // inverted sub-buckets
    uint32_t *fail = s.cursor;  // those left to the network
    for (uint32_t q = threadIdx.x; q < M; q += BLOCK)
        if (s.hist[q] && s.tcount[q] >= 2) inv[atomicAdd(&s.flag, 1u)] = q;
    __syncthreads();
    // each inverted sub-bucket: a short one by insertion (one lane), a longer
    // one by its warp as a stable counting sort over its distinct keys,
    // written straight to the output (hist = 2 marks it written); one with
    // more than WARP_DISTINCT_MAX distinct keys goes to the network below.
    // Several distinct keys, each repeated many times (the duplicate-heavy
    // leaves of small Zipf arrays), are what made insertion run long.
    const uint32_t ninv = s.flag;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long *dtab = reinterpret_cast<unsigned long long *>(s.u.la.cnt) + warp * (WARP_DISTINCT_MAX + 16);
    uint32_t *dcur = reinterpret_cast<uint32_t *>(dtab + WARP_DISTINCT_MAX);
    for (uint32_t f = warp; f < ninv; f += WARPS) {
        const uint32_t q = inv[f], a = s.tstart[q], c = s.tcount[q];
        if (c <= LEAF_INSERT_MAX) {
            if (lane == 0) insertion_sort_budget(key + a, val + a, c, 0xffffffffu);
        } else if (warp_distinct_sort<KV>(key, val, a, c, dtab, dcur, dk, dv)) {
            if (lane == 0) s.hist[q] = 2u;
        } else if (lane == 0) {
            fail[atomicAdd(&s.flag2, 1u)] = q;
        }
        __syncwarp();
    }
    __syncthreads();
    const uint32_t nfail = s.flag2;
    for (uint32_t f = 0; f < nfail; f++) {
        const uint32_t q = fail[f];
        bitonic_range(s, key, val, s.tstart[q], s.tcount[q]);
    }
    if (threadIdx.x == 0 && nfail) atomicAdd(&P.ctl->n_leaf_fb, 1ull);
    for (uint32_t p = threadIdx.x; p < len; p += BLOCK) {
        const unsigned long long kp = key[p];
        if (s.hist[leaf_sub(kp, mn, rshift, rmult)] == 2u) continue;  // written by its warp
        __stcg(dk + p, kp);
        if (KV) __stcg(dv + p, val[p]);
    }
}

// Leaf: a group of whole buckets, at most LEAF_CAP pairs, sorted in shared
// memory and written to the caller's arrays.  Mirrors the paper's finish
// (insertion sort of small clusters, counting sort of small ranges): one
// partition of the leaf into sub-buckets by the range map, an exact counting
// sort when the key range is smaller than the sub-bucket count, then each
// sub-bucket ordered (finish_fast / finish_stable).
template <bool KV>
__device__ __noinline__ void task_finish(const Params &P, const Item it, SmemTile &s, Pipe &pp)
{
    const unsigned long long off = it.off;
    const uint32_t len = it.len, buf = it.buf;
    const uint64_t *srck = keys_of(P, buf);
    const uint32_t *srcv = vals_of(P, buf);
    uint64_t *dk = P.ukeys + off;
    uint32_t *dv = KV ? P.uvals + off : nullptr;  // keys only: no payload
    unsigned long long *key;
    uint32_t *val;
    if (bulk_ok(P, buf)) {
        if (threadIdx.x == 0) {
            const unsigned long long a0 = off & ~1ull, a1 = min((off + len + 1) & ~1ull, P.n & ~1ull);
            const unsigned long long b0 = off & ~3ull, b1 = min((off + len + 3) & ~3ull, P.n & ~3ull);
            const uint32_t bk = a1 > a0 ? (uint32_t)(a1 - a0) * 8u : 0u;
            const uint32_t bv = KV && b1 > b0 ? (uint32_t)(b1 - b0) * 4u : 0u;
            mbar_expect_arrive(&s.bar[0], bk + bv);
            if (bk) bulk_g2s(s.u.la.leaf.key, srck + a0, bk, &s.bar[0]);
            if (bv) bulk_g2s(s.u.la.leaf.val, srcv + b0, bv, &s.bar[0]);
        }
        key = s.u.la.leaf.key + (off & 1ull);
        val = s.u.la.leaf.val + (off & 3ull);
        const bool ok = mbar_wait(&s.bar[0], pp.uses[0] & 1u, P.wait_ns);
        pp.uses[0]++;
        if (__syncthreads_or(!ok)) {  // CTA-uniform: every thread leaves together
            mbar_wait(&s.bar[0], (pp.uses[0] - 1u) & 1u, P.wait_ns);  // one more bounded wait
            set_error(P, ST_TIMEOUT);
            return;
        }
        const unsigned long long end = off + len;
        for (unsigned long long e = max(off, P.n & ~1ull) + threadIdx.x; e < end; e += BLOCK)
            key[e - off] = __ldcg(srck + e);
        if (KV)
            for (unsigned long long e = max(off, P.n & ~3ull) + threadIdx.x; e < end; e += BLOCK)
                val[e - off] = __ldcg(srcv + e);
    } else {
        key = s.u.la.leaf.key;
        val = s.u.la.leaf.val;
        for (uint32_t i = threadIdx.x; i < len; i += BLOCK) {
            key[i] = __ldcg(srck + off + i);
            if (KV) val[i] = __ldcg(srcv + off + i);
        }
    }
    __syncthreads();
    // this thread's pairs (leaf positions threadIdx.x + j * BLOCK) in registers
    unsigned long long kk[LEAF_IPT];
    uint32_t vv[LEAF_IPT];
    unsigned long long mn = ~0ull, mx = 0ull;
#pragma unroll
    for (int j = 0; j < LEAF_IPT; j++) {
        const uint32_t p = threadIdx.x + j * BLOCK;
        kk[j] = p < len ? key[p] : 0ull;
        vv[j] = p < len && KV ? val[p] : 0u;
        if (p < len) {
            mn = kk[j] < mn ? kk[j] : mn;
            mx = kk[j] > mx ? kk[j] : mx;
        }
    }
    const uint32_t M2 = min(LEAF_M2_MAX, pow2ceil32(len) / 2);
    uint32_t *cnt = s.u.la.cnt;
    for (uint32_t q = threadIdx.x; q < M2; q += BLOCK) cnt[q] = 0u;
    warp_minmax64(mn, mx);
    if ((threadIdx.x & 31) == 0) {
        s.red64[threadIdx.x >> 5] = mn;
        s.red64[WARPS + (threadIdx.x >> 5)] = mx;
    }
    __syncthreads();
    mn = s.red64[0];
    mx = s.red64[WARPS];
    for (int w = 1; w < WARPS; w++) {
        mn = s.red64[w] < mn ? s.red64[w] : mn;
        mx = s.red64[WARPS + w] > mx ? s.red64[WARPS + w] : mx;
    }
    if (threadIdx.x == 0) {
        atomicAdd(&P.ctl->n_leaves, 1ull);
        atomicAdd(&P.ctl->bytes, ((buf || mn != mx) ? 2ull : 1ull) * elem_bytes(P) * len);
    }
    if (mn == mx) {  // identical keys: in order already
        if (buf) {
#pragma unroll
            for (int j = 0; j < LEAF_IPT; j++) {
                const uint32_t p = threadIdx.x + j * BLOCK;
                if (p < len) {
                    __stcg(dk + p, kk[j]);
                    if (KV) __stcg(dv + p, vv[j]);
                }
            }
        }
        return;
    }
    if (len <= (uint32_t)RANK_SMALL) {
        const uint32_t t = threadIdx.x;
        if (t < len) {
            const unsigned long long kt = kk[0];
            uint32_t r = 0;
            for (uint32_t q = 0; q < len; q++) {
                const unsigned long long kq = key[q];
                r += (kq < kt) || (kq == kt && q < t);
            }
            __stcg(dk + r, kt);
            if (KV) __stcg(dv + r, vv[0]);
        }
        return;
    }
    // sub-buckets by the range map (the counting map when max - min < M2);
    // the atomic's old value is the pair's arrival slot in its sub-bucket
    uint32_t rs2, rm2;
    range_params(mx - mn, M2, &rs2, &rm2);
    uint32_t a[LEAF_IPT];
    bool big = false;
#pragma unroll
    for (int j = 0; j < LEAF_IPT; j++) {
        const uint32_t p = threadIdx.x + j * BLOCK;
        a[j] = p < len ? atomicAdd(&cnt[leaf_sub(kk[j], mn, rs2, rm2)], 1u) : 0u;
        big = big || a[j] >= LEAF_FAST_MAX;
    }
    if (!__syncthreads_or(big))
        finish_fast<KV>(s, key, val, len, mn, rs2, rm2, M2, kk, vv, a, dk, dv);
    else
        finish_stable<KV>(P, s, key, val, len, mn, mx, dk, dv);
}

// ------------------------------------------------------------ COPY
// All-equal large (sub)array living in scratch: one LEAF_CAP slice per task.
__device__ __noinline__ void task_copy(const Params &P, uint32_t sid, uint32_t tile)
{
    const Seg *S = &P.segs[sid];
    const unsigned long long off = __ldcg(&S->off) + (size_t)tile * LEAF_CAP;
    const uint32_t len = __ldcg(&S->len);
    const uint32_t cnt = min((uint32_t)LEAF_CAP, len - tile * LEAF_CAP);
    for (uint32_t p = threadIdx.x; p < cnt; p += BLOCK) {
        __stcg(P.ukeys + off + p, __ldcg(P.skeys + off + p));
        if (P.kv) __stcg(P.uvals + off + p, __ldcg(P.svals + off + p));
    }
    if (threadIdx.x == 0) atomicAdd(&P.ctl->bytes, 2ull * elem_bytes(P) * cnt);
}

}  // namespace zs
