// zsort_tasks.cuh -- the tasks of the persistent zSort executor.
//
// Every (sub)array goes through the steps of Alg. 1: statistics (exact
// min, max, mean and population sd), the bucket map (Eq. 1, or the learned
// map, or the range map of the progress guard), a histogram, an exclusive
// scan for the bucket starts, and a stable scatter; its buckets become the
// next level's (sub)arrays, or leaves finished in shared memory.
//   large (sub)arrays  -> one task per 4096-element tile and per phase, with
//                         a decoupled look-back across tiles in the scatter
//   medium (sub)arrays -> one task that runs every phase in one CTA
//   leaves             -> one task that sorts a group of small buckets in smem
#pragma once
#include "zsort_device.cuh"

namespace zs {

// ------------------------------------------------------------ queue
// Reserves `count` consecutive entries (thread 0 only) and counts them as
// pending; returns INVALID when the queue is full (error recorded).
__device__ uint32_t q_reserve(const Params &P, uint32_t count)
{
    if (count == 0) return 0;
    uint32_t e = atomicAdd(&P.ctl->q_alloc, count);
    if (e + count > P.qcap) {
        set_error(P, ST_CAPACITY);
        return INVALID;
    }
    atomicAdd(&P.ctl->pending, count);
    return e;
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

// Publishes entries [e, e+count): one fence, then the ready flags.
__device__ void q_release_all(const Params &P, uint32_t e, uint32_t count)
{
    __threadfence();
    for (uint32_t i = 0; i < count; i++) st_release(&P.ready[e + i], P.epoch);
}

// Thread 0: next (entry, tile) to run, or T_NONE when all work is done or an
// error was recorded.  A wait without any progress anywhere for longer than
// P.wait_ns records ST_TIMEOUT.
__device__ void dequeue(const Params &P, uint32_t *out)
{
    Ctl *C = P.ctl;
    unsigned long long last = ld_relaxed64(&C->progress);
    unsigned long long t0 = globaltimer();
    out[0] = T_NONE;
    for (;;) {
        if (ld_relaxed(&C->error)) return;
        uint32_t e = ld_relaxed(&C->q_head);
        if (e < P.qcap && ld_acquire(&P.ready[e]) == P.epoch) {
            uint32_t type = __ldcg(&P.entries[e].type);
            uint32_t arg = __ldcg(&P.entries[e].arg);
            uint32_t ntiles = __ldcg(&P.entries[e].ntiles);
            uint32_t t = atomicAdd(&P.tnext[e], 1u);
            if (t < ntiles) {
                out[0] = type;
                out[1] = arg;
                out[2] = t;
                out[3] = e;
                out[4] = ntiles;
                return;
            }
            atomicCAS(&C->q_head, e, e + 1);
            continue;
        }
        if (ld_acquire(&C->pending) == 0) return;
        unsigned long long pr = ld_relaxed64(&C->progress), now = globaltimer();
        if (pr != last) {
            last = pr;
            t0 = now;
        } else if (now - t0 > P.wait_ns) {
            set_error(P, ST_TIMEOUT);
            return;
        }
        __nanosleep(200);
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

__device__ __forceinline__ uint64_t *keys_of(const Params &P, uint32_t buf)
{
    return buf ? P.skeys : P.ukeys;
}
__device__ __forceinline__ uint32_t *vals_of(const Params &P, uint32_t buf)
{
    return buf ? P.svals : P.uvals;
}

// Buckets of one partition pass: enough for leaf_target elements per bucket.
__device__ __forceinline__ uint32_t choose_k(const Params &P, uint32_t len)
{
    uint32_t k = pow2ceil32((len + P.leaf_target - 1) / P.leaf_target);
    k = k < (uint32_t)MIN_K ? (uint32_t)MIN_K : k;
    return k > P.kmax ? P.kmax : k;
}

// Fills the map for a (sub)array from its exact sums: Eq. 1 (z-score) unless
// the depth reached the guard level, in which case the exact range map.
__device__ void map_from_sums(const Params &P, unsigned long long n, unsigned long long mn,
                              unsigned long long mx, const unsigned long long s1[2],
                              const unsigned long long s2[3], uint32_t k, uint32_t level, MapSm &m,
                              double *mean_d, double *sd)
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
    m.rshift = 0;
    m.rmult = 0;
    if (level >= P.guard_level || !(*sd > 0.0)) {
        m.kind = MAP_RANGE;
        range_params(range, k, &m.rshift, &m.rmult);
        atomicAdd(&P.ctl->n_guard, 1ull);
    } else {
        // scale = k/4 (Alg. 1); |z_min| = (mean - min)/sd cancels the mean.
        m.kind = MAP_Z;
        m.zc = (float)(((double)k / 4.0) / *sd);
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

// Loads a large segment's map into shared memory (all threads).
__device__ void load_seg_map(const Params &P, uint32_t sid, SmemTile &s)
{
    const Seg *S = &P.segs[sid];
    uint32_t kind = __ldcg(&S->kind);
    if (threadIdx.x == 0) {
        s.map.mn = __ldcg(&S->mn);
        s.map.kind = kind;
        s.map.k = __ldcg(&S->k);
        s.map.K = s.map.k >= PWL_P ? s.map.k / PWL_P : 1;
        s.map.zc = __ldcg(&S->zc);
        s.map.escale = __ldcg(&S->escale);
        s.map.rshift = __ldcg(&S->rshift);
        s.map.rmult = __ldcg(&S->rmult);
    }
    if (kind == MAP_PWL)
        for (int j = threadIdx.x; j <= PWL_P; j += BLOCK)
            s.map.q[j] = __ldcg(&P.pwl[(size_t)sid * (PWL_P + 1) + j]);
    __syncthreads();
}

// ------------------------------------------------------------ children
// After a partition of the (sub)array at absolute offset poff: bucket counts
// in s.hist[0..k), starts (relative) in s.bs[0..k).  Consecutive small
// buckets are grouped into leaves of at most LEAF_CAP elements (sorting a
// group of whole, ordered buckets gives the same result as sorting each);
// larger buckets become medium or large (sub)arrays of the next level.
__device__ void classify_children(const Params &P, unsigned long long poff, uint32_t k,
                                  uint32_t child_buf, uint32_t child_level, SmemTile &s)
{
    ChildList &L = *reinterpret_cast<ChildList *>(s.key);
    if (threadIdx.x == 0) {
        uint32_t nl = 0, nm = 0, ng = 0, glen = 0, gstart = 0;
        for (uint32_t b = 0; b < k; b++) {
            uint32_t c = s.hist[b];
            if (c == 0) continue;
            if (c > (uint32_t)LEAF_CAP) {
                if (glen) {
                    L.leaf_off[nl] = gstart;
                    L.leaf_len[nl++] = glen;
                    glen = 0;
                }
                if (c <= P.large_min) {
                    L.med_off[nm] = s.bs[b];
                    L.med_len[nm++] = c;
                } else {
                    L.lg_off[ng] = s.bs[b];
                    L.lg_len[ng++] = c;
                }
            } else {
                if (glen + c > (uint32_t)LEAF_CAP) {
                    L.leaf_off[nl] = gstart;
                    L.leaf_len[nl++] = glen;
                    glen = 0;
                }
                if (glen == 0) gstart = s.bs[b];
                glen += c;
            }
        }
        if (glen) {
            L.leaf_off[nl] = gstart;
            L.leaf_len[nl++] = glen;
        }
        if (child_level > (uint32_t)MAX_LEVEL && (nm + ng) > 0) set_error(P, ST_INTERNAL);
        // large children: descriptor + look-back rows, else demoted to medium
        uint32_t nok = 0;
        for (uint32_t g = 0; g < ng; g++) {
            uint32_t len = L.lg_len[g];
            uint32_t kk = choose_k(P, len);
            uint32_t tiles = (len + TILE - 1) / TILE;
            unsigned long long need = (unsigned long long)tiles * kk;
            uint32_t sid = atomicAdd(&P.ctl->seg_alloc, 1u);
            unsigned long long sb = ~0ull;
            if (sid < P.segcap) sb = atomicAdd(&P.ctl->status_alloc, need);
            if (sid < P.segcap && sb + need <= P.statuscap) {
                Seg *S = &P.segs[sid];
                S->off = poff + L.lg_off[g];
                S->mn = ~0ull;
                S->mx = 0ull;
                S->s1[0] = S->s1[1] = 0ull;
                S->s2[0] = S->s2[1] = S->s2[2] = 0ull;
                S->status_base = sb;
                S->len = len;
                S->k = kk;
                S->tiles = tiles;
                S->level = child_level;
                S->buf = child_buf;
                S->kind = MAP_Z;
                S->train_slot = INVALID;
                L.lg_sid[nok] = sid;
                L.lg_len[nok] = len;  // compacted in place (nok <= g)
                nok++;
            } else {
                if (sid < P.segcap) P.segs[sid].len = 0;
                L.med_off[nm] = L.lg_off[g];
                L.med_len[nm++] = len;
            }
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
    }
    __syncthreads();
    const uint32_t nl = s.n_leaf, nm = s.n_med, nok = s.n_large_ok, base = s.item_base;
    for (uint32_t i = threadIdx.x; i < nl + nm; i += BLOCK) {
        Item it;
        bool leaf = i < nl;
        it.off = poff + (leaf ? L.leaf_off[i] : L.med_off[i - nl]);
        it.len = leaf ? L.leaf_len[i] : L.med_len[i - nl];
        it.buf = (uint16_t)child_buf;
        it.level = (uint16_t)child_level;
        P.items[base + i] = it;
    }
    for (uint32_t g = 0; g < nok; g++) {
        uint32_t sid = L.lg_sid[g];
        uint32_t kk = choose_k(P, L.lg_len[g]);
        for (uint32_t q = threadIdx.x; q < kk; q += BLOCK) P.counts[(size_t)sid * NB_MAX + q] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t cnt = (nl > 0) + (nm > 0) + nok;
        uint32_t e = q_reserve(P, cnt);
        if (e != INVALID && cnt) {
            uint32_t j = e;
            if (nl) q_write(P, j++, T_FINISH, base, nl);
            if (nm) q_write(P, j++, T_MPART, base + nl, nm);
            for (uint32_t g = 0; g < nok; g++) {
                uint32_t sid = L.lg_sid[g];
                q_write(P, j++, T_LSTATS, sid, (L.lg_len[g] + TILE - 1) / TILE);
            }
            q_release_all(P, e, cnt);
        }
    }
    __syncthreads();
}

// ------------------------------------------------------------ tile loads
// Element (warp, slot i, lane) of a tile at `base`: base + warp*WARP_SPAN + i*32 + lane.
__device__ __forceinline__ uint32_t slot_index(int i)
{
    return (threadIdx.x >> 5) * WARP_SPAN + i * 32 + (threadIdx.x & 31);
}

// ------------------------------------------------------------ LSTATS
__device__ void task_lstats(const Params &P, uint32_t sid, uint32_t tile, SmemTile &s)
{
    const Seg *S = &P.segs[sid];
    const unsigned long long off = __ldcg(&S->off);
    const uint32_t len = __ldcg(&S->len), buf = __ldcg(&S->buf);
    const uint64_t *src = keys_of(P, buf) + off + (size_t)tile * TILE;
    const uint32_t cnt = min((uint32_t)TILE, len - tile * TILE);
    unsigned long long x[IPT];
#pragma unroll
    for (int i = 0; i < IPT; i++) {
        uint32_t p = slot_index(i);
        x[i] = p < cnt ? __ldcg(src + p) : 0ull;
    }
    Acc a;
    acc_init(a);
#pragma unroll
    for (int i = 0; i < IPT; i++)
        if (slot_index(i) < cnt) acc_key(a, x[i]);
    acc_block_reduce(a, s.acc);
    if (threadIdx.x == 0) {
        Seg *W = &P.segs[sid];
        atomicMin(&W->mn, a.mn);
        atomicMax(&W->mx, a.mx);
        unsigned long long v1[2] = {(unsigned long long)a.s1, (unsigned long long)(a.s1 >> 64)};
        unsigned long long v2[3] = {(unsigned long long)a.s2lo, (unsigned long long)(a.s2lo >> 64), a.s2hi};
        atomic_add_wide(W->s1, v1, 2);
        atomic_add_wide(W->s2, v2, 3);
        atomicAdd(&P.ctl->bytes, 8ull * cnt);
    }
}

__device__ void lstats_done(const Params &P, uint32_t sid, SmemTile &s)
{
    if (threadIdx.x == 0) {
        Seg *S = &P.segs[sid];
        const unsigned long long mn = __ldcg(&S->mn), mx = __ldcg(&S->mx);
        const uint32_t len = __ldcg(&S->len), level = __ldcg(&S->level), tiles = __ldcg(&S->tiles);
        const uint32_t sbuf = __ldcg(&S->buf), sk = __ldcg(&S->k);
        if (mn == mx) {  // a set of identical keys is sorted (Alg. 1 early exit)
            if (sbuf) {
                uint32_t e = q_reserve(P, 1);
                if (e != INVALID) {
                    q_write(P, e, T_COPY, sid, tiles);
                    q_release_all(P, e, 1);
                }
                atomicAdd(&P.ctl->n_copies, 1ull);
            }
        } else {
            unsigned long long s1[2] = {__ldcg(&S->s1[0]), __ldcg(&S->s1[1])};
            unsigned long long s2[3] = {__ldcg(&S->s2[0]), __ldcg(&S->s2[1]), __ldcg(&S->s2[2])};
            MapSm m;
            double mean_d, sd;
            map_from_sums(P, len, mn, mx, s1, s2, sk, level, m, &mean_d, &sd);
            S->mean_d = mean_d;
            S->sd = sd;
            S->kind = m.kind;
            S->zc = m.zc;
            S->escale = m.escale;
            S->rshift = m.rshift;
            S->rmult = m.rmult;
            if (level == 0 && sid == 0) record_top(P, m, mn, mx, mean_d, sd);
            uint32_t next = T_LHIST, nt = tiles;
            if (m.kind == MAP_Z && P.mapper == 1 && len >= P.learn_min && P.sample <= len &&
                sk >= (uint32_t)PWL_P) {
                uint32_t slot = atomicAdd(&P.ctl->train_alloc, 1u);
                if (slot < P.traincap) {
                    S->train_slot = slot;
                    next = T_LTRAIN;
                    nt = 1;
                }
            }
            uint32_t e = q_reserve(P, 1);
            if (e != INVALID) {
                q_write(P, e, next, sid, nt);
                q_release_all(P, e, 1);
            }
        }
    }
}

// ------------------------------------------------------------ LTRAIN
// One stable LSD pass (8-bit digit at `shift`) of m uint32 values, src -> dst,
// by one CTA: histogram, scan, then tile by tile in input order.
__device__ void cta_lsd_pass(const uint32_t *src, uint32_t *dst, uint32_t m, uint32_t shift, SmemTile &s)
{
    for (int q = threadIdx.x; q < 256; q += BLOCK) s.hist[q] = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < m; i += BLOCK) atomicAdd(&s.hist[(__ldcg(src + i) >> shift) & 255u], 1u);
    __syncthreads();
    block_exclusive_scan(s.hist, s.cursor, 256, s.wsum);
    for (uint32_t t0 = 0; t0 < m; t0 += TILE) {
        const uint32_t cnt = min((uint32_t)TILE, m - t0);
        uint32_t v[IPT], b[IPT], pos[IPT];
#pragma unroll
        for (int i = 0; i < IPT; i++) {
            uint32_t p = slot_index(i);
            v[i] = p < cnt ? __ldcg(src + t0 + p) : 0u;
            b[i] = p < cnt ? (v[i] >> shift) & 255u : INVALID;
        }
        tile_rank(b, pos, 256, s);
#pragma unroll
        for (int i = 0; i < IPT; i++)
            if (b[i] != INVALID) __stcg(dst + s.cursor[b[i]] + pos[i] - s.tstart[b[i]], v[i]);
        __syncthreads();
        for (int q = threadIdx.x; q < 256; q += BLOCK) s.cursor[q] += s.tcount[q];
        __syncthreads();
    }
}

// Bucket of a normalised key u under the learned map in s.map (the part of
// map_key after the normalisation).
__device__ __forceinline__ uint32_t pwl_bucket_u(const MapSm &m, float u)
{
    int s = 0;
#pragma unroll
    for (int st = PWL_P / 2; st; st >>= 1)
        if (m.q[s + st] <= u) s += st;
    float lo = m.q[s], hi = m.q[s + 1];
    float frac = 0.0f;
    if (hi > lo) frac = __fdiv_rn(__fsub_rn(u, lo), __fsub_rn(hi, lo));
    frac = fminf(fmaxf(frac, 0.0f), 0x1.fffffep-1f);
    uint32_t w = __float2uint_rz(__fmul_rn(frac, (float)m.K));
    w = w < m.K ? w : m.K - 1;
    return (uint32_t)s * m.K + w;
}

// Learned-map training: sample, exact sort of the normalised sample,
// breakpoints at the 1/256 quantiles, then the load test that keeps Eq. 1
// as the fallback.
__device__ void task_ltrain(const Params &P, uint32_t sid, SmemTile &s)
{
    Seg *S = &P.segs[sid];
    const unsigned long long off = __ldcg(&S->off), mn = __ldcg(&S->mn), mx = __ldcg(&S->mx);
    const uint32_t len = __ldcg(&S->len), buf = __ldcg(&S->buf), k = __ldcg(&S->k);
    const uint32_t slot = __ldcg(&S->train_slot), tiles = __ldcg(&S->tiles);
    const float escale = __ldcg(&S->escale), zc = __ldcg(&S->zc);
    const uint32_t m = P.sample;
    uint32_t *A = P.trainbuf + (size_t)slot * 2 * SAMPLE_MAX;
    uint32_t *B = A + SAMPLE_MAX;
    const uint64_t *src = keys_of(P, buf) + off;
    for (uint32_t i = threadIdx.x; i < m; i += BLOCK) {
        unsigned long long pos = sample_pos(P.seed, len, m, i);
        unsigned long long key = __ldcg(src + pos);
        float u = __fmul_rn(__ull2float_rn(key - mn), escale);
        __stcg(A + i, __float_as_uint(u));
    }
    __syncthreads();
    // non-negative floats order as their bit patterns
    cta_lsd_pass(A, B, m, 0, s);
    cta_lsd_pass(B, A, m, 8, s);
    cta_lsd_pass(A, B, m, 16, s);
    cta_lsd_pass(B, A, m, 24, s);
    if (threadIdx.x == 0) {
        s.map.mn = mn;
        s.map.kind = MAP_PWL;
        s.map.k = k;
        s.map.K = k / PWL_P;
        s.map.escale = escale;
        s.map.zc = zc;
    }
    for (int j = threadIdx.x; j <= PWL_P; j += BLOCK) {
        float q;
        if (j == 0)
            q = 0.0f;
        else if (j == PWL_P)
            q = __fmul_rn(__ull2float_rn(mx - mn), escale);
        else
            q = __uint_as_float(__ldcg(A + (size_t)j * m / PWL_P));
        s.map.q[j] = q;
        P.pwl[(size_t)sid * (PWL_P + 1) + j] = q;
    }
    for (uint32_t q = threadIdx.x; q < k; q += BLOCK) {
        s.hist[q] = 0;
        s.cursor[q] = 0;
    }
    __syncthreads();
    // load test on the sample: largest learned bucket vs largest Eq. 1 bucket
    // 2^E from escale = 2^-E (exponent field 127 - E -> 127 + E)
    const float two_e = __uint_as_float((uint32_t)(254 - ((__float_as_uint(escale) >> 23) & 0xff)) << 23);
    for (uint32_t i = threadIdx.x; i < m; i += BLOCK) {
        float u = __uint_as_float(__ldcg(A + i));
        atomicAdd(&s.hist[pwl_bucket_u(s.map, u)], 1u);
        float fd = __fmul_rn(u, two_e);  // = fl32(key - min), exactly
        uint32_t bz = __float2uint_rz(__fmul_rn(fd, zc));
        atomicAdd(&s.cursor[bz < k ? bz : k - 1], 1u);
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
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < WARPS; w++) {
            ml = max(ml, (uint32_t)s.red64[w]);
            mz = max(mz, (uint32_t)s.red64[WARPS + w]);
        }
        const bool ok = (float)ml <= P.fallback_ratio * (float)m / (float)k && ml <= mz;
        S->kind = ok ? MAP_PWL : MAP_Z;
        atomicAdd(ok ? &P.ctl->n_learn_ok : &P.ctl->n_learn_rej, 1ull);
        if (__ldcg(&S->level) == 0 && sid == 0) P.ctl->top_map = ok ? MAP_PWL : MAP_Z;
        uint32_t e = q_reserve(P, 1);
        if (e != INVALID) {
            q_write(P, e, T_LHIST, sid, tiles);
            q_release_all(P, e, 1);
        }
    }
}

// ------------------------------------------------------------ LHIST
__device__ void task_lhist(const Params &P, uint32_t sid, uint32_t tile, SmemTile &s)
{
    load_seg_map(P, sid, s);
    const Seg *S = &P.segs[sid];
    const unsigned long long off = __ldcg(&S->off), sbase = __ldcg(&S->status_base);
    const uint32_t len = __ldcg(&S->len), buf = __ldcg(&S->buf), k = s.map.k;
    const uint32_t cnt = min((uint32_t)TILE, len - tile * TILE);
    const uint64_t *src = keys_of(P, buf) + off + (size_t)tile * TILE;
    uint32_t *row = P.status + sbase + (size_t)tile * k;
    for (uint32_t q = threadIdx.x; q < k; q += BLOCK) {
        s.hist[q] = 0;
        __stcg(row + q, 0u);
    }
    unsigned long long x[IPT];
#pragma unroll
    for (int i = 0; i < IPT; i++) {
        uint32_t p = slot_index(i);
        x[i] = p < cnt ? __ldcg(src + p) : 0ull;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < IPT; i++) {
        uint32_t b = slot_index(i) < cnt ? map_key(s.map, x[i]) : INVALID;
        uint32_t peers = __match_any_sync(0xffffffffu, b);
        if (b != INVALID && lane == __ffs(peers) - 1) atomicAdd(&s.hist[b], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < k; q += BLOCK)
        if (s.hist[q]) atomicAdd(&P.counts[(size_t)sid * NB_MAX + q], s.hist[q]);
    if (threadIdx.x == 0) atomicAdd(&P.ctl->bytes, 8ull * cnt);
}

__device__ void lhist_done(const Params &P, uint32_t sid, SmemTile &s)
{
    const Seg *S = &P.segs[sid];
    const uint32_t k = __ldcg(&S->k), tiles = __ldcg(&S->tiles);
    for (uint32_t q = threadIdx.x; q < k; q += BLOCK) s.hist[q] = __ldcg(&P.counts[(size_t)sid * NB_MAX + q]);
    __syncthreads();
    block_exclusive_scan(s.hist, s.bs, k, s.wsum);
    for (uint32_t q = threadIdx.x; q < k; q += BLOCK) P.bstart[(size_t)sid * NB_MAX + q] = s.bs[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t e = q_reserve(P, 1);
        if (e != INVALID) {
            q_write(P, e, T_LSCATTER, sid, tiles);
            q_release_all(P, e, 1);
        }
    }
}

// ------------------------------------------------------------ LSCATTER
// Decoupled look-back: tile t publishes, per bucket, its count (FLAG_A) and
// then its inclusive prefix over tiles 0..t (FLAG_P); it finds its exclusive
// prefix by walking back over predecessors until one has FLAG_P.  Tiles are
// handed out in increasing order, so a predecessor is always running or done.
__device__ void task_lscatter(const Params &P, uint32_t sid, uint32_t tile, SmemTile &s)
{
    load_seg_map(P, sid, s);
    const Seg *S = &P.segs[sid];
    const unsigned long long off = __ldcg(&S->off), sbase = __ldcg(&S->status_base);
    const uint32_t len = __ldcg(&S->len), buf = __ldcg(&S->buf), k = s.map.k;
    const uint32_t cnt = min((uint32_t)TILE, len - tile * TILE);
    const uint64_t *srck = keys_of(P, buf) + off + (size_t)tile * TILE;
    const uint32_t *srcv = vals_of(P, buf) + off + (size_t)tile * TILE;
    uint64_t *dstk = keys_of(P, buf ^ 1u) + off;
    uint32_t *dstv = vals_of(P, buf ^ 1u) + off;
    unsigned long long x[IPT];
    uint32_t v[IPT], b[IPT], pos[IPT];
#pragma unroll
    for (int i = 0; i < IPT; i++) {
        uint32_t p = slot_index(i);
        x[i] = p < cnt ? __ldcg(srck + p) : 0ull;
        v[i] = p < cnt ? __ldcg(srcv + p) : 0u;
    }
#pragma unroll
    for (int i = 0; i < IPT; i++) b[i] = slot_index(i) < cnt ? map_key(s.map, x[i]) : INVALID;
    tile_rank(b, pos, k, s);
    uint32_t *status = P.status + sbase;
    uint32_t *row = status + (size_t)tile * k;
    for (uint32_t q = threadIdx.x; q < k; q += BLOCK) st_relaxed(row + q, (tile == 0 ? FLAG_P : FLAG_A) | s.tcount[q]);
    // look-back, up to NB_MAX / BLOCK buckets per thread, polled together
    constexpr int PER = NB_MAX / BLOCK;
    uint32_t excl[PER], j[PER];
    bool done[PER];
#pragma unroll
    for (int r = 0; r < PER; r++) {
        excl[r] = 0;
        j[r] = tile;
        done[r] = (threadIdx.x + r * BLOCK >= k) || tile == 0;
    }
    unsigned long long t0 = 0;
    uint32_t spins = 0;
    bool timed_out = false;
    for (;;) {
        bool all = true, moved = false;
#pragma unroll
        for (int r = 0; r < PER; r++) {
            if (done[r]) continue;
            const uint32_t q = threadIdx.x + r * BLOCK;
            uint32_t w = ld_relaxed(status + (size_t)(j[r] - 1) * k + q);
            uint32_t f = w & ~VAL_MASK;
            if (f == FLAG_P) {
                excl[r] += w & VAL_MASK;
                done[r] = true;
                st_relaxed(row + q, FLAG_P | (excl[r] + s.tcount[q]));
                moved = true;
            } else if (f == FLAG_A && j[r] > 1) {
                excl[r] += w & VAL_MASK;
                j[r]--;
                moved = true;
            } else if (f == FLAG_A || f == (FLAG_A | FLAG_P)) {
                set_error(P, ST_INTERNAL);  // tile 0 always publishes FLAG_P
                done[r] = true;
            } else {
                all = false;
            }
        }
#pragma unroll
        for (int r = 0; r < PER; r++) all = all && done[r];
        if (all) break;
        if (!moved) {
            if ((++spins & 31u) == 0) {
                unsigned long long now = globaltimer();
                if (t0 == 0)
                    t0 = now;
                else if (now - t0 > P.wait_ns) {
                    timed_out = true;
                    break;
                }
                if (has_error(P)) {
                    timed_out = true;
                    break;
                }
            }
        }
    }
    if (timed_out) set_error(P, ST_TIMEOUT);
#pragma unroll
    for (int r = 0; r < PER; r++) {
        const uint32_t q = threadIdx.x + r * BLOCK;
        if (q < k) s.gdelta[q] = __ldcg(&P.bstart[(size_t)sid * NB_MAX + q]) + excl[r] - s.tstart[q];
    }
    if (threadIdx.x == 0) s.flag = timed_out ? 1u : 0u;
    __syncthreads();
    const bool skip = s.flag != 0 || has_error(P);
#pragma unroll
    for (int i = 0; i < IPT; i++) {
        if (b[i] != INVALID) {
            s.key[pos[i]] = x[i];
            s.val[pos[i]] = v[i];
            s.bkt[pos[i]] = (uint16_t)b[i];
        }
    }
    __syncthreads();
    if (!skip) {
        for (uint32_t p = threadIdx.x; p < cnt; p += BLOCK) {
            uint32_t rel = s.gdelta[s.bkt[p]] + p;
            if (rel < len) {
                __stcg(dstk + rel, s.key[p]);
                __stcg(dstv + rel, s.val[p]);
            } else {
                set_error(P, ST_INTERNAL);
            }
        }
    }
    if (threadIdx.x == 0) atomicAdd(&P.ctl->bytes, 24ull * cnt);
}

__device__ void lscatter_done(const Params &P, uint32_t sid, SmemTile &s)
{
    const Seg *S = &P.segs[sid];
    const uint32_t k = __ldcg(&S->k), buf = __ldcg(&S->buf), level = __ldcg(&S->level);
    const unsigned long long off = __ldcg(&S->off);
    for (uint32_t q = threadIdx.x; q < k; q += BLOCK) {
        s.hist[q] = __ldcg(&P.counts[(size_t)sid * NB_MAX + q]);
        s.bs[q] = __ldcg(&P.bstart[(size_t)sid * NB_MAX + q]);
    }
    if (threadIdx.x == 0) {
        atomicAdd(&P.ctl->n_large, 1ull);
        note_level(P, level);
    }
    __syncthreads();
    classify_children(P, off, k, buf ^ 1u, level + 1, s);
}

// ------------------------------------------------------------ MPART
// A medium (sub)array: every step of Alg. 1 by one CTA, tile by tile in input
// order, so the scatter is stable with plain running bucket cursors.
__device__ void task_mpart(const Params &P, const Item it, SmemTile &s)
{
    const unsigned long long off = it.off;
    const uint32_t len = it.len, buf = it.buf, level = it.level;
    const uint64_t *srck = keys_of(P, buf) + off;
    const uint32_t *srcv = vals_of(P, buf) + off;
    // statistics (exact sums)
    Acc a;
    acc_init(a);
    for (uint32_t t0 = 0; t0 < len; t0 += TILE) {
        const uint32_t cnt = min((uint32_t)TILE, len - t0);
        unsigned long long x[IPT];
#pragma unroll
        for (int i = 0; i < IPT; i++) {
            uint32_t p = slot_index(i);
            x[i] = p < cnt ? __ldcg(srck + t0 + p) : 0ull;
        }
#pragma unroll
        for (int i = 0; i < IPT; i++)
            if (slot_index(i) < cnt) acc_key(a, x[i]);
    }
    acc_block_reduce(a, s.acc);
    if (threadIdx.x == 0) {
        if (a.mn == a.mx) {
            s.flag = 1;
        } else {
            s.flag = 0;
            unsigned long long s1[2] = {(unsigned long long)a.s1, (unsigned long long)(a.s1 >> 64)};
            unsigned long long s2[3] = {(unsigned long long)a.s2lo, (unsigned long long)(a.s2lo >> 64), a.s2hi};
            double mean_d, sd;
            map_from_sums(P, len, a.mn, a.mx, s1, s2, choose_k(P, len), level, s.map, &mean_d, &sd);
            if (level == 0 && off == 0) record_top(P, s.map, a.mn, a.mx, mean_d, sd);
        }
    }
    __syncthreads();
    if (s.flag) {  // identical keys: already sorted
        if (buf) {
            for (uint32_t p = threadIdx.x; p < len; p += BLOCK) {
                __stcg(P.ukeys + off + p, __ldcg(srck + p));
                __stcg(P.uvals + off + p, __ldcg(srcv + p));
            }
            if (threadIdx.x == 0) {
                atomicAdd(&P.ctl->n_copies, 1ull);
                atomicAdd(&P.ctl->bytes, 8ull * len + 24ull * len);
            }
        } else if (threadIdx.x == 0) {
            atomicAdd(&P.ctl->bytes, 8ull * len);
        }
        return;
    }
    const uint32_t k = s.map.k;
    const int lane = threadIdx.x & 31;
    // histogram
    for (uint32_t q = threadIdx.x; q < k; q += BLOCK) s.hist[q] = 0;
    __syncthreads();
    for (uint32_t t0 = 0; t0 < len; t0 += TILE) {
        const uint32_t cnt = min((uint32_t)TILE, len - t0);
        unsigned long long x[IPT];
#pragma unroll
        for (int i = 0; i < IPT; i++) {
            uint32_t p = slot_index(i);
            x[i] = p < cnt ? __ldcg(srck + t0 + p) : 0ull;
        }
#pragma unroll
        for (int i = 0; i < IPT; i++) {
            uint32_t b = slot_index(i) < cnt ? map_key(s.map, x[i]) : INVALID;
            uint32_t peers = __match_any_sync(0xffffffffu, b);
            if (b != INVALID && lane == __ffs(peers) - 1) atomicAdd(&s.hist[b], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    block_exclusive_scan(s.hist, s.bs, k, s.wsum);
    for (uint32_t q = threadIdx.x; q < k; q += BLOCK) s.cursor[q] = s.bs[q];
    __syncthreads();
    // stable scatter, tile by tile
    uint64_t *dstk = keys_of(P, buf ^ 1u) + off;
    uint32_t *dstv = vals_of(P, buf ^ 1u) + off;
    for (uint32_t t0 = 0; t0 < len; t0 += TILE) {
        const uint32_t cnt = min((uint32_t)TILE, len - t0);
        unsigned long long x[IPT];
        uint32_t v[IPT], b[IPT], pos[IPT];
#pragma unroll
        for (int i = 0; i < IPT; i++) {
            uint32_t p = slot_index(i);
            x[i] = p < cnt ? __ldcg(srck + t0 + p) : 0ull;
            v[i] = p < cnt ? __ldcg(srcv + t0 + p) : 0u;
        }
#pragma unroll
        for (int i = 0; i < IPT; i++) b[i] = slot_index(i) < cnt ? map_key(s.map, x[i]) : INVALID;
        tile_rank(b, pos, k, s);
        for (uint32_t q = threadIdx.x; q < k; q += BLOCK) s.gdelta[q] = s.cursor[q] - s.tstart[q];
#pragma unroll
        for (int i = 0; i < IPT; i++) {
            if (b[i] != INVALID) {
                s.key[pos[i]] = x[i];
                s.val[pos[i]] = v[i];
                s.bkt[pos[i]] = (uint16_t)b[i];
            }
        }
        __syncthreads();
        for (uint32_t p = threadIdx.x; p < cnt; p += BLOCK) {
            uint32_t rel = s.gdelta[s.bkt[p]] + p;
            if (rel < len) {
                __stcg(dstk + rel, s.key[p]);
                __stcg(dstv + rel, s.val[p]);
            } else {
                set_error(P, ST_INTERNAL);
            }
        }
        __syncthreads();
        for (uint32_t q = threadIdx.x; q < k; q += BLOCK) s.cursor[q] += s.tcount[q];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(&P.ctl->n_small, 1ull);
        atomicAdd(&P.ctl->bytes, 40ull * len);
        note_level(P, level);
    }
    classify_children(P, off, k, buf ^ 1u, level + 1, s);
}

// ------------------------------------------------------------ FINISH
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

// Bitonic sort of s.key/s.val[0..len) by (key, current position): stable.
__device__ void bitonic_fallback(SmemTile &s, uint32_t len)
{
    const uint32_t L = pow2ceil32(len);
    for (uint32_t p = threadIdx.x; p < L; p += BLOCK) {
        if (p >= len) {
            s.key[p] = ~0ull;
            s.val[p] = 0u;
            s.bkt[p] = 0xFFFFu;
        } else {
            s.bkt[p] = (uint16_t)p;
        }
    }
    __syncthreads();
    for (uint32_t size = 2; size <= L; size <<= 1) {
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (uint32_t t = threadIdx.x; t < L / 2; t += BLOCK) {
                uint32_t i = 2 * stride * (t / stride) + (t % stride);
                uint32_t jj = i + stride;
                bool asc = (i & size) == 0;
                unsigned long long ki = s.key[i], kj = s.key[jj];
                uint16_t ii = s.bkt[i], ij = s.bkt[jj];
                bool gt = ki > kj || (ki == kj && ii > ij);
                if (gt == asc) {
                    s.key[i] = kj;
                    s.key[jj] = ki;
                    s.bkt[i] = ij;
                    s.bkt[jj] = ii;
                    uint32_t tv = s.val[i];
                    s.val[i] = s.val[jj];
                    s.val[jj] = tv;
                }
            }
            __syncthreads();
        }
    }
}

// Leaf: a group of whole buckets, at most LEAF_CAP pairs, sorted in shared
// memory and written to the caller's arrays.  Mirrors the paper's finish
// (insertion sort of small clusters, counting sort of small ranges): a
// range-map partition into sub-buckets (exact counting sort when the key
// range is smaller than the sub-bucket count), then insertion sort of each
// sub-bucket; a bitonic sort is the fallback for a badly split leaf.
__device__ void task_finish(const Params &P, const Item it, SmemTile &s)
{
    const unsigned long long off = it.off;
    const uint32_t len = it.len, buf = it.buf;
    const uint64_t *srck = keys_of(P, buf) + off;
    const uint32_t *srcv = vals_of(P, buf) + off;
    uint64_t *dk = P.ukeys + off;
    uint32_t *dv = P.uvals + off;
    unsigned long long x[IPT];
    uint32_t v[IPT];
    unsigned long long mn = ~0ull, mx = 0ull;
#pragma unroll
    for (int i = 0; i < IPT; i++) {
        uint32_t p = slot_index(i);
        x[i] = p < len ? __ldcg(srck + p) : 0ull;
        v[i] = p < len ? __ldcg(srcv + p) : 0u;
        if (p < len) {
            mn = x[i] < mn ? x[i] : mn;
            mx = x[i] > mx ? x[i] : mx;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        unsigned long long a = shfl_down64(mn, o), b2 = shfl_down64(mx, o);
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
    if (threadIdx.x == 0) {
        atomicAdd(&P.ctl->n_leaves, 1ull);
        atomicAdd(&P.ctl->bytes, (buf || mn != mx) ? 24ull * len : 12ull * len);
    }
    if (mn == mx) {  // identical keys: in order already
        if (buf) {
#pragma unroll
            for (int i = 0; i < IPT; i++) {
                uint32_t p = slot_index(i);
                if (p < len) {
                    __stcg(dk + p, x[i]);
                    __stcg(dv + p, v[i]);
                }
            }
        }
        return;
    }
    if (len <= (uint32_t)RANK_SMALL) {
#pragma unroll
        for (int i = 0; i < IPT; i++) {
            uint32_t p = slot_index(i);
            if (p < len) {
                s.key[p] = x[i];
                s.val[p] = v[i];
            }
        }
        __syncthreads();
        const uint32_t t = threadIdx.x;
        if (t < len) {
            const unsigned long long kt = s.key[t];
            uint32_t r = 0;
            for (uint32_t q = 0; q < len; q++) {
                unsigned long long kq = s.key[q];
                r += (kq < kt) || (kq == kt && q < t);
            }
            __stcg(dk + r, kt);
            __stcg(dv + r, s.val[t]);
        }
        return;
    }
    // sub-buckets: range map with M buckets (counting map if max - min < M)
    const uint32_t M = min((uint32_t)NB_MAX, pow2ceil32(len) / 4);
    uint32_t rshift, rmult;
    range_params(mx - mn, M, &rshift, &rmult);
    uint32_t b[IPT], pos[IPT];
#pragma unroll
    for (int i = 0; i < IPT; i++) {
        if (slot_index(i) < len) {
            unsigned long long d = x[i] - mn;
            b[i] = rmult == 0 ? (uint32_t)d : __umulhi((uint32_t)(d >> rshift), rmult);
        } else {
            b[i] = INVALID;
        }
    }
    tile_rank(b, pos, M, s);
#pragma unroll
    for (int i = 0; i < IPT; i++) {
        if (b[i] != INVALID) {
            s.key[pos[i]] = x[i];
            s.val[pos[i]] = v[i];
        }
    }
    if (threadIdx.x == 0) s.flag = 0;
    __syncthreads();
    bool ok = true;
    for (uint32_t q = threadIdx.x; q < M; q += BLOCK) {
        const uint32_t c = s.tcount[q];
        if (c >= 2) ok = ok && insertion_sort_budget(s.key + s.tstart[q], s.val + s.tstart[q], c, 1024);
    }
    if (!ok) s.flag = 1;
    __syncthreads();
    if (s.flag) {
        bitonic_fallback(s, len);
        if (threadIdx.x == 0) atomicAdd(&P.ctl->n_leaf_fb, 1ull);
    }
    for (uint32_t p = threadIdx.x; p < len; p += BLOCK) {
        __stcg(dk + p, s.key[p]);
        __stcg(dv + p, s.val[p]);
    }
}

// ------------------------------------------------------------ COPY
__device__ void task_copy(const Params &P, uint32_t sid, uint32_t tile)
{
    const Seg *S = &P.segs[sid];
    const unsigned long long off = __ldcg(&S->off) + (size_t)tile * TILE;
    const uint32_t len = __ldcg(&S->len);
    const uint32_t cnt = min((uint32_t)TILE, len - tile * TILE);
    for (uint32_t p = threadIdx.x; p < cnt; p += BLOCK) {
        __stcg(P.ukeys + off + p, __ldcg(P.skeys + off + p));
        __stcg(P.uvals + off + p, __ldcg(P.svals + off + p));
    }
    if (threadIdx.x == 0) atomicAdd(&P.ctl->bytes, 24ull * cnt);
}

}  // namespace zs
