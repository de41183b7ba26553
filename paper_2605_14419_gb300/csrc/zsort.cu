// zsort.cu -- kernels and C ABI of the GB300 zSort (see include/zsort.h).
//
// One call = four stream-ordered operations: clear the control block,
// classify the (segment) inputs, publish the first queue entries, then ONE
// persistent kernel (one or two CTAs per SM) that pulls tasks from a device
// work queue until every (sub)array is sorted.  Nothing on the path runs on
// the host or falls back to it; the host only sizes the workspace and
// launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/zsort.h"
#include "zsort_tasks.cuh"

static_assert(sizeof(zsort_trace_rec) == sizeof(zs::TraceRec), "trace record layout");
static_assert(ZSORT_TILE_PAIRS == zs::TILE, "tile size in the header");
static_assert(ZSORT_SUB_SAMPLE == zs::SUB_SAMPLE, "sub-array sample size in the header");

using namespace zs;

// ---------------------------------------------------------------- kernels
// Thread 0: one record of the task trace (records past the buffer are
// counted, not written).
__device__ __noinline__ void trace_task(const Params &P, uint32_t type, uint32_t arg, uint32_t tile0, uint32_t count,
                                        unsigned long long t0, unsigned long long t1)
{
    const unsigned long long i = atomicAdd(&P.ctl->trace_n, 1ull);
    if (i >= P.trace_cap) return;
    uint32_t level = 0, a = arg;
    const uint32_t base = type & (TRACE_HANDLER - 1u);
    if (base == T_MPART || base == T_FINISH) {
        a = arg + tile0;
        level = load_item(P, a).level & (ITEM_RANGE_MAP - 1u);
    } else if (base != T_NONE && arg < P.segcap) {
        level = __ldcg(&P.segs[arg].level);
    }
    TraceRec r;
    r.t_start = t0;
    r.t_end = t1;
    r.cta = blockIdx.x;
    r.type = (uint16_t)type;
    r.level = (uint16_t)min(level, 0xffffu);
    r.arg = a;
    r.count = count;
    P.trace[i] = r;
}

__global__ void __launch_bounds__(BLOCK, 2) k_persistent(const __grid_constant__ Params P)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    SmemTile &s = *reinterpret_cast<SmemTile *>(smraw);
    if (threadIdx.x == 0) {
        s.drain = 0u;
        s.local_base = 0u;
        s.local_n = 0u;
        for (int w = 0; w < KEY_STAGES; w++) mbar_init(&s.bar[w]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    Pipe pp;
    for (int w = 0; w < KEY_STAGES; w++) pp.uses[w] = 0;
    unsigned long long t_idle0 = 0, t_task0 = 0, t_task1 = 0;
    const uint32_t ep = threadIdx.x < 32 ? call_epoch(P) : 0u;  // this call's queue epoch (set before launch)
    for (;;) {
        if (threadIdx.x < 32) {  // warp 0 finds the next work: this CTA's stash first, then the queue
            t_idle0 = globaltimer();
            uint32_t local = 0;
            if (threadIdx.x == 0 && s.local_n) {
                const uint32_t c = min(s.local_n, (uint32_t)LOCAL_CLAIM);
                s.task[0] = T_FINISH;
                s.task[1] = s.local_base;
                s.task[2] = 0;
                s.task[3] = INVALID;  // no queue entry
                s.task[4] = 0;
                s.task[5] = c;
                s.local_base += c;
                s.local_n -= c;
                local = 1;
            }
            if (!__shfl_sync(0xffffffffu, local, 0)) dequeue(P, ep, s.task);
            t_task0 = globaltimer();
            if (threadIdx.x == 0) {
                atomicAdd(&P.ctl->idle_ns, t_task0 - t_idle0);
                if (s.task[0] != T_NONE) atomicMin(&P.ctl->t_first, t_task0);
            }
        }
        __syncthreads();
        const uint32_t type = s.task[0], arg = s.task[1], tile0 = s.task[2];
        const uint32_t e = s.task[3], ntiles = s.task[4], count = s.task[5];
        __syncthreads();
        if (type == T_NONE) return;
        for (uint32_t j = 0; j < count; j++) {
            const uint32_t tile = tile0 + j;
            switch (type) {
            case T_LSTATS: task_lstats(P, arg, tile, s, pp); break;
            case T_LSAMPLE: task_lsample(P, arg, tile, s); break;
            case T_LFIT: task_lfit(P, arg, s); break;
            case T_SSTATS: task_sstats(P, arg, s); break;
            case T_LHIST: task_lhist(P, arg, tile, s, pp); break;
            case T_LSCATTER: task_lscatter(P, arg, tile, s, pp); break;
            case T_MPART: task_mpart(P, load_item(P, arg + tile), s, pp); break;
            case T_FINISH:
                if (threadIdx.x == 0 && j + 1 < count) prefetch_item_l2(P, load_item(P, arg + tile + 1));
                if (P.kv)
                    task_finish<true>(P, load_item(P, arg + tile), s, pp);
                else
                    task_finish<false>(P, load_item(P, arg + tile), s, pp);
                break;
            case T_COPY: task_copy(P, arg, tile); break;
            case T_DUMP: task_dump(P, arg, tile, s, pp); break;
            default: set_error(P, ST_INTERNAL); break;
            }
            fence_proxy_async();  // order this task's smem writes before later bulk copies
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const unsigned long long t1 = globaltimer();
            t_task1 = t1;
            // the learned map's fit counts as its training, a sampled
            // statistics task as statistics
            const uint32_t ti = type == T_LFIT ? (uint32_t)T_LSAMPLE : type == T_SSTATS ? (uint32_t)T_LSTATS : (type & 7u);
            atomicAdd(&P.ctl->task_ns[ti], t1 - t_task0);
            atomicAdd(&P.ctl->task_cnt[ti], (unsigned long long)count);
            __threadfence();
            if (e != INVALID) {
                const uint32_t old = atomicAdd(&P.tdone[e], count);
                s.flag2 = (old + count == ntiles) ? 1u : 0u;
            } else {
                s.flag2 = 0u;  // stashed leaves: no entry, no completion work
            }
            atomicAdd(&P.ctl->progress, 1ull);
            atomicAdd(&P.ctl->tasks, (unsigned long long)count);
        }
        __syncthreads();
        if (s.flag2) {
            __threadfence();
            switch (type) {
            case T_LSTATS: lstats_done(P, arg, s); break;
            case T_LHIST: lhist_done(P, arg, s); break;
            case T_LSCATTER: lscatter_done(P, arg, s); break;
            default: break;  // LSAMPLE, LFIT and SSTATS publish their successors themselves
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicSub(&P.ctl->pending, 1u);
            }
        }
        if (threadIdx.x == 0) {
            unsigned long long t2 = globaltimer();
            if (s.flag2) atomicAdd(&P.ctl->handler_ns, t2 - t_task1);  // the completion work alone
            atomicMax(&P.ctl->t_last, t2);
            if (P.trace) {
                trace_task(P, type, arg, tile0, count, t_task0, t_task1);
                if (s.flag2) trace_task(P, TRACE_HANDLER | type, arg, tile0, 0, t_task1, t2);
            }
        }
    }
}

// Classifies each input segment: leaf (<= LEAF_CAP), medium (<= large_min),
// or large (own descriptor and look-back rows).  off == nullptr means one
// segment [0, n).  Leaves are staged in items[0, nseg), mediums in
// items[nseg, 2 nseg).
__global__ void k_init_segments(Params P, const uint64_t *off, unsigned long long nseg)
{
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nseg) return;
    if (P.test_badoff) {  // injected: as if the offsets had failed the check, nothing is published
        if (i == 0) set_error(P, ST_BAD_OFFSETS);
        return;
    }
    const unsigned long long a = off ? off[i] : 0ull, b = off ? off[i + 1] : P.n;
    if (a > b || b > P.n) {
        set_error(P, ST_BAD_OFFSETS);
        return;
    }
    const unsigned long long len = b - a;
    if (len <= 1) return;
    if (len > (1ull << 30)) {  // per-(sub)array counts are 30-bit
        set_error(P, ST_BAD_OFFSETS);
        return;
    }
    Ctl *C = P.ctl;
    Item it;
    it.off = a;
    it.len = (uint32_t)len;
    it.buf = 0;
    it.level = 0;
    if (len <= (unsigned long long)P.leaf_cap && !P.plan_out) {
        uint32_t j = atomicAdd(&C->init_leaf, 1u);
        P.items[j] = it;
        return;
    }
    if (len > P.large_min || P.plan_out) {
        const uint32_t kk = choose_k(P, (uint32_t)len);
        const uint32_t tiles = (uint32_t)((len + P.tile - 1) / P.tile);
        const ChunkPlan cp = chunk_plan(P, tiles, (uint32_t)len);
        const uint32_t chunks = cp.chunks;
        const unsigned long long need = 2ull * chunks * kk;
        const uint32_t sid = atomicAdd(&C->seg_alloc, 1u);
        unsigned long long sb = ~0ull;
        if (sid < P.segcap) sb = atomicAdd(&C->status_alloc, need);
        if (sid < P.segcap && sb + need <= P.statuscap) {
            Seg *S = &P.segs[sid];
            S->off = a;
            S->mn = ~0ull;
            S->mx = 0ull;
            S->s1[0] = S->s1[1] = 0ull;
            S->s2[0] = S->s2[1] = S->s2[2] = 0ull;
            S->status_base = sb;
            S->len = (uint32_t)len;
            S->k = kk;
            S->tiles = tiles;
            S->chunk_tiles = cp.ct;
            S->chunk_tiles_small = cp.ct_small;
            S->chunks_big = cp.big;
            S->chunks = chunks;
            S->level = 0;
            S->buf = 0;
            S->kind = MAP_Z;
            S->range_map = 0;
            S->train_slot = take_train_slot(P, (uint32_t)len, kk, 0);
            S->join = 2;
            S->runs_left = SAMPLE_RUNS;
            S->max_learned = S->max_z = 0;
            return;
        }
        if (sid < P.segcap) P.segs[sid].len = 0;  // no room: partitioned by one CTA
    }
    uint32_t j = atomicAdd(&C->init_med, 1u);
    P.items[nseg + j] = it;
}

// Publishes the first entries (after k_init_segments, same stream).
__global__ void k_init_publish(Params P, unsigned long long nseg)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    Ctl *C = P.ctl;
    if (C->error) {
        C->pending = 0;
        return;
    }
    // a fresh epoch for this call: ready words of earlier calls never match
    uint32_t ep = *P.epoch_ctr + 1u;
    if (ep == 0) ep = 1;
    *P.epoch_ctr = ep;
    C->epoch = ep;
    const uint32_t nl = C->init_leaf, nm = C->init_med;
    const uint32_t ns = min(C->seg_alloc, P.segcap);
    uint32_t e = 0;  // partition queue; the leaf entry goes to the leaf queue
    if (nm) q_write(P, e++, T_MPART, (uint32_t)nseg, nm);
    for (uint32_t sid = 0; sid < ns; sid++) {
        if (P.segs[sid].len == 0) continue;
        if (e >= P.qcap) {
            C->error = (unsigned int)ST_CAPACITY;
            C->pending = 0;
            return;
        }
        if (P.segs[sid].train_slot != INVALID) {  // the sample runs beside the statistics
            if (e + 1 >= P.qcap) {
                C->error = (unsigned int)ST_CAPACITY;
                C->pending = 0;
                return;
            }
            q_write(P, e++, T_LSAMPLE, sid, SAMPLE_RUNS);
        }
        q_write(P, e++, T_LSTATS, sid, P.segs[sid].chunks);
    }
    C->t_first = ~0ull;
    if (P.test_stall) {  // test of the bounded waits: nothing published, one entry pending
        C->q_alloc[0] = C->q_alloc[1] = 0;
        C->pending = 1;
        C->item_alloc = (uint32_t)(2 * nseg);
        return;
    }
    const uint32_t eleaf = P.qcap;  // first entry of the leaf queue
    if (nl) q_write(P, eleaf, T_FINISH, 0, nl);
    C->q_alloc[0] = e;
    C->q_alloc[1] = nl ? 1u : 0u;
    C->pending = e + (nl ? 1u : 0u);
    C->item_alloc = (uint32_t)(2 * nseg);
    for (uint32_t i = 0; i < e; i++) P.ready[i] = ep;
    if (nl) P.ready[eleaf] = ep;
}

// Order-preserving encodings to uint64 and back (in place).
__global__ void k_encode(uint64_t *keys, unsigned long long n, uint32_t type, int inverse)
{
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        uint64_t x = keys[i];
        if (type == ZSORT_KEY_I64) {
            x ^= 0x8000000000000000ull;  // two's complement order -> unsigned order
        } else if (!inverse) {       // IEEE-754 totalOrder
            x = (x >> 63) ? ~x : (x | 0x8000000000000000ull);
        } else {
            x = (x >> 63) ? (x & 0x7fffffffffffffffull) : ~x;
        }
        keys[i] = x;
    }
}

// ---------------------------------------------------------------- host side
namespace {

// A captured launch sequence and the arguments it was captured with.
struct GraphCache {
    bool valid = false;
    uint64_t *keys = nullptr;
    uint32_t *vals = nullptr;
    const uint64_t *off = nullptr;
    unsigned long long n = 0, nseg = 0;
    uint32_t *plan = nullptr;
    zsort_opts o{};
    cudaGraphExec_t exec = nullptr;
};

struct Workspace {
    GraphCache graph;
    int device = -1;
    cudaStream_t stream = nullptr;
    unsigned long long n_cap = 0, nseg_cap = 0;
    unsigned long long large_min = 0;
    unsigned long long chunks_cap = 0;
    void *block = nullptr;
    size_t bytes = 0;
    Params P{};
    uint32_t epoch = 0;
    int sms = 0;
    int occ = 0;
    TraceRec *trace = nullptr;  // task trace buffer (ZSORT_TRACE_CAP records), on first traced call
    void *aux = nullptr;        // scratch of the 128-bit path, grown on demand
    size_t aux_bytes = 0;
};

// Names the host-side span of a public call in profiler timelines (NVTX).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

std::mutex g_mu;
std::vector<Workspace *> g_ws;
bool g_attr_set[64] = {false};
const size_t SMEM_BYTES = sizeof(SmemTile);

constexpr unsigned long long div_up(unsigned long long a, unsigned long long b) { return (a + b - 1) / b; }

constexpr size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

constexpr unsigned long long min_u64(unsigned long long a, unsigned long long b) { return a < b ? a : b; }

// Capacity plan for calls of up to n elements and nseg segments on a device
// of `sms` SMs (at most two persistent CTAs each).  The one source of the
// workspace capacities: the cached workspaces and the static scratch of
// zsort_pairs_noalloc are both laid out by it.
struct Plan {
    unsigned long long qcap, segcap, itemcap, statuscap, traincap;
    size_t off_skeys, off_svals, off_ids, off_ctl, off_epoch, off_entries, off_ready, off_tnext, off_tdone, off_segs,
        off_items, off_bstart, off_status, off_pwl, off_train, total;
};

constexpr Plan make_plan(unsigned long long n, unsigned long long nseg, unsigned long long large_min, int sms,
                         unsigned long long chunks_per_cta, unsigned long long traincap_max = 32)
{
    Plan p{};
    p.qcap = n / 128 + 4 * nseg + 4096;
    p.segcap = 3 * (n / (large_min + 1)) + 64;
    p.itemcap = 2 * nseg + n / 32 + 4096;
    // look-back rows: 2 x chunks x k words per large (sub)array; the chunks of
    // one level add up to ~chunks_per_cta per CTA plus at most 2 per
    // (sub)array; room for two such levels
    const unsigned long long nctas = 2ull * (unsigned long long)(sms > 0 ? sms : 160);
    p.statuscap = 2ull * NB_MAX *
                  (min_u64(2 * chunks_per_cta * nctas, n / TILE_MIN + 64) + min_u64(2 * p.segcap, 16384));
    p.traincap = min_u64(p.segcap, traincap_max);
    size_t o = 0;
    auto take = [&o](size_t bytes) {
        const size_t r = o;
        o = align_up(o + bytes);
        return r;
    };
    p.off_skeys = take(n * 8);
    p.off_svals = take(n * 4);
    p.off_ids = take(n * 2);
    p.off_ctl = take(sizeof(Ctl));
    p.off_epoch = take(16);
    p.off_entries = take(QUEUES * p.qcap * sizeof(Entry));
    p.off_ready = take(QUEUES * p.qcap * 4);
    p.off_tnext = take(QUEUES * p.qcap * 4);
    p.off_tdone = take(QUEUES * p.qcap * 4);
    p.off_segs = take(p.segcap * sizeof(Seg));
    p.off_items = take(p.itemcap * sizeof(Item));
    p.off_bstart = take(p.segcap * NB_MAX * 4);
    p.off_status = take(p.statuscap * 4);
    p.off_pwl = take(p.segcap * PWL_STRIDE * 4);
    p.off_train = take(p.traincap * 2 * SAMPLE_MAX * 8);
    p.total = o;
    return p;
}

// Points a launch's bookkeeping pointers into a block laid out by make_plan.
void bind_plan(Params &P, char *b, const Plan &p)
{
    P.skeys = reinterpret_cast<uint64_t *>(b + p.off_skeys);
    P.svals = reinterpret_cast<uint32_t *>(b + p.off_svals);
    P.ids = reinterpret_cast<uint16_t *>(b + p.off_ids);
    P.ctl = reinterpret_cast<Ctl *>(b + p.off_ctl);
    P.epoch_ctr = reinterpret_cast<uint32_t *>(b + p.off_epoch);
    P.entries = reinterpret_cast<Entry *>(b + p.off_entries);
    P.ready = reinterpret_cast<uint32_t *>(b + p.off_ready);
    P.tnext = reinterpret_cast<uint32_t *>(b + p.off_tnext);
    P.tdone = reinterpret_cast<uint32_t *>(b + p.off_tdone);
    P.qcap = (uint32_t)p.qcap;
    P.segs = reinterpret_cast<Seg *>(b + p.off_segs);
    P.segcap = (uint32_t)p.segcap;
    P.items = reinterpret_cast<Item *>(b + p.off_items);
    P.itemcap = (uint32_t)p.itemcap;
    P.bstart = reinterpret_cast<uint32_t *>(b + p.off_bstart);
    P.status = reinterpret_cast<uint32_t *>(b + p.off_status);
    P.statuscap = p.statuscap;
    P.pwl = reinterpret_cast<float *>(b + p.off_pwl);
    P.trainbuf = reinterpret_cast<unsigned long long *>(b + p.off_train);
    P.traincap = (uint32_t)p.traincap;
}

int cuda_err(cudaError_t e)
{
    if (e == cudaSuccess) return ZSORT_OK;
    if (e == cudaErrorMemoryAllocation) return ZSORT_ERR_NOMEM;
    return ZSORT_ERR_CUDA;
}

// Finds or (re)allocates the workspace of (current device, stream).
int get_workspace(cudaStream_t stream, unsigned long long n, unsigned long long nseg,
                  unsigned long long large_min, unsigned long long chunks_per_cta, Workspace **out)
{
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_err(ce);
    Workspace *ws = nullptr;
    for (Workspace *w : g_ws)
        if (w->device == dev && w->stream == stream) ws = w;
    if (!ws) {
        ws = new Workspace();
        ws->device = dev;
        ws->stream = stream;
        g_ws.push_back(ws);
    }
    if (!ws->block || ws->n_cap < n || ws->nseg_cap < nseg || ws->large_min != large_min ||
        ws->chunks_cap < chunks_per_cta) {
        unsigned long long ncap = std::max<unsigned long long>(n, ws->n_cap);
        unsigned long long scap = std::max<unsigned long long>(nseg, ws->nseg_cap);
        ncap = std::max<unsigned long long>(ncap, 1);
        scap = std::max<unsigned long long>(scap, 1);
        int sms = 0;
        ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (ce != cudaSuccess) return cuda_err(ce);
        const unsigned long long ccap = std::max<unsigned long long>(chunks_per_cta, ws->chunks_cap);
        Plan p = make_plan(ncap, scap, large_min, sms, ccap);
        if (ws->block) {
            ce = cudaStreamSynchronize(stream);  // the old block may still be in use
            if (ce != cudaSuccess) return cuda_err(ce);
            cudaFree(ws->block);
            ws->block = nullptr;
        }
        if (ws->graph.valid) {  // captured with the old block's addresses
            cudaGraphExecDestroy(ws->graph.exec);
            ws->graph = GraphCache{};
        }
        void *blk = nullptr;
        ce = cudaMalloc(&blk, p.total);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            return ZSORT_ERR_NOMEM;
        }
        // zero ready flags (epoch 0 is never used) on the call's own stream:
        // a plain cudaMemset runs on the legacy default stream, which a
        // non-blocking stream does not wait for, so it could still be
        // clearing the block while this call's kernels publish their work
        ce = cudaMemsetAsync(blk, 0, p.total, stream);
        if (ce != cudaSuccess) return cuda_err(ce);
        ws->block = blk;
        ws->bytes = p.total;
        ws->n_cap = ncap;
        ws->nseg_cap = scap;
        ws->large_min = large_min;
        ws->chunks_cap = ccap;
        Params &P = ws->P;
        P = Params{};
        bind_plan(P, static_cast<char *>(blk), p);
        ws->epoch = 0;
    }
    if (!ws->sms) {
        ce = cudaDeviceGetAttribute(&ws->sms, cudaDevAttrMultiProcessorCount, dev);
        if (ce != cudaSuccess) return cuda_err(ce);
        if (dev < 64 && !g_attr_set[dev]) {
            ce = cudaFuncSetAttribute(k_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)SMEM_BYTES);
            if (ce != cudaSuccess) return cuda_err(ce);
            g_attr_set[dev] = true;
        }
        ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ws->occ, k_persistent, BLOCK, SMEM_BYTES);
        if (ce != cudaSuccess) return cuda_err(ce);
        if (ws->occ < 1) return ZSORT_ERR_CUDA;
    }
    *out = ws;
    return ZSORT_OK;
}

bool opts_valid(const zsort_opts &o)
{
    if (o.struct_size != sizeof(zsort_opts)) return false;
    if (o.mapper > ZSORT_MAP_MLP) return false;
    if (o.kmax < MIN_K || o.kmax > NB_MAX || (o.kmax & (o.kmax - 1))) return false;
    if (o.leaf_target < 16 || o.leaf_target > (1u << 24)) return false;
    if (o.large_min < (uint32_t)LEAF_CAP || o.large_min >= (1u << 30)) return false;
    if (o.sample < (uint32_t)PWL_P || o.sample > (uint32_t)SAMPLE_MAX) return false;
    if (o.learn_min < o.sample) return false;
    if (!(o.fallback_ratio > 0.0f)) return false;
    if (o.guard_level < 1) return false;
    if (o.leaf_cap < (uint32_t)RANK_SMALL || o.leaf_cap > (uint32_t)LEAF_CAP) return false;
    if (o.chunks_per_cta < 1 || o.chunks_per_cta > 64) return false;
    if (o.ipt != (uint32_t)IPT && o.ipt != (uint32_t)IPT_SMALL) return false;
    return true;
}

// Host-side fault injection for failure-path tests: the environment variable
// ZSORT_FAULT, read at every call.  "alloc": the workspace allocation fails
// (ZSORT_ERR_NOMEM, nothing enqueued); "timeout": the call publishes no work
// and every device wait runs out after 50 ms (ZSORT_ERR_TIMEOUT from
// zsort_sync_status, as ZSORT_FLAG_TEST_STALL); "badoffsets": the segment
// check reports malformed offsets (ZSORT_ERR_BAD_OFFSETS).  No GPU fault is
// involved in any of them; keys and payloads are left untouched.
enum Fault { FAULT_NONE, FAULT_ALLOC, FAULT_TIMEOUT, FAULT_BADOFF };
Fault injected_fault()
{
    const char *f = std::getenv("ZSORT_FAULT");
    if (!f) return FAULT_NONE;
    if (std::strcmp(f, "alloc") == 0) return FAULT_ALLOC;
    if (std::strcmp(f, "timeout") == 0) return FAULT_TIMEOUT;
    if (std::strcmp(f, "badoffsets") == 0) return FAULT_BADOFF;
    return FAULT_NONE;
}

// Enqueues one sort (single array when off == nullptr).
int launch(uint64_t *keys, uint32_t *vals, unsigned long long n, const uint64_t *off,
           unsigned long long nseg, const zsort_opts &o_in, cudaStream_t stream, uint32_t *plan_out = nullptr)
{
    const Fault fault = injected_fault();
    if (fault == FAULT_ALLOC) return ZSORT_ERR_NOMEM;
    zsort_opts o = o_in;
    if (fault == FAULT_TIMEOUT) {
        o.flags = (o.flags | ZSORT_FLAG_TEST_STALL) & ~ZSORT_FLAG_GRAPH;
        o.wait_limit_ms = 50;
    }
    if (fault == FAULT_BADOFF) o.flags &= ~ZSORT_FLAG_GRAPH;
    std::lock_guard<std::mutex> lock(g_mu);
    Workspace *ws = nullptr;
    int rc = get_workspace(stream, n, nseg, o.large_min, o.chunks_per_cta, &ws);
    if (rc != ZSORT_OK) return rc;
    Params P = ws->P;
    P.ukeys = keys;
    P.uvals = vals;
    P.n = n;

    P.kmax = o.kmax;
    P.leaf_target = o.leaf_target;
    P.large_min = o.large_min;
    P.learn_min = o.learn_min;
    P.sample = o.sample;
    P.mapper = o.mapper;
    P.guard_level = o.guard_level;
    P.leaf_cap = o.leaf_cap;
    P.chunks_per_cta = o.chunks_per_cta;
    P.ipt = o.ipt;
    P.tile = (uint32_t)BLOCK * o.ipt;
    P.sub_sample = (o.flags & ZSORT_FLAG_EXACT_SUBSTATS) ? 0u : 1u;
    P.fallback_ratio = o.fallback_ratio;
    P.seed = o.seed;
    P.wait_ns = (unsigned long long)o.wait_limit_ms * 1000000ull;
    P.user_aligned = ((reinterpret_cast<uintptr_t>(keys) | reinterpret_cast<uintptr_t>(vals)) & 15u) == 0;
    P.kv = vals != nullptr;  // null vals: keys only
    P.test_stall = (o.flags & ZSORT_FLAG_TEST_STALL) ? 1u : 0u;
    P.test_badoff = fault == FAULT_BADOFF ? 1u : 0u;
    if (o.flags & ZSORT_FLAG_TRACE) {
        if (!ws->trace) {
            void *t = nullptr;
            if (cudaMalloc(&t, (size_t)ZSORT_TRACE_CAP * sizeof(TraceRec)) != cudaSuccess) {
                cudaGetLastError();
                return ZSORT_ERR_NOMEM;
            }
            ws->trace = static_cast<TraceRec *>(t);
        }
        P.trace = ws->trace;
        P.trace_cap = ZSORT_TRACE_CAP;
    }
    int per_sm = o.ctas_per_sm ? (int)std::min<uint32_t>(o.ctas_per_sm, (uint32_t)ws->occ) : ws->occ;
    P.nctas = (uint32_t)(ws->sms * per_sm);
    P.plan_out = plan_out;
    auto enqueue = [&]() -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(P.ctl, 0, sizeof(Ctl), stream);
        if (e != cudaSuccess) return e;
        const unsigned int gi = (unsigned int)div_up(nseg, 256);
        k_init_segments<<<gi, 256, 0, stream>>>(P, off, nseg);
        k_init_publish<<<1, 32, 0, stream>>>(P, nseg);
        k_persistent<<<P.nctas, BLOCK, SMEM_BYTES, stream>>>(P);
        return cudaGetLastError();
    };
    if (!(o.flags & ZSORT_FLAG_GRAPH) || stream == nullptr) return cuda_err(enqueue());
    GraphCache &g = ws->graph;
    const bool hit = g.valid && g.keys == keys && g.vals == vals && g.off == off && g.n == n && g.nseg == nseg &&
                     g.plan == plan_out && std::memcmp(&g.o, &o, sizeof(o)) == 0;
    if (!hit) {
        if (g.valid) cudaGraphExecDestroy(g.exec);
        g = GraphCache{};
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
        if (ce != cudaSuccess) return cuda_err(ce);
        cudaError_t le = enqueue();
        ce = cudaStreamEndCapture(stream, &graph);
        if (le != cudaSuccess || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_err(le != cudaSuccess ? le : ce);
        }
        cudaGraphExec_t exec = nullptr;
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return cuda_err(ce);
        g.valid = true;
        g.keys = keys;
        g.vals = vals;
        g.off = off;
        g.n = n;
        g.nseg = nseg;
        g.plan = plan_out;
        g.o = o;
        g.exec = exec;
    }
    return cuda_err(cudaGraphLaunch(g.exec, stream));
}

int encode(void *keys, unsigned long long n, uint32_t type, int inverse, cudaStream_t stream)
{
    if (type == ZSORT_KEY_U64 || n == 0) return ZSORT_OK;
    unsigned int grid = (unsigned int)std::min<unsigned long long>(div_up(n, 256), 4096);
    k_encode<<<grid, 256, 0, stream>>>(static_cast<uint64_t *>(keys), n, type, inverse);
    return cuda_err(cudaGetLastError());
}

// 128-bit keys, sorted by one zSort of a 64-bit window of each key (see
// zsort_pairs_u128).  A key is the word pair (lo, hi); d = key - min is taken
// exactly in 128 bits; the window is d >> s and the remainder the s bits
// below it, s = max(0, bitlen(max - min) - 64), so that (window, remainder)
// orders like the key and every window fits 64 bits.
struct U128Win {
    unsigned long long mn_lo, mn_hi;
    uint32_t s, pad;
    unsigned long long tied, groups;  // keys in runs of equal windows, runs
};

__device__ __forceinline__ bool lt128(unsigned long long alo, unsigned long long ahi, unsigned long long blo,
                                      unsigned long long bhi)
{
    return ahi < bhi || (ahi == bhi && alo < blo);
}

// Warp-wide 128-bit min and max (every lane gets them).
__device__ __forceinline__ void k128_warp_minmax(unsigned long long &mnl, unsigned long long &mnh,
                                                 unsigned long long &mxl, unsigned long long &mxh)
{
    for (int o = 16; o; o >>= 1) {
        const unsigned long long al = __shfl_xor_sync(0xffffffffu, mnl, o), ah = __shfl_xor_sync(0xffffffffu, mnh, o);
        const unsigned long long bl = __shfl_xor_sync(0xffffffffu, mxl, o), bh = __shfl_xor_sync(0xffffffffu, mxh, o);
        if (lt128(al, ah, mnl, mnh)) mnl = al, mnh = ah;
        if (lt128(mxl, mxh, bl, bh)) mxl = bl, mxh = bh;
    }
}

// Per block: the 128-bit min and max of its keys, as (lo, hi, lo, hi) in part[4b..].
__global__ void k128_minmax(const uint64_t *keys, unsigned long long n, unsigned long long *part)
{
    __shared__ unsigned long long sm[4][BLOCK / 32];
    unsigned long long mnl = ~0ull, mnh = ~0ull, mxl = 0, mxh = 0;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long lo = keys[2 * i], hi = keys[2 * i + 1];
        if (lt128(lo, hi, mnl, mnh)) mnl = lo, mnh = hi;
        if (lt128(mxl, mxh, lo, hi)) mxl = lo, mxh = hi;
    }
    k128_warp_minmax(mnl, mnh, mxl, mxh);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sm[0][warp] = mnl, sm[1][warp] = mnh, sm[2][warp] = mxl, sm[3][warp] = mxh;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < BLOCK / 32; w++) {
            if (lt128(sm[0][w], sm[1][w], mnl, mnh)) mnl = sm[0][w], mnh = sm[1][w];
            if (lt128(mxl, mxh, sm[2][w], sm[3][w])) mxl = sm[2][w], mxh = sm[3][w];
        }
        unsigned long long *p = part + 4ull * blockIdx.x;
        p[0] = mnl, p[1] = mnh, p[2] = mxl, p[3] = mxh;
    }
}

// One block of 1024 threads: the min and max over the blocks' parts, and the
// window shift.
__global__ void k128_window_shift(const unsigned long long *part, uint32_t nparts, U128Win *W)
{
    __shared__ unsigned long long sm[4][32];
    unsigned long long mnl = ~0ull, mnh = ~0ull, mxl = 0, mxh = 0;
    for (uint32_t b = threadIdx.x; b < nparts; b += blockDim.x) {
        const unsigned long long *p = part + 4ull * b;
        if (lt128(p[0], p[1], mnl, mnh)) mnl = p[0], mnh = p[1];
        if (lt128(mxl, mxh, p[2], p[3])) mxl = p[2], mxh = p[3];
    }
    k128_warp_minmax(mnl, mnh, mxl, mxh);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sm[0][warp] = mnl, sm[1][warp] = mnh, sm[2][warp] = mxl, sm[3][warp] = mxh;
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
        if (lt128(sm[0][w], sm[1][w], mnl, mnh)) mnl = sm[0][w], mnh = sm[1][w];
        if (lt128(mxl, mxh, sm[2][w], sm[3][w])) mxl = sm[2][w], mxh = sm[3][w];
    }
    const unsigned long long dl = mxl - mnl, dh = mxh - mnh - (mxl < mnl ? 1ull : 0ull);
    const uint32_t bits = dh ? 128u - (uint32_t)__clzll((long long)dh) : 64u - (uint32_t)__clzll((long long)dl);
    W->mn_lo = mnl;
    W->mn_hi = mnh;
    W->s = bits > 64u ? bits - 64u : 0u;
    W->tied = 0;
    W->groups = 0;
}

// d = key - min in 128 bits; the window d >> s and the remainder below it.
__device__ __forceinline__ void k128_split_key(unsigned long long lo, unsigned long long hi, const U128Win &W,
                                               unsigned long long *win, unsigned long long *rem)
{
    const unsigned long long dl = lo - W.mn_lo, dh = hi - W.mn_hi - (lo < W.mn_lo ? 1ull : 0ull);
    const uint32_t s = W.s;
    if (s == 0) {
        *win = dl;  // dh == 0: the range fits 64 bits
        *rem = 0;
    } else if (s == 64) {
        *win = dh;
        *rem = dl;
    } else {
        *win = (dl >> s) | (dh << (64u - s));
        *rem = dl & ((1ull << s) - 1ull);
    }
}

// The window of every key with its input index, and a copy of the keys and
// payloads as records (the final gather's source): (lo, hi) with no
// payloads, (lo, hi, payload, 0) with them, so that one record is one
// 16- or 32-byte aligned piece and the gather reads one sector a key.
__global__ void k128_window(const uint64_t *keys, const uint32_t *vals, unsigned long long n, const U128Win *Wp,
                            uint64_t *win, uint32_t *idx, uint64_t *rec)
{
    const U128Win W = *Wp;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long lo = keys[2 * i], hi = keys[2 * i + 1];
        unsigned long long w, r;
        k128_split_key(lo, hi, W, &w, &r);
        win[i] = w;
        idx[i] = (uint32_t)i;
        if (vals) {
            ulonglong2 *p = reinterpret_cast<ulonglong2 *>(rec + 4 * i);
            p[0] = make_ulonglong2(lo, hi);
            p[1] = make_ulonglong2((unsigned long long)vals[i], 0ull);
        } else {
            reinterpret_cast<ulonglong2 *>(rec)[i] = make_ulonglong2(lo, hi);
        }
    }
}

// Runs of equal windows in the sorted windows: element i of a run of two or
// more counts as tied (low 32 bits) and, if it starts the run, as a run head
// (high 32 bits).  TIE_PER consecutive elements per thread.
constexpr int TIE_PER = 16;
constexpr unsigned long long U128_RUNS_PER_LAUNCH = 1ull << 20;
constexpr unsigned long long TIE_TILE = (unsigned long long)BLOCK * TIE_PER;
__device__ __forceinline__ unsigned long long k128_tie_bits(const uint64_t *win, unsigned long long n,
                                                            unsigned long long i)
{
    const unsigned long long w = win[i];
    const bool eqp = i > 0 && win[i - 1] == w, eqn = i + 1 < n && win[i + 1] == w;
    const bool tied = eqp || eqn;
    return (tied ? 1ull : 0ull) | (tied && !eqp ? 1ull << 32 : 0ull);
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ unsigned long long k128_block_scan(unsigned long long v, unsigned long long *excl,
                                                             unsigned long long *wsum)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    unsigned long long before = 0, total = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
        before += w < warp ? wsum[w] : 0ull;
        total += wsum[w];
    }
    __syncthreads();
    *excl = before + x - v;
    return total;
}

// The block's count (the same TIE_TILE elements as k128_tie_emit's block,
// read here in coalesced rows: the count needs no order).
__global__ void k128_tie_count(const uint64_t *win, unsigned long long n, const U128Win *Wp, unsigned long long *bsum)
{
    __shared__ unsigned long long wsum[BLOCK / 32];
    unsigned long long c = 0;
    if (Wp->s != 0) {  // s == 0: equal windows are equal keys, already in input order
        const unsigned long long i0 = blockIdx.x * TIE_TILE + threadIdx.x;
#pragma unroll 4
        for (int u = 0; u < TIE_PER; u++) {
            const unsigned long long i = i0 + (unsigned long long)u * BLOCK;
            if (i < n) c += k128_tie_bits(win, n, i);
        }
    }
    unsigned long long excl;
    const unsigned long long t = k128_block_scan(c, &excl, wsum);
    if (threadIdx.x == 0) bsum[blockIdx.x] = t;
}

// One block: exclusive scan of the block counts; the totals into W.
__global__ void k128_tie_scan(unsigned long long *bsum, unsigned long long nb, U128Win *W)
{
    __shared__ unsigned long long wsum[32];
    const unsigned long long per = (nb + blockDim.x - 1) / blockDim.x, b0 = threadIdx.x * per;
    unsigned long long sum = 0;
    for (unsigned long long b = b0; b < b0 + per && b < nb; b++) sum += bsum[b];
    unsigned long long excl;
    const unsigned long long total = k128_block_scan(sum, &excl, wsum);
    for (unsigned long long b = b0; b < b0 + per && b < nb; b++) {
        const unsigned long long v = bsum[b];
        bsum[b] = excl;
        excl += v;
    }
    if (threadIdx.x == 0) {
        W->tied = total & 0xffffffffull;
        W->groups = total >> 32;
    }
}

// The tied keys, compacted in sorted order: remainder, sorted position (the
// segmented sort's payload, and a second copy that it leaves in place), and
// each run's start as a segment offset.
__global__ void k128_tie_emit(const uint64_t *win, const uint32_t *idx, const uint64_t *rec, uint32_t rs,
                              unsigned long long n, const unsigned long long *bofs, const U128Win *Wp, uint64_t *ck,
                              uint32_t *cv, uint32_t *pre, uint64_t *off)
{
    __shared__ unsigned long long wsum[BLOCK / 32];
    const U128Win W = *Wp;
    const unsigned long long i0 = blockIdx.x * TIE_TILE + (unsigned long long)threadIdx.x * TIE_PER;
    unsigned long long bits[TIE_PER], c = 0;
#pragma unroll
    for (int u = 0; u < TIE_PER; u++) {
        bits[u] = i0 + u < n ? k128_tie_bits(win, n, i0 + u) : 0ull;
        c += bits[u];
    }
    unsigned long long pos;
    k128_block_scan(c, &pos, wsum);
    pos += bofs[blockIdx.x];
#pragma unroll
    for (int u = 0; u < TIE_PER; u++) {
        if (bits[u] & 1ull) {
            const unsigned long long i = i0 + u, src = idx[i];
            const uint32_t j = (uint32_t)(pos & 0xffffffffull);
            unsigned long long w, r;
            k128_split_key(rec[rs * src], rec[rs * src + 1], W, &w, &r);
            ck[j] = r;
            cv[j] = (uint32_t)i;
            pre[j] = (uint32_t)i;
            if (bits[u] >> 32) off[pos >> 32] = j;
        }
        pos += bits[u];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) off[W.groups] = W.tied;
}

// After the runs are sorted by remainder: the index of each tied position,
// through a copy (gather, then scatter) so that no thread reads an entry
// another one rewrites.
__global__ void k128_tie_gather(const uint32_t *cv, const uint32_t *idx, unsigned long long t, uint32_t *tmp)
{
    for (unsigned long long j = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; j < t;
         j += (unsigned long long)gridDim.x * blockDim.x)
        tmp[j] = idx[cv[j]];
}
__global__ void k128_tie_place(const uint32_t *pre, const uint32_t *tmp, unsigned long long t, uint32_t *idx)
{
    for (unsigned long long j = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; j < t;
         j += (unsigned long long)gridDim.x * blockDim.x)
        idx[pre[j]] = tmp[j];
}

// The keys and payloads in sorted order, into the caller's arrays.
__global__ void k128_gather(const uint64_t *rec, const uint32_t *idx, unsigned long long n, uint64_t *keys,
                            uint32_t *vals)
{
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long src = idx[i];
        if (vals) {
            const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(rec + 4 * src);
            const ulonglong2 kv = p[0], pv = p[1];
            keys[2 * i] = kv.x;
            keys[2 * i + 1] = kv.y;
            vals[i] = (uint32_t)pv.x;
        } else {
            const ulonglong2 kv = reinterpret_cast<const ulonglong2 *>(rec)[src];
            keys[2 * i] = kv.x;
            keys[2 * i + 1] = kv.y;
        }
    }
}

// The stream's 128-bit scratch, at least bytes long (kept between calls: the
// call after the first one allocates nothing).  Growing it waits for the
// stream, whose earlier calls may still use the old area.  Takes g_mu.
int aux_scratch(cudaStream_t stream, size_t bytes, unsigned char **out)
{
    std::lock_guard<std::mutex> lock(g_mu);
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_err(ce);
    Workspace *ws = nullptr;
    for (Workspace *w : g_ws)
        if (w->device == dev && w->stream == stream) ws = w;
    if (!ws) {
        ws = new Workspace();
        ws->device = dev;
        ws->stream = stream;
        g_ws.push_back(ws);
    }
    if (ws->aux_bytes < bytes) {
        if (ws->aux) {
            ce = cudaStreamSynchronize(stream);
            if (ce != cudaSuccess) return cuda_err(ce);
            cudaFree(ws->aux);
            ws->aux = nullptr;
            ws->aux_bytes = 0;
        }
        ce = cudaMalloc(&ws->aux, bytes);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            ws->aux = nullptr;
            return ZSORT_ERR_NOMEM;
        }
        ws->aux_bytes = bytes;
    }
    *out = static_cast<unsigned char *>(ws->aux);
    return ZSORT_OK;
}

Workspace *find_ws(cudaStream_t stream)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    for (Workspace *w : g_ws)
        if (w->device == dev && w->stream == stream) return w;
    return nullptr;
}

}  // namespace

// ---------------------------------------------------------------- no-alloc entry
// Some callers cannot call cudaMalloc at all: real-time or embedded hosts
// that forbid device allocation once they have started, and processes whose
// device memory is owned by a fixed pool they may not grow.
// zsort_pairs_noalloc serves them: its scratch is one file-scope __device__
// array, sized for NA_MAX_N elements and held by every GPU that loads this
// library until the process exits.
namespace {

constexpr unsigned long long NA_MAX_N = ZSORT_NOALLOC_MAX_N;
constexpr unsigned long long NA_LARGE_MIN = 65536;  // the default large_min
constexpr unsigned long long NA_CHUNKS = 8;         // the default chunks_per_cta
constexpr int NA_MAX_SMS = 192;                     // launches use at most 2 x this many CTAs

// Layout of the static scratch: make_plan's regions for NA_MAX_N elements and
// one segment, with one learned-map training slot.
constexpr Plan NA = make_plan(NA_MAX_N, 1, NA_LARGE_MIN, NA_MAX_SMS, NA_CHUNKS, 1);

// Per-device set-up of the no-alloc path (the symbol's device address).
struct NaDevice {
    bool ready = false;
    char *base = nullptr;
    int sms = 0, occ = 0;
    uint32_t epoch = 0;
};
std::mutex g_na_mu;
NaDevice g_na_dev[64];

}  // namespace

// The scratch itself: zero at module load, reused (not cleared) by every call.
static __device__ __align__(256) unsigned char g_na_scratch[NA.total];
static_assert(NA.total < (32ull << 20), "the no-alloc scratch stays modest");

// Copies a call's device status word to the caller's int.
__global__ void k_na_status(const Ctl *ctl, int32_t *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *out = (int32_t)ctl->error;
}

// ---------------------------------------------------------------- C ABI
extern "C" {

void zsort_default_opts(zsort_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->struct_size = sizeof(zsort_opts);
    o->mapper = ZSORT_MAP_ZSCORE;
    o->kmax = 512;
    o->leaf_target = 2048;
    o->large_min = 65536;
    o->learn_min = 1u << 20;
    o->sample = 65536;
    o->fallback_ratio = 4.0f;
    o->seed = 0x5eed2605ull;
    o->guard_level = 8;
    o->ctas_per_sm = 0;
    o->wait_limit_ms = 2000;
    o->leaf_cap = LEAF_CAP;
    o->chunks_per_cta = 8;
    o->ipt = IPT;
}

int zsort_pairs_ex(void *keys, uint32_t key_type, uint32_t *vals, uint64_t n, const zsort_opts *opts,
                   zsort_stream_t stream)
{
    NvtxRange nv("zsort_pairs_ex");
    zsort_opts o;
    if (opts)
        o = *opts;
    else
        zsort_default_opts(&o);
    if (!opts_valid(o)) return ZSORT_ERR_INVALID;
    if (key_type > ZSORT_KEY_F64 || n > ZSORT_MAX_N) return ZSORT_ERR_INVALID;
    if (n <= 1) return ZSORT_OK;
    if (!keys) return ZSORT_ERR_INVALID;  // vals may be null: keys only
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int rc = encode(keys, n, key_type, 0, st);
    if (rc != ZSORT_OK) return rc;
    rc = launch(static_cast<uint64_t *>(keys), vals, n, nullptr, 1, o, st);
    if (rc != ZSORT_OK) return rc;
    return encode(keys, n, key_type, 1, st);
}

int zsort_pairs_u128(uint64_t *keys, uint32_t *vals, uint64_t n, const zsort_opts *opts, zsort_stream_t stream)
{
    NvtxRange nv("zsort_pairs_u128");
    zsort_opts o;
    if (opts)
        o = *opts;
    else
        zsort_default_opts(&o);
    if (!opts_valid(o) || n > ZSORT_MAX_N) return ZSORT_ERR_INVALID;
    if (n <= 1) return ZSORT_OK;
    if (!keys) return ZSORT_ERR_INVALID;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    auto a16 = [](size_t x) { return (x + 15) & ~size_t(15); };  // bulk copies want 16-byte bases
    const unsigned int grid = (unsigned int)std::min<unsigned long long>(div_up(n, 256), 4096);
    const unsigned int nparts = (unsigned int)std::min<unsigned long long>(div_up(n, 256), 1024);
    const unsigned long long nb = div_up(n, TIE_TILE);
    // scratch: records of keys (and payloads), windows, indices, block counts
    const uint32_t rs = vals ? 4u : 2u;  // 64-bit words a record
    const size_t o_win = a16(n * rs * 8), o_idx = a16(o_win + n * 8);
    const size_t o_part = a16(o_idx + n * 4), o_bs = a16(o_part + (size_t)nparts * 32);
    const size_t o_w = a16(o_bs + nb * 8), bytes = o_w + sizeof(U128Win);
    unsigned char *t = nullptr;
    int rc = aux_scratch(st, bytes, &t);
    if (rc != ZSORT_OK) return rc;
    cudaError_t ce = cudaSuccess;
    uint64_t *rec = reinterpret_cast<uint64_t *>(t);  // 256-byte aligned: a record never spans a sector
    uint64_t *win = reinterpret_cast<uint64_t *>(t + o_win);
    uint32_t *idx = reinterpret_cast<uint32_t *>(t + o_idx);
    unsigned long long *part = reinterpret_cast<unsigned long long *>(t + o_part);
    unsigned long long *bsum = reinterpret_cast<unsigned long long *>(t + o_bs);
    U128Win *W = reinterpret_cast<U128Win *>(t + o_w);
    // 1. min, max and the window shift; every key's window; one stable zSort
    //    of (window, input index)
    k128_minmax<<<nparts, BLOCK, 0, st>>>(keys, n, part);
    k128_window_shift<<<1, 1024, 0, st>>>(part, nparts, W);
    k128_window<<<grid, 256, 0, st>>>(keys, vals, n, W, win, idx, rec);
    rc = cuda_err(cudaGetLastError());
    if (rc == ZSORT_OK) rc = launch(win, idx, n, nullptr, 1, o, st);
    // 2. runs of equal windows (none for keys whose top 64 significant bits
    //    differ): counted on the device, the counts read back once
    U128Win hw{};
    if (rc == ZSORT_OK) {
        k128_tie_count<<<(unsigned int)nb, BLOCK, 0, st>>>(win, n, W, bsum);
        k128_tie_scan<<<1, 1024, 0, st>>>(bsum, nb, W);
        rc = cuda_err(cudaGetLastError());
    }
    if (rc == ZSORT_OK) rc = cuda_err(cudaMemcpyAsync(&hw, W, sizeof(hw), cudaMemcpyDeviceToHost, st));
    if (rc == ZSORT_OK) rc = cuda_err(cudaStreamSynchronize(st));
    // 3. the tied keys, compacted, each run sorted by the remainder below the
    //    window (one segmented zSort), their indices put back in that order
    if (rc == ZSORT_OK && hw.tied) {
        const unsigned long long T = hw.tied, G = hw.groups;
        const size_t c_cv = a16(T * 8), c_pre = a16(c_cv + T * 4), c_tmp = a16(c_pre + T * 4);
        const size_t c_off = a16(c_tmp + T * 4), cbytes = c_off + (G + 1) * 8;
        unsigned char *c = nullptr;
        ce = cudaMallocAsync(reinterpret_cast<void **>(&c), cbytes, st);
        if (ce != cudaSuccess) {
            rc = cuda_err(ce);
        } else {
            uint64_t *ck = reinterpret_cast<uint64_t *>(c);
            uint32_t *cv = reinterpret_cast<uint32_t *>(c + c_cv);
            uint32_t *pre = reinterpret_cast<uint32_t *>(c + c_pre);
            uint32_t *tmp = reinterpret_cast<uint32_t *>(c + c_tmp);
            uint64_t *off = reinterpret_cast<uint64_t *>(c + c_off);
            const unsigned int tg = (unsigned int)std::min<unsigned long long>(div_up(T, 256), 4096);
            k128_tie_emit<<<(unsigned int)nb, BLOCK, 0, st>>>(win, idx, rec, rs, n, bsum, W, ck, cv, pre, off);
            rc = cuda_err(cudaGetLastError());
            // at most U128_RUNS_PER_LAUNCH runs a launch, so that the
            // workspace's per-segment bookkeeping stays bounded however the
            // keys tie (the runs of one launch are a contiguous slice)
            for (unsigned long long g0 = 0; rc == ZSORT_OK && g0 < G; g0 += U128_RUNS_PER_LAUNCH)
                rc = launch(ck, cv, T, off + g0, std::min<unsigned long long>(U128_RUNS_PER_LAUNCH, G - g0), o, st);
            if (rc == ZSORT_OK) {
                k128_tie_gather<<<tg, 256, 0, st>>>(cv, idx, T, tmp);
                k128_tie_place<<<tg, 256, 0, st>>>(pre, tmp, T, idx);
                rc = cuda_err(cudaGetLastError());
            }
            const int rf = cuda_err(cudaFreeAsync(c, st));
            if (rc == ZSORT_OK) rc = rf;
        }
    }
    // 4. keys and payloads in that order, into the caller's arrays
    if (rc == ZSORT_OK) {
        k128_gather<<<grid, 256, 0, st>>>(rec, idx, n, keys, vals);
        rc = cuda_err(cudaGetLastError());
    }
    return rc;
}

int zsort_keys(uint64_t *keys, uint64_t n, zsort_stream_t stream)
{
    return zsort_pairs_ex(keys, ZSORT_KEY_U64, nullptr, n, nullptr, stream);
}

int zsort_pairs(uint64_t *keys, uint32_t *vals, uint64_t n, zsort_stream_t stream)
{
    return zsort_pairs_ex(keys, ZSORT_KEY_U64, vals, n, nullptr, stream);
}

int zsort_pairs_i64(int64_t *keys, uint32_t *vals, uint64_t n, zsort_stream_t stream)
{
    return zsort_pairs_ex(keys, ZSORT_KEY_I64, vals, n, nullptr, stream);
}

int zsort_pairs_f64(double *keys, uint32_t *vals, uint64_t n, zsort_stream_t stream)
{
    return zsort_pairs_ex(keys, ZSORT_KEY_F64, vals, n, nullptr, stream);
}

int zsort_segmented_ex(uint64_t *keys, uint32_t *vals, uint64_t n, const uint64_t *seg_offsets,
                       uint64_t nseg, const zsort_opts *opts, zsort_stream_t stream)
{
    NvtxRange nv("zsort_segmented_ex");
    zsort_opts o;
    if (opts)
        o = *opts;
    else
        zsort_default_opts(&o);
    if (!opts_valid(o)) return ZSORT_ERR_INVALID;
    if (n > ZSORT_MAX_SEG_TOTAL || nseg > (1ull << 31)) return ZSORT_ERR_INVALID;
    if (nseg == 0) return ZSORT_OK;
    if (!seg_offsets || (n > 0 && !keys)) return ZSORT_ERR_INVALID;
    return launch(keys, vals, n, seg_offsets, nseg, o, reinterpret_cast<cudaStream_t>(stream));
}

int zsort_segmented(uint64_t *keys, uint32_t *vals, uint64_t n, const uint64_t *seg_offsets, uint64_t nseg,
                    zsort_stream_t stream)
{
    return zsort_segmented_ex(keys, vals, n, seg_offsets, nseg, nullptr, stream);
}

int zsort_reserve(uint64_t n, uint64_t nseg, zsort_stream_t stream)
{
    if (n > ZSORT_MAX_SEG_TOTAL) return ZSORT_ERR_INVALID;
    zsort_opts o;
    zsort_default_opts(&o);
    std::lock_guard<std::mutex> lock(g_mu);
    Workspace *ws = nullptr;
    return get_workspace(reinterpret_cast<cudaStream_t>(stream), n, std::max<uint64_t>(nseg, 1),
                         o.large_min, o.chunks_per_cta, &ws);
}

int zsort_release(void)
{
    std::lock_guard<std::mutex> lock(g_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ZSORT_ERR_CUDA;
    int rc = ZSORT_OK;
    std::vector<Workspace *> keep;
    for (Workspace *w : g_ws) {
        if (w->device != dev) {
            keep.push_back(w);
            continue;
        }
        if (w->graph.valid) cudaGraphExecDestroy(w->graph.exec);
        if (w->block && cudaFree(w->block) != cudaSuccess) rc = ZSORT_ERR_CUDA;
        if (w->trace && cudaFree(w->trace) != cudaSuccess) rc = ZSORT_ERR_CUDA;
        if (w->aux && cudaFree(w->aux) != cudaSuccess) rc = ZSORT_ERR_CUDA;
        delete w;
    }
    g_ws.swap(keep);
    return rc;
}

int zsort_sync_status(zsort_stream_t stream)
{
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return cuda_err(ce);
    std::lock_guard<std::mutex> lock(g_mu);
    Workspace *ws = find_ws(st);
    if (!ws || !ws->block) return ZSORT_OK;
    unsigned int err = 0;
    ce = cudaMemcpy(&err, &ws->P.ctl->error, sizeof(err), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return cuda_err(ce);
    if (err) {  // cleared on the workspace's stream, ahead of its next call
        ce = cudaMemsetAsync(&ws->P.ctl->error, 0, sizeof(unsigned int), st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) return cuda_err(ce);
    }
    return (int)err;
}

int zsort_last_stats(zsort_stream_t stream, zsort_stats *out)
{
    if (!out) return ZSORT_ERR_INVALID;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return cuda_err(ce);
    std::lock_guard<std::mutex> lock(g_mu);
    Workspace *ws = find_ws(st);
    std::memset(out, 0, sizeof(*out));
    if (!ws || !ws->block) return ZSORT_OK;
    Ctl c;
    ce = cudaMemcpy(&c, ws->P.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return cuda_err(ce);
    out->n = ws->P.n;
    out->partitions_large = c.n_large;
    out->partitions_small = c.n_small;
    out->leaves = c.n_leaves;
    out->leaf_fallbacks = c.n_leaf_fb;
    out->copies = c.n_copies;
    out->learned_accepted = c.n_learn_ok;
    out->learned_rejected = c.n_learn_rej;
    out->guard_levels = c.n_guard;
    out->max_level = c.max_level;
    out->bytes_algorithmic = c.bytes;
    out->tasks = c.tasks;
    out->persistent_ctas = (uint64_t)ws->sms * ws->occ;
    out->top_mean_d = c.top_mean_d;
    out->top_sd = c.top_sd;
    out->top_min = c.top_min;
    out->top_max = c.top_max;
    out->top_k = c.top_k;
    out->top_map = c.top_map;
    for (int i = 0; i < 8; i++) {
        out->task_ns[i] = c.task_ns[i];
        out->task_count[i] = c.task_cnt[i];
    }
    out->handler_ns = c.handler_ns;
    out->idle_ns = c.idle_ns;
    out->busy_window_ns = (c.t_last > c.t_first && c.t_first != ~0ull) ? c.t_last - c.t_first : 0;
    out->sampled_stats = c.n_sampled;
    return ZSORT_OK;
}

int zsort_last_trace(zsort_stream_t stream, zsort_trace_rec *out, uint64_t cap, uint64_t *count)
{
    if (!count || (cap > 0 && !out)) return ZSORT_ERR_INVALID;
    *count = 0;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return cuda_err(ce);
    std::lock_guard<std::mutex> lock(g_mu);
    Workspace *ws = find_ws(st);
    if (!ws || !ws->block) return ZSORT_OK;
    unsigned long long nrec = 0;
    ce = cudaMemcpy(&nrec, &ws->P.ctl->trace_n, sizeof(nrec), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return cuda_err(ce);
    *count = nrec;
    const unsigned long long m = std::min<unsigned long long>(std::min<unsigned long long>(nrec, cap), ZSORT_TRACE_CAP);
    if (m == 0 || !ws->trace) return ZSORT_OK;
    return cuda_err(cudaMemcpy(out, ws->trace, m * sizeof(TraceRec), cudaMemcpyDeviceToHost));
}

int zsort_map_buckets(const uint64_t *keys, uint64_t n, const zsort_opts *opts, uint32_t *buckets,
                      zsort_map_info *info, zsort_stream_t stream)
{
    NvtxRange nv("zsort_map_buckets");
    zsort_opts o;
    if (opts)
        o = *opts;
    else
        zsort_default_opts(&o);
    if (!opts_valid(o)) return ZSORT_ERR_INVALID;
    if (n < 2 || n > ZSORT_MAX_N || !keys || !buckets || !info) return ZSORT_ERR_INVALID;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // inspection mode reads the keys only (no payload) and writes buckets
    int rc = launch(const_cast<uint64_t *>(keys), nullptr, n, nullptr, 1, o, st, buckets);
    if (rc != ZSORT_OK) return rc;
    cudaError_t ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return cuda_err(ce);
    std::lock_guard<std::mutex> lock(g_mu);
    Workspace *ws = find_ws(st);
    if (!ws) return ZSORT_ERR_INTERNAL;
    unsigned int err = 0;
    ce = cudaMemcpy(&err, &ws->P.ctl->error, sizeof(err), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return cuda_err(ce);
    if (err) {  // cleared on the workspace's stream, ahead of its next call
        ce = cudaMemsetAsync(&ws->P.ctl->error, 0, sizeof(unsigned int), st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) return cuda_err(ce);
        return (int)err;
    }
    Seg S;
    ce = cudaMemcpy(&S, ws->P.segs, sizeof(Seg), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return cuda_err(ce);
    std::memset(info, 0, sizeof(*info));
    info->map = S.kind == MAP_Z       ? ZSORT_MAPINFO_ZSCORE
                : S.kind == MAP_PWL   ? ZSORT_MAPINFO_LEARNED
                : S.kind == MAP_MLP   ? ZSORT_MAPINFO_MLP
                : S.kind == MAP_SPLIT ? ZSORT_MAPINFO_SPLIT
                                      : ZSORT_MAPINFO_RANGE;
    info->k = S.k;
    info->min = S.mn;
    info->max = S.mx;
    info->mean_d = S.mean_d;
    info->sd = S.sd;
    info->zc = S.zc;
    info->zsh = S.zsh;
    info->escale = S.escale;
    info->learned_max_load = S.max_learned;
    info->zscore_max_load = S.max_z;
    if (S.train_slot != INVALID && S.max_learned > 0) {  // the fit ran (it sets the loads)
        float t[PWL_STRIDE];
        ce = cudaMemcpy(t, ws->P.pwl, sizeof(t), cudaMemcpyDeviceToHost);
        if (ce != cudaSuccess) return cuda_err(ce);
        std::memcpy(info->q, t, sizeof(info->q));
        std::memcpy(info->r, t + PWL_P + 1, sizeof(info->r));
        std::memcpy(info->mlp, t + PWL_MLP_OFF, sizeof(info->mlp));
        info->trained = 1;
    }
    return ZSORT_OK;
}

// zsort_pairs_noalloc: see include/zsort.h.  The first call on a device
// looks up the address of the static scratch (cudaGetSymbolAddress, with
// that device current) and sets the kernel's shared-memory attribute; make
// that first call before any stream capture.
int zsort_pairs_noalloc(uint64_t *keys, uint32_t *vals, uint64_t n, int32_t *status, zsort_stream_t stream)
{
    NvtxRange nv("zsort_pairs_noalloc");
    if (n > NA_MAX_N) return ZSORT_ERR_INVALID;
    if (n <= 1) {
        if (status) {
            cudaError_t ce = cudaMemsetAsync(status, 0, sizeof(int32_t), reinterpret_cast<cudaStream_t>(stream));
            if (ce != cudaSuccess) return cuda_err(ce);
        }
        return ZSORT_OK;
    }
    if (!keys) return ZSORT_ERR_INVALID;  // vals may be null: keys only
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_err(ce);
    if (dev < 0 || dev >= 64) return ZSORT_ERR_INVALID;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lock(g_na_mu);
    NaDevice &D = g_na_dev[dev];
    if (!D.ready) {
        void *addr = nullptr;
        ce = cudaGetSymbolAddress(&addr, g_na_scratch);
        if (ce != cudaSuccess || !addr) return ZSORT_ERR_CUDA;
        ce = cudaDeviceGetAttribute(&D.sms, cudaDevAttrMultiProcessorCount, dev);
        if (ce != cudaSuccess) return cuda_err(ce);
        ce = cudaFuncSetAttribute(k_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
        if (ce != cudaSuccess) return cuda_err(ce);
        ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&D.occ, k_persistent, BLOCK, SMEM_BYTES);
        if (ce != cudaSuccess) return cuda_err(ce);
        if (D.occ < 1) return ZSORT_ERR_CUDA;
        D.base = static_cast<char *>(addr);
        D.ready = true;
    }
    zsort_opts o;
    zsort_default_opts(&o);
    Params P{};
    P.ukeys = keys;
    P.uvals = vals;
    P.n = n;
    bind_plan(P, D.base, NA);
    P.kmax = o.kmax;
    P.leaf_target = o.leaf_target;
    P.large_min = o.large_min;
    P.learn_min = o.learn_min;
    P.sample = o.sample;
    P.mapper = o.mapper;
    P.guard_level = o.guard_level;
    P.leaf_cap = o.leaf_cap;
    P.chunks_per_cta = o.chunks_per_cta;
    P.ipt = o.ipt;
    P.tile = (uint32_t)BLOCK * o.ipt;
    P.sub_sample = 1u;
    P.fallback_ratio = o.fallback_ratio;
    P.seed = o.seed;
    P.wait_ns = (unsigned long long)o.wait_limit_ms * 1000000ull;
    P.user_aligned = ((reinterpret_cast<uintptr_t>(keys) | reinterpret_cast<uintptr_t>(vals)) & 15u) == 0;
    P.kv = vals != nullptr;  // null vals: keys only
    // the plan's look-back rows are sized for at most 2 x NA_MAX_SMS CTAs
    P.nctas = (uint32_t)std::min(D.sms * D.occ, 2 * NA_MAX_SMS);
    ce = cudaMemsetAsync(P.ctl, 0, sizeof(Ctl), st);  // the control block must start at zero
    if (ce != cudaSuccess) return cuda_err(ce);
    k_init_segments<<<1, 256, 0, st>>>(P, nullptr, 1);
    k_init_publish<<<1, 32, 0, st>>>(P, 1);
    k_persistent<<<P.nctas, BLOCK, SMEM_BYTES, st>>>(P);
    if (status) k_na_status<<<1, 32, 0, st>>>(P.ctl, status);
    return cuda_err(cudaGetLastError());
}

const char *zsort_strerror(int code)
{
    switch (code) {
    case ZSORT_OK: return "ok";
    case ZSORT_ERR_INVALID: return "invalid argument";
    case ZSORT_ERR_NOMEM: return "device allocation failed";
    case ZSORT_ERR_CUDA: return "CUDA runtime error";
    case ZSORT_ERR_TIMEOUT: return "bounded device wait expired";
    case ZSORT_ERR_BAD_OFFSETS: return "segment offsets decrease or exceed n";
    case ZSORT_ERR_CAPACITY: return "internal device queue overflowed";
    case ZSORT_ERR_INTERNAL: return "device consistency check failed";
    default: return "unknown status";
    }
}

}  // extern "C"
