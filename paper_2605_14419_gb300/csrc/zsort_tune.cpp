// zsort_tune.cpp -- autotuner of zsort's runtime parameters (host code).
//
// A client of the library's own C ABI: it classifies a call from a strided
// key sample, looks the class up in a small JSON cache, and otherwise times
// candidate option sets on a device copy of the caller's data (coordinate
// descent over the knobs listed in include/zsort_tune.h).  The paper has no
// counterpart: its constants (Alg. 1) are fixed for one CPU thread, while the
// GPU executor's tile and bucket sizes are chosen here by measurement.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/zsort_tune.h"

namespace {

constexpr uint64_t SAMPLE_KEYS = 4096;

struct Knob {
    const char *name;
    uint32_t zsort_opts::*field;
    std::vector<uint32_t> values;
};

std::vector<Knob> knobs()
{
    return {
        {"kmax", &zsort_opts::kmax, {128, 256, 512}},
        {"leaf_target", &zsort_opts::leaf_target, {1024, 2048, 4096}},
        {"leaf_cap", &zsort_opts::leaf_cap, {2048, 3072, 4096}},
        {"large_min", &zsort_opts::large_min, {32768, 65536, 131072, 262144}},
        {"chunks_per_cta", &zsort_opts::chunks_per_cta, {4, 8, 16}},
        {"ipt", &zsort_opts::ipt, {8, 12}},
    };
}

// Range checks of the six tuned fields (as the library validates them).
bool tuned_fields_valid(const zsort_opts &o)
{
    if (o.kmax < 16 || o.kmax > 512 || (o.kmax & (o.kmax - 1))) return false;
    if (o.leaf_target < 16 || o.leaf_target > (1u << 24)) return false;
    if (o.leaf_cap < 256 || o.leaf_cap > 4096) return false;
    if (o.large_min < 4096 || o.large_min >= (1u << 30)) return false;
    if (o.chunks_per_cta < 1 || o.chunks_per_cta > 64) return false;
    if (o.ipt != 8 && o.ipt != 12) return false;
    return true;
}

int round_log2(uint64_t x)
{
    return x <= 1 ? 0 : (int)std::lround(std::log2((double)x));
}

const char *resolve_path(const char *path)
{
    if (path && *path) return path;
    const char *e = std::getenv("ZSORT_TUNE_CACHE");
    return (e && *e) ? e : nullptr;
}

// One cache line: "<class>": {"kmax": .., ..., "ms": ..}
struct Entry {
    std::string cls;
    zsort_opts o;
    double ms;
};

bool field_u32(const std::string &line, const char *name, uint32_t *v)
{
    const std::string pat = std::string("\"") + name + "\":";
    size_t p = line.find(pat);
    if (p == std::string::npos) return false;
    char *end = nullptr;
    const char *b = line.c_str() + p + pat.size();
    unsigned long long x = std::strtoull(b, &end, 10);
    if (end == b || x > 0xffffffffull) return false;
    *v = (uint32_t)x;
    return true;
}

bool field_f64(const std::string &line, const char *name, double *v)
{
    const std::string pat = std::string("\"") + name + "\":";
    size_t p = line.find(pat);
    if (p == std::string::npos) return false;
    char *end = nullptr;
    const char *b = line.c_str() + p + pat.size();
    double x = std::strtod(b, &end);
    if (end == b) return false;
    *v = x;
    return true;
}

// Parses one entry line; false for lines that are not entries ("{", "}").
// *bad is set for an entry line whose fields do not parse.
bool parse_entry(const std::string &line, Entry *e, bool *bad)
{
    *bad = false;
    size_t q0 = line.find('"');
    if (q0 == std::string::npos) return false;
    size_t q1 = line.find('"', q0 + 1);
    if (q1 == std::string::npos || line.find('{', q1) == std::string::npos) {
        *bad = true;
        return false;
    }
    e->cls = line.substr(q0 + 1, q1 - q0 - 1);
    std::memset(&e->o, 0, sizeof(e->o));
    e->ms = 0.0;
    const std::string rest = line.substr(q1 + 1);
    bool ok = field_u32(rest, "kmax", &e->o.kmax) && field_u32(rest, "leaf_target", &e->o.leaf_target) &&
              field_u32(rest, "leaf_cap", &e->o.leaf_cap) && field_u32(rest, "large_min", &e->o.large_min) &&
              field_u32(rest, "chunks_per_cta", &e->o.chunks_per_cta) && field_f64(rest, "ms", &e->ms);
    if (ok && !field_u32(rest, "ipt", &e->o.ipt)) e->o.ipt = 12;  // entries written before the knob existed
    if (!ok || !tuned_fields_valid(e->o)) {
        *bad = true;
        return false;
    }
    return true;
}

// Reads all entries; returns false if the file does not exist.  Entry lines
// that do not parse are reported through *bad_line (their class if known).
bool read_cache(const char *path, std::vector<Entry> *out, std::vector<std::string> *bad_lines)
{
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    std::string line;
    char buf[512];
    while (std::fgets(buf, sizeof(buf), f)) {
        line += buf;
        if (line.empty() || line.back() != '\n') {
            if (!std::feof(f)) continue;  // a long line: keep reading
        }
        Entry e;
        bool bad = false;
        if (parse_entry(line, &e, &bad))
            out->push_back(e);
        else if (bad && bad_lines)
            bad_lines->push_back(line);
        line.clear();
    }
    std::fclose(f);
    return true;
}

bool write_cache(const char *path, const std::vector<Entry> &entries)
{
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "w");
    if (!f) return false;
    std::fprintf(f, "{\n");
    for (size_t i = 0; i < entries.size(); i++) {
        const Entry &e = entries[i];
        std::fprintf(f,
                     "\"%s\": {\"kmax\": %u, \"leaf_target\": %u, \"leaf_cap\": %u, \"large_min\": %u, "
                     "\"chunks_per_cta\": %u, \"ipt\": %u, \"ms\": %.4f}%s\n",
                     e.cls.c_str(), e.o.kmax, e.o.leaf_target, e.o.leaf_cap, e.o.large_min, e.o.chunks_per_cta,
                     e.o.ipt, e.ms, i + 1 < entries.size() ? "," : "");
    }
    std::fprintf(f, "}\n");
    const bool ok = std::fflush(f) == 0;
    std::fclose(f);
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return false;
    }
    return true;
}

void copy_tuned(const zsort_opts &from, zsort_opts *to)
{
    to->kmax = from.kmax;
    to->leaf_target = from.leaf_target;
    to->leaf_cap = from.leaf_cap;
    to->large_min = from.large_min;
    to->chunks_per_cta = from.chunks_per_cta;
    to->ipt = from.ipt;
}

int sample_keys(const uint64_t *keys, uint64_t n, std::vector<uint64_t> *s, cudaStream_t st)
{
    const uint64_t m = std::min<uint64_t>(n, SAMPLE_KEYS);
    s->assign(m, 0);
    if (m == 0) return ZSORT_OK;
    // positions floor(i * n / m): one pitched copy when the stride is exact,
    // else one small copy per key
    if (n % m == 0) {
        const size_t stride = (size_t)(n / m) * sizeof(uint64_t);
        cudaError_t e = cudaMemcpy2DAsync(s->data(), sizeof(uint64_t), keys, stride, sizeof(uint64_t), (size_t)m,
                                          cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return ZSORT_ERR_CUDA;
    } else {
        for (uint64_t i = 0; i < m; i++) {
            const uint64_t p = (uint64_t)((unsigned __int128)i * n / m);
            cudaError_t e = cudaMemcpyAsync(&(*s)[i], keys + p, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) return ZSORT_ERR_CUDA;
        }
    }
    return cudaStreamSynchronize(st) == cudaSuccess ? ZSORT_OK : ZSORT_ERR_CUDA;
}

int device_sms(int *sms)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ZSORT_ERR_CUDA;
    if (cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ZSORT_ERR_CUDA;
    return ZSORT_OK;
}

// Device copies of the caller's data that every trial sorts.
struct Trial {
    const uint64_t *keys;
    const uint32_t *vals;
    uint64_t n;
    const uint64_t *off;
    uint64_t nseg;
    uint64_t *k2 = nullptr;
    uint32_t *v2 = nullptr;
    cudaStream_t st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;

    int init()
    {
        if (cudaMalloc(&k2, std::max<uint64_t>(n, 1) * 8) != cudaSuccess) return ZSORT_ERR_NOMEM;
        if (cudaMalloc(&v2, std::max<uint64_t>(n, 1) * 4) != cudaSuccess) return ZSORT_ERR_NOMEM;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return ZSORT_ERR_CUDA;
        return ZSORT_OK;
    }
    ~Trial()
    {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (k2) cudaFree(k2);
        if (v2) cudaFree(v2);
    }
    // Median time (ms) of `reps` sorts with options o; +inf on any error.
    double run(const zsort_opts &o, uint32_t reps)
    {
        std::vector<double> t;
        for (uint32_t r = 0; r < reps; r++) {
            if (cudaMemcpyAsync(k2, keys, n * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return INFINITY;
            if (cudaMemcpyAsync(v2, vals, n * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return INFINITY;
            cudaEventRecord(e0, st);
            int rc = off ? zsort_segmented_ex(k2, v2, n, off, nseg, &o, reinterpret_cast<zsort_stream_t>(st))
                         : zsort_pairs_ex(k2, ZSORT_KEY_U64, v2, n, &o, reinterpret_cast<zsort_stream_t>(st));
            cudaEventRecord(e1, st);
            if (rc != ZSORT_OK) return INFINITY;
            if (zsort_sync_status(reinterpret_cast<zsort_stream_t>(st)) != ZSORT_OK) return INFINITY;
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return INFINITY;
            t.push_back(ms);
        }
        std::sort(t.begin(), t.end());
        return t.empty() ? INFINITY : t[t.size() / 2];
    }
};

}  // namespace

extern "C" {

int zsort_tune_class_host(const uint64_t *sample, uint64_t m, uint64_t n, uint64_t nseg, int sms, char *cls,
                          size_t cls_len)
{
    if (!cls || cls_len < ZSORT_TUNE_CLASS_MAX || (m > 0 && !sample) || sms < 0) return ZSORT_ERR_INVALID;
    const char *dist = "flat";
    if (m >= 2) {
        std::vector<uint64_t> s(sample, sample + m);
        uint64_t asc = 0, desc = 0;
        for (uint64_t i = 0; i + 1 < m; i++) {
            asc += s[i] <= s[i + 1];
            desc += s[i] > s[i + 1];
        }
        std::sort(s.begin(), s.end());
        const uint64_t distinct = (uint64_t)(std::unique(s.begin(), s.end()) - s.begin());
        if (2 * distinct < m) {
            dist = "dup";
        } else if (10 * asc >= 9 * (m - 1)) {
            dist = "sorted";
        } else if (10 * desc >= 9 * (m - 1)) {
            dist = "reversed";
        } else {
            // Eq. 1 on the sample: k = 512 buckets, scale k/4, statistics of
            // d = key - min in double precision
            const uint64_t mn = s.front();
            double mean = 0.0;
            for (uint64_t x : s) mean += (double)(x - mn);
            mean /= (double)m;
            double var = 0.0;
            for (uint64_t x : s) {
                const double d = (double)(x - mn) - mean;
                var += d * d;
            }
            const double sd = std::sqrt(var / (double)m);
            const uint32_t k = 512;
            std::vector<uint32_t> load(k, 0);
            for (uint64_t x : s) {
                double h = sd > 0.0 ? (double)(x - mn) / sd * (k / 4.0) : 0.0;
                uint32_t b = h >= (double)(k - 1) ? k - 1 : (uint32_t)h;
                load[b]++;
            }
            const uint32_t mx = *std::max_element(load.begin(), load.end());
            dist = (double)mx <= 4.0 * (double)m / k ? "flat" : "skew";
        }
    }
    const int len = std::snprintf(cls, cls_len, "sm%d/n%d/s%d/%s", sms, round_log2(n), nseg <= 1 ? 0 : round_log2(nseg),
                                  dist);
    return (len > 0 && (size_t)len < cls_len) ? ZSORT_OK : ZSORT_ERR_INVALID;
}

int zsort_tune_class(const uint64_t *keys, uint64_t n, uint64_t nseg, char *cls, size_t cls_len,
                     zsort_stream_t stream)
{
    if (!cls || (n > 0 && !keys)) return ZSORT_ERR_INVALID;
    int sms = 0;
    int rc = device_sms(&sms);
    if (rc != ZSORT_OK) return rc;
    std::vector<uint64_t> s;
    rc = sample_keys(keys, n, &s, reinterpret_cast<cudaStream_t>(stream));
    if (rc != ZSORT_OK) return rc;
    return zsort_tune_class_host(s.data(), s.size(), n, nseg, sms, cls, cls_len);
}

int zsort_tune_cache_get(const char *path, const char *cls, zsort_opts *out, double *ms)
{
    if (!path || !cls || !out) return ZSORT_ERR_INVALID;
    std::vector<Entry> entries;
    std::vector<std::string> bad;
    if (!read_cache(path, &entries, &bad)) return ZSORT_NOT_TUNED;
    const std::string key = std::string("\"") + cls + "\"";
    for (const std::string &b : bad)
        if (b.find(key) != std::string::npos) return ZSORT_ERR_INVALID;
    for (const Entry &e : entries) {
        if (e.cls == cls) {
            copy_tuned(e.o, out);
            if (ms) *ms = e.ms;
            return ZSORT_OK;
        }
    }
    return ZSORT_NOT_TUNED;
}

int zsort_tune_cache_put(const char *path, const char *cls, const zsort_opts *o, double ms)
{
    if (!path || !cls || !o || !tuned_fields_valid(*o)) return ZSORT_ERR_INVALID;
    if (std::strchr(cls, '"') || std::strchr(cls, '\n') || !*cls) return ZSORT_ERR_INVALID;
    std::vector<Entry> entries;
    read_cache(path, &entries, nullptr);
    bool found = false;
    for (Entry &e : entries) {
        if (e.cls == cls) {
            copy_tuned(*o, &e.o);
            e.ms = ms;
            found = true;
        }
    }
    if (!found) {
        Entry e;
        e.cls = cls;
        std::memset(&e.o, 0, sizeof(e.o));
        copy_tuned(*o, &e.o);
        e.ms = ms;
        entries.push_back(e);
    }
    return write_cache(path, entries) ? ZSORT_OK : ZSORT_ERR_INVALID;
}

int zsort_tuned_opts(const uint64_t *keys, uint64_t n, uint64_t nseg, const zsort_opts *base,
                     const char *cache_path, zsort_opts *out, zsort_stream_t stream)
{
    if (!out) return ZSORT_ERR_INVALID;
    if (base)
        *out = *base;
    else
        zsort_default_opts(out);
    const char *path = resolve_path(cache_path);
    if (!path) return ZSORT_NOT_TUNED;
    char cls[ZSORT_TUNE_CLASS_MAX];
    int rc = zsort_tune_class(keys, n, nseg, cls, sizeof(cls), stream);
    if (rc != ZSORT_OK) return rc;
    zsort_opts t = *out;
    rc = zsort_tune_cache_get(path, cls, &t, nullptr);
    if (rc == ZSORT_OK) *out = t;
    return rc;
}

int zsort_autotune(const uint64_t *keys, const uint32_t *vals, uint64_t n, const uint64_t *seg_offsets,
                   uint64_t nseg, const zsort_opts *base, const char *cache_path, uint32_t budget_ms,
                   uint32_t reps, uint32_t flags, zsort_opts *out, zsort_stream_t stream)
{
    if (!out || !keys || !vals || n < 2) return ZSORT_ERR_INVALID;
    if (!seg_offsets && n > ZSORT_MAX_N) return ZSORT_ERR_INVALID;
    if (seg_offsets && (nseg == 0 || n > ZSORT_MAX_SEG_TOTAL)) return ZSORT_ERR_INVALID;
    zsort_opts cur;
    if (base)
        cur = *base;
    else
        zsort_default_opts(&cur);
    if (cur.struct_size != sizeof(zsort_opts)) return ZSORT_ERR_INVALID;
    const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const char *path = resolve_path(cache_path);
    const uint64_t segs = seg_offsets ? nseg : 0;
    char cls[ZSORT_TUNE_CLASS_MAX];
    int rc = zsort_tune_class(keys, n, segs, cls, sizeof(cls), stream);
    if (rc != ZSORT_OK) return rc;
    if (path && !(flags & ZSORT_TUNE_FORCE)) {
        zsort_opts t = cur;
        if (zsort_tune_cache_get(path, cls, &t, nullptr) == ZSORT_OK) {
            *out = t;
            return ZSORT_OK;
        }
    }
    Trial tr{keys, vals, n, seg_offsets, nseg};
    tr.st = st;
    rc = tr.init();
    if (rc != ZSORT_OK) return rc;
    if (reps == 0) reps = 3;
    const auto t_start = std::chrono::steady_clock::now();
    auto over_budget = [&]() {
        if (budget_ms == 0) return false;
        const auto el = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t_start);
        return el.count() >= (long long)budget_ms;
    };
    tr.run(cur, 1);  // warm-up: workspace allocation, first-launch costs
    double best = tr.run(cur, reps);
    const std::vector<Knob> ks = knobs();
    for (int pass = 0; pass < 3 && !over_budget(); pass++) {
        bool changed = false;
        for (const Knob &kb : ks) {
            for (uint32_t v : kb.values) {
                if (over_budget()) break;
                if (cur.*(kb.field) == v) continue;
                zsort_opts cand = cur;
                cand.*(kb.field) = v;
                if (cand.large_min < cand.leaf_cap) continue;
                const double t = tr.run(cand, reps);
                if (t < best * 0.99) {  // keep a change only for a clear gain
                    best = t;
                    cur = cand;
                    changed = true;
                }
            }
        }
        if (!changed) break;
    }
    if (!std::isfinite(best)) return ZSORT_ERR_CUDA;
    *out = cur;
    if (path) zsort_tune_cache_put(path, cls, &cur, best);
    return ZSORT_OK;
}

}  // extern "C"
