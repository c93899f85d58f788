// Batched form: many shards through one persistent launch, replayed from a CUDA graph, with the kernel
// geometry picked by timing the compiled variants on the batch itself.
//
// A plan fixes the shards (device buffers and sizes) once. Its device block holds one launch-wide
// result record, one result record per shard, the shard table and the look-back records of every tile;
// a shard's tiles are numbered from 0 for its own look-back chain and from tile0 in the launch-wide
// numbering from which the warps of the persistent kernel claim work. A run is: clear the block, zero
// the line index of empty shards, launch, copy the result records to pinned host memory. With a graph
// those steps are captured once and replayed by one cudaGraphLaunch.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "zs_common.cuh"

using zs::DevResult;
using zs::ShardView;
using zs::TileState;

struct zs_plan {
    const zs_dict *d = nullptr;
    zs_op op = ZS_OP_COMPRESS;
    unsigned flags = 0;
    int device = -1;
    std::vector<zs_shard> shards;
    int variant = 0;
    int cut_min = 0;               // span geometries: cut threshold (0: the geometry's default, < 0: never)
    bool use_graph = true;
    std::vector<double> tuned_ms;  // per variant (its best cut setting); < 0: not timed

    // device block: ShardView table[n] | DevResult g | DevResult res[n] | TileState tiles[max_tiles]
    void *dev = nullptr;
    size_t max_tiles = 0;
    uint64_t total_tiles = 0;
    uint8_t *slow = nullptr;
    size_t slow_cap = 0;
    DevResult *host = nullptr;  // pinned [n + 1]
    std::vector<ShardView> table;

    cudaStream_t cap = nullptr;  // private stream for capture
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    float last_ms = 0.f;

    size_t n() const { return shards.size(); }
    ShardView *dtable() const { return reinterpret_cast<ShardView *>(dev); }
    DevResult *dres() const { return reinterpret_cast<DevResult *>(dtable() + n()); }
    TileState *dtiles() const { return reinterpret_cast<TileState *>(dres() + n() + 1); }
    size_t clear_bytes() const { return (n() + 1) * sizeof(DevResult) + total_tiles * sizeof(TileState); }
};

namespace {

const zs::KernelVariant *variant_info(zs_op op, int v)
{
    return op == ZS_OP_COMPRESS ? zs::compress_warp_variant(v) : zs::decompress_variant(v);
}

int variant_count(zs_op op) { return op == ZS_OP_COMPRESS ? zs::compress_warp_variants() : zs::decompress_variants(); }

bool variant_usable(const zs_plan *p, int v)
{
    if (!variant_info(p->op, v)) return false;
    return p->op == ZS_OP_DECOMPRESS ? zs::decompress_fits(v, p->d) : zs::compress_warp_fits(v, p->d);
}

void drop_graph(zs_plan *p)
{
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->exec = nullptr;
    p->graph = nullptr;
}

// Lays the shards out for variant v (tile numbering, table) and uploads the table.
zs_status layout(zs_plan *p, int v)
{
    const uint32_t tb = variant_info(p->op, v)->tile_bytes;
    uint64_t t0 = 0;
    p->table.assign(p->n(), ShardView{});
    for (size_t i = 0; i < p->n(); ++i) {
        const zs_shard &s = p->shards[i];
        ShardView &v2 = p->table[i];
        const uint64_t nt = zs::tiles_for(s.in_len, tb);
        v2 = zs::single_shard(s.in, s.in_len, s.out, s.out_cap, p->op == ZS_OP_COMPRESS ? s.line_index : nullptr,
                              p->op == ZS_OP_COMPRESS && s.line_index ? s.index_cap : 0, nullptr,
                              p->dres() + 1 + i, nt);
        v2.tile0 = t0;
        v2.tiles = p->dtiles() + t0;
        t0 += nt;
    }
    p->total_tiles = t0;
    p->variant = v;
    cudaError_t e = cudaMemcpy(p->dtable(), p->table.data(), p->n() * sizeof(ShardView), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return zs::cuda_fail(e, "zs_plan: shard table upload");
    drop_graph(p);
    return ZS_OK;
}

cudaError_t issue(zs_plan *p, cudaStream_t s, bool capturing)
{
    cudaError_t e = cudaMemsetAsync(p->dres(), 0, p->clear_bytes(), s);
    if (p->op == ZS_OP_COMPRESS)
        for (const zs_shard &sh : p->shards)
            if (e == cudaSuccess && sh.in_len == 0 && sh.line_index && sh.index_cap >= 1)
                e = cudaMemsetAsync(sh.line_index, 0, sizeof(uint64_t), s);
    if (e != cudaSuccess) return e;
    if (p->total_tiles > 0) {
        zs::TiledLaunch L{};
        L.one = p->table.empty() ? ShardView{} : p->table[0];
        L.shards = p->dtable();
        L.n_shards = (uint32_t)p->n();
        L.total_tiles = p->total_tiles;
        L.g = p->dres();
        L.slow = p->slow;
        L.slow_cap = p->slow_cap;
        L.cut_min = p->cut_min;
        // under stream capture a plain record would only order streams: record external event nodes
        const unsigned rf = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
        e = cudaEventRecordWithFlags(p->ev0, s, rf);
        if (e == cudaSuccess)
            e = p->op == ZS_OP_COMPRESS ? zs::launch_compress_warp(p->variant, p->d, L, p->flags, s)
                                        : zs::launch_decompress(p->variant, p->d, L, s);
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(p->ev1, s, rf);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->host, p->dres(), (p->n() + 1) * sizeof(DevResult), cudaMemcpyDeviceToHost, s);
    return e;
}

zs_status build_graph(zs_plan *p)
{
    drop_graph(p);
    cudaError_t e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return zs::cuda_fail(e, "zs_plan: begin capture");
    cudaError_t e2 = issue(p, p->cap, true);
    e = cudaStreamEndCapture(p->cap, &p->graph);
    if (e2 != cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (e != cudaSuccess) {
        drop_graph(p);
        return zs::cuda_fail(e, "zs_plan: graph capture");
    }
    return ZS_OK;
}

zs_status grow_slow(zs_plan *p, size_t need)
{
    if (p->op != ZS_OP_COMPRESS || need <= p->slow_cap) return ZS_OK;
    if (p->slow) cudaFree(p->slow);
    p->slow = nullptr;
    p->slow_cap = 0;
    cudaError_t e = cudaMalloc(&p->slow, need);
    if (e != cudaSuccess) {
        cudaGetLastError();
        zs::set_error("zs_plan: out of device memory for the long-line scratch");
        return ZS_ERR_OOM;
    }
    p->slow_cap = need;
    drop_graph(p);
    return ZS_OK;
}

// One run on `s`, retried with a larger long-line scratch when it overflowed, and (when `fall_back`) with
// the general compression kernel when the span kernel met a line outside its fast path: the plan keeps that
// geometry from then on. Fills p->host.
zs_status run_once(zs_plan *p, cudaStream_t s, bool fall_back = true)
{
    for (int attempt = 0; attempt < 4; ++attempt) {
        cudaError_t e;
        if (p->use_graph) {
            if (!p->exec) {
                zs_status st = build_graph(p);
                if (st != ZS_OK) return st;
            }
            e = cudaGraphLaunch(p->exec, s);
        } else {
            e = issue(p, s, false);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return zs::cuda_fail(e, "zs_plan_run");
        p->last_ms = 0.f;
        if (p->total_tiles > 0 && cudaEventElapsedTime(&p->last_ms, p->ev0, p->ev1) != cudaSuccess) {
            cudaGetLastError();
            p->last_ms = 0.f;
        }
        const DevResult &g = p->host[0];
        if ((g.status & zs::kStFallback) && !(g.status & zs::kStTimeout) && fall_back &&
            p->op == ZS_OP_COMPRESS && zs::compress_variant_is_span(p->variant)) {
            const int gv = zs::compress_general_variant(p->d);
            if (gv < 0) {
                zs::set_error("zs_plan_run: no general kernel variant fits this dictionary");
                return ZS_ERR_BAD_DICT;
            }
            zs_status st = layout(p, gv);
            if (st != ZS_OK) return st;
            continue;
        }
        if (g.status & zs::kStSlowOverflow) {
            const size_t need = (size_t)g.slow_used + ((size_t)g.slow_used >> 2) + (1u << 20);
            zs_status st = grow_slow(p, need);
            if (st != ZS_OK) return st;
            continue;
        }
        return ZS_OK;
    }
    zs::set_error("zs_plan_run: long-line scratch could not be sized");
    return ZS_ERR_OOM;
}

// Per-shard results and the call's status from p->host.
zs_status collect(zs_plan *p, zs_result *res)
{
    const DevResult &g = p->host[0];
    zs_status first = ZS_OK;
    std::string msg;
    auto fail = [&](zs_status st, const std::string &m) {
        if (first == ZS_OK) {
            first = st;
            msg = m;
        }
    };
    if (g.status & zs::kStTimeout) fail(ZS_ERR_TIMEOUT, "zs_plan_run: a device-side wait expired");
    if (g.status & zs::kStTooBig) fail(ZS_ERR_INVALID_ARG, "zs_plan_run: a line longer than 1 GiB");
    for (size_t i = 0; i < p->n(); ++i) {
        const DevResult &r = p->host[1 + i];
        const zs_shard &sh = p->shards[i];
        zs_result out{r.out_len, r.n_lines, 0};
        if (r.err_key) out.err_offset = ~r.err_key;
        if (res) res[i] = out;
        const std::string tag = "zs_plan_run: shard " + std::to_string(i) + ": ";
        if (p->op == ZS_OP_DECOMPRESS && r.err_key)
            fail(ZS_ERR_MALFORMED, tag + "malformed input at byte " + std::to_string(out.err_offset));
        if (r.out_len > sh.out_cap) fail(ZS_ERR_CAPACITY, tag + "output buffer too small");
        if (p->op == ZS_OP_COMPRESS && sh.line_index && r.n_lines + 1 > sh.index_cap)
            fail(ZS_ERR_CAPACITY, tag + "line index buffer too small");
    }
    if (first != ZS_OK) zs::set_error(msg);
    return first;
}

// Times `reps` runs of the current layout (after one untimed run that also sizes the long-line scratch);
// *skip: the batch needs the general kernel (the span geometry cannot run it).
zs_status time_runs(zs_plan *p, int reps, double *ms, bool *skip)
{
    zs_status st = run_once(p, p->cap, false);
    *skip = st == ZS_OK && (p->host[0].status & zs::kStFallback);
    std::vector<float> t;
    for (int k = 0; k < reps && st == ZS_OK && !*skip; ++k) {
        st = run_once(p, p->cap, false);
        t.push_back(p->last_ms);
    }
    std::sort(t.begin(), t.end());
    *ms = t.empty() ? 0.0 : t[t.size() / 2];
    return st;
}

// Autotuning: every geometry that fits, and for span geometries the long-line cut setting both ways (the
// geometry's default and its opposite: cuts at 3/64 of a tile, or none); keeps the fastest.
zs_status tune(zs_plan *p, int reps)
{
    const int nv = variant_count(p->op);
    p->tuned_ms.assign(nv, -1.0);
    int best = -1, best_cut = 0;
    double best_ms = 0.0;
    const bool graph = p->use_graph;
    p->use_graph = false;
    for (int v = 0; v < nv; ++v) {
        if (!variant_usable(p, v)) continue;
        zs_status st = layout(p, v);
        if (st != ZS_OK) {
            p->use_graph = graph;
            return st;
        }
        const bool span = p->op == ZS_OP_COMPRESS && zs::compress_variant_is_span(v);
        const int ncut = span ? 2 : 1;
        for (int c = 0; c < ncut; ++c) {
            // cut setting c: 0 the geometry's default, 1 the opposite one
            const uint32_t dflt = span ? zs::span_cut_default(v) : 0u;
            p->cut_min = c == 0 ? 0 : (dflt ? -1 : (int)(3 * variant_info(p->op, v)->tile_bytes / 64));
            double ms = 0.0;
            bool skip = false;
            st = time_runs(p, reps, &ms, &skip);
            if (st != ZS_OK) {
                p->use_graph = graph;
                return st;
            }
            if (skip) break;  // this batch needs the general kernel
            if (p->tuned_ms[v] < 0 || ms < p->tuned_ms[v]) p->tuned_ms[v] = ms;
            if (best < 0 || ms < best_ms) {
                best = v;
                best_ms = ms;
                best_cut = p->cut_min;
            }
        }
    }
    p->use_graph = graph;
    if (best < 0) {
        zs::set_error("zs_plan_create: no kernel variant fits this dictionary");
        return ZS_ERR_BAD_DICT;
    }
    p->cut_min = best_cut;
    return layout(p, best);
}

// ---- tuning cache: (GPU model, dictionary, operation, flags, batch shape class) -> (variant, cut setting).
// The shape class is log2 of the batch's bytes, of its shard count and of its largest shard. Kept in the
// process; with ZS_TUNE_CACHE naming a file, loaded from it once and appended to. Plans use it only when
// their options ask (tune_cache).
std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune;
bool g_tune_loaded = false;

int ilog2(uint64_t x)
{
    int k = 0;
    while (x > 1) {
        x >>= 1;
        ++k;
    }
    return k;
}

std::string tune_key(const zs_plan *p)
{
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, p->device);
    uint64_t total = 0, mx = 0;
    for (const zs_shard &s : p->shards) {
        total += s.in_len;
        mx = std::max<uint64_t>(mx, s.in_len);
    }
    char buf[512];
    snprintf(buf, sizeof buf, "%s/sm%d.%d/x%d|%016llx|%d|%u|%d|%d|%d", prop.name, prop.major, prop.minor,
             prop.multiProcessorCount, (unsigned long long)p->d->digest, (int)p->op, p->flags, ilog2(total + 1),
             ilog2(p->shards.size() + 1), ilog2(mx + 1));
    for (char *c = buf; *c; ++c)
        if (*c == ' ') *c = '_';
    return buf;
}

void tune_cache_load()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = getenv("ZS_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char key[512];
    int v = 0, c = 0;
    while (fscanf(f, "%511s %d %d", key, &v, &c) == 3) g_tune[key] = {v, c};
    fclose(f);
}

bool tune_cache_get(const std::string &k, int *v, int *c)
{
    std::lock_guard<std::mutex> g(g_tune_mu);
    tune_cache_load();
    auto it = g_tune.find(k);
    if (it == g_tune.end()) return false;
    *v = it->second.first;
    *c = it->second.second;
    return true;
}

void tune_cache_put(const std::string &k, int v, int c)
{
    std::lock_guard<std::mutex> g(g_tune_mu);
    tune_cache_load();
    g_tune[k] = {v, c};
    const char *path = getenv("ZS_TUNE_CACHE");
    if (!path || !*path) return;
    if (FILE *f = fopen(path, "a")) {
        fprintf(f, "%s %d %d\n", k.c_str(), v, c);
        fclose(f);
    }
}

}  // namespace

extern "C" int zs_kernel_variants(zs_op op)
{
    return (op == ZS_OP_COMPRESS || op == ZS_OP_DECOMPRESS) ? variant_count(op) : 0;
}

extern "C" const char *zs_kernel_variant_name(zs_op op, int v)
{
    if (op != ZS_OP_COMPRESS && op != ZS_OP_DECOMPRESS) return nullptr;
    const zs::KernelVariant *k = variant_info(op, v);
    return k ? k->name : nullptr;
}

extern "C" void zs_plan_destroy(zs_plan *p)
{
    if (!p) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (p->device >= 0) cudaSetDevice(p->device);
    if (p->cap) cudaStreamSynchronize(p->cap);
    drop_graph(p);
    if (p->ev0) cudaEventDestroy(p->ev0);
    if (p->ev1) cudaEventDestroy(p->ev1);
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->dev) cudaFree(p->dev);
    if (p->slow) cudaFree(p->slow);
    if (p->host) cudaFreeHost(p->host);
    if (cur >= 0) cudaSetDevice(cur);
    delete p;
}

extern "C" zs_status zs_plan_create(const zs_dict *d, zs_op op, unsigned flags, const zs_shard *shards,
                                    size_t n_shards, const zs_plan_options *opt, zs_plan **out)
{
    zs::clear_error();
    if (!out) {
        zs::set_error("zs_plan_create: NULL argument");
        return ZS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (!d || (!shards && n_shards)) {
        zs::set_error("zs_plan_create: NULL argument");
        return ZS_ERR_INVALID_ARG;
    }
    if (op != ZS_OP_COMPRESS && op != ZS_OP_DECOMPRESS) {
        zs::set_error("zs_plan_create: unknown operation");
        return ZS_ERR_INVALID_ARG;
    }
    if (!zs::compress_flags_ok(flags)) {
        zs::set_error("zs_plan_create: unknown flag bits, or ZS_PREPROCESS_OUTER without ZS_PREPROCESS");
        return ZS_ERR_INVALID_ARG;
    }
    if (n_shards > (size_t)ZS_MAX_SHARDS) {
        zs::set_error("zs_plan_create: more than ZS_MAX_SHARDS shards");
        return ZS_ERR_INVALID_ARG;
    }
    for (size_t i = 0; i < n_shards; ++i) {
        const zs_shard &s = shards[i];
        if ((!s.in && s.in_len) || (!s.out && s.out_cap) || (op == ZS_OP_COMPRESS && !s.line_index && s.index_cap)) {
            zs::set_error("zs_plan_create: shard " + std::to_string(i) + " has a NULL buffer");
            return ZS_ERR_INVALID_ARG;
        }
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return zs::cuda_fail(e, "zs_plan_create: cudaGetDevice");
    if (dev != d->device) {
        zs::set_error("zs_plan_create: dictionary was loaded on another device");
        return ZS_ERR_INVALID_ARG;
    }
    const int nv = variant_count(op);
    const int want = opt ? opt->variant : -1;
    if (want >= nv) {
        zs::set_error("zs_plan_create: no such kernel variant");
        return ZS_ERR_INVALID_ARG;
    }

    zs_plan *p = new zs_plan;
    p->d = d;
    p->op = op;
    p->flags = flags;
    p->device = dev;
    p->shards.assign(shards, shards + n_shards);
    p->use_graph = opt ? opt->use_graph != 0 : true;
    // tile records for the variant with the smallest tiles
    for (int v = 0; v < nv; ++v) {
        const uint32_t tb = variant_info(op, v)->tile_bytes;
        size_t nt = 0;
        for (const zs_shard &s : p->shards) nt += zs::tiles_for(s.in_len, tb);
        p->max_tiles = std::max(p->max_tiles, nt);
    }
    const size_t bytes = (n_shards + 1) * sizeof(DevResult) + n_shards * sizeof(ShardView) +
                         p->max_tiles * sizeof(TileState);
    e = cudaMalloc(&p->dev, bytes);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&p->host), (n_shards + 1) * sizeof(DevResult));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&p->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&p->ev1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        zs_plan_destroy(p);
        zs::set_error("zs_plan_create: out of memory");
        return ZS_ERR_OOM;
    }
    zs_status st = grow_slow(p, op == ZS_OP_COMPRESS ? (16u << 20) : 0);
    if (st == ZS_OK) {
        if (want >= 0) {
            if (!variant_usable(p, want)) {
                zs::set_error("zs_plan_create: the kernel variant does not fit this dictionary");
                st = ZS_ERR_BAD_DICT;
            } else {
                p->tuned_ms.assign(nv, -1.0);
                p->cut_min = opt ? opt->cut_min : 0;
                st = layout(p, want);
            }
        } else {
            const bool cache = opt && opt->tune_cache;
            const std::string key = cache ? tune_key(p) : std::string();
            int cv = -1, cc = 0;
            if (cache && tune_cache_get(key, &cv, &cc) && cv >= 0 && cv < nv && variant_usable(p, cv)) {
                p->tuned_ms.assign(nv, -1.0);  // taken from the cache, not timed
                p->cut_min = cc;
                st = layout(p, cv);
            } else {
                st = tune(p, std::max(1, opt && opt->tune_reps > 0 ? opt->tune_reps : 3));
                if (st == ZS_OK && cache) tune_cache_put(key, p->variant, p->cut_min);
            }
        }
    }
    if (st != ZS_OK) {
        zs_plan_destroy(p);
        return st;
    }
    *out = p;
    return ZS_OK;
}

extern "C" zs_status zs_plan_run(zs_plan *p, zs_result *res, void *stream)
{
    zs::clear_error();
    if (!p) {
        zs::set_error("zs_plan_run: NULL plan");
        return ZS_ERR_INVALID_ARG;
    }
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != p->device) {
        zs::set_error("zs_plan_run: the plan was made on another device");
        return ZS_ERR_INVALID_ARG;
    }
    zs_status st = run_once(p, (cudaStream_t)stream);
    if (st != ZS_OK) return st;
    return collect(p, res);
}

extern "C" int zs_plan_variant(const zs_plan *p) { return p ? p->variant : -1; }

extern "C" int zs_plan_cut_min(const zs_plan *p)
{
    if (!p || p->op != ZS_OP_COMPRESS || !zs::compress_variant_is_span(p->variant)) return 0;
    if (p->cut_min > 0) return p->cut_min;
    return p->cut_min < 0 ? 0 : (int)zs::span_cut_default(p->variant);
}

extern "C" double zs_plan_tuned_ms(const zs_plan *p, int v)
{
    if (!p || v < 0 || v >= (int)p->tuned_ms.size()) return -1.0;
    return p->tuned_ms[v];
}

extern "C" double zs_plan_last_ms(const zs_plan *p) { return p ? (double)p->last_ms : 0.0; }

extern "C" zs_status zs_compress_batch(const zs_dict *d, const zs_shard *shards, size_t n_shards, unsigned flags,
                                       zs_result *res, void *stream)
{
    const int v = d ? zs::compress_default_variant(d) : -1;
    zs_plan_options o{v >= 0 ? v : zs::kDefaultVariant, 0, 0};
    zs_plan *p = nullptr;
    zs_status st = zs_plan_create(d, ZS_OP_COMPRESS, flags, shards, n_shards, &o, &p);
    if (st != ZS_OK) return st;
    st = zs_plan_run(p, res, stream);
    zs_plan_destroy(p);
    return st;
}

extern "C" zs_status zs_decompress_batch(const zs_dict *d, const zs_shard *shards, size_t n_shards, zs_result *res,
                                         void *stream)
{
    zs_plan_options o{d ? zs::decompress_default_variant(d) : zs::kDefaultVariant, 0, 0};
    zs_plan *p = nullptr;
    zs_status st = zs_plan_create(d, ZS_OP_DECOMPRESS, 0, shards, n_shards, &o, &p);
    if (st != ZS_OK) return st;
    st = zs_plan_run(p, res, stream);
    zs_plan_destroy(p);
    return st;
}
