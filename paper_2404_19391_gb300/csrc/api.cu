// Error reporting, scratch caching and small ABI helpers.
#include <stdio.h>
#include <stdlib.h>

#include "zs_common.cuh"

namespace zs {

static thread_local std::string t_error;
static thread_local double t_kernel_ms = 0.0;

void mark_kernel_start(Scratch *sc, cudaStream_t s)
{
    if (!sc->ev0) cudaEventCreate(&sc->ev0);
    if (!sc->ev1) cudaEventCreate(&sc->ev1);
    cudaEventRecord(sc->ev0, s);
}

void mark_kernel_end(Scratch *sc, cudaStream_t s) { cudaEventRecord(sc->ev1, s); }

void note_kernel_time(Scratch *sc)
{
    float ms = 0.f;
    if (sc->ev0 && sc->ev1 && cudaEventElapsedTime(&ms, sc->ev0, sc->ev1) == cudaSuccess) t_kernel_ms = ms;
    else cudaGetLastError();
}

void set_error(const std::string &msg) { t_error = msg; }
void clear_error() { t_error.clear(); }

zs_status cuda_fail(cudaError_t e, const char *what)
{
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return ZS_ERR_CUDA;
}

uint64_t wait_limit_ns()
{
    const char *v = getenv("ZS_WAIT_LIMIT_MS");
    if (v && *v) {
        long long ms = atoll(v);
        if (ms > 0) return (uint64_t)ms * 1000000ull;
    }
    return 20ull * 1000000000ull;  // 20 s: far above any legitimate wait
}

int64_t injected_stall_tile()
{
    const char *v = getenv("ZS_INJECT_STALL");
    if (v && *v) return atoll(v);
    return -1;
}

int64_t span_cut_min_override()
{
    const char *v = getenv("ZS_SPAN_CUT_MIN");
    if (v && *v) return atoll(v);
    return -1;
}

ScratchPool::~ScratchPool() { release_all(); }

void ScratchPool::release_all()
{
    std::lock_guard<std::mutex> g(mu_);
    int cur = -1;
    cudaGetDevice(&cur);
    for (auto &kv : map_) {
        Scratch &s = kv.second;
        if (s.device >= 0) cudaSetDevice(s.device);
        if (s.dev) cudaFree(s.dev);
        if (s.slow) cudaFree(s.slow);
        if (s.host) cudaFreeHost(s.host);
        if (s.ev0) cudaEventDestroy(s.ev0);
        if (s.ev1) cudaEventDestroy(s.ev1);
    }
    map_.clear();
    if (cur >= 0) cudaSetDevice(cur);
}

zs_status ScratchPool::get(void *stream, size_t tiles, size_t slow, Scratch **out)
{
    std::lock_guard<std::mutex> g(mu_);
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    Scratch &s = map_[std::make_pair(stream, std::this_thread::get_id())];
    if (s.device >= 0 && s.device != dev) {
        set_error("stream scratch belongs to another device");
        return ZS_ERR_INVALID_ARG;
    }
    s.device = dev;
    cudaStream_t st = (cudaStream_t)stream;
    if (!s.host) {
        e = cudaMallocHost((void **)&s.host, sizeof(DevResult));
        if (e != cudaSuccess) {
            s.host = nullptr;
            set_error("cudaMallocHost failed");
            return ZS_ERR_OOM;
        }
    }
    if (!s.dev || s.cap_tiles < tiles) {
        size_t cap = tiles < 1024 ? 1024 : tiles + tiles / 4;
        if (s.dev) {
            cudaStreamSynchronize(st);
            cudaFree(s.dev);
            s.dev = nullptr;
        }
        e = cudaMalloc(&s.dev, sizeof(DevResult) + cap * sizeof(TileState));
        if (e != cudaSuccess) {
            s.dev = nullptr;
            s.cap_tiles = 0;
            cudaGetLastError();
            set_error("cudaMalloc of tile scratch failed");
            return ZS_ERR_OOM;
        }
        s.cap_tiles = cap;
    }
    if (slow > s.slow_cap) {
        size_t cap = slow < (64u << 20) ? (64u << 20) : slow;
        if (s.slow) {
            cudaStreamSynchronize(st);
            cudaFree(s.slow);
            s.slow = nullptr;
        }
        e = cudaMalloc((void **)&s.slow, cap);
        if (e != cudaSuccess) {
            s.slow = nullptr;
            s.slow_cap = 0;
            cudaGetLastError();
            set_error("cudaMalloc of long-line scratch failed");
            return ZS_ERR_OOM;
        }
        s.slow_cap = cap;
    }
    *out = &s;
    return ZS_OK;
}

ScratchPool &global_pool()
{
    static ScratchPool *p = new ScratchPool();  // lives until exit (never destroyed after the CUDA runtime)
    return *p;
}

}  // namespace zs

extern "C" const char *zs_last_error(void) { return zs::t_error.c_str(); }

extern "C" double zs_last_kernel_ms(void) { return zs::t_kernel_ms; }

extern "C" const char *zs_version(void) { return "zsmiles-gb300 0.1 (sm_103a)"; }

extern "C" size_t zs_compress_bound(size_t in_len) { return 3 * in_len + 16; }

extern "C" size_t zs_decompress_bound(const zs_dict *d, size_t in_len)
{
    return d ? (size_t)d->lmax * in_len : 0;
}

extern "C" int zs_dictionary_lmax(const zs_dict *d) { return d ? d->lmax : 0; }
