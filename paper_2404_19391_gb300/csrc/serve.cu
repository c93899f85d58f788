// Serving form of random access (Sec. I: any line of a compressed library can be decoded alone): a
// resident compressed store plus its line index, and a request loop with continuous batching.
//
//   - Requests (sets of line ids) are submitted from any host thread and queue in arrival order.
//   - One scheduler thread admits the queue head into a free in-flight slot as soon as the slot and
//     the output arenas have room: every queued request that fits (ids per launch, arena bytes) joins
//     the batch, so requests that arrive while others are on the GPU ride the next launch. A batch is
//     one random-access launch over the concatenated ids; up to max_inflight batches run at once, each
//     on its own stream, so their copies and kernels overlap.
//   - Memory admission: a request of k ids reserves k times the store's longest decoded line (found
//     once, on the GPU, when the server is made; O(1) host work per request) in a device arena and in
//     a pinned, mapped host arena. Behind the random-access kernel, a copy kernel reads the exact decoded size on the device
//     and streams those bytes into the host arena with coalesced 16-byte stores, so one launch sequence
//     and one event complete a batch (no host round trip to learn the size). The device reservation is
//     released when the batch completes; the host bytes stay until the result is fetched or released.
//   - The batch's output offsets land in its host region too, behind its bytes, and stay there until its
//     last request is fetched or released: completing a batch costs O(1) host work per request (no per-id
//     copy); zs_server_fetch rebases a request's offsets as it copies them out.
//   - A request that arrives while no batch is in flight is launched by the submitting thread itself (no
//     hand-off to the scheduler); under load, requests queue and the scheduler batches them.
//   - Completion is observed by polling CUDA events (the scheduler yields between polls while work is
//     in flight); latency is arrival to the completion of the batch's host copy.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "zs_common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over [0, size) with coalescing; 256-byte granules.
class RangeAlloc {
   public:
    void reset(size_t size)
    {
        free_.clear();
        if (size) free_[0] = size;
        size_ = size;
    }
    static size_t round(size_t n) { return (std::max<size_t>(n, 1) + 255) & ~(size_t)255; }
    size_t largest() const
    {
        size_t m = 0;
        for (auto &kv : free_) m = std::max(m, kv.second);
        return m;
    }
    bool alloc(size_t n, size_t *off)
    {
        n = round(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const size_t rest = it->second - n, at = it->first + n;
            free_.erase(it);
            if (rest) free_[at] = rest;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        n = round(n);
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + n == next->first) {
            n += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += n;
                return;
            }
        }
        free_[off] = n;
    }
    size_t size() const { return size_; }

   private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0;
};

struct Batch;

struct Request {
    uint64_t ticket = 0;
    size_t k = 0;                     // ids
    const uint64_t *hid = nullptr;    // its ids: in the pinned ids arena (ids_off) or in heap_ids
    size_t ids_off = SIZE_MAX;        // byte offset in the ids arena, SIZE_MAX: heap_ids
    std::vector<uint64_t> heap_ids;   // used when the ids arena is full
    size_t bound = 0;
    Clock::time_point arrival, done_at;
    int state = 0;  // 0 queued, 1 on the GPU, 2 done, 3 failed
    zs_status err = ZS_OK;
    std::shared_ptr<Batch> batch;
    size_t first = 0;  // index of its first id in the batch
    uint64_t byte_off = 0, byte_len = 0;
    const uint64_t *off = nullptr;  // its k + 1 offsets in the batch's host region (relative to byte_off's base)
};

struct Batch {
    size_t dev_off = 0, host_off = 0, bound = 0;
    const uint64_t *d_ids = nullptr;  // the ids the launch reads (device address of pinned memory)
    size_t host_bound = 0;  // host region: the bytes (bound, rounded to 8) then the K + 1 offsets
    size_t slot = 0;        // the in-flight slot running it
    std::vector<Request *> reqs;
    size_t unfetched = 0;
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    // h_ids and h_res are pinned and mapped: the kernels read the ids and write the result record through
    // their device addresses (d_ids, h_res_dev), with no copy calls; the offsets go to the batch's host region
    uint64_t *h_ids = nullptr, *d_ids = nullptr, *d_off = nullptr;
    void *d_scratch = nullptr;
    zs::DevResult *h_res = nullptr, *h_res_dev = nullptr;
    int state = 0;  // 0 free, 1 batch in flight
    std::shared_ptr<Batch> batch;
    size_t K = 0;
};

// Copies the r->out_len decoded bytes of a batch from the device arena to the mapped host arena (both
// regions 256-byte aligned) with 16-byte loads and stores, grid-stride, and the batch's K + 1 output offsets
// (to the host region behind the bytes) and its result record to their mapped host copies, so the batch needs
// no copy calls of its own.
__global__ void copy_out_kernel(const uint8_t *__restrict__ src, uint8_t *__restrict__ dst, const zs::DevResult *r,
                                uint64_t cap, const uint64_t *__restrict__ off, uint64_t *__restrict__ h_off,
                                uint64_t n_off, zs::DevResult *h_res)
{
    const uint64_t n = min((uint64_t)r->out_len, cap);
    const uint64_t n16 = n >> 4;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (uint64_t i = tid; i < n16; i += stride)
        reinterpret_cast<uint4 *>(dst)[i] = reinterpret_cast<const uint4 *>(src)[i];
    for (uint64_t i = (n16 << 4) + tid; i < n; i += stride) dst[i] = src[i];
    for (uint64_t i = tid; i < n_off; i += stride) h_off[i] = off[i];
    if (tid == 0) *h_res = *r;
}

// The longest decoded line of a store (with its '\n'), and a count of index entries or lines that do
// not decode: one thread per line, the same escape rule as every decoder here (Sec. IV-D2).
__global__ void line_max_kernel(const uint8_t *__restrict__ comp, uint64_t comp_len, const uint64_t *__restrict__ index,
                                uint64_t n_lines, const uint8_t *__restrict__ plen, unsigned long long *out)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    unsigned long long mx = 0, bad = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_lines; i += stride) {
        const uint64_t a = index[i];
        uint64_t b = index[i + 1];
        if (a > b || b > comp_len) {
            ++bad;
            continue;
        }
        if (b > a && comp[b - 1] == '\n') --b;
        uint64_t len = 1;
        bool lit = false, ok = true;
        for (uint64_t p = a; p < b; ++p) {
            const uint8_t c = comp[p];
            if (lit) {
                len += 1;
                lit = false;
            } else if (c == ' ') {
                lit = true;
            } else {
                ok &= plen[c] != 0;
                len += plen[c];
            }
        }
        if (!ok || lit) ++bad;
        mx = max(mx, (unsigned long long)len);
    }
    if (mx) atomicMax(out, mx);
    if (bad) atomicAdd(out + 1, bad);
}

// Host region of a batch whose bytes take `bound`: the bytes, then the K + 1 offsets (8-byte aligned).
size_t offsets_at(size_t bound) { return (bound + 7) & ~(size_t)7; }
size_t host_bound(size_t bound, size_t K) { return offsets_at(bound) + (K + 1) * sizeof(uint64_t); }

double ms_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

double percentile(std::vector<double> v, double q)
{
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace

struct zs_server {
    const zs_dict *d = nullptr;
    int device = -1;
    const uint8_t *comp = nullptr;
    size_t comp_len = 0;
    const uint64_t *index = nullptr;
    size_t n_lines = 0;
    size_t max_line = 1;  // longest decoded line: a request of k ids reserves k * max_line bytes
    zs_server_options opt{};

    uint8_t *d_arena = nullptr;
    uint8_t *h_arena = nullptr;     // pinned, mapped
    // pinned, mapped ids arena: submit copies a request's ids here (no heap allocation, no page faults), and a
    // batch of one request is launched on them where they lie
    uint64_t *h_idsa = nullptr, *d_idsa = nullptr;
    RangeAlloc ids_alloc;
    uint8_t *h_arena_dev = nullptr;  // its device address
    RangeAlloc dev_alloc, host_alloc;
    std::vector<Slot> slots;
    size_t scratch_tiles = 0;

    std::mutex mu;
    std::condition_variable cv;       // scheduler wake-up (submit, stop)
    std::condition_variable done_cv;  // request completions
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_ticket = 1;
    // bumped (under mu) by submit, fetch/release and stop: the idle scheduler waits on it, the polling one
    // reads it without the lock to see that there is new work
    std::atomic<uint64_t> changes{0};
    bool stop = false;
    zs_status fatal = ZS_OK;
    std::string fatal_msg;
    std::thread worker;

    // statistics
    uint64_t n_submitted = 0, n_completed = 0, n_batches = 0, n_ids = 0, batch_reqs = 0;
    int max_inflight_seen = 0;
    std::vector<double> lat_ms;

    void loop();
    bool admit(Slot &s);
    void release_ids(Batch &b);
    void await(std::unique_lock<std::mutex> &lk, Request *r);
    void finish(Slot &s);
    void fail_batch(Slot &s, zs_status st, const std::string &msg);
};

namespace {

unsigned copy_blocks(size_t bound)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
    }
    const size_t want = (bound / 16 + 255) / 256;
    return (unsigned)std::max<size_t>(1, std::min<size_t>(want, (size_t)sms * 4));
}

// Longest decoded line of the store (checks the index and the store on the way).
zs_status store_max_line(const zs_dict *d, const uint8_t *comp, size_t comp_len, const uint64_t *index,
                         size_t n_lines, size_t *max_line, const char *what)
{
    unsigned long long *dv = nullptr, hv[2] = {0, 0};
    cudaError_t e = cudaMalloc(&dv, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(dv, 0, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess && n_lines) {
        const uint64_t blocks = std::min<uint64_t>((n_lines + 255) / 256, 4096);
        line_max_kernel<<<(unsigned)blocks, 256>>>(comp, comp_len, index, n_lines, d->d_dec, dv);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(hv, dv, sizeof hv, cudaMemcpyDeviceToHost);
    if (dv) cudaFree(dv);
    if (e != cudaSuccess) return zs::cuda_fail(e, what);
    if (hv[1]) {
        zs::set_error(std::string(what) + ": " + std::to_string(hv[1]) + " lines of the store do not decode");
        return ZS_ERR_MALFORMED;
    }
    *max_line = std::max<size_t>(1, (size_t)hv[0]);
    return ZS_OK;
}

cudaError_t issue_batch(zs_server *S, Slot &s)
{
    const size_t K = s.K;
    cudaError_t e = cudaMemsetAsync(s.d_scratch, 0,
                                    sizeof(zs::DevResult) + zs::lines_tiles(K) * sizeof(zs::TileState), s.st);
    zs::DevResult *dr = reinterpret_cast<zs::DevResult *>(s.d_scratch);
    zs::TileState *tiles = reinterpret_cast<zs::TileState *>(dr + 1);
    if (e == cudaSuccess)
        e = zs::launch_lines(S->d, S->comp, S->comp_len, S->index, S->n_lines, s.batch->d_ids, K,
                             S->d_arena + s.batch->dev_off, s.batch->bound, s.d_off, dr, tiles, s.st);
    if (e == cudaSuccess) {
        uint8_t *h = S->h_arena_dev + s.batch->host_off;
        copy_out_kernel<<<copy_blocks(s.batch->bound), 256, 0, s.st>>>(
            S->d_arena + s.batch->dev_off, h, dr, s.batch->bound, s.d_off,
            reinterpret_cast<uint64_t *>(h + offsets_at(s.batch->bound)), K + 1, s.h_res_dev);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(s.ev, s.st);
    return e;
}

}  // namespace

// Forms a batch from the queue head for free slot s. Caller holds mu.
bool zs_server::admit(Slot &s)
{
    if (queue.empty()) return false;
    const size_t droom = dev_alloc.largest(), hroom = host_alloc.largest();
    size_t K = 0, bound = 0;
    std::vector<Request *> take;
    for (Request *r : queue) {
        const size_t nb = RangeAlloc::round(bound + r->bound), nk = K + r->k;
        if (nk > opt.max_batch_ids || nb > droom || RangeAlloc::round(host_bound(nb, nk)) > hroom) break;
        K = nk;
        bound = nb;
        take.push_back(r);
    }
    if (take.empty()) return false;  // the head waits for memory (no overtaking)
    auto b = std::make_shared<Batch>();
    b->bound = bound;
    b->host_bound = host_bound(bound, K);
    if (!dev_alloc.alloc(bound, &b->dev_off)) return false;
    if (!host_alloc.alloc(b->host_bound, &b->host_off)) {
        dev_alloc.release(b->dev_off, bound);
        return false;
    }
    size_t at = 0;
    const bool in_place = take.size() == 1 && take[0]->ids_off != SIZE_MAX;  // launched on the arena copy
    for (Request *r : take) {
        if (!in_place) std::memcpy(s.h_ids + at, r->hid, r->k * sizeof(uint64_t));
        r->first = at;
        r->state = 1;
        r->batch = b;
        at += r->k;
        b->reqs.push_back(r);
        queue.pop_front();
    }
    b->d_ids = in_place ? d_idsa + take[0]->ids_off / sizeof(uint64_t) : s.d_ids;
    b->unfetched = take.size();
    b->slot = (size_t)(&s - slots.data());
    s.batch = b;
    s.K = K;
    s.state = 1;
    ++n_batches;
    batch_reqs += take.size();
    n_ids += K;
    cudaError_t e = issue_batch(this, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail_batch(s, ZS_ERR_CUDA, std::string("zs_server: launch failed: ") + cudaGetErrorString(e));
    }
    return true;
}

// The batch's launch has read its requests' ids: their arena space is free again. Holds mu.
void zs_server::release_ids(Batch &b)
{
    for (Request *r : b.reqs) {
        if (r->ids_off != SIZE_MAX) ids_alloc.release(r->ids_off, r->k * sizeof(uint64_t));
        r->ids_off = SIZE_MAX;
        r->hid = nullptr;
        r->heap_ids = std::vector<uint64_t>();
    }
}

void zs_server::fail_batch(Slot &s, zs_status st, const std::string &msg)
{
    auto b = s.batch;
    release_ids(*b);
    const Clock::time_point now = Clock::now();
    for (Request *r : b->reqs) {
        r->state = 3;
        r->err = st;
        r->done_at = now;
    }
    dev_alloc.release(b->dev_off, b->bound);
    if (fatal == ZS_OK && st == ZS_ERR_CUDA) {  // the server takes no more work: fail the queue too
        fatal = st;
        fatal_msg = msg;
        for (Request *r : queue) {
            r->state = 3;
            r->err = st;
            r->done_at = now;
            if (r->ids_off != SIZE_MAX) ids_alloc.release(r->ids_off, r->k * sizeof(uint64_t));
            r->ids_off = SIZE_MAX;
        }
        queue.clear();
    }
    s.state = 0;
    s.batch.reset();
    done_cv.notify_all();
}

// The batch's launches are done: check them, hand out per-request offsets and bytes.
void zs_server::finish(Slot &s)
{
    auto b = s.batch;
    const zs::DevResult r = *s.h_res;
    if (r.status & (zs::kStMalformed | zs::kStTimeout)) {
        fail_batch(s, (r.status & zs::kStTimeout) ? ZS_ERR_TIMEOUT : ZS_ERR_MALFORMED,
                   "zs_server: the random-access launch reported an error");
        return;
    }
    const Clock::time_point now = Clock::now();
    release_ids(*b);
    const uint64_t *offs = reinterpret_cast<const uint64_t *>(h_arena + b->host_off + offsets_at(b->bound));
    for (Request *q : b->reqs) {
        const size_t k = q->k;
        q->off = offs + q->first;
        q->byte_off = q->off[0];
        q->byte_len = q->off[k] - q->off[0];
        q->state = 2;
        q->done_at = now;
        lat_ms.push_back(ms_between(q->arrival, now));
        ++n_completed;
    }
    dev_alloc.release(b->dev_off, b->bound);
    s.state = 0;
    s.batch.reset();
    done_cv.notify_all();
}

// Waits (lk held on mu) until request r is done. While its batch is on the GPU the waiting thread polls the
// batch's event itself and completes the batch when it is done, so a result is seen without a hand-off
// through the scheduler thread (which polls the same events; whichever sees the event first finishes the batch).
void zs_server::await(std::unique_lock<std::mutex> &lk, Request *r)
{
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != device) cudaSetDevice(device);
    while (r->state < 2) {
        if (r->state == 1) {
            Slot &s = slots[r->batch->slot];
            const cudaEvent_t ev = s.ev;
            // poll without the lock for a while (the submitter and the scheduler need it), then look again
            lk.unlock();
            cudaError_t q = cudaErrorNotReady;
            for (int i = 0; i < 64 && q == cudaErrorNotReady; ++i) {
                q = cudaEventQuery(ev);
                if (q == cudaErrorNotReady) std::this_thread::yield();
            }
            lk.lock();
            if (r->state != 1 || s.batch != r->batch) continue;  // finished (or failed) meanwhile
            if (q == cudaErrorNotReady) continue;
            q = cudaEventQuery(ev);
            if (q == cudaSuccess) {
                finish(s);
            } else if (q != cudaErrorNotReady) {
                cudaGetLastError();
                fail_batch(s, ZS_ERR_CUDA, std::string("zs_server: ") + cudaGetErrorString(q));
            }
        } else {
            done_cv.wait(lk, [&] { return r->state != 0; });
        }
    }
    if (cur >= 0 && cur != device) cudaSetDevice(cur);
}

void zs_server::loop()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    std::vector<cudaEvent_t> polled;
    for (;;) {
        bool busy = false, progressed = false;
        for (Slot &s : slots) {
            if (s.state == 0) continue;
            busy = true;
            const cudaError_t q = cudaEventQuery(s.ev);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                cudaGetLastError();
                fail_batch(s, ZS_ERR_CUDA, std::string("zs_server: ") + cudaGetErrorString(q));
            } else {
                finish(s);
            }
            progressed = true;
        }
        int inflight = 0;
        bool free_slot = false;
        for (Slot &s : slots) {
            if (s.state == 0 && fatal == ZS_OK && admit(s)) progressed = true;
            inflight += s.state != 0;
            free_slot |= s.state == 0;
        }
        max_inflight_seen = std::max(max_inflight_seen, inflight);
        if (stop && inflight == 0) break;
        if (progressed) continue;
        if (busy || inflight) {
            // poll the in-flight events without the lock (submitters and waiters take it meanwhile) until one
            // completes, or new work arrives while a slot is free
            polled.clear();
            for (Slot &s : slots)
                if (s.state != 0) polled.push_back(s.ev);
            const uint64_t seen = changes.load();
            lk.unlock();
            for (bool go = true; go;) {
                for (cudaEvent_t ev : polled)
                    if (cudaEventQuery(ev) != cudaErrorNotReady) go = false;
                if (free_slot && changes.load() != seen) go = false;
                if (go) std::this_thread::yield();
            }
            lk.lock();
        } else {
            const uint64_t seen = changes.load();  // the queue head waits for arena room or a new request
            cv.wait(lk, [&] { return stop || changes.load() != seen; });
        }
    }
}

extern "C" zs_status zs_server_create(const zs_dict *d, const uint8_t *d_comp, size_t comp_len,
                                      const uint64_t *d_index, size_t n_lines, const zs_server_options *opt,
                                      zs_server **out)
{
    zs::clear_error();
    if (!out || !d || !d_index || (!d_comp && comp_len)) {
        zs::set_error("zs_server_create: NULL argument");
        return ZS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return zs::cuda_fail(e, "zs_server_create: cudaGetDevice");
    if (dev != d->device) {
        zs::set_error("zs_server_create: dictionary was loaded on another device");
        return ZS_ERR_INVALID_ARG;
    }
    auto S = std::make_unique<zs_server>();
    S->d = d;
    S->device = dev;
    S->comp = d_comp;
    S->comp_len = comp_len;
    S->index = d_index;
    S->n_lines = n_lines;
    S->opt.arena_bytes = opt && opt->arena_bytes ? opt->arena_bytes : (size_t)512 << 20;
    S->opt.max_batch_ids = opt && opt->max_batch_ids ? opt->max_batch_ids : (size_t)1 << 20;
    S->opt.max_inflight = opt && opt->max_inflight > 0 ? opt->max_inflight : 4;
    zs_status st = store_max_line(d, d_comp, comp_len, d_index, n_lines, &S->max_line, "zs_server_create");
    if (st != ZS_OK) return st;
    const size_t K = S->opt.max_batch_ids;
    S->scratch_tiles = zs::lines_tiles(K);
    const size_t ids_bytes = 4 * K * sizeof(uint64_t);
    e = cudaMalloc(&S->d_arena, S->opt.arena_bytes);
    if (e == cudaSuccess)
        e = cudaHostAlloc(reinterpret_cast<void **>(&S->h_idsa), ids_bytes, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&S->d_idsa), S->h_idsa, 0);
    if (e == cudaSuccess)
        e = cudaHostAlloc(reinterpret_cast<void **>(&S->h_arena), S->opt.arena_bytes, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&S->h_arena_dev), S->h_arena, 0);
    S->slots.resize(S->opt.max_inflight);
    for (Slot &s : S->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaHostAlloc(reinterpret_cast<void **>(&s.h_ids), K * sizeof(uint64_t), cudaHostAllocMapped);
        if (e == cudaSuccess)
            e = cudaHostAlloc(reinterpret_cast<void **>(&s.h_res), sizeof(zs::DevResult), cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&s.d_ids), s.h_ids, 0);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&s.h_res_dev), s.h_res, 0);
        if (e == cudaSuccess) e = cudaMalloc(&s.d_off, (K + 1) * sizeof(uint64_t));
        if (e == cudaSuccess)
            e = cudaMalloc(&s.d_scratch, sizeof(zs::DevResult) + S->scratch_tiles * sizeof(zs::TileState));
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        zs_server_destroy(S.release());
        zs::set_error("zs_server_create: out of memory");
        return ZS_ERR_OOM;
    }
    S->dev_alloc.reset(S->opt.arena_bytes);
    S->host_alloc.reset(S->opt.arena_bytes);
    S->ids_alloc.reset(ids_bytes);
    zs_server *raw = S.release();
    raw->worker = std::thread([raw] { raw->loop(); });
    *out = raw;
    return ZS_OK;
}

extern "C" void zs_server_destroy(zs_server *S)
{
    if (!S) return;
    if (S->worker.joinable()) {
        {
            std::lock_guard<std::mutex> g(S->mu);
            S->stop = true;
            for (Request *r : S->queue) {  // never started
                r->state = 3;
                r->err = ZS_ERR_INVALID_ARG;
            }
            S->queue.clear();
            ++S->changes;
        }
        S->cv.notify_all();
        S->done_cv.notify_all();
        S->worker.join();
    }
    int cur = -1;
    cudaGetDevice(&cur);
    if (S->device >= 0) cudaSetDevice(S->device);
    for (Slot &s : S->slots) {
        if (s.st) cudaStreamSynchronize(s.st);
        if (s.ev) cudaEventDestroy(s.ev);
        if (s.st) cudaStreamDestroy(s.st);
        if (s.h_ids) cudaFreeHost(s.h_ids);
        if (s.h_res) cudaFreeHost(s.h_res);
        if (s.d_off) cudaFree(s.d_off);
        if (s.d_scratch) cudaFree(s.d_scratch);
    }
    if (S->d_arena) cudaFree(S->d_arena);
    if (S->h_arena) cudaFreeHost(S->h_arena);
    if (S->h_idsa) cudaFreeHost(S->h_idsa);
    if (cur >= 0) cudaSetDevice(cur);
    delete S;
}

extern "C" zs_status zs_server_submit(zs_server *S, const uint64_t *ids, size_t k, uint64_t *ticket)
{
    zs::clear_error();
    if (!S || !ticket || (!ids && k)) {
        zs::set_error("zs_server_submit: NULL argument");
        return ZS_ERR_INVALID_ARG;
    }
    const Clock::time_point now = Clock::now();
    if (k > S->opt.max_batch_ids) {
        zs::set_error("zs_server_submit: more ids than one launch takes (max_batch_ids)");
        return ZS_ERR_INVALID_ARG;
    }
    auto r = std::make_unique<Request>();
    r->k = k;
    r->arrival = now;
    uint64_t top = 0;
    for (size_t j = 0; j < k; ++j) top = std::max(top, ids[j]);
    if (k && top >= S->n_lines) {
        zs::set_error("zs_server_submit: line id " + std::to_string(top) + " out of range");
        return ZS_ERR_INVALID_ARG;
    }
    const size_t bound = k * S->max_line;
    r->bound = bound;
    if (RangeAlloc::round(host_bound(bound, k)) > S->opt.arena_bytes) {
        zs::set_error("zs_server_submit: the request's output bound exceeds the arena");
        return ZS_ERR_CAPACITY;
    }
    // the ids are copied into the pinned ids arena (space reserved under the lock, copied outside it), or into
    // the heap when the arena is full
    if (k) {
        {
            std::lock_guard<std::mutex> g(S->mu);
            size_t off = 0;
            if (S->ids_alloc.alloc(k * sizeof(uint64_t), &off)) r->ids_off = off;
        }
        if (r->ids_off != SIZE_MAX) {
            uint64_t *dst = S->h_idsa + r->ids_off / sizeof(uint64_t);
            std::memcpy(dst, ids, k * sizeof(uint64_t));
            r->hid = dst;
        } else {
            r->heap_ids.assign(ids, ids + k);
            r->hid = r->heap_ids.data();
        }
    }
    std::lock_guard<std::mutex> g(S->mu);
    if (S->fatal != ZS_OK) {
        if (r->ids_off != SIZE_MAX) S->ids_alloc.release(r->ids_off, k * sizeof(uint64_t));
        zs::set_error(S->fatal_msg);
        return S->fatal;
    }
    r->ticket = S->next_ticket++;
    *ticket = r->ticket;
    ++S->n_submitted;
    Request *p = r.get();
    S->reqs[p->ticket] = std::move(r);
    if (k == 0) {
        p->state = 2;
        p->done_at = now;
        ++S->n_completed;
        S->lat_ms.push_back(0.0);
        S->done_cv.notify_all();
        return ZS_OK;
    }
    S->queue.push_back(p);
    ++S->changes;
    // an idle server (nothing in flight, nothing queued before this request) launches it at once from this
    // thread: no hand-off to the scheduler at low load; under load the scheduler batches the queue
    bool idle = S->fatal == ZS_OK && S->queue.size() == 1;
    for (const Slot &s : S->slots) idle &= s.state == 0;
    if (idle) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != S->device) cudaSetDevice(S->device);
        S->admit(S->slots[0]);
        if (cur >= 0 && cur != S->device) cudaSetDevice(cur);
    }
    S->cv.notify_all();
    return ZS_OK;
}

extern "C" zs_status zs_server_wait(zs_server *S, uint64_t ticket, double timeout_s, zs_result *res)
{
    zs::clear_error();
    if (!S) {
        zs::set_error("zs_server_wait: NULL argument");
        return ZS_ERR_INVALID_ARG;
    }
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) {
        zs::set_error("zs_server_wait: unknown ticket");
        return ZS_ERR_INVALID_ARG;
    }
    Request *r = it->second.get();
    auto ready = [&] { return r->state >= 2; };
    if (timeout_s < 0) {
        S->await(lk, r);
    } else if (!S->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
        zs::set_error("zs_server_wait: timed out");
        return ZS_ERR_TIMEOUT;
    }
    if (res) {
        res->out_len = r->byte_len;
        res->n_lines = r->k;
        res->err_offset = 0;
    }
    if (r->state == 3) {
        zs::set_error("zs_server_wait: the request failed");
        return r->err;
    }
    return ZS_OK;
}

namespace {

// Drops a finished request, releasing its batch's host bytes with the batch's last request. Holds mu.
void drop(zs_server *S, std::unordered_map<uint64_t, std::unique_ptr<Request>>::iterator it)
{
    Request *r = it->second.get();
    if (auto b = r->batch) {
        if (--b->unfetched == 0) S->host_alloc.release(b->host_off, b->host_bound);
        r->batch.reset();
    }
    S->reqs.erase(it);
    ++S->changes;
    S->cv.notify_all();  // host room may let the queue head in
}

// Waits for a request, notes when it finished, and drops it.
zs_status wait_release(zs_server *S, uint64_t ticket, Clock::time_point *done_at)
{
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return ZS_ERR_INVALID_ARG;
    Request *r = it->second.get();
    S->await(lk, r);
    const zs_status st = r->state == 3 ? r->err : ZS_OK;
    *done_at = r->done_at;
    drop(S, it);
    return st;
}

void wait_until(Clock::time_point t)
{
    if (t - Clock::now() > std::chrono::microseconds(200)) std::this_thread::sleep_until(t - std::chrono::microseconds(100));
    while (Clock::now() < t) std::this_thread::yield();
}

}  // namespace

extern "C" zs_status zs_server_fetch(zs_server *S, uint64_t ticket, uint8_t *out, size_t out_cap, uint64_t *off)
{
    zs::clear_error();
    if (!S) {
        zs::set_error("zs_server_fetch: NULL argument");
        return ZS_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) {
        zs::set_error("zs_server_fetch: unknown ticket");
        return ZS_ERR_INVALID_ARG;
    }
    Request *r = it->second.get();
    if (r->state < 2) {
        zs::set_error("zs_server_fetch: the request is not finished (call zs_server_wait first)");
        return ZS_ERR_INVALID_ARG;
    }
    if (r->state == 3) {
        const zs_status st = r->err;
        drop(S, it);
        zs::set_error("zs_server_fetch: the request failed");
        return st;
    }
    if ((r->byte_len && !out) || out_cap < r->byte_len) {
        zs::set_error("zs_server_fetch: output buffer too small");
        return ZS_ERR_CAPACITY;
    }
    if (r->byte_len) std::memcpy(out, S->h_arena + r->batch->host_off + r->byte_off, r->byte_len);
    if (off) {
        const size_t k = r->k;
        if (!r->off) off[0] = 0;  // an empty request
        for (size_t j = 0; r->off && j <= k; ++j) off[j] = r->off[j] - r->byte_off;
    }
    drop(S, it);
    return ZS_OK;
}

extern "C" zs_status zs_server_release(zs_server *S, uint64_t ticket)
{
    zs::clear_error();
    if (!S) {
        zs::set_error("zs_server_release: NULL argument");
        return ZS_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end() || it->second->state < 2) {
        zs::set_error("zs_server_release: unknown or unfinished ticket");
        return ZS_ERR_INVALID_ARG;
    }
    drop(S, it);
    return ZS_OK;
}

extern "C" zs_status zs_server_get_stats(zs_server *S, zs_server_stats *st)
{
    zs::clear_error();
    if (!S || !st) {
        zs::set_error("zs_server_get_stats: NULL argument");
        return ZS_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> g(S->mu);
    st->submitted = S->n_submitted;
    st->completed = S->n_completed;
    st->batches = S->n_batches;
    st->ids = S->n_ids;
    st->mean_batch_requests = S->n_batches ? (double)S->batch_reqs / (double)S->n_batches : 0.0;
    st->max_inflight = S->max_inflight_seen;
    st->p50_ms = percentile(S->lat_ms, 0.50);
    st->p99_ms = percentile(S->lat_ms, 0.99);
    return ZS_OK;
}

namespace {

zs_status check_replay_args(const double *arrival_s, const uint64_t *ids, const size_t *k, size_t n_req,
                            double *latency_ms, const char *what)
{
    if ((!arrival_s || !k || !latency_ms) && n_req) {
        zs::set_error(std::string(what) + ": NULL argument");
        return ZS_ERR_INVALID_ARG;
    }
    size_t total = 0;
    for (size_t r = 0; r < n_req; ++r) {
        if (r && arrival_s[r] < arrival_s[r - 1]) {
            zs::set_error(std::string(what) + ": arrival times must not decrease");
            return ZS_ERR_INVALID_ARG;
        }
        total += k[r];
    }
    if (total && !ids) {
        zs::set_error(std::string(what) + ": NULL ids");
        return ZS_ERR_INVALID_ARG;
    }
    return ZS_OK;
}

}  // namespace

extern "C" zs_status zs_server_replay(zs_server *S, const double *arrival_s, const uint64_t *ids, const size_t *k,
                                      size_t n_req, double *latency_ms, double *makespan_s)
{
    zs::clear_error();
    if (!S) {
        zs::set_error("zs_server_replay: NULL argument");
        return ZS_ERR_INVALID_ARG;
    }
    zs_status st = check_replay_args(arrival_s, ids, k, n_req, latency_ms, "zs_server_replay");
    if (st != ZS_OK) return st;
    std::vector<uint64_t> tickets(n_req, 0);
    std::vector<Clock::time_point> when(n_req);
    std::mutex tmu;
    std::condition_variable tcv;
    size_t posted = 0;
    zs_status col_st = ZS_OK;
    Clock::time_point last_done;
    const Clock::time_point t0 = Clock::now() + std::chrono::milliseconds(2);
    for (size_t r = 0; r < n_req; ++r)
        when[r] = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(arrival_s[r]));
    std::thread collector([&] {
        cudaSetDevice(S->device);
        last_done = t0;
        for (size_t r = 0; r < n_req; ++r) {
            uint64_t t;
            {
                std::unique_lock<std::mutex> lk(tmu);
                tcv.wait(lk, [&] { return posted > r; });
                t = tickets[r];
            }
            if (t == 0) {  // submission failed; the submitter stops
                latency_ms[r] = -1.0;
                continue;
            }
            Clock::time_point done;
            const zs_status s2 = wait_release(S, t, &done);
            if (s2 != ZS_OK && col_st == ZS_OK) col_st = s2;
            latency_ms[r] = ms_between(when[r], done);
            last_done = std::max(last_done, done);
        }
    });
    size_t at = 0;
    for (size_t r = 0; r < n_req; ++r) {
        wait_until(when[r]);
        uint64_t t = 0;
        if (st == ZS_OK) st = zs_server_submit(S, ids + at, k[r], &t);
        if (st != ZS_OK) t = 0;
        at += k[r];
        {
            std::lock_guard<std::mutex> g(tmu);
            tickets[r] = t;
            posted = r + 1;
        }
        tcv.notify_all();
    }
    collector.join();
    if (makespan_s) *makespan_s = std::chrono::duration<double>(last_done - t0).count();
    if (st == ZS_OK && col_st != ZS_OK) {
        zs::set_error("zs_server_replay: a request failed");
        st = col_st;
    }
    return st;
}

extern "C" zs_status zs_serial_replay(const zs_dict *d, const uint8_t *d_comp, size_t comp_len,
                                      const uint64_t *d_index, size_t n_lines, const double *arrival_s,
                                      const uint64_t *ids, const size_t *k, size_t n_req, double *latency_ms,
                                      double *makespan_s, void *stream)
{
    zs::clear_error();
    if (!d || !d_index || (!d_comp && comp_len)) {
        zs::set_error("zs_serial_replay: NULL argument");
        return ZS_ERR_INVALID_ARG;
    }
    zs_status st = check_replay_args(arrival_s, ids, k, n_req, latency_ms, "zs_serial_replay");
    if (st != ZS_OK) return st;
    size_t max_line = 1;
    st = store_max_line(d, d_comp, comp_len, d_index, n_lines, &max_line, "zs_serial_replay");
    if (st != ZS_OK) return st;
    size_t kmax = 1, at = 0;
    for (size_t r = 0; r < n_req; ++r) {
        for (size_t j = 0; j < k[r]; ++j)
            if (ids[at + j] >= n_lines) {
                zs::set_error("zs_serial_replay: line id out of range");
                return ZS_ERR_INVALID_ARG;
            }
        at += k[r];
        kmax = std::max(kmax, k[r]);
    }
    const size_t bmax = kmax * max_line;
    cudaError_t e = cudaSuccess;
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t *h_ids = nullptr, *d_ids = nullptr, *h_off = nullptr, *d_off = nullptr;
    uint8_t *h_out = nullptr, *d_out = nullptr;
    void *d_scr = nullptr;
    zs::DevResult *h_res = nullptr;
    const size_t scr = sizeof(zs::DevResult) + zs::lines_tiles(kmax) * sizeof(zs::TileState);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&h_ids), kmax * 8);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&h_off), (kmax + 1) * 8);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&h_out), bmax);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&h_res), sizeof(zs::DevResult));
    if (e == cudaSuccess) e = cudaMalloc(&d_ids, kmax * 8);
    if (e == cudaSuccess) e = cudaMalloc(&d_off, (kmax + 1) * 8);
    if (e == cudaSuccess) e = cudaMalloc(&d_out, bmax);
    if (e == cudaSuccess) e = cudaMalloc(&d_scr, scr);
    const Clock::time_point t0 = Clock::now() + std::chrono::milliseconds(2);
    Clock::time_point last = t0;
    at = 0;
    for (size_t r = 0; r < n_req && e == cudaSuccess; ++r) {
        const Clock::time_point when =
            t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(arrival_s[r]));
        wait_until(when);
        const size_t K = k[r];
        if (K) {
            std::memcpy(h_ids, ids + at, K * 8);
            zs::DevResult *dr = reinterpret_cast<zs::DevResult *>(d_scr);
            e = cudaMemcpyAsync(d_ids, h_ids, K * 8, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaMemsetAsync(d_scr, 0, scr, s);
            if (e == cudaSuccess)
                e = zs::launch_lines(d, d_comp, comp_len, d_index, n_lines, d_ids, K, d_out, bmax, d_off, dr,
                                     reinterpret_cast<zs::TileState *>(dr + 1), s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h_off, d_off, (K + 1) * 8, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h_res, dr, sizeof(zs::DevResult), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e == cudaSuccess && (h_res->status & (zs::kStMalformed | zs::kStTimeout))) {
                st = (h_res->status & zs::kStTimeout) ? ZS_ERR_TIMEOUT : ZS_ERR_MALFORMED;
                break;
            }
            if (e == cudaSuccess && h_res->out_len)
                e = cudaMemcpyAsync(h_out, d_out, h_res->out_len, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
        const Clock::time_point done = Clock::now();
        latency_ms[r] = ms_between(when, done);
        last = std::max(last, done);
        at += K;
    }
    if (makespan_s) *makespan_s = std::chrono::duration<double>(last - t0).count();
    const cudaError_t e_run = e;
    if (h_ids) cudaFreeHost(h_ids);
    if (h_off) cudaFreeHost(h_off);
    if (h_out) cudaFreeHost(h_out);
    if (h_res) cudaFreeHost(h_res);
    if (d_ids) cudaFree(d_ids);
    if (d_off) cudaFree(d_off);
    if (d_out) cudaFree(d_out);
    if (d_scr) cudaFree(d_scr);
    if (e_run != cudaSuccess) return zs::cuda_fail(e_run, "zs_serial_replay");
    if (st != ZS_OK) zs::set_error("zs_serial_replay: the random-access launch reported an error");
    return st;
}
