// Host-to-host pipelines: zs_compress_host / zs_decompress_host.
//
// The stream is cut into chunks at line ends. Lines are independent (Sec. I), so each chunk is coded on
// its own and the chunks' outputs, concatenated, are the output of the whole stream (every chunk but the
// last ends with '\n'). Up to n_streams chunks are in flight, each on its own stream with its own device
// buffers:
//   copy in (H2D) -> tiled kernel -> result record back to pinned host memory
// The host thread retires chunks in order. Once a chunk's output size is known it places the chunk, on the
// slot's own copy-out stream:
//   - rebases the chunk's line index by the bytes before it (a small kernel);
//   - copies output and index to their offsets in the caller's host buffers (D2H);
//   - then reuses the slot for a later chunk: its copy in starts at once, and only its kernel, which
//     rewrites the slot's output buffers, waits for the copy out.
// Copies in both directions and the kernels of different chunks overlap.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "zs_common.cuh"

namespace {

struct PipeSlot {
    cudaStream_t st = nullptr;      // copy in, kernel, result record
    cudaEvent_t ev = nullptr;       // the chunk's result record has landed
    cudaStream_t out_st = nullptr;  // rebase and copy out
    cudaEvent_t out_ev = nullptr;   // the slot's output buffers have been copied out
    bool out_pending = false;
    uint8_t *d_in = nullptr, *d_out = nullptr, *slow = nullptr;
    uint64_t *d_idx = nullptr;
    void *scratch = nullptr;  // DevResult + TileState[tiles]
    zs::DevResult *h_res = nullptr;
    size_t slow_cap = 0;
    // the chunk in flight
    bool busy = false;
    uint64_t off = 0, len = 0;
};

struct Pipe {
    zs_op op = ZS_OP_COMPRESS;
    size_t chunk = 0;
    std::vector<PipeSlot> slots;
};

__global__ void rebase_kernel(uint64_t *idx, uint64_t n, uint64_t base)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        idx[i] += base;
}

void free_pipe(Pipe &p)
{
    for (PipeSlot &s : p.slots) {
        if (s.st) cudaStreamSynchronize(s.st);
        if (s.out_st) cudaStreamSynchronize(s.out_st);
        if (s.ev) cudaEventDestroy(s.ev);
        if (s.out_ev) cudaEventDestroy(s.out_ev);
        if (s.st) cudaStreamDestroy(s.st);
        if (s.out_st) cudaStreamDestroy(s.out_st);
        if (s.d_in) cudaFree(s.d_in);
        if (s.d_out) cudaFree(s.d_out);
        if (s.d_idx) cudaFree(s.d_idx);
        if (s.scratch) cudaFree(s.scratch);
        if (s.slow) cudaFree(s.slow);
        if (s.h_res) cudaFreeHost(s.h_res);
    }
    p.slots.clear();
}

}  // namespace

struct zs_pipes {
    std::mutex mu;
    Pipe pipe[2];  // by zs_op
};

namespace zs {
void free_pipes(zs_dict *d)
{
    if (!d->pipes) return;
    for (Pipe &p : d->pipes->pipe) free_pipe(p);
    delete d->pipes;
    d->pipes = nullptr;
}
}  // namespace zs

namespace {

size_t out_bound(const zs_dict *d, zs_op op, size_t n)
{
    return op == ZS_OP_COMPRESS ? 3 * n + 16 : (size_t)std::max(1, d->lmax) * n + 16;
}

// Makes (or reuses) the pipeline of `op` with the given chunk size and stream count.
zs_status get_pipe(zs_dict *d, zs_op op, size_t chunk, int nst, Pipe **out)
{
    Pipe &p = d->pipes->pipe[op];
    if (p.chunk == chunk && (int)p.slots.size() == nst) {
        *out = &p;
        return ZS_OK;
    }
    free_pipe(p);
    p.op = op;
    p.chunk = chunk;
    p.slots.resize(nst);
    const uint64_t tiles = op == ZS_OP_COMPRESS ? zs::compress_scratch_tiles(d, chunk) : zs::decompress_tiles(chunk);
    cudaError_t e = cudaSuccess;
    for (PipeSlot &s : p.slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.out_st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.out_ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&s.d_in, chunk + 16);
        if (e == cudaSuccess) e = cudaMalloc(&s.d_out, out_bound(d, op, chunk));
        if (e == cudaSuccess && op == ZS_OP_COMPRESS) e = cudaMalloc(&s.d_idx, (chunk + 2) * sizeof(uint64_t));
        if (e == cudaSuccess) e = cudaMalloc(&s.scratch, sizeof(zs::DevResult) + tiles * sizeof(zs::TileState));
        if (e == cudaSuccess && op == ZS_OP_COMPRESS) {
            s.slow_cap = (size_t)64 << 20;
            e = cudaMalloc(&s.slow, s.slow_cap);
        }
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&s.h_res), sizeof(zs::DevResult));
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_pipe(p);
        p.chunk = 0;
        zs::set_error("zs pipeline: out of memory for the chunk buffers");
        return ZS_ERR_OOM;
    }
    *out = &p;
    return ZS_OK;
}

// End of the chunk starting at `off`: the last line end at most `chunk` bytes on, or the stream end if that
// is closer. Returns `off` when no line ends within `chunk` bytes (a line too long for the pipeline).
uint64_t chunk_end(const uint8_t *h, uint64_t n, uint64_t off, uint64_t chunk)
{
    if (n - off <= chunk) return n;
    for (uint64_t q = off + chunk; q > off; --q)
        if (h[q - 1] == '\n') return q;
    return off;
}

struct Totals {
    uint64_t out = 0, lines = 0;
    zs_status st = ZS_OK;
    std::string msg;
    uint64_t err_offset = 0;
};

}  // namespace

namespace {

zs_status run_pipeline(const zs_dict *dc, zs_op op, const uint8_t *h_in, size_t in_len, unsigned flags,
                       uint8_t *h_out, size_t out_cap, uint64_t *h_index, size_t index_cap, zs_result *res,
                       const zs_pipeline_options *opt, const char *what)
{
    zs::clear_error();
    if (!dc || !res || (!h_in && in_len) || (!h_out && out_cap) || (op == ZS_OP_COMPRESS && !h_index && index_cap)) {
        zs::set_error(std::string(what) + ": NULL argument");
        return ZS_ERR_INVALID_ARG;
    }
    if (!zs::compress_flags_ok(flags)) {
        zs::set_error(std::string(what) + ": unknown flag bits, or ZS_PREPROCESS_OUTER without ZS_PREPROCESS");
        return ZS_ERR_INVALID_ARG;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return zs::cuda_fail(e, what);
    if (dev != dc->device) {
        zs::set_error(std::string(what) + ": dictionary was loaded on another device");
        return ZS_ERR_INVALID_ARG;
    }
    res->out_len = res->n_lines = res->err_offset = 0;
    if (in_len == 0) {
        if (h_index) {
            if (index_cap < 1) {
                zs::set_error(std::string(what) + ": line index buffer too small");
                return ZS_ERR_CAPACITY;
            }
            h_index[0] = 0;
        }
        return ZS_OK;
    }
    const size_t chunk = opt && opt->chunk_bytes ? std::max<size_t>(opt->chunk_bytes, 4096) : ((size_t)32 << 20);
    const int nst = opt && opt->n_streams > 0 ? std::min(opt->n_streams, 16) : 4;
    zs_dict *d = const_cast<zs_dict *>(dc);
    {
        static std::mutex init_mu;
        std::lock_guard<std::mutex> g(init_mu);
        if (!d->pipes) d->pipes = new zs_pipes;
    }
    std::lock_guard<std::mutex> g(d->pipes->mu);  // calls on one dictionary run one at a time
    Pipe *p = nullptr;
    zs_status st = get_pipe(d, op, chunk, nst, &p);
    if (st != ZS_OK) return st;

    Totals T;
    auto issue = [&](PipeSlot &s, uint64_t off, uint64_t len) -> cudaError_t {
        s.busy = true;
        s.off = off;
        s.len = len;
        zs::DevResult *dr = reinterpret_cast<zs::DevResult *>(s.scratch);
        zs::TileState *tiles = reinterpret_cast<zs::TileState *>(dr + 1);
        const uint64_t ntiles = op == ZS_OP_COMPRESS ? zs::compress_scratch_tiles(d, len) : zs::decompress_tiles(len);
        cudaError_t e2 = cudaMemcpyAsync(s.d_in, h_in + off, len, cudaMemcpyHostToDevice, s.st);
        if (e2 == cudaSuccess)
            e2 = cudaMemsetAsync(s.scratch, 0, sizeof(zs::DevResult) + ntiles * sizeof(zs::TileState), s.st);
        if (e2 == cudaSuccess && s.out_pending) e2 = cudaStreamWaitEvent(s.st, s.out_ev, 0);
        s.out_pending = false;
        if (e2 == cudaSuccess)
            e2 = op == ZS_OP_COMPRESS
                     ? zs::launch_compress_any(d, s.d_in, len, flags, s.d_out, out_bound(d, op, len),
                                               h_index ? s.d_idx : nullptr, h_index ? len + 2 : 0, dr, tiles, s.slow,
                                               s.slow_cap, s.st)
                     : zs::launch_decompress_single(d, s.d_in, len, s.d_out, out_bound(d, op, len), dr, tiles, s.st);
        if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(s.h_res, dr, sizeof(zs::DevResult), cudaMemcpyDeviceToHost, s.st);
        if (e2 == cudaSuccess) e2 = cudaEventRecord(s.ev, s.st);
        return e2;
    };
    // Retires the slot's chunk: waits for its result, places its output and index.
    auto retire = [&](PipeSlot &s) -> cudaError_t {
        s.busy = false;
        cudaError_t e2 = cudaEventSynchronize(s.ev);
        if (e2 != cudaSuccess) return e2;
        zs::DevResult r = *s.h_res;
        if (op == ZS_OP_COMPRESS && (r.status & (zs::kStSlowOverflow | zs::kStFallback))) {
            // the long-line scratch of the slot was too small, or the chunk holds a line outside the span
            // kernel's fast path: code this chunk again through zs_compress, whose scratch grows as needed
            // and which runs the general kernel when the span kernel cannot
            zs_result rr{};
            const zs_status s2 = zs_compress(d, s.d_in, s.len, flags, s.d_out, out_bound(d, op, s.len),
                                             h_index ? s.d_idx : nullptr, h_index ? s.len + 2 : 0, &rr, s.st);
            if (s2 != ZS_OK && T.st == ZS_OK) {
                T.st = s2;
                T.msg = zs_last_error();
            }
            r = zs::DevResult{};
            r.out_len = rr.out_len;
            r.n_lines = rr.n_lines;
        }
        if (T.st == ZS_OK) {
            if (r.status & zs::kStTimeout) {
                T.st = ZS_ERR_TIMEOUT;
                T.msg = std::string(what) + ": a device-side wait expired";
            } else if (r.status & zs::kStTooBig) {
                T.st = ZS_ERR_INVALID_ARG;
                T.msg = std::string(what) + ": a line longer than 1 GiB";
            } else if (r.status & zs::kStMalformed) {
                T.st = ZS_ERR_MALFORMED;
                T.err_offset = s.off + ~r.err_key;
                T.msg = std::string(what) + ": malformed input at byte " + std::to_string(T.err_offset);
            }
        }
        // place the chunk (clipped to the caller's capacities; the totals still count everything), on the
        // copy-out stream; the slow-path recode above, if any, ran on the slot's stream, so order after it
        e2 = cudaEventRecord(s.ev, s.st);
        if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s.out_st, s.ev, 0);
        if (e2 == cudaSuccess && r.out_len && T.out < out_cap) {
            const uint64_t n = std::min<uint64_t>(r.out_len, out_cap - T.out);
            e2 = cudaMemcpyAsync(h_out + T.out, s.d_out, n, cudaMemcpyDeviceToHost, s.out_st);
        }
        if (e2 == cudaSuccess && op == ZS_OP_COMPRESS && h_index && r.n_lines && T.lines < index_cap) {
            const uint64_t n = std::min<uint64_t>(r.n_lines, index_cap - T.lines);
            if (T.out) {
                const unsigned blocks = (unsigned)std::min<uint64_t>((n + 255) / 256, 1024);
                rebase_kernel<<<blocks, 256, 0, s.out_st>>>(s.d_idx, n, T.out);
                e2 = cudaGetLastError();
            }
            if (e2 == cudaSuccess)
                e2 = cudaMemcpyAsync(h_index + T.lines, s.d_idx, n * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                                     s.out_st);
        }
        if (e2 == cudaSuccess) e2 = cudaEventRecord(s.out_ev, s.out_st);
        s.out_pending = e2 == cudaSuccess;
        T.out += r.out_len;
        T.lines += r.n_lines;
        return e2;
    };

    std::vector<int> order;  // slots in issue order
    uint64_t off = 0;
    size_t next = 0;
    e = cudaSuccess;
    while ((off < in_len || !order.empty()) && e == cudaSuccess) {
        // fill free slots
        while (off < in_len && (int)order.size() < nst && e == cudaSuccess) {
            const uint64_t end = chunk_end(h_in, in_len, off, chunk);
            if (end <= off) {  // a line longer than the chunk buffers: cannot be pipelined
                e = cudaErrorInvalidValue;
                T.st = ZS_ERR_CAPACITY;
                T.msg = std::string(what) + ": a line longer than the pipeline chunk (raise chunk_bytes)";
                break;
            }
            const int si = (int)(next++ % (size_t)nst);
            e = issue(p->slots[si], off, end - off);
            order.push_back(si);
            off = end;
        }
        if (order.empty() || e != cudaSuccess) break;
        const int si = order.front();
        order.erase(order.begin());
        e = retire(p->slots[si]);
    }
    for (PipeSlot &s : p->slots) {
        if (s.st) cudaStreamSynchronize(s.st);
        if (s.out_st) cudaStreamSynchronize(s.out_st);
        s.out_pending = false;
    }
    if (e != cudaSuccess && T.st == ZS_OK) return zs::cuda_fail(e, what);
    res->out_len = T.out;
    res->n_lines = T.lines;
    res->err_offset = T.err_offset;
    if (T.st != ZS_OK) {
        zs::set_error(T.msg);
        return T.st;
    }
    if (T.out > out_cap) {
        zs::set_error(std::string(what) + ": output buffer too small");
        return ZS_ERR_CAPACITY;
    }
    if (op == ZS_OP_COMPRESS && h_index) {
        if (T.lines + 1 > index_cap) {
            zs::set_error(std::string(what) + ": line index buffer too small");
            return ZS_ERR_CAPACITY;
        }
        h_index[T.lines] = T.out;
    }
    return ZS_OK;
}

}  // namespace

extern "C" zs_status zs_compress_host(const zs_dict *d, const uint8_t *h_in, size_t in_len, unsigned flags,
                                      uint8_t *h_out, size_t out_cap, uint64_t *h_index, size_t index_cap,
                                      zs_result *res, const zs_pipeline_options *opt)
{
    return run_pipeline(d, ZS_OP_COMPRESS, h_in, in_len, flags, h_out, out_cap, h_index, index_cap, res, opt,
                        "zs_compress_host");
}

extern "C" zs_status zs_decompress_host(const zs_dict *d, const uint8_t *h_in, size_t in_len, uint8_t *h_out,
                                        size_t out_cap, zs_result *res, const zs_pipeline_options *opt)
{
    return run_pipeline(d, ZS_OP_DECOMPRESS, h_in, in_len, 0, h_out, out_cap, nullptr, 0, res, opt,
                        "zs_decompress_host");
}
