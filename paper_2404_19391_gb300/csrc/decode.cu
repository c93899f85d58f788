// zs_decompress entry point, zs_build_line_index and zs_decompress_lines (random access, Sec. I). The
// decompression kernel itself is in decode_warp.cu.
#include <algorithm>

#include "zs_common.cuh"

namespace zs {
namespace {

// ------------------------------------------------------------------------------------------------
// Line index: newline ranks via warp-segmented 16-byte loads, a block scan and a warp-wide decoupled
// look-back, software-pipelined like the codec kernels:
//   - a CTA claims tile t+1 and issues its loads before it finishes tile t;
//   - it publishes a tile's aggregate as soon as the tile is scanned, but looks back for that tile only
//     after scanning the next one. By then the predecessors have had a whole tile's time to publish their
//     inclusive prefixes, so the walk back is short. Looking back at once would make every in-flight tile
//     walk back to the last finished one, 32 records per round trip.
// A tile's entries are staged in shared memory (two buffers, by rank within the tile) and written out as one
// contiguous run of coalesced 8-byte stores; a tile with more newlines than a buffer holds writes its entries
// directly.
// ------------------------------------------------------------------------------------------------
constexpr int kINT = 256;
constexpr int kIChunks = 8;                       // 16-byte chunks per lane: each warp 4 KiB = 8 x 512
constexpr int kIT = kINT / 32 * kIChunks * 512;   // bytes per tile (32 KiB)
constexpr uint32_t kIdxStage = 2048;              // staged index entries per tile and buffer (16 KiB)

struct IdxArgs {
    const uint8_t *in;
    uint64_t n;
    uint64_t *index;
    uint64_t index_cap;
    uint32_t in_aligned;
    uint64_t ntiles;
    DevResult *res;
    TileState *tiles;
    uint64_t limit_ns;
    int64_t stall_tile;
};

__device__ __forceinline__ uint32_t zero_bits4(uint32_t t)
{
    uint32_t z = ~(((t & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | t | 0x7F7F7F7Fu);
    return ((z >> 7) & 1u) | ((z >> 14) & 2u) | ((z >> 21) & 4u) | ((z >> 28) & 8u);
}

// The 16 bytes at p (bytes at or past n read as 0, which is no newline).
__device__ __forceinline__ uint4 load16(const uint8_t *in, uint64_t n, uint64_t p, bool aligned)
{
    if (aligned && p + 16 <= n) return __ldg(reinterpret_cast<const uint4 *>(in + p));
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    for (uint32_t q = 0; q < 16; ++q)
        if (p + q < n) w[q >> 2] |= (uint32_t)in[p + q] << (8 * (q & 3));
    return make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ uint32_t nl_bits16v(uint4 v)
{
    const uint32_t k = 0x0A0A0A0Au;
    return zero_bits4(v.x ^ k) | (zero_bits4(v.y ^ k) << 4) | (zero_bits4(v.z ^ k) << 8) |
           (zero_bits4(v.w ^ k) << 12);
}

__device__ __forceinline__ uint64_t tile_warp_base(uint64_t t, int warp)
{
    return t * (uint64_t)kIT + (uint64_t)warp * (kIChunks * 512u);
}

// Visits the newlines of a warp's part of a tile in byte order: f(rank, position after the newline), ranks
// counted from `rank` (the warp's first).
template <class F>
__device__ __forceinline__ void for_each_newline(const uint32_t *bits, uint64_t wbase, uint64_t rank, int lane, F f)
{
#pragma unroll
    for (int it = 0; it < kIChunks; ++it) {
        uint32_t b = bits[it];
        const uint32_t c = __popc(b);
        const uint32_t inc = warp_incl_u32(c);
        uint64_t rk = rank + inc - c;
        const uint64_t p0 = wbase + (uint64_t)it * 512u + (uint64_t)lane * 16u;
        while (b) {
            const int q = __ffs(b) - 1;
            b &= b - 1;
            f(rk, p0 + (uint64_t)q + 1u);
            ++rk;
        }
        rank += __shfl_sync(0xffffffffu, inc, 31);
    }
}

__global__ void __launch_bounds__(kINT) line_index_kernel(IdxArgs A)
{
    __shared__ uint64_t scan[2 * (kINT / 32 + 1)];
    __shared__ uint64_t s_tile, s_next, s_E;
    __shared__ uint64_t s_idx[2][kIdxStage];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool aligned = A.in_aligned != 0;
    uint32_t *status = &A.res->status;

    // the pending tile: scanned and its aggregate published, its look-back and writes still to do
    bool pending = false;
    uint64_t t_pend = 0, ta_pend = 0, wrank_pend = 0;
    uint32_t bits_pend[kIChunks];
    uint32_t buf = 0;
    auto finish = [&]() {  // looks back for the pending tile and writes its entries (whole block)
        const uint64_t tp = t_pend;
        if (warp == 0) {
            uint64_t ea = 0, eb = 0;
            if (tp > 0) lookback_warp(A.tiles, tp, &ea, &eb, A.limit_ns, status);
            if (lane == 0) {
                if (tp > 0 && (int64_t)tp != A.stall_tile) publish(&A.tiles[tp], 2u, ea + ta_pend, 0);
                s_E = ea;
                if (tp == 0 && A.index_cap > 0) A.index[0] = 0;
                if (tp == A.ntiles - 1) {
                    const uint64_t nl = ea + ta_pend;
                    const bool open_last = A.in[A.n - 1] != kNl;
                    const uint64_t lines = nl + (open_last ? 1u : 0u);
                    A.res->n_lines = lines;
                    if (open_last && lines < A.index_cap) A.index[lines] = A.n;
                }
            }
        }
        __syncthreads();
        const uint64_t E = s_E;
        if (ta_pend <= kIdxStage) {
            const uint64_t *src = s_idx[buf ^ 1u];
            for (uint32_t j = (uint32_t)tid; j < (uint32_t)ta_pend; j += kINT) {
                const uint64_t g = E + 1u + j;
                if (g < A.index_cap) A.index[g] = src[j];
            }
        } else {
            for_each_newline(bits_pend, tile_warp_base(tp, warp), E + wrank_pend, lane, [&](uint64_t rk, uint64_t v) {
                if (rk + 1 < A.index_cap) A.index[rk + 1] = v;
            });
        }
    };

    if (tid == 0) s_tile = atomicAdd(&A.res->tile_counter, 1ull);
    __syncthreads();
    uint64_t t = s_tile;
    uint4 v[kIChunks];
    if (t < A.ntiles) {
#pragma unroll
        for (int it = 0; it < kIChunks; ++it)
            v[it] = load16(A.in, A.n, tile_warp_base(t, warp) + (uint64_t)it * 512u + (uint64_t)lane * 16u, aligned);
    }
    while (t < A.ntiles) {
        uint32_t bits[kIChunks];
        uint32_t cnt = 0;
#pragma unroll
        for (int it = 0; it < kIChunks; ++it) {
            bits[it] = nl_bits16v(v[it]);
            cnt += __popc(bits[it]);
        }
        if (tid == 0) s_next = atomicAdd(&A.res->tile_counter, 1ull);
        uint64_t xa, xb, ta, tb;
        block_excl2_u64<kINT>(cnt, 0, scan, &xa, &xb, &ta, &tb);  // its barriers also publish s_next
        const uint64_t tn = s_next;
        if (tn < A.ntiles) {  // the next tile's reads, in flight while the pending tile looks back
#pragma unroll
            for (int it = 0; it < kIChunks; ++it)
                v[it] = load16(A.in, A.n, tile_warp_base(tn, warp) + (uint64_t)it * 512u + (uint64_t)lane * 16u,
                               aligned);
        }
        if (tid == 0 && (int64_t)t != A.stall_tile) publish(&A.tiles[t], t == 0 ? 2u : 1u, ta, 0);
        // each newline at p ends line k and starts line k+1 at p+1 (the last one marks the end)
        const uint64_t wrank = __shfl_sync(0xffffffffu, xa, 0);  // the warp's first rank within the tile
        if (ta <= kIdxStage) {  // the same for the whole block
            uint64_t *dst = s_idx[buf];
            for_each_newline(bits, tile_warp_base(t, warp), wrank, lane, [&](uint64_t rk, uint64_t v) {
                dst[rk] = v;
            });
        }
        if (pending) finish();
        __syncthreads();  // the written buffer and s_E are reused; s_next is rewritten
        pending = true;
        t_pend = t;
        ta_pend = ta;
        wrank_pend = wrank;
#pragma unroll
        for (int it = 0; it < kIChunks; ++it) bits_pend[it] = bits[it];
        buf ^= 1u;
        t = tn;
    }
    if (pending) {
        finish();
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------------
// Random access: one request per thread; decoded sizes, block scan + look-back over request tiles for
// the output offsets, then each thread decodes its line into a shared-memory stage at its offset within
// the tile, and the block writes the stage out as one contiguous run (coalesced); a tile whose lines
// decode to more than the stage holds writes them directly.
// ------------------------------------------------------------------------------------------------
constexpr int kRNT = 256;
constexpr uint32_t kRStage = 16384;  // staged decoded bytes per tile of requests

struct LinesArgs {
    const uint8_t *comp;
    uint64_t comp_len;
    uint32_t comp_aligned;  // comp is 4-byte aligned
    const uint64_t *index;
    uint64_t n_lines;
    const uint64_t *ids;
    uint64_t k;
    uint8_t *out;
    uint64_t out_cap;
    uint64_t *out_off;
    uint64_t ntiles;
    const uint8_t *dec;
    DevResult *res;
    TileState *tiles;
    uint64_t limit_ns;
    int64_t stall_tile;
};

// Calls f(c) for the bytes comp[a, b) in order, reading whole aligned 4-byte words where they lie inside
// [a, b) (so inside the buffer) and single bytes at the ends.
template <class F>
__device__ __forceinline__ void for_each_byte(const uint8_t *comp, uint64_t a, uint64_t b, bool aligned, F f)
{
    uint64_t p = a;
    if (aligned) {
        for (; p < b && (p & 3u); ++p) f((uint32_t)comp[p]);
#pragma unroll 4
        for (; p + 4 <= b; p += 4) {
            const uint32_t w = __ldg(reinterpret_cast<const uint32_t *>(comp + p));
            f(w & 255u);
            f((w >> 8) & 255u);
            f((w >> 16) & 255u);
            f(w >> 24);
        }
    }
    for (; p < b; ++p) f((uint32_t)comp[p]);
}

__global__ void __launch_bounds__(kRNT) lines_kernel(LinesArgs A)
{
    __shared__ __align__(16) uint8_t dec[kDecBytes];
    __shared__ __align__(16) uint8_t s_out[kRStage];
    __shared__ uint64_t scan[2 * (kRNT / 32 + 1)];
    __shared__ uint64_t s_tile, s_E;
    const int tid = threadIdx.x;
    uint32_t *status = &A.res->status;
    for (uint32_t j = tid; j < kDecBytes / 16; j += kRNT)
        reinterpret_cast<uint4 *>(dec)[j] = __ldg(reinterpret_cast<const uint4 *>(A.dec) + j);
    __syncthreads();
    const uint8_t *plen = dec;
    const uint8_t *pat = dec + 256;
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(&A.res->tile_counter, 1ull);
        __syncthreads();
        const uint64_t t = s_tile;
        if (t >= A.ntiles) break;
        const uint64_t r = t * (uint64_t)kRNT + (uint64_t)tid;
        uint64_t a = 0, b = 0, olen = 0;
        bool ok = false;
        if (r < A.k) {
            const uint64_t id = A.ids[r];
            ok = id < A.n_lines;
            if (ok) {
                a = A.index[id];
                b = A.index[id + 1];
                ok = a <= b && b <= A.comp_len;
            }
            if (ok && b > a && A.comp[b - 1] == kNl) --b;
            bool lit = false;
            if (ok) {
                for_each_byte(A.comp, a, b, A.comp_aligned != 0, [&](uint32_t c) {
                    if (lit) {
                        olen += 1;
                        lit = false;
                    } else if (c == kEsc) {
                        lit = true;
                    } else {
                        const uint32_t l = plen[c];
                        if (l == 0) ok = false;  // unknown symbol or a '\n' inside the line
                        olen += l;
                    }
                });
            }
            if (lit) ok = false;
            if (!ok) {
                note_error_offset(A.res, r);
                atomicOr(status, kStMalformed);
                olen = 0;
            } else {
                olen += 1;  // '\n'
            }
        }
        uint64_t xa, xb, ta, tb;
        block_excl2_u64<kRNT>(olen, 0, scan, &xa, &xb, &ta, &tb);
        if (tid < 32) {  // warp 0: publish, then look back 32 predecessors per round trip
            const bool stall = (int64_t)t == A.stall_tile;
            if (tid == 0 && !stall) publish(&A.tiles[t], t == 0 ? 2u : 1u, ta, 0);
            uint64_t ea = 0, eb = 0;
            if (t > 0) lookback_warp(A.tiles, t, &ea, &eb, A.limit_ns, status);
            if (tid == 0) {
                if (t > 0 && !stall) publish(&A.tiles[t], 2u, ea + ta, 0);
                s_E = ea;
                if (t == A.ntiles - 1) {
                    A.res->out_len = ea + ta;
                    A.out_off[A.k] = ea + ta;
                }
            }
        }
        __syncthreads();
        const uint64_t E = s_E;
        const bool staged = ta <= kRStage;  // the same for the whole block
        if (r < A.k) {
            A.out_off[r] = E + xa;
            if (ok) {
                // staged: bytes go to s_out at the line's offset within the tile; else straight to the output
                uint64_t pos = staged ? xa : E + xa;
                auto put = [&](uint8_t v) {
                    if (staged) s_out[pos] = v;
                    else if (pos < A.out_cap) A.out[pos] = v;
                    ++pos;
                };
                bool lit = false;
                for_each_byte(A.comp, a, b, A.comp_aligned != 0, [&](uint32_t c) {
                    if (!lit && c == kEsc) {
                        lit = true;
                        return;
                    }
                    if (lit) {
                        put((uint8_t)c);
                        lit = false;
                        return;
                    }
                    const uint32_t l = plen[c];
                    const uint8_t *src = pat + 16u * c;
                    for (uint32_t q = 0; q < l; ++q) put(src[q]);
                });
                put(kNl);
            }
        }
        if (staged) {
            __syncthreads();
            for (uint32_t j = (uint32_t)tid; j < (uint32_t)ta; j += kRNT) {
                const uint64_t g = E + j;
                if (g < A.out_cap) A.out[g] = s_out[j];
            }
        }
        __syncthreads();
    }
}

int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

template <class K>
int blocks_per_sm(K kernel, int nt, int smem)
{
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, nt, smem);
    return nb > 0 ? nb : 1;
}

}  // namespace

uint64_t index_tiles(uint64_t n) { return (n + kIT - 1) / kIT; }
uint64_t lines_tiles(uint64_t k) { return (k + kRNT - 1) / kRNT; }

cudaError_t launch_line_index(const uint8_t *in, uint64_t n, uint64_t *index, uint64_t index_cap, DevResult *res,
                              TileState *tiles, cudaStream_t s)
{
    IdxArgs a{};
    a.in = in;
    a.n = n;
    a.index = index;
    a.index_cap = index_cap;
    a.in_aligned = (((uintptr_t)in) & 15u) == 0;
    a.ntiles = index_tiles(n);
    a.res = res;
    a.tiles = tiles;
    a.limit_ns = wait_limit_ns();
    a.stall_tile = injected_stall_tile();
    static int per = -1;
    if (per < 0) per = blocks_per_sm(line_index_kernel, kINT, 0);
    const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(a.ntiles, (uint64_t)per * sm_count()));
    line_index_kernel<<<(unsigned)grid, kINT, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_lines(const zs_dict *d, const uint8_t *comp, uint64_t comp_len, const uint64_t *index,
                         uint64_t n_lines, const uint64_t *ids, uint64_t k, uint8_t *out, uint64_t out_cap,
                         uint64_t *out_off, DevResult *res, TileState *tiles, cudaStream_t s)
{
    LinesArgs a{};
    a.comp = comp;
    a.comp_len = comp_len;
    a.comp_aligned = (((uintptr_t)comp) & 3u) == 0;
    a.index = index;
    a.n_lines = n_lines;
    a.ids = ids;
    a.k = k;
    a.out = out;
    a.out_cap = out_cap;
    a.out_off = out_off;
    a.ntiles = lines_tiles(k);
    a.dec = d->d_dec;
    a.res = res;
    a.tiles = tiles;
    a.limit_ns = wait_limit_ns();
    a.stall_tile = injected_stall_tile();
    static int per = -1;
    if (per < 0) per = blocks_per_sm(lines_kernel, kRNT, 0);
    const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(a.ntiles, (uint64_t)per * sm_count()));
    lines_kernel<<<(unsigned)grid, kRNT, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace zs

namespace {

zs_status check_dict_device(const zs_dict *d, const char *what)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return zs::cuda_fail(e, what);
    if (dev != d->device) {
        zs::set_error(std::string(what) + ": dictionary was loaded on another device");
        return ZS_ERR_INVALID_ARG;
    }
    return ZS_OK;
}

// Zero the call's scratch, run `launch`, read the result back. *r receives the device result.
template <class F>
zs_status run(zs::ScratchPool &pool, void *stream, uint64_t ntiles, const char *what, F launch, zs::DevResult *r)
{
    zs::Scratch *sc = nullptr;
    zs_status st = pool.get(stream, ntiles, 0, &sc);
    if (st != ZS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    zs::DevResult *dr = reinterpret_cast<zs::DevResult *>(sc->dev);
    zs::TileState *tiles = reinterpret_cast<zs::TileState *>(dr + 1);
    cudaError_t e = cudaMemsetAsync(sc->dev, 0, sizeof(zs::DevResult) + ntiles * sizeof(zs::TileState), s);
    if (e == cudaSuccess) {
        zs::mark_kernel_start(sc, s);
        e = launch(dr, tiles, s);
        zs::mark_kernel_end(sc, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc->host, dr, sizeof(zs::DevResult), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return zs::cuda_fail(e, what);
    *r = *sc->host;
    zs::note_kernel_time(sc);
    if (r->status & zs::kStTimeout) {
        zs::set_error(std::string(what) + ": a device-side wait expired");
        return ZS_ERR_TIMEOUT;
    }
    return ZS_OK;
}

}  // namespace

extern "C" zs_status zs_decompress(const zs_dict *d, const uint8_t *d_in, size_t in_len, uint8_t *d_out,
                                   size_t out_cap, zs_result *res, void *stream)
{
    zs::clear_error();
    if (!d || !res || (!d_in && in_len) || (!d_out && out_cap)) {
        zs::set_error("zs_decompress: NULL argument");
        return ZS_ERR_INVALID_ARG;
    }
    zs_status st = check_dict_device(d, "zs_decompress");
    if (st != ZS_OK) return st;
    res->out_len = res->n_lines = res->err_offset = 0;
    if (in_len == 0) return ZS_OK;
    zs::DevResult r{};
    st = run(const_cast<zs_dict *>(d)->pool, stream, zs::decompress_tiles(in_len), "zs_decompress",
             [&](zs::DevResult *dr, zs::TileState *tiles, cudaStream_t s) {
                 return zs::launch_decompress_single(d, d_in, in_len, d_out, out_cap, dr, tiles, s);
             },
             &r);
    if (st != ZS_OK) return st;
    res->out_len = r.out_len;
    res->n_lines = r.n_lines;
    if (r.status & zs::kStMalformed) {
        res->err_offset = ~r.err_key;
        zs::set_error("zs_decompress: malformed input at byte " + std::to_string(res->err_offset));
        return ZS_ERR_MALFORMED;
    }
    if (r.out_len > out_cap) {
        zs::set_error("zs_decompress: output buffer too small");
        return ZS_ERR_CAPACITY;
    }
    return ZS_OK;
}

extern "C" zs_status zs_build_line_index(const uint8_t *d_in, size_t in_len, uint64_t *d_index, size_t index_cap,
                                         size_t *n_lines, void *stream)
{
    zs::clear_error();
    if (!n_lines || (!d_in && in_len) || (!d_index && index_cap)) {
        zs::set_error("zs_build_line_index: NULL argument");
        return ZS_ERR_INVALID_ARG;
    }
    *n_lines = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (in_len == 0) {
        if (index_cap < 1) {
            zs::set_error("zs_build_line_index: index buffer too small");
            return ZS_ERR_CAPACITY;
        }
        cudaError_t e = cudaMemsetAsync(d_index, 0, sizeof(uint64_t), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return e == cudaSuccess ? ZS_OK : zs::cuda_fail(e, "zs_build_line_index");
    }
    zs::DevResult r{};
    zs_status st = run(zs::global_pool(), stream, zs::index_tiles(in_len), "zs_build_line_index",
                       [&](zs::DevResult *dr, zs::TileState *tiles, cudaStream_t s2) {
                           return zs::launch_line_index(d_in, in_len, d_index, index_cap, dr, tiles, s2);
                       },
                       &r);
    if (st != ZS_OK) return st;
    *n_lines = r.n_lines;
    if (r.n_lines + 1 > index_cap) {
        zs::set_error("zs_build_line_index: index buffer too small");
        return ZS_ERR_CAPACITY;
    }
    return ZS_OK;
}

extern "C" zs_status zs_decompress_lines(const zs_dict *d, const uint8_t *d_comp, size_t comp_len,
                                         const uint64_t *d_index, size_t n_lines, const uint64_t *d_ids, size_t k,
                                         uint8_t *d_out, size_t out_cap, uint64_t *d_out_off, zs_result *res,
                                         void *stream)
{
    zs::clear_error();
    if (!d || !res || !d_out_off || (!d_comp && comp_len) || !d_index || (!d_ids && k) || (!d_out && out_cap)) {
        zs::set_error("zs_decompress_lines: NULL argument");
        return ZS_ERR_INVALID_ARG;
    }
    zs_status st = check_dict_device(d, "zs_decompress_lines");
    if (st != ZS_OK) return st;
    res->out_len = res->n_lines = res->err_offset = 0;
    if (k == 0) {
        cudaError_t e = cudaMemsetAsync(d_out_off, 0, sizeof(uint64_t), (cudaStream_t)stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
        return e == cudaSuccess ? ZS_OK : zs::cuda_fail(e, "zs_decompress_lines");
    }
    zs::DevResult r{};
    st = run(const_cast<zs_dict *>(d)->pool, stream, zs::lines_tiles(k), "zs_decompress_lines",
             [&](zs::DevResult *dr, zs::TileState *tiles, cudaStream_t s) {
                 return zs::launch_lines(d, d_comp, comp_len, d_index, n_lines, d_ids, k, d_out, out_cap, d_out_off,
                                         dr, tiles, s);
             },
             &r);
    if (st != ZS_OK) return st;
    res->out_len = r.out_len;
    res->n_lines = k;
    if (r.status & zs::kStMalformed) {
        res->err_offset = ~r.err_key;
        zs::set_error("zs_decompress_lines: bad request at position " + std::to_string(res->err_offset));
        return ZS_ERR_MALFORMED;
    }
    if (r.out_len > out_cap) {
        zs::set_error("zs_decompress_lines: output buffer too small");
        return ZS_ERR_CAPACITY;
    }
    return ZS_OK;
}
