// zs_decompress (Sec. IV-D2) with one warp per tile of compressed input (default 2176 bytes).
//
//   - Each warp of a persistent CTA claims tiles in launch order, stages its tile with one bulk (TMA)
//     copy and works on it alone: no CTA-wide barrier is on the per-tile path.
//   - Escapes without a sequential scan: a byte is verbatim exactly when the run of ' ' bytes just before
//     it has odd length (every unescaped ' ' escapes the byte after it, and a run always starts
//     unescaped), so each lane decodes its own slice (default 68 bytes) after counting the spaces in front of it
//     (an odd number of words per slice keeps the lanes' shared-memory reads on distinct banks).
//   - Small tiles and 20-32 warps per SM (22 by default): the per-lane loops are chains of dependent
//     shared-memory loads, so the kernel is bound by latency, and the warp count is what hides it.
//   - Sizes phase: per lane, the decoded size of its slice (pattern lengths from a shared table), then a
//     warp scan; the tile's aggregate is published for the decoupled look-back.
//   - Software pipeline: the warp computes the sizes of tile k+1 before it resolves tile k's output
//     offset (warp-wide look-back, 32 predecessors per round trip) and emits it, so predecessors have
//     long published by then.
//   - Emission: each lane expands its slice into a per-warp staging buffer aligned to the output's
//     16-byte grid, which is written with coalesced 16-byte stores (direct stores when a tile expands
//     past the buffer).
#include <algorithm>

#include "zs_common.cuh"

namespace zs {
namespace {

// Geometry of one compiled variant: warps per CTA and compressed bytes per lane slice (an odd number of
// 4-byte words, so lane l's word w sits in a bank of its own).
template <int W, int LANE, int OUTQ>
struct DwGeom {
    static constexpr int kWarps = W;
    static constexpr int kLane = LANE;
    static constexpr int kOutQ = OUTQ;  // staged output bytes per tile, in quarters of the tile's input bytes
};

constexpr unsigned kFullD = 0xffffffffu;

// Launch-wide arguments; the per-shard ones are in the ShardView of each claimed tile.
struct DwArgs {
    ShardView one;            // the shard when n_shards == 1
    const ShardView *shards;  // device shard table when n_shards > 1
    uint32_t n_shards;
    uint32_t _pad;
    uint64_t total_tiles;
    const uint8_t *dec;  // plen[256], pat[256][16]
    DevResult *g;        // tile counter and status bits
    uint64_t limit_ns;
    int64_t stall_tile;
};

// NARROW: every pattern is at most 7 bytes, so a pattern and its length fit one 64-bit table entry and
// the word-wise paths below apply; otherwise the byte loops run.
template <class Geo, bool NARROW>
struct DW {
    static constexpr int kDW = Geo::kWarps;
    static constexpr int kDNTW = 32 * kDW;
    static constexpr int kDLane = Geo::kLane;
    static constexpr int kDTile = 32 * kDLane;                  // compressed bytes per warp tile
    static constexpr int kDOut = (kDTile * Geo::kOutQ / 4 + 255) & ~255;  // staged output bytes per tile
    static_assert(kDLane % 8 == 4, "lane slices must be an odd number of 4-byte words and 16-byte tiles");

    struct alignas(16) DSlot {
        uint8_t in[kDTile + 16];
        uint32_t lane_off[32];  // output offset of each lane's slice within the tile
        uint8_t lit0[32];       // each lane's slice starts with an escaped byte
        uint64_t bar;
        uint64_t total;         // decoded bytes of the tile
        uint32_t nown, nls;     // owned bytes, newlines decoded
        ShardView sv;           // the shard of the staged tile
    };

    struct alignas(16) DWarpMem {
        DSlot slot[2];
        uint8_t ost[kDOut + 32];
    };

    struct DCtx {
        const DwArgs *P;
        const ShardView *A;
        DWarpMem *M;
        const uint8_t *plen;
        const uint8_t *pat;
        const uint32_t *szt;  // NARROW: decoded size per byte ('\n': 1, ' ': 0, not a symbol: 1 << 16)
        const uint64_t *pat8;  // NARROW: pattern bytes, length in byte 7 ('\n' -> "\n")
        uint32_t lane;
        uint32_t *status;
    };
    static constexpr uint32_t kBad = 1u << 16;  // szt entry of a byte that is no symbol

    static __device__ __forceinline__ void stage_d(const DCtx &C, DSlot &S, uint64_t t)
    {
        const ShardView &A = *C.A;
        const uint64_t base = t * (uint64_t)kDTile;
        const uint32_t nown = (uint32_t)(min(A.n, base + kDTile) - base);
        const uint32_t nbulk = A.in_aligned ? (nown & ~15u) : 0u;
        __syncwarp();
        if (C.lane == 0) {
            fence_proxy_async_smem();
            mbar_arrive_tx(&S.bar, nbulk);
            if (nbulk) bulk_g2s(S.in, A.in + base, nbulk, &S.bar);
            S.nown = nown;
        }
        for (uint32_t j = nbulk + C.lane; j < nown; j += 32) S.in[j] = A.in[base + j];
    }

    // Byte loop over the slice [p0, p1): decoded bytes and newlines, noting malformed bytes.
    static __device__ __forceinline__ void slice_bytes(const DCtx &C, const DSlot &S, uint64_t base, uint32_t p0,
                                                       uint32_t p1, bool lit, uint32_t *outb_, uint32_t *nls_,
                                                       bool *lit_end)
    {
        const ShardView &A = *C.A;
        uint32_t outb = 0, nls = 0;
        for (uint32_t p = p0; p < p1; ++p) {
            const uint8_t b = S.in[p];
            if (lit) {
                if (b == kNl) {  // a line ending in an unpaired escape
                    note_error_offset(A.res, base + p - 1);
                    atomicOr(C.status, kStMalformed);
                }
                outb += 1;
                nls += (b == kNl);
                lit = false;
            } else if (b == kEsc) {
                lit = true;
            } else if (b == kNl) {
                outb += 1;
                nls += 1;
            } else {
                const uint32_t l = C.plen[b];
                if (l == 0) {
                    note_error_offset(A.res, base + p);
                    atomicOr(C.status, kStMalformed);
                }
                outb += l;
            }
        }
        *outb_ = outb;
        *nls_ = nls;
        *lit_end = lit;
    }

    // The same sizes a 4-byte word at a time: four table lookups per word without a space; words with a
    // space (or after an escaping one) go byte by byte. Returns false if the slice holds a malformed byte
    // (the caller then reruns the byte loop, which notes where).
    static __device__ __forceinline__ bool slice_words(const DCtx &C, const DSlot &S, uint32_t p0, uint32_t p1,
                                                       bool lit, uint32_t *outb_, uint32_t *nls_, bool *lit_end)
    {
        const uint32_t *szt = C.szt;
        uint32_t acc = 0, nls = 0;
        bool bad = false;
        auto one = [&](uint32_t b) {
            if (lit) {
                bad |= (b == kNl);
                acc += 1;
                lit = false;
            } else if (b == kEsc) {
                lit = true;
            } else {
                acc += szt[b];
            }
            nls += (b == kNl);
        };
        uint32_t p = p0;
        const uint32_t pw = p0 + ((p1 - p0) & ~3u);
        for (; p < pw; p += 4) {
            const uint32_t w = *reinterpret_cast<const uint32_t *>(S.in + p);
            if (lit || __vcmpeq4(w, 0x20202020u)) {
#pragma unroll
                for (int j = 0; j < 4; ++j) one((w >> (8 * j)) & 255u);
                continue;
            }
            acc += szt[w & 255u] + szt[(w >> 8) & 255u] + szt[(w >> 16) & 255u] + szt[w >> 24];
            nls += __popc(__vcmpeq4(w, 0x0A0A0A0Au)) >> 3;
        }
        for (; p < p1; ++p) one(S.in[p]);
        *outb_ = acc & 0xFFFFu;
        *nls_ = nls;
        *lit_end = lit;
        return !bad && (acc >> 16) == 0;
    }

    // Decoded size of each lane's slice, warp scan, publication of the tile's aggregate.
    static __device__ __forceinline__ void sizes_d(const DCtx &C, DSlot &S, uint64_t t)
    {
        const ShardView &A = *C.A;
        const uint32_t lane = C.lane;
        const uint64_t base = t * (uint64_t)kDTile;
        const uint32_t nown = S.nown;
        uint32_t carry = 0;  // spaces immediately before the tile
        if (lane == 0)
            while (base > carry && A.in[base - 1 - carry] == kEsc) ++carry;
        carry = __shfl_sync(kFullD, carry, 0);
        const uint32_t p0 = min(nown, lane * (uint32_t)kDLane);
        const uint32_t p1 = min(nown, p0 + (uint32_t)kDLane);
        uint32_t run = 0;
        {
            int q = (int)p0 - 1;
            while (q >= 0 && S.in[q] == kEsc) {
                ++run;
                --q;
            }
            if (q < 0) run += carry;
        }
        const bool lit_start = (run & 1u) != 0;
        uint32_t outb = 0, nls = 0;
        bool lit = false;
        if (!NARROW || !slice_words(C, S, p0, p1, lit_start, &outb, &nls, &lit))
            slice_bytes(C, S, base, p0, p1, lit_start, &outb, &nls, &lit);
        if (lit && p1 > p0 && base + p1 == A.n) {  // the stream ends in an unpaired escape
            note_error_offset(A.res, A.n - 1);
            atomicOr(C.status, kStMalformed);
        }
        uint32_t inc = warp_incl_u32(outb);
        uint32_t incn = warp_incl_u32(nls);
        const uint32_t total = __shfl_sync(kFullD, inc, 31);
        const uint32_t totn = __shfl_sync(kFullD, incn, 31);
        S.lane_off[lane] = inc - outb;
        S.lit0[lane] = lit_start ? 1 : 0;
        if (lane == 0) {
            S.total = total;
            S.nls = totn;
            if ((int64_t)t != C.P->stall_tile) publish(&A.tiles[t], t == 0 ? 2u : 1u, total, totn);
        }
        __syncwarp();
    }

    // Word-wise expansion into the staging buffer (NARROW). Each lane funnels its pattern bytes into
    // aligned 32-bit stores. Its first word may start below its own first byte: those low bytes are
    // written as zeros, and belong to an earlier lane's last, partial word, which every lane writes byte
    // by byte only after the whole warp's word stores (the caller's second phase, expand_tail).
    struct Funnel {
        uint32_t a, n, wpos, head, pos0;
    };

    static __device__ __forceinline__ void expand_words(const DCtx &C, const DSlot &S, uint32_t p0, uint32_t p1,
                                                        bool lit, uint32_t pos, Funnel &F)
    {
        uint8_t *ost = C.M->ost;
        const uint64_t *pat8 = C.pat8;
        uint32_t a = 0, n = pos & 3u, wpos = pos & ~3u;
        auto push = [&](uint32_t lo, uint32_t hi, uint32_t l) {
            const uint32_t sh = 8u * n;
            const uint32_t w0 = a | (lo << sh);
            const uint32_t w1 = __funnelshift_l(lo, hi, sh);
            const uint32_t w2 = __funnelshift_l(hi, 0u, sh);
            const uint32_t tot = n + l;
            if (tot >= 4) *reinterpret_cast<uint32_t *>(ost + wpos) = w0;
            if (tot >= 8) *reinterpret_cast<uint32_t *>(ost + wpos + 4) = w1;
            const uint32_t k = tot >> 2;
            a = k == 0 ? w0 : (k == 1 ? w1 : w2);
            n = tot & 3u;
            wpos += 4u * k;
        };
        auto sym = [&](uint32_t b) {
            const uint64_t e = pat8[b];
            push((uint32_t)e, (uint32_t)(e >> 32) & 0x00FFFFFFu, (uint32_t)(e >> 56));
        };
        auto one = [&](uint32_t b) {
            if (lit) {
                push(b, 0u, 1u);
                lit = false;
            } else if (b == kEsc) {
                lit = true;
            } else {
                sym(b);
            }
        };
        uint32_t p = p0;
        const uint32_t pw = p0 + ((p1 - p0) & ~3u);
        for (; p < pw; p += 4) {
            const uint32_t w = *reinterpret_cast<const uint32_t *>(S.in + p);
            if (lit || __vcmpeq4(w, 0x20202020u)) {
#pragma unroll
                for (int j = 0; j < 4; ++j) one((w >> (8 * j)) & 255u);
                continue;
            }
            sym(w & 255u);
            sym((w >> 8) & 255u);
            sym((w >> 16) & 255u);
            sym(w >> 24);
        }
        for (; p < p1; ++p) one(S.in[p]);
        F.a = a;
        F.n = n;
        F.wpos = wpos;
        F.head = pos & 3u;
        F.pos0 = pos & ~3u;
    }

    // Second phase: the lane's last, partial word, byte by byte (never below its own first byte).
    static __device__ __forceinline__ void expand_tail(const DCtx &C, const Funnel &F)
    {
        uint8_t *ost = C.M->ost;
        const uint32_t j0 = F.wpos == F.pos0 ? F.head : 0u;
        for (uint32_t j = j0; j < F.n; ++j) ost[F.wpos + j] = (uint8_t)(F.a >> (8 * j));
    }

    template <bool STAGED>
    static __device__ __forceinline__ void expand_slice(const DCtx &C, const DSlot &S, uint32_t p0, uint32_t p1, bool lit,
                                                 uint64_t pos, uint64_t E_a, uint32_t so)
    {
        const ShardView &A = *C.A;
        uint8_t *ost = C.M->ost;
        for (uint32_t p = p0; p < p1; ++p) {
            const uint8_t b = S.in[p];
            if (!lit && b == kEsc) {
                lit = true;
                continue;
            }
            if (lit || b == kNl) {
                lit = false;
                if (STAGED) ost[so + pos] = b;
                else if (E_a + pos < A.out_cap) A.out[E_a + pos] = b;
                pos += 1;
                continue;
            }
            const uint32_t l = C.plen[b];
            const uint8_t *src = C.pat + 16u * b;
            if (STAGED) {
                uint8_t *d = ost + so + pos;
                for (uint32_t k = 0; k < l; ++k) d[k] = src[k];
            } else {
                for (uint32_t k = 0; k < l; ++k)
                    if (E_a + pos + k < A.out_cap) A.out[E_a + pos + k] = src[k];
            }
            pos += l;
        }
    }

    // Resolve the tile's output offset and write its decoded bytes.
    static __device__ void finish_d(const DCtx &C, DSlot &S, uint64_t t)
    {
        const ShardView &A = *C.A;
        const uint32_t lane = C.lane;
        uint64_t ea = 0, eb = 0;
        if (t > 0) lookback_warp(A.tiles, t, &ea, &eb, C.P->limit_ns, C.status);
        const uint64_t total = S.total;
        const uint32_t totn = S.nls;
        if (lane == 0 && t > 0 && (int64_t)t != C.P->stall_tile) publish(&A.tiles[t], 2u, ea + total, eb + totn);
        const uint32_t so = (uint32_t)(((uint64_t)(uintptr_t)A.out + ea) & 15u);
        const bool staged = total + 32 <= (uint64_t)kDOut;
        const uint32_t nown = S.nown;
        const uint32_t p0 = min(nown, lane * (uint32_t)kDLane);
        const uint32_t p1 = min(nown, p0 + (uint32_t)kDLane);
        if (NARROW && staged) {
            Funnel F;
            expand_words(C, S, p0, p1, S.lit0[lane] != 0, so + S.lane_off[lane], F);
            __syncwarp();
            expand_tail(C, F);
        } else if (staged) {
            expand_slice<true>(C, S, p0, p1, S.lit0[lane] != 0, S.lane_off[lane], ea, so);
        } else {
            expand_slice<false>(C, S, p0, p1, S.lit0[lane] != 0, S.lane_off[lane], ea, so);
        }
        __syncwarp();
        if (staged) warp_copy_out(C.M->ost, so, total, A.out + ea, A.out_cap > ea ? A.out_cap - ea : 0);
        if (lane == 0 && t == A.ntiles - 1) {
            A.res->out_len = ea + total;
            A.res->n_lines = eb + totn + ((A.in[A.n - 1] != kNl) ? 1u : 0u);
        }
        __syncwarp();
    }

    static __device__ void run(const DwArgs *P)
    {
        extern __shared__ __align__(128) uint8_t smem[];
        __shared__ uint64_t tab_bar;
        const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        DWarpMem &M = reinterpret_cast<DWarpMem *>(smem)[wid];
        uint8_t *tab = smem + kDW * sizeof(DWarpMem);
        DCtx C;
        C.P = P;
        C.A = nullptr;
        C.M = &M;
        C.plen = tab;
        C.pat = tab + 256;
        C.szt = reinterpret_cast<const uint32_t *>(tab + kDecBytes);
        C.pat8 = reinterpret_cast<const uint64_t *>(tab + kDecBytes + 1024);
        C.lane = lane;
        C.status = &P->g->status;
        if (threadIdx.x == 0) mbar_init(&tab_bar, 1);
        if (lane == 0) {
            mbar_init(&M.slot[0].bar, 1);
            mbar_init(&M.slot[1].bar, 1);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_arrive_tx(&tab_bar, kDecBytes);
            bulk_g2s(tab, P->dec, kDecBytes, &tab_bar);
        }
        const bool staged_ok = mbar_wait_bounded(&tab_bar, 0, P->limit_ns, C.status);
        if (!__syncthreads_and(staged_ok)) {
            mbar_wait_bounded(&tab_bar, 0, P->limit_ns, C.status);
            return;
        }
        if (NARROW) {  // word-path tables, built from the staged plen / pat tables
            uint32_t *szt = reinterpret_cast<uint32_t *>(tab + kDecBytes);
            uint64_t *pat8 = reinterpret_cast<uint64_t *>(tab + kDecBytes + 1024);
            for (uint32_t b = threadIdx.x; b < 256; b += blockDim.x) {
                const uint32_t l = tab[b];
                uint64_t e = 0;
                if (b == kNl) {
                    e = (uint64_t)kNl | (1ull << 56);
                } else if (l) {
                    for (uint32_t k = 0; k < l; ++k) e |= (uint64_t)tab[256 + 16 * b + k] << (8 * k);
                    e |= (uint64_t)l << 56;
                }
                szt[b] = b == kNl ? 1u : (l ? l : kBad);
                pat8[b] = e;
            }
            __syncthreads();
        }
        uint32_t ph = 0, s = 0;
        bool pending = false;
        uint64_t t_pend = 0;
        auto finish_pending = [&]() {
            DCtx Cp = C;
            Cp.A = &M.slot[s ^ 1u].sv;
            finish_d(Cp, M.slot[s ^ 1u], t_pend);
        };
        for (;;) {
            unsigned long long tt = 0;
            if (lane == 0) tt = atomicAdd(&P->g->tile_counter, 1ull);
            const uint64_t g = __shfl_sync(kFullD, tt, 0);
            if (g >= P->total_tiles) break;
            DSlot &S = M.slot[s];
            const uint32_t sh = P->n_shards == 1 ? 0u : find_shard(P->shards, P->n_shards, g);
            load_shard(&S.sv, P->one, P->shards, P->n_shards, sh);
            const uint64_t t = g - S.sv.tile0;  // tile number within the shard
            DCtx Cs = C;
            Cs.A = &S.sv;
            stage_d(Cs, S, t);
            if (!mbar_wait_bounded(&S.bar, (ph >> s) & 1u, P->limit_ns, C.status)) {
                mbar_wait_bounded(&S.bar, (ph >> s) & 1u, P->limit_ns, C.status);
                return;
            }
            ph ^= 1u << s;
            __syncwarp();
            sizes_d(Cs, S, t);
            if (pending) finish_pending();
            pending = true;
            t_pend = t;
            s ^= 1u;
        }
        if (pending) finish_pending();
    }
};

template <class Geo, bool NARROW>
__global__ void __launch_bounds__(Geo::kWarps * 32, 1) decompress_warp_kernel(const DwArgs P)
{
    DW<Geo, NARROW>::run(&P);
}

// Compiled geometries; variant 0 is the default: 22 warps, the output of a tile staged in 2.25 x its input
// bytes (a tile that expands more stores directly). Variant 1 is the same tile with 20 warps and 2.5 x for
// dictionaries that expand more; variants 2 and 3 hold smaller tiles with more warps.
using DwV0 = DwGeom<22, 68, 9>;
using DwV1 = DwGeom<20, 68, 10>;
using DwV2 = DwGeom<28, 52, 9>;
using DwV3 = DwGeom<32, 36, 10>;

template <class Geo, bool NARROW>
cudaError_t dw_launch_as(const DwArgs &a, uint64_t total_tiles, cudaStream_t s)
{
    using K = DW<Geo, NARROW>;
    const int smem = (int)(K::kDW * sizeof(typename K::DWarpMem) + kDecBytes + (NARROW ? 3072 : 0));
    static int per = -1;
    if (per < 0) {
        cudaError_t e = cudaFuncSetAttribute(decompress_warp_kernel<Geo, NARROW>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, decompress_warp_kernel<Geo, NARROW>, K::kDNTW, smem);
        if (per < 1) per = 1;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t grid = std::max<uint64_t>(
        1, std::min<uint64_t>((total_tiles + Geo::kWarps - 1) / Geo::kWarps, (uint64_t)per * (uint64_t)sms));
    decompress_warp_kernel<Geo, NARROW><<<(unsigned)grid, K::kDNTW, smem, s>>>(a);
    return cudaGetLastError();
}

template <class Geo>
cudaError_t dw_launch(const zs_dict *d, const TiledLaunch &L, cudaStream_t s)
{
    DwArgs a{};
    a.one = L.one;
    a.shards = L.shards;
    a.n_shards = L.n_shards;
    a.total_tiles = L.total_tiles;
    a.dec = d->d_dec;
    a.g = L.g;
    a.limit_ns = wait_limit_ns();
    a.stall_tile = injected_stall_tile();
    return d->max_plen <= 7 ? dw_launch_as<Geo, true>(a, L.total_tiles, s)
                            : dw_launch_as<Geo, false>(a, L.total_tiles, s);
}

struct DwEntry {
    KernelVariant info;
    cudaError_t (*launch)(const zs_dict *, const TiledLaunch &, cudaStream_t);
};

template <class Geo>
constexpr DwEntry dw_entry(const char *name)
{
    return DwEntry{KernelVariant{name, Geo::kWarps, 32 * Geo::kLane}, &dw_launch<Geo>};
}

const DwEntry kDwv[] = {
    dw_entry<DwV0>("decompress w22 t2176"),
    dw_entry<DwV1>("decompress w20 t2176"),
    dw_entry<DwV2>("decompress w28 t1664"),
    dw_entry<DwV3>("decompress w32 t1152"),
};
constexpr int kNumDw = (int)(sizeof(kDwv) / sizeof(kDwv[0]));

}  // namespace

// Variant numbering of the decompression kernels: the expansion kernel's geometries first
// (decode_expand.cu), then this kernel's.
int decompress_variants() { return expand_variants() + kNumDw; }

const KernelVariant *decompress_variant(int v)
{
    const int nx = expand_variants();
    if (v >= 0 && v < nx) return expand_variant(v);
    v -= nx;
    return (v >= 0 && v < kNumDw) ? &kDwv[v].info : nullptr;
}

bool decompress_fits(int v, const zs_dict *d)
{
    const int nx = expand_variants();
    if (v >= 0 && v < nx) return expand_fits(v, d);
    return v >= nx && v < nx + kNumDw;
}

int decompress_default_variant(const zs_dict *d) { return expand_fits(0, d) ? 0 : expand_variants(); }

cudaError_t launch_decompress(int v, const zs_dict *d, const TiledLaunch &L, cudaStream_t s)
{
    const int nx = expand_variants();
    if (v >= 0 && v < nx) return launch_expand(v, d, L, s);
    v -= nx;
    if (v < 0 || v >= kNumDw) return cudaErrorInvalidValue;
    return kDwv[v].launch(d, L, s);
}

// Look-back records for a single-stream call: enough for the smaller of the two default tiles.
uint64_t decompress_tile_bytes()
{
    return std::min<uint64_t>(expand_variant(0)->tile_bytes, kDwv[0].info.tile_bytes);
}

uint64_t decompress_tiles(uint64_t n) { return tiles_for(n, (uint32_t)decompress_tile_bytes()); }

cudaError_t launch_decompress_single(const zs_dict *d, const uint8_t *in, uint64_t n, uint8_t *out, uint64_t out_cap,
                                     DevResult *res, TileState *tiles, cudaStream_t s)
{
    const int v = decompress_default_variant(d);
    TiledLaunch L{};
    L.one = single_shard(in, n, out, out_cap, nullptr, 0, tiles, res, tiles_for(n, decompress_variant(v)->tile_bytes));
    L.n_shards = 1;
    L.total_tiles = L.one.ntiles;
    L.g = res;
    return launch_decompress(v, d, L, s);
}

}  // namespace zs
