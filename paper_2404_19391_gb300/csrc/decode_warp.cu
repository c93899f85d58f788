// zs_decompress (Sec. IV-D2) with one warp per 1408-byte tile of compressed input.
//
//   - Each warp of a persistent CTA claims tiles in launch order, stages its tile with one bulk (TMA)
//     copy and works on it alone: no CTA-wide barrier is on the per-tile path.
//   - Escapes without a sequential scan: a byte is verbatim exactly when the run of ' ' bytes just before
//     it has odd length (every unescaped ' ' escapes the byte after it, and a run always starts
//     unescaped), so each lane decodes its own 44-byte slice after counting the spaces in front of it
//     (an odd number of words per slice keeps the lanes' shared-memory reads on distinct banks).
//   - Small tiles and 28 warps per SM: the per-lane loops are chains of dependent shared-memory loads,
//     so the kernel is bound by latency, and the warp count is what hides it.
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
template <int W, int LANE>
struct DwGeom {
    static constexpr int kWarps = W;
    static constexpr int kLane = LANE;
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

template <class Geo>
struct DW {
    static constexpr int kDW = Geo::kWarps;
    static constexpr int kDNTW = 32 * kDW;
    static constexpr int kDLane = Geo::kLane;
    static constexpr int kDTile = 32 * kDLane;                  // compressed bytes per warp tile
    static constexpr int kDOut = (kDTile * 5 / 2 + 255) & ~255;  // staged output bytes per tile
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
        uint32_t lane;
        uint32_t *status;
    };

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
        bool lit = (run & 1u) != 0;
        const bool lit_start = lit;
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
        if (staged) expand_slice<true>(C, S, p0, p1, S.lit0[lane] != 0, S.lane_off[lane], ea, so);
        else expand_slice<false>(C, S, p0, p1, S.lit0[lane] != 0, S.lane_off[lane], ea, so);
        __syncwarp();
        if (staged) {
            uint8_t *gdst = A.out + ea - so;  // 16-byte aligned
            const uint32_t nchunks = (uint32_t)((so + total + 15) >> 4);
            for (uint32_t c = lane; c < nchunks; c += 32) {
                const uint32_t lo = c * 16u, hi = lo + 16u;
                if (lo >= so && hi <= so + total && ea - so + hi <= A.out_cap) {
                    *reinterpret_cast<uint4 *>(gdst + lo) = *reinterpret_cast<const uint4 *>(C.M->ost + lo);
                } else {
                    for (uint32_t k = lo; k < hi; ++k)
                        if (k >= so && k < so + total && ea - so + k < A.out_cap) gdst[k] = C.M->ost[k];
                }
            }
        }
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
        if (!mbar_wait_bounded(&tab_bar, 0, P->limit_ns, C.status)) {
            mbar_wait_bounded(&tab_bar, 0, P->limit_ns, C.status);
            return;
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

template <class Geo>
__global__ void __launch_bounds__(Geo::kWarps * 32, 1) decompress_warp_kernel(const DwArgs P)
{
    DW<Geo>::run(&P);
}

// Compiled geometries; variant 0 is the default.
using DwV0 = DwGeom<28, 44>;
using DwV1 = DwGeom<32, 36>;
using DwV2 = DwGeom<20, 68>;

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
    const int smem = (int)(DW<Geo>::kDW * sizeof(typename DW<Geo>::DWarpMem) + kDecBytes);
    static int per = -1;
    if (per < 0) {
        cudaError_t e = cudaFuncSetAttribute(decompress_warp_kernel<Geo>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             smem);
        if (e != cudaSuccess) return e;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, decompress_warp_kernel<Geo>, DW<Geo>::kDNTW, smem);
        if (per < 1) per = 1;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t grid = std::max<uint64_t>(
        1, std::min<uint64_t>((L.total_tiles + Geo::kWarps - 1) / Geo::kWarps, (uint64_t)per * (uint64_t)sms));
    decompress_warp_kernel<Geo><<<(unsigned)grid, DW<Geo>::kDNTW, smem, s>>>(a);
    return cudaGetLastError();
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
    dw_entry<DwV0>("decompress w28 t1408"),
    dw_entry<DwV1>("decompress w32 t1152"),
    dw_entry<DwV2>("decompress w20 t2176"),
};
constexpr int kNumDw = (int)(sizeof(kDwv) / sizeof(kDwv[0]));

}  // namespace

int decompress_variants() { return kNumDw; }

const KernelVariant *decompress_variant(int v) { return (v >= 0 && v < kNumDw) ? &kDwv[v].info : nullptr; }

cudaError_t launch_decompress(int v, const zs_dict *d, const TiledLaunch &L, cudaStream_t s)
{
    if (v < 0 || v >= kNumDw) return cudaErrorInvalidValue;
    return kDwv[v].launch(d, L, s);
}

uint64_t decompress_tiles(uint64_t n) { return tiles_for(n, kDwv[kDefaultVariant].info.tile_bytes); }

uint64_t decompress_tile_bytes() { return kDwv[kDefaultVariant].info.tile_bytes; }

cudaError_t launch_decompress_single(const zs_dict *d, const uint8_t *in, uint64_t n, uint8_t *out, uint64_t out_cap,
                                     DevResult *res, TileState *tiles, cudaStream_t s)
{
    TiledLaunch L{};
    L.one = single_shard(in, n, out, out_cap, nullptr, 0, tiles, res, decompress_tiles(n));
    L.n_shards = 1;
    L.total_tiles = L.one.ntiles;
    L.g = res;
    return launch_decompress(kDefaultVariant, d, L, s);
}

}  // namespace zs
