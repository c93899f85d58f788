// zs_decompress (Sec. IV-D2), expansion kernel: one warp per tile of compressed input, 512 bytes per round.
//
//   - Tiles and look-back as in the other tiled kernels: each warp of a persistent CTA claims tiles in
//     launch order, stages one (and the 16 bytes before it) with one bulk (TMA) copy, and resolves its
//     output offset by a warp-wide decoupled look-back. The next tile is claimed and its copy issued as soon
//     as the current one has expanded, so the copy lands while the warp looks back and copies out.
//   - Rounds: lane l takes the 16 bytes at 16 l of each 512-byte round (conflict-free 16-byte loads) and
//     looks up the 16 patterns at once. Each 64-bit entry holds the pattern (up to 7 bytes) and, in its top
//     byte, its length plus 128 for '\n', so one sum gives the lane's output bytes and newlines; ' ' and
//     bytes that are no symbol carry a flag instead, and such chunks (rare in SMILES text) take a byte loop.
//     The table is replicated 16 times so that the 16 lanes of each half-warp read 16 different bank pairs.
//   - A size pass over the entries' top words gives each lane's output bytes per round, a warp scan per
//     round places the lanes, and the tile publishes its size before it expands; the expansion then funnels
//     each lane's patterns into 32-bit words in a register and ORs each finished word into a cleared stage
//     (the first and last words of a lane may hold bytes of its neighbours, which the OR keeps).
//   - Escapes need no sequential scan: a byte is verbatim exactly when the run of ' ' before it has odd
//     length (every unescaped ' ' escapes the next byte, and a run starts unescaped).
//   - The stage leaves with aligned 16-byte stores once the look-back has given the tile's offset; a tile
//     that expands past its stage writes straight to memory after its look-back instead.
#include <algorithm>

#include "zs_common.cuh"

namespace zs {
namespace {

template <int W, int TB, int OUTB, int SLOTS, bool GIN = false>
struct DxGeom {
    static constexpr int kWarps = W;    // warps per CTA (one CTA per SM)
    static constexpr int kTile = TB;    // compressed bytes per warp tile
    static constexpr int kOut = OUTB;   // staged output bytes per tile
    static constexpr int kSlots = SLOTS;  // 2: a tile's look-back and copy-out wait until the next tile is
                                          // expanded (software pipeline); 1: they follow at once
    static constexpr bool kGlobalIn = GIN;  // the tile's compressed bytes are read from global memory (through
                                            // L1) instead of a staged copy: shared memory for more warps
};

constexpr unsigned kAllX = 0xffffffffu;

// *[addr] |= v in shared memory (32-bit shared-window address) when p holds: one predicated reduction, no branch.
__device__ __forceinline__ void red_or_shared(uint32_t addr, uint32_t v, bool p)
{
    asm volatile("{ .reg .pred q; setp.ne.u32 q, %2, 0; @q red.shared.or.b32 [%0], %1; }" ::"r"(addr), "r"(v),
                 "r"((uint32_t)p)
                 : "memory");
}

// Look-back records of this decoder: the first two words of a TileState, each single-copy atomic with its own
// valid bit: agg_a = the tile's output bytes (its aggregate), agg_b = the output bytes of tiles [0, this] (its
// inclusive prefix). One 16-byte load reads a record. Newlines are not carried: each tile adds its count to the
// shard's result with one atomic add.
__device__ __forceinline__ void dx_publish(TileState *ts, bool inclusive, uint64_t v)
{
    unsigned long long *p = inclusive ? &ts->agg_b : &ts->agg_a;
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"((unsigned long long)(v | kValidBit)) : "memory");
}

// Decoupled look-back by a whole warp over these records: each round trip, lane j reads the records of tiles
// t-1-j-32r for r < R, 32 R predecessors a trip. Sums aggregates from the nearest predecessor back to (and
// including) the nearest inclusive prefix. Every tile publishes its aggregate before it expands (a size pass),
// so the walk seldom waits; what it costs is round trips, and with thousands of tiles in flight the nearest
// inclusive prefix can be hundreds of tiles back. Called by all 32 lanes; all return the same sum. Waits are
// bounded (kStTimeout on expiry).
template <int R>
__device__ __forceinline__ uint64_t dx_lookback(TileState *tiles, uint64_t t, uint64_t limit_ns, uint32_t *status)
{
    const uint32_t lane = threadIdx.x & 31;
    uint64_t a = 0;
    int64_t top = (int64_t)t - 1;
    uint64_t t0 = 0;
    bool timed = false;
    while (top >= 0) {
        uint64_t v[R];
        uint32_t incl = 0, none = 0;  // bit r: record r holds an inclusive prefix / nothing yet
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int64_t p = top - (int64_t)lane - 32 * r;
            unsigned long long g = 0, i = kValidBit;  // before tile 0: an inclusive zero
            if (p >= 0) ld_pair(&tiles[p].agg_a, &g, &i);
            const bool fi = (i & kValidBit) != 0, fg = (g & kValidBit) != 0;
            incl |= (fi ? 1u : 0u) << r;
            none |= (!fi && !fg ? 1u : 0u) << r;
            v[r] = (fi ? i : g) & ~kValidBit;
        }
        // distance (32 r + lane) of the nearest record holding an inclusive prefix
        int stop = 32 * R;
#pragma unroll
        for (int r = R - 1; r >= 0; --r) {
            const uint32_t b = __ballot_sync(kAllX, (incl >> r) & 1u);
            if (b) stop = 32 * r + __ffs(b) - 1;
        }
        bool missing = false;  // a nearer tile has published nothing
#pragma unroll
        for (int r = 0; r < R; ++r) missing |= (32 * r + (int)lane < stop) && ((none >> r) & 1u);
        if (__any_sync(kAllX, missing)) {
            if (*((volatile uint32_t *)status) & kStTimeout) break;
            if (!timed) {
                t0 = gtime();
                timed = true;
            } else if (gtime() - t0 > limit_ns) {
                if (lane == 0) atomicOr(status, kStTimeout);
                break;
            }
            __nanosleep(64);
            continue;
        }
        timed = false;
        uint64_t sa = 0;
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (32 * r + (int)lane <= stop) sa += v[r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sa += __shfl_xor_sync(kAllX, sa, o);
        a += sa;
        if (stop < 32 * R) break;
        top -= 32 * R;
    }
    return a;
}
constexpr uint32_t kCopies = 16;       // replicas of the pattern table
constexpr uint32_t kFlag = 0x40000000u; // entry flag (top word): ' ' or a byte that is no symbol

struct DxArgs {
    ShardView one;
    const ShardView *shards;
    uint32_t n_shards;
    uint32_t _pad;
    uint64_t total_tiles;
    const uint8_t *dec;  // plen[256], pat[256][16]
    DevResult *g;
    uint64_t limit_ns;
    int64_t stall_tile;
};

template <class Geo>
struct DX {
    static constexpr int kW = Geo::kWarps;
    static constexpr int kNT = 32 * kW;
    static constexpr int kTB = Geo::kTile;
    static constexpr int kOutB = Geo::kOut;
    static constexpr int kRounds = kTB / 512;
    // look-back records per lane per round trip (64 tiles a trip: measured best against 1, 4 and 8)
    static constexpr int kLbR = 2;
    static_assert(kTB % 512 == 0 && kOutB % 16 == 0, "expansion geometry");

    struct alignas(16) OutSlot {
        uint8_t out[kOutB + 32];  // the tile's output at stage offset o = (destination address mod 16)
        ShardView sv;
    };

    struct alignas(16) WarpMem {
        uint8_t in[Geo::kGlobalIn ? 16 : 16 + kTB + 16];  // the 16 bytes before the tile, the tile (staged)
        OutSlot os[Geo::kSlots];
        ShardView nsv;              // shard of the staged tile (copied to its output slot when it expands)
        uint32_t pw[kRounds][32];   // from the size pass: lane's output offset in the round | kSlowChunk
        uint32_t run[kRounds];      // from the size pass: the round's output offset in the tile
        uint64_t bar;
    };
    static constexpr uint32_t kSlowChunk = 0x80000000u;

    struct Ctx {
        const DxArgs *P;
        const ShardView *A;
        WarpMem *M;
        const uint8_t *tin;  // the tile's first compressed byte: in the stage, or in global memory
        const uint8_t *tab;  // pat8[256][kCopies]
        const uint8_t *plen;
        const uint8_t *pat;
        uint32_t lane, lane8;
        uint32_t *status;
    };

    static __device__ __forceinline__ void stage(const Ctx &C, uint64_t t, uint32_t nown)
    {
        const ShardView &A = *C.A;
        WarpMem &M = *C.M;
        const uint64_t base = t * (uint64_t)kTB;
        const uint64_t lo = base >= 16 ? base - 16 : 0;
        const uint32_t j0 = (uint32_t)(lo + 16 - base);
        const uint32_t nbytes = (uint32_t)(base + nown - lo);
        const uint32_t nbulk = A.in_aligned ? (nbytes & ~15u) : 0u;
        __syncwarp();
        if (C.lane == 0) {
            fence_proxy_async_smem();
            mbar_arrive_tx(&M.bar, nbulk);
            if (nbulk) bulk_g2s(M.in + j0, A.in + lo, nbulk, &M.bar);
        }
        for (uint32_t j = nbulk + C.lane; j < nbytes; j += 32) M.in[j0 + j] = A.in[lo + j];
        if (t == 0 && C.lane == 0) M.in[15] = 0;  // nothing precedes the stream
    }

    // Whether the byte at tile offset c0 is verbatim: the run of ' ' before it has odd length (staged bytes
    // first, then global memory for a run that reaches past the stage).
    static __device__ __forceinline__ bool literal_at(const Ctx &C, uint64_t base, uint32_t c0)
    {
        uint32_t run = 0;
        if constexpr (Geo::kGlobalIn) {
            int64_t g = (int64_t)(base + c0) - 1;
            while (g >= 0 && C.A->in[g] == kEsc) {
                ++run;
                --g;
            }
            return (run & 1u) != 0;
        }
        const WarpMem &M = *C.M;
        int32_t q = 15 + (int32_t)c0;  // staged position of the byte before
        while (q >= 0 && M.in[q] == kEsc && base + (uint64_t)q >= 16) {
            ++run;
            --q;
        }
        if (q < 0) {  // the run continues before the stage
            int64_t g = (int64_t)base - 17;
            while (g >= 0 && C.A->in[g] == kEsc) {
                ++run;
                --g;
            }
        }
        return (run & 1u) != 0;
    }

    // The byte before tile offset c0 (0 before the stream's first byte).
    static __device__ __forceinline__ uint32_t byte_before(const Ctx &C, uint64_t base, uint32_t c0)
    {
        if (Geo::kGlobalIn && base + c0 == 0) return 0u;
        return C.tin[(int32_t)c0 - 1];
    }

    // The 16 compressed bytes at tile offset c0 (16-byte aligned in the stage; from global memory only when
    // the shard's input is 16-byte aligned, else byte by byte).
    static __device__ __forceinline__ uint4 load16(const Ctx &C, uint32_t c0)
    {
        if constexpr (!Geo::kGlobalIn) {
            return *reinterpret_cast<const uint4 *>(C.tin + c0);
        } else {
            if (C.A->in_aligned) return *reinterpret_cast<const uint4 *>(C.tin + c0);
            uint32_t w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                w[k] = (uint32_t)C.tin[c0 + 4 * k] | ((uint32_t)C.tin[c0 + 4 * k + 1] << 8) |
                       ((uint32_t)C.tin[c0 + 4 * k + 2] << 16) | ((uint32_t)C.tin[c0 + 4 * k + 3] << 24);
            return make_uint4(w[0], w[1], w[2], w[3]);
        }
    }

    // Byte loop over the staged bytes [p0, p1) (tile offsets): output bytes and newlines, noting malformed
    // bytes. *lit: in, the first byte is verbatim; out, the last byte was an unpaired ' '.
    static __device__ __forceinline__ void slow_size(const Ctx &C, uint64_t base, uint32_t p0, uint32_t p1, bool *lit,
                                                     uint32_t *outb, uint32_t *nls)
    {
        const ShardView &A = *C.A;
        const uint8_t *in = C.tin;
        uint32_t ob = 0, nl = 0;
        bool l = *lit;
        for (uint32_t p = p0; p < p1; ++p) {
            const uint8_t b = in[p];
            if (l) {
                if (b == kNl) {  // a line ending in an unpaired escape
                    note_error_offset(A.res, base + p - 1);
                    atomicOr(C.status, kStMalformed);
                }
                ob += 1;
                nl += (b == kNl);
                l = false;
            } else if (b == kEsc) {
                l = true;
            } else if (b == kNl) {
                ob += 1;
                nl += 1;
            } else {
                const uint32_t len = C.plen[b];
                if (len == 0) {
                    note_error_offset(A.res, base + p);
                    atomicOr(C.status, kStMalformed);
                }
                ob += len;
            }
        }
        *lit = l;
        *outb = ob;
        *nls = nl;
    }

    // The same walk writing the bytes to out[ea + pos] (those below the capacity): a tile that outgrew its stage.
    static __device__ __forceinline__ void slow_write(const Ctx &C, uint32_t p0, uint32_t p1, bool lit, uint32_t pos,
                                                      uint64_t ea)
    {
        const ShardView &A = *C.A;
        const uint8_t *in = C.tin;
        auto put = [&](uint32_t w, uint8_t v) {
            if (ea + w < A.out_cap) A.out[ea + w] = v;
        };
        for (uint32_t p = p0; p < p1; ++p) {
            const uint8_t b = in[p];
            if (!lit && b == kEsc) {
                lit = true;
                continue;
            }
            if (lit || b == kNl) {
                lit = false;
                put(pos++, b);
                continue;
            }
            const uint32_t l = C.plen[b];
            for (uint32_t k = 0; k < l; ++k) put(pos + k, C.pat[16u * b + k]);
            pos += l;
        }
    }

    // The byte loop of a slow chunk writing by atomic OR into the cleared stage (lanes share boundary words).
    static __device__ __forceinline__ void slow_or(const Ctx &C, uint32_t p0, uint32_t p1, bool lit, uint32_t pos,
                                                   uint8_t *stg)
    {
        const uint8_t *in = C.tin;
        uint32_t *w32 = reinterpret_cast<uint32_t *>(stg);
        auto put = [&](uint32_t w, uint8_t v) { atomicOr(w32 + (w >> 2), (uint32_t)v << (8 * (w & 3u))); };
        for (uint32_t p = p0; p < p1; ++p) {
            const uint8_t b = in[p];
            if (!lit && b == kEsc) {
                lit = true;
                continue;
            }
            if (lit || b == kNl) {
                lit = false;
                put(pos++, b);
                continue;
            }
            const uint32_t l = C.plen[b];
            for (uint32_t k = 0; k < l; ++k) put(pos + k, C.pat[16u * b + k]);
            pos += l;
        }
    }

    // Size pass over a staged tile, from the top words of the entries alone (chunks holding ' ' or a byte that
    // is no symbol take the byte loop, which also notes malformed bytes): each lane's output offset in each
    // round (warp scan) into pw, each round's offset in the tile into run; every lane returns the tile's
    // totals. It runs before the expansion so that the tile's size is published early and the look-backs of
    // later tiles seldom wait.
    static __device__ __forceinline__ void tile_sizes(const Ctx &C, uint64_t base, uint32_t nown, uint32_t *total,
                                                      uint32_t *nls)
    {
        WarpMem &M = *C.M;
        uint32_t run = 0, nl = 0;
        for (int r = 0; r < kRounds; ++r) {
            if ((uint32_t)r * 512u >= nown) break;
            const uint32_t c0 = (uint32_t)r * 512u + C.lane * 16u;
            const uint32_t p0 = min(c0, nown), p1 = min(c0 + 16u, nown);
            uint32_t ob = 0;
            bool fast = p1 - p0 == 16 && byte_before(C, base, c0) != kEsc;
            if (fast) {
                const uint4 v = load16(C, c0);
                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
                uint32_t acc = 0, fl = 0;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const uint32_t b = (w[k >> 2] >> (8 * (k & 3))) & 255u;
                    const uint32_t e = *reinterpret_cast<const uint32_t *>(C.tab + ((b << 7) | C.lane8) + 4);
                    acc += e >> 24;
                    fl |= e;
                }
                if (fl & kFlag) {
                    fast = false;
                } else {
                    ob = acc & 127u;
                    nl += acc >> 7;
                }
            }
            if (!fast && p1 > p0) {
                bool lit = literal_at(C, base, p0);
                uint32_t n1 = 0;
                slow_size(C, base, p0, p1, &lit, &ob, &n1);
                nl += n1;
                if (lit && base + p1 == C.A->n) {  // the stream ends in an unpaired escape
                    note_error_offset(C.A->res, C.A->n - 1);
                    atomicOr(C.status, kStMalformed);
                }
            }
            const uint32_t inc = warp_incl_u32(ob);
            M.pw[r][C.lane] = (inc - ob) | (fast ? 0u : kSlowChunk);
            if (C.lane == 31) M.run[r] = run;
            run += __shfl_sync(kAllX, inc, 31);
        }
        __syncwarp();
        *total = run;
        *nls = __reduce_add_sync(kAllX, nl);
    }

    // The 16 patterns of a fast chunk ORed into the (cleared) stage from shared address q on. The lane builds
    // each 32-bit word of its output in a register (a funnel of the patterns) and ORs a word into the stage once
    // it is complete, and the last, partial one at the end: about one reduction per two patterns, each with the
    // lanes that complete a word at that step, so the 32 lanes' random banks collide far less than with one
    // reduction per word a pattern touches. A lane's first and last words may hold bytes of its neighbours
    // (the OR keeps them).
    static __device__ __forceinline__ void or_patterns(const uint32_t (&lo)[16], const uint32_t (&hi)[16],
                                                       uint32_t q)
    {
        uint32_t w = q & ~3u;         // the word being filled
        uint32_t n8 = 8u * (q & 3u);  // its bits below this lane's next byte
        uint32_t acc = 0;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const uint32_t len8 = (hi[k] >> 21) & 56u;  // 8 x the pattern's length
            const uint32_t h = hi[k] & 0x00FFFFFFu;
            const uint32_t w0 = acc | (lo[k] << n8);
            const uint32_t w1 = __funnelshift_l(lo[k], h, n8);
            const uint32_t w2 = __funnelshift_l(h, 0u, n8);
            const uint32_t t8 = n8 + len8;  // below 88: the word and at most two more
            red_or_shared(w, w0, t8 >= 32u);
            red_or_shared(w + 4u, w1, t8 >= 64u);
            acc = t8 >= 64u ? w2 : (t8 >= 32u ? w1 : w0);
            w += (t8 >> 5) << 2;
            n8 = t8 & 31u;
        }
        red_or_shared(w, acc, n8 != 0u);
    }

    // Expansion of a sized tile into slot O's stage (which must hold total + 32 bytes): per round, each lane
    // looks up its 16 patterns and ORs them in at the offset the size pass gave it.
    static __device__ __forceinline__ void expand(const Ctx &C, OutSlot &O, uint64_t base, uint32_t nown,
                                                  uint32_t total)
    {
        const WarpMem &M = *C.M;
        uint8_t *stg = O.out;
        uint4 *s16 = reinterpret_cast<uint4 *>(stg);
        const uint32_t nclear = (total + 12u + 15u) / 16u;  // patterns OR zeros up to 12 bytes past the end
        for (uint32_t j = C.lane; j < nclear; j += 32) s16[j] = make_uint4(0, 0, 0, 0);
        __syncwarp();
        const uint32_t sbase = smem_u32(stg);
        for (int r = 0; r < kRounds; ++r) {
            if ((uint32_t)r * 512u >= nown) break;
            const uint32_t c0 = (uint32_t)r * 512u + C.lane * 16u;
            const uint32_t p0 = min(c0, nown), p1 = min(c0 + 16u, nown);
            if (p1 <= p0) continue;
            const uint32_t pw = M.pw[r][C.lane];
            const uint32_t pos = M.run[r] + (pw & ~kSlowChunk);
            if (!(pw & kSlowChunk)) {
                const uint4 v = load16(C, c0);
                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
                uint32_t lo[16], hi[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const uint32_t b = (w[k >> 2] >> (8 * (k & 3))) & 255u;
                    const uint2 e = *reinterpret_cast<const uint2 *>(C.tab + ((b << 7) | C.lane8));
                    lo[k] = e.x;
                    hi[k] = e.y;
                }
                or_patterns(lo, hi, sbase + pos);
            } else {
                slow_or(C, p0, p1, literal_at(C, base, p0), pos, stg);
            }
        }
        __syncwarp();
    }

    // A tile that outgrew its stage: the byte loop of every chunk, at the offsets of the size pass, straight to
    // out[ea + ...].
    static __device__ void expand_direct(const Ctx &C, uint64_t base, uint32_t nown, uint64_t ea)
    {
        const WarpMem &M = *C.M;
        for (int r = 0; r < kRounds; ++r) {
            if ((uint32_t)r * 512u >= nown) break;
            const uint32_t c0 = (uint32_t)r * 512u + C.lane * 16u;
            const uint32_t p0 = min(c0, nown), p1 = min(c0 + 16u, nown);
            if (p1 <= p0) continue;
            const uint32_t pw = M.pw[r][C.lane];
            const bool lit = (pw & kSlowChunk) ? literal_at(C, base, p0) : false;
            slow_write(C, p0, p1, lit, M.run[r] + (pw & ~kSlowChunk), ea);
        }
        __syncwarp();
    }

    // The shard's last tile writes the output size and counts the unterminated last line (newlines are added
    // to n_lines tile by tile).
    static __device__ __forceinline__ void finish_result(const Ctx &C, uint64_t t, uint64_t tot_a)
    {
        const ShardView &A = *C.A;
        if (C.lane == 0 && t == A.ntiles - 1) {
            A.res->out_len = tot_a;
            if (A.in[A.n - 1] != kNl) atomicAdd(&A.res->n_lines, 1ull);
        }
    }

    // Look-back, inclusive prefix, copy-out of a staged tile.
    static __device__ void finish_staged(const Ctx &C, OutSlot &O, uint64_t t, uint32_t total)
    {
        const ShardView &A = *C.A;
        const uint64_t ea = t > 0 ? dx_lookback<kLbR>(A.tiles, t, C.P->limit_ns, C.status) : 0;
        if (C.lane == 0 && t > 0 && (int64_t)t != C.P->stall_tile) dx_publish(&A.tiles[t], true, ea + total);
        if (total) warp_copy_realign<true>(O.out, total, A.out + ea, A.out_cap > ea ? A.out_cap - ea : 0);
        finish_result(C, t, ea + total);
        __syncwarp();
    }

    static __device__ void run(const DxArgs *P)
    {
        extern __shared__ __align__(128) uint8_t smem[];
        __shared__ uint64_t tab_bar;
        const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        WarpMem &M = reinterpret_cast<WarpMem *>(smem)[wid];
        uint8_t *tab = smem + kW * sizeof(WarpMem);  // pat8[256][kCopies], then plen[256] and pat[256][16]
        uint8_t *dec = tab + 256 * kCopies * 8;
        Ctx C;
        C.P = P;
        C.A = nullptr;
        C.M = &M;
        C.tin = nullptr;
        C.tab = tab;
        C.plen = dec;
        C.pat = dec + 256;
        C.lane = lane;
        C.lane8 = (lane & 15u) * 8u;
        C.status = &P->g->status;
        if (threadIdx.x == 0) mbar_init(&tab_bar, 1);
        if (lane == 0) mbar_init(&M.bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_arrive_tx(&tab_bar, kDecBytes);
            bulk_g2s(dec, P->dec, kDecBytes, &tab_bar);
        }
        const bool ok = mbar_wait_bounded(&tab_bar, 0, P->limit_ns, C.status);
        if (!__syncthreads_and(ok)) {
            mbar_wait_bounded(&tab_bar, 0, P->limit_ns, C.status);
            return;
        }
        // pat8: pattern bytes 0-6, top byte = length | 128 for '\n'; ' ' and non-symbols carry kFlag
        for (uint32_t i = threadIdx.x; i < 256 * kCopies; i += blockDim.x) {
            const uint32_t b = i / kCopies;
            const uint32_t l = dec[b];
            uint64_t e;
            if (b == kNl) {
                e = (uint64_t)kNl | (0x81ull << 56);
            } else if (b == kEsc || l == 0) {
                e = (uint64_t)kFlag << 32;
            } else {
                e = (uint64_t)l << 56;
                for (uint32_t k = 0; k < l; ++k) e |= (uint64_t)dec[256 + 16 * b + k] << (8 * k);
            }
            reinterpret_cast<uint64_t *>(tab)[i] = e;
        }
        __syncthreads();
        uint32_t ph = 0;
        constexpr uint32_t kWords = sizeof(ShardView) / 8;
        // Shard lookup (only when g leaves the shard of the last tile) and the bulk copy of launch-wide tile g.
        auto stage_tile = [&](uint64_t g) {
            if (g < M.nsv.tile0 || g >= M.nsv.tile0 + M.nsv.ntiles) {
                const uint32_t sh = P->n_shards == 1 ? 0u : find_shard(P->shards, P->n_shards, g);
                load_shard(&M.nsv, P->one, P->shards, P->n_shards, sh);
            }
            const uint64_t t = g - M.nsv.tile0;
            const uint64_t base = t * (uint64_t)kTB;
            if constexpr (!Geo::kGlobalIn) {  // else the bytes are read where they lie
                Ctx Cn = C;
                Cn.A = &M.nsv;
                stage(Cn, t, (uint32_t)(min(M.nsv.n, base + kTB) - base));
            }
        };
        if (lane == 0) {
            M.nsv.tile0 = 0;
            M.nsv.ntiles = 0;  // no shard loaded yet
        }
        __syncwarp();
        unsigned long long tt = 0;
        if (lane == 0) tt = atomicAdd(&P->g->tile_counter, 1ull);
        uint64_t g = __shfl_sync(kAllX, tt, 0);
        bool have = g < P->total_tiles;
        if (have) stage_tile(g);
        OutSlot &O = M.os[0];
        while (have) {
            if (lane < kWords) reinterpret_cast<uint64_t *>(&O.sv)[lane] = reinterpret_cast<const uint64_t *>(&M.nsv)[lane];
            __syncwarp();
            const ShardView &A = O.sv;
            const uint64_t t = g - A.tile0;
            Ctx Cs = C;
            Cs.A = &O.sv;
            const uint64_t base = t * (uint64_t)kTB;
            const uint32_t nown = (uint32_t)(min(A.n, base + kTB) - base);
            if constexpr (Geo::kGlobalIn) {
                Cs.tin = A.in + base;
            } else {
                Cs.tin = M.in + 16;
                if (!mbar_wait_bounded(&M.bar, ph, P->limit_ns, C.status)) {
                    mbar_wait_bounded(&M.bar, ph, P->limit_ns, C.status);
                    return;
                }
                ph ^= 1u;
            }
            __syncwarp();
            // size pass: the tile's size is published before it expands
            uint32_t total = 0, nls = 0;
            tile_sizes(Cs, base, nown, &total, &nls);
            if (lane == 0) {
                if ((int64_t)t != P->stall_tile) dx_publish(&A.tiles[t], t == 0, total);
                if (nls) atomicAdd(&A.res->n_lines, (unsigned long long)nls);
            }
            const bool fits = total + 32u <= (uint32_t)kOutB;
            if (fits) {
                expand(Cs, O, base, nown, total);
            } else {  // a tile that outgrows the stage looks back first and writes straight to memory
                const uint64_t ea = t > 0 ? dx_lookback<kLbR>(A.tiles, t, P->limit_ns, C.status) : 0;
                if (lane == 0 && t > 0 && (int64_t)t != P->stall_tile) dx_publish(&A.tiles[t], true, ea + total);
                expand_direct(Cs, base, nown, ea);
                finish_result(Cs, t, ea + total);
                __syncwarp();
            }
            // the staged bytes of this tile are dead from here on: the next tile's copy lands during the look-back
            // and copy-out of this one
            if (lane == 0) tt = atomicAdd(&P->g->tile_counter, 1ull);
            g = __shfl_sync(kAllX, tt, 0);
            have = g < P->total_tiles;
            if (have) stage_tile(g);
            if (fits) finish_staged(Cs, O, t, total);
        }
    }
};

template <class Geo>
__global__ void __launch_bounds__(Geo::kWarps * 32, 1) decompress_expand_kernel(const DxArgs P)
{
    DX<Geo>::run(&P);
}

// Compiled geometries, all with 2048-byte tiles (four rounds) and one stage of 2.25 x the tile beside the 36 KB
// of tables: the input staged by a bulk copy with 24 warps per SM (72 registers) or 20 warps (96), or read from
// global memory with 28 or 32 warps (the shared memory of the staged input left to more warps).
using DxV0 = DxGeom<24, 2048, 4608, 1>;
using DxV1 = DxGeom<20, 2048, 4608, 1>;
using DxV2 = DxGeom<28, 2048, 4608, 1, true>;
using DxV3 = DxGeom<32, 2048, 4608, 1, true>;
static_assert(DxV0::kWarps * sizeof(DX<DxV0>::WarpMem) + 256 * kCopies * 8 + kDecBytes <= 227 * 1024, "smem");
static_assert(DxV1::kWarps * sizeof(DX<DxV1>::WarpMem) + 256 * kCopies * 8 + kDecBytes <= 227 * 1024, "smem");
static_assert(DxV2::kWarps * sizeof(DX<DxV2>::WarpMem) + 256 * kCopies * 8 + kDecBytes <= 227 * 1024, "smem");
static_assert(DxV3::kWarps * sizeof(DX<DxV3>::WarpMem) + 256 * kCopies * 8 + kDecBytes <= 227 * 1024, "smem");

template <class Geo>
size_t dx_smem()
{
    return DX<Geo>::kW * sizeof(typename DX<Geo>::WarpMem) + 256 * kCopies * 8 + kDecBytes;
}

template <class Geo>
cudaError_t dx_launch(const zs_dict *d, const TiledLaunch &L, cudaStream_t s)
{
    DxArgs a{};
    a.one = L.one;
    a.shards = L.shards;
    a.n_shards = L.n_shards;
    a.total_tiles = L.total_tiles;
    a.dec = d->d_dec;
    a.g = L.g;
    a.limit_ns = wait_limit_ns();
    a.stall_tile = injected_stall_tile();
    const int smem = (int)dx_smem<Geo>();
    static int per = -1;
    if (per < 0) {
        cudaError_t e = cudaFuncSetAttribute(decompress_expand_kernel<Geo>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             smem);
        if (e != cudaSuccess) return e;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, decompress_expand_kernel<Geo>, DX<Geo>::kNT, smem);
        if (per < 1) per = 1;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t grid = std::max<uint64_t>(
        1, std::min<uint64_t>((L.total_tiles + Geo::kWarps - 1) / Geo::kWarps, (uint64_t)per * (uint64_t)sms));
    decompress_expand_kernel<Geo><<<(unsigned)grid, DX<Geo>::kNT, smem, s>>>(a);
    return cudaGetLastError();
}

struct DxEntry {
    KernelVariant info;
    size_t (*smem)();
    cudaError_t (*launch)(const zs_dict *, const TiledLaunch &, cudaStream_t);
};

template <class Geo>
constexpr DxEntry dx_entry(const char *name)
{
    return DxEntry{KernelVariant{name, Geo::kWarps, Geo::kTile}, &dx_smem<Geo>, &dx_launch<Geo>};
}

const DxEntry kDx[] = {
    dx_entry<DxV0>("decompress expand w24 t2048"),
    dx_entry<DxV1>("decompress expand w20 t2048"),
    dx_entry<DxV2>("decompress expand w28 t2048 global"),
    dx_entry<DxV3>("decompress expand w32 t2048 global"),
};
constexpr int kNumDx = (int)(sizeof(kDx) / sizeof(kDx[0]));

}  // namespace

int expand_variants() { return kNumDx; }

const KernelVariant *expand_variant(int v) { return (v >= 0 && v < kNumDx) ? &kDx[v].info : nullptr; }

bool expand_fits(int v, const zs_dict *d)
{
    if (v < 0 || v >= kNumDx || d->max_plen > 7) return false;  // patterns and length share a 64-bit entry
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return kDx[v].smem() <= (size_t)optin;
}

cudaError_t launch_expand(int v, const zs_dict *d, const TiledLaunch &L, cudaStream_t s)
{
    if (v < 0 || v >= kNumDx) return cudaErrorInvalidValue;
    return kDx[v].launch(d, L, s);
}

}  // namespace zs
