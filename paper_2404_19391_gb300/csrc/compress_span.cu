// zs_compress, span path: ring-ID pre-processing (Sec. IV-A) and the minimum-length parse (Sec. IV-D1) with
// one warp per tile and, within the tile, one contiguous span of whole lines per lane.
//
//   - Tiles and look-back as in the other tiled kernels: each warp of a persistent CTA claims tiles in
//     launch order, stages a tile (plus the byte before it and a halo for the last line) with one bulk
//     (TMA) copy, and resolves its output offset by a warp-wide decoupled look-back, one tile behind the
//     one it encodes (software pipeline).
//   - Token mask: the warp classifies the staged bytes 16 at a time with SIMD byte arithmetic (no table):
//     one bit per byte marks the bytes pre-processing looks at (digits, '%', '[', ']', ' ', tab, '\n'),
//     plus bytes >= 0x80 so that a tile holding any is known.
//   - Spans: lane l owns the lines that start between two boundaries, each the line start closest to
//     l / 32 of the tile, so every lane gets about 1/32 of the bytes whatever the line lengths. In geometries
//     that enable it, a target inside a long line may take a reset point of that line instead (a position
//     after a ring-bond token that leaves no ring open, found by all lanes at once over their own chunks with
//     segmented scans), so one line can be shared by several lanes.
//   - Pre-processing: each lane walks only the token bits of its span (digits inside bracket atoms masked
//     out); ring labels are rewritten in place when a ring closes (or opens, for the other reading), %nn labels
//     shrink (up to six open ones are followed in registers) and the span is compacted. Both relabelling rules
//     restart exactly at a reset point, so the units of a cut line are relabelled independently.
//   - Parse: the backward shortest-path scan is the minimal transducer of the dictionary, re-indexed by
//     the raw byte: per byte one byte-permute builds (state << 8 | 2 * byte) and one 16-bit shared load
//     gives the next state and the symbol chosen there. '\n' resets the state, so a whole span is one
//     scan, and the chosen symbols overwrite the text in place. A span ending at a cut starts from a short
//     read-ahead of the next span and is repaired from the true state (the next span's exit state) until the
//     two scans meet.
//   - Emission: a count walk over the chosen pieces gives each lane's output bytes, a warp scan places
//     them, and a write walk stores them into a per-warp staging buffer (and the line starts into an
//     index stage), which the finishing step copies out with aligned 16-byte stores. A span entered at a cut
//     starts where the previous span's walk left off and joins its own speculative chain where they meet.
//   - A line outside this fast path (a label above 9, more than six open %nn labels, longer than the stage)
//     is coded alone by its lane in global scratch. A cut that cannot be kept makes the tile be coded again
//     without cuts. Anything else (more such lines than a lane follows, an escaped input byte in a compacted
//     span) sets kStFallback, and the call is run again by the general kernel.
#include <algorithm>

#include "compress_shared.cuh"

namespace zs {
namespace {
using namespace cx;

template <int W, int TB, int HB, int OUTB, int MAXL, bool CUT>
struct SpGeom {
    static constexpr bool kCut = CUT;   // long lines are cut between lanes by default
    static constexpr int kWarps = W;    // warps per CTA (one CTA per SM)
    static constexpr int kTile = TB;    // owned input bytes per warp tile
    static constexpr int kHalo = HB;    // bytes staged past the tile for its last line
    static constexpr int kOut = OUTB;   // staged output bytes per tile (more: the tile writes directly)
    static constexpr int kMaxL = MAXL;  // staged index entries per tile (more: the tile writes directly)
};

constexpr unsigned kAll = 0xffffffffu;
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint8_t kDel = 0xFF;           // a deleted byte (digits of a rewritten %nn label); never staged text
constexpr uint32_t kOpen2 = 6;           // open %nn labels (>= 10) a lane follows (in registers)
constexpr uint32_t kChEscDigit = 0x10;   // choice 0x10 + d: escape of the (new) digit d
constexpr uint32_t kChEsc = 0x20;        // choice ' ': escape of the input byte at that position
constexpr uint32_t kPosBits = 13, kPosMask = (1u << kPosBits) - 1u;  // emission walks: position | out bytes << 13
// Aggregate published by a tile that met a line outside the fast path (and by every tile claimed after the
// call was marked for the general kernel): every later tile's output and index offsets then lie past any
// buffer's capacity, so nothing is written past what the general kernel's run will write.
constexpr uint64_t kPoison = 1ull << 40;
constexpr uint32_t kLongLine = 1u << 30;  // a line this long (or longer) is refused (ZS_ERR_INVALID_ARG)

// Launch-wide arguments; the per-shard ones are in the ShardView of each claimed tile.
struct SpArgs {
    ShardView one;
    const ShardView *shards;
    uint32_t n_shards;
    uint32_t flags;
    uint64_t total_tiles;
    const uint8_t *bimg;  // byte transducer image (ByteLayout)
    uint32_t img_bytes;
    uint32_t meta_off;    // offset of meta[256] in the image
    uint32_t q0;          // start state
    uint32_t rep_col;     // 2 * a byte below 0x80 that acts like every byte >= 0x80
    DevResult *g;
    uint8_t *slow;        // scratch of the lines coded one at a time (SlowLayout each)
    uint64_t slow_cap;
    uint64_t limit_ns;
    int64_t stall_tile;
    uint32_t cut_min;     // lines this long (or longer) may be cut between lanes at reset points; 0: never
    uint32_t cut_slack;   // a lane takes a cut only if its target is farther than this from a line start
    uint64_t slots_need;  // bytes of the tile slots at the start of the scratch (lines longer than the stage)
    uint64_t slots_bytes; // slots_need if the scratch holds them (lines are then coded before the launch), else 0
};

// Per-byte SIMD classification (bytes of a 32-bit word; the high bit of each result byte is the answer).
// Bytes >= 0x80 are in no class. Range tests add to the low seven bits, which never carries out of a byte.
struct Classes {
    uint32_t nl, dig, ob, cb, sp;  // '\n'; '0'-'9' and '%' (ring labels); '['; ']'; ' ' or tab
};

__device__ __forceinline__ Classes classify(uint32_t x)
{
    const uint32_t y = x & 0x7F7F7F7Fu, h = 0x80808080u & ~x;
    Classes c;
    c.nl = ~((y ^ 0x0A0A0A0Au) + 0x7F7F7F7Fu) & h;
    c.dig = (((y + 0x50505050u) & ~(y + 0x46464646u)) | ~((y ^ 0x25252525u) + 0x7F7F7F7Fu)) & h;  // 0-9, %
    c.ob = ~((y ^ 0x5B5B5B5Bu) + 0x7F7F7F7Fu) & h;
    c.cb = ~((y ^ 0x5D5D5D5Du) + 0x7F7F7F7Fu) & h;
    c.sp = ~(((y ^ 0x20202020u) + 0x7F7F7F7Fu) & ((y ^ 0x09090909u) + 0x7F7F7F7Fu)) & h;
    return c;
}

// The top bits of the four bytes of a high-bit mask, moved to bits 28..31 (byte i -> bit 28 + i).
__device__ __forceinline__ uint32_t top4(uint32_t hb) { return hb * 0x00204081u; }

// Bit masks of the 16 bytes of a chunk (byte i -> bit i) for each class.
__device__ __forceinline__ void class_bits16(uint4 v, uint32_t *nl, uint32_t *dig, uint32_t *ob, uint32_t *cb,
                                             uint32_t *sp)
{
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    uint32_t n = 0, d = 0, o = 0, c2 = 0, e = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const Classes c = classify(w[k]);
        n = (n >> 4) | (top4(c.nl) & 0xF0000000u);
        d = (d >> 4) | (top4(c.dig) & 0xF0000000u);
        o = (o >> 4) | (top4(c.ob) & 0xF0000000u);
        c2 = (c2 >> 4) | (top4(c.cb) & 0xF0000000u);
        e = (e >> 4) | (top4(c.sp) & 0xF0000000u);
    }
    *nl = n >> 16;
    *dig = d >> 16;
    *ob = o >> 16;
    *cb = c2 >> 16;
    *sp = e >> 16;
}

// Prefix XOR of the bits of x (bit i = XOR of bits 0..i).
__device__ __forceinline__ uint32_t prefix_xor(uint32_t x)
{
    x ^= x << 1;
    x ^= x << 2;
    x ^= x << 4;
    x ^= x << 8;
    x ^= x << 16;
    return x;
}

template <class Geo, bool OUTER>
struct SP {
    static constexpr int kW = Geo::kWarps;
    static constexpr int kNT = 32 * kW;
    static constexpr int kTB = Geo::kTile;
    static constexpr int kHB = Geo::kHalo;
    static constexpr int kSt = 16 + kTB + kHB;  // staged bytes: [0, 16) holds the byte before the tile at 15
    static constexpr int kOutB = Geo::kOut;
    static constexpr int kMaxL = Geo::kMaxL;
    static constexpr int kMaskWords = kSt / 32 + 2;
    static_assert(kTB % 512 == 0 && kHB % 16 == 0 && kOutB % 16 == 0 && kSt + 16 <= (int)kPosMask, "span geometry");

    struct alignas(16) OutSlot {
        uint8_t out[kOutB + 16];
        uint32_t idx[kMaxL];  // tile-relative output offset of each line start (entry 0 = 0)
        uint32_t total;       // output bytes of the tile
        uint32_t lines;       // lines starting in the tile
        uint32_t direct;      // 1: the tile's output did not fit the stage (written at finish time); 2: none
        uint32_t _pad;
        uint64_t t;
        ShardView sv;
    };

    struct alignas(16) WarpMem {
        uint8_t text[kSt + 16];
        uint32_t nmask[kMaskWords];  // one bit per staged byte: '\n'
        uint32_t dmask[kMaskWords];  // digits and '%'
        uint32_t omask[kMaskWords];  // '[', and ' ' tab
        uint32_t cmask[kMaskWords];  // ']', and ' ' tab (a byte in both masks always makes an exception)
        uint16_t ring[20 * 32];  // per lane (entry k of lane l at [k * 32 + l]): open positions of labels 0-9,
                                  // latest closes of new labels 0-9
        OutSlot os[2];
        uint64_t bar;
        uint32_t high;  // the staged tile holds a byte >= 0x80
        uint32_t _pad;
    };

    struct Ctx {
        const SpArgs *P;
        const ShardView *A;
        WarpMem *M;
        const uint8_t *tab;    // transducer table in shared memory
        const uint32_t *meta;  // per choice: input bytes consumed | output bytes << 13
        uint32_t lane;
        uint32_t *status;
    };

    // ---- staging and token mask ---------------------------------------------------------------------
    static __device__ __forceinline__ uint64_t tile_base(uint64_t t) { return t * (uint64_t)kTB; }

    static __device__ __forceinline__ void stage_issue(const Ctx &C, uint64_t t)
    {
        const ShardView &A = *C.A;
        WarpMem &M = *C.M;
        const uint64_t base = tile_base(t);
        const uint64_t stage_hi = min(A.n, base + (uint64_t)kTB + kHB);
        const uint64_t lo = base >= 16 ? base - 16 : 0;
        const uint32_t j0 = (uint32_t)(lo + 16 - base);
        const uint32_t nbytes = (uint32_t)(stage_hi - lo);
        const uint32_t nbulk = A.in_aligned ? (nbytes & ~15u) : 0u;
        __syncwarp();
        if (C.lane == 0) {
            fence_proxy_async_smem();
            mbar_arrive_tx(&M.bar, nbulk);
            if (nbulk) bulk_g2s(M.text + j0, A.in + lo, nbulk, &M.bar);
        }
        for (uint32_t j = nbulk + C.lane; j < nbytes; j += 32) M.text[j0 + j] = A.in[lo + j];
        if (t == 0 && C.lane == 0) M.text[15] = kNl;  // position 0 starts a line
    }

    // Class bits of the staged bytes [16 * c0, 16 * c1) (whole chunks); returns whether any byte >= 0x80.
    static __device__ __forceinline__ bool mask_chunks(const Ctx &C, uint32_t c0, uint32_t c1)
    {
        WarpMem &M = *C.M;
        uint32_t hi = 0;
        uint16_t *n16 = reinterpret_cast<uint16_t *>(M.nmask);
        uint16_t *d16 = reinterpret_cast<uint16_t *>(M.dmask);
        uint16_t *o16 = reinterpret_cast<uint16_t *>(M.omask);
        uint16_t *c16 = reinterpret_cast<uint16_t *>(M.cmask);
        for (uint32_t c = c0 + C.lane; c < c1; c += 32) {
            const uint4 v = *reinterpret_cast<const uint4 *>(M.text + 16 * c);
            hi |= (v.x | v.y | v.z | v.w);
            uint32_t n, d, o, cl, e;
            class_bits16(v, &n, &d, &o, &cl, &e);
            n16[c] = (uint16_t)n;
            d16[c] = (uint16_t)d;
            o16[c] = (uint16_t)(o | e);
            c16[c] = (uint16_t)(cl | e);
        }
        return __any_sync(kAll, (hi & 0x80808080u) != 0);
    }

    // ---- newline searches (every lane on its own) ---------------------------------------------------------
    // First '\n' at a staged position in [p, lim), or kNone.
    static __device__ __forceinline__ uint32_t next_nl(const WarpMem &M, uint32_t p, uint32_t lim)
    {
        while (p < lim) {
            const uint32_t w = p >> 5;
            const uint32_t bits = M.nmask[w] & (kAll << (p & 31));
            if (bits) {
                const uint32_t q = (w << 5) + (uint32_t)(__ffs(bits) - 1);
                return q < lim ? q : kNone;
            }
            p = (w + 1) << 5;
        }
        return kNone;
    }

    // Last '\n' at a staged position in [lo, p), or kNone.
    static __device__ __forceinline__ uint32_t prev_nl(const WarpMem &M, uint32_t p, uint32_t lo)
    {
        while (p > lo) {
            const uint32_t w = (p - 1) >> 5;
            const uint32_t bits = M.nmask[w] & (kAll >> (31u - ((p - 1) & 31u)));
            if (bits) {
                const uint32_t q = (w << 5) + 31u - (uint32_t)__clz(bits);
                return q >= lo ? q : kNone;
            }
            p = w << 5;
        }
        return kNone;
    }

    // Bits of mask m at staged positions [lo, hi) (all of them, one word at a time): their count.
    static __device__ __forceinline__ uint32_t count_bits(const uint32_t *m, uint32_t lo, uint32_t hi)
    {
        uint32_t n = 0;
        for (uint32_t w = lo >> 5; (w << 5) < hi; ++w) {
            uint32_t bits = m[w];
            if ((w << 5) < lo) bits &= kAll << (lo & 31);
            if (((w + 1) << 5) > hi) bits &= (1u << (hi & 31)) - 1u;
            n += __popc(bits);
        }
        return n;
    }

    // ---- spans ------------------------------------------------------------------------------------------
    struct Span {
        uint32_t a, b;      // this lane's lines: staged positions [a, b)
        uint32_t B0, B32;   // the tile's lines: [B0, B32)
        bool long_last;     // the tile's last line runs past the staged bytes
        bool cut_a, cut_b;  // the span starts (ends) inside a line, at a reset point
    };

    // ---- cuts inside long lines ---------------------------------------------------------------------------
    // A reset point is the position just after a ring-bond token (outside bracket atoms, before any space or
    // tab) that leaves no ring open. Both relabelling rules restart there exactly: every earlier ring has closed
    // before any later one opens, so all labels are free again (closing order), or none is held (opening
    // order). A long line can therefore be relabelled in independent units cut at reset points; the parse and
    // the emission walks are mended at each cut afterwards (their state does not restart there).
    static constexpr uint32_t kSync = 20;               // bytes recorded at a cut for the parse repair
    static constexpr uint32_t kLook = 12;               // bytes of the next span read ahead at a cut

    // Ring-token bits of word w within keep: digits and '%' outside bracket atoms and before the first space or
    // tab of their line, given the state at the word's start (inb: inside an atom, fd: past the field), which is
    // advanced to the last kept bit (a newline starts both afresh). The bracket state is the parity of the
    // bracket bytes since the line start; a malformed line only misplaces cuts, which the relabelling catches.
    static __device__ __forceinline__ uint32_t ring_tokens(const WarpMem &M, uint32_t w, uint32_t keep, uint32_t &inb,
                                                           uint32_t &fd)
    {
        const uint32_t om = M.omask[w] & keep, cm = M.cmask[w] & keep;
        const uint32_t sp = om & cm, t = (om | cm) & ~sp, d = M.dmask[w] & keep;
        uint32_t nl = M.nmask[w] & keep, rest = keep, toks = 0;
        while (rest) {
            const uint32_t seg = nl ? rest & ((nl & (0u - nl)) * 2u - 1u) : rest;  // up to the next newline
            const uint32_t ss = sp & seg;
            const uint32_t px = (prefix_xor(t & seg) ^ (0u - inb)) & seg;
            uint32_t live = fd ? 0u : seg;
            if (ss) live &= (ss & (0u - ss)) - 1u;
            toks |= d & live & ~px;
            if (!nl) {
                inb = (px >> (31 - __clz(seg))) & 1u;
                fd |= ss != 0;
                break;
            }
            rest &= ~seg;
            nl &= nl - 1u;
            inb = fd = 0;
        }
        return toks;
    }

    // Walk over the ring tokens and newlines of the chunk [c0, c1) from the given state: label parities P (bit
    // label % 32 of P[label / 32]) and open rings, restarted at each newline. FIND: note the first and last reset
    // points reached. *nl: the chunk holds a newline. skip_to: the two digits of a %nn that starts before c0.
    template <bool FIND>
    static __device__ __forceinline__ void chunk_walk(const WarpMem &M, uint32_t c0, uint32_t c1, uint32_t inb,
                                                      uint32_t fd, uint32_t skip_to, uint32_t P[4], uint32_t &open,
                                                      bool *nl, uint32_t *first, uint32_t *last)
    {
        for (uint32_t w = c0 >> 5; (w << 5) < c1; ++w) {
            uint32_t keep = kAll;
            if ((w << 5) < c0) keep &= kAll << (c0 & 31);
            if (((w + 1) << 5) > c1) keep &= (1u << (c1 & 31)) - 1u;
            const uint32_t n = M.nmask[w] & keep;
            uint32_t ev = ring_tokens(M, w, keep, inb, fd) | n;
            while (ev) {
                const uint32_t b = (uint32_t)(__ffs(ev) - 1), p = (w << 5) + b;
                ev &= ev - 1u;
                if ((n >> b) & 1u) {
                    P[0] = P[1] = P[2] = P[3] = 0;
                    open = 0;
                    skip_to = 0;
                    *nl = true;
                    continue;
                }
                if (p < skip_to) continue;
                const uint32_t ch = M.text[p];
                uint32_t label, end;
                if (ch == '%') {
                    const uint32_t d1 = (uint32_t)M.text[p + 1] - '0', d2 = (uint32_t)M.text[p + 2] - '0';
                    if (d1 > 9 || d2 > 9) continue;  // a bad %: the relabelling finds the line invalid
                    label = d1 * 10 + d2;
                    end = p + 3;
                    skip_to = end;
                } else {
                    label = ch - '0';
                    end = p + 1;
                }
                const uint32_t bit = 1u << (label & 31), q = label >> 5;
                const uint32_t was = (q == 0 ? P[0] : q == 1 ? P[1] : q == 2 ? P[2] : P[3]) & bit;
                P[0] ^= q == 0 ? bit : 0u;
                P[1] ^= q == 1 ? bit : 0u;
                P[2] ^= q == 2 ? bit : 0u;
                P[3] ^= q == 3 ? bit : 0u;
                open = was ? open - 1u : open + 1u;
                if (FIND && open == 0) {
                    if (*first == kNone) *first = end;
                    *last = end;
                }
            }
        }
    }

    // Reset points near the lane targets, all lanes at once. Lane l takes the chunk [c0, c1) between its target
    // and the next one. A first pass gives each chunk's effect on the bracket and field state of its last line,
    // a segmented scan over the lanes (a newline ends a segment) the state at each chunk's start; a second pass
    // and scan do the same for the label parities; a third pass finds the reset points of the chunk. *first and
    // *last: the first and last reset points reached in the chunk (kNone: none).
    static __device__ void chunk_resets(const Ctx &C, uint32_t c0, uint32_t c1, uint32_t *first, uint32_t *last)
    {
        const WarpMem &M = *C.M;
        const uint32_t lane = C.lane;
        c1 = max(c0, c1);
        // pass 1: bracket and field state
        uint32_t inb = 0, fd = 0;
        bool nl = false;
        for (uint32_t w = c0 >> 5; (w << 5) < c1; ++w) {
            uint32_t keep = kAll;
            if ((w << 5) < c0) keep &= kAll << (c0 & 31);
            if (((w + 1) << 5) > c1) keep &= (1u << (c1 & 31)) - 1u;
            nl |= (M.nmask[w] & keep) != 0;
            ring_tokens(M, w, keep, inb, fd);
        }
        uint32_t f = nl ? 1u : 0u;
#pragma unroll
        for (int k = 1; k < 32; k <<= 1) {  // inclusive segmented scan
            const uint32_t i2 = __shfl_up_sync(kAll, inb, k), f2 = __shfl_up_sync(kAll, fd, k);
            const uint32_t g2 = __shfl_up_sync(kAll, f, k);
            if ((int)lane >= k && !f) {
                inb ^= i2;
                fd |= f2;
            }
            if ((int)lane >= k) f |= g2;
        }
        uint32_t inb0 = __shfl_up_sync(kAll, inb, 1), fd0 = __shfl_up_sync(kAll, fd, 1);
        if (lane == 0) inb0 = fd0 = 0;
        // the two digits of a %nn whose '%' lies just before the chunk belong to the previous lane's token
        uint32_t skip_to = 0;
        if (!inb0 && !fd0) {
            if (M.text[c0 - 1] == '%') skip_to = c0 + 2;
            else if (M.text[c0 - 2] == '%' && (uint32_t)(M.text[c0 - 1] - '0') <= 9u) skip_to = c0 + 1;
        }
        // pass 2: label parities
        uint32_t P[4] = {0, 0, 0, 0}, open = 0, dummy = kNone;
        bool nl2 = false;
        chunk_walk<false>(M, c0, c1, inb0, fd0, skip_to, P, open, &nl2, &dummy, &dummy);
        f = nl2 ? 1u : 0u;
#pragma unroll
        for (int k = 1; k < 32; k <<= 1) {
            uint32_t q[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) q[j] = __shfl_up_sync(kAll, P[j], k);
            const uint32_t g2 = __shfl_up_sync(kAll, f, k);
            if ((int)lane >= k && !f) {
#pragma unroll
                for (int j = 0; j < 4; ++j) P[j] ^= q[j];
            }
            if ((int)lane >= k) f |= g2;
        }
        uint32_t P0[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            P0[j] = __shfl_up_sync(kAll, P[j], 1);
            if (lane == 0) P0[j] = 0;
        }
        // pass 3: the reset points
        open = (uint32_t)(__popc(P0[0]) + __popc(P0[1]) + __popc(P0[2]) + __popc(P0[3]));
        *first = *last = kNone;
        bool nl3 = false;
        chunk_walk<true>(M, c0, c1, inb0, fd0, skip_to, P0, open, &nl3, first, last);
    }

    // Tile segmentation and span boundaries. Line starts owned by the tile are staged positions
    // [16, 16 + nown) preceded by '\n'. Lane l's first line is the line start closest to 16 + l * nown / 32.
    // With cut_min > 0, a target inside a line of at least cut_min bytes (ending in the stage) may instead take
    // the closest reset point of that line; an inclusive max over the lanes keeps the boundaries in order.
    static __device__ __forceinline__ Span spans(const Ctx &C, uint64_t t, uint32_t nown, uint32_t stage_end,
                                                 bool stream_end_staged, uint32_t cut_min)
    {
        const WarpMem &M = *C.M;
        const uint32_t lane = C.lane;
        const uint32_t own_nl = 15u + nown;  // newlines at [15, own_nl) open owned lines
        Span s;
        uint32_t B0 = kNone, B32 = kNone;
        bool long_last = false;
        if (lane == 0) {
            const uint32_t q = next_nl(M, 15, own_nl);
            B0 = q == kNone ? kNone : q + 1;
        }
        B0 = __shfl_sync(kAll, B0, 0);
        if (B0 == kNone) {  // no line starts in this tile
            s.a = s.b = s.B0 = s.B32 = 16;
            s.long_last = false;
            s.cut_a = s.cut_b = false;
            return s;
        }
        if (lane == 31) {
            const uint32_t q = next_nl(M, own_nl, stage_end);
            if (q != kNone) {
                B32 = q + 1;
            } else {
                B32 = stage_end;
                long_last = !stream_end_staged;
            }
        }
        B32 = __shfl_sync(kAll, B32, 31);
        long_last = __shfl_sync(kAll, long_last, 31);
        uint32_t Bl = B0;
        const uint32_t target = 16u + (uint32_t)(((uint64_t)lane * nown) >> 5);
        bool want = false;
        uint32_t sm = kNone, sp = B32, le = kNone;
        if (lane > 0) {
            const uint32_t qm = prev_nl(M, target, B0 - 1u);
            const uint32_t qp = next_nl(M, target - 1u, own_nl);
            sm = qm == kNone ? kNone : qm + 1;
            sp = qp == kNone ? B32 : qp + 1;
            Bl = (sm != kNone && target - sm <= sp - target) ? sm : sp;
            // the target's line is [sm, le), le its '\n' (or the end of the data)
            le = qp;
            if (le == kNone) le = long_last ? kNone : (M.text[B32 - 1] == kNl ? B32 - 1u : B32);
            want = cut_min && sm != kNone && le != kNone && sm < target && target < sp && le - sm >= cut_min &&
                   min(target - sm, sp - target) > C.P->cut_slack;
        }
        if (__any_sync(kAll, want)) {
            const uint32_t tn = __shfl_down_sync(kAll, target, 1);  // every lane takes part in the shuffle
            const uint32_t c1 = lane == 31 ? 16u + nown : tn;
            uint32_t first, last;
            chunk_resets(C, lane == 0 ? 16u : target, min(c1, 16u + nown), &first, &last);
            const uint32_t rl = __shfl_up_sync(kAll, last, 1);  // the previous chunk's last reset point
            if (want) {
                uint32_t best = Bl, bd = Bl > target ? Bl - target : target - Bl;
                if (rl != kNone && rl > sm && rl < le) {
                    const uint32_t d = rl > target ? rl - target : target - rl;
                    if (d < bd || (d == bd && rl < best)) {
                        best = rl;
                        bd = d;
                    }
                }
                if (first != kNone && first > sm && first < le) {
                    const uint32_t d = first - target;
                    if (d < bd || (d == bd && first < best)) best = first;
                }
                Bl = best;
            }
        }
        if (lane > 0) Bl = min(max(Bl, B0), B32);
#pragma unroll
        for (int k = 1; k < 32; k <<= 1) {
            const uint32_t v = __shfl_up_sync(kAll, Bl, k);
            if ((int)lane >= k) Bl = max(Bl, v);
        }
        uint32_t Bn = __shfl_down_sync(kAll, Bl, 1);
        if (lane == 31) Bn = B32;
        s.a = Bl;
        s.b = Bn;
        s.B0 = B0;
        s.B32 = B32;
        s.long_last = long_last;
        s.cut_a = Bl < B32 && M.text[Bl - 1] != kNl;
        s.cut_b = __shfl_down_sync(kAll, s.cut_a, 1) && lane < 31;
        return s;
    }

    // ---- lines coded one at a time ---------------------------------------------------------------------
    // A line that needs a ring label above 9, more open %nn labels than a lane follows, or that runs past the
    // staged bytes is coded alone in global scratch (the exact slow pre-processing, then the byte transducer
    // one byte at a time) and emitted from there; the lane's other lines take the fast path around it.
    // Up to kMaxSlow such lines per lane; more make the call run again by the general kernel.
    static constexpr uint32_t kMaxSlow = 2;
    struct Slow {
        uint32_t n;
        uint32_t a[kMaxSlow], b[kMaxSlow];  // staged positions (after compaction) the line occupies
        uint32_t ga[kMaxSlow];              // its first byte as an original staged position
        uint32_t out[kMaxSlow];             // output bytes (with the '\n' of a line past the staged bytes)
        uint64_t ws[kMaxSlow];              // its work space in the scratch (offset), or ~0 if not coded
        uint32_t past;                      // bit k: line k runs past the staged bytes (found in memory)
        uint32_t pre;                       // bit k: line k was coded before the launch (its tile's slot)
    };

    // Allocates need bytes of the scratch after the tile slots; ~0 when they do not fit (the call runs again with
    // more: the first overflow also counts the slots, so that the host's new size holds both).
    static __device__ __forceinline__ uint64_t slow_alloc(const SpArgs *P, uint32_t *status, uint64_t need)
    {
        const unsigned long long o = atomicAdd(&P->g->slow_used, (unsigned long long)need);
        if (P->slots_bytes + o + need > P->slow_cap) {
            if (!(atomicOr(status, kStSlowOverflow) & kStSlowOverflow))
                atomicAdd(&P->g->slow_used, (unsigned long long)P->slots_need);
            return ~0ull;
        }
        return P->slots_bytes + o;
    }

    static __device__ __forceinline__ bool add_slow(Slow &S, uint32_t a, uint32_t b, uint32_t ga, bool past = false)
    {
        if (S.n >= kMaxSlow) return false;
        S.a[S.n] = a;
        S.b[S.n] = b;
        S.ga[S.n] = ga;
        S.out[S.n] = 0;
        S.ws[S.n] = ~0ull;
        if (past) S.past |= 1u << S.n;
        ++S.n;
        return true;
    }

    // Codes the lane's slow lines one at a time in the scratch: the exact slow pre-processing into the work
    // space's text (labels up to 99, any number of %nn), then the byte transducer, last byte first, into its
    // choices; notes each line's output bytes. A work space records {input bytes, coded bytes, '\n' follows}.
    static __device__ void code_slow(const Ctx &C, Slow &SL, uint64_t base)
    {
        const ShardView &A = *C.A;
        const uint8_t *tab = C.tab;
        const uint32_t rep = C.P->rep_col;
        for (uint32_t k = 0; k < SL.n; ++k) {
            if (((SL.past >> k) & 1u) && C.P->slots_bytes) {  // coded before the launch?
                const uint32_t sl = reinterpret_cast<const uint32_t *>(C.P->slow)[A.tile0 + base / (uint64_t)kTB];
                if (sl) {
                    SL.ws[k] = (uint64_t)sl << 4;
                    SL.out[k] = reinterpret_cast<const uint32_t *>(C.P->slow + SL.ws[k])[3];
                    SL.pre |= 1u << k;
                    continue;
                }
            }
            const uint64_t gs = base - 16 + SL.ga[k];  // the line's first byte in memory
            uint64_t glen = SL.b[k] - SL.a[k];
            bool nl_after = false;
            if ((SL.past >> k) & 1u) {  // find its end in memory
                uint64_t ge = base - 16 + SL.ga[k] + glen;
                while (ge < A.n && A.in[ge] != kNl) ++ge;
                nl_after = ge < A.n;
                glen = ge - gs;
            }
            if (glen >= kLongLine) {
                atomicOr(C.status, kStTooBig);
                continue;
            }
            const SlowLayout sl = slow_layout((uint32_t)glen);
            const uint64_t off = slow_alloc(C.P, C.status, sl.need);
            if (off == ~0ull) continue;  // the host retries with a larger scratch
            uint8_t *ws = C.P->slow + off;
            uint8_t *tx = ws + sl.text, *ch = ws + sl.chs;
            uint32_t m;
            if (C.P->flags & ZS_PREPROCESS) {
                m = preprocess_slow(A.in + gs, (uint32_t)glen, tx, ws + sl.tok, reinterpret_cast<int32_t *>(ws + sl.tables),
                                    reinterpret_cast<int32_t *>(ws + sl.tables) + 100, OUTER);
            } else {
                for (uint32_t i = 0; i < (uint32_t)glen; ++i) tx[i] = A.in[gs + i];
                m = (uint32_t)glen;
            }
            uint32_t st = C.P->q0;
            for (uint32_t i = m; i-- > 0;) {
                const uint32_t b = tx[i];
                st = look(tab, st, b >= 0x80u ? rep : (b << 1), 0x3204);
                ch[i] = (uint8_t)(st >> 8);
            }
            uint32_t outb = nl_after ? 1u : 0u;
            for (uint32_t i = 0; i < m;) {
                const uint32_t e = C.meta[ch[i]];
                i += e & kPosMask;
                outb += e >> kPosBits;
            }
            reinterpret_cast<uint32_t *>(ws)[0] = (uint32_t)glen;
            reinterpret_cast<uint32_t *>(ws)[1] = m;
            reinterpret_cast<uint32_t *>(ws)[2] = nl_after ? 1u : 0u;
            SL.out[k] = outb;
            SL.ws[k] = off;
        }
    }

    // Emission of a slow line from its work space at output offset w; returns the offset after it.
    template <class Sink>
    static __device__ uint32_t emit_slow(const Ctx &C, uint64_t wsoff, uint32_t w, Sink &S)
    {
        if (wsoff == ~0ull) return w;
        const uint8_t *ws = C.P->slow + wsoff;
        const uint32_t glen = reinterpret_cast<const uint32_t *>(ws)[0];
        const uint32_t m = reinterpret_cast<const uint32_t *>(ws)[1];
        const bool nl_after = reinterpret_cast<const uint32_t *>(ws)[2] != 0;
        const SlowLayout sl = slow_layout(glen);
        const uint8_t *tx = ws + sl.text, *ch = ws + sl.chs;
        for (uint32_t i = 0; i < m;) {
            const uint32_t c = ch[i];
            i += C.meta[c] & kPosMask;
            if (c > kChEsc) {
                S.put(w++, (uint8_t)c);
            } else {
                S.put(w++, kEsc);
                S.put(w++, c == kChEsc ? tx[i - 1] : (uint8_t)('0' + c - kChEscDigit));
            }
        }
        if (nl_after) S.put(w++, kNl);
        return w;
    }

    // ---- lines coded by the whole warp ----------------------------------------------------------------------
    // A line the lanes cannot code in the stage (longer than the stage, a label above 9, more open %nn labels
    // than a lane follows) is coded by all 32 lanes together in a work space of global scratch:
    //   header (32 bytes): input bytes n, pre-processed bytes m, flags (bit 0: a '\n' follows and is coded with
    //   the line), output bytes, then where the span kernel placed it (address, room); then the copied line (text), its pre-processed form (text2, up to 3n bytes:
    //   a label above 9 takes %nn), the choice and the state at each byte, the class masks (4 words per 32
    //   bytes), a nibble per byte with its digit value, the lane table (first piece, chunk end, output offset)
    //   and the tables of the one-lane exact pre-processing (taken when a label above 9 is needed).
    struct LongLayout {
        uint64_t text, text2, ch, st, masks, dv, table, tok, tables, need;
    };

    static __device__ __forceinline__ LongLayout long_layout(uint32_t n)
    {
        LongLayout L;
        const uint64_t n16 = ((uint64_t)n + 31u) & ~15ull;  // 16 bytes of slack for 16-byte reads
        const uint64_t nw = ((uint64_t)n + 31u) >> 5;
        L.text = 32;
        L.text2 = L.text + n16;
        L.ch = L.text2 + 3ull * n16;
        L.st = L.ch + 3ull * n16;
        L.masks = L.st + 3ull * n16;
        L.dv = L.masks + 16ull * nw;      // a nibble per byte: its digit value, 10 for '%', 15 otherwise
        L.table = L.dv + 16ull * (nw + 1);
        L.tok = L.table + 16ull * 32;
        L.tables = (L.tok + n + 16u + 15u) & ~15ull;
        L.need = (L.tables + 800u + 15u) & ~15ull;
        return L;
    }

    // Position (in the input) of the first '\n' at or after `from`, or the end of the input: all lanes, 512
    // bytes a round.
    static __device__ uint64_t find_nl_warp(const Ctx &C, uint64_t from)
    {
        const ShardView &A = *C.A;
        for (uint64_t base = from; base < A.n; base += 512) {
            const uint64_t p0 = base + 16u * C.lane;
            uint32_t bits = 0;
#pragma unroll
            for (uint32_t j = 0; j < 16; ++j)
                if (p0 + j < A.n && A.in[p0 + j] == kNl) bits |= 1u << j;
            const uint32_t any = __ballot_sync(kAll, bits != 0);
            if (any) {
                const int l = __ffs(any) - 1;
                const uint32_t b = __shfl_sync(kAll, bits, l);
                return base + 16u * (uint32_t)l + (uint32_t)(__ffs(b) - 1);
            }
        }
        return A.n;
    }

    // Copies the line (n bytes at src) into text, zero past its end, and writes its class masks: per 32 bytes,
    // the digits and '%', '[', ']', and space or tab. All lanes, 32 bytes each a round.
    static __device__ void long_copy(const Ctx &C, const uint8_t *src, uint32_t n, uint8_t *text, uint32_t *masks,
                                     uint32_t *dv)
    {
        const uint32_t nw = (n + 31u) >> 5;
        for (uint32_t w = C.lane; w <= nw; w += 32) {
            uint32_t v[8], nib[4] = {~0u, ~0u, ~0u, ~0u}, d = 0, o = 0, cb = 0, s = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                uint32_t x = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t p = 32u * w + 4u * q + j;
                    const uint32_t b = p < n ? src[p] : 0u;
                    x |= b << (8 * j);
                    const uint32_t bit = 1u << (4 * q + j);
                    const uint32_t dg = b - '0';
                    const uint32_t val = dg <= 9u ? dg : (b == '%' ? 10u : 15u);
                    nib[q >> 1] &= ~(0xFu << (4 * (4 * (q & 1) + j))) | (val << (4 * (4 * (q & 1) + j)));
                    if (val != 15u) d |= bit;
                    if (b == '[') o |= bit;
                    if (b == ']') cb |= bit;
                    if (b == ' ' || b == '\t') s |= bit;
                }
                v[q] = x;
            }
            if (w < nw) {
                uint4 *t4 = reinterpret_cast<uint4 *>(text + 32u * w);
                t4[0] = make_uint4(v[0], v[1], v[2], v[3]);
                t4[1] = make_uint4(v[4], v[5], v[6], v[7]);
                *reinterpret_cast<uint4 *>(masks + 4u * w) = make_uint4(d, o, cb, s);
            }
            *reinterpret_cast<uint4 *>(dv + 4u * w) = make_uint4(nib[0], nib[1], nib[2], nib[3]);  // w = nw: all 15
        }
    }

    // Pre-processing of the copied line by one lane (Sec. IV-A, the rules of preprocess_slow), visiting only the
    // bytes the masks mark and reading digit values from the nibbles (the next word's masks and nibbles are
    // loaded while a word is processed): new labels are written into text in place, and the two digits of each
    // %nn label become kDel. open_at/open_nl: 100 entries each, in shared memory. Returns 0: done; 1: done, with
    // %nn digits to squeeze out; 2: the line is left as it is (a bad %, an unclosed ring or atom; text is then
    // restored by the caller); 3: a label above 9 is needed.
    static __device__ uint32_t long_relabel(uint8_t *text, const uint32_t *masks, const uint32_t *dv, uint32_t n,
                                            uint32_t *open_at, uint8_t *open_nl)
    {
        // open_at[label]: open token position + 1 of each input label (bit 30: a %nn token), 0: closed;
        // open_nl[label]: opening order, the new label it took
        for (int k = 0; k < 100; ++k) open_at[k] = 0;
        uint32_t lc[10];  // closing order: latest close position + 1 of each new label
#pragma unroll
        for (int k = 0; k < 10; ++k) lc[k] = 0;
        uint32_t held = 0, nopen = 0, skip_to = 0;
        bool in_br = false, any_pct = false;
        const uint32_t nw = (n + 31u) >> 5;
        uint4 mk = *reinterpret_cast<const uint4 *>(masks), nv = *reinterpret_cast<const uint4 *>(dv);
        for (uint32_t w = 0; w < nw; ++w) {
            const uint4 mk1 = w + 1 < nw ? *reinterpret_cast<const uint4 *>(masks + 4u * (w + 1)) : make_uint4(0, 0, 0, 0);
            const uint4 nv1 = *reinterpret_cast<const uint4 *>(dv + 4u * (w + 1));
            auto nib = [&](uint32_t bit) -> uint32_t {  // digit value of byte bit of this word, bit < 34
                const uint32_t q = bit >> 3, sh = 4u * (bit & 7u);
                const uint32_t x = q == 0 ? nv.x : q == 1 ? nv.y : q == 2 ? nv.z : q == 3 ? nv.w : nv1.x;
                return (x >> sh) & 0xFu;
            };
            uint32_t ev = mk.x | mk.y | mk.z | mk.w;
            bool field_end = false;
            while (ev) {
                const uint32_t bit = (uint32_t)(__ffs(ev) - 1), p = 32u * w + bit, m1 = 1u << bit;
                ev &= ev - 1u;
                if (mk.w & m1) {  // the SMILES field ends at the first space or tab
                    field_end = true;
                    break;
                }
                if (in_br) {
                    if (mk.z & m1) in_br = false;
                    continue;
                }
                if (mk.y & m1) {
                    in_br = true;
                    continue;
                }
                if (!(mk.x & m1) || p < skip_to) continue;
                const uint32_t v0 = nib(bit);
                uint32_t label;
                bool pct = false;
                if (v0 == 10u) {  // '%': two digits must follow
                    if (p + 2 >= n) return 2;
                    const uint32_t d1 = nib(bit + 1), d2 = nib(bit + 2);
                    if (d1 > 9 || d2 > 9) return 2;
                    label = d1 * 10 + d2;
                    pct = true;
                    skip_to = p + 3;
                } else {
                    label = v0;
                }
                const uint32_t op = open_at[label];
                uint32_t nl;
                if (op == 0) {  // opens a ring
                    open_at[label] = (p + 1u) | (pct ? (1u << 30) : 0u);
                    ++nopen;
                    if (!OUTER) continue;
                    const uint32_t fr = ~held & 0x3FFu;
                    if (fr == 0) return 3;
                    nl = (uint32_t)__ffs(fr) - 1u;
                    held |= 1u << nl;
                    open_nl[label] = (uint8_t)nl;
                } else {  // closes the ring opened at o
                    const uint32_t o = (op & 0x3FFFFFFFu) - 1u;
                    open_at[label] = 0;
                    --nopen;
                    if (OUTER) {
                        nl = open_nl[label];
                        held &= ~(1u << nl);
                    } else {
                        nl = 10;
#pragma unroll
                        for (int x = 9; x >= 0; --x)
                            if (lc[x] <= o) nl = (uint32_t)x;
                        if (nl == 10) return 3;
                        text[o] = (uint8_t)('0' + nl);
                        if (op & (1u << 30)) {
                            text[o + 1] = kDel;
                            text[o + 2] = kDel;
                            any_pct = true;
                        }
#pragma unroll
                        for (int x = 0; x < 10; ++x)
                            if ((uint32_t)x == nl) lc[x] = p + 1u;
                    }
                }
                text[p] = (uint8_t)('0' + nl);
                if (pct) {
                    text[p + 1] = kDel;
                    text[p + 2] = kDel;
                    any_pct = true;
                }
            }
            if (field_end) break;
            mk = mk1;
            nv = nv1;
        }
        if (in_br || nopen != 0) return 2;
        return any_pct ? 1u : 0u;
    }

    // Squeezes the kDel bytes out of text[0, n) into out: all lanes, 32 bytes each a round. Returns the length.
    static __device__ uint32_t long_squeeze(const Ctx &C, const uint8_t *text, uint32_t n, uint8_t *out)
    {
        uint32_t base = 0;
        for (uint32_t r0 = 0; r0 < n; r0 += 1024) {
            const uint32_t p0 = r0 + 32u * C.lane;
            uint32_t keep = 0;
            for (uint32_t j = 0; j < 32; ++j) keep += (p0 + j < n && text[p0 + j] != kDel) ? 1u : 0u;
            const uint32_t inc = warp_incl_u32(keep);
            uint32_t o = base + inc - keep;
            for (uint32_t j = 0; j < 32; ++j) {
                const uint32_t p = p0 + j;
                if (p < n && text[p] != kDel) out[o++] = text[p];
            }
            base += __shfl_sync(kAll, inc, 31);
        }
        return base;
    }

    // Backward scan of the pre-processed line text[0, m) in 32 chunks, one a lane (Sec. IV-D1): each lane starts
    // from a read-ahead of the next chunk (16 bytes; exact at the line's end) and keeps the choice and the state
    // at every byte; a chunk whose entry state was wrong is scanned again from the true one (the next chunk's
    // state at its start) until the two scans meet. Returns the chunk length.
    static __device__ uint32_t long_parse(const Ctx &C, const uint8_t *text, uint32_t m, uint8_t *ch, uint8_t *st)
    {
        const uint8_t *tab = C.tab;
        const uint32_t rep = C.P->rep_col, lane = C.lane;
        auto col = [&](uint32_t b) -> uint32_t { return b >= 0x80u ? rep : (b << 1); };
        const uint32_t chunk = (((m + 31u) >> 5) + 15u) & ~15u;
        const uint32_t c0 = min(m, lane * chunk), c1 = min(m, c0 + chunk);
        uint32_t s = C.P->q0;
        for (uint32_t p = min(m, c1 + 16u); p-- > c1;) s = look(tab, s, col(text[p]), 0x3204);
        uint32_t entry = s;
        if (c0 < c1) {  // 16 bytes a load (chunk starts are 16-aligned; text has 16 bytes of slack)
            uint4 v = *reinterpret_cast<const uint4 *>(text + ((c1 - 1u) & ~15u));
            for (uint32_t blk = (c1 - 1u) & ~15u;; blk -= 16u) {
                const uint4 vn = blk > c0 ? *reinterpret_cast<const uint4 *>(text + blk - 16u) : v;  // the next block
                const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int j = 15; j >= 0; --j) {
                    const uint32_t p = blk + (uint32_t)j;
                    if (p < c1) {
                        s = look(tab, s, col((wv[j >> 2] >> (8 * (j & 3))) & 0xFFu), 0x3204);
                        ch[p] = (uint8_t)(s >> 8);
                        st[p] = (uint8_t)s;
                    }
                }
                if (blk == c0) break;
                v = vn;
            }
        }
        uint32_t exitv = s;
        for (int it = 0; it < 32; ++it) {
            const uint32_t T = __shfl_down_sync(kAll, exitv, 1);  // the next chunk's state at its start
            bool changed = false;
            if (lane < 31 && c1 < m && c0 < c1 && (T & 0xFFu) != (entry & 0xFFu)) {
                entry = T;
                uint32_t x = T;
                bool met = false;
                for (uint32_t p = c1; p-- > c0;) {
                    x = look(tab, x, col(text[p]), 0x3204);
                    ch[p] = (uint8_t)(x >> 8);
                    if ((x & 0xFFu) == st[p]) {
                        met = true;
                        break;
                    }
                    st[p] = (uint8_t)x;
                }
                if (!met) {
                    changed = (x & 0xFFu) != (exitv & 0xFFu);
                    exitv = x;
                }
            }
            if (!__any_sync(kAll, changed)) break;
        }
        return chunk;
    }

    // Forward byte reader over a buffer in global memory: 16 bytes a load, the next 16 already requested.
    // Positions only grow; the buffer has 32 bytes of slack past the last position read.
    struct Fwd {
        const uint8_t *b;
        uint32_t blk;
        uint4 cur, nxt;
        __device__ __forceinline__ void start(const uint8_t *base, uint32_t p)
        {
            b = base;
            blk = p & ~15u;
            cur = *reinterpret_cast<const uint4 *>(b + blk);
            nxt = *reinterpret_cast<const uint4 *>(b + blk + 16u);
        }
        __device__ __forceinline__ uint32_t at(uint32_t p)
        {
            while (p >= blk + 16u) {
                blk += 16u;
                cur = nxt;
                nxt = *reinterpret_cast<const uint4 *>(b + blk + 16u);
            }
            const uint32_t q = (p - blk) >> 2, sh = 8u * (p & 3u);
            const uint32_t w = q == 0 ? cur.x : q == 1 ? cur.y : q == 2 ? cur.z : cur.w;
            return (w >> sh) & 0xFFu;
        }
    };

    // Emission walks of the coded line, chunk by chunk: each lane walks the pieces that start in its chunk
    // (Sec. IV-D1), entering at the first piece the previous chunk's walk leaves to it; a lane walks its chunk
    // speculatively from its start, noting where its first 64 positions start pieces, and joins the true chain
    // where the two meet (or walks it out exactly), repeated until no chunk's exit moves. Fills the lane table
    // {first piece, chunk end, output offset} and returns the line's output bytes.
    static __device__ uint32_t long_walk(const Ctx &C, const uint8_t *ch, uint32_t m, uint32_t chunk, uint32_t *table)
    {
        const uint32_t *meta = C.meta, lane = C.lane;
        const uint32_t c0 = min(m, lane * chunk), c1 = min(m, c0 + chunk);
        uint64_t V = 0, E2 = 0;
        uint32_t pos = c0, out = 0;
        Fwd rd;
        if (c0 < c1) rd.start(ch, c0);
        while (pos < c1) {
            const uint32_t mt = meta[rd.at(pos)];
            const uint32_t r = pos - c0;
            if (r < 64u) {
                V |= 1ull << r;
                E2 |= (uint64_t)((mt >> kPosBits) == 2u) << r;
            }
            out += mt >> kPosBits;
            pos += mt & kPosMask;
        }
        const uint32_t out0 = out, x0 = pos;
        uint32_t xend = pos, entry = c0, last_in = kNone;
        for (int it = 0; it < 32; ++it) {
            uint32_t xin = __shfl_up_sync(kAll, xend, 1);
            bool changed = false;
            if (lane > 0 && c0 < c1 && xin != last_in) {
                last_in = xin;
                uint32_t p = xin, extra = 0;
                bool joined = false;
                Fwd rj;
                if (p < c1) rj.start(ch, p);
                while (p < c1) {
                    const uint32_t r = p - c0;
                    if (r < 64u && ((V >> r) & 1ull)) {
                        const uint64_t below = (1ull << r) - 1ull;
                        out = out0 + extra - (uint32_t)(__popcll(V & below) + __popcll(E2 & below));
                        joined = true;
                        break;
                    }
                    const uint32_t mt = meta[rj.at(p)];
                    extra += mt >> kPosBits;
                    p += mt & kPosMask;
                }
                uint32_t nx = x0;
                if (!joined) {
                    out = extra;
                    nx = p;
                }
                changed = nx != xend;
                xend = nx;
                entry = xin;
            }
            if (!__any_sync(kAll, changed)) break;
        }
        if (c0 >= c1) out = 0;
        const uint32_t inc = warp_incl_u32(out);
        *reinterpret_cast<uint4 *>(table + 4u * lane) = make_uint4(entry, c1, inc - out, 0u);
        return __shfl_sync(kAll, inc, 31);
    }

    // Writes the coded line at output offset w: each lane its chunk's pieces at its offset. An escape writes
    // ' ' and the pre-processed byte (or the escaped digit).
    template <class Sink>
    static __device__ void long_emit(const Ctx &C, const uint8_t *ws, uint32_t w, Sink &S)
    {
        const uint32_t n = reinterpret_cast<const uint32_t *>(ws)[0];
        const uint32_t flags = reinterpret_cast<const uint32_t *>(ws)[2];
        const uint32_t total = reinterpret_cast<const uint32_t *>(ws)[3];
        const LongLayout L = long_layout(n);
        const uint8_t *ch = ws + L.ch;
        const uint8_t *text = ws + ((flags & 2u) ? L.text2 : L.text);
        const uint4 row = *reinterpret_cast<const uint4 *>(ws + L.table + 16u * C.lane);
        uint32_t o = w + row.z;
        Fwd rd;
        if (row.x < row.y) rd.start(ch, row.x);
        for (uint32_t p = row.x; p < row.y;) {
            const uint32_t c = rd.at(p);
            p += C.meta[c] & kPosMask;
            if (c > kChEsc) {
                S.put(o++, (uint8_t)c);
            } else {
                S.put(o++, kEsc);
                S.put(o++, c == kChEsc ? text[p - 1] : (uint8_t)('0' + c - kChEscDigit));
            }
        }
        if (C.lane == 0 && (flags & 1u)) S.put(w + total - 1u, kNl);
    }

    // Codes one line [gs, gs + n) of the input with all lanes; nl_after: a '\n' follows, coded with the line.
    // Returns the work space offset (its header holds the output bytes), or ~0 when the scratch is too small
    // (the host runs the call again with more).
    static __device__ uint64_t code_long(const Ctx &C, uint64_t gs, uint32_t n, bool nl_after, uint32_t *tabs)
    {
        const LongLayout L = long_layout(n);
        uint64_t off = 0;
        if (C.lane == 0) off = slow_alloc(C.P, C.status, L.need);
        off = __shfl_sync(kAll, off, 0);
        if (off == ~0ull) return ~0ull;
        uint8_t *ws = C.P->slow + off;
        uint8_t *text = ws + L.text, *text2 = ws + L.text2;
        uint32_t *masks = reinterpret_cast<uint32_t *>(ws + L.masks);
        const uint8_t *src = C.A->in + gs;
        uint32_t *dv = reinterpret_cast<uint32_t *>(ws + L.dv);
        long_copy(C, src, n, text, masks, dv);
        __syncwarp();
        uint32_t m = n, flags = nl_after ? 1u : 0u;
        if (C.P->flags & ZS_PREPROCESS) {
            uint32_t r = 0;
            if (C.lane == 0)  // its tables in the warp's 512 bytes of shared memory
                r = long_relabel(text, masks, reinterpret_cast<const uint32_t *>(ws + L.dv), n, tabs,
                                 reinterpret_cast<uint8_t *>(tabs) + 400);
            r = __shfl_sync(kAll, r, 0);
            __syncwarp();
            if (r == 1) {  // squeeze out the %nn digits
                m = long_squeeze(C, text, n, text2);
                flags |= 2u;
            } else if (r == 2) {  // left as it is: copy it again
                long_copy(C, src, n, text, masks, dv);
            } else if (r == 3) {  // a label above 9: the exact pre-processing, one lane
                if (C.lane == 0)
                    m = preprocess_slow(src, n, text2, ws + L.tok, reinterpret_cast<int32_t *>(ws + L.tables),
                                        reinterpret_cast<int32_t *>(ws + L.tables) + 100, OUTER);
                m = __shfl_sync(kAll, m, 0);
                flags |= 2u;
            }
            __syncwarp();
        }
        const uint8_t *tx = (flags & 2u) ? text2 : text;
        uint8_t *ch = ws + L.ch;
        const uint32_t chunk = long_parse(C, tx, m, ch, ws + L.st);
        __syncwarp();
        const uint32_t total = long_walk(C, ch, m, chunk, reinterpret_cast<uint32_t *>(ws + L.table)) + (nl_after ? 1u : 0u);
        if (C.lane == 0) {
            *reinterpret_cast<uint4 *>(ws) = make_uint4(n, m, flags, total);
            *reinterpret_cast<uint4 *>(ws + 16) = make_uint4(0, 0, 0, 0);  // destination: noted by the span kernel
        }
        __syncwarp();
        return off;
    }

    // ---- pre-processing ---------------------------------------------------------------------------------
    // Open %nn labels (>= 10) of the current line, in registers: slot j holds (label + 1) << 16 | (open position
    // + 1) with bit 15 set (the open token is a written %nn), or 0 when free.
    static constexpr uint32_t kNoSlot = 0xFFu;
    struct OpenPct {
        uint32_t s[kOpen2];
        __device__ __forceinline__ void clear()
        {
#pragma unroll
            for (int j = 0; j < (int)kOpen2; ++j) s[j] = 0;
        }
        // The open entry of label, its slot freed; 0 if label is not open.
        __device__ __forceinline__ uint32_t take(uint32_t label)
        {
            uint32_t e = 0;
#pragma unroll
            for (int j = 0; j < (int)kOpen2; ++j)
                if ((s[j] >> 16) == label + 1u) {
                    e = s[j] & 0xFFFFu;
                    s[j] = 0;
                }
            return e;
        }
        // Records label as opened at position q; false if every slot is taken.
        __device__ __forceinline__ bool put(uint32_t label, uint32_t q)
        {
            bool done = false;
#pragma unroll
            for (int j = 0; j < (int)kOpen2; ++j)
                if (!done && s[j] == 0) {
                    s[j] = ((label + 1u) << 16) | (q + 1u) | 0x8000u;
                    done = true;
                }
            return done;
        }
    };

    // Walks the token bits of the lane's span [a, b) line by line and relabels ring IDs in place (closing
    // order by default: a ring takes, when it closes, the smallest label whose latest ring closed before this
    // one opened; opening order with OUTER: a ring takes, when it opens, the smallest label no open ring
    // holds). A line found invalid at its end (unclosed ring or bracket, bad %) is restored from the input.
    // %nn labels become one digit; their two digits are marked and squeezed out at the line's end, moving
    // the rest of the span down. Returns the span's end after compaction; *lines = lines in the span;
    // *shifted = some line was compacted; *fallback = a line needs the general kernel.
    static __device__ uint32_t relabel_general(const Ctx &C, uint32_t a, uint32_t b, const uint8_t *raw,
                                               uint32_t *lines_out, bool *shifted, bool last_slow, Slow &SL,
                                               bool *fallback, uint32_t cutf, bool *retry)
    {
        WarpMem &M = *C.M;
        uint8_t *text = M.text;
        uint16_t *ring = M.ring + C.lane;  // entry k at ring[32 * k]
        const bool pre = (C.P->flags & ZS_PREPROCESS) != 0;
        uint32_t shift = 0, lines = 0;
        bool fb = false;
        // per-line state
        uint32_t ls = a;  // line start (original positions)
        uint32_t dopen = 0, lcv = 0, held = 0, nopen2 = 0, skip_to = 0;
        bool in_br = false, field_done = false, bad = false, any_pct = false, wrote = false, slow = false;
        bool rt = false;
        OpenPct op;
        op.clear();
        auto finish_line = [&](uint32_t le) {  // le: the line's end (its '\n' or the span end), original
            const uint32_t cls = ls - shift, cle = le - shift;
            const bool split = ((cutf & 1u) && ls == a) || ((cutf & 2u) && le == b);  // a unit of a cut line
            if (split && (slow || bad || in_br || dopen != 0 || nopen2 != 0)) {
                rt = true;  // a cut line the units cannot code alone: the tile is coded again without cuts
            } else if (slow || (last_slow && le == b)) {  // coded alone; its bytes here are skipped
                if (!add_slow(SL, cls, cle, ls, last_slow && le == b)) fb = true;
            } else if (wrote && (bad || in_br || dopen != 0 || nopen2 != 0)) {  // left as it is
                for (uint32_t k = cls; k < cle; ++k) text[k] = raw[k + shift];
            } else if (wrote && any_pct) {  // squeeze out the deleted digits, then move the rest down
                uint32_t w = cls;
                for (uint32_t r = cls; r < cle; ++r) {
                    const uint8_t v = text[r];
                    if (v != kDel) text[w++] = v;
                }
                const uint32_t d = cle - w;
                const uint32_t bend = b - shift;
                for (uint32_t r = cle; r < bend; ++r) text[r - d] = text[r];
                shift += d;
            }
            ++lines;
            ls = le + 1;
            op.clear();
            dopen = lcv = held = nopen2 = 0;
            skip_to = 0;
            in_br = field_done = bad = any_pct = wrote = slow = false;
        };
        if (a < b) {
            uint32_t w = a >> 5;
            uint32_t bits = (M.nmask[w] | M.dmask[w] | M.omask[w] | M.cmask[w]) & (kAll << (a & 31));
            for (;;) {
                while (bits == 0) {
                    ++w;
                    if ((w << 5) >= b) break;
                    bits = M.nmask[w] | M.dmask[w] | M.omask[w] | M.cmask[w];
                }
                if (bits == 0) break;
                const uint32_t p = (w << 5) + (uint32_t)(__ffs(bits) - 1);
                bits &= bits - 1;
                if (p >= b) break;
                const uint32_t q = p - shift;  // current position
                const uint32_t c = text[q];
                if (c == kNl) {
                    finish_line(p);
                    continue;
                }
                if (!pre || field_done || bad || slow || p < skip_to || fb) continue;
                if (c == ' ' || c == '\t') {  // the SMILES field ends at the first space or tab
                    field_done = true;
                    continue;
                }
                if (in_br) {
                    if (c == ']') in_br = false;
                    continue;
                }
                if (c == '[') {
                    in_br = true;
                    continue;
                }
                uint32_t label;
                bool pct = false;
                if (c == '%') {  // %nn: two digits must follow within the line
                    const uint32_t d1 = (uint32_t)text[q + 1] - '0', d2 = (uint32_t)text[q + 2] - '0';
                    if (p + 2 >= b || d1 > 9 || d2 > 9) {
                        bad = true;
                        continue;
                    }
                    label = d1 * 10 + d2;
                    pct = true;
                    skip_to = p + 3;
                } else if (c >= '0' && c <= '9') {
                    label = c - '0';
                } else {
                    continue;  // a byte the token test passes but pre-processing ignores
                }
                // open_e: the ring's open token (position + 1, bit 15: written %nn) if this token closes it;
                // oslot: the entry that keeps an opening token's position
                uint32_t open_e = 0, oslot = label;
                if (label < 10) {
                    if ((dopen >> label) & 1u) open_e = ring[32 * label];
                    dopen ^= 1u << label;
                } else {
                    open_e = op.take(label);
                    if (open_e) {
                        --nopen2;
                    } else if (op.put(label, q)) {
                        oslot = kNoSlot;
                        ++nopen2;
                    } else {
                        slow = true;  // more open %nn labels than the lane follows
                        continue;
                    }
                }
                const bool opening = open_e == 0;
                uint32_t nl;
                if (OUTER) {
                    if (opening) {
                        const uint32_t fr = ~held & 0x3FFu;
                        if (fr == 0) {  // would need a two-digit label
                            slow = true;
                            continue;
                        }
                        nl = (uint32_t)__ffs(fr) - 1u;
                        held |= 1u << nl;
                        if (oslot != kNoSlot) ring[32 * oslot] = (uint16_t)((q + 1) | (pct ? 0x8000u : 0u));
                    } else {
                        nl = (uint32_t)text[(open_e & 0x7FFFu) - 1u] - '0';
                        held &= ~(1u << nl);
                    }
                } else {
                    if (opening) {
                        if (oslot != kNoSlot) ring[32 * oslot] = (uint16_t)((q + 1) | (pct ? 0x8000u : 0u));
                        continue;
                    }
                    const uint32_t o = (open_e & 0x7FFFu) - 1u;  // position of the open token
                    nl = 10;
                    for (uint32_t x = 0; x < 10; ++x) {
                        if (!((lcv >> x) & 1u) || ring[32 * (10 + x)] <= o) {
                            nl = x;
                            break;
                        }
                    }
                    if (nl == 10) {  // would need a two-digit label
                        slow = true;
                        continue;
                    }
                    text[o] = (uint8_t)('0' + nl);
                    if (open_e & 0x8000u) {
                        text[o + 1] = kDel;
                        text[o + 2] = kDel;
                        any_pct = true;
                    }
                    ring[32 * (10 + nl)] = (uint16_t)(q + 1);
                    lcv |= 1u << nl;
                }
                text[q] = (uint8_t)('0' + nl);
                if (pct) {
                    text[q + 1] = kDel;
                    text[q + 2] = kDel;
                    any_pct = true;
                }
                wrote = true;
            }
        }
        if (ls < b) finish_line(b);  // the stream's last line, without '\n' (or a unit ending at a cut)
        *lines_out = lines;
        *shifted = shift != 0;
        *fallback = fb;
        *retry = rt;
        return b - shift;
    }

    // Whether the span [a, b) can take the fast relabelling: no space or tab (a second field), and every
    // bracket atom opens and closes within its line, without nesting. Bit arithmetic over the class masks, one
    // 32-bit word at a time: the prefix XOR of the bracket bits is 1 from a '[' up to its ']'. Space and tab are
    // in both bracket masks, so each one is a '[' inside an atom or a ']' outside one. Digits inside an atom
    // (isotopes, charges, H counts) are not ring labels; the fast relabelling masks them out the same way.
    static __device__ __forceinline__ bool exception_free(const WarpMem &M, uint32_t a, uint32_t b, bool *dig_in)
    {
        uint32_t in = 0;  // inside a bracket atom at the start of the word
        uint32_t bad = 0, din = 0;
        for (uint32_t w = a >> 5; (w << 5) < b; ++w) {
            uint32_t keep = kAll;
            if ((w << 5) < a) keep &= kAll << (a & 31);
            if (((w + 1) << 5) > b) keep &= (1u << (b & 31)) - 1u;
            const uint32_t o = M.omask[w] & keep, c = M.cmask[w] & keep;
            const uint32_t t = o | c;
            const uint32_t px = prefix_xor(t) ^ (0u - in);   // 1 from each '[' up to, not including, its ']'
            const uint32_t before = px ^ t;                  // the state just before each bit
            bad |= (o & before)                              // '[' inside a bracket atom
                   | (c & ~before)                           // ']' outside one (space, tab: always one of
                                                             //  the two, being in both masks)
                   | (M.nmask[w] & keep & px);               // a line ending inside one
            din |= M.dmask[w] & keep & px & ~t;              // a digit inside one (isotope, charge, H count)
            in = (px >> 31) & 1u;
        }
        *dig_in = din != 0;
        return bad == 0 && in == 0;
    }

    // Ring-label bytes (digits and '%') of the line at original positions [ls, le) back to their input
    // bytes, the line sitting `shift` bytes lower in the stage (a line found invalid at its end).
    static __device__ __forceinline__ void restore_digits(const WarpMem &M, uint8_t *text, const uint8_t *raw,
                                                          uint32_t ls, uint32_t le, uint32_t shift)
    {
        for (uint32_t w = ls >> 5; (w << 5) < le; ++w) {
            uint32_t bits = M.dmask[w];
            while (bits) {
                const uint32_t q = (w << 5) + (uint32_t)(__ffs(bits) - 1);
                bits &= bits - 1;
                if (q >= ls && q < le) text[q - shift] = raw[q];
            }
        }
    }

    // Relabelling of the common span (Sec. IV-A): exception-free, no '%', no cut, no line past the stage, no digit
    // inside a bracket atom in the warp. Digit labels only, rewritten in place, nothing to squeeze: the ring
    // opened at o closes at p and takes the smallest label free since o (closing order; five registers hold the
    // latest closes as in relabel_fast) or keeps the label it took when it opened (opening order). A line left
    // with an open ring is put back. Returns false, with the span's digits put back, when it meets a '%' or a
    // line that needs a label above 9: the caller then takes relabel_fast.
    static __device__ __forceinline__ bool relabel_lean(const Ctx &C, uint32_t a, uint32_t b, const uint8_t *raw)
    {
        WarpMem &M = *C.M;
        uint8_t *text = M.text;
        uint16_t *openp = M.ring + C.lane;  // open position + 1 of digit label d at openp[32 * d]
        uint32_t ls = a, dopen = 0, held = 0;
        uint32_t L0 = 0, L1 = 0, L2 = 0, L3 = 0, L4 = 0;
        bool give_up = false;
        uint32_t w = a >> 5;
        uint32_t bits = (M.dmask[w] | M.nmask[w]) & (kAll << (a & 31));
        for (;;) {
            while (bits == 0) {
                ++w;
                if ((w << 5) >= b) break;
                bits = M.dmask[w] | M.nmask[w];
            }
            if (bits == 0) break;
            const uint32_t p = (w << 5) + (uint32_t)(__ffs(bits) - 1);
            bits &= bits - 1;
            if (p >= b) break;
            const uint32_t c = text[p];
            if (c == kNl) {  // end of a line: one with an unclosed ring stays as it is
                if (dopen) restore_digits(M, text, raw, ls, p, 0);
                dopen = held = 0;
                L0 = L1 = L2 = L3 = L4 = 0;
                ls = p + 1u;
                continue;
            }
            const uint32_t d = c - '0';
            if (d > 9u) {  // '%'
                give_up = true;
                break;
            }
            const uint32_t bit = 1u << d;
            if (dopen & bit) {  // closes the ring opened at o
                const uint32_t o = (uint32_t)openp[32 * d] - 1u;
                uint32_t nl;
                if (OUTER) {
                    nl = (uint32_t)text[o] - '0';
                    held &= ~(1u << nl);
                } else {
                    const uint32_t orep = (o * 0x00010001u) | 0x80008000u;
                    const uint32_t g = (((orep - L0) & 0x80008000u) >> 15) | (((orep - L1) & 0x80008000u) >> 14) |
                                       (((orep - L2) & 0x80008000u) >> 13) | (((orep - L3) & 0x80008000u) >> 12) |
                                       (((orep - L4) & 0x80008000u) >> 11);
                    const uint32_t f = (g & 0x1Fu) | ((g >> 11) & 0x3E0u);  // labels free since o, in order
                    if (f == 0) {  // would need a two-digit label
                        give_up = true;
                        break;
                    }
                    nl = (uint32_t)__ffs(f) - 1u;
                    text[o] = (uint8_t)('0' + nl);
                    const uint32_t r = nl < 5 ? nl : nl - 5u;
                    const uint32_t hm = nl < 5 ? 0x0000FFFFu : 0xFFFF0000u;
                    const uint32_t v = ((p + 1u) * 0x00010001u) & hm;
                    L0 = r == 0 ? (L0 & ~hm) | v : L0;
                    L1 = r == 1 ? (L1 & ~hm) | v : L1;
                    L2 = r == 2 ? (L2 & ~hm) | v : L2;
                    L3 = r == 3 ? (L3 & ~hm) | v : L3;
                    L4 = r == 4 ? (L4 & ~hm) | v : L4;
                }
                text[p] = (uint8_t)('0' + nl);
            } else {  // opens a ring
                openp[32 * d] = (uint16_t)(p + 1u);
                if (OUTER) {
                    const uint32_t fr = ~held & 0x3FFu;
                    if (fr == 0) {
                        give_up = true;
                        break;
                    }
                    const uint32_t nl = (uint32_t)__ffs(fr) - 1u;
                    held |= 1u << nl;
                    text[p] = (uint8_t)('0' + nl);
                }
            }
            dopen ^= bit;
        }
        if (give_up) {
            restore_digits(M, text, raw, a, b, 0);
            return false;
        }
        if (dopen) restore_digits(M, text, raw, ls, b, 0);
        return true;
    }

    // Relabelling of an exception-free span: only the digit bits outside bracket atoms (all of them ring labels)
    // and the newlines are visited. Labels
    // of a line are decided as in relabel_general; the latest close of each new label is kept in 16-bit
    // halves of five registers (label x in register x % 5, high half for x >= 5), so finding the smallest
    // label free since the ring opened is five subtractions and one find-first-set, without branches.
    template <bool MASK_ATOMS>  // some digit of the span sits inside a bracket atom: mask them out word by word
    static __device__ __forceinline__ uint32_t relabel_fast(const Ctx &C, uint32_t a, uint32_t b, const uint8_t *raw,
                                                            bool last_slow, Slow &SL, bool *shifted, bool *fallback,
                                                            uint32_t cutf, bool *retry)
    {
        WarpMem &M = *C.M;
        uint8_t *text = M.text;
        // ring[32 * d]: open position + 1 of digit label d (bit 15: written %0d); op: the open %nn labels
        uint16_t *ring = M.ring + C.lane;
        uint32_t ls = a, dopen = 0, held = 0, nopen2 = 0, skip_to = 0, shift = 0;
        uint32_t L0 = 0, L1 = 0, L2 = 0, L3 = 0, L4 = 0;
        bool fb = false, slow = false, bad = false, any_pct = false, rt = false;
        OpenPct op;
        op.clear();
        auto end_line = [&](uint32_t le) {  // le: the line's end (its '\n' or b), an original position
            const uint32_t cls = ls - shift, cle = le - shift;
            const bool split = ((cutf & 1u) && ls == a) || ((cutf & 2u) && le == b);  // a unit of a cut line
            if (split && (slow || bad || dopen != 0 || nopen2 != 0)) {
                rt = true;  // a cut line the units cannot code alone: the tile is coded again without cuts
            } else if (slow || (last_slow && le == b)) {  // coded alone; its bytes here are skipped
                if (!add_slow(SL, cls, cle, ls, last_slow && le == b)) fb = true;
            } else if (bad || dopen != 0 || nopen2 != 0) {  // an unclosed ring or a bad %: left as it is
                restore_digits(M, text, raw, ls, le, shift);
            } else if (any_pct) {  // squeeze out the deleted digits of %nn labels, then move the rest down
                uint32_t w2 = cls;
                for (uint32_t r = cls; r < cle; ++r) {
                    const uint8_t v = text[r];
                    if (v != kDel) text[w2++] = v;
                }
                const uint32_t d = cle - w2, bend = b - shift;
                for (uint32_t r = cle; r < bend; ++r) text[r - d] = text[r];
                shift += d;
            }
            op.clear();
            dopen = held = nopen2 = 0;
            L0 = L1 = L2 = L3 = L4 = 0;
            slow = bad = any_pct = false;
            skip_to = 0;
        };
        // token bits of word w: newlines, and digits and '%' outside bracket atoms (inb: inside one at the
        // word's start; the span is exception-free, so the bracket masks hold only '[' and ']')
        uint32_t inb = 0;
        auto word_tokens = [&](uint32_t w, uint32_t keep) -> uint32_t {
            if (!MASK_ATOMS) return (M.dmask[w] | M.nmask[w]) & keep;
            const uint32_t t = (M.omask[w] | M.cmask[w]) & keep;
            const uint32_t px = prefix_xor(t) ^ (0u - inb);
            inb = px >> 31;
            return ((M.dmask[w] & ~px) | M.nmask[w]) & keep;
        };
        uint32_t w = a >> 5;
        uint32_t bits = word_tokens(w, kAll << (a & 31));
        for (;;) {
            while (bits == 0) {
                ++w;
                if ((w << 5) >= b) break;
                bits = word_tokens(w, kAll);
            }
            if (bits == 0) break;
            const uint32_t p = (w << 5) + (uint32_t)(__ffs(bits) - 1);
            bits &= bits - 1;
            if (p >= b) break;
            const uint32_t q = p - shift;  // where the byte sits now
            const uint32_t c = text[q];
            if (c == kNl) {
                end_line(p);
                ls = p + 1u;
                continue;
            }
            if (slow || bad || p < skip_to) continue;
            uint32_t label;
            bool pct = false;
            if (c == '%') {  // %nn: two digits must follow within the line
                const uint32_t d1 = (uint32_t)text[q + 1] - '0', d2 = (uint32_t)text[q + 2] - '0';
                if (p + 2 >= b || d1 > 9 || d2 > 9) {
                    bad = true;
                    continue;
                }
                label = d1 * 10 + d2;
                pct = true;
                skip_to = p + 3;
            } else {
                label = c - '0';
            }
            uint32_t open_e = 0, oslot = label;  // open_e: the ring's open token if this token closes it
            if (label < 10) {
                if ((dopen >> label) & 1u) open_e = ring[32 * label];
                dopen ^= 1u << label;
            } else {
                open_e = op.take(label);
                if (open_e) {
                    --nopen2;
                } else if (op.put(label, q)) {
                    oslot = kNoSlot;
                    ++nopen2;
                } else {  // more open %nn labels than the lane follows: the line is coded alone
                    slow = true;
                    continue;
                }
            }
            uint32_t nl;
            if (open_e == 0) {  // opens a ring
                if (oslot != kNoSlot) ring[32 * oslot] = (uint16_t)((q + 1u) | (pct ? 0x8000u : 0u));
                if (!OUTER) continue;
                const uint32_t fr = ~held & 0x3FFu;
                if (fr == 0) {  // would need a two-digit label
                    slow = true;
                    continue;
                }
                nl = (uint32_t)__ffs(fr) - 1u;
                held |= 1u << nl;
            } else if (OUTER) {  // closes a ring: it repeats the label taken when it opened
                nl = (uint32_t)text[(open_e & 0x7FFFu) - 1u] - '0';
                held &= ~(1u << nl);
            } else {  // closes the ring opened at o: the smallest label free since o
                const uint32_t o = (open_e & 0x7FFFu) - 1u;
                const uint32_t orep = (o * 0x00010001u) | 0x80008000u;
                const uint32_t g = (((orep - L0) & 0x80008000u) >> 15) | (((orep - L1) & 0x80008000u) >> 14) |
                                   (((orep - L2) & 0x80008000u) >> 13) | (((orep - L3) & 0x80008000u) >> 12) |
                                   (((orep - L4) & 0x80008000u) >> 11);
                const uint32_t f = (g & 0x1Fu) | ((g >> 11) & 0x3E0u);  // labels free since o, in order
                if (f == 0) {  // would need a two-digit label: the line is coded alone
                    slow = true;
                    continue;
                }
                nl = (uint32_t)__ffs(f) - 1u;
                text[o] = (uint8_t)('0' + nl);
                if (open_e & 0x8000u) {
                    text[o + 1] = kDel;
                    text[o + 2] = kDel;
                    any_pct = true;
                }
                const uint32_t r = nl < 5 ? nl : nl - 5u;
                const uint32_t hm = nl < 5 ? 0x0000FFFFu : 0xFFFF0000u;
                const uint32_t v = ((q + 1u) * 0x00010001u) & hm;
                L0 = r == 0 ? (L0 & ~hm) | v : L0;
                L1 = r == 1 ? (L1 & ~hm) | v : L1;
                L2 = r == 2 ? (L2 & ~hm) | v : L2;
                L3 = r == 3 ? (L3 & ~hm) | v : L3;
                L4 = r == 4 ? (L4 & ~hm) | v : L4;
            }
            text[q] = (uint8_t)('0' + nl);
            if (pct) {
                text[q + 1] = kDel;
                text[q + 2] = kDel;
                any_pct = true;
            }
        }
        if (ls < b) end_line(b);  // the span's last line has no '\n' here (or is a unit ending at a cut)
        *shifted = shift != 0;
        *fallback = fb;
        *retry = rt;
        return b - shift;
    }

    // Pre-processing of the lane's span (Sec. IV-A): the fast relabelling when the span allows it, else the
    // general walk. Returns the span's end after compaction; *lines = lines starting in the span (a span that
    // starts at a cut continues the previous lane's line). cutf: bit 0 the span starts at a cut, bit 1 it ends
    // at one; *retry: a unit of a cut line needs what only a whole line can have.
    static __device__ __forceinline__ uint32_t preprocess(const Ctx &C, uint32_t a, uint32_t b, const uint8_t *raw,
                                                          bool last_slow, uint32_t cutf, uint32_t *lines,
                                                          bool *shifted, Slow &SL, bool *fallback, bool *retry)
    {
        const WarpMem &M = *C.M;
        // exception test first, by every lane, so that the choice of masking is warp-wide (lanes taking both
        // forms of the loop would run one after the other)
        bool dig_in = false, ef = false;
        if (a < b && (C.P->flags & ZS_PREPROCESS)) ef = exception_free(M, a, b, &dig_in);
        const bool mask_atoms = __any_sync(kAll, dig_in);
        *lines = a < b ? count_bits(M.nmask, a, b) + (M.text[b - 1] != kNl ? 1u : 0u) - (cutf & 1u) : 0u;
        *shifted = false;
        *fallback = false;
        *retry = false;
        SL.n = 0;
        SL.past = 0;
        SL.pre = 0;
        if (a >= b) return b;
        if (!(C.P->flags & ZS_PREPROCESS)) {
            if (last_slow) {  // the last line runs past the staged bytes: coded alone
                const uint32_t q = prev_nl(M, b, a);
                const uint32_t ls = q == kNone ? a : q + 1u;
                add_slow(SL, ls, b, ls, true);
            }
            return b;
        }
        if (ef) {
            if (!mask_atoms && cutf == 0 && !last_slow && relabel_lean(C, a, b, raw)) return b;
            return mask_atoms ? relabel_fast<true>(C, a, b, raw, last_slow, SL, shifted, fallback, cutf, retry)
                              : relabel_fast<false>(C, a, b, raw, last_slow, SL, shifted, fallback, cutf, retry);
        }
        uint32_t l2 = 0;
        return relabel_general(C, a, b, raw, &l2, shifted, last_slow, SL, fallback, cutf, retry);
    }

    // ---- parse ------------------------------------------------------------------------------------------
    // Table lookup of the byte transducer: entry (next state | choice << 8) at byte offset
    // (state << 8) | (2 * byte XOR (state mod 32) * 4): one byte-permute builds (state << 8) | 2 * byte from the
    // previous entry and the doubled bytes, and the swizzle (the state's low five bits, from the same entry)
    // moves the entry to a bank of its own, so lanes on the same byte in different states do not conflict.
    static __device__ __forceinline__ uint32_t look(const uint8_t *tab, uint32_t prev, uint32_t x2, uint32_t sel)
    {
        return *reinterpret_cast<const uint16_t *>(tab + (__byte_perm(prev, x2, sel) ^ ((prev << 2) & 0x7Cu)));
    }

    // Backward scan of the lane's span [a, e): each byte is replaced by the choice made there. HIGH: the tile
    // holds bytes >= 0x80, which read the column of rep_col (they match no pattern). Returns the last table
    // entry (the state at a in its low byte). rec (a span ending at a cut, where the scan starts from the start
    // state on speculation): the first kSync bytes scanned and the state after each, as byte | state << 8.
    template <bool HIGH>
    static __device__ __forceinline__ uint32_t parse(const Ctx &C, uint32_t a, uint32_t e, uint16_t *rec, uint32_t st)
    {
        uint8_t *text = C.M->text;
        const uint8_t *tab = C.tab;
        const uint32_t rep = C.P->rep_col;
        int32_t p = (int32_t)e - 1;
        const int32_t lo = (int32_t)a;
        auto col = [&](uint32_t b) -> uint32_t { return (HIGH && b >= 0x80u) ? rep : (b << 1); };
        if (rec) {
            for (uint32_t k = 0; k < kSync && p >= lo; ++k, --p) {
                const uint32_t b = text[p];
                st = look(tab, st, col(b), 0x3204);
                text[p] = (uint8_t)(st >> 8);
                rec[32 * k] = (uint16_t)(b | (st << 8));
            }
        }
        while (p >= lo && ((p + 1) & 3) != 0) {
            st = look(tab, st, col(text[p]), 0x3204);
            text[p] = (uint8_t)(st >> 8);
            --p;
        }
        while (p - 3 >= lo) {
            const int32_t wp = p - 3;
            const uint32_t x = *reinterpret_cast<const uint32_t *>(text + wp);
            uint32_t x2;
            if (HIGH) {
                x2 = (x & 0x7F7F7F7Fu) << 1;
                const uint32_t hb = x & 0x80808080u;
                if (hb) {
                    const uint32_t hm = (hb >> 7) * 0xFFu;
                    x2 = (x2 & ~hm) | ((rep * 0x01010101u) & hm);
                }
            } else {
                x2 = (x + x) & 0xFEFEFEFEu;  // every byte is below 0x80; the mask keeps each address even
            }
            const uint32_t e3 = look(tab, st, x2, 0x3207);
            const uint32_t e2 = look(tab, e3, x2, 0x3206);
            const uint32_t e1 = look(tab, e2, x2, 0x3205);
            const uint32_t e0 = look(tab, e1, x2, 0x3204);
            *reinterpret_cast<uint32_t *>(text + wp) =
                __byte_perm(__byte_perm(e0, e1, 0x0051), __byte_perm(e2, e3, 0x0051), 0x5410);
            st = e0;
            p -= 4;
        }
        while (p >= lo) {
            st = look(tab, st, col(text[p]), 0x3204);
            text[p] = (uint8_t)(st >> 8);
            --p;
        }
        return st;
    }

    // State at a cut, read ahead from the bytes [b0, lim) that follow it (the start of the next span): exact if
    // they hold a newline (the scan starts there), else a guess that the repair below checks.
    template <bool HIGH>
    static __device__ __forceinline__ uint32_t lookahead(const Ctx &C, uint32_t b0, uint32_t lim)
    {
        const uint8_t *text = C.M->text;
        const uint32_t rep = C.P->rep_col;
        for (uint32_t p = b0; p < lim; ++p)
            if (text[p] == kNl) {
                lim = p + 1;
                break;
            }
        uint32_t st = C.P->q0;
        for (uint32_t p = lim; p-- > b0;) {
            const uint32_t b = text[p];
            st = look(C.tab, st, (HIGH && b >= 0x80u) ? rep : (b << 1), 0x3204);
        }
        return st;
    }

    // Repair of a span that ends at a cut: the recorded bytes are scanned again from the true state there (the
    // state the next span's scan reached at its start), rewriting their choices, until the state meets the one
    // the speculative scan had at the same byte; from there on the two scans agree. lo: the start of the scan
    // that ends at the cut. Returns false if they do not meet within the recorded bytes.
    template <bool HIGH>
    static __device__ bool repair_parse(const Ctx &C, uint32_t e, uint32_t lo, uint32_t st, const uint16_t *rec)
    {
        uint8_t *text = C.M->text;
        const uint8_t *tab = C.tab;
        const uint32_t rep = C.P->rep_col;
        int32_t p = (int32_t)e - 1;
        for (uint32_t k = 0; k < kSync && p >= (int32_t)lo; ++k, --p) {
            const uint32_t r = rec[32 * k];
            const uint32_t b = r & 0xFFu;
            st = look(tab, st, (HIGH && b >= 0x80u) ? rep : (b << 1), 0x3204);
            text[p] = (uint8_t)(st >> 8);
            if ((st & 0xFFu) == (r >> 8)) return true;
        }
        return false;
    }

    // ---- emission ---------------------------------------------------------------------------------------
    // Walk over the pieces chosen along [a, e): returns position | output bytes << 13 after the last piece (the
    // position may lie past e, inside the piece that crosses it). *gen_esc: an escape of an input byte was chosen.
    // head (a span starting at a cut, entered on speculation): *V gets bit r for each of the first 64 positions
    // a + r where a piece starts, *E2 bit r where that piece emits two bytes.
    static __device__ __forceinline__ uint32_t count_out(const Ctx &C, uint32_t a, uint32_t e, bool check, bool *gen_esc,
                                                         bool head = false, uint64_t *V = nullptr, uint64_t *E2 = nullptr)
    {
        const uint8_t *text = C.M->text;
        const uint32_t *meta = C.meta;
        uint32_t acc = a;
        bool ge = false;
        if (head) {
            uint64_t v = 0, e2 = 0;
            while ((acc & kPosMask) < e) {
                const uint32_t pos = acc & kPosMask, r = pos - a;
                if (r >= 64) break;
                const uint32_t c = text[pos];
                const uint32_t m = meta[c];
                v |= 1ull << r;
                e2 |= (uint64_t)((m >> kPosBits) == 2u) << r;
                ge |= c == kChEsc;
                acc += m;
            }
            *V = v;
            *E2 = e2;
        }
        if (!check) {
            while ((acc & kPosMask) < e) acc += meta[text[acc & kPosMask]];
        } else {
            while ((acc & kPosMask) < e) {
                const uint32_t c = text[acc & kPosMask];
                ge |= c == kChEsc;
                acc += meta[c];
            }
        }
        *gen_esc = ge;
        return acc;
    }

    struct SmemOut {
        uint8_t *o;
        uint32_t *idx;
        uint32_t nidx;
        __device__ __forceinline__ void put(uint32_t w, uint8_t v) { o[w] = v; }
        __device__ __forceinline__ void line(uint32_t r, uint32_t w) { if (r < nidx) idx[r] = w; }
        __device__ __forceinline__ void long_dst(uint8_t *, uint32_t) {}  // such tiles are never staged
    };
    struct GlobalOut {  // direct writes: output offset ea, lines from eb
        uint8_t *out;
        uint64_t cap, ea;
        uint64_t *index;
        uint64_t index_cap, eb;
        uint32_t nlines;
        __device__ __forceinline__ void put(uint32_t w, uint8_t v)
        {
            if (ea + w < cap) out[ea + w] = v;
        }
        __device__ __forceinline__ void line(uint32_t r, uint32_t w)
        {
            if (index && r < nlines && eb + r < index_cap) index[eb + r] = ea + w;
        }
        // a line coded before the launch: its destination and room, for the patch kernel (header bytes 16-31)
        __device__ __forceinline__ void long_dst(uint8_t *ws, uint32_t w)
        {
            uint64_t *h = reinterpret_cast<uint64_t *>(ws + 16);
            h[0] = reinterpret_cast<uint64_t>(out + ea + w);
            h[1] = ea + w < cap ? cap - (ea + w) : 0;
        }
    };

    struct LongSink {  // a line coded before the launch, written at dst (room bytes)
        uint8_t *dst;
        uint64_t room;
        __device__ __forceinline__ void put(uint32_t w, uint8_t v)
        {
            if (w < room) dst[w] = v;
        }
    };

    // Write walk of the span [a, e) from output offset w, the lane's first line being line `rank` of the
    // tile: symbols as they are, escapes as ' ' + byte, and each new line's start offset.
    template <class Sink>
    static __device__ __forceinline__ void write_out(const Ctx &C, uint32_t a, uint32_t e, uint32_t &w, uint32_t &rank,
                                                     const uint8_t *raw, Sink &S)
    {
        const uint8_t *text = C.M->text;
        const uint32_t *meta = C.meta;
        uint32_t acc = a;
        while ((acc & kPosMask) < e) {
            const uint32_t i = acc & kPosMask;
            const uint32_t c = text[i];
            acc += meta[c];
            if (c > kChEsc) {
                S.put(w++, (uint8_t)c);
            } else if (c == kNl) {
                S.put(w++, kNl);
                S.line(++rank, w);
            } else {
                S.put(w++, kEsc);
                S.put(w++, c == kChEsc ? raw[i] : (uint8_t)('0' + c - kChEscDigit));
            }
        }
    }

    // ---- one tile -----------------------------------------------------------------------------------------
    struct Enc {
        uint32_t a, e;      // the lane's span after pre-processing
        uint32_t entry;     // where its first piece starts (past a for a span entered at a cut)
        uint32_t off;       // its output offset within the tile
        uint32_t rank;      // the line its first piece belongs to, within the tile
        uint32_t total, lines;
        bool retry;         // a cut could not be kept: the tile is staged and coded again without cuts
        Slow sl;            // its lines coded one at a time (skipped by the walks over the span)
    };

    // The walks over the lane's span, around its slow lines: parse (returns the span's exit state, the state
    // at its start), output bytes, writes.
    template <bool HIGH>
    static __device__ __forceinline__ uint32_t parse_all(const Ctx &C, const Enc &E, uint16_t *rec, uint32_t st0)
    {
        uint32_t p = E.a, x = 0;
        for (uint32_t k = 0; k < E.sl.n; ++k) {
            const uint32_t st = parse<HIGH>(C, p, E.sl.a[k], nullptr, C.P->q0);
            if (k == 0) x = st;
            p = E.sl.b[k];
        }
        const uint32_t st = parse<HIGH>(C, p, E.e, rec, st0);
        return E.sl.n ? x : st;
    }

    // Output bytes of the span; *xend: where the walk of its last stretch ended (a position past e when the
    // piece crossing a cut runs into the next span). head, V, E2: as count_out, for the span's first stretch.
    static __device__ __forceinline__ uint32_t count_all(const Ctx &C, const Enc &E, bool check, bool *gen_esc,
                                                         uint32_t *xend, bool head, uint64_t *V, uint64_t *E2,
                                                         uint32_t *n1)
    {
        uint32_t p = E.a, n = 0;
        bool ge = false, g2 = false;
        for (uint32_t k = 0; k < E.sl.n; ++k) {
            const uint32_t c = count_out(C, p, E.sl.a[k], check, &g2, head && k == 0, V, E2) >> kPosBits;
            if (k == 0) *n1 = c;
            n += c + E.sl.out[k];
            ge |= g2;
            p = E.sl.b[k];
        }
        const uint32_t acc = count_out(C, p, E.e, check, &g2, head && E.sl.n == 0, V, E2);
        if (E.sl.n == 0) *n1 = acc >> kPosBits;
        n += acc >> kPosBits;
        *xend = acc & kPosMask;
        *gen_esc = ge | g2;
        return n;
    }

    template <class Sink>
    static __device__ __forceinline__ void write_all(const Ctx &C, const Enc &E, const uint8_t *raw, Sink &S)
    {
        uint32_t w = E.off, rank = E.rank, p = E.entry;
        for (uint32_t k = 0; k < E.sl.n; ++k) {
            write_out(C, p, E.sl.a[k], w, rank, raw, S);
            if ((E.sl.pre >> k) & 1u) {
                S.long_dst(C.P->slow + E.sl.ws[k], w);
                w += E.sl.out[k];
            } else {
                w = emit_slow(C, E.sl.ws[k], w, S);
            }
            p = E.sl.b[k];
        }
        write_out(C, p, E.e, w, rank, raw, S);
    }

    // Everything up to the tile's aggregate: masks, spans, pre-processing, parse, sizes (and, when the tile
    // fits its stage, the staged output). Publishes the aggregate, unless a cut could not be kept (E.retry:
    // nothing published, the stage overwritten; the caller stages the tile again and codes it without cuts).
    static __device__ Enc encode(const Ctx &C, OutSlot &O, uint64_t t, bool cuts)
    {
        const ShardView &A = *C.A;
        WarpMem &M = *C.M;
        const uint32_t lane = C.lane;
        const uint64_t base = tile_base(t);
        const uint32_t nown = (uint32_t)(min(A.n, base + kTB) - base);
        const uint64_t stage_hi = min(A.n, base + (uint64_t)kTB + kHB);
        const uint32_t stage_end = (uint32_t)(stage_hi - base) + 16u;
        const uint8_t *raw = A.in + base - 16;  // global address of staged position 0
        bool high = mask_chunks(C, 0, (16u + nown + 15u) >> 4);
        // end of the tile's last line: the first '\n' at or after the last owned byte
        uint32_t lastnl = kNone;
        for (uint32_t off = (15u + nown) & ~15u; off < stage_end; off += 512) {
            const uint32_t p0 = off + 16u * lane;
            uint32_t bits = 0;
            if (p0 < stage_end) {
                bits = nl_bits16(*reinterpret_cast<const uint4 *>(M.text + p0));
                if (p0 < 15u + nown) bits &= kAll << (15u + nown - p0);
                if (p0 + 16u > stage_end) bits &= (1u << (stage_end - p0)) - 1u;
            }
            lastnl = __reduce_min_sync(kAll, bits ? p0 + (uint32_t)(__ffs(bits) - 1) : kNone);
            if (lastnl != kNone) break;
        }
        const uint32_t tail_end = lastnl != kNone ? lastnl + 1u : stage_end;
        high |= mask_chunks(C, (16u + nown) >> 4, (tail_end + 15u) >> 4);
        // the tile's last line runs past the halo: lane 31 codes it alone, reading it from memory
        const bool past = lastnl == kNone && stage_hi != A.n;
        const Span sp = spans(C, t, nown, tail_end, stage_hi == A.n, cuts ? C.P->cut_min : 0u);
        const uint32_t cutf = (sp.cut_a ? 1u : 0u) | (sp.cut_b ? 2u : 0u);
        const bool any_cut = __any_sync(kAll, cutf != 0);
        Enc E;
        uint32_t lines = 0;
        bool shifted = false, fb = false, rt = false;
        E.a = sp.a;
        E.retry = false;
        E.e = preprocess(C, sp.a, sp.b, raw, past && sp.a < sp.b && sp.b == sp.B32, cutf, &lines, &shifted, E.sl,
                         &fb, &rt);
        E.entry = E.a;
        __syncwarp();
        if (E.sl.n) code_slow(C, E.sl, base);
        uint16_t *rec = (cutf & 2u) ? M.ring + lane : nullptr;  // the relabelling is done with the ring entries
        const uint32_t ne = __ballot_sync(kAll, sp.a < sp.b);  // lanes with a span
        const uint32_t nx = ne & ~((2u << lane) - 1u), pv = ne & ((1u << lane) - 1u);
        const int next_lane = nx ? __ffs(nx) - 1 : (int)lane, prev_lane = pv ? 31 - __clz(pv) : (int)lane;
        uint32_t st0 = C.P->q0;
        if (any_cut) {  // a span ending at a cut starts its scan from a short read-ahead into the next span
            const uint32_t nend = __shfl_sync(kAll, E.e, next_lane);
            if ((cutf & 2u) && sp.a < sp.b)
                st0 = high ? lookahead<true>(C, sp.b, min(nend, sp.b + kLook)) : lookahead<false>(C, sp.b, min(nend, sp.b + kLook));
            __syncwarp();  // read before the next span's scan overwrites it
        }
        const uint32_t xst = high ? parse_all<true>(C, E, rec, st0) : parse_all<false>(C, E, rec, st0);
        if (any_cut) {  // the parse at each cut: the true state there is the next span's exit state
            const uint32_t T = __shfl_sync(kAll, xst, next_lane);
            if ((cutf & 2u) && sp.a < sp.b) {
                const uint32_t lo = E.sl.n ? E.sl.b[E.sl.n - 1] : E.a;
                const bool ok = high ? repair_parse<true>(C, E.e, lo, T, rec) : repair_parse<false>(C, E.e, lo, T, rec);
                rt |= !ok;
            }
        }
        bool gen_esc = false;
        uint32_t xend = 0, n1 = 0;
        uint64_t V = 0, E2 = 0;
        uint32_t ob = count_all(C, E, shifted, &gen_esc, &xend, (cutf & 1u) != 0, &V, &E2, &n1);
        if (any_cut) {
            // the walk at each cut: a span entered at a cut starts where the previous span's walk left it (its
            // exit, past the cut, as a position of this span), joins its own speculative chain where the two
            // meet, and walks its first stretch out exactly if they do not meet within 64 bytes. A changed exit
            // changes the next span's entry: repeat until no exit changes.
            const uint32_t ob0 = ob, x0 = xend;
            uint32_t last_in = kNone;
            for (int it = 0; it < 32; ++it) {
                const uint32_t xo = (cutf & 2u) ? xend - E.e + sp.b : 0u;
                const uint32_t xin = __shfl_sync(kAll, xo, prev_lane);
                bool changed = false;
                if ((cutf & 1u) && sp.a < sp.b && xin != last_in) {
                    last_in = xin;
                    const uint32_t lim = E.sl.n ? E.sl.a[0] : E.e;
                    uint32_t pos = xin, extra = 0;
                    bool joined = false;
                    while (pos < lim) {
                        const uint32_t r = pos - E.a;
                        if (r < 64u && ((V >> r) & 1ull)) {
                            const uint64_t below = (1ull << r) - 1ull;
                            ob = ob0 + extra - (uint32_t)(__popcll(V & below) + __popcll(E2 & below));
                            joined = true;
                            break;
                        }
                        const uint32_t c = M.text[pos];
                        const uint32_t m = C.meta[c];
                        gen_esc |= c == kChEsc;
                        extra += m >> kPosBits;
                        pos += m & kPosMask;
                    }
                    uint32_t nx_end = x0;
                    if (!joined) {
                        ob = ob0 - n1 + extra;
                        if (E.sl.n == 0) nx_end = pos;
                    }
                    changed = nx_end != xend;
                    xend = nx_end;
                    E.entry = xin;
                }
                if (!__any_sync(kAll, changed)) break;
            }
        }
        if (__any_sync(kAll, rt)) {
            E.retry = true;
            return E;
        }
        fb |= shifted && gen_esc;  // an escaped input byte no longer sits at its input position
        fb = __any_sync(kAll, fb);
        if (fb && lane == 0) atomicOr(C.status, kStFallback);
        const uint32_t oinc = warp_incl_u32(ob), linc = warp_incl_u32(lines);
        E.off = oinc - ob;
        E.rank = linc - lines - (cutf & 1u);  // a span entered at a cut starts inside the previous lane's line
        E.total = __shfl_sync(kAll, oinc, 31);
        E.lines = __shfl_sync(kAll, linc, 31);
        const bool staged = !fb && E.total + 16u <= (uint32_t)kOutB && E.lines <= (uint32_t)kMaxL &&
                            !__any_sync(kAll, E.sl.pre != 0);  // a line coded before: written by the patch kernel
        if (staged) {
            SmemOut so{O.out, O.idx, E.lines};
            if (lane == 0) O.idx[0] = 0;
            write_all(C, E, raw, so);
        }
        if (fb) {  // the call is run again by the general kernel: this tile and every later one write nothing
            E.total = E.lines = 0;
            E.e = E.a;
            E.sl.n = 0;
        }
        if (lane == 0) {
            O.total = E.total;
            O.lines = E.lines;
            O.direct = fb ? 2u : (staged ? 0u : 1u);  // 2: nothing left to do (poison published)
            O.t = t;
            if ((int64_t)t != C.P->stall_tile) {
                if (fb) publish(&A.tiles[t], 2u, kPoison, kPoison);
                else publish(&A.tiles[t], t == 0 ? 2u : 1u, E.total, E.lines);
            }
        }
        __syncwarp();
        return E;
    }

    static __device__ __forceinline__ void finish_result(const Ctx &C, uint64_t t, uint64_t tot_a, uint64_t tot_b)
    {
        const ShardView &A = *C.A;
        if (C.lane == 0 && t == A.ntiles - 1) {
            A.res->out_len = tot_a;
            A.res->n_lines = tot_b;
            if (A.index && tot_b < A.index_cap) A.index[tot_b] = tot_a;
        }
    }

    // Output offset by look-back, then the staged output and index.
    static __device__ void finish_staged(const Ctx &C, OutSlot &O)
    {
        const ShardView &A = *C.A;
        const uint64_t t = O.t;
        uint64_t ea = 0, eb = 0;
        if (t > 0) lookback_warp(A.tiles, t, &ea, &eb, C.P->limit_ns, C.status);
        const uint32_t total = O.total, lines = O.lines;
        if (C.lane == 0 && t > 0 && (int64_t)t != C.P->stall_tile) publish(&A.tiles[t], 2u, ea + total, eb + lines);
        if (total) warp_copy_realign(O.out, total, A.out + ea, A.out_cap > ea ? A.out_cap - ea : 0);
        if (A.index)
            for (uint32_t r = C.lane; r < lines; r += 32)
                if (eb + r < A.index_cap) A.index[eb + r] = ea + O.idx[r];
        finish_result(C, t, ea + total, eb + lines);
        __syncwarp();
    }

    // A tile whose output or lines do not fit the stage: look back first, then write straight to memory.
    static __device__ void finish_direct(const Ctx &C, OutSlot &O, const Enc &E)
    {
        const ShardView &A = *C.A;
        const uint64_t t = O.t;
        uint64_t ea = 0, eb = 0;
        if (t > 0) lookback_warp(A.tiles, t, &ea, &eb, C.P->limit_ns, C.status);
        if (C.lane == 0 && t > 0 && (int64_t)t != C.P->stall_tile)
            publish(&A.tiles[t], 2u, ea + E.total, eb + E.lines);
        if (C.lane == 0 && A.index && E.lines > 0 && eb < A.index_cap) A.index[eb] = ea;
        GlobalOut go{A.out, A.out_cap, ea, A.index, A.index_cap, eb, E.lines};
        write_all(C, E, A.in + tile_base(t) - 16, go);
        finish_result(C, t, ea + E.total, eb + E.lines);
        __syncwarp();
    }

    // ---- lines longer than the stage: coded before the span kernel, written after it ----------------------
    // The tile slots (one uint32 per tile of the launch, at the start of the scratch) hold the work space (offset
    // / 16) of the tile's last line when that line runs past the tile's stage: the span kernel takes its size
    // from there and the patch kernel writes its bytes. Nothing waits on these lines while they are coded.
    static constexpr int kPreWarps = 8;
    static constexpr uint32_t kPreTab = 512;  // bytes of relabelling tables per warp

    static __host__ __device__ size_t pre_smem(uint32_t img_bytes)  // called by the launch
    {
        return ((img_bytes + 127u) & ~127u) + kPreWarps * (sizeof(ShardView) + kPreTab);
    }

    // Whether the last line of tile t of shard A runs past the tile's stage, and where that line starts: a '\n'
    // neither at or after the last owned byte within the stage, nor the stage at the end of the input. The
    // probe of four tiles at once (each lane 16 bytes of each) is done by precode_run.
    static __device__ void precode_run(const SpArgs *P)
    {
        extern __shared__ __align__(128) uint8_t smem[];
        __shared__ uint64_t img_bar;
        const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        uint8_t *img = smem;
        ShardView *svs = reinterpret_cast<ShardView *>(smem + ((P->img_bytes + 127u) & ~127u));
        uint32_t *tabs = reinterpret_cast<uint32_t *>(reinterpret_cast<uint8_t *>(svs + kPreWarps) + wid * kPreTab);
        Ctx C;
        C.P = P;
        C.A = &svs[wid];
        C.M = nullptr;
        C.tab = img;
        C.meta = reinterpret_cast<const uint32_t *>(img + P->meta_off);
        C.lane = lane;
        C.status = &P->g->status;
        if (threadIdx.x == 0) mbar_init(&img_bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_arrive_tx(&img_bar, P->img_bytes);
            bulk_g2s(img, P->bimg, P->img_bytes, &img_bar);
        }
        const bool ok = mbar_wait_bounded(&img_bar, 0, P->limit_ns, C.status);
        if (!__syncthreads_and(ok)) {
            mbar_wait_bounded(&img_bar, 0, P->limit_ns, C.status);
            return;
        }
        uint32_t *slot = reinterpret_cast<uint32_t *>(P->slow);
        const uint64_t nwarps = (uint64_t)gridDim.x * kPreWarps;
        // each warp a contiguous run of tiles, so that the shard changes rarely; eight tiles a round, four lanes
        // a tile, each lane 16 of the 64 bytes from the tile's last owned byte (the first '\n' after it is
        // nearly always there); a tile without one there is probed over its whole stage window on its own
        const uint64_t per = (P->total_tiles + nwarps - 1) / nwarps;
        const uint64_t g_begin = ((uint64_t)blockIdx.x * kPreWarps + wid) * per;
        const uint64_t g_end = min(P->total_tiles, g_begin + per);
        uint64_t s_t0 = 1, s_t1 = 0;  // tiles [s_t0, s_t1) of the cached shard
        uint32_t sh = 0;
        for (uint64_t g0 = g_begin; g0 < g_end; g0 += 8) {
            if (g0 < s_t0 || g0 >= s_t1) {
                sh = P->n_shards == 1 ? 0u : find_shard(P->shards, P->n_shards, g0);
                const ShardView &S0 = P->n_shards == 1 ? P->one : P->shards[sh];
                s_t0 = S0.tile0;
                s_t1 = S0.tile0 + S0.ntiles;
            }
            const ShardView &A0 = P->n_shards == 1 ? P->one : P->shards[sh];
            const uint32_t j = C.lane >> 2, q = C.lane & 3u;
            const uint64_t g = g0 + j;
            bool mine = false, cand = false, f = false;
            if (g < g_end && g < s_t1) {  // tiles of the cached shard (the rest are taken next round)
                mine = true;
                const uint64_t base = (g - A0.tile0) * (uint64_t)kTB;
                const uint64_t own_end = min(A0.n, base + kTB), stage_hi = min(A0.n, base + kTB + kHB);
                cand = stage_hi < A0.n;
                if (cand) {
                    const uint64_t p0 = own_end - 1 + 16u * q;
#pragma unroll
                    for (uint32_t i = 0; i < 16; ++i)
                        if (p0 + i < stage_hi && A0.in[p0 + i] == kNl) f = true;
                }
            }
            if (mine && q == 0) slot[g] = 0;  // set below if the line is coded
            // a tile is done when one of its four lanes saw a '\n' or it is not a candidate
            const uint32_t seen = __ballot_sync(kAll, f), cands = __ballot_sync(kAll, cand && q == 0);
            const uint32_t took = __ballot_sync(kAll, mine && q == 0);
            uint32_t left = 0;  // tiles (bit j) whose first 64 bytes hold no '\n'
            for (uint32_t jj = 0; jj < 8; ++jj)
                if (((cands >> (4 * jj)) & 1u) && !((seen >> (4 * jj)) & 0xFu)) left |= 1u << jj;
            const uint32_t ntook = __popc(took);
            __syncwarp();
            while (left) {
                const uint32_t jj = (uint32_t)(__ffs(left) - 1);
                left &= left - 1u;
                precode_tile(C, g0 + jj, sh, slot, tabs, svs + wid);
            }
            if (ntook < 8) g0 -= 8 - ntook;  // the round stopped at the shard's end: resume there
        }
    }

    // One tile whose first 64 bytes after its last owned byte hold no '\n': probe the rest of its stage window,
    // and if the last line runs past the stage, find the line and code it (all lanes).
    static __device__ void precode_tile(Ctx &C, uint64_t g, uint32_t sh, uint32_t *slot, uint32_t *tabs,
                                        ShardView *sv)
    {
        const SpArgs *P = C.P;
        load_shard(sv, P->one, P->shards, P->n_shards, sh);
        C.A = sv;
        const ShardView &A = *sv;
        const uint32_t lane = C.lane;
        const uint64_t t = g - A.tile0, base = t * (uint64_t)kTB;
        const uint64_t own_end = min(A.n, base + kTB), stage_hi = min(A.n, base + kTB + kHB);
        bool nl = false;
        for (uint64_t q0 = own_end - 1 + 64; q0 < stage_hi && !nl; q0 += 512) {
            const uint64_t p0 = q0 + 16u * lane;
            bool f = false;
#pragma unroll
            for (uint32_t i = 0; i < 16; ++i)
                if (p0 + i < stage_hi && A.in[p0 + i] == kNl) f = true;
            nl = __any_sync(kAll, f);
        }
        if (nl) return;
        // the tile's last line start: after the last '\n' in [base - 1, own_end - 1) (the input's start counts
        // as one); none: the tile holds no line start
        uint64_t ls = ~0ull;
        const uint64_t lo = base == 0 ? 0 : base - 1;
        for (uint64_t hi = own_end - 1; hi > lo && ls == ~0ull;) {
            const uint64_t w0 = hi > lo + 512 ? hi - 512 : lo;
            uint32_t bits = 0;
            const uint64_t p0 = w0 + 16u * lane;
#pragma unroll
            for (uint32_t i = 0; i < 16; ++i)
                if (p0 + i < hi && A.in[p0 + i] == kNl) bits |= 1u << i;
            const uint32_t any = __ballot_sync(kAll, bits != 0);
            if (any) {
                const int l = 31 - __clz(any);
                const uint32_t bb = __shfl_sync(kAll, bits, l);
                ls = w0 + 16u * (uint32_t)l + (uint32_t)(31 - __clz(bb)) + 1u;
            }
            hi = w0;
        }
        if (ls == ~0ull) {
            if (base != 0) return;
            ls = 0;
        }
        const uint64_t ge = find_nl_warp(C, stage_hi);
        if (ge - ls >= kLongLine) return;  // refused by the span kernel
        const uint64_t off = code_long(C, ls, (uint32_t)(ge - ls), ge < A.n, tabs);
        if (lane == 0 && off != ~0ull) slot[g] = (uint32_t)(off >> 4);
    }

    // Writes the lines coded before the launch where the span kernel placed them: one warp per slot.
    static __device__ void patch_run(const SpArgs *P)
    {
        const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        Ctx C;
        C.P = P;
        C.A = nullptr;
        C.M = nullptr;
        C.tab = nullptr;
        C.meta = reinterpret_cast<const uint32_t *>(P->bimg + P->meta_off);
        C.lane = lane;
        C.status = &P->g->status;
        const uint32_t *slot = reinterpret_cast<const uint32_t *>(P->slow);
        const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
        for (uint64_t g0 = ((uint64_t)blockIdx.x * (blockDim.x >> 5) + wid) * 32u; g0 < P->total_tiles;
             g0 += nwarps * 32u) {
            const uint64_t g = g0 + lane;
            uint32_t todo = __ballot_sync(kAll, g < P->total_tiles && slot[g] != 0);
            while (todo) {
                const int l = __ffs(todo) - 1;
                todo &= todo - 1u;
                const uint8_t *ws = P->slow + ((uint64_t)slot[g0 + (uint32_t)l] << 4);
                const uint64_t *h = reinterpret_cast<const uint64_t *>(ws + 16);
                LongSink S{reinterpret_cast<uint8_t *>(h[0]), h[1]};
                if (S.dst) long_emit(C, ws, 0, S);  // no address: the tile was not written (a rerun follows)
            }
        }
    }

    static __device__ void run(const SpArgs *P)
    {
        extern __shared__ __align__(128) uint8_t smem[];
        __shared__ uint64_t img_bar;
        const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        WarpMem &M = reinterpret_cast<WarpMem *>(smem)[wid];
        uint8_t *img = smem + kW * sizeof(WarpMem);
        Ctx C;
        C.P = P;
        C.A = nullptr;
        C.M = &M;
        C.tab = img;
        C.meta = reinterpret_cast<const uint32_t *>(img + P->meta_off);
        C.lane = lane;
        C.status = &P->g->status;
        if (threadIdx.x == 0) mbar_init(&img_bar, 1);
        if (lane == 0) mbar_init(&M.bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_arrive_tx(&img_bar, P->img_bytes);
            bulk_g2s(img, P->bimg, P->img_bytes, &img_bar);
        }
        const bool ok = mbar_wait_bounded(&img_bar, 0, P->limit_ns, C.status);
        if (!__syncthreads_and(ok)) {
            mbar_wait_bounded(&img_bar, 0, P->limit_ns, C.status);
            return;
        }
        uint32_t ph = 0, s = 0;
        bool pending = false;
        for (;;) {
            unsigned long long tt = 0;
            if (lane == 0) tt = atomicAdd(&P->g->tile_counter, 1ull);
            const uint64_t g = __shfl_sync(kAll, tt, 0);
            if (g >= P->total_tiles) break;
            OutSlot &O = M.os[s];
            const uint32_t sh = P->n_shards == 1 ? 0u : find_shard(P->shards, P->n_shards, g);
            load_shard(&O.sv, P->one, P->shards, P->n_shards, sh);
            const uint64_t t = g - O.sv.tile0;
            Ctx Cs = C;
            Cs.A = &O.sv;
            if (*((volatile uint32_t *)C.status) & kStFallback) {  // the call is redone: just unblock successors
                if (lane == 0 && (int64_t)t != P->stall_tile) publish(&O.sv.tiles[t], 2u, kPoison, kPoison);
                __syncwarp();
                continue;
            }
            stage_issue(Cs, t);
            if (!mbar_wait_bounded(&M.bar, ph, P->limit_ns, C.status)) {
                mbar_wait_bounded(&M.bar, ph, P->limit_ns, C.status);
                return;
            }
            ph ^= 1u;
            __syncwarp();
            Enc E = encode(Cs, O, t, P->cut_min != 0);
            if (E.retry) {  // a cut could not be kept: stage the tile again and code it whole-line only
                stage_issue(Cs, t);
                if (!mbar_wait_bounded(&M.bar, ph, P->limit_ns, C.status)) {
                    mbar_wait_bounded(&M.bar, ph, P->limit_ns, C.status);
                    return;
                }
                ph ^= 1u;
                __syncwarp();
                E = encode(Cs, O, t, false);
            }
            if (pending) {
                Ctx Cp = C;
                Cp.A = &M.os[s ^ 1u].sv;
                finish_staged(Cp, M.os[s ^ 1u]);
                pending = false;
            }
            if (O.direct == 1u) {
                finish_direct(Cs, O, E);
            } else if (O.direct == 0u) {
                pending = true;
                s ^= 1u;
            }
        }
        if (pending) {
            Ctx Cp = C;
            Cp.A = &M.os[s ^ 1u].sv;
            finish_staged(Cp, M.os[s ^ 1u]);
        }
    }
};

template <class Geo, bool OUTER>
__global__ void __launch_bounds__(Geo::kWarps * 32, 1) compress_span_kernel(const SpArgs P)
{
    SP<Geo, OUTER>::run(&P);
}

template <class Geo, bool OUTER>
__global__ void __launch_bounds__(SP<Geo, OUTER>::kPreWarps * 32) compress_span_precode_kernel(const SpArgs P)
{
    SP<Geo, OUTER>::precode_run(&P);
}

template <class Geo, bool OUTER>
__global__ void __launch_bounds__(256) compress_span_patch_kernel(const SpArgs P)
{
    SP<Geo, OUTER>::patch_run(&P);
}

// Compiled geometries: 2048-byte tiles (about 44 lines of 46 bytes, so a lane span holds one or two lines)
// with 20 warps per SM, the most whose stages fit beside a 170-state table; a variant with 4096-byte tiles
// (longer spans, better balance across lanes, 11 warps) for long-line mixes.
// Cuts: with 2048-byte tiles the reset-point search costs about what the balance gains on the long-tail mix
// (measured), so they are off by default; with 4096-byte tiles they are on.
using SpV0 = SpGeom<20, 2048, 512, 1152, 128, false>;
using SpV1 = SpGeom<11, 4096, 512, 2560, 320, true>;
// beside the table of a 170-state transducer (the frozen default dictionary; larger tables are checked at
// run time by span_fits)
static_assert(20 * sizeof(SP<SpV0, false>::WarpMem) + 170 * 256 + 1024 <= 227 * 1024, "shared memory");
static_assert(11 * sizeof(SP<SpV1, false>::WarpMem) + 170 * 256 + 1024 <= 227 * 1024, "shared memory");

template <class Geo>
size_t sp_smem(const zs_dict *d)
{
    return SP<Geo, false>::kW * sizeof(typename SP<Geo, false>::WarpMem) + d->blayout.img_bytes;
}

template <class Geo, bool OUTER>
cudaError_t sp_launch_as(const zs_dict *d, const TiledLaunch &L, unsigned flags, cudaStream_t s)
{
    SpArgs a{};
    a.one = L.one;
    a.shards = L.shards;
    a.n_shards = L.n_shards;
    a.flags = flags;
    a.total_tiles = L.total_tiles;
    a.bimg = d->d_bimg;
    a.img_bytes = d->blayout.img_bytes;
    a.meta_off = d->blayout.meta_off;
    a.q0 = d->blayout.q0;
    a.rep_col = d->blayout.rep_col;
    a.g = L.g;
    a.slow = L.slow;
    a.slow_cap = L.slow_cap;
    a.limit_ns = wait_limit_ns();
    a.stall_tile = injected_stall_tile();
    // lines of at least 3/64 of a tile (1.5 lane shares) may be cut, in the geometries where that pays (Geo::kCut);
    // a target within 1/128 of a tile of a line start takes the line start
    // the caller's threshold (a plan's tuned one), else the geometry's default; the test knob overrides both
    const int64_t cm = span_cut_min_override();
    a.cut_min = L.cut_min > 0 ? (uint32_t)L.cut_min : (L.cut_min < 0 ? 0u : (Geo::kCut ? (uint32_t)(3 * Geo::kTile / 64) : 0u));
    if (cm >= 0) a.cut_min = (uint32_t)cm;
    a.cut_slack = Geo::kTile / 128;
    const int smem = (int)sp_smem<Geo>(d);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    static int set_smem = -1;
    if (set_smem != smem) {
        cudaError_t e = cudaFuncSetAttribute(compress_span_kernel<Geo, OUTER>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        set_smem = smem;
    }
    // lines longer than the stage: a slot per tile at the start of the scratch, when it holds them
    a.slots_need = (L.total_tiles * 4u + 255u) & ~255ull;
    a.slots_bytes = (L.slow && L.slow_cap >= a.slots_need) ? a.slots_need : 0;
    if (a.slots_bytes && L.total_tiles) {
        cudaError_t e = cudaSuccess;
        using S = SP<Geo, OUTER>;  // the precode kernel writes every tile's slot
        const int psm = (int)S::pre_smem(d->blayout.img_bytes);
        static int set_pre = -1;
        if (set_pre != psm) {
            e = cudaFuncSetAttribute(compress_span_precode_kernel<Geo, OUTER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     psm);
            if (e != cudaSuccess) return e;
            set_pre = psm;
        }
        const uint64_t pg = std::min<uint64_t>((L.total_tiles + 4 * S::kPreWarps - 1) / (4 * S::kPreWarps),
                                               (uint64_t)sms * 4u);
        compress_span_precode_kernel<Geo, OUTER><<<(unsigned)pg, S::kPreWarps * 32, psm, s>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, compress_span_kernel<Geo, OUTER>, SP<Geo, OUTER>::kNT, smem);
    if (per < 1) per = 1;
    uint64_t grid = std::min<uint64_t>((L.total_tiles + Geo::kWarps - 1) / Geo::kWarps, (uint64_t)per * (uint64_t)sms);
    if (grid == 0) grid = 1;
    compress_span_kernel<Geo, OUTER><<<(unsigned)grid, SP<Geo, OUTER>::kNT, smem, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !a.slots_bytes || !L.total_tiles) return e;
    const uint64_t tg = std::min<uint64_t>((L.total_tiles + 255) / 256, (uint64_t)sms * 2u);
    compress_span_patch_kernel<Geo, OUTER><<<(unsigned)tg, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <class Geo>
cudaError_t sp_launch(const zs_dict *d, const TiledLaunch &L, unsigned flags, cudaStream_t s)
{
    return (flags & ZS_PREPROCESS_OUTER) ? sp_launch_as<Geo, true>(d, L, flags, s)
                                         : sp_launch_as<Geo, false>(d, L, flags, s);
}

struct SpEntry {
    KernelVariant info;
    size_t (*smem)(const zs_dict *);
    cudaError_t (*launch)(const zs_dict *, const TiledLaunch &, unsigned, cudaStream_t);
    uint32_t cut_default;
};

template <class Geo>
constexpr SpEntry sp_entry(const char *name)
{
    return SpEntry{KernelVariant{name, Geo::kWarps, Geo::kTile}, &sp_smem<Geo>, &sp_launch<Geo>,
                   Geo::kCut ? (uint32_t)(3 * Geo::kTile / 64) : 0u};
}

const SpEntry kSp[] = {
    sp_entry<SpV0>("compress span w20 t2048"),
    sp_entry<SpV1>("compress span w11 t4096"),
};
constexpr int kNumSp = (int)(sizeof(kSp) / sizeof(kSp[0]));

}  // namespace

int span_variants() { return kNumSp; }

const KernelVariant *span_variant(int v) { return (v >= 0 && v < kNumSp) ? &kSp[v].info : nullptr; }

uint32_t span_cut_default(int v)
{
    if (v < 0 || v >= kNumSp) return 0;
    return kSp[v].cut_default;
}

bool span_fits(int v, const zs_dict *d)
{
    if (v < 0 || v >= kNumSp || !d->has_bytes) return false;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return kSp[v].smem(d) <= (size_t)optin;
}

cudaError_t launch_span(int v, const zs_dict *d, const TiledLaunch &L, unsigned flags, cudaStream_t s)
{
    if (v < 0 || v >= kNumSp) return cudaErrorInvalidValue;
    return kSp[v].launch(d, L, flags, s);
}

}  // namespace zs
