// zs_compress, transducer path: ring-ID pre-processing (Sec. IV-A) and the minimum-length parse
// (Sec. IV-D1) with one warp per tile (default: 20 warps per SM, 1408-byte tiles, about 30 lines each).
//
//   - Each warp of a persistent CTA claims tiles on its own (atomic counter in launch order) and stages
//     each tile, the byte before it and a halo (512 bytes by default) with one bulk (TMA) copy. No
//     CTA-wide barrier is on the per-tile path.
//   - Software pipeline: a warp encodes tile k+1 (publishing its aggregate) before it resolves tile k's
//     output offset by look-back and emits it, so by the time it looks back, its predecessors have long
//     published; two staging slots per warp hold the two tiles.
//   - Segmentation counts and ranks line starts on the raw bytes (16-byte shared loads, warp prefix sums);
//     then only the bytes the tile's lines cover are replaced by class codes (coalesced 16-byte chunks, a
//     lane-replicated class table so lookups never conflict on a bank), with per-chunk flags for the bytes
//     pre-processing must look at (digits; '%', brackets, space, tab). Lines are sorted by length (per-warp
//     counting sort) and dealt to lanes longest first, in snake order when a batch needs several rounds.
//   - Pre-processing: a line of at most 112 bytes without '%' and with at most kTok ring labels takes the
//     bit-mask path (lanes in lockstep over the ring tokens, per-label state in register byte lanes); any
//     other line walks its flagged bytes once and relabels in place. Either way the new labels are written
//     into the class codes (the class of digit d is d), %nn labels shrinking in place.
//   - Parse: the backward shortest-path scan is the minimal transducer built by zs_load_dictionary: per
//     byte one transition lookup on the class code gives the next state, the increment of the path cost
//     and the symbol chosen at that byte. Codes are read and symbols written a 4-byte word at a time;
//     only the state lookups form a dependent chain.
//   - Emission walks the chosen symbols front to back into a per-warp staging buffer aligned to the
//     output's 16-byte grid, written out with coalesced 16-byte stores.
//   - Lines longer than 2047 bytes or past the halo, lines needing a two-digit label or holding more open
//     %nn labels than the lane's column has slots, and lines whose relabelled text needs an escape of a
//     byte that is not a digit take the exact slow path in global scratch (one lane). A tile with more lines
//     than a batch holds is processed batch by batch, look-back first.
#include <algorithm>

#include "compress_shared.cuh"

namespace zs {
namespace {
using namespace cx;

// Tile geometry of one compiled variant of the kernel.
template <int W, int TW, int HW, int MAXL, int OUTW, int TOK>
struct CwGeom {
    static constexpr int kWarps = W;        // warps per CTA
    static constexpr int kTile = TW;        // owned bytes per warp tile
    static constexpr int kHalo = HW;        // bytes staged past the tile for the tile's last line
    static constexpr int kMaxLines = MAXL;  // lines per batch
    static constexpr int kOut = OUTW;       // staged output bytes per tile
    static constexpr int kTok = TOK;        // per-lane column: ring labels of a line on the bit-mask path, and
                                            // the class-code path's open-ring slots (10 + 2 per open %nn label)
};
constexpr int kFastMax = 2047;        // longest line on the fast path (token positions use 11 bits)
constexpr uint32_t kLongLine = 1u << 30;
constexpr uint8_t kLfNl = 1, kLfSlow = 2;
constexpr unsigned kFull = 0xffffffffu;

// Launch-wide arguments; the per-shard ones are in the ShardView of each claimed tile.
struct CwArgs {
    ShardView one;            // the shard when n_shards == 1
    const ShardView *shards;  // device shard table when n_shards > 1 (tile0 ascending, shards[0].tile0 == 0)
    uint32_t n_shards;
    uint32_t flags;
    uint64_t total_tiles;
    const uint8_t *mimg;
    uint32_t img_bytes;
    uint32_t n_classes;
    uint32_t start_state;
    uint32_t esc_digits;      // the table codes an escaped digit d as choice 1 + d (MachineLayout::esc_digits)
    DevResult *g;             // tile counter, status bits, long-line scratch use
    uint8_t *slow;
    uint64_t slow_cap;
    uint64_t limit_ns;
    int64_t stall_tile;
};

// OUTER: ring IDs renumbered in opening order (ZS_PREPROCESS_OUTER) instead of closing order; a template
// parameter so that the default kernel carries none of the other reading's code.
template <class Geo, bool OUTER>
struct CW {
    static constexpr int kMW = Geo::kWarps;
    static constexpr int kMNT = 32 * kMW;
    static constexpr int kTW = Geo::kTile;
    static constexpr int kHW = Geo::kHalo;
    static constexpr int kStW = 16 + kTW + kHW;  // staged bytes: the byte before the tile (index 15), tile, halo
    static constexpr int kMaxLW = Geo::kMaxLines;
    static constexpr int kOutW = Geo::kOut;
    static constexpr int kTokMax = Geo::kTok;
    static constexpr uint32_t kImaskChunks = (kStW + 31) / 16 + 2;
    static_assert(kTW % 16 == 0 && kHW % 16 == 0 && kOutW % 16 == 0 && kMaxLW % 8 == 0 && kMaxLW <= 256 &&
                      kTokMax >= 12 && kTokMax <= 32,
                  "tile geometry");

    struct alignas(16) Slot {
        uint8_t st[kStW + 48];
        uint16_t start[kMaxLW + 8];
        uint16_t plen[kMaxLW];
        uint32_t olen[kMaxLW];  // per line: length bucket (sort), output bytes, then (in place) output offset
        uint32_t soff[kMaxLW];  // per line: rank in its bucket (sort), then slow-path work space / 16
        uint8_t flag[kMaxLW];
        uint8_t perm[kMaxLW];
        uint64_t bar;
        uint64_t btotal;
        uint32_t Lt, first_start, last_end, last_nl, last_long, any_slow, nown, pad;
        ShardView sv;  // the shard of the staged tile
    };

    struct alignas(16) WarpMem {
        Slot slot[2];
        uint8_t ost[kOutW + 32];
        uint16_t tok[kTokMax * 32];  // per lane (entry k of lane l at [k * 32 + l]): the ring tokens of the
                                     // lane's line (bit-mask path) or its open rings (in-place path)
        uint32_t hist[64];
        uint32_t imask[kImaskChunks];  // per 16-byte chunk of the staged tile: digit bytes (bits 0-15) and the
                                       // other bytes pre-processing looks at: '%', brackets, space, tab (16-31)
    };

    struct Ctx {
        const CwArgs *P;      // launch-wide arguments
        const ShardView *A;   // shard of the tile being worked on
        WarpMem *M;
        const uint8_t *clsrep;
        const uint8_t *plen_tab;
        const uint32_t *T;
        uint32_t nc, q0, lane;
        uint32_t *status;
    };

    static __device__ __forceinline__ uint32_t cls_of(const uint8_t *clsrep, uint32_t c, uint32_t lane)
    {
        return clsrep[((((c >> 2) << 5) + lane) << 2) | (c & 3u)];
    }

    // One transducer step (last byte first): returns the chosen symbol, updates state and cost.
    // q is the current state's row offset (state * classes).
    static __device__ __forceinline__ uint32_t step(const uint32_t *T, uint32_t nc, uint32_t k, uint32_t &q, int32_t &cost)
    {
        (void)nc;
        const uint32_t t = T[q + k];
        q = t & 0xFFFFu;
        cost += (int32_t)((t >> 16) & 31u) - 16;
        return t >> 24;
    }

    // Transducer walk over the class codes st[a, a+n) in place (last byte first); each code is replaced by
    // the symbol chosen at that byte. Whole 4-byte words where the word belongs to the line. *esc: the line
    // has an escape the input bytes must supply (an escaped digit, when the table codes it as 1 + d, does not
    // count: see MachineLayout::esc_digits).
    static __device__ __forceinline__ uint32_t parse_classes(uint8_t *st, uint32_t a, uint32_t n, const Ctx &C, bool *esc)
    {
        uint32_t q = C.q0, e = 0;
        int32_t cost = 0;
        int32_t p = (int32_t)(a + n) - 1;
        const int32_t lo = (int32_t)a;
        while (p >= lo && ((p + 1) & 3) != 0) {
            const uint32_t sy = step(C.T, C.nc, st[p], q, cost);
            e |= (sy == kEsc);
            st[p] = (uint8_t)sy;
            --p;
        }
        while (p - 3 >= lo) {
            const int32_t wp = p - 3;
            const uint32_t w = *reinterpret_cast<const uint32_t *>(st + wp);
            const uint32_t s3 = step(C.T, C.nc, w >> 24, q, cost);
            const uint32_t s2 = step(C.T, C.nc, (w >> 16) & 255u, q, cost);
            const uint32_t s1 = step(C.T, C.nc, (w >> 8) & 255u, q, cost);
            const uint32_t s0 = step(C.T, C.nc, w & 255u, q, cost);
            e |= (s3 == kEsc) | (s2 == kEsc) | (s1 == kEsc) | (s0 == kEsc);
            *reinterpret_cast<uint32_t *>(st + wp) = s0 | (s1 << 8) | (s2 << 16) | (s3 << 24);
            p -= 4;
        }
        while (p >= lo) {
            const uint32_t sy = step(C.T, C.nc, st[p], q, cost);
            e |= (sy == kEsc);
            st[p] = (uint8_t)sy;
            --p;
        }
        *esc = e != 0;
        return (uint32_t)cost;
    }

    // The same walk over separate global arrays (slow path).
    static __device__ uint32_t parse_global(const uint8_t *text, uint8_t *choice, uint32_t n, const Ctx &C)
    {
        uint32_t q = C.q0;
        int32_t cost = 0;
        for (uint32_t i = n; i-- > 0;) choice[i] = (uint8_t)step(C.T, C.nc, cls_of(C.clsrep, text[i], C.lane), q, cost);
        return (uint32_t)cost;
    }

    // Pre-processing of the class codes st[a, a+n) in place (Sec. IV-A), in one pass over the bytes flagged
    // in imask (digits, '%', brackets, space, tab), for any line the bit-mask path does not take. Rings
    // are labelled in the order they close, each with the smallest label that no ring closed since it
    // opened still holds: lc[x] = position + 1 of the latest close that took label x. Both label bytes of
    // a ring are written when it closes (a %nn label's '%' becomes the digit and its two digits a deletion
    // mark, squeezed out at the end), so only the open rings are remembered, in the lane's column of `opn`
    // (stride 32): slot x < 10 = position + 1 of the open label x (bit 15 set if it was written %0x), slots
    // 10 + 2j / 11 + 2j = (label + 1, position) of up to kOpen2 open %nn labels. A line found invalid at its end (unclosed ring or bracket, bad
    // %) is restored from its raw bytes and left as it is.
    // Returns the new length, or -1 for the slow path (a label >= 10 needed, more than kOpen2 open %nn labels,
    // or more than kFastMax bytes). *modified: some ring label was rewritten.
    static constexpr uint8_t kClsDel = 0xFE;  // a deleted byte (the digits of a rewritten %nn label)
    static constexpr int kOpen2 = (kTokMax - 10) / 2;  // open %nn labels the class-code path follows

    static __device__ __forceinline__ int preprocess_classes(uint8_t *st, const uint32_t *imask, uint32_t a, uint32_t n,
                                                             const uint8_t *raw, const Ctx &C, uint16_t *opn,
                                                             bool *modified)
    {
        *modified = false;
        if (n > (uint32_t)kFastMax) return -1;
        if (n == 0) return 0;
        const uint32_t end = a + n;
        uint32_t lc[10];
    #pragma unroll
        for (int x = 0; x < 10; ++x) lc[x] = 0;
        for (int x = 0; x < 10 + 2 * kOpen2; ++x) opn[x * 32] = 0;
        uint32_t dopen = 0, nopen2 = 0, skipto = 0, held = 0;
        bool in_br = false, bad = false, any_pct = false, done = false, need_slow = false, wrote = false;
        const uint32_t clast = (end - 1) >> 4;
        uint32_t c = a >> 4;
        auto chunk_mask = [&](uint32_t cc) -> uint32_t {
            const uint32_t cb = cc << 4;
            uint32_t mm = (imask[cc] | (imask[cc] >> 16)) & 0xFFFFu;
            if (cb < a) mm &= 0xFFFFu << (a - cb);
            if (cb + 16 > end) mm &= (1u << (end - cb)) - 1u;
            return mm;
        };
        // writes new label nl at line position q (a %nn token: the '%' becomes the digit, its digits go)
        auto put = [&](uint32_t q, uint32_t nl, bool pct) {
            st[a + q] = (uint8_t)nl;  // the class of digit d is d
            if (pct) {
                st[a + q + 1] = kClsDel;
                st[a + q + 2] = kClsDel;
            }
        };
        uint32_t m = chunk_mask(c);
        for (;;) {
            while (m == 0 && c < clast) m = chunk_mask(++c);
            if (m == 0 || done) break;
            const uint32_t p = (c << 4) + (uint32_t)(__ffs(m) - 1);
            m &= m - 1;
            const uint32_t k = st[p];
            const bool live = p >= skipto;  // not one of the two digits of a %nn label
            const bool ws = live & ((k == kClsSpace) | (k == kClsTab));
            done = ws;  // the SMILES field ends at the first space or tab
            const bool lb = live & !ws & !in_br & (k == kClsLbr);
            const bool rb = live & in_br & (k == kClsRbr);
            const bool ring = live & !in_br & (k <= kClsPct);  // a digit or a '%'
            in_br = (in_br | lb) & !rb;
            if (!ring) continue;
            uint32_t label = k;
            bool pct = false;
            if (k == kClsPct) {  // %nn: two digits must follow inside the line
                if (p + 2 >= end || st[p + 1] >= 10 || st[p + 2] >= 10) {
                    bad = true;
                    break;
                }
                label = st[p + 1] * 10u + st[p + 2];
                pct = true;
                any_pct = true;
                skipto = p + 3;
            }
            const uint32_t q = p - a;
            int po = -1;  // position of the ring's open token, if this token closes it
            bool opct = false;
            if (label < 10) {  // a digit, or %0d; bit 15 of the slot: the opening token was %0d
                if ((dopen >> label) & 1u) {
                    const uint32_t v = opn[label * 32];
                    po = (int)(v & 0x7FFFu) - 1;
                    opct = (v >> 15) != 0;
                    dopen &= ~(1u << label);
                } else {
                    opn[label * 32] = (uint16_t)((q + 1) | (pct ? 0x8000u : 0u));
                    dopen |= 1u << label;
                }
            } else {
                int hit = -1, empty = -1;
                for (int j = 0; j < kOpen2; ++j) {
                    const uint32_t v = opn[(10 + 2 * j) * 32];
                    if (v == 0) {
                        if (empty < 0) empty = j;
                    } else if (v == label + 1) {
                        hit = j;
                    }
                }
                if (hit >= 0) {
                    po = (int)opn[(11 + 2 * hit) * 32];
                    opct = true;
                    opn[(10 + 2 * hit) * 32] = 0;
                    --nopen2;
                } else if (empty >= 0) {
                    opn[(10 + 2 * empty) * 32] = (uint16_t)(label + 1);
                    opn[(11 + 2 * empty) * 32] = (uint16_t)q;
                    ++nopen2;
                } else {
                    need_slow = true;
                    break;
                }
            }
            if (OUTER) {  // opening order: an opening ring takes the smallest free label at once
                if (po < 0) {
                    const uint32_t fr = ~held & 0x3FFu;
                    if (fr == 0) {  // needs a two-digit label
                        need_slow = true;
                        break;
                    }
                    const uint32_t nl = (uint32_t)__ffs(fr) - 1u;
                    held |= 1u << nl;
                    put(q, nl, pct);
                } else {
                    const uint32_t nl = st[a + (uint32_t)po];
                    held &= ~(1u << nl);
                    put(q, nl, pct);
                }
                wrote = true;
                continue;
            }
            if (po < 0) continue;
            int nl = -1;
    #pragma unroll
            for (int x = 9; x >= 0; --x)
                if (lc[x] <= (uint32_t)po + 1) nl = x;
            if (nl < 0) {  // needs a two-digit label
                need_slow = true;
                break;
            }
    #pragma unroll
            for (int x = 0; x < 10; ++x)
                if (x == nl) lc[x] = q + 1;
            put((uint32_t)po, (uint32_t)nl, opct);
            put(q, (uint32_t)nl, pct);
            wrote = true;
        }
        if (need_slow) return -1;
        if (bad || in_br || dopen != 0 || nopen2 != 0 || !wrote) {  // left as it is
            if (wrote)
                for (uint32_t i = 0; i < n; ++i) st[a + i] = (uint8_t)cls_of(C.clsrep, raw[i], C.lane);
            return (int)n;
        }
        *modified = true;
        if (!any_pct) return (int)n;
        uint32_t w = 0;
        for (uint32_t r = 0; r < n; ++r) {
            const uint8_t v = st[a + r];
            if (v != kClsDel) st[a + w++] = v;
        }
        return (int)w;
    }

    // Writes the new labels of a valid line back into its class codes (the class of digit d is d); %nn
    // labels shrink to one digit, so the line is compacted then. Returns the new length.
    static __device__ __forceinline__ int write_labels(uint8_t *st, uint32_t a, uint32_t n, const uint16_t *tok,
                                                       uint32_t ntok, bool any_pct)
    {
        if (!any_pct) {
            for (uint32_t k = 0; k < ntok; ++k) {
                const uint32_t e = tok[k * 32];
                st[a + (e & 0x7FFu)] = (uint8_t)(e >> 12);
            }
            return (int)n;
        }
        uint32_t w = 0, r = 0;
        for (uint32_t k = 0; k < ntok; ++k) {
            const uint32_t e = tok[k * 32];
            const uint32_t p = e & 0x7FFu;
            for (; r < p; ++r, ++w) st[a + w] = st[a + r];
            st[a + w] = (uint8_t)(e >> 12);
            ++w;
            r = p + ((e & 0x800u) ? 3u : 1u);
        }
        for (; r < n; ++r, ++w) st[a + w] = st[a + r];
        return (int)w;
    }

    // Bits below window position t in word k of a 128-bit window (t - 32k clamped to [0, 32]).
    static __device__ __forceinline__ uint32_t below(int t, int k)
    {
        return __funnelshift_lc(0xFFFFFFFFu, 0u, (uint32_t)max(t - 32 * k, 0));
    }

    // A 128-bit bit set in four registers (no array, so it never lands in local memory).
    struct Bits128 {
        uint32_t w0, w1, w2, w3;
        __device__ __forceinline__ bool any() const { return (w0 | w1 | w2 | w3) != 0; }
        __device__ __forceinline__ uint32_t count() const { return __popc(w0) + __popc(w1) + __popc(w2) + __popc(w3); }
        // Removes and returns the lowest set bit (an empty set returns 127 and stays empty).
        __device__ __forceinline__ int pop()
        {
            const bool z0 = w0 == 0, z1 = w1 == 0, z2 = w2 == 0;
            const uint32_t w = !z0 ? w0 : (!z1 ? w1 : (!z2 ? w2 : w3));
            const int base = !z0 ? 0 : (!z1 ? 32 : (!z2 ? 64 : 96));
            const uint32_t c = w & (w - 1u);
            w0 = !z0 ? c : w0;
            w1 = (z0 && !z1) ? c : w1;
            w2 = (z0 && z1 && !z2) ? c : w2;
            w3 = (z0 && z1 && z2) ? c : w3;
            return w ? base + __ffs(w) - 1 : 127;
        }
        __device__ __forceinline__ void keep_below(int t)
        {
            w0 &= below(t, 0);
            w1 &= below(t, 1);
            w2 &= below(t, 2);
            w3 &= below(t, 3);
        }
        __device__ __forceinline__ void clear_range(int lo_b, int hi_b)  // [lo_b, hi_b)
        {
            w0 &= ~below(hi_b, 0) | below(lo_b, 0);
            w1 &= ~below(hi_b, 1) | below(lo_b, 1);
            w2 &= ~below(hi_b, 2) | below(lo_b, 2);
            w3 &= ~below(hi_b, 3) | below(lo_b, 3);
        }
    };

    // Pre-processing of a line of at most kBitMax bytes without '%' (the usual drug-like line), from bit
    // masks and with the lanes in lockstep over the ring tokens.
    //   - The digit and other-flag masks of the line's chunks form two 128-bit register windows (window bit
    //     i = staged byte 16 * (a / 16) + i). The few other flags (brackets, the end of the first field)
    //     are walked first: they remove the digits inside brackets and after the field. What remains are
    //     the ring tokens.
    //   - The tokens are then visited in order by every lane at once, as many steps as the lane with the
    //     most tokens, each step predicated rather than branched. lc (latest close position + 1 of each
    //     label, positions <= 112) lives in the byte lanes of three registers, so finding the smallest
    //     label free since the ring opened is three 32-bit subtractions and one find-first-set.
    //   - A token's new label goes to the lane's column of `tok` (position | label << 12); the labels are
    //     written into the class codes once the line is known to be valid.
    // Returns as preprocess_classes, or -2 when the line holds a '%' or more than kTokMax ring labels (the
    // caller then runs preprocess_classes). Every lane of the calling group must call it.
    static constexpr uint32_t kBitMax = 112;

    static __device__ __forceinline__ int preprocess_bits(uint8_t *st, const uint32_t *imask, uint32_t nchunks,
                                                          uint32_t a, uint32_t n, bool eligible, uint16_t *tok,
                                                          bool *modified)
    {
        *modified = false;
        const uint32_t am = __activemask();
        int result = 0x7FFFFFFF;  // decided early: the line's result; else the token pass decides
        uint32_t ntok = 0;
        Bits128 D{0u, 0u, 0u, 0u};
        const uint32_t lo = a & 15u;
        if (!eligible) {
            result = -2;
        } else {
            const uint32_t c0 = a >> 4;
            const int hi = (int)(lo + n);  // the line is window bits [lo, hi), hi <= 127
            uint32_t m[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) m[k] = c0 + k < nchunks ? imask[c0 + k] : 0u;
            D = Bits128{(m[0] & 0xFFFFu) | (m[1] << 16), (m[2] & 0xFFFFu) | (m[3] << 16),
                        (m[4] & 0xFFFFu) | (m[5] << 16), (m[6] & 0xFFFFu) | (m[7] << 16)};
            Bits128 O{(m[0] >> 16) | (m[1] & 0xFFFF0000u), (m[2] >> 16) | (m[3] & 0xFFFF0000u),
                      (m[4] >> 16) | (m[5] & 0xFFFF0000u), (m[6] >> 16) | (m[7] & 0xFFFF0000u)};
            D.keep_below(hi);
            O.keep_below(hi);
            D.w0 &= 0xFFFFFFFFu << lo;
            O.w0 &= 0xFFFFFFFFu << lo;
            bool in_br = false;
            int obr = 0;
            while (O.any()) {
                const int wb = O.pop();
                const uint32_t c = st[a + (uint32_t)wb - lo];
                if (c == kClsPct) {
                    result = -2;
                    break;
                }
                if (c == kClsSpace || c == kClsTab) {  // the first field ends here
                    D.keep_below(wb);
                    break;
                }
                if (c == kClsLbr) {
                    if (!in_br) obr = wb;
                    in_br = true;
                } else if (in_br) {  // ']' closes the bracket atom: its digits are no ring labels
                    D.clear_range(obr + 1, wb);
                    in_br = false;
                }
            }
            ntok = D.count();
            if (result == 0x7FFFFFFF) {
                if (in_br || ntok == 0) result = (int)n;       // unclosed bracket, or no ring: left as it is
                else if (ntok > (uint32_t)kTokMax) result = -2;  // more tokens than the lane's column holds
            }
        }
        const uint32_t my_steps = result == 0x7FFFFFFF ? ntok : 0u;
        const uint32_t steps = __reduce_max_sync(am, my_steps);
        // lc: latest close position + 1 of each new label, label x in byte x / 3 of register x % 3 (positions
        // are at most 112); the bytes of labels 10 and 11 hold 127, never free
        uint32_t lc0 = 0u, lc1 = 0x7F000000u, lc2 = 0x7F000000u;
        uint64_t dmap = 0;
        uint32_t dopen = 0;
        bool need_slow = false;
        uint32_t held = 0;  // opening order: bit x set while label x is held
        for (uint32_t it = 0; it < steps; ++it) {
            const bool act = it < my_steps;
            const int wb = D.pop();
            const uint32_t rel = (uint32_t)wb - lo;
            const uint32_t label = act ? st[a + rel] : 0u;
            const bool open = (dopen >> label) & 1u;
            const uint32_t ko = open ? (uint32_t)(dmap >> (5 * label)) & 31u : 0u;
            const uint32_t eo = tok[ko * 32];
            if (OUTER) {  // an opening ring takes the smallest free label, its closing token repeats it
                const bool opening = act && !open, closing = act && open;
                const uint32_t fr = ~held & 0x3FFu;
                need_slow = need_slow || (opening && fr == 0u);  // would need a two-digit label
                const uint32_t nl = closing ? (eo >> 12) : (fr ? (uint32_t)__ffs(fr) - 1u : 0u);
                held = (opening && fr != 0u) ? (held | (1u << nl)) : held;
                held = closing ? (held & ~(1u << nl)) : held;
                if (act) tok[it * 32] = (uint16_t)(rel | (nl << 12));
                dmap = opening ? ((dmap & ~(31ull << (5 * label))) | ((uint64_t)it << (5 * label))) : dmap;
                dopen ^= act ? (1u << label) : 0u;
                continue;
            }
            // label x is free when lc[x] <= open position + 1 = p. Per byte, (0x80 + p) - lc[x] stays within the
            // byte (both are below 128) and has its top bit set exactly then; one find-first-set over the three
            // registers' top bits (bit 8 * byte + register) gives the smallest free label
            const uint32_t t = (((eo & 0x7Fu) + 1u) * 0x01010101u) | 0x80808080u;
            const uint32_t y = (((t - lc0) & 0x80808080u) >> 7) | (((t - lc1) & 0x80808080u) >> 6) |
                               (((t - lc2) & 0x80808080u) >> 5);
            const bool closing = act && open;
            const uint32_t fb = (uint32_t)__ffs(y) - 1u;
            const uint32_t by = fb >> 3, rg = fb & 7u;
            const int nl = (int)(3u * by + rg);
            need_slow = need_slow || (closing && y == 0u);  // would need a two-digit label
            const bool upd = closing && y != 0u;
            lc0 = (upd && rg == 0) ? put_byte(lc0, rel + 1u, by) : lc0;
            lc1 = (upd && rg == 1) ? put_byte(lc1, rel + 1u, by) : lc1;
            lc2 = (upd && rg == 2) ? put_byte(lc2, rel + 1u, by) : lc2;
            if (upd) tok[ko * 32] = (uint16_t)(eo | ((uint32_t)nl << 12));
            if (act) tok[it * 32] = (uint16_t)(upd ? (rel | ((uint32_t)nl << 12)) : rel);
            const bool opening = act && !open;
            dmap = opening ? ((dmap & ~(31ull << (5 * label))) | ((uint64_t)it << (5 * label))) : dmap;
            dopen ^= act ? (1u << label) : 0u;
        }
        if (result != 0x7FFFFFFF) return result;
        if (need_slow) return -1;
        if (dopen != 0) return (int)n;  // an unclosed ring: left as it is
        *modified = true;
        return write_labels(st, a, n, tok, ntok, false);
    }

    // Byte lane b of x (b = 0..3) replaced by the low 8 bits of v.
    static __device__ __forceinline__ uint32_t put_byte(uint32_t x, uint32_t v, uint32_t b)
    {
        uint32_t r;
        asm("bfi.b32 %0, %1, %2, %3, 8;" : "=r"(r) : "r"(v), "r"(x), "r"(8u * b));
        return r;
    }

    // Packs the 0x00 / 0xFF byte lanes of x into 4 bits (byte i -> bit i).
    static __device__ __forceinline__ uint32_t pack4(uint32_t x) { return ((x & 0x01010101u) * 0x01020408u) >> 24; }

    // Replace the staged bytes by their classes (coalesced 16-byte chunks, lane-replicated table) and flag,
    // per chunk, the bytes pre-processing has to look at.
    static __device__ __forceinline__ void to_classes(const Ctx &C, Slot &S, uint32_t stage_end)
    {
        const uint32_t nchunks = (stage_end + 15) >> 4;
        for (uint32_t c = C.lane; c < nchunks; c += 32) {
            const uint4 v = *reinterpret_cast<const uint4 *>(S.st + c * 16);
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
            uint32_t o[4], dmask = 0, omask = 0;
    #pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t b0 = cls_of(C.clsrep, w[i] & 255u, C.lane), b1 = cls_of(C.clsrep, (w[i] >> 8) & 255u, C.lane);
                const uint32_t b2 = cls_of(C.clsrep, (w[i] >> 16) & 255u, C.lane), b3 = cls_of(C.clsrep, w[i] >> 24, C.lane);
                o[i] = b0 | (b1 << 8) | (b2 << 16) | (b3 << 24);
                const uint32_t dig = __vcmpltu4(o[i], 0x0A0A0A0Au);  // 0xFF per digit byte
                const uint32_t flg = __vcmpltu4(o[i], kClsNl * 0x01010101u);
                dmask |= pack4(dig) << (4 * i);
                omask |= pack4(flg & ~dig) << (4 * i);
            }
            *reinterpret_cast<uint4 *>(S.st + c * 16) = make_uint4(o[0], o[1], o[2], o[3]);
            C.M->imask[c] = dmask | (omask << 16);
        }
        __syncwarp();
    }

    // Newline bits of the 16 staged bytes at p0 (nl: the newline byte, raw or as its class), below lim.
    static __device__ __forceinline__ uint32_t nl_bits_masked(const uint8_t *st, uint32_t p0, uint32_t lim,
                                                              uint32_t nl = kClsNl)
    {
        if (p0 >= lim) return 0;
        uint32_t bits = eq_bits16(*reinterpret_cast<const uint4 *>(st + p0), nl * 0x01010101u);
        if (p0 + 16 > lim) bits &= (1u << (lim - p0)) - 1u;
        return bits;
    }

    static __device__ __forceinline__ uint64_t tile_base(uint64_t t) { return t * (uint64_t)kTW; }

    // Issue the bulk copy of tile t into slot S (lane 0), plus the unaligned tail bytes (all lanes).
    static __device__ __forceinline__ void stage_issue(const Ctx &C, Slot &S, uint64_t t)
    {
        const ShardView &A = *C.A;
        const uint64_t base = tile_base(t);
        const uint64_t stage_hi = min(A.n, base + (uint64_t)kTW + kHW);
        const uint64_t lo = base >= 16 ? base - 16 : 0;
        const uint32_t j0 = (uint32_t)(lo + 16 - base);
        const uint32_t nbytes = (uint32_t)(stage_hi - lo);
        const uint32_t nbulk = A.in_aligned ? (nbytes & ~15u) : 0u;
        __syncwarp();
        if (C.lane == 0) {
            fence_proxy_async_smem();
            mbar_arrive_tx(&S.bar, nbulk);
            if (nbulk) bulk_g2s(S.st + j0, A.in + lo, nbulk, &S.bar);
        }
        for (uint32_t j = nbulk + C.lane; j < nbytes; j += 32) S.st[j0 + j] = A.in[lo + j];
        if (t == 0 && C.lane == 0) S.st[15] = kNl;  // position 0 starts a line
    }

    // Segmentation of the staged tile: line count, first start, end of the last line.
    // Segmentation of the staged tile on its raw bytes: line count, first start, end of the last line.
    // Then only the bytes the tile's lines cover (the owned bytes and the last line's overhang into the
    // halo) are turned into classes.
    static __device__ __forceinline__ void segment(const Ctx &C, Slot &S, uint64_t t)
    {
        const ShardView &A = *C.A;
        const uint64_t base = tile_base(t);
        const uint32_t nown = (uint32_t)(min(A.n, base + kTW) - base);
        const uint64_t stage_hi = min(A.n, base + (uint64_t)kTW + kHW);
        const uint32_t stage_end = (uint32_t)(stage_hi - base) + 16u;
        const uint8_t *st = S.st;
        const uint32_t lim = 15u + nown;
        const uint32_t first_start = (st[15] == kNl && nown > 0) ? 1u : 0u;
        uint32_t Lt = first_start;
    #pragma unroll
        for (int it = 0; it < (kTW + 511) / 512; ++it)
            Lt += __reduce_add_sync(kFull, __popc(nl_bits_masked(st, 16u + it * 512u + C.lane * 16u, lim, kNl)));
        uint32_t last_end = 0, last_nl = 0, last_long = 0;
        uint32_t conv_end = 16u + nown;  // staged bytes [0, conv_end) become classes
        if (Lt > 0) {
            uint32_t end = 0xFFFFFFFFu;
            if (st[15 + nown] == kNl) {
                end = 15 + nown;
            } else {
                for (uint32_t off = 16 + nown; off < stage_end && end == 0xFFFFFFFFu; off += 512) {
                    const uint32_t p0 = off + C.lane * 16u;
                    uint32_t bits = 0;
                    if (p0 < stage_end) {
                        if (p0 + 16 <= stage_end && (p0 & 15u) == 0) {
                            bits = eq_bits16(*reinterpret_cast<const uint4 *>(st + p0), kNl * 0x01010101u);
                        } else {
                            for (uint32_t q = 0; q < 16 && p0 + q < stage_end; ++q)
                                if (st[p0 + q] == kNl) bits |= 1u << q;
                        }
                    }
                    const uint32_t cand = bits ? p0 + (uint32_t)(__ffs(bits) - 1) : 0xFFFFFFFFu;
                    end = __reduce_min_sync(kFull, cand);
                }
            }
            if (end != 0xFFFFFFFFu) {
                last_end = end;
                last_nl = 1;
                conv_end = max(conv_end, end + 1u);
            } else if (stage_hi == A.n) {
                last_end = stage_end;
                conv_end = stage_end;
            } else {
                last_long = 1;  // the slow path reads this line from global memory
            }
        }
        to_classes(C, S, conv_end);
        if (C.lane == 0) {
            S.Lt = Lt;
            S.first_start = first_start;
            S.last_end = last_end;
            S.last_nl = last_nl;
            S.last_long = last_long;
            S.nown = nown;
        }
        __syncwarp();
    }

    // Lines [r0, r1) of the staged tile: starts, extents, length sort, encode, output offsets.
    // Returns the batch's output bytes; *any_slow reports slow-path lines.
    static __device__ uint64_t prepare_batch(const Ctx &C, Slot &S, uint64_t t, uint32_t r0, uint32_t r1, bool *any_slow)
    {
        const ShardView &A = *C.A;
        WarpMem &M = *C.M;
        const uint32_t lane = C.lane;
        uint8_t *st = S.st;
        const uint32_t nb = r1 - r0, Lt = S.Lt, first_start = S.first_start;
        const uint32_t lim = 15u + S.nown;
        const uint64_t base = tile_base(t);
        const uint8_t *gbase = A.in + base - 16;  // global address of staged byte 0

        if (lane == 0 && first_start && r0 == 0) S.start[0] = 16;
        {
            uint32_t rank = first_start;
    #pragma unroll 1
            for (int it = 0; it < (kTW + 511) / 512; ++it) {
                const uint32_t p0 = 16u + it * 512u + lane * 16u;
                uint32_t bits = nl_bits_masked(st, p0, lim);
                const uint32_t c = __popc(bits);
                const uint32_t inc = warp_incl_u32(c);
                uint32_t rk = rank + inc - c;
                while (bits) {
                    const int q = __ffs(bits) - 1;
                    bits &= bits - 1;
                    if (rk >= r0 && rk <= r1) S.start[rk - r0] = (uint16_t)(p0 + (uint32_t)q + 1u);
                    ++rk;
                }
                rank += __shfl_sync(kFull, inc, 31);
            }
        }
        M.hist[lane] = 0;
        M.hist[lane + 32] = 0;
        __syncwarp();
        for (uint32_t r = lane; r < nb; r += 32) {
            const uint32_t s = S.start[r];
            uint32_t end;
            uint8_t fl;
            if (r0 + r + 1 < Lt) {
                end = (uint32_t)S.start[r + 1] - 1u;
                fl = kLfNl;
            } else if (S.last_long) {
                end = s;  // found by the slow path
                fl = kLfSlow;
            } else {
                end = S.last_end;
                fl = S.last_nl ? kLfNl : 0;
            }
            const uint32_t len = end - s;
            S.plen[r] = (uint16_t)min(len, 65535u);
            S.flag[r] = fl;
            const uint32_t bucket = 63u - min(len >> 3, 63u);
            S.olen[r] = bucket;
            S.soff[r] = atomicAdd(&M.hist[bucket], 1u);
        }
        __syncwarp();
        {
            const uint32_t h0 = M.hist[2 * lane], h1 = M.hist[2 * lane + 1];
            const uint32_t ex = warp_incl_u32(h0 + h1) - (h0 + h1);
            M.hist[2 * lane] = ex;
            M.hist[2 * lane + 1] = ex + h0;
        }
        __syncwarp();
        for (uint32_t r = lane; r < nb; r += 32) S.perm[M.hist[S.olen[r]] + S.soff[r]] = (uint8_t)r;
        __syncwarp();

        // Lines go to lanes longest first in snake order (round k: lane l takes sorted line 32k + l for even
        // k, 32k + 31 - l for odd k), so a lane with a long line in one round gets a short one in the next.
        bool lane_slow = false;
        for (uint32_t q0 = 0; q0 < nb; q0 += 32) {
            const uint32_t qd = q0 + ((q0 & 32u) ? 31u - lane : lane);
            if (qd >= nb) continue;
            const uint32_t r = S.perm[qd];
            const uint32_t a = S.start[r];
            uint8_t fl = S.flag[r];
            uint32_t n = S.plen[r];
            uint32_t cost = 0;
            bool slow = (fl & kLfSlow) != 0;
            if (!slow) {
                bool modified = false;
                int m = (int)n;
                if (C.P->flags & ZS_PREPROCESS) {
                    m = preprocess_bits(st, M.imask, kImaskChunks, a, n, n <= kBitMax, M.tok + lane,
                                               &modified);
                    if (m == -2)
                        m = preprocess_classes(st, M.imask, a, n, gbase + a, C, M.tok + lane, &modified);
                }
                if (m < 0) {
                    slow = true;
                } else {
                    bool esc = false;
                    cost = parse_classes(st, a, (uint32_t)m, C, &esc);
                    // escapes of other bytes are emitted from the input bytes, whose positions a compacted
                    // (%nn-shortened) line no longer matches
                    if (esc && modified && (!C.P->esc_digits || m != (int)n)) slow = true;
                    n = (uint32_t)m;
                }
            }
            if (slow) {
                const uint64_t gs = base - 16 + a;
                uint64_t glen;
                if (fl & kLfSlow) {
                    uint64_t ge = gs;
                    while (ge < A.n && A.in[ge] != kNl) ++ge;
                    if (ge < A.n) fl |= kLfNl;
                    glen = ge - gs;
                } else {
                    glen = S.plen[r];
                }
                cost = 0;
                n = 0;
                S.soff[r] = 0xFFFFFFFFu;
                if (glen >= kLongLine) {
                    atomicOr(C.status, kStTooBig);
                } else {
                    const SlowLayout sl = slow_layout((uint32_t)glen);
                    const unsigned long long off = atomicAdd(&C.P->g->slow_used, (unsigned long long)sl.need);
                    if (off + sl.need > C.P->slow_cap) {
                        atomicOr(C.status, kStSlowOverflow);
                    } else {
                        uint8_t *ws = C.P->slow + off;
                        uint32_t m;
                        if (C.P->flags & ZS_PREPROCESS) {
                            m = preprocess_slow(A.in + gs, (uint32_t)glen, ws + sl.text, ws + sl.tok,
                                                reinterpret_cast<int32_t *>(ws + sl.tables),
                                                reinterpret_cast<int32_t *>(ws + sl.tables) + 100,
                                                OUTER);
                        } else {
                            for (uint32_t i = 0; i < glen; ++i) ws[sl.text + i] = A.in[gs + i];
                            m = (uint32_t)glen;
                        }
                        cost = parse_global(ws + sl.text, ws + sl.chs, m, C);
                        reinterpret_cast<uint32_t *>(ws)[0] = (uint32_t)glen;
                        reinterpret_cast<uint32_t *>(ws)[1] = m;
                        S.soff[r] = (uint32_t)(off >> 4);
                    }
                }
                fl |= kLfSlow;
                lane_slow = true;
            }
            S.flag[r] = fl;
            S.plen[r] = (uint16_t)min(n, 65535u);
            S.olen[r] = cost + ((fl & kLfNl) ? 1u : 0u);
        }
        *any_slow = __any_sync(kFull, lane_slow);
        __syncwarp();

        const uint32_t per = (nb + 31) / 32;
        uint64_t local = 0;
        for (uint32_t k = 0; k < per; ++k) {
            const uint32_t r = lane * per + k;
            if (r < nb) local += S.olen[r];
        }
        uint64_t inc = local;
    #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t u = __shfl_up_sync(kFull, inc, o);
            if (lane >= (uint32_t)o) inc += u;
        }
        const uint64_t btotal = __shfl_sync(kFull, inc, 31);
        {
            uint64_t acc = inc - local;
            for (uint32_t k = 0; k < per; ++k) {
                const uint32_t r = lane * per + k;
                if (r < nb) {
                    const uint32_t o = S.olen[r];
                    S.olen[r] = (uint32_t)acc;  // output bytes become the output offset
                    acc += o;
                }
            }
        }
        if (lane == 0 && btotal >= 0xFFFFFFFFull) atomicOr(C.status, kStTooBig);
        __syncwarp();
        return btotal;
    }

    // Emit lines [0, nb) of slot S at output offset out_at (lines numbered from line0).
    static __device__ void emit_batch(const Ctx &C, Slot &S, uint64_t t, uint32_t nb, uint64_t out_at, uint64_t line0,
                               uint64_t btotal, bool staged)
    {
        const ShardView &A = *C.A;
        WarpMem &M = *C.M;
        const uint32_t lane = C.lane;
        const uint8_t *gbase = A.in + tile_base(t) - 16;
        const uint32_t so = (uint32_t)(((uint64_t)(uintptr_t)A.out + out_at) & 15u);
        for (uint32_t q0 = 0; q0 < nb; q0 += 32) {  // the same snake order as the encode loop
            const uint32_t qd = q0 + ((q0 & 32u) ? 31u - lane : lane);
            if (qd >= nb) continue;
            const uint32_t r = S.perm[qd];
            const uint32_t a = S.start[r];
            const uint8_t fl = S.flag[r];
            const uint32_t loff = S.olen[r];  // the output offset by now
            if (A.index && line0 + r < A.index_cap) A.index[line0 + r] = out_at + loff;
            if (fl & kLfSlow) {
                if (S.soff[r] == 0xFFFFFFFFu) continue;
                uint8_t *ws = C.P->slow + ((uint64_t)S.soff[r] << 4);
                const uint32_t glen = reinterpret_cast<const uint32_t *>(ws)[0];
                const uint32_t m = reinterpret_cast<const uint32_t *>(ws)[1];
                const SlowLayout sl = slow_layout(glen);
                GlobalSink sink{A.out, out_at + loff, A.out_cap};
                if (C.P->esc_digits) emit_line<true>(ws + sl.chs, ws + sl.text, m, C.plen_tab, sink);
                else emit_line<false>(ws + sl.chs, ws + sl.text, m, C.plen_tab, sink);
                if (fl & kLfNl) sink.put(kNl);
            } else if (staged) {
                SmemSink sink{M.ost + so + loff};
                if (C.P->esc_digits) emit_line<true>(S.st + a, gbase + a, S.plen[r], C.plen_tab, sink);
                else emit_line<false>(S.st + a, gbase + a, S.plen[r], C.plen_tab, sink);
                if (fl & kLfNl) sink.put(kNl);
            } else {
                GlobalSink sink{A.out, out_at + loff, A.out_cap};
                if (C.P->esc_digits) emit_line<true>(S.st + a, gbase + a, S.plen[r], C.plen_tab, sink);
                else emit_line<false>(S.st + a, gbase + a, S.plen[r], C.plen_tab, sink);
                if (fl & kLfNl) sink.put(kNl);
            }
        }
        __syncwarp();
        if (staged)
            warp_copy_out(M.ost, so, btotal, A.out + out_at, A.out_cap > out_at ? A.out_cap - out_at : 0);
        __syncwarp();
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

    // Encode a tile of at most kMaxLW lines and publish its aggregate.
    static __device__ void encode_single(const Ctx &C, Slot &S, uint64_t t)
    {
        bool any_slow = false;
        const uint64_t btotal = prepare_batch(C, S, t, 0, S.Lt, &any_slow);
        if (C.lane == 0) {
            S.btotal = btotal;
            S.any_slow = any_slow ? 1u : 0u;
            if ((int64_t)t != C.P->stall_tile) publish(&C.A->tiles[t], t == 0 ? 2u : 1u, btotal, S.Lt);
        }
        __syncwarp();
    }

    // Resolve the offset of an encoded tile and emit it.
    static __device__ void finish_single(const Ctx &C, Slot &S, uint64_t t)
    {
        const ShardView &A = *C.A;
        uint64_t ea = 0, eb = 0;
        if (t > 0) lookback_warp(A.tiles, t, &ea, &eb, C.P->limit_ns, C.status);
        const uint64_t btotal = S.btotal;
        const uint32_t Lt = S.Lt;
        if (C.lane == 0 && t > 0 && (int64_t)t != C.P->stall_tile) publish(&A.tiles[t], 2u, ea + btotal, eb + Lt);
        const bool staged = !S.any_slow && btotal + 48 <= (uint64_t)kOutW;
        emit_batch(C, S, t, Lt, ea, eb, btotal, staged);
        finish_result(C, t, ea + btotal, eb + Lt);
    }

    // A tile with more lines than one batch holds: look back first, then encode and emit batch by batch.
    static __device__ void process_batched(const Ctx &C, Slot &S, uint64_t t)
    {
        const ShardView &A = *C.A;
        const uint32_t Lt = S.Lt;
        uint64_t ea = 0, eb = 0;
        if (t > 0) lookback_warp(A.tiles, t, &ea, &eb, C.P->limit_ns, C.status);
        uint64_t run = 0;
        for (uint32_t r0 = 0; r0 < Lt; r0 += kMaxLW) {
            const uint32_t r1 = min(Lt, r0 + kMaxLW);
            bool any_slow = false;
            const uint64_t btotal = prepare_batch(C, S, t, r0, r1, &any_slow);
            emit_batch(C, S, t, r1 - r0, ea + run, eb + r0, btotal, false);
            run += btotal;
        }
        if (C.lane == 0 && (int64_t)t != C.P->stall_tile) publish(&A.tiles[t], 2u, ea + run, eb + Lt);
        finish_result(C, t, ea + run, eb + Lt);
        __syncwarp();
    }

    static __device__ void run(const CwArgs *P)
    {
        extern __shared__ __align__(128) uint8_t smem[];
        __shared__ uint64_t img_bar;
        const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        WarpMem &M = reinterpret_cast<WarpMem *>(smem)[wid];
        uint8_t *img = smem + kMW * sizeof(WarpMem);
        Ctx C;
        C.P = P;
        C.A = nullptr;
        C.M = &M;
        C.clsrep = img + kMOffClsRep;
        C.plen_tab = img + kMOffPlen;
        C.T = reinterpret_cast<const uint32_t *>(img + kMOffTable);
        C.nc = P->n_classes;
        C.q0 = P->start_state;
        C.lane = lane;
        C.status = &P->g->status;

        if (threadIdx.x == 0) mbar_init(&img_bar, 1);
        if (lane == 0) {
            mbar_init(&M.slot[0].bar, 1);
            mbar_init(&M.slot[1].bar, 1);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_arrive_tx(&img_bar, P->img_bytes);
            bulk_g2s(img, P->mimg, P->img_bytes, &img_bar);
        }
        if (!mbar_wait_bounded(&img_bar, 0, P->limit_ns, C.status)) {
            mbar_wait_bounded(&img_bar, 0, P->limit_ns, C.status);
            return;
        }

        uint32_t ph = 0;  // phase bit of each slot's barrier (bit s)
        uint32_t s = 0;
        bool pending = false;
        uint64_t t_pend = 0;
        auto finish_pending = [&]() {
            Ctx Cp = C;
            Cp.A = &M.slot[s ^ 1u].sv;
            finish_single(Cp, M.slot[s ^ 1u], t_pend);
        };
        for (;;) {
            unsigned long long tt = 0;
            if (lane == 0) tt = atomicAdd(&P->g->tile_counter, 1ull);
            const uint64_t g = __shfl_sync(kFull, tt, 0);
            if (g >= P->total_tiles) break;
            Slot &S = M.slot[s];
            const uint32_t sh = P->n_shards == 1 ? 0u : find_shard(P->shards, P->n_shards, g);
            load_shard(&S.sv, P->one, P->shards, P->n_shards, sh);
            const uint64_t t = g - S.sv.tile0;  // tile number within the shard
            Ctx Cs = C;
            Cs.A = &S.sv;
            stage_issue(Cs, S, t);
            if (!mbar_wait_bounded(&S.bar, (ph >> s) & 1u, P->limit_ns, C.status)) {
                mbar_wait_bounded(&S.bar, (ph >> s) & 1u, P->limit_ns, C.status);
                return;
            }
            ph ^= 1u << s;
            __syncwarp();
            segment(Cs, S, t);
            if (S.Lt <= (uint32_t)kMaxLW) {
                encode_single(Cs, S, t);
                if (pending) finish_pending();
                pending = true;
                t_pend = t;
                s ^= 1u;
            } else {
                if (pending) finish_pending();
                pending = false;
                process_batched(Cs, S, t);
            }
        }
        if (pending) finish_pending();
    }
};

template <class Geo, bool OUTER>
__global__ void __launch_bounds__(Geo::kWarps * 32, 1) compress_warp_kernel(const CwArgs P)
{
    CW<Geo, OUTER>::run(&P);
}

// The compiled geometries. Variant 0 (about 30 lines of 46 bytes per warp tile, so mostly one lane round;
// 20 warps per SM, five per scheduler, the most that keep 96 registers a thread) is the default, and
// variant 1 the same tile with 19 warps for a dictionary whose transducer image leaves too little shared
// memory for 20; variant 2 keeps long lines (hundreds of bytes) several to a tile; variant 3 (about 60
// lines per tile: two lane rounds, which the snake order balances) suits a mix with a long tail of lines.
using CwV0 = CwGeom<20, 1408, 512, 64, 960, 26>;
using CwV1 = CwGeom<19, 1408, 512, 64, 960, 26>;
using CwV2 = CwGeom<8, 4096, 1024, 192, 1728, 26>;
using CwV3 = CwGeom<12, 2816, 512, 128, 1920, 26>;

template <class Geo>
size_t cw_smem(const zs_dict *d)
{
    return CW<Geo, false>::kMW * sizeof(typename CW<Geo, false>::WarpMem) + d->mlayout.img_bytes;
}

template <class Geo, bool OUTER>
cudaError_t cw_launch_as(const zs_dict *d, const TiledLaunch &L, unsigned flags, cudaStream_t s)
{
    CwArgs a{};
    a.one = L.one;
    a.shards = L.shards;
    a.n_shards = L.n_shards;
    a.flags = flags;
    a.total_tiles = L.total_tiles;
    a.mimg = d->d_mimg;
    a.img_bytes = d->mlayout.img_bytes;
    a.n_classes = d->mlayout.n_classes;
    a.start_state = d->mlayout.start;
    a.esc_digits = d->mlayout.esc_digits;
    a.g = L.g;
    a.slow = L.slow;
    a.slow_cap = L.slow_cap;
    a.limit_ns = wait_limit_ns();
    a.stall_tile = injected_stall_tile();
    const int smem = (int)cw_smem<Geo>(d);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    static int set_smem = -1;
    if (set_smem != smem) {
        cudaError_t e = cudaFuncSetAttribute(compress_warp_kernel<Geo, OUTER>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        set_smem = smem;
    }
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, compress_warp_kernel<Geo, OUTER>, CW<Geo, OUTER>::kMNT,
                                                  smem);
    if (per < 1) per = 1;
    uint64_t grid = std::min<uint64_t>((L.total_tiles + Geo::kWarps - 1) / Geo::kWarps, (uint64_t)per * (uint64_t)sms);
    if (grid == 0) grid = 1;
    compress_warp_kernel<Geo, OUTER><<<(unsigned)grid, CW<Geo, OUTER>::kMNT, smem, s>>>(a);
    return cudaGetLastError();
}

template <class Geo>
cudaError_t cw_launch(const zs_dict *d, const TiledLaunch &L, unsigned flags, cudaStream_t s)
{
    return (flags & ZS_PREPROCESS_OUTER) ? cw_launch_as<Geo, true>(d, L, flags, s)
                                         : cw_launch_as<Geo, false>(d, L, flags, s);
}

struct CwEntry {
    KernelVariant info;
    size_t (*smem)(const zs_dict *);
    cudaError_t (*launch)(const zs_dict *, const TiledLaunch &, unsigned, cudaStream_t);
};

template <class Geo>
constexpr CwEntry cw_entry(const char *name)
{
    return CwEntry{KernelVariant{name, Geo::kWarps, Geo::kTile}, &cw_smem<Geo>, &cw_launch<Geo>};
}

const CwEntry kCw[] = {
    cw_entry<CwV0>("compress w20 t1408"),
    cw_entry<CwV1>("compress w19 t1408"),
    cw_entry<CwV2>("compress w8 t4096"),
    cw_entry<CwV3>("compress w12 t2816"),
};
constexpr int kNumCw = (int)(sizeof(kCw) / sizeof(kCw[0]));

}  // namespace

// Variant numbering of the tiled compression kernels: the span kernel's geometries first
// (compress_span.cu), then this kernel's.
int compress_warp_variants() { return span_variants() + kNumCw; }

const KernelVariant *compress_warp_variant(int v)
{
    const int ns = span_variants();
    if (v >= 0 && v < ns) return span_variant(v);
    v -= ns;
    return (v >= 0 && v < kNumCw) ? &kCw[v].info : nullptr;
}

bool compress_warp_fits(int v, const zs_dict *d)
{
    const int ns = span_variants();
    if (v >= 0 && v < ns) return span_fits(v, d);
    v -= ns;
    if (v < 0 || v >= kNumCw || !d->has_machine) return false;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return kCw[v].smem(d) <= (size_t)optin;
}

bool compress_variant_is_span(int v) { return v >= 0 && v < span_variants(); }

cudaError_t launch_compress_warp(int v, const zs_dict *d, const TiledLaunch &L, unsigned flags, cudaStream_t s)
{
    const int ns = span_variants();
    if (v >= 0 && v < ns) return launch_span(v, d, L, flags, s);
    v -= ns;
    if (v < 0 || v >= kNumCw) return cudaErrorInvalidValue;
    return kCw[v].launch(d, L, flags, s);
}

}  // namespace zs
