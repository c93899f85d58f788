// zs_compress: ring-ID pre-processing (Sec. IV-A) + minimum-length dictionary parse (Sec. IV-D1) of every
// line of a stream, in one persistent single-pass kernel.
//
// Work decomposition
//   - The input is cut into tiles of kTB bytes. A tile owns the lines that START inside it and reads up
//     to kHalo bytes past its end to finish its last line. Tiles are claimed in launch order through an
//     atomic counter, so every tile's predecessors are already running (forward progress for the scan).
//   - Staging: one bulk (TMA) copy moves the tile (plus the byte before it and the halo) into shared
//     memory; the encoder tables are bulk-copied once per CTA.
//   - Segmentation: each warp scans 2 KiB with 16-byte shared loads, finds '\n' bytes with SIMD-in-word
//     compares, and ranks line starts with warp prefix sums.
//   - Lines are sorted by length (counting sort) and dealt to threads so that the 32 lanes of a warp get
//     lines of similar length; each lane then runs one line: pre-processing in place, then the backward
//     shortest-path scan driven by a reverse Aho-Corasick automaton (one shared-memory lookup per byte
//     gives every dictionary match starting at that byte), which overwrites each byte with the symbol
//     chosen there.
//   - Output offsets and line numbers come from a block scan plus a decoupled look-back across tiles.
//   - Emission walks the chosen symbols front to back into a shared staging buffer aligned to the
//     output's 16-byte grid, which is then written with coalesced 16-byte stores.
//   - Lines longer than the halo, or whose pre-processing needs a 3-byte %nn label or more than 16 open
//     rings, or that both had ring labels rewritten and need an escape, take an exact slow path in global
//     scratch.
#include <algorithm>

#include "compress_shared.cuh"

namespace zs {
namespace {
using namespace cx;

constexpr int kNT = 256;                  // threads per CTA
constexpr int kTB = 16384;                // owned bytes per tile
constexpr int kHalo = 4096;               // bytes read past the tile to finish its last line
constexpr int kStage = 16 + kTB + kHalo;  // staging: 16 bytes before the tile, the tile, the halo
constexpr int kMaxL = 1024;               // lines handled per batch
constexpr int kOutCap = 16384 + 64;       // staged output bytes per tile
constexpr int kSlowOpen = 16;             // open rings tracked by the in-place pre-processor
constexpr uint32_t kLongLine = 1u << 30;  // longest line the slow path accepts

static_assert(kTB == (kNT / 32) * 2048, "each warp segments 2 KiB");

// line flag bits
constexpr uint8_t kLfNl = 1, kLfSlow = 2;

struct CompressArgs {
    const uint8_t *in;
    uint64_t n;
    uint8_t *out;
    uint64_t out_cap;
    uint64_t *index;
    uint64_t index_cap;
    uint32_t flags;
    uint32_t in_aligned;
    uint64_t ntiles;
    const uint8_t *enc;
    EncLayout L;
    DevResult *res;
    TileState *tiles;
    uint8_t *slow;
    uint64_t slow_cap;
    uint64_t limit_ns;
    int64_t stall_tile;
};

// ---- shared memory carve-up ----
constexpr int align16(int x) { return (x + 15) & ~15; }
constexpr int kOffStage = 0;
constexpr int kOffOut = kOffStage + align16(kStage + 16);
constexpr int kOffStart = kOffOut + align16(kOutCap + 32);
constexpr int kOffPlenL = kOffStart + align16(2 * (kMaxL + 1));
constexpr int kOffOlen = kOffPlenL + align16(2 * kMaxL);
constexpr int kOffLoff = kOffOlen + align16(4 * kMaxL);
constexpr int kOffSoff = kOffLoff + align16(4 * kMaxL);
constexpr int kOffPerm = kOffSoff + align16(4 * kMaxL);
constexpr int kOffTmp = kOffPerm + align16(2 * kMaxL);
constexpr int kOffFlag = kOffTmp + align16(2 * kMaxL);
constexpr int kOffHist = kOffFlag + align16(kMaxL);
constexpr int kOffScan = kOffHist + align16(4 * 128);
constexpr int kOffWarp = kOffScan + align16(8 * (kNT / 32 + 2));
constexpr int kOffVars = kOffWarp + align16(4 * (kNT / 32 + 1));
constexpr int kOffBar = kOffVars + align16(8 * 24);
constexpr int kOffDict = kOffBar + 16;
constexpr int kSmemFixed = kOffDict;

struct Vars {
    uint64_t tile;
    uint64_t E_a, E_b;        // exclusive prefix: output bytes, lines
    uint64_t run_a;           // running output offset within the tile (multi-batch)
    uint32_t L;               // lines starting in the tile
    uint32_t first_start;     // 1 if the tile's first byte starts a line
    uint32_t last_end;        // staging index of the newline (or end) of the tile's last line
    uint32_t last_nl;         // last line ends with '\n'
    uint32_t last_long;       // last line extends past the halo
    uint32_t any_slow;
    uint32_t staged;          // emission goes through the shared staging buffer
    uint32_t stage_off;       // (absolute output address) & 15
    uint64_t batch_total;
    uint32_t halo_hit;
    uint32_t pad;
};

// Block exclusive scan of 64-bit values (NT threads).
__device__ __forceinline__ uint64_t block_excl_u64(uint64_t v, uint64_t *tmp, uint64_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) tmp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = lane < kNT / 32 ? tmp[lane] : 0ull;
        uint64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t u = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += u;
        }
        if (lane < kNT / 32) tmp[lane] = wi - w;
        if (lane == kNT / 32 - 1) tmp[kNT / 32] = wi;
    }
    __syncthreads();
    uint64_t r = tmp[warp] + inc - v;
    *total = tmp[kNT / 32];
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------------------------------------
// Pre-processing, fast path: in place in shared memory (Sec. IV-A).
//
// Streaming form of "label intervals in ascending closing order with the smallest label not held by an
// already-labelled overlapping interval": an interval that closes now overlaps every earlier-closed
// interval that closed after it opened, so label x is taken iff the latest interval labelled x closed
// after this one opened. lc[x] keeps (that close position + 1). The opening token is written as a
// placeholder and patched when its ring closes; %nn labels shrink to one digit as they are copied.
// With outer (rings labelled in opening order), an opening ring takes at once the smallest label no open
// ring holds (held: bit x set while label x is held) and its closing token copies it.
// Returns the new length, or -1 when the line needs the slow path (label >= 10, more than kSlowOpen
// open rings). *modified is set if any ring label was rewritten (the line no longer equals its input
// bytes). Invalid lines are restored from global memory.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ int preprocess_inplace(uint8_t *st, int a, int n, const uint8_t *gsrc, bool *modified,
                                                  bool outer)
{
    const uint32_t kEmpty = 0xFFFFFFFFu;
    uint32_t slot[kSlowOpen];
#pragma unroll
    for (int k = 0; k < kSlowOpen; ++k) slot[k] = kEmpty;
    uint32_t lc[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) lc[k] = 0;
    int nopen = 0;
    uint32_t held = 0;
    int w = 0, r = 0;
    bool in_br = false, bad = false;
    *modified = false;
    while (r < n) {
        uint8_t c = st[a + r];
        if (c == ' ' || c == '\t') {  // end of the SMILES field: the rest is copied verbatim
            if (w != r) {
                for (; r < n; ++r, ++w) st[a + w] = st[a + r];
            } else {
                w = n;
                r = n;
            }
            break;
        }
        if (in_br) {
            if (c == ']') in_br = false;
        } else if (c == '[') {
            in_br = true;
        } else if ((c >= '0' && c <= '9') || c == '%') {
            int lab, tl;
            if (c == '%') {
                if (r + 2 >= n) { bad = true; break; }
                uint8_t d1 = st[a + r + 1], d2 = st[a + r + 2];
                if (d1 < '0' || d1 > '9' || d2 < '0' || d2 > '9') { bad = true; break; }
                lab = (d1 - '0') * 10 + (d2 - '0');
                tl = 3;
            } else {
                lab = c - '0';
                tl = 1;
            }
            int hit = -1;
            uint32_t o = 0;
#pragma unroll
            for (int k = 0; k < kSlowOpen; ++k)
                if ((slot[k] & 0xFFu) == (uint32_t)lab) {
                    hit = k;
                    o = slot[k] >> 8;
                }
            if (hit >= 0 && outer) {  // closes the ring opened at write position o: same label
                const uint32_t nl = (uint32_t)(st[a + (int)o] - '0');
                st[a + w] = (uint8_t)('0' + nl);
                held &= ~(1u << nl);
#pragma unroll
                for (int k = 0; k < kSlowOpen; ++k)
                    if (k == hit) slot[k] = kEmpty;
                --nopen;
            } else if (hit >= 0) {  // closes the ring opened at write position o
                int nl = -1;
#pragma unroll
                for (int x = 9; x >= 0; --x)
                    if (lc[x] <= o + 1) nl = x;
                if (nl < 0) return -1;  // needs a two-digit label
                st[a + (int)o] = (uint8_t)('0' + nl);
                st[a + w] = (uint8_t)('0' + nl);
#pragma unroll
                for (int x = 0; x < 10; ++x)
                    if (x == nl) lc[x] = (uint32_t)w + 1;
#pragma unroll
                for (int k = 0; k < kSlowOpen; ++k)
                    if (k == hit) slot[k] = kEmpty;
                --nopen;
            } else {  // opens a ring
                if (nopen == kSlowOpen) return -1;
                bool done = false;
#pragma unroll
                for (int k = 0; k < kSlowOpen; ++k)
                    if (!done && slot[k] == kEmpty) {
                        slot[k] = ((uint32_t)w << 8) | (uint32_t)lab;
                        done = true;
                    }
                ++nopen;
                if (outer) {
                    const uint32_t fr = ~held & 0x3FFu;
                    if (fr == 0) return -1;  // needs a two-digit label
                    const int nl = __ffs(fr) - 1;
                    held |= 1u << nl;
                    st[a + w] = (uint8_t)('0' + nl);
                } else {
                    st[a + w] = '0';
                }
            }
            w += 1;
            r += tl;
            *modified = true;
            continue;
        }
        if (w != r) st[a + w] = c;
        ++w;
        ++r;
    }
    if (bad || in_br || nopen > 0) {  // not a well-formed ring structure: the line stays as it is
        for (int i = 0; i < n; ++i) st[a + i] = gsrc[i];
        *modified = false;
        return n;
    }
    return w;
}

// ------------------------------------------------------------------------------------------------
// Backward shortest-path scan (Sec. IV-D1). best[i] = min(best[i+1] + (s[i] in D ? 1 : 2),
// min over matches l >= 2 at i of best[i+l] + 1); ties go to the longest piece (an escape loses to
// everything). Writes at choice[i] the symbol chosen at i (kEsc for an escape); text and choice may
// alias (each byte is read before it is overwritten). Returns best[0] = compressed length.
// ------------------------------------------------------------------------------------------------
template <int LMAX, bool COMPACT, class TP, class CP>
__device__ __forceinline__ uint32_t parse_backward(TP text, CP choice, uint32_t n, const uint8_t *enc,
                                                   uint32_t n_classes, uint32_t off_trans, uint32_t off_sym,
                                                   bool *esc)
{
    const uint8_t *cls = enc + kOffCls;
    const uint32_t *masks = reinterpret_cast<const uint32_t *>(enc + kOffMasks);
    const uint16_t *t16 = reinterpret_cast<const uint16_t *>(enc + off_trans);
    const uint32_t *t32 = reinterpret_cast<const uint32_t *>(enc + off_trans);
    const uint8_t *sym = enc + off_sym;
    uint32_t w[LMAX];
#pragma unroll
    for (int l = 0; l < LMAX; ++l) w[l] = 0;
    uint32_t state = 0;
    bool e = false;
    for (uint32_t i = n; i-- > 0;) {
        uint8_t c = text[i];
        uint32_t idx = state * n_classes + cls[c];
        uint32_t mask;
        if (COMPACT) {
            uint32_t t = t16[idx];
            state = t & 0x7FFu;
            mask = masks[t >> 11];
        } else {
            uint32_t t = t32[idx];
            state = t & 0xFFFFu;
            mask = t >> 16;
        }
        uint32_t best = w[0] + ((mask & 1u) ? 1u : 2u);
        uint32_t pick = 1;
#pragma unroll
        for (int l = 2; l <= LMAX; ++l) {
            uint32_t cand = w[l - 1] + 1u;
            if (((mask >> (l - 1)) & 1u) && cand <= best) {
                best = cand;
                pick = (uint32_t)l;
            }
        }
        uint8_t out;
        if (pick == 1 && !(mask & 1u)) {
            out = kEsc;
            e = true;
        } else {
            out = sym[state * 16u + pick - 1u];
        }
        choice[i] = out;
#pragma unroll
        for (int l = LMAX - 1; l > 0; --l) w[l] = w[l - 1];
        w[0] = best;
    }
    *esc = e;
    return w[0];
}

template <int LMAX, bool COMPACT>
__global__ void __launch_bounds__(kNT) compress_kernel(CompressArgs A)
{
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t *st = smem + kOffStage;
    uint8_t *ost = smem + kOffOut;
    uint16_t *s_start = reinterpret_cast<uint16_t *>(smem + kOffStart);
    uint16_t *s_plen = reinterpret_cast<uint16_t *>(smem + kOffPlenL);
    uint32_t *s_olen = reinterpret_cast<uint32_t *>(smem + kOffOlen);
    uint32_t *s_loff = reinterpret_cast<uint32_t *>(smem + kOffLoff);
    uint32_t *s_soff = reinterpret_cast<uint32_t *>(smem + kOffSoff);
    uint16_t *s_perm = reinterpret_cast<uint16_t *>(smem + kOffPerm);
    uint16_t *s_tmp = reinterpret_cast<uint16_t *>(smem + kOffTmp);
    uint8_t *s_flag = smem + kOffFlag;
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(smem + kOffHist);
    uint64_t *s_scan = reinterpret_cast<uint64_t *>(smem + kOffScan);
    uint32_t *s_warp = reinterpret_cast<uint32_t *>(smem + kOffWarp);
    Vars *V = reinterpret_cast<Vars *>(smem + kOffVars);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kOffBar);
    uint8_t *enc = smem + kOffDict;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const EncLayout &L = A.L;
    uint32_t *status = &A.res->status;

    if (tid == 0) mbar_init(bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    if (tid == 0) {
        mbar_arrive_tx(bar, L.img_bytes);
        bulk_g2s(enc, A.enc, L.img_bytes, bar);
    }
    if (!mbar_wait_bounded(bar, phase, A.limit_ns, status)) {
        mbar_wait_bounded(bar, phase, A.limit_ns, status);
        return;
    }
    phase ^= 1u;
    const uint8_t *plen_tab = enc + kOffPlen;

    for (;;) {
        if (tid == 0) V->tile = atomicAdd(&A.res->tile_counter, 1ull);
        __syncthreads();
        const uint64_t t = V->tile;
        if (t >= A.ntiles) break;

        const uint64_t base = t * (uint64_t)kTB;
        const uint64_t own_end = min(A.n, base + kTB);
        const uint32_t nown = (uint32_t)(own_end - base);
        const uint64_t stage_hi = min(A.n, base + (uint64_t)kTB + kHalo);
        const uint64_t lo = base >= 16 ? base - 16 : 0;  // global position of staging index j0
        const uint32_t j0 = (uint32_t)(lo + 16 - base);  // 16 - (base - lo): 0, or 16 for tile 0
        const uint32_t nbytes = (uint32_t)(stage_hi - lo);
        const uint32_t stage_end = j0 + nbytes;          // staging index one past the last staged byte
        const uint8_t *gbase = A.in + base - 16;         // staging index j <-> gbase[j] (never read below 16 for t=0)

        // ---- stage the tile ----
        const uint32_t nbulk = A.in_aligned ? (nbytes & ~15u) : 0u;
        if (tid == 0) {
            fence_proxy_async_smem();
            mbar_arrive_tx(bar, nbulk);
            if (nbulk) bulk_g2s(st + j0, A.in + lo, nbulk, bar);
        }
        for (uint32_t j = nbulk + tid; j < nbytes; j += kNT) st[j0 + j] = A.in[lo + j];
        if (t == 0 && tid == 0) st[15] = kNl;  // position 0 starts a line
        if (!mbar_wait_bounded(bar, phase, A.limit_ns, status)) {
            mbar_wait_bounded(bar, phase, A.limit_ns, status);
            return;
        }
        phase ^= 1u;
        __syncthreads();

        // ---- segmentation: newline count per warp segment [16 + 2048 w, +2048) ----
        // a newline at staging p (16 <= p < 15 + nown) starts a line at p + 1; index 16 starts one if st[15] is '\n'
        const uint32_t lim = 15u + nown;  // newlines at p >= lim do not start an owned line
        uint32_t wcount = 0;
        for (int it = 0; it < 4; ++it) {
            uint32_t p0 = 16u + (uint32_t)warp * 2048u + (uint32_t)it * 512u + (uint32_t)lane * 16u;
            uint32_t bits = 0;
            if (p0 < lim) {
                uint4 v = *reinterpret_cast<const uint4 *>(st + p0);
                bits = nl_bits16(v);
                if (p0 + 16 > lim) bits &= (1u << (lim - p0)) - 1u;
            }
            wcount += __popc(bits);
        }
        wcount = __reduce_add_sync(0xffffffffu, wcount);
        if (lane == 0) s_warp[warp] = wcount;
        if (tid == 0) V->first_start = (st[15] == kNl && nown > 0) ? 1u : 0u;
        __syncthreads();
        if (tid == 0) {
            uint32_t acc = V->first_start;
            for (int w2 = 0; w2 < kNT / 32; ++w2) {
                uint32_t c = s_warp[w2];
                s_warp[w2] = acc;
                acc += c;
            }
            V->L = acc;
        }
        __syncthreads();
        const uint32_t Lt = V->L;

        // ---- end of the tile's last line (staging index of its '\n', or of the end of input) ----
        if (warp == 0 && Lt > 0) {
            uint32_t end = 0xFFFFFFFFu;
            if (nown > 0 && st[15 + nown] == kNl) {
                end = 15 + nown;
            } else {
                for (uint32_t off = 16 + nown; off < stage_end && end == 0xFFFFFFFFu; off += 512) {
                    uint32_t p0 = off + (uint32_t)lane * 16u;
                    uint32_t bits = 0;
                    if (p0 < stage_end) {
                        if (p0 + 16 <= stage_end && (p0 & 15u) == 0) {
                            bits = nl_bits16(*reinterpret_cast<const uint4 *>(st + p0));
                        } else {
                            for (uint32_t q = 0; q < 16 && p0 + q < stage_end; ++q)
                                if (st[p0 + q] == kNl) bits |= 1u << q;
                        }
                    }
                    uint32_t cand = bits ? p0 + (uint32_t)(__ffs(bits) - 1) : 0xFFFFFFFFu;
                    end = __reduce_min_sync(0xffffffffu, cand);
                }
            }
            if (lane == 0) {
                if (end != 0xFFFFFFFFu) {
                    V->last_end = end;
                    V->last_nl = 1;
                    V->last_long = 0;
                } else if (stage_hi == A.n) {
                    V->last_end = stage_end;
                    V->last_nl = 0;
                    V->last_long = 0;
                } else {
                    V->last_end = 0;
                    V->last_nl = 0;
                    V->last_long = 1;
                }
            }
        }
        if (tid == 0) {
            V->any_slow = 0;
            V->run_a = 0;
        }
        __syncthreads();

        const uint32_t nbatch = Lt == 0 ? 1u : (Lt + kMaxL - 1) / kMaxL;
        const bool single = nbatch == 1;

        for (uint32_t b = 0; b < nbatch; ++b) {
            const uint32_t r0 = b * kMaxL;
            const uint32_t r1 = min(Lt, r0 + kMaxL);
            const uint32_t nb = r1 - r0;

            // ---- starts of lines [r0, r1] (one extra to bound the batch's last line) ----
            if (tid == 0 && V->first_start && r0 == 0) s_start[0] = 16;
            {
                uint32_t rank = s_warp[warp];
                for (int it = 0; it < 4; ++it) {
                    uint32_t p0 = 16u + (uint32_t)warp * 2048u + (uint32_t)it * 512u + (uint32_t)lane * 16u;
                    uint32_t bits = 0;
                    if (p0 < lim) {
                        uint4 v = *reinterpret_cast<const uint4 *>(st + p0);
                        bits = nl_bits16(v);
                        if (p0 + 16 > lim) bits &= (1u << (lim - p0)) - 1u;
                    }
                    uint32_t c = __popc(bits);
                    uint32_t inc = warp_incl_u32(c);
                    uint32_t rk = rank + inc - c;
                    while (bits) {
                        int q = __ffs(bits) - 1;
                        bits &= bits - 1;
                        if (rk >= r0 && rk <= r1) s_start[rk - r0] = (uint16_t)(p0 + (uint32_t)q + 1u);
                        ++rk;
                    }
                    rank += __shfl_sync(0xffffffffu, inc, 31);
                }
            }
            if (tid < 128) s_hist[tid] = 0;
            __syncthreads();

            // ---- extents, length sort ----
            for (uint32_t r = tid; r < nb; r += kNT) {
                uint32_t s = s_start[r];
                uint32_t end;
                uint8_t fl;
                if (r0 + r + 1 < Lt) {
                    end = (uint32_t)s_start[r + 1] - 1u;
                    fl = kLfNl;
                } else if (V->last_long) {
                    end = s;  // unknown here; the slow path finds it
                    fl = kLfSlow;
                } else {
                    end = V->last_end;
                    fl = V->last_nl ? kLfNl : 0;
                }
                uint32_t len = end - s;
                s_plen[r] = (uint16_t)min(len, 65535u);
                s_flag[r] = fl;
                uint32_t bucket = len >= 1016u ? 127u : len >> 3;
                s_tmp[r] = (uint16_t)atomicAdd(&s_hist[127 - bucket], 1u);
                s_olen[r] = 127u - bucket;  // bucket id, reused below
            }
            __syncthreads();
            if (warp == 0) {
                uint32_t h0 = s_hist[lane * 4], h1 = s_hist[lane * 4 + 1], h2 = s_hist[lane * 4 + 2],
                         h3 = s_hist[lane * 4 + 3];
                uint32_t sum = h0 + h1 + h2 + h3;
                uint32_t ex = warp_incl_u32(sum) - sum;
                s_hist[lane * 4] = ex;
                s_hist[lane * 4 + 1] = ex + h0;
                s_hist[lane * 4 + 2] = ex + h0 + h1;
                s_hist[lane * 4 + 3] = ex + h0 + h1 + h2;
            }
            __syncthreads();
            for (uint32_t r = tid; r < nb; r += kNT) s_perm[s_hist[s_olen[r]] + s_tmp[r]] = (uint16_t)r;
            __syncthreads();

            // ---- encode: one line per lane, longest lines first ----
            for (uint32_t q = tid; q < nb; q += kNT) {
                const uint32_t r = s_perm[q];
                const uint32_t a = s_start[r];
                uint8_t fl = s_flag[r];
                uint32_t n = s_plen[r];
                uint32_t cost = 0;
                bool slow = (fl & kLfSlow) != 0;
                if (!slow) {
                    bool modified = false;
                    int m = (int)n;
                    if (A.flags & ZS_PREPROCESS)
                        m = preprocess_inplace(st, (int)a, (int)n, gbase + a, &modified,
                                               (A.flags & ZS_PREPROCESS_OUTER) != 0);
                    if (m < 0) {
                        slow = true;
                    } else {
                        bool esc = false;
                        cost = parse_backward<LMAX, COMPACT>(st + a, st + a, (uint32_t)m, enc, L.n_classes,
                                                            L.off_trans, L.off_sym, &esc);
                        // an escape is emitted from the input bytes: only valid if pre-processing changed nothing
                        if (esc && modified) slow = true;
                        n = (uint32_t)m;
                    }
                }
                if (slow) {
                    const uint64_t gs = base - 16 + a;  // input position of the line
                    uint64_t glen;
                    if (fl & kLfSlow) {                 // longer than the halo: find its end in global memory
                        uint64_t ge = gs;
                        while (ge < A.n && A.in[ge] != kNl) ++ge;
                        if (ge < A.n) fl |= kLfNl;
                        glen = ge - gs;
                    } else {
                        glen = s_plen[r];  // unchanged: the original length
                    }
                    cost = 0;
                    n = 0;
                    s_soff[r] = 0xFFFFFFFFu;
                    if (glen >= kLongLine) {
                        atomicOr(status, kStTooBig);
                    } else {
                        const SlowLayout sl = slow_layout((uint32_t)glen);
                        unsigned long long off = atomicAdd(&A.res->slow_used, (unsigned long long)sl.need);
                        if (off + sl.need > A.slow_cap) {
                            atomicOr(status, kStSlowOverflow);
                        } else {
                            uint8_t *ws = A.slow + off;
                            uint32_t m;
                            if (A.flags & ZS_PREPROCESS) {
                                m = preprocess_slow(A.in + gs, (uint32_t)glen, ws + sl.text, ws + sl.tok,
                                                    reinterpret_cast<int32_t *>(ws + sl.tables),
                                                    reinterpret_cast<int32_t *>(ws + sl.tables) + 100,
                                                    (A.flags & ZS_PREPROCESS_OUTER) != 0);
                            } else {
                                for (uint32_t i = 0; i < glen; ++i) ws[sl.text + i] = A.in[gs + i];
                                m = (uint32_t)glen;
                            }
                            bool esc = false;
                            cost = parse_backward<LMAX, COMPACT>(ws + sl.text, ws + sl.chs, m, enc, L.n_classes,
                                                                L.off_trans, L.off_sym, &esc);
                            reinterpret_cast<uint32_t *>(ws)[0] = (uint32_t)glen;
                            reinterpret_cast<uint32_t *>(ws)[1] = m;
                            s_soff[r] = (uint32_t)(off >> 4);
                        }
                    }
                    fl |= kLfSlow;
                    atomicOr(&V->any_slow, 1u);
                }
                s_flag[r] = fl;
                s_plen[r] = (uint16_t)min(n, 65535u);
                s_olen[r] = cost + ((fl & kLfNl) ? 1u : 0u);
            }
            __syncthreads();

            // ---- per-line output offsets within the batch ----
            const uint32_t per = (nb + kNT - 1) / kNT;
            uint64_t local = 0;
            for (uint32_t k = 0; k < per; ++k) {
                uint32_t r = tid * per + k;
                if (r < nb) local += s_olen[r];
            }
            uint64_t btotal;
            uint64_t ex = block_excl_u64(local, s_scan, &btotal);
            {
                uint64_t acc = ex;
                for (uint32_t k = 0; k < per; ++k) {
                    uint32_t r = tid * per + k;
                    if (r < nb) {
                        s_loff[r] = (uint32_t)acc;
                        acc += s_olen[r];
                    }
                }
            }
            if (tid == 0 && btotal >= 0xFFFFFFFFull) atomicOr(status, kStTooBig);

            // ---- publish / look back ----
            if (tid == 0) {
                V->batch_total = btotal;
                const bool stall = (int64_t)t == A.stall_tile;
                if (b == 0) {
                    uint64_t agg_lines = Lt;
                    if (single && !stall) publish(&A.tiles[t], t == 0 ? 2u : 1u, btotal, agg_lines);
                    uint64_t ea = 0, eb = 0;
                    if (t > 0) lookback(A.tiles, t, &ea, &eb, A.limit_ns, status);
                    V->E_a = ea;
                    V->E_b = eb;
                    if (single && t > 0 && !stall) publish(&A.tiles[t], 2u, ea + btotal, eb + agg_lines);
                }
                const uint64_t out_at = V->E_a + V->run_a;
                const uint64_t abs_addr = (uint64_t)(uintptr_t)(A.out) + out_at;
                V->stage_off = (uint32_t)(abs_addr & 15u);
                V->staged = (single && !V->any_slow && btotal + 16 <= (uint64_t)kOutCap - 32) ? 1u : 0u;
            }
            __syncthreads();

            // ---- emit ----
            const uint64_t out_at = V->E_a + V->run_a;
            const uint64_t line0 = V->E_b + r0;
            const bool staged = V->staged != 0;
            const uint32_t so = V->stage_off;
            for (uint32_t q = tid; q < nb; q += kNT) {
                const uint32_t r = s_perm[q];
                const uint32_t a = s_start[r];
                const uint8_t fl = s_flag[r];
                const uint32_t loff = s_loff[r];
                if (A.index && line0 + r < A.index_cap) A.index[line0 + r] = out_at + loff;
                if (fl & kLfSlow) {
                    if (s_soff[r] == 0xFFFFFFFFu) continue;
                    uint8_t *ws = A.slow + ((uint64_t)s_soff[r] << 4);
                    const uint32_t glen = reinterpret_cast<const uint32_t *>(ws)[0];
                    const uint32_t m = reinterpret_cast<const uint32_t *>(ws)[1];
                    const SlowLayout sl = slow_layout(glen);
                    GlobalSink sink{A.out, out_at + loff, A.out_cap};
                    emit_line<false>(ws + sl.chs, ws + sl.text, m, plen_tab, sink);
                    if (fl & kLfNl) sink.put(kNl);
                } else if (staged) {
                    SmemSink sink{ost + so + loff};
                    emit_line<false>(st + a, gbase + a, s_plen[r], plen_tab, sink);
                    if (fl & kLfNl) sink.put(kNl);
                } else {
                    GlobalSink sink{A.out, out_at + loff, A.out_cap};
                    emit_line<false>(st + a, gbase + a, s_plen[r], plen_tab, sink);
                    if (fl & kLfNl) sink.put(kNl);
                }
            }
            __syncthreads();

            // ---- staged copy-out: 16-byte stores on the output's 16-byte grid ----
            if (staged) {
                const uint64_t total = V->batch_total;
                uint8_t *gdst = A.out + out_at - so;  // 16-byte aligned address
                const uint64_t cap_end = A.out_cap;   // bytes at output offset >= out_cap are dropped
                const uint32_t nchunks = (uint32_t)((so + total + 15) >> 4);
                for (uint32_t c = tid; c < nchunks; c += kNT) {
                    const uint32_t lo_b = c * 16u, hi_b = lo_b + 16u;
                    const uint64_t g_lo = out_at - so + lo_b;  // output offset of this chunk's first byte
                    if (lo_b >= so && hi_b <= so + total && g_lo + 16 <= cap_end) {
                        *reinterpret_cast<uint4 *>(gdst + lo_b) = *reinterpret_cast<const uint4 *>(ost + lo_b);
                    } else {
                        for (uint32_t k = lo_b; k < hi_b; ++k)
                            if (k >= so && k < so + total && out_at - so + k < cap_end) gdst[k] = ost[k];
                    }
                }
            }
            if (tid == 0) V->run_a += V->batch_total;
            __syncthreads();
        }

        if (tid == 0) {
            if (!single && (int64_t)t != A.stall_tile) {
                publish(&A.tiles[t], 2u, V->E_a + V->run_a, V->E_b + Lt);
            }
            if (t == A.ntiles - 1) {
                const uint64_t tot_a = V->E_a + V->run_a, tot_b = V->E_b + Lt;
                A.res->out_len = tot_a;
                A.res->n_lines = tot_b;
                if (A.index && tot_b < A.index_cap) A.index[tot_b] = tot_a;
            }
        }
        __syncthreads();
    }
}

template <int LMAX, bool COMPACT>
int max_blocks_per_sm(int smem)
{
    static int cached = -1;
    static int cached_smem = -1;
    if (cached < 0 || cached_smem != smem) {
        cudaFuncSetAttribute(compress_kernel<LMAX, COMPACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, compress_kernel<LMAX, COMPACT>, kNT, smem);
        cached = nb > 0 ? nb : 1;
        cached_smem = smem;
    }
    return cached;
}

template <int LMAX, bool COMPACT>
cudaError_t launch(const CompressArgs &a, int smem, int sms, cudaStream_t s)
{
    int per = max_blocks_per_sm<LMAX, COMPACT>(smem);
    uint64_t grid = std::min<uint64_t>(a.ntiles, (uint64_t)per * (uint64_t)sms);
    if (grid == 0) grid = 1;
    compress_kernel<LMAX, COMPACT><<<(unsigned)grid, kNT, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

// Launch the compress kernel for one stream (used by zs_compress and the batched entry points).
cudaError_t launch_compress(const zs_dict *d, const uint8_t *in, uint64_t n, unsigned flags, uint8_t *out,
                            uint64_t out_cap, uint64_t *index, uint64_t index_cap, DevResult *res,
                            TileState *tiles, uint8_t *slow, uint64_t slow_cap, cudaStream_t s)
{
    CompressArgs a{};
    a.in = in;
    a.n = n;
    a.out = out;
    a.out_cap = out_cap;
    a.index = index;
    a.index_cap = index_cap;
    a.flags = flags;
    a.in_aligned = (((uintptr_t)in) & 15u) == 0 ? 1u : 0u;
    a.ntiles = (n + kTB - 1) / kTB;
    a.enc = d->d_enc;
    a.L = d->layout;
    a.res = res;
    a.tiles = tiles;
    a.slow = slow;
    a.slow_cap = slow_cap;
    a.limit_ns = wait_limit_ns();
    a.stall_tile = injected_stall_tile();
    const int smem = kSmemFixed + (int)d->layout.img_bytes;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool compact = d->layout.compact != 0;
    if (d->lmax <= 8) return compact ? launch<8, true>(a, smem, sms, s) : launch<8, false>(a, smem, sms, s);
    return compact ? launch<16, true>(a, smem, sms, s) : launch<16, false>(a, smem, sms, s);
}

uint64_t compress_tiles(uint64_t n) { return (n + kTB - 1) / kTB; }

// The tiled geometry zs_compress uses for a dictionary: the span kernel's default geometry when the
// dictionary has a byte-indexed transducer, else the general transducer kernel's fastest geometry that
// leaves its image room in shared memory (20 warps, the same tile with 19, 12 warps, 8 warps); -1 when none
// fits, and the generic kernel (automaton + window scan per byte) runs.
int compress_general_variant(const zs_dict *d)
{
    const int ns = span_variants();
    for (int v : {0, 1, 3, 2})
        if (compress_warp_fits(ns + v, d)) return ns + v;
    return -1;
}

int compress_default_variant(const zs_dict *d)
{
    if (compress_warp_fits(0, d)) return 0;
    return compress_general_variant(d);
}

bool use_transducer(const zs_dict *d) { return compress_default_variant(d) >= 0; }

}  // namespace zs

extern "C" int zs_dictionary_uses_transducer(const zs_dict *d) { return d && zs::use_transducer(d) ? 1 : 0; }

namespace zs {

// Look-back records for a call: enough for the default geometry and for the general one it may fall back to.
uint64_t compress_scratch_tiles(const zs_dict *d, uint64_t n)
{
    uint64_t m = compress_tiles(n);
    for (int v : {compress_default_variant(d), compress_general_variant(d)})
        if (v >= 0) m = std::max<uint64_t>(m, tiles_for(n, compress_warp_variant(v)->tile_bytes));
    return m;
}

cudaError_t launch_compress_any(const zs_dict *d, const uint8_t *in, uint64_t n, unsigned flags, uint8_t *out,
                                uint64_t out_cap, uint64_t *index, uint64_t index_cap, DevResult *res,
                                TileState *tiles, uint8_t *slow, uint64_t slow_cap, cudaStream_t s, bool general)
{
    const int v = general ? compress_general_variant(d) : compress_default_variant(d);
    if (v < 0) return launch_compress(d, in, n, flags, out, out_cap, index, index_cap, res, tiles, slow, slow_cap, s);
    TiledLaunch L{};
    L.one = single_shard(in, n, out, out_cap, index, index_cap, tiles, res,
                         tiles_for(n, compress_warp_variant(v)->tile_bytes));
    L.n_shards = 1;
    L.total_tiles = L.one.ntiles;
    L.g = res;
    L.slow = slow;
    L.slow_cap = slow_cap;
    return launch_compress_warp(v, d, L, flags, s);
}

}  // namespace zs

namespace {

zs_status finish_status(const zs::DevResult &r, const char *what, uint64_t out_cap, uint64_t index_cap,
                        bool has_index)
{
    if (r.status & zs::kStTimeout) {
        zs::set_error(std::string(what) + ": a device-side wait expired");
        return ZS_ERR_TIMEOUT;
    }
    if (r.status & zs::kStTooBig) {
        zs::set_error(std::string(what) + ": a line longer than 1 GiB");
        return ZS_ERR_INVALID_ARG;
    }
    if (r.out_len > out_cap) {
        zs::set_error(std::string(what) + ": output buffer too small");
        return ZS_ERR_CAPACITY;
    }
    if (has_index && r.n_lines + 1 > index_cap) {
        zs::set_error(std::string(what) + ": line index buffer too small");
        return ZS_ERR_CAPACITY;
    }
    return ZS_OK;
}

}  // namespace

extern "C" zs_status zs_compress(const zs_dict *d, const uint8_t *d_in, size_t in_len, unsigned flags,
                                 uint8_t *d_out, size_t out_cap, uint64_t *d_line_index, size_t index_cap,
                                 zs_result *res, void *stream)
{
    zs::clear_error();
    if (!d || !res || (!d_in && in_len) || (!d_out && out_cap)) {
        zs::set_error("zs_compress: NULL argument");
        return ZS_ERR_INVALID_ARG;
    }
    if (!zs::compress_flags_ok(flags)) {
        zs::set_error("zs_compress: unknown flag bits, or ZS_PREPROCESS_OUTER without ZS_PREPROCESS");
        return ZS_ERR_INVALID_ARG;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return zs::cuda_fail(e, "cudaGetDevice");
    if (dev != d->device) {
        zs::set_error("zs_compress: dictionary was loaded on another device");
        return ZS_ERR_INVALID_ARG;
    }
    res->out_len = res->n_lines = res->err_offset = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (in_len == 0) {
        if (d_line_index) {
            if (index_cap < 1) {
                zs::set_error("zs_compress: line index buffer too small");
                return ZS_ERR_CAPACITY;
            }
            e = cudaMemsetAsync(d_line_index, 0, sizeof(uint64_t), s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return zs::cuda_fail(e, "zs_compress");
        }
        return ZS_OK;
    }
    const uint64_t ntiles = zs::compress_scratch_tiles(d, in_len);
    size_t slow_need = 16u << 20;
    bool general = false;  // the span kernel met a line outside its fast path: run the general kernel
    for (int attempt = 0; attempt < 4; ++attempt) {
        zs::Scratch *sc = nullptr;
        zs_status st = const_cast<zs_dict *>(d)->pool.get(stream, ntiles, slow_need, &sc);
        if (st != ZS_OK) return st;
        zs::DevResult *dr = reinterpret_cast<zs::DevResult *>(sc->dev);
        zs::TileState *tiles = reinterpret_cast<zs::TileState *>(dr + 1);
        e = cudaMemsetAsync(sc->dev, 0, sizeof(zs::DevResult) + ntiles * sizeof(zs::TileState), s);
        if (e != cudaSuccess) return zs::cuda_fail(e, "zs_compress: memset");
        zs::mark_kernel_start(sc, s);
        e = zs::launch_compress_any(d, d_in, in_len, flags, d_out, out_cap, d_line_index,
                                    d_line_index ? index_cap : 0, dr, tiles, sc->slow, sc->slow_cap, s, general);
        if (e != cudaSuccess) return zs::cuda_fail(e, "zs_compress: launch");
        zs::mark_kernel_end(sc, s);
        e = cudaMemcpyAsync(sc->host, dr, sizeof(zs::DevResult), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return zs::cuda_fail(e, "zs_compress");
        const zs::DevResult r = *sc->host;
        zs::note_kernel_time(sc);
        if ((r.status & zs::kStFallback) && !(r.status & zs::kStTimeout) && !general) {
            general = true;
            continue;
        }
        if (r.status & zs::kStSlowOverflow) {
            slow_need = (size_t)r.slow_used + ((size_t)r.slow_used >> 2) + (1u << 20);
            continue;
        }
        res->out_len = r.out_len;
        res->n_lines = r.n_lines;
        return finish_status(r, "zs_compress", out_cap, index_cap, d_line_index != nullptr);
    }
    zs::set_error("zs_compress: long-line scratch could not be sized");
    return ZS_ERR_OOM;
}
