// Internal declarations shared by the ZSMILES CUDA translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <utility>

#include "../../include/zsmiles.h"

namespace zs {

constexpr int kMaxPat = 16;       // longest pattern a dictionary may hold
constexpr uint8_t kEsc = ' ';     // escape byte (Sec. IV-D1/IV-D2)
constexpr uint8_t kNl = '\n';     // line separator

// ------------------------------------------------------------------------------------------------
// Encoder tables. The host builds one contiguous image that each compress CTA copies into shared
// memory with a single bulk (TMA) copy. Offsets are 16-byte aligned.
//
//   [0, 256)                  cls[256]    byte -> character class (0: the byte occurs in no pattern)
//   [256, 512)                plen[256]   symbol -> pattern length (0: not a symbol)
//   [512, 640)                masks[32]   compact layout: mask id -> set of match lengths
//   [off_trans, +trans_bytes) trans       reverse Aho-Corasick automaton, next state + match set
//   [off_sym, +S*16)          sym[S][16]  symbol of the pattern of length l+1 that starts at the
//                                          byte just read
//
// The automaton reads a line from its last byte to its first; after reading byte i its state is the
// longest suffix of (s[n-1] ... s[i]) that is a prefix of some reversed pattern, so the match set of
// the state is exactly {l : s[i..i+l) is a pattern of D} - the out-edges of node i in the paper's
// graph G (Sec. IV-D1), in the order the backward shortest-path scan needs them.
//
// Transition entry: compact (u16) = next state (bits 0-10) | mask id (bits 11-15), used when the
// automaton has <= 2048 states and <= 32 distinct match sets; wide (u32) = next state (bits 0-15) |
// match set (bits 16-31).
// ------------------------------------------------------------------------------------------------
struct EncLayout {
    uint32_t n_states;
    uint32_t n_classes;
    uint32_t compact;
    uint32_t lmax;
    uint32_t off_trans;
    uint32_t off_sym;
    uint32_t img_bytes;
    uint32_t _pad;
};

constexpr uint32_t kOffCls = 0, kOffPlen = 256, kOffMasks = 512, kOffTrans = 640;

// Fixed byte classes (the automaton's input alphabet): pre-processing and segmentation read these
// directly from class-coded text. Interesting bytes for pre-processing have classes below kClsNl.
constexpr uint8_t kClsPct = 10, kClsLbr = 11, kClsRbr = 12, kClsSpace = 13, kClsTab = 14, kClsNl = 15,
                  kClsOther = 16, kClsFirstFree = 17;

// Parse-transducer image (shared memory of the compress kernel):
//   [0, 8192)          class of each byte, replicated for the 32 lanes: byte c of lane l is at
//                      ((c >> 2) * 32 + l) * 4 + (c & 3), so a warp-wide lookup never conflicts on a bank
//   [8192, 8448)       plen[256]: symbol -> pattern length
//   [8448, ...)        table[states][classes] (u32): next state * classes | (delta + 16) << 16 | symbol << 24
struct MachineLayout {
    uint32_t n_states;
    uint32_t n_classes;
    uint32_t start;
    uint32_t off_table;
    uint32_t img_bytes;
    // 1 when every symbol byte is above ' ': the table then codes an escape chosen at a digit d (class d)
    // as the choice 1 + d, so the emitter writes the digit itself (a new ring label that the input bytes no
    // longer show) rather than the input byte
    uint32_t esc_digits;
    uint32_t _pad[2];
};
constexpr uint32_t kMOffClsRep = 0, kMOffPlen = 8192, kMOffTable = 8448;

// Byte-indexed parse transducer (the span kernel): the minimal transducer above with its columns indexed by
// the raw byte (bytes 0-127; bytes >= 0x80 read the column of a byte below 0x80 in no pattern), so a lookup
// needs no class table.
//   [0, 256 * n_states)    table[state][128] (u16): next state | choice << 8, at byte offset state * 256 +
//                          (2 * byte XOR (state mod 32) * 4): the swizzle spreads one byte's entries over the 32
//                          banks, so lanes reading the same byte in different states do not conflict.
//                          Choices: a symbol (every symbol is above ' '); ' ' = escape of the input
//                          byte; 0x10 + d = escape of the digit d; '\n' = end of line (next state: the start)
//   [meta_off, +1024)      meta[256] (u32) per choice: input bytes consumed | output bytes << 13
struct ByteLayout {
    uint32_t n_states;
    uint32_t q0;         // start state
    uint32_t meta_off;
    uint32_t img_bytes;
    uint32_t rep_col;    // 2 * the stand-in byte for bytes >= 0x80
    uint32_t _pad[3];
};
constexpr uint32_t kMaxMachineBytes = 64u * 1024u;  // transition table budget in shared memory

// Decoder tables (global, staged per CTA): plen[256] then pat[256][16].
constexpr uint32_t kDecBytes = 256 + 256 * kMaxPat;

// ------------------------------------------------------------------------------------------------
// Per-call device scratch
// ------------------------------------------------------------------------------------------------
// Look-back record of one tile. Every word carries its own validity (bit 63 set once written; the record
// starts zeroed), so a reader learns what is published and its value from the same load, and reads a whole
// record in one round trip.
struct alignas(32) TileState {
    unsigned long long agg_a, agg_b;  // this tile's totals (a: bytes, b: lines)
    unsigned long long inc_a, inc_b;  // totals of tiles [0, this]
};
constexpr unsigned long long kValidBit = 1ull << 63;

enum : uint32_t {
    kStTimeout = 1u,       // a bounded wait expired
    kStMalformed = 2u,     // bad compressed byte / request
    kStSlowOverflow = 4u,  // the long/irregular-line scratch was too small (host retries larger)
    kStTooBig = 8u,        // a single line needs more than 4 GiB of work space
    kStFallback = 16u,     // the span kernel met a line outside its fast path: the call is run again by the
                           // general kernel
};

struct alignas(16) DevResult {
    unsigned long long tile_counter;  // dynamic tile ids, claimed in launch order
    uint32_t status;                  // kSt* bits
    uint32_t _pad;
    unsigned long long out_len;       // total output bytes (written by the last tile)
    unsigned long long n_lines;       // total lines / requests
    unsigned long long err_key;       // max of (~offset): the smallest bad offset, 0 = none
    unsigned long long slow_used;     // bytes of long-line scratch claimed
    unsigned long long _pad2[2];
};

// Host-side scratch cached per (device, stream).
struct Scratch {
    int device = -1;
    void *dev = nullptr;            // DevResult + TileState[cap_tiles]
    size_t cap_tiles = 0;
    uint8_t *slow = nullptr;        // long/irregular-line work space
    size_t slow_cap = 0;
    DevResult *host = nullptr;      // pinned mirror of DevResult
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // bracket the call's main kernel (zs_last_kernel_ms)
};

class ScratchPool {
   public:
    ~ScratchPool();
    // Returns the scratch of `stream` for the calling host thread, grown to hold `tiles` tile states and
    // `slow` long-line bytes. Keyed by thread as well as stream: calls from several threads on one stream
    // are ordered on the device by the stream, but each needs its own host-side result record.
    zs_status get(void *stream, size_t tiles, size_t slow, Scratch **out);
    void release_all();

   private:
    std::mutex mu_;
    std::map<std::pair<void *, std::thread::id>, Scratch> map_;
};

ScratchPool &global_pool();

// Kernel timing: record ev0/ev1 of `sc` around a launch on `s`; after the stream is synchronised,
// note_kernel_time() stores the elapsed milliseconds for zs_last_kernel_ms().
void mark_kernel_start(Scratch *sc, cudaStream_t s);
void mark_kernel_end(Scratch *sc, cudaStream_t s);
void note_kernel_time(Scratch *sc);

// Thread-local error message.
void set_error(const std::string &msg);
void clear_error();
zs_status cuda_fail(cudaError_t e, const char *what);

// Bounded-wait default (device waits give up after this many nanoseconds).
uint64_t wait_limit_ns();
// Debug/fault-injection knobs, set from the environment of the calling process (tests only):
//   ZS_WAIT_LIMIT_MS    overrides the wait limit
//   ZS_INJECT_STALL     tile index whose look-back record is never published
//   ZS_SPAN_CUT_MIN     shortest line the span kernel may cut between lanes (0: never); -1 when unset
int64_t injected_stall_tile();
int64_t span_cut_min_override();

}  // namespace zs

// The dictionary handle.
struct zs_dict {
    int device = -1;
    int lmax = 0;      // the file's L_max
    int max_plen = 0;  // the longest pattern actually present (alphabet singles count as 1)
    zs::EncLayout layout{};
    zs::MachineLayout mlayout{};
    bool has_machine = false;
    zs::ByteLayout blayout{};
    bool has_bytes = false;     // the byte-indexed transducer exists (span kernel)
    uint8_t *d_bimg = nullptr;  // its image (blayout.img_bytes)
    uint8_t *d_enc = nullptr;  // encoder image (layout.img_bytes)
    uint8_t *d_mimg = nullptr; // parse-transducer image (mlayout.img_bytes), if it fits
    uint8_t *d_dec = nullptr;  // decoder tables (kDecBytes)
    uint8_t plen[256];
    uint8_t pat[256][zs::kMaxPat];
    uint64_t digest = 0;        // FNV-1a of the dictionary file (the plan tuning cache's key)
    zs::ScratchPool pool;
    struct zs_pipes *pipes = nullptr;  // host-to-host pipelines (pipeline.cu), made on first use
};

namespace zs {
// zs_compress flags: ZS_PREPROCESS, optionally with ZS_PREPROCESS_OUTER; nothing else.
inline bool compress_flags_ok(unsigned flags)
{
    return (flags & ~(unsigned)(ZS_PREPROCESS | ZS_PREPROCESS_OUTER)) == 0 &&
           (!(flags & ZS_PREPROCESS_OUTER) || (flags & ZS_PREPROCESS));
}
void free_pipes(zs_dict *d);
uint64_t compress_scratch_tiles(const zs_dict *d, uint64_t n);
cudaError_t launch_compress_any(const zs_dict *d, const uint8_t *in, uint64_t n, unsigned flags, uint8_t *out,
                                uint64_t out_cap, uint64_t *index, uint64_t index_cap, DevResult *res,
                                TileState *tiles, uint8_t *slow, uint64_t slow_cap, cudaStream_t s,
                                bool general = false);
}  // namespace zs

// ------------------------------------------------------------------------------------------------
// Device helpers
// ------------------------------------------------------------------------------------------------
#ifdef __CUDACC__
namespace zs {

__device__ __forceinline__ uint64_t gtime()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// A pair of 64-bit words, written and read at gpu scope (each word is single-copy atomic on its own).
__device__ __forceinline__ void st_pair(unsigned long long *p, unsigned long long x, unsigned long long y)
{
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(x), "l"(y) : "memory");
}

__device__ __forceinline__ void ld_pair(const unsigned long long *p, unsigned long long *x, unsigned long long *y)
{
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(*x), "=l"(*y) : "l"(p) : "memory");
}

// One tile's record: 2 = inclusive prefix published (values in *a, *b), 1 = aggregate only, 0 = nothing yet.
__device__ __forceinline__ uint32_t read_tile(const TileState *ts, uint64_t *a, uint64_t *b)
{
    unsigned long long ga, gb, ia, ib;
    ld_pair(&ts->agg_a, &ga, &gb);
    ld_pair(&ts->inc_a, &ia, &ib);
    if (ia & ib & kValidBit) {
        *a = ia & ~kValidBit;
        *b = ib & ~kValidBit;
        return 2u;
    }
    if (ga & gb & kValidBit) {
        *a = ga & ~kValidBit;
        *b = gb & ~kValidBit;
        return 1u;
    }
    *a = *b = 0;
    return 0u;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Waits for the phase with the thread suspended in hardware for up to ~20 us (the suspend-time hint),
// so a waiting warp does not take issue slots from the warps that are working.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase), "r"(20000u)
        : "memory");
    return ok != 0;
}

// Make generic-proxy writes to shared memory visible to a following bulk copy into the same bytes.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One-dimensional bulk copy global -> shared (cp.async.bulk): src, dst 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Waits for phase `phase` of `bar`; gives up after `limit_ns` (sets kStTimeout). Returns false on
// timeout. A timed-out copy may still be in flight: the caller stops issuing new ones and the kernel
// only finishes after the copy lands (see drain_bulk), so no write hits shared memory after exit.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase, uint64_t limit_ns,
                                                  uint32_t *status)
{
    if (mbar_try_wait(bar, phase)) return true;
    uint64_t t0 = gtime();
    for (;;) {
        if (mbar_try_wait(bar, phase)) return true;
        if (gtime() - t0 > limit_ns) {
            atomicOr(status, kStTimeout);
            return false;
        }
    }
}

// Warp-level inclusive sum.
__device__ __forceinline__ uint32_t warp_incl_u32(uint32_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Block-wide exclusive sum of one value per thread; `tmp` holds NT/32 + 1 words. Returns the
// exclusive prefix; *total gets the block total. Contains __syncthreads().
template <int NT>
__device__ __forceinline__ uint32_t block_excl_u32(uint32_t v, uint32_t *tmp, uint32_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = warp_incl_u32(v);
    if (lane == 31) tmp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < NT / 32 ? tmp[lane] : 0u;
        uint32_t wi = warp_incl_u32(w);
        if (lane < NT / 32) tmp[lane] = wi - w;
        if (lane == NT / 32 - 1) tmp[NT / 32] = wi;
    }
    __syncthreads();
    uint32_t r = tmp[warp] + inc - v;
    *total = tmp[NT / 32];
    __syncthreads();
    return r;
}

// Block-wide exclusive sums of two 64-bit values per thread (NT threads, NT/32 <= 32). `tmp` holds
// 2 * (NT/32 + 1) words. Returns the exclusive prefixes in *xa, *xb and the block totals in *ta, *tb.
// Contains __syncthreads().
template <int NT>
__device__ __forceinline__ void block_excl2_u64(uint64_t a, uint64_t b, uint64_t *tmp, uint64_t *xa, uint64_t *xb,
                                                uint64_t *ta, uint64_t *tb)
{
    constexpr int W = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t ua = __shfl_up_sync(0xffffffffu, ia, o);
        uint64_t ub = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) {
            ia += ua;
            ib += ub;
        }
    }
    if (lane == 31) {
        tmp[warp] = ia;
        tmp[W + 1 + warp] = ib;
    }
    __syncthreads();
    if (warp == 0) {
        uint64_t wa = lane < W ? tmp[lane] : 0ull, wb = lane < W ? tmp[W + 1 + lane] : 0ull;
        uint64_t sa = wa, sb = wb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t ua = __shfl_up_sync(0xffffffffu, sa, o);
            uint64_t ub = __shfl_up_sync(0xffffffffu, sb, o);
            if (lane >= o) {
                sa += ua;
                sb += ub;
            }
        }
        if (lane < W) {
            tmp[lane] = sa - wa;
            tmp[W + 1 + lane] = sb - wb;
        }
        if (lane == W - 1) {
            tmp[W] = sa;
            tmp[2 * W + 1] = sb;
        }
    }
    __syncthreads();
    *xa = tmp[warp] + ia - a;
    *xb = tmp[W + 1 + warp] + ib - b;
    *ta = tmp[W];
    *tb = tmp[2 * W + 1];
    __syncthreads();
}

// Decoupled look-back (single thread): publish-free part. Sums the aggregates of tiles t-1, t-2, ...
// until one has published its inclusive prefix. Waits are bounded; on expiry kStTimeout is set and
// the sums so far are returned.
__device__ __forceinline__ void lookback(TileState *tiles, uint64_t t, uint64_t *ea, uint64_t *eb,
                                         uint64_t limit_ns, uint32_t *status)
{
    uint64_t a = 0, b = 0;
    int64_t p = (int64_t)t - 1;
    uint64_t t0 = 0;
    bool timed = false;
    while (p >= 0) {
        uint64_t va, vb;
        const uint32_t f = read_tile(&tiles[p], &va, &vb);
        if (f == 0) {
            if (*((volatile uint32_t *)status) & kStTimeout) break;
            if (!timed) {
                t0 = gtime();
                timed = true;
            } else if (gtime() - t0 > limit_ns) {
                atomicOr(status, kStTimeout);
                break;
            }
            __nanosleep(64);
            continue;
        }
        a += va;
        b += vb;
        if (f == 2) break;
        --p;
        timed = false;
    }
    *ea = a;
    *eb = b;
}

// Decoupled look-back by a whole warp: each round, lane j reads the record of tile t-1-j, so one round trip
// to L2 covers 32 predecessors. Sums aggregates from the nearest predecessor back to (and including) the
// nearest one that has published its inclusive prefix. Called by all 32 lanes; every lane returns the
// same sums. Waits are bounded (kStTimeout on expiry).
__device__ __forceinline__ void lookback_warp(TileState *tiles, uint64_t t, uint64_t *ea, uint64_t *eb,
                                              uint64_t limit_ns, uint32_t *status)
{
    const uint32_t lane = threadIdx.x & 31;
    uint64_t a = 0, b = 0;
    int64_t top = (int64_t)t - 1;
    uint64_t t0 = 0;
    bool timed = false;
    while (top >= 0) {
        const int64_t p = top - (int64_t)lane;
        uint64_t va = 0, vb = 0;
        const uint32_t f = p >= 0 ? read_tile(&tiles[p], &va, &vb) : 2u;  // before tile 0: a zero prefix
        const uint32_t incl = __ballot_sync(0xffffffffu, f == 2u);
        const int stop = incl ? __ffs(incl) - 1 : 32;  // nearest lane holding an inclusive prefix
        if (__any_sync(0xffffffffu, (int)lane < stop && f == 0u)) {  // a nearer tile has published nothing
            if (*((volatile uint32_t *)status) & kStTimeout) break;
            if (!timed) {
                t0 = gtime();
                timed = true;
            } else if (gtime() - t0 > limit_ns) {
                if (lane == 0) atomicOr(status, kStTimeout);
                break;
            }
            __nanosleep(128);
            continue;
        }
        timed = false;
        if ((int)lane > stop) va = vb = 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            va += __shfl_xor_sync(0xffffffffu, va, o);
            vb += __shfl_xor_sync(0xffffffffu, vb, o);
        }
        a += va;
        b += vb;
        if (stop < 32) break;
        top -= 32;
    }
    *ea = a;
    *eb = b;
}

__device__ __forceinline__ void publish(TileState *ts, uint32_t flag, uint64_t a, uint64_t b)
{
    if (flag == 1) st_pair(&ts->agg_a, a | kValidBit, b | kValidBit);
    else st_pair(&ts->inc_a, a | kValidBit, b | kValidBit);
}

// Copies a warp's staged output to global memory: staged bytes [so, so + len) go to dst[0, len), where
// dst - so is 16-byte aligned and bytes at or past cap (relative to dst) are not written. Whole 16-byte
// chunks go as one store each; the partial chunks at either end byte by byte. Called by all 32 lanes.
__device__ __forceinline__ void warp_copy_out(const uint8_t *stage, uint32_t so, uint64_t len, uint8_t *dst,
                                              uint64_t cap)
{
    const uint32_t lane = threadIdx.x & 31;
    uint8_t *g = dst - so;
    const uint32_t end = so + (uint32_t)min(len, cap);  // staged bytes [so, end) are written
    const uint32_t c0 = (so + 15u) >> 4, c1 = end >> 4;  // whole chunks [c0, c1)
    for (uint32_t c = c0 + lane; c < c1; c += 32)
        reinterpret_cast<uint4 *>(g)[c] = reinterpret_cast<const uint4 *>(stage)[c];
    const uint32_t h1 = min(c0 * 16u, end);
    for (uint32_t k = so + lane; k < h1; k += 32) g[k] = stage[k];
    for (uint32_t k = max(c1 * 16u, h1) + lane; k < end; k += 32) g[k] = stage[k];
}

// Copies a warp's stage [0, len) to dst[0, len) for any alignment of dst (bytes at or past cap are not
// written): each whole 16-byte chunk of the destination is one store, its bytes taken from two 16-byte
// chunks of the stage by funnel shifts; the partial chunks at either end go byte by byte. The stage is
// 16-byte aligned and readable up to 16 bytes past len. Called by all 32 lanes.
template <int Q>
__device__ __forceinline__ uint4 shift_chunk(const uint4 A, const uint4 B, uint32_t sh)
{
    const uint32_t v[8] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w};
    return make_uint4(__funnelshift_r(v[Q], v[Q + 1], sh), __funnelshift_r(v[Q + 1], v[Q + 2], sh),
                      __funnelshift_r(v[Q + 2], v[Q + 3], sh), __funnelshift_r(v[Q + 3], v[Q + 4], sh));
}

template <int Q>
__device__ __forceinline__ void realign_loop(const uint4 *s16, uint4 *g, uint32_t j, uint32_t j1, uint32_t sh)
{
    for (; j < j1; j += 32) g[j] = shift_chunk<Q>(s16[j - 1], s16[j], sh);
}

// HOIST: the word offset's four cases are separate loops (the decoder), else one loop that switches per chunk
// (the span kernel, whose register allocation is tuned around it).
template <bool HOIST = false>
__device__ __forceinline__ void warp_copy_realign(const uint8_t *stg, uint64_t len64, uint8_t *dst, uint64_t cap)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t len = (uint32_t)min(len64, cap);
    const uint32_t so = (uint32_t)((uintptr_t)dst & 15u);
    uint4 *g = reinterpret_cast<uint4 *>(dst - so);
    const uint4 *s16 = reinterpret_cast<const uint4 *>(stg);
    const uint32_t j0 = so ? 1u : 0u, j1 = (len + so) >> 4;  // whole destination chunks [j0, j1)
    if (so == 0) {
        for (uint32_t j = lane; j < j1; j += 32) g[j] = s16[j];
    } else {
        // destination chunk j = stage bytes [16 j - so, 16 j - so + 16): chunk j - 1 from byte r = 16 - so on
        const uint32_t r = 16u - so, q = r >> 2, sh = 8u * (r & 3u);
        if constexpr (HOIST) {  // the word offset q is the same for every chunk: choose the loop once
            switch (q) {
                case 0: realign_loop<0>(s16, g, j0 + lane, j1, sh); break;
                case 1: realign_loop<1>(s16, g, j0 + lane, j1, sh); break;
                case 2: realign_loop<2>(s16, g, j0 + lane, j1, sh); break;
                default: realign_loop<3>(s16, g, j0 + lane, j1, sh); break;
            }
        } else {
            for (uint32_t j = j0 + lane; j < j1; j += 32) {
                const uint4 A = s16[j - 1], B = s16[j];
                uint4 o;
                switch (q) {
                    case 0: o = shift_chunk<0>(A, B, sh); break;
                    case 1: o = shift_chunk<1>(A, B, sh); break;
                    case 2: o = shift_chunk<2>(A, B, sh); break;
                    default: o = shift_chunk<3>(A, B, sh); break;
                }
                g[j] = o;
            }
        }
    }
    const uint32_t h1 = min(len, j0 * 16u - so);  // head bytes [0, h1)
    for (uint32_t k = lane; k < h1; k += 32) dst[k] = stg[k];
    const uint32_t t0 = j1 > j0 ? max(h1, j1 * 16u - so) : h1;  // tail bytes [t0, len)
    for (uint32_t k = t0 + lane; k < len; k += 32) dst[k] = stg[k];
}

__device__ __forceinline__ void note_error_offset(DevResult *r, uint64_t off)
{
    atomicMax(&r->err_key, ~(unsigned long long)off);
}

// One shard of a launch: a whole input stream for the single-stream calls, one entry of the shard table
// for the batched calls. Tiles are numbered per shard (look-back never crosses a shard); tile0 is the
// shard's first tile in the launch-wide numbering that warps claim from.
struct alignas(16) ShardView {
    const uint8_t *in;
    uint64_t n;
    uint8_t *out;
    uint64_t out_cap;
    uint64_t *index;      // compress: line index (nullable); unused by decompression
    uint64_t index_cap;
    uint64_t tile0;
    uint64_t ntiles;
    TileState *tiles;     // look-back records of this shard's tiles
    DevResult *res;       // out_len, n_lines, err_key of this shard
    uint32_t in_aligned;  // in is 16-byte aligned (bulk copies allowed)
    uint32_t _pad[3];
};

// One launch of a tiled kernel over one shard (`one`, n_shards == 1) or a device shard table.
struct TiledLaunch {
    ShardView one;
    const ShardView *shards = nullptr;
    uint32_t n_shards = 1;
    uint64_t total_tiles = 0;
    DevResult *g = nullptr;  // launch-wide counters and status (the shard's own result when n_shards == 1)
    uint8_t *slow = nullptr;  // compression's long-line scratch
    uint64_t slow_cap = 0;
    int32_t cut_min = 0;      // span kernel: shortest line cut between lanes (0: the geometry's default; < 0: never)
};

// A compiled geometry of a tiled kernel.
struct KernelVariant {
    const char *name;
    uint32_t warps;       // warps per CTA (one CTA per SM)
    uint32_t tile_bytes;  // input bytes per warp tile
};

constexpr int kDefaultVariant = 0;

inline uint64_t tiles_for(uint64_t n, uint32_t tile_bytes) { return (n + tile_bytes - 1) / tile_bytes; }

inline ShardView single_shard(const uint8_t *in, uint64_t n, uint8_t *out, uint64_t out_cap, uint64_t *index,
                              uint64_t index_cap, TileState *tiles, DevResult *res, uint64_t ntiles)
{
    ShardView v{};
    v.in = in;
    v.n = n;
    v.out = out;
    v.out_cap = out_cap;
    v.index = index;
    v.index_cap = index_cap;
    v.tile0 = 0;
    v.ntiles = ntiles;
    v.tiles = tiles;
    v.res = res;
    v.in_aligned = (((uintptr_t)in) & 15u) == 0 ? 1u : 0u;
    return v;
}

// Span kernel (compress_span.cu): compiled geometries, fit, launch.
int span_variants();
const KernelVariant *span_variant(int v);
bool span_fits(int v, const zs_dict *d);
cudaError_t launch_span(int v, const zs_dict *d, const TiledLaunch &L, unsigned flags, cudaStream_t s);
uint32_t span_cut_default(int v);  // the geometry's default cut threshold (0: cuts off), or 0 for no such geometry

// Compiled variants of the tiled compression (transducer) and decompression kernels.
int compress_warp_variants();
const KernelVariant *compress_warp_variant(int v);
bool compress_warp_fits(int v, const zs_dict *d);
int compress_default_variant(const zs_dict *d);  // the geometry zs_compress uses, or -1: the generic kernel
int compress_general_variant(const zs_dict *d);  // the same without the span kernel (its fallback)
bool compress_variant_is_span(int v);
cudaError_t launch_compress_warp(int v, const zs_dict *d, const TiledLaunch &L, unsigned flags, cudaStream_t s);
int decompress_variants();
const KernelVariant *decompress_variant(int v);
bool decompress_fits(int v, const zs_dict *d);
int decompress_default_variant(const zs_dict *d);  // the expansion kernel unless a pattern exceeds 7 bytes
// Expansion kernel (decode_expand.cu): compiled geometries, fit, launch.
int expand_variants();
const KernelVariant *expand_variant(int v);
bool expand_fits(int v, const zs_dict *d);
cudaError_t launch_expand(int v, const zs_dict *d, const TiledLaunch &L, cudaStream_t s);
cudaError_t launch_decompress(int v, const zs_dict *d, const TiledLaunch &L, cudaStream_t s);
// Random access (decode.cu): tile records a launch over k requested ids needs, and the launch itself
// (out_off[k + 1] receives each line's output offset and the total).
uint64_t lines_tiles(uint64_t k);
cudaError_t launch_lines(const zs_dict *d, const uint8_t *comp, uint64_t comp_len, const uint64_t *index,
                         uint64_t n_lines, const uint64_t *ids, uint64_t k, uint8_t *out, uint64_t out_cap,
                         uint64_t *out_off, DevResult *res, TileState *tiles, cudaStream_t s);
// The default variant over one stream: tiles and launch.
uint64_t decompress_tiles(uint64_t n);
uint64_t decompress_tile_bytes();
cudaError_t launch_decompress_single(const zs_dict *d, const uint8_t *in, uint64_t n, uint8_t *out, uint64_t out_cap,
                                     DevResult *res, TileState *tiles, cudaStream_t s);

// The shard owning launch-wide tile g: the last shard whose tile0 <= g (called by a whole warp; a
// 32-way search per round, so two rounds cover 1024 shards). tab[0].tile0 must be 0.
__device__ __forceinline__ uint32_t find_shard(const ShardView *tab, uint32_t n, uint64_t g)
{
    const uint32_t lane = threadIdx.x & 31;
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint32_t step = (hi - lo + 31) / 32;
        const uint32_t idx = lo + lane * step;
        const bool ok = idx < hi && tab[idx].tile0 <= g;
        const uint32_t b = __ballot_sync(0xffffffffu, ok);  // lane 0 (idx == lo) always holds
        lo += (uint32_t)(31 - __clz(b)) * step;
        hi = min(hi, lo + step);
    }
    return lo;
}

// Copy shard `s` (or the single shard `one`) into a warp's shared-memory view; all lanes call.
__device__ __forceinline__ void load_shard(ShardView *dst, const ShardView &one, const ShardView *tab, uint32_t n,
                                           uint32_t s)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t *src = reinterpret_cast<const uint64_t *>(n == 1 ? &one : tab + s);
    constexpr uint32_t kWords = sizeof(ShardView) / 8;
    __syncwarp();
    if (lane < kWords) reinterpret_cast<uint64_t *>(dst)[lane] = src[lane];
    __syncwarp();
}

}  // namespace zs
#endif
