// Device helpers shared by the two compress kernels (internal).
#pragma once

#include "zs_common.cuh"

namespace zs {
namespace cx {

__device__ __forceinline__ uint32_t zero_byte_bits(uint32_t t)
{
    uint32_t z = ~(((t & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | t | 0x7F7F7F7Fu);
    return ((z >> 7) & 1u) | ((z >> 14) & 2u) | ((z >> 21) & 4u) | ((z >> 28) & 8u);
}

// bit i set iff byte i of the 16-byte chunk equals the byte repeated in k (k = b * 0x01010101)
__device__ __forceinline__ uint32_t eq_bits16(uint4 v, uint32_t k)
{
    return zero_byte_bits(v.x ^ k) | (zero_byte_bits(v.y ^ k) << 4) | (zero_byte_bits(v.z ^ k) << 8) |
           (zero_byte_bits(v.w ^ k) << 12);
}

// bit i set iff byte i of the 16-byte chunk is '\n'
__device__ __forceinline__ uint32_t nl_bits16(uint4 v) { return eq_bits16(v, 0x0A0A0A0Au); }

// ------------------------------------------------------------------------------------------------
// Pre-processing, slow path: any line, work space in global memory. Two passes: label every ring
// token (labels up to 99), then write the relabelled line (1- or 3-byte labels).
//   - closing order (the default): a ring that closes takes the smallest label whose latest ring closed
//     before this one opened; lcv[x] = (latest close of label x) + 1;
//   - opening order (outer): a ring that opens takes the smallest label no open ring holds, and its
//     closing token repeats it; lcv[x] = 1 while label x is held.
// tok: one byte per ring token; lcv/open_tok: 100 ints each. Returns the new length.
// ------------------------------------------------------------------------------------------------
static __device__ uint32_t preprocess_slow(const uint8_t *s, uint32_t n, uint8_t *out, uint8_t *tok, int32_t *lcv,
                                           int32_t *open_tok, bool outer)
{
    for (int k = 0; k < 100; ++k) {
        lcv[k] = 0;
        open_tok[k] = -1;
    }
    uint32_t f = 0;
    while (f < n && s[f] != ' ' && s[f] != '\t') ++f;
    bool ok = true, in_br = false;
    int32_t ord = 0;
    for (uint32_t r = 0; r < f && ok;) {
        uint8_t c = s[r];
        if (in_br) {
            if (c == ']') in_br = false;
            ++r;
            continue;
        }
        if (c == '[') {
            in_br = true;
            ++r;
            continue;
        }
        int lab = -1, tl = 1;
        if (c == '%') {
            if (r + 2 < f && s[r + 1] >= '0' && s[r + 1] <= '9' && s[r + 2] >= '0' && s[r + 2] <= '9') {
                lab = (s[r + 1] - '0') * 10 + (s[r + 2] - '0');
                tl = 3;
            } else {
                ok = false;
                break;
            }
        } else if (c >= '0' && c <= '9') {
            lab = c - '0';
        }
        if (lab >= 0 && outer) {
            if (open_tok[lab] < 0) {
                int nl = 0;
                while (nl < 100 && lcv[nl] != 0) ++nl;
                if (nl > 99) {
                    ok = false;
                    break;
                }
                lcv[nl] = 1;
                tok[ord] = (uint8_t)nl;
                open_tok[lab] = ord;
            } else {
                const uint8_t nl = tok[open_tok[lab]];
                tok[ord] = nl;
                lcv[nl] = 0;
                open_tok[lab] = -1;
            }
            ++ord;
        } else if (lab >= 0) {
            if (open_tok[lab] < 0) {
                open_tok[lab] = ord;
            } else {
                int32_t o = open_tok[lab];
                int nl = 0;
                while (nl < 100 && lcv[nl] > o + 1) ++nl;
                if (nl > 99) {
                    ok = false;
                    break;
                }
                tok[o] = (uint8_t)nl;
                tok[ord] = (uint8_t)nl;
                lcv[nl] = ord + 1;
                open_tok[lab] = -1;
            }
            ++ord;
        }
        r += tl;
    }
    if (in_br) ok = false;
    for (int k = 0; k < 100 && ok; ++k)
        if (open_tok[k] >= 0) ok = false;
    if (!ok) {
        for (uint32_t i = 0; i < n; ++i) out[i] = s[i];
        return n;
    }
    uint32_t w = 0;
    ord = 0;
    in_br = false;
    for (uint32_t r = 0; r < f;) {
        uint8_t c = s[r];
        if (in_br) {
            if (c == ']') in_br = false;
            out[w++] = c;
            ++r;
            continue;
        }
        if (c == '[') {
            in_br = true;
            out[w++] = c;
            ++r;
            continue;
        }
        if (c == '%' || (c >= '0' && c <= '9')) {
            int nl = tok[ord++];
            if (nl < 10) {
                out[w++] = (uint8_t)('0' + nl);
            } else {
                out[w++] = '%';
                out[w++] = (uint8_t)('0' + nl / 10);
                out[w++] = (uint8_t)('0' + nl % 10);
            }
            r += (c == '%') ? 3 : 1;
            continue;
        }
        out[w++] = c;
        ++r;
    }
    for (uint32_t r = f; r < n; ++r) out[w++] = s[r];
    return w;
}

// Emission of one line: walk the choices front to back. A ' ' choice escapes the input byte at that
// position. With ESC_DIGITS (the dictionary has no symbol byte below 0x20, so every choice up to ' ' is an
// escape), a choice 1 + d (d = 0..9) is an escaped digit d, written as such.
template <bool ESC_DIGITS, class CP, class TP, class Sink>
__device__ __forceinline__ void emit_line(CP choice, TP raw, uint32_t n, const uint8_t *plen, Sink &out)
{
    for (uint32_t i = 0; i < n;) {
        uint8_t s = choice[i];
        if (ESC_DIGITS ? (s <= kEsc) : (s == kEsc)) {
            out.put(kEsc);
            out.put((ESC_DIGITS && s != kEsc) ? (uint8_t)('0' + s - 1) : raw[i]);
            i += 1;
        } else {
            out.put(s);
            i += plen[s] ? plen[s] : 1u;  // every symbol on the path has a pattern; never stall
        }
    }
}

struct SmemSink {
    uint8_t *p;
    __device__ __forceinline__ void put(uint8_t b) { *p++ = b; }
};

struct GlobalSink {
    uint8_t *out;
    uint64_t pos, cap;
    __device__ __forceinline__ void put(uint8_t b)
    {
        if (pos < cap) out[pos] = b;
        ++pos;
    }
};

// Work space of one slow line of n input bytes: a 16-byte header {n, pre-processed length}, the
// pre-processed text (<= 3n bytes: a 1-byte label can become %nn), the chosen symbols, one label byte per
// ring token, and the 2 x 100 ints of the relabelling tables.
struct SlowLayout {
    uint64_t text, chs, tok, tables, need;
};

__device__ __forceinline__ SlowLayout slow_layout(uint32_t n)
{
    SlowLayout s;
    s.text = 16;
    s.chs = s.text + 3ull * n + 16;
    s.tok = s.chs + 3ull * n + 16;
    s.tables = (s.tok + n + 16 + 15) & ~15ull;
    s.need = (s.tables + 800 + 15) & ~15ull;
    return s;
}

}  // namespace cx
}  // namespace zs
