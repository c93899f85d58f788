// zs_load_dictionary: parse the dictionary file and build the encoder automaton and decoder tables.
#include <string.h>

#include <stdlib.h>

#include <algorithm>
#include <deque>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>

#include "zs_common.cuh"

namespace {

struct Entry {
    uint8_t sym;
    std::string pat;
};

int hexv(int c)
{
    if (c >= '0' && c <= '9') return c - '0';
    if (c >= 'a' && c <= 'f') return c - 'a' + 10;
    if (c >= 'A' && c <= 'F') return c - 'A' + 10;
    return -1;
}

bool unhex(const std::string &h, std::string *out)
{
    if (h.size() % 2) return false;
    out->clear();
    for (size_t i = 0; i < h.size(); i += 2) {
        int a = hexv((unsigned char)h[i]), b = hexv((unsigned char)h[i + 1]);
        if (a < 0 || b < 0) return false;
        out->push_back((char)(a * 16 + b));
    }
    return true;
}

bool parse_uint(const std::string &s, size_t *pos, long *v)
{
    while (*pos < s.size() && s[*pos] == ' ') ++*pos;
    if (*pos >= s.size() || s[*pos] < '0' || s[*pos] > '9') return false;
    long x = 0;
    while (*pos < s.size() && s[*pos] >= '0' && s[*pos] <= '9') {
        x = x * 10 + (s[*pos] - '0');
        if (x > 1000000) return false;
        ++*pos;
    }
    *v = x;
    return true;
}

// Parse the text format documented in zsmiles.h. Returns "" on success, else a message.
std::string parse(const uint8_t *bytes, size_t len, int *lmax_out, std::vector<Entry> *entries)
{
    std::vector<std::string> lines;
    size_t i = 0;
    while (i < len) {
        size_t j = i;
        while (j < len && bytes[j] != '\n') ++j;
        lines.emplace_back((const char *)bytes + i, j - i);
        i = j + 1;
    }
    if (lines.size() < 3 || lines[0] != "ZSDICT 1") return "missing 'ZSDICT 1' header";
    size_t p = 0;
    long lmin, lmax, T;
    if (!parse_uint(lines[1], &p, &lmin) || !parse_uint(lines[1], &p, &lmax) || !parse_uint(lines[1], &p, &T))
        return "bad '<lmin> <lmax> <T>' line";
    while (p < lines[1].size() && lines[1][p] == ' ') ++p;
    if (p != lines[1].size()) return "trailing characters after '<lmin> <lmax> <T>'";
    if (lmin < 1 || lmax < lmin || lmax > zs::kMaxPat) return "lmin/lmax out of range (1 <= lmin <= lmax <= 16)";
    if (T > 254) return "too many patterns";
    const std::string &al = lines[2];
    if (al.compare(0, 9, "alphabet ") != 0 || al.size() < 10) return "bad 'alphabet' line";
    std::string alpha;
    if (al.substr(9) != "-" && !unhex(al.substr(9), &alpha)) return "alphabet is not hex";
    bool sym_used[256] = {false};
    std::vector<std::string> pats;
    auto add = [&](uint8_t sym, const std::string &pat) -> std::string {
        if (sym == zs::kNl || sym == zs::kEsc) return "symbol is '\\n' or ' '";
        if (sym_used[sym]) return "duplicate symbol";
        if (pat.empty() || (long)pat.size() > lmax) return "pattern length outside 1..lmax";
        for (unsigned char c : pat)
            if (c == zs::kNl || c == zs::kEsc) return "pattern holds '\\n' or ' '";
        for (const auto &q : pats)
            if (q == pat) return "duplicate pattern";
        sym_used[sym] = true;
        pats.push_back(pat);
        entries->push_back({sym, pat});
        return "";
    };
    for (unsigned char c : alpha) {
        std::string err = add(c, std::string(1, (char)c));
        if (!err.empty()) return "alphabet: " + err;
    }
    if ((long)lines.size() < 3 + T) return "fewer pattern lines than T";
    for (long t = 0; t < T; ++t) {
        const std::string &l = lines[3 + t];
        size_t sp = l.find(' ');
        std::string s, pat;
        if (sp != 2 || !unhex(l.substr(0, 2), &s) || !unhex(l.substr(3), &pat)) return "bad pattern line";
        std::string err = add((uint8_t)s[0], pat);
        if (!err.empty()) return "pattern line " + std::to_string(t) + ": " + err;
    }
    for (size_t k = 3 + T; k < lines.size(); ++k)
        if (!lines[k].empty()) return "extra lines after the T pattern lines";
    *lmax_out = (int)lmax;
    return "";
}

struct Node {
    int child[256];
    int fail = 0;
    int term_len = 0;
    int term_sym = -1;
    Node() { std::fill(child, child + 256, -1); }
};

}  // namespace

// ------------------------------------------------------------------------------------------------
// Parse transducer.
//
// The backward shortest-path scan (Sec. IV-D1) needs, at position i, the match set of i (a function of
// the automaton state after reading s[i]) and best[i+1 .. i+Lp] for the longest pattern length Lp. The
// choice at i and the increment best[i] - best[i+1] depend on those values only through their
// differences, and with match cost 1 and escape cost 2 the differences stay bounded. So the pair
// (automaton state, window of best values relative to best[i]) ranges over a finite set, and the
// whole scan is a finite-state transducer: per byte class it moves to a next state and outputs the
// increment of best and the symbol chosen at that byte (' ' for an escape). Its reachable states are
// enumerated breadth-first and then merged by Moore partition refinement (states with identical output
// sequences for every input are equivalent); the minimal table is what the kernel walks, one lookup
// per byte. Returns false when the state space or the table exceeds the given limits.
// ------------------------------------------------------------------------------------------------
struct Machine {
    std::vector<uint32_t> table;  // [states][classes]: next | (delta + 16) << 16 | symbol << 24
    int states = 0;
    int start = 0;
};

bool build_machine(const std::vector<std::vector<int>> &delta, const std::vector<uint32_t> &mask,
                   const std::vector<std::vector<uint8_t>> &sym, int n_classes, int Lp, size_t max_states,
                   size_t max_table_bytes, Machine *out)
{
    const int W = Lp > 1 ? Lp - 1 : 0;  // window: best[i+1..i+Lp-1] - best[i]
    const int8_t INF = 127;
    struct Entry {
        int next;
        int delta;
        uint8_t sym;
    };
    std::unordered_map<std::string, int> id;
    std::vector<std::string> keys;
    auto key_of = [&](int ac, const int8_t *w) {
        std::string k(2 + W, '\0');
        k[0] = (char)(ac & 0xFF);
        k[1] = (char)(ac >> 8);
        for (int j = 0; j < W; ++j) k[2 + j] = (char)w[j];
        return k;
    };
    std::vector<int8_t> w0(W > 0 ? W : 1, INF);
    std::string k0 = key_of(0, w0.data());
    id[k0] = 0;
    keys.push_back(k0);
    std::vector<std::vector<Entry>> rows;
    for (size_t qi = 0; qi < keys.size(); ++qi) {
        const std::string cur = keys[qi];
        const int ac = (uint8_t)cur[0] | ((uint8_t)cur[1] << 8);
        const int8_t *w = reinterpret_cast<const int8_t *>(cur.data() + 2);
        std::vector<Entry> row(n_classes);
        for (int c = 0; c < n_classes; ++c) {
            const int a2 = delta[ac][c];
            const uint32_t m = mask[a2];
            int best = (m & 1u) ? 1 : 2, pick = 1;
            for (int l = 2; l <= Lp; ++l) {
                if (!((m >> (l - 1)) & 1u)) continue;
                const int v = w[l - 2];
                if (v == INF) return false;  // cannot happen: matches never reach past the line end
                if (1 + v <= best) {
                    best = 1 + v;
                    pick = l;
                }
            }
            const uint8_t sy = (pick == 1 && !(m & 1u)) ? (uint8_t)' ' : sym[a2][pick - 1];
            std::vector<int8_t> nw(W > 0 ? W : 1, INF);
            if (W > 0) {
                nw[0] = (int8_t)(-best);
                for (int j = 1; j < W; ++j) nw[j] = (w[j - 1] == INF) ? INF : (int8_t)(w[j - 1] - best);
            }
            std::string nk = key_of(a2, nw.data());
            auto it = id.find(nk);
            int nid;
            if (it == id.end()) {
                if (keys.size() >= max_states) return false;
                nid = (int)keys.size();
                id.emplace(nk, nid);
                keys.push_back(nk);
            } else {
                nid = it->second;
            }
            row[c] = {nid, best, sy};
        }
        rows.push_back(std::move(row));
    }
    const int N = (int)rows.size();

    // Moore refinement: start from the partition by output rows, split by successor classes
    std::vector<int> part(N), np(N);
    {
        std::map<std::vector<int>, int> sig;
        for (int i = 0; i < N; ++i) {
            std::vector<int> v(2 * n_classes);
            for (int c = 0; c < n_classes; ++c) {
                v[2 * c] = rows[i][c].delta;
                v[2 * c + 1] = rows[i][c].sym;
            }
            auto it = sig.emplace(std::move(v), (int)sig.size()).first;
            part[i] = it->second;
        }
    }
    int nparts = 0;
    for (int i = 0; i < N; ++i) nparts = std::max(nparts, part[i] + 1);
    for (;;) {
        std::map<std::vector<int>, int> sig;
        for (int i = 0; i < N; ++i) {
            std::vector<int> v(n_classes + 1);
            v[0] = part[i];
            for (int c = 0; c < n_classes; ++c) v[c + 1] = part[rows[i][c].next];
            auto it = sig.emplace(std::move(v), (int)sig.size()).first;
            np[i] = it->second;
        }
        const int n2 = (int)sig.size();
        part.swap(np);
        if (n2 == nparts) break;
        nparts = n2;
    }
    if (nparts > 65535 || (size_t)nparts * n_classes * 4 > max_table_bytes) return false;
    std::vector<int> rep(nparts, -1);
    for (int i = 0; i < N; ++i)
        if (rep[part[i]] < 0) rep[part[i]] = i;
    out->states = nparts;
    out->start = part[0];
    out->table.assign((size_t)nparts * n_classes, 0);
    for (int p2 = 0; p2 < nparts; ++p2)
        for (int c = 0; c < n_classes; ++c) {
            const Entry &e = rows[rep[p2]][c];
            out->table[(size_t)p2 * n_classes + c] =
                (uint32_t)part[e.next] | ((uint32_t)(e.delta + 16) << 16) | ((uint32_t)e.sym << 24);
        }
    return true;
}

extern "C" zs_status zs_load_dictionary(const uint8_t *file_bytes, size_t len, zs_dict **out)
{
    zs::clear_error();
    if (!out || (!file_bytes && len)) {
        zs::set_error("zs_load_dictionary: NULL argument");
        return ZS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    int lmax = 0;
    std::vector<Entry> entries;
    std::string err = parse(file_bytes, len, &lmax, &entries);
    if (!err.empty()) {
        zs::set_error("dictionary: " + err);
        return ZS_ERR_BAD_DICT;
    }

    // Character classes. The bytes that pre-processing and segmentation look at get fixed classes:
    // digit d -> d, '%' -> 10, '[' -> 11, ']' -> 12, ' ' -> 13, '\t' -> 14, '\n' -> 15. Every other byte
    // that occurs in some pattern gets its own class from 17 up (ascending byte order); all remaining
    // bytes share class 16.
    uint8_t cls[256];
    int n_classes = zs::kClsFirstFree;
    {
        bool seen[256] = {false};
        for (auto &e : entries)
            for (unsigned char c : e.pat) seen[c] = true;
        for (int b = 0; b < 256; ++b) cls[b] = zs::kClsOther;
        for (int dg = 0; dg < 10; ++dg) cls['0' + dg] = (uint8_t)dg;
        cls['%'] = zs::kClsPct;
        cls['['] = zs::kClsLbr;
        cls[']'] = zs::kClsRbr;
        cls[' '] = zs::kClsSpace;
        cls['\t'] = zs::kClsTab;
        cls['\n'] = zs::kClsNl;
        for (int b = 0; b < 256; ++b)
            if (seen[b] && cls[b] == zs::kClsOther) cls[b] = (uint8_t)n_classes++;
    }

    // trie of reversed patterns
    std::vector<Node> nodes(1);
    for (auto &e : entries) {
        int u = 0;
        for (int k = (int)e.pat.size() - 1; k >= 0; --k) {
            int c = cls[(unsigned char)e.pat[k]];
            if (nodes[u].child[c] < 0) {
                nodes[u].child[c] = (int)nodes.size();
                nodes.emplace_back();
            }
            u = nodes[u].child[c];
        }
        nodes[u].term_len = (int)e.pat.size();
        nodes[u].term_sym = e.sym;
    }
    const int S = (int)nodes.size();
    if (S > 65535) {
        zs::set_error("dictionary: automaton has too many states");
        return ZS_ERR_BAD_DICT;
    }

    // failure links and the complete transition function, breadth first
    std::vector<int> order;
    std::vector<std::vector<int>> delta(S, std::vector<int>(n_classes, 0));
    {
        std::deque<int> q;
        for (int c = 0; c < n_classes; ++c) {
            int v = nodes[0].child[c];
            if (v >= 0) {
                nodes[v].fail = 0;
                delta[0][c] = v;
                q.push_back(v);
            } else {
                delta[0][c] = 0;
            }
        }
        while (!q.empty()) {
            int u = q.front();
            q.pop_front();
            order.push_back(u);
            for (int c = 0; c < n_classes; ++c) {
                int v = nodes[u].child[c];
                if (v >= 0) {
                    nodes[v].fail = delta[nodes[u].fail][c];
                    delta[u][c] = v;
                    q.push_back(v);
                } else {
                    delta[u][c] = delta[nodes[u].fail][c];
                }
            }
        }
    }
    // match sets and symbols along each failure chain
    std::vector<uint32_t> mask(S, 0);
    std::vector<std::vector<uint8_t>> sym(S, std::vector<uint8_t>(zs::kMaxPat, 0));
    auto fill = [&](int u) {
        int f = nodes[u].fail;
        mask[u] = (u == 0) ? 0u : mask[f];
        if (u != 0) sym[u] = sym[f];
        if (nodes[u].term_len) {
            mask[u] |= 1u << (nodes[u].term_len - 1);
            sym[u][nodes[u].term_len - 1] = (uint8_t)nodes[u].term_sym;
        }
    };
    fill(0);
    for (int u : order) fill(u);

    std::vector<uint32_t> distinct;
    for (int u = 0; u < S; ++u)
        if (std::find(distinct.begin(), distinct.end(), mask[u]) == distinct.end()) distinct.push_back(mask[u]);
    const bool compact = S <= 2048 && distinct.size() <= 32;

    zs::EncLayout L{};
    L.n_states = (uint32_t)S;
    L.n_classes = (uint32_t)n_classes;
    L.compact = compact ? 1u : 0u;
    L.lmax = (uint32_t)lmax;
    L.off_trans = zs::kOffTrans;
    uint32_t trans_bytes = (uint32_t)S * (uint32_t)n_classes * (compact ? 2u : 4u);
    trans_bytes = (trans_bytes + 15u) & ~15u;
    L.off_sym = L.off_trans + trans_bytes;
    L.img_bytes = L.off_sym + (uint32_t)S * 16u;
    const uint32_t kMaxImg = 150u * 1024u;
    if (L.img_bytes > kMaxImg) {
        zs::set_error("dictionary: encoder automaton (" + std::to_string(L.img_bytes) +
                      " bytes) exceeds the 150 KiB shared-memory budget");
        return ZS_ERR_BAD_DICT;
    }

    std::vector<uint8_t> img(L.img_bytes, 0);
    memcpy(img.data() + zs::kOffCls, cls, 256);
    uint8_t plen[256] = {0};
    uint8_t pat[256][zs::kMaxPat];
    memset(pat, 0, sizeof pat);
    for (auto &e : entries) {
        plen[e.sym] = (uint8_t)e.pat.size();
        memcpy(pat[e.sym], e.pat.data(), e.pat.size());
    }
    memcpy(img.data() + zs::kOffPlen, plen, 256);
    if (compact) {
        uint32_t *m = (uint32_t *)(img.data() + zs::kOffMasks);
        for (size_t k = 0; k < distinct.size(); ++k) m[k] = distinct[k];
        uint16_t *t = (uint16_t *)(img.data() + L.off_trans);
        for (int u = 0; u < S; ++u)
            for (int c = 0; c < n_classes; ++c) {
                int v = delta[u][c];
                uint32_t id = (uint32_t)(std::find(distinct.begin(), distinct.end(), mask[v]) - distinct.begin());
                t[u * n_classes + c] = (uint16_t)(v | (id << 11));
            }
    } else {
        uint32_t *t = (uint32_t *)(img.data() + L.off_trans);
        for (int u = 0; u < S; ++u)
            for (int c = 0; c < n_classes; ++c) {
                int v = delta[u][c];
                t[u * n_classes + c] = (uint32_t)v | (mask[v] << 16);
            }
    }
    for (int u = 0; u < S; ++u) memcpy(img.data() + L.off_sym + 16 * u, sym[u].data(), 16);

    // parse transducer image: replicated class table, pattern lengths, transition table
    int Lp = 1;
    for (auto &en : entries) Lp = std::max(Lp, (int)en.pat.size());
    Machine mach;
    const char *force_generic = getenv("ZS_FORCE_GENERIC");
    const bool use_machine = !(force_generic && *force_generic && *force_generic != '0') &&
                             build_machine(delta, mask, sym, n_classes, Lp, 1u << 20, zs::kMaxMachineBytes, &mach);
    std::vector<uint8_t> mimg;
    zs::MachineLayout ML{};
    if (use_machine) {
        ML.n_states = (uint32_t)mach.states;
        ML.n_classes = (uint32_t)n_classes;
        ML.start = (uint32_t)mach.start * (uint32_t)n_classes;  // row offset of the start state
        ML.off_table = zs::kMOffTable;
        ML.img_bytes = zs::kMOffTable + (uint32_t)(mach.table.size() * 4);
        ML.img_bytes = (ML.img_bytes + 15u) & ~15u;
        mimg.assign(ML.img_bytes, 0);
        for (int c = 0; c < 256; ++c)
            for (int ln = 0; ln < 32; ++ln) mimg[zs::kMOffClsRep + ((c >> 2) * 32 + ln) * 4 + (c & 3)] = cls[c];
        for (auto &en : entries) mimg[zs::kMOffPlen + en.sym] = (uint8_t)en.pat.size();
        // the image stores each next state as its row offset (state * classes, < 2^16 within the table
        // budget), so the kernel's per-byte lookup needs no multiply
        std::vector<uint32_t> rows(mach.table);
        for (uint32_t &e : rows) e = (e & 0xFFFF0000u) | ((e & 0xFFFFu) * (uint32_t)n_classes);
        ML.esc_digits = 1;  // needs every symbol byte above ' ' (so choices up to ' ' are escapes)
        for (auto &en : entries)
            if (en.sym < 0x20) ML.esc_digits = 0;
        if (ML.esc_digits)  // an escape chosen at digit class d becomes the choice 1 + d
            for (size_t i = 0; i < rows.size(); ++i) {
                const uint32_t k = (uint32_t)(i % (size_t)n_classes);
                if (k < 10 && (rows[i] >> 24) == (uint32_t)' ') rows[i] = (rows[i] & 0x00FFFFFFu) | ((1u + k) << 24);
            }
        memcpy(mimg.data() + zs::kMOffTable, rows.data(), rows.size() * 4);
    }

    // byte-indexed transducer for the span kernel: at most 256 states (8-bit next state), every symbol
    // above ' ' (so choices up to ' ' are free for escapes and '\n'), every pattern byte below 0x80 and
    // some byte below 0x80 in no pattern that stands for the bytes >= 0x80
    std::vector<uint8_t> bimg;
    zs::ByteLayout BL{};
    if (use_machine && mach.states <= 256) {
        bool ok = true;
        for (auto &en : entries) {
            if (en.sym <= zs::kEsc) ok = false;
            for (unsigned char c : en.pat)
                if (c >= 0x80) ok = false;
        }
        int rep = -1;
        for (int b = 1; b < 128 && rep < 0; ++b)
            if (cls[b] == zs::kClsOther) rep = b;
        if (ok && rep > 0) {
            const uint32_t S = (uint32_t)mach.states;
            BL.n_states = S;
            BL.q0 = (uint32_t)mach.start;
            BL.meta_off = S * 256u;
            BL.img_bytes = BL.meta_off + 1024u;
            BL.rep_col = 2u * (uint32_t)rep;
            bimg.assign(BL.img_bytes, 0);
            uint16_t *t16 = reinterpret_cast<uint16_t *>(bimg.data());
            for (uint32_t q = 0; q < S; ++q)
                for (uint32_t b = 0; b < 128; ++b) {
                    uint32_t ns, ch;
                    if (b == zs::kNl) {
                        ns = BL.q0;
                        ch = zs::kNl;
                    } else {
                        const uint32_t e2 = mach.table[(size_t)q * n_classes + cls[b]];
                        ns = e2 & 0xFFFFu;
                        ch = e2 >> 24;
                        if (ch == zs::kEsc && b >= '0' && b <= '9') ch = 0x10u + (b - '0');
                    }
                    t16[q * 128 + (b ^ ((q & 31u) << 1))] = (uint16_t)(ns | (ch << 8));  // bank swizzle
                }
            uint32_t *meta = reinterpret_cast<uint32_t *>(bimg.data() + BL.meta_off);
            for (uint32_t c = 0; c < 256; ++c) {
                uint32_t step = 1, outb = 1;
                if (c == zs::kEsc || (c >= 0x10 && c < 0x1A)) outb = 2;
                else if (c > zs::kEsc && plen[c]) step = plen[c];
                meta[c] = step | (outb << 13);
            }
        }
    }

    std::vector<uint8_t> dec(zs::kDecBytes, 0);
    memcpy(dec.data(), plen, 256);
    memcpy(dec.data() + 256, pat, sizeof pat);

    zs_dict *d = new zs_dict();
    d->digest = 1469598103934665603ull;  // FNV-1a, 64-bit
    for (size_t i = 0; i < len; ++i) d->digest = (d->digest ^ file_bytes[i]) * 1099511628211ull;
    cudaError_t e = cudaGetDevice(&d->device);
    if (e != cudaSuccess) {
        delete d;
        return zs::cuda_fail(e, "cudaGetDevice");
    }
    d->lmax = lmax;
    d->max_plen = 1;
    for (int b = 0; b < 256; ++b) d->max_plen = std::max(d->max_plen, (int)plen[b]);
    d->layout = L;
    d->mlayout = ML;
    d->has_machine = use_machine;
    d->blayout = BL;
    d->has_bytes = !bimg.empty();
    memcpy(d->plen, plen, 256);
    memcpy(d->pat, pat, sizeof pat);
    e = cudaMalloc((void **)&d->d_enc, L.img_bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&d->d_dec, zs::kDecBytes);
    if (e == cudaSuccess) e = cudaMemcpy(d->d_enc, img.data(), L.img_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d->d_dec, dec.data(), zs::kDecBytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && use_machine) {
        e = cudaMalloc((void **)&d->d_mimg, ML.img_bytes);
        if (e == cudaSuccess) e = cudaMemcpy(d->d_mimg, mimg.data(), ML.img_bytes, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && d->has_bytes) {
        e = cudaMalloc((void **)&d->d_bimg, BL.img_bytes);
        if (e == cudaSuccess) e = cudaMemcpy(d->d_bimg, bimg.data(), BL.img_bytes, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (d->d_bimg) cudaFree(d->d_bimg);
        if (d->d_enc) cudaFree(d->d_enc);
        if (d->d_dec) cudaFree(d->d_dec);
        if (d->d_mimg) cudaFree(d->d_mimg);
        delete d;
        return zs::cuda_fail(e, "uploading dictionary tables");
    }
    *out = d;
    return ZS_OK;
}

extern "C" void zs_free_dictionary(zs_dict *d)
{
    if (!d) return;
    int cur = -1;
    cudaGetDevice(&cur);
    cudaSetDevice(d->device);
    d->pool.release_all();
    zs::free_pipes(d);
    if (d->d_enc) cudaFree(d->d_enc);
    if (d->d_dec) cudaFree(d->d_dec);
    if (d->d_mimg) cudaFree(d->d_mimg);
    if (d->d_bimg) cudaFree(d->d_bimg);
    if (cur >= 0) cudaSetDevice(cur);
    delete d;
}
