// zs_train_dictionary: dictionary generation (Algorithm 1 with the rank of Eq. 1, Sec. IV-C) on the GPU.
//
//   1. Pre-processing (Sec. IV-A) of the training lines, if asked: a round trip through a dictionary of
//      the alphabet alone (decompress(compress(x)) is the pre-processed x), all on the device.
//   2. Counting, one pattern length at a time: every window of the training stream of that length that
//      holds no ' ' and no '\n' is inserted into an open-addressing hash table in device memory (the
//      window's bytes packed into a 64-bit key, the count by atomic add). The table's occupied slots are
//      then gathered into a candidate list (pattern, count).
//   3. Selection on the host: T picks of the highest rank occ * (len - overlap) (Eq. 1), overlap being the
//      largest overlap with a pattern picked before. It uses a lazily re-evaluated max-heap: ranks only
//      fall as patterns are picked, so the first popped entry whose fresh rank still beats the heap top is
//      the argmax. Ties go to the higher count, then the longer pattern, then the bytewise smaller one. It
//      stops early once the best rank is <= 0.
//   4. The .zsd text: header, pre-populated alphabet, then one symbol per pick, in pick order, symbols from
//      the code space (printable bytes 0x21-0x7E outside the alphabet, then 0xA1-0xFF) in ascending order.
// Patterns are at most 8 bytes here (one 64-bit key); training bytes must not be 0 (a packed key of 0
// marks an empty slot).
#include <algorithm>
#include <cstring>
#include <queue>
#include <string>
#include <vector>

#include "zs_common.cuh"

namespace {

// SMILES alphabet pre-populated as identity entries (Sec. IV-B): digits, bond, branch, bracket, charge and
// chirality marks, the organic-subset element letters, the second letters of Cl and Br, aromatic atoms.
const char kSmilesAlphabet[] = "0123456789()[]=#$:/\\.+-@%*BCNOPSFIHlrbcnops";

struct Cand {
    uint64_t key;  // pattern bytes, little-endian (byte 0 first)
    uint32_t count;
    uint32_t len;
};

__device__ __forceinline__ uint64_t mix64(uint64_t x)
{
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

// Counts every window of length l of s[0, n) that holds no ' ' and no '\n'. flags[0] |= 1: the table
// overflowed (never with the sizing below; the host then reports an error).
__global__ void count_kernel(const uint8_t *__restrict__ s, uint64_t n, uint32_t l, unsigned long long *keys,
                             uint32_t *counts, uint64_t mask, uint32_t *flags)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i + l <= n; i += stride) {
        uint64_t key = 0;
        bool ok = true;
        for (uint32_t k = 0; k < l; ++k) {
            const uint8_t b = s[i + k];
            ok &= (b != ' ') & (b != '\n');
            key |= (uint64_t)b << (8 * k);
        }
        if (!ok) continue;
        uint64_t h = mix64(key) & mask;
        for (uint64_t probe = 0;; ++probe) {
            if (probe > mask) {
                atomicOr(flags, 1u);
                break;
            }
            const unsigned long long prev = atomicCAS(&keys[h], 0ull, (unsigned long long)key);
            if (prev == 0ull || prev == key) {
                atomicAdd(&counts[h], 1u);
                break;
            }
            h = (h + 1) & mask;
        }
    }
}

__global__ void gather_kernel(const unsigned long long *keys, const uint32_t *counts, uint64_t slots, uint32_t l,
                              Cand *out, unsigned long long *n_out)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < slots; i += stride) {
        if (keys[i] == 0ull) continue;
        const unsigned long long at = atomicAdd(n_out, 1ull);
        out[at] = Cand{keys[i], counts[i], l};
    }
}

// Finds a zero byte in s[0, n) (flags[0] |= 2).
__global__ void nul_kernel(const uint8_t *s, uint64_t n, uint32_t *flags)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        if (s[i] == 0) atomicOr(flags, 2u);
}

std::string pattern_of(const Cand &c)
{
    std::string p(c.len, '\0');
    for (uint32_t k = 0; k < c.len; ++k) p[k] = (char)((c.key >> (8 * k)) & 0xFF);
    return p;
}

// overlap_{p,w}: |p| if p occurs inside w; else |w| if w occurs inside p; else the longest proper suffix of
// one that is a prefix of the other (either order); else 0.
int overlap(const std::string &p, const std::string &w)
{
    if (w.find(p) != std::string::npos) return (int)p.size();
    if (p.find(w) != std::string::npos) return (int)w.size();
    int best = 0;
    const int m = (int)std::min(p.size(), w.size());
    for (int k = 1; k < m; ++k) {
        const bool a = p.compare(p.size() - k, k, w, 0, k) == 0;
        const bool b = w.compare(w.size() - k, k, p, 0, k) == 0;
        if (a || b) best = k;
    }
    return best;
}

struct Key {  // ordered so that the best entry is the largest
    int64_t rank;
    int64_t occ;
    int len;
    std::string pat;
    bool operator<(const Key &o) const
    {
        if (rank != o.rank) return rank < o.rank;
        if (occ != o.occ) return occ < o.occ;
        if (len != o.len) return len < o.len;
        return pat > o.pat;  // bytewise smaller wins
    }
};

std::vector<std::string> select_patterns(const std::vector<Cand> &cands, int T)
{
    std::priority_queue<Key> heap;
    for (const Cand &c : cands) heap.push(Key{(int64_t)c.count * (int64_t)c.len, (int64_t)c.count, (int)c.len,
                                              pattern_of(c)});
    std::vector<std::string> selected;
    while (!heap.empty() && (int)selected.size() < T) {
        Key top = heap.top();
        heap.pop();
        int ov = 0;
        for (const std::string &w : selected) ov = std::max(ov, overlap(top.pat, w));
        top.rank = top.occ * ((int64_t)top.len - ov);
        if (!heap.empty() && top < heap.top()) {  // no longer the best: put it back with its fresh rank
            heap.push(top);
            continue;
        }
        if (top.rank <= 0) break;
        selected.push_back(top.pat);
    }
    return selected;
}

std::string hex(const std::string &s)
{
    static const char *d = "0123456789abcdef";
    std::string o;
    for (unsigned char c : s) {
        o.push_back(d[c >> 4]);
        o.push_back(d[c & 15]);
    }
    return o;
}

std::vector<int> code_space(const std::string &alphabet)
{
    std::vector<int> out;
    auto in_alpha = [&](int b) { return alphabet.find((char)b) != std::string::npos; };
    for (int b = 0x21; b < 0x7F; ++b)
        if (!in_alpha(b)) out.push_back(b);
    for (int b = 0xA1; b < 0x100; ++b)
        if (!in_alpha(b)) out.push_back(b);
    return out;
}

std::string dictionary_text(const std::vector<std::string> &pats, const std::string &alphabet, int lmin, int lmax)
{
    const std::vector<int> space = code_space(alphabet);
    std::string t = "ZSDICT 1\n" + std::to_string(lmin) + " " + std::to_string(lmax) + " " +
                    std::to_string(pats.size()) + "\nalphabet " + (alphabet.empty() ? "-" : hex(alphabet)) + "\n";
    for (size_t i = 0; i < pats.size(); ++i) {
        char sym[4];
        snprintf(sym, sizeof sym, "%02x", space[i]);
        t += std::string(sym) + " " + hex(pats[i]) + "\n";
    }
    return t;
}

}  // namespace

extern "C" zs_status zs_train_dictionary(const uint8_t *d_train, size_t n, unsigned flags, const zs_train_options *opt,
                                         uint8_t *out, size_t out_cap, size_t *out_len, void *stream)
{
    zs::clear_error();
    if (!out_len || (!d_train && n) || (!out && out_cap)) {
        zs::set_error("zs_train_dictionary: NULL argument");
        return ZS_ERR_INVALID_ARG;
    }
    *out_len = 0;
    if (!zs::compress_flags_ok(flags)) {
        zs::set_error("zs_train_dictionary: unknown flag bits, or ZS_PREPROCESS_OUTER without ZS_PREPROCESS");
        return ZS_ERR_INVALID_ARG;
    }
    const int lmin = opt && opt->lmin > 0 ? opt->lmin : 2;
    const int lmax = opt && opt->lmax > 0 ? opt->lmax : 8;
    const std::string alphabet = (opt && opt->no_alphabet) ? std::string() : std::string(kSmilesAlphabet);
    const int space = (int)code_space(alphabet).size();
    const int T = std::min(opt && opt->T > 0 ? opt->T : space, space);
    if (lmin < 1 || lmax < lmin || lmax > 8) {
        zs::set_error("zs_train_dictionary: need 1 <= lmin <= lmax <= 8");
        return ZS_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<void *> owned;
    auto alloc = [&](void **p, size_t bytes) -> bool {
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        owned.push_back(*p);
        return true;
    };
    auto cleanup = [&]() {
        for (void *p : owned) cudaFree(p);
    };
    zs_status st = ZS_OK;
    const uint8_t *text = d_train;
    uint64_t tn = n;
    uint32_t *d_flags = nullptr;
    if (!alloc(reinterpret_cast<void **>(&d_flags), sizeof(uint32_t))) {
        zs::set_error("zs_train_dictionary: out of device memory");
        return ZS_ERR_OOM;
    }
    cudaMemsetAsync(d_flags, 0, sizeof(uint32_t), s);
    if (n) nul_kernel<<<1024, 256, 0, s>>>(d_train, n, d_flags);

    if ((flags & ZS_PREPROCESS) && n) {  // pre-processing: a round trip through the alphabet alone
        const std::string a(kSmilesAlphabet);
        const std::string file = "ZSDICT 1\n1 1 0\nalphabet " + hex(a) + "\n";
        zs_dict *alpha = nullptr;
        st = zs_load_dictionary(reinterpret_cast<const uint8_t *>(file.data()), file.size(), &alpha);
        uint8_t *comp = nullptr, *pre = nullptr;
        const size_t ccap = zs_compress_bound(n), pcap = zs_decompress_bound(alpha, ccap);
        if (st == ZS_OK && (!alloc(reinterpret_cast<void **>(&comp), ccap) ||
                            !alloc(reinterpret_cast<void **>(&pre), pcap))) {
            zs::set_error("zs_train_dictionary: out of device memory");
            st = ZS_ERR_OOM;
        }
        zs_result r{};
        if (st == ZS_OK) st = zs_compress(alpha, d_train, n, flags, comp, ccap, nullptr, 0, &r, stream);
        zs_result r2{};
        if (st == ZS_OK) st = zs_decompress(alpha, comp, r.out_len, pre, pcap, &r2, stream);
        if (alpha) zs_free_dictionary(alpha);
        if (st != ZS_OK) {
            cleanup();
            return st;
        }
        text = pre;
        tn = r2.out_len;
    }

    // counting, one length at a time, into one reused table
    uint64_t slots = 1024;
    while (slots < 2 * std::max<uint64_t>(tn, 1)) slots <<= 1;
    unsigned long long *keys = nullptr, *d_ncand = nullptr;
    uint32_t *counts = nullptr;
    Cand *d_cand = nullptr;
    if (!alloc(reinterpret_cast<void **>(&keys), slots * 8) || !alloc(reinterpret_cast<void **>(&counts), slots * 4) ||
        !alloc(reinterpret_cast<void **>(&d_cand), slots * sizeof(Cand)) ||
        !alloc(reinterpret_cast<void **>(&d_ncand), 8)) {
        cleanup();
        zs::set_error("zs_train_dictionary: out of device memory for the count table");
        return ZS_ERR_OOM;
    }
    std::vector<Cand> cands;
    cudaError_t e = cudaSuccess;
    for (int l = lmin; l <= lmax && e == cudaSuccess && tn >= (uint64_t)l; ++l) {
        e = cudaMemsetAsync(keys, 0, slots * 8, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, slots * 4, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_ncand, 0, 8, s);
        if (e != cudaSuccess) break;
        count_kernel<<<2048, 256, 0, s>>>(text, tn, (uint32_t)l, keys, counts, slots - 1, d_flags);
        gather_kernel<<<2048, 256, 0, s>>>(keys, counts, slots, (uint32_t)l, d_cand, d_ncand);
        unsigned long long nc = 0;
        e = cudaMemcpyAsync(&nc, d_ncand, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        const size_t at = cands.size();
        cands.resize(at + nc);
        if (nc) e = cudaMemcpy(cands.data() + at, d_cand, nc * sizeof(Cand), cudaMemcpyDeviceToHost);
    }
    uint32_t hflags = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&hflags, d_flags, sizeof hflags, cudaMemcpyDeviceToHost);
    cleanup();
    if (e != cudaSuccess) return zs::cuda_fail(e, "zs_train_dictionary");
    if (hflags & 2u) {
        zs::set_error("zs_train_dictionary: the training text holds a zero byte");
        return ZS_ERR_INVALID_ARG;
    }
    if (hflags & 1u) {
        zs::set_error("zs_train_dictionary: count table overflow");
        return ZS_ERR_OOM;
    }
    const std::vector<std::string> pats = select_patterns(cands, T);
    const std::string file = dictionary_text(pats, alphabet, lmin, lmax);
    *out_len = file.size();
    if (file.size() > out_cap) {
        zs::set_error("zs_train_dictionary: output buffer too small");
        return ZS_ERR_CAPACITY;
    }
    memcpy(out, file.data(), file.size());
    return ZS_OK;
}
