/*
 * ZSMILES CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow, single-threaded restatement of the ZSMILES codec of
 * arXiv 2404.19391, written to check the CUDA library against. Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it. It shares no code, header, table or helper with the CUDA path.
 *
 * What it computes, by paper section:
 *   - ring-ID pre-processing (Sec. IV-A): ring-closure labels are renumbered from 0 and reused once a
 *     ring has closed; among overlapping rings the innermost (first to close) gets the lower label;
 *   - compression (Sec. IV-D1): the minimum-output-length parse of a line over the dictionary D, a
 *     shortest path in the graph whose edges are matches of D (cost 1) or escapes (cost 2);
 *   - decompression (Sec. IV-D2): symbol -> pattern lookup; a space escapes the next byte;
 *   - line separability (Sec. I): one output line per input line, in order, plus a line-offset index.
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   - only the first whitespace-free field of a line is pre-processed; '[...]' atoms are opaque;
 *     a line with an unclosed ring label, an unclosed '[' or a '%' not followed by two digits, or one
 *     that would need a label above 99, is left unchanged;
 *   - "innermost gets the lower ID" = intervals are labelled in ascending order of their closing
 *     token, each with the smallest label not held by an already-labelled interval overlapping it;
 *   - the other reading of that sentence, kept as an experiment (flags bit 1): intervals are labelled in
 *     ascending order of their opening token by the same rule, so among nested rings the outermost gets
 *     the lower label;
 *   - parse tie-break: among minimum-cost parses, at each step take the longest piece (an escape is a
 *     piece of length 1 and loses every tie);
 *   - an escape is written as ' ' followed by the raw byte (the decoder reads the space first).
 *
 * Parity status: pre-processing, compression, decompression and the line index are pinned by the
 * tests (paper's worked example, closed forms, invariants, brute-force enumeration).
 */
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OZ_OK = 0, OZ_ERR_INVALID_ARG = 1, OZ_ERR_BAD_DICT = 2, OZ_ERR_CAPACITY = 3, OZ_ERR_MALFORMED = 4 };

#define OZ_MAX_PLEN 16

typedef struct {
    int lmin, lmax, n_alpha, n_learned;
    int n;                                  /* entries: alphabet singles first, then learned patterns */
    unsigned char sym[256];
    unsigned char plen[256];
    unsigned char pat[256][OZ_MAX_PLEN];
    int sym_entry[256];                     /* symbol byte -> entry, or -1 */
    int n_len[OZ_MAX_PLEN + 1];             /* entries of each pattern length ... */
    int by_len[OZ_MAX_PLEN + 1][256];       /* ... sorted by pattern bytes (for bsearch membership) */
} oz_dict;

/* ------------------------------------------------------------------------------------------------ */
/* Dictionary file                                                                                   */
/*   ZSDICT 1                                                                                        */
/*   <lmin> <lmax> <T>                                                                               */
/*   alphabet <hex of the pre-populated characters, or '-'>                                          */
/*   T lines: <symbol as 2 hex digits> <pattern as hex>                                              */
/* Each alphabet character c is the identity entry c -> "c". Symbols and patterns are unique, never   */
/* contain '\n' or ' ', and patterns are 1..lmax (<= 16) bytes long.                                 */
/* ------------------------------------------------------------------------------------------------ */

static int hexval(int c)
{
    if (c >= '0' && c <= '9') return c - '0';
    if (c >= 'a' && c <= 'f') return c - 'a' + 10;
    if (c >= 'A' && c <= 'F') return c - 'A' + 10;
    return -1;
}

typedef struct {
    const uint8_t *p, *end;
} cursor;

/* next line (without '\n') */
static int next_line(cursor *c, const uint8_t **ls, size_t *ln)
{
    if (c->p >= c->end) return 0;
    const uint8_t *s = c->p;
    while (c->p < c->end && *c->p != '\n') c->p++;
    *ls = s;
    *ln = (size_t)(c->p - s);
    if (c->p < c->end) c->p++;
    return 1;
}

static int parse_hex(const uint8_t *s, size_t n, unsigned char *out, size_t cap, size_t *outn)
{
    if (n % 2 != 0 || n / 2 > cap) return -1;
    for (size_t i = 0; i < n; i += 2) {
        int a = hexval(s[i]), b = hexval(s[i + 1]);
        if (a < 0 || b < 0) return -1;
        out[i / 2] = (unsigned char)(a * 16 + b);
    }
    *outn = n / 2;
    return 0;
}

static int add_entry(oz_dict *d, unsigned char sym, const unsigned char *pat, size_t len)
{
    if (sym == '\n' || sym == ' ' || len < 1 || len > (size_t)d->lmax || d->n >= 256) return -1;
    if (d->sym_entry[sym] >= 0) return -1;
    for (size_t i = 0; i < len; ++i)
        if (pat[i] == '\n' || pat[i] == ' ') return -1;
    for (int e = 0; e < d->n; ++e)
        if (d->plen[e] == len && memcmp(d->pat[e], pat, len) == 0) return -1;
    d->sym[d->n] = sym;
    d->plen[d->n] = (unsigned char)len;
    memcpy(d->pat[d->n], pat, len);
    d->sym_entry[sym] = d->n;
    d->n++;
    return 0;
}

int oz_dict_parse(const uint8_t *bytes, size_t len, oz_dict *d)
{
    memset(d, 0, sizeof *d);
    for (int i = 0; i < 256; ++i) d->sym_entry[i] = -1;
    cursor c = {bytes, bytes + len};
    const uint8_t *ls;
    size_t ln;
    if (!next_line(&c, &ls, &ln) || ln != 8 || memcmp(ls, "ZSDICT 1", 8) != 0) return OZ_ERR_BAD_DICT;
    if (!next_line(&c, &ls, &ln) || ln >= 64) return OZ_ERR_BAD_DICT;
    char hdr[64];
    memcpy(hdr, ls, ln);
    hdr[ln] = 0;
    char *q = hdr;
    long v[3];
    for (int k = 0; k < 3; ++k) {
        while (*q == ' ') ++q;
        if (*q < '0' || *q > '9') return OZ_ERR_BAD_DICT;
        v[k] = strtol(q, &q, 10);
    }
    while (*q == ' ') ++q;
    if (*q != 0) return OZ_ERR_BAD_DICT;
    d->lmin = (int)v[0];
    d->lmax = (int)v[1];
    d->n_learned = (int)v[2];
    if (d->lmin < 1 || d->lmax < d->lmin || d->lmax > OZ_MAX_PLEN || d->n_learned < 0 || d->n_learned > 254)
        return OZ_ERR_BAD_DICT;
    if (!next_line(&c, &ls, &ln) || ln < 10 || memcmp(ls, "alphabet ", 9) != 0) return OZ_ERR_BAD_DICT;
    unsigned char alpha[256];
    size_t na = 0;
    if (!(ln == 10 && ls[9] == '-')) {
        if (parse_hex(ls + 9, ln - 9, alpha, sizeof alpha, &na) != 0) return OZ_ERR_BAD_DICT;
    }
    for (size_t i = 0; i < na; ++i)
        if (add_entry(d, alpha[i], &alpha[i], 1) != 0) return OZ_ERR_BAD_DICT;
    d->n_alpha = (int)na;
    for (int t = 0; t < d->n_learned; ++t) {
        if (!next_line(&c, &ls, &ln)) return OZ_ERR_BAD_DICT;
        size_t sp = 0;
        while (sp < ln && ls[sp] != ' ') ++sp;
        unsigned char symb[1], pat[OZ_MAX_PLEN];
        size_t ns, np;
        if (sp != 2 || parse_hex(ls, 2, symb, 1, &ns) != 0) return OZ_ERR_BAD_DICT;
        if (sp + 1 >= ln || parse_hex(ls + sp + 1, ln - sp - 1, pat, sizeof pat, &np) != 0) return OZ_ERR_BAD_DICT;
        if (add_entry(d, symb[0], pat, np) != 0) return OZ_ERR_BAD_DICT;
    }
    while (next_line(&c, &ls, &ln))
        if (ln != 0) return OZ_ERR_BAD_DICT;
    for (int l = 1; l <= OZ_MAX_PLEN; ++l) {
        d->n_len[l] = 0;
        for (int e = 0; e < d->n; ++e)
            if (d->plen[e] == l) d->by_len[l][d->n_len[l]++] = e;
        /* insertion sort by pattern bytes */
        for (int a = 1; a < d->n_len[l]; ++a) {
            int e = d->by_len[l][a], b = a;
            while (b > 0 && memcmp(d->pat[d->by_len[l][b - 1]], d->pat[e], (size_t)l) > 0) {
                d->by_len[l][b] = d->by_len[l][b - 1];
                --b;
            }
            d->by_len[l][b] = e;
        }
    }
    return OZ_OK;
}

/* entry whose pattern equals s[0..l), or -1 ("s[i:i+l] in D") */
typedef struct {
    const oz_dict *d;
    const unsigned char *s;
    int l;
} lookup_key;

static int cmp_lookup(const void *key, const void *elem)
{
    const lookup_key *k = (const lookup_key *)key;
    int e = *(const int *)elem;
    return memcmp(k->s, k->d->pat[e], (size_t)k->l);
}

static int dict_find(const oz_dict *d, const unsigned char *s, int l)
{
    if (l < 1 || l > OZ_MAX_PLEN || d->n_len[l] == 0) return -1;
    lookup_key k = {d, s, l};
    const int *hit = (const int *)bsearch(&k, d->by_len[l], (size_t)d->n_len[l], sizeof(int), cmp_lookup);
    return hit ? *hit : -1;
}

int oz_dict_lmax(const oz_dict *d) { return d->lmax; }
int oz_dict_entries(const oz_dict *d) { return d->n; }
size_t oz_dict_size(void) { return sizeof(oz_dict); }

/* ------------------------------------------------------------------------------------------------ */
/* Pre-processing (Sec. IV-A)                                                                        */
/* ------------------------------------------------------------------------------------------------ */

typedef struct {
    size_t start, len;  /* span in the input line */
    int ring;           /* 1 if this token is a ring-closure label */
    int label;          /* original label value (ring tokens) */
    int interval;       /* interval index (ring tokens) */
} token;

typedef struct {
    size_t o, c;        /* token indices of the opening and the closing label */
    int label;          /* new label */
} interval;

static size_t copy_unchanged(const uint8_t *s, size_t n, uint8_t *out)
{
    memcpy(out, s, n);
    return n;
}

/* Pre-process one line (no '\n'); out needs 3*n bytes. Returns the new length. outer = 0: intervals are
 * labelled in closing order (the default reading); outer = 1: in opening order. */
size_t oz_preprocess_line_ex(const uint8_t *s, size_t n, uint8_t *out, int outer)
{
    size_t f = 0;
    while (f < n && s[f] != ' ' && s[f] != '\t') ++f;

    token *tok = (token *)malloc((f + 1) * sizeof(token));
    interval *iv = (interval *)malloc((f / 2 + 1) * sizeof(interval));
    size_t nt = 0, niv = 0;
    int ok = 1;

    /* tokenize the first field */
    for (size_t i = 0; i < f && ok;) {
        token t = {i, 1, 0, -1, -1};
        if (s[i] == '[') {
            size_t j = i + 1;
            while (j < f && s[j] != ']') ++j;
            if (j >= f) { ok = 0; break; }
            t.len = j - i + 1;
        } else if (s[i] == '%') {
            if (i + 2 < f && s[i + 1] >= '0' && s[i + 1] <= '9' && s[i + 2] >= '0' && s[i + 2] <= '9') {
                t.len = 3;
                t.ring = 1;
                t.label = (s[i + 1] - '0') * 10 + (s[i + 2] - '0');
            } else {
                ok = 0;
                break;
            }
        } else if (s[i] >= '0' && s[i] <= '9') {
            t.ring = 1;
            t.label = s[i] - '0';
        }
        tok[nt++] = t;
        i += t.len;
    }

    /* pair labels: a label opens if not open, else closes the open one */
    if (ok) {
        long open_tok[100];
        for (int l = 0; l < 100; ++l) open_tok[l] = -1;
        for (size_t k = 0; k < nt; ++k) {
            if (!tok[k].ring) continue;
            int l = tok[k].label;
            if (open_tok[l] < 0) {
                open_tok[l] = (long)k;
            } else {
                iv[niv].o = (size_t)open_tok[l];
                iv[niv].c = k;
                iv[niv].label = -1;
                tok[open_tok[l]].interval = (int)niv;
                tok[k].interval = (int)niv;
                ++niv;
                open_tok[l] = -1;
            }
        }
        for (int l = 0; l < 100; ++l)
            if (open_tok[l] >= 0) ok = 0;
    }

    /* visiting order: intervals were recorded in ascending closing position; for the opening-order
     * reading, visit them by ascending opening position instead (the opening tokens, left to right) */
    size_t *order = (size_t *)malloc((niv + 1) * sizeof(size_t));
    if (ok) {
        if (!outer) {
            for (size_t k = 0; k < niv; ++k) order[k] = k;
        } else {
            size_t q = 0;
            for (size_t k = 0; k < nt; ++k)
                if (tok[k].ring && iv[tok[k].interval].o == k) order[q++] = (size_t)tok[k].interval;
        }
    }

    /* label each interval, in that order, with the smallest label not held by an already-labelled
     * interval that overlaps it */
    if (ok) {
        for (size_t q = 0; q < niv && ok; ++q) {
            size_t k = order[q];
            int used[101];
            memset(used, 0, sizeof used);
            for (size_t p = 0; p < q; ++p) {
                size_t j = order[p];
                int overlap = iv[j].o < iv[k].c && iv[k].o < iv[j].c;
                if (overlap && iv[j].label <= 100) used[iv[j].label] = 1;
            }
            int lab = 0;
            while (lab <= 100 && used[lab]) ++lab;
            if (lab > 99) ok = 0;
            iv[k].label = lab;
        }
    }
    free(order);

    size_t m;
    if (!ok) {
        m = copy_unchanged(s, n, out);
    } else {
        m = 0;
        for (size_t k = 0; k < nt; ++k) {
            if (tok[k].ring) {
                int lab = iv[tok[k].interval].label;
                if (lab < 10) {
                    out[m++] = (uint8_t)('0' + lab);
                } else {
                    out[m++] = '%';
                    out[m++] = (uint8_t)('0' + lab / 10);
                    out[m++] = (uint8_t)('0' + lab % 10);
                }
            } else {
                memcpy(out + m, s + tok[k].start, tok[k].len);
                m += tok[k].len;
            }
        }
        memcpy(out + m, s + f, n - f);
        m += n - f;
    }
    free(tok);
    free(iv);
    return m;
}

size_t oz_preprocess_line(const uint8_t *s, size_t n, uint8_t *out) { return oz_preprocess_line_ex(s, n, out, 0); }

/* ------------------------------------------------------------------------------------------------ */
/* Compression of one line (Sec. IV-D1): shortest path, match cost 1, escape cost 2                  */
/* ------------------------------------------------------------------------------------------------ */

/* out needs 2*n bytes. Returns the compressed length. */
size_t oz_compress_line(const oz_dict *d, const uint8_t *s, size_t n, uint8_t *out)
{
    size_t *best = (size_t *)malloc((n + 1) * sizeof(size_t));
    best[n] = 0;
    for (size_t i = n; i-- > 0;) {
        size_t b = 2 + best[i + 1];                         /* escape */
        for (int l = 1; l <= d->lmax && (size_t)l <= n - i; ++l)
            if (dict_find(d, s + i, l) >= 0 && 1 + best[i + l] < b) b = 1 + best[i + l];
        best[i] = b;
    }
    size_t m = 0, i = 0;
    while (i < n) {
        int chosen = -1, lchosen = 0;
        int lmax = (size_t)d->lmax < n - i ? d->lmax : (int)(n - i);
        for (int l = lmax; l >= 1; --l) {
            int e = dict_find(d, s + i, l);
            if (e >= 0 && 1 + best[i + l] == best[i]) {
                chosen = e;
                lchosen = l;
                break;
            }
        }
        if (chosen >= 0) {
            out[m++] = d->sym[chosen];
            i += (size_t)lchosen;
        } else {
            out[m++] = ' ';
            out[m++] = s[i];
            i += 1;
        }
    }
    free(best);
    return m;
}

/* Cost of the optimal parse (= compressed length) of one line. */
size_t oz_parse_cost(const oz_dict *d, const uint8_t *s, size_t n)
{
    uint8_t *tmp = (uint8_t *)malloc(2 * n + 1);
    size_t m = oz_compress_line(d, s, n, tmp);
    free(tmp);
    return m;
}

/* ------------------------------------------------------------------------------------------------ */
/* Decompression of one line (Sec. IV-D2)                                                            */
/* ------------------------------------------------------------------------------------------------ */

/* out needs n * lmax bytes. Returns OZ_OK or OZ_ERR_MALFORMED (bad byte offset in *err). */
int oz_decompress_line(const oz_dict *d, const uint8_t *s, size_t n, uint8_t *out, size_t *outn, size_t *err)
{
    size_t m = 0;
    for (size_t i = 0; i < n;) {
        if (s[i] == ' ') {
            if (i + 1 >= n) { *err = i; return OZ_ERR_MALFORMED; }
            out[m++] = s[i + 1];
            i += 2;
        } else {
            int e = d->sym_entry[s[i]];
            if (e < 0) { *err = i; return OZ_ERR_MALFORMED; }
            memcpy(out + m, d->pat[e], d->plen[e]);
            m += d->plen[e];
            i += 1;
        }
    }
    *outn = m;
    return OZ_OK;
}

/* ------------------------------------------------------------------------------------------------ */
/* Streams: split at '\n', code each line, rejoin; the final-newline state is preserved              */
/* ------------------------------------------------------------------------------------------------ */

/* Number of lines: '\n' count, plus one for a last line without '\n'. */
size_t oz_count_lines(const uint8_t *s, size_t n)
{
    size_t k = 0;
    for (size_t i = 0; i < n; ++i) k += s[i] == '\n';
    if (n > 0 && s[n - 1] != '\n') ++k;
    return k;
}

/* index[0..n_lines] = start offset of each line, then n. Returns n_lines. */
size_t oz_line_index(const uint8_t *s, size_t n, uint64_t *index)
{
    size_t k = 0;
    size_t start = 0;
    for (size_t i = 0; i < n; ++i) {
        if (s[i] == '\n') {
            if (index) index[k] = start;
            ++k;
            start = i + 1;
        }
    }
    if (n > 0 && s[n - 1] != '\n') {
        if (index) index[k] = start;
        ++k;
    }
    if (index) index[k] = n;
    return k;
}

size_t oz_preprocess_bound(size_t n) { return 3 * n + 16; }
size_t oz_compress_bound(size_t n) { return 6 * n + 16; }

/* Pre-process every line of a stream; outer selects the opening-order reading. */
int oz_preprocess_stream_ex(const uint8_t *in, size_t n, int outer, uint8_t *out, size_t cap, size_t *out_len)
{
    size_t m = 0, i = 0;
    while (i < n) {
        size_t j = i;
        while (j < n && in[j] != '\n') ++j;
        if (m + 3 * (j - i) + 1 > cap) return OZ_ERR_CAPACITY;
        m += oz_preprocess_line_ex(in + i, j - i, out + m, outer);
        if (j < n) out[m++] = '\n';
        i = j + 1;
    }
    *out_len = m;
    return OZ_OK;
}

int oz_preprocess_stream(const uint8_t *in, size_t n, uint8_t *out, size_t cap, size_t *out_len)
{
    return oz_preprocess_stream_ex(in, n, 0, out, cap, out_len);
}

/* Compress a stream; flags bit 0 = pre-process each line first, bit 1 (with bit 0) = in the
 * opening-order reading. index (nullable) gets n_lines+1 offsets into the output. */
int oz_compress_stream(const oz_dict *d, const uint8_t *in, size_t n, unsigned flags, uint8_t *out, size_t cap,
                       uint64_t *index, size_t *out_len, size_t *n_lines)
{
    size_t m = 0, i = 0, k = 0;
    if ((flags & ~3u) || (flags & 3u) == 2u) return OZ_ERR_INVALID_ARG;
    uint8_t *pre = (uint8_t *)malloc(3 * 65536);
    size_t pre_cap = 3 * 65536;
    while (i < n) {
        size_t j = i;
        while (j < n && in[j] != '\n') ++j;
        size_t ln = j - i;
        if (3 * ln + 1 > pre_cap) {
            pre_cap = 3 * ln + 1;
            pre = (uint8_t *)realloc(pre, pre_cap);
        }
        size_t pn;
        if (flags & 1u) pn = oz_preprocess_line_ex(in + i, ln, pre, (flags & 2u) != 0);
        else { memcpy(pre, in + i, ln); pn = ln; }
        if (m + 2 * pn + 1 > cap) { free(pre); return OZ_ERR_CAPACITY; }
        if (index) index[k] = m;
        ++k;
        m += oz_compress_line(d, pre, pn, out + m);
        if (j < n) out[m++] = '\n';
        i = j + 1;
    }
    free(pre);
    if (index) index[k] = m;
    *out_len = m;
    *n_lines = k;
    return OZ_OK;
}

/* Decompress a stream. On malformed input, *err is the offset of the first bad byte. */
int oz_decompress_stream(const oz_dict *d, const uint8_t *in, size_t n, uint8_t *out, size_t cap,
                         size_t *out_len, size_t *err)
{
    size_t m = 0, i = 0;
    while (i < n) {
        size_t j = i;
        while (j < n && in[j] != '\n') ++j;
        if (m + (size_t)d->lmax * (j - i) + 1 > cap) return OZ_ERR_CAPACITY;
        size_t ln, e;
        int st = oz_decompress_line(d, in + i, j - i, out + m, &ln, &e);
        if (st != OZ_OK) { *err = i + e; return st; }
        m += ln;
        if (j < n) out[m++] = '\n';
        i = j + 1;
    }
    *out_len = m;
    return OZ_OK;
}

/* Random access: decode lines ids[0..k) of a compressed stream with its index, in request order, each
 * followed by '\n'; out_off gets k+1 offsets. An id >= n_lines is malformed (*err = its position). */
int oz_decompress_lines(const oz_dict *d, const uint8_t *comp, size_t comp_len, const uint64_t *index,
                        size_t n_lines, const uint64_t *ids, size_t k, uint8_t *out, size_t cap,
                        uint64_t *out_off, size_t *out_len, size_t *err)
{
    size_t m = 0;
    for (size_t r = 0; r < k; ++r) {
        if (ids[r] >= n_lines) { *err = r; return OZ_ERR_MALFORMED; }
        size_t a = (size_t)index[ids[r]], b = (size_t)index[ids[r] + 1];
        if (a > b || b > comp_len) { *err = r; return OZ_ERR_MALFORMED; }
        if (b > a && comp[b - 1] == '\n') --b;
        out_off[r] = m;
        if (m + (size_t)d->lmax * (b - a) + 1 > cap) return OZ_ERR_CAPACITY;
        size_t ln, e;
        int st = oz_decompress_line(d, comp + a, b - a, out + m, &ln, &e);
        if (st != OZ_OK) { *err = r; return st; }
        m += ln;
        out[m++] = '\n';
    }
    out_off[k] = m;
    *out_len = m;
    return OZ_OK;
}
