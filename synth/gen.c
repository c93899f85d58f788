/*
 * Seeded synthetic SMILES-like line generator.
 *
 * This module only produces inputs. It holds none of the codec's arithmetic (no ring relabelling, no
 * dictionary, no parse), and both the CPU oracle and the CUDA path consume what it writes.
 *
 * Counter-based: line `i` of seed `s` is drawn from its own PCG32 stream whose state and increment come
 * from SplitMix64 over (s, i). Any range of lines can therefore be generated independently, in any
 * order, by any number of threads, with identical bytes. Everything is integer arithmetic, so x86_64
 * and aarch64 hosts produce the same bytes.
 *
 * Grammar (shaped like drug-like SMILES libraries):
 *   - atoms C N O S F Cl Br P (aliphatic) and c n o s (aromatic); aromatic atoms are likely while an
 *     "aromatic" ring is open;
 *   - bracket atoms with probability p_bracket from a small set ([nH] [C@@H] [N+] [O-]) or, for long
 *     lines, from a wider set;
 *   - bonds '=' and '#' occasionally, '/' and '\' stereo bonds on long lines;
 *   - branches '(' ... ')' nested at most 4 deep, never empty;
 *   - ring bonds open with a label drawn uniformly from the currently free labels 1-9 (or, for 30% of
 *     the rings of long lines, from %10-%99) and close after 3-7 further atoms, so the labels are not
 *     canonical;
 *   - the line stops once it reaches its drawn target length, then closes open rings and branches.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef struct {
    uint64_t seed;
    int32_t len_mean_milli; /* mean of the normal line-length target, in thousandths of a char */
    int32_t len_sd_milli;   /* its standard deviation, same unit */
    int32_t len_lo, len_hi; /* clip range of the target */
    uint32_t p_long16;      /* probability (out of 65536) that a line is a long line */
    int32_t long_lo, long_hi; /* uniform target range of long lines */
} synth_params;

typedef struct {
    uint64_t state, inc;
} rng_t;

static uint64_t splitmix64_next(uint64_t *x)
{
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static uint32_t pcg32_next(rng_t *r)
{
    uint64_t old = r->state;
    r->state = old * 6364136223846793005ULL + r->inc;
    uint32_t xs = (uint32_t)(((old >> 18) ^ old) >> 27);
    uint32_t rot = (uint32_t)(old >> 59);
    return (xs >> rot) | (xs << ((32u - rot) & 31u));
}

static void rng_for_line(rng_t *r, uint64_t seed, uint64_t line)
{
    uint64_t x = seed * 0xD1B54A32D192ED03ULL ^ line;
    uint64_t init_state = splitmix64_next(&x);
    r->inc = (splitmix64_next(&x) << 1) | 1u;
    r->state = 0;
    pcg32_next(r);
    r->state += init_state;
    pcg32_next(r);
}

/* uniform integer in [0, n) */
static uint32_t below(rng_t *r, uint32_t n)
{
    return (uint32_t)(((uint64_t)pcg32_next(r) * n) >> 32);
}

/* true with probability p16 / 65536 */
static int chance(rng_t *r, uint32_t p16)
{
    return (pcg32_next(r) >> 16) < p16;
}

/* approximately normal target length: Irwin-Hall sum of 12 uniforms (mean 6, variance 1) */
static int32_t normal_len(rng_t *r, int32_t mean_milli, int32_t sd_milli, int32_t lo, int32_t hi)
{
    int64_t s = 0;
    for (int k = 0; k < 12; ++k) s += (int64_t)(pcg32_next(r) >> 16);
    int64_t z65536 = s - 6 * 65536;  /* N(0,1) scaled by 65536 */
    int64_t num = (int64_t)mean_milli * 65536 + (int64_t)sd_milli * z65536;
    int64_t den = (int64_t)65536 * 1000;
    int64_t v = num >= 0 ? (num + den / 2) / den : -((-num + den / 2) / den);
    if (v < lo) v = lo;
    if (v > hi) v = hi;
    return (int32_t)v;
}

#define P16(x) ((uint32_t)((x) * 65536.0 + 0.5))
#define MAX_OPEN 12

typedef struct {
    uint8_t *buf;
    size_t len, cap;
    int overflow;
} sink_t;

static void put(sink_t *s, const char *t, size_t n)
{
    if (s->len + n > s->cap) { s->overflow = 1; return; }
    memcpy(s->buf + s->len, t, n);
    s->len += n;
}

static void put1(sink_t *s, char c) { put(s, &c, 1); }

typedef struct {
    int label;      /* 1..99 */
    int countdown;  /* atoms left before closure */
    int aromatic;
    int opened_at;  /* atom ordinal that carries the opening label */
} ring_t;

static const char *const brackets_small[] = {"[nH]", "[C@@H]", "[N+]", "[O-]"};
static const char *const brackets_wide[] = {"[C@H]", "[C@@H]", "[NH3+]", "[N+]",
                                            "[O-]", "[nH]", "[NH2+]", "[S@@]"};

static void put_label(sink_t *s, int label)
{
    if (label < 10) {
        put1(s, (char)('0' + label));
    } else {
        char t[3] = {'%', (char)('0' + label / 10), (char)('0' + label % 10)};
        put(s, t, 3);
    }
}

static void put_atom(sink_t *s, rng_t *r, int aromatic_ctx, int long_line)
{
    uint32_t pb = long_line ? P16(0.30) : P16(0.05);
    if (chance(r, pb)) {
        if (long_line) {
            const char *b = brackets_wide[below(r, 8)];
            put(s, b, strlen(b));
        } else {
            const char *b = brackets_small[below(r, 4)];
            put(s, b, strlen(b));
        }
        return;
    }
    int aromatic = aromatic_ctx ? chance(r, P16(0.85)) : chance(r, P16(0.04));
    uint32_t u = below(r, 100);
    if (aromatic) {
        put1(s, u < 75 ? 'c' : u < 90 ? 'n' : u < 95 ? 'o' : 's');
    } else {
        if (u < 62) put1(s, 'C');
        else if (u < 74) put1(s, 'N');
        else if (u < 86) put1(s, 'O');
        else if (u < 90) put1(s, 'S');
        else if (u < 93) put1(s, 'F');
        else if (u < 96) put(s, "Cl", 2);
        else if (u < 98) put(s, "Br", 2);
        else put1(s, 'P');
    }
}

/* Emit one line (without its newline). */
static void gen_line(sink_t *s, const synth_params *p, uint64_t line)
{
    rng_t r;
    rng_for_line(&r, p->seed, line);
    int long_line = p->p_long16 ? chance(&r, p->p_long16) : 0;
    int32_t target = long_line
        ? p->long_lo + (int32_t)below(&r, (uint32_t)(p->long_hi - p->long_lo + 1))
        : normal_len(&r, p->len_mean_milli, p->len_sd_milli, p->len_lo, p->len_hi);
    size_t start = s->len;

    ring_t rings[MAX_OPEN];
    int nrings = 0;
    int max_open = long_line ? 8 : 3;
    int depth = 0;
    int atoms_in_branch[5] = {0, 0, 0, 0, 0};
    int atom_ordinal = 0;

    for (;;) {
        /* one atom step: optional bond, atom, ring closures, ring opening */
        int aromatic_ctx = 0;
        for (int k = 0; k < nrings; ++k) aromatic_ctx |= rings[k].aromatic;
        if (atom_ordinal > 0) {
            if (long_line && chance(&r, P16(0.06))) put1(s, chance(&r, P16(0.5)) ? '/' : '\\');
            else if (chance(&r, P16(0.07))) put1(s, '=');
            else if (chance(&r, P16(0.01))) put1(s, '#');
        }
        put_atom(s, &r, aromatic_ctx, long_line);
        ++atom_ordinal;
        atoms_in_branch[depth] += 1;

        /* labels closing at this atom are not reusable for an opening at the same atom */
        int used[100];
        memset(used, 0, sizeof used);
        for (int k = 0; k < nrings; ++k) used[rings[k].label] = 1;
        for (int k = 0; k < nrings;) {
            if (--rings[k].countdown <= 0) {
                put_label(s, rings[k].label);
                rings[k] = rings[--nrings];
            } else {
                ++k;
            }
        }
        if (nrings < max_open && chance(&r, long_line ? P16(0.16) : P16(0.13))) {
            int lo = 1, hi = 9;
            if (long_line && chance(&r, P16(0.30))) { lo = 10; hi = 99; }
            int free_labels[99], nfree = 0;
            for (int l = lo; l <= hi; ++l)
                if (!used[l]) free_labels[nfree++] = l;
            if (nfree > 0) {
                ring_t g;
                g.label = free_labels[below(&r, (uint32_t)nfree)];
                g.countdown = 3 + (int)below(&r, 5);
                g.aromatic = chance(&r, long_line ? P16(0.5) : P16(0.6));
                g.opened_at = atom_ordinal;
                rings[nrings++] = g;
                put_label(s, g.label);
            }
        }

        if ((int32_t)(s->len - start) >= target || s->overflow) break;

        /* branch structure between atoms */
        if (depth > 0 && atoms_in_branch[depth] >= 1 && chance(&r, P16(0.22))) {
            put1(s, ')');
            --depth;
            if (depth > 0 && atoms_in_branch[depth] >= 1 && chance(&r, P16(0.15))) {
                put1(s, ')');
                --depth;
            }
        }
        if (depth < 4 && chance(&r, P16(0.16))) {
            put1(s, '(');
            ++depth;
            atoms_in_branch[depth] = 0;
        }
    }

    /* close open rings on a fresh atom (a ring cannot close on the atom that opened it) */
    if (nrings > 0) {
        int need_atom = 0;
        for (int k = 0; k < nrings; ++k) need_atom |= (rings[k].opened_at == atom_ordinal);
        if (need_atom) {
            put1(s, rings[0].aromatic ? 'c' : 'C');
            ++atom_ordinal;
        }
        for (int k = 0; k < nrings; ++k) put_label(s, rings[k].label);
    }
    while (depth > 0) {
        put1(s, ')');
        --depth;
    }
}

/* Lines [first, first + count) into out, each followed by '\n'. Returns bytes written, or
 * (size_t)-1 if cap is too small. */
size_t synth_lines(const synth_params *p, uint64_t first, uint64_t count, uint8_t *out, size_t cap)
{
    sink_t s = {out, 0, cap, 0};
    for (uint64_t i = 0; i < count; ++i) {
        gen_line(&s, p, first + i);
        put1(&s, '\n');
        if (s.overflow) return (size_t)-1;
    }
    return s.len;
}

/* Byte count of lines [first, first + count) without storing them. */
static size_t synth_count(const synth_params *p, uint64_t first, uint64_t count)
{
    uint8_t line[4096];
    size_t total = 0;
    for (uint64_t i = 0; i < count; ++i) {
        sink_t s = {line, 0, sizeof line, 0};
        gen_line(&s, p, first + i);
        total += s.len + 1;
    }
    return total;
}

typedef struct {
    const synth_params *p;
    uint64_t first, count;
    uint8_t *out;
    size_t cap, result;
} job_t;

static void *count_job(void *a)
{
    job_t *j = (job_t *)a;
    j->result = synth_count(j->p, j->first, j->count);
    return NULL;
}

static void *fill_job(void *a)
{
    job_t *j = (job_t *)a;
    j->result = synth_lines(j->p, j->first, j->count, j->out, j->cap);
    return NULL;
}

#define MAX_THREADS 256

/* Two passes over `nthreads` line ranges: count the bytes of each range, then, if `out` is not NULL
 * and cap suffices, write every range at its offset. Returns the total byte count (or (size_t)-1 if
 * cap is too small). With out == NULL only the size is computed. */
size_t synth_lines_mt(const synth_params *p, uint64_t first, uint64_t count, int nthreads,
                      uint8_t *out, size_t cap)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > MAX_THREADS) nthreads = MAX_THREADS;
    if ((uint64_t)nthreads > count) nthreads = count ? (int)count : 1;
    job_t jobs[MAX_THREADS];
    pthread_t th[MAX_THREADS];
    uint64_t per = count / (uint64_t)nthreads, extra = count % (uint64_t)nthreads, at = first;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].p = p;
        jobs[t].first = at;
        jobs[t].count = per + ((uint64_t)t < extra ? 1 : 0);
        at += jobs[t].count;
    }
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, count_job, &jobs[t]);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    size_t total = 0;
    for (int t = 0; t < nthreads; ++t) total += jobs[t].result;
    if (out == NULL) return total;
    if (total > cap) return (size_t)-1;
    size_t off = 0;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].out = out + off;
        jobs[t].cap = jobs[t].result;
        off += jobs[t].result;
    }
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, fill_job, &jobs[t]);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    for (int t = 0; t < nthreads; ++t)
        if (jobs[t].result != jobs[t].cap) return (size_t)-1;
    return total;
}

/* Uniform draws for host-side workload shaping (shard sizes, request streams): `n` values in
 * [0, 2^32) from stream (seed, index0 + k). */
void synth_u32(uint64_t seed, uint64_t index0, uint64_t n, uint32_t *out)
{
    for (uint64_t k = 0; k < n; ++k) {
        rng_t r;
        rng_for_line(&r, seed ^ 0x5DEECE66DULL, index0 + k);
        out[k] = pcg32_next(&r);
    }
}
