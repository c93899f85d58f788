/*
 * zsmiles.h - C ABI of the GB300 ZSMILES codec (libzsmiles.so).
 *
 * ZSMILES (arXiv 2404.19391) stores SMILES libraries one molecule per line. Each line is optionally
 * pre-processed (ring-ID renumbering, Sec. IV-A), then encoded against one fixed, input-independent
 * dictionary D (Sec. I, IV-B, IV-C) by the parse of minimum output length (a shortest path where a
 * dictionary match costs 1 byte and an escaped character 2, Sec. IV-D1). Decoding replaces each symbol
 * by its pattern and copies the byte after a space verbatim (Sec. IV-D2). The output stays readable and
 * keeps every molecule on its own line, so any line can be cut out and decoded alone (Sec. I).
 *
 * Conventions for every call below:
 *   - Pointers named d_* are DEVICE pointers on the device that was current when the dictionary was
 *     loaded (for calls without a dictionary: the current device). The caller owns every buffer; the
 *     library owns only the zs_dict handle and the scratch it caches per (dictionary, stream) pair.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream). Work is
 *     stream-ordered. Calls that fill a zs_result wait for their own work on `stream` before returning,
 *     so *res is valid on return.
 *   - Streams: a stream is a sequence of lines separated by '\n'. A trailing '\n' does not open an
 *     extra, empty line; whether the last line ends with '\n' is preserved by every call. A line
 *     index has n_lines + 1 uint64 entries: the byte offset where each line starts, then the total
 *     length.
 *   - Errors never abort, trap or print. The return value says what went wrong, zs_last_error()
 *     gives a message. On ZS_ERR_CAPACITY the output buffers may have been partly written and
 *     res->out_len holds the size that would have been needed.
 *   - The library never falls back to a CPU path: without a usable CUDA device every call returns
 *     ZS_ERR_CUDA.
 */
#ifndef ZSMILES_H
#define ZSMILES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct zs_dict zs_dict; /* opaque, library-owned */

typedef enum {
    ZS_OK = 0,
    ZS_ERR_INVALID_ARG = 1, /* NULL where a pointer is required, wrong device, size out of range */
    ZS_ERR_BAD_DICT = 2,    /* dictionary file does not parse (format below) */
    ZS_ERR_CAPACITY = 3,    /* an output buffer is too small; res->out_len / *n_lines say how large */
    ZS_ERR_MALFORMED = 4,   /* compressed input is not a valid ZSMILES stream; see res->err_offset */
    ZS_ERR_CUDA = 5,        /* a CUDA runtime call failed */
    ZS_ERR_TIMEOUT = 6,     /* a device-side wait ran past its limit; the call's output is invalid */
    ZS_ERR_OOM = 7          /* the library could not allocate its scratch */
} zs_status;

/* zs_compress flags */
enum {
    ZS_PREPROCESS = 1u,      /* renumber ring IDs before encoding (Sec. IV-A); "optionally", Sec. IV-D */
    ZS_PREPROCESS_OUTER = 2u /* with ZS_PREPROCESS only: the other reading of Sec. IV-A, kept as an
                              * experiment - rings are labelled in the order they open, each with the
                              * smallest ID held by no ring open at that point (the outermost of a nest
                              * then gets the lower ID). Alone it is ZS_ERR_INVALID_ARG. */
};

typedef struct {
    uint64_t out_len;    /* bytes written to the output (or needed, on ZS_ERR_CAPACITY) */
    uint64_t n_lines;    /* lines (compress/decompress) or requests (decompress_lines) processed */
    uint64_t err_offset; /* ZS_ERR_MALFORMED: offset of the first bad byte, or index of the bad request */
} zs_result;

/*
 * zs_load_dictionary - parse a dictionary file and build its device tables.
 *
 * D maps a symbol byte to a pattern (Sec. IV: "a dictionary that associates a common string pattern to
 * an ASCII character"); it is fixed and input-independent (Sec. I), pre-populated with single
 * characters (Sec. IV-B) and filled with learned patterns by Algorithm 1 (Sec. IV-C). The paper compiles
 * D into its executable (Sec. IV-D); here it is loaded at run time from this text format:
 *
 *     ZSDICT 1
 *     <lmin> <lmax> <T>
 *     alphabet <hex of the pre-populated characters, or ->
 *     T lines of: <symbol as 2 hex digits> <pattern as hex>
 *
 * Each alphabet character c is the entry c -> "c". Symbols and patterns must be unique, may not hold
 * '\n' or ' ' (the line separator and the escape), and patterns are 1..lmax bytes, lmax <= 16.
 *
 * file_bytes: host memory, len bytes, read during the call only. *out: receives a handle owned by the
 * caller until zs_free_dictionary. The device tables live on the current device. Returns ZS_OK,
 * ZS_ERR_INVALID_ARG, ZS_ERR_BAD_DICT, ZS_ERR_CUDA or ZS_ERR_OOM.
 */
zs_status zs_load_dictionary(const uint8_t *file_bytes, size_t len, zs_dict **out);

/* Releases the handle, its device tables and every scratch buffer cached for it. The caller must not
 * have work in flight that uses the handle. NULL is ignored. */
void zs_free_dictionary(zs_dict *d);

/* 1 if zs_compress with this dictionary runs the parse-transducer kernel on the current device (the
 * shortest-path scan of Sec. IV-D1 compiled into one table lookup per byte, built at load time), 0 if it
 * runs the generic kernel (automaton walk plus window scan per byte) because the transducer's state space
 * or table does not fit. Both produce identical output. (Informational; the paper has no counterpart.) */
int zs_dictionary_uses_transducer(const zs_dict *d);

/* Longest pattern of D (the most bytes one symbol can expand to). */
int zs_dictionary_lmax(const zs_dict *d);

/* Output capacity that always suffices for zs_compress of in_len bytes: 3 * in_len + 16. Escaping
 * doubles a byte (Sec. IV-B) and renumbering can turn a 1-byte ring label into a 3-byte %nn label. */
size_t zs_compress_bound(size_t in_len);

/* Output capacity that always suffices for zs_decompress of in_len bytes under d: lmax * in_len. */
size_t zs_decompress_bound(const zs_dict *d, size_t in_len);

/*
 * zs_compress - encode every line of a stream (Sec. IV-D1).
 *
 * Per line: if flags has ZS_PREPROCESS, renumber ring IDs (Sec. IV-A: IDs restart at 0, are reused once
 * a ring closes, and among overlapping rings the one that closes first - the innermost - gets the lower
 * ID; only the first space/tab-free field is touched; a line with an unclosed ring or bracket, a bad %
 * label, or one needing an ID above 99 is left as is). ZS_PREPROCESS | ZS_PREPROCESS_OUTER labels the
 * rings in opening order instead (see the flag). Then write the minimum-length sequence of
 * dictionary symbols (cost 1) and escapes (' ' + raw byte, cost 2) that spells the line (Sec. IV-D1);
 * among equally short encodings the one taking the longest piece at each step, front to back. Each
 * output line ends with '\n' exactly when its input line did.
 *
 * d_in:  device, in_len bytes (any alignment; 16-byte alignment is faster).
 * d_out: device, out_cap bytes; zs_compress_bound(in_len) always suffices.
 * d_line_index: device, nullable; if given, receives n_lines + 1 offsets into d_out (index_cap entries
 *        available; ZS_ERR_CAPACITY if fewer are needed than given).
 * res:   host; out_len = compressed bytes, n_lines = lines.
 * Returns ZS_OK, ZS_ERR_INVALID_ARG, ZS_ERR_CAPACITY, ZS_ERR_CUDA, ZS_ERR_TIMEOUT or ZS_ERR_OOM.
 */
zs_status zs_compress(const zs_dict *d, const uint8_t *d_in, size_t in_len, unsigned flags, uint8_t *d_out,
                      size_t out_cap, uint64_t *d_line_index, size_t index_cap, zs_result *res, void *stream);

/*
 * zs_decompress - decode every line of a compressed stream (Sec. IV-D2).
 *
 * Each byte b of a line: ' ' -> output the next byte verbatim (escape); any other b -> output D[b].
 * '\n' separates lines and is copied. An undefined symbol, or a line ending in an unpaired ' ', is
 * ZS_ERR_MALFORMED with res->err_offset = offset of the first bad byte in d_in.
 *
 * d_in: device, in_len bytes. d_out: device, out_cap bytes (zs_decompress_bound suffices).
 * res: host; out_len = decoded bytes, n_lines = lines.
 * Returns ZS_OK, ZS_ERR_INVALID_ARG, ZS_ERR_CAPACITY, ZS_ERR_MALFORMED, ZS_ERR_CUDA, ZS_ERR_TIMEOUT, ZS_ERR_OOM.
 */
zs_status zs_decompress(const zs_dict *d, const uint8_t *d_in, size_t in_len, uint8_t *d_out, size_t out_cap,
                        zs_result *res, void *stream);

/*
 * zs_build_line_index - line-start offsets of any '\n'-separated stream (Sec. I: every molecule keeps
 * its own line, which is what makes random access possible).
 *
 * d_in: device, in_len bytes. d_index: device, index_cap uint64 entries; receives n_lines + 1 offsets.
 * *n_lines: host, receives the line count (also on ZS_ERR_CAPACITY, so the caller can size d_index).
 * Returns ZS_OK, ZS_ERR_INVALID_ARG, ZS_ERR_CAPACITY, ZS_ERR_CUDA, ZS_ERR_TIMEOUT or ZS_ERR_OOM.
 */
zs_status zs_build_line_index(const uint8_t *d_in, size_t in_len, uint64_t *d_index, size_t index_cap,
                              size_t *n_lines, void *stream);

/*
 * zs_decompress_lines - random access: decode the requested lines of a compressed stream (Sec. I:
 * "random access" = lines keep their order and stay separable, so one line can be decoded alone with
 * the shared dictionary).
 *
 * d_comp, comp_len: device, the compressed stream. d_index: device, its n_lines + 1 line offsets (from
 * zs_compress or zs_build_line_index). d_ids: device, k line numbers, any order, repeats allowed.
 * d_out: device, out_cap bytes; receives the decoded lines in request order, each followed by '\n'.
 * d_out_off: device, k + 1 entries; the offset of each decoded line in d_out, then the total.
 * res: host; out_len = total bytes, n_lines = k. An id >= n_lines, or a malformed line, is
 * ZS_ERR_MALFORMED with res->err_offset = the position of the first bad request in d_ids.
 * Returns ZS_OK, ZS_ERR_INVALID_ARG, ZS_ERR_CAPACITY, ZS_ERR_MALFORMED, ZS_ERR_CUDA, ZS_ERR_TIMEOUT, ZS_ERR_OOM.
 */
zs_status zs_decompress_lines(const zs_dict *d, const uint8_t *d_comp, size_t comp_len, const uint64_t *d_index,
                              size_t n_lines, const uint64_t *d_ids, size_t k, uint8_t *d_out, size_t out_cap,
                              uint64_t *d_out_off, zs_result *res, void *stream);

/*
 * zs_decompress_noalloc - zs_decompress for callers that cannot allocate. (The paper has no counterpart:
 * this concerns how the library obtains memory, not what it computes.)
 *
 * Some callers cannot let a library allocate memory: their device memory is entirely reserved by another
 * allocator (a framework's caching allocator that already holds the free HBM, a fixed arena in an
 * embedded service), or they run latency-critical loops in which cudaMalloc, cudaFree or cudaMallocHost
 * would implicitly synchronise the device. This call decodes exactly like zs_decompress (same
 * arguments, same output, same errors) but allocates nothing: its scratch is a fixed 8 MiB array of
 * device memory compiled into the library, which every GPU that loads the library holds until the
 * process exits, and its result is copied straight into *res.
 *
 * Limit: the scratch holds 262,142 tile records of 2,048 bytes of compressed input each, so in_len may be
 * at most 536,866,816 bytes (zs_decompress_noalloc_limit() returns this figure); a larger input returns
 * ZS_ERR_INVALID_ARG without touching the device (use zs_decompress instead).
 *
 * Set-up: every call looks up the array's device address on the current device (cudaGetSymbolAddress),
 * so nothing is cached across a cudaDeviceReset. The call clears the scratch it uses, launches the
 * decoder, copies the result record to host memory and waits for its stream before returning.
 * Concurrency: every call shares the one array, and the call clears what must start at zero. Calls whose
 * work overlaps on the GPU (from several host threads or streams at once) race on the array: the caller
 * must serialise them.
 */
zs_status zs_decompress_noalloc(const zs_dict *d, const uint8_t *d_in, size_t in_len, uint8_t *d_out,
                                size_t out_cap, zs_result *res, void *stream);

/* The largest in_len that zs_decompress_noalloc accepts, in bytes. Host-only; never fails. */
size_t zs_decompress_noalloc_limit(void);

/* ---- Batched form: many shards, one persistent launch, CUDA graph replay ---------------------------
 *
 * Library files are often split into many shards of very uneven sizes (the paper's method works line
 * by line, Sec. IV, so shards are independent). These calls run the compression (or decompression) of
 * a whole set of shards as ONE launch of the persistent kernel: the warps claim fixed-size tiles from a
 * launch-wide numbering that runs through all shards, and each shard's output offsets come from its own
 * look-back chain, so every shard gets exactly the bytes (and line index) that zs_compress /
 * zs_decompress give it alone. The batching itself is not in the paper.
 */

/* One shard. Device pointers; the caller owns every buffer. For compression, in is the SMILES text,
 * out receives the compressed stream (capacity zs_compress_bound(in_len) always suffices) and
 * line_index (nullable, index_cap entries) the line index. For decompression, in is a compressed stream,
 * out receives the decoded text (zs_decompress_bound), and line_index must be NULL with index_cap 0. */
typedef struct zs_shard {
    const uint8_t *in;
    size_t in_len;
    uint8_t *out;
    size_t out_cap;
    uint64_t *line_index;
    size_t index_cap;
} zs_shard;

typedef enum { ZS_OP_COMPRESS = 0, ZS_OP_DECOMPRESS = 1 } zs_op;

enum { ZS_MAX_SHARDS = 1 << 20 };

/* Kernel variants: each operation is compiled for a few tile geometries (warps per SM x input bytes per
 * warp tile; for compression this sets how many lines a warp holds at once). All give identical
 * output; their speed depends on the line-length mix. */
int zs_kernel_variants(zs_op op);                     /* number of compiled variants (0 for a bad op) */
const char *zs_kernel_variant_name(zs_op op, int v);  /* static string, or NULL */

/* One-shot batched calls: one launch of the default variant over all shards, then a wait. flags: as for
 * zs_compress (here and in zs_plan_create; not used by decompression). res: host
 * array of n_shards results (out_len, n_lines and err_offset of each shard). Errors: as for
 * zs_compress / zs_decompress; the first failing shard is named in zs_last_error(), and every shard's
 * res entry is filled. A dictionary whose transducer does not fit in shared memory (see
 * zs_dictionary_uses_transducer) cannot be used here: ZS_ERR_BAD_DICT. */
zs_status zs_compress_batch(const zs_dict *d, const zs_shard *shards, size_t n_shards, unsigned flags,
                            zs_result *res, void *stream);
zs_status zs_decompress_batch(const zs_dict *d, const zs_shard *shards, size_t n_shards, zs_result *res,
                              void *stream);

/* Plans: a fixed set of shards run many times (new data in the same buffers). */
typedef struct zs_plan zs_plan; /* opaque, library-owned */

typedef struct zs_plan_options {
    int variant;    /* -1: autotune (time every variant on this batch, keep the fastest); else a variant */
    int use_graph;  /* nonzero: capture clear + launch + result copy in a CUDA graph, replay it per run */
    int tune_reps;  /* timed runs per variant when autotuning (<= 0: 3) */
    int cut_min;    /* span geometries, fixed variant: shortest line cut between lanes (0: the geometry's
                       default; < 0: never). Autotuning times the default and its opposite and keeps the faster */
    int tune_cache; /* nonzero: an autotuned plan first looks up, then records, its choice (variant, cut) under
                       (GPU model, dictionary digest, operation, flags, log2 of the batch bytes, shard count and
                       largest shard); the cache lives in the process, and in the file ZS_TUNE_CACHE names */
} zs_plan_options;

/* Makes a plan for `op` over the shards (host array, copied). opt may be NULL: autotune, with a graph.
 * Autotuning RUNS the operation on the shards (writing their outputs) a few times per variant, on a
 * private stream, and waits for it. Allocates the plan's device scratch (results, shard table, tile
 * records, long-line work space) and pinned host memory. */
zs_status zs_plan_create(const zs_dict *d, zs_op op, unsigned flags, const zs_shard *shards, size_t n_shards,
                         const zs_plan_options *opt, zs_plan **out);
/* Runs the plan on `stream` and waits for it; res (host, n_shards entries, nullable) as above. Calls on
 * one plan must not overlap (the plan's scratch is reused). */
zs_status zs_plan_run(zs_plan *p, zs_result *res, void *stream);
int zs_plan_variant(const zs_plan *p);             /* the variant the plan runs */
int zs_plan_cut_min(const zs_plan *p);             /* its span cut threshold in bytes (0: no cuts) */
double zs_plan_tuned_ms(const zs_plan *p, int v);  /* median kernel ms of variant v when tuned, else -1 */
double zs_plan_last_ms(const zs_plan *p);          /* kernel ms of the last run */
void zs_plan_destroy(zs_plan *p);

/* ---- Dictionary generation (Algorithm 1, Eq. 1; Sec. IV-B, IV-C) -------------------------------------
 *
 * Trains a dictionary on a device training stream ('\n'-separated lines; no zero bytes) and writes the
 * .zsd file text to `out` (host, out_cap bytes; *out_len receives its size, also on ZS_ERR_CAPACITY).
 *
 * Steps:
 *   - with ZS_PREPROCESS, the lines are ring-ID pre-processed first (Sec. IV-A), in opening order if
 *     ZS_PREPROCESS_OUTER is set too;
 *   - every substring of lmin..lmax bytes that holds no ' ' and no '\n' is counted on the GPU, overlapping
 *     occurrences included;
 *   - then T patterns are picked greedily by occ * (len - overlap) (Eq. 1), where overlap is the largest
 *     overlap with a pattern already picked: |p| if p lies inside it, its length if it lies inside p, else
 *     the longest suffix/prefix overlap either way;
 *   - ties go to the higher count, then the longer pattern, then the bytewise smaller one; selection stops
 *     once the best rank is <= 0.
 *
 * Symbols: the pre-populated SMILES alphabet (unless no_alphabet) maps each of its characters to itself;
 * picks take the free printable bytes 0x21-0x7E, then 0xA1-0xFF, in pick order. Patterns are at most 8
 * bytes here. Not in the paper: how overlap, ties and the symbol bytes are chosen (readings of Sec. IV-C).
 */
typedef struct zs_train_options {
    int lmin;        /* shortest pattern (0: 2) */
    int lmax;        /* longest pattern, <= 8 (0: 8) */
    int T;           /* patterns to pick (0 or more than the free symbol bytes: all free symbol bytes) */
    int no_alphabet; /* nonzero: no pre-populated alphabet */
} zs_train_options;

zs_status zs_train_dictionary(const uint8_t *d_train, size_t n, unsigned flags, const zs_train_options *opt,
                              uint8_t *out, size_t out_cap, size_t *out_len, void *stream);

/* ---- Host-to-host pipelines ------------------------------------------------------------------------
 *
 * zs_compress / zs_decompress take device buffers. These take HOST buffers and hide the copies: the stream
 * is cut into chunks at line ends (lines are independent, Sec. I, so the chunks' outputs concatenated are
 * the output of the whole stream), and up to n_streams chunks are in flight at once, each on its own
 * stream: host-to-device copy, kernel, then its output and line index copied to their place in the
 * caller's buffers. Copies in both directions overlap the kernels of other chunks. Output, line index,
 * errors and capacities are exactly those of zs_compress / zs_decompress on the same bytes. The buffers
 * should be page-locked (cudaMallocHost / cudaHostRegister) for the copies to overlap; pageable memory
 * works but serialises them. Calls on one dictionary run one at a time (the pipeline's device buffers
 * belong to the dictionary and are kept for the next call). A line longer than chunk_bytes returns
 * ZS_ERR_CAPACITY (raise chunk_bytes). Not in the paper.
 */
typedef struct zs_pipeline_options {
    size_t chunk_bytes; /* input bytes per chunk (0: 32 MiB; at least 4 KiB) */
    int n_streams;      /* chunks in flight (0: 4; at most 16) */
} zs_pipeline_options;

zs_status zs_compress_host(const zs_dict *d, const uint8_t *h_in, size_t in_len, unsigned flags, uint8_t *h_out,
                           size_t out_cap, uint64_t *h_line_index, size_t index_cap, zs_result *res,
                           const zs_pipeline_options *opt);
zs_status zs_decompress_host(const zs_dict *d, const uint8_t *h_in, size_t in_len, uint8_t *h_out, size_t out_cap,
                             zs_result *res, const zs_pipeline_options *opt);

/* ---- Serving form: continuous batching of random-access requests over a resident store -----------
 *
 * A server keeps a compressed store and its line index resident in device memory (the caller's
 * buffers, which must outlive the server) and answers requests for sets of line ids (random access,
 * Sec. I). Requests queue in arrival order. A scheduler thread admits the queue head as soon as one of
 * max_inflight slots is free and the output arenas have room for it: every queued request that fits
 * joins that launch (continuous batching), so requests arriving while others are on the GPU ride the
 * next launch, and up to max_inflight launches (each with its own stream) overlap. Admission reserves
 * an upper bound of the request's decoded size (k ids times the store's longest decoded line, measured
 * on the GPU when the server is made) in a device arena and in a pinned host arena; the host bytes
 * stay reserved until the result is fetched or released. A request's result is exactly what
 * zs_decompress_lines gives for its ids alone. The batching is not in the paper.
 */
typedef struct zs_server zs_server; /* opaque, library-owned */

typedef struct zs_server_options {
    size_t arena_bytes;   /* device arena and pinned host arena, bytes each (0: 512 MiB) */
    size_t max_batch_ids; /* ids per launch, and the largest request (0: 1,048,576) */
    int max_inflight;     /* launches on the GPU at once (0: 4) */
} zs_server_options;

typedef struct zs_server_stats {
    uint64_t submitted, completed, batches, ids;
    double mean_batch_requests; /* requests per launch */
    int max_inflight;           /* most launches seen in flight at once */
    double p50_ms, p99_ms;      /* submit-to-result latency of completed requests */
} zs_server_stats;

/* d_comp/comp_len: the compressed store; d_index: its line index (n_lines + 1 entries, as written by
 * zs_compress or zs_build_line_index). One GPU pass over the store checks that every line decodes
 * (else ZS_ERR_MALFORMED) and finds the longest decoded line. opt may be NULL. Starts the scheduler
 * thread. */
zs_status zs_server_create(const zs_dict *d, const uint8_t *d_comp, size_t comp_len, const uint64_t *d_index,
                           size_t n_lines, const zs_server_options *opt, zs_server **out);
/* Queues a request for the k line ids in ids (host array, copied); returns at once with a ticket.
 * Thread-safe. ZS_ERR_INVALID_ARG for an id >= n_lines or k > max_batch_ids; ZS_ERR_CAPACITY when the
 * request's bound exceeds the arena. */
zs_status zs_server_submit(zs_server *s, const uint64_t *ids, size_t k, uint64_t *ticket);
/* Waits (timeout_s < 0: without limit) until the request is done; res->out_len = its decoded bytes,
 * res->n_lines = k. ZS_ERR_TIMEOUT if the time ran out (the request stays queued). */
zs_status zs_server_wait(zs_server *s, uint64_t ticket, double timeout_s, zs_result *res);
/* Copies a finished request's lines (out: out_cap bytes; off: k + 1 host offsets, nullable) and
 * forgets the ticket. */
zs_status zs_server_fetch(zs_server *s, uint64_t ticket, uint8_t *out, size_t out_cap, uint64_t *off);
/* Forgets a finished request without copying it. */
zs_status zs_server_release(zs_server *s, uint64_t ticket);
zs_status zs_server_get_stats(zs_server *s, zs_server_stats *st);
/* Stops the scheduler (queued requests fail, launches in flight finish) and frees everything. */
void zs_server_destroy(zs_server *s);

/* Open-loop load replay. Request r (k[r] ids, consecutive in ids) is submitted at arrival_s[r] seconds
 * after the call starts (non-decreasing), whether or not earlier ones are done; latency_ms[r] runs
 * from that scheduled arrival to the request's completion; *makespan_s (nullable) from the start to
 * the last completion. Results are released, not returned. */
zs_status zs_server_replay(zs_server *s, const double *arrival_s, const uint64_t *ids, const size_t *k,
                           size_t n_req, double *latency_ms, double *makespan_s);
/* The same replay served one request at a time, in arrival order, each by its own random-access launch
 * with a wait and the copy of its bytes to the host (decompress-per-request, the unbatched baseline). */
zs_status zs_serial_replay(const zs_dict *d, const uint8_t *d_comp, size_t comp_len, const uint64_t *d_index,
                           size_t n_lines, const double *arrival_s, const uint64_t *ids, const size_t *k,
                           size_t n_req, double *latency_ms, double *makespan_s, void *stream);

/* Device time, in milliseconds, of the main kernel of the last successful zs_compress, zs_decompress,
 * zs_build_line_index or zs_decompress_lines on this thread, measured with CUDA events recorded on the
 * call's stream just before and just after the kernel launch (no paper counterpart: instrumentation). */
double zs_last_kernel_ms(void);

/* Message for the last failing call on this thread ("" if none). Valid until the next call. */
const char *zs_last_error(void);

/* Library version string. */
const char *zs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ZSMILES_H */
