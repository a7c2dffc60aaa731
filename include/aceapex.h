/*
 * aceapex.h -- C ABI of the GB300 ACEAPEX stream decoder (libaceapex.so).
 *
 * ACEAPEX is an LZ77 format whose back-references are absolute positions in the decoded output and whose
 * output is cut into self-contained blocks of B bytes (paper §3.1); each block carries four arrays:
 * literal bytes, match lengths, absolute offsets and the command sequence of literal-run lengths (§3.2).
 * The byte layout is the ACEAPEX stream format, fixed once for this library.  Decoding places every
 * sequence with a prefix sum, scatters the literals and runs the match copies in dependency order (§7.1);
 * a stream whose matches all read literal bytes (chain flattening, §3.3) decodes in one pass.
 *
 * Conventions for every call:
 *   - pointers named d_* and the comp/out arguments of the decode calls are DEVICE pointers owned by the
 *     caller; pointers named h_* are HOST pointers owned by the caller; the library never frees them;
 *   - `stream` is a cudaStream_t (passed as void*); work is enqueued on it in order;
 *   - return values are aceapex_status codes (0 = OK, negative = error); no C++ exception crosses the ABI;
 *   - malformed input never faults the GPU: every device load and store is bounds-checked and a violation
 *     becomes a status code;
 *   - calls on one context are serialised by an internal lock; use one stream per concurrent decode.
 */
#ifndef ACEAPEX_H
#define ACEAPEX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ACEAPEX_OK = 0,
    ACEAPEX_ERR_ARG = -1,     /* null pointer, misaligned comp (needs 16 B), bad size argument */
    ACEAPEX_ERR_FORMAT = -2,  /* bad magic/version/flags/fields, block index, header counts, varint, sync table */
    ACEAPEX_ERR_SIZE = -3,    /* out_len differs from the decoded size, comp_len differs from the header */
    ACEAPEX_ERR_OFFSET = -4,  /* a match source not before its destination, or a sequence leaving its block */
    ACEAPEX_ERR_TIMEOUT = -5, /* a bounded device wait expired (the result is unusable, the context is fine) */
    ACEAPEX_ERR_CUDA = -6,    /* a CUDA runtime call failed */
    ACEAPEX_ERR_NOMEM = -7,   /* workspace allocation failed, or the caller's workspace is too small */
    ACEAPEX_ERR_DEPTH = -8    /* the stream's max_depth is smaller than the depth of one of its matches */
} aceapex_status;

/* Header fields of a stream (stream format §1.1). */
typedef struct {
    uint64_t decoded_len;   /* N */
    uint64_t n_blocks;      /* ceil(N / B) */
    uint64_t comp_len;      /* total stream bytes */
    uint64_t n_match;       /* matches over all blocks */
    uint64_t n_seq;         /* sequences over all blocks */
    uint64_t n_tiles;       /* sync-point tiles over all blocks */
    uint32_t block_log2;    /* B = 2^block_log2 */
    uint32_t tile_log2;     /* T = 2^tile_log2 */
    uint32_t min_match;
    uint32_t flatten;       /* 0 none, 1 within-block, 2 global (§3.3) */
    uint32_t depth_cap;     /* 0 = none (§7.4) */
    uint32_t max_depth;     /* largest match depth; <= 1 selects the one-pass decode */
} aceapex_info;

/* Statistics of the last decode on this context (aceapex_get_stats). */
#define ACEAPEX_HIST_MAX 4096
typedef struct {
    uint64_t decoded_len, comp_len, n_match, n_tiles;
    uint32_t max_depth;         /* largest match depth of the stream */
    uint32_t one_pass;          /* 1 when the one-pass (flattened) path ran */
    uint32_t n_levels;          /* depth levels executed by the wavefront (0 on the one-pass path) */
    uint32_t hist_len;          /* valid entries of level_hist */
    uint64_t level_hist[ACEAPEX_HIST_MAX]; /* level_hist[k] = matches of depth k (k >= 1), clipped */
    /* with aceapex_profile(1), one-pass path only: SM cycles summed over CTAs spent in each tile phase --
     * open, parse, literals, store + publish, wait, matches, store -- and [7] = tiles processed */
    uint64_t phase_cycles[8];
} aceapex_stats;

/* Host-side header parse (paper §3.1: the stream is a sequence of self-contained blocks; the header gives
 * their size and count, and the depth information of §7.1 that picks the decode schedule).  host_prefix
 * holds at least the first 64 bytes of the stream.  Checks magic, version, flags and field ranges (stream
 * format §1.1); returns ACEAPEX_ERR_FORMAT / ACEAPEX_ERR_SIZE on a bad header, ACEAPEX_ERR_ARG on null. */
int aceapex_peek_header(const void *host_prefix, size_t len, aceapex_info *info);

/* Device workspace bytes needed by aceapex_decode_async for this stream. */
size_t aceapex_workspace_size(const aceapex_info *info);

/*
 * Decode one stream (blocking) -- the operation of paper §3.1-§3.2: every sequence of every block is placed
 * by a prefix sum of its literal-run and match lengths, its literal run is copied from lit[], and each
 * match copies bytes from an absolute position of the output ("copy N bytes from position P"), matches of
 * increasing dependency depth after the ones they read (§7.1).  comp: device bytes of the stream, 16-byte
 * aligned, comp_len bytes.
 * out: device buffer of out_len bytes, which must equal the header's decoded length.  Reads the 64-byte
 * header back to the host, takes workspace from a cached pool, enqueues the decode on `stream`,
 * synchronises `stream` and returns the device status.
 */
int aceapex_decode(const void *comp, size_t comp_len, void *out, size_t out_len, void *stream);

/*
 * Decode one stream without any host synchronisation (the same operation as aceapex_decode, paper §3.1-§3.2,
 * §7.1; the caller supplies the workspace and receives the status on the device).  info: from
 * aceapex_peek_header on a host copy of
 * the header.  d_ws: caller-owned device workspace of at least aceapex_workspace_size(info) bytes,
 * zero-filled before its first use (it may then be reused without clearing by calls that do not
 * overlap in time).  d_status: device int32 that receives the status.  Returns an argument error at
 * once; device-side errors go to *d_status.
 */
int aceapex_decode_async(const void *comp, size_t comp_len, void *out, size_t out_len, const aceapex_info *info,
                         void *d_ws, size_t ws_len, int32_t *d_status, void *stream);

/*
 * Decode one stream without allocating anything (the paper has no counterpart: this serves callers that
 * cannot allocate device memory while decoding -- a process whose memory was budgeted up front, real-time
 * code, or a library that must not use the application's allocator).  Same arguments as
 * aceapex_decode_async minus the workspace: the scratch is a 16 MiB array in the library's static device
 * memory, which every GPU that loads the library holds until the process exits.  It holds a flag per tile
 * and the literal bitmap (one bit per output byte), so only streams whose matches all have depth <= 1
 * (chain-flattened), with tiles of at most 4 KiB and flags plus bitmap within 16 MiB (about 127 MiB of
 * output at 4 KiB tiles), fit: anything else returns ACEAPEX_ERR_NOMEM at once.  The
 * first call on a device looks up the array's device address (cudaGetSymbolAddress); make that first
 * call before any stream capture.  Every call on a device shares the one array: calls that overlap on the
 * GPU race and must not be issued (serialise them on one stream).  Enqueued on `stream`, no host
 * synchronisation; the status goes to *d_status.
 */
int aceapex_decode_noalloc(const void *comp, size_t comp_len, void *out, size_t out_len, const aceapex_info *info,
                           int32_t *d_status, void *stream);

/*
 * Decode a stream held in HOST memory into a host buffer (blocking; §3.1 blocks, §7.1 decode).
 * h_comp: comp_len bytes of an ACEAPEX stream in host memory; h_out: out_len = decoded length bytes of host
 * memory; both are the caller's and are only read / written during the call.  The library copies the
 * stream to device memory it owns (kept for later calls, grown on demand), decodes, and copies the output
 * back.  Streams the one-pass kernel takes are cut into up to 16 slices of whole blocks: a slice's stream
 * bytes are copied in, its tiles decoded and its output copied out on three CUDA streams, so transfers in
 * both directions overlap the decode.  Deeper streams are copied, decoded whole, and copied back.  With
 * pinned (page-locked) buffers the copies are asynchronous; pageable buffers work but serialise.  Work
 * is ordered after the caller's earlier work on `stream`.  Returns the decode status; ACEAPEX_ERR_ARG for
 * null pointers, ACEAPEX_ERR_SIZE when the lengths disagree with the header, ACEAPEX_ERR_NOMEM when the
 * device buffers cannot be allocated.
 */
int aceapex_decode_host(const void *h_comp, size_t comp_len, void *h_out, size_t out_len, void *stream);

/*
 * Decode n independent streams (blocking) -- paper §7.5: streams have no dependency on each other, so they
 * decode together without any exchange; each stream is decoded as in aceapex_decode (§3.1-§3.2, §7.1).
 * comps/outs: host arrays of n device pointers; comp_lens and
 * out_lens: host arrays; statuses: host array of n int32 that receives each stream's status.  The streams
 * the one-pass kernel takes (see aceapex_set_force_wavefront) are decoded together by one persistent launch
 * over a global tile queue; the others are decoded one after another.  Returns 0 when every stream decoded, else the first
 * failing status.
 */
int aceapex_decode_batch(int n, const void *const *comps, const size_t *comp_lens, void *const *outs,
                         const size_t *out_lens, int32_t *statuses, void *stream);

/*
 * Decode n independent streams held in HOST memory into host buffers (blocking; §7.5 batching of
 * independent streams, each decoded as in aceapex_decode, §3.1-§3.2 and §7.1).  h_comps/h_outs: host
 * arrays of n host pointers (any alignment; pinned memory lets the copies run asynchronously, pageable
 * memory works but serialises); comp_lens/out_lens: host arrays; statuses: host array of n int32 that
 * receives each stream's status (ACEAPEX_ERR_ARG for a null pointer or a stream shorter than its header,
 * ACEAPEX_ERR_SIZE when the lengths disagree with the header, else the decode status).
 * The streams are cut into about 32 groups of consecutive streams.  A group's stream bytes are copied to
 * device memory that the library owns (kept for later calls, grown on demand), its streams are decoded
 * together (one persistent one-pass launch; deeper streams one after another) and its outputs are copied
 * back, on three CUDA streams, so both copy directions overlap the decodes of other groups.  Streams whose
 * host bytes follow each other share one copy: copies in also carry host gaps of up to 64 KiB between
 * streams (read only), copies out join only outputs that are back to back, so no byte outside the outputs
 * is written.  Host buffers are only read / written during the call; work is ordered after the caller's
 * earlier work on `stream`.  Returns 0 when every stream decoded, else the first failing status in stream
 * order; ACEAPEX_ERR_ARG when n < 0 or an array is null (statuses untouched); ACEAPEX_ERR_NOMEM when the
 * device or pinned buffers cannot be allocated.  The call holds the context's lock until it returns.
 */
int aceapex_decode_batch_host(int n, const void *const *h_comps, const size_t *comp_lens, void *const *h_outs,
                              const size_t *out_lens, int32_t *statuses, void *stream);

/*
 * Reusable batch plan (for repeated decodes of the same set of buffers): reads the headers once, builds the
 * device descriptor table and workspace.  plan_launch enqueues the decode; with graph != 0 the launch
 * sequence is captured into a CUDA graph on first use and replayed afterwards.  plan_statuses copies the
 * per-stream statuses to the host (synchronising `stream`).
 */
typedef struct aceapex_batch_plan aceapex_batch_plan;
int aceapex_batch_plan_create(int n, const void *const *comps, const size_t *comp_lens, void *const *outs,
                              const size_t *out_lens, void *stream, aceapex_batch_plan **plan);
int aceapex_batch_plan_launch(aceapex_batch_plan *plan, int graph, void *stream);
int aceapex_batch_plan_statuses(aceapex_batch_plan *plan, int32_t *statuses, void *stream);
/* The same statuses written to the device array d_statuses (n int32), enqueued on `stream` after the
 * plan's launch, with no host synchronization (the device-status form of the batch decode). */
int aceapex_batch_plan_statuses_device(aceapex_batch_plan *plan, int32_t *d_statuses, void *stream);
int aceapex_batch_plan_destroy(aceapex_batch_plan *plan);

/* Launch shape of the one-pass kernel: warps per CTA (2, 4 or 8; default 4) and CTAs per SM (0 = as many as
 * fit, the default).  Applies to later launches on this context.  Returns ACEAPEX_ERR_ARG for another value. */
int aceapex_set_launch_config(int warps_per_cta, int ctas_per_sm);
int aceapex_get_launch_config(int *warps_per_cta, int *ctas_per_sm);

/* Scheduler of streams whose matches are deeper than 1: 1 per-level work queues drained level by level
 * by one persistent cooperative kernel with a bounded grid barrier between levels; 0 dataflow: each
 * match is copied by its thread as soon as every match that wrote its source has published its depth
 * (no level barrier); 2 (default) warp-granular dataflow: a warp takes 32 consecutive matches and copies
 * them in rounds as their writers finish.  All compute the same per-match depths (§7.1) and the same
 * bytes.  Returns ACEAPEX_ERR_ARG for another value. */
int aceapex_set_wave_scheduler(int kind);

/* Decode every stream with the wavefront path, even streams the one-pass kernel would take (for testing
 * and comparison).  Applies to later calls on this context.  The one-pass kernel takes the streams whose
 * max_depth is at most 1, with tiles of at most 4 KiB and at most 0xFFF00000 bytes of output; it checks
 * every source byte against the literal bitmap it builds, so a stream whose depth fields understate its
 * matches' depths ends in ACEAPEX_ERR_DEPTH on either path. */
int aceapex_set_force_wavefront(int on);

/* Limit of every bounded device wait in nanoseconds (0 restores the default of 4 s).  withhold_tile is a
 * test hook: the one-pass kernel's tile with that global index never publishes its literals, so that
 * every later tile's wait runs out and the call returns ACEAPEX_ERR_TIMEOUT without faulting the GPU
 * (UINT64_MAX = none).  Applies to later launches on this context. */
int aceapex_set_wait_limit(uint64_t ns, uint64_t withhold_tile);

/* Kernel timing.  aceapex_profile(1) clears the totals and starts recording a CUDA event pair on the launch
 * stream around every kernel the library launches (not inside CUDA-graph capture); aceapex_profile(0)
 * stops.  aceapex_profile_read synchronises on the recorded events, adds them to the per-kernel totals
 * and fills up to max_kernels entries (kernel name, total milliseconds, launch count); it returns the
 * number of kernels the library has. */
int aceapex_profile(int enable);
int aceapex_profile_read(int max_kernels, const char **names, double *total_ms, uint64_t *launches);

/* Statistics of the last aceapex_decode on this context (level histogram only when the wavefront ran). */
int aceapex_get_stats(aceapex_stats *stats);

/* Pre-scan choice between a CPU and a GPU decode (paper §8, data characteristics and GPU suitability: the
 * size and the depth of a stream, read from its header, decide which processor decodes it faster).  The
 * model is in decoded GB/s and microseconds; fields left at 0 take the defaults measured on GB300
 * (one-pass 260 GB/s; wavefront 200 GB/s plus 16.5 us per dependency level; 30 us fixed per decode).
 * cpu_gbps (required, > 0) is the caller's own CPU decode rate, measured on its host; link_gbps > 0 adds
 * the copy of the stream and the output between host and device to the GPU time (0: device-resident). */
typedef struct {
    double cpu_gbps, gpu_one_pass_gbps, gpu_wave_gbps, gpu_level_us, gpu_fixed_us, link_gbps;
} aceapex_device_model;

/* Returns 1 when the GPU decode is estimated faster, 0 when the CPU decode is, ACEAPEX_ERR_ARG for a null
 * pointer or cpu_gbps <= 0.  *cpu_s and *gpu_s (may be null) receive the two estimates in seconds.  Streams
 * the one-pass kernel takes (see aceapex_set_force_wavefront) are estimated at the one-pass rate. */
int aceapex_choose_device(const aceapex_info *info, const aceapex_device_model *model, double *cpu_s, double *gpu_s);

/* Human-readable name of a status code. */
const char *aceapex_strerror(int code);

/* ------------------------------------------------------------------------------------- entropy stage */
/*
 * Entropy container (stream format §6): the entropy stage the paper names without fixing one (§6 of the
 * paper, an FSE stage over the arrays), read here as canonical Huffman coding (codes of at most 12 bits) of
 * segments of at most 4096 bytes of a stream, 32 interleaved lanes per segment; decoding it gives back the
 * wrapped stream byte for byte, which the decode calls above then take.
 *
 * aceapex_entropy_peek: the container header from host memory (len >= 64 bytes): ACEAPEX_ERR_FORMAT for a
 *   bad magic/version/field, ACEAPEX_ERR_SIZE for a bad e_len.
 * aceapex_entropy_decode: decodes the device container e (16-byte aligned, e_len bytes, header info from
 *   aceapex_entropy_peek of its first 64 bytes) into the device buffer raw (raw_len = info->raw_len bytes),
 *   enqueued on `stream` without a host synchronization; *d_status (device int32) receives 0 or
 *   ACEAPEX_ERR_FORMAT (any malformed segment, table, length, Kraft sum or bitstream).  Returns
 *   ACEAPEX_ERR_ARG / ACEAPEX_ERR_SIZE for bad arguments, ACEAPEX_ERR_CUDA if the launch fails.  It uses no
 *   workspace; one launch, one warp per segment.
 */
typedef struct {
    uint64_t raw_len, n_seg, e_len;
} aceapex_entropy_info;
int aceapex_entropy_peek(const void *host_prefix, size_t len, aceapex_entropy_info *info);
/* Wrap the host stream raw (raw_len bytes) in an entropy container, on the host: stored stream header, block
 * index, block headers and sync tables; each block section coded with its own code (a segment stored when
 * coding would not shrink it).  *out is allocated (release with aceapex_free), *out_len its length. */
int aceapex_entropy_encode(const void *raw, size_t raw_len, void **out, size_t *out_len);
int aceapex_entropy_decode(const void *e, size_t e_len, const aceapex_entropy_info *info, void *raw, size_t raw_len,
                           int32_t *d_status, void *stream);

/* ---------------------------------------------------------------------------------------- transcoder */
/*
 * Global chain flattening of an existing stream (§3.3, applied after the fact; §7.1 orders the work): the
 * result decodes to the same bytes and every one of its matches reads literal bytes only (depth 1), so the
 * one-pass kernel decodes it.  Every match byte has a root, the literal byte it ultimately copies (a literal
 * byte is its own root; byte k of a match with destination d, source s, period p = d - s has the root of
 * byte s + (k mod p)).  Each match becomes: itself, if it overlaps itself and its effective source [s, d) is
 * literal; else, for a short repeat (p < L, p <= 32, L - p >= min_match), its first period as literal bytes
 * and the self-overlapping match (d + p, d, L - p); else the maximal runs of its bytes with consecutive
 * roots, those of at least min_match bytes as matches from the root of their first byte, the rest as
 * literal bytes.  The result keeps block_log2, tile_log2 and min_match, with flatten mode 2 and depth_cap 0.
 *
 * aceapex_transcode_create: comp is a device stream (16-byte aligned) of at most 2^32 - 1 decoded bytes.
 *   Runs every step on the GPU (decode, roots, rewritten matches, block layout) and synchronizes `stream`;
 *   *out_len receives the size of the result and *plan the object holding the intermediate device buffers
 *   (about 4 bytes per decoded byte plus the wavefront workspace).  Returns the decode's status for a
 *   malformed stream, ACEAPEX_ERR_SIZE for a stream over 2^32 - 1 bytes, ACEAPEX_ERR_NOMEM if a buffer
 *   cannot be allocated (nothing is kept then).
 * aceapex_transcode_write: writes the result into the device buffer out (16-byte aligned, out_cap >= out_len
 *   bytes, else ACEAPEX_ERR_SIZE) on `stream` and synchronizes it.
 * aceapex_transcode_info: matches and sequences of the result.
 * aceapex_transcode_destroy: frees the plan (synchronizes the device).
 */
typedef struct aceapex_transcode aceapex_transcode;
int aceapex_transcode_create(const void *comp, size_t comp_len, aceapex_transcode **plan, size_t *out_len, void *stream);
int aceapex_transcode_write(aceapex_transcode *plan, void *out, size_t out_cap, void *stream);
int aceapex_transcode_info(const aceapex_transcode *plan, uint64_t *n_match, uint64_t *n_seq);
int aceapex_transcode_destroy(aceapex_transcode *plan);

/* -------------------------------------------------------------------------------------------- server */
/*
 * Continuous-batching decode server.  Requests are device-resident streams (16-byte aligned) with their
 * header info.  aceapex_server_step admits queued requests in arrival order while stream + output bytes fit
 * hbm_budget and one of max_slots slots is free (the server allocates each output with the stream-ordered
 * allocator), then enqueues ONE one-pass launch that advances every admitted request by a slice of its tiles
 * (each request gets an equal share of tiles_per_step); requests admitted while others are running join the
 * next launch.  A stream the one-pass kernel does not take (deeper than 1, tiles over 4 KiB) is decoded
 * whole by the wavefront path on a stream the server owns, enqueued in the step that admits it, so the
 * other requests' launches do not wait for it.  poll returns 1 once a
 * request's last launch has completed (with its status and output pointer), 0 while pending; release frees
 * its output and budget (stream-ordered on `stream`).  step returns the number of queued + running
 * requests.  One host thread drives a server; the budget counts stream + output bytes (plus, for a request
 * the one-pass kernel takes, its literal bitmap: one bit per output byte).  A request is admitted only once
 * its first work is enqueued: if that fails, step returns the error and the request stays queued, holding
 * nothing.
 */
typedef struct aceapex_server aceapex_server;
int aceapex_server_create(size_t hbm_budget, int max_slots, uint64_t tiles_per_step, aceapex_server **server);
int64_t aceapex_server_submit(aceapex_server *server, const void *comp, size_t comp_len, const aceapex_info *info);
int aceapex_server_step(aceapex_server *server, void *stream);
int aceapex_server_poll(aceapex_server *server, int64_t id, int32_t *status, void **out);
int aceapex_server_release(aceapex_server *server, int64_t id, void *stream);
int aceapex_server_destroy(aceapex_server *server);

/* ------------------------------------------------------------------------------------------- encoder */
/* Encoder parameters (host side, CPU).  Defaults: block_log2 20, tile_log2 12, min_match 4,
 * hash_bits 20, chain_limit 16, flatten 0, depth_cap 0, use_first 1, min_emit 0, long_bits 0 (off),
 * long_chain 4.  long_bits > 0 adds a second candidate chain keyed by the 12 bytes at each position
 * (2^long_bits hash values, long_chain most recent positions each, tried first), which finds long repeats
 * on small alphabets (DNA bases) where 4-byte keys take few values. */
typedef struct {
    uint32_t block_log2, tile_log2, min_match, hash_bits, chain_limit, flatten, depth_cap, use_first, min_emit;
    uint32_t long_bits, long_chain;
} aceapex_enc_params;

/*
 * Encode n host bytes into a newly allocated host buffer (*out, release with aceapex_free).  Greedy
 * hash-chain parse with absolute offsets (§3.1, §3.4), optional chain flattening (§3.3) and depth cap
 * (§7.4).  Returns the stream length or a negative status.  Inputs must be shorter than 4 GiB;
 * chain_limit <= 16, 8 <= hash_bits <= 24; long_bits 0 or 8..28 with 1 <= long_chain <= 16.
 */
int64_t aceapex_encode(const void *in, size_t n, const aceapex_enc_params *params, void **out);
void aceapex_free(void *p);

#ifdef __cplusplus
}
#endif
#endif /* ACEAPEX_H */
