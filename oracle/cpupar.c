/*
 * Block-parallel multi-core CPU decoder -- TEST AND BENCHMARK INFRASTRUCTURE ONLY (a CPU baseline).
 *
 * The paper's CPU decoder (§3.1, last paragraph of "Absolute Offsets"; methodology §4.3): absolute offsets
 * make every block self-contained, so I threads decode blocks in parallel.  Threads take blocks in
 * stream order from a shared counter and decode each one sequentially (literal run, then the match byte by
 * byte from its absolute source).  A match whose source lies in an earlier block that another thread is
 * still decoding waits until that block has published its progress past the source bytes; a source in
 * the thread's own block is already written.  The lowest unfinished block never waits (its sources lie in
 * finished blocks), so the decode always completes.
 *
 * A batch of independent streams (§7.5) is decoded the same way from one queue of (stream, block) units in
 * order -- stream 0's blocks, then stream 1's, ... -- so that small streams of one or a few blocks keep
 * every thread busy.  Waits stay inside a stream; the lowest unfinished unit still never waits.
 *
 * Not the oracle: it checks the stream's structure only as far as needed to stay in bounds and returns
 * -2/-3/-4 on a stream it cannot decode; the oracle (oracle.c) is the definition of the decoded bytes.
 * Shares no code with the GPU library or with oracle.c.
 */
#include <pthread.h>
#include <sched.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define CP_ERR_FORMAT (-2)
#define CP_ERR_SIZE (-3)
#define CP_ERR_OFFSET (-4)
#define CP_ERR_NOMEM (-7)
#define CP_PUBLISH 4096  /* a block publishes its progress every this many output bytes */

static uint64_t le(const uint8_t *p, int n) {
    uint64_t v = 0;
    for (int i = n - 1; i >= 0; i--) v = (v << 8) | p[i];
    return v;
}
static uint64_t up16(uint64_t x) { return (x + 15) & ~(uint64_t)15; }

typedef struct {
    const uint8_t *c;
    uint64_t comp_len, N, n_blocks, B;
    uint32_t min_match;
    uint8_t *out;
    _Atomic uint64_t *done;       /* per block: output bytes written so far (block-relative) */
    _Atomic int err;              /* first failing status of this stream */
} stream_t;

typedef struct {
    stream_t *s;
    int n;
    const uint64_t *unit0;        /* n + 1 prefix sums of the streams' block counts */
    _Atomic uint64_t next;        /* next (stream, block) unit to take */
} job_t;

/* Wait until block b of stream S has written its first `upto` bytes (block-relative). */
static void wait_for(stream_t *S, uint64_t b, uint64_t upto) {
    while (atomic_load_explicit(&S->done[b], memory_order_acquire) < upto) {
        if (atomic_load_explicit(&S->err, memory_order_relaxed)) return;
        sched_yield();
    }
}

static int varint(const uint8_t *p, uint64_t end, uint64_t *pos, uint32_t *v) {
    uint64_t x = 0;
    for (int i = 0; i < 5; i++) {
        if (*pos >= end) return -1;
        const uint8_t b = p[(*pos)++];
        x |= (uint64_t)(b & 0x7F) << (7 * i);
        if (!(b & 0x80)) {
            if (x > 0xFFFFFFFFull) return -1;
            *v = (uint32_t)x;
            return 0;
        }
    }
    return -1;
}

static int decode_block(stream_t *J, uint64_t b) {
    const uint8_t *c = J->c;
    const uint64_t off = le(c + 64 + 8 * b, 8), end = b + 1 < J->n_blocks ? le(c + 64 + 8 * (b + 1), 8) : J->comp_len;
    if ((off & 15) || end <= off || end > J->comp_len || end - off < 32) return CP_ERR_FORMAT;
    const uint8_t *h = c + off;
    const uint32_t n_seq = (uint32_t)le(h, 4), n_match = (uint32_t)le(h + 4, 4), n_lit = (uint32_t)le(h + 8, 4);
    const uint32_t cmd_bytes = (uint32_t)le(h + 12, 4), len_bytes = (uint32_t)le(h + 16, 4), w = h[20];
    const uint32_t n_tiles = (uint32_t)le(h + 28, 4);
    if (w < 1 || w > 8) return CP_ERR_FORMAT;
    const uint64_t o_cmd = off + up16(32 + 20 * (uint64_t)n_tiles), o_len = up16(o_cmd + cmd_bytes);
    const uint64_t o_off = up16(o_len + len_bytes), o_lit = up16(o_off + (uint64_t)n_match * w);
    if (up16(o_lit + n_lit) != end) return CP_ERR_FORMAT;
    const uint64_t b0 = b * J->B, b1 = b0 + J->B < J->N ? b0 + J->B : J->N;
    uint8_t *out = J->out;
    uint64_t pos = b0, cp = 0, lp = 0, lt = 0, pub = 0;
    for (uint32_t i = 0; i < n_seq; i++) {
        uint32_t r, Lraw = 0;
        if (varint(c + o_cmd, cmd_bytes, &cp, &r)) return CP_ERR_FORMAT;
        if (pos + r > b1 || lt + r > n_lit) return CP_ERR_OFFSET;
        memcpy(out + pos, c + o_lit + lt, r);
        pos += r;
        lt += r;
        if (i < n_match) {
            if (varint(c + o_len, len_bytes, &lp, &Lraw)) return CP_ERR_FORMAT;
            const uint64_t L = (uint64_t)Lraw + J->min_match, s = le(c + o_off + (uint64_t)i * w, (int)w);
            if (s >= pos || pos + L > b1) return CP_ERR_OFFSET;
            const uint64_t eff = L < pos - s ? L : pos - s;  /* bytes written before the match */
            if (s < b0) {
                /* source bytes in earlier blocks: each must have published past them */
                for (uint64_t sb = s / J->B; sb * J->B < s + eff && sb < b; sb++) {
                    const uint64_t hi = s + eff < (sb + 1) * J->B ? s + eff - sb * J->B : J->B;
                    wait_for(J, sb, hi);
                }
            }
            if (pos - s >= L) {
                memcpy(out + pos, out + s, L);  /* source and destination do not overlap */
            } else {
                for (uint64_t k = 0; k < L; k++) out[pos + k] = out[s + k];  /* byte-sequential: RLE overlap */
            }
            pos += L;
        }
        if (pos - b0 >= pub + CP_PUBLISH) {
            pub = pos - b0;
            atomic_store_explicit(&J->done[b], pub, memory_order_release);
        }
    }
    if (pos != b1) return CP_ERR_FORMAT;
    atomic_store_explicit(&J->done[b], b1 - b0, memory_order_release);
    return 0;
}

/* Header checks and the per-stream state: 0, a negative status, or 1 for an empty stream (nothing to do). */
static int stream_init(stream_t *S, const uint8_t *comp, uint64_t comp_len, uint8_t *out, uint64_t out_len) {
    memset(S, 0, sizeof(*S));
    atomic_init(&S->err, 0);
    if (!comp || comp_len < 64 || (comp_len & 15)) return CP_ERR_SIZE;
    if (le(comp, 4) != 0x58454341u || le(comp + 4, 2) != 1) return CP_ERR_FORMAT;
    const uint32_t bl = comp[8];
    if (bl < 2 || bl > 24) return CP_ERR_FORMAT;
    S->c = comp;
    S->comp_len = comp_len;
    S->N = le(comp + 16, 8);
    S->n_blocks = le(comp + 24, 8);
    S->B = 1ull << bl;
    S->min_match = comp[10];
    S->out = out;
    if (S->N != out_len || le(comp + 32, 8) != comp_len) return CP_ERR_SIZE;
    if (S->n_blocks != (S->N + S->B - 1) / S->B || 64 + 8 * S->n_blocks > comp_len) return CP_ERR_FORMAT;
    if (S->N == 0) return 1;
    S->done = (_Atomic uint64_t *)calloc(S->n_blocks, sizeof(_Atomic uint64_t));
    return S->done ? 0 : CP_ERR_NOMEM;
}

static void *worker(void *arg) {
    job_t *J = (job_t *)arg;
    const uint64_t total = J->unit0[J->n];
    int k = 0;  /* stream of the last unit taken: a thread's units only increase */
    for (;;) {
        const uint64_t u = atomic_fetch_add(&J->next, 1);
        if (u >= total) break;
        while (J->unit0[k + 1] <= u) k++;
        stream_t *S = &J->s[k];
        const uint64_t b = u - J->unit0[k];
        /* the blocks of a stream that has failed are skipped */
        const int rc = atomic_load(&S->err) ? 1 : decode_block(S, b);
        if (rc) {
            if (rc < 0) {
                int z = 0;
                atomic_compare_exchange_strong(&S->err, &z, rc);
            }
            /* unblock waiters: mark the block as written (the stream's result is discarded with the error) */
            atomic_store_explicit(&S->done[b], S->B, memory_order_release);
        }
    }
    return NULL;
}

static void run(job_t *J, int threads) {
    const uint64_t total = J->unit0[J->n];
    if (total == 0) return;
    if (threads < 1) threads = 1;
    if ((uint64_t)threads > total) threads = (int)total;
    pthread_t *tid = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    int started = 0;
    if (tid)
        for (; started < threads - 1; started++)
            if (pthread_create(&tid[started], NULL, worker, J)) break;
    worker(J);  /* the calling thread works too */
    for (int k = 0; k < started; k++) pthread_join(tid[k], NULL);
    free(tid);
}

/* Decode a stream with `threads` threads (<= 0: one).  Returns 0 or a negative status. */
int cpupar_decode(const uint8_t *comp, uint64_t comp_len, uint8_t *out, uint64_t out_len, int threads) {
    stream_t S;
    const int rc = stream_init(&S, comp, comp_len, out, out_len);
    if (rc) return rc > 0 ? 0 : rc;
    uint64_t unit0[2] = {0, S.n_blocks};
    job_t J;
    J.s = &S;
    J.n = 1;
    J.unit0 = unit0;
    atomic_init(&J.next, 0);
    run(&J, threads);
    free((void *)S.done);
    return atomic_load(&S.err);
}

/* Decode n independent streams with `threads` threads from one queue of (stream, block) units; comps/outs:
 * arrays of n pointers, comp_lens/out_lens: arrays of n lengths, statuses: n int32 that receive each
 * stream's status.  Returns 0 when every stream decoded, else the first failing status in stream order. */
int cpupar_decode_batch(int n, const uint8_t *const *comps, const uint64_t *comp_lens, uint8_t *const *outs,
                        const uint64_t *out_lens, int32_t *statuses, int threads) {
    if (n < 0 || (n > 0 && (!comps || !comp_lens || !outs || !out_lens || !statuses))) return CP_ERR_SIZE;
    stream_t *S = (stream_t *)calloc(n > 0 ? (size_t)n : 1, sizeof(stream_t));
    uint64_t *unit0 = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    if (!S || !unit0) {
        free(S);
        free(unit0);
        return CP_ERR_NOMEM;
    }
    unit0[0] = 0;
    for (int i = 0; i < n; i++) {
        const int rc = stream_init(&S[i], comps[i], comp_lens[i], outs[i], out_lens[i]);
        statuses[i] = rc < 0 ? rc : 0;
        unit0[i + 1] = unit0[i] + (rc == 0 ? S[i].n_blocks : 0);
    }
    job_t J;
    J.s = S;
    J.n = n;
    J.unit0 = unit0;
    atomic_init(&J.next, 0);
    run(&J, threads);
    int first = 0;
    for (int i = 0; i < n; i++) {
        if (S[i].done) {
            statuses[i] = atomic_load(&S[i].err);
            free((void *)S[i].done);
        }
        if (statuses[i] && !first) first = statuses[i];
    }
    free(S);
    free(unit0);
    return first;
}
