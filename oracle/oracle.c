/*
 * ACEAPEX CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, sequential restatement of the method (paper §3.1-§3.4, §7.1, §7.4) used to check the
 * GPU decoder.  Only the test suite, the smoke check and the benchmark's CPU-baseline leg may load it;
 * the product library never does, and this file shares no code with it.
 *
 * Contents
 *   oracle_encode     greedy hash-chain encoder with absolute offsets (§3.1), self-contained blocks,
 *                     optional chain flattening (§3.3, global or within-block) and depth cap (§7.4)
 *   oracle_serialize  writes a parse (match list) in the ACEAPEX stream format
 *   oracle_decode     the definition of the decoded bytes: blocks in order, sequences in order,
 *                     literal run then byte-by-byte match copy from the absolute source (§3.2); a
 *                     stream whose block max_depth understates a match's depth (§7.1) is rejected
 *                     with ERR_DEPTH after every other check
 *   oracle_parse      lists every sequence (literal-run length, match length, absolute source)
 *   oracle_lz77_rel_decode  textbook LZ77 with backward distances (§2) on the same parse
 *   oracle_depths     per-match dependency depth by byte-level simulation (§7.1)
 *   oracle_check      invariants: flattened sources are literal (§3.3), depth cap honoured (§7.4),
 *                     block depth fields equal the recomputed ones (§7.1)
 *   oracle_transcode_flat  global chain flattening (§3.3) of an existing stream: every match rewritten as
 *                     the maximal runs of its bytes with consecutive roots, each copying from its root
 *
 * Pins (tests/test_oracle_*.py): encode->decode round trip on every generator, agreement with the
 * textbook relative decoder, brute force over every legal parse of tiny strings, hand-assembled golden
 * streams, the §3.1 worked example, and the invariants above.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_FORMAT (-2)
#define OR_ERR_SIZE (-3)
#define OR_ERR_OFFSET (-4)
#define OR_ERR_NOMEM (-7)
#define OR_ERR_DEPTH (-8)

#define MAGIC 0x58454341u
#define NONE UINT64_MAX
#define CHAIN_MAX 256
#define LONG_CHAIN_MAX 16
#define LONG_KEY 12
#define PERIOD_MAX 16
#define PERIOD_RESTART 32
#define TRANSCODE_PERIOD_MAX 32  /* transcoder: repeats of at most this period restart from literal bytes */

typedef struct {
    uint32_t block_log2, tile_log2, min_match, hash_bits, chain_limit, flatten, depth_cap, use_first, min_emit;
    uint32_t long_bits, long_chain;
} or_params;

typedef struct {
    uint64_t N, n_blocks, comp_len, n_match, n_seq;
    uint32_t block_log2, tile_log2, min_match, flatten, depth_cap, max_depth;
} or_info;

/* ------------------------------------------------------------------------------------------ bytes */
static uint64_t rd(const uint8_t *p, int n) {
    uint64_t v = 0;
    for (int i = n - 1; i >= 0; i--) v = (v << 8) | p[i];
    return v;
}
static void wr(uint8_t *p, uint64_t v, int n) {
    for (int i = 0; i < n; i++) { p[i] = (uint8_t)(v & 0xFF); v >>= 8; }
}
static uint64_t align16(uint64_t x) { return (x + 15) & ~(uint64_t)15; }

/* LEB128: 7 bits per byte, low group first, high bit set on every byte but the last */
static int put_varint(uint8_t *p, uint32_t v) {
    int n = 0;
    while (v >= 0x80) { p[n++] = (uint8_t)(v | 0x80); v >>= 7; }
    p[n++] = (uint8_t)v;
    return n;
}
static int varint_size(uint32_t v) { int n = 1; while (v >= 0x80) { v >>= 7; n++; } return n; }
/* reads one varint from p[*pos], p has `end` bytes; returns 0 on success */
static int get_varint(const uint8_t *p, uint64_t end, uint64_t *pos, uint32_t *out) {
    uint64_t v = 0;
    for (int i = 0; i < 5; i++) {
        if (*pos >= end) return OR_ERR_FORMAT;
        uint8_t c = p[(*pos)++];
        v |= (uint64_t)(c & 0x7F) << (7 * i);
        if (!(c & 0x80)) {
            if (v > 0xFFFFFFFFull) return OR_ERR_FORMAT;
            *out = (uint32_t)v;
            return OR_OK;
        }
    }
    return OR_ERR_FORMAT;
}
static int bytes_for(uint64_t v) { int w = 1; while (w < 8 && (v >> (8 * w))) w++; return w; }

/* ------------------------------------------------------------------------------------------ depth of a parse */
/*
 * §7.1: a literal byte has depth 0; a match has depth 1 + the largest depth among the bytes of its
 * effective source [s, s + min(L, d - s)); each byte it writes takes that depth.
 */
static uint32_t *parse_depths(uint64_t N, const uint64_t *d, const uint64_t *s, const uint32_t *L, uint64_t nm,
                              uint32_t *mdepth) {
    uint32_t *wdepth = (uint32_t *)calloc(N ? N : 1, sizeof(uint32_t));
    if (!wdepth) return NULL;
    for (uint64_t m = 0; m < nm; m++) {
        uint64_t eff = L[m] < d[m] - s[m] ? L[m] : d[m] - s[m];
        uint32_t mx = 0;
        for (uint64_t x = s[m]; x < s[m] + eff; x++) if (wdepth[x] > mx) mx = wdepth[x];
        mdepth[m] = mx + 1;
        for (uint64_t k = 0; k < L[m]; k++) wdepth[d[m] + k] = mx + 1;
    }
    return wdepth;
}

/* ------------------------------------------------------------------------------------------ serializer */
/*
 * Writes the parse (matches sorted by destination; every other byte is a literal taken from `in`) in the
 * layout of the ACEAPEX stream format.  *out is malloc'ed; returns the stream length or a negative error.
 */
int64_t oracle_serialize(const uint8_t *in, uint64_t N, const uint64_t *d, const uint64_t *s, const uint32_t *L,
                         uint64_t nm, const or_params *prm, uint8_t **out) {
    *out = NULL;
    if (prm->block_log2 < 2 || prm->block_log2 > 24 || prm->tile_log2 < 2 || prm->tile_log2 > prm->block_log2 ||
        prm->min_match < 1 || prm->min_match > 255 || prm->flatten > 2)
        return OR_ERR_ARG;
    const uint64_t B = 1ull << prm->block_log2, T = 1ull << prm->tile_log2;
    const uint64_t n_blocks = (N + B - 1) / B;
    /* validate the parse */
    for (uint64_t m = 0; m < nm; m++) {
        if (L[m] < prm->min_match || s[m] >= d[m] || d[m] + L[m] > N) return OR_ERR_OFFSET;
        if (m > 0 && d[m] < d[m - 1] + L[m - 1]) return OR_ERR_OFFSET;
        if ((d[m] >> prm->block_log2) != ((d[m] + L[m] - 1) >> prm->block_log2)) return OR_ERR_OFFSET;
    }
    uint32_t *mdepth = (uint32_t *)malloc((nm ? nm : 1) * sizeof(uint32_t));
    uint32_t *wdepth = mdepth ? parse_depths(N, d, s, L, nm, mdepth) : NULL;
    if (!wdepth) { free(mdepth); return OR_ERR_NOMEM; }
    free(wdepth);

    /* pass 1: sizes of every block */
    uint64_t *bsize = (uint64_t *)calloc(n_blocks ? n_blocks : 1, sizeof(uint64_t));
    uint64_t total = align16(64 + 8 * n_blocks), m = 0, n_seq_total = 0;
    uint32_t max_depth = 0;
    for (uint64_t b = 0; b < n_blocks; b++) {
        uint64_t b0 = b * B, b1 = (b0 + B < N) ? b0 + B : N, pos = b0, cmd = 0, len = 0, lit = 0, ns = 0, nmb = 0;
        uint64_t maxoff = 0;
        while (m < nm && d[m] < b1) {
            cmd += varint_size((uint32_t)(d[m] - pos));
            len += varint_size(L[m] - prm->min_match);
            lit += d[m] - pos;
            if (s[m] > maxoff) maxoff = s[m];
            pos = d[m] + L[m]; ns++; nmb++; m++;
        }
        if (pos < b1) { cmd += varint_size((uint32_t)(b1 - pos)); lit += b1 - pos; ns++; }
        uint64_t n_tiles = (b1 - b0 + T - 1) / T;
        int w = bytes_for(maxoff);
        uint64_t sz = align16(32 + 20 * n_tiles);
        sz = align16(sz + cmd); sz = align16(sz + len); sz = align16(sz + nmb * (uint64_t)w); sz = align16(sz + lit);
        bsize[b] = sz; total += sz; n_seq_total += ns;
    }
    for (uint64_t i = 0; i < nm; i++) if (mdepth[i] > max_depth) max_depth = mdepth[i];
    uint8_t *o = (uint8_t *)calloc(total, 1);
    if (!o) { free(bsize); free(mdepth); return OR_ERR_NOMEM; }

    /* stream header */
    wr(o + 0, MAGIC, 4); wr(o + 4, 1, 2); wr(o + 6, prm->flatten, 2);
    o[8] = (uint8_t)prm->block_log2; o[9] = (uint8_t)prm->tile_log2; o[10] = (uint8_t)prm->min_match;
    wr(o + 12, prm->depth_cap, 4); wr(o + 16, N, 8); wr(o + 24, n_blocks, 8); wr(o + 32, total, 8);
    wr(o + 40, nm, 8); wr(o + 48, max_depth, 4); wr(o + 56, n_seq_total, 8);

    /* pass 2: blocks */
    uint64_t at = align16(64 + 8 * n_blocks);
    m = 0;
    for (uint64_t b = 0; b < n_blocks; b++) {
        wr(o + 64 + 8 * b, at, 8);
        uint64_t b0 = b * B, b1 = (b0 + B < N) ? b0 + B : N, n_tiles = (b1 - b0 + T - 1) / T;
        uint64_t m0 = m, m1 = m;
        while (m1 < nm && d[m1] < b1) m1++;
        uint64_t nmb = m1 - m0, maxoff = 0;
        uint32_t bdepth = 0;
        for (uint64_t i = m0; i < m1; i++) { if (s[i] > maxoff) maxoff = s[i]; if (mdepth[i] > bdepth) bdepth = mdepth[i]; }
        int w = bytes_for(maxoff);
        uint64_t last_pos = (m1 > m0) ? d[m1 - 1] + L[m1 - 1] : b0;
        uint64_t ns = nmb + (last_pos < b1 ? 1 : 0);
        /* section sizes */
        uint64_t cmd = 0, len = 0, lit = 0, pos = b0;
        for (uint64_t i = m0; i < m1; i++) {
            cmd += varint_size((uint32_t)(d[i] - pos)); len += varint_size(L[i] - prm->min_match);
            lit += d[i] - pos; pos = d[i] + L[i];
        }
        if (pos < b1) { cmd += varint_size((uint32_t)(b1 - pos)); lit += b1 - pos; }
        uint8_t *h = o + at;
        wr(h + 0, ns, 4); wr(h + 4, nmb, 4); wr(h + 8, lit, 4); wr(h + 12, cmd, 4); wr(h + 16, len, 4);
        h[20] = (uint8_t)w; wr(h + 24, bdepth, 4); wr(h + 28, n_tiles, 4);
        uint64_t o_cmd = align16(32 + 20 * n_tiles), o_len = align16(o_cmd + cmd), o_off = align16(o_len + len),
                 o_lit = align16(o_off + nmb * (uint64_t)w);
        /* sequences, sync table */
        uint64_t cp = 0, lp = 0, lt = 0, tile = 0;
        pos = b0;
        for (uint64_t i = 0; i < ns; i++) {
            int has_match = (m0 + i < m1);
            uint64_t r = has_match ? d[m0 + i] - pos : b1 - pos;
            uint64_t seq_end = pos + r + (has_match ? L[m0 + i] : 0);
            /* tiles whose first byte lies in this sequence */
            while (tile < n_tiles && b0 + tile * T < seq_end) {
                uint8_t *e = h + 32 + 20 * tile;
                wr(e + 0, i, 4); wr(e + 4, cp, 4); wr(e + 8, lp, 4); wr(e + 12, lt, 4); wr(e + 16, pos - b0, 4);
                tile++;
            }
            cp += (uint64_t)put_varint(h + o_cmd + cp, (uint32_t)r);
            memcpy(h + o_lit + lt, in + pos, r);
            lt += r;
            if (has_match) {
                lp += (uint64_t)put_varint(h + o_len + lp, L[m0 + i] - prm->min_match);
                wr(h + o_off + (uint64_t)w * i, s[m0 + i], w);
            }
            pos = seq_end;
        }
        at += bsize[b];
        m = m1;
    }
    free(bsize); free(mdepth);
    *out = o;
    return (int64_t)total;
}

/* ------------------------------------------------------------------------------------------ encoder */
static uint32_t hash4(const uint8_t *p, uint32_t bits) {
    uint32_t v = (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
    return (uint32_t)(v * 2654435761u) >> (32 - bits);
}

/* Hash of the 12 bytes at p (little-endian 8-byte and 4-byte words, multiplied and added mod 2^64). */
static uint32_t hash12(const uint8_t *p, uint32_t bits) {
    uint64_t lo = rd(p, 8), hi = rd(p + 8, 4);
    uint64_t v = lo * 0x9E3779B97F4A7C15ull + hi * 0xC2B2AE3D27D4EB4Full;
    return (uint32_t)(v >> (64 - bits));
}

typedef struct { uint64_t *d, *s; uint32_t *L; uint64_t n, cap; } mlist;
static int ml_push(mlist *ml, uint64_t d, uint64_t s, uint32_t L) {
    if (ml->n == ml->cap) {
        uint64_t c = ml->cap ? 2 * ml->cap : 1024;
        uint64_t *nd = (uint64_t *)realloc(ml->d, c * 8), *ns = (uint64_t *)realloc(ml->s, c * 8);
        uint32_t *nl = (uint32_t *)realloc(ml->L, c * 4);
        if (nd) ml->d = nd;
        if (ns) ml->s = ns;
        if (nl) ml->L = nl;
        if (!nd || !ns || !nl) return OR_ERR_NOMEM;
        ml->cap = c;
    }
    ml->d[ml->n] = d; ml->s[ml->n] = s; ml->L[ml->n] = L; ml->n++;
    return OR_OK;
}
static void ml_free(mlist *ml) { free(ml->d); free(ml->s); free(ml->L); memset(ml, 0, sizeof(*ml)); }

/*
 * Greedy parse with a view of the whole input (§3.4): positions are hashed over all of it (absolute
 * positions, no window).  The candidates for position p are, when long_bits is set, the long_chain most
 * recent earlier positions with the same hash of the 12 bytes at p (a key that stays selective on small
 * alphabets such as DNA, where 4-byte keys take few values), then the chain_limit most recent earlier
 * positions with the same 4-byte hash, then (if use_first) the first position ever seen with that hash.
 * Every position is entered in the 4-byte chain; in flatten modes only literal positions (their own root)
 * enter the 12-byte chain, so that its candidates start on bytes a flattened match may point at.  A match
 * never leaves its destination block.  The longest candidate wins; equal lengths go to the smaller depth, then to the
 * candidate found first.
 *
 * Chain flattening (§3.3) is applied while parsing: every byte x carries root[x], the literal position
 * whose byte it copies (global mode), or -- block mode -- the first position reached outside x's own
 * block when following its chain.  Seen from position p, a source byte x has root R(x) = root[x] if x
 * lies in p's block or the mode is global, else x itself.  A candidate c is usable only over the prefix
 * where R(c), R(c)+1, ... are consecutive, and the match then points at R(c): it reads only literal bytes
 * (global) or literal and earlier-block bytes (block).  A candidate that runs into p itself continues as a
 * self-overlapping copy only when its source bytes [c, p) are their own roots.
 *
 * Depth cap D (§7.4): a candidate is cut before the first byte of its effective source whose depth is
 * at least D, so the match depth stays at most D.
 */
static int greedy_parse(const uint8_t *in, uint64_t N, const or_params *prm, mlist *ml) {
    const uint32_t bits = prm->hash_bits ? prm->hash_bits : 20;
    const uint64_t HS = 1ull << bits;
    const int flat = (int)prm->flatten, bl = (int)prm->block_log2;
    const uint32_t lbits = prm->long_bits;
    const uint64_t LS = lbits ? 1ull << lbits : 1;
    uint64_t *head = (uint64_t *)malloc(HS * 8), *first = (uint64_t *)malloc(HS * 8);
    uint64_t *prev = (uint64_t *)malloc((N ? N : 1) * 8);
    uint64_t *head2 = (uint64_t *)malloc(LS * 8), *prev2 = lbits ? (uint64_t *)malloc((N ? N : 1) * 8) : NULL;
    uint64_t *root = flat ? (uint64_t *)malloc((N ? N : 1) * 8) : NULL;
    uint32_t *wdepth = (uint32_t *)calloc(N ? N : 1, 4);
#define FREE_ALL() do { free(head); free(first); free(prev); free(head2); free(prev2); free(root); free(wdepth); } while (0)
    if (!head || !first || !prev || !head2 || (lbits && !prev2) || !wdepth || (flat && !root)) {
        FREE_ALL();
        return OR_ERR_NOMEM;
    }
    for (uint64_t i = 0; i < HS; i++) { head[i] = NONE; first[i] = NONE; }
    for (uint64_t i = 0; i < LS; i++) head2[i] = NONE;
    const uint64_t mm = prm->min_match > prm->min_emit ? prm->min_match : prm->min_emit, cap = prm->depth_cap;
    uint64_t p = 0;
#define R(x) ((flat == 2 || ((x) >> bl) == (p >> bl)) ? root[x] : (x))
    while (p < N) {
        uint64_t blk_end = ((p >> bl) + 1) << bl;
        if (blk_end > N) blk_end = N;
        uint64_t maxL = blk_end - p, best_L = 0, best_s = 0;
        uint32_t best_dep = 0;
        if (maxL >= mm && p + 4 <= N) {
            uint32_t h = hash4(in + p, bits);
            /* candidate list: the long-key chain's most recent positions, the 4-byte chain's most recent
               positions, then the first position of the 4-byte hash */
            uint64_t cand[LONG_CHAIN_MAX + CHAIN_MAX + 1];
            uint32_t nc = 0;
            if (lbits && p + LONG_KEY <= N) {
                uint32_t nl = 0;
                for (uint64_t c = head2[hash12(in + p, lbits)]; c != NONE && nl < prm->long_chain; c = prev2[c])
                    cand[nc++] = c, nl++;
            }
            for (uint64_t c = head[h], k = 0; c != NONE && k < prm->chain_limit; c = prev[c], k++) cand[nc++] = c;
            if (prm->use_first && first[h] != NONE) cand[nc++] = first[h];
            for (uint32_t j = 0; j < nc; j++) {
                uint64_t c = cand[j], Lc = 0, src = c;
                while (Lc < maxL && in[c + Lc] == in[p + Lc]) Lc++;
                if (flat && Lc > 0) {
                    uint64_t r0 = R(c), k = 1;
                    while (k < Lc && c + k < p && R(c + k) == r0 + k) k++;
                    if (k < Lc && c + k == p && r0 == c) k = Lc;  /* overlap on bytes that are their own roots */
                    Lc = k;
                    src = r0;
                }
                if (cap > 0) {  /* cut before the first effective-source byte of depth >= cap */
                    uint64_t eff = Lc < p - src ? Lc : p - src;
                    for (uint64_t x = src; x < src + eff; x++)
                        if (wdepth[x] >= cap) { Lc = x - src; break; }
                }
                if (Lc < mm) continue;
                uint64_t eff = Lc < p - src ? Lc : p - src;
                uint32_t mx = 0;
                for (uint64_t x = src; x < src + eff; x++) if (wdepth[x] > mx) mx = wdepth[x];
                if (Lc > best_L || (Lc == best_L && mx + 1 < best_dep)) { best_L = Lc; best_s = src; best_dep = mx + 1; }
            }
        }
        uint64_t adv = 1, lits = 1;
        if (flat && best_L < PERIOD_RESTART) {
            /* period restart: when the input ahead repeats with a short period, emit one period as
               literals so that the next position can copy them as a self-overlapping match */
            for (uint64_t per = 1; per <= PERIOD_MAX && p + per + PERIOD_RESTART + 4 * per <= blk_end; per++) {
                uint64_t run = 0;
                while (p + per + run < blk_end && in[p + per + run] == in[p + run]) run++;
                if (run >= PERIOD_RESTART + 4 * per) { lits = per; best_L = 0; break; }
            }
        }
        if (best_L >= mm) {
            if (ml_push(ml, p, best_s, (uint32_t)best_L)) {
                FREE_ALL();
                return OR_ERR_NOMEM;
            }
            uint64_t per = p - best_s;
            for (uint64_t k = 0; k < best_L; k++) {
                wdepth[p + k] = best_dep;
                if (flat) root[p + k] = R(best_s + (k % per));
            }
            adv = best_L;
        } else {
            for (uint64_t k = 0; k < lits; k++) {
                wdepth[p + k] = 0;
                if (flat) root[p + k] = p + k;
            }
            adv = lits;
        }
        for (uint64_t q = p; q < p + adv; q++) {
            if (q + 4 <= N) {
                uint32_t h = hash4(in + q, bits);
                prev[q] = head[h]; head[h] = q;
                if (first[h] == NONE) first[h] = q;
            }
            if (lbits && q + LONG_KEY <= N && (!flat || root[q] == q)) {
                uint32_t h2 = hash12(in + q, lbits);
                prev2[q] = head2[h2]; head2[h2] = q;
            }
        }
        p += adv;
    }
#undef R
    FREE_ALL();
#undef FREE_ALL
    return OR_OK;
}

int64_t oracle_encode(const uint8_t *in, uint64_t N, const or_params *prm, uint8_t **out) {
    *out = NULL;
    if (prm->block_log2 < 2 || prm->block_log2 > 24 || prm->min_match < 1 || prm->flatten > 2 ||
        prm->chain_limit > CHAIN_MAX || (prm->hash_bits && (prm->hash_bits < 8 || prm->hash_bits > 28)) ||
        (prm->long_bits && (prm->long_bits < 8 || prm->long_bits > 28 || prm->long_chain < 1 ||
                            prm->long_chain > LONG_CHAIN_MAX)))
        return OR_ERR_ARG;
    mlist ml = {0};
    int rc = greedy_parse(in, N, prm, &ml);
    if (rc) { ml_free(&ml); return rc; }
    int64_t n = oracle_serialize(in, N, ml.d, ml.s, ml.L, ml.n, prm, out);
    ml_free(&ml);
    return n;
}

void oracle_free(void *p) { free(p); }

/* ------------------------------------------------------------------------------------------ reading a stream */
typedef struct {
    uint64_t off, end;          /* block extent in the stream */
    uint32_t n_seq, n_match, n_lit, cmd_bytes, len_bytes, w, max_depth, n_tiles;
    uint64_t o_cmd, o_len, o_off, o_lit;  /* absolute section offsets */
} blk_t;

int oracle_peek(const uint8_t *c, uint64_t comp_len, or_info *info) {
    if (!c || !info) return OR_ERR_ARG;
    if (comp_len < 64) return OR_ERR_SIZE;
    if (rd(c, 4) != MAGIC || rd(c + 4, 2) != 1) return OR_ERR_FORMAT;
    uint32_t flags = (uint32_t)rd(c + 6, 2);
    if (flags > 2) return OR_ERR_FORMAT;
    info->flatten = flags;
    info->block_log2 = c[8]; info->tile_log2 = c[9]; info->min_match = c[10];
    if (info->block_log2 < 2 || info->block_log2 > 24 || info->tile_log2 < 2 || info->tile_log2 > info->block_log2 ||
        info->min_match < 1 || c[11] != 0)
        return OR_ERR_FORMAT;
    info->depth_cap = (uint32_t)rd(c + 12, 4);
    info->N = rd(c + 16, 8); info->n_blocks = rd(c + 24, 8); info->comp_len = rd(c + 32, 8);
    info->n_match = rd(c + 40, 8); info->max_depth = (uint32_t)rd(c + 48, 4); info->n_seq = rd(c + 56, 8);
    uint64_t B = 1ull << info->block_log2;
    if (info->n_blocks != (info->N + B - 1) / B) return OR_ERR_FORMAT;
    if (info->comp_len != comp_len || (comp_len & 15)) return OR_ERR_SIZE;
    if (info->n_blocks > (comp_len - 64) / 8) return OR_ERR_FORMAT;
    return OR_OK;
}

static int read_block(const uint8_t *c, const or_info *I, uint64_t b, blk_t *k) {
    uint64_t first = align16(64 + 8 * I->n_blocks);
    k->off = rd(c + 64 + 8 * b, 8);
    k->end = (b + 1 < I->n_blocks) ? rd(c + 64 + 8 * (b + 1), 8) : I->comp_len;
    if ((k->off & 15) || (b == 0 && k->off != first) || k->end <= k->off || k->end > I->comp_len || k->end - k->off < 32)
        return OR_ERR_FORMAT;
    const uint8_t *h = c + k->off;
    k->n_seq = (uint32_t)rd(h, 4); k->n_match = (uint32_t)rd(h + 4, 4); k->n_lit = (uint32_t)rd(h + 8, 4);
    k->cmd_bytes = (uint32_t)rd(h + 12, 4); k->len_bytes = (uint32_t)rd(h + 16, 4); k->w = h[20];
    k->max_depth = (uint32_t)rd(h + 24, 4); k->n_tiles = (uint32_t)rd(h + 28, 4);
    uint64_t B = 1ull << I->block_log2, T = 1ull << I->tile_log2;
    uint64_t b0 = b * B, Nb = (I->N - b0 < B) ? I->N - b0 : B;
    if (k->n_seq < 1 || (k->n_match != k->n_seq && k->n_match + 1 != k->n_seq) || k->w < 1 || k->w > 8 ||
        h[21] || h[22] || h[23] || k->n_tiles != (Nb + T - 1) / T || k->n_lit > Nb)
        return OR_ERR_FORMAT;
    k->o_cmd = k->off + align16(32 + 20 * (uint64_t)k->n_tiles);
    k->o_len = align16(k->o_cmd + k->cmd_bytes);
    k->o_off = align16(k->o_len + k->len_bytes);
    k->o_lit = align16(k->o_off + (uint64_t)k->n_match * k->w);
    if (align16(k->o_lit + k->n_lit) != k->end) return OR_ERR_FORMAT;
    return OR_OK;
}

/*
 * Walks every sequence of every block in order.  If `out` is given, performs the decode of the stream format (§3 of the format):
 * literal run, then the match byte after byte (so a self-overlapping copy repeats its period).  If
 * `seq_r/seq_L/seq_s/lits` are given, lists the sequences instead (seq_L = 0 when the sequence has no
 * match).  Validates every rule of the stream format, sync table included.
 */
static int walk_(const uint8_t *c, const or_info *Ip, uint8_t *out, uint32_t *wd, uint64_t *seq_r, uint64_t *seq_L,
                 uint64_t *seq_s, uint8_t *lits, uint64_t cap_seq, uint64_t *n_seq_out) {
    const or_info I = *Ip;
    int rc, depth_lie = 0;
    const uint64_t B = 1ull << I.block_log2, T = 1ull << I.tile_log2;
    uint64_t si = 0, li = 0, tot_match = 0, tot_seq = 0;
    uint32_t max_depth = 0;
    for (uint64_t b = 0; b < I.n_blocks; b++) {
        blk_t k;
        rc = read_block(c, &I, b, &k);
        if (rc) return rc;
        if (k.max_depth > max_depth) max_depth = k.max_depth;
        tot_match += k.n_match; tot_seq += k.n_seq;
        const uint64_t b0 = b * B, b1 = (I.N - b0 < B) ? I.N : b0 + B;
        uint64_t pos = b0, cp = 0, lp = 0, lt = 0, tile = 0;
        for (uint32_t i = 0; i < k.n_seq; i++) {
            uint64_t cpos0 = cp, lpos0 = lp;
            uint32_t r, Lraw = 0;
            if (get_varint(c + k.o_cmd, k.cmd_bytes, &cp, &r)) return OR_ERR_FORMAT;
            int has_match = i < k.n_match;
            uint64_t L = 0, s = 0;
            if (has_match) {
                if (get_varint(c + k.o_len, k.len_bytes, &lp, &Lraw)) return OR_ERR_FORMAT;
                L = (uint64_t)Lraw + I.min_match;
                s = rd(c + k.o_off + (uint64_t)i * k.w, (int)k.w);
            } else if (r == 0) {
                return OR_ERR_FORMAT;  /* a final sequence without match writes at least one byte */
            }
            uint64_t seq_end = pos + r + L;
            if (seq_end > b1) return OR_ERR_OFFSET;
            if (lt + r > k.n_lit) return OR_ERR_FORMAT;
            /* sync entries of the tiles whose first byte lies in this sequence */
            while (tile < k.n_tiles && b0 + tile * T < seq_end) {
                const uint8_t *e = c + k.off + 32 + 20 * tile;
                if (rd(e, 4) != i || rd(e + 4, 4) != cpos0 || rd(e + 8, 4) != lpos0 || rd(e + 12, 4) != lt ||
                    rd(e + 16, 4) != pos - b0)
                    return OR_ERR_FORMAT;
                tile++;
            }
            if (out) memcpy(out + pos, c + k.o_lit + lt, r);
            if (lits) memcpy(lits + li, c + k.o_lit + lt, r);
            li += r; lt += r; pos += r;
            if (has_match) {
                if (s >= pos) return OR_ERR_OFFSET;
                if (out) for (uint64_t j = 0; j < L; j++) out[pos + j] = out[s + j];
                if (wd) {
                    /* depth (format §4, paper §7.1): 1 + the deepest byte of the effective source; literal
                       bytes are 0 (wd is zero-filled and literal bytes are never rewritten) */
                    uint64_t eff = L < pos - s ? L : pos - s;
                    uint32_t mx = 0;
                    for (uint64_t x = s; x < s + eff; x++) if (wd[x] > mx) mx = wd[x];
                    for (uint64_t j = 0; j < L; j++) wd[pos + j] = mx + 1;
                    if (mx + 1 > k.max_depth) depth_lie = 1;
                }
                pos += L;
            }
            if (seq_r) {
                if (si >= cap_seq) return OR_ERR_SIZE;
                seq_r[si] = r; seq_L[si] = L; seq_s[si] = s;
            }
            si++;
        }
        if (pos != b1 || lt != k.n_lit || cp != k.cmd_bytes || lp != k.len_bytes || tile != k.n_tiles)
            return OR_ERR_FORMAT;
    }
    if (tot_match != I.n_match || tot_seq != I.n_seq || max_depth != I.max_depth) return OR_ERR_FORMAT;
    /* a block whose max_depth is below the depth of one of its matches: the stream is malformed (format §4),
       reported after every other error, as the last check of the stream */
    if (depth_lie) return OR_ERR_DEPTH;
    if (n_seq_out) *n_seq_out = si;
    return OR_OK;
}

/* `out` given: decode, and track every byte's depth to validate the blocks' max_depth fields. */
static int walk(const uint8_t *c, uint64_t comp_len, uint8_t *out, uint64_t out_len, uint64_t *seq_r, uint64_t *seq_L,
                uint64_t *seq_s, uint8_t *lits, uint64_t cap_seq, uint64_t *n_seq_out) {
    or_info I;
    int rc = oracle_peek(c, comp_len, &I);
    if (rc) return rc;
    if (out && I.N != out_len) return OR_ERR_SIZE;
    uint32_t *wd = NULL;
    if (out) {
        wd = (uint32_t *)calloc(I.N ? I.N : 1, sizeof(uint32_t));
        if (!wd) return OR_ERR_NOMEM;
    }
    rc = walk_(c, &I, out, wd, seq_r, seq_L, seq_s, lits, cap_seq, n_seq_out);
    free(wd);
    return rc;
}

int oracle_decode(const uint8_t *comp, uint64_t comp_len, uint8_t *out, uint64_t out_len) {
    if (!comp || (!out && out_len)) return OR_ERR_ARG;
    return walk(comp, comp_len, out ? out : (uint8_t *)"", out_len, NULL, NULL, NULL, NULL, 0, NULL);
}

int64_t oracle_parse(const uint8_t *comp, uint64_t comp_len, uint64_t *seq_r, uint64_t *seq_L, uint64_t *seq_s,
                     uint8_t *lits, uint64_t cap_seq) {
    uint64_t n = 0;
    int rc = walk(comp, comp_len, NULL, 0, seq_r, seq_L, seq_s, lits, cap_seq, &n);
    return rc ? rc : (int64_t)n;
}

/*
 * Textbook LZ77 (§2): a match is (length, distance) measured backward from the current write position.
 * Used on the same parse with dist = d - s to check the absolute-offset decoder (§3.1).
 */
int oracle_lz77_rel_decode(uint64_t n_seq, const uint64_t *r, const uint64_t *L, const uint64_t *dist,
                           const uint8_t *lits, uint8_t *out, uint64_t out_len) {
    uint64_t op = 0, lp = 0;
    for (uint64_t i = 0; i < n_seq; i++) {
        if (op + r[i] + L[i] > out_len) return OR_ERR_SIZE;
        for (uint64_t j = 0; j < r[i]; j++) out[op++] = lits[lp++];
        if (L[i]) {
            if (dist[i] == 0 || dist[i] > op) return OR_ERR_OFFSET;
            for (uint64_t j = 0; j < L[i]; j++) { out[op] = out[op - dist[i]]; op++; }
        }
    }
    return op == out_len ? OR_OK : OR_ERR_SIZE;
}

/* Per-match depth (§7.1) recomputed from the stream by byte-level simulation; returns the match count. */
int64_t oracle_depths(const uint8_t *comp, uint64_t comp_len, uint32_t *depth, uint64_t cap) {
    or_info I;
    int rc = oracle_peek(comp, comp_len, &I);
    if (rc) return rc;
    uint64_t ns = I.n_seq;
    uint64_t *r = (uint64_t *)malloc((ns ? ns : 1) * 8), *L = (uint64_t *)malloc((ns ? ns : 1) * 8),
             *s = (uint64_t *)malloc((ns ? ns : 1) * 8);
    uint8_t *lits = (uint8_t *)malloc(I.N ? I.N : 1);
    uint32_t *wd = (uint32_t *)calloc(I.N ? I.N : 1, 4);
    int64_t res = OR_ERR_NOMEM;
    if (!r || !L || !s || !lits || !wd) goto done;
    res = oracle_parse(comp, comp_len, r, L, s, lits, ns);
    if (res < 0) goto done;
    {
        uint64_t pos = 0, m = 0;
        for (uint64_t i = 0; i < (uint64_t)res; i++) {
            pos += r[i];
            if (L[i]) {
                uint64_t d = pos, eff = L[i] < d - s[i] ? L[i] : d - s[i];
                uint32_t mx = 0;
                for (uint64_t x = s[i]; x < s[i] + eff; x++) if (wd[x] > mx) mx = wd[x];
                for (uint64_t k = 0; k < L[i]; k++) wd[d + k] = mx + 1;
                if (m < cap) depth[m] = mx + 1;
                m++;
                pos += L[i];
            }
        }
        res = (int64_t)m;
    }
done:
    free(r); free(L); free(s); free(lits); free(wd);
    return res;
}

/*
 * Invariants of a stream: 0 when all hold, else the first failing one:
 *   2  a block's max_depth differs from the recomputed one (§7.1)
 *   4  global flattening: a match reads a non-literal byte (§3.3)
 *   5  block flattening: a match reads a non-literal byte of its own block (§3.3)
 *   6  a match deeper than the depth cap (§7.4)
 * negative: the stream does not parse.  Two further invariants need no code of their own: a source that
 * does not precede its destination (§3.1) fails the parse (ERR_OFFSET), and a stream whose max_depth is
 * not the largest block max_depth fails it too (ERR_FORMAT), so once every block passes 2 the stream's
 * max_depth equals the recomputed one.
 */
int oracle_check(const uint8_t *comp, uint64_t comp_len) {
    or_info I;
    int rc = oracle_peek(comp, comp_len, &I);
    if (rc) return rc;
    uint64_t ns = I.n_seq;
    uint64_t *r = (uint64_t *)malloc((ns ? ns : 1) * 8), *L = (uint64_t *)malloc((ns ? ns : 1) * 8),
             *s = (uint64_t *)malloc((ns ? ns : 1) * 8);
    uint8_t *lits = (uint8_t *)malloc(I.N ? I.N : 1), *islit = (uint8_t *)malloc(I.N ? I.N : 1);
    uint32_t *wd = (uint32_t *)calloc(I.N ? I.N : 1, 4);
    int res = OR_ERR_NOMEM;
    if (!r || !L || !s || !lits || !islit || !wd) goto done;
    {
        int64_t n = oracle_parse(comp, comp_len, r, L, s, lits, ns);
        if (n < 0) { res = (int)n; goto done; }
        const uint64_t B = 1ull << I.block_log2;
        uint64_t pos = 0, nb = I.n_blocks;
        uint32_t *bdepth = (uint32_t *)calloc(nb ? nb : 1, 4);
        res = 0;
        for (uint64_t i = 0; i < (uint64_t)n && !res; i++) {
            for (uint64_t j = 0; j < r[i]; j++) { islit[pos + j] = 1; wd[pos + j] = 0; }
            pos += r[i];
            if (!L[i]) continue;
            uint64_t d = pos;
            uint64_t eff = L[i] < d - s[i] ? L[i] : d - s[i];
            uint32_t mx = 0;
            for (uint64_t x = s[i]; x < s[i] + eff; x++) {
                if (wd[x] > mx) mx = wd[x];
                if (I.flatten == 2 && !islit[x]) res = 4;
                if (I.flatten == 1 && !islit[x] && (x / B) == (d / B)) res = 5;
            }
            if (res) break;
            for (uint64_t k = 0; k < L[i]; k++) { wd[d + k] = mx + 1; islit[d + k] = 0; }
            if (mx + 1 > bdepth[d / B]) bdepth[d / B] = mx + 1;
            if (I.depth_cap && mx + 1 > I.depth_cap) res = 6;
            pos += L[i];
        }
        for (uint64_t b = 0; b < nb && !res; b++) {
            blk_t k;
            if (read_block(comp, &I, b, &k)) { res = OR_ERR_FORMAT; break; }
            if (k.max_depth != bdepth[b]) res = 2;
        }
        free(bdepth);
    }
done:
    free(r); free(L); free(s); free(lits); free(islit); free(wd);
    return res;
}

/* ------------------------------------------------------------------------------------------ transcoding */
/*
 * Global chain flattening (§3.3) of an existing stream.  Every output byte has a root: a literal byte is
 * its own root, and byte k of a match with destination d, source s and period p = d - s has the root of
 * byte s + (k mod p) (which precedes d, so roots are settled in decode order).  Each match is rewritten
 * as the maximal runs of its bytes whose roots are consecutive (root of byte k+1 = root of byte k, plus
 * one); a run becomes a match copying from the root of its first byte when it is at least min_match long,
 * else its bytes become literal bytes.  Self-overlapping matches (p < L) are taken first:
 *   - one whose effective source [s, d) is all literal bytes already reads only literal bytes and stays;
 *   - else, when its period is short (p <= 32) and L - p >= min_match, its first period [d, d + p) becomes
 *     literal bytes and the rest a self-overlapping match (d + p, d, L - p) reading them (a repeat whose
 *     source is not literal would otherwise break into a run per period);
 *   - else it is split into runs like any other match.
 * Every match of the result reads literal bytes only, so it has depth 1 (§7.1).
 *
 * The result keeps the input's block_log2, tile_log2 and min_match, has flatten mode 2 and depth cap 0,
 * and decodes to the same bytes.  *out is malloc'ed; returns its length or a negative status (the input
 * is validated by oracle_decode first).
 */
int64_t oracle_transcode_flat(const uint8_t *comp, uint64_t comp_len, uint8_t **out) {
    *out = NULL;
    or_info I;
    int rc = oracle_peek(comp, comp_len, &I);
    if (rc) return rc;
    const uint64_t N = I.N, ns = I.n_seq;
    uint8_t *x = (uint8_t *)malloc(N ? N : 1);
    uint64_t *root = (uint64_t *)malloc((N ? N : 1) * 8);
    uint64_t *r = (uint64_t *)malloc((ns ? ns : 1) * 8), *L = (uint64_t *)malloc((ns ? ns : 1) * 8),
             *s = (uint64_t *)malloc((ns ? ns : 1) * 8);
    mlist ml;
    memset(&ml, 0, sizeof(ml));
    int64_t res = OR_ERR_NOMEM;
    if (!x || !root || !r || !L || !s) goto done;
    rc = oracle_decode(comp, comp_len, x, N);
    if (rc) { res = rc; goto done; }
    {
        const int64_t n = oracle_parse(comp, comp_len, r, L, s, NULL, ns);
        if (n < 0) { res = n; goto done; }
        /* roots, in decode order */
        uint64_t pos = 0;
        for (uint64_t i = 0; i < (uint64_t)n; i++) {
            for (uint64_t j = 0; j < r[i]; j++) root[pos + j] = pos + j;
            pos += r[i];
            const uint64_t d = pos, p = d - s[i];
            for (uint64_t k = 0; k < L[i]; k++) root[d + k] = root[s[i] + k % p];
            pos += L[i];
        }
        /* the rewritten matches, in destination order */
        pos = 0;
        res = 0;
        for (uint64_t i = 0; i < (uint64_t)n && !res; i++) {
            pos += r[i];
            const uint64_t d = pos, p = d - s[i], len = L[i];
            pos += len;
            if (!len) continue;
            if (p < len) {
                int lit_src = 1;
                for (uint64_t j = 0; lit_src && j < p; j++) lit_src = root[s[i] + j] == s[i] + j;
                if (lit_src) { res = ml_push(&ml, d, s[i], (uint32_t)len); continue; }
                if (p <= TRANSCODE_PERIOD_MAX && len - p >= I.min_match) {
                    res = ml_push(&ml, d + p, d, (uint32_t)(len - p));
                    continue;
                }
            }
            uint64_t k0 = 0;
            for (uint64_t k = 1; k <= len && !res; k++) {
                if (k < len && root[d + k] == root[d + k - 1] + 1) continue;
                if (k - k0 >= I.min_match) res = ml_push(&ml, d + k0, root[d + k0], (uint32_t)(k - k0));
                k0 = k;
            }
        }
        if (res) goto done;
        or_params prm;
        memset(&prm, 0, sizeof(prm));
        prm.block_log2 = I.block_log2;
        prm.tile_log2 = I.tile_log2;
        prm.min_match = I.min_match;
        prm.flatten = 2;
        res = oracle_serialize(x, N, ml.d, ml.s, ml.L, ml.n, &prm, out);
    }
done:
    free(x); free(root); free(r); free(L); free(s);
    ml_free(&ml);
    return res;
}
