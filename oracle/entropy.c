/*
 * Entropy container of the ACEAPEX stream format (format §6) -- TEST INFRASTRUCTURE ONLY, part of the CPU
 * oracle (same rules as oracle.c: only tests, the smoke check and the benchmark's CPU legs use it; it
 * shares no code with the GPU library).
 *
 * The paper names an entropy stage (an FSE stage after the four arrays, §6) without fixing one.  The
 * container read here wraps a stream byte for byte: segments of at most 4096 bytes, each stored or coded
 * with a canonical Huffman code of at most 12-bit codes, 32 interleaved lanes per segment.
 *
 *   oracle_huff_lengths     code lengths from symbol counts: Huffman's construction (repeatedly merge the
 *                           two lightest trees), then lengths above 12 cut and the Kraft sum restored
 *   oracle_entropy_encode   wraps a stream: stored stream header, block index, block headers and sync
 *                           tables; each block section (cmd, len, off, lit) coded with its own code, chunked
 *                           at 4096 bytes; a chunk is stored when coding would not make it smaller
 *   oracle_entropy_decode   the definition of the wrapped bytes: every field checked, every lane decoded bit
 *                           by bit against the canonical code
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define E_MAGIC 0x45454341u
#define E_SEG 4096
#define E_MAXLEN 12
#define E_LANES 32
#define E_ERR_ARG (-1)
#define E_ERR_FORMAT (-2)
#define E_ERR_SIZE (-3)
#define E_ERR_NOMEM (-7)

static uint64_t e_rd(const uint8_t *p, int n) {
    uint64_t v = 0;
    for (int i = n - 1; i >= 0; i--) v = (v << 8) | p[i];
    return v;
}
static void e_wr(uint8_t *p, uint64_t v, int n) {
    for (int i = 0; i < n; i++) p[i] = (uint8_t)(v >> (8 * i));
}
static uint64_t e_align16(uint64_t x) { return (x + 15) & ~(uint64_t)15; }

/* ------------------------------------------------------------------------------------------ code lengths */
/*
 * Huffman's construction over the symbols with nonzero count: repeatedly merge the two lightest trees
 * (ties: the tree created first; leaves are created in symbol order before any merged tree); a symbol's
 * length is its leaf depth.  A single symbol gets length 1.  Lengths above 12 are then set to 12 and, while
 * the Kraft sum sum 2^(12 - len) exceeds 2^12, the longest code below 12 (ties: the smaller count, then
 * the larger symbol) is made one bit longer.  Returns the number of symbols with a code.
 */
int oracle_huff_lengths(const uint64_t *count, uint8_t *len) {
    uint64_t w[511];
    int parent[511], alive[511], n = 0, used = 0;
    memset(len, 0, 256);
    for (int s = 0; s < 256; s++) {
        w[s] = count[s];
        parent[s] = -1;
        alive[s] = count[s] > 0;
        used += alive[s];
    }
    if (used == 0) return 0;
    if (used == 1) {
        for (int s = 0; s < 256; s++) if (count[s]) len[s] = 1;
        return 1;
    }
    n = 256;
    for (int merges = 0; merges < used - 1; merges++) {
        int a = -1, b = -1;
        for (int i = 0; i < n; i++) {
            if (!alive[i]) continue;
            if (a < 0 || w[i] < w[a]) { b = a; a = i; }
            else if (b < 0 || w[i] < w[b]) b = i;
        }
        w[n] = w[a] + w[b];
        parent[n] = -1;
        alive[n] = 1;
        parent[a] = n;
        parent[b] = n;
        alive[a] = alive[b] = 0;
        n++;
    }
    for (int s = 0; s < 256; s++) {
        if (!count[s]) continue;
        int d = 0;
        for (int x = s; parent[x] >= 0; x = parent[x]) d++;
        len[s] = (uint8_t)(d > E_MAXLEN ? E_MAXLEN : d);
    }
    for (;;) {
        uint64_t kraft = 0;
        for (int s = 0; s < 256; s++) if (len[s]) kraft += 1ull << (E_MAXLEN - len[s]);
        if (kraft <= (1ull << E_MAXLEN)) break;
        int best = -1;
        for (int s = 0; s < 256; s++) {
            if (!len[s] || len[s] >= E_MAXLEN) continue;
            if (best < 0 || len[s] > len[best] || (len[s] == len[best] && count[s] <= count[best])) best = s;
        }
        len[best]++;
    }
    return used;
}

/* Canonical codes of lengths len[] (format §6.3): symbols ordered by (length, value), consecutive codes. */
static void canon_codes(const uint8_t *len, uint32_t *code) {
    uint32_t c = 0;
    int prev = 0, first = 1;
    for (int L = 1; L <= E_MAXLEN; L++) {
        for (int s = 0; s < 256; s++) {
            if (len[s] != L) continue;
            if (first) { c = 0; first = 0; }
            else c = (c + 1) << (L - prev);
            prev = L;
            code[s] = c;
        }
    }
}

/* ------------------------------------------------------------------------------------------ encoder */
typedef struct { uint64_t a, b; int coded; } region_t;

typedef struct { uint8_t *p; uint64_t n, cap; } buf_t;
static int buf_put(buf_t *b, const void *src, uint64_t n) {
    if (b->n + n > b->cap) {
        uint64_t c = b->cap ? b->cap : 1 << 16;
        while (c < b->n + n) c *= 2;
        uint8_t *q = (uint8_t *)realloc(b->p, c);
        if (!q) return E_ERR_NOMEM;
        b->p = q;
        b->cap = c;
    }
    if (src) memcpy(b->p + b->n, src, n);
    else memset(b->p + b->n, 0, n);
    b->n += n;
    return 0;
}

/* Regions of a wrapped ACEAPEX stream: stored header and index, per block its stored header and sync
   table, then its four sections coded (one code each).  Anything that does not parse is one coded region. */
static int stream_regions(const uint8_t *raw, uint64_t n, region_t **out, int *nr) {
    int cap = 16, k = 0;
    region_t *r = (region_t *)malloc(sizeof(region_t) * cap);
    if (!r) return E_ERR_NOMEM;
#define ADD(A, B, C)                                                                      \
    do {                                                                                  \
        if ((B) > (A)) {                                                                  \
            if (k == cap) {                                                               \
                region_t *q = (region_t *)realloc(r, sizeof(region_t) * (cap *= 2));      \
                if (!q) { free(r); return E_ERR_NOMEM; }                                  \
                r = q;                                                                    \
            }                                                                             \
            r[k].a = (A); r[k].b = (B); r[k].coded = (C); k++;                            \
        }                                                                                 \
    } while (0)
    int ok = n >= 64 && e_rd(raw, 4) == 0x58454341u;
    uint64_t nb = ok ? e_rd(raw + 24, 8) : 0;
    uint64_t first = e_align16(64 + 8 * nb);
    if (ok && (nb > n / 8 || first > n)) ok = 0;
    for (uint64_t b = 0; ok && b < nb; b++) {
        /* blocks follow each other from the end of the index to the end of the stream */
        uint64_t off = e_rd(raw + 64 + 8 * b, 8), end = b + 1 < nb ? e_rd(raw + 64 + 8 * (b + 1), 8) : n;
        if ((b == 0 && off != first) || end > n || end < off + 32) { ok = 0; break; }
        const uint8_t *h = raw + off;
        uint64_t tiles = e_rd(h + 28, 4), cmd = e_rd(h + 12, 4), lenb = e_rd(h + 16, 4), w = h[20], nm = e_rd(h + 4, 4);
        uint64_t o_cmd = off + e_align16(32 + 20 * tiles), o_len = e_align16(o_cmd + cmd), o_off = e_align16(o_len + lenb);
        uint64_t o_lit = e_align16(o_off + nm * w);
        if (o_lit > end) { ok = 0; break; }
    }
    if (!ok) {
        ADD(0, n, 1);
    } else {
        ADD(0, first, 0);
        for (uint64_t b = 0; b < nb; b++) {
            uint64_t off = e_rd(raw + 64 + 8 * b, 8), end = b + 1 < nb ? e_rd(raw + 64 + 8 * (b + 1), 8) : n;
            const uint8_t *h = raw + off;
            uint64_t tiles = e_rd(h + 28, 4), cmd = e_rd(h + 12, 4), lenb = e_rd(h + 16, 4), w = h[20], nm = e_rd(h + 4, 4);
            uint64_t o_cmd = off + e_align16(32 + 20 * tiles), o_len = e_align16(o_cmd + cmd), o_off = e_align16(o_len + lenb);
            uint64_t o_lit = e_align16(o_off + nm * w);
            ADD(off, o_cmd, 0);
            ADD(o_cmd, o_len, 1);
            ADD(o_len, o_off, 1);
            ADD(o_off, o_lit, 1);
            ADD(o_lit, end, 1);
        }
    }
#undef ADD
    *out = r;
    *nr = k;
    return 0;
}

/* Bits of one lane of a coded segment: bytes l, l+32, ... of seg[0, n), codes MSB first. */
static uint64_t lane_bits(const uint8_t *seg, uint64_t n, int l, const uint8_t *len) {
    uint64_t bits = 0;
    for (uint64_t j = (uint64_t)l; j < n; j += E_LANES) bits += len[seg[j]];
    return bits;
}
static void lane_pack(const uint8_t *seg, uint64_t n, int l, const uint8_t *len, const uint32_t *code, uint8_t *out) {
    uint64_t bit = 0;
    for (uint64_t j = (uint64_t)l; j < n; j += E_LANES) {
        const int L = len[seg[j]];
        for (int i = L - 1; i >= 0; i--, bit++)
            if ((code[seg[j]] >> i) & 1u) out[bit / 8] |= (uint8_t)(0x80u >> (bit % 8));
    }
}

int64_t oracle_entropy_encode(const uint8_t *raw, uint64_t raw_len, uint8_t **out) {
    *out = NULL;
    if (!raw && raw_len) return E_ERR_ARG;
    region_t *reg = NULL;
    int nr = 0, rc = 0;
    if (raw_len && (rc = stream_regions(raw, raw_len, &reg, &nr))) return rc;
    /* segments: every region cut at 4096 bytes */
    uint64_t n_seg = 0;
    for (int i = 0; i < nr; i++) n_seg += (reg[i].b - reg[i].a + E_SEG - 1) / E_SEG;
    uint64_t *raw_off = (uint64_t *)malloc(8 * (n_seg + 1)), *e_off = (uint64_t *)malloc(8 * (n_seg + 1));
    buf_t pay = {0};
    if (!raw_off || !e_off) { free(reg); free(raw_off); free(e_off); return E_ERR_NOMEM; }
    const uint64_t base = e_align16(64 + 16 * n_seg);
    uint64_t k = 0;
    for (int i = 0; i < nr && !rc; i++) {
        uint8_t len[256];
        uint32_t code[256];
        uint64_t cnt[256] = {0};
        for (uint64_t x = reg[i].a; x < reg[i].b; x++) cnt[raw[x]]++;
        oracle_huff_lengths(cnt, len);
        canon_codes(len, code);
        int64_t table_seg = -1;  /* segment carrying this region's code */
        for (uint64_t a = reg[i].a; a < reg[i].b && !rc; a += E_SEG, k++) {
            const uint64_t n = reg[i].b - a < E_SEG ? reg[i].b - a : E_SEG;
            const uint8_t *seg = raw + a;
            raw_off[k] = a;
            e_off[k] = base + pay.n;
            uint64_t lb[E_LANES], coded = 8 + (table_seg < 0 ? 128 : 0) + 2 * E_LANES;
            for (int l = 0; l < E_LANES; l++) { lb[l] = (lane_bits(seg, n, l, len) + 7) / 8; coded += lb[l]; }
            uint8_t hdr[8] = {0};
            if (!reg[i].coded || coded >= 8 + n) {
                rc = buf_put(&pay, hdr, 8);
                if (!rc) rc = buf_put(&pay, seg, n);
            } else {
                if (table_seg < 0) table_seg = (int64_t)k;
                hdr[0] = 1;
                e_wr(hdr + 4, (uint64_t)table_seg, 4);
                rc = buf_put(&pay, hdr, 8);
                if (!rc && table_seg == (int64_t)k) {
                    uint8_t nib[128];
                    for (int s = 0; s < 128; s++) nib[s] = (uint8_t)(len[2 * s] | (len[2 * s + 1] << 4));
                    rc = buf_put(&pay, nib, 128);
                }
                for (int l = 0; l < E_LANES && !rc; l++) {
                    uint8_t b2[2];
                    e_wr(b2, lb[l], 2);
                    rc = buf_put(&pay, b2, 2);
                }
                for (int l = 0; l < E_LANES && !rc; l++) {
                    const uint64_t at = pay.n;
                    rc = buf_put(&pay, NULL, lb[l]);
                    if (!rc) lane_pack(seg, n, l, len, code, pay.p + at);
                }
            }
            if (!rc) rc = buf_put(&pay, NULL, e_align16(pay.n) - pay.n);
        }
    }
    free(reg);
    if (rc) { free(raw_off); free(e_off); free(pay.p); return rc; }
    const uint64_t e_len = base + pay.n;
    uint8_t *o = (uint8_t *)calloc(e_len ? e_len : 1, 1);
    if (!o) { free(raw_off); free(e_off); free(pay.p); return E_ERR_NOMEM; }
    e_wr(o, E_MAGIC, 4); e_wr(o + 4, 1, 2); e_wr(o + 12, E_MAXLEN, 4);
    e_wr(o + 16, raw_len, 8); e_wr(o + 24, n_seg, 8); e_wr(o + 32, e_len, 8);
    for (uint64_t i = 0; i < n_seg; i++) { e_wr(o + 64 + 16 * i, raw_off[i], 8); e_wr(o + 72 + 16 * i, e_off[i], 8); }
    if (pay.n) memcpy(o + base, pay.p, pay.n);
    free(raw_off); free(e_off); free(pay.p);
    *out = o;
    return (int64_t)e_len;
}

/* ------------------------------------------------------------------------------------------ decoder */
/* Header of a container: raw_len and n_seg; ERR_FORMAT / ERR_SIZE as the format says. */
int oracle_entropy_peek(const uint8_t *e, uint64_t e_len, uint64_t *raw_len, uint64_t *n_seg) {
    if (!e) return E_ERR_ARG;
    if (e_len < 64 || (e_len & 15)) return E_ERR_SIZE;
    if (e_rd(e, 4) != E_MAGIC || e_rd(e + 4, 2) != 1 || e_rd(e + 6, 2) != 0 || e_rd(e + 8, 4) != 0 ||
        e_rd(e + 12, 4) != E_MAXLEN)
        return E_ERR_FORMAT;
    for (int i = 40; i < 64; i++) if (e[i]) return E_ERR_FORMAT;
    if (e_rd(e + 32, 8) != e_len) return E_ERR_SIZE;
    const uint64_t rl = e_rd(e + 16, 8), ns = e_rd(e + 24, 8);
    if ((rl == 0) != (ns == 0) || ns > rl || ns > (e_len - 64) / 16) return E_ERR_FORMAT;
    *raw_len = rl;
    *n_seg = ns;
    return 0;
}

/* Code lengths of a coded segment's table (the payload of segment t), checked: at most 12, Kraft sum at
   most 2^12, at least one code. */
static int read_lengths(const uint8_t *e, uint64_t e_len, uint64_t n_seg, uint64_t t, uint8_t *len) {
    const uint64_t eo = e_rd(e + 72 + 16 * t, 8), ee = t + 1 < n_seg ? e_rd(e + 72 + 16 * (t + 1), 8) : e_len;
    if (ee < eo + 8 + 128 || e[eo] != 1 || e_rd(e + eo + 4, 4) != t) return E_ERR_FORMAT;
    uint64_t kraft = 0;
    for (int s = 0; s < 256; s++) {
        len[s] = (uint8_t)((e[eo + 8 + s / 2] >> (4 * (s & 1))) & 15);
        if (len[s] > E_MAXLEN) return E_ERR_FORMAT;
        if (len[s]) kraft += 1ull << (E_MAXLEN - len[s]);
    }
    if (kraft == 0 || kraft > (1ull << E_MAXLEN)) return E_ERR_FORMAT;
    return 0;
}

/* The wrapped stream (raw_len bytes into raw).  Segments in order; lanes decoded bit by bit: a code is
   read one bit at a time until the bits read are the code of some symbol (canonical code, format §6.3). */
int oracle_entropy_decode(const uint8_t *e, uint64_t e_len, uint8_t *raw, uint64_t raw_len) {
    uint64_t rl = 0, ns = 0;
    int rc = oracle_entropy_peek(e, e_len, &rl, &ns);
    if (rc) return rc;
    if (rl != raw_len) return E_ERR_SIZE;
    if (!raw && raw_len) return E_ERR_ARG;
    for (uint64_t k = 0; k < ns; k++) {
        const uint64_t ro = e_rd(e + 64 + 16 * k, 8), eo = e_rd(e + 72 + 16 * k, 8);
        const uint64_t re = k + 1 < ns ? e_rd(e + 64 + 16 * (k + 1), 8) : rl;
        const uint64_t ee = k + 1 < ns ? e_rd(e + 72 + 16 * (k + 1), 8) : e_len;
        if ((k == 0 && (ro != 0 || eo != e_align16(64 + 16 * ns))) || re <= ro || re - ro > E_SEG || re > rl ||
            (eo & 15) || ee <= eo || ee > e_len || ee - eo < 8)
            return E_ERR_FORMAT;
        const uint64_t n = re - ro, P = ee - eo;
        const uint8_t *q = e + eo;
        const uint32_t mode = q[0], table = (uint32_t)e_rd(q + 4, 4);
        if (q[1] || q[2] || q[3] || mode > 1) return E_ERR_FORMAT;
        if (mode == 0) {
            if (table != 0 || P < 8 + n) return E_ERR_FORMAT;
            memcpy(raw + ro, q + 8, n);
            continue;
        }
        if (table > k) return E_ERR_FORMAT;
        uint8_t len[256];
        if ((rc = read_lengths(e, e_len, ns, table, len))) return rc;
        /* the canonical code per length: first code, number of codes, and the symbols in code order */
        uint32_t first[E_MAXLEN + 2] = {0}, cnt[E_MAXLEN + 2] = {0}, base[E_MAXLEN + 2] = {0};
        uint8_t sorted[256];
        int ns_sorted = 0;
        for (int L = 1; L <= E_MAXLEN; L++) {
            base[L] = (uint32_t)ns_sorted;
            for (int s = 0; s < 256; s++) if (len[s] == L) { sorted[ns_sorted++] = (uint8_t)s; cnt[L]++; }
        }
        for (int L = 1, c = 0; L <= E_MAXLEN; L++) {
            c = (c + (int)cnt[L - 1]) << 1;
            first[L] = (uint32_t)c;
        }
        const uint64_t lb_at = 8 + (table == k ? 128 : 0);
        if (P < lb_at + 2 * E_LANES) return E_ERR_FORMAT;
        uint64_t at = lb_at + 2 * E_LANES, sum = 0;
        for (int l = 0; l < E_LANES; l++) sum += e_rd(q + lb_at + 2 * l, 2);
        if (P < at + sum) return E_ERR_FORMAT;
        for (int l = 0; l < E_LANES; l++) {
            const uint64_t nbytes = e_rd(q + lb_at + 2 * l, 2), nbits = 8 * nbytes;
            const uint8_t *bits = q + at;
            uint64_t bit = 0;
            for (uint64_t j = (uint64_t)l; j < n; j += E_LANES) {
                uint32_t c = 0;
                int L = 0, sym = -1;
                while (sym < 0) {
                    if (L == E_MAXLEN || bit >= nbits) return E_ERR_FORMAT;
                    c = (c << 1) | ((bits[bit / 8] >> (7 - bit % 8)) & 1u);
                    bit++;
                    L++;
                    if (c - first[L] < cnt[L]) sym = sorted[base[L] + c - first[L]];
                }
                raw[ro + j] = (uint8_t)sym;
            }
            at += nbytes;
        }
    }
    return 0;
}
