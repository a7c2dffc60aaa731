/*
 * Seeded synthetic inputs shaped like the paper's workloads (§4.2: a Wikipedia-XML text corpus and
 * whole-genome FASTQ reads).  None of those datasets is reproduced: only their statistical shape is
 * mimicked, from seeded pseudo-random tables.  This module holds no codec arithmetic; both the oracle
 * and the GPU decoder's tests and benchmark draw their inputs from it.
 *
 * Every generator is deterministic for a given seed on one platform.  Generators that use libm
 * (log/pow/cos) may differ in rare last-ulp decisions across C libraries, so no stored test value is
 * derived from their output.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- PRNG: splitmix64 + xoshiro256** */
typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static void rng_seed(rng_t *r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; i++) r->s[i] = splitmix64(&x);
}
static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static inline uint64_t rng_next(rng_t *r) {
    uint64_t *s = r->s;
    uint64_t res = rotl(s[1] * 5, 7) * 9, t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3]; s[2] ^= t; s[3] = rotl(s[3], 45);
    return res;
}
static inline double rng_unit(rng_t *r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }
static inline uint32_t rng_below(rng_t *r, uint32_t n) { return (uint32_t)(((rng_next(r) >> 32) * (uint64_t)n) >> 32); }
static double rng_gauss(rng_t *r) {
    double u1 = rng_unit(r), u2 = rng_unit(r);
    if (u1 < 1e-300) u1 = 1e-300;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* ---------------------------------------------------------------- uniform random bytes */
void synth_random(uint64_t seed, uint8_t *out, size_t n) {
    rng_t r; rng_seed(&r, seed ^ 0x52414E44ull);
    size_t i = 0;
    for (; i + 8 <= n; i += 8) { uint64_t v = rng_next(&r); memcpy(out + i, &v, 8); }
    if (i < n) { uint64_t v = rng_next(&r); memcpy(out + i, &v, n - i); }
}

/* ---------------------------------------------------------------- period-7 motif with 0.1 % mutations */
void synth_rle7(uint64_t seed, uint8_t *out, size_t n) {
    rng_t r; rng_seed(&r, seed ^ 0x524C4537ull);
    uint8_t motif[7];
    for (int i = 0; i < 7; i++) motif[i] = (uint8_t)rng_next(&r);
    for (size_t i = 0; i < n; i++) out[i] = motif[i % 7];
    /* mutate about 0.1 % of the bytes: geometric gaps with mean 1000 */
    size_t p = 0;
    for (;;) {
        double u = rng_unit(&r);
        if (u < 1e-12) u = 1e-12;
        size_t gap = (size_t)(-log(u) * 1000.0);
        p += gap + 1;
        if (p >= n) break;
        out[p] = (uint8_t)rng_next(&r);
    }
}

/* ---------------------------------------------------------------- order-2 Markov text with Zipf(1.1) word reuse */
#define MK_SYM 96
static uint8_t mk_char(int i) { return i == 95 ? (uint8_t)'\n' : (uint8_t)(0x20 + i); }
static int mk_index(uint8_t c) { return c == '\n' ? 95 : (c >= 0x20 && c < 0x7F ? c - 0x20 : 0); }

void synth_markov_text(uint64_t seed, uint8_t *out, size_t n) {
    rng_t r; rng_seed(&r, seed ^ 0x4D4B5632ull);
    /* cumulative transition weights per context (a, b): skewed weights u^8 give a few likely successors */
    uint32_t *cdf = (uint32_t *)malloc(sizeof(uint32_t) * MK_SYM * MK_SYM * MK_SYM);
    for (int ctx = 0; ctx < MK_SYM * MK_SYM; ctx++) {
        double w[MK_SYM], tot = 0.0;
        for (int j = 0; j < MK_SYM; j++) {
            double u = rng_unit(&r);
            w[j] = u * u * u * u * u * u * u * u;
            if (j == 0) w[j] += 1.5;  /* space: words of ~7 symbols on average */
            tot += w[j];
        }
        double acc = 0.0;
        for (int j = 0; j < MK_SYM; j++) {
            acc += w[j] / tot;
            uint64_t v = (uint64_t)(acc * 4294967295.0);
            cdf[(size_t)ctx * MK_SYM + j] = (uint32_t)(v > 0xFFFFFFFFull ? 0xFFFFFFFFull : v);
        }
        cdf[(size_t)ctx * MK_SYM + MK_SYM - 1] = 0xFFFFFFFFu;
    }
    /* growing word list */
    size_t cap_words = 1u << 16, n_words = 0, pool_cap = 1u << 20, pool_used = 0;
    uint32_t *w_off = (uint32_t *)malloc(sizeof(uint32_t) * cap_words);
    uint8_t *w_len = (uint8_t *)malloc(cap_words);
    uint8_t *pool = (uint8_t *)malloc(pool_cap);
    int a = 0, b = 0;
    size_t pos = 0;
    while (pos < n) {
        if (n_words > 0 && rng_unit(&r) < 0.5) {
            /* reuse: rank ~ Zipf(1.1) over the list in order of first appearance */
            double s = 1.1, u = rng_unit(&r);
            double hi = pow((double)n_words + 1.0, 1.0 - s);
            size_t k = (size_t)pow(1.0 + u * (hi - 1.0), 1.0 / (1.0 - s));
            if (k < 1) k = 1;
            if (k > n_words) k = n_words;
            k -= 1;
            for (uint32_t t = 0; t < w_len[k] && pos < n; t++) out[pos++] = pool[w_off[k] + t];
            if (pos < n) out[pos++] = ' ';
            a = mk_index(pool[w_off[k] + w_len[k] - 1]); b = 0;
        } else {
            /* new word from the Markov source, ended by a space or newline (at most 20 symbols) */
            uint8_t word[21]; int wl = 0;
            for (;;) {
                uint32_t u = (uint32_t)(rng_next(&r) >> 32);
                const uint32_t *row = cdf + ((size_t)a * MK_SYM + b) * MK_SYM;
                int j = 0;
                while (j < MK_SYM - 1 && row[j] < u) j++;
                a = b; b = j;
                uint8_t c = mk_char(j);
                if (pos < n) out[pos++] = c;
                if (c == ' ' || c == '\n' || wl == 20) break;
                word[wl++] = c;
            }
            if (wl > 0 && n_words < cap_words && pool_used + (size_t)wl <= pool_cap) {
                w_off[n_words] = (uint32_t)pool_used; w_len[n_words] = (uint8_t)wl;
                memcpy(pool + pool_used, word, (size_t)wl);
                pool_used += (size_t)wl; n_words++;
            }
        }
    }
    free(cdf); free(w_off); free(w_len); free(pool);
}

/* ---------------------------------------------------------------- English-like text: Zipf(1.0) vocabulary */
#define ZT_VOCAB 200000
typedef struct {
    uint64_t seed;
    double *cdf;          /* ZT_VOCAB cumulative Zipf(1.0) probabilities */
    uint32_t *guide;      /* guide[i] = first rank whose cdf >= i / 2^16 */
    uint32_t *off;        /* word start in pool */
    uint8_t *len;
    uint8_t *pool;
    uint32_t *succ;       /* 4 favourite successors per word: bigram structure */
    char **markup;        /* invented markup tokens */
    int n_markup;
} zt_tables;

typedef struct zt_node { zt_tables *t; struct zt_node *next; } zt_node;
static pthread_mutex_t g_lock = PTHREAD_MUTEX_INITIALIZER;
static zt_node *g_zt = NULL;  /* table sets by seed; built once, kept until exit */

static uint32_t zipf_draw(const double *cdf, uint32_t n, double u) {
    uint32_t lo = 0, hi = n - 1;
    while (lo < hi) { uint32_t mid = (lo + hi) >> 1; if (cdf[mid] < u) lo = mid + 1; else hi = mid; }
    return lo;
}
static uint32_t zipf_draw_g(const zt_tables *t, double u) {
    uint32_t g = (uint32_t)(u * 65536.0);
    uint32_t lo = t->guide[g], hi = (g + 1 < 65536) ? t->guide[g + 1] : ZT_VOCAB - 1;
    const double *cdf = t->cdf;
    while (lo < hi) { uint32_t mid = (lo + hi) >> 1; if (cdf[mid] < u) lo = mid + 1; else hi = mid; }
    return lo;
}

static zt_tables *zt_get(uint64_t vocab_seed) {
    pthread_mutex_lock(&g_lock);
    for (zt_node *q = g_zt; q; q = q->next)
        if (q->t->seed == vocab_seed) { pthread_mutex_unlock(&g_lock); return q->t; }
    zt_tables *t = (zt_tables *)calloc(1, sizeof(zt_tables));
    t->seed = vocab_seed;
    rng_t r; rng_seed(&r, vocab_seed ^ 0x564F4341ull);
    /* unigram letter distribution: an English-like profile, perturbed by the seed */
    static const double base[26] = {8.2, 1.5, 2.8, 4.3, 12.7, 2.2, 2.0, 6.1, 7.0, 0.15, 0.77, 4.0, 2.4,
                                    6.7, 7.5, 1.9, 0.095, 6.0, 6.3, 9.1, 2.8, 0.98, 2.4, 0.15, 2.0, 0.074};
    double lc[26], tot = 0.0;
    for (int i = 0; i < 26; i++) { lc[i] = base[i] * (0.6 + 0.8 * rng_unit(&r)); tot += lc[i]; }
    double acc = 0.0;
    for (int i = 0; i < 26; i++) { acc += lc[i] / tot; lc[i] = acc; }
    lc[25] = 1.0;
    t->cdf = (double *)malloc(sizeof(double) * ZT_VOCAB);
    double h = 0.0;
    for (int i = 0; i < ZT_VOCAB; i++) { h += 1.0 / (double)(i + 1); t->cdf[i] = h; }
    for (int i = 0; i < ZT_VOCAB; i++) t->cdf[i] /= h;
    t->cdf[ZT_VOCAB - 1] = 1.0;
    t->guide = (uint32_t *)malloc(sizeof(uint32_t) * 65536);
    for (uint32_t g = 0, k = 0; g < 65536; g++) {
        while (k < ZT_VOCAB - 1 && t->cdf[k] < (double)g / 65536.0) k++;
        t->guide[g] = k;
    }
    t->off = (uint32_t *)malloc(sizeof(uint32_t) * ZT_VOCAB);
    t->len = (uint8_t *)malloc(ZT_VOCAB);
    t->pool = (uint8_t *)malloc((size_t)ZT_VOCAB * 12);
    size_t used = 0;
    for (int i = 0; i < ZT_VOCAB; i++) {
        int L = 2 + (int)rng_below(&r, 11);  /* uniform 2..12 */
        t->off[i] = (uint32_t)used; t->len[i] = (uint8_t)L;
        for (int k = 0; k < L; k++) {
            double u = rng_unit(&r);
            int c = 0;
            while (c < 25 && lc[c] < u) c++;
            t->pool[used++] = (uint8_t)('a' + c);
        }
    }
    t->succ = (uint32_t *)malloc(sizeof(uint32_t) * 4 * ZT_VOCAB);
    for (int i = 0; i < 4 * ZT_VOCAB; i++) t->succ[i] = zipf_draw(t->cdf, ZT_VOCAB, rng_unit(&r));
    /* invented markup: tags, brackets, pipes, entity-like sequences */
    static const char *fixed[] = {"[[", "]]", "{{", "}}", "|", "&amp;", "&quot;", "&lt;br&gt;", "'''", "''",
                                  "==", "<ref>", "</ref>", "<tt>", "</tt>", "* ", "#"};
    int nf = (int)(sizeof(fixed) / sizeof(fixed[0]));
    t->n_markup = nf + 24;
    t->markup = (char **)malloc(sizeof(char *) * (size_t)t->n_markup);
    for (int i = 0; i < nf; i++) t->markup[i] = strdup(fixed[i]);
    for (int i = nf; i < t->n_markup; i++) {
        char buf[32]; int L = 3 + (int)rng_below(&r, 6), k = 0;
        buf[k++] = '<';
        if (rng_below(&r, 2)) buf[k++] = '/';
        for (int j = 0; j < L; j++) buf[k++] = (char)('a' + rng_below(&r, 26));
        buf[k++] = '>'; buf[k] = 0;
        t->markup[i] = strdup(buf);
    }
    zt_node *node = (zt_node *)malloc(sizeof(zt_node));
    node->t = t; node->next = g_zt; g_zt = node;
    pthread_mutex_unlock(&g_lock);
    return t;
}

typedef struct { uint8_t *out; size_t n, pos; } sink_t;
static inline void put(sink_t *s, uint8_t c) { if (s->pos < s->n) s->out[s->pos++] = c; }
static inline void puts_(sink_t *s, const uint8_t *p, size_t L) {
    size_t k = s->n - s->pos < L ? s->n - s->pos : L;
    memcpy(s->out + s->pos, p, k); s->pos += k;
}

void synth_zipf_text(uint64_t vocab_seed, uint64_t seed, uint8_t *out, size_t n) {
    zt_tables *t = zt_get(vocab_seed);
    rng_t r; rng_seed(&r, seed ^ 0x5A495046ull);
    sink_t s = {out, n, 0};
    uint32_t prev = 0;
    while (s.pos < n) {
        int words = 5 + (int)rng_below(&r, 26);  /* sentence of 5..30 words */
        for (int w = 0; w < words && s.pos < n; w++) {
            if (rng_unit(&r) < 0.05) {  /* markup-like token */
                const char *m = t->markup[rng_below(&r, (uint32_t)t->n_markup)];
                puts_(&s, (const uint8_t *)m, strlen(m));
                if (rng_below(&r, 2)) {
                    uint32_t k = zipf_draw_g(t, rng_unit(&r));
                    puts_(&s, t->pool + t->off[k], t->len[k]);
                }
            } else {
                uint32_t k;
                if (w > 0 && rng_unit(&r) < 0.35) k = t->succ[4 * prev + rng_below(&r, 4)];
                else k = zipf_draw_g(t, rng_unit(&r));
                prev = k;
                const uint8_t *p = t->pool + t->off[k];
                if (w == 0) { put(&s, (uint8_t)(p[0] - 32)); puts_(&s, p + 1, t->len[k] - 1u); }
                else puts_(&s, p, t->len[k]);
            }
            if (w + 1 < words) {
                if (rng_unit(&r) < 0.08) put(&s, ',');
                put(&s, ' ');
            }
        }
        double u = rng_unit(&r);
        put(&s, u < 0.8 ? '.' : (u < 0.9 ? '?' : '!'));
        if (rng_unit(&r) < 0.15) { put(&s, '\n'); put(&s, '\n'); } else put(&s, ' ');
    }
}

/* ---------------------------------------------------------------- FASTQ-like reads */
#define FQ_SEGS 64
#define FQ_SEGLEN (1u << 20)
#define FQ_READ 150
typedef struct {
    uint64_t seed;
    uint8_t *ref;               /* FQ_SEGS × FQ_SEGLEN bases */
    uint8_t qtab[FQ_READ][1024]; /* per-position inverse CDF of the quality score */
} fq_tables;
typedef struct fq_node { fq_tables *t; struct fq_node *next; } fq_node;
static fq_node *g_fq = NULL;  /* table sets by seed; built once, kept until exit */

static fq_tables *fq_get(uint64_t ref_seed) {
    pthread_mutex_lock(&g_lock);
    for (fq_node *q = g_fq; q; q = q->next)
        if (q->t->seed == ref_seed) { pthread_mutex_unlock(&g_lock); return q->t; }
    fq_tables *t = (fq_tables *)calloc(1, sizeof(fq_tables));
    t->seed = ref_seed;
    rng_t r; rng_seed(&r, ref_seed ^ 0x46415351ull);
    size_t total = (size_t)FQ_SEGS * FQ_SEGLEN;
    t->ref = (uint8_t *)malloc(total);
    static const uint8_t acgt[4] = {'A', 'C', 'G', 'T'};
    for (size_t i = 0; i < total; i += 32) {
        uint64_t v = rng_next(&r);
        for (int k = 0; k < 32 && i + k < total; k++) t->ref[i + k] = acgt[(v >> (2 * k)) & 3];
    }
    /* Phred score at position i ~ round(N(mean_i, 3)), mean declining from 31 to 28, clipped to [2, 41] */
    for (int i = 0; i < FQ_READ; i++) {
        double mean = 31.0 - 3.0 * (double)i / (double)(FQ_READ - 1);
        double cdf[42], acc = 0.0;
        for (int q = 0; q <= 41; q++) {
            double lo = (q == 2) ? -1e9 : (double)q - 0.5, hi = (q == 41) ? 1e9 : (double)q + 0.5;
            double p = (q < 2) ? 0.0 : 0.5 * (erf((hi - mean) / (3.0 * sqrt(2.0))) - erf((lo - mean) / (3.0 * sqrt(2.0))));
            acc += p; cdf[q] = acc;
        }
        for (int j = 0; j < 1024; j++) {
            double u = ((double)j + 0.5) / 1024.0 * acc;
            int q = 2;
            while (q < 41 && cdf[q] < u) q++;
            t->qtab[i][j] = (uint8_t)(q + 33);
        }
    }
    fq_node *node = (fq_node *)malloc(sizeof(fq_node));
    node->t = t; node->next = g_fq; g_fq = node;
    pthread_mutex_unlock(&g_lock);
    return t;
}

void synth_fastq(uint64_t ref_seed, uint64_t seed, uint8_t *out, size_t n) {
    fq_tables *t = fq_get(ref_seed);
    rng_t r; rng_seed(&r, seed ^ 0x52454144ull);
    sink_t s = {out, n, 0};
    static const uint8_t acgt[4] = {'A', 'C', 'G', 'T'};
    uint64_t id = 1, next_sub = 0;
    char hdr[64];
    while (s.pos < n) {
        uint32_t seg = rng_below(&r, FQ_SEGS);
        uint32_t at = rng_below(&r, FQ_SEGLEN - FQ_READ);
        /* header: '@' + name + incrementing id */
        int hl = 0;
        const char *pre = "@SYNTH.";
        while (pre[hl]) { hdr[hl] = pre[hl]; hl++; }
        char num[24]; int nl = 0; uint32_t sv = seg;
        do { num[nl++] = (char)('0' + sv % 10); sv /= 10; } while (sv);
        while (nl) hdr[hl++] = num[--nl];
        hdr[hl++] = '.';
        uint64_t iv = id++;
        do { num[nl++] = (char)('0' + iv % 10); iv /= 10; } while (iv);
        while (nl) hdr[hl++] = num[--nl];
        hdr[hl++] = '\n';
        puts_(&s, (const uint8_t *)hdr, (size_t)hl);
        /* 150 bases copied from the reference with 1 % substitutions */
        uint8_t bases[FQ_READ + 1];
        memcpy(bases, t->ref + (size_t)seg * FQ_SEGLEN + at, FQ_READ);
        /* substitutions at geometric gaps (rate 1 %), carried across reads */
        while (next_sub < FQ_READ) {
            int i = (int)next_sub;
            int cur = bases[i] == 'A' ? 0 : bases[i] == 'C' ? 1 : bases[i] == 'G' ? 2 : 3;
            bases[i] = acgt[(cur + 1 + (int)rng_below(&r, 3)) & 3];
            double u = rng_unit(&r);
            if (u < 1e-12) u = 1e-12;
            next_sub += 1 + (uint64_t)(-log(u) * 99.5);
        }
        next_sub -= FQ_READ;
        bases[FQ_READ] = '\n';
        puts_(&s, bases, FQ_READ + 1);
        put(&s, '+'); put(&s, '\n');
        uint8_t qual[FQ_READ + 1];
        for (int i = 0; i < FQ_READ; i += 6) {
            uint64_t v = rng_next(&r);
            for (int k = 0; k < 6 && i + k < FQ_READ; k++) qual[i + k] = t->qtab[i + k][(v >> (10 * k)) & 1023];
        }
        qual[FQ_READ] = '\n';
        puts_(&s, qual, FQ_READ + 1);
    }
}

/* ---------------------------------------------------------------- Box-Muller, exported for size sampling tests */
double synth_gauss(uint64_t seed) { rng_t r; rng_seed(&r, seed); return rng_gauss(&r); }
