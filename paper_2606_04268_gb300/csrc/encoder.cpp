// ACEAPEX encoder (host CPU): greedy hash-chain parse with absolute offsets over the whole input (§3.1,
// §3.4), self-contained blocks, chain flattening applied while parsing (§3.3) and an
// optional depth cap (§7.4); output in the ACEAPEX stream format.
//
// Parse rules (deterministic, so that a stream is a pure function of input and parameters):
//   * every position q with q+4 <= N is hashed (4 bytes LE x 2654435761, top hash_bits) and chained;
//     the first position of each hash value is also remembered;
//   * with long_bits set, every position q with q+12 <= N is also chained under a hash of its 12 bytes
//     (8-byte and 4-byte LE words times two odd constants, summed mod 2^64, top long_bits): a key that
//     stays selective on small alphabets such as DNA bases, where 4-byte keys take few values; in flatten
//     modes only literal positions (their own root) enter this chain, so that its candidates start on
//     bytes a flattened match may point at;
//   * candidates at p: up to long_chain most recent positions of the 12-byte chain, then up to chain_limit
//     most recent positions of the 4-byte chain, then the 4-byte hash's first position;
//   * a candidate's length is its common prefix with the input at p, cut at p's block end; in flatten
//     modes it is also cut where the roots of its source bytes stop being consecutive, and the match then
//     points at the first root (a self-overlapping candidate keeps its full length only when its source
//     bytes are their own roots); with a depth cap D it is cut before the first source byte of depth >= D;
//   * lengths below max(min_match, min_emit) are ignored; the longest candidate wins, then the smaller
//     depth, then the earlier candidate;
//   * flatten modes: when the best match is shorter than 32 bytes and the input ahead repeats with a
//     period of at most 16 for at least 32 + 4*period bytes, one period is emitted as literals (the next
//     position then copies it as a self-overlapping match).
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <sys/mman.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/aceapex.h"
#include "layout.h"

namespace {

using aceapex::align16;

constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kPeriodMax = 16, kPeriodRestart = 32, kRing = 16;

// The chain_limit most recent earlier positions of each hash value, most recent first.  Kept as a small
// ring per hash value (one 64-byte line) instead of a linked chain through every position: the candidate
// set and its order are the same, without a dependent cache miss per candidate.
struct alignas(64) Ring {
    uint32_t pos[kRing];
};

// A table of n elements of T, all set to v.  Large tables are placed on 2 MiB boundaries and the kernel is
// asked to back them with huge pages: the parse reads them at random, and with small pages nearly every
// access would also miss the TLB.
template <typename T>
struct Table {
    T *p = nullptr;
    size_t n = 0;
    Table() = default;
    Table(const Table &) = delete;
    Table &operator=(const Table &) = delete;
    ~Table() { free(p); }
    bool init(size_t count, const T &v) {
        free(p);
        p = nullptr;
        n = count;
        const size_t bytes = count * sizeof(T), huge = (size_t)2 << 20;
        void *q = nullptr;
        if (bytes >= huge) {
            if (posix_memalign(&q, huge, (bytes + huge - 1) / huge * huge) != 0) return false;
            madvise(q, (bytes + huge - 1) / huge * huge, MADV_HUGEPAGE);  // a hint: failure changes nothing
        } else {
            q = malloc(bytes ? bytes : 1);
            if (!q) return false;
        }
        p = (T *)q;
        for (size_t i = 0; i < count; i++) p[i] = v;
        return true;
    }
    T &operator[](size_t i) { return p[i]; }
    const T &operator[](size_t i) const { return p[i]; }
};

struct Match {
    uint32_t d, s, L;
};

inline uint32_t load32(const uint8_t *p) {
    uint32_t v;
    memcpy(&v, p, 4);
    return v;  // little-endian host assumed (x86-64, aarch64)
}
inline uint32_t hash4(const uint8_t *p, uint32_t bits) { return (load32(p) * 2654435761u) >> (32 - bits); }
inline uint32_t hash12(const uint8_t *p, uint32_t bits) {
    uint64_t lo;
    memcpy(&lo, p, 8);
    const uint64_t v = lo * 0x9E3779B97F4A7C15ull + (uint64_t)load32(p + 8) * 0xC2B2AE3D27D4EB4Full;
    return (uint32_t)(v >> (64 - bits));
}
constexpr uint32_t kLongKey = 12, kLongMax = 16;

// Common prefix of a[0..) and b[0..), at most lim bytes, 8 bytes at a time.
inline uint32_t common_prefix(const uint8_t *a, const uint8_t *b, uint32_t lim) {
    uint32_t n = 0;
    while (n + 8 <= lim) {
        uint64_t x, y;
        memcpy(&x, a + n, 8);
        memcpy(&y, b + n, 8);
        const uint64_t z = x ^ y;
        if (z) return n + (uint32_t)(__builtin_ctzll(z) >> 3);
        n += 8;
    }
    while (n < lim && a[n] == b[n]) n++;
    return n;
}

struct Parser {
    const uint8_t *in;
    uint32_t N;
    aceapex_enc_params P;
    Table<Ring> ring;
    Table<uint32_t> ring2;  // long-key chain: long_chain most recent positions per hash, most recent first
    Table<uint32_t> first, root, wdepth;
    std::vector<Match> out;

    bool init() {
        try {
            Ring empty;
            for (uint32_t i = 0; i < kRing; i++) empty.pos[i] = kNone;
            if (!ring.init((size_t)1 << P.hash_bits, empty) || !first.init((size_t)1 << P.hash_bits, kNone) ||
                (P.long_bits && !ring2.init((size_t)P.long_chain << P.long_bits, kNone)) || !wdepth.init(N, 0) ||
                (P.flatten && !root.init(N, 0)))
                return false;
            out.reserve(N / 16 + 16);
        } catch (...) {
            return false;
        }
        return true;
    }

    inline uint32_t R(uint32_t x, uint32_t p) const {
        const uint32_t bl = P.block_log2;
        return (P.flatten == 2 || (x >> bl) == (p >> bl)) ? root[x] : x;
    }

    // The hash tables are far larger than the caches and every position is entered in order: while entering
    // q, fetch the buckets of position q + 2 kAhead and the bytes (and roots) of the long-key candidates of
    // q + kAhead, whose bucket was fetched kAhead positions ago, so that their misses overlap.
    static constexpr uint32_t kAhead = 32;
    void prefetch(uint32_t q) {
        const uint32_t q2 = q + 2 * kAhead;
        if ((uint64_t)q2 + kLongKey <= N) {
            const uint32_t h = hash4(in + q2, P.hash_bits);
            __builtin_prefetch(&ring[h], 1);
            __builtin_prefetch(&first[h], 1);
            if (P.long_bits) __builtin_prefetch(&ring2[(size_t)hash12(in + q2, P.long_bits) * P.long_chain], 1);
        }
        const uint32_t q1 = q + kAhead;
        if ((uint64_t)q1 + kLongKey <= N) {
            if (P.long_bits) {
                const uint32_t *r2 = &ring2[(size_t)hash12(in + q1, P.long_bits) * P.long_chain];
                for (uint32_t k = 0; k < P.long_chain && r2[k] != kNone; k++) {
                    __builtin_prefetch(in + r2[k]);
                    if (P.flatten) __builtin_prefetch(&root[r2[k]]);
                }
            }
            const Ring &rg = ring[hash4(in + q1, P.hash_bits)];
            for (uint32_t k = 0; k < P.chain_limit && rg.pos[k] != kNone; k++) __builtin_prefetch(in + rg.pos[k]);
        }
    }

    void insert(uint32_t q) {
        prefetch(q);
        if ((uint64_t)q + 4 > N) return;
        const uint32_t h = hash4(in + q, P.hash_bits);
        Ring &r = ring[h];
        memmove(&r.pos[1], &r.pos[0], sizeof(uint32_t) * (kRing - 1));
        r.pos[0] = q;
        if (first[h] == kNone) first[h] = q;
        if (P.long_bits && (uint64_t)q + kLongKey <= N && (!P.flatten || root[q] == q)) {
            uint32_t *r2 = &ring2[(size_t)hash12(in + q, P.long_bits) * P.long_chain];
            memmove(r2 + 1, r2, sizeof(uint32_t) * (P.long_chain - 1));
            r2[0] = q;
        }
    }

    void run() {
        const uint32_t mm = std::max(P.min_match, P.min_emit), cap = P.depth_cap, bl = P.block_log2;
        const bool flat = P.flatten != 0;
        uint32_t cand[kLongMax + kRing + 1];
        uint32_t p = 0;
        while (p < N) {
            const uint32_t blk_end = (uint32_t)std::min<uint64_t>(((uint64_t)(p >> bl) + 1) << bl, N);
            const uint32_t maxL = blk_end - p;
            uint32_t best_L = 0, best_s = 0, best_dep = 0;
            if (maxL >= mm && (uint64_t)p + 4 <= N) {
                const uint32_t h = hash4(in + p, P.hash_bits);
                uint32_t nc = 0;
                if (P.long_bits && (uint64_t)p + kLongKey <= N) {
                    const uint32_t *r2 = &ring2[(size_t)hash12(in + p, P.long_bits) * P.long_chain];
                    for (uint32_t k = 0; k < P.long_chain && r2[k] != kNone; k++) cand[nc++] = r2[k];
                }
                const Ring &rg = ring[h];
                for (uint32_t k = 0; k < P.chain_limit && rg.pos[k] != kNone; k++) cand[nc++] = rg.pos[k];
                if (P.use_first && first[h] != kNone) cand[nc++] = first[h];
                for (uint32_t j = 0; j < nc; j++) __builtin_prefetch(in + cand[j]);
                for (uint32_t j = 0; j < nc; j++) {
                    const uint32_t c = cand[j];
                    uint32_t Lc = common_prefix(in + c, in + p, maxL), src = c;
                    if (Lc < mm || Lc < best_L) continue;  // cuts below only shorten it: it cannot win
                    if (flat) {
                        const uint32_t r0 = R(c, p);
                        uint32_t k = 1;
                        while (k < Lc && c + k < p && R(c + k, p) == r0 + k) k++;
                        if (k < Lc && c + k == p && r0 == c) k = Lc;
                        Lc = k;
                        src = r0;
                    }
                    uint32_t mx = 0;
                    if (P.flatten != 2) {  // global roots are literal bytes: depth 0, never cut by a cap
                        const uint32_t eff = std::min(Lc, p - src);
                        for (uint32_t x = src; x < src + eff; x++) {
                            if (cap && wdepth[x] >= cap) { Lc = x - src; break; }
                            mx = std::max(mx, wdepth[x]);
                        }
                    }
                    if (Lc < mm || Lc < best_L) continue;
                    if (Lc > best_L || mx + 1 < best_dep) { best_L = Lc; best_s = src; best_dep = mx + 1; }
                }
            }
            uint32_t adv = 1, lits = 1;
            if (flat && best_L < kPeriodRestart) {
                for (uint32_t per = 1; per <= kPeriodMax && (uint64_t)p + per + kPeriodRestart + 4 * per <= blk_end; per++) {
                    const uint32_t run = common_prefix(in + p + per, in + p, blk_end - p - per);
                    if (run >= kPeriodRestart + 4 * per) { lits = per; best_L = 0; break; }
                }
            }
            if (best_L >= mm) {
                out.push_back({p, best_s, best_L});
                const uint32_t per = p - best_s;
                for (uint32_t k = 0, y = 0; k < best_L; k++) {
                    wdepth[p + k] = best_dep;
                    if (flat) root[p + k] = R(best_s + y, p);
                    if (++y == per) y = 0;
                }
                adv = best_L;
            } else {
                for (uint32_t k = 0; k < lits; k++) {
                    wdepth[p + k] = 0;
                    if (flat) root[p + k] = p + k;
                }
                adv = lits;
            }
            for (uint32_t q = p; q < p + adv; q++) insert(q);
            p += adv;
        }
    }
};

inline void put(uint8_t *p, uint64_t v, int n) {
    for (int i = 0; i < n; i++) { p[i] = (uint8_t)v; v >>= 8; }
}
inline uint32_t vsize(uint32_t v) { return v < 0x80 ? 1 : v < 0x4000 ? 2 : v < 0x200000 ? 3 : v < 0x10000000 ? 4 : 5; }
inline uint32_t vput(uint8_t *p, uint32_t v) {
    uint32_t n = 0;
    while (v >= 0x80) { p[n++] = (uint8_t)(v | 0x80); v >>= 7; }
    p[n++] = (uint8_t)v;
    return n;
}
inline uint32_t width_of(uint64_t v) { uint32_t w = 1; while (w < 8 && (v >> (8 * w))) w++; return w; }

// Writes the match list (sorted, literals in between) as a stream.  Depth of every match from the byte
// depths recomputed here (literal 0; match 1 + max over its effective source).
int64_t serialize(const uint8_t *in, uint64_t N, const std::vector<Match> &ms, const aceapex_enc_params &P, void **outp) {
    const uint64_t B = 1ull << P.block_log2, T = 1ull << P.tile_log2;
    const uint64_t nb = (N + B - 1) / B;
    std::vector<uint32_t> mdepth(ms.size());
    {
        std::vector<uint32_t> wd;
        try { wd.assign(N, 0); } catch (...) { return aceapex::kErrNomem; }
        for (size_t m = 0; m < ms.size(); m++) {
            const Match &x = ms[m];
            const uint32_t eff = std::min<uint32_t>(x.L, x.d - x.s);
            uint32_t mx = 0;
            for (uint32_t y = x.s; y < x.s + eff; y++) mx = std::max(mx, wd[y]);
            mdepth[m] = mx + 1;
            std::fill(wd.begin() + x.d, wd.begin() + x.d + x.L, mx + 1);
        }
    }
    struct Blk { size_t m0, m1; uint64_t cmd, len, lit, ns, ntiles, size; uint32_t w, depth; };
    std::vector<Blk> blks(nb);
    uint64_t total = align16(64 + 8 * nb), nseq = 0;
    uint32_t maxd = 0;
    size_t m = 0;
    for (uint64_t b = 0; b < nb; b++) {
        Blk &k = blks[b];
        const uint64_t b0 = b * B, b1 = std::min(b0 + B, N);
        k.m0 = m; k.cmd = k.len = k.lit = 0; k.depth = 0;
        uint64_t pos = b0, maxoff = 0;
        while (m < ms.size() && ms[m].d < b1) {
            k.cmd += vsize((uint32_t)(ms[m].d - pos));
            k.len += vsize(ms[m].L - P.min_match);
            k.lit += ms[m].d - pos;
            maxoff = std::max<uint64_t>(maxoff, ms[m].s);
            k.depth = std::max(k.depth, mdepth[m]);
            pos = (uint64_t)ms[m].d + ms[m].L;
            m++;
        }
        k.m1 = m;
        k.ns = (k.m1 - k.m0) + (pos < b1 ? 1 : 0);
        if (pos < b1) { k.cmd += vsize((uint32_t)(b1 - pos)); k.lit += b1 - pos; }
        k.w = width_of(maxoff);
        k.ntiles = (b1 - b0 + T - 1) / T;
        uint64_t sz = align16(32 + 20 * k.ntiles);
        sz = align16(sz + k.cmd); sz = align16(sz + k.len); sz = align16(sz + (k.m1 - k.m0) * k.w); sz = align16(sz + k.lit);
        k.size = sz;
        total += sz;
        nseq += k.ns;
        maxd = std::max(maxd, k.depth);
    }
    uint8_t *o = (uint8_t *)calloc(total, 1);
    if (!o) return aceapex::kErrNomem;
    put(o, aceapex::kMagic, 4); put(o + 4, 1, 2); put(o + 6, P.flatten, 2);
    o[8] = (uint8_t)P.block_log2; o[9] = (uint8_t)P.tile_log2; o[10] = (uint8_t)P.min_match;
    put(o + 12, P.depth_cap, 4); put(o + 16, N, 8); put(o + 24, nb, 8); put(o + 32, total, 8);
    put(o + 40, ms.size(), 8); put(o + 48, maxd, 4); put(o + 56, nseq, 8);
    uint64_t at = align16(64 + 8 * nb);
    for (uint64_t b = 0; b < nb; b++) {
        const Blk &k = blks[b];
        put(o + 64 + 8 * b, at, 8);
        uint8_t *h = o + at;
        const uint64_t nm = k.m1 - k.m0;
        put(h, k.ns, 4); put(h + 4, nm, 4); put(h + 8, k.lit, 4); put(h + 12, k.cmd, 4); put(h + 16, k.len, 4);
        h[20] = (uint8_t)k.w; put(h + 24, k.depth, 4); put(h + 28, k.ntiles, 4);
        const uint64_t ocmd = align16(32 + 20 * k.ntiles), olen = align16(ocmd + k.cmd), ooff = align16(olen + k.len),
                       olit = align16(ooff + nm * k.w);
        const uint64_t b0 = b * B, b1 = std::min(b0 + B, N);
        uint64_t pos = b0, cp = 0, lp = 0, lt = 0, tile = 0;
        for (uint64_t i = 0; i < k.ns; i++) {
            const bool hm = i < nm;
            const Match *x = hm ? &ms[k.m0 + i] : nullptr;
            const uint64_t r = hm ? x->d - pos : b1 - pos;
            const uint64_t end = pos + r + (hm ? x->L : 0);
            while (tile < k.ntiles && b0 + tile * T < end) {
                uint8_t *e = h + 32 + 20 * tile;
                put(e, i, 4); put(e + 4, cp, 4); put(e + 8, lp, 4); put(e + 12, lt, 4); put(e + 16, pos - b0, 4);
                tile++;
            }
            cp += vput(h + ocmd + cp, (uint32_t)r);
            memcpy(h + olit + lt, in + pos, r);
            lt += r;
            if (hm) {
                lp += vput(h + olen + lp, x->L - P.min_match);
                put(h + ooff + k.w * i, x->s, (int)k.w);
            }
            pos = end;
        }
        at += k.size;
    }
    *outp = o;
    return (int64_t)total;
}

}  // namespace

extern "C" {

int64_t aceapex_encode(const void *in, size_t n, const aceapex_enc_params *params, void **out) {
    if (!out || (!in && n) || !params) return aceapex::kErrArg;
    *out = nullptr;
    aceapex_enc_params P = *params;
    if (!P.hash_bits) P.hash_bits = 20;
    if (n >= 0xFFFFFFFFull || P.block_log2 < 2 || P.block_log2 > 24 || P.tile_log2 < 2 || P.tile_log2 > P.block_log2 ||
        P.min_match < 1 || P.min_match > 255 || P.flatten > 2 || P.chain_limit > kRing || P.hash_bits < 8 ||
        P.hash_bits > 24 ||
        (P.long_bits && (P.long_bits < 8 || P.long_bits > 28 || P.long_chain < 1 || P.long_chain > kLongMax)))
        return aceapex::kErrArg;
    Parser ps;
    ps.in = (const uint8_t *)in;
    ps.N = (uint32_t)n;
    ps.P = P;
    if (!ps.init()) return aceapex::kErrNomem;
    ps.run();
    // release the parse state before serializing
    ps.ring.init(0, Ring{});
    ps.ring2.init(0, 0u);
    ps.first.init(0, 0u);
    ps.root.init(0, 0u);
    ps.wdepth.init(0, 0u);
    return serialize(ps.in, n, ps.out, P, out);
}

void aceapex_free(void *p) { free(p); }

}  // extern "C"
