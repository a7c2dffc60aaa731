// One-pass decode with one warp per tile (tiles of at most 2^kWarpImgLog2 bytes).
//
// Every warp of the persistent grid takes tiles from the global ticket queue and decodes each one alone,
// with warp-synchronous primitives only: no CTA barrier, so 32 or more independent tiles per SM hide
// each other's memory latency.  For each tile:
//
//   phase A: sequences are parsed 32 at a time (lane k <- sequence k of the group): LEB128 values found
//            by a ballot over terminator bytes, output positions and literal offsets by shuffle scans
//            (§3.2: the running position of a sequential decoder); each lane copies its literal run into
//            the warp's shared-memory image of the tile; the image goes to HBM with 16-byte stores and the
//            tile's flag is published.
//   phase B: after every earlier tile of the stream has published (bounded wait), the tile is parsed
//            again (its varints are in L1/L2) with the absolute offsets (§3.1); each lane copies its match
//            out[d+k] = out[s + (k mod (d-s))] into the image -- sources inside the tile from the image,
//            earlier ones from HBM -- and the image is stored again.
//
// Copies of at most 16 bytes are done by their lane: two aligned 16-byte loads, a byte permute to realign,
// predicated byte stores.  Longer literal runs and matches are copied by the whole warp: lanes over bytes,
// or -- from 256 bytes on -- lanes over 16-byte chunks aligned to the image.
#pragma once
#include "decode.h"
#include "tile.cuh"

namespace aceapex {

constexpr int kWarpImgLog2 = 12;   // largest tile of the warp kernel
constexpr int kWarpsPerCta = 4;

struct WarpTile {                   // per-warp tile context (shared memory, written by lane 0)
    const uint8_t *cmd, *len, *off, *lit;
    unsigned long long b0, tile_abs;
    uint32_t Nb, n_seq, n_match, n_lit, cmd_bytes, len_bytes, w, min_match;
    uint32_t lo, hi, shift;
    uint32_t e_seq, e_cmd, e_len, e_lit, e_out;
    uint32_t chk_seq, chk_cmd, chk_len, chk_lit, chk_out, seq_end;
    uint32_t vals[2][32];           // varint hand-off: terminator lane -> lane of its rank
};

struct WarpSmem {
    WarpTile ctx;
    alignas(16) uint8_t img[(1 << kWarpImgLog2) + 32];
};

// ------------------------------------------------------------------------------------------ tile open
// All lanes: read and check the block index entry, block header and the tile's sync entries.  Returns the
// status code; lane 0 fills ctx (the values are uniform, lanes load the same words).
__device__ int warp_tile_open(WarpTile &c, const StreamDesc &sd, uint64_t b, uint32_t j, StreamState *acc) {
    const uint8_t *cp = sd.comp;
    const uint64_t first = align16(kStreamHeader + 8ull * sd.n_blocks);
    const uint64_t boff = ld64(cp + kStreamHeader + 8 * b);
    const uint64_t bend = (b + 1 < sd.n_blocks) ? ld64(cp + kStreamHeader + 8 * (b + 1)) : sd.comp_len;
    if ((boff & 15) || boff < first || (b == 0 && boff != first) || bend <= boff || bend > sd.comp_len ||
        bend - boff < kBlockHeader)
        return kErrFormat;
    const uint8_t *h = cp + boff;
    // lanes 0..7 read the header words; once the header is checked, lanes 0..4 read sync entry j and
    // lanes 5..9 entry j+1 (when present)
    const uint32_t lane = threadIdx.x & 31;
    uint32_t word = lane < 8 ? ld32(h + 4 * lane) : 0u;
    uint32_t f[18];
#pragma unroll
    for (int k = 0; k < 8; k++) f[k] = __shfl_sync(0xffffffffu, word, k);
    const uint32_t n_seq = f[0], n_match = f[1], n_lit = f[2], cmd_bytes = f[3], len_bytes = f[4], word5 = f[5],
                   depth = f[6], n_tiles = f[7];
    const uint32_t w = word5 & 0xFF;
    const uint64_t B = 1ull << sd.block_log2, T = 1ull << sd.tile_log2;
    const uint64_t b0 = b * B, Nb = (sd.N - b0 < B) ? sd.N - b0 : B;
    if (n_seq < 1 || (n_match != n_seq && n_match + 1 != n_seq) || w < 1 || w > 8 || (word5 >> 8) ||
        n_tiles != (Nb + T - 1) / T || n_lit > Nb || j >= n_tiles)
        return kErrFormat;
    const uint64_t o_cmd = boff + align16(kBlockHeader + (uint64_t)kSyncEntry * n_tiles);
    const uint64_t o_len = align16(o_cmd + cmd_bytes), o_off = align16(o_len + len_bytes);
    const uint64_t o_lit = align16(o_off + (uint64_t)n_match * w);
    if (align16(o_lit + n_lit) != bend) return kErrFormat;
    word = 0;
    if (lane < 5) word = ld32(h + kBlockHeader + kSyncEntry * (uint64_t)j + 4 * lane);
    else if (lane < 10 && j + 1 < n_tiles) word = ld32(h + kBlockHeader + kSyncEntry * (uint64_t)(j + 1) + 4 * (lane - 5));
#pragma unroll
    for (int k = 0; k < 10; k++) f[8 + k] = __shfl_sync(0xffffffffu, word, k);
    const uint32_t e_seq = f[8], e_cmd = f[9], e_len = f[10], e_lit = f[11], e_out = f[12];
    const uint32_t lo = (uint32_t)(j * T), hi = (uint32_t)((j + 1) * T < Nb ? (j + 1) * T : Nb);
    if (j == 0 && (e_seq | e_cmd | e_len | e_lit | e_out)) return kErrFormat;
    if (e_seq >= n_seq || e_out > lo || e_cmd > cmd_bytes || e_len > len_bytes || e_lit > n_lit) return kErrFormat;
    uint32_t chk_seq, chk_cmd, chk_len, chk_lit, chk_out, seq_end;
    if (j + 1 < n_tiles) {
        chk_seq = f[13]; chk_cmd = f[14]; chk_len = f[15]; chk_lit = f[16]; chk_out = f[17];
        if (chk_seq < e_seq || chk_seq >= n_seq) return kErrFormat;
        seq_end = chk_seq + 1;
    } else {
        chk_seq = n_seq; chk_cmd = cmd_bytes; chk_len = len_bytes; chk_lit = n_lit; chk_out = (uint32_t)Nb;
        seq_end = n_seq;
    }
    if (lane == 0) {
        c.cmd = cp + o_cmd; c.len = cp + o_len; c.off = cp + o_off; c.lit = cp + o_lit;
        c.b0 = b0; c.tile_abs = b0 + lo; c.Nb = (uint32_t)Nb; c.n_seq = n_seq; c.n_match = n_match; c.n_lit = n_lit;
        c.cmd_bytes = cmd_bytes; c.len_bytes = len_bytes; c.w = w; c.min_match = sd.min_match;
        c.lo = lo; c.hi = hi; c.shift = (uint32_t)((uintptr_t)(sd.out + b0 + lo) & 15);
        c.e_seq = e_seq; c.e_cmd = e_cmd; c.e_len = e_len; c.e_lit = e_lit; c.e_out = e_out;
        c.chk_seq = chk_seq; c.chk_cmd = chk_cmd; c.chk_len = chk_len; c.chk_lit = chk_lit; c.chk_out = chk_out;
        c.seq_end = seq_end;
        if (acc && j == 0) {
            atomicAdd(&acc->seq_sum, (unsigned long long)n_seq);
            atomicAdd(&acc->match_sum, (unsigned long long)n_match);
            atomicMax(&acc->depth_max, depth);
        }
    }
    __syncwarp();
    return kOK;
}

// ------------------------------------------------------------------------------------------ warp varints
// Decode `count` (<= 32) LEB128 values starting at sec[pos]: lane k receives value k.  *start_of receives
// the byte offset of varint `want` (want <= count; == the end when want == count).  Returns the offset
// after the last varint, or -1 on a malformed varint or a short section.
__device__ __forceinline__ int64_t warp_varints(const uint8_t *sec, uint32_t sec_len, uint32_t pos, uint32_t count,
                                                uint32_t *hand, uint32_t want, uint32_t &start_of, uint32_t &val) {
    const uint32_t lane = threadIdx.x & 31;
    uint32_t got = 0;
    val = 0;
    if (want == 0) start_of = pos;
    if (count == 0) return pos;
    {
        // common case: the next `count` bytes are all one-byte varints
        const uint32_t q = pos + lane;
        const uint32_t byte = q < sec_len ? __ldg(sec + q) : 0x80u;
        const uint32_t T = __ballot_sync(0xffffffffu, byte < 0x80u);
        const uint32_t need = count == 32 ? 0xffffffffu : (1u << count) - 1u;
        if ((T & need) == need) {
            val = lane < count ? byte : 0u;
            if (want <= count) start_of = pos + want;
            return pos + count;
        }
    }
    while (got < count) {
        const uint32_t q = pos + lane;
        const uint32_t byte = q < sec_len ? __ldg(sec + q) : 0x80u;
        const uint32_t T = __ballot_sync(0xffffffffu, byte < 0x80u);
        if (T == 0) return -1;  // no terminator in 32 bytes: a varint longer than 5 bytes or a short section
        // value of the varint ending at this lane: its bytes run from the previous terminator + 1
        const uint32_t below = T & ((1u << lane) - 1u);
        const uint32_t vstart = below ? 32 - __clz(below) : 0;  // first byte of this lane's varint
        const uint32_t x = byte & 0x7Fu;
        uint64_t v = 0;
#pragma unroll
        for (int m = 0; m <= 4; m++) {  // terminator (most significant group) first
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, m);
            if (lane >= (uint32_t)m && lane - m >= vstart) v = (v << 7) | y;
        }
        const bool term = (T >> lane) & 1u;
        const uint32_t rank = __popc(below);
        const uint32_t k = __popc(T);
        const uint32_t take = (count - got) < k ? count - got : k;
        bool bad = term && rank < take && (lane - vstart >= 5 || v > 0xFFFFFFFFull);
        if (__any_sync(0xffffffffu, bad)) return -1;
        if (term && rank < take) hand[got + rank] = (uint32_t)v;
        // byte offset of varint `want`: one past the terminator of varint want-1 (rank want-1-got here)
        if (want > got && want <= got + take) {
            const uint32_t bl = __ballot_sync(0xffffffffu, term && rank == want - 1 - got);
            start_of = pos + (uint32_t)__ffs(bl);
        }
        // advance past the last varint taken
        const uint32_t last = __reduce_or_sync(0xffffffffu, (term && rank == take - 1) ? lane : 0u);
        pos += last + 1;
        got += take;
    }
    __syncwarp();
    if (lane < count) val = hand[lane];
    __syncwarp();
    return pos;
}

// ------------------------------------------------------------------------------------------ copies
// Word i (0..3) of v, selected without local-memory indexing.
__device__ __forceinline__ uint32_t pick4(const uint4 &v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }

// Realign: the 16 bytes that start at byte `o` (0..15) of the 32-byte pair (a, b).
__device__ __forceinline__ uint4 realign16(const uint4 &a, const uint4 &b, uint32_t o) {
    const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    const uint32_t base = o >> 2, sel = 0x3210u + 0x1111u * (o & 3u);
    uint32_t r[5];
#pragma unroll
    for (int k = 0; k < 5; k++) {
        uint32_t v = w[k];
#pragma unroll
        for (int m = 1; m < 4; m++) v = base == (uint32_t)m ? w[k + m] : v;
        r[k] = v;
    }
    return make_uint4(__byte_perm(r[0], r[1], sel), __byte_perm(r[1], r[2], sel), __byte_perm(r[2], r[3], sel),
                      __byte_perm(r[3], r[4], sel));
}

// Up to 16 bytes from a global source (read-only stream or decoded output) into the image, one lane.
template <bool COHERENT>
__device__ __forceinline__ void lane_copy_global(uint8_t *dst, const uint8_t *src, uint32_t len) {
    const uintptr_t addr = (uintptr_t)src, al = addr & ~(uintptr_t)15;
    const uint32_t o = (uint32_t)(addr - al);
    const uint4 *g = reinterpret_cast<const uint4 *>(al);
    const uint4 a = COHERENT ? __ldca(g) : __ldg(g);
    uint4 b = make_uint4(0, 0, 0, 0);
    if (o + len > 16) b = COHERENT ? __ldca(g + 1) : __ldg(g + 1);
    const uint4 v = realign16(a, b, o);
    const uint32_t r[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 16; j++)
        if ((uint32_t)j < len) dst[j] = (uint8_t)(r[j >> 2] >> (8 * (j & 3)));
}

// Warp-cooperative copy of `len` bytes dst[0..len) <- src bytes; src_at(k) gives the absolute source of
// byte k for self-overlapping matches (period p < 16); otherwise the source is contiguous.
__device__ __forceinline__ uint8_t fetch_byte(const uint8_t *img_tile, uint64_t tile_abs, const uint8_t *out,
                                              uint64_t src) {
    return src >= tile_abs ? img_tile[src - tile_abs] : __ldca(out + src);
}

// ------------------------------------------------------------------------------------------ kernel
__global__ void __launch_bounds__(32 * kWarpsPerCta) k_flat3(WsHead *head, StreamState *sst, uint32_t *flags,
                                                             const StreamDesc *descs, LaunchArgs a) {
    extern __shared__ uint4 dyn_smem[];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpSmem &ws = reinterpret_cast<WarpSmem *>(dyn_smem)[warp];
    WarpTile &c = ws.ctx;
    const uint32_t epoch = head->epoch;
    unsigned long long ph[kPhases] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long tc = clock64();
#define WPHASE(k) do { if (a.phase && lane == 0) { const long long now = clock64(); ph[k] += now - tc; tc = now; } } while (0)
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(&head->ticket, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= a.total_tiles) break;
        int si = 0;
        if (a.n_streams > 1) {
            if (lane == 0) si = find_stream(descs, a.n_streams, t);
            si = __shfl_sync(0xffffffffu, si, 0);
        }
        const StreamDesc &sd = a.n_streams == 1 ? a.one : descs[si];
        StreamState *st = sd.state ? sd.state : &sst[si];
        const unsigned long long order = t - sd.tile_base + sd.tile_off;
        const uint32_t sh = sd.block_log2 - sd.tile_log2;
        int err = *(volatile int *)&st->status ? 1 : 0;
        err = __shfl_sync(0xffffffffu, err, 0);
        if (!err) err = warp_tile_open(c, sd, order >> sh, (uint32_t)(order & ((1ull << sh) - 1)), st);
        __syncwarp();
        WPHASE(0);
        ph[7] += 1;
        uint8_t *img = ws.img + c.shift;  // img[x - lo] = block-relative byte x
        // ---------------------------------------------------------------- phase A: literals
        for (int pass = 0; pass < 2 && err == 0; pass++) {
            const bool matches = pass == 1;
            if (matches) {
                // wait for the literals of every earlier tile of this stream (bounded)
                unsigned long long f = ld_acquire_u64(&st->front);
                if (f < sd.tile_base) f = sd.tile_base;
                const uint64_t t0 = global_ns();
                bool timed_out = false;
                while (f < t) {
                    const unsigned long long k = f + lane;
                    const bool done = k >= t || ld_acquire_u32(&flags[k]) == epoch;
                    const unsigned ball = __ballot_sync(0xffffffffu, done);
                    if (ball == 0xffffffffu) { f += 32; continue; }
                    f += __ffs(~ball) - 1;
                    if (global_ns() - t0 > a.wait_ns) { timed_out = true; break; }
                    __nanosleep(64);
                }
                if (timed_out) { if (lane == 0) report(st, kErrTimeout, kOrderTimeout); err = kErrTimeout; break; }
                if (lane == 0) atomicMax(&st->front, t < f ? t : f);
                WPHASE(4);
            }
            uint32_t seq = c.e_seq, cmd_pos = c.e_cmd, len_pos = c.e_len, lit_pos = c.e_lit, out_pos = c.e_out;
            const uint32_t seq_end = c.seq_end, lo = c.lo, hi = c.hi;
            while (seq < seq_end) {
                const uint32_t n = (seq_end - seq) < 32u ? seq_end - seq : 32u;
                const uint32_t nm = seq < c.n_match ? ((c.n_match - seq) < n ? c.n_match - seq : n) : 0u;
                const uint32_t want = (c.chk_seq >= seq && c.chk_seq <= seq + n) ? c.chk_seq - seq : 0xFFFFFFFFu;
                uint32_t at_cmd = 0, at_len = 0, r = 0, Lraw = 0;
                const int64_t cp = warp_varints(c.cmd, c.cmd_bytes, cmd_pos, n, c.vals[0], want, at_cmd, r);
                const uint32_t want_l = want <= nm ? want : (want == 0xFFFFFFFFu ? want : nm);
                const int64_t lp = warp_varints(c.len, c.len_bytes, len_pos, nm, c.vals[1], want_l, at_len, Lraw);
                if (cp < 0 || lp < 0) { err = kErrFormat; break; }
                uint64_t L = lane < nm ? (uint64_t)Lraw + c.min_match : 0;
                if (lane >= n) r = 0;
                const bool bad = lane < n && (r > c.Nb || L > c.Nb || r + L == 0);
                // exclusive scans of (r + L) and r
                uint32_t tot = (uint32_t)(r + L), rr = r, ex_tot = tot, ex_r = rr;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y1 = __shfl_up_sync(0xffffffffu, ex_tot, o), y2 = __shfl_up_sync(0xffffffffu, ex_r, o);
                    if (lane >= (uint32_t)o) { ex_tot += y1; ex_r += y2; }
                }
                const uint32_t sum_tot = __shfl_sync(0xffffffffu, ex_tot, 31), sum_r = __shfl_sync(0xffffffffu, ex_r, 31);
                ex_tot -= tot; ex_r -= rr;
                const uint64_t start = (uint64_t)out_pos + ex_tot, loff = (uint64_t)lit_pos + ex_r;
                if (__any_sync(0xffffffffu, bad) || (uint64_t)out_pos + sum_tot > c.Nb || (uint64_t)lit_pos + sum_r > c.n_lit) {
                    err = kErrOffset; break;
                }
                // sync checks: the first sequence holds the tile's first byte; the next entry matches
                if (seq == c.e_seq && __shfl_sync(0xffffffffu, (uint32_t)start + tot, 0) <= lo) { err = kErrFormat; break; }
                if (want != 0xFFFFFFFFu) {
                    const uint32_t lit_at = want < n ? __shfl_sync(0xffffffffu, (uint32_t)loff, want & 31) : lit_pos + sum_r;
                    const uint32_t out_at = want < n ? __shfl_sync(0xffffffffu, (uint32_t)start, want & 31) : out_pos + sum_tot;
                    if (at_cmd != c.chk_cmd || at_len != c.chk_len || lit_at != c.chk_lit || out_at != c.chk_out) {
                        err = kErrFormat; break;
                    }
                }
                // this lane's segment inside the tile: literal run (pass 0) or match (pass 1)
                uint64_t s = 0;
                uint32_t x0, x1;
                if (!matches) {
                    x0 = (uint32_t)(start > lo ? start : lo);
                    x1 = (uint32_t)((start + r) < hi ? start + r : hi);
                } else {
                    const uint64_t d = start + r;
                    x0 = (uint32_t)(d > lo ? d : lo);
                    x1 = (uint32_t)((d + L) < hi ? d + L : hi);
                    if (lane < nm) {
                        // w-byte little-endian field: aligned word loads and a funnel shift (the section is
                        // padded to 16 bytes, so the covering words stay inside the stream)
                        const uintptr_t addr = (uintptr_t)(c.off + (uint64_t)(seq + lane) * c.w);
                        const uint32_t *wp = reinterpret_cast<const uint32_t *>(addr & ~(uintptr_t)3);
                        const uint32_t sh8 = 8 * (uint32_t)(addr & 3);
                        // load only words that hold a byte of the field, so no load leaves the stream
                        const uint32_t span = (uint32_t)(addr & 3) + c.w;
                        const uint32_t w0 = __ldg(wp), w1 = span > 4 ? __ldg(wp + 1) : 0u;
                        uint64_t v = __funnelshift_r(w0, w1, sh8);
                        if (c.w > 4) {
                            const uint32_t w2 = span > 8 ? __ldg(wp + 2) : 0u;
                            v |= (uint64_t)__funnelshift_r(w1, w2, sh8) << 32;
                        }
                        s = c.w >= 8 ? v : (v & ((1ull << (8 * c.w)) - 1));
                        if (s >= c.b0 + d) err = kErrOffset;
                    }
                    if (__any_sync(0xffffffffu, err != 0)) { err = kErrOffset; break; }
                }
                const uint32_t len = (lane < n && x1 > x0) ? x1 - x0 : 0;
                // source of the segment's first byte, and the match period
                uint64_t src0 = 0, per = 0;
                if (!matches) src0 = loff + (x0 - start);
                else if (len) { const uint64_t d = c.b0 + start + r; per = d - s; src0 = s + (c.b0 + x0 - d); }
                const bool contiguous = !matches || per >= (uint64_t)(x0 - (start + r)) + len;  // no wrap
                const bool mine = len > 0 && len <= 16 && contiguous &&
                                  (!matches || src0 + len <= c.tile_abs || src0 >= c.tile_abs);
                if (mine) {
                    uint8_t *dst = img + (x0 - lo);
                    if (!matches) {
                        lane_copy_global<false>(dst, c.lit + src0, len);
                    } else if (src0 >= c.tile_abs) {
                        const uint8_t *sp = img + (src0 - c.tile_abs);
                        for (uint32_t j = 0; j < len; j++) dst[j] = sp[j];
                    } else {
                        lane_copy_global<true>(dst, sd.out + src0, len);
                    }
                }
                // the rest, one segment at a time with the whole warp
                uint32_t todo = __ballot_sync(0xffffffffu, len > 0 && !mine);
                while (todo) {
                    const int l = __ffs(todo) - 1;
                    todo &= todo - 1;
                    const uint32_t X0 = __shfl_sync(0xffffffffu, x0, l), LEN = __shfl_sync(0xffffffffu, len, l);
                    const uint64_t S0 = __shfl_sync(0xffffffffu, src0, l);
                    const uint64_t PER = __shfl_sync(0xffffffffu, per, l);
                    const uint32_t K0 = X0 - (uint32_t)__shfl_sync(0xffffffffu, (uint32_t)(start + r), l);
                    const bool contig = !matches || PER >= (uint64_t)K0 + LEN;
                    const bool from_lit = !matches, from_img = matches && S0 >= c.tile_abs;
                    if (LEN >= 256 && contig && (from_lit || from_img || S0 + LEN <= c.tile_abs)) {
                        // 16-byte chunks aligned to the image: lane g fills image bytes [16g, 16g + 16) of the
                        // segment's span; the first and last chunk are partial and use byte stores
                        const uint32_t d0 = X0 - lo + c.shift, d1 = d0 + LEN;  // image byte range
                        const uint32_t g0 = d0 >> 4, g1 = (d1 + 15) >> 4;
                        const uint8_t *sbase = from_lit ? c.lit + S0 : (from_img ? img + (S0 - c.tile_abs) : sd.out + S0);
                        for (uint32_t g = g0 + lane; g < g1; g += 32) {
                            const uint32_t a0 = g << 4;  // image byte of the chunk start
                            // source of image byte a0 is sbase + (a0 - d0) (may start before the segment)
                            const uint8_t *sp = sbase + ((int64_t)a0 - (int64_t)d0);
                            uint4 v;
                            if (from_img) {
                                // image source: byte loads (the chunk may start before the image)
                                uint32_t wv[4] = {0, 0, 0, 0};
                                for (uint32_t j = 0; j < 16; j++) {
                                    const uint32_t ab = a0 + j;
                                    if (ab >= d0 && ab < d1) wv[j >> 2] |= (uint32_t)sp[j] << (8 * (j & 3));
                                }
                                v = make_uint4(wv[0], wv[1], wv[2], wv[3]);
                            } else {
                                // aligned 16-byte loads that hold at least one byte of the segment's source
                                const uint32_t j0 = a0 < d0 ? d0 - a0 : 0u, j1 = (a0 + 16) > d1 ? d1 - a0 : 16u;
                                const uintptr_t first = (uintptr_t)(sp + j0), al = first & ~(uintptr_t)15;
                                const uint4 *gp = reinterpret_cast<const uint4 *>(al);
                                const uint4 va = from_lit ? __ldg(gp) : __ldca(gp);
                                uint4 vb = make_uint4(0, 0, 0, 0);
                                if ((uintptr_t)(sp + j1 - 1) >= al + 16) vb = from_lit ? __ldg(gp + 1) : __ldca(gp + 1);
                                // realign so that byte j0 of the result is byte (first - al) of (va, vb)
                                const uint32_t o = (uint32_t)(first - al);
                                const uint4 t = realign16(va, vb, o);
                                // t holds source bytes j0.. at positions 0..; shift them to position j0
                                uint32_t wv[4];
                                const uint32_t bs = j0 >> 2, bb = 8 * (j0 & 3);
#pragma unroll
                                for (int k = 0; k < 4; k++) {
                                    const int ia = k - (int)bs, ib = ia - 1;
                                    const uint32_t hiw = ia >= 0 ? pick4(t, ia) : 0u, low = ib >= 0 ? pick4(t, ib) : 0u;
                                    wv[k] = ia < 0 ? 0u : (bb ? __funnelshift_l(low, hiw, bb) : hiw);
                                }
                                v = make_uint4(wv[0], wv[1], wv[2], wv[3]);
                            }
                            if (a0 >= d0 && a0 + 16 <= d1) {
                                *reinterpret_cast<uint4 *>(ws.img + a0) = v;
                            } else {
                                const uint32_t u0 = a0 < d0 ? d0 : a0, u1 = (a0 + 16) < d1 ? a0 + 16 : d1;
                                const uint32_t vw[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                                for (uint32_t j = 0; j < 16; j++)
                                    if (a0 + j >= u0 && a0 + j < u1) ws.img[a0 + j] = (uint8_t)(vw[j >> 2] >> (8 * (j & 3)));
                            }
                        }
                    } else if (!matches) {
                        for (uint32_t j = lane; j < LEN; j += 32) img[X0 - lo + j] = __ldg(c.lit + S0 + j);
                    } else {
                        // match byte k = K0 + j reads s + (k mod PER); S0 = s + K0 when no wrap
                        const uint64_t s_ = S0 - K0;
                        for (uint32_t j = lane; j < LEN; j += 32) {
                            const uint64_t k = K0 + j;
                            const uint64_t srcb = s_ + (k < PER ? k : k % PER);
                            img[X0 - lo + j] = fetch_byte(img, c.tile_abs, sd.out, srcb);
                        }
                    }
                }
                __syncwarp();
                seq += n;
                cmd_pos = (uint32_t)cp;
                len_pos = (uint32_t)lp;
                lit_pos += sum_r;
                out_pos += sum_tot;
            }
            if (err) break;
            WPHASE(matches ? 5 : 1);
            // image -> HBM
            {
                uint8_t *base = sd.out + c.b0 + lo - c.shift;
                const uint32_t total = c.shift + (hi - lo), ng = (total + 15) >> 4;
                for (uint32_t g = lane; g < ng; g += 32) {
                    const uint32_t a0 = g << 4, a1 = a0 + 16;
                    if (a0 >= c.shift && a1 <= total) {
                        *reinterpret_cast<uint4 *>(base + a0) = *reinterpret_cast<const uint4 *>(ws.img + a0);
                    } else {
                        const uint32_t u = a0 > c.shift ? a0 : c.shift, z = a1 < total ? a1 : total;
                        for (uint32_t x = u; x < z; x++) base[x] = ws.img[x];
                    }
                }
            }
            if (!matches) {
                __threadfence();
                __syncwarp();
                if (lane == 0 && t != a.withhold) st_release_u32(&flags[t], epoch);
                __syncwarp();
                WPHASE(3);
            } else {
                WPHASE(6);
            }
        }
        if (err) {
            if (lane == 0) {
                if (err < 0 && err != kErrTimeout) report(st, err, order);
                // a tile that failed before publishing still publishes, so that no later tile waits on it
                st_release_u32(&flags[t], epoch);
            }
        }
        __syncwarp();
    }
    if (a.phase && lane == 0)
        for (int k = 0; k < kPhases; k++) atomicAdd(&a.phase[k], ph[k]);
#undef WPHASE
}

}  // namespace aceapex
