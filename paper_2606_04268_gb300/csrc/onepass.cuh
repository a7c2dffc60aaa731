// One-pass decode with one warp per tile (tiles of at most 4 KiB), sections staged in shared memory by the
// bulk-copy engine and copies merged into the tile image word by word.
//
// A stream whose matches are all of depth 1 reads literal bytes only (§3.3, §7.1), so two passes per tile
// decode it:
//
//   stage   lane 0 issues cp.async.bulk copies of the tile's ranges of cmd[], len[], off[] and lit[] (§3.2)
//           into the warp's shared memory, completing on the warp's mbarrier; meanwhile the warp clears its
//           image of the tile and the tile's literal bitmap;
//   pass A  sequences are parsed 32 at a time from the staged bytes (lane k <- sequence k of the group:
//           LEB128 values by a ballot over terminator bytes, output positions by shuffle scans, §3.2); each
//           lane ORs the part of its literal run that falls in the tile into the zeroed image, a 16-byte piece
//           at a time (five aligned word ORs per piece, no byte stores), and marks those bytes in the tile's
//           literal bitmap (one bit per output byte); the image and the bitmap go to HBM and the tile's flag
//           is published;
//   pass B  the staged varints are parsed again with the absolute offsets (§3.1); each lane waits (bounded)
//           until the tiles holding its match's source bytes have published their literals -- only those
//           tiles, so no tile waits on the slowest of all earlier ones -- checks that every source byte is
//           a literal byte (a match that reads a match byte has depth >= 2, which the stream's
//           max_depth <= 1 denies: ACEAPEX_ERR_DEPTH), and ORs its match into the image, reading the source
//           bytes from HBM; the image is stored again.
//
// Pieces: a lane copies the first 16 bytes of its segment itself; the later pieces of longer segments are
// dealt round-robin to all lanes (exclusive scan of the piece counts, binary search for the owner).  A
// self-overlapping match (source period p < length) is copied byte-exactly by splitting each piece at the
// period boundaries: byte k of the match reads s + (k mod p).
//
// Sections that do not fit the stage, or a group whose bytes lie outside the staged ranges (possible only in
// a malformed stream), are read from global memory instead, with the same results.  Positions are 32-bit:
// streams of up to ~4 GiB of output (kF4MaxN).
#pragma once
#include "warp_tile.cuh"

namespace aceapex {

constexpr uint32_t kF4Warps = 4;                              // warps per CTA
constexpr uint32_t kF4Stage = 5120;                           // staged section bytes per warp
constexpr uint32_t kF4Slack = 48;                             // readable bytes after the staged data
constexpr uint32_t kF4LitCap = (1u << kWarpImgLog2) + 512;    // literal window staged per tile
constexpr uint32_t kFull = 0xffffffffu;
constexpr unsigned long long kF4MaxN = kOnePassMaxN;       // streams up to ~4 GiB: positions fit 32 bits
static_assert(kWarpImgLog2 == (int)kOnePassMaxTileLog2, "one warp per tile of at most 4 KiB");

constexpr uint32_t kF4Img = (1u << kWarpImgLog2) + 32;       // image: alignment shift + tile + slack
constexpr uint32_t kF4LbmWords = kF4Img / 32 + 4;

struct alignas(16) F4Warp {
    WarpTile c;                                               // tile context, varint hand-off
    unsigned long long mbar;                                  // completion of the staging copies
    uint32_t pad_[2];
    alignas(16) uint8_t stage[kF4Stage + kF4Slack];
    alignas(16) uint8_t img[kF4Img];
    uint32_t lbm[kF4LbmWords];                                // bit i: image byte i is a literal byte
};

// ------------------------------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *m) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(m)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *m, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *m, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(m)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bulk copy global -> this CTA's shared memory; dst, src and bytes are multiples of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, unsigned long long *m) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(m))
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ------------------------------------------------------------------------------------------ word ORs
// OR window bytes [a, a + len) into the image words d[0..4]; u0..u5 are consecutive source words and window
// byte i sits at bit 8 * (i + sh/8) of the 192-bit value u5:...:u0 (sh in {0, 8, 16, 24}).  Bytes outside
// the window are masked off, so the neighbours' bytes of a shared word stay as they are.
__device__ __forceinline__ void or_window(uint32_t *d, uint32_t a, uint32_t len, uint32_t u0, uint32_t u1,
                                          uint32_t u2, uint32_t u3, uint32_t u4, uint32_t u5, uint32_t sh) {
    const uint32_t nb = a + len;  // window end, 1..19
    uint32_t w = __funnelshift_r(u0, u1, sh) & (0xFFFFFFFFu << (8 * a));
    atomicOr(d, w & __funnelshift_lc(0xFFFFFFFFu, 0u, 8 * nb));
    if (nb > 4) atomicOr(d + 1, __funnelshift_r(u1, u2, sh) & __funnelshift_lc(0xFFFFFFFFu, 0u, 8 * (nb - 4)));
    if (nb > 8) atomicOr(d + 2, __funnelshift_r(u2, u3, sh) & __funnelshift_lc(0xFFFFFFFFu, 0u, 8 * (nb - 8)));
    if (nb > 12) atomicOr(d + 3, __funnelshift_r(u3, u4, sh) & __funnelshift_lc(0xFFFFFFFFu, 0u, 8 * (nb - 12)));
    if (nb > 16) atomicOr(d + 4, __funnelshift_r(u4, u5, sh) & __funnelshift_lc(0xFFFFFFFFu, 0u, 8 * (nb - 16)));
}

// Piece from shared memory: `so` is the byte offset of the source inside the warp's F4Warp (which is 16-byte
// aligned, so word boundaries of `base` are shared-memory word boundaries).  Reads at most 6 bytes before
// and 24 bytes after the source, all inside the warp's F4Warp.
__device__ __forceinline__ void or_piece_smem(const uint32_t *base, uint32_t *imgw, uint32_t ib, uint32_t so,
                                              uint32_t len) {
    const uint32_t a = ib & 3u;
    const uint32_t P = so - a;  // window byte 0
    const uint32_t *s = base + (P >> 2);
    or_window(imgw + (ib >> 2), a, len, s[0], s[1], s[2], s[3], s[4], s[5], 8 * (P & 3u));
}

// Piece from global memory: bytes base[off .. off + len).  Loads only the aligned 16-byte blocks (and at
// most one word of a third) that hold a byte of that range; the address arithmetic is 32-bit relative to
// base's 16-byte aligned floor.  NC: read-only data (the compressed stream); else decoded output of this
// launch, read through L2.
template <bool NC>
__device__ __forceinline__ void or_piece_glob(uint32_t *imgw, uint32_t ib, const uint8_t *base, uint32_t off,
                                              uint32_t len) {
    const uint32_t a = ib & 3u;
    const uint32_t ba = (uint32_t)(uintptr_t)base & 15u;
    const uint8_t *abase = base - ba;
    const int32_t g = (int32_t)(ba + off) - (int32_t)a;   // window byte 0, relative to abase
    const int32_t al = g & ~15;
    const uint32_t o = (uint32_t)(g - al);               // window byte i is byte o + i of the blocks at al
    const int32_t s0 = (int32_t)(ba + off), s1 = s0 + (int32_t)len;
    const uint4 *p = reinterpret_cast<const uint4 *>(abase + al);
    uint4 b0 = make_uint4(0, 0, 0, 0), b1 = make_uint4(0, 0, 0, 0);
    uint32_t b2 = 0;
    if (s0 < al + 16) b0 = NC ? __ldg(p) : __ldcg(p);
    if (s1 > al + 16 && s0 < al + 32) b1 = NC ? __ldg(p + 1) : __ldcg(p + 1);
    if (s1 > al + 32) {
        const uint32_t *q = reinterpret_cast<const uint32_t *>(abase + al + 32);
        b2 = NC ? __ldg(q) : __ldcg(q);
    }
    // words w[q .. q + 5] with q = o >> 2 in 0..3, by a two-stage shifter
    const uint32_t q = o >> 2;
    uint32_t t0, t1, t2, t3, t4, t5, t6;
    if (q & 2) { t0 = b0.z; t1 = b0.w; t2 = b1.x; t3 = b1.y; t4 = b1.z; t5 = b1.w; t6 = b2; }
    else       { t0 = b0.x; t1 = b0.y; t2 = b0.z; t3 = b0.w; t4 = b1.x; t5 = b1.y; t6 = b1.z; }
    uint32_t u0, u1, u2, u3, u4, u5;
    if (q & 1) { u0 = t1; u1 = t2; u2 = t3; u3 = t4; u4 = t5; u5 = t6; }
    else       { u0 = t0; u1 = t1; u2 = t2; u3 = t3; u4 = t4; u5 = t5; }
    or_window(imgw + (ib >> 2), a, len, u0, u1, u2, u3, u4, u5, 8 * (o & 3u));
}

// ------------------------------------------------------------------------------------------ varints
// Lane k receives byte pos + k of a section (0x80 past its end) from the staged copy when the 32 bytes lie
// in the staged range [slo, shi) (or past the section end), else from global memory.
__device__ __forceinline__ uint32_t f4_window(const uint8_t *g, const uint8_t *stg, uint32_t slo, uint32_t shi,
                                              uint32_t sec_len, uint32_t pos) {
    const uint32_t lane = threadIdx.x & 31, q = pos + lane;
    uint32_t byte = 0x80u;
    if (pos >= slo && (pos + 32 <= shi || shi >= sec_len)) {
        if (q < sec_len) byte = stg[q - slo];
    } else {
        if (q < sec_len) byte = __ldg(g + q);
    }
    return byte;
}

// Decode `count` (<= 32) LEB128 values starting at section offset pos: lane k receives value k.
// *start_of receives the byte offset of varint `want` (want <= count; == the end when want == count).
// Returns the offset after the last varint, or -1 on a malformed varint or a short section.
__device__ __forceinline__ int64_t f4_varints(const uint8_t *g, const uint8_t *stg, uint32_t slo, uint32_t shi,
                                              uint32_t sec_len, uint32_t pos, uint32_t count, uint32_t *hand,
                                              uint32_t want, uint32_t &start_of, uint32_t &val) {
    const uint32_t lane = threadIdx.x & 31;
    val = 0;
    if (want == 0) start_of = pos;
    if (count == 0) return pos;
    uint32_t byte = f4_window(g, stg, slo, shi, sec_len, pos);
    uint32_t T = __ballot_sync(kFull, byte < 0x80u);
    {
        // common case: the next `count` bytes are all one-byte varints
        const uint32_t need = count == 32 ? kFull : (1u << count) - 1u;
        if ((T & need) == need) {
            val = lane < count ? byte : 0u;
            if (want <= count) start_of = pos + want;
            return pos + count;
        }
    }
    uint32_t got = 0;
    for (;;) {
        if (T == 0) return -1;  // no terminator in 32 bytes: a varint longer than 5 bytes or a short section
        const uint32_t below = T & ((1u << lane) - 1u);
        const uint32_t vstart = below ? 32 - __clz(below) : 0;  // first byte of this lane's varint
        const uint32_t x = byte & 0x7Fu;
        uint64_t v = 0;
#pragma unroll
        for (int m = 0; m <= 4; m++) {  // terminator (most significant group) first
            const uint32_t y = __shfl_up_sync(kFull, x, m);
            if (lane >= (uint32_t)m && lane - m >= vstart) v = (v << 7) | y;
        }
        const bool term = (T >> lane) & 1u;
        const uint32_t rank = __popc(below);
        const uint32_t k = __popc(T);
        const uint32_t take = (count - got) < k ? count - got : k;
        const bool bad = term && rank < take && (lane - vstart >= 5 || v > 0xFFFFFFFFull);
        if (__any_sync(kFull, bad)) return -1;
        if (term && rank < take) hand[got + rank] = (uint32_t)v;
        if (want > got && want <= got + take) {
            const uint32_t bl = __ballot_sync(kFull, term && rank == want - 1 - got);
            start_of = pos + (uint32_t)__ffs(bl);
        }
        const uint32_t last = __reduce_or_sync(kFull, (term && rank == take - 1) ? lane : 0u);
        pos += last + 1;
        got += take;
        if (got >= count) break;
        byte = f4_window(g, stg, slo, shi, sec_len, pos);
        T = __ballot_sync(kFull, byte < 0x80u);
    }
    __syncwarp();
    if (lane < count) val = hand[lane];
    __syncwarp();
    return pos;
}

// Owner of round-robin piece i: the largest lane k with ex_k <= i (ex non-decreasing over lanes).
__device__ __forceinline__ uint32_t f4_owner(uint32_t ex, uint32_t i) {
    uint32_t k = 0;
#pragma unroll
    for (uint32_t st = 16; st; st >>= 1) {
        const uint32_t e = __shfl_sync(kFull, ex, k + st);
        if (e <= i) k += st;
    }
    return k;
}

// Rarely taken paths are kept out of line (not inlined at each call site), which keeps the kernel's hot loop
// small in the instruction cache: literals read from global memory (a section larger than the stage) and the
// period-split copy of a self-overlapping match.
__device__ __noinline__ void or_piece_lit_glob(uint32_t *imgw, uint32_t ib, const uint8_t *base, uint32_t off,
                                              uint32_t len) {
    or_piece_glob<true>(imgw, ib, base, off, len);
}
// Byte k of a self-overlapping match reads s + (k mod p): the piece is split at the period boundaries.
__device__ __noinline__ void f4_match_wrap(uint32_t *imgw, uint32_t ib, const uint8_t *out, uint32_t s, uint32_t p,
                                           uint32_t k, uint32_t len) {
    uint32_t r = k % p;
    while (len) {
        const uint32_t c = (p - r) < len ? p - r : len;
        or_piece_glob<false>(imgw, ib, out, s + r, c);
        ib += c; len -= c;
        r += c; if (r == p) r = 0;
    }
}
// Match bytes [k, k + len) of a match with source s and period p (p >= length: no wrap) into the image.
__device__ __forceinline__ void f4_match_piece(uint32_t *imgw, uint32_t ib, const uint8_t *out, uint32_t s,
                                               uint32_t p, uint32_t k, uint32_t len, bool wrap) {
    if (!wrap) or_piece_glob<false>(imgw, ib, out, s + k, len);
    else f4_match_wrap(imgw, ib, out, s, p, k, len);
}

// ------------------------------------------------------------------------------------------ literal bits
// Mark image bytes [ib, ib + n) (n <= 32) as literal bytes.
__device__ __forceinline__ void f4_mark(uint32_t *lbm, uint32_t ib, uint32_t n) {
    const uint32_t q = ib >> 5, o = ib & 31u;
    const unsigned long long m = (n >= 32 ? 0xFFFFFFFFull : ((1ull << n) - 1)) << o;
    atomicOr(&lbm[q], (uint32_t)m);
    if (m >> 32) atomicOr(&lbm[q + 1], (uint32_t)(m >> 32));
}

// Bits [a, b) (a < b) of a bit array all set: GLOB reads the array through L2 (written by other warps of
// this launch), else from shared memory.  Bit positions are stream positions, below kF4MaxN < 2^32.
template <bool GLOB>
__device__ __forceinline__ bool f4_bits(const uint32_t *w, uint32_t a, uint32_t b) {
    const uint32_t q0 = a >> 5, q1 = (b - 1) >> 5;
    bool ok = true;
    for (uint32_t q = q0; q <= q1 && ok; q++) {
        const uint32_t lo = q == q0 ? (uint32_t)(a & 31u) : 0u, hi = q == q1 ? (uint32_t)((b - 1) & 31u) + 1 : 32u;
        const uint32_t m = __funnelshift_lc(0xFFFFFFFFu, 0u, hi) & ~__funnelshift_lc(0xFFFFFFFFu, 0u, lo);
        const uint32_t v = GLOB ? __ldcg(w + q) : w[q];
        ok = (v & m) == m;
    }
    return ok;
}

// The slow part of a match's wait for its source tiles, out of line (most matches find their sources
// published at the first look): poll the flags of stream tiles [need, need_hi] (flag of tile u at fl[u - toff])
// every 64 ns until all lanes' tiles are published, or until wait_ns has passed (kErrTimeout).
__device__ __noinline__ int f4_wait_slow(const uint32_t *fl, uint32_t toff, uint32_t need, uint32_t need_hi,
                                         uint32_t epoch, unsigned long long wait_ns) {
    const uint64_t t0 = global_ns();
    for (;;) {
        __nanosleep(64);
        bool ok = true;
        while (need <= need_hi) {
            if (ld_acquire_u32(&fl[need - toff]) != epoch) { ok = false; break; }
            need++;
        }
        if (__all_sync(kFull, ok)) return 0;
        if (__any_sync(kFull, global_ns() - t0 > wait_ns)) return kErrTimeout;
    }
}

// ------------------------------------------------------------------------------------------ kernel
template <int WARPS>
__global__ void __launch_bounds__(32 * WARPS, 20 / WARPS) k_flat(WsHead *head, StreamState *sst, uint32_t *flags,
                                                         const StreamDesc *descs, LaunchArgs a) {
    extern __shared__ uint4 dyn_smem[];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    F4Warp &W = reinterpret_cast<F4Warp *>(dyn_smem)[warp];
    WarpTile &c = W.c;
    const uint32_t *wbase = reinterpret_cast<const uint32_t *>(&W);
    uint32_t *imgw = reinterpret_cast<uint32_t *>(W.img);
    const uint32_t stage_off = (uint32_t)((const uint8_t *)W.stage - (const uint8_t *)&W);
    const uint32_t epoch = head->epoch;
    uint32_t parity = 0;
    if (lane == 0) mbar_init(&W.mbar);
    __syncwarp();
    unsigned long long ph[kPhases] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long tc = clock64();
#define WPHASE(k) do { if (a.phase && lane == 0) { const long long now = clock64(); ph[k] += now - tc; tc = now; } } while (0)
    bool dead = false;  // a staging copy never completed: stop taking tiles
    while (!dead) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(&head->ticket, 1ull);
        t = __shfl_sync(kFull, t, 0);
        if (t >= a.total_tiles) break;
        int si = 0;
        if (a.n_streams > 1) {
            if (lane == 0) si = find_stream(descs, a.n_streams, t);
            si = __shfl_sync(kFull, si, 0);
        }
        const StreamDesc &sd = a.n_streams == 1 ? a.one : descs[si];
        StreamState *st = sd.state ? sd.state : &sst[si];
        const unsigned long long order = t - sd.tile_base + sd.tile_off;
        const uint32_t bsh = sd.block_log2 - sd.tile_log2;
        int err = *(volatile int *)&st->status ? 1 : 0;
        err = __shfl_sync(kFull, err, 0);
        __syncwarp();  // every lane is done with the previous tile's stage and image
        if (!err) err = warp_tile_open(c, sd, order >> bsh, (uint32_t)(order & ((1ull << bsh) - 1)), st);
        __syncwarp();
        // ---------------------------------------------------------------- staging
        // section k: [slo[k], shi[k]) of its offsets is staged at W.stage + soff[k] (slo = ~0 when not staged)
        uint32_t slo[4], shi[4], soff[4];
        const uint8_t *sbase[4];
        uint32_t staged = 0;
        if (!err) {
            // a block's header denies matches while having some (depth 1 > 0)
            if (lane == 0 && (order & ((1ull << bsh) - 1)) == 0 && c.n_match > 0) {
                const uint64_t boff = ld64(sd.comp + kStreamHeader + 8 * (order >> bsh));
                if (ld32(sd.comp + boff + 24) == 0) report_depth(st);
            }
            const uint32_t w = c.w;
            const uint32_t m_lo = c.e_seq < c.n_match ? c.e_seq : c.n_match;
            const uint32_t m_hi = c.seq_end < c.n_match ? c.seq_end : c.n_match;
            const uint32_t bx0 = c.chk_lit + (c.hi > c.chk_out ? c.hi - c.chk_out : 0u);
            const uint32_t bx = bx0 < c.n_lit ? bx0 : c.n_lit;
            const uint32_t lit_lo = bx > c.e_lit + kF4LitCap ? bx - kF4LitCap : c.e_lit;
            const uint32_t want_lo[4] = {c.e_cmd, c.e_len, m_lo * w, lit_lo};
            const uint32_t ch = c.chk_cmd + 32, lh = c.chk_len + 32;
            const uint32_t want_hi[4] = {ch < c.cmd_bytes ? ch : c.cmd_bytes, lh < c.len_bytes ? lh : c.len_bytes,
                                         m_hi * w, bx};
            sbase[0] = c.cmd; sbase[1] = c.len; sbase[2] = c.off; sbase[3] = c.lit;
            uint32_t used = 0;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint32_t l16 = want_lo[k] & ~15u, h16 = (uint32_t)align16(want_hi[k]);
                slo[k] = ~0u; shi[k] = 0; soff[k] = 0;
                if (want_hi[k] > want_lo[k] && used + (h16 - l16) <= kF4Stage) {
                    slo[k] = l16; shi[k] = h16; soff[k] = used;
                    used += h16 - l16;
                }
            }
            staged = used;
            if (staged && lane == 0) {
                fence_proxy_async();
                mbar_expect_tx(&W.mbar, staged);
#pragma unroll
                for (int k = 0; k < 4; k++)
                    if (shi[k]) bulk_g2s(W.stage + soff[k], sbase[k] + slo[k], shi[k] - slo[k], &W.mbar);
            }
        }
        // clear the image while the copies run
        for (uint32_t g = lane; g < sizeof(W.img) / 16; g += 32) reinterpret_cast<uint4 *>(W.img)[g] = make_uint4(0, 0, 0, 0);
        for (uint32_t g = lane; g < kF4LbmWords; g += 32) W.lbm[g] = 0;
        if (staged) {
            const uint64_t t0 = global_ns();
            bool ok = mbar_try_wait(&W.mbar, parity);
            while (!__all_sync(kFull, ok)) {
                if (__any_sync(kFull, global_ns() - t0 > a.wait_ns)) break;
                ok = mbar_try_wait(&W.mbar, parity);
            }
            ok = __all_sync(kFull, ok);
            if (!ok) {
                // the copy did not complete in time: report, give it one more bounded wait, stop this warp
                if (lane == 0) report(st, kErrTimeout, kOrderTimeout);
                err = kErrTimeout;
                const uint64_t t1 = global_ns();
                while (!mbar_try_wait(&W.mbar, parity) && global_ns() - t1 < a.wait_ns) {}
                dead = true;
            }
            parity ^= 1u;
        }
        __syncwarp();
        WPHASE(0);
        ph[7] += 1;
        const uint32_t ishift = c.shift;
        // ---------------------------------------------------------------- passes
        for (int pass = 0; pass < 2 && err == 0; pass++) {
            const bool matches = pass == 1;
            uint32_t seq = c.e_seq, cmd_pos = c.e_cmd, len_pos = c.e_len, lit_pos = c.e_lit, out_pos = c.e_out;
            const uint32_t seq_end = c.seq_end, lo = c.lo, hi = c.hi;
            while (seq < seq_end) {
                const uint32_t n = (seq_end - seq) < 32u ? seq_end - seq : 32u;
                const uint32_t nm = seq < c.n_match ? ((c.n_match - seq) < n ? c.n_match - seq : n) : 0u;
                const uint32_t want = (!matches && c.chk_seq >= seq && c.chk_seq <= seq + n) ? c.chk_seq - seq
                                                                                           : 0xFFFFFFFFu;
                uint32_t at_cmd = 0, at_len = 0, r = 0, Lraw = 0;
                const int64_t cp = f4_varints(c.cmd, W.stage + soff[0], slo[0], shi[0], c.cmd_bytes, cmd_pos, n,
                                              c.vals[0], want, at_cmd, r);
                const uint32_t want_l = want <= nm ? want : (want == 0xFFFFFFFFu ? want : nm);
                const int64_t lp = f4_varints(c.len, W.stage + soff[1], slo[1], shi[1], c.len_bytes, len_pos, nm,
                                              c.vals[1], want_l, at_len, Lraw);
                if (cp < 0 || lp < 0) { err = kErrFormat; break; }
                const uint64_t L64 = lane < nm ? (uint64_t)Lraw + c.min_match : 0ull;
                const uint32_t L = (uint32_t)L64;  // < 2^24 once pass A has checked it
                if (lane >= n) r = 0;
                // inclusive scans of (r + L) and r (pass B needs the first only)
                const uint32_t tot = r + L;
                uint32_t in_tot = tot, in_r = r;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y1 = __shfl_up_sync(kFull, in_tot, o);
                    if (lane >= (uint32_t)o) in_tot += y1;
                    if (!matches) {
                        const uint32_t y2 = __shfl_up_sync(kFull, in_r, o);
                        if (lane >= (uint32_t)o) in_r += y2;
                    }
                }
                const uint32_t sum_tot = __shfl_sync(kFull, in_tot, 31);
                const uint32_t start = out_pos + (in_tot - tot);  // block-relative (< 2^24 once checked)
                uint32_t sum_r = 0;
                if (!matches) {
                    sum_r = __shfl_sync(kFull, in_r, 31);
                    const bool bad = lane < n && ((uint64_t)r > c.Nb || L64 > c.Nb || r + L64 == 0);
                    if (__any_sync(kFull, bad) || (uint64_t)out_pos + sum_tot > c.Nb ||
                        (uint64_t)lit_pos + sum_r > c.n_lit) {
                        err = kErrOffset; break;
                    }
                    // sync checks: the first sequence holds the tile's first byte; the next entry matches
                    if (seq == c.e_seq && __shfl_sync(kFull, start + tot, 0) <= lo) { err = kErrFormat; break; }
                    if (want != 0xFFFFFFFFu) {
                        const uint32_t loff = lit_pos + (in_r - r);
                        const uint32_t lit_at = want < n ? __shfl_sync(kFull, loff, want & 31) : lit_pos + sum_r;
                        const uint32_t out_at = want < n ? __shfl_sync(kFull, start, want & 31)
                                                         : out_pos + sum_tot;
                        if (at_cmd != c.chk_cmd || at_len != c.chk_len || lit_at != c.chk_lit || out_at != c.chk_out) {
                            err = kErrFormat; break;
                        }
                    }
                    // ---- literal run: this lane's part inside the tile
                    const uint32_t x0 = start > lo ? start : lo;
                    const uint32_t x1 = (start + r) < hi ? start + r : hi;
                    const uint32_t len = (lane < n && x1 > x0) ? x1 - x0 : 0u;
                    const uint32_t src = lit_pos + (in_r - r) + (x0 - start);  // offset in lit[]
                    const uint32_t ib = x0 - lo + ishift;
                    const bool in_stage = len == 0 || (src >= slo[3] && src + len <= shi[3]);
                    const bool smem_src = __all_sync(kFull, in_stage);
                    const uint32_t so = stage_off + soff[3] + (src - slo[3]);
                    const uint32_t first = len < 16 ? len : 16u;
                    if (first) {
                        if (smem_src) or_piece_smem(wbase, imgw, ib, so, first);
                        else or_piece_lit_glob(imgw, ib, c.lit, src, first);
                        f4_mark(W.lbm, ib, first);
                    }
                    if (__any_sync(kFull, len > 16)) {
                        const uint32_t second = len > 32 ? 16u : (len > 16 ? len - 16 : 0u);
                        if (second) {
                            if (smem_src) or_piece_smem(wbase, imgw, ib + 16, so + 16, second);
                            else or_piece_lit_glob(imgw, ib + 16, c.lit, src + 16, second);
                            f4_mark(W.lbm, ib + 16, second);
                        }
                    }
                    // pieces from the third on: round-robin over the warp
                    const uint32_t extra = len > 32 ? (len - 17) >> 4 : 0u;
                    if (__any_sync(kFull, extra != 0)) {
                        uint32_t ex = extra;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const uint32_t y = __shfl_up_sync(kFull, ex, o);
                            if (lane >= (uint32_t)o) ex += y;
                        }
                        const uint32_t total = __shfl_sync(kFull, ex, 31);
                        ex -= extra;
                        for (uint32_t base = 0; base < total; base += 32) {
                            const uint32_t i = base + lane;
                            const uint32_t k = f4_owner(ex, i);
                            const uint32_t o_ib = __shfl_sync(kFull, ib, k), o_len = __shfl_sync(kFull, len, k);
                            const uint32_t o_src = __shfl_sync(kFull, src, k), o_so = __shfl_sync(kFull, so, k);
                            const uint32_t o_ex = __shfl_sync(kFull, ex, k);
                            if (i < total) {
                                const uint32_t off = 16 * (2 + i - o_ex);
                                const uint32_t pl = (o_len - off) < 16 ? o_len - off : 16u;
                                if (smem_src) or_piece_smem(wbase, imgw, o_ib + off, o_so + off, pl);
                                else or_piece_lit_glob(imgw, o_ib + off, c.lit, o_src + off, pl);
                                f4_mark(W.lbm, o_ib + off, pl);
                            }
                        }
                    }
                } else {
                    // ---- match: absolute source (§3.1), this lane's part inside the tile
                    const uint32_t d = start + r;  // block-relative destination
                    const uint32_t x0 = d > lo ? d : lo;
                    const uint32_t x1 = (d + L) < hi ? d + L : hi;
                    uint32_t s = 0;
                    const uint32_t b0 = (uint32_t)c.b0;
                    if (lane < nm) {
                        const uint32_t q = (seq + lane) * c.w;  // field offset in off[]
                        const bool st_ok = q >= slo[2] && q + c.w <= shi[2];
                        // w-byte little-endian field: aligned word loads and a funnel shift (the field's words
                        // lie inside the staged range, or inside the stream's 16-byte padded section)
                        uint32_t w0, w1, w2;
                        uint32_t sh8;
                        if (st_ok) {
                            const uint32_t so = stage_off + soff[2] + (q - slo[2]);
                            const uint32_t *wp = wbase + (so >> 2);
                            sh8 = 8 * (so & 3u);
                            const uint32_t span = (so & 3u) + c.w;
                            w0 = wp[0]; w1 = span > 4 ? wp[1] : 0u; w2 = span > 8 ? wp[2] : 0u;
                        } else {
                            const uintptr_t addr = (uintptr_t)(c.off + q);
                            const uint32_t *wp = reinterpret_cast<const uint32_t *>(addr & ~(uintptr_t)3);
                            sh8 = 8 * (uint32_t)(addr & 3);
                            const uint32_t span = (uint32_t)(addr & 3) + c.w;
                            w0 = __ldg(wp); w1 = span > 4 ? __ldg(wp + 1) : 0u; w2 = span > 8 ? __ldg(wp + 2) : 0u;
                        }
                        uint64_t v = __funnelshift_r(w0, w1, sh8);
                        if (c.w > 4) v |= (uint64_t)__funnelshift_r(w1, w2, sh8) << 32;
                        const uint64_t s64 = c.w >= 8 ? v : (v & ((1ull << (8 * c.w)) - 1));
                        if (s64 >= (uint64_t)b0 + d) err = kErrOffset;
                        s = (uint32_t)s64;
                    }
                    if (__any_sync(kFull, err != 0)) { err = kErrOffset; break; }
                    const uint32_t len = (lane < nm && x1 > x0) ? x1 - x0 : 0u;
                    const uint32_t p = b0 + d - s;             // source period (valid lanes: s < b0 + d)
                    const bool wrap = p < L;
                    const uint32_t k0 = x0 - d;                // first match byte inside the tile
                    const uint32_t ib = x0 - lo + ishift;
                    // the stream tiles holding the source bytes this lane reads must have published their
                    // literals (bounded wait); this tile's own literals are in place since pass A, and tiles
                    // before tile_off were decoded by an earlier launch
                    WPHASE(5);
                    {
                        uint32_t need = 0xFFFFFFFFu, need_hi = 0;
                        const uint32_t ord32 = (uint32_t)order, toff = (uint32_t)sd.tile_off;
                        if (len) {
                            const uint32_t sa = wrap ? s : s + k0, sb = wrap ? b0 + d : s + k0 + len;
                            const uint32_t ua = sa >> sd.tile_log2, ub = (sb - 1) >> sd.tile_log2;
                            if (ua < ord32 && ub >= toff) {
                                need = ua > toff ? ua : toff;
                                need_hi = ub < ord32 ? ub : ord32 - 1;
                            }
                        }
                        bool ok = true;
                        const uint32_t *fl = flags + sd.tile_base;  // fl[u - toff]: flag of stream tile u
                        while (need <= need_hi) {
                            if (ld_acquire_u32(&fl[need - toff]) != epoch) { ok = false; break; }
                            need++;
                        }
                        if (!__all_sync(kFull, ok)) err = f4_wait_slow(fl, toff, need, need_hi, epoch, a.wait_ns);
                        err = __shfl_sync(kFull, err, 0);
                        if (err) { if (lane == 0) report(st, kErrTimeout, kOrderTimeout); break; }
                        __syncwarp();
                    }
                    WPHASE(4);
                    // every source byte read must be a literal byte: this tile's part against the bits in
                    // shared memory, earlier tiles' against the published bits in HBM (one or two words loaded
                    // directly, longer ranges word by word).  32-bit stream positions: the source range ends at
                    // or before b0 + d < kF4MaxN.
                    const uint32_t tile_abs = (uint32_t)(c.b0 + lo);
                    const uint32_t ra = wrap ? s : s + k0, rb = wrap ? b0 + d : s + k0 + len;
                    const uint32_t rg = rb < tile_abs ? rb : tile_abs;
                    uint32_t gv0 = 0, gv1 = 0, gm0 = 0, gm1 = 0;
                    bool glong = false;
                    if (len && ra < rg) {
                        const uint32_t q0 = ra >> 5, q1 = (rg - 1) >> 5;
                        const uint32_t lo0 = ra & 31u, hi1 = ((rg - 1) & 31u) + 1u;
                        if (q1 == q0) {
                            gm0 = __funnelshift_lc(kFull, 0u, hi1) & ~__funnelshift_lc(kFull, 0u, lo0);
                            gv0 = __ldcg(sd.litmap + q0);
                        } else if (q1 == q0 + 1) {
                            gm0 = ~__funnelshift_lc(kFull, 0u, lo0);
                            gm1 = __funnelshift_lc(kFull, 0u, hi1);
                            gv0 = __ldcg(sd.litmap + q0);
                            gv1 = __ldcg(sd.litmap + q1);
                        } else {
                            glong = true;
                        }
                    }
                    const bool lit_glob = (gv0 & gm0) == gm0 && (gv1 & gm1) == gm1;
                    const uint32_t first = len < 16 ? len : 16u;
                    if (first) f4_match_piece(imgw, ib, sd.out, s, p, k0, first, wrap);
                    if (len) {
                        bool lit = lit_glob;
                        if (glong) lit = f4_bits<true>(sd.litmap, ra, rg);
                        if (lit && rb > tile_abs) {
                            const uint32_t a2 = ra > tile_abs ? ra : tile_abs;
                            lit = f4_bits<false>(W.lbm, a2 - tile_abs + ishift, rb - tile_abs + ishift);
                        }
                        if (!lit) report_depth(st);
                    }
                    const uint32_t extra = len > 16 ? (len - 1) >> 4 : 0u;
                    if (__any_sync(kFull, extra != 0)) {
                        uint32_t ex = extra;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const uint32_t y = __shfl_up_sync(kFull, ex, o);
                            if (lane >= (uint32_t)o) ex += y;
                        }
                        const uint32_t total = __shfl_sync(kFull, ex, 31);
                        ex -= extra;
                        for (uint32_t base = 0; base < total; base += 32) {
                            const uint32_t i = base + lane;
                            const uint32_t k = f4_owner(ex, i);
                            const uint32_t o_ib = __shfl_sync(kFull, ib, k), o_len = __shfl_sync(kFull, len, k);
                            const uint32_t o_k0 = __shfl_sync(kFull, k0, k), o_ex = __shfl_sync(kFull, ex, k);
                            const uint32_t o_s = __shfl_sync(kFull, s, k), o_p = __shfl_sync(kFull, p, k);
                            const bool o_wrap = __shfl_sync(kFull, (uint32_t)wrap, k) != 0;
                            if (i < total) {
                                const uint32_t off = 16 * (1 + i - o_ex);
                                const uint32_t pl = (o_len - off) < 16 ? o_len - off : 16u;
                                f4_match_piece(imgw, o_ib + off, sd.out, o_s, o_p, o_k0 + off, pl, o_wrap);
                            }
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
                uint8_t *base = sd.out + c.b0 + lo - ishift;
                const uint32_t total = ishift + (hi - lo), ng = (total + 15) >> 4;
                for (uint32_t g = lane; g < ng; g += 32) {
                    const uint32_t a0 = g << 4, a1 = a0 + 16;
                    if (a0 >= ishift && a1 <= total) {
                        *reinterpret_cast<uint4 *>(base + a0) = *reinterpret_cast<const uint4 *>(W.img + a0);
                    } else {
                        const uint32_t u = a0 > ishift ? a0 : ishift, z = a1 < total ? a1 : total;
                        for (uint32_t x = u; x < z; x++) base[x] = W.img[x];
                    }
                }
            }
            if (!matches) {
                // the tile's literal bits (bit x: output byte x of the stream), published with the flag
                const uint32_t nbits = hi - lo;
                const unsigned long long tile_abs = c.b0 + lo;
                if (sd.tile_log2 >= 5) {
                    uint32_t *gw = sd.litmap + (tile_abs >> 5);
                    const uint32_t nwd = (nbits + 31) >> 5;
                    for (uint32_t w = lane; w < nwd; w += 32) {
                        uint32_t v = __funnelshift_r(W.lbm[w], W.lbm[w + 1], ishift);
                        if (w == nwd - 1 && (nbits & 31u)) v &= (1u << (nbits & 31u)) - 1u;
                        gw[w] = v;
                    }
                } else if (lane == 0) {
                    // tiles of 4, 8 or 16 bytes share a word with their neighbours
                    const uint32_t m = (1u << nbits) - 1u, off = (uint32_t)(tile_abs & 31u);
                    const uint32_t v = __funnelshift_r(W.lbm[0], W.lbm[1], ishift) & m;
                    uint32_t *gw = sd.litmap + (tile_abs >> 5);
                    atomicAnd(gw, ~(m << off));
                    atomicOr(gw, v << off);
                }
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
