// Warp-level building blocks of the tile decoders: the tile context one warp works on, the check of a
// block's index entry, header and sync entries, the warp-wide LEB128 decoder, and single-lane copies of up
// to 16 bytes.
//
// A warp owns one tile (at most 2^kWarpImgLog2 output bytes) at a time and works with warp-synchronous
// primitives only (no CTA barrier), so many independent tiles per SM hide each other's memory latency.
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

}  // namespace aceapex
