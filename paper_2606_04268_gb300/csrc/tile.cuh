// Tile parsing shared by the one-pass kernel and the wavefront path's parse kernel.
//
// A tile is the T-byte slice [j*T, (j+1)*T) of block b's output (stream format §2.3).  Its sync entry gives the
// state of the sequence that contains its first byte, so a CTA can parse it with no reference to earlier
// tiles.  Sequences are handled in chunks of CH = NT*SPT: the CH literal-run lengths (cmd[]) and match
// lengths (len[]) are decoded block-wide, an exclusive prefix sum places every sequence in the output
// (§3.2; the running position of a sequential decoder), and the chunk's output bytes are then mapped onto
// threads.  Every field read from the stream is checked against the block's extent, and the parse of each
// tile is checked against the next tile's sync entry, so a malformed stream yields a status code and never
// an out-of-bounds access.
#pragma once
#include "device_common.cuh"

namespace aceapex {

template <int NT, int SPT>
struct TileSmem {
    static constexpr int CH = NT * SPT;
    uint32_t start[CH + 1];        // block-relative output start of each chunk sequence, then the chunk end
    uint32_t rlen[CH];             // literal-run length
    uint32_t mlen[CH];             // match length (min_match included), 0 for a sequence without match
    uint32_t loff[CH];             // block-relative offset of the literal run in lit[]
    alignas(16) uint32_t ends[CH]; // varint scratch
    unsigned long long soff[CH];   // absolute match source
    ScanSmem<NT> scan;
    // block and tile context (written by thread 0, read by all)
    const uint8_t *cmd, *len, *off, *lit;
    unsigned long long b0;         // absolute output position of the block's first byte
    uint32_t Nb, n_seq, n_match, n_lit, cmd_bytes, len_bytes, w, n_tiles, min_match, block_depth;
    uint32_t tile_lo, tile_hi;     // block-relative output range of the tile
    // entry state of the tile (kept for the second pass) and running parse state
    uint32_t e_seq, e_cmd, e_len, e_lit, e_out;
    uint32_t seq, cmd_pos, len_pos, lit_pos, out_pos, seq_end, chunk_seq, chunk_n, chunk_nm;
    // sync-point check: the state at sequence chk_seq must equal (chk_cmd, chk_len, chk_lit, chk_out)
    uint32_t chk_seq, chk_cmd, chk_len, chk_lit, chk_out, got_cmd, got_len;
    int err, verr;
};

// Thread 0: read the block index entry and block header, check them, set up the tile context.  Returns
// the status code (0 = fine).  `acc` (when non-null) receives the block's header totals, once per block.
template <int NT, int SPT>
__device__ int tile_open(TileSmem<NT, SPT> &sm, const StreamDesc &sd, uint64_t b, uint32_t j, StreamState *acc) {
    const uint8_t *c = sd.comp;
    const uint64_t first = align16(kStreamHeader + 8ull * sd.n_blocks);
    const uint64_t boff = ld64(c + kStreamHeader + 8 * b);
    const uint64_t bend = (b + 1 < sd.n_blocks) ? ld64(c + kStreamHeader + 8 * (b + 1)) : sd.comp_len;
    if ((boff & 15) || boff < first || (b == 0 && boff != first) || bend <= boff || bend > sd.comp_len ||
        bend - boff < kBlockHeader)
        return kErrFormat;
    const uint8_t *h = c + boff;
    const uint32_t n_seq = ld32(h), n_match = ld32(h + 4), n_lit = ld32(h + 8), cmd_bytes = ld32(h + 12),
                   len_bytes = ld32(h + 16), word5 = ld32(h + 20), depth = ld32(h + 24), n_tiles = ld32(h + 28);
    const uint32_t w = word5 & 0xFF;
    const uint64_t B = 1ull << sd.block_log2, T = 1ull << sd.tile_log2;
    const uint64_t b0 = b * B, Nb = (sd.N - b0 < B) ? sd.N - b0 : B;
    if (n_seq < 1 || (n_match != n_seq && n_match + 1 != n_seq) || w < 1 || w > 8 || (word5 >> 8) ||
        n_tiles != (Nb + T - 1) / T || n_lit > Nb)
        return kErrFormat;
    const uint64_t o_cmd = boff + align16(kBlockHeader + (uint64_t)kSyncEntry * n_tiles);
    const uint64_t o_len = align16(o_cmd + cmd_bytes), o_off = align16(o_len + len_bytes);
    const uint64_t o_lit = align16(o_off + (uint64_t)n_match * w);
    if (align16(o_lit + n_lit) != bend) return kErrFormat;
    if (j >= n_tiles) return kErrFormat;
    const uint8_t *e = h + kBlockHeader + (uint64_t)kSyncEntry * j;
    sm.e_seq = ld32(e); sm.e_cmd = ld32(e + 4); sm.e_len = ld32(e + 8); sm.e_lit = ld32(e + 12); sm.e_out = ld32(e + 16);
    sm.tile_lo = (uint32_t)(j * T);
    sm.tile_hi = (uint32_t)((j + 1) * T < Nb ? (j + 1) * T : Nb);
    if (j == 0 && (sm.e_seq | sm.e_cmd | sm.e_len | sm.e_lit | sm.e_out)) return kErrFormat;
    if (sm.e_seq >= n_seq || sm.e_out > sm.tile_lo || sm.e_cmd > cmd_bytes || sm.e_len > len_bytes ||
        sm.e_lit > n_lit)
        return kErrFormat;
    if (j + 1 < n_tiles) {
        const uint8_t *e2 = e + kSyncEntry;
        sm.chk_seq = ld32(e2); sm.chk_cmd = ld32(e2 + 4); sm.chk_len = ld32(e2 + 8); sm.chk_lit = ld32(e2 + 12);
        sm.chk_out = ld32(e2 + 16);
        if (sm.chk_seq < sm.e_seq || sm.chk_seq >= n_seq) return kErrFormat;
        sm.seq_end = sm.chk_seq + 1;
    } else {
        sm.chk_seq = n_seq; sm.chk_cmd = cmd_bytes; sm.chk_len = len_bytes; sm.chk_lit = n_lit;
        sm.chk_out = (uint32_t)Nb;
        sm.seq_end = n_seq;
    }
    sm.cmd = c + o_cmd; sm.len = c + o_len; sm.off = c + o_off; sm.lit = c + o_lit;
    sm.b0 = b0; sm.Nb = (uint32_t)Nb; sm.n_seq = n_seq; sm.n_match = n_match; sm.n_lit = n_lit;
    sm.cmd_bytes = cmd_bytes; sm.len_bytes = len_bytes; sm.w = w; sm.n_tiles = n_tiles;
    sm.min_match = sd.min_match; sm.block_depth = depth;
    if (acc && j == 0) {
        atomicAdd(&acc->seq_sum, (unsigned long long)n_seq);
        atomicAdd(&acc->match_sum, (unsigned long long)n_match);
        atomicMax(&acc->depth_max, depth);
    }
    return kOK;
}

// All threads: rewind the running parse state to the tile's sync entry.
template <int NT, int SPT>
__device__ __forceinline__ void tile_rewind(TileSmem<NT, SPT> &sm) {
    if (threadIdx.x == 0) {
        sm.seq = sm.e_seq; sm.cmd_pos = sm.e_cmd; sm.len_pos = sm.e_len; sm.lit_pos = sm.e_lit; sm.out_pos = sm.e_out;
        sm.verr = 0;
    }
    __syncthreads();
}

// All threads: parse the next chunk of sequences.  Fills start/rlen/mlen/loff (and soff when with_off),
// checks them, advances the running state.  Returns false on a format error (sm.err is then set).
template <int NT, int SPT>
__device__ bool chunk_parse(TileSmem<NT, SPT> &sm, bool with_off) {
    constexpr int CH = NT * SPT;
    const uint32_t seq = sm.seq;
    const uint32_t n = (sm.seq_end - seq) < (uint32_t)CH ? sm.seq_end - seq : (uint32_t)CH;
    const uint32_t nm = seq < sm.n_match ? ((sm.n_match - seq) < n ? sm.n_match - seq : n) : 0;
    const uint32_t want = (sm.chk_seq >= seq && sm.chk_seq <= seq + n) ? sm.chk_seq - seq : 0xFFFFFFFFu;
    const int64_t cpos = block_varints<NT>(sm.cmd, sm.cmd_bytes, sm.cmd_pos, n, sm.rlen, sm.ends, sm.scan, &sm.verr,
                                           want, &sm.got_cmd);
    const uint32_t want_l = want <= nm ? want : (want == 0xFFFFFFFFu ? want : nm);
    const int64_t lpos = block_varints<NT>(sm.len, sm.len_bytes, sm.len_pos, nm, sm.mlen, sm.ends, sm.scan, &sm.verr,
                                           want_l, &sm.got_len);
    if (cpos < 0 || lpos < 0) {
        if (threadIdx.x == 0) sm.err = kErrFormat;
        __syncthreads();
        return false;
    }
    // per thread: SPT consecutive sequences
    const uint32_t i0 = threadIdx.x * SPT;
    unsigned long long tot_loc = 0, lit_loc = 0;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < SPT; k++) {
        const uint32_t i = i0 + k;
        if (i < n) {
            const uint32_t r = sm.rlen[i];
            uint64_t L = 0;
            if (i < nm) {
                L = (uint64_t)sm.mlen[i] + sm.min_match;
                sm.mlen[i] = (uint32_t)(L <= sm.Nb ? L : 0);
            } else {
                sm.mlen[i] = 0;
            }
            if (r > sm.Nb || L > sm.Nb || r + L == 0) bad = true;
            tot_loc += r + L;
            lit_loc += r;
        }
    }
    unsigned long long tot_all, lit_all;
    unsigned long long tot_ex = block_excl_scan<NT>(tot_loc, sm.scan, tot_all);
    unsigned long long lit_ex = block_excl_scan<NT>(lit_loc, sm.scan, lit_all);
    const unsigned long long out0 = sm.out_pos, lit0 = sm.lit_pos;
    if (out0 + tot_all > sm.Nb || lit0 + lit_all > sm.n_lit) bad = true;
#pragma unroll
    for (int k = 0; k < SPT; k++) {
        const uint32_t i = i0 + k;
        if (i < n && !bad) {
            sm.start[i] = (uint32_t)(out0 + tot_ex);
            sm.loff[i] = (uint32_t)(lit0 + lit_ex);
            tot_ex += sm.rlen[i] + sm.mlen[i];
            lit_ex += sm.rlen[i];
            if (with_off && i < nm) {
                const uint64_t s = ld_le(sm.off + (uint64_t)(seq + i) * sm.w, sm.w);
                sm.soff[i] = s;
                if (s >= sm.b0 + sm.start[i] + sm.rlen[i]) atomicCAS(&sm.err, 0, kErrOffset);
            }
        }
    }
    if (bad) atomicCAS(&sm.err, 0, kErrOffset);
    __syncthreads();
    if (threadIdx.x == 0 && !sm.err) {
        sm.start[n] = (uint32_t)(out0 + tot_all);
        // the tile's first sequence must contain the tile's first byte
        if (seq == sm.e_seq && sm.start[1] <= sm.tile_lo) sm.err = kErrFormat;
        if (want != 0xFFFFFFFFu) {
            const uint32_t lit_at = want < n ? sm.loff[want] : (uint32_t)(lit0 + lit_all);
            const uint32_t out_at = want < n ? sm.start[want] : (uint32_t)(out0 + tot_all);
            if (sm.got_cmd != sm.chk_cmd || sm.got_len != sm.chk_len || lit_at != sm.chk_lit || out_at != sm.chk_out)
                sm.err = kErrFormat;
        }
        sm.chunk_seq = seq; sm.chunk_n = n; sm.chunk_nm = nm;
        sm.seq = seq + n; sm.cmd_pos = (uint32_t)cpos; sm.len_pos = (uint32_t)lpos;
        sm.lit_pos = (uint32_t)(lit0 + lit_all); sm.out_pos = (uint32_t)(out0 + tot_all);
    }
    __syncthreads();
    return sm.err == 0;
}

// Stream of global tile t in a batch (descs sorted by tile_base).
__device__ __forceinline__ int find_stream(const StreamDesc *descs, int n, uint64_t t) {
    int a = 0, z = n;
    while (z - a > 1) {
        const int mid = (a + z) >> 1;
        if (descs[mid].tile_base <= t) a = mid; else z = mid;
    }
    return a;
}

// Index of the chunk sequence whose output range holds block-relative byte q (start[i] <= q < start[i+1]).
template <int NT, int SPT>
__device__ __forceinline__ uint32_t seq_of(const TileSmem<NT, SPT> &sm, uint32_t n, uint32_t q) {
    uint32_t a = 0, z = n;
    while (z - a > 1) {
        const uint32_t mid = (a + z) >> 1;
        if (sm.start[mid] <= q) a = mid; else z = mid;
    }
    return a;
}

// All threads: write the chunk's literal bytes that fall inside the tile.
template <int NT, int SPT>
__device__ void chunk_literals(const TileSmem<NT, SPT> &sm, uint8_t *out) {
    const uint32_t n = sm.chunk_n;
    const uint32_t lo = sm.start[0] > sm.tile_lo ? sm.start[0] : sm.tile_lo;
    const uint32_t hi = sm.start[n] < sm.tile_hi ? sm.start[n] : sm.tile_hi;
    uint8_t *ob = out + sm.b0;
    for (uint32_t q = lo + threadIdx.x; q < hi; q += NT) {
        const uint32_t i = seq_of(sm, n, q);
        const uint32_t rel = q - sm.start[i];
        if (rel < sm.rlen[i]) ob[q] = __ldg(sm.lit + sm.loff[i] + rel);
    }
}

}  // namespace aceapex
