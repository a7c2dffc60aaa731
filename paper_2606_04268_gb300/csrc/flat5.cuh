// One-pass decode, one warp per tile (tiles of at most 4 KiB), 128 sequences per warp step.
//
// The structure is the staged two-pass kernel's (§3.3, §7.1: every match of a depth-1 stream reads literal
// bytes only): the tile's ranges of cmd[], len[], off[] and lit[] (§3.2) are bulk-copied into shared memory;
// pass A places the sequences and ORs the literal runs into a zeroed shared image of the tile, which is
// stored and published; pass B copies every match once the tiles holding its source bytes have published.
//
// What changes is the unit of work: lane l owns the four consecutive sequences 4l .. 4l+3 of a group of
// 128.  Their LEB128 values come from one 128-byte window (lane l reads bytes 4l .. 4l+3) when every value
// is a single byte, the common case; one warp scan of the lanes' run+match totals and one of their literal
// totals place all 128 (§3.2: the running position of a sequential decoder).  The per-step costs of the
// 32-sequence kernel (window tests, ballots, scans, loop control) are paid once per 128 sequences.  Each
// lane then copies the first 16 bytes of each of its segments; the remaining 16-byte pieces of longer
// segments are dealt round-robin to the warp.
//
// Errors are reported in the order the 32-sequence kernel reports them: sub-groups of 32 sequences in
// stream order, and within one: a malformed varint, then a run or match length out of range, then the sync
// entries' checks.
#pragma once
#include "flat4.cuh"

namespace aceapex {

constexpr int kF5Warps = 4;
constexpr uint32_t kF5Seq = 4;                  // sequences per lane per step
constexpr uint32_t kF5Group = 32 * kF5Seq;      // sequences per warp step
constexpr uint32_t kF5Stage = 5120;             // staged section bytes per warp

struct alignas(16) F5Warp {
    WarpTile c;                                 // tile context, 32-varint hand-off
    unsigned long long mbar;
    uint32_t pad_[2];
    uint32_t tr[kF5Group];                      // general varint path: values in sequence order
    alignas(16) uint8_t stage[kF5Stage + kF4Slack];
    alignas(16) uint8_t img[(1u << kWarpImgLog2) + 32];
};

template <int N>
__device__ __forceinline__ uint32_t pick(const uint32_t (&v)[N], uint32_t i) {
    uint32_t r = v[0];
#pragma unroll
    for (int k = 1; k < N; k++) r = i == (uint32_t)k ? v[k] : r;
    return r;
}

// `count` (<= 128) LEB128 values starting at section offset pos: lane l receives values 4l .. 4l+3 in v[]
// (0 past count).  *start_of receives the offset of varint `want` (want <= count).  ok32 receives how many
// leading sub-groups of 32 values decoded without error (4 when all did).  Returns the offset after the
// last good varint.
__device__ __forceinline__ uint32_t f5_varints(const uint8_t *g, const uint8_t *stg, uint32_t slo, uint32_t shi,
                                               uint32_t sec_len, uint32_t pos, uint32_t count, uint32_t *hand,
                                               uint32_t *tr, uint32_t want, uint32_t &start_of, uint32_t (&v)[kF5Seq],
                                               uint32_t &ok32) {
    const uint32_t lane = threadIdx.x & 31;
#pragma unroll
    for (uint32_t i = 0; i < kF5Seq; i++) v[i] = 0;
    ok32 = 4;
    if (want == 0) start_of = pos;
    if (count == 0) return pos;
    // common case: the count bytes at pos are all one-byte varints
    const bool st = pos >= slo && (pos + count <= shi || shi >= sec_len);
    uint32_t b[kF5Seq];
    bool big = false;
#pragma unroll
    for (uint32_t i = 0; i < kF5Seq; i++) {
        const uint32_t k = kF5Seq * lane + i, q = pos + k;
        b[i] = 0;
        if (k < count) {
            b[i] = q < sec_len ? (st ? (uint32_t)stg[q - slo] : (uint32_t)__ldg(g + q)) : 0x80u;
            big |= b[i] >= 0x80u;
        }
    }
    if (!__any_sync(kFull, big)) {
#pragma unroll
        for (uint32_t i = 0; i < kF5Seq; i++) v[i] = b[i];
        if (want <= count) start_of = pos + want;
        return pos + count;
    }
    // general case: 32 values at a time, through shared memory back to lane order
    uint32_t p = pos;
    for (uint32_t j = 0; j < count; j += 32) {
        const uint32_t cnt = (count - j) < 32u ? count - j : 32u;
        const uint32_t wj = (want >= j && want <= j + cnt) ? want - j : 0xFFFFFFFFu;
        uint32_t so = 0, val = 0;
        const int64_t np = f4_varints(g, stg, slo, shi, sec_len, p, cnt, hand, wj, so, val);
        if (np < 0) { ok32 = j / 32; break; }
        if (wj != 0xFFFFFFFFu) start_of = so;
        if (lane < cnt) tr[j + lane] = val;
        p = (uint32_t)np;
    }
    __syncwarp();
    const uint32_t good = ok32 * 32 < count ? ok32 * 32 : count;
#pragma unroll
    for (uint32_t i = 0; i < kF5Seq; i++) {
        const uint32_t k = kF5Seq * lane + i;
        v[i] = k < good ? tr[k] : 0u;
    }
    __syncwarp();
    return p;
}

// ------------------------------------------------------------------------------------------ kernel
__global__ void __launch_bounds__(32 * kF5Warps) k_flat5(WsHead *head, StreamState *sst, uint32_t *flags,
                                                         const StreamDesc *descs, LaunchArgs a) {
    extern __shared__ uint4 dyn_smem[];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    F5Warp &W = reinterpret_cast<F5Warp *>(dyn_smem)[warp];
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
        uint32_t slo[4], shi[4], soff[4];
        uint32_t staged = 0;
        if (!err) {
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
            const uint8_t *sbase[4] = {c.cmd, c.len, c.off, c.lit};
            uint32_t used = 0;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint32_t l16 = want_lo[k] & ~15u, h16 = (uint32_t)align16(want_hi[k]);
                slo[k] = ~0u; shi[k] = 0; soff[k] = 0;
                if (want_hi[k] > want_lo[k] && used + (h16 - l16) <= kF5Stage) {
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
        for (uint32_t g = lane; g < sizeof(W.img) / 16; g += 32) reinterpret_cast<uint4 *>(W.img)[g] = make_uint4(0, 0, 0, 0);
        if (staged) {
            const uint64_t t0 = global_ns();
            bool ok = mbar_try_wait(&W.mbar, parity);
            while (!__all_sync(kFull, ok)) {
                if (__any_sync(kFull, global_ns() - t0 > a.wait_ns)) break;
                ok = mbar_try_wait(&W.mbar, parity);
            }
            ok = __all_sync(kFull, ok);
            if (!ok) {
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
                const uint32_t n = (seq_end - seq) < kF5Group ? seq_end - seq : kF5Group;
                const uint32_t nm = seq < c.n_match ? ((c.n_match - seq) < n ? c.n_match - seq : n) : 0u;
                const uint32_t want = (!matches && c.chk_seq >= seq && c.chk_seq <= seq + n) ? c.chk_seq - seq
                                                                                           : 0xFFFFFFFFu;
                uint32_t at_cmd = 0, at_len = 0, rv[kF5Seq], lv[kF5Seq], okc = 4, okl = 4;
                const uint32_t cp = f5_varints(c.cmd, W.stage + soff[0], slo[0], shi[0], c.cmd_bytes, cmd_pos, n,
                                               c.vals[0], W.tr, want, at_cmd, rv, okc);
                const uint32_t want_l = want <= nm ? want : (want == 0xFFFFFFFFu ? want : nm);
                // the len[] values are needed only where cmd[] decoded
                const uint32_t nm_dec = okc < 4 ? (nm < okc * 32 ? nm : okc * 32) : nm;
                const uint32_t lp = f5_varints(c.len, W.stage + soff[1], slo[1], shi[1], c.len_bytes, len_pos, nm_dec,
                                               c.vals[1], W.tr, want_l <= nm_dec ? want_l : 0xFFFFFFFFu, at_len, lv, okl);
                // sub-groups of 32 whose varints all decoded
                const uint32_t okv = okc < okl ? okc : okl;
                const uint32_t nv = okv < 4 ? (n < okv * 32 ? n : okv * 32) : n;
                uint32_t r[kF5Seq], L[kF5Seq];
                uint32_t lane_tot = 0, lane_r = 0;
                bool bad = false;
#pragma unroll
                for (uint32_t i = 0; i < kF5Seq; i++) {
                    const uint32_t k = kF5Seq * lane + i;
                    const uint64_t L64 = k < nm ? (uint64_t)lv[i] + c.min_match : 0ull;
                    r[i] = k < nv ? rv[i] : 0u;
                    L[i] = k < nv ? (uint32_t)L64 : 0u;
                    if (!matches && k < nv) bad |= (uint64_t)r[i] > c.Nb || L64 > c.Nb || r[i] + L64 == 0;
                    lane_tot += r[i] + L[i];
                    lane_r += r[i];
                }
                uint32_t in_tot = lane_tot, in_r = lane_r;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y1 = __shfl_up_sync(kFull, in_tot, o);
                    const uint32_t y2 = __shfl_up_sync(kFull, in_r, o);
                    if (lane >= (uint32_t)o) { in_tot += y1; in_r += y2; }
                }
                const uint32_t sum_tot = __shfl_sync(kFull, in_tot, 31), sum_r = __shfl_sync(kFull, in_r, 31);
                uint32_t start[kF5Seq], loff[kF5Seq];
                start[0] = out_pos + (in_tot - lane_tot);
                loff[0] = lit_pos + (in_r - lane_r);
#pragma unroll
                for (uint32_t i = 1; i < kF5Seq; i++) { start[i] = start[i - 1] + r[i - 1] + L[i - 1]; loff[i] = loff[i - 1] + r[i - 1]; }
                if (!matches) {
                    // ---- checks, in the order of the 32-sequence kernel: sub-group by sub-group
                    int e = 0;
                    const unsigned bad_lanes = __ballot_sync(kFull, bad);
                    // cumulative totals at the end of each sub-group (lanes 8j+7)
                    const uint32_t tot_end[4] = {__shfl_sync(kFull, in_tot, 7), __shfl_sync(kFull, in_tot, 15),
                                                 __shfl_sync(kFull, in_tot, 23), sum_tot};
                    const uint32_t r_end[4] = {__shfl_sync(kFull, in_r, 7), __shfl_sync(kFull, in_r, 15),
                                               __shfl_sync(kFull, in_r, 23), sum_r};
                    const uint32_t first_end = __shfl_sync(kFull, start[0] + r[0] + L[0], 0);
                    const uint32_t wl = want >> 2, wsl = want & 3u;
                    const uint32_t w_lit = __shfl_sync(kFull, pick(loff, wsl), wl & 31);
                    const uint32_t w_out = __shfl_sync(kFull, pick(start, wsl), wl & 31);
#pragma unroll
                    for (uint32_t j = 0; j < 4; j++) {
                        const uint32_t beg = 32 * j;
                        if (e || beg >= n) break;
                        if (j >= okv) { e = kErrFormat; break; }
                        const uint32_t end = (beg + 32) < nv ? beg + 32 : nv;
                        if (((bad_lanes >> (8 * j)) & 0xFFu) || (uint64_t)out_pos + tot_end[j] > c.Nb ||
                            (uint64_t)lit_pos + r_end[j] > c.n_lit) { e = kErrOffset; break; }
                        if (j == 0 && seq == c.e_seq && first_end <= lo) { e = kErrFormat; break; }
                        if (want != 0xFFFFFFFFu && want >= beg && want <= end) {
                            const uint32_t lit_at = want < nv ? w_lit : lit_pos + sum_r;
                            const uint32_t out_at = want < nv ? w_out : out_pos + sum_tot;
                            if (at_cmd != c.chk_cmd || at_len != c.chk_len || lit_at != c.chk_lit || out_at != c.chk_out) {
                                e = kErrFormat; break;
                            }
                        }
                    }
                    if (e) { err = e; break; }
                    // ---- literal runs: this lane's parts inside the tile
                    uint32_t len[kF5Seq], src[kF5Seq], ib[kF5Seq];
                    bool in_stage = true;
#pragma unroll
                    for (uint32_t i = 0; i < kF5Seq; i++) {
                        const uint32_t x0 = start[i] > lo ? start[i] : lo;
                        const uint32_t x1 = (start[i] + r[i]) < hi ? start[i] + r[i] : hi;
                        len[i] = x1 > x0 ? x1 - x0 : 0u;
                        src[i] = loff[i] + (x0 - start[i]);
                        ib[i] = x0 - lo + ishift;
                        in_stage &= len[i] == 0 || (src[i] >= slo[3] && src[i] + len[i] <= shi[3]);
                    }
                    const bool smem_src = __all_sync(kFull, in_stage);
                    const uint32_t sbias = stage_off + soff[3] - slo[3];  // stage offset of lit[] offset x: x + sbias
#pragma unroll
                    for (uint32_t i = 0; i < kF5Seq; i++) {
                        const uint32_t f = len[i] < 16 ? len[i] : 16u;
                        if (f) {
                            if (smem_src) or_piece_smem(wbase, imgw, ib[i], src[i] + sbias, f);
                            else or_piece_glob<true>(imgw, ib[i], c.lit, src[i], f);
                        }
                    }
                    // later pieces: round-robin over the warp
                    uint32_t ex4[kF5Seq], lane_e = 0;
#pragma unroll
                    for (uint32_t i = 0; i < kF5Seq; i++) { ex4[i] = len[i] > 16 ? (len[i] - 1) >> 4 : 0u; lane_e += ex4[i]; }
                    if (__any_sync(kFull, lane_e != 0)) {
                        uint32_t ex = lane_e;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const uint32_t y = __shfl_up_sync(kFull, ex, o);
                            if (lane >= (uint32_t)o) ex += y;
                        }
                        const uint32_t total = __shfl_sync(kFull, ex, 31);
                        ex -= lane_e;
                        const uint32_t c1 = ex4[0], c2 = c1 + ex4[1], c3 = c2 + ex4[2];
                        for (uint32_t base = 0; base < total; base += 32) {
                            const uint32_t jj = base + lane;
                            const uint32_t k = f4_owner(ex, jj);
                            const uint32_t rel = jj - __shfl_sync(kFull, ex, k);
                            const uint32_t o1 = __shfl_sync(kFull, c1, k), o2 = __shfl_sync(kFull, c2, k),
                                           o3 = __shfl_sync(kFull, c3, k);
                            const uint32_t i = rel < o1 ? 0u : rel < o2 ? 1u : rel < o3 ? 2u : 3u;
                            const uint32_t before = i == 0 ? 0u : i == 1 ? o1 : i == 2 ? o2 : o3;
                            uint32_t oib[kF5Seq], olen[kF5Seq], osrc[kF5Seq];
#pragma unroll
                            for (uint32_t q = 0; q < kF5Seq; q++) {
                                oib[q] = __shfl_sync(kFull, ib[q], k);
                                olen[q] = __shfl_sync(kFull, len[q], k);
                                osrc[q] = __shfl_sync(kFull, src[q], k);
                            }
                            if (jj < total) {
                                const uint32_t off = 16 * (1 + rel - before);
                                const uint32_t sl = pick(olen, i), sb = pick(oib, i), ss = pick(osrc, i);
                                const uint32_t pl = (sl - off) < 16 ? sl - off : 16u;
                                if (smem_src) or_piece_smem(wbase, imgw, sb + off, ss + off + sbias, pl);
                                else or_piece_glob<true>(imgw, sb + off, c.lit, ss + off, pl);
                            }
                        }
                    }
                } else {
                    // ---- matches: absolute sources (§3.1)
                    const uint32_t b0 = (uint32_t)c.b0;
                    uint32_t s[kF5Seq], d[kF5Seq];
                    bool off_bad = false;
#pragma unroll
                    for (uint32_t i = 0; i < kF5Seq; i++) {
                        const uint32_t k = kF5Seq * lane + i;
                        d[i] = start[i] + r[i];
                        s[i] = 0;
                        if (k < nm) {
                            const uint32_t q = (seq + k) * c.w;  // field offset in off[]
                            uint32_t w0, w1, w2, sh8;
                            if (q >= slo[2] && q + c.w <= shi[2]) {
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
                            off_bad |= s64 >= (uint64_t)b0 + d[i];
                            s[i] = (uint32_t)s64;
                        }
                    }
                    if (__any_sync(kFull, off_bad)) { err = kErrOffset; break; }
                    uint32_t len[kF5Seq], k0[kF5Seq], ib[kF5Seq], p[kF5Seq];
                    bool wrap[kF5Seq];
#pragma unroll
                    for (uint32_t i = 0; i < kF5Seq; i++) {
                        const uint32_t x0 = d[i] > lo ? d[i] : lo;
                        const uint32_t x1 = (d[i] + L[i]) < hi ? d[i] + L[i] : hi;
                        len[i] = (kF5Seq * lane + i < nm && x1 > x0) ? x1 - x0 : 0u;
                        k0[i] = x0 - d[i];
                        ib[i] = x0 - lo + ishift;
                        p[i] = b0 + d[i] - s[i];
                        wrap[i] = p[i] < L[i];
                    }
                    WPHASE(5);
                    // the tiles holding the source bytes must have published their literals (bounded wait);
                    // this tile's own literals are in place, tiles before tile_off were decoded earlier
                    {
                        const uint32_t ord32 = (uint32_t)order, toff = (uint32_t)sd.tile_off;
                        uint32_t need[kF5Seq], need_hi[kF5Seq];
#pragma unroll
                        for (uint32_t i = 0; i < kF5Seq; i++) {
                            need[i] = 0xFFFFFFFFu; need_hi[i] = 0;
                            if (len[i]) {
                                const uint32_t sa = wrap[i] ? s[i] : s[i] + k0[i];
                                const uint32_t sb = wrap[i] ? b0 + d[i] : s[i] + k0[i] + len[i];
                                const uint32_t ua = sa >> sd.tile_log2, ub = (sb - 1) >> sd.tile_log2;
                                if (ua < ord32 && ub >= toff) {
                                    need[i] = ua > toff ? ua : toff;
                                    need_hi[i] = ub < ord32 ? ub : ord32 - 1;
                                }
                            }
                        }
                        const uint64_t t0 = global_ns();
                        for (;;) {
                            bool ok = true;
#pragma unroll
                            for (uint32_t i = 0; i < kF5Seq; i++) {
                                while (ok && need[i] <= need_hi[i]) {
                                    if (ld_acquire_u32(&flags[need[i] - toff + (uint32_t)sd.tile_base]) != epoch) ok = false;
                                    else need[i]++;
                                }
                            }
                            if (__all_sync(kFull, ok)) break;
                            if (__any_sync(kFull, global_ns() - t0 > a.wait_ns)) { err = kErrTimeout; break; }
                            __nanosleep(64);
                        }
                        if (err) { if (lane == 0) report(st, kErrTimeout, kOrderTimeout); break; }
                        __syncwarp();
                    }
                    WPHASE(4);
#pragma unroll
                    for (uint32_t i = 0; i < kF5Seq; i++) {
                        const uint32_t f = len[i] < 16 ? len[i] : 16u;
                        if (f) f4_match_piece(imgw, ib[i], sd.out, s[i], p[i], k0[i], f, wrap[i]);
                    }
                    uint32_t ex4[kF5Seq], lane_e = 0;
#pragma unroll
                    for (uint32_t i = 0; i < kF5Seq; i++) { ex4[i] = len[i] > 16 ? (len[i] - 1) >> 4 : 0u; lane_e += ex4[i]; }
                    if (__any_sync(kFull, lane_e != 0)) {
                        uint32_t ex = lane_e;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const uint32_t y = __shfl_up_sync(kFull, ex, o);
                            if (lane >= (uint32_t)o) ex += y;
                        }
                        const uint32_t total = __shfl_sync(kFull, ex, 31);
                        ex -= lane_e;
                        const uint32_t c1 = ex4[0], c2 = c1 + ex4[1], c3 = c2 + ex4[2];
                        for (uint32_t base = 0; base < total; base += 32) {
                            const uint32_t jj = base + lane;
                            const uint32_t k = f4_owner(ex, jj);
                            const uint32_t rel = jj - __shfl_sync(kFull, ex, k);
                            const uint32_t o1 = __shfl_sync(kFull, c1, k), o2 = __shfl_sync(kFull, c2, k),
                                           o3 = __shfl_sync(kFull, c3, k);
                            const uint32_t i = rel < o1 ? 0u : rel < o2 ? 1u : rel < o3 ? 2u : 3u;
                            const uint32_t before = i == 0 ? 0u : i == 1 ? o1 : i == 2 ? o2 : o3;
                            uint32_t oib[kF5Seq], olen[kF5Seq], os[kF5Seq], op[kF5Seq], ok0[kF5Seq], ow[kF5Seq];
#pragma unroll
                            for (uint32_t q = 0; q < kF5Seq; q++) {
                                oib[q] = __shfl_sync(kFull, ib[q], k);
                                olen[q] = __shfl_sync(kFull, len[q], k);
                                os[q] = __shfl_sync(kFull, s[q], k);
                                op[q] = __shfl_sync(kFull, p[q], k);
                                ok0[q] = __shfl_sync(kFull, k0[q], k);
                                ow[q] = __shfl_sync(kFull, (uint32_t)wrap[q], k);
                            }
                            if (jj < total) {
                                const uint32_t off = 16 * (1 + rel - before);
                                const uint32_t sl = pick(olen, i);
                                const uint32_t pl = (sl - off) < 16 ? sl - off : 16u;
                                f4_match_piece(imgw, pick(oib, i) + off, sd.out, pick(os, i), pick(op, i),
                                               pick(ok0, i) + off, pl, pick(ow, i) != 0);
                            }
                        }
                    }
                }
                __syncwarp();
                seq += n;
                cmd_pos = cp;
                len_pos = lp;
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
