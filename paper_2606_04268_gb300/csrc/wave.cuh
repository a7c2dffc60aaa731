// Wavefront path, warp-parallel parts: the tile parse (one warp per tile) and the level drain (one lane
// per match).
//
// k_parse_w: literal bytes -> out (through a per-warp image of the tile, as in the one-pass kernel; match
//   positions receive don't-care bytes that the level drain overwrites), and for every match whose first
//   byte lies in the tile a record (absolute destination, absolute source, length) at its global match index,
//   plus the granule index gidx[g] = first match whose range ends after the granule's first byte.
// k_wave_w: levels 1, 2, ... in one cooperative launch with a bounded grid barrier in between; inside a
//   level, lane k of a warp copies match k of a group of 32 (at most 16 bytes: aligned 16-byte loads through
//   L2, since the previous level's bytes were written by other SMs), longer or self-overlapping matches are
//   copied by the whole warp.
#pragma once
#include "flat3.cuh"

namespace aceapex {

__global__ void __launch_bounds__(32 * kWarpsPerCta) k_parse_w(StreamState *sst, LaunchArgs a, WaveBufs wb) {
    extern __shared__ uint4 dyn_smem[];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpSmem &ws = reinterpret_cast<WarpSmem *>(dyn_smem)[warp];
    WarpTile &c = ws.ctx;
    const StreamDesc &sd = a.one;
    StreamState *st = &sst[0];
    const uint32_t sh = sd.block_log2 - sd.tile_log2;
    const uint32_t gl = sd.tile_log2 < kGranuleLog2 ? sd.tile_log2 : kGranuleLog2;
    const uint64_t nwarps = (uint64_t)gridDim.x * kWarpsPerCta;
    for (uint64_t t = (uint64_t)blockIdx.x * kWarpsPerCta + warp; t < sd.n_tiles; t += nwarps) {
        int err = *(volatile int *)&st->status ? 1 : 0;
        err = __shfl_sync(0xffffffffu, err, 0);
        if (err) return;
        const uint64_t b = t >> sh;
        err = warp_tile_open(c, sd, b, (uint32_t)(t & ((1ull << sh) - 1)), st);
        if (err) { if (lane == 0) report(st, err, t); return; }
        const unsigned long long mb = wb.block_base[b], mb_next = wb.block_base[b + 1];
        uint8_t *img = ws.img + c.shift;
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
            const uint64_t L = lane < nm ? (uint64_t)Lraw + c.min_match : 0;
            if (lane >= n) r = 0;
            const bool bad = lane < n && (r > c.Nb || L > c.Nb || r + L == 0);
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
            if (seq == c.e_seq && __shfl_sync(0xffffffffu, (uint32_t)start + tot, 0) <= lo) { err = kErrFormat; break; }
            if (want != 0xFFFFFFFFu) {
                const uint32_t lit_at = want < n ? __shfl_sync(0xffffffffu, (uint32_t)loff, want & 31) : lit_pos + sum_r;
                const uint32_t out_at = want < n ? __shfl_sync(0xffffffffu, (uint32_t)start, want & 31) : out_pos + sum_tot;
                if (at_cmd != c.chk_cmd || at_len != c.chk_len || lit_at != c.chk_lit || out_at != c.chk_out) {
                    err = kErrFormat; break;
                }
            }
            // match record of a match that starts in this tile
            const uint64_t d = start + r;
            if (lane < nm && d >= lo && d < hi) {
                const uintptr_t addr = (uintptr_t)(c.off + (uint64_t)(seq + lane) * c.w);
                const uint32_t *wp = reinterpret_cast<const uint32_t *>(addr & ~(uintptr_t)3);
                const uint32_t sh8 = 8 * (uint32_t)(addr & 3), span = (uint32_t)(addr & 3) + c.w;
                const uint32_t w0 = __ldg(wp), w1 = span > 4 ? __ldg(wp + 1) : 0u;
                uint64_t v = __funnelshift_r(w0, w1, sh8);
                if (c.w > 4) {
                    const uint32_t w2 = span > 8 ? __ldg(wp + 2) : 0u;
                    v |= (uint64_t)__funnelshift_r(w1, w2, sh8) << 32;
                }
                const uint64_t s = c.w >= 8 ? v : (v & ((1ull << (8 * c.w)) - 1));
                const unsigned long long m = mb + seq + lane;
                if (s >= c.b0 + d) err = kErrOffset;
                else if (m >= mb_next || m >= sd.n_match) err = kErrFormat;
                else {
                    wb.mdst[m] = c.b0 + d;
                    wb.msrc[m] = s;
                    wb.mlen[m] = (uint32_t)L;
                    wb.depth[m] = 0;
                }
            }
            if (__any_sync(0xffffffffu, err != 0)) { err = __reduce_min_sync(0xffffffffu, (unsigned)(err + 16)) - 16; break; }
            // granule index: granule starts in this group's range inside the tile
            {
                const uint32_t G = 1u << gl;
                const uint64_t g_lo64 = start > lo ? start : lo;  // per lane; the group range is [lane 0 start, end)
                const uint32_t grp_lo = (uint32_t)__shfl_sync(0xffffffffu, (uint32_t)g_lo64, 0);
                const uint32_t grp_hi = (out_pos + sum_tot) < hi ? out_pos + sum_tot : hi;
                uint32_t q = (grp_lo + G - 1) & ~(G - 1);
                c.vals[0][lane] = (uint32_t)start;  // group starts for the search
                __syncwarp();
                for (; q < grp_hi; q += 32 * G) {
                    const uint32_t qq = q + lane * G;
                    if (qq < grp_hi) {
                        uint32_t a0 = 0, z = n;
                        while (z - a0 > 1) {
                            const uint32_t mid = (a0 + z) >> 1;
                            if (c.vals[0][mid] <= qq) a0 = mid; else z = mid;
                        }
                        wb.gidx[(c.b0 + qq) >> gl] = (seq + a0 < c.n_match) ? (uint32_t)(mb + seq + a0) : (uint32_t)mb_next;
                    }
                }
                __syncwarp();
            }
            // literal run -> image
            const uint32_t x0 = (uint32_t)(start > lo ? start : lo);
            const uint32_t x1 = (uint32_t)((start + r) < hi ? start + r : hi);
            const uint32_t len = (lane < n && x1 > x0) ? x1 - x0 : 0;
            const uint64_t src0 = loff + (x0 - start);
            if (len > 0 && len <= 16) lane_copy_global<false>(img + (x0 - lo), c.lit + src0, len);
            uint32_t todo = __ballot_sync(0xffffffffu, len > 16);
            while (todo) {
                const int l = __ffs(todo) - 1;
                todo &= todo - 1;
                const uint32_t X0 = __shfl_sync(0xffffffffu, x0, l), LEN = __shfl_sync(0xffffffffu, len, l);
                const uint64_t S0 = __shfl_sync(0xffffffffu, src0, l);
                for (uint32_t j = lane; j < LEN; j += 32) img[X0 - lo + j] = __ldg(c.lit + S0 + j);
            }
            __syncwarp();
            seq += n; cmd_pos = (uint32_t)cp; len_pos = (uint32_t)lp; lit_pos += sum_r; out_pos += sum_tot;
        }
        if (err) { if (lane == 0) report(st, err, t); return; }
        // image -> out
        uint8_t *base = sd.out + c.b0 + lo - c.shift;
        const uint32_t total = c.shift + (hi - lo), ng = (total + 15) >> 4;
        for (uint32_t g = lane; g < ng; g += 32) {
            const uint32_t a0 = g << 4, a1 = a0 + 16;
            if (a0 >= c.shift && a1 <= total) *reinterpret_cast<uint4 *>(base + a0) = *reinterpret_cast<const uint4 *>(ws.img + a0);
            else {
                const uint32_t u = a0 > c.shift ? a0 : c.shift, z = a1 < total ? a1 : total;
                for (uint32_t x = u; x < z; x++) base[x] = ws.img[x];
            }
        }
        __syncwarp();
    }
}

// Up to 16 bytes out[d..d+len) <- out[s..s+len) (no overlap), one lane; loads through L2.
__device__ __forceinline__ void lane_copy_out(uint8_t *out, uint64_t d, uint64_t s, uint32_t len) {
    const uintptr_t addr = (uintptr_t)(out + s), al = addr & ~(uintptr_t)15;
    const uint32_t o = (uint32_t)(addr - al);
    const uint4 *g = reinterpret_cast<const uint4 *>(al);
    const uint4 va = __ldcg(g);
    uint4 vb = make_uint4(0, 0, 0, 0);
    if (o + len > 16) vb = __ldcg(g + 1);
    const uint4 v = realign16(va, vb, o);
    const uint32_t rw[4] = {v.x, v.y, v.z, v.w};
    uint8_t *dp = out + d;
#pragma unroll
    for (int j = 0; j < 16; j++)
        if ((uint32_t)j < len) dp[j] = (uint8_t)(rw[j >> 2] >> (8 * (j & 3)));
}

__global__ void __launch_bounds__(1024) k_wave_w(WsHead *head, StreamState *sst, LaunchArgs a, WaveBufs wb) {
    if (*(volatile int *)&sst[0].status) return;  // uniform: the status is final before this launch
    const uint32_t nlev = head->depth_seen;
    const uint64_t t0 = global_ns();
    const uint32_t lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    uint8_t *out = a.one.out;
    const uint64_t N = a.one.N, nmatch = a.one.n_match;
    for (uint32_t k = 1; k <= nlev; k++) {
        const uint32_t beg = wb.lvl[k], end = wb.lvl[k + 1];
        // two matches per warp step: a half-warp copies a match of at most 16 bytes, lane j <- byte j, so the
        // loads and stores of a match coalesce; four steps are issued together (8 matches in flight per
        // warp); longer or self-overlapping matches take the whole warp
        constexpr int U = 4;
        for (uint64_t g = beg + warp * 2 * U; g < end; g += nwarps * 2 * U) {
            uint64_t d[U], s[U], L[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const uint64_t i = g + 2 * u + half;
                d[u] = 0; s[u] = 0; L[u] = 0;
                if (i < end) {
                    d[u] = wb.qd[i]; s[u] = wb.qs[i]; L[u] = wb.ql[i];
                    if (s[u] >= d[u] || d[u] + L[u] > N) L[u] = 0;  // never true for records k_parse_w checked
                }
            }
            uint32_t v[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const bool small = L[u] <= 16 && d[u] - s[u] >= L[u];
                v[u] = (small && hl < L[u]) ? (uint32_t)__ldcg(out + s[u] + hl) : 0x100u;
            }
#pragma unroll
            for (int u = 0; u < U; u++)
                if (v[u] < 0x100u) out[d[u] + hl] = (uint8_t)v[u];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const bool small = L[u] <= 16 && d[u] - s[u] >= L[u];
                uint32_t todo = __ballot_sync(0xffffffffu, L[u] > 0 && !small && hl == 0);
                while (todo) {
                    const int l = __ffs(todo) - 1;
                    todo &= todo - 1;
                    const uint64_t D = __shfl_sync(0xffffffffu, d[u], l), S = __shfl_sync(0xffffffffu, s[u], l);
                    const uint64_t LL = __shfl_sync(0xffffffffu, L[u], l), P = D - S;
                    for (uint64_t j = lane; j < LL; j += 32) out[D + j] = __ldcg(out + S + (j < P ? j : j % P));
                }
            }
        }
        if (k < nlev && !grid_barrier(head, &sst[0], t0, a.wait_ns)) return;
    }
}

// Level queues by counting: pass 1 counts the levels of a CTA's contiguous range of matches in shared
// memory and reserves one slice per (CTA, level) of the global queue; pass 2 writes the entries.
constexpr int kScatterLevels = 4096;  // levels handled in shared memory; deeper ones use global atomics
__global__ void __launch_bounds__(256) k_scatter_w(LaunchArgs a, WaveBufs wb) {
    __shared__ uint32_t cnt[kScatterLevels];
    const uint64_t n = a.one.n_match;
    const uint32_t maxd = a.one.max_depth;
    const uint32_t nl = (maxd + 1) < (uint32_t)kScatterLevels ? maxd + 1 : (uint32_t)kScatterLevels;
    const uint64_t per = (n + gridDim.x - 1) / gridDim.x;
    const uint64_t m0 = (uint64_t)blockIdx.x * per, m1 = (m0 + per) < n ? m0 + per : n;
    for (uint32_t i = threadIdx.x; i < nl; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    for (uint64_t m = m0 + threadIdx.x; m < m1; m += blockDim.x) {
        const uint32_t d = wb.depth[m];
        if (d <= maxd && d < (uint32_t)kScatterLevels) atomicAdd(&cnt[d], 1u);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nl; i += blockDim.x)
        if (cnt[i]) cnt[i] = atomicAdd(&wb.cursor[i], cnt[i]);  // base of this CTA's slice
    __syncthreads();
    for (uint64_t m = m0 + threadIdx.x; m < m1; m += blockDim.x) {
        const uint32_t d = wb.depth[m];
        if (d > maxd) continue;
        const uint32_t pos = d < (uint32_t)kScatterLevels ? atomicAdd(&cnt[d], 1u) : atomicAdd(&wb.cursor[d], 1u);
        wb.queue[pos] = (uint32_t)m;
        // the record itself, in level order, so that the drain reads it without an index indirection
        wb.qd[pos] = wb.mdst[m];
        wb.qs[pos] = wb.msrc[m];
        wb.ql[pos] = wb.mlen[m];
    }
}

}  // namespace aceapex
