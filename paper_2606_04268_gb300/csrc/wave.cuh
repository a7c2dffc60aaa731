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
#include "warp_tile.cuh"

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

// Copy the matches of queue entries [beg, end) with warps warp, warp + nwarps, ...: two matches per warp
// step -- a half-warp copies a match of at most 16 bytes, lane j <- byte j, so the loads and stores of a
// match coalesce; four steps are issued together (8 matches in flight per warp); longer or self-overlapping
// matches take the whole warp, out[d+k] = out[s + (k mod (d-s))].
__device__ __forceinline__ void wave_level(const WaveBufs &wb, uint8_t *out, uint64_t N, uint64_t beg, uint64_t end,
                                           uint64_t warp, uint64_t nwarps) {
    const uint32_t lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
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
}

// Levels of at most kSmallLevel matches are drained by CTA 0 alone, a run of consecutive ones separated by
// CTA barriers only; the grid meets again at the next larger level.  Deep streams end in long runs of small
// levels, where a grid barrier per level would cost more than the level's copies.
constexpr uint32_t kSmallLevel = 512;

__global__ void __launch_bounds__(1024) k_wave_w(WsHead *head, StreamState *sst, LaunchArgs a, WaveBufs wb) {
    __shared__ uint32_t s_run_end;
    if (*(volatile int *)&sst[0].status) return;  // uniform: the status is final before this launch
    const uint32_t nlev = head->depth_seen;
    const uint64_t t0 = global_ns();
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    uint8_t *out = a.one.out;
    const uint64_t N = a.one.N;
    uint32_t k = 1;
    while (k <= nlev) {
        const uint32_t beg = wb.lvl[k], end = wb.lvl[k + 1];
        if (end - beg > kSmallLevel) {
            wave_level(wb, out, N, beg, end, warp, nwarps);
            k++;
        } else {
            // the run of small levels [k, k2): every CTA finds k2 the same way
            uint32_t k2 = k;
            for (;;) {
                if (threadIdx.x == 0) s_run_end = 0xFFFFFFFFu;
                __syncthreads();
                const uint32_t j = k2 + threadIdx.x;
                if (j <= nlev && wb.lvl[j + 1] - wb.lvl[j] > kSmallLevel) atomicMin(&s_run_end, j);
                __syncthreads();
                const uint32_t e = s_run_end;
                __syncthreads();
                if (e != 0xFFFFFFFFu) { k2 = e; break; }
                k2 += blockDim.x;
                if (k2 > nlev) { k2 = nlev + 1; break; }
            }
            if (blockIdx.x == 0) {
                const uint64_t cw = threadIdx.x >> 5, cn = blockDim.x >> 5;
                for (uint32_t q = k; q < k2; q++) {
                    wave_level(wb, out, N, wb.lvl[q], wb.lvl[q + 1], cw, cn);
                    __syncthreads();
                }
            }
            k = k2;
        }
        if (k <= nlev && !grid_barrier(head, &sst[0], t0, a.wait_ns)) return;
    }
}

// Match phase as a warp-granular dataflow (§7.1 without level barriers).  A warp takes 32 consecutive matches
// (a ticket); lane l owns match m = m0 + l.  Its writers -- the matches whose output overlaps its effective
// source [s, s + min(L, d - s)) -- have smaller indices and are found through the granule index.  In rounds,
// every lane whose writers have all finished copies its match, out[d+k] = out[s + (k mod (d-s))], and
// publishes depth = 1 + the writers' largest depth (nonzero: "finished").  Writers in the same 32 are seen
// through shared memory (the warp barrier orders their bytes); earlier ones through their published depth,
// read with an acquire load that a writer's release store of the depth, after its bytes, pairs with.  The lowest unfinished
// match only waits on finished ones, so the persistent grid always progresses; waits are bounded.

constexpr int kFlowWarps = 8;
constexpr int kFlowWidth = 32;  // lanes of one worker: a worker takes kFlowWidth consecutive matches
__global__ void __launch_bounds__(32 * kFlowWarps, 8) k_flow_w(WsHead *head, StreamState *sst, LaunchArgs a, WaveBufs wb) {
    constexpr int G = kFlowWidth;
    __shared__ uint32_t s_dep[kFlowWarps * 32];
    const StreamDesc &sd = a.one;
    const uint64_t nmatch = sd.n_match, N = sd.N;
    if (*(volatile int *)&sst[0].status) return;  // the parse failed: the records are not usable
    const uint32_t gl = sd.tile_log2 < kGranuleLog2 ? sd.tile_log2 : kGranuleLog2;
    const uint32_t cap = sd.max_depth > 0 ? sd.max_depth : 1;
    const uint32_t lane = threadIdx.x & 31, sub = lane % G, grp = lane / G;
    const unsigned mask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (G * grp));
    volatile uint32_t *mydep = s_dep + (threadIdx.x - sub);
    uint8_t *out = sd.out;
    const uint64_t t0 = global_ns();
    uint32_t dmax = 0;
    for (;;) {
        unsigned long long g = 0;
        if (sub == 0) g = atomicAdd(&head->ticket2, 1ull);
        g = __shfl_sync(mask, g, 0, G);
        const uint64_t m0 = g * G;
        if (m0 >= nmatch) break;
        const uint64_t m = m0 + sub;
        mydep[sub] = 0;
        uint64_t d = 0, s = 0, L = 0, send = 0, w = m;
        bool done = m >= nmatch;
        if (!done) {
            d = __ldg(&wb.mdst[m]); s = __ldg(&wb.msrc[m]); L = __ldg(&wb.mlen[m]);
            if (s < d && d + L <= N) {  // records are checked by the parse; stale ones (after an error) read nothing
                send = s + (L < d - s ? L : d - s);
                w = __ldg(&wb.gidx[s >> gl]);
                while (w < m && __ldg(&wb.mdst[w]) + __ldg(&wb.mlen[w]) <= s) w++;
            } else {
                L = 0; w = m;
            }
        }
        __syncwarp(mask);
        uint32_t mx = 0, spins = 0;
        while (!__all_sync(mask, done)) {
            bool ready = false;
            if (!done) {
                // advance over finished writers; stop at the first unfinished one
                while (w < m && __ldg(&wb.mdst[w]) < send) {
                    // acquire: a finished writer's bytes are visible to this thread's loads below
                    const uint32_t dw = w >= m0 ? mydep[w - m0] : ld_acquire_u32(&wb.depth[w]);
                    if (dw == 0) break;
                    mx = dw > mx ? dw : mx;
                    w++;
                }
                ready = !(w < m && __ldg(&wb.mdst[w]) < send);
            }
            if (__any_sync(mask, ready)) {
                if (ready) {
                    const uint64_t p = d - s;
                    if (p >= L) {
                        for (uint64_t o = 0; o < L; o += 16)
                            lane_copy_out(out, d + o, s + o, (uint32_t)(L - o < 16 ? L - o : 16));
                    } else {
                        uint32_t km = 0;
                        for (uint64_t k = 0; k < L; k++) {
                            out[d + k] = __ldcg(out + s + km);
                            if (++km == (uint32_t)p) km = 0;
                        }
                    }
                    if (a.root) {
                        // transcoding: every byte's root travels with it, root[d+k] = root[s + (k mod p)]
                        uint64_t km = 0;
                        for (uint64_t k = 0; k < L; k++) {
                            a.root[d + k] = __ldcg(a.root + s + km);
                            if (++km == p) km = 0;
                        }
                    }
                    uint32_t dep = mx + 1;
                    // a match deeper than its block's max_depth field: the stream understates its depth
                    if (L && dep > wb.bdepth[d >> sd.block_log2]) report_depth(&sst[0]);
                    if (dep > cap) dep = cap;
                    st_release_u32(&wb.depth[m], dep);  // the bytes (and roots) above are visible before the depth
                    mydep[sub] = dep;
                    dmax = dep > dmax ? dep : dmax;
                    done = true;
                }
                __syncwarp(mask);
            } else {
                if ((++spins & 15) == 0 && __any_sync(mask, global_ns() - t0 > a.wait_ns)) {
                    if (sub == 0) report(&sst[0], kErrTimeout, kOrderTimeout);
                    return;
                }
                __nanosleep(64);
            }
        }
    }
    dmax = __reduce_max_sync(mask, dmax);
    if (sub == 0 && dmax) atomicMax(&head->depth_seen, dmax);
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
    // counts and positions are taken once per group of equal levels in a warp (most matches of a range
    // share a few shallow levels, so per-thread atomics would serialise on the same counters)
    const uint32_t lane = threadIdx.x & 31;
    for (uint64_t m0w = m0; m0w < m1; m0w += blockDim.x) {
        const uint64_t m = m0w + threadIdx.x;
        const uint32_t d = m < m1 ? wb.depth[m] : 0xFFFFFFFFu;
        const bool take = d <= maxd && d < (uint32_t)kScatterLevels;
        const unsigned peers = __match_any_sync(0xffffffffu, take ? d : 0xFFFFFFFFu);
        if (take && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&cnt[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nl; i += blockDim.x)
        if (cnt[i]) cnt[i] = atomicAdd(&wb.cursor[i], cnt[i]);  // base of this CTA's slice
    __syncthreads();
    for (uint64_t m0w = m0; m0w < m1; m0w += blockDim.x) {
        const uint64_t m = m0w + threadIdx.x;
        const uint32_t d = m < m1 ? wb.depth[m] : 0xFFFFFFFFu;
        const bool take = d <= maxd;
        const unsigned peers = __match_any_sync(0xffffffffu, take ? d : 0xFFFFFFFFu);
        const int leader = __ffs(peers) - 1;
        const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        uint32_t base = 0;
        if (take && (int)lane == leader)
            base = d < (uint32_t)kScatterLevels ? atomicAdd(&cnt[d], (uint32_t)__popc(peers))
                                                : atomicAdd(&wb.cursor[d], (uint32_t)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (!take) continue;
        const uint32_t pos = base + rank;
        wb.queue[pos] = (uint32_t)m;
        // the record itself, in level order, so that the drain reads it without an index indirection
        wb.qd[pos] = wb.mdst[m];
        wb.qs[pos] = wb.msrc[m];
        wb.ql[pos] = wb.mlen[m];
    }
}

}  // namespace aceapex
