// ACEAPEX decode kernels for sm_103a and their host-side launch sequences.
//
// One-pass path (every match has depth <= 1, i.e. reads only literal bytes: chain flattening, §3.3):
//   k_flat (onepass.cuh) -- persistent warps take tiles from a global ticket queue (one queue over all the
//   streams of a batch).  Pass A parses the tile, writes its literal bytes and literal bits and publishes a
//   per-tile flag; pass B copies its matches from absolute offsets (§3.1) once the tiles they read have
//   published.  Tickets are handed out in order and pass A never waits, so every wait ends; no per-match
//   metadata reaches HBM.
//
// Wavefront path (§7.1, any depth): k_parse writes the literals and one record (destination, source,
//   length) per match plus a granule index that finds the writers of any byte range; k_flow_w (default)
//   copies each match as soon as the matches that wrote its source have finished, computing its depth on
//   the way; the alternatives compute every depth first (k_depth) and then either copy with them (the
//   per-thread dataflow) or bucket the matches into per-level queues (k_hist/k_levels/k_scatter_w) that
//   one cooperative persistent launch (k_wave_w) drains level by level with a bounded grid barrier in
//   between, instead of one kernel launch per level as in the paper's H100 design.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "decode.h"
#include "tile.cuh"
#include "onepass.cuh"
#include "wave.cuh"

namespace aceapex {


// ------------------------------------------------------------------------------------------ reset
__global__ void k_reset(WsHead *head, StreamState *sst, const StreamDesc *descs, LaunchArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        head->epoch = head->epoch + 1 == 0 ? 1 : head->epoch + 1;
        head->ticket = 0; head->ticket2 = 0; head->bar_count = 0; head->bar_gen = 0;
        head->depth_seen = 0; head->n_levels = 0;
        for (int k = 0; k < 8; k++) head->phase[k] = 0;
    }
    if (i < a.n_streams) {
        const StreamDesc &sd = a.n_streams == 1 ? a.one : descs[i];
        if (sd.state) {
            sd.state->front = sd.tile_base;  // persistent state: only the launch-local frontier restarts
        } else {
            sst[i].front = sd.tile_base; sst[i].seq_sum = 0; sst[i].match_sum = 0; sst[i].depth_max = 0;
            sst[i].status = 0; sst[i].err_key = ~0ull;
        }
    }
}

// Header totals against the blocks' fields, then the status out (async API).
__global__ void k_finalize(StreamState *sst, const StreamDesc *descs, LaunchArgs a, int32_t *status_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_streams) return;
    const StreamDesc &sd = a.n_streams == 1 ? a.one : descs[i];
    StreamState &st = sd.state ? *sd.state : sst[i];
    // the header totals are checked when every tile ran to its end (no error, or only depth errors)
    const bool complete = st.err_key == ~0ull || (st.err_key >> 4) == kOrderDepth;
    if ((sd.flags & kDescLast) && complete &&
        (st.seq_sum != sd.n_seq || st.match_sum != sd.n_match || st.depth_max != sd.max_depth))
        st.err_key = (kOrderTotals << 4) | (unsigned long long)(-kErrFormat);
    st.status = st.err_key == ~0ull ? 0 : -(int)(st.err_key & 15);
    if (status_out) status_out[i] = st.status;
}


// ------------------------------------------------------------------------------------------ wavefront path
constexpr int kNT = 256, kSPT = 4;

// Prefix sum of the blocks' match counts (one CTA); block_base[n_blocks] = total, which must equal the
// header's n_match (the record arrays are sized from it).
__global__ void __launch_bounds__(kNT) k_match_base(StreamState *sst, LaunchArgs a, unsigned long long *block_base,
                                                    uint32_t *bdepth) {
    __shared__ ScanSmem<kNT> scan;
    __shared__ unsigned int s_depth;
    const StreamDesc &sd = a.one;
    if (threadIdx.x == 0) s_depth = 0;
    __syncthreads();
    unsigned long long run = 0;
    for (uint64_t b0 = 0; b0 < sd.n_blocks; b0 += kNT) {
        const uint64_t b = b0 + threadIdx.x;
        unsigned long long nm = 0;
        if (b < sd.n_blocks) {
            const uint64_t boff = ld64(sd.comp + kStreamHeader + 8 * b);
            if ((boff & 15) == 0 && boff + kBlockHeader <= sd.comp_len) {
                nm = ld32(sd.comp + boff + 4);
                const uint32_t bd = ld32(sd.comp + boff + 24);
                atomicMax(&s_depth, bd);
                bdepth[b] = bd;
            } else {
                report(&sst[0], kErrFormat, b << (sd.block_log2 - sd.tile_log2));
            }
        }
        unsigned long long tot;
        const unsigned long long ex = block_excl_scan<kNT>(nm, scan, tot);
        if (b < sd.n_blocks) block_base[b] = run + ex;
        run += tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        block_base[sd.n_blocks] = run;
        // header totals against the blocks, before any depth is computed (the level arrays are sized
        // from the header's max_depth)
        if (run != sd.n_match || s_depth != sd.max_depth) report(&sst[0], kErrFormat, kOrderTotals);
    }
}

// Parse every tile: literals to `out`, one record per match that starts in the tile, granule index.
__global__ void __launch_bounds__(kNT) k_parse(StreamState *sst, LaunchArgs a, WaveBufs wb) {
    __shared__ TileSmem<kNT, kSPT> sm;
    const StreamDesc &sd = a.one;
    StreamState *st = &sst[0];
    const uint32_t sh = sd.block_log2 - sd.tile_log2;
    const uint32_t gl = sd.tile_log2 < kGranuleLog2 ? sd.tile_log2 : kGranuleLog2;
    for (uint64_t t = blockIdx.x; t < sd.n_tiles; t += gridDim.x) {
        const uint64_t b = t >> sh;
        if (threadIdx.x == 0) {
            sm.err = 0; sm.verr = 0;
            sm.err = *(volatile int *)&st->status ? 1 : tile_open(sm, sd, b, (uint32_t)(t & ((1ull << sh) - 1)), st);
        }
        __syncthreads();
        if (sm.err) { if (threadIdx.x == 0 && sm.err < 0) report(st, sm.err, t); return; }
        tile_rewind(sm);
        const unsigned long long mb = wb.block_base[b], mb_next = wb.block_base[b + 1];
        while (sm.seq < sm.seq_end) {
            if (!chunk_parse(sm, true)) break;
            chunk_literals(sm, sd.out);
            const uint32_t n = sm.chunk_n, nm = sm.chunk_nm, cs = sm.chunk_seq;
            // match records: owned by the tile that holds the match's first byte
            for (uint32_t i = threadIdx.x; i < nm; i += kNT) {
                const uint32_t drel = sm.start[i] + sm.rlen[i];
                if (drel >= sm.tile_lo && drel < sm.tile_hi) {
                    const unsigned long long m = mb + cs + i;
                    if (m < mb_next && m < sd.n_match) {
                        wb.mdst[m] = sm.b0 + drel;
                        wb.msrc[m] = sm.soff[i];
                        wb.mlen[m] = sm.mlen[i];
                        wb.depth[m] = 0;
                    } else {
                        report(st, kErrFormat, t);
                    }
                }
            }
            // granule index: gidx[g] = first match whose range ends after the granule's first byte
            const uint32_t G = 1u << gl;
            uint32_t lo = sm.start[0] > sm.tile_lo ? sm.start[0] : sm.tile_lo;
            const uint32_t hi = sm.start[n] < sm.tile_hi ? sm.start[n] : sm.tile_hi;
            lo = (lo + G - 1) & ~(G - 1);
            for (uint32_t q = lo + threadIdx.x * G; q < hi; q += kNT * G) {
                const uint32_t i = seq_of(sm, n, q);
                wb.gidx[(sm.b0 + q) >> gl] = (i < nm) ? (uint32_t)(mb + cs + i) : (uint32_t)mb_next;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0 && sm.err) report(st, sm.err, t);
        __syncthreads();
    }
}

// Depth of every match (§7.1): 1 + the largest depth among the matches that wrote its effective source
// [s, s + min(L, d - s)); literal bytes count as depth 0.  Chunks of kNT matches are taken in index order;
// a writer always has a smaller index than its reader, so the lowest unfinished chunk can always finish.
// One thread copies its match once every writer of its source has published (COPY variant of k_depth):
// out[d+k] = out[s + (k mod (d-s))], loads through L2, pieces of at most 16 bytes.
__device__ __forceinline__ void thread_copy(uint8_t *out, uint64_t d, uint64_t s, uint64_t L) {
    const uint64_t p = d - s;
    if (p >= L) {
        for (uint64_t o = 0; o < L; o += 16) lane_copy_out(out, d + o, s + o, (uint32_t)(L - o < 16 ? L - o : 16));
    } else {
        uint32_t km = 0;
        for (uint64_t k = 0; k < L; k++) {
            out[d + k] = __ldcg(out + s + km);
            if (++km == (uint32_t)p) km = 0;
        }
    }
}

template <bool COPY>
__global__ void __launch_bounds__(kNT) k_depth(WsHead *head, StreamState *sst, LaunchArgs a, WaveBufs wb) {
    __shared__ unsigned long long s_c;
    __shared__ int s_abort;
    __shared__ unsigned int s_dmax;
    __shared__ uint32_t s_dep[kNT];  // depths of this chunk's matches (0 = not known yet)
    const StreamDesc &sd = a.one;
    const uint64_t nmatch = sd.n_match;
    const uint32_t gl = sd.tile_log2 < kGranuleLog2 ? sd.tile_log2 : kGranuleLog2;
    const uint32_t cap = sd.max_depth > 0 ? sd.max_depth : 1;
    const uint64_t t0 = global_ns();
    if (*(volatile int *)&sst[0].status) return;  // the parse failed: the records are not usable
    for (;;) {
        if (threadIdx.x == 0) { s_c = atomicAdd(&head->ticket2, 1ull); s_abort = 0; s_dmax = 0; }
        s_dep[threadIdx.x] = 0;
        __syncthreads();
        const uint64_t base = s_c * kNT;
        const uint64_t m = base + threadIdx.x;
        if (s_c * kNT >= nmatch) break;
        bool done = m >= nmatch;
        uint64_t s = 0, send = 0, w = 0, d = 0, L = 0;
        uint32_t mx = 0;
        if (!done) {
            d = wb.mdst[m];
            s = wb.msrc[m];
            L = wb.mlen[m];
            if (s < d && d + L <= sd.N) {  // records are checked by k_parse; stale ones (after an error) read nothing
                send = s + (L < d - s ? L : d - s);
                w = wb.gidx[s >> gl];
                while (w < m && wb.mdst[w] + wb.mlen[w] <= s) w++;
            } else {
                s = send = 0; w = m; L = 0;
            }
        }
        int iter = 0;
        while (__syncthreads_or(!done)) {
            if (!done) {
                // advance over writers whose depth is known; stop at the first unknown one
                while (w < m && wb.mdst[w] < send) {
                    // a writer of this chunk: its depth (and, COPY, its bytes) are visible after the CTA barrier
                    // of the loop; an earlier chunk's writer publishes its depth after its bytes (release/acquire)
                    const uint32_t dw = w >= base ? *(volatile uint32_t *)&s_dep[w - base]
                                                  : (COPY ? ld_acquire_u32(&wb.depth[w]) : ld_relaxed_u32(&wb.depth[w]));
                    if (dw == 0) break;
                    mx = dw > mx ? dw : mx;
                    w++;
                }
                if (!(w < m && wb.mdst[w] < send)) {
                    uint32_t dep = mx + 1;
                    // a match deeper than its block's max_depth field: the stream understates its depth
                    if (L && dep > wb.bdepth[d >> sd.block_log2]) report_depth(&sst[0]);
                    if (dep > cap) dep = cap;
                    if (COPY) {
                        if (L) thread_copy(sd.out, d, s, L);
                        __threadfence();
                        st_release_u32(&wb.depth[m], dep);
                    } else {
                        st_relaxed_u32(&wb.depth[m], dep);
                    }
                    s_dep[threadIdx.x] = dep;
                    atomicMax(&s_dmax, dep);  // one global atomic per chunk (below), not per match
                    done = true;
                }
            }
            if (++iter % 64 == 0 && threadIdx.x == 0 && global_ns() - t0 > a.wait_ns) {
                report(&sst[0], kErrTimeout, kOrderTimeout);
                s_abort = 1;
            }
            __syncthreads();
            if (s_abort) return;
        }
        if (threadIdx.x == 0 && s_dmax) atomicMax(&head->depth_seen, s_dmax);
    }
}

// Level histogram (shared-memory privatised for the first kHistSmem levels).
constexpr int kHistSmem = 2048;
__global__ void __launch_bounds__(kNT) k_hist(LaunchArgs a, WaveBufs wb) {
    __shared__ unsigned int h[kHistSmem];
    for (int i = threadIdx.x; i < kHistSmem; i += kNT) h[i] = 0;
    __syncthreads();
    const uint64_t n = a.one.n_match;
    for (uint64_t m = (uint64_t)blockIdx.x * kNT + threadIdx.x; m < n; m += (uint64_t)gridDim.x * kNT) {
        const uint32_t d = wb.depth[m];
        if (d > a.one.max_depth) continue;  // only after an error (k_depth clamps to max_depth)
        if (d < kHistSmem) atomicAdd(&h[d], 1u);
        else atomicAdd(&wb.hist[d], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kHistSmem && i <= (int)a.one.max_depth; i += kNT)
        if (h[i]) atomicAdd(&wb.hist[i], h[i]);
}

// Exclusive scan of the histogram into level offsets; cursor = offsets.
__global__ void __launch_bounds__(kNT) k_levels(WsHead *head, LaunchArgs a, WaveBufs wb) {
    __shared__ ScanSmem<kNT> scan;
    const uint32_t nl = a.one.max_depth + 1;  // levels 0..max_depth
    unsigned long long run = 0;
    for (uint32_t k0 = 0; k0 < nl; k0 += kNT) {
        const uint32_t k = k0 + threadIdx.x;
        const unsigned long long v = k < nl ? wb.hist[k] : 0;
        unsigned long long tot;
        const unsigned long long ex = block_excl_scan<kNT>(v, scan, tot);
        if (k < nl) { wb.lvl[k] = (uint32_t)(run + ex); wb.cursor[k] = (uint32_t)(run + ex); }
        run += tot;
    }
    if (threadIdx.x == 0) { wb.lvl[nl] = (uint32_t)run; head->n_levels = head->depth_seen; }
}

// ------------------------------------------------------------------------------------------ host side
const char *const kKernelNames[kKCount] = {"k_reset", "k_flat", "k_finalize", "k_match_base", "k_parse",
                                           "k_depth", "k_hist", "k_levels", "k_scatter", "k_wave", "k_flow"};
namespace {
struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<int> ids;  // kernel id of each recorded (start, stop) pair
    double ms[kKCount] = {};
    unsigned long long launches[kKCount] = {};
};
Prof &prof() {
    static Prof *p = new Prof();
    return *p;
}
cudaEvent_t prof_event() {
    Prof &P = prof();
    if (P.used == P.pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        P.pool.push_back(e);
    }
    return P.pool[P.used++];
}
}  // namespace

void prof_enable(bool on) {
    Prof &P = prof();
    P.on = on;
    P.used = 0;
    P.ids.clear();
    for (int i = 0; i < kKCount; i++) { P.ms[i] = 0; P.launches[i] = 0; }
}
bool prof_enabled() { return prof().on; }
void prof_mark(int id, bool start, cudaStream_t stream) {
    Prof &P = prof();
    if (!P.on) return;
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) return;
    if (start) P.ids.push_back(id);
    cudaEventRecord(prof_event(), stream);
}
int prof_collect(double *ms, unsigned long long *launches) {
    Prof &P = prof();
    for (size_t k = 0; k < P.ids.size() && 2 * k + 1 < P.used; k++) {
        cudaEventSynchronize(P.pool[2 * k + 1]);
        float t = 0;
        cudaEventElapsedTime(&t, P.pool[2 * k], P.pool[2 * k + 1]);
        P.ms[P.ids[k]] += t;
        P.launches[P.ids[k]] += 1;
    }
    P.used = 0;
    P.ids.clear();
    for (int i = 0; i < kKCount; i++) { ms[i] = P.ms[i]; launches[i] = P.launches[i]; }
    return kKCount;
}

#define PROF(id, ...) do { prof_mark(id, true, stream); __VA_ARGS__; prof_mark(id, false, stream); } while (0)

// The one-pass kernel with `warps` warps per CTA (2, 4 or 8): persistent grid of as many CTAs per SM as
// fit (or cfg.ctas_per_sm), at most one warp per tile.
template <int WARPS>
static cudaError_t launch_k_flat(const LaunchCfg &cfg, WsHead *head, StreamState *sst, uint32_t *flags,
                                 const StreamDesc *descs, const LaunchArgs &a, cudaStream_t stream) {
    const size_t dyn = sizeof(F4Warp) * WARPS;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_flat<WARPS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_flat<WARPS>, 32 * WARPS, dyn);
    if (e != cudaSuccess) return e;
    if (cfg.ctas_per_sm > 0 && cfg.ctas_per_sm < occ) occ = cfg.ctas_per_sm;
    if (occ < 1) occ = 1;
    uint64_t grid = (uint64_t)occ * cfg.num_sms;
    const uint64_t need = (a.total_tiles + WARPS - 1) / WARPS;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    PROF(kKFlat, k_flat<WARPS><<<(unsigned)grid, 32 * WARPS, dyn, stream>>>(head, sst, flags, descs, a));
    return cudaGetLastError();
}

cudaError_t launch_flat(const LaunchCfg &cfg, WsHead *head, StreamState *sst, uint32_t *flags, const StreamDesc *descs,
                        const LaunchArgs &a, int32_t *status_out, cudaStream_t stream) {
    const int ns = a.n_streams;
    PROF(kKReset, k_reset<<<(ns + 255) / 256, 256, 0, stream>>>(head, sst, descs, a));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (a.total_tiles > 0) {
        // the one-pass kernel keeps positions in 32 bits and needs tiles of at most 4 KiB; the host sends
        // every other stream down the wavefront path
        if (a.max_tile_log2 > (unsigned)kWarpImgLog2 || a.max_n > kF4MaxN || a.total_tiles >= (1ull << 31))
            return cudaErrorInvalidValue;
        e = cfg.warps == 2 ? launch_k_flat<2>(cfg, head, sst, flags, descs, a, stream)
          : cfg.warps == 8 ? launch_k_flat<8>(cfg, head, sst, flags, descs, a, stream)
                           : launch_k_flat<4>(cfg, head, sst, flags, descs, a, stream);
        if (e != cudaSuccess) return e;
    }
    PROF(kKFinalize, k_finalize<<<(ns + 255) / 256, 256, 0, stream>>>(sst, descs, a, status_out));
    return cudaGetLastError();
}

cudaError_t launch_wave(const LaunchCfg &cfg, WsHead *head, StreamState *sst, const LaunchArgs &a, const WaveBufs &wb,
                        int32_t *status_out, cudaStream_t stream) {
    PROF(kKReset, k_reset<<<1, 256, 0, stream>>>(head, sst, nullptr, a));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const StreamDesc &sd = a.one;
    if (sd.N > 0) {
        cudaMemsetAsync(wb.hist, 0, sizeof(uint32_t) * (sd.max_depth + 2), stream);
        PROF(kKMatchBase, k_match_base<<<1, kNT, 0, stream>>>(sst, a, wb.block_base, wb.bdepth));
        if (sd.tile_log2 <= (uint32_t)kWarpImgLog2) {
            const size_t dyn = sizeof(WarpSmem) * kWarpsPerCta;
            static bool attr = false;
            if (!attr) {
                e = cudaFuncSetAttribute(k_parse_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
                if (e != cudaSuccess) return e;
                attr = true;
            }
            int pocc = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pocc, k_parse_w, 32 * kWarpsPerCta, dyn);
            const uint64_t need = (sd.n_tiles + kWarpsPerCta - 1) / kWarpsPerCta;
            const uint64_t pg = std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)std::max(pocc, 1) * cfg.num_sms));
            PROF(kKParse, k_parse_w<<<(unsigned)pg, 32 * kWarpsPerCta, dyn, stream>>>(sst, a, wb));
        } else {
            const uint64_t ptiles = std::min<uint64_t>(sd.n_tiles, (uint64_t)cfg.num_sms * 8);
            PROF(kKParse, k_parse<<<(unsigned)std::max<uint64_t>(ptiles, 1), kNT, 0, stream>>>(sst, a, wb));
        }
        if (sd.n_match > 0 && cfg.wave_sched == 2) {
            // warp-granular dataflow: copies and depths in one persistent launch, then the level histogram
            int occ = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_flow_w, 32 * kFlowWarps, 0);
            const uint64_t groups = (sd.n_match + 31) / 32;
            const uint64_t fgrid = std::min<uint64_t>((groups + kFlowWarps - 1) / kFlowWarps,
                                                      (uint64_t)std::max(occ, 1) * cfg.num_sms);
            PROF(kKFlow, k_flow_w<<<(unsigned)fgrid, 32 * kFlowWarps, 0, stream>>>(head, sst, a, wb));
            const unsigned g = (unsigned)std::min<uint64_t>((sd.n_match + kNT - 1) / kNT, (uint64_t)cfg.num_sms * 4);
            PROF(kKHist, k_hist<<<g, kNT, 0, stream>>>(a, wb));
            PROF(kKFinalize, k_finalize<<<1, 32, 0, stream>>>(sst, nullptr, a, status_out));
            return cudaGetLastError();
        }
        if (sd.n_match > 0) {
            int occ = 0;
            const bool flow = cfg.wave_sched == 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, flow ? k_depth<true> : k_depth<false>, kNT, 0);
            const uint64_t chunks = (sd.n_match + kNT - 1) / kNT;
            const uint64_t dgrid = std::min<uint64_t>(chunks, (uint64_t)std::max(occ, 1) * cfg.num_sms);
            if (flow) PROF(kKDepth, k_depth<true><<<(unsigned)dgrid, kNT, 0, stream>>>(head, sst, a, wb));
            else PROF(kKDepth, k_depth<false><<<(unsigned)dgrid, kNT, 0, stream>>>(head, sst, a, wb));
            const unsigned g = (unsigned)std::min<uint64_t>(chunks, (uint64_t)cfg.num_sms * 4);
            PROF(kKHist, k_hist<<<g, kNT, 0, stream>>>(a, wb));
            if (flow) {  // matches were copied as their writers published: no level queues needed
                PROF(kKFinalize, k_finalize<<<1, 32, 0, stream>>>(sst, nullptr, a, status_out));
                return cudaGetLastError();
            }
            PROF(kKLevels, k_levels<<<1, kNT, 0, stream>>>(head, a, wb));
            PROF(kKScatter, k_scatter_w<<<g, 256, 0, stream>>>(a, wb));
            // one 1024-thread CTA per SM: few arrivals per grid barrier
            unsigned wgrid = (unsigned)cfg.num_sms;
            void *args[] = {(void *)&head, (void *)&sst, (void *)&a, (void *)&wb};
            PROF(kKWave, e = cudaLaunchCooperativeKernel((void *)k_wave_w, wgrid, 1024, args, 0, stream));
            if (e != cudaSuccess) return e;
        }
    }
    PROF(kKFinalize, k_finalize<<<1, 32, 0, stream>>>(sst, nullptr, a, status_out));
    return cudaGetLastError();
}

}  // namespace aceapex

namespace aceapex {
__global__ void k_gather_status(int n, const int32_t *map, const int32_t *flat, const int32_t *wave, int32_t *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t kind = map[2 * i], v = map[2 * i + 1];
    out[i] = kind == 0 ? v : kind == 1 ? flat[v] : wave[v];
}
cudaError_t launch_gather_status(int n, const int32_t *map, const int32_t *flat, const int32_t *wave, int32_t *out,
                                 cudaStream_t stream) {
    k_gather_status<<<(n + 255) / 256, 256, 0, stream>>>(n, map, flat, wave, out);
    return cudaGetLastError();
}
}  // namespace aceapex

// Fresh persistent state of a served request (stream-ordered, no host memory involved).
namespace aceapex {
__global__ void k_state_init(StreamState *st) {
    st->front = 0; st->seq_sum = 0; st->match_sum = 0; st->err_key = ~0ull; st->depth_max = 0; st->status = 0;
}
}  // namespace aceapex
namespace aceapex_host {
int init_state(aceapex::StreamState *st, cudaStream_t stream) {
    aceapex::k_state_init<<<1, 1, 0, stream>>>(st);
    return cudaGetLastError() == cudaSuccess ? 0 : -6;
}
}  // namespace aceapex_host

// ================================================================================================ no-alloc entry
// Some callers cannot allocate device memory at decode time: code running under a memory budget that
// was fixed up front (a serving process that pre-sized its pools), real-time or embedded callers that
// forbid allocation on the decode path, or libraries that must not touch the application's allocator.
// aceapex_decode_noalloc decodes with scratch that exists before any call: a fixed array in the module's
// static device memory, held by every GPU that loads the library until the process exits.
#include "../../include/aceapex.h"
using namespace aceapex;
namespace {

// Scratch of the one-pass decode: launch head | stream state | per-tile flags | literal bitmap (one bit per
// output byte).  16 MiB: streams of up to ~127 MiB of output at 4 KiB tiles.
constexpr size_t kNoAllocBytes = 16u << 20;
constexpr size_t kNoAllocFlags = 1024;  // byte offset of the flags region
static_assert(sizeof(WsHead) <= 512 && sizeof(StreamState) <= 256, "no-alloc scratch layout");
__device__ __align__(256) static uint8_t g_noalloc_scratch[kNoAllocBytes];

// In host code the array's name is only a stand-in: the device address comes from cudaGetSymbolAddress,
// looked up once per device (with that device current, under a lock) and kept here.
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices];
int g_noalloc_sms[kMaxDevices];

}  // namespace

extern "C" int aceapex_decode_noalloc(const void *comp, size_t comp_len, void *out, size_t out_len,
                                      const aceapex_info *info, int32_t *d_status, void *stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    if (!comp || comp_len < kStreamHeader || ((uintptr_t)comp & 15) || (!out && out_len) || !info || !d_status)
        return kErrArg;
    if (info->comp_len != comp_len || info->decoded_len != out_len) return kErrSize;
    // only the one-pass kernel fits the fixed scratch: streams of depth <= 1 and tiles of at most 4 KiB whose
    // flags and literal bitmap fit
    const uint64_t flag_bytes = (4 * info->n_tiles + 255) & ~255ull;
    if (info->max_depth > 1 || info->tile_log2 > (uint32_t)kWarpImgLog2 || info->decoded_len > kF4MaxN ||
        info->n_tiles > (kNoAllocBytes - kNoAllocFlags) / 4 ||
        kNoAllocFlags + flag_bytes + 4 * litmap_words(info->decoded_len) > kNoAllocBytes)
        return kErrNomem;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) { cudaGetLastError(); return kErrCuda; }
    void *addr = nullptr;
    int sms = 0;
    {
        std::lock_guard<std::mutex> g(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) { cudaGetLastError(); return kErrCuda; }
            int n = 0;
            if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
                cudaGetLastError();
                return kErrCuda;
            }
            g_noalloc_sms[dev] = n;
            g_noalloc_addr[dev] = p;
        }
        addr = g_noalloc_addr[dev];
        sms = g_noalloc_sms[dev];
    }
    uint8_t *base = (uint8_t *)addr;
    WsHead *head = (WsHead *)base;
    StreamState *sst = (StreamState *)(base + 512);
    uint32_t *flags = (uint32_t *)(base + kNoAllocFlags);
    uint32_t *litmap = (uint32_t *)(base + kNoAllocFlags + flag_bytes);
    if (info->decoded_len == 0) return cudaMemsetAsync(d_status, 0, 4, stream) == cudaSuccess ? kOK : kErrCuda;
    LaunchArgs a{};
    StreamDesc &d = a.one;
    d.comp = (const uint8_t *)comp; d.out = (uint8_t *)out; d.comp_len = comp_len; d.N = info->decoded_len;
    d.n_blocks = info->n_blocks; d.n_seq = info->n_seq; d.n_match = info->n_match; d.tile_base = 0;
    d.n_tiles = info->n_tiles; d.tile_off = 0; d.state = nullptr; d.litmap = litmap; d.block_log2 = info->block_log2;
    d.tile_log2 = info->tile_log2; d.min_match = info->min_match; d.max_depth = info->max_depth; d.flags = kDescLast;
    a.n_streams = 1;
    a.total_tiles = info->n_tiles;
    a.wait_ns = 4000000000ull;
    a.withhold = ~0ull;
    a.max_tile_log2 = info->tile_log2;
    a.phase = nullptr;
    // k_reset zeroes the launch head and stream state of every call; the tile flags need no clearing (they
    // hold the epoch of the call that last published them, and each call runs with a new epoch), nor does
    // the literal bitmap (every tile writes all of its bits before it publishes)
    k_reset<<<1, 256, 0, stream>>>(head, sst, nullptr, a);
    const size_t dyn = sizeof(F4Warp) * kF4Warps;  // below the 48 KiB default: no attribute needed
    static_assert(sizeof(F4Warp) * kF4Warps <= 48 * 1024, "no-alloc launch needs no shared-memory attribute");
    const uint64_t need = (a.total_tiles + kF4Warps - 1) / kF4Warps;
    const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)sms * 4));
    k_flat<kF4Warps><<<(unsigned)grid, 32 * kF4Warps, dyn, stream>>>(head, sst, flags, nullptr, a);
    k_finalize<<<1, 32, 0, stream>>>(sst, nullptr, a, d_status);
    return cudaGetLastError() == cudaSuccess ? kOK : kErrCuda;
}
