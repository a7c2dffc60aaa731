// One-pass decode of a tile through a shared-memory image of its output (tiles of at most 2^kImgLog2
// bytes).  Compared with writing bytes straight to HBM, the image turns every global store into a
// coalesced 16-byte vector store, lets sources inside the tile be read from shared memory, and keeps the
// per-sequence arrays of a tile in shared memory between the two phases so that a tile is parsed once.
//
//   phase A: parse, literal bytes -> image, image -> out, publish the tile's flag
//   phase B: wait for earlier tiles' literals, match bytes -> image (sources: image or out), image -> out
//
// Bytes are placed warp-window by warp-window: lane j of a warp handles output byte q + j, so that the
// image stores, the literal loads (consecutive runs are adjacent in lit[]) and the match-source loads
// (consecutive bytes of one match are consecutive source bytes) of a warp instruction touch a few cache
// sectors.  The sequence that covers each lane's byte comes from one warp-wide OR of the next 31
// sequence starts and a population count, with no per-byte search.
#pragma once
#include "decode.h"
#include "tile.cuh"

namespace aceapex {

constexpr int kImgLog2 = 14;  // largest tile handled through the image

template <int NT, int SPT>
struct FlatSmem {
    TileSmem<NT, SPT> t;
    alignas(16) uint8_t img[(1 << kImgLog2) + 16];
    uint32_t shift;  // image byte of the tile's first byte (aligns the image with HBM)
};

// Image bytes [shift, shift + (hi-lo)) -> out[b0+lo .. b0+hi): 16-byte stores, byte stores at the edges.
template <int NT, int SPT>
__device__ void image_store(const FlatSmem<NT, SPT> &fs, uint8_t *out) {
    const TileSmem<NT, SPT> &sm = fs.t;
    uint8_t *base = out + sm.b0 + sm.tile_lo - fs.shift;  // 16-byte aligned
    const uint32_t total = fs.shift + (sm.tile_hi - sm.tile_lo);
    const uint32_t ng = (total + 15) >> 4;
    for (uint32_t g = threadIdx.x; g < ng; g += NT) {
        const uint32_t lo = g << 4, hi = lo + 16;
        if (lo >= fs.shift && hi <= total) {
            *reinterpret_cast<uint4 *>(base + lo) = *reinterpret_cast<const uint4 *>(fs.img + lo);
        } else {
            const uint32_t a = lo > fs.shift ? lo : fs.shift, z = hi < total ? hi : total;
            for (uint32_t x = a; x < z; x++) base[x] = fs.img[x];
        }
    }
}

// The chunk's bytes inside the tile -> image.  MATCHES = false: literal bytes (from lit[]); true: match
// bytes, out[d+k] = out[s + (k mod (d-s))], read from the image when the source lies in this tile (its
// literal bytes are there) and from out otherwise (earlier tiles' literal bytes, published).
template <int NT, int SPT, bool MATCHES>
__device__ void image_window_pass(FlatSmem<NT, SPT> &fs, const uint8_t *out) {
    const TileSmem<NT, SPT> &sm = fs.t;
    const uint32_t n = sm.chunk_n;
    const uint32_t lo = sm.start[0] > sm.tile_lo ? sm.start[0] : sm.tile_lo;
    const uint32_t hi = sm.start[n] < sm.tile_hi ? sm.start[n] : sm.tile_hi;
    if (hi <= lo) return;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr uint32_t NW = NT / 32;
    const uint32_t per = (((hi - lo) + NW - 1) / NW + 31) & ~31u;  // contiguous stretch per warp
    const uint32_t w0 = lo + warp * per;
    const uint32_t w1 = (w0 + per) < hi ? w0 + per : hi;
    if (w0 >= w1) return;
    const uint64_t tile_abs = sm.b0 + sm.tile_lo;
    uint8_t *img = const_cast<uint8_t *>(fs.img) + fs.shift;  // img[x - tile_lo] holds block-relative byte x
    uint32_t i0 = seq_of(sm, n, w0);                           // sequence containing w0
    constexpr int U = 8;  // windows in flight per warp: their loads are issued before any is consumed
    for (uint32_t q = w0; q < w1; q += 32 * U) {
        uint32_t seq_u[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint32_t qq = q + 32 * u;
            // starts of the next 31 sequences that fall in [qq, qq+32) -> bit mask (start[i0+k] > qq, k >= 1)
            uint32_t bit = 0;
            if (lane >= 1 && i0 + lane < n) {
                const uint32_t sk = sm.start[i0 + lane] - qq;
                if (sk < 32) bit = 1u << sk;
            }
            const uint32_t M = __reduce_or_sync(0xffffffffu, bit);
            seq_u[u] = i0 + __popc(M & ((2u << lane) - 1u));
            // sequence containing qq + 32: the one holding qq + 31, or the next one if it starts there
            i0 += __popc(M);
            if (i0 + 1 < n && sm.start[i0 + 1] <= qq + 32) i0++;
        }
        uint32_t val[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint32_t x = q + 32 * u + lane;
            val[u] = 0x100;  // nothing to write
            if (x < w1) {
                const uint32_t i = seq_u[u];
                const uint32_t rel = x - sm.start[i], r = sm.rlen[i];
                if (!MATCHES) {
                    if (rel < r) val[u] = __ldg(sm.lit + sm.loff[i] + rel);
                } else if (rel >= r) {
                    const uint64_t k = rel - r, d = sm.b0 + sm.start[i] + r, s = sm.soff[i], p = d - s;
                    const uint64_t src = s + (k < p ? k : (uint64_t)((uint32_t)k % (uint32_t)p));
                    val[u] = src >= tile_abs ? img[src - tile_abs] : __ldca(out + src);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++)
            if (val[u] < 0x100) img[q + 32 * u + lane - sm.tile_lo] = (uint8_t)val[u];
    }
}

template <int NT, int SPT>
__global__ void __launch_bounds__(NT) k_flat2(WsHead *head, StreamState *sst, uint32_t *flags,
                                              const StreamDesc *descs, LaunchArgs a) {
    extern __shared__ uint4 dyn_smem[];
    FlatSmem<NT, SPT> &fs = *reinterpret_cast<FlatSmem<NT, SPT> *>(dyn_smem);
    TileSmem<NT, SPT> &sm = fs.t;
    __shared__ unsigned long long s_t;
    __shared__ int s_si;
    constexpr uint32_t CH = NT * SPT;
    const uint32_t epoch = head->epoch;
    unsigned long long ph[kPhases] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long tc = clock64();
#define PHASE(k) do { if (a.phase && threadIdx.x == 0) { const long long now = clock64(); ph[k] += now - tc; tc = now; } } while (0)
    for (;;) {
        if (threadIdx.x == 0) {
            s_t = atomicAdd(&head->ticket, 1ull);
            s_si = (s_t < a.total_tiles) ? (a.n_streams == 1 ? 0 : find_stream(descs, a.n_streams, s_t)) : 0;
        }
        __syncthreads();
        const unsigned long long t = s_t;
        if (t >= a.total_tiles) break;
        const int si = s_si;
        const StreamDesc &sd = a.n_streams == 1 ? a.one : descs[si];
        StreamState *st = sd.state ? sd.state : &sst[si];
        const unsigned long long order = t - sd.tile_base + sd.tile_off;
        if (threadIdx.x == 0) {
            const uint32_t sh = sd.block_log2 - sd.tile_log2;
            sm.err = 0; sm.verr = 0;
            sm.err = *(volatile int *)&st->status ? 1 : tile_open(sm, sd, order >> sh, (uint32_t)(order & ((1ull << sh) - 1)), st);
            fs.shift = (uint32_t)((uintptr_t)(sd.out + sm.b0 + sm.tile_lo) & 15);
        }
        __syncthreads();
        PHASE(0);
        ph[7] += 1;
        // a tile whose sequences fit one chunk is parsed once; its arrays serve both phases
        const bool single = !sm.err && (sm.seq_end - sm.e_seq) <= CH;
        if (!sm.err) {
            tile_rewind(sm);
            while (sm.seq < sm.seq_end) {
                if (!chunk_parse(sm, single)) break;
                PHASE(1);
                image_window_pass<NT, SPT, false>(fs, sd.out);
                __syncthreads();
                PHASE(2);
            }
            if (!sm.err) image_store(fs, sd.out);
        }
        __threadfence();
        __syncthreads();
        const int err_a = sm.err;
        if (threadIdx.x == 0) {
            if (err_a < 0) report(st, err_a, order);
            if (t != a.withhold) st_release_u32(&flags[t], epoch);
        }
        PHASE(3);
        if (!err_a) {
            if (threadIdx.x < 32) {
                unsigned long long f = ld_acquire_u64(&st->front);
                if (f < sd.tile_base) f = sd.tile_base;
                const uint64_t t0 = global_ns();
                bool timed_out = false;
                while (f < t) {
                    const unsigned long long k = f + threadIdx.x;
                    const bool done = k >= t || ld_acquire_u32(&flags[k]) == epoch;
                    const unsigned ball = __ballot_sync(0xffffffffu, done);
                    if (ball == 0xffffffffu) { f += 32; continue; }
                    f += __ffs(~ball) - 1;
                    if (global_ns() - t0 > a.wait_ns) { timed_out = true; break; }
                    __nanosleep(64);
                }
                if (threadIdx.x == 0) {
                    if (timed_out) { report(st, kErrTimeout, kOrderTimeout); sm.err = kErrTimeout; }
                    else atomicMax(&st->front, t < f ? t : f);
                }
            }
            __syncthreads();
            PHASE(4);
            if (!sm.err) {
                if (single) {
                    image_window_pass<NT, SPT, true>(fs, sd.out);
                    __syncthreads();
                } else {
                    tile_rewind(sm);
                    while (sm.seq < sm.seq_end) {
                        if (!chunk_parse(sm, true)) break;
                        image_window_pass<NT, SPT, true>(fs, sd.out);
                        __syncthreads();
                    }
                }
                PHASE(5);
                if (!sm.err) image_store(fs, sd.out);
                __syncthreads();
                PHASE(6);
                if (threadIdx.x == 0 && sm.err) report(st, sm.err, order);
            }
        }
        __syncthreads();
    }
    if (a.phase && threadIdx.x == 0)
        for (int k = 0; k < kPhases; k++) atomicAdd(&a.phase[k], ph[k]);
#undef PHASE
}

}  // namespace aceapex
