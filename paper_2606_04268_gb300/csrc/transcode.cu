// Transcoding a stream into a globally chain-flattened stream, on the GPU (chain flattening of §3.3 applied
// to an existing stream; the match dependencies of §7.1 order the root computation).  Every match byte has a root, the
// literal byte it ultimately copies: a literal byte is its own root, and byte k of a match with destination
// d, source s and period p = d - s has the root of byte s + (k mod p).  Each match becomes
//   - itself, when it overlaps itself (p < L) and its effective source [s, d) is literal;
//   - else, for a short repeat (p < L, p <= 32, L - p >= min_match): its first period as literal bytes, then
//     the self-overlapping match (d + p, d, L - p) that reads them;
//   - else the maximal runs of its bytes with consecutive roots, each at least min_match long a match copying
//     from the root of its first byte; shorter runs become literal bytes.
// Every match of the result reads literal bytes only (depth 1).  The result keeps the stream's block size,
// tile size and min_match, and has flatten mode 2 and no depth cap.
//
// Device steps:
//   1. k_tc_root_init: root[y] = y for every output byte;
//   2. the decode by the wavefront path's warp dataflow (api.cpp, k_flow_w): every match is copied once the
//      matches that wrote its source bytes are done, and its bytes' roots with it, root[d + k] =
//      root[s + (k mod p)] (§7.1 orders the work without level barriers); each match's record stays in the
//      workspace in stream order;
//   3. k_tc_pieces<false> counts the matches each match becomes, k_tc_scan_* turn the counts into offsets,
//      k_tc_pieces<true> writes them (destination, source, length) in destination order;
//   4. k_tc_block_sizes: per block its sequence count, section sizes, offset width and size; the host lays
//      out the stream header and the block index;
//   5. k_tc_write: per block the block header, the sync table, the cmd/len varints, the offsets and the
//      literal bytes.
// Positions are 32-bit: streams of up to 2^32 - 1 decoded bytes.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/aceapex.h"
#include "decode.h"
#include "device_common.cuh"

using namespace aceapex;

namespace aceapex_host {
int tc_parse_header(const uint8_t *h, size_t len, aceapex_info *info);
size_t tc_workspace_size(const aceapex_info &I);
int tc_decode(const void *comp, void *out, const aceapex_info &I, uint8_t *ws, WaveBufs *wb, uint32_t *root,
              int32_t *status, int *num_sms, cudaStream_t stream);
}  // namespace aceapex_host

namespace aceapex {

constexpr uint32_t kTcPeriodMax = 32;  // short repeats restart from literal bytes up to this period
constexpr uint32_t kTcLaneMax = 64;    // matches up to this length are examined by one lane, longer by a warp
constexpr int kTcNT = 256;
constexpr int kTcItems = 16;           // scan items per thread

struct TcBlock {  // per block of the result
    uint32_t n_seq, n_match, n_lit, cmd_bytes, len_bytes, w, n_tiles, pad;
    unsigned long long size;
};

__device__ __forceinline__ uint32_t vlen(uint32_t v) { return v < (1u << 7) ? 1 : v < (1u << 14) ? 2 : v < (1u << 21) ? 3 : v < (1u << 28) ? 4 : 5; }
__device__ __forceinline__ uint32_t put_varint(uint8_t *p, uint32_t v) {
    uint32_t n = 0;
    while (v >= 0x80) { p[n++] = (uint8_t)(v | 0x80); v >>= 7; }
    p[n++] = (uint8_t)v;
    return n;
}
__device__ __forceinline__ void put_le(uint8_t *p, uint64_t v, uint32_t n) {
    for (uint32_t i = 0; i < n; i++) p[i] = (uint8_t)(v >> (8 * i));
}
__device__ __forceinline__ void put32(uint8_t *p, uint32_t v) { put_le(p, v, 4); }

// ------------------------------------------------------------------------------------------ roots
__global__ void k_tc_root_init(uint32_t *root, uint64_t n4) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t y = (uint32_t)(4 * i);
        reinterpret_cast<uint4 *>(root)[i] = make_uint4(y, y + 1, y + 2, y + 3);
    }
}

// ------------------------------------------------------------------------------------------ pieces
__device__ __forceinline__ void tc_put(uint32_t *pd, uint32_t *ps, uint32_t *pl, uint32_t at, uint32_t d, uint32_t s,
                                       uint32_t L) {
    pd[at] = d; ps[at] = s; pl[at] = L;
}

// The matches that match (d, s, L) becomes, examined by one lane; written from index `at` when EMIT.
template <bool EMIT>
__device__ uint32_t tc_match_lane(uint32_t d, uint32_t s, uint32_t L, const uint32_t *__restrict__ root, uint32_t mm,
                                  uint32_t *pd, uint32_t *ps, uint32_t *pl, uint32_t at) {
    const uint32_t p = d - s;
    if (p < L) {
        bool lit = true;
        for (uint32_t j = 0; j < p && lit; j++) lit = __ldg(root + s + j) == s + j;
        if (lit) { if (EMIT) tc_put(pd, ps, pl, at, d, s, L); return 1; }
        if (p <= kTcPeriodMax && L - p >= mm) { if (EMIT) tc_put(pd, ps, pl, at, d + p, d, L - p); return 1; }
    }
    uint32_t n = 0, k0 = 0, r0 = __ldg(root + d), prev = r0;
    for (uint32_t k = 1; k <= L; k++) {
        uint32_t v = 0;
        if (k < L) {
            v = __ldg(root + d + k);
            if (v == prev + 1) { prev = v; continue; }
        }
        if (k - k0 >= mm) { if (EMIT) tc_put(pd, ps, pl, at + n, d + k0, r0, k - k0); n++; }
        k0 = k; r0 = v; prev = v;
    }
    return n;
}

// The same, examined by the whole warp (every lane passes the same match); lane 0 writes.
template <bool EMIT>
__device__ uint32_t tc_match_warp(uint32_t d, uint32_t s, uint32_t L, const uint32_t *__restrict__ root, uint32_t mm,
                                  uint32_t *pd, uint32_t *ps, uint32_t *pl, uint32_t at) {
    const uint32_t lane = threadIdx.x & 31, p = d - s;
    if (p < L) {
        bool lit = true;
        for (uint32_t j0 = 0; j0 < p && lit; j0 += 32) {
            const uint32_t j = j0 + lane;
            lit = __all_sync(0xffffffffu, j >= p || __ldg(root + s + j) == s + j);
        }
        if (lit) { if (EMIT && lane == 0) tc_put(pd, ps, pl, at, d, s, L); return 1; }
        if (p <= kTcPeriodMax && L - p >= mm) {
            if (EMIT && lane == 0) tc_put(pd, ps, pl, at, d + p, d, L - p);
            return 1;
        }
    }
    uint32_t n = 0, k0 = 0, r0 = 0, carry = 0;
    for (uint32_t base = 0; base < L; base += 32) {
        const uint32_t k = base + lane;
        const uint32_t v = k < L ? __ldg(root + d + k) : 0u;
        uint32_t up = __shfl_up_sync(0xffffffffu, v, 1);
        if (lane == 0) up = carry;
        unsigned brk = __ballot_sync(0xffffffffu, k < L && (k == 0 || v != up + 1));
        while (brk) {
            const int o = __ffs(brk) - 1;
            brk &= brk - 1;
            const uint32_t kb = base + o, rb = __shfl_sync(0xffffffffu, v, o);
            if (kb > 0 && kb - k0 >= mm) {
                if (EMIT && lane == 0) tc_put(pd, ps, pl, at + n, d + k0, r0, kb - k0);
                n++;
            }
            k0 = kb; r0 = rb;
        }
        carry = __shfl_sync(0xffffffffu, v, 31);
    }
    if (L - k0 >= mm) {
        if (EMIT && lane == 0) tc_put(pd, ps, pl, at + n, d + k0, r0, L - k0);
        n++;
    }
    return n;
}

// Matches in stream order, 32 per warp: cnt[m] = the number of matches match m becomes (!EMIT), or those
// matches written from base[m] on (EMIT).
template <bool EMIT>
__global__ void __launch_bounds__(kTcNT) k_tc_pieces(WaveBufs wb, unsigned long long nm, const uint32_t *__restrict__ root,
                                                     uint32_t mm, uint32_t *cnt, const uint32_t *base, uint32_t *pd,
                                                     uint32_t *ps, uint32_t *pl) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (kTcNT / 32);
    for (uint64_t g = 32 * ((uint64_t)blockIdx.x * (kTcNT / 32) + (threadIdx.x >> 5)); g < nm; g += 32 * warps) {
        const uint64_t m = g + lane;
        const bool valid = m < nm;
        uint32_t d = 0, s = 0, L = 0, at = 0, n = 0;
        if (valid) {
            d = (uint32_t)wb.mdst[m]; s = (uint32_t)wb.msrc[m]; L = wb.mlen[m];
            if (EMIT) at = base[m];
        }
        if (valid && L <= kTcLaneMax) n = tc_match_lane<EMIT>(d, s, L, root, mm, pd, ps, pl, at);
        unsigned longs = __ballot_sync(0xffffffffu, valid && L > kTcLaneMax);
        while (longs) {
            const int o = __ffs(longs) - 1;
            longs &= longs - 1;
            const uint32_t c = tc_match_warp<EMIT>(__shfl_sync(0xffffffffu, d, o), __shfl_sync(0xffffffffu, s, o),
                                                   __shfl_sync(0xffffffffu, L, o), root, mm, pd, ps, pl,
                                                   __shfl_sync(0xffffffffu, at, o));
            if ((int)lane == o) n = c;
        }
        if (!EMIT && valid) cnt[m] = n;
    }
}

// ------------------------------------------------------------------------------------------ scan
// Exclusive prefix sum of cnt[0, n) into out[0, n]; out[n] = the total.  Three launches: per-CTA sums of
// kTcNT * kTcItems items, a one-CTA scan of those sums, then each CTA's items.
__global__ void __launch_bounds__(kTcNT) k_tc_scan_part(const uint32_t *cnt, unsigned long long n,
                                                        unsigned long long *part) {
    __shared__ ScanSmem<kTcNT> sm;
    const uint64_t i0 = ((uint64_t)blockIdx.x * kTcNT + threadIdx.x) * kTcItems;
    unsigned long long v = 0;
    for (int j = 0; j < kTcItems; j++) if (i0 + j < n) v += cnt[i0 + j];
    unsigned long long tot;
    block_excl_scan<kTcNT>(v, sm, tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}
__global__ void __launch_bounds__(kTcNT) k_tc_scan_top(unsigned long long *part, unsigned long long np, uint32_t *out,
                                                       unsigned long long n) {
    __shared__ ScanSmem<kTcNT> sm;
    unsigned long long run = 0;
    for (uint64_t c0 = 0; c0 < np; c0 += kTcNT) {
        const uint64_t c = c0 + threadIdx.x;
        const unsigned long long v = c < np ? part[c] : 0ull;
        unsigned long long tot;
        const unsigned long long ex = block_excl_scan<kTcNT>(v, sm, tot);
        if (c < np) part[c] = run + ex;
        run += tot;
    }
    if (threadIdx.x == 0) out[n] = (uint32_t)run;
}
__global__ void __launch_bounds__(kTcNT) k_tc_scan_down(const uint32_t *cnt, unsigned long long n,
                                                        const unsigned long long *part, uint32_t *out) {
    __shared__ ScanSmem<kTcNT> sm;
    const uint64_t i0 = ((uint64_t)blockIdx.x * kTcNT + threadIdx.x) * kTcItems;
    uint32_t v[kTcItems];
    unsigned long long sum = 0;
    for (int j = 0; j < kTcItems; j++) { v[j] = i0 + j < n ? cnt[i0 + j] : 0u; sum += v[j]; }
    unsigned long long tot;
    unsigned long long at = part[blockIdx.x] + block_excl_scan<kTcNT>(sum, sm, tot);
    for (int j = 0; j < kTcItems; j++) {
        if (i0 + j < n) out[i0 + j] = (uint32_t)at;
        at += v[j];
    }
}

// ------------------------------------------------------------------------------------------ serializing
struct TcArgs {
    const unsigned long long *block_base;  // per block of the input: its first match (stream order)
    const uint32_t *base;                  // per input match: its first result match; base[n_match] = total
    const uint32_t *pd, *ps, *pl;          // result matches in destination order
    const uint8_t *x;                      // decoded bytes
    unsigned long long N, n_blocks;
    uint32_t block_log2, tile_log2, min_match;
    TcBlock *blk;
    const unsigned long long *boff;        // per block: offset of its header in the result
    uint8_t *out;
};

__device__ __forceinline__ void tc_block_range(const TcArgs &a, uint64_t b, uint32_t &P0, uint32_t &P1, uint32_t &b0,
                                               uint32_t &b1) {
    P0 = a.base[a.block_base[b]];
    P1 = a.base[a.block_base[b + 1]];
    b0 = (uint32_t)(b << a.block_log2);
    const uint64_t e = (uint64_t)b0 + (1ull << a.block_log2);
    b1 = (uint32_t)(e < a.N ? e : a.N);
}

// Layout of one block of the result (one CTA per block).
__global__ void __launch_bounds__(kTcNT) k_tc_block_sizes(TcArgs a) {
    __shared__ ScanSmem<kTcNT> sm;
    __shared__ uint32_t s_maxoff;
    for (uint64_t b = blockIdx.x; b < a.n_blocks; b += gridDim.x) {
        uint32_t P0, P1, b0, b1;
        tc_block_range(a, b, P0, P1, b0, b1);
        if (threadIdx.x == 0) s_maxoff = 0;
        __syncthreads();
        unsigned long long cmd = 0, len = 0, lit = 0;
        for (uint32_t j = P0 + threadIdx.x; j < P1; j += kTcNT) {
            const uint32_t d = a.pd[j], L = a.pl[j];
            const uint32_t prev = j > P0 ? a.pd[j - 1] + a.pl[j - 1] : b0;
            cmd += vlen(d - prev);
            len += vlen(L - a.min_match);
            lit += d - prev;
            atomicMax(&s_maxoff, a.ps[j]);
        }
        unsigned long long t_cmd, t_len, t_lit;
        block_excl_scan<kTcNT>(cmd, sm, t_cmd);
        block_excl_scan<kTcNT>(len, sm, t_len);
        block_excl_scan<kTcNT>(lit, sm, t_lit);
        if (threadIdx.x == 0) {
            const uint32_t last = P1 > P0 ? a.pd[P1 - 1] + a.pl[P1 - 1] : b0;
            const uint32_t trail = b1 - last, np = P1 - P0;
            if (trail) { t_cmd += vlen(trail); t_lit += trail; }
            const uint32_t mo = s_maxoff;  // offsets are 32-bit: at most 4 bytes wide
            uint32_t w = 1;
            while (w < 4 && (mo >> (8 * w))) w++;
            const uint32_t T = 1u << a.tile_log2;
            const uint32_t n_tiles = (b1 - b0 + T - 1) / T;
            unsigned long long sz = align16(kBlockHeader + (unsigned long long)kSyncEntry * n_tiles);
            sz = align16(sz + t_cmd);
            sz = align16(sz + t_len);
            sz = align16(sz + (unsigned long long)np * w);
            sz = align16(sz + t_lit);
            TcBlock &k = a.blk[b];
            k.n_seq = np + (trail ? 1u : 0u);
            k.n_match = np;
            k.n_lit = (uint32_t)t_lit;
            k.cmd_bytes = (uint32_t)t_cmd;
            k.len_bytes = (uint32_t)t_len;
            k.w = w;
            k.n_tiles = n_tiles;
            k.size = sz;
        }
        __syncthreads();
    }
}

// One block of the result (one CTA per block): header, sync table, sections.  The result buffer is zeroed
// first (padding), so only the fields and sections are written.  Sequences are taken kTcWNT at a time; their
// section offsets come from CTA scans; a thread copies its own literal run when it is short, a warp each
// medium one, the whole CTA each long one.
constexpr int kTcWNT = 1024;
constexpr uint32_t kTcShortRun = 32, kTcLongRun = 512;
__global__ void __launch_bounds__(kTcWNT) k_tc_write(TcArgs a) {
    __shared__ ScanSmem<kTcWNT> sm;
    __shared__ uint32_t s_src[kTcWNT], s_dst[kTcWNT], s_len[kTcWNT], s_med[kTcWNT], s_long[kTcWNT];
    __shared__ uint32_t s_nmed, s_nlong;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint8_t *__restrict__ x = a.x;
    for (uint64_t b = blockIdx.x; b < a.n_blocks; b += gridDim.x) {
        uint32_t P0, P1, b0, b1;
        tc_block_range(a, b, P0, P1, b0, b1);
        const TcBlock k = a.blk[b];
        uint8_t *__restrict__ h = a.out + a.boff[b];
        if (threadIdx.x == 0) {
            put32(h + 0, k.n_seq); put32(h + 4, k.n_match); put32(h + 8, k.n_lit); put32(h + 12, k.cmd_bytes);
            put32(h + 16, k.len_bytes); h[20] = (uint8_t)k.w; put32(h + 24, k.n_match ? 1u : 0u); put32(h + 28, k.n_tiles);
        }
        const uint64_t o_cmd = align16(kBlockHeader + (uint64_t)kSyncEntry * k.n_tiles);
        const uint64_t o_len = align16(o_cmd + k.cmd_bytes), o_off = align16(o_len + k.len_bytes);
        const uint64_t o_lit = align16(o_off + (uint64_t)k.n_match * k.w);
        const uint32_t np = P1 - P0, tl = a.tile_log2, T = 1u << tl;
        unsigned long long cp = 0, lp = 0, lt = 0;
        for (uint32_t i0 = 0; i0 < k.n_seq; i0 += kTcWNT) {
            if (threadIdx.x == 0) { s_nmed = 0; s_nlong = 0; }  // ordered by the scans' barriers below
            const uint32_t i = i0 + threadIdx.x;
            const bool valid = i < k.n_seq, has = i < np;
            uint32_t pos = 0, r = 0, L = 0, s = 0;
            if (valid) {
                const uint32_t j = P0 + i;
                pos = i == 0 ? b0 : a.pd[j - 1] + a.pl[j - 1];
                if (has) { r = a.pd[j] - pos; L = a.pl[j]; s = a.ps[j]; }
                else r = b1 - pos;
            }
            const uint32_t vr = valid ? vlen(r) : 0u, vl = has ? vlen(L - a.min_match) : 0u;
            unsigned long long tc, tlp, tlt;
            const unsigned long long ec = cp + block_excl_scan<kTcWNT>(vr, sm, tc);
            const unsigned long long el = lp + block_excl_scan<kTcWNT>(vl, sm, tlp);
            const unsigned long long et = lt + block_excl_scan<kTcWNT>(valid ? r : 0u, sm, tlt);
            if (valid) {
                put_varint(h + o_cmd + ec, r);
                if (has) {
                    put_varint(h + o_len + el, L - a.min_match);
                    put_le(h + o_off + (uint64_t)k.w * i, s, k.w);
                }
                // sync entries of the tiles whose first byte lies in this sequence
                const uint32_t rel = pos - b0, end = rel + r + L;
                for (uint32_t t = (rel + T - 1) >> tl; t < ((end + T - 1) >> tl); t++) {
                    uint8_t *e = h + kBlockHeader + (uint64_t)kSyncEntry * t;
                    put32(e, i); put32(e + 4, (uint32_t)ec); put32(e + 8, (uint32_t)el); put32(e + 12, (uint32_t)et);
                    put32(e + 16, rel);
                }
                if (r <= kTcShortRun) {
                    const uint8_t *src = x + pos;
                    uint8_t *dst = h + o_lit + et;
                    for (uint32_t q = 0; q < r; q++) dst[q] = __ldg(src + q);
                } else if (r < kTcLongRun) {
                    s_med[atomicAdd(&s_nmed, 1u)] = threadIdx.x;
                } else {
                    s_long[atomicAdd(&s_nlong, 1u)] = threadIdx.x;
                }
            }
            s_src[threadIdx.x] = pos;
            s_dst[threadIdx.x] = (uint32_t)et;
            s_len[threadIdx.x] = valid ? r : 0u;
            __syncthreads();
            const uint32_t nmed = s_nmed, nlong = s_nlong;
            for (uint32_t q = warp; q < nmed; q += kTcWNT / 32) {
                const uint32_t t = s_med[q], n = s_len[t];
                const uint8_t *src = x + s_src[t];
                uint8_t *dst = h + o_lit + s_dst[t];
                for (uint32_t j = lane; j < n; j += 32) dst[j] = __ldg(src + j);
            }
            for (uint32_t q = 0; q < nlong; q++) {
                const uint32_t t = s_long[q], n = s_len[t];
                const uint8_t *src = x + s_src[t];
                uint8_t *dst = h + o_lit + s_dst[t];
                uint32_t j = threadIdx.x;
                for (; j + 3 * kTcWNT < n; j += 4 * kTcWNT) {
                    const uint8_t v0 = __ldg(src + j), v1 = __ldg(src + j + kTcWNT), v2 = __ldg(src + j + 2 * kTcWNT),
                                  v3 = __ldg(src + j + 3 * kTcWNT);
                    dst[j] = v0; dst[j + kTcWNT] = v1; dst[j + 2 * kTcWNT] = v2; dst[j + 3 * kTcWNT] = v3;
                }
                for (; j < n; j += kTcWNT) dst[j] = __ldg(src + j);
            }
            __syncthreads();
            cp += tc; lp += tlp; lt += tlt;
        }
    }
}

}  // namespace aceapex

// ================================================================================================ host
struct aceapex_transcode {
    aceapex_info in{};
    uint8_t *x = nullptr;        // decoded bytes
    uint32_t *root = nullptr;
    uint8_t *ws = nullptr;       // wavefront workspace (records, level queues)
    WaveBufs wb{};
    uint32_t *cnt = nullptr, *base = nullptr;
    unsigned long long *part = nullptr;
    uint32_t *pd = nullptr, *ps = nullptr, *pl = nullptr;
    TcBlock *blk = nullptr;
    unsigned long long *boff = nullptr;
    unsigned long long *zero_bb = nullptr;  // block match ranges of a stream without matches (all [0, 0))
    int32_t *d_status = nullptr;
    std::vector<uint8_t> head;   // stream header + block index + padding of the result
    unsigned long long n_out_match = 0, n_out_seq = 0, out_len = 0;
    int num_sms = 0;
};

namespace {

int tc_fail(cudaError_t e) {
    if (e == cudaSuccess) return kOK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? kErrNomem : kErrCuda;
}

void tc_free(aceapex_transcode *t) {
    if (!t) return;
    cudaFree(t->x); cudaFree(t->root); cudaFree(t->ws); cudaFree(t->cnt); cudaFree(t->base);
    cudaFree(t->part); cudaFree(t->pd); cudaFree(t->ps); cudaFree(t->pl); cudaFree(t->blk); cudaFree(t->boff);
    cudaFree(t->zero_bb); cudaFree(t->d_status);
    delete t;
}

void wr_le(uint8_t *p, uint64_t v, int n) {
    for (int i = 0; i < n; i++) p[i] = (uint8_t)(v >> (8 * i));
}

template <typename T>
int tc_alloc(T **p, size_t n) {
    return tc_fail(cudaMalloc((void **)p, std::max<size_t>(n, 1) * sizeof(T)));
}

int tc_status(aceapex_transcode *t, cudaStream_t stream) {
    int32_t st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, t->d_status, 4, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return tc_fail(e);
    return st;
}

int tc_build(aceapex_transcode *t, const void *comp, cudaStream_t stream) {
    const aceapex_info &I = t->in;
    const uint64_t N = I.decoded_len, nm = I.n_match, nb = I.n_blocks;
    int rc;
    if ((rc = tc_alloc(&t->d_status, 1)) || (rc = tc_fail(cudaMemsetAsync(t->d_status, 0, 4, stream)))) return rc;
    if (N > 0) {
        // 1-2. roots start as root[y] = y; the decode by the warp dataflow copies every match byte's root with
        // the byte (a match is copied once the matches that wrote its source are done, so the roots it reads
        // are final) and leaves every match's record in stream order
        const uint64_t n4 = (N + 3) / 4;
        if ((rc = tc_alloc(&t->x, N)) || (rc = tc_alloc(&t->ws, aceapex_host::tc_workspace_size(I))) ||
            (rc = tc_alloc(&t->root, 4 * n4)))
            return rc;
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        k_tc_root_init<<<(unsigned)std::min<uint64_t>((n4 + kTcNT - 1) / kTcNT, (uint64_t)sms * 16), kTcNT, 0,
                         stream>>>(t->root, n4);
        if ((rc = tc_fail(cudaGetLastError()))) return rc;
        if ((rc = aceapex_host::tc_decode(comp, t->x, I, t->ws, &t->wb, t->root, t->d_status, &t->num_sms, stream)))
            return rc;
        if ((rc = tc_status(t, stream))) return rc;
    }
    if (nm > 0) {
        // 3. the matches each match becomes
        const uint64_t per = (uint64_t)kTcNT * kTcItems, nparts = (nm + per - 1) / per;
        if ((rc = tc_alloc(&t->cnt, nm)) || (rc = tc_alloc(&t->base, nm + 1)) || (rc = tc_alloc(&t->part, nparts)))
            return rc;
        const unsigned pgrid = (unsigned)std::min<uint64_t>((nm + kTcNT - 1) / kTcNT, (uint64_t)t->num_sms * 8);
        k_tc_pieces<false><<<pgrid, kTcNT, 0, stream>>>(t->wb, nm, t->root, I.min_match, t->cnt, nullptr, nullptr,
                                                         nullptr, nullptr);
        k_tc_scan_part<<<(unsigned)nparts, kTcNT, 0, stream>>>(t->cnt, nm, t->part);
        k_tc_scan_top<<<1, kTcNT, 0, stream>>>(t->part, nparts, t->base, nm);
        k_tc_scan_down<<<(unsigned)nparts, kTcNT, 0, stream>>>(t->cnt, nm, t->part, t->base);
        uint32_t total = 0;
        cudaError_t e = cudaMemcpyAsync(&total, t->base + nm, 4, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return tc_fail(e);
        t->n_out_match = total;
        if ((rc = tc_alloc(&t->pd, total)) || (rc = tc_alloc(&t->ps, total)) || (rc = tc_alloc(&t->pl, total))) return rc;
        k_tc_pieces<true><<<pgrid, kTcNT, 0, stream>>>(t->wb, nm, t->root, I.min_match, nullptr, t->base, t->pd, t->ps,
                                                        t->pl);
        if ((rc = tc_fail(cudaGetLastError()))) return rc;
    } else if (nb > 0) {
        // no match: every block is one literal run; the per-match arrays are empty
        if ((rc = tc_alloc(&t->base, 1)) || (rc = tc_fail(cudaMemsetAsync(t->base, 0, 4, stream)))) return rc;
    }
    // 4. block layout
    const uint64_t head_len = align16(kStreamHeader + 8 * nb);
    t->head.assign(head_len, 0);
    unsigned long long at = head_len, n_seq = 0;
    if (nb > 0) {
        if ((rc = tc_alloc(&t->blk, nb)) || (rc = tc_alloc(&t->boff, nb))) return rc;
        if (nm == 0 && ((rc = tc_alloc(&t->zero_bb, nb + 1)) ||
                        (rc = tc_fail(cudaMemsetAsync(t->zero_bb, 0, 8 * (nb + 1), stream)))))
            return rc;
        TcArgs a = {};
        a.block_base = nm > 0 ? t->wb.block_base : t->zero_bb;
        a.base = t->base; a.pd = t->pd; a.ps = t->ps; a.pl = t->pl; a.x = t->x;
        a.N = N; a.n_blocks = nb; a.block_log2 = I.block_log2; a.tile_log2 = I.tile_log2; a.min_match = I.min_match;
        a.blk = t->blk;
        const unsigned bgrid = (unsigned)std::min<uint64_t>(nb, 65535);
        k_tc_block_sizes<<<bgrid, kTcNT, 0, stream>>>(a);
        std::vector<TcBlock> hb(nb);
        cudaError_t e = cudaMemcpyAsync(hb.data(), t->blk, sizeof(TcBlock) * nb, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return tc_fail(e);
        std::vector<unsigned long long> off(nb);
        for (uint64_t b = 0; b < nb; b++) {
            off[b] = at;
            wr_le(t->head.data() + kStreamHeader + 8 * b, at, 8);
            at += hb[b].size;
            n_seq += hb[b].n_seq;
        }
        if ((rc = tc_fail(cudaMemcpyAsync(t->boff, off.data(), 8 * nb, cudaMemcpyHostToDevice, stream)))) return rc;
        if ((rc = tc_fail(cudaStreamSynchronize(stream)))) return rc;
    }
    t->out_len = at;
    t->n_out_seq = n_seq;
    uint8_t *o = t->head.data();
    wr_le(o + 0, kMagic, 4); wr_le(o + 4, kVersion, 2); wr_le(o + 6, 2, 2);
    o[8] = (uint8_t)I.block_log2; o[9] = (uint8_t)I.tile_log2; o[10] = (uint8_t)I.min_match;
    wr_le(o + 12, 0, 4); wr_le(o + 16, N, 8); wr_le(o + 24, nb, 8); wr_le(o + 32, at, 8);
    wr_le(o + 40, t->n_out_match, 8); wr_le(o + 48, t->n_out_match ? 1 : 0, 4); wr_le(o + 56, n_seq, 8);
    return kOK;
}

}  // namespace

extern "C" {

int aceapex_transcode_create(const void *comp, size_t comp_len, aceapex_transcode **plan, size_t *out_len, void *stream_) {
    if (!plan || !out_len || !comp || comp_len < kStreamHeader || ((uintptr_t)comp & 15)) return kErrArg;
    *plan = nullptr;
    cudaStream_t stream = (cudaStream_t)stream_;
    uint8_t h[kStreamHeader];
    cudaError_t e = cudaMemcpyAsync(h, comp, kStreamHeader, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return tc_fail(e);
    aceapex_transcode *t = new (std::nothrow) aceapex_transcode();
    if (!t) return kErrNomem;
    int rc = aceapex_host::tc_parse_header(h, kStreamHeader, &t->in);
    if (!rc && t->in.comp_len != comp_len) rc = kErrSize;
    if (!rc && t->in.decoded_len > 0xFFFFFFFFull) rc = kErrSize;  // 32-bit positions
    if (!rc) rc = tc_build(t, comp, stream);
    if (rc) {
        cudaStreamSynchronize(stream);
        tc_free(t);
        return rc;
    }
    *plan = t;
    *out_len = t->out_len;
    return kOK;
}

int aceapex_transcode_write(aceapex_transcode *t, void *out, size_t out_cap, void *stream_) {
    if (!t || !out || ((uintptr_t)out & 15)) return kErrArg;
    if (out_cap < t->out_len) return kErrSize;
    cudaStream_t stream = (cudaStream_t)stream_;
    const aceapex_info &I = t->in;
    cudaError_t e = cudaMemsetAsync(out, 0, t->out_len, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, t->head.data(), t->head.size(), cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return tc_fail(e);
    if (I.n_blocks > 0) {
        TcArgs a = {};
        a.block_base = I.n_match > 0 ? t->wb.block_base : t->zero_bb;
        a.base = t->base; a.pd = t->pd; a.ps = t->ps; a.pl = t->pl; a.x = t->x;
        a.N = I.decoded_len; a.n_blocks = I.n_blocks; a.block_log2 = I.block_log2; a.tile_log2 = I.tile_log2;
        a.min_match = I.min_match; a.blk = t->blk; a.boff = t->boff; a.out = (uint8_t *)out;
        k_tc_write<<<(unsigned)std::min<uint64_t>(I.n_blocks, 65535), kTcWNT, 0, stream>>>(a);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return tc_fail(e);
    } else if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) {
        return tc_fail(e);
    }
    return kOK;
}

int aceapex_transcode_info(const aceapex_transcode *t, uint64_t *n_match, uint64_t *n_seq) {
    if (!t) return kErrArg;
    if (n_match) *n_match = t->n_out_match;
    if (n_seq) *n_seq = t->n_out_seq;
    return kOK;
}

int aceapex_transcode_destroy(aceapex_transcode *t) {
    if (!t) return kErrArg;
    cudaDeviceSynchronize();
    tc_free(t);
    return kOK;
}

}  // extern "C"
