// Decoder of the entropy container (stream format §6; the entropy stage the paper leaves for later, §6):
// segments of at most 4096 bytes of the wrapped stream, each stored or coded with a canonical Huffman code
// (codes of at most 12 bits) in 32 interleaved lanes, decoded back into the wrapped stream in HBM, ahead of
// the decode kernels on the same CUDA stream.
//
// One warp per segment, warps taking consecutive segments (consecutive segments usually share a code): lane
// l decodes the bytes l, l + 32, ... of the segment from its own bitstream, one code per step, with a
// 4096-entry lookup table (12-bit prefix -> symbol, length) that the warp builds in shared memory whenever
// the code changes.  Stored segments are copied.  Every field, bound, Kraft sum and code is checked; a
// malformed container sets ACEAPEX_ERR_FORMAT and no access leaves the container or the output.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>

#include "../../include/aceapex.h"
#include "layout.h"

namespace aceapex {

constexpr uint32_t kEMagic = 0x45454341u;
constexpr uint32_t kESeg = 4096;      // bytes of the wrapped stream per segment, at most
constexpr uint32_t kEMaxLen = 12;     // longest code
constexpr int kEWarps = 4;            // warps per CTA

constexpr uint32_t kEStage = 8 + 128 + 64 + kESeg;  // payloads up to this size are staged in shared memory

struct alignas(16) EWarp {
    uint16_t tbl[1u << kEMaxLen];     // 12-bit prefix -> symbol | length << 8 (0: no code)
    uint16_t code[256];
    uint8_t len[256];
    uint32_t running[kEMaxLen + 1];
    alignas(16) uint8_t pay[kEStage + 16];  // the segment's payload (16-byte copies), when it fits; the
                                            // 16 spare bytes keep a two-word read at the end inside
};

__device__ __forceinline__ uint64_t e_ld64(const uint8_t *p) {  // 8-aligned
    return __ldg(reinterpret_cast<const unsigned long long *>(p));
}
__device__ __forceinline__ uint32_t e_ld32(const uint8_t *p) {  // 4-aligned
    return __ldg(reinterpret_cast<const uint32_t *>(p));
}

__device__ __forceinline__ void e_fail(int32_t *status) { atomicCAS(status, 0, kErrFormat); }

// The code of segment t (its inline code lengths), checked, into the warp's table.  Returns false when the
// table segment or its lengths are malformed.
__device__ bool e_load_code(EWarp &W, const uint8_t *e, uint64_t e_len, uint64_t n_seg, uint64_t t) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t eo = e_ld64(e + 72 + 16 * t);
    const uint64_t ee = t + 1 < n_seg ? e_ld64(e + 72 + 16 * (t + 1)) : e_len;
    // payload bounds: 16-aligned, inside the container, room for the header and the 128 bytes of lengths
    bool ok = !(eo & 15) && ee <= e_len && eo < ee && ee - eo >= 8 + 128;
    if (!__all_sync(0xffffffffu, ok)) return false;
    ok = e[eo] == 1 && e_ld32(e + eo + 4) == (uint32_t)t;
    // lane l: bytes 4l .. 4l+3 of the lengths, symbols 8l .. 8l+7
    const uint32_t w = e_ld32(e + eo + 8 + 4 * lane);
    uint32_t kraft = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const uint32_t L = (w >> (4 * j)) & 15u;
        if (L > kEMaxLen) ok = false;
        else if (L) kraft += 1u << (kEMaxLen - L);
        W.len[8 * lane + j] = (uint8_t)L;
    }
    kraft = __reduce_add_sync(0xffffffffu, kraft);
    if (!__all_sync(0xffffffffu, ok) || kraft == 0 || kraft > (1u << kEMaxLen)) return false;
    __syncwarp();
    // canonical codes: first code of each length, then symbols in value order, 32 per round
    if (lane <= kEMaxLen) W.running[lane] = 0;
    __syncwarp();
    uint32_t cnt_l = 0;  // lane L (1..12): number of symbols of length L
    for (int s0 = 0; s0 < 256; s0 += 32) {
        const uint32_t L = W.len[s0 + lane];
        const unsigned peers = __match_any_sync(0xffffffffu, L);
        if (lane == (uint32_t)(__ffs(peers) - 1) && L) atomicAdd(&W.running[L], (uint32_t)__popc(peers));
    }
    __syncwarp();
    if (lane <= kEMaxLen) cnt_l = W.running[lane];
    // first[L] = (first[L-1] + cnt[L-1]) << 1, first[1] = 0: a running sum over lanes 1..12
    uint32_t first = 0;
    for (uint32_t L = 1; L <= kEMaxLen; L++) {
        const uint32_t prev_first = __shfl_sync(0xffffffffu, first, L - 1), prev_cnt = __shfl_sync(0xffffffffu, cnt_l, L - 1);
        if (lane == L) first = L == 1 ? 0u : (prev_first + prev_cnt) << 1;
    }
    __syncwarp();
    if (lane <= kEMaxLen) W.running[lane] = first;  // next code of each length
    __syncwarp();
    for (int s0 = 0; s0 < 256; s0 += 32) {
        const uint32_t s = s0 + lane, L = W.len[s];
        const unsigned peers = __match_any_sync(0xffffffffu, L);
        const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        const uint32_t base = L ? W.running[L] : 0u;
        W.code[s] = (uint16_t)(base + rank);
        __syncwarp();
        if (lane == (uint32_t)(__ffs(peers) - 1) && L) W.running[L] = base + __popc(peers);
        __syncwarp();
    }
    // lookup table: every 12-bit prefix that starts with a symbol's code
    for (uint32_t i = lane; i < (1u << kEMaxLen); i += 32) W.tbl[i] = 0;
    __syncwarp();
    for (int s = 0; s < 256; s++) {
        const uint32_t L = W.len[s];
        if (!L) continue;
        const uint32_t b = (uint32_t)W.code[s] << (kEMaxLen - L), n = 1u << (kEMaxLen - L);
        for (uint32_t j = lane; j < n; j += 32) W.tbl[b + j] = (uint16_t)(s | (L << 8));
    }
    __syncwarp();
    return true;
}

__global__ void __launch_bounds__(32 * kEWarps) k_entropy(const uint8_t *e, uint64_t e_len, uint64_t n_seg,
                                                          uint64_t raw_len, uint8_t *raw, int32_t *status) {
    extern __shared__ uint4 e_smem[];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    EWarp &W = reinterpret_cast<EWarp *>(e_smem)[warp];
    const uint64_t nw = (uint64_t)gridDim.x * kEWarps, gw = (uint64_t)blockIdx.x * kEWarps + warp;
    const uint64_t k0 = gw * n_seg / nw, k1 = (gw + 1) * n_seg / nw;
    uint64_t cur = ~0ull;  // segment whose code is in the table
    for (uint64_t k = k0; k < k1; k++) {
        const uint64_t ro = e_ld64(e + 64 + 16 * k), eo = e_ld64(e + 72 + 16 * k);
        const uint64_t re = k + 1 < n_seg ? e_ld64(e + 64 + 16 * (k + 1)) : raw_len;
        const uint64_t ee = k + 1 < n_seg ? e_ld64(e + 72 + 16 * (k + 1)) : e_len;
        if ((k == 0 && (ro != 0 || eo != align16(64 + 16 * n_seg))) || re <= ro || re - ro > kESeg || re > raw_len ||
            (eo & 15) || ee <= eo || ee > e_len || ee - eo < 8) {
            if (lane == 0) e_fail(status);
            return;
        }
        const uint32_t n = (uint32_t)(re - ro);
        const uint64_t P = ee - eo;
        const uint8_t *q = e + eo;
        const uint32_t h = e_ld32(q), table = e_ld32(q + 4), mode = h & 0xFFu;
        if ((h >> 8) || mode > 1) { if (lane == 0) e_fail(status); return; }
        if (mode == 0) {
            if (table != 0 || P < 8 + (uint64_t)n) { if (lane == 0) e_fail(status); return; }
            if ((ro & 7) == 0) {  // 8-byte words (the payload's bytes start 8-aligned), then the tail
                const unsigned long long *src = reinterpret_cast<const unsigned long long *>(q + 8);
                unsigned long long *dst = reinterpret_cast<unsigned long long *>(raw + ro);
                for (uint32_t i = lane; i < n / 8; i += 32) dst[i] = __ldg(src + i);
                for (uint32_t j = (n & ~7u) + lane; j < n; j += 32) raw[ro + j] = __ldg(q + 8 + j);
            } else {
                for (uint32_t j = lane; j < n; j += 32) raw[ro + j] = __ldg(q + 8 + j);
            }
            continue;
        }
        if (table > k) { if (lane == 0) e_fail(status); return; }
        if (table != cur) {
            if (!e_load_code(W, e, e_len, n_seg, table)) { if (lane == 0) e_fail(status); return; }
            cur = table;
        }
        const uint64_t lb_at = 8 + (table == k ? 128 : 0);
        if (P < lb_at + 64) { if (lane == 0) e_fail(status); return; }
        // lane l's bitstream: its byte length, and where it starts (exclusive scan over the lanes)
        const uint32_t nbytes = (uint32_t)__ldg(q + lb_at + 2 * lane) | ((uint32_t)__ldg(q + lb_at + 2 * lane + 1) << 8);
        uint32_t start = nbytes;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, start, o);
            if (lane >= (uint32_t)o) start += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, start, 31);
        start -= nbytes;
        if (P < lb_at + 64 + total) { if (lane == 0) e_fail(status); return; }
        bool bad = false;
        if (P <= kEStage) {
            // the payload in shared memory (one 16-byte copy per lane per step); the next 12 bits of a lane are
            // read from the two big-endian words around its bit position
            const uint4 *src = reinterpret_cast<const uint4 *>(q);
            uint4 *dst = reinterpret_cast<uint4 *>(W.pay);
            for (uint32_t i = lane; i < (uint32_t)(P >> 4); i += 32) dst[i] = __ldg(src + i);
            __syncwarp();
            const uint32_t *wd = reinterpret_cast<const uint32_t *>(W.pay);
            uint32_t bit = 8 * (uint32_t)(lb_at + 64 + start);
            const uint32_t bit_end = bit + 8 * nbytes;
            // words idx and idx + 1 of the payload (big-endian) hold the next bits; a code is at most 12 bits,
            // so the window moves by at most one word per code
            uint32_t idx = bit >> 5;
            uint32_t w0 = __byte_perm(wd[idx], 0, 0x0123), w1 = __byte_perm(wd[idx + 1], 0, 0x0123);
            uint8_t *dst_b = raw + ro + lane;
            for (uint32_t j = lane; j < n; j += 32, dst_b += 32) {
                const uint32_t peek = __funnelshift_l(w1, w0, bit & 31u);
                const uint32_t ent = W.tbl[peek >> (32 - kEMaxLen)], L = ent >> 8;
                if (L == 0 || bit + L > bit_end) { bad = true; break; }
                *dst_b = (uint8_t)ent;
                bit += L;
                if ((bit >> 5) != idx) {
                    idx++;
                    w0 = w1;
                    w1 = __byte_perm(wd[idx + 1], 0, 0x0123);
                }
            }
        } else {
            // straight from the container, a byte at a time
            const uint8_t *p = q + lb_at + 64 + start, *pe = p + nbytes;
            uint64_t buf = 0;
            uint32_t nb = 0;
            for (uint32_t j = lane; j < n; j += 32) {
                while (nb <= 56 && p < pe) { buf |= (uint64_t)__ldg(p++) << (56 - nb); nb += 8; }
                const uint32_t ent = W.tbl[buf >> (64 - kEMaxLen)], L = ent >> 8;
                if (L == 0 || L > nb) { bad = true; break; }
                raw[ro + j] = (uint8_t)ent;
                buf <<= L;
                nb -= L;
            }
        }
        if (__any_sync(0xffffffffu, bad)) { if (lane == 0) e_fail(status); return; }
        __syncwarp();  // the staged payload is read by every lane before the next segment overwrites it
    }
}

}  // namespace aceapex

using namespace aceapex;

extern "C" {

int aceapex_entropy_peek(const void *host_prefix, size_t len, aceapex_entropy_info *info) {
    const uint8_t *h = (const uint8_t *)host_prefix;
    if (!h || !info) return kErrArg;
    if (len < 64) return kErrSize;
    auto rd = [&](int off, int n) {
        uint64_t v = 0;
        for (int i = n - 1; i >= 0; i--) v = (v << 8) | h[off + i];
        return v;
    };
    if (rd(0, 4) != kEMagic || rd(4, 2) != 1 || rd(6, 2) != 0 || rd(8, 4) != 0 || rd(12, 4) != kEMaxLen)
        return kErrFormat;
    for (int i = 40; i < 64; i++) if (h[i]) return kErrFormat;
    info->raw_len = rd(16, 8);
    info->n_seg = rd(24, 8);
    info->e_len = rd(32, 8);
    if (info->e_len < 64 || (info->e_len & 15)) return kErrSize;
    if ((info->raw_len == 0) != (info->n_seg == 0) || info->n_seg > info->raw_len || info->n_seg > (info->e_len - 64) / 16)
        return kErrFormat;
    return kOK;
}

int aceapex_entropy_decode(const void *e, size_t e_len, const aceapex_entropy_info *info, void *raw, size_t raw_len,
                           int32_t *d_status, void *stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    if (!e || !info || !d_status || ((uintptr_t)e & 15) || (!raw && raw_len)) return kErrArg;
    if (info->e_len != e_len || info->raw_len != raw_len) return kErrSize;
    if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), stream) != cudaSuccess) { cudaGetLastError(); return kErrCuda; }
    if (info->n_seg == 0) return kOK;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t dyn = sizeof(EWarp) * kEWarps;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_entropy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess) {
            cudaGetLastError();
            return kErrCuda;
        }
        attr = true;
    }
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_entropy, 32 * kEWarps, dyn);
    const uint64_t want = (info->n_seg + kEWarps - 1) / kEWarps;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)std::max(occ, 1) * sms));
    k_entropy<<<grid, 32 * kEWarps, dyn, stream>>>((const uint8_t *)e, info->e_len, info->n_seg, info->raw_len,
                                                  (uint8_t *)raw, d_status);
    if (cudaGetLastError() != cudaSuccess) return kErrCuda;
    return kOK;
}

}  // extern "C"
