// Device-side building blocks shared by the decode kernels: little-endian reads of the stream layout,
// acquire/release flags, bounded waits, block-wide scans and the block-wide LEB128 decoder.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "layout.h"

namespace aceapex {

// ------------------------------------------------------------------------------------------ errors
// Record an error of a stream.  `order` places it in stream order (tile index, or one of the kOrder*
// constants); the final status is the error a sequential decoder would meet first.
__device__ __forceinline__ void report(StreamState *st, int code, unsigned long long order) {
    atomicMin(&st->err_key, (order << 4) | (unsigned long long)(-code));
    atomicCAS(&st->status, 0, code);
}
// A match deeper than its block's max_depth field: recorded after every tile error and the header totals,
// as the last check of a stream, without stopping the other tiles (their errors still come first).
__device__ __forceinline__ void report_depth(StreamState *st) {
    atomicMin(&st->err_key, (kOrderDepth << 4) | (unsigned long long)(-kErrDepth));
}

// ------------------------------------------------------------------------------------------ memory
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Loads of decoded output written during the same launch go through L2 (never a stale L1 line).
__device__ __forceinline__ uint8_t ld_out(const uint8_t *p) { return __ldcg(p); }

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Little-endian field reads from the (read-only) compressed stream.  Header fields sit at 4- or 8-byte
// aligned offsets of a 16-byte aligned stream; variable-width offsets use byte loads.
__device__ __forceinline__ uint32_t ld32(const uint8_t *p) { return __ldg(reinterpret_cast<const uint32_t *>(p)); }
__device__ __forceinline__ uint64_t ld64(const uint8_t *p) {
    return __ldg(reinterpret_cast<const unsigned long long *>(p));
}
__device__ __forceinline__ uint64_t ld_le(const uint8_t *p, uint32_t w) {
    uint64_t v = 0;
    for (uint32_t i = 0; i < w; i++) v |= (uint64_t)__ldg(p + i) << (8 * i);
    return v;
}

// ------------------------------------------------------------------------------------------ scans
template <int NT>
struct ScanSmem {
    unsigned long long w[NT / 32];
};

// Exclusive block-wide prefix sum of 64-bit values; every thread receives the block total.
template <int NT>
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v, ScanSmem<NT> &sm,
                                                              unsigned long long &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm.w[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long s = lane < NT / 32 ? sm.w[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < NT / 32) sm.w[lane] = s;
    }
    __syncthreads();
    unsigned long long base = wid ? sm.w[wid - 1] : 0ull;
    total = sm.w[NT / 32 - 1];
    __syncthreads();
    return base + x - v;
}

// ------------------------------------------------------------------------------------------ LEB128
// Block-wide decode of `count` LEB128 varints that start at sec[pos]; sec has sec_len bytes.  Values go to
// vals[0..count); ends[] is scratch of at least `count` entries.  If want <= count, *want_pos receives the
// byte offset where varint `want` begins (== the returned offset when want == count), used to check sync
// points.  Returns the offset after the last varint, or -1 on a malformed varint or a short section.
// All threads of the block must call it with the same arguments.
template <int NT>
__device__ int64_t block_varints(const uint8_t *sec, uint32_t sec_len, uint32_t pos, uint32_t count, uint32_t *vals,
                                 uint32_t *ends, ScanSmem<NT> &sm, int *s_err, uint32_t want, uint32_t *want_pos) {
    if (count == 0) {
        if (want == 0 && threadIdx.x == 0) *want_pos = pos;
        __syncthreads();
        return pos;
    }
    uint32_t found = 0, base = pos;
    // pass 1: locate the first `count` terminating bytes (high bit clear); their rank comes from a scan
    while (found < count) {
        if (base >= sec_len) return -1;
        const uint32_t b0 = base + threadIdx.x * 4u;
        uint32_t mask = 0;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint32_t q = b0 + j;
            if (q < sec_len && !(__ldg(sec + q) & 0x80)) mask |= 1u << j;
        }
        unsigned long long total;
        unsigned long long ex = block_excl_scan<NT>((unsigned long long)__popc(mask), sm, total);
        uint32_t idx = found + (uint32_t)ex;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if ((mask >> j) & 1u) {
                if (idx < count) ends[idx] = b0 + j;
                idx++;
            }
        }
        found += (uint32_t)total;
        base += NT * 4u;
        __syncthreads();
    }
    const uint32_t after = ends[count - 1] + 1;
    if (threadIdx.x == 0 && want <= count) *want_pos = want == 0 ? pos : ends[want - 1] + 1;
    // pass 2: value i spans (end of varint i-1, end of varint i]
    for (uint32_t i = threadIdx.x; i < count; i += NT) {
        const uint32_t en = ends[i];
        const uint32_t st = i ? ends[i - 1] + 1 : pos;
        uint64_t v = 0;
        if (en - st >= 5) {
            *s_err = 1;
        } else {
            for (uint32_t q = st; q <= en; q++) v |= (uint64_t)(__ldg(sec + q) & 0x7F) << (7 * (q - st));
            if (v > 0xFFFFFFFFull) *s_err = 1;
        }
        vals[i] = (uint32_t)v;
    }
    __syncthreads();
    return *s_err ? -1 : (int64_t)after;
}

// Bounded grid barrier of a cooperative launch.  Returns false when the wait timed out.
__device__ __forceinline__ bool grid_barrier(WsHead *head, StreamState *st, uint64_t t0, uint64_t wait_ns) {
    __shared__ int s_ok;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        s_ok = 1;
        const unsigned gen = ld_acquire_u32(&head->bar_gen);
        const unsigned arrived = atomicAdd(&head->bar_count, 1u) + 1;
        if (arrived == gridDim.x) {
            atomicExch(&head->bar_count, 0u);
            __threadfence();
            st_release_u32(&head->bar_gen, gen + 1);
        } else {
            while (ld_acquire_u32(&head->bar_gen) == gen) {
                if (global_ns() - t0 > wait_ns) { report(st, kErrTimeout, kOrderTimeout); s_ok = 0; break; }
                __nanosleep(32);
            }
        }
    }
    __syncthreads();
    return s_ok;
}

}  // namespace aceapex
