// Launch interface between the host API (api.cpp) and the decode kernels (decode.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "layout.h"

namespace aceapex {

// Kernel arguments: a single stream travels by value, a batch through a device descriptor array.
struct LaunchArgs {
    StreamDesc one;
    int n_streams;
    unsigned long long total_tiles;
    unsigned long long wait_ns;   // limit of every bounded device wait
    unsigned long long withhold;  // test hook: this tile never publishes its flag (~0 = none)
    unsigned int max_tile_log2;   // largest tile of the launch's streams (selects the image kernel)
    unsigned long long max_n;     // largest decoded length of the launch's streams (0 = unknown)
    unsigned long long *phase;    // when profiling: per-phase SM cycles of the one-pass kernel (kPhases)
    uint32_t *root;               // transcoding (warp dataflow only): per output byte, its root, copied with it
};
constexpr int kPhases = 8;  // open, parse, literals, store+publish, wait, matches, store, tiles

// Launch shape and schedulers.
struct LaunchCfg {
    int num_sms;
    int warps;        // one-pass kernel: warps per CTA (2, 4 or 8)
    int ctas_per_sm;  // one-pass kernel: CTAs per SM (0 = as many as fit)
    int wave_sched;   // deep streams: 0 per-match dataflow, 1 level queues, 2 warp dataflow (default)
};

// Device buffers of the wavefront path (carved from the workspace).
struct WaveBufs {
    unsigned long long *block_base;  // n_blocks + 1 prefix sums of per-block match counts
    uint32_t *bdepth;                // per block: its header's max_depth field
    unsigned long long *mdst, *msrc; // per match: absolute destination and source
    uint32_t *mlen, *depth, *queue;  // per match: length, depth, level-queue entry
    uint32_t *gidx;                  // per granule: first match ending after the granule start
    uint32_t *hist, *lvl, *cursor;   // per level (max_depth + 2 entries)
    unsigned long long *qd, *qs;     // level-ordered match records: destination, source
    uint32_t *ql;                    //   and length
};

// Kernel timing (opt-in): CUDA events recorded on the launch stream around each kernel.
enum KernelId { kKReset = 0, kKFlat, kKFinalize, kKMatchBase, kKParse, kKDepth, kKHist, kKLevels, kKScatter, kKWave,
                kKFlow, kKCount };
extern const char *const kKernelNames[kKCount];
void prof_enable(bool on);
bool prof_enabled();
void prof_mark(int id, bool start, cudaStream_t stream);
int prof_collect(double *ms, unsigned long long *launches);  // kKCount entries each; syncs on the events

cudaError_t launch_flat(const LaunchCfg &cfg, WsHead *head, StreamState *sst, uint32_t *flags, const StreamDesc *descs,
                        const LaunchArgs &a, int32_t *status_out, cudaStream_t stream);
// Batch plan statuses into device memory: out[i] = map (0, v): v; (1, k): flat[k]; (2, k): wave[k].
cudaError_t launch_gather_status(int n, const int32_t *map, const int32_t *flat, const int32_t *wave, int32_t *out,
                                 cudaStream_t stream);
cudaError_t launch_wave(const LaunchCfg &cfg, WsHead *head, StreamState *sst, const LaunchArgs &a, const WaveBufs &wb,
                        int32_t *status_out, cudaStream_t stream);

}  // namespace aceapex
