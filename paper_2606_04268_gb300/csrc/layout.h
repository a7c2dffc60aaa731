// Stream layout constants of the ACEAPEX stream format and the descriptor / workspace structures the
// host code hands to the decode kernels.  Included by host C++ and by CUDA code.
#pragma once
#include <stdint.h>

namespace aceapex {

constexpr uint32_t kMagic = 0x58454341u;  // "ACEX"
constexpr uint32_t kVersion = 1;
constexpr uint32_t kStreamHeader = 64;    // stream header bytes (stream format §1.1)
constexpr uint32_t kBlockHeader = 32;     // block header bytes (§2.1)
constexpr uint32_t kSyncEntry = 20;       // sync-table entry bytes (§2.3)
constexpr uint32_t kMinBlockLog2 = 2, kMaxBlockLog2 = 24;
constexpr uint32_t kGranuleLog2 = 6;      // writer-index granule: 64 output bytes (or the tile, if smaller)
constexpr uint32_t kOnePassMaxTileLog2 = 12;          // largest tile of the one-pass kernel (one warp per tile)
constexpr unsigned long long kOnePassMaxN = 0xFFF00000ull;  // its positions are 32-bit: ~4 GiB of output

// status codes (mirror aceapex_status)
enum : int { kOK = 0, kErrArg = -1, kErrFormat = -2, kErrSize = -3, kErrOffset = -4, kErrTimeout = -5,
             kErrCuda = -6, kErrNomem = -7, kErrDepth = -8 };

#ifdef __CUDACC__
#define ACEAPEX_HD __host__ __device__
#else
#define ACEAPEX_HD
#endif
ACEAPEX_HD inline uint64_t align16(uint64_t x) { return (x + 15) & ~uint64_t(15); }

// One stream of a launch (built on the host from the header it read back, copied to the device).
struct StreamDesc {
    const uint8_t *comp;
    uint8_t *out;
    uint64_t comp_len;
    uint64_t N;           // decoded bytes
    uint64_t n_blocks;
    uint64_t n_seq;       // header totals, checked against the blocks
    uint64_t n_match;
    uint64_t tile_base;   // global index of this launch's first tile of the stream in the launch's tile space
    uint64_t n_tiles;     // tiles of the stream decoded by this launch
    uint64_t tile_off;    // index (within the stream) of the first of them: earlier tiles are already decoded
    struct StreamState *state;  // persistent per-stream state (served requests), else the launch's own array
    uint32_t *litmap;     // one-pass path: bit x set once output byte x is known to be a literal byte
    uint32_t block_log2, tile_log2, min_match, max_depth;
    uint32_t flags;       // bit 0: this launch completes the stream: check the header totals at the end
    uint32_t pad;
};
constexpr uint32_t kDescLast = 1;

// Per-stream device state (zeroed by the reset kernel, or once per request by the server).
struct StreamState {
    unsigned long long front;      // tiles [tile_base, front) are known to have published their literals
    unsigned long long seq_sum;    // sum of the blocks' n_seq
    unsigned long long match_sum;  // sum of the blocks' n_match
    unsigned long long err_key;    // min over errors of (order << 4 | -code): the earliest error wins
    unsigned int depth_max;        // max of the blocks' max_depth fields
    int status;                    // nonzero once any error was seen (quick test); final code after k_finalize
};

// Order of an error not tied to a tile: after every tile error, as a sequential decoder would meet it.
constexpr unsigned long long kOrderTotals = (1ull << 58) - 3, kOrderDepth = (1ull << 58) - 2,
                             kOrderTimeout = (1ull << 58) - 1;

// Head of every workspace.
struct WsHead {
    unsigned long long ticket;     // tile (or match-chunk) tickets of the running persistent kernel
    unsigned long long ticket2;
    unsigned int epoch;            // launch counter: a tile flag equal to it means "published in this launch"
    unsigned int bar_count, bar_gen;
    unsigned int depth_seen;       // largest computed match depth (wavefront path)
    unsigned int n_levels;
    unsigned int pad[7];
    unsigned long long phase[8];   // per-phase SM cycles of the one-pass kernel (profiling only)
};

// 32-bit words of a stream's literal bitmap (one bit per output byte, one spare word).
inline uint64_t litmap_words(uint64_t N) { return (N + 31) / 32 + 1; }

// Tiles of a stream: every block but the last has 2^(block_log2 - tile_log2) tiles.
inline uint64_t stream_tiles(uint64_t N, uint32_t block_log2, uint32_t tile_log2) {
    if (N == 0) return 0;
    const uint64_t B = 1ull << block_log2, T = 1ull << tile_log2;
    const uint64_t nb = (N + B - 1) / B, last = N - (nb - 1) * B;
    return (nb - 1) * (B / T) + (last + T - 1) / T;
}

}  // namespace aceapex
