// Host side of the C ABI (include/aceapex.h): header checks, workspace layout and pool, path selection,
// the batch plan with CUDA-graph replay, statistics.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/aceapex.h"
#include "decode.h"

using namespace aceapex;

namespace {

// ------------------------------------------------------------------------------------------ header
uint64_t rd(const uint8_t *p, int n) {
    uint64_t v = 0;
    for (int i = n - 1; i >= 0; i--) v = (v << 8) | p[i];
    return v;
}

int parse_header(const uint8_t *h, size_t len, aceapex_info *info) {
    if (!h || !info) return kErrArg;
    if (len < kStreamHeader) return kErrSize;
    if (rd(h, 4) != kMagic || rd(h + 4, 2) != kVersion) return kErrFormat;
    const uint32_t flags = (uint32_t)rd(h + 6, 2);
    if (flags > 2) return kErrFormat;
    memset(info, 0, sizeof(*info));
    info->flatten = flags;
    info->block_log2 = h[8];
    info->tile_log2 = h[9];
    info->min_match = h[10];
    if (info->block_log2 < kMinBlockLog2 || info->block_log2 > kMaxBlockLog2 || info->tile_log2 < 2 ||
        info->tile_log2 > info->block_log2 || info->min_match < 1 || h[11] != 0)
        return kErrFormat;
    info->depth_cap = (uint32_t)rd(h + 12, 4);
    info->decoded_len = rd(h + 16, 8);
    info->n_blocks = rd(h + 24, 8);
    info->comp_len = rd(h + 32, 8);
    info->n_match = rd(h + 40, 8);
    info->max_depth = (uint32_t)rd(h + 48, 4);
    info->n_seq = rd(h + 56, 8);
    const uint64_t B = 1ull << info->block_log2;
    if (info->n_blocks != (info->decoded_len + B - 1) / B) return kErrFormat;
    if (info->comp_len & 15) return kErrSize;
    if (info->comp_len < kStreamHeader || info->n_blocks > (info->comp_len - kStreamHeader) / 8) return kErrFormat;
    if (info->n_match > info->decoded_len || info->n_seq > info->decoded_len) return kErrFormat;
    info->n_tiles = stream_tiles(info->decoded_len, info->block_log2, info->tile_log2);
    return kOK;
}

// ------------------------------------------------------------------------------------------ workspace
constexpr size_t kAlign = 256;
size_t up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct WsLayout {
    size_t head, sst, flags, litmap, descs, status, block_base, bdepth, mdst, msrc, mlen, depth, queue, gidx, qd, qs, ql,
        hist, lvl, cursor, total;
};

// Regions of a workspace.  One-pass: flags per tile and the literal bitmaps of the streams (lm_words 32-bit
// words in all).  Wavefront: per-match records, granule index, per-block depth fields, per-level arrays.
WsLayout layout(int n_streams, uint64_t total_tiles, bool wave, const aceapex_info *wi, uint64_t lm_words) {
    WsLayout L{};
    size_t at = 0;
    L.head = at; at = up(at + sizeof(WsHead));
    L.sst = at; at = up(at + sizeof(StreamState) * (size_t)std::max(n_streams, 1));
    L.status = at; at = up(at + sizeof(int32_t) * (size_t)std::max(n_streams, 1));
    L.descs = at; at = up(at + (n_streams > 1 ? sizeof(StreamDesc) * (size_t)n_streams : 0));
    L.flags = at; at = up(at + sizeof(uint32_t) * (size_t)(wave ? 0 : total_tiles));
    L.litmap = at; at = up(at + sizeof(uint32_t) * (size_t)(wave ? 0 : lm_words));
    if (wave && wi) {
        const uint64_t nm = wi->n_match, nb = wi->n_blocks;
        const uint32_t gl = std::min<uint32_t>(wi->tile_log2, kGranuleLog2);
        const uint64_t ng = (wi->decoded_len + (1ull << gl) - 1) >> gl;
        const uint64_t nl = (uint64_t)wi->max_depth + 2;
        L.block_base = at; at = up(at + 8 * (nb + 1));
        L.bdepth = at; at = up(at + 4 * (nb + 1));
        L.mdst = at; at = up(at + 8 * nm);
        L.msrc = at; at = up(at + 8 * nm);
        L.mlen = at; at = up(at + 4 * nm);
        L.depth = at; at = up(at + 4 * nm);
        L.queue = at; at = up(at + 4 * nm);
        L.gidx = at; at = up(at + 4 * ng);
        L.qd = at; at = up(at + 8 * nm);
        L.qs = at; at = up(at + 8 * nm);
        L.ql = at; at = up(at + 4 * nm);
        L.hist = at; at = up(at + 4 * nl);
        L.lvl = at; at = up(at + 4 * (nl + 1));
        L.cursor = at; at = up(at + 4 * nl);
    }
    L.total = at;
    return L;
}

WaveBufs wave_bufs(uint8_t *ws, const WsLayout &L) {
    WaveBufs w;
    w.block_base = (unsigned long long *)(ws + L.block_base);
    w.bdepth = (uint32_t *)(ws + L.bdepth);
    w.mdst = (unsigned long long *)(ws + L.mdst);
    w.msrc = (unsigned long long *)(ws + L.msrc);
    w.mlen = (uint32_t *)(ws + L.mlen);
    w.depth = (uint32_t *)(ws + L.depth);
    w.queue = (uint32_t *)(ws + L.queue);
    w.gidx = (uint32_t *)(ws + L.gidx);
    w.hist = (uint32_t *)(ws + L.hist);
    w.lvl = (uint32_t *)(ws + L.lvl);
    w.cursor = (uint32_t *)(ws + L.cursor);
    w.qd = (unsigned long long *)(ws + L.qd);
    w.qs = (unsigned long long *)(ws + L.qs);
    w.ql = (uint32_t *)(ws + L.ql);
    return w;
}

// Workspace of one stream decoded alone.
WsLayout layout_one(const aceapex_info &I, bool wave) {
    return layout(1, I.n_tiles, wave, &I, wave ? 0 : litmap_words(I.decoded_len));
}

StreamDesc make_desc(const void *comp, void *out, const aceapex_info &I, uint64_t tile_base) {
    StreamDesc d{};
    d.comp = (const uint8_t *)comp;
    d.out = (uint8_t *)out;
    d.comp_len = I.comp_len;
    d.N = I.decoded_len;
    d.n_blocks = I.n_blocks;
    d.n_seq = I.n_seq;
    d.n_match = I.n_match;
    d.tile_base = tile_base;
    d.n_tiles = I.n_tiles;
    d.tile_off = 0;
    d.state = nullptr;
    d.litmap = nullptr;
    d.flags = kDescLast;
    d.block_log2 = I.block_log2;
    d.tile_log2 = I.tile_log2;
    d.min_match = I.min_match;
    d.max_depth = I.max_depth;
    return d;
}

// ------------------------------------------------------------------------------------------ context
constexpr int kHostSlices = 16;  // most slices of one overlapped host-buffer decode

struct DevPool {
    uint8_t *ws = nullptr;
    size_t cap = 0;
    uint8_t *host = nullptr;  // pinned: header read-back, status, level histogram
    size_t host_cap = 0;
    int num_sms = 0;
    // host-buffer decodes: device copies of the stream and the output, one persistent stream state, and the
    // copy-in / copy-out streams and events of the overlap
    uint8_t *hd_comp = nullptr, *hd_out = nullptr;
    size_t hd_comp_cap = 0, hd_out_cap = 0;
    StreamState *hd_state = nullptr;
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev_in[kHostSlices]{}, ev_dec[kHostSlices]{};
    // host-buffer batch decodes: device copies of the streams and outputs, the groups' workspaces, and pinned
    // staging of the descriptors and statuses
    uint8_t *hb_comp = nullptr, *hb_out = nullptr, *hb_ws = nullptr, *hb_pin = nullptr;
    size_t hb_comp_cap = 0, hb_out_cap = 0, hb_ws_cap = 0, hb_pin_cap = 0;
};

struct Context {
    std::mutex mu;
    std::map<int, DevPool> pools;
    LaunchCfg cfg{0, 4, 0, 2};
    bool force_wave = false;
    unsigned long long wait_ns = 4000000000ull;  // bounded device waits give up after 4 s
    unsigned long long withhold = ~0ull;
    aceapex_stats stats{};
};
Context &ctx() {
    static Context *c = new Context();  // never destroyed: safe against exit-time ordering
    return *c;
}

int cuda_fail(cudaError_t e) {
    if (e == cudaSuccess) return kOK;
    cudaGetLastError();
    return kErrCuda;
}

int pool_for_device(DevPool **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cuda_fail(cudaErrorInvalidDevice);
    DevPool &p = ctx().pools[dev];
    if (!p.num_sms) {
        if (cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return kErrCuda;
        p.host_cap = 64 * 1024;
        if (cudaMallocHost((void **)&p.host, p.host_cap) != cudaSuccess) { p.host = nullptr; return kErrCuda; }
    }
    *out = &p;
    return kOK;
}

int pool_reserve(DevPool &p, size_t bytes, cudaStream_t stream) {
    if (bytes <= p.cap) return kOK;
    if (p.ws) {
        cudaStreamSynchronize(stream);
        cudaFree(p.ws);
        p.ws = nullptr;
        p.cap = 0;
    }
    size_t want = std::max(bytes, (size_t)1 << 20);
    if (cudaMalloc((void **)&p.ws, want) != cudaSuccess) { cudaGetLastError(); p.ws = nullptr; return kErrNomem; }
    // a fresh workspace is zero-filled once: tile flags hold launch epochs and must start below epoch 1
    if (cudaMemsetAsync(p.ws, 0, want, stream) != cudaSuccess) return kErrCuda;
    p.cap = want;
    return kOK;
}

// The one-pass kernel takes streams whose matches all have depth <= 1, with tiles of at most 4 KiB and at
// most ~4 GiB of output (its positions are 32-bit); every other stream takes the wavefront path.
bool one_pass_fits(const aceapex_info &I) {
    return I.max_depth <= 1 && I.tile_log2 <= (uint32_t)kOnePassMaxTileLog2 && I.decoded_len <= kOnePassMaxN;
}
bool use_wave(const aceapex_info &I) { return !one_pass_fits(I) || ctx().force_wave; }

// Enqueue the decode of one stream into workspace ws (layout L); the status goes to status_out.
// wave_sched >= 0 overrides the scheduler of the wavefront path.
int enqueue_one(const void *comp, void *out, const aceapex_info &I, uint8_t *ws, const WsLayout &L,
                int32_t *status_out, int num_sms, cudaStream_t stream, int wave_sched = -1,
                uint32_t *root = nullptr) {
    LaunchCfg cfg = ctx().cfg;
    cfg.num_sms = num_sms;
    if (wave_sched >= 0) cfg.wave_sched = wave_sched;
    LaunchArgs a{};
    a.one = make_desc(comp, out, I, 0);
    a.one.litmap = (uint32_t *)(ws + L.litmap);
    a.n_streams = 1;
    a.total_tiles = I.n_tiles;
    a.wait_ns = ctx().wait_ns;
    a.withhold = ctx().withhold;
    a.max_tile_log2 = I.tile_log2;
    a.max_n = I.decoded_len;
    WsHead *head = (WsHead *)(ws + L.head);
    a.phase = prof_enabled() ? head->phase : nullptr;
    a.root = root;
    StreamState *sst = (StreamState *)(ws + L.sst);
    cudaError_t e;
    if (use_wave(I) || wave_sched >= 0) e = launch_wave(cfg, head, sst, a, wave_bufs(ws, L), status_out, stream);
    else e = launch_flat(cfg, head, sst, (uint32_t *)(ws + L.flags), nullptr, a, status_out, stream);
    return cuda_fail(e);
}

bool check_ptrs(const void *comp, size_t comp_len, const void *out, size_t out_len) {
    if (!comp || comp_len < kStreamHeader || ((uintptr_t)comp & 15)) return false;
    if (!out && out_len) return false;
    return true;
}

}  // namespace

// Host helpers of the serving engine (serve.cpp); init_state is defined with the kernels (decode.cu).
namespace aceapex_host {
int init_state(aceapex::StreamState *st, cudaStream_t stream);
bool one_pass_stream(const aceapex_info &I) {
    std::lock_guard<std::mutex> g(ctx().mu);
    return !use_wave(I);
}
LaunchCfg launch_cfg() {
    std::lock_guard<std::mutex> g(ctx().mu);
    return ctx().cfg;
}
int num_sms() {
    std::lock_guard<std::mutex> g(ctx().mu);
    DevPool *p = nullptr;
    return pool_for_device(&p) ? 1 : p->num_sms;
}
// Decode one stream whole into a workspace that the caller keeps (grown on demand).
int server_enqueue_whole(const void *comp, void *out, const aceapex_info &I, uint8_t **ws, size_t *ws_cap,
                         int32_t *status_out, cudaStream_t stream) {
    std::lock_guard<std::mutex> g(ctx().mu);
    DevPool *p = nullptr;
    int rc = pool_for_device(&p);
    if (rc) return rc;
    const WsLayout L = layout_one(I, use_wave(I));
    if (L.total > *ws_cap) {
        cudaStreamSynchronize(stream);
        cudaFree(*ws);
        *ws = nullptr;
        *ws_cap = 0;
        if (cudaMalloc((void **)ws, L.total) != cudaSuccess) { cudaGetLastError(); *ws = nullptr; return kErrNomem; }
        if (cudaMemsetAsync(*ws, 0, L.total, stream) != cudaSuccess) return kErrCuda;
        *ws_cap = L.total;
    }
    return enqueue_one(comp, out, I, *ws, L, status_out ? status_out : (int32_t *)(*ws + L.status), p->num_sms, stream);
}

// Transcoder (transcode.cu): header parsing, and a decode by the wavefront path's warp dataflow that leaves
// every match's record (stream order) in the caller's workspace and copies every byte's root with the byte
// (root[] holds y at every position beforehand).
int tc_parse_header(const uint8_t *h, size_t len, aceapex_info *info) { return parse_header(h, len, info); }
size_t tc_workspace_size(const aceapex_info &I) { return layout_one(I, true).total; }
int tc_decode(const void *comp, void *out, const aceapex_info &I, uint8_t *ws, WaveBufs *wb, uint32_t *root,
              int32_t *status, int *num_sms, cudaStream_t stream) {
    std::lock_guard<std::mutex> g(ctx().mu);
    DevPool *p = nullptr;
    int rc = pool_for_device(&p);
    if (rc) return rc;
    const WsLayout L = layout_one(I, true);
    if (cudaMemsetAsync(ws, 0, L.total, stream) != cudaSuccess) return cuda_fail(cudaErrorUnknown);
    *wb = wave_bufs(ws, L);
    *num_sms = p->num_sms;
    return enqueue_one(comp, out, I, ws, L, status, p->num_sms, stream, 2, root);
}
}  // namespace aceapex_host

// ================================================================================================ C ABI
extern "C" {

int aceapex_peek_header(const void *host_prefix, size_t len, aceapex_info *info) {
    return parse_header((const uint8_t *)host_prefix, len, info);
}

size_t aceapex_workspace_size(const aceapex_info *info) {
    if (!info) return 0;
    std::lock_guard<std::mutex> g(ctx().mu);
    return layout_one(*info, use_wave(*info)).total;
}

int aceapex_decode(const void *comp, size_t comp_len, void *out, size_t out_len, void *stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    if (!check_ptrs(comp, comp_len, out, out_len)) return kErrArg;
    std::lock_guard<std::mutex> g(ctx().mu);
    DevPool *p = nullptr;
    int rc = pool_for_device(&p);
    if (rc) return rc;
    if (cudaMemcpyAsync(p->host, comp, kStreamHeader, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return cuda_fail(cudaErrorUnknown);
    aceapex_info I;
    rc = parse_header(p->host, kStreamHeader, &I);
    if (rc) return rc;
    if (I.comp_len != comp_len || I.decoded_len != out_len) return kErrSize;
    aceapex_stats &S = ctx().stats;
    memset(&S, 0, sizeof(S));
    S.decoded_len = I.decoded_len; S.comp_len = I.comp_len; S.n_match = I.n_match; S.n_tiles = I.n_tiles;
    S.max_depth = I.max_depth;
    S.one_pass = !use_wave(I);
    if (I.decoded_len == 0) return (I.n_blocks || I.n_match || I.n_seq || I.max_depth) ? kErrFormat : kOK;
    const bool wave = use_wave(I);
    const WsLayout L = layout_one(I, wave);
    rc = pool_reserve(*p, L.total, stream);
    if (rc) return rc;
    int32_t *d_status = (int32_t *)(p->ws + L.status);
    rc = enqueue_one(comp, out, I, p->ws, L, d_status, p->num_sms, stream);
    if (rc) return rc;
    int32_t *h_status = (int32_t *)p->host;
    if (cudaMemcpyAsync(h_status, d_status, 4, cudaMemcpyDeviceToHost, stream) != cudaSuccess) return kErrCuda;
    uint32_t *h_hist = (uint32_t *)(p->host + 64);
    const uint32_t nh = std::min<uint32_t>(I.max_depth + 1, ACEAPEX_HIST_MAX);
    if (wave) {
        if (cudaMemcpyAsync(h_hist, p->ws + L.hist, 4 * nh, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaMemcpyAsync(p->host + 32, p->ws + L.head + offsetof(WsHead, depth_seen), 4, cudaMemcpyDeviceToHost,
                            stream) != cudaSuccess)
            return kErrCuda;
    }
    if (prof_enabled() &&
        cudaMemcpyAsync(p->host + 32768, p->ws + L.head + offsetof(WsHead, phase), 64, cudaMemcpyDeviceToHost, stream) != cudaSuccess)
        return kErrCuda;
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e);
    if (prof_enabled()) memcpy(S.phase_cycles, p->host + 32768, 64);
    if (wave) {
        S.n_levels = *(uint32_t *)(p->host + 32);
        S.hist_len = nh;
        for (uint32_t k = 0; k < nh; k++) S.level_hist[k] = h_hist[k];
    }
    return *h_status;
}

int aceapex_decode_async(const void *comp, size_t comp_len, void *out, size_t out_len, const aceapex_info *info,
                         void *d_ws, size_t ws_len, int32_t *d_status, void *stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    if (!check_ptrs(comp, comp_len, out, out_len) || !info || !d_status || ((uintptr_t)d_ws & 15)) return kErrArg;
    if (info->comp_len != comp_len || info->decoded_len != out_len) return kErrSize;
    std::lock_guard<std::mutex> g(ctx().mu);
    DevPool *p = nullptr;
    int rc = pool_for_device(&p);
    if (rc) return rc;
    if (info->decoded_len == 0) return cuda_fail(cudaMemsetAsync(d_status, 0, 4, stream));
    const WsLayout L = layout_one(*info, use_wave(*info));
    if (!d_ws || ws_len < L.total) return kErrNomem;
    return enqueue_one(comp, out, *info, (uint8_t *)d_ws, L, d_status, p->num_sms, stream);
}

// ------------------------------------------------------------------------------------------ batch
struct aceapex_batch_plan {
    int n = 0;
    int device = 0;
    int num_sms = 0;
    std::vector<int32_t> arg_status;       // status known on the host (argument / header errors)
    std::vector<int> flat_idx, wave_idx;    // stream indices per path
    std::vector<aceapex_info> info;
    std::vector<const void *> comps;
    std::vector<void *> outs;
    LaunchArgs flat_args{};
    uint8_t *ws = nullptr;                 // flat workspace: head, states, statuses, descriptors, flags
    WsLayout flat_L{};
    uint8_t *wave_ws = nullptr;            // shared by the wave streams, decoded one after another
    size_t wave_cap = 0;
    int32_t *wave_status = nullptr;        // one device status per wave stream
    int32_t *status_map = nullptr;         // device, 2 per stream: where its status comes from (plan_statuses_device)
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
};

// Read the 64-byte header of every stream back to the host (one small copy per stream, one sync).
static int read_headers(int n, const void *const *comps, std::vector<uint8_t> &hdr, cudaStream_t stream) {
    uint8_t *pinned = nullptr;
    if (cudaMallocHost((void **)&pinned, (size_t)n * kStreamHeader) != cudaSuccess) return kErrNomem;
    for (int i = 0; i < n; i++) {
        if (!comps[i]) continue;
        if (cudaMemcpyAsync(pinned + (size_t)i * kStreamHeader, comps[i], kStreamHeader, cudaMemcpyDeviceToHost,
                            stream) != cudaSuccess) {
            cudaFreeHost(pinned);
            return cuda_fail(cudaErrorUnknown);
        }
    }
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) hdr.assign(pinned, pinned + (size_t)n * kStreamHeader);
    cudaFreeHost(pinned);
    return cuda_fail(e);
}

int aceapex_batch_plan_create(int n, const void *const *comps, const size_t *comp_lens, void *const *outs,
                              const size_t *out_lens, void *stream_, aceapex_batch_plan **plan_out) {
    cudaStream_t stream = (cudaStream_t)stream_;
    if (n < 0 || (n > 0 && (!comps || !comp_lens || !outs || !out_lens)) || !plan_out) return kErrArg;
    std::lock_guard<std::mutex> g(ctx().mu);
    DevPool *p = nullptr;
    int rc = pool_for_device(&p);
    if (rc) return rc;
    aceapex_batch_plan *P = new (std::nothrow) aceapex_batch_plan();
    if (!P) return kErrNomem;
    P->n = n;
    cudaGetDevice(&P->device);
    P->num_sms = p->num_sms;
    P->arg_status.assign(n, 0);
    P->info.resize(n);
    P->comps.assign(comps, comps + n);
    P->outs.assign(outs, outs + n);
    std::vector<const void *> valid(n, nullptr);
    for (int i = 0; i < n; i++) {
        if (!check_ptrs(comps[i], comp_lens[i], outs[i], out_lens[i])) P->arg_status[i] = kErrArg;
        else valid[i] = comps[i];
    }
    std::vector<uint8_t> hdr;
    rc = read_headers(n, valid.data(), hdr, stream);
    if (rc) { delete P; return rc; }
    std::vector<StreamDesc> descs;
    std::vector<uint64_t> lm_at;  // word offset of each one-pass stream's literal bitmap
    uint64_t tiles = 0, lm_words = 0;
    size_t wave_need = 0;
    for (int i = 0; i < n; i++) {
        if (P->arg_status[i]) continue;
        aceapex_info &I = P->info[i];
        int r = parse_header(hdr.data() + (size_t)i * kStreamHeader, kStreamHeader, &I);
        if (!r && (I.comp_len != comp_lens[i] || I.decoded_len != out_lens[i])) r = kErrSize;
        if (!r && I.decoded_len == 0 && (I.n_blocks || I.n_match || I.n_seq || I.max_depth)) r = kErrFormat;
        if (r) { P->arg_status[i] = r; continue; }
        if (I.decoded_len == 0) continue;  // nothing to do, status 0
        if (use_wave(I)) {
            P->wave_idx.push_back(i);
            wave_need = std::max(wave_need, layout_one(I, true).total);
        } else {
            P->flat_idx.push_back(i);
            P->flat_args.max_tile_log2 = std::max(P->flat_args.max_tile_log2, I.tile_log2);
            P->flat_args.max_n = std::max<unsigned long long>(P->flat_args.max_n, I.decoded_len);
            descs.push_back(make_desc(comps[i], outs[i], I, tiles));
            tiles += I.n_tiles;
            lm_at.push_back(lm_words);
            lm_words += litmap_words(I.decoded_len);
        }
    }
    const int nf = (int)P->flat_idx.size();
    // >= 2 streams: the descriptor table always lives in memory
    P->flat_L = layout(std::max(nf, 2), tiles, false, nullptr, lm_words);
    if (nf > 0) {
        if (cudaMalloc((void **)&P->ws, P->flat_L.total) != cudaSuccess) { cudaGetLastError(); delete P; return kErrNomem; }
        for (int k = 0; k < nf; k++) descs[k].litmap = (uint32_t *)(P->ws + P->flat_L.litmap) + lm_at[k];
        cudaMemsetAsync(P->ws, 0, P->flat_L.total, stream);
        cudaMemcpyAsync(P->ws + P->flat_L.descs, descs.data(), sizeof(StreamDesc) * nf, cudaMemcpyHostToDevice, stream);
        P->flat_args.n_streams = nf;
        P->flat_args.total_tiles = tiles;
        if (nf == 1) P->flat_args.one = descs[0];
    }
    if (!P->wave_idx.empty()) {
        P->wave_cap = wave_need;
        if (cudaMalloc((void **)&P->wave_ws, wave_need) != cudaSuccess ||
            cudaMalloc((void **)&P->wave_status, 4 * P->wave_idx.size()) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(P->ws); cudaFree(P->wave_ws);
            delete P;
            return kErrNomem;
        }
        cudaMemsetAsync(P->wave_ws, 0, wave_need, stream);
    }
    // per stream: (0, status known on the host) | (1, index among the one-pass streams) | (2, index among the
    // wavefront streams), for the stream-ordered status gather
    std::vector<int32_t> map(2 * (size_t)std::max(n, 1), 0);
    for (int i = 0; i < n; i++) map[2 * i + 1] = P->arg_status[i];
    for (size_t k = 0; k < P->flat_idx.size(); k++) { map[2 * P->flat_idx[k]] = 1; map[2 * P->flat_idx[k] + 1] = (int32_t)k; }
    for (size_t k = 0; k < P->wave_idx.size(); k++) { map[2 * P->wave_idx[k]] = 2; map[2 * P->wave_idx[k] + 1] = (int32_t)k; }
    cudaError_t e = cudaMalloc((void **)&P->status_map, 4 * map.size());
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->status_map, map.data(), 4 * map.size(), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        cudaFree(P->ws); cudaFree(P->wave_ws); cudaFree(P->wave_status); cudaFree(P->status_map);
        delete P;
        return cuda_fail(e);
    }
    *plan_out = P;
    return kOK;
}

int aceapex_batch_plan_statuses_device(aceapex_batch_plan *P, int32_t *d_statuses, void *stream_) {
    if (!P || (!d_statuses && P->n)) return kErrArg;
    if (P->n == 0) return kOK;
    return cuda_fail(launch_gather_status(P->n, P->status_map, (const int32_t *)(P->ws + P->flat_L.status),
                                          P->wave_status, d_statuses, (cudaStream_t)stream_));
}

static int plan_enqueue(aceapex_batch_plan *P, cudaStream_t stream) {
    LaunchCfg cfg = ctx().cfg;
    cfg.num_sms = P->num_sms;
    if (!P->flat_idx.empty()) {
        P->flat_args.wait_ns = ctx().wait_ns;
        P->flat_args.withhold = ctx().withhold;
        uint8_t *ws = P->ws;
        const WsLayout &L = P->flat_L;
        const StreamDesc *descs = P->flat_args.n_streams > 1 ? (const StreamDesc *)(ws + L.descs) : nullptr;
        cudaError_t e = launch_flat(cfg, (WsHead *)(ws + L.head), (StreamState *)(ws + L.sst), (uint32_t *)(ws + L.flags),
                                    descs, P->flat_args, (int32_t *)(ws + L.status), stream);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    for (size_t k = 0; k < P->wave_idx.size(); k++) {
        const int i = P->wave_idx[k];
        const aceapex_info &I = P->info[i];
        const WsLayout L = layout_one(I, true);
        int rc = enqueue_one(P->comps[i], P->outs[i], I, P->wave_ws, L, P->wave_status + k, P->num_sms, stream);
        if (rc) return rc;
    }
    return kOK;
}

int aceapex_batch_plan_launch(aceapex_batch_plan *P, int graph, void *stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    if (!P) return kErrArg;
    std::lock_guard<std::mutex> g(ctx().mu);
    if (!graph) return plan_enqueue(P, stream);
    if (!P->exec) {
        // capture on a private stream: the caller's may be the legacy default stream, which cannot capture
        cudaStream_t cap = nullptr;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return cuda_fail(cudaErrorUnknown);
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaStreamDestroy(cap);
            return cuda_fail(cudaErrorUnknown);
        }
        int rc = plan_enqueue(P, cap);
        cudaGraph_t gr = nullptr;
        cudaError_t e = cudaStreamEndCapture(cap, &gr);
        cudaStreamDestroy(cap);
        if (rc || e != cudaSuccess) { if (gr) cudaGraphDestroy(gr); return rc ? rc : cuda_fail(e); }
        e = cudaGraphInstantiate(&P->exec, gr, 0);
        if (e != cudaSuccess) { cudaGraphDestroy(gr); P->exec = nullptr; return cuda_fail(e); }
        P->graph = gr;
    }
    return cuda_fail(cudaGraphLaunch(P->exec, stream));
}

int aceapex_batch_plan_statuses(aceapex_batch_plan *P, int32_t *statuses, void *stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    if (!P || (!statuses && P->n)) return kErrArg;
    std::vector<int32_t> fs(P->flat_idx.size()), wsts(P->wave_idx.size());
    if (!fs.empty() && cudaMemcpyAsync(fs.data(), P->ws + P->flat_L.status, 4 * fs.size(), cudaMemcpyDeviceToHost,
                                       stream) != cudaSuccess)
        return cuda_fail(cudaErrorUnknown);
    if (!wsts.empty() &&
        cudaMemcpyAsync(wsts.data(), P->wave_status, 4 * wsts.size(), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
        return cuda_fail(cudaErrorUnknown);
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e);
    int first = 0;
    for (int i = 0; i < P->n; i++) statuses[i] = P->arg_status[i];
    for (size_t k = 0; k < fs.size(); k++) statuses[P->flat_idx[k]] = fs[k];
    for (size_t k = 0; k < wsts.size(); k++) statuses[P->wave_idx[k]] = wsts[k];
    for (int i = 0; i < P->n; i++) if (statuses[i] && !first) first = statuses[i];
    return first;
}

int aceapex_batch_plan_destroy(aceapex_batch_plan *P) {
    if (!P) return kErrArg;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    cudaFree(P->ws);
    cudaFree(P->wave_ws);
    cudaFree(P->wave_status);
    cudaFree(P->status_map);
    delete P;
    return kOK;
}

int aceapex_decode_batch(int n, const void *const *comps, const size_t *comp_lens, void *const *outs,
                         const size_t *out_lens, int32_t *statuses, void *stream) {
    if (n < 0 || (n > 0 && !statuses)) return kErrArg;
    aceapex_batch_plan *P = nullptr;
    int rc = aceapex_batch_plan_create(n, comps, comp_lens, outs, out_lens, stream, &P);
    if (rc) return rc;
    rc = aceapex_batch_plan_launch(P, 0, stream);
    int rs = rc ? rc : aceapex_batch_plan_statuses(P, statuses, stream);
    aceapex_batch_plan_destroy(P);
    return rs;
}

// ------------------------------------------------------------------------------------------ config, stats
int aceapex_set_launch_config(int warps_per_cta, int ctas_per_sm) {
    if ((warps_per_cta != 2 && warps_per_cta != 4 && warps_per_cta != 8) || ctas_per_sm < 0) return kErrArg;
    std::lock_guard<std::mutex> g(ctx().mu);
    ctx().cfg.warps = warps_per_cta;
    ctx().cfg.ctas_per_sm = ctas_per_sm;
    return kOK;
}

int aceapex_get_launch_config(int *warps_per_cta, int *ctas_per_sm) {
    if (!warps_per_cta || !ctas_per_sm) return kErrArg;
    std::lock_guard<std::mutex> g(ctx().mu);
    *warps_per_cta = ctx().cfg.warps;
    *ctas_per_sm = ctx().cfg.ctas_per_sm;
    return kOK;
}

int aceapex_set_wave_scheduler(int kind) {
    if (kind < 0 || kind > 2) return kErrArg;
    std::lock_guard<std::mutex> g(ctx().mu);
    ctx().cfg.wave_sched = kind;
    return kOK;
}

int aceapex_set_force_wavefront(int on) {
    std::lock_guard<std::mutex> g(ctx().mu);
    ctx().force_wave = on != 0;
    return kOK;
}

int aceapex_set_wait_limit(uint64_t ns, uint64_t withhold_tile) {
    std::lock_guard<std::mutex> g(ctx().mu);
    ctx().wait_ns = ns ? ns : 4000000000ull;
    ctx().withhold = withhold_tile;
    return kOK;
}

int aceapex_profile(int enable) {
    std::lock_guard<std::mutex> g(ctx().mu);
    prof_enable(enable != 0);
    return kOK;
}

int aceapex_profile_read(int max_kernels, const char **names, double *total_ms, uint64_t *launches) {
    if (max_kernels < 0 || (max_kernels > 0 && (!names || !total_ms || !launches))) return kErrArg;
    std::lock_guard<std::mutex> g(ctx().mu);
    double ms[kKCount];
    unsigned long long n[kKCount];
    prof_collect(ms, n);
    const int k = std::min(max_kernels, (int)kKCount);
    for (int i = 0; i < k; i++) { names[i] = kKernelNames[i]; total_ms[i] = ms[i]; launches[i] = n[i]; }
    return kKCount;
}

int aceapex_get_stats(aceapex_stats *s) {
    if (!s) return kErrArg;
    std::lock_guard<std::mutex> g(ctx().mu);
    *s = ctx().stats;
    return kOK;
}

// ------------------------------------------------------------------------------------------ host buffers
namespace {
int grow(uint8_t **buf, size_t *cap, size_t need) {
    if (need <= *cap) return kOK;
    cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    if (cudaMalloc((void **)buf, need) != cudaSuccess) { cudaGetLastError(); *buf = nullptr; return kErrNomem; }
    *cap = need;
    return kOK;
}
int host_path_init(DevPool &p) {
    if (p.s_in) return kOK;
    bool ok = cudaStreamCreateWithFlags(&p.s_in, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p.s_out, cudaStreamNonBlocking) == cudaSuccess &&
              cudaMalloc((void **)&p.hd_state, sizeof(StreamState)) == cudaSuccess;
    for (int k = 0; ok && k < kHostSlices; k++)
        ok = cudaEventCreateWithFlags(&p.ev_in[k], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&p.ev_dec[k], cudaEventDisableTiming) == cudaSuccess;
    return ok ? kOK : cuda_fail(cudaErrorUnknown);
}
}  // namespace

int aceapex_decode_host(const void *h_comp, size_t comp_len, void *h_out, size_t out_len, void *stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    if (!h_comp || comp_len < kStreamHeader || (!h_out && out_len)) return kErrArg;
    aceapex_info I;
    int rc = parse_header((const uint8_t *)h_comp, kStreamHeader, &I);
    if (rc) return rc;
    if (I.comp_len != comp_len || I.decoded_len != out_len) return kErrSize;
    if (I.decoded_len == 0) return (I.n_blocks || I.n_match || I.n_seq || I.max_depth) ? kErrFormat : kOK;
    std::lock_guard<std::mutex> g(ctx().mu);
    DevPool *p = nullptr;
    rc = pool_for_device(&p);
    if (!rc) rc = host_path_init(*p);
    if (!rc) rc = grow(&p->hd_comp, &p->hd_comp_cap, comp_len);
    if (!rc) rc = grow(&p->hd_out, &p->hd_out_cap, out_len);
    if (rc) return rc;
    const bool wave = use_wave(I);
    const WsLayout L = layout_one(I, wave);
    rc = pool_reserve(*p, L.total, stream);
    if (rc) return rc;
    aceapex_stats &S = ctx().stats;
    memset(&S, 0, sizeof(S));
    S.decoded_len = I.decoded_len; S.comp_len = I.comp_len; S.n_match = I.n_match; S.n_tiles = I.n_tiles;
    S.max_depth = I.max_depth;
    S.one_pass = !wave;
    const uint8_t *hc = (const uint8_t *)h_comp;
    uint8_t *ho = (uint8_t *)h_out;
    int32_t *d_status = (int32_t *)(p->ws + L.status);
    int32_t *h_status = (int32_t *)p->host;
    // slices: whole blocks of the stream in order; a slice's stream bytes end where its last block ends
    const uint64_t B = 1ull << I.block_log2, T = 1ull << I.tile_log2, tpb = B / T;
    int ns = (int)std::min<uint64_t>((uint64_t)kHostSlices, (I.decoded_len + (32ull << 20) - 1) / (32ull << 20));
    if (ns < 1) ns = 1;
    if (wave || I.n_blocks < (uint64_t)ns) ns = 1;
    // the block index must be usable to cut the stream; otherwise copy it whole (the kernels report the error)
    std::vector<uint64_t> cut(ns + 1, 0);
    uint64_t t_beg[kHostSlices + 1];
    for (int k = 0; k <= ns; k++) {
        const uint64_t bb = (I.n_blocks * (uint64_t)k) / (uint64_t)ns;  // first block of slice k
        t_beg[k] = k == ns ? I.n_tiles : bb * tpb;
        if (k == ns || k == 0) { cut[k] = k == ns ? comp_len : 0; continue; }
        cut[k] = rd(hc + kStreamHeader + 8 * bb, 8);
    }
    for (int k = 1; k <= ns; k++)
        if (cut[k] < cut[k - 1] || cut[k] > comp_len || (cut[k] & 15)) { ns = 1; cut[1] = comp_len; t_beg[1] = I.n_tiles; break; }
    // every copy and launch below waits for the caller's earlier work on its stream
    if (cudaEventRecord(p->ev_dec[0], stream) != cudaSuccess || cudaStreamWaitEvent(p->s_in, p->ev_dec[0], 0) != cudaSuccess)
        return cuda_fail(cudaErrorUnknown);
    for (int k = 0; k < ns; k++) {
        if (cudaMemcpyAsync(p->hd_comp + cut[k], hc + cut[k], cut[k + 1] - cut[k], cudaMemcpyHostToDevice, p->s_in) !=
                cudaSuccess ||
            cudaEventRecord(p->ev_in[k], p->s_in) != cudaSuccess)
            return cuda_fail(cudaErrorUnknown);
    }
    LaunchCfg cfg = ctx().cfg;
    cfg.num_sms = p->num_sms;
    if (wave) {
        if (cudaStreamWaitEvent(stream, p->ev_in[0], 0) != cudaSuccess) return kErrCuda;
        rc = enqueue_one(p->hd_comp, p->hd_out, I, p->ws, L, d_status, p->num_sms, stream);
        if (rc) return rc;
        if (cudaEventRecord(p->ev_dec[0], stream) != cudaSuccess) return kErrCuda;
    } else {
        if (aceapex_host::init_state(p->hd_state, stream)) return kErrCuda;
        for (int k = 0; k < ns; k++) {
            if (cudaStreamWaitEvent(stream, p->ev_in[k], 0) != cudaSuccess) return kErrCuda;
            LaunchArgs a{};
            a.one = make_desc(p->hd_comp, p->hd_out, I, 0);
            a.one.n_tiles = t_beg[k + 1] - t_beg[k];
            a.one.tile_off = t_beg[k];
            a.one.state = p->hd_state;
            a.one.litmap = (uint32_t *)(p->ws + L.litmap);
            a.one.flags = k + 1 == ns ? kDescLast : 0u;
            a.n_streams = 1;
            a.total_tiles = a.one.n_tiles;
            a.wait_ns = ctx().wait_ns;
            a.withhold = ~0ull;
            a.max_tile_log2 = I.tile_log2;
            a.max_n = I.decoded_len;
            WsHead *head = (WsHead *)(p->ws + L.head);
            StreamState *sst = (StreamState *)(p->ws + L.sst);
            cudaError_t e = launch_flat(cfg, head, sst, (uint32_t *)(p->ws + L.flags), nullptr, a,
                                        k + 1 == ns ? d_status : nullptr, stream);
            if (e != cudaSuccess) return cuda_fail(e);
            if (cudaEventRecord(p->ev_dec[k], stream) != cudaSuccess) return kErrCuda;
            // this slice's output is final once its launch has completed (its sources lie before it)
            const uint64_t o0 = t_beg[k] * T, o1 = std::min<uint64_t>(t_beg[k + 1] * T, I.decoded_len);
            if (k + 1 < ns && o1 > o0) {
                if (cudaStreamWaitEvent(p->s_out, p->ev_dec[k], 0) != cudaSuccess ||
                    cudaMemcpyAsync(ho + o0, p->hd_out + o0, o1 - o0, cudaMemcpyDeviceToHost, p->s_out) != cudaSuccess)
                    return cuda_fail(cudaErrorUnknown);
            }
        }
    }
    // the last slice (or the whole stream), then the status
    const uint64_t o0 = wave ? 0 : t_beg[ns - 1] * T;
    if (cudaStreamWaitEvent(p->s_out, p->ev_dec[wave ? 0 : ns - 1], 0) != cudaSuccess ||
        cudaMemcpyAsync(ho + o0, p->hd_out + o0, I.decoded_len - o0, cudaMemcpyDeviceToHost, p->s_out) != cudaSuccess ||
        cudaMemcpyAsync(h_status, d_status, 4, cudaMemcpyDeviceToHost, p->s_out) != cudaSuccess)
        return cuda_fail(cudaErrorUnknown);
    cudaError_t e = cudaStreamSynchronize(p->s_out);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e);
    return *h_status;
}

// ------------------------------------------------------------------------------------------ batch, host buffers
namespace {
constexpr uint64_t kBatchHostGap = 64 * 1024;  // a host gap up to this size between streams is copied in too
constexpr int kBatchHostGroups = 32;           // about this many copy-in / decode / copy-out groups per call

struct HostRun {  // one copy of len bytes between host memory and device offset dev
    uint64_t dev;
    uint8_t *host;
    uint64_t len;
};
struct HostGroup {
    std::vector<int> flat, wave;    // the group's streams by path, in stream order
    std::vector<uint64_t> lm_at;    // per one-pass stream: word offset of its literal bitmap
    std::vector<HostRun> in, out;   // copies in and out
    WsLayout L{};                   // one-pass workspace, at ws_at in the batch workspace
    uint64_t ws_at = 0, tiles = 0, lm_words = 0;
    uint64_t pin_desc = 0, pin_status = 0;  // descriptors and statuses in the pinned staging buffer
    unsigned int max_tile_log2 = 0;
    unsigned long long max_n = 0;
};

int grow_pinned(uint8_t **buf, size_t *cap, size_t need) {
    if (need <= *cap) return kOK;
    cudaFreeHost(*buf);
    *buf = nullptr;
    *cap = 0;
    if (cudaMallocHost((void **)buf, need) != cudaSuccess) { cudaGetLastError(); *buf = nullptr; return kErrNomem; }
    *cap = need;
    return kOK;
}

// Cut the live streams into groups and lay out their device copies, workspaces and pinned staging.
// Consecutive streams whose host bytes follow each other share one copy: copies in bridge gaps of up to
// kBatchHostGap bytes and keep 16-byte offsets (the device streams stay 16-byte aligned); copies out join
// back-to-back outputs only, so no caller byte outside an output is written.
void plan_host_groups(int n, const void *const *h_comps, const size_t *comp_lens, void *const *h_outs,
                      const size_t *out_lens, const std::vector<aceapex_info> &info, const std::vector<char> &live,
                      uint64_t target, std::vector<HostGroup> &groups, std::vector<uint64_t> &d_comp,
                      std::vector<uint64_t> &d_out, uint64_t &c_end, uint64_t &o_end, uint64_t &ws_end,
                      uint64_t &pin_end, uint64_t &wave_need, uint64_t &n_wave) {
    c_end = o_end = ws_end = pin_end = wave_need = n_wave = 0;
    for (int i = 0; i < n;) {
        HostGroup G;
        uint64_t acc = 0, in_d = 0, out_d = 0;
        uint8_t *in_h = nullptr, *in_e = nullptr, *out_h = nullptr, *out_e = nullptr;
        for (; i < n && acc < target; i++) {
            if (!live[i]) continue;
            const aceapex_info &I = info[i];
            uint8_t *hc = (uint8_t *)h_comps[i], *ho = (uint8_t *)h_outs[i];
            if (in_h && hc >= in_e && (uint64_t)(hc - in_e) <= kBatchHostGap && ((hc - in_h) & 15) == 0) {
                in_e = std::max(in_e, hc + comp_lens[i]);
            } else {
                if (in_h) { G.in.push_back({in_d, in_h, (uint64_t)(in_e - in_h)}); c_end = in_d + (uint64_t)(in_e - in_h); }
                in_d = align16(c_end);
                in_h = hc;
                in_e = hc + comp_lens[i];
            }
            d_comp[i] = in_d + (uint64_t)(hc - in_h);
            if (out_h && ho == out_e) {
                out_e += out_lens[i];
            } else {
                if (out_h) { G.out.push_back({out_d, out_h, (uint64_t)(out_e - out_h)}); o_end = out_d + (uint64_t)(out_e - out_h); }
                out_d = align16(o_end) + ((uintptr_t)ho & 15);  // the device copy keeps the host's alignment
                out_h = ho;
                out_e = ho + out_lens[i];
            }
            d_out[i] = out_d + (uint64_t)(ho - out_h);
            acc += I.decoded_len;
            if (use_wave(I)) {
                G.wave.push_back(i);
                wave_need = std::max<uint64_t>(wave_need, layout_one(I, true).total);
                n_wave++;
            } else {
                G.flat.push_back(i);
                G.max_tile_log2 = std::max(G.max_tile_log2, I.tile_log2);
                G.max_n = std::max<unsigned long long>(G.max_n, I.decoded_len);
                G.lm_at.push_back(G.lm_words);
                G.tiles += I.n_tiles;
                G.lm_words += litmap_words(I.decoded_len);
            }
        }
        if (in_h) { G.in.push_back({in_d, in_h, (uint64_t)(in_e - in_h)}); c_end = in_d + (uint64_t)(in_e - in_h); }
        if (out_h) { G.out.push_back({out_d, out_h, (uint64_t)(out_e - out_h)}); o_end = out_d + (uint64_t)(out_e - out_h); }
        if (G.flat.empty() && G.wave.empty()) continue;
        const size_t nf = G.flat.size();
        if (nf) {
            G.L = layout(std::max<int>((int)nf, 2), G.tiles, false, nullptr, G.lm_words);  // descriptor table in memory
            G.ws_at = ws_end;
            ws_end = up(ws_end + G.L.total);
            G.pin_desc = pin_end;
            pin_end = up(pin_end + sizeof(StreamDesc) * nf);
        }
        G.pin_status = pin_end;
        pin_end = up(pin_end + 4 * (nf + G.wave.size()));
        groups.push_back(std::move(G));
    }
}
}  // namespace

int aceapex_decode_batch_host(int n, const void *const *h_comps, const size_t *comp_lens, void *const *h_outs,
                              const size_t *out_lens, int32_t *statuses, void *stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    if (n < 0 || (n > 0 && (!h_comps || !comp_lens || !h_outs || !out_lens || !statuses))) return kErrArg;
    // headers straight from host memory: argument and header errors are known before any device work
    std::vector<aceapex_info> info(n);
    std::vector<char> live(n, 0);
    uint64_t n_total = 0;
    for (int i = 0; i < n; i++) {
        statuses[i] = 0;
        if (!h_comps[i] || comp_lens[i] < kStreamHeader || (!h_outs[i] && out_lens[i])) { statuses[i] = kErrArg; continue; }
        aceapex_info &I = info[i];
        int r = parse_header((const uint8_t *)h_comps[i], kStreamHeader, &I);
        if (!r && (I.comp_len != comp_lens[i] || I.decoded_len != out_lens[i])) r = kErrSize;
        if (!r && I.decoded_len == 0 && (I.n_blocks || I.n_match || I.n_seq || I.max_depth)) r = kErrFormat;
        if (r) { statuses[i] = r; continue; }
        if (I.decoded_len == 0) continue;
        live[i] = 1;
        n_total += I.decoded_len;
    }
    auto first_error = [&]() {
        for (int i = 0; i < n; i++) if (statuses[i]) return (int)statuses[i];
        return (int)kOK;
    };
    if (n_total == 0) return first_error();
    std::lock_guard<std::mutex> g(ctx().mu);
    DevPool *p = nullptr;
    int rc = pool_for_device(&p);
    if (!rc) rc = host_path_init(*p);
    if (rc) return rc;
    std::vector<HostGroup> groups;
    std::vector<uint64_t> d_comp(n, 0), d_out(n, 0);
    uint64_t c_end, o_end, ws_end, pin_end, wave_need, n_wave;
    plan_host_groups(n, h_comps, comp_lens, h_outs, out_lens, info, live,
                     std::max<uint64_t>(n_total / kBatchHostGroups, 16ull << 20), groups, d_comp, d_out, c_end, o_end,
                     ws_end, pin_end, wave_need, n_wave);
    const uint64_t wave_at = ws_end, wst_at = up(wave_at + wave_need);
    ws_end = up(wst_at + 4 * (n_wave + 1));
    // every buffer is in place before the first copy: growing one frees the old one, which synchronises
    rc = grow(&p->hb_comp, &p->hb_comp_cap, c_end + 16);
    if (!rc) rc = grow(&p->hb_out, &p->hb_out_cap, o_end + 16);
    if (!rc) rc = grow(&p->hb_ws, &p->hb_ws_cap, ws_end);
    if (!rc) rc = grow_pinned(&p->hb_pin, &p->hb_pin_cap, pin_end + 16);
    if (rc) return rc;
    uint8_t *ws = p->hb_ws;
    for (HostGroup &G : groups) {
        StreamDesc *D = (StreamDesc *)(p->hb_pin + G.pin_desc);
        uint64_t tb = 0;
        for (size_t k = 0; k < G.flat.size(); k++) {
            const int i = G.flat[k];
            D[k] = make_desc(p->hb_comp + d_comp[i], p->hb_out + d_out[i], info[i], tb);
            D[k].litmap = (uint32_t *)(ws + G.ws_at + G.L.litmap) + G.lm_at[k];
            tb += info[i].n_tiles;
        }
    }
    // on a failure after work was enqueued, the call returns only once no copy touches the caller's buffers
    auto fail = [&](int code) {
        cudaStreamSynchronize(p->s_in);
        cudaStreamSynchronize(stream);
        cudaStreamSynchronize(p->s_out);
        return code;
    };
    // ordered after the caller's earlier work on `stream`; the groups' control regions (head, states,
    // statuses, descriptors, tile flags: flags hold launch epochs) start zeroed, the wavefront workspace too
    if (cudaEventRecord(p->ev_dec[0], stream) != cudaSuccess || cudaStreamWaitEvent(p->s_in, p->ev_dec[0], 0) != cudaSuccess ||
        cudaStreamWaitEvent(p->s_out, p->ev_dec[0], 0) != cudaSuccess)
        return fail(cuda_fail(cudaErrorUnknown));
    for (const HostGroup &G : groups) {
        if (G.flat.empty()) continue;
        if (cudaMemsetAsync(ws + G.ws_at, 0, G.L.litmap, stream) != cudaSuccess ||
            cudaMemcpyAsync(ws + G.ws_at + G.L.descs, p->hb_pin + G.pin_desc, sizeof(StreamDesc) * G.flat.size(),
                            cudaMemcpyHostToDevice, stream) != cudaSuccess)
            return fail(cuda_fail(cudaErrorUnknown));
    }
    if (n_wave && cudaMemsetAsync(ws + wave_at, 0, wave_need, stream) != cudaSuccess) return fail(cuda_fail(cudaErrorUnknown));
    LaunchCfg cfg = ctx().cfg;
    cfg.num_sms = p->num_sms;
    int32_t *wave_status = (int32_t *)(ws + wst_at);
    uint64_t wk = 0;
    for (size_t gi = 0; gi < groups.size(); gi++) {
        const HostGroup &G = groups[gi];
        const int e = (int)(gi % kHostSlices);  // an event is re-recorded only after its waits were enqueued
        for (const HostRun &r : G.in)
            if (cudaMemcpyAsync(p->hb_comp + r.dev, r.host, r.len, cudaMemcpyHostToDevice, p->s_in) != cudaSuccess)
                return fail(cuda_fail(cudaErrorUnknown));
        if (cudaEventRecord(p->ev_in[e], p->s_in) != cudaSuccess || cudaStreamWaitEvent(stream, p->ev_in[e], 0) != cudaSuccess)
            return fail(cuda_fail(cudaErrorUnknown));
        const size_t nf = G.flat.size();
        uint8_t *gws = ws + G.ws_at;
        if (nf) {
            LaunchArgs a{};
            a.n_streams = (int)nf;
            a.total_tiles = G.tiles;
            a.wait_ns = ctx().wait_ns;
            a.withhold = ctx().withhold;
            a.max_tile_log2 = G.max_tile_log2;
            a.max_n = G.max_n;
            if (nf == 1) a.one = *(const StreamDesc *)(p->hb_pin + G.pin_desc);
            cudaError_t ce = launch_flat(cfg, (WsHead *)(gws + G.L.head), (StreamState *)(gws + G.L.sst),
                                         (uint32_t *)(gws + G.L.flags), nf > 1 ? (const StreamDesc *)(gws + G.L.descs) : nullptr,
                                         a, (int32_t *)(gws + G.L.status), stream);
            if (ce != cudaSuccess) return fail(cuda_fail(ce));
        }
        const uint64_t wk0 = wk;
        for (int i : G.wave) {
            rc = enqueue_one(p->hb_comp + d_comp[i], p->hb_out + d_out[i], info[i], ws + wave_at, layout_one(info[i], true),
                             wave_status + wk, p->num_sms, stream);
            if (rc) return fail(rc);
            wk++;
        }
        if (cudaEventRecord(p->ev_dec[e], stream) != cudaSuccess || cudaStreamWaitEvent(p->s_out, p->ev_dec[e], 0) != cudaSuccess)
            return fail(cuda_fail(cudaErrorUnknown));
        for (const HostRun &r : G.out)
            if (cudaMemcpyAsync(r.host, p->hb_out + r.dev, r.len, cudaMemcpyDeviceToHost, p->s_out) != cudaSuccess)
                return fail(cuda_fail(cudaErrorUnknown));
        if ((nf && cudaMemcpyAsync(p->hb_pin + G.pin_status, gws + G.L.status, 4 * nf, cudaMemcpyDeviceToHost, p->s_out) !=
                       cudaSuccess) ||
            (!G.wave.empty() && cudaMemcpyAsync(p->hb_pin + G.pin_status + 4 * nf, wave_status + wk0, 4 * G.wave.size(),
                                                cudaMemcpyDeviceToHost, p->s_out) != cudaSuccess))
            return fail(cuda_fail(cudaErrorUnknown));
    }
    cudaError_t ce = cudaStreamSynchronize(p->s_out);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(p->s_in);
    if (ce != cudaSuccess) return fail(cuda_fail(ce));
    for (const HostGroup &G : groups) {
        const int32_t *st = (const int32_t *)(p->hb_pin + G.pin_status);
        for (size_t k = 0; k < G.flat.size(); k++) statuses[G.flat[k]] = st[k];
        for (size_t k = 0; k < G.wave.size(); k++) statuses[G.wave[k]] = st[G.flat.size() + k];
    }
    return first_error();
}

int aceapex_choose_device(const aceapex_info *info, const aceapex_device_model *model, double *cpu_s, double *gpu_s) {
    if (!info || !model || !(model->cpu_gbps > 0)) return kErrArg;
    const double one = model->gpu_one_pass_gbps > 0 ? model->gpu_one_pass_gbps : 260.0;
    const double wave = model->gpu_wave_gbps > 0 ? model->gpu_wave_gbps : 200.0;
    const double level_s = 1e-6 * (model->gpu_level_us > 0 ? model->gpu_level_us : 16.5);
    const double fixed_s = 1e-6 * (model->gpu_fixed_us > 0 ? model->gpu_fixed_us : 30.0);
    const double N = (double)info->decoded_len, C = (double)info->comp_len;
    const double tc = N / (model->cpu_gbps * 1e9);
    bool one_pass;
    {
        std::lock_guard<std::mutex> g(ctx().mu);
        one_pass = !use_wave(*info);
    }
    double tg = fixed_s + (one_pass ? N / (one * 1e9) : N / (wave * 1e9) + level_s * info->max_depth);
    if (model->link_gbps > 0) tg += (C + N) / (model->link_gbps * 1e9);
    if (cpu_s) *cpu_s = tc;
    if (gpu_s) *gpu_s = tg;
    return tg < tc ? 1 : 0;
}

const char *aceapex_strerror(int code) {
    switch (code) {
        case kOK: return "ok";
        case kErrArg: return "invalid argument";
        case kErrFormat: return "malformed stream";
        case kErrSize: return "size mismatch";
        case kErrOffset: return "match offset out of range";
        case kErrTimeout: return "device wait timed out";
        case kErrCuda: return "CUDA runtime error";
        case kErrNomem: return "out of memory / workspace too small";
        case kErrDepth: return "match depth above the stream's max_depth";
        default: return "unknown status";
    }
}

}  // extern "C"
