// Continuous-batching decode server (C ABI: aceapex_server_*).
//
// Requests arrive with a device-resident compressed stream.  step() first admits queued requests in
// arrival order while their bytes (stream + output) fit the HBM budget and a slot is free -- the server
// allocates the output with the stream-ordered allocator -- then enqueues ONE one-pass launch that advances
// every admitted request by a slice of its tiles: a request's slices run in order (consecutive steps on one
// stream), each starting after the tiles that earlier steps decoded, so requests that arrive while others
// are on the GPU join the next launch and share it.  A request is done when the launch holding its last
// slice has completed (CUDA event).  Streams whose matches are deeper than 1 are decoded whole by the
// wavefront path on the server's own side stream, enqueued in the step that admits them: the sliced
// launches of the other requests do not wait behind them.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <deque>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/aceapex.h"
#include "decode.h"

using namespace aceapex;

namespace aceapex_host {
int server_enqueue_whole(const void *comp, void *out, const aceapex_info &I, uint8_t **ws, size_t *ws_cap,
                         int32_t *status_out, cudaStream_t stream);
LaunchCfg launch_cfg();
bool one_pass_stream(const aceapex_info &I);
int num_sms();
int init_state(StreamState *st, cudaStream_t stream);
}  // namespace aceapex_host

namespace {

struct Req {
    const void *comp = nullptr;
    size_t comp_len = 0;
    aceapex_info info{};
    void *out = nullptr;
    bool whole = false;          // decoded whole by the wavefront path (else in slices by the one-pass kernel)
    uint32_t *litmap = nullptr;  // one-pass requests: literal bitmap, allocated right after the output
    size_t out_alloc = 0;     // output bytes (+ literal bitmap) allocated at admission
    size_t bytes = 0;         // budget share: stream + output allocation
    uint64_t next_tile = 0;   // tiles [0, next_tile) are enqueued
    int slot = -1;
    int phase = 0;            // 0 queued, 1 admitted, 2 last slice enqueued, 3 released
    long done_step = -1;      // step whose event marks completion
    int32_t *h_status = nullptr;
};

constexpr int kMaxStepsInFlight = 4;
constexpr unsigned kEvFlags = cudaEventDisableTiming;

}  // namespace

struct aceapex_server {
    std::mutex mu;
    size_t budget = 0, used = 0;
    int max_slots = 0;
    uint64_t tiles_per_step = 0;
    std::vector<Req> reqs;
    std::deque<int64_t> queue;
    std::vector<int64_t> slot_owner;  // -1 = free
    // device: persistent per-slot stream states; per-step launch workspace
    StreamState *d_state = nullptr;
    uint8_t *d_ws = nullptr;          // head | flags | descs (per ring entry)
    size_t ws_stride = 0, flags_cap = 0;
    StreamDesc *h_descs = nullptr;    // pinned, one block per ring entry
    int32_t *h_status = nullptr;      // pinned, one per slot
    cudaEvent_t ev[kMaxStepsInFlight]{};
    long step_no = 0;
    uint8_t *whole_ws = nullptr;      // wavefront workspace for deep streams (used in order on `side`)
    size_t whole_cap = 0;
    cudaStream_t side = nullptr;      // whole decodes of deep streams
    cudaEvent_t admitted = nullptr;   // side waits for the admission work (allocation, state) on the step stream
    std::vector<cudaEvent_t> slot_ev; // per slot: completion of a whole decode (created on first use)
};

namespace {

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

bool event_done(aceapex_server *S, const Req &r) {
    if (r.whole && r.info.decoded_len > 0) return cudaEventQuery(S->slot_ev[r.slot]) == cudaSuccess;
    const long step = r.done_step;
    if (step < 0) return false;
    // the ring entry of step k is waited for at the start of step k + kMaxStepsInFlight
    if (step + kMaxStepsInFlight < S->step_no) return true;
    return cudaEventQuery(S->ev[step % kMaxStepsInFlight]) == cudaSuccess;
}

}  // namespace

extern "C" {

int aceapex_server_create(size_t hbm_budget, int max_slots, uint64_t tiles_per_step, aceapex_server **out) {
    if (!out || max_slots < 1 || max_slots > 65536 || tiles_per_step < 1) return kErrArg;
    aceapex_server *S = new (std::nothrow) aceapex_server();
    if (!S) return kErrNomem;
    S->budget = hbm_budget;
    S->max_slots = max_slots;
    S->tiles_per_step = tiles_per_step;
    S->slot_owner.assign(max_slots, -1);
    S->flags_cap = tiles_per_step + (uint64_t)max_slots;  // slices are rounded up to at least one tile
    S->ws_stride = up256(sizeof(WsHead)) + up256(sizeof(StreamState) * 2) + up256(4 * S->flags_cap) +
                   up256(sizeof(StreamDesc) * (size_t)max_slots) + up256(4 * (size_t)max_slots);
    bool ok = cudaMalloc((void **)&S->d_state, sizeof(StreamState) * max_slots) == cudaSuccess &&
              cudaMalloc((void **)&S->d_ws, S->ws_stride * kMaxStepsInFlight) == cudaSuccess &&
              cudaMallocHost((void **)&S->h_descs, sizeof(StreamDesc) * max_slots * kMaxStepsInFlight) == cudaSuccess &&
              cudaMallocHost((void **)&S->h_status, sizeof(int32_t) * max_slots) == cudaSuccess &&
              cudaMemset(S->d_ws, 0, S->ws_stride * kMaxStepsInFlight) == cudaSuccess;
    for (int k = 0; ok && k < kMaxStepsInFlight; k++)
        ok = cudaEventCreateWithFlags(&S->ev[k], kEvFlags) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&S->side, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&S->admitted, kEvFlags) == cudaSuccess;
    if (ok) S->slot_ev.assign(max_slots, nullptr);
    if (!ok) {
        cudaGetLastError();
        for (int k = 0; k < kMaxStepsInFlight; k++) if (S->ev[k]) cudaEventDestroy(S->ev[k]);
        if (S->admitted) cudaEventDestroy(S->admitted);
        if (S->side) cudaStreamDestroy(S->side);
        cudaFree(S->d_state); cudaFree(S->d_ws); cudaFreeHost(S->h_descs); cudaFreeHost(S->h_status);
        delete S;
        return kErrNomem;
    }
    *out = S;
    return kOK;
}

int aceapex_server_destroy(aceapex_server *S) {
    if (!S) return kErrArg;
    cudaDeviceSynchronize();
    for (auto &r : S->reqs) if (r.out && r.phase != 3) cudaFree(r.out);
    for (int k = 0; k < kMaxStepsInFlight; k++) if (S->ev[k]) cudaEventDestroy(S->ev[k]);
    for (cudaEvent_t e : S->slot_ev) if (e) cudaEventDestroy(e);
    if (S->admitted) cudaEventDestroy(S->admitted);
    if (S->side) cudaStreamDestroy(S->side);
    cudaFree(S->d_state); cudaFree(S->d_ws); cudaFree(S->whole_ws);
    cudaFreeHost(S->h_descs); cudaFreeHost(S->h_status);
    delete S;
    return kOK;
}

int64_t aceapex_server_submit(aceapex_server *S, const void *comp, size_t comp_len, const aceapex_info *info) {
    if (!S || !comp || !info || ((uintptr_t)comp & 15) || info->comp_len != comp_len) return kErrArg;
    std::lock_guard<std::mutex> g(S->mu);
    Req r;
    r.comp = comp;
    r.comp_len = comp_len;
    r.info = *info;
    const uint64_t N = info->decoded_len;
    r.whole = !aceapex_host::one_pass_stream(*info);
    r.out_alloc = r.whole ? (N ? N : 1) : align16(N) + 4 * litmap_words(N);
    r.bytes = comp_len + r.out_alloc;
    if (r.bytes > S->budget) return kErrNomem;
    S->reqs.push_back(r);
    const int64_t id = (int64_t)S->reqs.size() - 1;
    S->queue.push_back(id);
    return id;
}

int aceapex_server_step(aceapex_server *S, void *stream_) {
    if (!S) return kErrArg;
    cudaStream_t stream = (cudaStream_t)stream_;
    std::lock_guard<std::mutex> g(S->mu);
    // ring entry of this step: wait for the step that used it before
    const int ring = (int)(S->step_no % kMaxStepsInFlight);
    if (S->step_no >= kMaxStepsInFlight && cudaEventSynchronize(S->ev[ring]) != cudaSuccess) return kErrCuda;
    // 1. admission: arrival order, budget and slots.  A request is admitted only once its first work is
    //    enqueued; if that fails it goes back to the head of the queue holding nothing, and step returns
    //    the error (a later step retries it).
    while (!S->queue.empty()) {
        const int64_t id = S->queue.front();
        Req &r = S->reqs[id];
        int slot = -1;
        for (int k = 0; k < S->max_slots; k++) if (S->slot_owner[k] < 0) { slot = k; break; }
        if (slot < 0 || S->used + r.bytes > S->budget) break;
        if (cudaMallocAsync(&r.out, r.out_alloc, stream) != cudaSuccess) {
            cudaGetLastError();
            r.out = nullptr;
            break;  // retry in a later step
        }
        r.litmap = r.whole ? nullptr : (uint32_t *)((uint8_t *)r.out + align16(r.info.decoded_len));
        auto undo = [&](int rc) {
            if (r.whole) cudaStreamSynchronize(S->side);  // nothing of a failed whole decode may still run
            cudaFreeAsync(r.out, stream);
            cudaGetLastError();
            r.out = nullptr;
            r.litmap = nullptr;
            return rc;
        };
        if (aceapex_host::init_state(&S->d_state[slot], stream)) return undo(kErrCuda);
        if (r.info.decoded_len > 0 && r.whole) {
            // deep stream (or one the one-pass kernel does not take): decoded whole on the side stream, after
            // the admission work above; its status is left in the shared workspace's state and copied out
            // before the next whole decode can reuse the workspace (same stream)
            if (!S->slot_ev[slot] && cudaEventCreateWithFlags(&S->slot_ev[slot], kEvFlags) != cudaSuccess) {
                S->slot_ev[slot] = nullptr;
                return undo(kErrCuda);
            }
            if (cudaEventRecord(S->admitted, stream) != cudaSuccess ||
                cudaStreamWaitEvent(S->side, S->admitted, 0) != cudaSuccess)
                return undo(kErrCuda);
            const int rc = aceapex_host::server_enqueue_whole(r.comp, r.out, r.info, &S->whole_ws, &S->whole_cap,
                                                              nullptr, S->side);
            if (rc) return undo(rc);
            if (cudaMemcpyAsync(&S->h_status[slot], S->whole_ws + up256(sizeof(WsHead)) + offsetof(StreamState, status),
                                4, cudaMemcpyDeviceToHost, S->side) != cudaSuccess ||
                cudaEventRecord(S->slot_ev[slot], S->side) != cudaSuccess)
                return undo(kErrCuda);
        }
        S->queue.pop_front();
        S->used += r.bytes;
        r.slot = slot;
        r.phase = 1;
        S->slot_owner[slot] = id;
        if (r.info.decoded_len == 0) {
            S->h_status[slot] = 0;
            r.phase = 2;
            r.done_step = S->step_no;
        } else if (r.whole) {
            r.phase = 2;
            r.done_step = S->step_no;
            r.next_tile = r.info.n_tiles;
        }
    }
    // 2. slices: every admitted request with tiles left gets a share of the step's tile budget
    std::vector<int64_t> act;
    for (int k = 0; k < S->max_slots; k++) {
        const int64_t id = S->slot_owner[k];
        if (id >= 0 && S->reqs[id].phase == 1 && !S->reqs[id].whole) act.push_back(id);
    }
    std::sort(act.begin(), act.end());
    StreamDesc *hd = S->h_descs + (size_t)ring * S->max_slots;
    uint8_t *ws = S->d_ws + (size_t)ring * S->ws_stride;
    WsHead *head = (WsHead *)ws;
    StreamState *sst = (StreamState *)(ws + up256(sizeof(WsHead)));
    uint32_t *flags = (uint32_t *)(ws + up256(sizeof(WsHead)) + up256(sizeof(StreamState) * 2));
    StreamDesc *dd = (StreamDesc *)((uint8_t *)flags + up256(4 * S->flags_cap));
    int32_t *d_out_status = (int32_t *)((uint8_t *)dd + up256(sizeof(StreamDesc) * (size_t)S->max_slots));
    uint64_t total = 0;
    int nd = 0;
    uint32_t max_tl = 0;
    std::vector<int64_t> finishing;
    if (!act.empty()) {
        const uint64_t quota = std::max<uint64_t>(1, S->tiles_per_step / act.size());
        for (int64_t id : act) {
            Req &r = S->reqs[id];
            const uint64_t left = r.info.n_tiles - r.next_tile;
            const uint64_t take = std::min(left, quota);
            StreamDesc d{};
            d.comp = (const uint8_t *)r.comp; d.out = (uint8_t *)r.out; d.comp_len = r.info.comp_len;
            d.N = r.info.decoded_len; d.n_blocks = r.info.n_blocks; d.n_seq = r.info.n_seq; d.n_match = r.info.n_match;
            d.tile_base = total; d.n_tiles = take; d.tile_off = r.next_tile; d.state = &S->d_state[r.slot];
            d.litmap = r.litmap;
            d.block_log2 = r.info.block_log2; d.tile_log2 = r.info.tile_log2; d.min_match = r.info.min_match;
            d.max_depth = r.info.max_depth;
            d.flags = (r.next_tile + take == r.info.n_tiles) ? kDescLast : 0u;
            hd[nd++] = d;
            total += take;
            max_tl = std::max(max_tl, r.info.tile_log2);
            r.next_tile += take;
            if (d.flags & kDescLast) finishing.push_back(id);
        }
        if (cudaMemcpyAsync(dd, hd, sizeof(StreamDesc) * nd, cudaMemcpyHostToDevice, stream) != cudaSuccess)
            return kErrCuda;
        LaunchCfg cfg = aceapex_host::launch_cfg();
        cfg.num_sms = aceapex_host::num_sms();
        LaunchArgs a{};
        a.n_streams = nd;
        a.total_tiles = total;
        a.wait_ns = 4000000000ull;
        a.withhold = ~0ull;
        a.max_tile_log2 = max_tl;
        for (int k = 0; k < nd; k++) a.max_n = std::max<unsigned long long>(a.max_n, hd[k].N);
        if (nd == 1) a.one = hd[0];
        // launch_flat reads descs[] (device) when n_streams > 1, and a.one otherwise
        cudaError_t e = launch_flat(cfg, head, sst, flags, nd > 1 ? dd : nullptr, a, d_out_status, stream);
        if (e != cudaSuccess) { cudaGetLastError(); return kErrCuda; }
        for (int64_t id : finishing) {
            Req &r = S->reqs[id];
            r.phase = 2;
            r.done_step = S->step_no;
            if (cudaMemcpyAsync(&S->h_status[r.slot], &S->d_state[r.slot].status, 4, cudaMemcpyDeviceToHost, stream) !=
                cudaSuccess)
                return kErrCuda;
        }
    }
    if (cudaEventRecord(S->ev[ring], stream) != cudaSuccess) return kErrCuda;
    S->step_no++;
    int pending = (int)S->queue.size();
    for (int k = 0; k < S->max_slots; k++) if (S->slot_owner[k] >= 0 && S->reqs[S->slot_owner[k]].phase == 1) pending++;
    return pending;
}

int aceapex_server_poll(aceapex_server *S, int64_t id, int32_t *status, void **out) {
    if (!S) return kErrArg;
    std::lock_guard<std::mutex> g(S->mu);
    if (id < 0 || id >= (int64_t)S->reqs.size()) return kErrArg;
    Req &r = S->reqs[id];
    if (r.phase != 2 || !event_done(S, r)) return 0;
    if (status) *status = S->h_status[r.slot];
    if (out) *out = r.out;
    return 1;
}

int aceapex_server_release(aceapex_server *S, int64_t id, void *stream_) {
    if (!S) return kErrArg;
    std::lock_guard<std::mutex> g(S->mu);
    if (id < 0 || id >= (int64_t)S->reqs.size()) return kErrArg;
    Req &r = S->reqs[id];
    if (r.phase != 2) return kErrArg;
    // a whole decode runs on the side stream: the free waits for it (stream-ordered)
    if (r.whole && r.info.decoded_len > 0 && cudaStreamWaitEvent((cudaStream_t)stream_, S->slot_ev[r.slot], 0) != cudaSuccess)
        return kErrCuda;
    cudaFreeAsync(r.out, (cudaStream_t)stream_);
    r.out = nullptr;
    r.litmap = nullptr;
    r.phase = 3;
    S->used -= r.bytes;
    S->slot_owner[r.slot] = -1;
    return kOK;
}

}  // extern "C"

