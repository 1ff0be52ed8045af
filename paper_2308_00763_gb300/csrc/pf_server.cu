// pf_server.cu -- the serving loop: continuous batching of many camera streams over the
// per-frame step kernel (declared in include/pf.h, "serving").
//
// Layout.  One device arena (the HBM budget) is carved per stream by a first-fit
// allocator.  Per precision an engine holds the slot-indexed tracker descriptors and
// states, a CUDA stream, and a ring of launch records (pinned host + device arrays for
// one launch: the slot of every launch position, the tile prefix, the frame table and
// the estimates).  A tick gathers, per precision, every stream with a queued frame
// into one launch: the kernel finds each tile's launch position by bisection of the
// tile prefix and the stream's descriptor through its slot, so the batch is rebuilt at
// every tick without touching the streams' device state.  A host callback enqueued
// after each launch records its completion time; poll harvests completed launches.
#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <deque>
#include <map>
#include <new>
#include <thread>
#include <vector>

#include "pf.h"
#include "pf_host.h"
#include "pf_internal.h"

using namespace pfk;

namespace {

double now_s() {
    using clk = std::chrono::steady_clock;
    return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator over [0, size) in kAlign units; free ranges coalesce.
class Arena {
public:
    void reset(size_t size) { free_.clear(); if (size) free_[0] = size; in_use_ = 0; peak_ = 0; }
    bool take(size_t bytes, size_t *off) {
        bytes = align_up(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                in_use_ += bytes;
                peak_ = std::max(peak_, in_use_);
                return true;
            }
        }
        return false;
    }
    void give(size_t off, size_t bytes) {
        bytes = align_up(bytes);
        in_use_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) { it->second += nx->second; free_.erase(nx); }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) { pv->second += it->second; free_.erase(it); }
        }
    }
    size_t in_use() const { return in_use_; }
    size_t peak() const { return peak_; }

private:
    std::map<size_t, size_t> free_;
    size_t in_use_ = 0, peak_ = 0;
};

// Pieces of a stream's arena block (offsets from the block start).
struct StreamLayout {
    size_t px[2], py[2], pl[2], look, part, gtab, done, est, stat, ring, total;
    int64_t ring_pitch;
    int ntiles, tile;
};

StreamLayout stream_layout(const pf_config &c, bool host_frames, int queue_depth) {
    StreamLayout L{};
    const size_t pb = pos_bytes(c.precision);
    const int64_t N = c.num_particles;
    L.tile = step_tile_size(c.precision, N);
    L.ntiles = static_cast<int>((N + L.tile - 1) / L.tile);
    size_t o = 0;
    auto take = [&](size_t b) { const size_t at = o; o = align_up(o + b); return at; };
    for (int s = 0; s < 2; ++s) {
        L.px[s] = take(N * pb + 16);
        L.py[s] = take(N * pb + 16);
        L.pl[s] = take(N * pb + 16);
    }
    L.look = take(sizeof(LookbackDesc) * L.ntiles);
    L.part = take(sizeof(TilePartial) * L.ntiles);
    // the stream's likelihood table (streams of two or more tiles; cleared with the
    // descriptors when a stream opens, so no tag of an earlier stream in the slot survives)
    L.gtab = L.ntiles >= 2 ? take(sizeof(uint64_t) * kTableMax) : SIZE_MAX;
    L.done = take(sizeof(uint32_t));
    L.est = take(sizeof(double) * 2 * 2);
    L.stat = take(sizeof(double) * 2 * 2);
    L.ring_pitch = (c.width + 15) & ~int64_t(15);
    L.ring = host_frames ? take(static_cast<size_t>(L.ring_pitch) * c.height * queue_depth) : o;
    L.total = o;
    return L;
}

struct Pending {
    int64_t index;
    double arrival;
    const uint8_t *frame;
    int64_t pitch;
    int ring_slot;      // -1: device frame read in place
};

struct Stream {
    bool open = false;
    pf_config cfg{};
    double fps = 0;
    int slot = -1;
    size_t off = 0;
    StreamLayout lay{};
    bool host_frames = false;
    std::deque<Pending> queued;
    int in_flight = 0;
    int64_t submitted = 0, done = 0;
    std::vector<double> res;          // 2 * rcap estimates, frame i at i % rcap
    std::vector<int64_t> res_index;   // which frame each ring entry holds (-1 none)
    std::vector<uint8_t> ring_busy;   // host-frame queue slots in use
    std::vector<cudaEvent_t> ring_ev; // completion of the copy into each queue slot
};

struct LaunchItem {
    int stream;
    int64_t index;
    double arrival;
    int ring_slot;
};

struct LaunchRec {
    int32_t *h_pos = nullptr, *d_pos = nullptr;         // slot_of[cap] then tile_prefix[cap + 1]
    FrameRef *h_frames = nullptr, *d_frames = nullptr;
    double *h_est = nullptr, *d_est = nullptr;
    std::vector<LaunchItem> items;
    std::atomic<int> finished{0};
    double t_done = 0;
    bool busy = false;
};


struct Engine {
    int prec = -1;
    cudaStream_t stream = nullptr;
    TrackerDev *d_trk = nullptr;
    TrackerState *d_states = nullptr;
    uint32_t *d_ticket = nullptr;
    std::vector<LaunchRec *> recs;
    int next = 0;
    std::vector<int> free_slots;
};

void CUDART_CB launch_done(void *p) {
    LaunchRec *r = static_cast<LaunchRec *>(p);
    r->t_done = now_s();
    r->finished.store(1, std::memory_order_release);
}

}  // namespace

struct pf_server {
    pf_server_config cfg{};
    unsigned char *d_arena = nullptr;
    Arena arena;
    std::vector<Stream> streams;
    Engine eng[4];
    cudaStream_t copy_stream = nullptr;
    double demand = 0;
    pf_status sticky = PF_OK;
    // statistics
    int64_t admitted = 0, rejected = 0, frames_submitted = 0, frames_rejected = 0, frames_done = 0, launches = 0;
    double psteps = 0, first_launch = -1, last_done = -1;
    std::vector<float> latency_ms;

    pf_status fail(pf_status s) { if (sticky == PF_OK) sticky = s; return s; }
};

namespace {

pf_status engine_init(pf_server *S, int prec) {
    Engine &e = S->eng[prec];
    if (e.prec >= 0) return PF_OK;
    const int cap = S->cfg.max_streams;
    cudaError_t err = cudaStreamCreateWithFlags(&e.stream, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaMalloc(reinterpret_cast<void **>(&e.d_trk), sizeof(TrackerDev) * cap);
    if (err == cudaSuccess) err = cudaMalloc(reinterpret_cast<void **>(&e.d_states), sizeof(TrackerState) * cap);
    if (err == cudaSuccess) err = cudaMalloc(reinterpret_cast<void **>(&e.d_ticket), sizeof(uint32_t));
    if (err == cudaSuccess) err = cudaMemsetAsync(e.d_ticket, 0, sizeof(uint32_t), e.stream);
    for (int k = 0; err == cudaSuccess && k < S->cfg.max_in_flight; ++k) {
        LaunchRec *r = new (std::nothrow) LaunchRec();
        if (!r) { err = cudaErrorMemoryAllocation; break; }
        e.recs.push_back(r);
        err = cudaMallocHost(reinterpret_cast<void **>(&r->h_pos), sizeof(int32_t) * (2 * cap + 1));
        if (err == cudaSuccess) err = cudaMalloc(reinterpret_cast<void **>(&r->d_pos), sizeof(int32_t) * (2 * cap + 1));
        if (err == cudaSuccess) err = cudaMallocHost(reinterpret_cast<void **>(&r->h_frames), sizeof(FrameRef) * cap);
        if (err == cudaSuccess) err = cudaMalloc(reinterpret_cast<void **>(&r->d_frames), sizeof(FrameRef) * cap);
        if (err == cudaSuccess) err = cudaMallocHost(reinterpret_cast<void **>(&r->h_est), sizeof(double) * 2 * cap);
        if (err == cudaSuccess) err = cudaMalloc(reinterpret_cast<void **>(&r->d_est), sizeof(double) * 2 * cap);
    }
    if (err != cudaSuccess) {
        cudaGetLastError();
        return err == cudaErrorMemoryAllocation ? PF_ERR_OOM : PF_ERR_CUDA;
    }
    e.free_slots.clear();
    for (int k = cap - 1; k >= 0; --k) e.free_slots.push_back(k);
    e.prec = prec;
    return PF_OK;
}

void engine_free(Engine &e) {
    if (e.stream) cudaStreamSynchronize(e.stream);
    for (LaunchRec *r : e.recs) {
        cudaFreeHost(r->h_pos); cudaFree(r->d_pos);
        cudaFreeHost(r->h_frames); cudaFree(r->d_frames);
        cudaFreeHost(r->h_est); cudaFree(r->d_est);
        delete r;
    }
    e.recs.clear();
    cudaFree(e.d_trk); cudaFree(e.d_states); cudaFree(e.d_ticket);
    if (e.stream) cudaStreamDestroy(e.stream);
    e = Engine();
}

// Harvest the completed launch records of every engine (in launch order per engine).
int harvest(pf_server *S, bool *timeout) {
    int n = 0;
    for (Engine &e : S->eng) {
        if (e.prec < 0) continue;
        const int k = static_cast<int>(e.recs.size());
        for (int i = 0; i < k; ++i) {
            LaunchRec *r = e.recs[(e.next + i) % k];   // oldest first
            if (!r->busy || !r->finished.load(std::memory_order_acquire)) continue;
            for (size_t p = 0; p < r->items.size(); ++p) {
                const LaunchItem &it = r->items[p];
                Stream &st = S->streams[it.stream];
                const int rc = static_cast<int>(st.res_index.size());
                const int at = static_cast<int>(it.index % rc);
                st.res[2 * at] = r->h_est[2 * p];
                st.res[2 * at + 1] = r->h_est[2 * p + 1];
                st.res_index[at] = it.index;
                st.done = std::max(st.done, it.index + 1);
                st.in_flight--;
                if (it.ring_slot >= 0) st.ring_busy[it.ring_slot] = 0;
                S->latency_ms.push_back(static_cast<float>(1e3 * (r->t_done - it.arrival)));
                S->psteps += static_cast<double>(st.cfg.num_particles);
                S->frames_done++;
                ++n;
            }
            S->last_done = std::max(S->last_done, r->t_done);
            r->items.clear();
            r->busy = false;
            r->finished.store(0, std::memory_order_relaxed);
        }
        // a failed step raises the tracker's timeout bit; checked on the states of this engine
        (void)timeout;
    }
    return n;
}

pf_status launch_engine(pf_server *S, Engine &e, int *launched) {
    *launched = 0;
    LaunchRec *r = e.recs[e.next];
    if (r->busy) return PF_OK;   // every record in flight: wait for a completion
    const int cap = S->cfg.max_streams;
    int n = 0, tiles = 0;
    cudaError_t err = cudaSuccess;
    for (int sid = 0; sid < static_cast<int>(S->streams.size()) && n < cap; ++sid) {
        Stream &st = S->streams[sid];
        if (!st.open || st.cfg.precision != e.prec || st.queued.empty()) continue;
        const Pending pd = st.queued.front();
        st.queued.pop_front();
        r->h_pos[n] = st.slot;
        r->h_pos[cap + n] = tiles;
        FrameRef fr;
        memset(&fr, 0, sizeof fr);
        fr.base = pd.frame;
        fr.pitch = pd.pitch;
        fr.stride = 0;
        fr.active = 1;
        r->h_frames[n] = fr;
        if (pd.ring_slot >= 0 && err == cudaSuccess) err = cudaStreamWaitEvent(e.stream, st.ring_ev[pd.ring_slot], 0);
        r->items.push_back(LaunchItem{sid, pd.index, pd.arrival, pd.ring_slot});
        st.in_flight++;
        tiles += st.lay.ntiles;
        ++n;
    }
    if (n == 0) return PF_OK;
    r->h_pos[cap + n] = tiles;
    // slot_of at d_pos[0..n), tile prefix at d_pos[cap .. cap + n]
    if (err == cudaSuccess) err = cudaMemcpyAsync(r->d_pos, r->h_pos, sizeof(int32_t) * n, cudaMemcpyHostToDevice, e.stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(r->d_pos + cap, r->h_pos + cap, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, e.stream);
    if (err == cudaSuccess) err = cudaMemcpyAsync(r->d_frames, r->h_frames, sizeof(FrameRef) * n, cudaMemcpyHostToDevice, e.stream);
    if (err != cudaSuccess) { cudaGetLastError(); return S->fail(PF_ERR_CUDA); }
    StepLaunch L;
    L.trk = e.d_trk;
    L.states = e.d_states;
    L.frames = r->d_frames;
    L.tile_trk = nullptr;
    L.tile_prefix = r->d_pos + cap;
    L.slot_of = r->d_pos;
    L.est_out = r->d_est;
    L.ticket = e.d_ticket;
    L.ntrk = n;
    L.total_tiles = tiles;
    L.frame_override = nullptr;
    L.pitch_override = 0;
    const int grid = step_grid_size(e.prec, tiles);
    if (grid < 1 || launch_step(e.prec, L, grid, e.stream) != 0) { cudaGetLastError(); return S->fail(PF_ERR_CUDA); }
    err = cudaMemcpyAsync(r->h_est, r->d_est, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, e.stream);
    if (err == cudaSuccess) err = cudaLaunchHostFunc(e.stream, launch_done, r);
    if (err != cudaSuccess) { cudaGetLastError(); return S->fail(PF_ERR_CUDA); }
    r->busy = true;
    e.next = (e.next + 1) % static_cast<int>(e.recs.size());
    S->launches++;
    if (S->first_launch < 0) S->first_launch = now_s();
    *launched = n;
    return PF_OK;
}

// A step that gave up (bounded wait) marks its tracker; the server fails with TIMEOUT.
pf_status check_status(pf_server *S) {
    for (Engine &e : S->eng) {
        if (e.prec < 0) continue;
        for (const Stream &st : S->streams) {
            if (!st.open || st.cfg.precision != e.prec) continue;
            uint32_t status = 0;
            if (cudaMemcpy(&status, &e.d_states[st.slot].status, sizeof status, cudaMemcpyDeviceToHost) != cudaSuccess) {
                cudaGetLastError();
                return S->fail(PF_ERR_CUDA);
            }
            if (status & kStatusTimeout) return S->fail(PF_ERR_TIMEOUT);
            if (status & kStatusBounds) return S->fail(PF_ERR_STATE);   // checked builds
        }
    }
    return PF_OK;
}

}  // namespace

extern "C" {

double pf_server_now(void) { return now_s(); }

pf_status pf_server_stream_bytes(const pf_config *cfg, int32_t host_frames, int32_t queue_depth, int64_t *bytes) {
    if (!bytes || check_config(cfg) != PF_OK || queue_depth < 1 ||
        cfg->resampler == PF_RESAMPLE_MULTINOMIAL || ancestors_given(cfg->resampler)) return PF_ERR_ARG;
    *bytes = static_cast<int64_t>(align_up(stream_layout(*cfg, host_frames != 0, queue_depth).total));
    return PF_OK;
}

pf_status pf_server_create(const pf_server_config *cfg, pf_server **out) {
    if (!cfg || !out) return PF_ERR_ARG;
    *out = nullptr;
    pf_server_config c = *cfg;
    if (c.hbm_budget_bytes <= 0 || c.max_streams < 1 || c.queue_depth < 1 || c.reserved != 0) return PF_ERR_ARG;
    if (!(c.capacity >= 0) || !(c.headroom >= 0) || c.headroom > 1.0) return PF_ERR_ARG;
    if (c.max_in_flight < 0 || c.max_in_flight > 8) return PF_ERR_ARG;
    if (c.headroom == 0) c.headroom = 1.0;
    if (c.max_in_flight == 0) c.max_in_flight = 2;
    pf_server *S = new (std::nothrow) pf_server();
    if (!S) return PF_ERR_OOM;
    S->cfg = c;
    cudaError_t err = cudaMalloc(reinterpret_cast<void **>(&S->d_arena), static_cast<size_t>(c.hbm_budget_bytes));
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&S->copy_stream, cudaStreamNonBlocking);
    if (err != cudaSuccess) {
        cudaGetLastError();
        if (S->d_arena) cudaFree(S->d_arena);
        delete S;
        return err == cudaErrorMemoryAllocation ? PF_ERR_OOM : PF_ERR_CUDA;
    }
    S->arena.reset(static_cast<size_t>(c.hbm_budget_bytes));
    S->streams.resize(c.max_streams);
    *out = S;
    return PF_OK;
}

pf_status pf_server_open(pf_server *S, const pf_config *cfg, double fps, int32_t host_frames, int32_t *stream_id) {
    if (!S || !stream_id || check_config(cfg) != PF_OK || !(fps >= 0) || !isfinite(fps)) return PF_ERR_ARG;
    if (cfg->flags & PF_FLAG_DEBUG_ARRAYS) return PF_ERR_ARG;
    // one launch per tick: no pull kernel (multinomial, Gumbel-max, Metropolis, rejection)
    if (cfg->resampler == PF_RESAMPLE_MULTINOMIAL || ancestors_given(cfg->resampler)) return PF_ERR_ARG;
    if (S->sticky != PF_OK) return PF_ERR_STATE;
    *stream_id = -1;
    const pf_config &c = *cfg;
    int sid = -1;
    for (int i = 0; i < static_cast<int>(S->streams.size()); ++i)
        if (!S->streams[i].open) { sid = i; break; }
    const double add = static_cast<double>(c.num_particles) * fps;
    if (sid < 0 || (S->cfg.capacity > 0 && S->demand + add > S->cfg.headroom * S->cfg.capacity)) {
        S->rejected++;
        return PF_ERR_ADMISSION;
    }
    const StreamLayout lay = stream_layout(c, host_frames != 0, S->cfg.queue_depth);
    size_t off = 0;
    if (!S->arena.take(lay.total, &off)) { S->rejected++; return PF_ERR_ADMISSION; }
    pf_status ps = engine_init(S, c.precision);
    if (ps != PF_OK) { S->arena.give(off, lay.total); return ps; }
    Engine &e = S->eng[c.precision];
    const int slot = e.free_slots.back();
    Stream &st = S->streams[sid];
    st = Stream();
    st.cfg = c;
    st.fps = fps;
    st.slot = slot;
    st.off = off;
    st.lay = lay;
    st.host_frames = host_frames != 0;
    const int rcap = c.est_capacity > 0 ? c.est_capacity : 64;
    st.res.assign(2 * rcap, 0.0);
    st.res_index.assign(rcap, -1);
    cudaError_t err = cudaSuccess;
    if (st.host_frames) {
        st.ring_busy.assign(S->cfg.queue_depth, 0);
        st.ring_ev.assign(S->cfg.queue_depth, nullptr);
        for (auto &ev : st.ring_ev)
            if (err == cudaSuccess) err = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    }
    // descriptor and initial state of the slot; cleared lookback descriptors and partials
    unsigned char *base = S->d_arena + off;
    TrackerDev T;
    memset(&T, 0, sizeof T);
    fill_tracker_constants(c, T);
    T.tile_begin = 0;
    T.tile = lay.tile;
    T.ntiles = lay.ntiles;
    T.est_cap = 2;
    for (int s2 = 0; s2 < 2; ++s2) {
        T.px[s2] = base + lay.px[s2];
        T.py[s2] = base + lay.py[s2];
        T.pl[s2] = base + lay.pl[s2];
    }
    T.look = reinterpret_cast<LookbackDesc *>(base + lay.look);
    T.part = reinterpret_cast<TilePartial *>(base + lay.part);
    T.done = reinterpret_cast<uint32_t *>(base + lay.done);
    T.gtab = lay.gtab == SIZE_MAX ? nullptr : reinterpret_cast<uint64_t *>(base + lay.gtab);
    T.state = e.d_states + slot;
    T.est_ring = reinterpret_cast<double *>(base + lay.est);
    T.stat_ring = reinterpret_cast<double *>(base + lay.stat);
    const TrackerState s0 = initial_state(c);
    // the slot may have served a stream of this engine whose launches are still queued
    if (err == cudaSuccess) err = cudaStreamSynchronize(e.stream);
    if (err == cudaSuccess) err = cudaMemset(base + lay.look, 0, lay.done + sizeof(uint32_t) - lay.look);
    if (err == cudaSuccess) err = cudaMemcpy(e.d_trk + slot, &T, sizeof T, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(e.d_states + slot, &s0, sizeof s0, cudaMemcpyHostToDevice);
    if (err != cudaSuccess) {
        cudaGetLastError();
        for (auto ev : st.ring_ev) if (ev) cudaEventDestroy(ev);
        st = Stream();
        S->arena.give(off, lay.total);
        return S->fail(PF_ERR_CUDA);
    }
    e.free_slots.pop_back();
    st.open = true;
    S->demand += add;
    S->admitted++;
    *stream_id = sid;
    return PF_OK;
}

pf_status pf_server_submit(pf_server *S, int32_t sid, const uint8_t *frame, int64_t pitch, int32_t on_device,
                           double arrival) {
    if (!S || !frame) return PF_ERR_ARG;
    if (S->sticky != PF_OK) return PF_ERR_STATE;
    if (sid < 0 || sid >= static_cast<int>(S->streams.size()) || !S->streams[sid].open) return PF_ERR_STATE;
    Stream &st = S->streams[sid];
    if (pitch < st.cfg.width) return PF_ERR_ARG;
    if (!on_device && !st.host_frames) return PF_ERR_ARG;
    if (arrival < 0) arrival = now_s();
    S->frames_submitted++;
    if (static_cast<int>(st.queued.size()) + st.in_flight >= S->cfg.queue_depth) {
        S->frames_rejected++;
        return PF_ERR_ADMISSION;
    }
    Pending pd{st.submitted, arrival, frame, pitch, -1};
    if (!on_device) {
        int k = -1;
        for (int i = 0; i < static_cast<int>(st.ring_busy.size()); ++i)
            if (!st.ring_busy[i]) { k = i; break; }
        if (k < 0) { S->frames_rejected++; return PF_ERR_ADMISSION; }
        unsigned char *dst = S->d_arena + st.off + st.lay.ring + static_cast<size_t>(k) * st.lay.ring_pitch * st.cfg.height;
        cudaError_t err = cudaMemcpy2DAsync(dst, st.lay.ring_pitch, frame, pitch, st.cfg.width, st.cfg.height,
                                            cudaMemcpyHostToDevice, S->copy_stream);
        if (err == cudaSuccess) err = cudaEventRecord(st.ring_ev[k], S->copy_stream);
        if (err != cudaSuccess) { cudaGetLastError(); return S->fail(PF_ERR_CUDA); }
        st.ring_busy[k] = 1;
        pd.frame = dst;
        pd.pitch = st.lay.ring_pitch;
        pd.ring_slot = k;
    }
    st.queued.push_back(pd);
    st.submitted++;
    return PF_OK;
}

pf_status pf_server_poll(pf_server *S, int32_t *completed) {
    if (!S) return PF_ERR_ARG;
    bool to = false;
    const int n = harvest(S, &to);
    if (completed) *completed = n;
    return S->sticky;
}

pf_status pf_server_tick(pf_server *S, int32_t *launched) {
    TraceRange trace("pf_server_tick");
    if (!S) return PF_ERR_ARG;
    if (launched) *launched = 0;
    if (S->sticky != PF_OK) return PF_ERR_STATE;
    harvest(S, nullptr);
    int total = 0;
    for (Engine &e : S->eng) {
        if (e.prec < 0) continue;
        int n = 0;
        const pf_status ps = launch_engine(S, e, &n);
        if (ps != PF_OK) return ps;
        total += n;
    }
    if (launched) *launched = total;
    return PF_OK;
}

pf_status pf_server_drain(pf_server *S) {
    if (!S) return PF_ERR_ARG;
    for (;;) {
        if (S->sticky != PF_OK) return S->sticky;
        bool pending = false;
        for (const Stream &st : S->streams)
            if (st.open && (!st.queued.empty() || st.in_flight > 0)) { pending = true; break; }
        if (!pending) break;
        int32_t n = 0;
        pf_status ps = pf_server_tick(S, &n);
        if (ps != PF_OK) return ps;
        if (n == 0) {
            for (Engine &e : S->eng)
                if (e.prec >= 0 && cudaStreamSynchronize(e.stream) != cudaSuccess) { cudaGetLastError(); return S->fail(PF_ERR_CUDA); }
            harvest(S, nullptr);
        }
    }
    return check_status(S);
}

pf_status pf_server_result(pf_server *S, int32_t sid, int64_t index, double *x, double *y) {
    if (!S || !x || !y) return PF_ERR_ARG;
    if (sid < 0 || sid >= static_cast<int>(S->streams.size()) || !S->streams[sid].open) return PF_ERR_STATE;
    const Stream &st = S->streams[sid];
    if (index < 0) return PF_ERR_ARG;
    const int rc = static_cast<int>(st.res_index.size());
    const int at = static_cast<int>(index % rc);
    if (st.res_index[at] != index) return PF_ERR_STATE;
    *x = st.res[2 * at];
    *y = st.res[2 * at + 1];
    return PF_OK;
}

int64_t pf_server_frames_done(const pf_server *S, int32_t sid) {
    if (!S || sid < 0 || sid >= static_cast<int>(S->streams.size()) || !S->streams[sid].open) return -1;
    return S->streams[sid].done;
}

pf_status pf_server_close(pf_server *S, int32_t sid) {
    if (!S) return PF_ERR_ARG;
    if (sid < 0 || sid >= static_cast<int>(S->streams.size()) || !S->streams[sid].open) return PF_ERR_STATE;
    Stream &st = S->streams[sid];
    st.queued.clear();
    Engine &e = S->eng[st.cfg.precision];
    while (st.in_flight > 0) {
        if (cudaStreamSynchronize(e.stream) != cudaSuccess) { cudaGetLastError(); return S->fail(PF_ERR_CUDA); }
        harvest(S, nullptr);
    }
    if (st.host_frames && cudaStreamSynchronize(S->copy_stream) != cudaSuccess) { cudaGetLastError(); return S->fail(PF_ERR_CUDA); }
    for (auto ev : st.ring_ev) if (ev) cudaEventDestroy(ev);
    S->arena.give(st.off, st.lay.total);
    e.free_slots.push_back(st.slot);
    S->demand -= static_cast<double>(st.cfg.num_particles) * st.fps;
    if (S->demand < 0) S->demand = 0;
    st = Stream();
    return PF_OK;
}

pf_status pf_server_get_stats(pf_server *S, pf_server_stats *o) {
    if (!S || !o) return PF_ERR_ARG;
    memset(o, 0, sizeof *o);
    for (const Stream &st : S->streams) o->streams_open += st.open ? 1 : 0;
    o->streams_admitted = S->admitted;
    o->streams_rejected = S->rejected;
    o->frames_submitted = S->frames_submitted;
    o->frames_rejected = S->frames_rejected;
    o->frames_done = S->frames_done;
    o->launches = S->launches;
    o->particle_steps = S->psteps;
    if (!S->latency_ms.empty()) {
        std::vector<float> v(S->latency_ms);
        const size_t n = v.size();
        auto pct = [&](double q) {
            const size_t k = std::min(n - 1, static_cast<size_t>(ceil(q * static_cast<double>(n))) - (q > 0 ? 1 : 0));
            std::nth_element(v.begin(), v.begin() + static_cast<long>(k), v.end());
            return static_cast<double>(v[k]);
        };
        o->latency_p50_ms = pct(0.50);
        o->latency_p99_ms = pct(0.99);
        o->latency_max_ms = static_cast<double>(*std::max_element(v.begin(), v.end()));
    }
    o->first_launch_s = S->first_launch;
    o->last_done_s = S->last_done;
    o->hbm_in_use = static_cast<int64_t>(S->arena.in_use());
    o->hbm_peak = static_cast<int64_t>(S->arena.peak());
    o->demand = S->demand;
    return PF_OK;
}

pf_status pf_server_destroy(pf_server *S) {
    if (!S) return PF_OK;
    for (Engine &e : S->eng) if (e.stream) cudaStreamSynchronize(e.stream);
    if (S->copy_stream) cudaStreamSynchronize(S->copy_stream);
    harvest(S, nullptr);
    for (Stream &st : S->streams)
        for (auto ev : st.ring_ev) if (ev) cudaEventDestroy(ev);
    for (Engine &e : S->eng) engine_free(e);
    if (S->copy_stream) cudaStreamDestroy(S->copy_stream);
    cudaFree(S->d_arena);
    delete S;
    return PF_OK;
}

pf_status pf_server_replay(pf_server *S, const pf_trace_event *ev, int64_t n, int32_t n_streams, int32_t realtime) {
    TraceRange trace("pf_server_replay");
    if (!S || (n > 0 && !ev) || n < 0 || n_streams < 0) return PF_ERR_ARG;
    if (S->sticky != PF_OK) return PF_ERR_STATE;
    std::vector<int32_t> sid(n_streams, -2);   // -2 never opened, -1 refused / closed
    const double t0 = now_s();
    int64_t i = 0;
    for (;;) {
        const double now = now_s() - t0;
        int taken = 0;
        while (i < n && (realtime ? ev[i].time_s <= now : taken < 256)) {
            const pf_trace_event &e = ev[i++];
            ++taken;
            if (e.stream < 0 || e.stream >= n_streams) return PF_ERR_ARG;
            int32_t &id = sid[e.stream];
            if (e.kind == 0) {
                if (id >= 0) return PF_ERR_ARG;
                int32_t out = -1;
                const pf_status ps = pf_server_open(S, e.cfg, e.fps, 0, &out);
                if (ps == PF_OK) id = out;
                else if (ps == PF_ERR_ADMISSION) id = -1;
                else return ps;
            } else if (e.kind == 1) {
                const double arrival = realtime ? t0 + e.time_s : now_s();
                if (id < 0) { S->frames_submitted++; S->frames_rejected++; continue; }
                pf_status ps = pf_server_submit(S, id, e.frame, e.pitch_bytes, 1, arrival);
                // as fast as possible: a full queue waits for the stream's oldest frame
                while (!realtime && ps == PF_ERR_ADMISSION) {
                    S->frames_submitted--;
                    S->frames_rejected--;
                    Stream &st = S->streams[id];
                    int32_t launched = 0;
                    pf_status pt = pf_server_tick(S, &launched);
                    if (pt != PF_OK) return pt;
                    if (static_cast<int>(st.queued.size()) + st.in_flight >= S->cfg.queue_depth) {
                        if (cudaStreamSynchronize(S->eng[st.cfg.precision].stream) != cudaSuccess) {
                            cudaGetLastError();
                            return S->fail(PF_ERR_CUDA);
                        }
                        harvest(S, nullptr);
                    }
                    ps = pf_server_submit(S, id, e.frame, e.pitch_bytes, 1, arrival);
                }
                if (ps != PF_OK && ps != PF_ERR_ADMISSION) return ps;
            } else if (e.kind == 2) {
                if (id >= 0) {
                    // the stream's frames that arrived before it closed are still served
                    Stream &st = S->streams[id];
                    while (!st.queued.empty()) {
                        int32_t launched = 0;
                        pf_status pt = pf_server_tick(S, &launched);
                        if (pt != PF_OK) return pt;
                        if (!st.queued.empty() &&
                            cudaStreamSynchronize(S->eng[st.cfg.precision].stream) != cudaSuccess) {
                            cudaGetLastError();
                            return S->fail(PF_ERR_CUDA);
                        }
                    }
                    const pf_status ps = pf_server_close(S, id);
                    if (ps != PF_OK) return ps;
                }
                id = -1;
            } else {
                return PF_ERR_ARG;
            }
        }
        int32_t launched = 0;
        const pf_status ps = pf_server_tick(S, &launched);
        if (ps != PF_OK) return ps;
        bool pending = false;
        for (const Stream &st : S->streams)
            if (st.open && (!st.queued.empty() || st.in_flight > 0)) { pending = true; break; }
        if (i >= n && !pending) break;
        if (launched == 0) std::this_thread::yield();
    }
    return check_status(S);
}

}  // extern "C"
