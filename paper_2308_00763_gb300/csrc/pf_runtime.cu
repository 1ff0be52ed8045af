// pf_runtime.cu -- host runtime behind the C ABI of include/pf.h: handles, device
// buffers, frame staging, launches, estimates, checkpoints.
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>
#include <stdlib.h>
#include <stddef.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "pf.h"
#include "pf_internal.h"
#include "pf_host.h"

using namespace pfk;

namespace {

// ---------------------------------------------------------------- launch-shape cache
struct TuneKey {
    int prec, lg, sq, r, fb, sms;
    bool operator<(const TuneKey &o) const {
        if (prec != o.prec) return prec < o.prec;
        if (lg != o.lg) return lg < o.lg;
        if (sq != o.sq) return sq < o.sq;
        if (r != o.r) return r < o.r;
        if (fb != o.fb) return fb < o.fb;
        return sms < o.sms;
    }
};

std::mutex g_tune_lock;
std::map<TuneKey, pf_tuning> g_tune;

// shape bucket: precision, floor(log2 N), the larger sigma in quarter pixels, the disk
// radius, floor(log2 (W H)) and the current device's SM count
TuneKey tune_key(const pf_config &c) {
    int lg = 0;
    while (lg < 62 && (int64_t(1) << (lg + 1)) <= c.num_particles) ++lg;
    const double sg = std::max(c.sigma_x, c.sigma_y);
    const int sq = static_cast<int>(std::min(4.0 * sg + 0.5, 1.0e6));
    const int64_t px = static_cast<int64_t>(c.width) * c.height;
    int fb = 0;
    while (fb < 62 && (int64_t(1) << (fb + 1)) <= px) ++fb;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = 0;                           // no device (host-only use of the cache)
    }
    return TuneKey{c.precision, lg, sq, c.disk_radius, fb, sms};
}

bool valid_tuning(const pf_tuning &t) {
    return (t.tile == 0 || (t.tile % 8 == 0 && t.tile >= 1024 && t.tile <= kTile)) && t.window >= 0 &&
           t.window <= 2 && t.ctas_per_sm >= 0 && t.ctas_per_sm <= 32 && t.reserved == 0;
}

// the launch shape a tracker takes: forced, else its bucket's (PF_FLAG_TUNED), else default
pf_tuning tuning_for(const pf_config &c, const pf_tuning *force) {
    if (force) return *force;
    pf_tuning t{0, 0, 0, 0};
    if (c.flags & PF_FLAG_TUNED) {
        std::lock_guard<std::mutex> g(g_tune_lock);
        auto it = g_tune.find(tune_key(c));
        if (it != g_tune.end()) t = it->second;
    }
    return t;
}

// One allocation carved into aligned pieces.
struct Arena {
    char *base = nullptr;
    size_t size = 0, used = 0;
    size_t take(size_t bytes) {
        const size_t off = (used + 255) & ~size_t(255);
        used = off + bytes;
        return off;
    }
};

}  // namespace

// A set of trackers of one precision, stepped by one launch.
struct Engine {
    int prec = 0;
    int n = 0;
    cudaStream_t stream = nullptr;
    std::vector<pf_config> cfg;
    std::vector<TrackerDev> h_trk;     // host copy; device pointers inside
    std::vector<FrameRef> h_frames;
    std::vector<int64_t> done_frames;  // per tracker
    std::vector<const uint8_t *> video_start;  // resident videos: first frame (pf_batch_reset)
    TrackerDev *d_trk = nullptr;
    FrameRef *d_frames = nullptr;
    FrameRef *h_frames_pinned = nullptr;
    int32_t *d_tile_trk = nullptr;
    // an ancestor kernel's trackers: device table of [n] slots, then [n + 1] CTA prefix
    struct AncestorTable {
        int32_t *d = nullptr;
        int n = 0;
        int ctas = 0;
    };
    AncestorTable gumbel, metro, rej;  // Gumbel-max, Metropolis, rejection
    uint32_t *d_ticket = nullptr;
    char *d_arena = nullptr;
    int total_tiles = 0;               // tiles of the step kernel's trackers (systematic, stratified)
    int pull_tiles = 0;                // tiles of the pull kernel's trackers (multinomial, Gumbel-max,
                                       // Metropolis, rejection)
    int n_multi = 0;                   // multinomial trackers (the CDF kernel runs when > 0)
    int grid = 0;
    int grid_pull = 0;
    int ctas_cap = 0;                  // CTAs per SM (0: as many as fit)
    pf_status sticky = PF_OK;
    uint8_t *d_frame_buf = nullptr;    // single tracker: staging of host frames
    TrackerState *h_init_pinned = nullptr;  // initial state of every tracker (pf_reset)
    cudaEvent_t frames_copied = nullptr;     // the pinned frame table may be rewritten after it
    cudaStream_t capture_stream = nullptr;   // private stream used to capture step graphs
    std::vector<std::pair<int32_t, cudaGraphExec_t>> graphs;   // count consecutive steps, replayed
    // host-frame runs: a ring of two chunks of staged frames, filled on a copy stream
    uint8_t *d_ring = nullptr;
    int64_t ring_pitch = 0;
    int32_t ring_chunk = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ring_copied[2] = {nullptr, nullptr}, ring_free[2] = {nullptr, nullptr};
    int64_t frame_buf_pitch = 0;
    // counters (pf_get_counters): launches enqueued, graph replays, host frame bytes copied
    int64_t n_step_launches = 0, n_kernels = 0, n_graphs = 0, n_host_bytes = 0;
    int kernels_per_step() const {
        return (total_tiles > 0 ? 1 : 0) + (pull_tiles > 0 ? 1 : 0) + (n_multi > 0 ? 1 : 0) + (gumbel.n > 0 ? 1 : 0) +
               (metro.n > 0 ? 1 : 0) + (rej.n > 0 ? 1 : 0);
    }

    pf_status fail(pf_status s) {
        if (sticky == PF_OK) sticky = s;
        return s;
    }
};

struct pf_filter {
    Engine e;
};

struct pf_batch {
    Engine e;
};

static void engine_free(Engine &e) {
    cudaStreamSynchronize(e.stream);
    for (auto &g : e.graphs) cudaGraphExecDestroy(g.second);
    e.graphs.clear();
    if (e.capture_stream) cudaStreamDestroy(e.capture_stream);
    if (e.frames_copied) cudaEventDestroy(e.frames_copied);
    e.capture_stream = nullptr; e.frames_copied = nullptr;
    if (e.copy_stream) { cudaStreamSynchronize(e.copy_stream); cudaStreamDestroy(e.copy_stream); }
    for (int k = 0; k < 2; ++k) {
        if (e.ring_copied[k]) cudaEventDestroy(e.ring_copied[k]);
        if (e.ring_free[k]) cudaEventDestroy(e.ring_free[k]);
        e.ring_copied[k] = e.ring_free[k] = nullptr;
    }
    cudaFree(e.d_ring);
    e.d_ring = nullptr; e.copy_stream = nullptr; e.ring_chunk = 0;
    cudaFree(e.d_trk);
    cudaFree(e.d_frames);
    cudaFree(e.d_tile_trk);
    cudaFree(e.gumbel.d);
    cudaFree(e.metro.d);
    cudaFree(e.rej.d);
    cudaFree(e.d_ticket);
    cudaFree(e.d_arena);
    cudaFree(e.d_frame_buf);
    if (e.h_frames_pinned) cudaFreeHost(e.h_frames_pinned);
    if (e.h_init_pinned) cudaFreeHost(e.h_init_pinned);
    e.h_init_pinned = nullptr;
    e.d_trk = nullptr; e.d_frames = nullptr; e.d_tile_trk = nullptr; e.d_ticket = nullptr;
    e.gumbel.d = nullptr; e.metro.d = nullptr; e.rej.d = nullptr;
    e.d_arena = nullptr; e.d_frame_buf = nullptr; e.h_frames_pinned = nullptr;
}

static pf_status engine_init(Engine &e, const pf_config *cfgs, int n, void *stream, bool stage_frames,
                             const pf_tuning *force = nullptr) {
    if (n < 1 || !cfgs) return PF_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        pf_status s = check_config(&cfgs[i]);
        if (s != PF_OK) return s;
        if (cfgs[i].precision != cfgs[0].precision) return PF_ERR_ARG;
    }
    e.prec = cfgs[0].precision;
    e.n = n;
    e.stream = static_cast<cudaStream_t>(stream);
    e.cfg.assign(cfgs, cfgs + n);
    e.h_trk.assign(n, TrackerDev{});
    e.h_frames.assign(n, FrameRef{});
    e.done_frames.assign(n, 0);
    e.video_start.assign(n, nullptr);

    // sizes
    const size_t pb = pos_bytes(e.prec);
    const size_t cdf_b = e.prec == PF_REF64 ? 8 : 4;
    Arena a;
    struct Off { size_t px[2], py[2], pl[2], look, part, done, state, est, stat, dbga, dbgc, dbgw, cdf, gtab; };
    std::vector<Off> off(n);
    // the trackers' states form one array (the kernel indexes it by tracker)
    const size_t states_off = a.take(sizeof(TrackerState) * n);
    // Tiles are numbered per kernel family: the step kernel's trackers first, then the
    // pull kernel's (multinomial, Gumbel-max, Metropolis, rejection), so no launch carries
    // tiles it skips.  The ancestor kernels number their CTAs per scheme.
    int64_t tiles = 0, mtiles = 0;
    std::vector<int32_t> atab[3], aprefix[3] = {{0}, {0}, {0}};   // Gumbel-max, Metropolis, rejection
    for (int i = 0; i < n; ++i) {
        const pf_config &c = cfgs[i];
        const int64_t N = c.num_particles;
        const pf_tuning tun = tuning_for(c, force);
        if (!valid_tuning(tun)) return PF_ERR_ARG;
        const int tile = tun.tile ? tun.tile : step_tile_size(e.prec, N);
        e.ctas_cap = (i == 0 || (e.ctas_cap > 0 && tun.ctas_per_sm > 0)) ? std::max(e.ctas_cap, tun.ctas_per_sm) : 0;
        const int64_t nt64 = (N + tile - 1) / tile;
        if (nt64 > 0x7fffffff) return PF_ERR_ARG;
        const int nt = static_cast<int>(nt64);
        if (tiles + mtiles + nt > 0x7fffffff) return PF_ERR_ARG;
        const int cap = c.est_capacity ? c.est_capacity : 4096;
        Off &o = off[i];
        for (int s = 0; s < 2; ++s) {
            o.px[s] = a.take(N * pb + 16);
            o.py[s] = a.take(N * pb + 16);
            o.pl[s] = a.take(N * pb + 16);
        }
        o.look = a.take(sizeof(LookbackDesc) * nt);
        o.part = a.take(sizeof(TilePartial) * nt);
        o.done = a.take(sizeof(uint32_t));
        // the tracker's likelihood table (step-family trackers of two or more tiles)
        o.gtab = SIZE_MAX;
        if (nt >= 2 && !(c.resampler == PF_RESAMPLE_MULTINOMIAL || ancestors_given(c.resampler)))
            o.gtab = a.take(sizeof(uint64_t) * kTableMax);
        o.state = states_off + sizeof(TrackerState) * i;
        o.est = a.take(sizeof(double) * 2 * cap);
        o.stat = a.take(sizeof(double) * 2 * cap);
        const bool given = ancestors_given(c.resampler);          // Gumbel-max, Metropolis, rejection
        const bool multi = c.resampler == PF_RESAMPLE_MULTINOMIAL || given;   // the pull family
        if (c.flags & PF_FLAG_DEBUG_ARRAYS) {
            o.dbga = a.take(sizeof(int32_t) * N);
            if (!multi) o.dbgc = a.take(cdf_b * N);
            o.dbgw = a.take(sizeof(int32_t) * 4 * static_cast<size_t>(nt));
        }
        if (multi) o.cdf = a.take((given ? sizeof(int32_t) : cdf_b) * N + 16);
        if (given) {
            const int s = c.resampler == PF_RESAMPLE_GUMBEL ? 0 : c.resampler == PF_RESAMPLE_METROPOLIS ? 1 : 2;
            const int per = s == 0 ? kGumbelOffspring : s == 1 ? kMetropolisThreads : kRejectionOffspring;
            const int64_t ctas = aprefix[s].back() + (N + per - 1) / per;
            if (ctas > 0x7fffffff) return PF_ERR_ARG;
            atab[s].push_back(i);
            aprefix[s].push_back(static_cast<int32_t>(ctas));
        }
        e.n_multi += (c.resampler == PF_RESAMPLE_MULTINOMIAL) ? 1 : 0;
        TrackerDev &T = e.h_trk[i];
        fill_tracker_constants(c, T);
        T.tile_begin = static_cast<int32_t>(multi ? mtiles : tiles);
        T.tile = tile;
        T.ntiles = nt;
        T.est_cap = cap;
        T.window = tun.window;
        (multi ? mtiles : tiles) += nt;
    }
    e.total_tiles = static_cast<int>(tiles);
    e.pull_tiles = static_cast<int>(mtiles);
    Engine::AncestorTable *tabs[3] = {&e.gumbel, &e.metro, &e.rej};
    for (int s = 0; s < 3; ++s) {
        tabs[s]->n = static_cast<int>(atab[s].size());
        tabs[s]->ctas = aprefix[s].back();
        atab[s].insert(atab[s].end(), aprefix[s].begin(), aprefix[s].end());   // slots, then prefix
    }
    a.size = a.used + 256;

    cudaError_t err = cudaMalloc(reinterpret_cast<void **>(&e.d_arena), a.size);
    if (err != cudaSuccess) { cudaGetLastError(); engine_free(e); return PF_ERR_OOM; }
    err = cudaMemsetAsync(e.d_arena, 0, a.size, e.stream);
    if (err == cudaSuccess) err = cudaMalloc(reinterpret_cast<void **>(&e.d_trk), sizeof(TrackerDev) * n);
    if (err == cudaSuccess) err = cudaMalloc(reinterpret_cast<void **>(&e.d_frames), sizeof(FrameRef) * n);
    if (err == cudaSuccess)
        err = cudaMalloc(reinterpret_cast<void **>(&e.d_tile_trk), sizeof(int32_t) * (e.total_tiles + e.pull_tiles + 1));
    for (int s = 0; s < 3 && err == cudaSuccess; ++s)
        if (tabs[s]->n > 0) err = cudaMalloc(reinterpret_cast<void **>(&tabs[s]->d), sizeof(int32_t) * atab[s].size());
    if (err == cudaSuccess) err = cudaMalloc(reinterpret_cast<void **>(&e.d_ticket), sizeof(uint32_t));
    if (err == cudaSuccess) err = cudaMallocHost(reinterpret_cast<void **>(&e.h_frames_pinned), sizeof(FrameRef) * n);
    if (err == cudaSuccess) err = cudaMallocHost(reinterpret_cast<void **>(&e.h_init_pinned), sizeof(TrackerState) * n);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e.frames_copied, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&e.capture_stream, cudaStreamNonBlocking);
    if (err == cudaSuccess && stage_frames) {
        e.frame_buf_pitch = (cfgs[0].width + 15) & ~15;
        err = cudaMalloc(reinterpret_cast<void **>(&e.d_frame_buf), static_cast<size_t>(e.frame_buf_pitch) * cfgs[0].height);
    }
    if (err != cudaSuccess) {
        cudaGetLastError();
        engine_free(e);
        return err == cudaErrorMemoryAllocation ? PF_ERR_OOM : PF_ERR_CUDA;
    }
    std::vector<int32_t> tile_trk(e.total_tiles + e.pull_tiles + 1);   // step family, then pull family
    std::vector<TrackerState> st(n);
    for (int i = 0; i < n; ++i) {
        TrackerDev &T = e.h_trk[i];
        const Off &o = off[i];
        for (int s = 0; s < 2; ++s) {
            T.px[s] = e.d_arena + o.px[s];
            T.py[s] = e.d_arena + o.py[s];
            T.pl[s] = e.d_arena + o.pl[s];
        }
        T.look = reinterpret_cast<LookbackDesc *>(e.d_arena + o.look);
        T.part = reinterpret_cast<TilePartial *>(e.d_arena + o.part);
        T.done = reinterpret_cast<uint32_t *>(e.d_arena + o.done);
        T.gtab = o.gtab == SIZE_MAX ? nullptr : reinterpret_cast<uint64_t *>(e.d_arena + o.gtab);
        T.state = reinterpret_cast<TrackerState *>(e.d_arena + o.state);
        T.est_ring = reinterpret_cast<double *>(e.d_arena + o.est);
        T.stat_ring = reinterpret_cast<double *>(e.d_arena + o.stat);
        if (e.cfg[i].flags & PF_FLAG_DEBUG_ARRAYS) {
            T.dbg_anc = reinterpret_cast<int32_t *>(e.d_arena + o.dbga);
            T.dbg_cdf = e.d_arena + o.dbgc;
            T.dbg_win = reinterpret_cast<int32_t *>(e.d_arena + o.dbgw);
        }
        if (e.cfg[i].resampler == PF_RESAMPLE_MULTINOMIAL) {
            // written by the CDF kernel, read by the pull kernel and by pf_get_debug
            T.cdf = e.d_arena + o.cdf;
            T.dbg_cdf = T.cdf;
        }
        if (ancestors_given(e.cfg[i].resampler)) {
            // written by the ancestor kernel, read by the pull kernel; no CDF exists
            T.anc = reinterpret_cast<int32_t *>(e.d_arena + o.cdf);
            T.dbg_cdf = nullptr;
        }
        const int base = (e.cfg[i].resampler == PF_RESAMPLE_MULTINOMIAL || ancestors_given(e.cfg[i].resampler))
                             ? e.total_tiles : 0;
        for (int k = 0; k < T.ntiles; ++k) tile_trk[base + T.tile_begin + k] = i;
        st[i] = initial_state(e.cfg[i]);
        e.h_frames[i].active = 1;
    }
    err = cudaMemcpyAsync(e.d_trk, e.h_trk.data(), sizeof(TrackerDev) * n, cudaMemcpyHostToDevice, e.stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(e.d_tile_trk, tile_trk.data(), sizeof(int32_t) * tile_trk.size(),
                              cudaMemcpyHostToDevice, e.stream);
    for (int s = 0; s < 3 && err == cudaSuccess; ++s)
        if (tabs[s]->n > 0)
            err = cudaMemcpyAsync(tabs[s]->d, atab[s].data(), sizeof(int32_t) * atab[s].size(), cudaMemcpyHostToDevice,
                                  e.stream);
    if (err == cudaSuccess) err = cudaMemsetAsync(e.d_ticket, 0, sizeof(uint32_t), e.stream);
    memcpy(e.h_init_pinned, st.data(), sizeof(TrackerState) * n);
    for (int i = 0; i < n && err == cudaSuccess; ++i)
        err = cudaMemcpyAsync(e.h_trk[i].state, &e.h_init_pinned[i], sizeof(TrackerState), cudaMemcpyHostToDevice,
                              e.stream);
    if (err == cudaSuccess) {
        memcpy(e.h_frames_pinned, e.h_frames.data(), sizeof(FrameRef) * n);
        err = cudaMemcpyAsync(e.d_frames, e.h_frames_pinned, sizeof(FrameRef) * n, cudaMemcpyHostToDevice, e.stream);
    }
    if (err == cudaSuccess) err = cudaStreamSynchronize(e.stream);   // host vectors go out of scope
    if (err != cudaSuccess) { cudaGetLastError(); engine_free(e); return PF_ERR_CUDA; }
    e.grid = e.total_tiles ? step_grid_size(e.prec, e.total_tiles) : 0;
    e.grid_pull = e.pull_tiles ? step_grid_size(e.prec, e.pull_tiles) : 0;
    if ((e.total_tiles && e.grid < 1) || (e.pull_tiles && e.grid_pull < 1)) {
        engine_free(e);
        return PF_ERR_CUDA;                  // no launchable kernel for this precision
    }
    if (e.ctas_cap > 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms > 0) {
            e.grid = std::min(e.grid, sms * e.ctas_cap);
            e.grid_pull = std::min(e.grid_pull, sms * e.ctas_cap);
        }
    }
    return PF_OK;
}

static AncestorLaunch ancestor_launch(const Engine &e, const Engine::AncestorTable &tab) {
    AncestorLaunch G;
    G.trk = e.d_trk;
    G.frames = e.d_frames;
    G.slots = tab.d;
    G.cta_prefix = tab.d + tab.n;
    G.ntrk = tab.n;
    G.total_ctas = tab.ctas;
    return G;
}

// One frame's launches: the step kernel over its family's tiles, then, for the pull
// family, the CDF kernel (multinomial trackers), the ancestor kernels (Gumbel-max,
// Metropolis, rejection) and the pull kernel over the pull family's tiles (tile table entries after
// the step family's).  L carries the step family's table and count.
static int engine_enqueue(const Engine &e, StepLaunch L, cudaStream_t stream) {
    int rc = 0;
    if (e.total_tiles > 0) rc = launch_step(e.prec, L, e.grid, stream);
    if (rc == 0 && e.gumbel.n > 0) rc = launch_gumbel(e.prec, ancestor_launch(e, e.gumbel), stream);
    if (rc == 0 && e.metro.n > 0) rc = launch_metropolis(e.prec, ancestor_launch(e, e.metro), stream);
    if (rc == 0 && e.rej.n > 0) rc = launch_rejection(e.prec, ancestor_launch(e, e.rej), stream);
    if (rc == 0 && e.pull_tiles > 0) {
        L.tile_trk = e.d_tile_trk + e.total_tiles;
        L.total_tiles = e.pull_tiles;
        rc = launch_pull(e.prec, L, e.grid_pull, e.n_multi > 0, stream);
    }
    return rc;
}

static pf_status engine_launch(Engine &e, const uint8_t *override_frame, int64_t override_pitch) {
    StepLaunch L;
    L.trk = e.d_trk;
    L.states = e.h_trk[0].state;
    L.frames = e.d_frames;
    L.tile_trk = e.d_tile_trk;
    L.tile_prefix = nullptr;
    L.slot_of = nullptr;
    L.est_out = nullptr;
    L.ticket = e.d_ticket;
    L.ntrk = e.n;
    L.total_tiles = e.total_tiles;
    L.frame_override = override_frame;
    L.pitch_override = override_pitch;
    if (engine_enqueue(e, L, e.stream) != 0) { cudaGetLastError(); return e.fail(PF_ERR_CUDA); }
    e.n_step_launches += 1;
    e.n_kernels += e.kernels_per_step();
    return PF_OK;
}

// Upload the frame table (pinned staging -> device) on the handle's stream.  The staging
// copy is only rewritten once the previous upload has been consumed.
static pf_status engine_upload_frames(Engine &e) {
    cudaError_t err = cudaMemcpyAsync(e.d_frames, e.h_frames_pinned, sizeof(FrameRef) * e.n,
                                      cudaMemcpyHostToDevice, e.stream);
    if (err == cudaSuccess) err = cudaEventRecord(e.frames_copied, e.stream);
    if (err != cudaSuccess) { cudaGetLastError(); return e.fail(PF_ERR_CUDA); }
    return PF_OK;
}

static pf_status engine_wait_staging(Engine &e) {
    if (cudaEventSynchronize(e.frames_copied) != cudaSuccess) { cudaGetLastError(); return e.fail(PF_ERR_CUDA); }
    return PF_OK;
}

// `count` steps that read their frames through the frame table (base + t * stride), as
// one CUDA graph of identical kernel nodes, captured once per count and replayed.
static pf_status engine_run_resident(Engine &e, int32_t count) {
    if (count <= 0) return PF_OK;
    cudaGraphExec_t exec = nullptr;
    for (auto &g : e.graphs)
        if (g.first == count) exec = g.second;
    if (!exec) {
        if (e.graphs.size() >= 4) {   // keep a few counts (a run's chunk and its tail)
            cudaGraphExecDestroy(e.graphs.front().second);
            e.graphs.erase(e.graphs.begin());
        }
        StepLaunch L;
        L.trk = e.d_trk;
        L.states = e.h_trk[0].state;
        L.frames = e.d_frames;
        L.tile_trk = e.d_tile_trk;
        L.tile_prefix = nullptr;
        L.slot_of = nullptr;
        L.est_out = nullptr;
        L.ticket = e.d_ticket;
        L.ntrk = e.n;
        L.total_tiles = e.total_tiles;
        L.frame_override = nullptr;
        L.pitch_override = 0;
        cudaGraph_t g = nullptr;
        cudaError_t err = cudaStreamBeginCapture(e.capture_stream, cudaStreamCaptureModeThreadLocal);
        int rc = 0;
        for (int32_t i = 0; i < count && err == cudaSuccess && rc == 0; ++i)
            rc = engine_enqueue(e, L, e.capture_stream);
        const cudaError_t end = cudaStreamEndCapture(e.capture_stream, &g);
        if (err == cudaSuccess) err = end;
        if (err == cudaSuccess && rc != 0) err = cudaErrorLaunchFailure;
        if (err == cudaSuccess) err = cudaGraphInstantiate(&exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (err != cudaSuccess) { cudaGetLastError(); return e.fail(PF_ERR_CUDA); }
        e.graphs.emplace_back(count, exec);
    }
    if (cudaGraphLaunch(exec, e.stream) != cudaSuccess) { cudaGetLastError(); return e.fail(PF_ERR_CUDA); }
    e.n_graphs += 1;
    e.n_step_launches += count;
    e.n_kernels += static_cast<int64_t>(count) * e.kernels_per_step();
    return PF_OK;
}

// Host frames, `count` of them `frame_stride` bytes apart: copied chunk by chunk into a
// ring of two chunks on the device by a copy stream, each chunk stepped by a replayed
// graph on the handle's stream as soon as its copy lands, so copies overlap the steps
// of the previous chunk.  The frame table points the kernel at the ring
// (frame t at ring + (t % 2C) * frame bytes).
static pf_status engine_run_host_frames(Engine &e, const uint8_t *frames, int64_t pitch_bytes,
                                        int64_t frame_stride, int32_t count) {
    const pf_config &c = e.cfg[0];
    constexpr int32_t kChunk = 8;
    cudaError_t err = cudaSuccess;
    if (!e.d_ring) {
        e.ring_pitch = (c.width + 15) & ~int64_t(15);
        err = cudaMalloc(reinterpret_cast<void **>(&e.d_ring), static_cast<size_t>(e.ring_pitch) * c.height * 2 * kChunk);
        if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&e.copy_stream, cudaStreamNonBlocking);
        for (int k = 0; k < 2 && err == cudaSuccess; ++k) {
            err = cudaEventCreateWithFlags(&e.ring_copied[k], cudaEventDisableTiming);
            if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e.ring_free[k], cudaEventDisableTiming);
        }
        if (err != cudaSuccess) {
            cudaGetLastError();
            return err == cudaErrorMemoryAllocation ? PF_ERR_OOM : e.fail(PF_ERR_CUDA);
        }
        e.ring_chunk = kChunk;
    }
    const int64_t fbytes = e.ring_pitch * c.height;
    const int64_t t0 = e.done_frames[0];
    pf_status s = engine_wait_staging(e);
    if (s != PF_OK) return s;
    FrameRef &fr = e.h_frames_pinned[0];
    fr.base = e.d_ring;
    fr.pitch = e.ring_pitch;
    fr.stride = fbytes;
    fr.active = 1;
    fr.ring = 2 * kChunk;
    s = engine_upload_frames(e);
    if (s != PF_OK) return s;
    // the copy stream must not overwrite frames earlier steps on the handle's stream still read
    err = cudaEventRecord(e.ring_free[0], e.stream);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(e.copy_stream, e.ring_free[0], 0);
    for (int32_t done = 0; done < count && err == cudaSuccess;) {
        const int32_t n = std::min(kChunk, count - done);
        // a chunk of up to kChunk frames may span both halves of the ring (its first frame
        // in half kc, its last in half kl); before overwriting them the copies wait for the
        // steps that last read those halves
        const int kc = static_cast<int>(((t0 + done) / kChunk) % 2);
        const int kl = static_cast<int>(((t0 + done + n - 1) / kChunk) % 2);
        if (done > 0) {
            err = cudaStreamWaitEvent(e.copy_stream, e.ring_free[kc], 0);
            if (err == cudaSuccess && kl != kc) err = cudaStreamWaitEvent(e.copy_stream, e.ring_free[kl], 0);
        }
        for (int32_t i = 0; i < n && err == cudaSuccess; ++i) {
            const int64_t t = t0 + done + i;
            err = cudaMemcpy2DAsync(e.d_ring + (t % (2 * kChunk)) * fbytes, e.ring_pitch,
                                    frames + static_cast<int64_t>(done + i) * frame_stride, pitch_bytes, c.width,
                                    c.height, cudaMemcpyHostToDevice, e.copy_stream);
        }
        if (err == cudaSuccess) e.n_host_bytes += static_cast<int64_t>(n) * c.width * c.height;
        if (err == cudaSuccess) err = cudaEventRecord(e.ring_copied[kc], e.copy_stream);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(e.stream, e.ring_copied[kc], 0);
        if (err != cudaSuccess) break;
        s = engine_run_resident(e, n);
        if (s != PF_OK) return s;
        err = cudaEventRecord(e.ring_free[kl], e.stream);
        if (err == cudaSuccess && kl != kc) err = cudaEventRecord(e.ring_free[kc], e.stream);
        done += n;
        e.done_frames[0] += n;
    }
    if (err != cudaSuccess) { cudaGetLastError(); return e.fail(PF_ERR_CUDA); }
    return PF_OK;
}

static pf_status engine_sync_status(Engine &e) {
    if (e.sticky != PF_OK) return e.sticky;
    cudaError_t err = cudaStreamSynchronize(e.stream);
    if (err != cudaSuccess) { cudaGetLastError(); return e.fail(PF_ERR_CUDA); }
    for (int i = 0; i < e.n; ++i) {
        uint32_t status = 0;
        err = cudaMemcpy(&status, &e.h_trk[i].state->status, sizeof status, cudaMemcpyDeviceToHost);
        if (err != cudaSuccess) { cudaGetLastError(); return e.fail(PF_ERR_CUDA); }
        if (status & kStatusTimeout) return e.fail(PF_ERR_TIMEOUT);
        if (status & kStatusBounds) return e.fail(PF_ERR_STATE);   // checked builds
    }
    return PF_OK;
}

static pf_status engine_read_frame(Engine &e, int i, int64_t idx, double *xy, double *ms) {
    const TrackerDev &T = e.h_trk[i];
    if (idx < 0 || idx >= e.done_frames[i] || idx < e.done_frames[i] - T.est_cap) return PF_ERR_ARG;
    const int64_t slot = idx % T.est_cap;
    cudaError_t err = cudaMemcpy(xy, T.est_ring + 2 * slot, 2 * sizeof(double), cudaMemcpyDeviceToHost);
    if (err == cudaSuccess && ms) err = cudaMemcpy(ms, T.stat_ring + 2 * slot, 2 * sizeof(double), cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) { cudaGetLastError(); return e.fail(PF_ERR_CUDA); }
    return PF_OK;
}

// ---------------------------------------------------------------------------- C ABI
extern "C" {

const char *pf_status_string(pf_status s) {
    switch (s) {
        case PF_OK: return "ok";
        case PF_ERR_ARG: return "invalid argument";
        case PF_ERR_OOM: return "out of memory";
        case PF_ERR_CUDA: return "CUDA error";
        case PF_ERR_TIMEOUT: return "device wait timed out";
        case PF_ERR_STATE: return "handle in failed state or wrong state";
        case PF_ERR_ADMISSION: return "admission refused";
    }
    return "unknown status";
}

pf_status pf_create(const pf_config *cfg, void *cuda_stream, pf_filter **out) {
    if (!cfg || !out) return PF_ERR_ARG;
    *out = nullptr;
    pf_filter *f = new (std::nothrow) pf_filter();
    if (!f) return PF_ERR_OOM;
    pf_status s = engine_init(f->e, cfg, 1, cuda_stream, true);
    if (s != PF_OK) { delete f; return s; }
    *out = f;
    return PF_OK;
}

pf_status pf_step_frame(pf_filter *f, const uint8_t *frame, int64_t pitch_bytes, int32_t frame_on_device) {
    TraceRange trace("pf_step_frame");
    if (!f || !frame) return PF_ERR_ARG;
    Engine &e = f->e;
    if (e.sticky != PF_OK) return PF_ERR_STATE;
    const pf_config &c = e.cfg[0];
    if (pitch_bytes < c.width) return PF_ERR_ARG;
    const uint8_t *dev = frame;
    int64_t pitch = pitch_bytes;
    if (!frame_on_device) {
        cudaError_t err = cudaMemcpy2DAsync(e.d_frame_buf, e.frame_buf_pitch, frame, pitch_bytes, c.width,
                                            c.height, cudaMemcpyHostToDevice, e.stream);
        if (err != cudaSuccess) { cudaGetLastError(); return e.fail(PF_ERR_CUDA); }
        dev = e.d_frame_buf;
        pitch = e.frame_buf_pitch;
        e.n_host_bytes += static_cast<int64_t>(c.width) * c.height;
    }
    pf_status s = engine_launch(e, dev, pitch);
    if (s != PF_OK) return s;
    e.done_frames[0] += 1;
    return PF_OK;
}

pf_status pf_run_frames(pf_filter *f, const uint8_t *frames, int64_t pitch_bytes, int64_t frame_stride,
                        int32_t count, int32_t frames_on_device) {
    TraceRange trace("pf_run_frames");
    if (!f || !frames || count < 0) return PF_ERR_ARG;
    Engine &e = f->e;
    if (e.sticky != PF_OK) return PF_ERR_STATE;
    if (pitch_bytes < e.cfg[0].width) return PF_ERR_ARG;
    if (!frames_on_device) {
        if (count == 0) return PF_OK;
        if (frame_stride < pitch_bytes * e.cfg[0].height) return PF_ERR_ARG;
        return engine_run_host_frames(e, frames, pitch_bytes, frame_stride, count);
    }
    if (count == 0) return PF_OK;
    // Device frames: the kernel finds frame t at base + t * stride, with base chosen so
    // that the tracker's next frame (t = frames done) is `frames`; then `count` identical
    // steps replay as one graph.
    pf_status s = engine_wait_staging(e);
    if (s != PF_OK) return s;
    FrameRef &fr = e.h_frames_pinned[0];
    fr.base = frames - e.done_frames[0] * frame_stride;
    fr.pitch = pitch_bytes;
    fr.stride = frame_stride;
    fr.active = 1;
    fr.ring = 0;
    s = engine_upload_frames(e);
    if (s == PF_OK) s = engine_run_resident(e, count);
    if (s != PF_OK) return s;
    e.done_frames[0] += count;
    return PF_OK;
}

pf_status pf_estimate(pf_filter *f, int64_t frame_index, double *x, double *y) {
    if (!f || !x || !y) return PF_ERR_ARG;
    Engine &e = f->e;
    pf_status s = engine_sync_status(e);
    if (s != PF_OK) return s;
    double xy[2];
    s = engine_read_frame(e, 0, frame_index, xy, nullptr);
    if (s != PF_OK) return s;
    *x = xy[0];
    *y = xy[1];
    return PF_OK;
}

pf_status pf_estimates(pf_filter *f, int64_t first, int32_t count, double *xy, double *max_and_sum) {
    if (!f || !xy || count < 0) return PF_ERR_ARG;
    Engine &e = f->e;
    pf_status s = engine_sync_status(e);
    if (s != PF_OK) return s;
    const TrackerDev &T = e.h_trk[0];
    const int64_t done = e.done_frames[0];
    if (count == 0) return PF_OK;
    if (first < 0 || first + count > done || first < done - T.est_cap) return PF_ERR_ARG;
    // copy in at most two contiguous pieces of the ring
    int64_t idx = first;
    int32_t left = count;
    while (left > 0) {
        const int64_t slot = idx % T.est_cap;
        int64_t run = T.est_cap - slot;
        if (run > left) run = left;
        cudaError_t err = cudaMemcpy(xy + 2 * (idx - first), T.est_ring + 2 * slot, run * 2 * sizeof(double),
                                     cudaMemcpyDeviceToHost);
        if (err == cudaSuccess && max_and_sum)
            err = cudaMemcpy(max_and_sum + 2 * (idx - first), T.stat_ring + 2 * slot, run * 2 * sizeof(double),
                             cudaMemcpyDeviceToHost);
        if (err != cudaSuccess) { cudaGetLastError(); return e.fail(PF_ERR_CUDA); }
        idx += run;
        left -= static_cast<int32_t>(run);
    }
    return PF_OK;
}

int64_t pf_frames_done(const pf_filter *f) { return f ? f->e.done_frames[0] : -1; }

static void fill_counters(const Engine &e, pf_counters *out) {
    memset(out, 0, sizeof *out);
    int64_t frames = 0;
    for (int i = 0; i < e.n; ++i) frames += e.done_frames[i];
    out->frames = frames;
    out->step_launches = e.n_step_launches;
    out->kernel_launches = e.n_kernels;
    out->graph_launches = e.n_graphs;
    out->host_frame_bytes = e.n_host_bytes;
    out->status = e.sticky;
}

pf_status pf_get_counters(const pf_filter *f, pf_counters *out) {
    if (!f || !out) return PF_ERR_ARG;
    fill_counters(f->e, out);
    return PF_OK;
}

// Clear tracker i's lookback descriptors on the engine's stream.
static cudaError_t clear_lookback(Engine &e, int i) {
    const TrackerDev &T = e.h_trk[i];
    return cudaMemsetAsync(T.look, 0, sizeof(LookbackDesc) * static_cast<size_t>(T.ntiles), e.stream);
}

pf_status pf_reset(pf_filter *f) {
    if (!f) return PF_ERR_ARG;
    Engine &e = f->e;
    if (e.sticky != PF_OK) return PF_ERR_STATE;
    // Rewrite every field of the state except the launch counter (epoch) and the status
    // word, and clear the lookback descriptors (their tags are launch counters modulo
    // 65535: cleared words can never look current).
    TrackerState *d = e.h_trk[0].state;
    const TrackerState *h = &e.h_init_pinned[0];
    const size_t tail = sizeof(TrackerState) - offsetof(TrackerState, M);
    cudaError_t err = cudaMemcpyAsync(&d->t, &h->t, sizeof(int64_t), cudaMemcpyHostToDevice, e.stream);
    if (err == cudaSuccess) err = cudaMemcpyAsync(&d->M, &h->M, tail, cudaMemcpyHostToDevice, e.stream);
    if (err == cudaSuccess) err = clear_lookback(e, 0);
    if (err != cudaSuccess) { cudaGetLastError(); return e.fail(PF_ERR_CUDA); }
    e.done_frames[0] = 0;
    return PF_OK;
}

pf_status pf_destroy(pf_filter *f) {
    if (!f) return PF_OK;
    engine_free(f->e);
    delete f;
    return PF_OK;
}

pf_status pf_get_state(pf_filter *f, void *host_buf, size_t *bytes) {
    if (!f || !bytes) return PF_ERR_ARG;
    Engine &e = f->e;
    const TrackerDev &T = e.h_trk[0];
    const size_t pb = pos_bytes(e.prec);
    const size_t need = sizeof(pf_state_header) + 3 * pb * static_cast<size_t>(T.N);
    if (!host_buf) { *bytes = need; return PF_OK; }
    if (*bytes < need) return PF_ERR_ARG;
    cudaError_t err = cudaStreamSynchronize(e.stream);
    TrackerState st;
    if (err == cudaSuccess) err = cudaMemcpy(&st, T.state, sizeof st, cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) { cudaGetLastError(); return e.fail(PF_ERR_CUDA); }
    pf_state_header h;
    memset(&h, 0, sizeof h);
    h.magic = 0x31534650u;
    h.precision = e.prec;
    h.num_particles = T.N;
    h.t = st.t;
    h.max_l = st.M;
    h.sum_e = st.S;
    h.anchor_x = st.ax;
    h.anchor_y = st.ay;
    h.next_anchor_x = st.nx;
    h.next_anchor_y = st.ny;
    h.est_x = st.est_x;
    h.est_y = st.est_y;
    char *p = static_cast<char *>(host_buf);
    memcpy(p, &h, sizeof h);
    p += sizeof h;
    const int slot = static_cast<int>((st.t + 1) & 1);
    const size_t nb = pb * static_cast<size_t>(T.N);
    err = cudaMemcpy(p, T.px[slot], nb, cudaMemcpyDeviceToHost);
    if (err == cudaSuccess) err = cudaMemcpy(p + nb, T.py[slot], nb, cudaMemcpyDeviceToHost);
    if (err == cudaSuccess) err = cudaMemcpy(p + 2 * nb, T.pl[slot], nb, cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) { cudaGetLastError(); return e.fail(PF_ERR_CUDA); }
    *bytes = need;
    return PF_OK;
}

pf_status pf_set_state(pf_filter *f, const void *host_buf, size_t bytes) {
    if (!f || !host_buf) return PF_ERR_ARG;
    Engine &e = f->e;
    if (e.sticky != PF_OK) return PF_ERR_STATE;
    const TrackerDev &T = e.h_trk[0];
    const size_t pb = pos_bytes(e.prec);
    const size_t need = sizeof(pf_state_header) + 3 * pb * static_cast<size_t>(T.N);
    if (bytes < need) return PF_ERR_ARG;
    pf_state_header h;
    memcpy(&h, host_buf, sizeof h);
    if (h.magic != 0x31534650u || h.precision != e.prec || h.num_particles != T.N || h.t < 0) return PF_ERR_ARG;
    if (!(h.sum_e > 0) || !isfinite(h.max_l)) return PF_ERR_ARG;
    cudaError_t err = cudaStreamSynchronize(e.stream);
    TrackerState st;
    if (err == cudaSuccess) err = cudaMemcpy(&st, T.state, sizeof st, cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) { cudaGetLastError(); return e.fail(PF_ERR_CUDA); }
    st.t = h.t;
    st.M = h.max_l;
    st.S = h.sum_e;
    st.invS = e.prec == PF_REF64 ? 1.0 / h.sum_e
                                 : static_cast<double>(1.0f / static_cast<float>(h.sum_e));
    st.ax = h.anchor_x;
    st.ay = h.anchor_y;
    st.nx = h.next_anchor_x;
    st.ny = h.next_anchor_y;
    st.est_x = h.est_x;
    st.est_y = h.est_y;
    bbox_unknown(st);   // the next step tabulates the likelihood per tile
    state_copies(st);
    const char *p = static_cast<const char *>(host_buf) + sizeof h;
    const int slot = static_cast<int>((h.t + 1) & 1);
    const size_t nb = pb * static_cast<size_t>(T.N);
    err = cudaMemcpy(T.state, &st, sizeof st, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemset(T.look, 0, sizeof(LookbackDesc) * static_cast<size_t>(T.ntiles));
    if (err == cudaSuccess) err = cudaMemcpy(T.px[slot], p, nb, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(T.py[slot], p + nb, nb, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(T.pl[slot], p + 2 * nb, nb, cudaMemcpyHostToDevice);
    if (err != cudaSuccess) { cudaGetLastError(); return e.fail(PF_ERR_CUDA); }
    e.done_frames[0] = h.t;
    return PF_OK;
}

pf_status pf_get_debug(pf_filter *f, int32_t which, void *host_buf, size_t bytes) {
    if (!f || !host_buf) return PF_ERR_ARG;
    Engine &e = f->e;
    const TrackerDev &T = e.h_trk[0];
    if (!T.dbg_anc) return PF_ERR_STATE;
    if (which == 1 && !T.dbg_cdf) return PF_ERR_ARG;   // Gumbel-max, Metropolis, rejection: no CDF
    if (which == 2) {   // per-tile windows
        const size_t wb = sizeof(int32_t) * 4 * static_cast<size_t>(T.ntiles);
        if (bytes < wb) return PF_ERR_ARG;
        cudaError_t err = cudaStreamSynchronize(e.stream);
        if (err == cudaSuccess) err = cudaMemcpy(host_buf, T.dbg_win, wb, cudaMemcpyDeviceToHost);
        if (err != cudaSuccess) { cudaGetLastError(); return e.fail(PF_ERR_CUDA); }
        return PF_OK;
    }
    const size_t elem = which == 0 ? 4 : (e.prec == PF_REF64 ? 8 : 4);
    if (which < 0 || which > 1 || bytes < elem * static_cast<size_t>(T.N)) return PF_ERR_ARG;
    cudaError_t err = cudaStreamSynchronize(e.stream);
    if (err == cudaSuccess)
        err = cudaMemcpy(host_buf, which == 0 ? static_cast<void *>(T.dbg_anc) : T.dbg_cdf,
                         elem * static_cast<size_t>(T.N), cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) { cudaGetLastError(); return e.fail(PF_ERR_CUDA); }
    return PF_OK;
}

pf_status pf_debug_philox(const uint32_t *ctrs, int64_t n, uint64_t seed, uint32_t *out) {
    if (!ctrs || !out || n < 0) return PF_ERR_ARG;
    if (n == 0) return PF_OK;
    uint32_t *d = nullptr;
    cudaError_t err = cudaMalloc(reinterpret_cast<void **>(&d), static_cast<size_t>(n) * 32);
    if (err != cudaSuccess) { cudaGetLastError(); return PF_ERR_OOM; }
    err = cudaMemcpy(d, ctrs, static_cast<size_t>(n) * 16, cudaMemcpyHostToDevice);
    if (err == cudaSuccess && launch_debug_philox(d, n, seed, d + 4 * n, nullptr) != 0) err = cudaErrorLaunchFailure;
    if (err == cudaSuccess) err = cudaMemcpy(out, d + 4 * n, static_cast<size_t>(n) * 16, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (err != cudaSuccess) { cudaGetLastError(); return PF_ERR_CUDA; }
    return PF_OK;
}

pf_status pf_debug_wait_timeout(uint32_t spin_limit, uint32_t *status_out) {
    if (!status_out || spin_limit == 0 || spin_limit > (1u << 20)) return PF_ERR_ARG;
    void *d = nullptr;
    const size_t bytes = sizeof(LookbackDesc) + sizeof(TrackerState);
    cudaError_t err = cudaMalloc(&d, bytes);
    if (err != cudaSuccess) { cudaGetLastError(); return PF_ERR_OOM; }
    err = cudaMemset(d, 0, bytes);   // the descriptor's words stay untagged: nobody publishes it
    char *base = static_cast<char *>(d);
    if (err == cudaSuccess && launch_wait_probe(base, base + sizeof(LookbackDesc), spin_limit, nullptr) != 0)
        err = cudaErrorLaunchFailure;
    TrackerState st;
    if (err == cudaSuccess) err = cudaMemcpy(&st, base + sizeof(LookbackDesc), sizeof st, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (err != cudaSuccess) { cudaGetLastError(); return PF_ERR_CUDA; }
    *status_out = st.status;
    if (st.status & kStatusBounds) return PF_ERR_STATE;   // checked builds
    return (st.status & kStatusTimeout) ? PF_ERR_TIMEOUT : PF_OK;
}

// ---------------------------------------------------------------------------- batches
pf_status pf_batch_create(const pf_config *cfgs, int32_t n, void *cuda_stream, pf_batch **out) {
    if (!cfgs || !out || n < 1) return PF_ERR_ARG;
    *out = nullptr;
    pf_batch *b = new (std::nothrow) pf_batch();
    if (!b) return PF_ERR_OOM;
    pf_status s = engine_init(b->e, cfgs, n, cuda_stream, false);
    if (s != PF_OK) { delete b; return s; }
    *out = b;
    return PF_OK;
}

pf_status pf_batch_step(pf_batch *b, const uint8_t *const *frames, const int64_t *pitches,
                        const uint8_t *active_mask) {
    TraceRange trace("pf_batch_step");
    if (!b || !frames || !pitches) return PF_ERR_ARG;
    Engine &e = b->e;
    if (e.sticky != PF_OK) return PF_ERR_STATE;
    for (int i = 0; i < e.n; ++i) {
        const int act = active_mask ? (active_mask[i] != 0) : 1;
        if (act && (!frames[i] || pitches[i] < e.cfg[i].width)) return PF_ERR_ARG;
    }
    pf_status s = engine_wait_staging(e);
    if (s != PF_OK) return s;
    for (int i = 0; i < e.n; ++i) {
        const int act = active_mask ? (active_mask[i] != 0) : 1;
        FrameRef &fr = e.h_frames_pinned[i];
        fr.base = act ? frames[i] : nullptr;
        fr.pitch = act ? pitches[i] : 0;
        fr.stride = 0;
        fr.active = act;
        e.video_start[i] = nullptr;
    }
    s = engine_upload_frames(e);
    if (s == PF_OK) s = engine_launch(e, nullptr, 0);
    if (s != PF_OK) return s;
    for (int i = 0; i < e.n; ++i)
        if (e.h_frames_pinned[i].active) e.done_frames[i] += 1;
    return PF_OK;
}

static pf_status engine_set_videos(Engine &e, const uint8_t *const *videos, const int64_t *pitches,
                                   const int64_t *frame_strides) {
    for (int i = 0; i < e.n; ++i)
        if (!videos[i] || pitches[i] < e.cfg[i].width || frame_strides[i] < pitches[i] * e.cfg[i].height)
            return PF_ERR_ARG;
    pf_status s = engine_wait_staging(e);
    if (s != PF_OK) return s;
    for (int i = 0; i < e.n; ++i) {
        FrameRef &fr = e.h_frames_pinned[i];
        e.video_start[i] = videos[i];
        fr.base = videos[i] - e.done_frames[i] * frame_strides[i];
        fr.pitch = pitches[i];
        fr.stride = frame_strides[i];
        fr.active = 1;
        fr.ring = 0;
    }
    return engine_upload_frames(e);
}

pf_status pf_batch_set_videos(pf_batch *b, const uint8_t *const *videos, const int64_t *pitches,
                              const int64_t *frame_strides) {
    if (!b || !videos || !pitches || !frame_strides) return PF_ERR_ARG;
    if (b->e.sticky != PF_OK) return PF_ERR_STATE;
    return engine_set_videos(b->e, videos, pitches, frame_strides);
}

pf_status pf_batch_run(pf_batch *b, int32_t count) {
    TraceRange trace("pf_batch_run");
    if (!b || count < 0) return PF_ERR_ARG;
    Engine &e = b->e;
    if (e.sticky != PF_OK) return PF_ERR_STATE;
    for (int i = 0; i < e.n; ++i)
        if (!e.h_frames_pinned[i].active || e.h_frames_pinned[i].stride == 0) return PF_ERR_STATE;
    pf_status s = engine_run_resident(e, count);
    if (s != PF_OK) return s;
    for (int i = 0; i < e.n; ++i) e.done_frames[i] += count;
    return PF_OK;
}

pf_status pf_batch_get_counters(const pf_batch *b, pf_counters *out) {
    if (!b || !out) return PF_ERR_ARG;
    fill_counters(b->e, out);
    return PF_OK;
}

static pf_status engine_reset(Engine &e) {
    const size_t tail = sizeof(TrackerState) - offsetof(TrackerState, M);
    pf_status s = engine_wait_staging(e);
    if (s != PF_OK) return s;
    for (int i = 0; i < e.n; ++i) {
        TrackerState *d = e.h_trk[i].state;
        const TrackerState *h = &e.h_init_pinned[i];
        cudaError_t err = cudaMemcpyAsync(&d->t, &h->t, sizeof(int64_t), cudaMemcpyHostToDevice, e.stream);
        if (err == cudaSuccess) err = cudaMemcpyAsync(&d->M, &h->M, tail, cudaMemcpyHostToDevice, e.stream);
        if (err == cudaSuccess) err = clear_lookback(e, i);
        if (err != cudaSuccess) { cudaGetLastError(); return e.fail(PF_ERR_CUDA); }
        // resident videos: frame 0 is again the video's first frame
        FrameRef &fr = e.h_frames_pinned[i];
        if (fr.stride && e.video_start[i]) fr.base = e.video_start[i];
        e.done_frames[i] = 0;
    }
    return engine_upload_frames(e);
}

pf_status pf_batch_reset(pf_batch *b) {
    if (!b) return PF_ERR_ARG;
    if (b->e.sticky != PF_OK) return PF_ERR_STATE;
    return engine_reset(b->e);
}

pf_status pf_batch_estimates(pf_batch *b, int64_t frame_index, double *xy) {
    if (!b || !xy) return PF_ERR_ARG;
    Engine &e = b->e;
    pf_status s = engine_sync_status(e);
    if (s != PF_OK) return s;
    for (int i = 0; i < e.n; ++i) {
        double v[2];
        if (engine_read_frame(e, i, frame_index, v, nullptr) == PF_OK) {
            xy[2 * i] = v[0];
            xy[2 * i + 1] = v[1];
        } else {
            xy[2 * i] = NAN;
            xy[2 * i + 1] = NAN;
        }
    }
    return e.sticky;
}

pf_status pf_batch_destroy(pf_batch *b) {
    if (!b) return PF_OK;
    engine_free(b->e);
    delete b;
    return PF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------- autotuning
pf_status pf_tuning_lookup(const pf_config *cfg, pf_tuning *out) {
    if (!out || check_config(cfg) != PF_OK) return PF_ERR_ARG;
    std::lock_guard<std::mutex> g(g_tune_lock);
    auto it = g_tune.find(tune_key(*cfg));
    if (it == g_tune.end()) return PF_ERR_STATE;
    *out = it->second;
    return PF_OK;
}

pf_status pf_tuning_store(const pf_config *cfg, const pf_tuning *t) {
    if (!t || check_config(cfg) != PF_OK || !valid_tuning(*t)) return PF_ERR_ARG;
    std::lock_guard<std::mutex> g(g_tune_lock);
    g_tune[tune_key(*cfg)] = *t;
    return PF_OK;
}

pf_status pf_tuning_clear(void) {
    std::lock_guard<std::mutex> g(g_tune_lock);
    g_tune.clear();
    return PF_OK;
}

// Time every candidate shape, applied to all trackers alike, on a batch of these trackers
// over their resident videos; the fastest shape and its time per frame.
static pf_status sweep_shapes(std::vector<pf_config> cfgs, const std::vector<const uint8_t *> &vids,
                              const std::vector<int64_t> &pitches, const std::vector<int64_t> &strides,
                              int32_t n_frames, pf_tuning *best, double *best_us) {
    const int n = static_cast<int>(cfgs.size());
    for (pf_config &c : cfgs) {
        c.flags &= ~(PF_FLAG_DEBUG_ARRAYS | PF_FLAG_TUNED);
        c.est_capacity = n_frames + 1;
    }
    cudaStream_t stream = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    if (err != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        if (stream) cudaStreamDestroy(stream);
        return PF_ERR_CUDA;
    }
    static const int32_t kTiles[] = {0, 1024, 2048, 3072, 4096};
    pf_tuning win{0, 0, 0, 0};
    double win_ms = -1.0;
    pf_status result = PF_OK;
    for (int32_t tile : kTiles) {
        if (tile > kTile) continue;
        for (int32_t window = 0; window <= 2 && result == PF_OK; ++window) {
            for (int32_t ctas = 0; ctas <= 1 && result == PF_OK; ++ctas) {
                const pf_tuning cand{tile, window, ctas, 0};
                pf_batch *b = new (std::nothrow) pf_batch();
                if (!b) { result = PF_ERR_OOM; break; }
                pf_status st = engine_init(b->e, cfgs.data(), n, stream, false, &cand);
                if (st != PF_OK) { delete b; if (st != PF_ERR_OOM) result = st; continue; }
                Engine &e = b->e;
                float ms = 0.0f;
                st = engine_set_videos(e, vids.data(), pitches.data(), strides.data());
                if (st == PF_OK) st = engine_run_resident(e, n_frames);       // warm-up (and graph capture)
                if (st == PF_OK) st = engine_reset(e);
                if (st == PF_OK && cudaEventRecord(e0, stream) != cudaSuccess) st = PF_ERR_CUDA;
                if (st == PF_OK) st = engine_run_resident(e, n_frames);
                if (st == PF_OK && (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                    cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                    st = PF_ERR_CUDA;
                if (st == PF_OK) st = engine_sync_status(e);
                engine_free(e);
                delete b;
                if (st != PF_OK) { cudaGetLastError(); result = st; break; }
                if (win_ms < 0 || ms < win_ms) { win_ms = ms; win = cand; }
            }
        }
        if (result != PF_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(stream);
    if (result != PF_OK) return result;
    if (win_ms < 0) return PF_ERR_OOM;
    *best = win;
    if (best_us) *best_us = 1e3 * win_ms / n_frames;
    return PF_OK;
}

pf_status pf_autotune(const pf_config *cfg, int32_t copies, const uint8_t *video, int64_t pitch_bytes,
                      int64_t frame_stride, int32_t n_frames, pf_tuning *best, double *best_us_per_frame) {
    TraceRange trace("pf_autotune");
    if (!best || check_config(cfg) != PF_OK || copies < 1 || copies > 4096 || !video || n_frames < 1) return PF_ERR_ARG;
    if (pitch_bytes < cfg->width || frame_stride < pitch_bytes * cfg->height) return PF_ERR_ARG;
    std::vector<pf_config> cfgs(copies, *cfg);
    for (int i = 0; i < copies; ++i) cfgs[i].tracker_id = cfg->tracker_id + static_cast<uint32_t>(i);
    pf_status s = sweep_shapes(cfgs, std::vector<const uint8_t *>(copies, video), std::vector<int64_t>(copies, pitch_bytes),
                               std::vector<int64_t>(copies, frame_stride), n_frames, best, best_us_per_frame);
    if (s != PF_OK) return s;
    std::lock_guard<std::mutex> g(g_tune_lock);
    g_tune[tune_key(*cfg)] = *best;
    return PF_OK;
}

pf_status pf_autotune_batch(const pf_config *cfgs, int32_t n, const uint8_t *const *videos, const int64_t *pitches,
                            const int64_t *frame_strides, int32_t n_frames, pf_tuning *best, double *best_us_per_frame) {
    TraceRange trace("pf_autotune_batch");
    if (!best || !cfgs || n < 1 || !videos || !pitches || !frame_strides || n_frames < 1) return PF_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        if (check_config(&cfgs[i]) != PF_OK || cfgs[i].precision != cfgs[0].precision || !videos[i]) return PF_ERR_ARG;
        if (pitches[i] < cfgs[i].width || frame_strides[i] < pitches[i] * cfgs[i].height) return PF_ERR_ARG;
    }
    pf_status s = sweep_shapes(std::vector<pf_config>(cfgs, cfgs + n), std::vector<const uint8_t *>(videos, videos + n),
                               std::vector<int64_t>(pitches, pitches + n), std::vector<int64_t>(frame_strides, frame_strides + n),
                               n_frames, best, best_us_per_frame);
    if (s != PF_OK) return s;
    std::lock_guard<std::mutex> g(g_tune_lock);
    for (int i = 0; i < n; ++i) g_tune[tune_key(cfgs[i])] = *best;
    return PF_OK;
}
