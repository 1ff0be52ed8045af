// pf_shard.cu -- one tracker sharded by particles across ranks (one GPU per rank).
//
// Rank q of R holds the contiguous particles [k_q, k_q + n_q) of an N-particle tracker
// (k_q even, so a Philox pair never straddles two ranks).  A frame of the sharded filter
// (the exchanges between the calls are the caller's; paper_2308_00763_gb300/sharded.py
// drives them over a torch.distributed process group):
//   pf_shard_stats     the shard's (M_q, S_q, estimate) of the frame it stepped last;
//   (all-gather: every rank forms the global M, S and the prefix P_q of the rescaled
//    totals before it, in rank order)
//   pf_shard_resample  the CDF of the shard's particles against the global weights
//                      (C_k = (P_q + local prefix) / S, from P_q to P_(q+1)) and, over the
//                      global strata u_j = (j + u0) / N, the ancestor position of every
//                      offspring of its run [J(P_q / S), J(P_(q+1) / S)) -- the resampling
//                      of Sec. IV, "Resampling", cut at the shard's boundaries;
//   (all-to-all: each slice of the runs goes to the rank that owns those offspring slots)
//   pf_shard_step      the received ancestor positions become the previous frame's
//                      particles of the shard's slots, and the pull kernel propagates them
//                      (draws keyed by the global particle index), scores them (Eq. 3-4)
//                      and forms the shard's statistics (Eq. 5).
// REF64 and F32 shards (absolute positions travel between ranks); systematic resampling.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "pf.h"
#include "pf_host.h"
#include "pf_internal.h"

using namespace pfk;

struct pf_shard {
    pf_config cfg{};          // the shard's own configuration (num_particles = n_q)
    int64_t n_global = 0;
    int64_t j_base = 0;
    int32_t rank = 0, nranks = 1;
    int prec = 0;
    cudaStream_t stream = nullptr;
    TrackerDev h_trk{};
    TrackerDev *d_trk = nullptr;
    FrameRef *d_frame = nullptr;
    FrameRef *h_frame = nullptr;      // pinned
    uint32_t *d_ticket = nullptr;
    char *d_arena = nullptr;
    int64_t *d_run = nullptr;         // [2] offspring run of the last resample, then status word
    int64_t *h_run = nullptr;         // pinned [3]
    TrackerState *h_state = nullptr;  // pinned
    int grid = 0;
    int64_t t = 0;                    // frames stepped
    pf_status sticky = PF_OK;
    pf_status fail(pf_status s) {
        if (sticky == PF_OK) sticky = s;
        return s;
    }
};

namespace {

__global__ void iota_kernel(int32_t *a, int64_t n) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        a[i] = static_cast<int32_t>(i);
}

size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

void shard_free(pf_shard *h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    cudaFree(h->d_trk);
    cudaFree(h->d_frame);
    cudaFree(h->d_ticket);
    cudaFree(h->d_arena);
    cudaFree(h->d_run);
    if (h->h_frame) cudaFreeHost(h->h_frame);
    if (h->h_run) cudaFreeHost(h->h_run);
    if (h->h_state) cudaFreeHost(h->h_state);
    delete h;
}

StepLaunch single_launch(const pf_shard *h) {
    StepLaunch L;
    L.trk = h->d_trk;
    L.states = h->h_trk.state;
    L.frames = h->d_frame;
    L.tile_trk = nullptr;
    L.tile_prefix = nullptr;
    L.slot_of = nullptr;
    L.est_out = nullptr;
    L.ticket = h->d_ticket;
    L.ntrk = 1;
    L.total_tiles = h->h_trk.ntiles;
    L.frame_override = nullptr;
    L.pitch_override = 0;
    return L;
}

}  // namespace

extern "C" pf_status pf_shard_partition(int64_t n_global, int32_t nranks, int32_t rank, int64_t *first,
                                        int64_t *count) {
    if (nranks < 1 || rank < 0 || rank >= nranks || n_global < 2 * static_cast<int64_t>(nranks) || !first || !count)
        return PF_ERR_ARG;
    const int64_t base = (n_global / nranks) & ~int64_t(1);
    *first = base * rank;
    *count = rank == nranks - 1 ? n_global - base * (nranks - 1) : base;
    return PF_OK;
}

extern "C" pf_status pf_shard_create(const pf_config *cfg, int32_t rank, int32_t nranks, void *cuda_stream,
                                     pf_shard **out) {
    if (!cfg || !out) return PF_ERR_ARG;
    *out = nullptr;
    pf_status s = check_config(cfg);
    if (s != PF_OK) return s;
    if (cfg->precision != PF_REF64 && cfg->precision != PF_F32) return PF_ERR_ARG;
    if (cfg->resampler != PF_RESAMPLE_SYSTEMATIC || (cfg->flags & ~PF_FLAG_ACCUM32)) return PF_ERR_ARG;
    int64_t first = 0, count = 0;
    s = pf_shard_partition(cfg->num_particles, nranks, rank, &first, &count);
    if (s != PF_OK) return s;
    pf_shard *h = new pf_shard();
    h->cfg = *cfg;
    h->cfg.num_particles = count;
    h->cfg.est_capacity = 2;
    h->n_global = cfg->num_particles;
    h->j_base = first;
    h->rank = rank;
    h->nranks = nranks;
    h->prec = cfg->precision;
    h->stream = static_cast<cudaStream_t>(cuda_stream);

    TrackerDev &T = h->h_trk;
    fill_tracker_constants(h->cfg, T);
    T.resampler = kResampleShard;
    T.j_base = first;
    T.tile = step_tile_size(h->prec, count);
    T.ntiles = static_cast<int32_t>((count + T.tile - 1) / T.tile);
    T.tile_begin = 0;
    T.est_cap = 2;
    const size_t pb = pos_bytes(h->prec);
    size_t off = 0;
    auto take = [&](size_t b) { const size_t at = off; off = align_up(off + b); return at; };
    size_t px[2], py[2], pl[2];
    for (int k = 0; k < 2; ++k) {
        px[k] = take(count * pb + 16);
        py[k] = take(count * pb + 16);
        pl[k] = take(count * pb + 16);
    }
    const size_t o_look = take(sizeof(LookbackDesc) * T.ntiles), o_part = take(sizeof(TilePartial) * T.ntiles);
    const size_t o_done = take(sizeof(uint32_t)), o_state = take(sizeof(TrackerState));
    const size_t o_est = take(sizeof(double) * 4), o_stat = take(sizeof(double) * 4);
    const size_t o_cdf = take(pb * count + 16), o_anc = take(sizeof(int32_t) * count + 16);
    cudaError_t err = cudaMalloc(reinterpret_cast<void **>(&h->d_arena), off);
    if (err == cudaSuccess) err = cudaMemsetAsync(h->d_arena, 0, off, h->stream);
    if (err == cudaSuccess) err = cudaMalloc(reinterpret_cast<void **>(&h->d_trk), sizeof(TrackerDev));
    if (err == cudaSuccess) err = cudaMalloc(reinterpret_cast<void **>(&h->d_frame), sizeof(FrameRef));
    if (err == cudaSuccess) err = cudaMalloc(reinterpret_cast<void **>(&h->d_ticket), sizeof(uint32_t));
    if (err == cudaSuccess) err = cudaMalloc(reinterpret_cast<void **>(&h->d_run), 3 * sizeof(int64_t));
    if (err == cudaSuccess) err = cudaMallocHost(reinterpret_cast<void **>(&h->h_frame), sizeof(FrameRef));
    if (err == cudaSuccess) err = cudaMallocHost(reinterpret_cast<void **>(&h->h_run), 3 * sizeof(int64_t));
    if (err == cudaSuccess) err = cudaMallocHost(reinterpret_cast<void **>(&h->h_state), sizeof(TrackerState));
    if (err != cudaSuccess) {
        cudaGetLastError();
        shard_free(h);
        return err == cudaErrorMemoryAllocation ? PF_ERR_OOM : PF_ERR_CUDA;
    }
    for (int k = 0; k < 2; ++k) {
        T.px[k] = h->d_arena + px[k];
        T.py[k] = h->d_arena + py[k];
        T.pl[k] = h->d_arena + pl[k];
    }
    T.look = reinterpret_cast<LookbackDesc *>(h->d_arena + o_look);
    T.part = reinterpret_cast<TilePartial *>(h->d_arena + o_part);
    T.done = reinterpret_cast<uint32_t *>(h->d_arena + o_done);
    T.state = reinterpret_cast<TrackerState *>(h->d_arena + o_state);
    T.est_ring = reinterpret_cast<double *>(h->d_arena + o_est);
    T.stat_ring = reinterpret_cast<double *>(h->d_arena + o_stat);
    T.cdf = h->d_arena + o_cdf;
    T.anc = reinterpret_cast<int32_t *>(h->d_arena + o_anc);
    *h->h_state = initial_state(h->cfg);
    bbox_unknown(*h->h_state);
    memset(h->h_frame, 0, sizeof(FrameRef));
    h->h_frame->active = 1;
    err = cudaMemcpyAsync(h->d_trk, &T, sizeof T, cudaMemcpyHostToDevice, h->stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(h->d_frame, h->h_frame, sizeof(FrameRef), cudaMemcpyHostToDevice, h->stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(T.state, h->h_state, sizeof(TrackerState), cudaMemcpyHostToDevice, h->stream);
    if (err == cudaSuccess) err = cudaMemsetAsync(h->d_ticket, 0, sizeof(uint32_t), h->stream);
    if (err == cudaSuccess) {
        iota_kernel<<<static_cast<unsigned>(std::min<int64_t>((count + 255) / 256, 4096)), 256, 0, h->stream>>>(T.anc,
                                                                                                           count);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaStreamSynchronize(h->stream);   // the stack copy of T goes out of scope
    h->grid = step_grid_size(h->prec, T.ntiles);
    if (err != cudaSuccess || h->grid < 1) {
        cudaGetLastError();
        shard_free(h);
        return PF_ERR_CUDA;
    }
    *out = h;
    return PF_OK;
}

extern "C" pf_status pf_shard_stats(pf_shard *h, double *out4) {
    if (!h || !out4) return PF_ERR_ARG;
    if (h->sticky != PF_OK) return PF_ERR_STATE;
    if (h->t < 1) return PF_ERR_STATE;
    cudaError_t err = cudaMemcpyAsync(h->h_state, h->h_trk.state, sizeof(TrackerState), cudaMemcpyDeviceToHost,
                                      h->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(h->stream);
    if (err != cudaSuccess) { cudaGetLastError(); return h->fail(PF_ERR_CUDA); }
    if (h->h_state->status & kStatusTimeout) return h->fail(PF_ERR_TIMEOUT);
    if (h->h_state->status & kStatusBounds) return h->fail(PF_ERR_STATE);
    out4[0] = h->h_state->M;
    out4[1] = h->h_state->S;
    out4[2] = h->h_state->est_x;
    out4[3] = h->h_state->est_y;
    return PF_OK;
}

extern "C" pf_status pf_shard_resample(pf_shard *h, const double *global4, int32_t last, void *send_x, void *send_y,
                                       int64_t send_capacity, int64_t *run_out) {
    if (!h || !global4 || !send_x || !send_y || !run_out || send_capacity < 0) return PF_ERR_ARG;
    if (h->sticky != PF_OK) return PF_ERR_STATE;
    if (h->t < 1) return PF_ERR_STATE;    // frame 0 resamples nothing
    const double gM = global4[0], gS = global4[1], lo = global4[2], hi = global4[3];
    if (!isfinite(gM) || !(gS > 0) || !(lo >= 0) || !(hi >= lo)) return PF_ERR_ARG;
    StepLaunch L = single_launch(h);
    L.shard = 1;
    L.shard_last = last ? 1 : 0;
    L.shard_lo = lo;
    L.shard_hi = hi;
    L.g_M = gM;
    // 1/S in the CDF's precision, as a single tracker saves it
    L.g_invS = h->prec == PF_REF64 ? 1.0 / gS : static_cast<double>(1.0f / static_cast<float>(gS));
    // the normalised CDF value where this shard starts: the arithmetic the shard before it
    // uses for its last element (PF_NORM of shard_hi, capped at 1)
    double c_lo;
    if (h->prec == PF_REF64) c_lo = std::min(lo * L.g_invS, 1.0);
    else c_lo = static_cast<double>(std::min(static_cast<float>(lo) * static_cast<float>(L.g_invS), 1.0f));
    if (launch_cdf(h->prec, L, h->grid, h->stream) != 0) { cudaGetLastError(); return h->fail(PF_ERR_CUDA); }
    const int in = static_cast<int>((h->t + 1) & 1);
    cudaError_t err = cudaMemsetAsync(h->d_run, 0, 3 * sizeof(int64_t), h->stream);
    if (err != cudaSuccess) { cudaGetLastError(); return h->fail(PF_ERR_CUDA); }
    if (launch_shard_expand(h->prec, h->h_trk.cdf, h->h_trk.px[in], h->h_trk.py[in], h->cfg.num_particles, h->n_global,
                            h->t, h->h_trk.key_lo, h->h_trk.key_hi, h->h_trk.tracker_id, c_lo, send_x, send_y,
                            send_capacity, h->d_run, reinterpret_cast<uint32_t *>(h->d_run + 2), h->stream) != 0) {
        cudaGetLastError();
        return h->fail(PF_ERR_CUDA);
    }
    err = cudaMemcpyAsync(h->h_run, h->d_run, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(h->stream);
    if (err != cudaSuccess) { cudaGetLastError(); return h->fail(PF_ERR_CUDA); }
    if (h->h_run[2] != 0) return PF_ERR_ARG;     // send_capacity is short of the run
    run_out[0] = h->h_run[0];
    run_out[1] = h->h_run[1];
    return PF_OK;
}

extern "C" pf_status pf_shard_step(pf_shard *h, const void *recv_x, const void *recv_y, const uint8_t *frame,
                                   int64_t pitch_bytes, int32_t frame_on_device) {
    if (!h || !frame || pitch_bytes < h->cfg.width || !frame_on_device) return PF_ERR_ARG;
    if (h->sticky != PF_OK) return PF_ERR_STATE;
    TraceRange tr("pf_shard_step");
    cudaError_t err = cudaSuccess;
    if (h->t > 0) {
        if (!recv_x || !recv_y) return PF_ERR_ARG;
        // the ancestors of the shard's slots become its previous frame (ancestors = identity)
        const int in = static_cast<int>((h->t + 1) & 1);
        const size_t nb = pos_bytes(h->prec) * static_cast<size_t>(h->cfg.num_particles);
        err = cudaMemcpyAsync(h->h_trk.px[in], recv_x, nb, cudaMemcpyDeviceToDevice, h->stream);
        if (err == cudaSuccess) err = cudaMemcpyAsync(h->h_trk.py[in], recv_y, nb, cudaMemcpyDeviceToDevice, h->stream);
        if (err != cudaSuccess) { cudaGetLastError(); return h->fail(PF_ERR_CUDA); }
    }
    StepLaunch L = single_launch(h);
    L.frame_override = frame;
    L.pitch_override = pitch_bytes;
    if (launch_pull(h->prec, L, h->grid, false, h->stream) != 0) { cudaGetLastError(); return h->fail(PF_ERR_CUDA); }
    h->t += 1;
    return PF_OK;
}

extern "C" int64_t pf_shard_frames_done(const pf_shard *h) { return h ? h->t : -1; }

extern "C" pf_status pf_shard_destroy(pf_shard *h) {
    shard_free(h);
    return PF_OK;
}
