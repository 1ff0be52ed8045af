// pf_noalloc.cu -- pf_step_frame_noalloc: one frame of the filter for callers that
// cannot allocate device memory.
//
// Some embedders cannot call cudaMalloc: a host program whose CUDA memory is owned and
// budgeted by another runtime (a graphics or inference engine that hands out buffers), a
// real-time loop that forbids allocation after start-up, or code running inside a
// stream-ordered section where an allocation would synchronise the device.  They can still
// provide their own input and output buffers; what the step needs beyond those (the
// decoupled-lookback descriptors, per-tile partial sums, counters and the tracker's
// descriptor) lives here, in a file-scope device array that exists in every GPU's memory
// as soon as the library is loaded and stays there until the process exits.
#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "pf.h"
#include "pf_internal.h"
#include "pf_host.h"

using namespace pfk;

namespace {

constexpr int64_t kMaxParticles = int64_t(1) << 22;
constexpr int kMaxTiles = static_cast<int>(kMaxParticles / (kTile / 2));   // a tile holds >= kTile / 2
constexpr int kMaxDevices = 64;
// tracker descriptor, state, frame and counters, then the per-tile descriptors and partials
constexpr size_t kScratchBytes = 8192 + (sizeof(LookbackDesc) + sizeof(TilePartial)) * size_t(kMaxTiles);

// The scratch array.  In host code its name is only a stand-in for the symbol; the
// device address comes from cudaGetSymbolAddress (per device).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Layout inside the scratch array.
struct ScratchLayout {
    size_t trk, state, frame, ticket, done, est, stat, look, part, end;
};

constexpr size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

constexpr ScratchLayout layout() {
    ScratchLayout L{};
    L.trk = 0;
    L.state = align256(L.trk + sizeof(TrackerDev));
    L.frame = align256(L.state + sizeof(TrackerState));
    L.ticket = align256(L.frame + sizeof(FrameRef));
    L.done = L.ticket + 16;
    L.est = L.done + 16;
    L.stat = L.est + 16;
    L.look = align256(L.stat + 16);
    L.part = align256(L.look + sizeof(LookbackDesc) * kMaxTiles);
    L.end = L.part + sizeof(TilePartial) * kMaxTiles;
    return L;
}
static_assert(layout().end <= kScratchBytes, "scratch layout exceeds the array");

// Writes the tracker descriptor, its state and the frame reference into the scratch array
// and clears what every step must find at zero there (the ticket, the tile counter, the
// lookback descriptors and tile partials of the nt tiles).  The three structures travel as
// kernel parameters, so no host buffer has to outlive the call.
__global__ void noalloc_setup_kernel(const TrackerDev T, const TrackerState st, const FrameRef fr,
                                     unsigned char *scr, int nt) {
    constexpr ScratchLayout LY = layout();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    if (i == 0) {
        *reinterpret_cast<TrackerDev *>(scr + LY.trk) = T;
        *reinterpret_cast<TrackerState *>(scr + LY.state) = st;
        *reinterpret_cast<FrameRef *>(scr + LY.frame) = fr;
    }
    uint4 *z = reinterpret_cast<uint4 *>(scr + LY.ticket);
    for (int k = i; k < static_cast<int>((LY.est - LY.ticket) / 16); k += stride) z[k] = make_uint4(0u, 0u, 0u, 0u);
    uint4 *look = reinterpret_cast<uint4 *>(scr + LY.look);
    for (int k = i; k < nt * static_cast<int>(sizeof(LookbackDesc) / 16); k += stride) look[k] = make_uint4(0u, 0u, 0u, 0u);
    uint4 *part = reinterpret_cast<uint4 *>(scr + LY.part);
    for (int k = i; k < nt * static_cast<int>(sizeof(TilePartial) / 16); k += stride) part[k] = make_uint4(0u, 0u, 0u, 0u);
}
static_assert(sizeof(LookbackDesc) % 16 == 0 && sizeof(TilePartial) % 16 == 0, "16-byte clears");
static_assert(layout().ticket % 16 == 0 && layout().est % 16 == 0 && layout().look % 16 == 0 &&
              layout().part % 16 == 0, "16-byte aligned scratch regions");

// True if the byte ranges [a, a + n) and [b, b + n) overlap.
bool overlaps(const void *a, const void *b, size_t n) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + n && y < x + n;
}

std::mutex g_lock;
unsigned char *g_scratch_dev[kMaxDevices] = {};
int g_grid[kMaxDevices][4] = {};

// Device address of the scratch array on the current device (looked up once per device).
pf_status scratch_for_current_device(int *dev_out, unsigned char **ptr_out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return PF_ERR_CUDA; }
    if (dev < 0 || dev >= kMaxDevices) return PF_ERR_ARG;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return PF_ERR_CUDA;
        }
        g_scratch_dev[dev] = static_cast<unsigned char *>(p);
    }
    *dev_out = dev;
    *ptr_out = g_scratch_dev[dev];
    return PF_OK;
}

}  // namespace

extern "C" pf_status pf_step_frame_noalloc(const pf_config *cfg, const pf_state_header *state_in,
                                           const void *x_in, const void *y_in, const void *l_in,
                                           const uint8_t *frame, int64_t pitch_bytes,
                                           void *x_out, void *y_out, void *l_out,
                                           pf_state_header *state_out, void *cuda_stream) {
    if (!cfg || !state_in || !frame || !x_out || !y_out || !l_out || !state_out) return PF_ERR_ARG;
    const pf_config &c = *cfg;
    if (c.width < 1 || c.width > 65535 || c.height < 1 || c.height > 65535) return PF_ERR_ARG;
    if (c.num_particles < 1 || c.num_particles > kMaxParticles) return PF_ERR_ARG;
    if (c.disk_radius < 0 || c.disk_radius > kMaxRadius) return PF_ERR_ARG;
    if (c.precision < PF_REF64 || c.precision > PF_BF16) return PF_ERR_ARG;
    if (!(c.sigma_x >= 0) || !(c.sigma_y >= 0) || !isfinite(c.sigma_x) || !isfinite(c.sigma_y)) return PF_ERR_ARG;
    if (!isfinite(c.init_x) || !isfinite(c.init_y) || fabs(c.init_x) > 1.0e6 || fabs(c.init_y) > 1.0e6) return PF_ERR_ARG;
    if (!isfinite(c.drift_x) || !isfinite(c.drift_y) || !isfinite(c.bg_level) || !isfinite(c.fg_level)) return PF_ERR_ARG;
    if (c.flags & ~PF_FLAG_ACCUM32) return PF_ERR_ARG;   // no debug arrays here
    if (c.resampler != PF_RESAMPLE_SYSTEMATIC && c.resampler != PF_RESAMPLE_STRATIFIED) return PF_ERR_ARG;
    if (c.resampler_steps != 0 || c.reserved != 0) return PF_ERR_ARG;
    if (pitch_bytes < c.width) return PF_ERR_ARG;
    const pf_state_header &h = *state_in;
    if (h.magic != 0x31534650u || h.precision != c.precision || h.num_particles != c.num_particles || h.t < 0)
        return PF_ERR_ARG;
    if (h.t > 0 && (!x_in || !y_in || !l_in || !(h.sum_e > 0) || !isfinite(h.max_l))) return PF_ERR_ARG;
    // the step moves particles in 16-byte vectors
    const auto misaligned = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0u; };
    if (misaligned(x_out) || misaligned(y_out) || misaligned(l_out)) return PF_ERR_ARG;
    if (h.t > 0 && (misaligned(x_in) || misaligned(y_in) || misaligned(l_in))) return PF_ERR_ARG;
    // the step gathers ancestors from the inputs while it writes the outputs: no buffer
    // may overlap another
    {
        const size_t nb = static_cast<size_t>(c.num_particles) * pos_bytes(c.precision);
        const void *bufs[6] = {x_out, y_out, l_out, x_in, y_in, l_in};
        const int nbuf = h.t > 0 ? 6 : 3;
        for (int a = 0; a < nbuf; ++a)
            for (int b = a + 1; b < nbuf; ++b)
                if (overlaps(bufs[a], bufs[b], nb)) return PF_ERR_ARG;
    }

    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    // the call waits for its step and reads the new state back: it cannot be captured
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) { cudaGetLastError(); return PF_ERR_CUDA; }
        if (cs != cudaStreamCaptureStatusNone) return PF_ERR_ARG;
    }
    int dev = 0;
    unsigned char *scr = nullptr;
    pf_status s = scratch_for_current_device(&dev, &scr);
    if (s != PF_OK) return s;
    constexpr ScratchLayout LY = layout();

    // descriptor of the tracker: the caller's buffers are the ping-pong slots of frame t
    const int64_t N = c.num_particles;
    const int tile = step_tile_size(c.precision, N);
    const int nt = static_cast<int>((N + tile - 1) / tile);
    if (nt > kMaxTiles) return PF_ERR_ARG;
    const int in = static_cast<int>((h.t + 1) & 1), out = static_cast<int>(h.t & 1);
    TrackerDev T;
    memset(&T, 0, sizeof T);
    fill_tracker_constants(c, T);
    T.tile_begin = 0; T.ntiles = nt; T.tile = tile; T.est_cap = 1;
    T.px[in] = const_cast<void *>(x_in); T.py[in] = const_cast<void *>(y_in); T.pl[in] = const_cast<void *>(l_in);
    T.px[out] = x_out; T.py[out] = y_out; T.pl[out] = l_out;
    T.look = reinterpret_cast<LookbackDesc *>(scr + LY.look);
    T.part = reinterpret_cast<TilePartial *>(scr + LY.part);
    T.done = reinterpret_cast<uint32_t *>(scr + LY.done);
    T.state = reinterpret_cast<TrackerState *>(scr + LY.state);
    T.est_ring = reinterpret_cast<double *>(scr + LY.est);
    T.stat_ring = reinterpret_cast<double *>(scr + LY.stat);

    // the scalars the step reads (frame 0: every particle at the initial position)
    TrackerState st;
    memset(&st, 0, sizeof st);
    st.t = h.t;
    st.epoch = 1;   // the lookback descriptors and tile partials are cleared below
    if (h.t == 0) {
        st.M = 0.0; st.S = 1.0;
        st.ax = st.nx = round_half_up(c.init_x);
        st.ay = st.ny = round_half_up(c.init_y);
        st.est_x = c.init_x; st.est_y = c.init_y;
    } else {
        st.M = h.max_l; st.S = h.sum_e;
        st.ax = h.anchor_x; st.ay = h.anchor_y; st.nx = h.next_anchor_x; st.ny = h.next_anchor_y;
        st.est_x = h.est_x; st.est_y = h.est_y;
    }
    st.invS = c.precision == PF_REF64 ? 1.0 / st.S : static_cast<double>(1.0f / static_cast<float>(st.S));
    bbox_unknown(st);   // (no tracker table here: every tile tabulates its own window)
    state_copies(st);
    FrameRef fr;
    memset(&fr, 0, sizeof fr);
    fr.base = frame; fr.pitch = pitch_bytes; fr.stride = 0; fr.active = 1;

    // Every call shares the scratch array and finds the previous call's contents in it:
    // the lookback descriptors, the tile partials (their words carry the launch counter,
    // which is 1 on every call), the tile counter and the ticket must start at zero.  One
    // small kernel writes the descriptor, state and frame reference (its parameters) and
    // clears those.
    noalloc_setup_kernel<<<8, 256, 0, stream>>>(T, st, fr, scr, nt);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return PF_ERR_CUDA;
    int grid;
    {
        std::lock_guard<std::mutex> guard(g_lock);
        if (!g_grid[dev][c.precision]) g_grid[dev][c.precision] = step_grid_size(c.precision, kMaxTiles);
        grid = g_grid[dev][c.precision];
    }
    if (grid < 1) return PF_ERR_CUDA;
    if (grid > nt) grid = nt;
    StepLaunch L;
    L.trk = reinterpret_cast<const TrackerDev *>(scr + LY.trk);
    L.states = T.state;
    L.frames = reinterpret_cast<const FrameRef *>(scr + LY.frame);
    L.tile_trk = nullptr;   // one tracker: every tile belongs to it
    L.tile_prefix = nullptr;
    L.slot_of = nullptr;
    L.est_out = nullptr;
    L.ticket = reinterpret_cast<uint32_t *>(scr + LY.ticket);
    L.ntrk = 1;
    L.total_tiles = nt;
    L.frame_override = nullptr;
    L.pitch_override = 0;
    if (launch_step(c.precision, L, grid, stream) != 0) { cudaGetLastError(); return PF_ERR_CUDA; }

    // the new state header: read back once the step has run (the call waits for it), with
    // the device status a failed wait or a checked build's index test left there
    {
        TrackerState res;
        err = cudaMemcpyAsync(&res, scr + LY.state, sizeof res, cudaMemcpyDeviceToHost, stream);
        if (err == cudaSuccess) err = cudaStreamSynchronize(stream);
        if (err != cudaSuccess) { cudaGetLastError(); return PF_ERR_CUDA; }
        if (res.status & kStatusTimeout) return PF_ERR_TIMEOUT;
        if (res.status & kStatusBounds) return PF_ERR_STATE;   // checked builds
        pf_state_header o;
        memset(&o, 0, sizeof o);
        o.magic = 0x31534650u;
        o.precision = c.precision;
        o.num_particles = N;
        o.t = res.t;
        o.max_l = res.M;
        o.sum_e = res.S;
        o.anchor_x = res.ax; o.anchor_y = res.ay;
        o.next_anchor_x = res.nx; o.next_anchor_y = res.ny;
        o.est_x = res.est_x; o.est_y = res.est_y;
        *state_out = o;
    }
    return PF_OK;
}
