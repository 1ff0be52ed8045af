// pf_internal.h -- data shared by the host runtime and the sm_103a kernels.
//
// Layout in HBM (one tracker; a batch is an array of these):
//   positions  x[2][N], y[2][N]   ping-pong: step t reads slot (t+1)&1, writes slot t&1
//   likelihood L[2][N]            same ping-pong
//     REF64: double  F32: float  F16: __half  BF16: __nv_bfloat16 (positions are offsets
//     from an integer anchor in F16/BF16)
//   per tile  LookbackDesc[ntiles]  decoupled-lookback status of the CDF scan
//             TilePartial[ntiles]   (max L, sum e, sum e*dx, sum e*dy) of the tile's outputs
//   per tracker TrackerState      frame counter, M, S, 1/S, anchors, last estimate, status
//               est ring [cap][2], stat ring [cap][2] (M, S) in double
#pragma once
#include <stdint.h>

namespace pfk {

// Threads per CTA of the step kernel: 512 (measured best on GB300 for large trackers).
// Other builds (-DPF_STEP_THREADS=128/256/1024) exist for the thread-block study only.
#ifndef PF_STEP_THREADS
#define PF_STEP_THREADS 512
#endif
constexpr int kThreads = PF_STEP_THREADS;
static_assert(kThreads == 128 || kThreads == 256 || kThreads == 512 || kThreads == 1024,
              "the step kernel is built for 128, 256, 512 or 1024 threads per CTA");
constexpr int kItems = 8;                 // CDF elements per thread
constexpr int kTile = kThreads * kItems;  // largest tile (particles of the resampled frame)
constexpr int kMaxRadius = 64;
// Pixels of a likelihood table (a tile's table in shared memory, and a tracker's table in
// device memory, which tiles copy into theirs).
constexpr int kTableMax = kTile < 4096 ? kTile : 4096;

// Resampling schemes (pf_config.resampler).
constexpr int kResampleSystematic = 0;
constexpr int kResampleStratified = 1;
constexpr int kResampleMultinomial = 2;   // CDF by the step kernel, offspring by the pull kernel
constexpr int kResampleGumbel = 3;        // ancestors by the Gumbel-max kernel, offspring by the pull kernel
constexpr int kResampleMetropolis = 4;    // ancestors by the Metropolis kernel, offspring by the pull kernel
constexpr int kResampleRejection = 5;     // ancestors by the rejection kernel, offspring by the pull kernel
// One shard of a tracker sharded by particles (pf_shard_*; not a pf_config value): the
// ancestors' positions arrive from the other ranks into the previous-frame slots, so the
// ancestors are the identity (T.anc[k] = k) and the pull kernel takes the offspring.
constexpr int kResampleShard = 6;
constexpr int64_t kGumbelMaxN = 1ll << 16; // N^2 draws a frame
constexpr int64_t kMetropolisMaxN = 1ll << 24;   // offspring index in the Philox tag
constexpr int kMetropolisMaxSteps = 4096;
constexpr int kMetropolisDefaultSteps = 64;
constexpr int kRejectionMaxTries = 65536;
constexpr int kRejectionDefaultTries = 4096;

// Schemes whose ancestors an ancestor kernel writes to T.anc before the pull kernel runs.
__host__ __device__ constexpr bool ancestors_given(int resampler) {
    return resampler == kResampleGumbel || resampler == kResampleMetropolis || resampler == kResampleRejection ||
           resampler == kResampleShard;
}

// Device status bits (sticky, per tracker).
constexpr uint32_t kStatusTimeout = 0x1u;
constexpr uint32_t kStatusBounds = 0x2u;    // checked builds: an index left its array (the access was redirected)

// Lookback descriptor of one tile: its aggregate and its inclusive prefix, each an exact
// 128-bit fixed-point value (value * 2^kFixShift; the inter-tile prefix then does not
// depend on the order in which a tile collects its predecessors' aggregates).  Each value
// is split into three 64-bit words (48 + 48 + 32 payload bits) whose top 16 bits carry a
// tag of the launch (the tracker's epoch).  A word is written once per launch by a single
// 64-bit store, so a reader that finds the current tag in all three words of a value holds
// the whole value: neither side needs a fence.  Layout: w[0..1] aggregate words 0-1,
// w[2..3] inclusive words 0-1 (16-byte aligned pairs), w[4] aggregate word 2, w[5]
// inclusive word 2.
struct alignas(16) LookbackDesc {
    uint64_t w[6];
};

// Per-tile (max L, sum exp(L - max), sum exp(L - max) * dx, * dy).  REF64 stores four
// doubles (published by an acquire-release count); the FP32/FP16/BF16 kernels store four
// 64-bit words (tag << 32 | float bits), the tag being the launch counter, so the tile
// that completes the tracker can wait for each word without any fence.
struct alignas(16) TilePartial {
    union {
        double d[4];
        uint64_t w[4];
    };
    // bounding box of the tile's new positions (x0, x1, y0, y1, absolute pixel units): four
    // tagged words (tag << 32 | float bits), as the FP32 statistics
    uint64_t b[4];
};

struct alignas(16) TrackerState {
    int64_t t;             // index of the frame the next step processes
    uint32_t epoch;        // launch counter of this tracker (lookback flag tag), never reset
    uint32_t status;       // sticky kStatus* bits
    double M;              // max L of frame t-1
    double S;              // sum exp(L - M) of frame t-1
    double invS;           // 1 / S
    double ax, ay;         // integer anchor of the stored positions (frame t-1)
    double nx, ny;         // integer anchor the next step writes against
    double est_x, est_y;   // estimate of frame t-1
    // the same scalars for the FP32 kernels (no FP64 instruction on their path)
    float M_f, invS_f;
    int32_t axi, ayi, nxi, nyi;
    // bounding box of the stored positions (frame t-1; absolute pixel units), which sizes
    // the tracker's likelihood table of the next step; NaN when unknown
    float bb_x0, bb_x1, bb_y0, bb_y1;
};

struct FrameRef {
    const uint8_t *base;   // frame pointer (device)
    int64_t pitch;         // bytes between rows
    int64_t stride;        // if nonzero, frame of step t is base + t * stride
    int32_t active;        // 0: tracker not stepped this launch
    int32_t ring;          // if nonzero (with stride): frame of step t is base + (t % ring) * stride
};

struct TrackerDev {
    int64_t N;
    int32_t W, H;
    int32_t r, D;              // radius and |D|
    int32_t tile_begin, ntiles;
    uint32_t key_lo, key_hi, tracker_id, flags;
    int32_t est_cap;
    int32_t tile;              // particles per tile (multiple of 8, <= kTile)
    // likelihood constants: L = c1 * (2 s - c2 * D) / den  (exact-integer form of Eq. 3)
    double c1, c2, den;
    float kappa, bg_f, fg_f, pad1;   // Eq. 4 scaled form: kappa = 1 / sqrt(50 |D|)
    double init_x, init_y, sigma_x, sigma_y, drift_x, drift_y;
    double inv_n;              // 1.0 / N
    float inv_n_f;             // 1.0f / (float)N
    int32_t resampler;         // pf_resampler
    int32_t steps;             // Metropolis: chain length B; rejection: tries R
    // FP32 copies for the FP32 kernels
    float init_xf, init_yf, drift_xf, drift_yf, sigma_xf, sigma_yf;
    float c1f, c2Df, denf;
    int32_t window;            // likelihood window: 0 adaptive, 1 always 3.5 sigma, 2 always the full draw range
    int64_t j_base;            // global index of particle 0 (a shard of a sharded tracker; even), else 0
    void *px[2], *py[2], *pl[2];
    int32_t *dbg_anc;          // NULL unless PF_FLAG_DEBUG_ARRAYS
    void *dbg_cdf;
    int32_t *dbg_win;          // NULL unless PF_FLAG_DEBUG_ARRAYS: each tile's table window [4 * ntiles]
    void *cdf;                 // multinomial: the normalised CDF of the previous frame [N] (FP64 / FP32)
    int32_t *anc;              // Gumbel-max, Metropolis, rejection: the ancestor of every offspring [N]
    LookbackDesc *look;
    TilePartial *part;
    // The tracker's likelihood table of the current step, kTableMax cells of one 64-bit word
    // (launch tag << 32 | payload: the integer disk sum of Eq. 3, or the bits of the half
    // form of Eq. 4); null = every tile builds its own table.
    uint64_t *gtab;
    uint32_t *done;
    TrackerState *state;
    double *est_ring;          // [est_cap][2]
    double *stat_ring;         // [est_cap][2] = (M, S)
};

// Launch of one step over a batch of trackers of one precision.
// The launch steps ntrk trackers; launch position p (0 <= p < ntrk) is the tracker in
// slot slot_of[p] of the descriptor and state arrays (slot p if slot_of is null).
struct StepLaunch {
    const TrackerDev *trk;     // device array indexed by slot
    TrackerState *states;      // device array indexed by slot (trk[s].state == states + s)
    const FrameRef *frames;    // device array [ntrk], by launch position
    const int32_t *tile_trk;   // device array [total_tiles]: launch position of each tile, or null
    const int32_t *tile_prefix;  // device array [ntrk + 1]: first tile of each position (when
                                 // tile_trk is null and ntrk > 1: positions found by bisection)
    const int32_t *slot_of;    // device array [ntrk], or null
    double *est_out;           // device array [2 * ntrk], or null: each position's new estimate
    uint32_t *ticket;          // device counter, 0 between launches
    int32_t ntrk;
    int32_t total_tiles;
    const uint8_t *frame_override;  // single tracker: frame pointer passed by the call
    int64_t pitch_override;
    // A shard's CDF launch (pf_shard_resample): the global M and 1/S replace the tracker's
    // own, the shard's prefix starts at shard_lo and its last element is pinned to shard_hi
    // (to 1 on the last shard).  shard = 0 for every other launch.
    int32_t shard = 0, shard_last = 0;
    double shard_lo = 0.0, shard_hi = 0.0, g_M = 0.0, g_invS = 0.0;
};

// Host entry points into the kernel translation unit.
int launch_step(int precision, const StepLaunch &L, int grid, void *stream);
// The pull family's kernels after launch_step on the same stream: the multinomial
// trackers' CDF kernel (when with_cdf), then the pull kernel (the offspring of the
// multinomial, Gumbel-max, Metropolis and rejection trackers; the last three read the
// ancestors that launch_gumbel / launch_metropolis / launch_rejection wrote, enqueued
// before it).
int launch_pull(int precision, const StepLaunch &L, int grid, bool with_cdf, void *stream);
// The CDF kernel alone (a shard's resampling).
int launch_cdf(int precision, const StepLaunch &L, int grid, void *stream);
// A shard's offspring run: the counts J_k = #{j : u_j <= C_k} over the global strata
// u_j = (j + u0) / N_global (u0 of frame t - 1) for the shard's CDF C[0..n), and the
// ancestor position of every offspring j of its run [J(c_lo), J(C[n-1])) written to
// sx / sy[j - J(c_lo)] (at most cap); run[0..1] = the run; status |= 1 if cap is short.
int launch_shard_expand(int precision, const void *cdf, const void *x, const void *y, int64_t n, int64_t n_global,
                        int64_t t, uint32_t key_lo, uint32_t key_hi, uint32_t tracker, double c_lo, void *sx,
                        void *sy, int64_t cap, int64_t *run, uint32_t *status, void *stream);

// An ancestor kernel over the trackers in slots[0 .. ntrk-1]: CTA b works on tracker g with
// cta_prefix[g] <= b < cta_prefix[g + 1], offspring (b - cta_prefix[g]) * (offspring per
// CTA) onwards.  A tracker at frame 0, with a failed step, or inactive in frames[] is
// skipped.
constexpr int kGumbelOffspring = 8;       // Gumbel-max: offspring per CTA
constexpr int kGumbelThreads = 256;
constexpr int kMetropolisThreads = 256;   // Metropolis: one offspring per thread
constexpr int kRejectionThreads = 256;    // rejection: threads per CTA
constexpr int kRejectionOffspring = 2048; // rejection: offspring per CTA (a pool its threads share)
struct AncestorLaunch {
    const TrackerDev *trk;     // device array indexed by slot
    const FrameRef *frames;    // device array indexed by slot
    const int32_t *slots;      // device array [ntrk]
    const int32_t *cta_prefix; // device array [ntrk + 1]
    int32_t ntrk;
    int32_t total_ctas;
};
int launch_gumbel(int precision, const AncestorLaunch &G, void *stream);
int launch_metropolis(int precision, const AncestorLaunch &G, void *stream);
int launch_rejection(int precision, const AncestorLaunch &G, void *stream);
int step_grid_size(int precision, int total_tiles);
// Particles per tile for a tracker of n particles.  A tracker of at least half a device
// of full tiles (SMs x CTAs per SM x kTile / 2 particles) takes the smallest multiple of
// 8 that splits it into a whole number of waves of the device's resident CTAs, so every
// tile carries the same load (between kTile / 2 and kTile); a smaller tracker takes
// kTile.  A function of (precision, n, device model) only, so a tracker tiles the same
// alone, in a batch and through the allocation-free entry point.
int step_tile_size(int precision, int64_t n);
int launch_debug_philox(const uint32_t *d_ctrs, int64_t n, uint64_t seed, uint32_t *d_out,
                        void *stream);
int launch_wait_probe(void *d_desc, void *d_state, uint32_t limit, void *stream);

}  // namespace pfk
