/*
 * pf.h -- C ABI of the GB300 (sm_103a) particle-filter library: the per-frame SIR
 * (sequential importance resampling) step of a video object tracker, after
 * Schieffer et al., "Boosting the Performance of Object Tracking with a
 * Half-Precision Particle Filter on GPU" (arXiv 2308.00763).
 *
 * The problem (Sec. I and Sec. IV): track one object in a monochrome video.  Each
 * frame, every particle is propagated around its ancestor (Eq. 1-2), scored against
 * the frame under a disk template (Eq. 3, in its overflow-safe scaled form Eq. 4 for
 * half precision), weighted by exp(L - max L) (Eq. 5, log-sum-exp), normalised, summed
 * into a cumulative distribution by an inclusive prefix sum, and resampled
 * systematically (Sec. IV, "Resampling").  The paper switches the whole filter between
 * double, single and half precision by a template argument (Sec. IV, "Implementation");
 * here the precision is a field of the configuration.
 *
 * Conventions for every entry point:
 *  - Pointers are plain host or device addresses, as each argument states; sizes are
 *    in bytes unless stated otherwise.  No entry point takes ownership of a caller's
 *    buffer.  Handles (pf_filter, pf_batch) are owned by the library and released only
 *    by their destroy call.
 *  - Every call returns a pf_status; nothing is thrown across the ABI.  A handle whose
 *    device work has failed (a CUDA error, or a device wait that gave up) keeps that
 *    status and answers PF_ERR_STATE to every later call except get/destroy.
 *  - Work is enqueued on the handle's CUDA stream and is asynchronous unless the entry
 *    point says it synchronises.  One host thread at a time per handle.
 *  - Frames: width x height uint8 pixels, row-major (x = column, y = row), rows
 *    pitch_bytes apart (pitch_bytes >= width).
 */
#ifndef PF_GB300_H
#define PF_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PF_OK = 0,
    PF_ERR_ARG = 1,        /* an argument is out of range or NULL */
    PF_ERR_OOM = 2,        /* device or pinned memory could not be allocated */
    PF_ERR_CUDA = 3,       /* a CUDA runtime call or kernel launch failed */
    PF_ERR_TIMEOUT = 4,    /* a bounded device-side wait gave up (results of that step are invalid) */
    PF_ERR_STATE = 5,      /* the handle failed earlier, or the call does not fit its state
                              (also: a checked build, -DPF_CHECKED, found an index out of range) */
    PF_ERR_ADMISSION = 6   /* serving: a stream was refused by the memory or compute budget */
} pf_status;

/* Arithmetic of the filter (Sec. IV: double / float / half specialisations). */
typedef enum {
    PF_REF64 = 0,  /* FP64 everywhere: the reference mode */
    PF_F32 = 1,    /* FP32 everywhere */
    PF_F16 = 2,    /* half2 propagation and likelihood (Eq. 4 form, half accumulation),
                      half positions as offsets from an integer anchor, FP32 weights, sums, CDF */
    PF_BF16 = 3    /* as PF_F16 in bfloat16, with the likelihood accumulated in FP32 */
} pf_precision;

/* Resampling scheme (pf_config.resampler).  SYSTEMATIC and STRATIFIED cut the unit
 * interval into N strata [j/N, (j+1)/N), draw one point u_j in each and give offspring j
 * the first particle whose
 * normalised CDF value reaches u_j (Sec. IV, "Resampling"; Sec. III names the standard
 * multinomial, stratified and systematic schemes).  The points are evaluated in the CDF's
 * precision exactly as ((A)j + v_j) * (A)(1/N), A = double (PF_REF64) or float.
 *   SYSTEMATIC: v_j = u0 for every j, u0 = uniform word 0 of Philox(0, t, 1, tracker_id)
 *               (the paper's scheme; the default).
 *   STRATIFIED: v_j independent, v_j = uniform word (j mod 4) of Philox(j / 4, t, 1,
 *               tracker_id), so v_0 = u0.  With a FP32 CDF it needs N <= 2^24 (beyond,
 *               (float)j rounds and the points would no longer be ordered).
 *   MULTINOMIAL: no strata: offspring j takes the first particle whose CDF value reaches
 *               u_j = v_j, the stratified offsets used as N independent uniforms (Sec. IV
 *               describes this categorical draw).  Two kernels per frame (the CDF is
 *               written to device memory, then every offspring searches it); trackers
 *               and batches only (pf_server_open and pf_step_frame_noalloc reject it).
 *   GUMBEL:     the same categorical draw in the log domain (the Gumbel-max alternative to
 *               log-sum-exp that Sec. IV weighs): offspring j takes the particle
 *               a_j = argmax_k (L_k + g_jk), ties to the smallest k, where L_k is the
 *               unnormalised log weight, g_jk = -ln(-ln u_jk) and u_jk = uniform word
 *               (k mod 4) of Philox(k / 4, t, 4 + 256 j, tracker_id); evaluated in FP64
 *               (PF_REF64) or FP32 (the others, L widened from its stored type).  No
 *               maximum, sum or CDF of the weights is needed for the draw, but it costs N^2
 *               variates a frame, so N <= 2^16 (PF_ERR_ARG beyond).  Two kernels per frame
 *               (the argmax, then the pull kernel); trackers and batches only, as
 *               MULTINOMIAL.  pf_get_debug(which = 1) answers PF_ERR_ARG (no CDF).
 *   METROPOLIS: Metropolis resampling (Sec. III cites it, after Murray, Lee and Jacob, as a
 *               scheme with no global sum): offspring j runs a chain of B =
 *               pf_config.resampler_steps steps over the particle indices with target
 *               exp(L_k), started at k = j; step b proposes k' = floor(w N / 2^32) and
 *               moves there when ln u <= L_k' - L_k, with w and u the words 2 (b mod 2)
 *               and 2 (b mod 2) + 1 of Philox(b / 2, t, 5 + 256 j, tracker_id) (u uniform
 *               as above); a_j is the state after B steps.  The test runs in FP64
 *               (PF_REF64) or FP32 (the others), as for GUMBEL.  Biased for small B (the
 *               chain has not mixed); no maximum, sum or CDF is needed for the draw and
 *               the cost is B steps per offspring at any N (N <= 2^24, PF_ERR_ARG beyond).
 *               Two kernels per frame (the chains, then the
 *               pull kernel); trackers and batches only; pf_get_debug(which = 1) answers
 *               PF_ERR_ARG.
 *   REJECTION:  rejection resampling (Sec. III cites it beside METROPOLIS): offspring j
 *               tests candidate j, then proposals k' = floor(w N / 2^32), and keeps the
 *               first candidate k with ln u <= L_k - M, M the maximum of L the previous
 *               step computed (w_k / w_max = exp(L_k - M)); try i reads words 2 (i mod 2)
 *               (proposal; unused by try 0) and 2 (i mod 2) + 1 (u) of Philox(i / 2, t,
 *               6 + 256 j, tracker_id).  Offspring j keeps j with probability w_j / w_max,
 *               else draws from the normalised weights, so expected offspring counts are
 *               N w_k / sum w.  At most R = pf_config.resampler_steps tries (0 = 4096,
 *               at most 65536); after R refusals the last candidate is kept.  Expected
 *               tries per offspring: N w_max / sum w.  Same precision, limits (N <= 2^24)
 *               and launches as METROPOLIS. */
typedef enum {
    PF_RESAMPLE_SYSTEMATIC = 0,
    PF_RESAMPLE_STRATIFIED = 1,
    PF_RESAMPLE_MULTINOMIAL = 2,
    PF_RESAMPLE_GUMBEL = 3,
    PF_RESAMPLE_METROPOLIS = 4,
    PF_RESAMPLE_REJECTION = 5
} pf_resampler;

/* pf_config.flags */
#define PF_FLAG_DEBUG_ARRAYS 0x1u  /* keep the last step's CDF and ancestor indices (pf_get_debug) */
#define PF_FLAG_ACCUM32      0x2u  /* PF_F16: accumulate the likelihood in FP32 instead of half */
#define PF_FLAG_TUNED        0x4u  /* take the launch shape pf_autotune cached for this shape bucket */

typedef struct {
    int32_t width, height;     /* frame size in pixels, each in [1, 65535] */
    int64_t num_particles;     /* N, in [1, 2^31 - 1] */
    int32_t disk_radius;       /* r, in [0, 64]: template = {(dx,dy): dx^2 + dy^2 <= r^2} */
    int32_t precision;         /* pf_precision */
    double  bg_level, fg_level;/* background / foreground intensity of Eq. 3 (100, 228) */
    double  init_x, init_y;    /* every particle starts here (pixel units) */
    double  sigma_x, sigma_y;  /* std of the transition noise, Eq. 1-2 (paper: 5, 2) */
    double  drift_x, drift_y;  /* mean displacement per frame, Eq. 1-2 (paper: 1, 2) */
    uint64_t seed;             /* Philox4x32-10 key */
    uint32_t tracker_id;       /* Philox counter word 3: separates trackers sharing a seed */
    uint32_t flags;            /* PF_FLAG_* */
    int32_t est_capacity;      /* frames of estimates kept on the device; 0 = 4096 */
    int32_t resampler;         /* pf_resampler (0 = systematic) */
    int32_t resampler_steps;   /* METROPOLIS: chain length B in [1, 4096], 0 = 64; REJECTION: tries
                                  R in [1, 65536], 0 = 4096.  Others: 0 */
    int32_t reserved;          /* must be 0 */
} pf_config;

typedef struct pf_filter pf_filter;
typedef struct pf_batch pf_batch;

/* Human-readable name of a status code (static storage; never NULL). */
const char *pf_status_string(pf_status s);

/* Create one tracker (Sec. IV, Fig. 1 "initialisation"): validates *cfg, allocates its
 * device buffers on the current CUDA device and binds it to `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream).  *out receives the handle.
 * Errors: PF_ERR_ARG (bad field, NULL pointer), PF_ERR_OOM, PF_ERR_CUDA. */
pf_status pf_create(const pf_config *cfg, void *cuda_stream, pf_filter **out);

/* One frame of the filter (Sec. IV, Fig. 1: propagation, likelihood, max finding,
 * weighting, normalising, resampling).  `frame` is a host pointer if frame_on_device
 * is 0 (copied to the library's device buffer on the handle's stream before the
 * call returns for pageable memory; pinned memory must stay unchanged until the step
 * has run) or a device pointer if 1 (must stay valid until the step has run).
 * Resampling of the previous frame's particles happens at the start of this step;
 * the estimate of this frame is available to pf_estimate afterwards.  Asynchronous.
 * Errors: PF_ERR_ARG, PF_ERR_STATE, PF_ERR_CUDA. */
pf_status pf_step_frame(pf_filter *f, const uint8_t *frame, int64_t pitch_bytes,
                        int32_t frame_on_device);

/* Run `count` frames in one call: frame i at frames + i * frame_stride (bytes), rows
 * pitch_bytes apart, all on the host (frames_on_device = 0) or all on the device (1).
 * Equivalent to `count` calls of pf_step_frame.  With device frames the `count` steps
 * are replayed from a CUDA graph captured on the first call with this count.  Host
 * frames (frame_stride >= pitch_bytes * height) are copied chunk by chunk into a
 * library ring of 16 frames on a copy stream while the previous chunk is stepped (each
 * chunk of up to 8 frames replayed from a graph); pageable frames may be reused when
 * the call returns, pinned frames once a synchronising call (pf_estimate) has returned.
 * Asynchronous. */
pf_status pf_run_frames(pf_filter *f, const uint8_t *frames, int64_t pitch_bytes,
                        int64_t frame_stride, int32_t count, int32_t frames_on_device);

/* State estimate of frame `frame_index`: the tracked object position that the paper
 * plots against the ground truth trajectory (Sec. V, "Verification & Accuracy Results",
 * Fig. 4), taken as the weighted mean of the propagated particles before resampling
 * (reading C7: the paper does not state which summary of the cloud it plots).  Synchronises the handle's stream; checks the sticky
 * device status.  Only the last est_capacity frames are kept.  x, y: host pointers.
 * Errors: PF_ERR_ARG (index not stepped yet or overwritten), PF_ERR_TIMEOUT,
 * PF_ERR_STATE, PF_ERR_CUDA. */
pf_status pf_estimate(pf_filter *f, int64_t frame_index, double *x, double *y);

/* Estimates of frames first .. first+count-1 into xy[2*count] (host), plus, if
 * max_and_sum is not NULL, (max L, sum of exp(L - max L)) of each frame into
 * max_and_sum[2*count].  Synchronises like pf_estimate. */
pf_status pf_estimates(pf_filter *f, int64_t first, int32_t count, double *xy,
                       double *max_and_sum);

/* Restart the tracker at frame 0 with every particle back at (init_x, init_y), as
 * after pf_create, without reallocating.  Enqueued on the handle's stream (asynchronous);
 * estimates of earlier frames become unavailable.  Errors: PF_ERR_STATE, PF_ERR_CUDA. */
pf_status pf_reset(pf_filter *f);

/* Number of frames stepped so far (host-side count; no synchronisation). */
int64_t pf_frames_done(const pf_filter *f);

/* Host-side counters of a handle or batch (no synchronisation): what was enqueued, not
 * what has completed. */
typedef struct {
    int64_t frames;            /* tracker-frames stepped (a batch: summed over its trackers) */
    int64_t step_launches;     /* frame steps enqueued (one per frame of the handle) */
    int64_t kernel_launches;   /* kernels enqueued, graph nodes included: per step 1 for the
                                  systematic and stratified trackers, 1 pull kernel for the
                                  others, plus 1 CDF kernel (multinomial) and 1 ancestor
                                  kernel per scheme present (Gumbel-max, Metropolis,
                                  rejection) */
    int64_t graph_launches;    /* CUDA graph replays (pf_run_frames, pf_batch_run) */
    int64_t host_frame_bytes;  /* frame bytes copied from host memory to the device */
    int32_t status;            /* the handle's sticky pf_status */
    int32_t reserved;
} pf_counters;
pf_status pf_get_counters(const pf_filter *f, pf_counters *out);

/* Release the handle and every device buffer it owns (synchronises its stream first).
 * The end of a tracking run (Sec. IV, Fig. 1: the filter runs frame by frame until the
 * video ends); the paper states no teardown, so this is the library's own.
 * NULL is accepted. */
pf_status pf_destroy(pf_filter *f);

/* Checkpoint.  The state that the next step reads: the particles of the last frame
 * (positions before resampling and their log-likelihoods) and the frame scalars.
 * Layout (all little-endian, host memory):
 *   pf_state_header, then x[N], y[N], L[N] in the precision's storage type:
 *   REF64: double, double, double   F32: float, float, float
 *   F16:   half,   half,   half     BF16: bfloat16 x3
 *   (F16/BF16 positions are offsets from the integer anchor (anchor_x, anchor_y)).
 * pf_get_state: with host_buf NULL, writes the size to *bytes; otherwise *bytes must
 * be at least that size.  Synchronises.  pf_set_state: replaces the state (same
 * precision and N required); the next step resamples from it. */
typedef struct {
    uint32_t magic;            /* 'PFS1' = 0x31534650 */
    int32_t  precision;
    int64_t  num_particles;
    int64_t  t;                /* index of the next frame to step (frames done) */
    double   max_l;            /* M = max L of the stored frame */
    double   sum_e;            /* S = sum exp(L - M) */
    double   anchor_x, anchor_y;       /* anchor of the stored positions (integers) */
    double   next_anchor_x, next_anchor_y; /* anchor the next step writes against */
    double   est_x, est_y;     /* estimate of the stored frame */
} pf_state_header;

pf_status pf_get_state(pf_filter *f, void *host_buf, size_t *bytes);
pf_status pf_set_state(pf_filter *f, const void *host_buf, size_t bytes);

/* Test hooks (flags & PF_FLAG_DEBUG_ARRAYS): after a step, `which` = 0 copies the
 * ancestor index a_j of every particle j of that step (int32[N]; undefined at frame
 * 0), `which` = 1 the CDF C_k of the previous frame as the step computed it (double[N]
 * for REF64, float[N] otherwise; PF_ERR_ARG for the schemes that build no CDF: Gumbel-max,
 * Metropolis, rejection), `which` = 2 the likelihood-table window of every tile of the
 * step (x0, y0, width, height in pixels as int32, width 0 when the tile built none; the
 * tracker has ntiles <= ceil(N / 1024) tiles, so `bytes` >= 16 * ceil(N / 1024) always
 * suffices; the 4-word entries of the ntiles tiles are written, the rest of the buffer is
 * left as it was).  Synchronises.  host_buf: host pointer of `bytes`.
 * Errors: PF_ERR_STATE (no debug arrays), PF_ERR_ARG, PF_ERR_CUDA. */
pf_status pf_get_debug(pf_filter *f, int32_t which, void *host_buf, size_t bytes);

/* Test hook: Philox4x32-10 on the device, the same generator the step uses: for each
 * of the n counters ctrs[4*i..4*i+3] (host) with key = seed, writes four words to
 * out[4*i..] (host).  Synchronises the legacy default stream. */
pf_status pf_debug_philox(const uint32_t *ctrs, int64_t n, uint64_t seed, uint32_t *out);

/* One frame of the filter for callers that cannot allocate device memory: an engine or
 * runtime that owns all CUDA memory and hands out buffers, a real-time loop that forbids
 * allocation after start-up, or code that must not synchronise the device the way an
 * allocation can.  The paper has no counterpart; this is a deployment form of
 * pf_step_frame.  The caller owns every buffer (device pointers): the previous frame's
 * particles x_in, y_in, l_in (ignored when state_in->t == 0) and the new frame's
 * x_out, y_out, l_out (N elements each, in the precision's storage type, 16-byte aligned;
 * F16/BF16 positions are offsets from the anchor in the header), and the frame (rows
 * pitch_bytes apart).  No two of the particle buffers may overlap (the step gathers
 * ancestors from the inputs while it writes the outputs; PF_ERR_ARG otherwise).
 * state_in (host) carries the scalars of the previous frame in the pf_get_state header
 * layout (t = 0: a fresh tracker); state_out (host, required) receives the new frame's
 * scalars (its t is state_in->t + 1, its est_x/est_y the estimate of this frame): the
 * call waits for the step to finish on cuda_stream and reads them back, with any error the
 * device recorded (PF_ERR_TIMEOUT: a bounded wait gave up).
 * Everything else the step needs (lookback descriptors, per-tile sums, counters, the
 * tracker descriptor) lives in one array (about 170 KiB) in the library's device memory, present
 * on every GPU from the moment the library is loaded until the process exits; it limits
 * num_particles to 2^22 (PF_ERR_ARG beyond).  The call waits for its step and reads the
 * state back, so it cannot be captured into a CUDA graph (PF_ERR_ARG while cuda_stream is
 * capturing).  All calls share the array; a
 * small kernel of each call writes the descriptor and clears what must start at zero;
 * calls whose GPU work overlaps (other streams, other threads) race on it and must be
 * serialised by the caller.  No device or pinned memory is allocated.
 * Errors: PF_ERR_ARG, PF_ERR_CUDA, PF_ERR_TIMEOUT. */
pf_status pf_step_frame_noalloc(const pf_config *cfg, const pf_state_header *state_in,
                                const void *x_in, const void *y_in, const void *l_in,
                                const uint8_t *frame, int64_t pitch_bytes,
                                void *x_out, void *y_out, void *l_out,
                                pf_state_header *state_out, void *cuda_stream);

/* Test hook for failure detection: runs the step kernel's bounded lookback wait on a
 * descriptor that nobody publishes, giving up after spin_limit polls (1 .. 2^20); writes
 * the resulting status bits to *status_out (host) and returns PF_ERR_TIMEOUT when the wait
 * gave up, as it must.  The device stays usable afterwards.  Synchronises. */
pf_status pf_debug_wait_timeout(uint32_t spin_limit, uint32_t *status_out);

/* ---------------------------------------------------------------- one tracker on several GPUs
 * A tracker of N particles sharded by particles across R ranks, one GPU per rank: rank q
 * holds the contiguous particles [first_q, first_q + count_q) (pf_shard_partition).  The
 * per-frame step (Sec. IV, Fig. 1) couples particles only through the previous frame's
 * maximum log-likelihood M and weight sum S (Eq. 5 and the normalising kernel), the
 * inclusive prefix of the weights that resampling searches (Sec. IV, "Resampling") and the
 * ancestors themselves, so a frame of the sharded filter is, on every rank:
 *   1. pf_shard_stats: the shard's (M_q, S_q, est_x_q, est_y_q) of its last frame; the
 *      caller all-gathers them and forms, in rank order and identically on every rank,
 *      the global M = max M_q, the rescaled totals s_q = S_q exp(M_q - M), S = sum s_q,
 *      P_q = sum of s_r for r < q, and the frame's estimate sum s_q est_q / S;
 *   2. pf_shard_resample: the shard's particles are the ancestors of the contiguous
 *      offspring run [j0, j1) of the global systematic strata u_j = (j + u0) / N (reading
 *      C8); their positions are written in offspring order;
 *   3. the caller's all-to-all delivers to every rank the ancestor positions of its own
 *      slots [first_q, first_q + count_q), in order; pf_shard_step propagates them (draws
 *      keyed by the global particle index, Eq. 1-2), scores them on the frame (Eq. 3) and
 *      forms the shard's statistics.
 * Frame 0 has no steps 1-3: every particle starts at init_x, init_y.  The result is the
 * unsharded filter's method (the CDF is summed in a different order, so its last bits
 * differ).  REF64 and F32 shards, systematic resampling; positions travel as absolute
 * coordinates in the precision's type (double / float).  All calls on one handle run on its
 * stream; pf_shard_stats and pf_shard_resample synchronise it.  The paper tracks on one GPU;
 * this splitting is the library's.  Errors: PF_ERR_ARG, PF_ERR_OOM, PF_ERR_CUDA,
 * PF_ERR_STATE (failed handle, or a call out of order), PF_ERR_TIMEOUT. */
typedef struct pf_shard pf_shard;
/* Rank `rank`'s particles of an n_global-particle tracker over nranks ranks: first (even)
 * and count; the last rank takes the remainder.  n_global >= 2 nranks.  No device needed. */
pf_status pf_shard_partition(int64_t n_global, int32_t nranks, int32_t rank, int64_t *first, int64_t *count);
/* Create rank `rank`'s shard of the tracker *cfg (cfg->num_particles = N, the whole
 * tracker; precision PF_REF64 or PF_F32; resampler SYSTEMATIC; flags 0) on the current
 * device, bound to cuda_stream. */
pf_status pf_shard_create(const pf_config *cfg, int32_t rank, int32_t nranks, void *cuda_stream, pf_shard **out);
/* out4[0..3] = (M_q, S_q, est_x_q, est_y_q) of the shard's last stepped frame (host).
 * Synchronises.  PF_ERR_STATE before the first step. */
pf_status pf_shard_stats(pf_shard *h, double *out4);
/* Resample the shard's previous frame against the global weights: global4 = (M, S, P_q,
 * P_(q+1)) of that frame (host; P_(q+1) = S on the last rank, which passes last = 1).  The
 * ancestor position of every offspring j of the shard's run [run_out[0], run_out[1]) is
 * written to send_x / send_y[j - run_out[0]] (device, the precision's type, capacity
 * send_capacity elements; PF_ERR_ARG if short).  Consecutive ranks' runs meet; the first
 * starts at 0 and the last ends at N.  Synchronises.  PF_ERR_STATE at frame 0. */
pf_status pf_shard_resample(pf_shard *h, const double *global4, int32_t last, void *send_x, void *send_y,
                            int64_t send_capacity, int64_t *run_out);
/* Step the shard's slots on `frame` (a device pointer, rows pitch_bytes apart;
 * frame_on_device must be 1): from frame 1 on, recv_x / recv_y (device, count_q elements)
 * are the ancestor positions of slots first_q .. first_q + count_q - 1.  Asynchronous. */
pf_status pf_shard_step(pf_shard *h, const void *recv_x, const void *recv_y, const uint8_t *frame,
                        int64_t pitch_bytes, int32_t frame_on_device);
/* Frames stepped so far (host-side count). */
int64_t pf_shard_frames_done(const pf_shard *h);
/* Release the shard (synchronises its stream).  NULL is accepted. */
pf_status pf_shard_destroy(pf_shard *h);

/* ---------------------------------------------------------------- batches
 * Many independent trackers (different N, frame sizes, radii, seeds), stepped together
 * by one persistent segmented launch per frame.  All trackers of a batch share one
 * precision.  Frames: frames[i] is tracker i's frame (device pointers), rows
 * pitches[i] bytes apart; a tracker whose active_mask[i] is 0 is not stepped (its
 * frame pointer may be NULL).  active_mask NULL = all active. */
pf_status pf_batch_create(const pf_config *cfgs, int32_t n, void *cuda_stream, pf_batch **out);
pf_status pf_batch_step(pf_batch *b, const uint8_t *const *frames, const int64_t *pitches,
                        const uint8_t *active_mask);
/* Resident videos: tracker i reads its next frame at videos[i] (device), later frames
 * frame_strides[i] bytes apart, rows pitches[i] bytes apart (every video must hold all
 * the frames that pf_batch_run will step).  Asynchronous. */
pf_status pf_batch_set_videos(pf_batch *b, const uint8_t *const *videos, const int64_t *pitches,
                              const int64_t *frame_strides);
/* Step every tracker `count` frames through its resident video: one launch per frame,
 * replayed from a CUDA graph captured on the first call with this count.  Asynchronous. */
pf_status pf_batch_run(pf_batch *b, int32_t count);
/* Restart every tracker at frame 0 (as after pf_batch_create); resident videos restart
 * at their first frame.  Asynchronous. */
pf_status pf_batch_reset(pf_batch *b);
/* Counters of a batch (see pf_counters). */
pf_status pf_batch_get_counters(const pf_batch *b, pf_counters *out);

/* Estimates of frame `frame_index` of every tracker into xy[2*n] (host); trackers that
 * have not stepped that frame get NaN.  Synchronises. */
pf_status pf_batch_estimates(pf_batch *b, int64_t frame_index, double *xy);
pf_status pf_batch_destroy(pf_batch *b);

/* ---------------------------------------------------------------- autotuning
 * Launch shapes of the step: the tile (particles of the previous frame per CTA task, a
 * multiple of 8 from 1024 to 4096; 0 = the default rule), the likelihood window policy
 * (0 adaptive, 1 always 3.5 sigma, 2 always the full draw range) and the CTAs per SM
 * (0 = as many as fit, else at most this many).  They change no formula, but the tile
 * partitions the FP scan and so the rounding of the CDF.
 *
 * pf_autotune times candidate shapes for one configuration on the caller's resident video
 * (n_frames frames of rows pitch_bytes apart, frame_stride bytes apart, on the device)
 * with `copies` trackers of that configuration in one batch (1 = the tracker alone; more
 * = throughput with the device full, as in a batch), and caches the fastest for the
 * configuration's shape bucket: (precision, floor(log2 N), the larger sigma in quarter
 * pixels, disk radius, floor(log2 (width x height)), the device's SM count).  Trackers
 * created with PF_FLAG_TUNED take their bucket's cached
 * shape (the default shape if none), so equal configurations tile alike alone and in a
 * batch.  The cache lives in the process (pf_tuning_clear empties it).  Synchronises. */
typedef struct {
    int32_t tile;
    int32_t window;
    int32_t ctas_per_sm;
    int32_t reserved;           /* 0 */
} pf_tuning;

pf_status pf_autotune(const pf_config *cfg, int32_t copies, const uint8_t *video, int64_t pitch_bytes,
                      int64_t frame_stride, int32_t n_frames, pf_tuning *best, double *best_us_per_frame);
/* The same sweep with every candidate applied to a whole batch (trackers cfgs[0..n) over
 * their resident videos, as pf_batch_set_videos takes them): the fastest shape is cached
 * for every bucket of the batch. */
pf_status pf_autotune_batch(const pf_config *cfgs, int32_t n, const uint8_t *const *videos, const int64_t *pitches,
                            const int64_t *frame_strides, int32_t n_frames, pf_tuning *best,
                            double *best_us_per_frame);
/* The cached shape of cfg's bucket; PF_ERR_STATE if none. */
pf_status pf_tuning_lookup(const pf_config *cfg, pf_tuning *out);
/* Cache a shape for cfg's bucket (checked as pf_autotune's candidates are). */
pf_status pf_tuning_store(const pf_config *cfg, const pf_tuning *t);
pf_status pf_tuning_clear(void);

/* ---------------------------------------------------------------- serving
 * Continuous batching over many camera streams whose frames arrive over time.  The
 * paper tracks one video; this is the deployment form of the same per-frame step.
 *
 * A server owns one device arena of hbm_budget_bytes, carved per stream (particles of
 * both ping-pong slots, lookback descriptors, tile partials, and a queue of
 * queue_depth frames for streams fed from host memory).  pf_server_open admits a stream
 * while its bytes fit the arena AND the admitted demand (sum of N * fps over open
 * streams) stays within headroom * capacity particle-steps/s; otherwise it returns
 * PF_ERR_ADMISSION and the caller may retry once streams close.  Every stream keeps its
 * particles on the device from open to close.
 *
 * pf_server_tick launches, for each precision with queued frames, one step over every
 * stream of that precision that has a frame queued (its oldest one), on that precision's
 * own CUDA stream: streams join and leave the batch from one tick to the next, launches
 * of FP16 and FP32 streams overlap on the device, and up to max_in_flight launches per
 * precision are queued behind one another.  A stream's result does not depend on which
 * other streams share its launches (every tracker's arithmetic reads only its own state).
 * Completions are signalled by a host callback at the end of each launch;
 * pf_server_poll harvests them: estimates, and per frame the latency from its arrival
 * time to the callback (arrival times are on pf_server_now's clock).
 *
 * Threading: one host thread drives a server.  Errors: PF_ERR_ARG, PF_ERR_OOM,
 * PF_ERR_CUDA, PF_ERR_ADMISSION (stream refused, or the stream's frame queue is full),
 * PF_ERR_STATE (closed stream or failed server), PF_ERR_TIMEOUT (a step gave up; the
 * server is failed afterwards). */
typedef struct pf_server pf_server;

typedef struct {
    int64_t hbm_budget_bytes;   /* device memory for all streams (> 0) */
    double  capacity;           /* particle-steps/s the device serves; 0 = no compute budget */
    double  headroom;           /* admitted demand <= headroom * capacity (0 = 1.0) */
    int32_t max_streams;        /* open streams at once (>= 1) */
    int32_t queue_depth;        /* frames per stream queued or in flight (>= 1) */
    int32_t max_in_flight;      /* launches per precision in flight (1..8; 0 = 2) */
    int32_t reserved;           /* 0 */
} pf_server_config;

typedef struct {
    int64_t streams_open, streams_admitted, streams_rejected;
    int64_t frames_submitted, frames_rejected, frames_done;
    int64_t launches;
    double  particle_steps;     /* sum of N over completed frames */
    double  latency_p50_ms, latency_p99_ms, latency_max_ms;   /* arrival -> estimate available */
    double  first_launch_s, last_done_s;   /* pf_server_now times of the first launch / last completion */
    int64_t hbm_in_use, hbm_peak;
    double  demand;             /* admitted sum of N * fps */
} pf_server_stats;

/* seconds on a monotonic clock (the clock of arrival times and latencies) */
double pf_server_now(void);
pf_status pf_server_create(const pf_server_config *cfg, pf_server **out);
/* Admit a stream (cfg->est_capacity = results kept on the host, 0 = 64; debug flags are
 * not allowed).  host_frames: 1 if its frames will come from host memory (reserves the
 * frame queue in the arena), 0 for device frames.  *stream_id >= 0 on success. */
pf_status pf_server_open(pf_server *s, const pf_config *cfg, double fps, int32_t host_frames,
                         int32_t *stream_id);
/* Queue the stream's next frame (frame index = submission order).  Device frames
 * (frame_on_device = 1) are read in place and must stay valid until the frame completes;
 * host frames are copied into the stream's queue (asynchronously; the caller's buffer
 * may be reused once this returns if it is pageable, after the frame completes if it is
 * pinned).  arrival_time_s < 0 means now. */
pf_status pf_server_submit(pf_server *s, int32_t stream_id, const uint8_t *frame, int64_t pitch_bytes,
                           int32_t frame_on_device, double arrival_time_s);
/* Launch every precision's ready streams; *frames_launched (may be NULL) counts them. */
pf_status pf_server_tick(pf_server *s, int32_t *frames_launched);
/* Harvest completed launches; *frames_completed (may be NULL) counts their frames. */
pf_status pf_server_poll(pf_server *s, int32_t *frames_completed);
/* Launch and complete everything queued (blocking). */
pf_status pf_server_drain(pf_server *s);
/* Estimate of frame `frame_index` of a stream (the last est_capacity completed frames are
 * kept); PF_ERR_STATE if it has not completed or was dropped from the ring. */
pf_status pf_server_result(pf_server *s, int32_t stream_id, int64_t frame_index, double *x, double *y);
/* Frames of the stream completed so far. */
int64_t pf_server_frames_done(const pf_server *s, int32_t stream_id);
/* Close a stream: its in-flight frames complete first, queued ones are dropped; its
 * memory and compute budget return to the server. */
pf_status pf_server_close(pf_server *s, int32_t stream_id);
pf_status pf_server_get_stats(pf_server *s, pf_server_stats *out);
pf_status pf_server_destroy(pf_server *s);
/* Bytes a stream of this configuration takes from the arena (no device needed). */
pf_status pf_server_stream_bytes(const pf_config *cfg, int32_t host_frames, int32_t queue_depth,
                                 int64_t *bytes);

/* Trace replay: the server's request loop.  Events in time order: kind 0 opens trace
 * stream `stream` (cfg, fps; its frames are device frames), kind 1 submits a device frame
 * to it, kind 2 closes it (after its queued frames are served).  A stream refused at
 * open drops its frames (counted as rejected); in real time a full queue drops the frame,
 * otherwise the replay waits for room.  realtime = 1 processes every event at its
 * time (seconds from the start of the replay) while ticking and polling continuously;
 * realtime = 0 takes events as fast as the loop runs.  Returns after every event is
 * processed and every launched frame has completed; streams left open stay open. */
typedef struct {
    double time_s;
    int32_t kind;               /* 0 open, 1 frame, 2 close */
    int32_t stream;             /* trace stream index, 0 <= stream < n_streams */
    const uint8_t *frame;       /* kind 1 */
    int64_t pitch_bytes;        /* kind 1 */
    const pf_config *cfg;       /* kind 0 */
    double fps;                 /* kind 0 */
} pf_trace_event;
pf_status pf_server_replay(pf_server *s, const pf_trace_event *events, int64_t n_events,
                           int32_t n_streams, int32_t realtime);

#ifdef __cplusplus
}
#endif

#endif /* PF_GB300_H */
