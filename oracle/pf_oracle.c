/*
 * pf_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle of the per-frame
 * SIR (sequential importance resampling) step of the half-precision particle filter
 * for object tracking (Schieffer et al., arXiv 2308.00763).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the bench's
 * CPU-baseline leg load this library.  It shares no code, header, table, constant or
 * helper with the CUDA library; neither includes nor links the other.
 *
 * The step follows Sec. IV of the paper in the paper's order (Fig. 1 workflow):
 *   propagation  Eq. 1-2            orc_propagate
 *   likelihood   Eq. 3 (Sec. IV)      orc_likelihood_at / orc_likelihood_all
 *   max finding + weighting Eq. 5   orc_weights
 *   normalising (sum + estimate)    orc_normalise
 *   normalising (CDF, inclusive prefix sum)  orc_cdf
 *   systematic resampling (Sec. IV)  orc_resample_f64 / orc_resample_f32
 *     (naive form, points by division)  orc_resample_div_f64 / orc_resample_div_f32
 *   stratified resampling (Sec. III)  orc_stratified_offsets, orc_resample_strat_f64 / _f32
 *   multinomial resampling (Sec. IV) orc_resample_multi_f64 / _f32 (draws: orc_stratified_offsets)
 *   Gumbel-max resampling (Sec. IV)  orc_gumbel_f64 / _f32 (argmax of L + Gumbel variates)
 *   Metropolis resampling (Sec. III)  orc_metropolis_f64 / _f32 (B-step chains on exp(L))
 *   rejection resampling (Sec. III)   orc_rejection_f64 / _f32 (first candidate with u <= w/w_max)
 * Where the paper is silent the readings are (numbered as in the design notes):
 *   C1  Eq. 3 is summed over the template pixels and divided by 50*|D|.
 *   C2  template D = integer offsets with dx^2+dy^2 <= r^2 (centre included).
 *   C3  pixel of a position v: floor(v) + (v - floor(v) >= 0.5); x = column, y = row.
 *   C4  template pixels outside the frame are clamped to the nearest edge pixel.
 *   C5  motion: x += drift_x + sigma_x*n_x, y += drift_y + sigma_y*n_y (Eq. 1-2 with
 *       the drift and the standard deviations as parameters).
 *   C6  resampling every frame, so w_{t-1} = 1/N drops out of Eq. 5.
 *   C7  estimate = weighted mean of the propagated particles, before resampling.
 *   C8  systematic: one u0 per frame, u_j = (j + u0) * (1/N) in the CDF's precision,
 *       a_j = min{k : C_k >= u_j}, N-1 if there is none.
 *       Stratified (alternative scheme): u_j = (j + v_j) * (1/N), v_j independent.
 *       Multinomial (alternative scheme): u_j = v_j, N independent draws.
 *       Gumbel-max (alternative scheme): a_j = argmax_k L_k - ln(-ln u_jk), ties to the
 *       smallest k, N draws per offspring (tag 4 + 256 j).
 *       Metropolis (alternative scheme): a B-step chain from k = j, proposals uniform,
 *       accepted when ln u <= L_k' - L_k (tag 5 + 256 j, two steps per draw).
 *       Rejection (alternative scheme): candidates j, then uniform proposals, the first
 *       with ln u <= L_k - max L kept; R tries at most (tag 6 + 256 j, two tries per draw).
 *   C11 draws: Philox4x32-10 words -> 23-bit uniforms -> Box-Muller in FP64.
 *   C12 at t = 0 every ancestor sits at (init_x, init_y).
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written here
 * from that paper's description, keyed by the 64-bit seed with the counter
 * (index, frame t, tag, tracker id); tag 0 = propagation, 1 = resampling u0.  One
 * propagation block (four words) serves the particle pair (2i, 2i+1): counter index i,
 * words 0-1 for particle 2i and words 2-3 for particle 2i+1.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fPIC -shared (no FMA contraction,
 * so x86-64 and aarch64 produce the same bits).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#if defined(__FAST_MATH__)
#error "the oracle must not be built with -ffast-math"
#endif

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (SC'11, Sec. "Philox"): 10 rounds of two 32x32->64 multiplies,   */
/* the high halves xored with the other counter words and the round key; the key */
/* advances by the two Weyl constants between rounds.                             */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)mul0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)mul1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        if (round < 9) { k0 += weyl0; k1 += weyl1; }
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Philox draw for (seed, counter = (j, t, tag, tracker)). */
void orc_philox_draw(uint64_t seed, uint32_t j, uint32_t t, uint32_t tag, uint32_t tracker,
                     uint32_t out[4])
{
    uint32_t ctr[4] = { j, t, tag, tracker };
    uint32_t key[2] = { (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) };
    orc_philox4x32_10(ctr, key, out);
}

/* Uniform in (0, 1) from the top 23 bits of a word: ((w >> 9) + 1/2) * 2^-23.  The
 * value has at most 24 significant bits, so FP32 and FP64 hold it exactly (C11). */
double orc_uniform(uint32_t w)
{
    return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* Box-Muller transform of two uniforms into two independent N(0,1) draws, FP64.
 * The paper samples the transition noise in double precision (Sec. IV, after Eq. 2). */
void orc_box_muller(double ua, double ub, double *nx, double *ny)
{
    const double two_pi = 6.283185307179586476925286766559;
    double radius = sqrt(-2.0 * log(ua));
    double angle = two_pi * ub;
    *nx = radius * cos(angle);
    *ny = radius * sin(angle);
}

/* Batch forms for the tests (one call per array instead of one per element). */
void orc_philox_batch(int64_t n, const uint32_t *ctrs, uint64_t seed, uint32_t *out)
{
    uint32_t key[2] = { (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) };
    for (int64_t i = 0; i < n; ++i) orc_philox4x32_10(ctrs + 4 * i, key, out + 4 * i);
}

void orc_uniform_batch(int64_t n, const uint32_t *w, double *u)
{
    for (int64_t i = 0; i < n; ++i) u[i] = orc_uniform(w[i]);
}

void orc_box_muller_batch(int64_t n, const double *ua, const double *ub, double *nx, double *ny)
{
    for (int64_t i = 0; i < n; ++i) orc_box_muller(ua[i], ub[i], nx + i, ny + i);
}

/* The propagation draw of particle j at frame t (tag 0): block j/2, words 2(j%2), 2(j%2)+1. */
void orc_normal2(uint64_t seed, uint32_t j, uint32_t t, uint32_t tracker, double *nx, double *ny)
{
    uint32_t w[4];
    orc_philox_draw(seed, j >> 1, t, 0u, tracker, w);
    const uint32_t h = 2u * (j & 1u);
    orc_box_muller(orc_uniform(w[h]), orc_uniform(w[h + 1]), nx, ny);
}

void orc_normal2_batch(uint64_t seed, uint32_t t, uint32_t tracker, int64_t start, int64_t n,
                       double *nx, double *ny)
{
    for (int64_t i = 0; i < n; ++i)
        orc_normal2(seed, (uint32_t)(start + i), t, tracker, nx + i, ny + i);
}

/* The systematic-resampling offset u0 of frame t (tag 1, particle word 0). */
double orc_resample_u0(uint64_t seed, uint32_t t, uint32_t tracker)
{
    uint32_t w[4];
    orc_philox_draw(seed, 0u, t, 1u, tracker, w);
    return orc_uniform(w[0]);
}

/* ------------------------------------------------------------------------- */
/* Template and pixel rounding (C2, C3).                                       */
/* ------------------------------------------------------------------------- */
int orc_disk_count(int r)
{
    int n = 0;
    for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx)
            if (dx * dx + dy * dy <= r * r) ++n;
    return n;
}

int64_t orc_round_pixel(double v)
{
    double f = floor(v);
    return (int64_t)f + ((v - f) >= 0.5 ? 1 : 0);
}

void orc_round_pixel_batch(int64_t n, const double *v, int64_t *p)
{
    for (int64_t i = 0; i < n; ++i) p[i] = orc_round_pixel(v[i]);
}

static int64_t clamp_i64(int64_t v, int64_t lo, int64_t hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

/* ------------------------------------------------------------------------- */
/* Likelihood, Eq. 3 (reading C1): over every template pixel I around the       */
/* particle's pixel, sum (I - bg)^2 - (I - fg)^2 and divide by 50 * |D|.          */
/* bg = 100 and fg = 228 in the paper.  Literal per-pixel FP64 form.              */
/* ------------------------------------------------------------------------- */
double orc_likelihood_at(const uint8_t *frame, int W, int H, int64_t pitch, int r,
                         double bg, double fg, int64_t px, int64_t py)
{
    double num = 0.0;
    int count = 0;
    for (int dy = -r; dy <= r; ++dy) {
        for (int dx = -r; dx <= r; ++dx) {
            if (dx * dx + dy * dy > r * r) continue;
            int64_t row = clamp_i64(py + dy, 0, H - 1);
            int64_t col = clamp_i64(px + dx, 0, W - 1);
            double I = (double)frame[row * pitch + col];
            num += (I - bg) * (I - bg) - (I - fg) * (I - fg);
            ++count;
        }
    }
    return num / (50.0 * (double)count);
}

/* Plain integer sum of the template pixels: the second, independent calculation
 * that the exact-integer form of Eq. 3 is checked against. */
int64_t orc_disk_sum(const uint8_t *frame, int W, int H, int64_t pitch, int r,
                     int64_t px, int64_t py)
{
    int64_t s = 0;
    for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx) {
            if (dx * dx + dy * dy > r * r) continue;
            s += frame[clamp_i64(py + dy, 0, H - 1) * pitch + clamp_i64(px + dx, 0, W - 1)];
        }
    return s;
}

/* ------------------------------------------------------------------------- */
/* Per-particle work split over threads (results do not depend on the split).  */
/* ------------------------------------------------------------------------- */
typedef struct {
    int kind;                 /* 0 = propagate, 1 = likelihood */
    int64_t lo, hi;
    /* propagate */
    uint32_t t; uint64_t seed; uint32_t tracker;
    const double *xa, *ya; const int64_t *anc;
    double init_x, init_y, drift_x, drift_y, sigma_x, sigma_y;
    double *x, *y;
    /* likelihood */
    const double *xs, *ys; const uint8_t *frame; int W, H; int64_t pitch; int r;
    double bg, fg; double *L;
} orc_job;

static void run_job_range(const orc_job *jb)
{
    if (jb->kind == 0) {
        for (int64_t j = jb->lo; j < jb->hi; ++j) {
            double xa, ya;
            if (jb->anc) { xa = jb->xa[jb->anc[j]]; ya = jb->ya[jb->anc[j]]; }
            else { xa = jb->init_x; ya = jb->init_y; }
            double nx, ny;
            orc_normal2(jb->seed, (uint32_t)j, jb->t, jb->tracker, &nx, &ny);
            jb->x[j] = xa + jb->drift_x + jb->sigma_x * nx;
            jb->y[j] = ya + jb->drift_y + jb->sigma_y * ny;
        }
    } else {
        for (int64_t j = jb->lo; j < jb->hi; ++j) {
            int64_t px = orc_round_pixel(jb->xs[j]);
            int64_t py = orc_round_pixel(jb->ys[j]);
            jb->L[j] = orc_likelihood_at(jb->frame, jb->W, jb->H, jb->pitch, jb->r,
                                         jb->bg, jb->fg, px, py);
        }
    }
}

static void *job_thread(void *arg)
{
    run_job_range((const orc_job *)arg);
    return NULL;
}

static void run_jobs(const orc_job *proto, int64_t N, int nthreads)
{
    if (nthreads <= 1 || N < 4096) {
        orc_job jb = *proto; jb.lo = 0; jb.hi = N;
        run_job_range(&jb);
        return;
    }
    if (nthreads > 256) nthreads = 256;
    pthread_t tid[256];
    orc_job jobs[256];
    int started[256];
    int64_t chunk = (N + nthreads - 1) / nthreads;
    for (int i = 0; i < nthreads; ++i) {
        jobs[i] = *proto;
        jobs[i].lo = (int64_t)i * chunk < N ? (int64_t)i * chunk : N;
        jobs[i].hi = jobs[i].lo + chunk < N ? jobs[i].lo + chunk : N;
        started[i] = pthread_create(&tid[i], NULL, job_thread, &jobs[i]) == 0;
        if (!started[i]) run_job_range(&jobs[i]);
    }
    for (int i = 0; i < nthreads; ++i)
        if (started[i]) pthread_join(tid[i], NULL);
}

/* Propagation, Eq. 1-2 (reading C5, C12): the new particle j is drawn around its
 * ancestor a_j, x_j = x_{a_j} + drift_x + sigma_x * n_x (same for y).  anc == NULL
 * means frame 0: every ancestor sits at (init_x, init_y). */
void orc_propagate(int64_t N, uint32_t t, uint64_t seed, uint32_t tracker,
                   const double *xa, const double *ya, const int64_t *anc,
                   double init_x, double init_y, double drift_x, double drift_y,
                   double sigma_x, double sigma_y, double *x, double *y, int nthreads)
{
    orc_job jb;
    memset(&jb, 0, sizeof jb);
    jb.kind = 0; jb.t = t; jb.seed = seed; jb.tracker = tracker;
    jb.xa = xa; jb.ya = ya; jb.anc = anc;
    jb.init_x = init_x; jb.init_y = init_y; jb.drift_x = drift_x; jb.drift_y = drift_y;
    jb.sigma_x = sigma_x; jb.sigma_y = sigma_y; jb.x = x; jb.y = y;
    run_jobs(&jb, N, nthreads);
}

/* Likelihood of every particle, Eq. 3 at the rounded pixel (C3, C4). */
void orc_likelihood_all(int64_t N, const double *x, const double *y, const uint8_t *frame,
                        int W, int H, int64_t pitch, int r, double bg, double fg, double *L,
                        int nthreads)
{
    orc_job jb;
    memset(&jb, 0, sizeof jb);
    jb.kind = 1; jb.xs = x; jb.ys = y; jb.frame = frame; jb.W = W; jb.H = H;
    jb.pitch = pitch; jb.r = r; jb.bg = bg; jb.fg = fg; jb.L = L;
    run_jobs(&jb, N, nthreads);
}

/* ------------------------------------------------------------------------- */
/* Max finding and weighting, Eq. 5 with log-sum-exp (Sec. IV, numerical         */
/* stability): M = max_k L_k, e_k = exp(L_k - M).  Returns M. (C6)                */
/* ------------------------------------------------------------------------- */
double orc_weights(int64_t N, const double *L, double *e)
{
    double M = -INFINITY;
    for (int64_t k = 0; k < N; ++k)
        if (L[k] > M) M = L[k];
    for (int64_t k = 0; k < N; ++k)
        e[k] = exp(L[k] - M);
    return M;
}

/* Neumaier-compensated running sum, in index order. */
typedef struct { double sum, comp; } orc_ksum;

static void ksum_add(orc_ksum *s, double v)
{
    double t = s->sum + v;
    if (fabs(s->sum) >= fabs(v)) s->comp += (s->sum - t) + v;
    else s->comp += (v - t) + s->sum;
    s->sum = t;
}

static double ksum_value(const orc_ksum *s) { return s->sum + s->comp; }

/* Normalising: S = sum_k e_k and the state estimate (C7)
 * xhat = sum_k e_k x_k / S, yhat = sum_k e_k y_k / S.  Returns S. */
double orc_normalise(int64_t N, const double *e, const double *x, const double *y,
                     double *xhat, double *yhat)
{
    orc_ksum s = {0, 0}, sx = {0, 0}, sy = {0, 0};
    for (int64_t k = 0; k < N; ++k) {
        ksum_add(&s, e[k]);
        ksum_add(&sx, e[k] * x[k]);
        ksum_add(&sy, e[k] * y[k]);
    }
    double S = ksum_value(&s);
    *xhat = ksum_value(&sx) / S;
    *yhat = ksum_value(&sy) / S;
    return S;
}

/* Normalising, CDF: the normalised inclusive prefix sum, C_k = (sum_{i<=k} e_i) / S,
 * with the last entry set to exactly 1. */
void orc_cdf(int64_t N, const double *e, double S, double *C)
{
    orc_ksum p = {0, 0};
    for (int64_t k = 0; k < N; ++k) {
        ksum_add(&p, e[k]);
        C[k] = ksum_value(&p) / S;
    }
    if (N > 0) C[N - 1] = 1.0;
}

/* Systematic resampling (Sec. IV; reading C8), decided in FP64: the unit interval is
 * cut into N strata and stratum j is sampled at u_j = (j + u0) / N; its ancestor is
 * the first particle whose CDF value reaches u_j.  Linear scan with a moving pointer. */
void orc_resample_f64(int64_t N, const double *C, double u0, int64_t *a)
{
    double inv_n = 1.0 / (double)N;
    int64_t k = 0;
    for (int64_t j = 0; j < N; ++j) {
        double u = ((double)j + u0) * inv_n;
        while (k < N && C[k] < u) ++k;
        a[j] = k < N ? k : N - 1;
    }
}

/* The same decision taken in FP32, for a CDF held in FP32. */
void orc_resample_f32(int64_t N, const float *C, float u0, int64_t *a)
{
    volatile float inv_n = 1.0f / (float)N;  /* volatile: keep FP32 rounding explicit */
    int64_t k = 0;
    for (int64_t j = 0; j < N; ++j) {
        volatile float jf = (float)j;
        volatile float s = jf + u0;
        volatile float u = s * inv_n;
        while (k < N && C[k] < u) ++k;
        a[j] = k < N ? k : N - 1;
    }
}

/* Stratified resampling (Sec. III lists it with multinomial and systematic resampling as
 * the standard schemes): the same N strata, each sampled at its own offset, u_j =
 * (j + v_j) * (1/N).  Offset v_j of frame t is the uniform of word (j mod 4) of the
 * Philox draw (j / 4, t, tag 1, tracker), so v_0 is the systematic u0 of that frame. */
void orc_stratified_offsets(uint64_t seed, uint32_t t, uint32_t tracker, int64_t N, double *v)
{
    for (int64_t j = 0; j < N; ++j) {
        uint32_t w[4];
        orc_philox_draw(seed, (uint32_t)(j / 4), t, 1u, tracker, w);
        v[j] = orc_uniform(w[j % 4]);
    }
}

/* a_j = min{k : C_k >= u_j} (N - 1 if there is none), by bisection for every j, with
 * u_j = (j + v_j) * (1/N) in FP64. */
void orc_resample_strat_f64(int64_t N, const double *C, const double *v, int64_t *a)
{
    double inv_n = 1.0 / (double)N;
    for (int64_t j = 0; j < N; ++j) {
        double u = ((double)j + v[j]) * inv_n;
        int64_t lo = 0, hi = N;          /* first index in [lo, hi] with C >= u; N: none */
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (C[mid] >= u) hi = mid; else lo = mid + 1;
        }
        a[j] = lo < N ? lo : N - 1;
    }
}

/* The same decision taken in FP32, for a CDF held in FP32. */
void orc_resample_strat_f32(int64_t N, const float *C, const float *v, int64_t *a)
{
    volatile float inv_n = 1.0f / (float)N;
    for (int64_t j = 0; j < N; ++j) {
        volatile float jf = (float)j;
        volatile float s = jf + v[j];
        volatile float u = s * inv_n;
        int64_t lo = 0, hi = N;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (C[mid] >= u) hi = mid; else lo = mid + 1;
        }
        a[j] = lo < N ? lo : N - 1;
    }
}

/* Multinomial resampling (Sec. IV describes it as drawing each ancestor from the
 * categorical distribution of the normalised weights): offspring j takes the first
 * particle whose CDF value reaches an independent uniform v_j (the same Philox words as
 * the stratified offsets), N - 1 if there is none. */
void orc_resample_multi_f64(int64_t N, const double *C, const double *v, int64_t *a)
{
    for (int64_t j = 0; j < N; ++j) {
        int64_t lo = 0, hi = N;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (C[mid] >= v[j]) hi = mid; else lo = mid + 1;
        }
        a[j] = lo < N ? lo : N - 1;
    }
}

/* The same decision taken in FP32, for a CDF held in FP32. */
void orc_resample_multi_f32(int64_t N, const float *C, const float *v, int64_t *a)
{
    for (int64_t j = 0; j < N; ++j) {
        int64_t lo = 0, hi = N;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (C[mid] >= v[j]) hi = mid; else lo = mid + 1;
        }
        a[j] = lo < N ? lo : N - 1;
    }
}

/* Gumbel-max resampling, the log-domain alternative Sec. IV weighs against log-sum-exp:
 * with g_jk = -ln(-ln u_jk) independent standard Gumbel variates, offspring j takes
 * a_j = argmax_k (L_k + g_jk) over the unnormalised log weights L (the smallest k among
 * equal values).  The Gumbel-max property makes a_j a draw from the categorical law
 * exp(L_k) / sum_i exp(L_i) -- the multinomial draw, with no maximum, sum or CDF.
 * u_jk is the uniform of word (k mod 4) of the Philox draw (k / 4, t, 4 + 256 j,
 * tracker); j < 2^24.  N^2 draws, so for small trackers only. */
void orc_gumbel_f64(uint64_t seed, uint32_t t, uint32_t tracker, int64_t N, const double *L, int64_t *a)
{
    for (int64_t j = 0; j < N; ++j) {
        double best = 0.0;
        int64_t arg = -1;
        for (int64_t k = 0; k < N; ++k) {
            uint32_t w[4];
            orc_philox_draw(seed, (uint32_t)(k / 4), t, 4u + 256u * (uint32_t)j, tracker, w);
            double g = -log(-log(orc_uniform(w[k % 4])));
            double v = L[k] + g;
            if (arg < 0 || v > best) { best = v; arg = k; }
        }
        a[j] = arg;
    }
}

/* The same decisions taken in FP32 (L held in FP32, the variates from logf). */
void orc_gumbel_f32(uint64_t seed, uint32_t t, uint32_t tracker, int64_t N, const float *L, int64_t *a)
{
    for (int64_t j = 0; j < N; ++j) {
        float best = 0.0f;
        int64_t arg = -1;
        for (int64_t k = 0; k < N; ++k) {
            uint32_t w[4];
            orc_philox_draw(seed, (uint32_t)(k / 4), t, 4u + 256u * (uint32_t)j, tracker, w);
            volatile float u = (float)orc_uniform(w[k % 4]);
            volatile float e = -logf(u);
            volatile float g = -logf(e);
            volatile float v = L[k] + g;
            if (arg < 0 || v > best) { best = v; arg = k; }
        }
        a[j] = arg;
    }
}

/* Metropolis resampling (Sec. III cites it, with rejection resampling, as a scheme that
 * needs no global sum; Murray, Lee and Jacob, 2016): offspring j runs a Metropolis chain
 * of B steps over the particle indices with target exp(L_k), started at k = j.  Step b
 * proposes k' uniform on {0, ..., N-1} and moves there when u <= exp(L_k' - L_k), taken in
 * the log form ln u <= L_k' - L_k; a_j is the state after B steps.  Step b of offspring j
 * reads the Philox draw (b / 2, t, 5 + 256 j, tracker): word 2 (b mod 2) gives the
 * proposal k' = floor(w N / 2^32), word 2 (b mod 2) + 1 the uniform u; j < 2^24. */
void orc_metropolis_f64(uint64_t seed, uint32_t t, uint32_t tracker, int64_t N, const double *L, int B, int64_t *a)
{
    for (int64_t j = 0; j < N; ++j) {
        int64_t k = j;
        for (int b = 0; b < B; ++b) {
            uint32_t w[4];
            orc_philox_draw(seed, (uint32_t)(b / 2), t, 5u + 256u * (uint32_t)j, tracker, w);
            int64_t kp = (int64_t)(((uint64_t)w[2 * (b % 2)] * (uint64_t)N) >> 32);
            double u = orc_uniform(w[2 * (b % 2) + 1]);
            if (log(u) <= L[kp] - L[k]) k = kp;
        }
        a[j] = k;
    }
}

/* The same chains with the acceptance test in FP32 (L held in FP32, ln u from logf). */
void orc_metropolis_f32(uint64_t seed, uint32_t t, uint32_t tracker, int64_t N, const float *L, int B, int64_t *a)
{
    for (int64_t j = 0; j < N; ++j) {
        int64_t k = j;
        for (int b = 0; b < B; ++b) {
            uint32_t w[4];
            orc_philox_draw(seed, (uint32_t)(b / 2), t, 5u + 256u * (uint32_t)j, tracker, w);
            int64_t kp = (int64_t)(((uint64_t)w[2 * (b % 2)] * (uint64_t)N) >> 32);
            volatile float u = (float)orc_uniform(w[2 * (b % 2) + 1]);
            volatile float lu = logf(u);
            volatile float d = L[kp] - L[k];
            if (lu <= d) k = kp;
        }
        a[j] = k;
    }
}

/* Rejection resampling (Sec. III cites it beside Metropolis resampling; Murray, Lee and
 * Jacob, 2016): offspring j tests k = j first, then proposals k' uniform on
 * {0, ..., N-1}, and takes the first candidate k that passes u <= w_k / w_max, in the log
 * form ln u <= L_k - M with M = max L (so w_k / w_max = exp(L_k - M)).  Offspring j thus
 * keeps j with probability w_j / w_max at the first try and otherwise draws from the
 * categorical law p_k = exp(L_k) / sum exp(L) (the later tries are plain rejection
 * sampling): P(a_j = k) = (w_j / w_max) [k = j] + (1 - w_j / w_max) p_k, so particle k's
 * expected offspring count is N p_k, with less spread than multinomial.  Try i of
 * offspring j reads the Philox draw (i / 2, t, 6 + 256 j, tracker): word 2 (i mod 2) gives
 * the proposal (not used by try 0, which tests j itself), word 2 (i mod 2) + 1 the uniform
 * u.  After R tries without acceptance the offspring keeps the last candidate (R = 4096 in
 * the library: a truncation of probability (1 - S/N)^R, S = sum exp(L - M)); j < 2^24. */
void orc_rejection_f64(uint64_t seed, uint32_t t, uint32_t tracker, int64_t N, const double *L, double M, int R,
                       int64_t *a)
{
    for (int64_t j = 0; j < N; ++j) {
        int64_t k = j;
        for (int i = 0; i < R; ++i) {
            uint32_t w[4];
            orc_philox_draw(seed, (uint32_t)(i / 2), t, 6u + 256u * (uint32_t)j, tracker, w);
            if (i > 0) k = (int64_t)(((uint64_t)w[2 * (i % 2)] * (uint64_t)N) >> 32);
            if (log(orc_uniform(w[2 * (i % 2) + 1])) <= L[k] - M) break;
        }
        a[j] = k;
    }
}

/* The same tries with the test in FP32 (L and M held in FP32, ln u from logf). */
void orc_rejection_f32(uint64_t seed, uint32_t t, uint32_t tracker, int64_t N, const float *L, float M, int R,
                       int64_t *a)
{
    for (int64_t j = 0; j < N; ++j) {
        int64_t k = j;
        for (int i = 0; i < R; ++i) {
            uint32_t w[4];
            orc_philox_draw(seed, (uint32_t)(i / 2), t, 6u + 256u * (uint32_t)j, tracker, w);
            if (i > 0) k = (int64_t)(((uint64_t)w[2 * (i % 2)] * (uint64_t)N) >> 32);
            volatile float u = (float)orc_uniform(w[2 * (i % 2) + 1]);
            volatile float lu = logf(u);
            volatile float d = L[k] - M;
            if (lu <= d) break;
        }
        a[j] = k;
    }
}

/* The same systematic decisions with the stratum points formed by a division,
 * u_j = (j + u0) / N, and no saved reciprocal: the naive form of Sec. IV's performance
 * optimisation (the GPU's naive study build takes these decisions). */
void orc_resample_div_f64(int64_t N, const double *C, double u0, int64_t *a)
{
    int64_t k = 0;
    for (int64_t j = 0; j < N; ++j) {
        double u = ((double)j + u0) / (double)N;
        while (k < N && C[k] < u) ++k;
        a[j] = k < N ? k : N - 1;
    }
}

void orc_resample_div_f32(int64_t N, const float *C, float u0, int64_t *a)
{
    int64_t k = 0;
    for (int64_t j = 0; j < N; ++j) {
        volatile float jf = (float)j;
        volatile float s = jf + u0;
        volatile float nf = (float)N;
        volatile float u = s / nf;
        while (k < N && C[k] < u) ++k;
        a[j] = k < N ? k : N - 1;
    }
}

/* ------------------------------------------------------------------------- */
/* The whole tracker (Fig. 1): for t = 0..T-1 propagate, weigh, normalise,      */
/* estimate, resample.  Outputs per frame: estimate (x, y), M and S.             */
/* frames: T frames of H rows of `pitch` bytes, frame t at frames + t*frame_stride.*/
/* Returns 0, or -1 if memory could not be had.                                   */
/* ------------------------------------------------------------------------- */
int orc_run(const uint8_t *frames, int64_t frame_stride, int T, int W, int H, int64_t pitch,
            int64_t N, int r, double bg, double fg, double init_x, double init_y,
            double sigma_x, double sigma_y, double drift_x, double drift_y,
            uint64_t seed, uint32_t tracker, int nthreads, int resampler, int iters,
            double *est, double *M_out, double *S_out)
{
    double *xa = malloc((size_t)N * sizeof(double));
    double *ya = malloc((size_t)N * sizeof(double));
    double *x = malloc((size_t)N * sizeof(double));
    double *y = malloc((size_t)N * sizeof(double));
    double *L = malloc((size_t)N * sizeof(double));
    double *e = malloc((size_t)N * sizeof(double));
    double *C = malloc((size_t)N * sizeof(double));
    int64_t *a = malloc((size_t)N * sizeof(int64_t));
    double *v = resampler ? malloc((size_t)N * sizeof(double)) : NULL;
    int ok = xa && ya && x && y && L && e && C && a && (v || !resampler);
    if (ok) {
        for (int t = 0; t < T; ++t) {
            const uint8_t *frame = frames + (int64_t)t * frame_stride;
            orc_propagate(N, (uint32_t)t, seed, tracker, xa, ya, t > 0 ? a : NULL,
                          init_x, init_y, drift_x, drift_y, sigma_x, sigma_y, x, y, nthreads);
            orc_likelihood_all(N, x, y, frame, W, H, pitch, r, bg, fg, L, nthreads);
            double M = orc_weights(N, L, e);
            double xh, yh;
            double S = orc_normalise(N, e, x, y, &xh, &yh);
            est[2 * t] = xh; est[2 * t + 1] = yh;
            if (M_out) M_out[t] = M;
            if (S_out) S_out[t] = S;
            orc_cdf(N, e, S, C);
            if (resampler == 3) {
                orc_gumbel_f64(seed, (uint32_t)t, tracker, N, L, a);
            } else if (resampler == 4) {
                orc_metropolis_f64(seed, (uint32_t)t, tracker, N, L, iters, a);
            } else if (resampler == 5) {
                orc_rejection_f64(seed, (uint32_t)t, tracker, N, L, M, iters, a);
            } else if (resampler) {
                orc_stratified_offsets(seed, (uint32_t)t, tracker, N, v);
                if (resampler == 2) orc_resample_multi_f64(N, C, v, a);
                else orc_resample_strat_f64(N, C, v, a);
            } else {
                orc_resample_f64(N, C, orc_resample_u0(seed, (uint32_t)t, tracker), a);
            }
            double *sw;
            sw = xa; xa = x; x = sw;
            sw = ya; ya = y; y = sw;
        }
    }
    free(xa); free(ya); free(x); free(y); free(L); free(e); free(C); free(a); free(v);
    return ok ? 0 : -1;
}
