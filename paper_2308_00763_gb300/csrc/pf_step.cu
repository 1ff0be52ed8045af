// pf_step.cu -- the fused per-frame SIR step for sm_103a.
//
// One launch per frame for a whole batch of trackers.  A tile is kTile consecutive
// particles k of one tracker's previous frame.  Per tile (dynamic ticket order):
//   1. resampling of the previous frame (Sec. IV, "Normalizing" and "Resampling"):
//      e_k = exp(L_k - M) (Eq. 5 with the max of the previous step), a block scan, and a
//      decoupled lookback over the tracker's earlier tiles give the inclusive prefix
//      P_k; C_k = P_k * (1/S) (the reciprocal saved by the previous step); the strata
//      j with C_{k-1} < u_j <= C_k are the offspring of k.  The tile's offspring form a
//      contiguous range of j, and their ancestors all lie in the tile, so the gather of
//      ancestor positions is a read of the tile's own particles staged in shared memory.
//   2. propagation (Eq. 1-2) of every offspring j with Philox draws keyed by (j, t),
//   3. likelihood (Eq. 3; Eq. 4 scaled half form in F16/BF16) on the new frame.  The
//      likelihood is a function of the particle's pixel only, so each tile first tabulates
//      it in shared memory over the window its offspring can reach (the ancestors'
//      bounding box widened by the drift and the largest draw the 23-bit Box-Muller can
//      produce), from a copy of the frame region staged in shared memory, and each
//      offspring reads its pixel's value; a pixel outside the window is evaluated directly
//      from global memory by the same arithmetic in the same order, so the two routes
//      give identical bits.
//   4. per-tile (max L, sum e, sum e*dx, sum e*dy), merged with rescaling,
//   5. the tile that completes a tracker merges its tiles' partials in index order:
//      M, S, 1/S and the estimate of the frame (the weighted mean of the propagated
//      particles).
// Frame t = 0 has no resampling: every particle starts at the initial position.
//
// Multinomial trackers (Sec. IV: each ancestor drawn from the categorical distribution of
// the weights) are not in the step kernel's launch; they take two other launches per
// frame (the same code in other modes): the CDF kernel runs phase 1 up to the CDF and writes it to
// T.cdf; the pull kernel then gives each offspring j the first particle whose CDF value
// reaches an independent uniform v_j (a binary search over T.cdf), gathers the ancestors'
// positions of its tile's offspring into shared memory, sizes the likelihood window by
// them and runs phases 2-5 as the step kernel does.  Gumbel-max trackers (the log-domain
// form of the same draw, Sec. IV), Metropolis and rejection trackers (Sec. III) skip the CDF
// kernel: the pull kernel reads the ancestors their kernel (pf_gumbel.cu, pf_metropolis.cu,
// pf_rejection.cu) wrote to T.anc instead of searching.
//
// Scan boundaries.  The prefix between tiles is an exact 128-bit fixed-point sum of
// the tiles' aggregates, so every tile obtains the same boundary value whichever
// predecessors its lookback visits.  Inside a tile the prefix is an FP scan made
// non-decreasing by a running max and clamped to the exact value at the tile's end.
// Hence C is non-decreasing, the strata ranges of consecutive tiles meet exactly, and
// every j is written by exactly one tile.
#include <cuda_runtime.h>
#include <float.h>
#include <stddef.h>
#include <math.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "pf_device.cuh"
#include "pf_internal.h"

// The pull kernel's offspring have no likelihood table (window width 0), so its bounds
// tests against the window compare unsigned values with a constant 0.
#pragma nv_diag_suppress 186

namespace pfk {

namespace {

constexpr int kWarps = kThreads / 32;
constexpr int kRoiMax = 2 * kTableMax;     // staged frame pixels (window + template margin)
constexpr int kMapMax = 2 * kTile;         // offspring of a tile served by the ancestor map
constexpr uint32_t kSpinLimit = 1u << 22;  // bounded waits: ~1 s with backoff
// Half-width of the likelihood window in standard deviations of the transition noise.
// Every draw is below sqrt(-2 ln 2^-24) = 5.77 in magnitude (kDrawMax, rounded up).  When
// that window has more cells than the block has threads, a window of 3.5 sigma is used:
// a tile's few offspring beyond it (probability 4.7e-4 per coordinate) are cheaper to
// evaluate directly (same arithmetic, same bits) than a window twice as wide.
constexpr float kDrawMax = 5.7683f;
constexpr float kWindowSigmas = 3.5f;

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t atom_add_acq_rel(uint32_t *p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ bool timed_out(const TrackerState *st) {
    return (ld_relaxed_u32(&st->status) & kStatusTimeout) != 0u;
}

// Checked builds (-DPF_CHECKED): every index below that is in range by construction is
// tested; one out of range raises the tracker's bounds bit and is redirected to element 0
// (the host then reports the step as failed).  Other builds use the index as it is.
#ifdef PF_CHECKED
__device__ __forceinline__ int checked_index(int i, int n, TrackerState *st) {
    if (static_cast<unsigned>(i) >= static_cast<unsigned>(n)) {
        atomicOr(&st->status, kStatusBounds);
        return 0;
    }
    return i;
}
#define PF_IDX(i, n) checked_index((i), (n), st)
#else
#define PF_IDX(i, n) (i)
#endif

// The normalised CDF value of a prefix P: P * (1/S) with the reciprocal saved by the
// previous step (the paper's saved constant); the naive study build (-DPF_NAIVE_RESAMPLE)
// divides by S for every element instead.
#ifdef PF_NAIVE_RESAMPLE
#define PF_NORM(P) div_rn((P), Sdiv)
#else
#define PF_NORM(P) mul_rn((P), invS)
#endif

// ---- lookback descriptor words (see LookbackDesc): 16-bit launch tag | 48-bit payload
constexpr uint64_t kPayload48 = (1ull << 48) - 1ull;

__device__ __forceinline__ uint64_t desc_tag(uint32_t ep) {   // never 0 (cleared memory)
    return static_cast<uint64_t>(ep % 65535u + 1u) << 48;
}

__device__ __forceinline__ void st_relaxed_v2(uint64_t *p, uint64_t a, uint64_t b) {
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t a) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(a) : "memory");
}
__device__ __forceinline__ void ld_relaxed_v2(const uint64_t *p, uint64_t &a, uint64_t &b) {
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}

// Publish a tile's aggregate (which = 0) or inclusive prefix (which = 1).
__device__ __forceinline__ void desc_publish(LookbackDesc *d, int which, U128 v, uint64_t tag) {
    const uint64_t w0 = (v.lo & kPayload48) | tag;
    const uint64_t w1 = (((v.lo >> 48) | (v.hi << 16)) & kPayload48) | tag;
    const uint64_t w2 = (v.hi >> 32) | tag;
    st_relaxed_v2(&d->w[2 * which], w0, w1);
    st_relaxed_u64(&d->w[4 + which], w2);
}

__device__ __forceinline__ U128 desc_value(uint64_t w0, uint64_t w1, uint64_t w2) {
    U128 v;
    v.lo = (w0 & kPayload48) | (w1 << 48);
    v.hi = ((w1 & kPayload48) >> 16) | ((w2 & kPayload48) << 32);
    return v;
}

// Wait (bounded) until a predecessor tile has published this launch's inclusive prefix
// (returns 2) or aggregate (returns 1), with its value in v.  Returns 0 on timeout (and
// raises the tracker's timeout bit).
__device__ uint32_t wait_desc(const LookbackDesc *d, uint64_t tag, TrackerState *st, U128 &v,
                              uint32_t limit = kSpinLimit) {
    uint32_t ns = 8;
    for (uint32_t it = 0; it < limit; ++it) {
        // all six words in one round trip (the predecessor has usually published only its
        // aggregate when the tiles of a wave look back together)
        uint64_t a0, a1, i0, i1, w4, w5;
        ld_relaxed_v2(&d->w[0], a0, a1);
        ld_relaxed_v2(&d->w[2], i0, i1);
        ld_relaxed_v2(&d->w[4], w4, w5);
        const uint64_t hm = ~kPayload48;
        if ((i0 & hm) == tag && (i1 & hm) == tag && (w5 & hm) == tag) { v = desc_value(i0, i1, w5); return 2u; }
        if ((a0 & hm) == tag && (a1 & hm) == tag && (w4 & hm) == tag) { v = desc_value(a0, a1, w4); return 1u; }
        if ((it & 1023u) == 1023u && timed_out(st)) return 0u;   // another wait already gave up
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
    }
    atomicOr(&st->status, kStatusTimeout);
    return 0u;
}

__device__ __forceinline__ uint32_t atom_add_relaxed(uint32_t *p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.relaxed.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Tile partials of the FP32/FP16/BF16 kernels: 32-bit launch tag | float bits per word.
__device__ __forceinline__ uint64_t partial_tag(uint32_t ep) {   // never 0 (cleared memory)
    return static_cast<uint64_t>(ep % 0x7fffffffu + 1u) << 32;
}

// Wait (bounded) until the words of a tile partial (statistics, and the bounding box when
// the launch tracks it) carry this launch's tag; on timeout the tracker's timeout bit is
// raised and the words read last are returned.
__device__ void wait_partial(const TilePartial *p, uint64_t tag, TrackerState *st, uint64_t (&q)[8], bool with_box,
                             uint32_t limit = kSpinLimit) {
    uint32_t ns = 8;
    const uint64_t hm = 0xffffffff00000000ull;
    q[4] = q[5] = q[6] = q[7] = tag;
    for (uint32_t it = 0; it < limit; ++it) {
        ld_relaxed_v2(&p->w[0], q[0], q[1]);
        ld_relaxed_v2(&p->w[2], q[2], q[3]);
        if (with_box) {
            ld_relaxed_v2(&p->b[0], q[4], q[5]);
            ld_relaxed_v2(&p->b[2], q[6], q[7]);
        }
        if ((q[0] & hm) == tag && (q[1] & hm) == tag && (q[2] & hm) == tag && (q[3] & hm) == tag &&
            (q[4] & hm) == tag && (q[5] & hm) == tag && (q[6] & hm) == tag && (q[7] & hm) == tag)
            return;
        if ((it & 1023u) == 1023u && timed_out(st)) return;
        __nanosleep(ns);
        if (ns < 64) ns <<= 1;
    }
    atomicOr(&st->status, kStatusTimeout);
}

// exp(d) for d <= 0 with the two exact shortcuts: exp(0) = 1, and 0 below the point
// where the precision underflows to zero anyway.
__device__ __forceinline__ double exp_le0(double d) {
    return d == 0.0 ? 1.0 : (d < -746.0 ? 0.0 : exp(d));
}
__device__ __forceinline__ float exp_le0(float d) {
    return d == 0.0f ? 1.0f : (d < -104.0f ? 0.0f : expf(d));
}
// The FP16/BF16 filters weigh with the hardware exp2 approximation (their likelihoods
// carry ~11 bits); the scan and the statistics use the same function, so they agree.
template <bool kFast, typename A> __device__ __forceinline__ A wexp(A d) { return exp_le0(d); }
template <> __device__ __forceinline__ float wexp<true, float>(float d) {
    return d == 0.0f ? 1.0f : (d < -104.0f ? 0.0f : __expf(d));
}

template <typename A>
struct Stats {
    A m, s, sx, sy;
};

// Merge of two partial (max, sums) with rescaling to the larger max.  Symmetric:
// stats_merge(a, b) and stats_merge(b, a) give the same bits (no fused multiply-add).
template <bool F, typename A>
__device__ __forceinline__ Stats<A> stats_merge(const Stats<A> &a, const Stats<A> &b) {
    const A m = a.m > b.m ? a.m : b.m;
    if (m == neg_inf<A>()) return a;
    const A sa = (a.m == neg_inf<A>()) ? static_cast<A>(0) : wexp<F>(a.m - m);
    const A sb = (b.m == neg_inf<A>()) ? static_cast<A>(0) : wexp<F>(b.m - m);
    Stats<A> r;
    r.m = m;
    r.s = add_rn(mul_rn(a.s, sa), mul_rn(b.s, sb));
    r.sx = add_rn(mul_rn(a.sx, sa), mul_rn(b.sx, sb));
    r.sy = add_rn(mul_rn(a.sy, sa), mul_rn(b.sy, sb));
    return r;
}

// Two particles at once (a particle whose flag is false is skipped).  The rescale to a new
// maximum is applied without a branch: when the maximum does not move the factor is
// wexp(0) = 1 exactly (and 1 while no particle has been seen), so the sums are unchanged,
// the same bits as skipping it.
template <bool F, typename A>
__device__ __forceinline__ void stats_add2(Stats<A> &a, bool v0, A L0, A dx0, A dy0, bool v1, A L1, A dx1, A dy1) {
    const A l0 = v0 ? L0 : neg_inf<A>(), l1 = v1 ? L1 : neg_inf<A>();
    const A mx = l0 > l1 ? l0 : l1;
    const A nm = mx > a.m ? mx : a.m;
    const A sc = (nm == neg_inf<A>()) ? static_cast<A>(1)
                                      : ((a.m == neg_inf<A>()) ? static_cast<A>(0) : wexp<F>(a.m - nm));
    a.s *= sc; a.sx *= sc; a.sy *= sc;
    a.m = nm;
    const A e0 = v0 ? wexp<F>(l0 - a.m) : static_cast<A>(0);
    const A e1 = v1 ? wexp<F>(l1 - a.m) : static_cast<A>(0);
    a.s += e0 + e1;
    a.sx += e0 * dx0 + e1 * dx1;
    a.sy += e0 * dy0 + e1 * dy1;
}

// Pixel of a position (reading C3): floor(v) + (v - floor(v) >= 0.5).  For |v| below
// 2^22 (float) or 2^51 (double) this equals floor(v + 0.5): adding 1/2 is exact unless
// it crosses into the next binade, which happens only when the fraction is >= 1/2 and
// then rounds to the same integer.  Positions are first clamped to +-2^20, far outside
// any frame (template pixels are clamped to the frame, reading C4).
__device__ __forceinline__ int pixel_of(float v) {
    return __float2int_rd(fminf(fmaxf(v, -1048576.0f), 1048576.0f) + 0.5f);
}
__device__ __forceinline__ int pixel_of(double v) {
    return __double2int_rd(fmin(fmax(v, -1048576.0), 1048576.0) + 0.5);
}

// kItems consecutive elements between memory and registers as 16-byte vectors (kItems *
// sizeof(T) is a multiple of 16 for every element type here; the address is 16-byte
// aligned).  The elements are unpacked from (packed into) the vector words with bit
// operations on constant indices, so the register arrays never need an address (an
// array whose address is taken lives in local memory).
__device__ __forceinline__ uint32_t vword(const uint4 &v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}
__device__ __forceinline__ void set_vword(uint4 &v, int k, uint32_t w) {
    if (k == 0) v.x = w; else if (k == 1) v.y = w; else if (k == 2) v.z = w; else v.w = w;
}
template <typename T> struct Bits;
template <> struct Bits<double> {
    __device__ static __forceinline__ double get(const uint4 *v, int m) {
        return __hiloint2double(static_cast<int>(vword(v[m >> 1], 2 * (m & 1) + 1)),
                                static_cast<int>(vword(v[m >> 1], 2 * (m & 1))));
    }
    __device__ static __forceinline__ void put(uint4 *v, int m, double x) {
        set_vword(v[m >> 1], 2 * (m & 1), static_cast<uint32_t>(__double2loint(x)));
        set_vword(v[m >> 1], 2 * (m & 1) + 1, static_cast<uint32_t>(__double2hiint(x)));
    }
};
template <> struct Bits<float> {
    __device__ static __forceinline__ float get(const uint4 *v, int m) { return __uint_as_float(vword(v[m >> 2], m & 3)); }
    __device__ static __forceinline__ void put(uint4 *v, int m, float x) { set_vword(v[m >> 2], m & 3, __float_as_uint(x)); }
};
template <> struct Bits<int32_t> {
    __device__ static __forceinline__ int32_t get(const uint4 *v, int m) { return static_cast<int32_t>(vword(v[m >> 2], m & 3)); }
    __device__ static __forceinline__ void put(uint4 *v, int m, int32_t x) { set_vword(v[m >> 2], m & 3, static_cast<uint32_t>(x)); }
};
template <> struct Bits<__half> {
    __device__ static __forceinline__ __half get(const uint4 *v, int m) {
        const uint32_t w = vword(v[m >> 3], (m >> 1) & 3);
        return __ushort_as_half(static_cast<unsigned short>((m & 1) ? (w >> 16) : (w & 0xffffu)));
    }
    __device__ static __forceinline__ void put(uint4 *v, int m, __half x) {
        const uint32_t h = __half_as_ushort(x);
        uint32_t w = vword(v[m >> 3], (m >> 1) & 3);
        w = (m & 1) ? ((w & 0xffffu) | (h << 16)) : ((w & 0xffff0000u) | h);
        set_vword(v[m >> 3], (m >> 1) & 3, w);
    }
};
template <> struct Bits<__nv_bfloat16> {
    __device__ static __forceinline__ __nv_bfloat16 get(const uint4 *v, int m) {
        const uint32_t w = vword(v[m >> 3], (m >> 1) & 3);
        return __ushort_as_bfloat16(static_cast<unsigned short>((m & 1) ? (w >> 16) : (w & 0xffffu)));
    }
    __device__ static __forceinline__ void put(uint4 *v, int m, __nv_bfloat16 x) {
        const uint32_t h = __bfloat16_as_ushort(x);
        uint32_t w = vword(v[m >> 3], (m >> 1) & 3);
        w = (m & 1) ? ((w & 0xffffu) | (h << 16)) : ((w & 0xffff0000u) | h);
        set_vword(v[m >> 3], (m >> 1) & 3, w);
    }
};

template <typename T>
__device__ __forceinline__ void load_items(T (&dst)[kItems], const T *src) {
    constexpr int kVec = static_cast<int>(sizeof(T)) * kItems / 16;
    static_assert(kVec * 16 == static_cast<int>(sizeof(T)) * kItems, "kItems elements must fill 16-byte vectors");
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    uint4 v[kVec];
#pragma unroll
    for (int k = 0; k < kVec; ++k) v[k] = s[k];
#pragma unroll
    for (int m = 0; m < kItems; ++m) dst[m] = Bits<T>::get(v, m);
}
template <typename T>
__device__ __forceinline__ void store_items(T *dst, const T (&src)[kItems]) {
    constexpr int kVec = static_cast<int>(sizeof(T)) * kItems / 16;
    uint4 v[kVec];
#pragma unroll
    for (int k = 0; k < kVec; ++k) v[k] = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int m = 0; m < kItems; ++m) Bits<T>::put(v, m, src[m]);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
#pragma unroll
    for (int k = 0; k < kVec; ++k) d[k] = v[k];
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Half-width of template row dy (reading C2): the largest w with w^2 + dy^2 <= r^2
// (|dy| <= r <= 64; the float square root is corrected to the exact integer).
__device__ __forceinline__ int row_half_width(int r, int dy) {
    const int q = r * r - dy * dy;
    int w = static_cast<int>(sqrtf(static_cast<float>(q)));
    if ((w + 1) * (w + 1) <= q) ++w;
    if (w * w > q) --w;
    return w;
}

struct FrameView {
    const uint8_t *p;
    int64_t pitch;
    int W, H, r;
    __device__ __forceinline__ uint32_t at(int x, int y) const {
        return __ldg(p + static_cast<int64_t>(clampi(y, 0, H - 1)) * pitch + clampi(x, 0, W - 1));
    }
};

// Integer sum of the template pixels around (px, py) (the exact form of Eq. 3; reading
// C4 clamps template pixels to the frame).  w[i] = half-width of template row dy = i - r.
__device__ uint32_t disk_sum(const FrameView &f, const int8_t *w, int px, int py) {
    uint32_t s = 0;
    const int r = f.r;
    if (px - r >= 0 && px + r < f.W && py - r >= 0 && py + r < f.H) {
        const uint8_t *row = f.p + static_cast<int64_t>(py - r) * f.pitch + px;
        for (int i = 0; i <= 2 * r; ++i, row += f.pitch) {
            const int hw = w[i];
            for (int dx = -hw; dx <= hw; ++dx) s += __ldg(row + dx);
        }
    } else {
        for (int dy = -r; dy <= r; ++dy) {
            const int hw = w[dy + r];
            for (int dx = -hw; dx <= hw; ++dx) s += f.at(px + dx, py + dy);
        }
    }
    return s;
}

// Eq. 3 from the integer disk sum: sum (I-bg)^2 - (I-fg)^2 = (fg-bg)(2 sum I - (bg+fg)|D|).
template <typename A>
__device__ __forceinline__ A lik_from_sum(uint32_t s, A c1, A c2D, A den) {
    return (c1 * (static_cast<A>(2) * static_cast<A>(s) - c2D)) / den;
}

// ----------------------------------------------------------------------------------
// Eq. 4 per-pixel scaled form in half precision: a = (I - bg) kappa, b = (I - fg) kappa,
// term = a*a - b*b, summed over the template row by row, left to right, in the lane type
// (F16, the paper's form) or in FP32 (BF16 and PF_FLAG_ACCUM32).
// ----------------------------------------------------------------------------------
template <typename H> struct HalfOps;

template <>
struct HalfOps<__half> {
    using h2 = __half2;
#ifndef PF_NAIVE_RESAMPLE
    // (1024 + I) has the bit pattern 0x6400 | I in binary16, so the pixel enters the
    // half arithmetic without a conversion instruction: h - (1024 + level) is exact.
    static constexpr float kLevelOffset = 1024.0f;
    __device__ static __forceinline__ __half pix(uint32_t i) { return __ushort_as_half(static_cast<unsigned short>(0x6400u | i)); }
#else
    // study build: an integer-to-half conversion per pixel (the same exact value of I - level)
    static constexpr float kLevelOffset = 0.0f;
    __device__ static __forceinline__ __half pix(uint32_t i) { return __uint2half_rn(i); }
#endif
    __device__ static __forceinline__ __half from_f(float v) { return __float2half_rn(v); }
    __device__ static __forceinline__ float to_f(__half v) { return __half2float(v); }
    __device__ static __forceinline__ h2 pack(__half a, __half b) { return __halves2half2(a, b); }
    __device__ static __forceinline__ h2 from_f2(float a, float b) { return __floats2half2_rn(a, b); }
    __device__ static __forceinline__ float lo(h2 v) { return __low2float(v); }
    __device__ static __forceinline__ float hi(h2 v) { return __high2float(v); }
    __device__ static __forceinline__ __half lo_h(h2 v) { return __low2half(v); }
    __device__ static __forceinline__ __half hi_h(h2 v) { return __high2half(v); }
};

template <>
struct HalfOps<__nv_bfloat16> {
    using h2 = __nv_bfloat162;
    static constexpr float kLevelOffset = 0.0f;
    __device__ static __forceinline__ __nv_bfloat16 pix(uint32_t i) { return __float2bfloat16_rn(static_cast<float>(i)); }
    __device__ static __forceinline__ __nv_bfloat16 from_f(float v) { return __float2bfloat16_rn(v); }
    __device__ static __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ static __forceinline__ h2 pack(__nv_bfloat16 a, __nv_bfloat16 b) { return __halves2bfloat162(a, b); }
    __device__ static __forceinline__ h2 from_f2(float a, float b) { return __floats2bfloat162_rn(a, b); }
    __device__ static __forceinline__ float lo(h2 v) { return __low2float(v); }
    __device__ static __forceinline__ float hi(h2 v) { return __high2float(v); }
    __device__ static __forceinline__ __nv_bfloat16 lo_h(h2 v) { return __low2bfloat16(v); }
    __device__ static __forceinline__ __nv_bfloat16 hi_h(h2 v) { return __high2bfloat16(v); }
};

// The half-form sum (reading C10): each template row summed left to right, then the row
// sums added top to bottom, every addition in the lane type (F16, the paper's half
// accumulation) or in FP32 (BF16 and PF_FLAG_ACCUM32) and the result rounded to the lane
// type.  Every route below (a thread over the frame, a thread over staged terms, a warp
// over the frame) performs exactly these operations in this order.
template <typename H>
struct HalfLik {
    H kap, bgo, fgo;
    bool half_acc;
    __device__ __forceinline__ H term(uint32_t i) const {
        const H h = HalfOps<H>::pix(i);
        const H a = __hmul(__hsub(h, bgo), kap);
        const H b = __hmul(__hsub(h, fgo), kap);
        return __hfma(a, a, __hneg(__hmul(b, b)));
    }
    // direct evaluation from the frame by one thread
    __device__ H at(const FrameView &f, const int8_t *w, int px, int py) const {
        H hacc = HalfOps<H>::from_f(0.0f);
        float facc = 0.0f;
        for (int dy = -f.r; dy <= f.r; ++dy) {
            const int hw = w[dy + f.r];
            H hrow = HalfOps<H>::from_f(0.0f);
            float frow = 0.0f;
            for (int dx = -hw; dx <= hw; ++dx) {
                const H tm = term(f.at(px + dx, py + dy));
                if (half_acc) hrow = __hadd(hrow, tm); else frow += HalfOps<H>::to_f(tm);
            }
            if (half_acc) hacc = __hadd(hacc, hrow); else facc += frow;
        }
        return half_acc ? hacc : HalfOps<H>::from_f(facc);
    }
    // from per-pixel terms staged in shared memory (row pitch rw, template centred at
    // column cx + r, row cy + r)
    __device__ H from_terms(const H *tm, int rw, const int8_t *w, int r, int cx, int cy) const {
        if (half_acc) {
            H acc = HalfOps<H>::from_f(0.0f);
            for (int i = 0; i <= 2 * r; ++i) {
                const int hw = w[i];
                const H *row = tm + (cy + i) * rw + cx + r;
                H rs = HalfOps<H>::from_f(0.0f);
#pragma unroll 4
                for (int dx = -hw; dx <= hw; ++dx) rs = __hadd(rs, row[dx]);
                acc = __hadd(acc, rs);
            }
            return acc;
        }
        float acc = 0.0f;
        for (int i = 0; i <= 2 * r; ++i) {
            const int hw = w[i];
            const H *row = tm + (cy + i) * rw + cx + r;
            float rs = 0.0f;
#pragma unroll 4
            for (int dx = -hw; dx <= hw; ++dx) rs += HalfOps<H>::to_f(row[dx]);
            acc += rs;
        }
        return HalfOps<H>::from_f(acc);
    }
    // by one warp from the frame: lane l sums rows l, l + 32, ... (each left to right);
    // lane 0 adds the row sums top to bottom.  Valid in lane 0.
    __device__ H warp_at(const FrameView &f, int px, int py) const {
        const int lane = threadIdx.x & 31, nrow = 2 * f.r + 1;
        H hacc = HalfOps<H>::from_f(0.0f);
        float facc = 0.0f;
        for (int base = 0; base < nrow; base += 32) {
            const int i = base + lane;
            H hrow = HalfOps<H>::from_f(0.0f);
            float frow = 0.0f;
            if (i < nrow) {
                const int dy = i - f.r;
                const int hw = row_half_width(f.r, dy);
                for (int dx = -hw; dx <= hw; ++dx) {
                    const H tm = term(f.at(px + dx, py + dy));
                    if (half_acc) hrow = __hadd(hrow, tm); else frow += HalfOps<H>::to_f(tm);
                }
            }
            const int n = nrow - base < 32 ? nrow - base : 32;
            for (int k = 0; k < n; ++k) {
                if (half_acc) {
                    const H v = __shfl_sync(0xffffffffu, hrow, k);
                    hacc = __hadd(hacc, v);
                } else {
                    facc += __shfl_sync(0xffffffffu, frow, k);
                }
            }
        }
        return half_acc ? hacc : HalfOps<H>::from_f(facc);
    }
};

// The half-form constants of a tracker: kappa, and the two levels offset so that a pixel
// enters half arithmetic without a conversion (HalfOps<H>::pix).
template <typename H>
__device__ __forceinline__ HalfLik<H> half_lik(const TrackerDev &T) {
    HalfLik<H> hk;
    const float lo = HalfOps<H>::kLevelOffset;
    hk.kap = HalfOps<H>::from_f(T.kappa);
    hk.bgo = HalfOps<H>::from_f(lo + T.bg_f);
    hk.fgo = HalfOps<H>::from_f(lo + T.fg_f);
    hk.half_acc = std::is_same<H, __half>::value && !(T.flags & 0x2u);
    return hk;
}

// Integer disk sum by one warp (lanes take template rows; exact, so the order is free).
__device__ __forceinline__ uint32_t warp_disk_sum(const FrameView &f, int px, int py) {
    const int lane = threadIdx.x & 31, nrow = 2 * f.r + 1;
    uint32_t s = 0;
    for (int i = lane; i < nrow; i += 32) {
        const int hw = row_half_width(f.r, i - f.r);
        for (int dx = -hw; dx <= hw; ++dx) s += f.at(px + dx, py + i - f.r);
    }
    return __reduce_add_sync(0xffffffffu, s);
}

// Shared memory of the step kernel (dynamic: sizeof(StepSmem<P>) bytes).
template <int P>
struct __align__(16) StepSmem {
    using Tr = Prec<P>;
    using pos_t = typename Tr::pos_t;
    using lik_t = typename Tr::lik_t;
    using acc_t = typename Tr::acc_t;
    pos_t ax[kTile];          // ancestor positions of the tile (previous frame)
    pos_t ay[kTile];
    int32_t J[kTile];         // J[e] = strata assigned to particles k0..k0+e (cumulative)
    lik_t table[kTableMax];   // likelihood of each pixel of the tile's window
    union {
        uint16_t pre[kRoiMax];      // integer form: row prefix sums of the staged region
        lik_t term[Tr::kHalf ? kRoiMax : 1];   // half form: per-pixel Eq. 4 terms of the staged region
        // F16 half accumulation, staged regions of up to kRoiMax / 2 pixels: the terms of
        // pixels x and x + 1 of a row side by side, so one half2 addition advances the sums
        // of two neighbouring cells
        __half2 term2[P == 2 ? kRoiMax / 2 : 1];
    } u;
    alignas(16) uint16_t map[kMapMax];   // ancestor (tile element + 1) of each offspring
    alignas(16) int warp_imax[kWarps];
    alignas(16) acc_t warp_sum[kWarps];
    alignas(16) acc_t warp_max[kWarps];
    alignas(16) float box[kWarps][4];
    U128 red128[kWarps];
    alignas(16) int warp_incl[kWarps];
    Stats<acc_t> red[kWarps];
    U128 agg_x;               // the tile aggregate (fixed point)
    int jbeg, jend;
    double u0d;               // resampling offset u0 of the previous frame
    float u0f;
    uint32_t skeys[4];        // stratified resampling: key_lo, key_hi, frame t - 1, tracker id
    int win_x0, win_y0, win_w, win_h;   // likelihood table window (win_w = 0: none)
    int qmin;
    int8_t w[2 * kMaxRadius + 1];
    uint32_t ticket;
    uint32_t last;
    int cached;               // tracker whose descriptor / state / frame are loaded below
    TrackerDev trk;
    TrackerState st;
    FrameRef fr;
};

// Block-wide merge of per-thread stats, result valid in thread 0.  Each warp takes its
// max of m (butterfly), rescales every lane's sums to it (one exp a lane) and adds them
// (butterfly); warp 0 does the same over the warps' results.  Max, rescale and sums run
// in a fixed order, so the result is deterministic.  The caller synchronises before
// sm.red is written again.
// Warp max / min of floats by redux.sync on an order-preserving integer image (the sign bit
// kept, the other bits flipped for negative values); exact, -inf included (no NaN here).
__device__ __forceinline__ int float_key(float x) {
    const int b = __float_as_int(x);
    return b ^ ((b >> 31) & 0x7fffffff);
}
__device__ __forceinline__ float key_float(int k) { return __int_as_float(k ^ ((k >> 31) & 0x7fffffff)); }
__device__ __forceinline__ float warp_max(float x) { return key_float(__reduce_max_sync(0xffffffffu, float_key(x))); }
__device__ __forceinline__ float warp_min(float x) { return key_float(__reduce_min_sync(0xffffffffu, float_key(x))); }
__device__ __forceinline__ double warp_max(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double y = __shfl_xor_sync(0xffffffffu, x, o);
        x = y > x ? y : x;
    }
    return x;
}

template <int P, typename A>
__device__ __forceinline__ Stats<A> warp_stats(Stats<A> v) {
    constexpr bool F = Prec<P>::kHalf;
    const A m = warp_max(v.m);
    if (m == neg_inf<A>()) return Stats<A>{m, 0, 0, 0};
    const A sc = (v.m == neg_inf<A>()) ? static_cast<A>(0) : wexp<F>(v.m - m);
    A s = mul_rn(v.s, sc), sx = mul_rn(v.sx, sc), sy = mul_rn(v.sy, sc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s = add_rn(s, __shfl_xor_sync(0xffffffffu, s, o));
        sx = add_rn(sx, __shfl_xor_sync(0xffffffffu, sx, o));
        sy = add_rn(sy, __shfl_xor_sync(0xffffffffu, sy, o));
    }
    return Stats<A>{m, s, sx, sy};
}

// Warp-level min / max of a bounding box (x0, x1, y0, y1), returned to every lane; lane 0
// also leaves it in sm.box for merge_warp_boxes after the next barrier.
template <int P>
__device__ __forceinline__ float4 warp_box(float4 b, StepSmem<P> &sm) {
    b = make_float4(warp_min(b.x), warp_max(b.y), warp_min(b.z), warp_max(b.w));
    if ((threadIdx.x & 31) == 0) *reinterpret_cast<float4 *>(sm.box[threadIdx.x >> 5]) = b;
    return b;
}
// The block's box from the warps' boxes in sm.box, by one whole warp (lane w reads warp w's),
// returned to every lane of that warp.
template <int P>
__device__ __forceinline__ float4 merge_warp_boxes(const StepSmem<P> &sm) {
    const int lane = threadIdx.x & 31;
    const float4 b = lane < kWarps ? *reinterpret_cast<const float4 *>(sm.box[lane])
                                   : make_float4(FLT_MAX, -FLT_MAX, FLT_MAX, -FLT_MAX);
    return make_float4(warp_min(b.x), warp_max(b.y), warp_min(b.z), warp_max(b.w));
}

template <int P, typename A>
__device__ Stats<A> block_stats(Stats<A> v, StepSmem<P> &sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_stats<P>(v);
    if (lane == 0) sm.red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = (lane < kWarps) ? sm.red[lane] : Stats<A>{neg_inf<A>(), 0, 0, 0};
        v = warp_stats<P>(v);
    }
    return v;
}

// Decoupled lookback over the tracker's earlier tiles, kThreads tiles per round (thread
// i inspects tile base - i).  Sums the fixed-point aggregates back to the nearest tile
// that has published its inclusive prefix.  Whole block, one barrier per round; the
// result is valid in every thread.
template <int P>
__device__ U128 lookback(const LookbackDesc *look, int lt, uint64_t tag, TrackerState *st, StepSmem<P> &sm) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    U128 total{0ull, 0ull};
    for (int base = lt - 1; base >= 0; base -= kThreads) {
        const int idx = base - tid;
        uint32_t f = 0u;
        U128 v{0ull, 0ull};
        if (idx >= 0) {
            f = wait_desc(&look[idx], tag, st, v);
            if (f == 0u) { f = 2u; v = U128{0ull, 0ull}; }   // timed out: an inclusive zero (step flagged invalid)
        }
        // the warp's nearest inclusive predecessor (lowest lane); lanes past it contribute 0
        const uint32_t incl = __ballot_sync(0xffffffffu, f == 2u);
        const int first = incl ? __ffs(static_cast<int>(incl)) - 1 : 32;
        if (lane > first) v = U128{0ull, 0ull};
        if (base - warp * 32 >= 0) {          // the warp has predecessors in this round
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = add128(v, shfl_down128(v, o));
        }
        if (lane == 0) { sm.red128[warp] = v; sm.warp_incl[warp] = incl != 0u; }
        const int found = __syncthreads_or(incl != 0u);
        {   // every warp: the warp sums up to the first warp with an inclusive predecessor
            U128 x{0ull, 0ull};
            int inc = 0;
            if (lane < kWarps) { x = sm.red128[lane]; inc = sm.warp_incl[lane]; }
            const uint32_t im = __ballot_sync(0xffffffffu, inc != 0);
            const int fw = im ? __ffs(static_cast<int>(im)) - 1 : 32;
            if (lane > fw) x = U128{0ull, 0ull};
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) x = add128(x, shfl_xor128(x, o));
            total = add128(total, x);
        }
        if (found) break;
        __syncthreads();           // red128 is rewritten by the next round
    }
    return total;
}

// First index e in [0, n) with J[e] > j (J non-decreasing, J[n-1] > j).
__device__ __forceinline__ int upper_index(const int32_t *J, int n, int j) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (J[mid] > j) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// Merge of the tracker's tile partials (one per thread, all loads in flight, then the
// block merge: deterministic) and the new state, by the tile that completed the tracker.
template <int P>
__device__ void finalize_tracker(const TrackerDev &T, TrackerState *st, StepSmem<P> &sm, double *est_out,
                                 bool track_box) {
    using acc_t = typename Prec<P>::acc_t;
    constexpr bool kF64 = sizeof(acc_t) == 8;
    constexpr bool F = Prec<P>::kHalf;
    Stats<acc_t> v{neg_inf<acc_t>(), 0, 0, 0};
    float4 bb = make_float4(FLT_MAX, -FLT_MAX, FLT_MAX, -FLT_MAX);
    const uint64_t tg = partial_tag(sm.st.epoch);
    for (int i = threadIdx.x; i < T.ntiles; i += kThreads) {
        Stats<acc_t> w;
        uint64_t q[8];
        if constexpr (kF64) {
            const double *p = T.part[i].d;
            w = Stats<acc_t>{__ldcg(p + 0), __ldcg(p + 1), __ldcg(p + 2), __ldcg(p + 3)};
            const unsigned long long *pb = reinterpret_cast<const unsigned long long *>(T.part[i].b);
#pragma unroll
            for (int k = 0; k < 4; ++k) q[4 + k] = track_box ? __ldcg(pb + k) : 0ull;
        } else {
            wait_partial(&T.part[i], tg, st, q, track_box);
            w = Stats<acc_t>{__uint_as_float(static_cast<uint32_t>(q[0])), __uint_as_float(static_cast<uint32_t>(q[1])),
                             __uint_as_float(static_cast<uint32_t>(q[2])), __uint_as_float(static_cast<uint32_t>(q[3]))};
        }
        v = stats_merge<F>(v, w);
        bb.x = fminf(bb.x, __uint_as_float(static_cast<uint32_t>(q[4])));
        bb.y = fmaxf(bb.y, __uint_as_float(static_cast<uint32_t>(q[5])));
        bb.z = fminf(bb.z, __uint_as_float(static_cast<uint32_t>(q[6])));
        bb.w = fmaxf(bb.w, __uint_as_float(static_cast<uint32_t>(q[7])));
    }
    if (track_box) warp_box(bb, sm);
    v = block_stats<P>(v, sm);
    if (track_box && threadIdx.x < 32) bb = merge_warp_boxes(sm);
    if (threadIdx.x < 32) {
        // The new state, from the block's statistics (thread 0's, broadcast) and this launch's
        // starting state (the copy in shared memory, which no tile changes), written field by
        // field with stores only by four lanes in parallel: lane 0 the x estimate and
        // anchors, lane 1 the y ones, lane 2 the weight scalars, lane 3 the rest.  The status
        // word is not written (another tile may have raised it).
        const int lane = threadIdx.x;
        Stats<acc_t> r;
        r.m = __shfl_sync(0xffffffffu, v.m, 0);
        r.s = __shfl_sync(0xffffffffu, v.s, 0);
        r.sx = __shfl_sync(0xffffffffu, v.sx, 0);
        r.sy = __shfl_sync(0xffffffffu, v.sy, 0);
        const TrackerState &o = sm.st;
        const int64_t slot = (o.t >= 0 && o.t < 0x7fffffffll)
                                 ? static_cast<int64_t>(static_cast<uint32_t>(o.t) % static_cast<uint32_t>(T.est_cap))
                                 : o.t % T.est_cap;
        if (lane < 2) {
            const bool ly = lane == 1;
            const acc_t rs = ly ? r.sy : r.sx;
            const double on = ly ? o.ny : o.nx;        // the anchor the positions were written against
            const int32_t oni = ly ? o.nyi : o.nxi;
            double e, nn;
            int32_t ni;
            if constexpr (kF64) {
                e = on + rs / r.s;
                nn = on;
                if (isfinite(e) && fabs(e) < 1.0e6) nn = floor(e) + ((e - floor(e)) >= 0.5 ? 1.0 : 0.0);
                ni = static_cast<int32_t>(nn);
            } else {
                // FP32 quotient; the next anchor in FP32 / integers (FP64 only to widen the
                // results the host reads)
                const float q = rs / r.s;
                const float fq = static_cast<float>(oni) + q;
                ni = oni;
                if (isfinite(fq) && fabsf(fq) < 1.0e6f) ni = __float2int_rd(fq + 0.5f);
                nn = static_cast<double>(ni);
                e = on + static_cast<double>(q);
            }
            if (ly) { st->ay = on; st->ayi = oni; st->ny = nn; st->nyi = ni; st->est_y = e; }
            else { st->ax = on; st->axi = oni; st->nx = nn; st->nxi = ni; st->est_x = e; }
            T.est_ring[2 * slot + lane] = e;
            if (est_out) est_out[lane] = e;
        } else if (lane == 2) {
            const acc_t inv = static_cast<acc_t>(1) / r.s;
            st->M = static_cast<double>(r.m);
            st->S = static_cast<double>(r.s);
            st->invS = static_cast<double>(inv);
            st->M_f = static_cast<float>(r.m);
            st->invS_f = static_cast<float>(inv);
            T.stat_ring[2 * slot] = static_cast<double>(r.m);
            T.stat_ring[2 * slot + 1] = static_cast<double>(r.s);
        } else if (lane == 3) {
            // the box of the new positions sizes the next step's tracker table (unknown if
            // the launch did not track it, or empty)
            const bool box_ok = track_box && bb.x <= bb.y && bb.z <= bb.w;
            st->bb_x0 = box_ok ? bb.x : __int_as_float(0x7fc00000);
            st->bb_x1 = box_ok ? bb.y : __int_as_float(0x7fc00000);
            st->bb_y0 = box_ok ? bb.z : __int_as_float(0x7fc00000);
            st->bb_y1 = box_ok ? bb.w : __int_as_float(0x7fc00000);
            st->t = o.t + 1;
            st->epoch = o.epoch + 1u;
            // every tile of this launch has counted; the next launch sees the reset after the
            // kernel boundary
            *T.done = 0u;
        }
    }
}

// The tracker's likelihood table of this launch into the tile's shared-memory table: each
// cell's word if it carries this launch's tag, else the cell computed here (the builder
// has not reached it yet; the same operations give the same bits).
template <int P, typename A>
__device__ __forceinline__ void fetch_table(const TrackerDev &T, StepSmem<P> &sm, int gx0, int gy0, int gw, int cells,
                                            const FrameView &fv, A c1, A c2D, A den, TrackerState *st) {
    (void)st;
    using H = typename std::conditional<Prec<P>::kHalf, typename Prec<P>::pos_t, __half>::type;
    const uint64_t gtag = static_cast<uint64_t>(sm.st.epoch % 0x7fffffffu + 1u) << 32;
    for (int c = threadIdx.x; c < cells; c += kThreads) {
        const uint64_t v = __ldcg(reinterpret_cast<const unsigned long long *>(T.gtab) + PF_IDX(c, kTableMax));
        uint32_t payload;
        const bool built = (v & 0xffffffff00000000ull) == gtag;
        if constexpr (Prec<P>::kHalf) {
            if (built) {
                payload = static_cast<uint32_t>(v);
            } else {
                const H h = half_lik<H>(T).at(fv, sm.w, gx0 + c % gw, gy0 + c / gw);
                payload = static_cast<uint32_t>(*reinterpret_cast<const unsigned short *>(&h));
            }
            const unsigned short bits = static_cast<unsigned short>(payload);
            sm.table[PF_IDX(c, kTableMax)] = *reinterpret_cast<const H *>(&bits);
        } else {
            payload = built ? static_cast<uint32_t>(v) : disk_sum(fv, sm.w, gx0 + c % gw, gy0 + c / gw);
            sm.table[PF_IDX(c, kTableMax)] = lik_from_sum<A>(payload, c1, c2D, den);
        }
    }
}

// The strata counts of a thread's elements (phase 1d): C_k of each element from the tile's
// local prefix loc[m] pinned to the exact boundaries excl / pend, and J = the number of
// strata points at or below C_k (repeated C values reuse the count: on a peaked posterior
// most elements repeat the previous C).  nrm is the saved 1/S (the naive study build: S
// itself).  Force-inlined so that loc and Jr stay in registers.
template <typename A, typename Str>
__device__ __forceinline__ void strata_counts(const Str &str, const A (&loc)[kItems], int (&Jr)[kItems], A excl,
                                              A pend, A nrm, int eb, int cnt, int k0, int N, A *dbg_cdf,
                                              TrackerState *st) {
    (void)st;
#ifdef PF_NAIVE_RESAMPLE
    const A Sdiv = nrm;
#else
    const A invS = nrm;
#endif
    A cprev = static_cast<A>(-1);
    int jprev = 0;
#pragma unroll
    for (int m = 0; m < kItems; ++m) {
        const int e = eb + m;
        int J = N;                                   // (elements past the tile: unused)
        if (e < cnt) {
            const int k = k0 + e;
            const A Pk = (e == cnt - 1) ? pend : fmin(add_rn(excl, loc[m]), pend);
            // the normalised CDF cannot exceed 1; the FP32 scan can round above it
            A C = fmin(PF_NORM(Pk), static_cast<A>(1));
            if (k == N - 1) { C = static_cast<A>(1); J = N; }
            else if (C == cprev) J = jprev;          // same CDF value, same count
            else J = str.count_le(C);
            cprev = C;
            jprev = J;
            if (dbg_cdf) dbg_cdf[PF_IDX(k, N)] = C;
        }
        Jr[m] = J;
    }
}

// The descriptor, state and frame reference of launch position ti (slot `slot`) into shared
// memory, by the whole block (the caller synchronises).
template <int P>
__device__ __forceinline__ void load_descriptor(const StepLaunch &Lp, int slot, int ti, StepSmem<P> &sm) {
    const uint32_t *src_t = reinterpret_cast<const uint32_t *>(Lp.trk + slot);
    const uint32_t *src_s = reinterpret_cast<const uint32_t *>(Lp.states + slot);
    const uint32_t *src_f = reinterpret_cast<const uint32_t *>(Lp.frames + ti);
    uint32_t *dt = reinterpret_cast<uint32_t *>(&sm.trk);
    uint32_t *ds = reinterpret_cast<uint32_t *>(&sm.st);
    uint32_t *df = reinterpret_cast<uint32_t *>(&sm.fr);
    constexpr int nt = sizeof(TrackerDev) / 4, ns = sizeof(TrackerState) / 4, nf = sizeof(FrameRef) / 4;
    for (int i = threadIdx.x; i < nt + ns + nf; i += kThreads) {
        if (i < nt) dt[i] = __ldg(src_t + i);
        else if (i < nt + ns) ds[i - nt] = __ldcg(src_s + i - nt);
        else df[i - nt - ns] = __ldcg(src_f + i - nt - ns);
    }
}

// Kernel modes: the step kernel (systematic and stratified trackers, every phase), and for
// multinomial trackers the CDF kernel (phase 1 up to the CDF, written to T.cdf) and the
// pull kernel (resampling from T.cdf, phases 2-5), launched in that order; the pull kernel
// also takes the Gumbel-max, Metropolis and rejection trackers (ancestors from T.anc).
constexpr int kModeStep = 0, kModeCdf = 1, kModePull = 2;
// The step kernel with the tracker table (phase 0) and the bounding box that sizes it: a
// separate instantiation, launched for a tracker of at least two waves of tiles, so that the
// common launch carries none of its code or registers.
constexpr int kModeStepBig = 3;

// One tile of a launch in mode kMode (trackers of the other modes are skipped).
template <int P, int kMode>
__device__ void run_tile(const StepLaunch &Lp, int g, StepSmem<P> &sm) {
    constexpr bool kPull = kMode == kModePull;
    using Tr = Prec<P>;
    using pos_t = typename Tr::pos_t;
    using lik_t = typename Tr::lik_t;
    using acc_t = typename Tr::acc_t;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // launch position of the tile, its first tile and its slot
    int ti = 0;
    if (Lp.ntrk > 1) {
        if (Lp.tile_trk) {
            ti = __ldg(&Lp.tile_trk[g]);
        } else {   // last position whose first tile is <= g
            int lo = 0, hi = Lp.ntrk - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(&Lp.tile_prefix[mid]) <= g) lo = mid; else hi = mid - 1;
            }
            ti = lo;
        }
    }
    const int slot = Lp.slot_of ? __ldg(&Lp.slot_of[ti]) : ti;
    TrackerState *const st = Lp.states + slot;

    // ---- the tracker's descriptor, state and frame reference, loaded in one round trip
    // and kept for the CTA's later tiles of the same tracker (none of them changes
    // before the tracker's last tile of this launch has finished)
    if (ti != sm.cached) {
        load_descriptor(Lp, slot, ti, sm);
        __syncthreads();
        if (tid == 0) sm.cached = ti;
    }
    const TrackerDev &T = sm.trk;
    if (!sm.fr.active) return;
    if (sm.st.status & kStatusTimeout) return;   // a failed step: results are invalid
    // (the host gives each launch only its own family's tiles; the CDF and pull kernels
    // check as well)
    if constexpr (kMode == kModeCdf) {
        if (T.resampler != kResampleMultinomial && T.resampler != kResampleShard) return;
    } else if constexpr (kMode == kModePull) {
        if (T.resampler != kResampleMultinomial && !ancestors_given(T.resampler)) return;
    }

    const int N = static_cast<int>(T.N);
    const int lt = g - (Lp.tile_prefix ? __ldg(&Lp.tile_prefix[ti]) : T.tile_begin);
    const int k0 = lt * T.tile;
    const int cnt = (N - k0) < T.tile ? (N - k0) : T.tile;
    const int64_t t = sm.st.t;
    if constexpr (kMode == kModeCdf) {
        if (t == 0) return;                        // frame 0 resamples nothing
    }
    const uint64_t dtag = desc_tag(sm.st.epoch);    // this launch's lookback tag
    constexpr bool kF64 = sizeof(acc_t) == 8;    // REF64; the other kernels use no FP64
    const int nxi = sm.st.nxi, nyi = sm.st.nyi;     // anchor of the offspring
    const int axi_anc = sm.st.axi, ayi_anc = sm.st.ayi;   // anchor of the ancestors
    const int in = static_cast<int>((t + 1) & 1), out = static_cast<int>(t & 1);
    acc_t *const dbg_cdf = static_cast<acc_t *>(T.dbg_cdf);
    LookbackDesc *const look = T.look;

    FrameView fv;
    fv.W = T.W; fv.H = T.H; fv.r = T.r;
    if (Lp.frame_override) { fv.p = Lp.frame_override; fv.pitch = Lp.pitch_override; }
    else {
        const int64_t ft = sm.fr.ring ? t % sm.fr.ring : t;   // a ring of staged frames, or a resident video
        fv.p = sm.fr.base + (sm.fr.stride ? ft * sm.fr.stride : 0);
        fv.pitch = sm.fr.pitch;
    }
    const int r = fv.r;
    for (int i = tid; i <= 2 * r; i += kThreads) sm.w[i] = static_cast<int8_t>(row_half_width(r, i - r));

    using H = typename std::conditional<Tr::kHalf, pos_t, __half>::type;

    // ------------------------------------------------------------ 0. the tracker's table
    // A step launch of a tracker of at least two waves of tiles (twice as many tiles as the
    // launch has CTAs) whose previous positions' bounding box is known shares one likelihood
    // table per frame: the window every offspring can reach (the box widened by the drift
    // and the largest draw, kDrawMax sigma, plus one pixel of rounding), tabulated once in
    // device memory instead of once per tile.  (With a single wave the per-tile tables are
    // built while the tiles wait for their predecessors' aggregates, at no cost; so are the
    // builders' cells here, after the aggregate is published.)  The tracker's first
    // min(ntiles, grid) tiles build it, one cell per warp; every cell carries this launch's
    // tag, and a tile that finds a cell not yet built computes it itself (same operations,
    // same bits), so no tile waits for another.
    const bool track_box = kMode == kModeStepBig && T.gtab != nullptr &&
                           T.ntiles >= 2 * static_cast<int>(gridDim.x);
    bool gt = false;
    int gx0 = 0, gy0 = 0, gw = 0, gh = 0;
    if constexpr (kMode == kModeStepBig) {
        const float b0 = sm.st.bb_x0, b1 = sm.st.bb_x1, c0 = sm.st.bb_y0, c1b = sm.st.bb_y1;
        if (track_box && b0 <= b1 && c0 <= c1b && fabsf(b0) < 1.0e6f && fabsf(b1) < 1.0e6f &&
            fabsf(c0) < 1.0e6f && fabsf(c1b) < 1.0e6f) {
            const float mxr = fabsf(T.drift_xf) + kDrawMax * T.sigma_xf + 1.0f;
            const float myr = fabsf(T.drift_yf) + kDrawMax * T.sigma_yf + 1.0f;
            if (mxr < 4096.0f && myr < 4096.0f && b1 - b0 < 4096.0f && c1b - c0 < 4096.0f) {
                gx0 = static_cast<int>(floorf(b0 - mxr));
                gy0 = static_cast<int>(floorf(c0 - myr));
                gw = static_cast<int>(ceilf(b1 + mxr)) - gx0 + 1;
                gh = static_cast<int>(ceilf(c1b + myr)) - gy0 + 1;
                gt = static_cast<int64_t>(gw) * gh <= kTableMax;
            }
        }
        // the window for the rest of the tile (ordered by the barrier of phase 1b)
        if (gt && tid == 0) { sm.win_x0 = gx0; sm.win_y0 = gy0; sm.win_w = gw; sm.win_h = gh; }
    }

    // ------------------------------------------------------------ 1a. local scan of e
    acc_t loc[kItems];
    acc_t mex = static_cast<acc_t>(0);   // running max of the preceding lanes of the warp
    // bounding box of the ancestors with non-negligible weight (absolute pixel units)
    float bx0 = FLT_MAX, bx1 = -FLT_MAX, by0 = FLT_MAX, by1 = -FLT_MAX;
    const int eb = tid * kItems;  // blocked arrangement: thread tid owns elements eb .. eb+kItems-1
    if (!kPull && t > 0) {
        const lik_t *__restrict__ Lin = static_cast<const lik_t *>(T.pl[in]);
        const pos_t *__restrict__ Xin = static_cast<const pos_t *>(T.px[in]);
        const pos_t *__restrict__ Yin = static_cast<const pos_t *>(T.py[in]);
        const acc_t M = Lp.shard ? static_cast<acc_t>(Lp.g_M)
                                 : (kF64 ? static_cast<acc_t>(sm.st.M) : static_cast<acc_t>(sm.st.M_f));
        lik_t lv[kItems];
        // the thread's kItems positions as raw 16-byte vectors: copied to shared memory as
        // they are (the offspring loop reads its ancestors there), unpacked only where the
        // window's bounding box needs a value
        constexpr int kVp = static_cast<int>(sizeof(pos_t)) * kItems / 16;
        uint4 xr[kVp], yr[kVp];
        if (eb + kItems <= cnt) {
            // kItems consecutive values of each array, 16-byte aligned (k0 and eb are
            // multiples of kItems = 8 and the buffers are 16-byte aligned)
            load_items(lv, Lin + k0 + eb);
#pragma unroll
            for (int k = 0; k < kVp; ++k) {
                xr[k] = reinterpret_cast<const uint4 *>(Xin + k0 + eb)[k];
                yr[k] = reinterpret_cast<const uint4 *>(Yin + k0 + eb)[k];
            }
        } else {
            pos_t xv[kItems], yv[kItems];
#pragma unroll
            for (int m = 0; m < kItems; ++m) {
                const int e = eb + m;
                lv[m] = (e < cnt) ? Lin[k0 + e] : lik_t{};
                xv[m] = (e < cnt) ? Xin[k0 + e] : pos_t{};
                yv[m] = (e < cnt) ? Yin[k0 + e] : pos_t{};
            }
#pragma unroll
            for (int k = 0; k < kVp; ++k) { xr[k] = make_uint4(0u, 0u, 0u, 0u); yr[k] = xr[k]; }
#pragma unroll
            for (int m = 0; m < kItems; ++m) { Bits<pos_t>::put(xr, m, xv[m]); Bits<pos_t>::put(yr, m, yv[m]); }
        }
#pragma unroll
        for (int k = 0; k < kVp; ++k) {
            reinterpret_cast<uint4 *>(sm.ax + eb)[k] = xr[k];
            reinterpret_cast<uint4 *>(sm.ay + eb)[k] = yr[k];
        }
        // clear the ancestor map (its heads are written after the strata are counted)
#pragma unroll
        for (int i = 0; i < kMapMax / 8 / kThreads; ++i)
            reinterpret_cast<uint4 *>(sm.map)[tid + i * kThreads] = make_uint4(0u, 0u, 0u, 0u);
        const float sx = Tr::kHalf ? static_cast<float>(axi_anc) : 0.0f;
        const float sy = Tr::kHalf ? static_cast<float>(ayi_anc) : 0.0f;
        acc_t run = static_cast<acc_t>(0);
#pragma unroll
        for (int m = 0; m < kItems; ++m) {
            const int e = eb + m;
            acc_t v = static_cast<acc_t>(0);
            if (e < cnt) v = wexp<Tr::kHalf>(to_acc(lv[m]) - M);
            if (!gt && v > static_cast<acc_t>(9.3132257461547852e-10)) {   // weight above 2^-30 of the max
                const float xa = static_cast<float>(to_acc(Bits<pos_t>::get(xr, m))) + sx;
                const float ya = static_cast<float>(to_acc(Bits<pos_t>::get(yr, m))) + sy;
                bx0 = fminf(bx0, xa); bx1 = fmaxf(bx1, xa);
                by0 = fminf(by0, ya); by1 = fmaxf(by1, ya);
            }
            run = (m == 0) ? v : run + v;
            loc[m] = run;
        }
        // block exclusive scan of the thread totals
        acc_t x = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const acc_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sm.warp_sum[warp] = x;
        acc_t xex = __shfl_up_sync(0xffffffffu, x, 1);
        if (lane == 0) xex = static_cast<acc_t>(0);
        __syncthreads();
        acc_t wpre = static_cast<acc_t>(0);
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const acc_t v = sm.warp_sum[w];
            if (w < warp) wpre += v;
        }
        const acc_t off = wpre + xex;
        if (tid != 0) {
#pragma unroll
            for (int m = 0; m < kItems; ++m) loc[m] = off + loc[m];
        }
        // The tile aggregate is the prefix at its last particle; the thread that holds it
        // publishes it at once (tile 0: as the inclusive prefix) and leaves it for thread 0,
        // which reads it after the next barrier.  (Every prefix of the tile is later clamped
        // to the exact boundary excl + aggregate.)
        {
            const int el = cnt - 1;
            if (el / kItems == tid) {
                acc_t a = loc[0];
#pragma unroll
                for (int m = 1; m < kItems; ++m)
                    if (m == el % kItems) a = loc[m];
                const U128 ax = to_fixed(a);
                desc_publish(&look[lt], lt == 0 ? 1 : 0, ax, dtag);
                sm.agg_x = ax;
            }
        }
        // running max across threads, which makes the tile-local prefix non-decreasing: the
        // warp part here, the block part after the next barrier (phase 1d)
        acc_t mx = loc[kItems - 1];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const acc_t y = __shfl_up_sync(0xffffffffu, mx, o);
            if (lane >= o) mx = fmax(mx, y);
        }
        if (lane == 31) sm.warp_max[warp] = mx;
        mex = __shfl_up_sync(0xffffffffu, mx, 1);
    } else if (kPull && t > 0) {
        // The pull kernel's gather: offspring j = k0 + e takes the first particle a whose
        // CDF value reaches v_j (word j mod 4 of Philox(j / 4, t - 1, 1, tracker)); the
        // eight searches of a thread advance together.  a goes to J[e], the ancestor's
        // position (previous frame) to ax/ay[e], and the box of the gathered positions
        // sizes the likelihood window as in the step kernel.
        const acc_t *cdf = static_cast<const acc_t *>(T.cdf);
        const pos_t *__restrict__ Xin = static_cast<const pos_t *>(T.px[in]);
        const pos_t *__restrict__ Yin = static_cast<const pos_t *>(T.py[in]);
        acc_t uq[kItems];
        int lo[kItems], hi[kItems];
        if (ancestors_given(T.resampler)) {
            // Gumbel-max, Metropolis, rejection: the ancestor kernel wrote every offspring's ancestor
#pragma unroll
            for (int m = 0; m < kItems; ++m) {
                const int a = (eb + m < cnt) ? __ldg(T.anc + PF_IDX(k0 + eb + m, N)) : 0;
                lo[m] = hi[m] = a > 0 ? a : 0;
            }
        } else {
#pragma unroll
            for (int h = 0; h < kItems; h += 4) {
                const uint32_t blk = static_cast<uint32_t>(k0 + eb + h) >> 2;   // k0 + eb is a multiple of 8
                const uint4 wv = philox4x32_10(make_uint4(blk, static_cast<uint32_t>(t - 1), 1u, T.tracker_id),
                                               T.key_lo, T.key_hi);
                const uint32_t ws[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if constexpr (kF64) uq[h + i] = uniform_f64(ws[i]); else uq[h + i] = uniform_f32(ws[i]);
                    lo[h + i] = 0;
                    hi[h + i] = (eb + h + i < cnt) ? N : 0;
                }
            }
            // A coarse table of the CDF in shared memory (the staging area is free until the
            // likelihood table): cs[i] = C at the last index of block i of 2^lb entries, 2^lb
            // the smallest power of two that gives at most kCoarse blocks.  The first block
            // whose last value reaches u holds the answer (C is non-decreasing), so a search
            // is a search of the table and then lb global steps inside that block, with the
            // same result as a search of the whole CDF.
            constexpr int kCoarse = static_cast<int>(sizeof(sm.u) / sizeof(acc_t));
            int lb = 0;
            while (((static_cast<int64_t>(N) + (1ll << lb) - 1) >> lb) > kCoarse) ++lb;
            const int nb = static_cast<int>((static_cast<int64_t>(N) + (1ll << lb) - 1) >> lb);
            acc_t *cs = reinterpret_cast<acc_t *>(&sm.u);
            for (int i = tid; i < nb; i += kThreads) {
                const int64_t last = ((static_cast<int64_t>(i) + 1) << lb) - 1;
                cs[PF_IDX(i, kCoarse)] = __ldg(cdf + (last < N ? last : N - 1));
            }
            __syncthreads();
#pragma unroll
            for (int m = 0; m < kItems; ++m) {
                if (hi[m] > 0) {
                    int a = 0, b = nb - 1;        // first block whose last value reaches u
                    while (a < b) {
                        const int mid = (a + b) >> 1;
                        if (cs[PF_IDX(mid, kCoarse)] >= uq[m]) b = mid; else a = mid + 1;
                    }
                    const int64_t bl = static_cast<int64_t>(a) << lb, bh = ((static_cast<int64_t>(a) + 1) << lb) - 1;
                    lo[m] = static_cast<int>(bl);
                    hi[m] = static_cast<int>(bh < N ? bh : N - 1);
                }
            }
        }
        for (bool more = true; more;) {           // first k with C_k >= u, in [lo, hi]
            more = false;
#pragma unroll
            for (int m = 0; m < kItems; ++m) {
                if (lo[m] < hi[m]) {
                    const int mid = lo[m] + ((hi[m] - lo[m]) >> 1);
                    if (__ldg(cdf + mid) >= uq[m]) hi[m] = mid; else lo[m] = mid + 1;
                    more = true;
                }
            }
        }
        const float sx = Tr::kHalf ? static_cast<float>(axi_anc) : 0.0f;
        const float sy = Tr::kHalf ? static_cast<float>(ayi_anc) : 0.0f;
#pragma unroll
        for (int m = 0; m < kItems; ++m) {
            const int e = eb + m;
            if (e < cnt) {
                const int a = lo[m] < N ? lo[m] : N - 1;
                const pos_t xa = Xin[PF_IDX(a, N)], ya = Yin[PF_IDX(a, N)];
                sm.J[PF_IDX(e, kTile)] = a;
                sm.ax[PF_IDX(e, kTile)] = xa;
                sm.ay[PF_IDX(e, kTile)] = ya;
                const float xf = static_cast<float>(to_acc(xa)) + sx, yf = static_cast<float>(to_acc(ya)) + sy;
                bx0 = fminf(bx0, xf); bx1 = fmaxf(bx1, xf);
                by0 = fminf(by0, yf); by1 = fmaxf(by1, yf);
            }
        }
    } else {
        bx0 = bx1 = T.init_xf;
        by0 = by1 = T.init_yf;
    }

    // ------------------------------------------------------------ 1b. likelihood window
    // The bounding box of the heavy ancestors, widened by the drift and 3.5 sigma of the
    // draw: almost all of their offspring's pixels fall inside it.  Computed before the
    // lookback, so that the predecessors publish meanwhile.  (The pull kernel sizes it by
    // the gathered ancestors; the CDF kernel has none.)
    if constexpr (kMode != kModeCdf) {
        if (!gt) warp_box(make_float4(bx0, bx1, by0, by1), sm);   // warp 0 merges them after the barrier
        // the tracker table's share of this tile (after the aggregate is out)
        if (gt) {
            const uint64_t gtag = static_cast<uint64_t>(sm.st.epoch % 0x7fffffffu + 1u) << 32;
            const int K = T.ntiles < static_cast<int>(gridDim.x) ? T.ntiles : static_cast<int>(gridDim.x);
            const int gcells = gw * gh;
            for (int c = lt + K * warp; lt < K && c < gcells; c += K * kWarps) {
                const int px = gx0 + c % gw, py = gy0 + c / gw;
                uint32_t payload;
                if constexpr (Tr::kHalf) {
                    const H v = half_lik<H>(T).warp_at(fv, px, py);
                    payload = static_cast<uint32_t>(*reinterpret_cast<const unsigned short *>(&v));
                } else {
                    payload = warp_disk_sum(fv, px, py);
                }
                if (lane == 0) st_relaxed_u64(&T.gtab[PF_IDX(c, kTableMax)], gtag | payload);
            }
        }
        // the resampling offset u0 of frame t - 1 (Philox tag 1, index 0), once per tile
        if (t > 0 && tid == 32) {
            const uint32_t w0 =
                philox4x32_10(make_uint4(0u, static_cast<uint32_t>(t - 1), 1u, T.tracker_id), T.key_lo, T.key_hi).x;
            if constexpr (kF64) sm.u0d = uniform_f64(w0); else sm.u0f = uniform_f32(w0);
            sm.skeys[0] = T.key_lo; sm.skeys[1] = T.key_hi;
            sm.skeys[2] = static_cast<uint32_t>(t - 1); sm.skeys[3] = T.tracker_id;
        }
        __syncthreads();
        if (!gt && warp == 0) {   // the block's box, in every lane of warp 0
            const float4 b = merge_warp_boxes(sm);
            bx0 = b.x; bx1 = b.y; by0 = b.z; by1 = b.w;
        }
        if (!gt && tid == 0) {
            // Every draw lies within kDrawMax sigma: if that window takes a single pass of
            // the block, no offspring needs the direct route; otherwise kWindowSigmas
            // (the tracker's window policy may force either).
            float mxr = fabsf(T.drift_xf) + kDrawMax * T.sigma_xf + 1.0f;
            float myr = fabsf(T.drift_yf) + kDrawMax * T.sigma_yf + 1.0f;
            if (T.window == 1 ||
                (T.window == 0 && (ceilf(bx1 + mxr) - floorf(bx0 - mxr) + 1.0f) * (ceilf(by1 + myr) - floorf(by0 - myr) + 1.0f) >
                                      static_cast<float>(kThreads))) {
                mxr = fabsf(T.drift_xf) + kWindowSigmas * T.sigma_xf + 1.0f;
                myr = fabsf(T.drift_yf) + kWindowSigmas * T.sigma_yf + 1.0f;
            }
            int ww = 0, wh = 0, x0 = 0, y0 = 0;
            if (bx0 <= bx1 && by0 <= by1 && bx1 - bx0 < 4096.0f && by1 - by0 < 4096.0f &&
                fabsf(bx0) < 1.0e6f && fabsf(by0) < 1.0e6f && mxr < 4096.0f && myr < 4096.0f) {
                x0 = static_cast<int>(floorf(bx0 - mxr));
                y0 = static_cast<int>(floorf(by0 - myr));
                ww = static_cast<int>(ceilf(bx1 + mxr)) - x0 + 1;
                wh = static_cast<int>(ceilf(by1 + myr)) - y0 + 1;
                const int64_t cells = static_cast<int64_t>(ww) * wh;
                const int64_t roi = static_cast<int64_t>(ww + 2 * r + 1) * (wh + 2 * r);
                // (a table is built even for fewer particles than cells: 81-odd global loads
                // in a dependent chain per particle cost more than the table's shared loads)
                if (cells > kTableMax || roi > kRoiMax) { ww = 0; wh = 0; }
            }
            sm.win_x0 = x0; sm.win_y0 = y0; sm.win_w = ww; sm.win_h = wh;
        }
        if (!gt) __syncthreads();
    }
    const bool no_table = kMode == kModeCdf;
    const int wx0 = no_table ? 0 : sm.win_x0, wy0 = no_table ? 0 : sm.win_y0;
    const int ww = no_table ? 0 : sm.win_w, wh = no_table ? 0 : sm.win_h;
    const int cells = ww * wh;
    if (kMode != kModeCdf && T.dbg_win && tid == 0) {   // test hook: the tile's window
        int32_t *dw = T.dbg_win + PF_IDX(4 * lt, 4 * T.ntiles);
        dw[0] = wx0; dw[1] = wy0; dw[2] = ww; dw[3] = wh;
    }
    HalfLik<H> hk;
    if constexpr (Tr::kHalf) hk = half_lik<H>(T);

    const acc_t c1 = kF64 ? static_cast<acc_t>(T.c1) : static_cast<acc_t>(T.c1f);
    const acc_t c2D = kF64 ? static_cast<acc_t>(T.c2 * T.D) : static_cast<acc_t>(T.c2Df);
    const acc_t den = kF64 ? static_cast<acc_t>(T.den) : static_cast<acc_t>(T.denf);

    // ------------------------------------------------------------ 1c. likelihood table
    if (kMode != kModeCdf && cells > 0 && !gt) {
        // stage the frame region the window's templates cover (clamped to the frame);
        // warp w takes rows w, w + kWarps, ...; its lanes walk the row
        const int rx0 = wx0 - r, ry0 = wy0 - r, rw = ww + 2 * r, rh = wh + 2 * r;
        bool paired = false;
        if constexpr (P == 2) paired = hk.half_acc && rw * rh <= kRoiMax / 2;
        for (int yy = warp; yy < rh; yy += kWarps) {
            const uint8_t *row = fv.p + static_cast<int64_t>(clampi(ry0 + yy, 0, fv.H - 1)) * fv.pitch;
            if constexpr (P == 2) {
                if (paired) {
                    // term2[x] = (term x, term x + 1): the right neighbour from the next lane
                    // (lane 31 loads it; x + 1 = rw reads the clamped pixel after the row)
                    for (int x0 = 0; x0 < rw; x0 += 32) {
                        const int xx = x0 + lane;
                        const H tx = hk.term(__ldg(row + clampi(rx0 + xx, 0, fv.W - 1)));
                        H tn = __shfl_down_sync(0xffffffffu, tx, 1);
                        if (lane == 31) tn = hk.term(__ldg(row + clampi(rx0 + xx + 1, 0, fv.W - 1)));
                        if (xx < rw) sm.u.term2[PF_IDX(yy * rw + xx, kRoiMax / 2)] = __halves2half2(tx, tn);
                    }
                    continue;
                }
            }
            if constexpr (Tr::kHalf) {
                for (int xx = lane; xx < rw; xx += 32)
                    sm.u.term[PF_IDX(yy * rw + xx, kRoiMax)] = hk.term(__ldg(row + clampi(rx0 + xx, 0, fv.W - 1)));
            } else {
                // integer form: exclusive row prefix sums pre[y * (rw + 1) + x] = sum of the
                // row's pixels 0 .. x-1 (uint16, modular), by a warp scan per 32 columns
                const int last = yy * (rw + 1) + rw;      // the row's last prefix entry
                uint16_t *pre = sm.u.pre + (PF_IDX(last, kRoiMax) == last ? last - rw : 0);
                if (lane == 0) pre[0] = 0;
                uint32_t carry = 0;
                for (int x0 = 0; x0 < rw; x0 += 32) {
                    const int xx = x0 + lane;
                    uint32_t v = (xx < rw) ? static_cast<uint32_t>(__ldg(row + clampi(rx0 + xx, 0, fv.W - 1))) : 0u;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
                        if (lane >= o) v += y;
                    }
                    if (xx < rw) pre[xx + 1] = static_cast<uint16_t>(carry + v);
                    carry += __shfl_sync(0xffffffffu, v, 31);
                }
            }
        }
        __syncthreads();
        if (paired) {
            // two neighbouring cells (cx, cx + 1) a thread, one in each half2 lane: each lane
            // performs its cell's additions of from_terms in the same order (an odd row's
            // last pair computes a cell past the row and drops it)
            const int hpr = (ww + 1) >> 1;
            for (int pi = tid; pi < hpr * wh; pi += kThreads) {
                const int cy = pi / hpr, cx = 2 * (pi - cy * hpr);
                __half2 acc = __float2half2_rn(0.0f);
                for (int i = 0; i <= 2 * r; ++i) {
                    const int hw = sm.w[i];
                    const int b = (cy + i) * rw + cx + r;
                    __half2 rs = __float2half2_rn(0.0f);
#pragma unroll 4
                    for (int dx = -hw; dx <= hw; ++dx) rs = __hadd2(rs, sm.u.term2[PF_IDX(b + dx, kRoiMax / 2)]);
                    acc = __hadd2(acc, rs);
                }
                const int c = cy * ww + cx;
                const __half2 a2 = acc;
                lik_t *tab = sm.table;
                tab[PF_IDX(c, kTableMax)] = *reinterpret_cast<const lik_t *>(&a2);
                if (cx + 1 < ww) tab[PF_IDX(c + 1, kTableMax)] = reinterpret_cast<const lik_t *>(&a2)[1];
            }
        }
        const int wdiv = kMode != kModeCdf ? ww : 1;    // (no table in the CDF kernel)
        for (int c = paired ? cells : tid, cy = tid / wdiv, cx = tid - (tid / wdiv) * wdiv; c < cells; c += kThreads) {
            if constexpr (Tr::kHalf) {
                sm.table[PF_IDX(c, kTableMax)] = hk.from_terms(sm.u.term, rw, sm.w, r, cx, cy);
            } else {
                uint32_t ssum = 0;
#pragma unroll 4
                for (int i = 0; i <= 2 * r; ++i) {
                    const uint16_t *p = sm.u.pre + (cy + i) * (rw + 1) + cx + r;
                    const int hw = sm.w[i];
                    ssum += static_cast<uint32_t>(static_cast<uint16_t>(p[hw + 1] - p[-hw]));
                }
                sm.table[PF_IDX(c, kTableMax)] = lik_from_sum<acc_t>(ssum, c1, c2D, den);
            }
            cx += kThreads;               // next cell: kThreads further in row-major order
            while (cx >= ww) { cx -= ww; ++cy; }
        }
        // (no barrier: the next one, before the offspring, orders the table's writes)
    }

    // ------------------------------------------------------------ 1d. lookback, CDF, strata
    int Jr[kItems];           // J of the thread's elements (frames t > 0)
    int jb, je;               // the tile's offspring are j in [jb, je)
    if (!kPull && t > 0) {
        // the step kernel's window phase ordered the tile aggregate (sm.agg_x) and the warps'
        // running maxima before this point; the CDF kernel has no window phase
        if constexpr (kMode == kModeCdf) __syncthreads();
        {   // the block part of the running max
            acc_t wmax = static_cast<acc_t>(0);
            if constexpr (kF64) {
#pragma unroll
                for (int w = 0; w < kWarps; ++w) {
                    const acc_t v = sm.warp_max[w];
                    if (w < warp) wmax = fmax(wmax, v);
                }
            } else {   // lane w < warp holds warp w's maximum (prefixes are >= 0): one redux
                wmax = warp_max(lane < warp ? sm.warp_max[lane] : static_cast<acc_t>(0));
            }
            if (lane == 0) mex = wmax; else mex = fmax(mex, wmax);
#pragma unroll
            for (int m = 0; m < kItems; ++m) loc[m] = fmax(loc[m], mex);
        }
        const acc_t invS = Lp.shard ? static_cast<acc_t>(Lp.g_invS)
                                    : (kF64 ? static_cast<acc_t>(sm.st.invS) : static_cast<acc_t>(sm.st.invS_f));
#ifdef PF_NAIVE_RESAMPLE
        const acc_t Sdiv = static_cast<acc_t>(sm.st.S);   // study build: a division per element
#endif
        const acc_t u0 = kF64 ? static_cast<acc_t>(sm.u0d) : static_cast<acc_t>(sm.u0f);
#ifdef PF_NAIVE_RESAMPLE
        const acc_t inv_n = static_cast<acc_t>(N);     // the study build divides by N per point
#else
        const acc_t inv_n = sizeof(acc_t) == 8 ? static_cast<acc_t>(T.inv_n) : static_cast<acc_t>(T.inv_n_f);
#endif
        // exact prefix before the tile (every thread) and after it (published as inclusive)
        const U128 exclx = (lt > 0) ? lookback<P>(look, lt, dtag, st, sm) : U128{0ull, 0ull};
        const U128 endx = add128(exclx, sm.agg_x);
        if (tid == 0 && lt > 0) desc_publish(&look[lt], 1, endx, dtag);
        // Prefix of the tile's elements: FP inside the tile, pinned to the exact fixed-point
        // values at both tile boundaries, so neighbouring tiles see the same boundary.
        acc_t excl, pend;
        if constexpr (kF64) { excl = from_fixed(exclx); pend = from_fixed(endx); }
        else { excl = from_fixed_f(exclx); pend = from_fixed_f(endx); }
        if constexpr (kMode == kModeCdf) {
            acc_t *const cdf = static_cast<acc_t *>(T.cdf);
            // a shard: its prefix starts at the other ranks' total before it and ends pinned
            // at shard_hi, the value its successor starts from
            const acc_t slo = static_cast<acc_t>(Lp.shard_lo), shi = static_cast<acc_t>(Lp.shard_hi);
            if (Lp.shard) { excl = add_rn(excl, slo); pend = add_rn(pend, slo); }
#pragma unroll
            for (int m = 0; m < kItems; ++m) {
                const int e = eb + m;
                if (e < cnt) {
                    const int k = k0 + e;
                    acc_t Pk = (e == cnt - 1) ? pend : fmin(add_rn(excl, loc[m]), pend);
                    if (Lp.shard) Pk = (k == N - 1) ? shi : fmin(Pk, shi);
                    acc_t C = fmin(PF_NORM(Pk), static_cast<acc_t>(1));
                    if (k == N - 1 && (!Lp.shard || Lp.shard_last)) C = static_cast<acc_t>(1);
                    cdf[PF_IDX(k, N)] = C;
                }
            }
            return;                       // the pull kernel takes the offspring
        }
        // J of the tile's first element and of each element, for either resampling scheme
#ifdef PF_NAIVE_RESAMPLE
        const acc_t nrm = Sdiv;
#else
        const acc_t nrm = invS;
#endif
        int jbl = 0, jprev0 = 0;   // the tile's first count; the count before the thread's first element
        if (T.resampler == kResampleStratified) {
            // (key_lo, key_hi, frame t - 1, tracker id) of the stratum offsets
            Strata<acc_t, true> str;
            str.init(N, static_cast<acc_t>(0.5), inv_n, sm.skeys);   // u0 = 1/2 only centres the estimate
            strata_counts(str, loc, Jr, excl, pend, nrm, eb, cnt, k0, N, dbg_cdf, st);
            jbl = (lt == 0) ? 0 : str.count_le(fmin(PF_NORM(excl), static_cast<acc_t>(1)));
            // (see the systematic branch for the count before the thread's first element)
            if (lane == 0 && tid != 0 && eb < cnt)
                jprev0 = str.count_le(fmin(PF_NORM(fmin(add_rn(excl, mex), pend)), static_cast<acc_t>(1)));
            if (tid == 0) jprev0 = jbl;
        } else {
            Strata<acc_t, false> str;
            str.init(N, u0, inv_n);
            strata_counts(str, loc, Jr, excl, pend, nrm, eb, cnt, k0, N, dbg_cdf, st);
            jbl = (lt == 0) ? 0 : str.count_le(fmin(PF_NORM(excl), static_cast<acc_t>(1)));
            // The count before a warp's first element: that element's predecessor is the
            // previous warp's last, whose clamped prefix is the running max of all preceding
            // warps (the running max at lane 0 of this warp, mex), so the count is taken here
            // from the same value, with the same arithmetic, as its owner takes it.
            if (lane == 0 && tid != 0 && eb < cnt)
                jprev0 = str.count_le(fmin(PF_NORM(fmin(add_rn(excl, mex), pend)), static_cast<acc_t>(1)));
            if (tid == 0) jprev0 = jbl;
        }
        // Every thread knows the tile's first count and the count before its first element,
        // so the ancestor map's heads go in now (phase 1e fills the gaps): map[jp - jb] =
        // 1 + element, jp the first offspring of each element that has offspring.
        {
            int jpt = __shfl_up_sync(0xffffffffu, Jr[kItems - 1], 1);
            if (lane == 0) jpt = jprev0;
#pragma unroll
            for (int m = 0; m < kItems; ++m) {
                const int jp = m ? Jr[m - 1] : jpt;
                if (eb + m < cnt && Jr[m] > jp && jp - jbl < kMapMax)
                    sm.map[PF_IDX(jp - jbl, kMapMax)] = static_cast<uint16_t>(eb + m + 1);
            }
        }
        if (tid == 0) sm.jbeg = jbl;
        store_items(sm.J + eb, Jr);
        if (gt) fetch_table<P>(T, sm, wx0, wy0, ww, cells, fv, c1, c2D, den, st);
        __syncthreads();          // J, jbeg and the likelihood table are complete
        jb = sm.jbeg;
        je = sm.J[cnt - 1];
    } else {
        jb = k0;
        je = k0 + cnt;
        if (gt) fetch_table<P>(T, sm, wx0, wy0, ww, cells, fv, c1, c2D, den, st);
        __syncthreads();          // the likelihood table is complete
    }
    const int nout = je - jb;

    // ------------------------------------------------------------ 1e. ancestor map
    // map[j - jb] = 1 + tile element that is the ancestor of offspring j: the heads (phase
    // 1d; the map was cleared at the start of the tile), then a block-wide running max fills
    // the gaps.
    const bool use_map = !kPull && (t > 0) && nout <= kMapMax;
    if (use_map) {
        // thread tid fills entries [tid*ch, tid*ch + ch), ch = 8 or 16 (16-byte vectors)
        const int nv = (nout > kThreads * 8) ? 2 : 1;
        uint4 *mv = reinterpret_cast<uint4 *>(sm.map) + tid * nv;
        uint4 c0 = mv[0], c1 = make_uint4(0u, 0u, 0u, 0u);
        if (nv == 2) c1 = mv[1];
        uint32_t m2 = __vmaxu2(__vmaxu2(__vmaxu2(c0.x, c0.y), __vmaxu2(c0.z, c0.w)),
                               __vmaxu2(__vmaxu2(c1.x, c1.y), __vmaxu2(c1.z, c1.w)));
        int xm = static_cast<int>(max(m2 & 0xffffu, m2 >> 16));
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, xm, o);
            if (lane >= o) xm = max(xm, y);
        }
        if (lane == 31) sm.warp_imax[warp] = xm;
        int run = __shfl_up_sync(0xffffffffu, xm, 1);
        if (lane == 0) run = 0;
        __syncthreads();
        // the maxima of the preceding warps: lane w < warp holds warp w's (entries are >= 0)
        run = max(run, __reduce_max_sync(0xffffffffu, lane < warp ? sm.warp_imax[lane] : 0));
        uint32_t w4[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (i < 4 * nv) {
                const int r1 = max(run, static_cast<int>(w4[i] & 0xffffu));
                const int r2 = max(r1, static_cast<int>(w4[i] >> 16));
                w4[i] = static_cast<uint32_t>(r1) | (static_cast<uint32_t>(r2) << 16);
                run = r2;
            }
        }
        mv[0] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        if (nv == 2) mv[1] = make_uint4(w4[4], w4[5], w4[6], w4[7]);
        __syncthreads();
    }

    // ------------------------------------------------------------ 2-4. offspring
    pos_t *__restrict__ Xout = static_cast<pos_t *>(T.px[out]);
    pos_t *__restrict__ Yout = static_cast<pos_t *>(T.py[out]);
    lik_t *__restrict__ Lout = static_cast<lik_t *>(T.pl[out]);
    int32_t *__restrict__ dbg_anc = T.dbg_anc;
    const uint32_t tctr = static_cast<uint32_t>(t);
    const uint32_t trk_id = T.tracker_id, key_lo = T.key_lo, key_hi = T.key_hi;
    const int jpair0 = static_cast<int>(T.j_base >> 1);   // global pair index of local pair 0
    Stats<acc_t> stats{neg_inf<acc_t>(), 0, 0, 0};
    const acc_t nxa_a = static_cast<acc_t>(nxi), nya_a = static_cast<acc_t>(nyi);
    const int axi = nxi, ayi = nyi;
    const acc_t dxm = kF64 ? static_cast<acc_t>(T.drift_x) : static_cast<acc_t>(T.drift_xf);
    const acc_t dym = kF64 ? static_cast<acc_t>(T.drift_y) : static_cast<acc_t>(T.drift_yf);
    const acc_t sgx = kF64 ? static_cast<acc_t>(T.sigma_x) : static_cast<acc_t>(T.sigma_xf);
    const acc_t sgy = kF64 ? static_cast<acc_t>(T.sigma_y) : static_cast<acc_t>(T.sigma_yf);
    // offsets: the ancestors' anchor minus the offspring's anchor (integers)
    const float shx = static_cast<float>(axi_anc - nxi), shy = static_cast<float>(ayi_anc - nyi);
    const float ix0 = T.init_xf - static_cast<float>(nxi), iy0 = T.init_yf - static_cast<float>(nyi);

    // bounding box of the thread's new positions (for the next step's tracker table, when
    // the tracker is large enough to use one): absolute in REF64 / F32, anchor offsets in
    // half2 lanes in F16 / BF16
    acc_t pbx0 = static_cast<acc_t>(FLT_MAX), pbx1 = static_cast<acc_t>(-FLT_MAX);
    acc_t pby0 = static_cast<acc_t>(FLT_MAX), pby1 = static_cast<acc_t>(-FLT_MAX);
    using HB2 = typename HalfOps<H>::h2;
    HB2 hbx0 = HalfOps<H>::from_f2(65504.0f, 65504.0f), hbx1 = HalfOps<H>::from_f2(-65504.0f, -65504.0f);
    HB2 hby0 = hbx0, hby1 = hbx1;

    // One pair of offspring (j0, j1) = (2q, 2q + 1).  Compile-time flags: V0 / V1, the
    // particle lies in [jb, je); FAST, frame t > 0 with the ancestor map and no debug
    // arrays (the interior pairs of a tile in production take the FAST copy).
    auto pair = [&](const int q, auto V0c, auto V1c, auto FASTc) {
        constexpr bool v0 = decltype(V0c)::value, v1 = decltype(V1c)::value;
        constexpr bool kFast = decltype(FASTc)::value;
        const int j0 = 2 * q, j1 = j0 + 1;
        int e0 = 0, e1 = 0;
        if (kFast) {
            if (v0) e0 = static_cast<int>(sm.map[PF_IDX(j0 - jb, kMapMax)]) - 1;
            if (v1) e1 = static_cast<int>(sm.map[PF_IDX(j1 - jb, kMapMax)]) - 1;
            if (!v0) e0 = e1;
            if (!v1) e1 = e0;
        } else if (t > 0) {
            if constexpr (kPull) {
                // multinomial: the ancestors were gathered into ax/ay at the tile's own
                // output positions (J holds their indices)
                e0 = j0 - k0;
                e1 = j1 - k0;
            } else if (use_map) {
                e0 = v0 ? static_cast<int>(sm.map[PF_IDX(j0 - jb, kMapMax)]) - 1 : 0;
                e1 = v1 ? static_cast<int>(sm.map[PF_IDX(j1 - jb, kMapMax)]) - 1 : 0;
            } else {
                if (v0) e0 = upper_index(sm.J, cnt, j0);
                if (v1) e1 = (v0 && sm.J[e0] > j1) ? e0 : upper_index(sm.J, cnt, j1);
            }
            if (!v0) e0 = e1;
            if (!v1) e1 = e0;
            if (dbg_anc) {
                if constexpr (kPull) {
                    if (v0) dbg_anc[PF_IDX(j0, N)] = sm.J[e0];
                    if (v1) dbg_anc[PF_IDX(j1, N)] = sm.J[e1];
                } else {
                    if (v0) dbg_anc[PF_IDX(j0, N)] = k0 + e0;
                    if (v1) dbg_anc[PF_IDX(j1, N)] = k0 + e1;
                }
            }
        }
        // one Philox block per particle pair: words (x, y) for j0, (z, w) for j1 (a shard's
        // pairs are numbered globally)
        const uint4 wd = philox4x32_10(make_uint4(static_cast<uint32_t>(q + jpair0), tctr, 0u, trk_id), key_lo, key_hi);

        if constexpr (!Tr::kHalf) {
            // ---------------- REF64 / F32: absolute positions, exact-integer likelihood
            acc_t xa0, ya0, xa1, ya1;
            if (t > 0) {
                xa0 = sm.ax[PF_IDX(e0, kTile)]; ya0 = sm.ay[PF_IDX(e0, kTile)];
                xa1 = sm.ax[PF_IDX(e1, kTile)]; ya1 = sm.ay[PF_IDX(e1, kTile)];
            }
            else {
                xa0 = xa1 = kF64 ? static_cast<acc_t>(T.init_x) : static_cast<acc_t>(T.init_xf);
                ya0 = ya1 = kF64 ? static_cast<acc_t>(T.init_y) : static_cast<acc_t>(T.init_yf);
            }
            acc_t n0x, n0y, n1x, n1y;
            if constexpr (sizeof(acc_t) == 8) {
                box_muller(uniform_f64(wd.x), uniform_f64(wd.y), n0x, n0y);
                box_muller(uniform_f64(wd.z), uniform_f64(wd.w), n1x, n1y);
            } else {
                box_muller(uniform_f32(wd.x), uniform_f32(wd.y), n0x, n0y);
                box_muller(uniform_f32(wd.z), uniform_f32(wd.w), n1x, n1y);
            }
            const acc_t x0 = add_rn(add_rn(xa0, dxm), mul_rn(sgx, n0x));
            const acc_t y0 = add_rn(add_rn(ya0, dym), mul_rn(sgy, n0y));
            const acc_t x1 = add_rn(add_rn(xa1, dxm), mul_rn(sgx, n1x));
            const acc_t y1 = add_rn(add_rn(ya1, dym), mul_rn(sgy, n1y));
            const int px0 = pixel_of(x0), py0 = pixel_of(y0), px1 = pixel_of(x1), py1 = pixel_of(y1);
            const unsigned cx0 = static_cast<unsigned>(px0 - wx0), cy0 = static_cast<unsigned>(py0 - wy0);
            const unsigned cx1 = static_cast<unsigned>(px1 - wx0), cy1 = static_cast<unsigned>(py1 - wy0);
            acc_t L0 = static_cast<acc_t>(0), L1 = static_cast<acc_t>(0);
            if (v0) {
                if (cx0 < static_cast<unsigned>(ww) && cy0 < static_cast<unsigned>(wh)) L0 = sm.table[cy0 * ww + cx0];
                else L0 = lik_from_sum<acc_t>(disk_sum(fv, sm.w, px0, py0), c1, c2D, den);
            }
            if (v1) {
                if (cx1 < static_cast<unsigned>(ww) && cy1 < static_cast<unsigned>(wh)) L1 = sm.table[cy1 * ww + cx1];
                else L1 = lik_from_sum<acc_t>(disk_sum(fv, sm.w, px1, py1), c1, c2D, den);
            }
            if (v0 && v1) {
                if constexpr (sizeof(acc_t) == 8) {
                    reinterpret_cast<double2 *>(Xout)[PF_IDX(q, N / 2)] = make_double2(x0, x1);
                    reinterpret_cast<double2 *>(Yout)[q] = make_double2(y0, y1);
                    reinterpret_cast<double2 *>(Lout)[q] = make_double2(L0, L1);
                } else {
                    reinterpret_cast<float2 *>(Xout)[PF_IDX(q, N / 2)] = make_float2(x0, x1);
                    reinterpret_cast<float2 *>(Yout)[q] = make_float2(y0, y1);
                    reinterpret_cast<float2 *>(Lout)[q] = make_float2(L0, L1);
                }
            } else if (v0) {
                Xout[PF_IDX(j0, N)] = x0; Yout[j0] = y0; Lout[j0] = L0;
            } else if (v1) {
                Xout[PF_IDX(j1, N)] = x1; Yout[j1] = y1; Lout[j1] = L1;
            }
            stats_add2<false>(stats, v0, L0, x0 - nxa_a, y0 - nya_a, v1, L1, x1 - nxa_a, y1 - nya_a);
            if (track_box) {
                if (v0) { pbx0 = fmin(pbx0, x0); pbx1 = fmax(pbx1, x0); pby0 = fmin(pby0, y0); pby1 = fmax(pby1, y0); }
                if (v1) { pbx0 = fmin(pbx0, x1); pbx1 = fmax(pbx1, x1); pby0 = fmin(pby0, y1); pby1 = fmax(pby1, y1); }
            }
        } else {
            // ---------------- F16 / BF16: half2 lanes = particles (j0, j1), offsets from the anchor
            using OPS = HalfOps<H>;
            using h2 = typename OPS::h2;
            h2 ox, oy;
            if (t > 0) {
                ox = OPS::pack(sm.ax[PF_IDX(e0, kTile)], sm.ax[PF_IDX(e1, kTile)]);
                oy = OPS::pack(sm.ay[PF_IDX(e0, kTile)], sm.ay[PF_IDX(e1, kTile)]);
                if (shx != 0.0f || shy != 0.0f) {
                    ox = __hadd2(ox, OPS::from_f2(shx, shx));
                    oy = __hadd2(oy, OPS::from_f2(shy, shy));
                }
            } else {
                ox = OPS::from_f2(ix0, ix0);
                oy = OPS::from_f2(iy0, iy0);
            }
            float a, b, c, d;
            box_muller_fast(uniform_f32(wd.x), uniform_f32(wd.y), a, b);
            box_muller_fast(uniform_f32(wd.z), uniform_f32(wd.w), c, d);
            ox = __hadd2(ox, OPS::from_f2(dxm + sgx * a, dxm + sgx * c));
            oy = __hadd2(oy, OPS::from_f2(dym + sgy * b, dym + sgy * d));
            const int px0 = axi + pixel_of(OPS::lo(ox)), py0 = ayi + pixel_of(OPS::lo(oy));
            const int px1 = axi + pixel_of(OPS::hi(ox)), py1 = ayi + pixel_of(OPS::hi(oy));
            const unsigned cx0 = static_cast<unsigned>(px0 - wx0), cy0 = static_cast<unsigned>(py0 - wy0);
            const unsigned cx1 = static_cast<unsigned>(px1 - wx0), cy1 = static_cast<unsigned>(py1 - wy0);
            const bool in0 = cx0 < static_cast<unsigned>(ww) && cy0 < static_cast<unsigned>(wh);
            const bool in1 = cx1 < static_cast<unsigned>(ww) && cy1 < static_cast<unsigned>(wh);
            H l0 = in0 ? sm.table[cy0 * ww + cx0] : OPS::from_f(0.0f);
            H l1 = in1 ? sm.table[cy1 * ww + cx1] : OPS::from_f(0.0f);
            if (v0 && !in0) l0 = hk.at(fv, sm.w, px0, py0);
            if (v1 && !in1) l1 = hk.at(fv, sm.w, px1, py1);
            if (v0 && v1) {
                reinterpret_cast<h2 *>(Xout)[PF_IDX(q, N / 2)] = ox;
                reinterpret_cast<h2 *>(Yout)[q] = oy;
                reinterpret_cast<h2 *>(Lout)[q] = OPS::pack(l0, l1);
            } else if (v0) {
                Xout[PF_IDX(j0, N)] = OPS::lo_h(ox); Yout[j0] = OPS::lo_h(oy); Lout[j0] = l0;
            } else if (v1) {
                Xout[PF_IDX(j1, N)] = OPS::hi_h(ox); Yout[j1] = OPS::hi_h(oy); Lout[j1] = l1;
            }
            stats_add2<true>(stats, v0, OPS::to_f(l0), OPS::lo(ox), OPS::lo(oy), v1, OPS::to_f(l1), OPS::hi(ox), OPS::hi(oy));
            // (a lane outside [jb, je) holds a draw around a valid ancestor: inside the reach
            // of the next step's table all the same)
            if (track_box) {
                hbx0 = __hmin2(hbx0, ox); hbx1 = __hmax2(hbx1, ox);
                hby0 = __hmin2(hby0, oy); hby1 = __hmax2(hby1, oy);
            }
        }
    };
    {
        using TT = std::true_type;
        using FF = std::false_type;
        const int qi0 = (jb + 1) >> 1, qi1 = je >> 1;   // pairs with both particles in [jb, je)
        if (t > 0 && use_map && !dbg_anc) {
            for (int q = qi0 + tid; q < qi1; q += kThreads) pair(q, TT{}, TT{}, TT{});
        } else {
            for (int q = qi0 + tid; q < qi1; q += kThreads) pair(q, TT{}, TT{}, FF{});
        }
        // the pairs that straddle the ends of [jb, je)
        if (tid == 0 && (jb & 1) && jb < je) pair(jb >> 1, FF{}, TT{}, FF{});
        if (tid == kThreads - 1 && (je & 1) && je > jb) pair(je >> 1, TT{}, FF{}, FF{});
    }

    // ------------------------------------------------------------ 5. tile partial + finalise
    float4 bb;
    if constexpr (Tr::kHalf) {
        const float ax = static_cast<float>(nxi), ay = static_cast<float>(nyi);
        bb = make_float4(fminf(HalfOps<H>::lo(hbx0), HalfOps<H>::hi(hbx0)) + ax,
                         fmaxf(HalfOps<H>::lo(hbx1), HalfOps<H>::hi(hbx1)) + ax,
                         fminf(HalfOps<H>::lo(hby0), HalfOps<H>::hi(hby0)) + ay,
                         fmaxf(HalfOps<H>::lo(hby1), HalfOps<H>::hi(hby1)) + ay);
    } else {
        // widened to whole pixels outwards, so the float box still contains every position
        bb = make_float4(static_cast<float>(floor(pbx0)), static_cast<float>(ceil(pbx1)),
                         static_cast<float>(floor(pby0)), static_cast<float>(ceil(pby1)));
    }
    if (track_box) warp_box(bb, sm);
    const Stats<acc_t> tot = block_stats<P>(stats, sm);
    if (track_box && warp == 0) bb = merge_warp_boxes(sm);
    if (tid == 0) {
        TilePartial *p = &T.part[PF_IDX(lt, T.ntiles)];
        if (track_box) {
            const uint64_t btg = partial_tag(sm.st.epoch);
            st_relaxed_v2(&p->b[0], btg | __float_as_uint(bb.x), btg | __float_as_uint(bb.y));
            st_relaxed_v2(&p->b[2], btg | __float_as_uint(bb.z), btg | __float_as_uint(bb.w));
        }
        uint32_t prev;
        if constexpr (kF64) {
            p->d[0] = tot.m;
            p->d[1] = tot.s;
            p->d[2] = tot.sx;
            p->d[3] = tot.sy;
            // release: the partial is visible before the count; acquire: the last tile sees all
            prev = atom_add_acq_rel(T.done, 1u);
        } else {
            const uint64_t tg = partial_tag(sm.st.epoch);
            st_relaxed_v2(&p->w[0], tg | __float_as_uint(tot.m), tg | __float_as_uint(tot.s));
            st_relaxed_v2(&p->w[2], tg | __float_as_uint(tot.sx), tg | __float_as_uint(tot.sy));
            // the tracker's last tile finalises, waiting for every partial's tag: no tile waits
            // for a counter's round trip (the tiles before it hold lower tickets, so they are
            // running or done)
            prev = static_cast<uint32_t>(lt);
        }
        sm.last = (prev == static_cast<uint32_t>(T.ntiles - 1)) ? 1u : 0u;
    }
    __syncthreads();
    if (sm.last) finalize_tracker<P>(T, st, sm, Lp.est_out ? Lp.est_out + 2 * ti : nullptr, track_box);
}

// CTAs per SM the register allocation must allow: 1024 threads per SM (64 registers a
// thread) for the FP32/FP16/BF16 kernels, 512 for REF64 (its FP64 Box-Muller needs ~128);
// measured best on GB300 for the latency-bound step.
template <int P> struct MinBlocks {
    static constexpr int value = (P == 0 ? 512 : 1024) / kThreads > 0 ? (P == 0 ? 512 : 1024) / kThreads : 1;
};

template <int P, int kMode>
__global__ void __launch_bounds__(kThreads, MinBlocks<P>::value) step_kernel(const StepLaunch Lp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StepSmem<P> &sm = *reinterpret_cast<StepSmem<P> *>(smem_raw);
    // Programmatic dependent launch: a launch that follows another step on the same stream
    // may be scheduled while that one drains; everything it reads (ticket, descriptors,
    // state, particles) is written by its predecessor, so it first waits for the
    // predecessor grid to complete, then lets its own successor be scheduled.  (Both are
    // no-ops for a launch without the programmatic-serialization attribute.)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (threadIdx.x == 0) sm.cached = -1;
    if (Lp.ntrk == 1) {
        // one tracker: its descriptor and state load while the first ticket is drawn
        load_descriptor(Lp, Lp.slot_of ? __ldg(&Lp.slot_of[0]) : 0, 0, sm);
        if (threadIdx.x == 0) sm.cached = 0;
    }
    for (;;) {
        if (threadIdx.x == 0) sm.ticket = atomicAdd(Lp.ticket, 1u);
        __syncthreads();
        const uint32_t g = sm.ticket;
        __syncthreads();
        if (g >= static_cast<uint32_t>(Lp.total_tiles)) {
            if (threadIdx.x == 0 && g == static_cast<uint32_t>(Lp.total_tiles) + gridDim.x - 1u)
                atomicExch(Lp.ticket, 0u);
            return;
        }
        run_tile<P, kMode>(Lp, static_cast<int>(g), sm);
        __syncthreads();
    }
}

// Test hook: the lookback wait on a descriptor that nobody publishes, with a short limit;
// it must give up, raise the timeout bit and return.
__global__ void wait_probe_kernel(const LookbackDesc *d, TrackerState *st, uint32_t limit) {
    U128 v;
    wait_desc(d, desc_tag(1u), st, v, limit);
}

__global__ void philox_kernel(const uint4 *ctrs, int64_t n, uint32_t k0, uint32_t k1, uint4 *out) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(ctrs[i], k0, k1);
}

template <int P>
int configure_and_grid(int total_tiles) {
    // MinBlocks CTAs must fit in an SM's 228 KB of shared memory (1 KB reserved per CTA)
    // (the 1024-thread study build has no REF64 kernel: its tile does not fit)
    static_assert((sizeof(StepSmem<P>) + 1024) * MinBlocks<P>::value <= 228 * 1024 || kThreads > 512,
                  "shared memory of the step kernel exceeds its CTAs per SM");
    if (sizeof(StepSmem<P>) + 1024 > 228 * 1024) return -1;
    const int bytes = static_cast<int>(sizeof(StepSmem<P>));
    if (cudaFuncSetAttribute(step_kernel<P, kModeStep>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess ||
        cudaFuncSetAttribute(step_kernel<P, kModeStepBig>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess ||
        cudaFuncSetAttribute(step_kernel<P, kModeCdf>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess ||
        cudaFuncSetAttribute(step_kernel<P, kModePull>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess)
        return -1;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_kernel<P, kModeStep>, kThreads, bytes);
    if (per_sm < 1) per_sm = 1;
    const int g = sms * per_sm;
    return total_tiles < g ? total_tiles : g;
}

}  // namespace

namespace {
// resident CTAs of the step kernel on the current device (cached per device and precision)
int slots_of(int precision) {
    static std::atomic<int> cache[64][4];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return -1; }
    if (precision < 0 || precision > 3) return -1;
    if (dev >= 0 && dev < 64) {
        const int c = cache[dev][precision].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int g = -1;
    switch (precision) {
        case 0: g = configure_and_grid<0>(0x7fffffff); break;
        case 1: g = configure_and_grid<1>(0x7fffffff); break;
        case 2: g = configure_and_grid<2>(0x7fffffff); break;
        case 3: g = configure_and_grid<3>(0x7fffffff); break;
    }
    if (g > 0 && dev >= 0 && dev < 64) cache[dev][precision].store(g, std::memory_order_relaxed);
    return g;
}
}  // namespace

int step_tile_size(int precision, int64_t n) {
    const int64_t slots = slots_of(precision);
    // a tracker that cannot fill half the device with full tiles keeps full tiles (in a
    // batch, other trackers fill the device)
    if (slots < 1 || n < slots * (kTile / 2)) return kTile;
    const int64_t waves = (n + slots * kTile - 1) / (slots * kTile);
    int64_t tile = (n + slots * waves - 1) / (slots * waves);   // >= kTile / 2 here
    tile = (tile + 7) & ~int64_t(7);
    if (tile > kTile) tile = kTile;
    return static_cast<int>(tile);
}

int step_grid_size(int precision, int total_tiles) {
    switch (precision) {
        case 0: return configure_and_grid<0>(total_tiles);
        case 1: return configure_and_grid<1>(total_tiles);
        case 2: return configure_and_grid<2>(total_tiles);
        case 3: return configure_and_grid<3>(total_tiles);
    }
    return -1;
}

// A step-family launch with programmatic stream serialization: when the previous work on
// the stream is a step kernel (the previous frame), this launch is scheduled while that one
// drains and waits for it on the device (griddepcontrol.wait) instead of the stream
// serialising the two; captured into a CUDA graph as a programmatic dependency.
template <int P, int kMode>
int launch_one(int grid, const StepLaunch &L, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(grid));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = sizeof(StepSmem<P>);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return static_cast<int>(cudaLaunchKernelEx(&cfg, step_kernel<P, kMode>, L));
}

template <int kMode>
int launch_mode(int precision, const StepLaunch &L, int grid, void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (grid < 1) grid = 1;
    int rc = -1;
    switch (precision) {
        case 0: rc = launch_one<0, kMode>(grid, L, s); break;
        case 1: rc = launch_one<1, kMode>(grid, L, s); break;
        case 2: rc = launch_one<2, kMode>(grid, L, s); break;
        case 3: rc = launch_one<3, kMode>(grid, L, s); break;
        default: return -1;
    }
    if (rc != 0) return rc;
    return static_cast<int>(cudaGetLastError());
}

int launch_step(int precision, const StepLaunch &L, int grid, void *stream) {
    // a single tracker of at least two waves of tiles takes the instantiation with the
    // tracker table (the kernel checks the condition again per tile)
    if (L.ntrk == 1 && L.total_tiles >= 2 * grid) return launch_mode<kModeStepBig>(precision, L, grid, stream);
    return launch_mode<kModeStep>(precision, L, grid, stream);
}

int launch_pull(int precision, const StepLaunch &L, int grid, bool with_cdf, void *stream) {
    const int rc = with_cdf ? launch_mode<kModeCdf>(precision, L, grid, stream) : 0;
    return rc != 0 ? rc : launch_mode<kModePull>(precision, L, grid, stream);
}

int launch_cdf(int precision, const StepLaunch &L, int grid, void *stream) {
    return launch_mode<kModeCdf>(precision, L, grid, stream);
}

// A shard's offspring run (see pf_internal.h): one thread per element of the shard's CDF,
// the count at its predecessor (J(c_lo) before the first) and at itself over the global
// strata, and the element's position copied to every offspring slot in between.
template <typename A>
__global__ void shard_expand_kernel(const A *C, const A *x, const A *y, int64_t n, int64_t n_global, int64_t t,
                                    uint32_t key_lo, uint32_t key_hi, uint32_t tracker, A c_lo, A *sx, A *sy,
                                    int64_t cap, int64_t *run, uint32_t *status) {
    const uint32_t w0 = philox4x32_10(make_uint4(0u, static_cast<uint32_t>(t - 1), 1u, tracker), key_lo, key_hi).x;
    const A u0 = sizeof(A) == 8 ? static_cast<A>(uniform_f64(w0)) : static_cast<A>(uniform_f32(w0));
    const A inv_n = sizeof(A) == 8 ? static_cast<A>(1.0 / static_cast<double>(n_global))
                                   : static_cast<A>(1.0f / static_cast<float>(n_global));
    Strata<A, false> str;
    str.init(static_cast<int>(n_global), u0, inv_n);
    const int64_t jb = str.count_le(c_lo);
    for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < n;
         k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t j0 = k == 0 ? jb : str.count_le(C[k - 1]);
        const int64_t j1 = str.count_le(C[k]);
        const A xa = x[k], ya = y[k];
        for (int64_t j = j0; j < j1; ++j) {
            const int64_t i = j - jb;
            if (i >= 0 && i < cap) { sx[i] = xa; sy[i] = ya; }
            else atomicOr(status, 1u);
        }
        if (k == 0) run[0] = jb;
        if (k == n - 1) run[1] = j1;
    }
}

int launch_shard_expand(int precision, const void *cdf, const void *x, const void *y, int64_t n, int64_t n_global,
                        int64_t t, uint32_t key_lo, uint32_t key_hi, uint32_t tracker, double c_lo, void *sx,
                        void *sy, int64_t cap, int64_t *run, uint32_t *status, void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const unsigned blocks = static_cast<unsigned>(std::min<int64_t>((n + 255) / 256, 4096));
    if (precision == 0)
        shard_expand_kernel<double><<<blocks, 256, 0, s>>>(
            static_cast<const double *>(cdf), static_cast<const double *>(x), static_cast<const double *>(y), n, n_global,
            t, key_lo, key_hi, tracker, c_lo, static_cast<double *>(sx), static_cast<double *>(sy), cap, run, status);
    else if (precision == 1)
        shard_expand_kernel<float><<<blocks, 256, 0, s>>>(
            static_cast<const float *>(cdf), static_cast<const float *>(x), static_cast<const float *>(y), n, n_global,
            t, key_lo, key_hi, tracker, static_cast<float>(c_lo), static_cast<float *>(sx), static_cast<float *>(sy),
            cap, run, status);
    else
        return -1;
    return static_cast<int>(cudaGetLastError());
}

int launch_wait_probe(void *d_desc, void *d_state, uint32_t limit, void *stream) {
    wait_probe_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const LookbackDesc *>(d_desc), static_cast<TrackerState *>(d_state), limit);
    return static_cast<int>(cudaGetLastError());
}

int launch_debug_philox(const uint32_t *d_ctrs, int64_t n, uint64_t seed, uint32_t *d_out, void *stream) {
    if (n <= 0) return 0;
    const int64_t blocks = (n + 255) / 256;
    philox_kernel<<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const uint4 *>(d_ctrs), n, static_cast<uint32_t>(seed & 0xffffffffu),
        static_cast<uint32_t>(seed >> 32), reinterpret_cast<uint4 *>(d_out));
    return static_cast<int>(cudaGetLastError());
}

}  // namespace pfk
