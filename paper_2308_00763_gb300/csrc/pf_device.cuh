// pf_device.cuh -- device building blocks of the SIR step (sm_103a, CUDA cores only).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace pfk {

// ----------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): a counter-based generator, so the
// draw of particle j at frame t is a pure function of (seed, j, t, tag, tracker) and no
// generator state is stored (the paper draws with cuRAND, Sec. IV after Eq. 2).
// ----------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        if (round < 9) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
    }
    return c;
}

// Uniform on (0,1) from the top 23 bits: ((w >> 9) + 1/2) * 2^-23, exact in FP32 and
// FP64, so every precision sees the same uniforms.
__device__ __forceinline__ float uniform_f32(uint32_t w) {
    return (static_cast<float>(w >> 9) + 0.5f) * 1.1920928955078125e-07f;
}
__device__ __forceinline__ double uniform_f64(uint32_t w) {
    return (static_cast<double>(w >> 9) + 0.5) * 1.1920928955078125e-07;
}

// Box-Muller: two N(0,1) draws from two uniforms.
__device__ __forceinline__ void box_muller(double ua, double ub, double &nx, double &ny) {
    const double rad = sqrt(-2.0 * log(ua));
    double s, c;
    sincospi(2.0 * ub, &s, &c);
    nx = rad * c;
    ny = rad * s;
}
__device__ __forceinline__ void box_muller(float ua, float ub, float &nx, float &ny) {
    const float rad = sqrtf(-2.0f * logf(ua));
    float s, c;
    sincospif(2.0f * ub, &s, &c);
    nx = rad * c;
    ny = rad * s;
}

// Box-Muller with the hardware approximations (log2, sqrt, sin/cos special-function
// units), for the FP16/BF16 filters whose positions keep ~11 bits anyway.  The angle
// is taken in [-pi, pi), where the sin/cos approximations are most accurate:
// (cos, sin)(2 pi u - pi) = -(cos, sin)(2 pi u).
__device__ __forceinline__ float sqrt_approx(float v) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ void box_muller_fast(float ua, float ub, float &nx, float &ny) {
    const float rad = sqrt_approx(-1.3862943611198906f * __log2f(ua));   // -2 ln u = -2 ln2 log2 u
    const float ang = 6.2831853071795865f * (ub - 0.5f);
    float s, c;
    __sincosf(ang, &s, &c);
    nx = -rad * c;
    ny = -rad * s;
}

// ----------------------------------------------------------------------------------
// Explicitly rounded arithmetic (no contraction), used where the result must equal the
// same expression evaluated elsewhere.
// ----------------------------------------------------------------------------------
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }

__device__ __forceinline__ double exp_acc(double x) { return exp(x); }
__device__ __forceinline__ float exp_acc(float x) { return expf(x); }

template <typename A> __device__ __forceinline__ A neg_inf();
template <> __device__ __forceinline__ double neg_inf<double>() { return -__longlong_as_double(0x7ff0000000000000ll); }
template <> __device__ __forceinline__ float neg_inf<float>() { return -__int_as_float(0x7f800000); }

// ----------------------------------------------------------------------------------
// Resampling points (Sec. IV, "Resampling"): stratum j is sampled at u_j = (j + v_j) * (1/N),
// evaluated in the CDF's precision A; systematic resampling takes v_j = u0 for every j,
// stratified resampling an independent v_j per stratum.  count_le(c) is the number of
// strata with u_j <= c; particle k receives strata [count_le(C_{k-1}), count_le(C_k)),
// which is exactly a_j = min{k : C_k >= u_j} for a non-decreasing C.  u_j is
// non-decreasing in j (both roundings are monotone, and (A)j + v_j stays within
// [j, j + 1] while (A)j is exact), so the count is found from an arithmetic estimate and a
// short galloping search.
// ----------------------------------------------------------------------------------
template <typename A>
__device__ __forceinline__ A stratum_point32(int j, A u0, A inv_n) {
#ifdef PF_NAIVE_RESAMPLE
    // study build: a reciprocal per point, (j + u0) / N (inv_n carries N here)
    return div_rn(add_rn(static_cast<A>(j), u0), inv_n);
#else
    return mul_rn(add_rn(static_cast<A>(j), u0), inv_n);
#endif
}

// Strata of one tracker's frame: n = N, 1/N, the offsets and the first / last points.
// kStrat: stratified, v_j = uniform word j % 4 of Philox(j / 4, tf, 1, trk), with
// (key_lo, key_hi, tf, trk) read from `keys` (shared memory); else systematic, v_j = u0.
template <typename A, bool kStrat>
struct Strata {
    A u0, inv_n, first, last, nf;
    int n;
    const uint32_t *keys;
    __device__ __forceinline__ void init(int n_, A u0_, A inv_n_, const uint32_t *keys_ = nullptr) {
        n = n_; u0 = u0_; inv_n = inv_n_; keys = keys_;
        first = point(0);
        last = point(n - 1);
        nf = static_cast<A>(n);
    }
    __device__ __forceinline__ uint4 strat_block(int j) const {
        return philox4x32_10(make_uint4(static_cast<uint32_t>(j) >> 2, keys[2], 1u, keys[3]), keys[0], keys[1]);
    }
    __device__ __forceinline__ A strat_point_from(const uint4 &w, int j) const {
        const int q = j & 3;
        const uint32_t x = q == 0 ? w.x : (q == 1 ? w.y : (q == 2 ? w.z : w.w));
        const A v = sizeof(A) == 8 ? static_cast<A>(uniform_f64(x)) : static_cast<A>(uniform_f32(x));
        return stratum_point32<A>(j, v, inv_n);
    }
    __device__ __noinline__ A strat_point(int j) const { return strat_point_from(strat_block(j), j); }
    // The two probes of count_le for stratified points: one Philox block serves both when
    // the neighbour shares it (three times in four).
    __device__ __noinline__ int strat_probes(A c, int j) const {
        const uint4 w = strat_block(j);
        const bool a = strat_point_from(w, j) <= c;
        const int nb = a ? j + 1 : j - 1;
        const bool b = ((nb >> 2) == (j >> 2) ? strat_point_from(w, nb) : strat_point(nb)) <= c;
        if (a != b) return a ? j + 1 : j;
        return -1;
    }
    __device__ __forceinline__ A point(int j) const {
        if constexpr (kStrat) return strat_point(j);
        else return stratum_point32<A>(j, u0, inv_n);
    }
    // number of strata j with u_j <= c
    __device__ __forceinline__ int count_le(A c) const {
        if (!(first <= c)) return 0;   // also NaN
        if (last <= c) return n;
        const A est = c * nf - u0;
        int j = (est > static_cast<A>(0)) ? static_cast<int>(est) : 0;
        if (j > n - 2) j = n - 2;
        // The estimate is almost always within one stratum of the answer: probe u_j and its
        // neighbour on the far side (j = 0 has u_0 = first <= c, so j - 1 is never probed
        // below 0), and search only when both probes fall on the same side.
        if constexpr (kStrat) {
            const int r = strat_probes(c, j);
            return r >= 0 ? r : search(c, j);
        } else {
            const bool a = point(j) <= c;
            const bool b = point(a ? j + 1 : j - 1) <= c;
            if (a != b) return a ? j + 1 : j;
            return search(c, j);
        }
    }
    // the count for u_0 <= c < u_{n-1}, from the start point j (galloping, then bisection)
    __device__ __noinline__ int search(A c, int j) const {
        // invariant wanted: u(lo) <= c < u(hi), 0 <= lo < hi <= n - 1
        int lo, hi;
        if (point(j) <= c) {
            lo = j;
            hi = j + 1;
            long long step = 1;
            while (hi < n - 1 && point(hi) <= c) {
                lo = hi;
                step <<= 1;
                hi = (hi + step < n - 1) ? static_cast<int>(hi + step) : n - 1;
            }
        } else {
            hi = j;
            lo = j - 1;
            long long step = 1;
            while (lo > 0 && !(point(lo) <= c)) {
                hi = lo;
                step <<= 1;
                lo = (lo > step) ? static_cast<int>(lo - step) : 0;
            }
        }
        while (hi - lo > 1) {
            const int mid = lo + ((hi - lo) >> 1);
            if (point(mid) <= c) lo = mid; else hi = mid;
        }
        return lo + 1;
    }
};

// ----------------------------------------------------------------------------------
// 128-bit fixed point for the inter-tile prefix of the CDF scan: x -> round-down(x * 2^90).
// Tile aggregates are at most 2^12 and a tracker's total at most 2^31, so 2^121 bounds
// every value; the sum of integers is exact and associative.
// ----------------------------------------------------------------------------------
constexpr int kFixShift = 90;

struct U128 {
    uint64_t lo, hi;
};

__device__ __forceinline__ U128 add128(U128 a, U128 b) {
    U128 r;
    r.lo = a.lo + b.lo;
    r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
    return r;
}

// Non-negative finite double -> floor(v * 2^90) (values below 2^-90 become 0).
__device__ __forceinline__ U128 to_fixed(double v) {
    U128 r{0ull, 0ull};
    if (!(v > 0.0)) return r;
    const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(v));
    const int ex = static_cast<int>((bits >> 52) & 0x7ff);
    if (ex == 0) return r;  // subnormal: far below 2^-90
    const uint64_t mant = (bits & 0xfffffffffffffull) | 0x10000000000000ull;  // 53 bits
    const int sh = ex - 1075 + kFixShift;   // v * 2^90 = mant * 2^sh
    if (sh <= -53) return r;
    if (sh < 0) { r.lo = mant >> (-sh); return r; }
    if (sh == 0) { r.lo = mant; return r; }
    if (sh < 64) { r.lo = mant << sh; r.hi = mant >> (64 - sh); return r; }
    r.hi = mant << (sh - 64);
    return r;
}

// Non-negative finite float -> floor(v * 2^90).
__device__ __forceinline__ U128 to_fixed(float v) {
    U128 r{0ull, 0ull};
    if (!(v > 0.0f)) return r;
    const uint32_t bits = __float_as_uint(v);
    const int ex = static_cast<int>((bits >> 23) & 0xff);
    if (ex == 0) return r;  // subnormal: far below 2^-90
    const uint64_t mant = (bits & 0x7fffffu) | 0x800000u;  // 24 bits
    const int sh = ex - 150 + kFixShift;   // v * 2^90 = mant * 2^sh
    if (sh <= -24) return r;
    if (sh < 0) { r.lo = mant >> (-sh); return r; }
    if (sh == 0) { r.lo = mant; return r; }
    if (sh < 64) { r.lo = mant << sh; r.hi = mant >> (64 - sh); return r; }
    r.hi = mant << (sh - 64);
    return r;
}

// Fixed point -> float: the top 64 significant bits rounded to nearest (monotone,
// deterministic); no FP64 instruction.
__device__ __forceinline__ float from_fixed_f(U128 x) {
    if (x.hi == 0ull && (x.lo >> 32) == 0ull)
        return __uint2float_rn(static_cast<uint32_t>(x.lo)) * 8.0779356694631609e-28f;   // 2^-90
    // normalise so the top set bit is bit 63 of `top`, value = top * 2^e2
    const int lz = x.hi ? __clzll(static_cast<long long>(x.hi)) : 64 + __clzll(static_cast<long long>(x.lo));
    uint64_t top;
    if (lz == 0) top = x.hi;
    else if (lz < 64) top = (x.hi << lz) | (x.lo >> (64 - lz));
    else top = x.lo << (lz - 64);
    const int e2 = 64 - lz - kFixShift;                     // in [-121, -26]
    // round to nearest on the top 32 bits with the rest folded into a sticky bit: the
    // same result as converting all 64 bits (24 + guard + round bits are inside the 32),
    // without a 64-bit integer conversion
    const uint32_t t32 = static_cast<uint32_t>(top >> 32) | (static_cast<uint32_t>(top) != 0u ? 1u : 0u);
    return __uint2float_rn(t32) * __int_as_float((127 + 32 + e2) << 23);
}

// Fixed point -> double: the top 64 significant bits rounded to nearest; monotone
// non-decreasing and deterministic, which is all the scan boundaries rely on.
__device__ __forceinline__ double from_fixed(U128 x) {
    if (x.hi == 0ull) return __ull2double_rn(x.lo) * 8.0779356694631609e-28;   // 2^-90
    const int lz = __clzll(static_cast<long long>(x.hi));
    const uint64_t top = (x.hi << lz) | (lz ? (x.lo >> (64 - lz)) : 0ull);
    const int e2 = 64 - lz - kFixShift;                     // value = top * 2^e2
    const double scale = __longlong_as_double(static_cast<long long>(1023 + e2) << 52);
    return __ull2double_rn(top) * scale;
}

__device__ __forceinline__ U128 shfl_xor128(U128 v, int o) {
    U128 r;
    r.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    r.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    return r;
}
__device__ __forceinline__ U128 shfl_down128(U128 v, int o) {
    U128 r;
    r.lo = __shfl_down_sync(0xffffffffu, v.lo, o);
    r.hi = __shfl_down_sync(0xffffffffu, v.hi, o);
    return r;
}

// ----------------------------------------------------------------------------------
// Precision traits.  acc_t is the precision of the weights, sums, scan and CDF.
// ----------------------------------------------------------------------------------
template <int P> struct Prec;
template <> struct Prec<0> {   // PF_REF64
    using pos_t = double; using lik_t = double; using acc_t = double;
    static constexpr bool kHalf = false;
};
template <> struct Prec<1> {   // PF_F32
    using pos_t = float; using lik_t = float; using acc_t = float;
    static constexpr bool kHalf = false;
};
template <> struct Prec<2> {   // PF_F16
    using pos_t = __half; using lik_t = __half; using acc_t = float;
    static constexpr bool kHalf = true;
};
template <> struct Prec<3> {   // PF_BF16
    using pos_t = __nv_bfloat16; using lik_t = __nv_bfloat16; using acc_t = float;
    static constexpr bool kHalf = true;
};

__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ float to_acc(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }

}  // namespace pfk
