// pf_rejection.cu -- rejection resampling (sm_103a, CUDA cores only).
//
// Sec. III cites rejection resampling (Murray, Lee and Jacob, 2016) beside Metropolis
// resampling as avoiding the prefix sum of the standard schemes.  Offspring j tests the
// candidate k = j, then proposals k' uniform on {0, ..., N-1}, and keeps the first
// candidate with u <= w_k / w_max, in the log form ln u <= L_k - M where M is the maximum
// of L the previous step already computed (the state's M).  Offspring j keeps j with
// probability w_j / w_max and otherwise draws from the normalised weights, so particle k's
// expected offspring count is N w_k / sum w.  Expected tries: N w_max / sum w.
//
// Draws: try i of offspring j reads Philox(i / 2, t - 1, 6 + 256 j, tracker); word
// 2 (i mod 2) gives the proposal k' = floor(w N / 2^32) (unused by try 0), word
// 2 (i mod 2) + 1 the uniform u.  At most R = T.steps tries: after R refusals the last
// candidate is kept (the loop is bounded whatever the weights).  The test runs in FP64 for
// REF64 and FP32 for the others (L widened exactly from its stored type).
//
// Layout: CTA b takes kRejectionOffspring consecutive offspring as a pool its
// kRejectionThreads threads share: each loop iteration is eight tries of every lane's
// current offspring (their gathers in flight together), and a lane whose offspring is
// decided takes the next undecided one from a shared counter.  A warp therefore stays busy until the pool is empty instead of waiting,
// for each group of 32 offspring, for the largest of 32 geometric try counts; every
// offspring's tries and decision are those of its own Philox stream either way.
#include <math.h>

#include "pf_ancestor.cuh"
#include "pf_device.cuh"
#include "pf_internal.h"

namespace pfk {
namespace {

__device__ __forceinline__ double log_uniform(uint32_t w, double) { return log(uniform_f64(w)); }
__device__ __forceinline__ float log_uniform(uint32_t w, float) { return logf(uniform_f32(w)); }

template <int P>
__global__ void __launch_bounds__(kRejectionThreads) rejection_kernel(const AncestorLaunch G) {
    using lik_t = typename Prec<P>::lik_t;
    using acc_t = typename Prec<P>::acc_t;
    constexpr bool kF64 = sizeof(acc_t) == 8;
    __shared__ unsigned int s_next;   // next undecided offspring of the pool (local index)
    const int b = static_cast<int>(blockIdx.x);
    const int g = ancestor_tracker(G, b);
    const int slot = __ldg(G.slots + g);
    const TrackerDev &T = G.trk[slot];
    const TrackerState *st = T.state;
    const int64_t t = st->t;
    if (t <= 0 || (st->status & kStatusTimeout) || !G.frames[slot].active) return;
    const int N = static_cast<int>(T.N);
    const int64_t j0 = static_cast<int64_t>(b - __ldg(G.cta_prefix + g)) * kRejectionOffspring;
    const int pool = static_cast<int>(N - j0 < kRejectionOffspring ? N - j0 : kRejectionOffspring);
    if (threadIdx.x == 0) s_next = kRejectionThreads;
    __syncthreads();
    const lik_t *__restrict__ L = static_cast<const lik_t *>(T.pl[static_cast<int>((t + 1) & 1)]);
    const acc_t M = kF64 ? static_cast<acc_t>(st->M) : static_cast<acc_t>(st->M_f);
    const uint32_t tctr = static_cast<uint32_t>(t - 1);
    const uint32_t key_lo = T.key_lo, key_hi = T.key_hi, trk_id = T.tracker_id;
    const uint32_t n = static_cast<uint32_t>(N);
    const int R = T.steps > 0 ? T.steps : 1;   // >= 1: every offspring is decided within R tries

    int e = static_cast<int>(threadIdx.x);   // the lane's offspring (pool index); >= pool: none
    int i = 0;                               // its next try (a multiple of 8)
    while (e < pool) {
        const int jj = static_cast<int>(j0) + e;
        const uint32_t tag = 6u + (static_cast<uint32_t>(jj) << 8);
        // eight tries at a time: proposals (four Philox blocks) and gathers first, all eight
        // loads in flight, then the tests in try order; the first accepted try (or the last
        // try allowed) decides, later loads of the batch go unused
        uint32_t wk[8], wu[8];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            uint4 w = make_uint4(0u, 0u, 0u, 0u);
            if (i + 2 * h < R)
                w = philox4x32_10(make_uint4(static_cast<uint32_t>((i >> 1) + h), tctr, tag, trk_id), key_lo, key_hi);
            wk[2 * h] = w.x; wu[2 * h] = w.y; wk[2 * h + 1] = w.z; wu[2 * h + 1] = w.w;
        }
        int kq[8];
        acc_t lq[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            kq[q] = (i + q == 0) ? jj : static_cast<int>(__umulhi(wk[q], n));
            lq[q] = (i + q < R) ? to_acc(L[kq[q]]) : acc_t{};
        }
        int dec = -1;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (dec < 0 && i + q < R && (log_uniform(wu[q], acc_t{}) <= lq[q] - M || i + q + 1 >= R)) dec = q;
        if (dec >= 0) {
            int kd = kq[0];
#pragma unroll
            for (int q = 1; q < 8; ++q) if (q == dec) kd = kq[q];
            T.anc[jj] = kd;
            e = static_cast<int>(atomicAdd(&s_next, 1u));
            i = 0;
        } else {
            i += 8;
        }
    }
}

template <int P>
int launch_p(const AncestorLaunch &G, cudaStream_t s) {
    rejection_kernel<P><<<G.total_ctas, kRejectionThreads, 0, s>>>(G);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

}  // namespace

int launch_rejection(int precision, const AncestorLaunch &G, void *stream) {
    if (G.total_ctas <= 0 || G.ntrk <= 0) return 0;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (precision) {
        case 0: return launch_p<0>(G, s);
        case 1: return launch_p<1>(G, s);
        case 2: return launch_p<2>(G, s);
        case 3: return launch_p<3>(G, s);
        default: return 1;
    }
}

}  // namespace pfk
