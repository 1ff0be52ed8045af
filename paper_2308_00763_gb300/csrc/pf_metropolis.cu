// pf_metropolis.cu -- Metropolis resampling (sm_103a, CUDA cores only).
//
// Sec. III cites Metropolis resampling (Murray, Lee and Jacob, 2016) as a scheme that avoids
// the global reduction of multinomial, stratified and systematic resampling.  Offspring j
// runs a Metropolis chain of B steps over the particle indices with target exp(L_k),
// started at k = j: step b proposes k' uniform on {0, ..., N-1} and moves there when
// ln u <= L_k' - L_k.  Neither the maximum of L, nor the sum of the weights, nor a CDF is
// read; the chain's limit is the categorical law exp(L_k) / sum exp(L), and for small B the
// draw is biased towards the start.
//
// Draws: step b of offspring j reads Philox(b / 2, t - 1, 5 + 256 j, tracker); word
// 2 (b mod 2) gives k' = floor(w N / 2^32) (an integer multiply-high, so every precision
// proposes the same k'), word 2 (b mod 2) + 1 the uniform u.  The test is evaluated in the
// weight precision: FP64 for REF64, FP32 for the others (L widened exactly from its stored
// type).
//
// Layout: one thread per offspring, 256 offspring per CTA.  The proposals do not depend on
// the chain's state, so the random gathers L[k'] of successive steps are independent loads:
// a thread issues eight steps' gathers together, then takes their accept tests in order
// (L of a tracker is 2-8 bytes per particle and stays in L2 here); the state's own L_k is
// kept in a register.  The pull kernel gathers the ancestors written here.
#include <math.h>

#include "pf_ancestor.cuh"
#include "pf_device.cuh"
#include "pf_internal.h"

namespace pfk {
namespace {

__device__ __forceinline__ double log_uniform(uint32_t w, double) { return log(uniform_f64(w)); }
__device__ __forceinline__ float log_uniform(uint32_t w, float) { return logf(uniform_f32(w)); }

template <int P>
__global__ void __launch_bounds__(kMetropolisThreads) metropolis_kernel(const AncestorLaunch G) {
    using lik_t = typename Prec<P>::lik_t;
    using acc_t = typename Prec<P>::acc_t;
    const int b = static_cast<int>(blockIdx.x);
    const int g = ancestor_tracker(G, b);
    const int slot = __ldg(G.slots + g);
    const TrackerDev &T = G.trk[slot];
    const TrackerState *st = T.state;
    const int64_t t = st->t;
    if (t <= 0 || (st->status & kStatusTimeout) || !G.frames[slot].active) return;
    const int N = static_cast<int>(T.N);
    const int j = (b - __ldg(G.cta_prefix + g)) * kMetropolisThreads + static_cast<int>(threadIdx.x);
    if (j >= N) return;
    const lik_t *__restrict__ L = static_cast<const lik_t *>(T.pl[static_cast<int>((t + 1) & 1)]);
    const uint32_t tctr = static_cast<uint32_t>(t - 1);
    const uint32_t tag = 5u + (static_cast<uint32_t>(j) << 8);
    const uint32_t key_lo = T.key_lo, key_hi = T.key_hi, trk_id = T.tracker_id;
    const uint32_t n = static_cast<uint32_t>(N);
    const int B = T.steps;

    int k = j;
    acc_t lk = to_acc(L[j]);
    // eight steps at a time: their proposals (four Philox blocks) and gathers first, all
    // eight loads in flight, then the eight accept tests in step order
    for (int s = 0; s < B; s += 8) {
        uint32_t wk[8], wu[8];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            uint4 w = make_uint4(0u, 0u, 0u, 0u);
            if (s + 2 * h < B)
                w = philox4x32_10(make_uint4(static_cast<uint32_t>((s >> 1) + h), tctr, tag, trk_id), key_lo, key_hi);
            wk[2 * h] = w.x; wu[2 * h] = w.y; wk[2 * h + 1] = w.z; wu[2 * h + 1] = w.w;
        }
        int kq[8];
        acc_t lq[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            kq[q] = static_cast<int>(__umulhi(wk[q], n));
            lq[q] = (s + q < B) ? to_acc(L[kq[q]]) : acc_t{};
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (s + q < B && log_uniform(wu[q], acc_t{}) <= lq[q] - lk) {
                k = kq[q];
                lk = lq[q];
            }
        }
    }
    T.anc[j] = k;
}

template <int P>
int launch_p(const AncestorLaunch &G, cudaStream_t s) {
    metropolis_kernel<P><<<G.total_ctas, kMetropolisThreads, 0, s>>>(G);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

}  // namespace

int launch_metropolis(int precision, const AncestorLaunch &G, void *stream) {
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
