// pf_gumbel.cu -- Gumbel-max resampling (sm_103a, CUDA cores only).
//
// Multinomial resampling in the log domain, the alternative to log-sum-exp that Sec. IV
// ("Numerical Stability Optimization") weighs: with g_jk = -ln(-ln u_jk) independent
// standard Gumbel variates, argmax_k (L_k + g_jk) follows the categorical law
// exp(L_k) / sum_i exp(L_i), so offspring j needs no maximum, no sum and no CDF of the
// weights -- only N draws of its own, hence N^2 draws a frame (trackers of at most
// kGumbelMaxN particles).
//
// u_jk is the uniform of word (k mod 4) of Philox(k / 4, t - 1, 4 + 256 j, tracker), and
// the sum is taken in the filter's weight precision: FP64 for REF64, FP32 for the others
// (L widened from its stored type).  Ties go to the smallest k.
//
// Layout: CTA b takes kGumbelOffspring consecutive offspring of one tracker.  Its threads
// stride over the particle quads q (particles 4q .. 4q+3): one Philox block per (quad,
// offspring) gives that offspring's four draws, the quad's four L are loaded once for all
// of the CTA's offspring, and each thread keeps a running best per offspring (k rises
// within a thread, so a strict comparison keeps the smallest k of equal values).  The CTA
// then reduces each offspring's (value, index) pairs: warp shuffles, then one thread per
// offspring over the warps' results.  The pull kernel gathers the ancestors written here.
#include <math.h>

#include "pf_ancestor.cuh"
#include "pf_device.cuh"
#include "pf_internal.h"

namespace pfk {
namespace {

__device__ __forceinline__ double gumbel_of(uint32_t w, double) { return -log(-log(uniform_f64(w))); }
__device__ __forceinline__ float gumbel_of(uint32_t w, float) { return -logf(-logf(uniform_f32(w))); }

// (v, k) <- (v2, k2) when v2 is larger, or equal with the smaller index
template <typename A>
__device__ __forceinline__ void take_best(A &v, int &k, A v2, int k2) {
    if (v2 > v || (v2 == v && k2 < k)) {
        v = v2;
        k = k2;
    }
}

template <int P>
__global__ void __launch_bounds__(kGumbelThreads) gumbel_kernel(const AncestorLaunch G) {
    using lik_t = typename Prec<P>::lik_t;
    using acc_t = typename Prec<P>::acc_t;
    constexpr int kJ = kGumbelOffspring;
    constexpr int kWarps = kGumbelThreads / 32;
    __shared__ acc_t s_v[kWarps][kJ];
    __shared__ int s_k[kWarps][kJ];

    const int b = static_cast<int>(blockIdx.x);
    const int g = ancestor_tracker(G, b);
    const int slot = __ldg(G.slots + g);
    const TrackerDev &T = G.trk[slot];
    const TrackerState *st = T.state;
    const int64_t t = st->t;
    if (t <= 0 || (st->status & kStatusTimeout) || !G.frames[slot].active) return;
    const int N = static_cast<int>(T.N);
    const int j0 = (b - __ldg(G.cta_prefix + g)) * kJ;
    const lik_t *__restrict__ L = static_cast<const lik_t *>(T.pl[static_cast<int>((t + 1) & 1)]);
    const uint32_t tctr = static_cast<uint32_t>(t - 1);
    const uint32_t key_lo = T.key_lo, key_hi = T.key_hi, trk_id = T.tracker_id;

    acc_t best[kJ];
    int arg[kJ];
#pragma unroll
    for (int jj = 0; jj < kJ; ++jj) {
        best[jj] = -INFINITY;
        arg[jj] = N;
    }
    const int nq = (N + 3) >> 2;
    for (int q = threadIdx.x; q < nq; q += kGumbelThreads) {
        const int k = 4 * q;
        acc_t l[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) l[i] = (k + i < N) ? to_acc(L[k + i]) : static_cast<acc_t>(-INFINITY);
#pragma unroll
        for (int jj = 0; jj < kJ; ++jj) {
            const int j = j0 + jj;
            if (j >= N) break;
            const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(q), tctr, 4u + (static_cast<uint32_t>(j) << 8),
                                                     trk_id),
                                          key_lo, key_hi);
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (k + i < N) {
                    const acc_t v = l[i] + gumbel_of(ws[i], acc_t{});
                    if (v > best[jj]) {
                        best[jj] = v;
                        arg[jj] = k + i;
                    }
                }
            }
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int jj = 0; jj < kJ; ++jj) {
        acc_t v = best[jj];
        int k = arg[jj];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const acc_t v2 = __shfl_xor_sync(0xffffffffu, v, o);
            const int k2 = __shfl_xor_sync(0xffffffffu, k, o);
            take_best(v, k, v2, k2);
        }
        if (lane == 0) {
            s_v[wid][jj] = v;
            s_k[wid][jj] = k;
        }
    }
    __syncthreads();
    if (threadIdx.x < kJ) {
        const int jj = threadIdx.x, j = j0 + jj;
        acc_t v = s_v[0][jj];
        int k = s_k[0][jj];
#pragma unroll
        for (int w = 1; w < kWarps; ++w) take_best(v, k, s_v[w][jj], s_k[w][jj]);
        // k = N only if no value compared larger than -inf (a NaN likelihood)
        if (j < N) T.anc[j] = k < N ? k : N - 1;
    }
}

template <int P>
int launch_p(const AncestorLaunch &G, cudaStream_t s) {
    gumbel_kernel<P><<<G.total_ctas, kGumbelThreads, 0, s>>>(G);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

}  // namespace

int launch_gumbel(int precision, const AncestorLaunch &G, void *stream) {
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
