// pf_ancestor.cuh -- shared piece of the ancestor kernels (Gumbel-max, Metropolis).
#pragma once
#include "pf_internal.h"

namespace pfk {

// The tracker g of CTA b: cta_prefix[g] <= b < cta_prefix[g + 1] (bisection; every tracker
// has at least one CTA, so the prefix is strictly increasing).
__device__ __forceinline__ int ancestor_tracker(const AncestorLaunch &G, int b) {
    int lo = 0, hi = G.ntrk - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(G.cta_prefix + mid) <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace pfk
