// fgt_hermite.cuh -- device pieces shared by the FP32 and tensor-core forms of
// the FGT Hermite evaluation (Sec. 4.2, Eq. hermite).
#pragma once

#include "common.cuh"

namespace fmmgb {

// h_n(t) = exp(-t^2) H_n(t), n < P, by the three-term recurrence
// h_{n+1} = 2t h_n - 2n h_{n-1} (h_0 = exp(-t^2), h_1 = 2t exp(-t^2)).
template <int P>
__device__ __forceinline__ void hermite_functions(float t, float (&h)[P])
{
    const float tt = t + t;
    h[0] = __expf(-t * t);
    if (P > 1) h[1] = tt * h[0];
#pragma unroll
    for (int m = 1; m + 1 < P; ++m) h[m + 1] = fmaf(tt, h[m], -(float)(2 * m) * h[m - 1]);
}

// The run of binned targets that claim k covers: claims[b] is the exclusive
// prefix over boxes of ceil(targets of b / ch) (launch_h2p_claims), so claim k
// belongs to the box b with claims[b] <= k < claims[b+1] and covers
// [box_start[b] + (k - claims[b]) ch, ... + ch) clipped to the box.  An
// inconsistent box_start gives first >= end.
__device__ __forceinline__ void h2p_claim_range(const int* __restrict__ claims, const int* __restrict__ box_start,
                                                int nbox, int n, int ch, int k, int* first, int* end, int* box)
{
    int lo = 0, hi = nbox;  // largest b with claims[b] <= k
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(claims + mid) <= k) lo = mid;
        else hi = mid;
    }
    const int f = __ldg(box_start + lo) + (k - __ldg(claims + lo)) * ch;
    const int e = min(min(f + ch, __ldg(box_start + lo + 1)), n);
    const bool ok = 0 <= f && f < e;
    *first = ok ? f : 0;
    *end = ok ? e : 0;
    *box = lo;
}

// The same with the claim table over the boxes in `order` (position i holds box order[i]).
__device__ __forceinline__ void h2p_claim_range_ordered(const int* __restrict__ claims, const int* __restrict__ order,
                                                        const int* __restrict__ box_start, int nbox, int n, int ch,
                                                        int k, int* first, int* end, int* box)
{
    int lo = 0, hi = nbox;  // largest position i with claims[i] <= k
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(claims + mid) <= k) lo = mid;
        else hi = mid;
    }
    const int b = __ldg(order + lo);
    const bool inb = (unsigned)b < (unsigned)nbox;
    const int f = inb ? __ldg(box_start + b) + (k - __ldg(claims + lo)) * ch : 0;
    const int e = inb ? min(min(f + ch, __ldg(box_start + b + 1)), n) : 0;
    const bool ok = inb && 0 <= f && f < e;
    *first = ok ? f : 0;
    *end = ok ? e : 0;
    *box = ok ? b : 0;
}

// Host: claims[0..nbox] for runs of ch targets (one CTA, on `st`).
int launch_h2p_claims(int nbox, const int* box_start, int ch, int* claims, int* err, cudaStream_t st);

// Host: the tensor-core evaluation (p = 16); claims must have been built with ch = 128.
int launch_fgt_h2p_tc(int g, int ncut, double d, bool split, const float* A, const double* y, int n, const int* perm,
                      const int* box_start, const int* claims, float* G, bool accumulate, int* err, cudaStream_t st);

}  // namespace fmmgb
