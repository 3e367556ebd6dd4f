// fgt_eval.cu -- Taylor-series evaluation of the fast Gauss transform at
// target points (Sec. 2.2, Eq. taylor): each target takes the Taylor
// coefficients C of its own box of the uniform grid,
//   G(y) (+)= sum_{b1,b2 < p} C[box][b1][b2] t1^b1 t2^b2,  t = (y - t_C) / (sqrt(2) sigma).
// With P2H and H2T this completes the transform on the device.  Horner in
// FP32 on t formed in FP64 (|t| <= 0.36 on the workload grids).
#include "common.cuh"

namespace fmmgb {

template <int P>
__global__ void fgt_t2p_kernel(int g, double inv_scale, const float* __restrict__ C, int64_t n,
                               const double* __restrict__ y, float* __restrict__ G, int accumulate)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int side = 1 << g;
    const double px = y[2 * i] * side, py = y[2 * i + 1] * side;
    int ix = (int)floor(px), iy = (int)floor(py);
    ix = ix < 0 ? 0 : (ix > side - 1 ? side - 1 : ix);
    iy = iy < 0 ? 0 : (iy > side - 1 ? side - 1 : iy);
    const float t1 = (float)((px - (ix + 0.5)) / side * inv_scale);
    const float t2 = (float)((py - (iy + 0.5)) / side * inv_scale);
    const float4* cb = reinterpret_cast<const float4*>(C + ((size_t)iy * side + ix) * P * P);
    float outer = 0.f;
#pragma unroll 1
    for (int b1 = P - 1; b1 >= 0; --b1) {
        float row[P];
#pragma unroll
        for (int q = 0; q < P / 4; ++q) {
            const float4 v = __ldg(cb + b1 * (P / 4) + q);
            row[4 * q] = v.x;
            row[4 * q + 1] = v.y;
            row[4 * q + 2] = v.z;
            row[4 * q + 3] = v.w;
        }
        float inner = 0.f;
#pragma unroll
        for (int b2 = P - 1; b2 >= 0; --b2) inner = fmaf(inner, t2, row[b2]);
        outer = fmaf(outer, t1, inner);
    }
    G[i] = accumulate ? G[i] + outer : outer;
}

template <int P>
static int t2p_p(int g, double sigma, const float* C, int64_t n, const double* y, float* G, bool acc, cudaStream_t st)
{
    fgt_t2p_kernel<P><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, 1.0 / (sqrt(2.0) * sigma), C, n, y, G,
                                                                   acc ? 1 : 0);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

// T2P at targets binned by box (fgt_bin_points): one block per box holds the
// box's p x p Taylor coefficients in shared memory (every lane reads the same
// entry: a broadcast) and evaluates them at each of the box's targets, whose
// offsets from the box centre are read off the bits of their FP64 coordinates.
// The per-target kernel above reads a random box's 1 KB of coefficients per
// target from L1/L2.
constexpr int kT2pThreads = 128;

template <int P>
__global__ void __launch_bounds__(kT2pThreads) fgt_t2p_binned_kernel(int g, double inv_scale, float dcell,
                                                                     const float* __restrict__ C, int n,
                                                                     const double* __restrict__ y,
                                                                     const int* __restrict__ perm,
                                                                     const int* __restrict__ box_start,
                                                                     float* __restrict__ G, int accumulate, int* err)
{
    __shared__ float s_c[P * P];
    const int side = 1 << g;
    const int b = blockIdx.x, tid = threadIdx.x;
    const int bx = b & (side - 1), by = b >> g;
    const int first = box_start[b], end = box_start[b + 1];
    if (first < 0 || end > n || first > end) {
        if (tid == 0) atomicOr(err, DEV_ERR_CHECK);
        return;
    }
    if (first == end) return;
    for (int k = tid; k < P * P; k += kT2pThreads) s_c[k] = C[(size_t)b * P * P + k];
    __syncthreads();
    for (int q = first + tid; q < end; q += kT2pThreads) {
        const int j = perm[q];
        if ((unsigned)j >= (unsigned)n) {
            atomicOr(err, DEV_ERR_CHECK);
            continue;
        }
        const double y0 = y[2 * (size_t)j], y1 = y[2 * (size_t)j + 1];
        long long X0, X1;
        float t1, t2;
        if (grid_fixed31(y0, g, X0) && grid_fixed31(y1, g, X1) && (int)(X0 >> 31) == bx && (int)(X1 >> 31) == by) {
            t1 = cell_offset31(X0) * dcell;
            t2 = cell_offset31(X1) * dcell;
        } else {  // outside the unit square (the nearest box): offset in FP64
            t1 = (float)((y0 * side - (bx + 0.5)) / side * inv_scale);
            t2 = (float)((y1 * side - (by + 0.5)) / side * inv_scale);
        }
        float outer = 0.f;
#pragma unroll 4
        for (int b1 = P - 1; b1 >= 0; --b1) {
            float inner = 0.f;
#pragma unroll
            for (int b2 = P - 1; b2 >= 0; --b2) inner = fmaf(inner, t2, s_c[b1 * P + b2]);
            outer = fmaf(outer, t1, inner);
        }
        G[j] = accumulate ? G[j] + outer : outer;
    }
}

template <int P>
static int t2p_binned_p(int g, double sigma, const float* C, int n, const double* y, const int* perm,
                        const int* box_start, float* G, bool acc, int* err, cudaStream_t st)
{
    const double inv_scale = 1.0 / (sqrt(2.0) * sigma);
    fgt_t2p_binned_kernel<P><<<1u << (2 * g), kT2pThreads, 0, st>>>(
        g, inv_scale, (float)(ldexp(1.0, -g) * inv_scale), C, n, y, perm, box_start, G, acc ? 1 : 0, err);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

}  // namespace fmmgb

using namespace fmmgb;

extern "C" int fgt_t2p_binned(int32_t grid_log2, int32_t p, double sigma, const float* C, const double* y, int64_t n,
                              const int32_t* perm, const int32_t* box_start, float* G, int32_t flags, void* stream)
{
    clear_error();
    if (grid_log2 < 0 || grid_log2 > 10)
        return fail(FMM_EINVAL, "fgt_t2p_binned: grid_log2 %d outside 0..10", grid_log2);
    if (!fgt_supported(p)) return fail(FMM_EINVAL, "fgt_t2p_binned: unsupported p = %d (4, 8, 12, 16)", p);
    if (!(sigma > 0.0) || !(sigma < 1e300)) return fail(FMM_EINVAL, "fgt_t2p_binned: sigma must be positive and finite");
    if (n < 0 || n > INT32_MAX) return fail(FMM_EINVAL, "fgt_t2p_binned: n = %lld outside 0..2^31-1", (long long)n);
    if (!C || !box_start || (n > 0 && (!y || !G || !perm))) return fail(FMM_EINVAL, "fgt_t2p_binned: NULL pointer");
    if (((uintptr_t)C & 3) || ((uintptr_t)y & 7) || ((uintptr_t)G & 3) || ((uintptr_t)perm & 3) ||
        ((uintptr_t)box_start & 3))
        return fail(FMM_EINVAL, "fgt_t2p_binned: misaligned pointer");
    if (flags & ~FMM_ACCUMULATE) return fail(FMM_EINVAL, "fgt_t2p_binned: unknown flags 0x%x", flags);
    if (n == 0) return FMM_OK;
    int* err = nullptr;
    if (int rc = device_error_word(&err)) return rc;
    const bool acc = (flags & FMM_ACCUMULATE) != 0;
    cudaStream_t st = (cudaStream_t)stream;
    const int nn = (int)n;
    switch (p) {
        case 4: return t2p_binned_p<4>(grid_log2, sigma, C, nn, y, perm, box_start, G, acc, err, st);
        case 8: return t2p_binned_p<8>(grid_log2, sigma, C, nn, y, perm, box_start, G, acc, err, st);
        case 12: return t2p_binned_p<12>(grid_log2, sigma, C, nn, y, perm, box_start, G, acc, err, st);
        default: return t2p_binned_p<16>(grid_log2, sigma, C, nn, y, perm, box_start, G, acc, err, st);
    }
}

extern "C" int fgt_t2p(int32_t grid_log2, int32_t p, double sigma, const float* C, const double* y, int64_t n,
                       float* G, int32_t flags, void* stream)
{
    clear_error();
    if (grid_log2 < 0 || grid_log2 > 12) return fail(FMM_EINVAL, "fgt_t2p: grid_log2 %d outside 0..12", grid_log2);
    if (!fgt_supported(p)) return fail(FMM_EINVAL, "fgt_t2p: unsupported p = %d (4, 8, 12, 16)", p);
    if (!(sigma > 0.0) || !(sigma < 1e300)) return fail(FMM_EINVAL, "fgt_t2p: sigma must be positive and finite");
    if (n < 0) return fail(FMM_EINVAL, "fgt_t2p: n < 0");
    if (!C || (n > 0 && (!y || !G))) return fail(FMM_EINVAL, "fgt_t2p: NULL pointer");
    if (((uintptr_t)C & 15) || ((uintptr_t)y & 7) || ((uintptr_t)G & 3))
        return fail(FMM_EINVAL, "fgt_t2p: misaligned pointer (C 16 bytes, y 8, G 4)");
    if (flags & ~FMM_ACCUMULATE) return fail(FMM_EINVAL, "fgt_t2p: unknown flags 0x%x", flags);
    if (n == 0) return FMM_OK;
    const bool acc = (flags & FMM_ACCUMULATE) != 0;
    cudaStream_t st = (cudaStream_t)stream;
    switch (p) {
        case 4: return t2p_p<4>(grid_log2, sigma, C, n, y, G, acc, st);
        case 8: return t2p_p<8>(grid_log2, sigma, C, n, y, G, acc, st);
        case 12: return t2p_p<12>(grid_log2, sigma, C, n, y, G, acc, st);
        default: return t2p_p<16>(grid_log2, sigma, C, n, y, G, acc, st);
    }
}
