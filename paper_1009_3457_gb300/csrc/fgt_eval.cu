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

}  // namespace fmmgb

using namespace fmmgb;

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
