// upward.cu -- device construction of M2L inputs (upward sweep, Sec. 2.1
// stage 2): P2M of particles into the boxes of one level and M2M from a level
// to its parents (and M2M's conjugate transpose, for gradients), in
// radius-scaled units.  Support for the translation path, not part of it;
// kept simple (atomic accumulation in P2M).
#include "common.cuh"

namespace fmmgb {

// M~_b[k] += c_i w^k,  w = (y_i - x_b) / r_l  (|w| <= 1/sqrt 2): w read off the bits of
// the FP64 coordinates (points outside the unit square: the clamped box, in FP64), the
// powers in FP32, added by FP32 atomics.
__global__ void p2m_kernel(int level, int p, const double* __restrict__ xy, const double* __restrict__ c, int64_t n,
                           float2* __restrict__ M)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int side = 1 << level;
    const double x = xy[2 * i], y = xy[2 * i + 1];
    int ix, iy;
    float wr, wi;
    long long X, Y;
    if (grid_fixed31(x, level, X) && grid_fixed31(y, level, Y)) {
        ix = (int)(X >> 31);
        iy = (int)(Y >> 31);
        wr = cell_offset31(X);
        wi = cell_offset31(Y);
    } else {
        const double xs = x * side, ys = y * side;
        ix = (int)floor(xs);
        iy = (int)floor(ys);
        ix = ix < 0 ? 0 : (ix > side - 1 ? side - 1 : ix);
        iy = iy < 0 ? 0 : (iy > side - 1 ? side - 1 : iy);
        wr = (float)(xs - (ix + 0.5));
        wi = (float)(ys - (iy + 0.5));
    }
    float pr = (float)c[i], pi = 0.f;
    float2* mb = M + ((size_t)iy * side + ix) * p;
    for (int k = 0; k < p; ++k) {
        atomicAdd(&mb[k].x, pr);
        atomicAdd(&mb[k].y, pi);
        const float t = fmaf(pr, wr, -pi * wi);
        pi = fmaf(pr, wi, pi * wr);
        pr = t;
    }
}

// P2M from points binned by box (fmm_bin_points at `level`): one warp per box
// (four boxes per CTA) sums its points' c d^k (d read off the bits of the FP64
// coordinates, powers in FP32: |d| <= 1/sqrt(2)), each lane over a strided
// share of the box's points; the lanes' partial sums meet through a transpose in
// shared memory (lane t < 2p adds up real t of the 32 lanes' partials), so a
// box costs 2p + 32 shared-memory accesses per lane instead of a shuffle tree
// per coefficient.  One store per real, no atomics, a fixed summation order.
constexpr int kP2mThreads = 128;
constexpr int kP2mBoxes = kP2mThreads / 32;

template <int P>
__global__ void __launch_bounds__(kP2mThreads) p2m_binned_kernel(int level, const double* __restrict__ xy,
                                                                 const double* __restrict__ c, int n,
                                                                 const int* __restrict__ perm,
                                                                 const int* __restrict__ box_start,
                                                                 float2* __restrict__ M, int accumulate, int* err)
{
    constexpr int R = 2 * P + 1;  // padded row of one lane's reals: conflict-free column reads
    __shared__ float s_red[kP2mBoxes][32 * R];
    const int side = 1 << level, nbox = side * side;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = blockIdx.x * kP2mBoxes + warp;
    if (b >= nbox) return;  // whole warps only: no block barrier below
    const int bx = b & (side - 1), by = b >> level;
    int first = box_start[b], end = box_start[b + 1];
    if (first < 0 || end > n || first > end) {
        if (lane == 0) atomicOr(err, DEV_ERR_CHECK);
        first = end = 0;
    }
    float2 acc[P];
#pragma unroll
    for (int k = 0; k < P; ++k) acc[k] = make_float2(0.f, 0.f);
    for (int q = first + lane; q < end; q += 32) {
        const int i = perm[q];
        if ((unsigned)i >= (unsigned)n) {
            atomicOr(err, DEV_ERR_CHECK);
            continue;
        }
        const double x = xy[2 * (size_t)i], y = xy[2 * (size_t)i + 1];
        long long X, Y;
        float wr, wi;  // offset from the box centre in box sides
        if (grid_fixed31(x, level, X) && grid_fixed31(y, level, Y) && (int)(X >> 31) == bx && (int)(Y >> 31) == by) {
            wr = cell_offset31(X);  // no FP64 arithmetic for a point inside its box
            wi = cell_offset31(Y);
        } else {
            wr = (float)(x * side - (bx + 0.5));
            wi = (float)(y * side - (by + 0.5));
        }
        float pr = (float)c[i], pi = 0.f;
#pragma unroll
        for (int k = 0; k < P; ++k) {
            acc[k].x += pr;
            acc[k].y += pi;
            const float t = fmaf(pr, wr, -pi * wi);
            pi = fmaf(pr, wi, pi * wr);
            pr = t;
        }
    }
    float* red = s_red[warp];
#pragma unroll
    for (int k = 0; k < P; ++k) {
        red[lane * R + 2 * k] = acc[k].x;
        red[lane * R + 2 * k + 1] = acc[k].y;
    }
    __syncwarp();
    for (int t = lane; t < 2 * P; t += 32) {
        float v = 0.f;
#pragma unroll 8
        for (int l = 0; l < 32; ++l) v += red[l * R + t];
        float* dst = reinterpret_cast<float*>(M + (size_t)b * P) + t;
        if (accumulate) v += *dst;
        *dst = v;
    }
}

int launch_p2m_binned(int level, int p, const double* xy, const double* c, int n, const int* perm,
                      const int* box_start, float2* M, bool acc, int* err, cudaStream_t st)
{
    const unsigned nbox = 1u << (2 * level), grid = (nbox + kP2mBoxes - 1) / kP2mBoxes;
    switch (p) {
        case 6: p2m_binned_kernel<6><<<grid, kP2mThreads, 0, st>>>(level, xy, c, n, perm, box_start, M, acc, err); break;
        case 8: p2m_binned_kernel<8><<<grid, kP2mThreads, 0, st>>>(level, xy, c, n, perm, box_start, M, acc, err); break;
        case 12: p2m_binned_kernel<12><<<grid, kP2mThreads, 0, st>>>(level, xy, c, n, perm, box_start, M, acc, err); break;
        case 16: p2m_binned_kernel<16><<<grid, kP2mThreads, 0, st>>>(level, xy, c, n, perm, box_start, M, acc, err); break;
        case 24: p2m_binned_kernel<24><<<grid, kP2mThreads, 0, st>>>(level, xy, c, n, perm, box_start, M, acc, err); break;
        default: return fail(FMM_EINVAL, "fmm_p2m_binned: unsupported p = %d (6, 8, 12, 16, 24)", p);
    }
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

// Scaled M2M: parent box side R = 2r, child offset z = (x_c - x_P)/R = (+-1/4, +-1/4):
//   M~P_j = sum_{k<=j} C(j,k) z^(j-k) 2^-k M~c_k, summed over the 4 children.
// The entries (binomials, powers of (+-1 +- i)/4, powers of 2) are exact in FP32;
// the binomials come from the compile-time table.
__global__ void m2m_kernel(int child_level, int p, const float2* __restrict__ Mc, float2* __restrict__ Mp,
                           int accumulate)
{
    const int np = 1 << (child_level - 1);
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)np * np * p) return;
    const int j = (int)(idx % p);
    const int64_t pb = idx / p;
    const int px = (int)(pb % np), py = (int)(pb / np);
    const int nc = 2 * np;
    float sr = 0.f, si = 0.f;
    for (int cyy = 0; cyy < 2; ++cyy)
        for (int cxx = 0; cxx < 2; ++cxx) {
            const float zr = cxx ? 0.25f : -0.25f, zi = cyy ? 0.25f : -0.25f;
            const float2* mc = Mc + ((size_t)(2 * py + cyy) * nc + (2 * px + cxx)) * p;
            // k from j down to 0: term C(j,k) z^(j-k) 2^-k m_k
            const float* brow = kBinom.v + j * 64;
            float zpr = 1.f, zpi = 0.f;  // z^(j-k)
            for (int k = j; k >= 0; --k) {
                const float sc = brow[k] * pow2_neg(k);
                const float2 m = mc[k];
                sr = fmaf(sc, zpr * m.x - zpi * m.y, sr);
                si = fmaf(sc, zpr * m.y + zpi * m.x, si);
                const float nr = zpr * zr - zpi * zi;
                zpi = zpr * zi + zpi * zr;
                zpr = nr;
            }
        }
    float2* out = Mp + (size_t)pb * p + j;
    float2 o = make_float2(sr, si);
    if (accumulate) {
        o.x += out->x;
        o.y += out->y;
    }
    *out = o;
}

// Conjugate transpose of M2M: one thread per (child box, k):
//   Wc[child][k] (+)= sum_{j>=k} conj(C(j,k) z^(j-k) 2^-k) WP[parent][j]
// (binomials from the compile-time table).
__global__ void m2m_adjoint_kernel(int child_level, int p, const float2* __restrict__ Wp, float2* __restrict__ Wc,
                                   int accumulate)
{
    const int side = 1 << child_level, np = side >> 1;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)side * side * p) return;
    const int k = (int)(idx % p);
    const int64_t b = idx / p;
    const int ix = (int)(b % side), iy = (int)(b / side);
    const float zr = (ix & 1) ? 0.25f : -0.25f, zi = (iy & 1) ? 0.25f : -0.25f;
    const float2* wp = Wp + ((size_t)(iy >> 1) * np + (ix >> 1)) * p;
    float sr = 0.f, si = 0.f, pr = 1.f, pim = 0.f;  // z^(j-k)
    for (int j = k; j < p; ++j) {
        const float2 w = wp[j];
        const float binom = kBinom.v[j * 64 + k];  // C(j, k)
        // conj(z^(j-k)) w
        sr = fmaf(binom, pr * w.x + pim * w.y, sr);
        si = fmaf(binom, pr * w.y - pim * w.x, si);
        const float nr = pr * zr - pim * zi;
        pim = pr * zi + pim * zr;
        pr = nr;
    }
    const float sc = pow2_neg(k);
    float2* out = Wc + (size_t)b * p + k;
    float2 o = make_float2(sc * sr, sc * si);
    if (accumulate) {
        o.x += out->x;
        o.y += out->y;
    }
    *out = o;
}

// FGT Hermite coefficients of every box of a 2^g grid (Eq. A_alpha):
//   A_b[a1][a2] += q_j t1^a1 t2^a2 / (a1! a2!),  t = (x_j - s_b) / (sqrt(2) sigma)
__global__ void fgt_p2h_kernel(int g, int p, double inv_scale, const double* __restrict__ x,
                               const double* __restrict__ q, int64_t n, float* __restrict__ A)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int side = 1 << g;
    const double px = x[2 * j] * side, py = x[2 * j + 1] * side;
    int ix = (int)floor(px), iy = (int)floor(py);
    ix = ix < 0 ? 0 : (ix > side - 1 ? side - 1 : ix);
    iy = iy < 0 ? 0 : (iy > side - 1 ? side - 1 : iy);
    const double t1 = (px - (ix + 0.5)) / side * inv_scale, t2 = (py - (iy + 0.5)) / side * inv_scale;
    float* Ab = A + ((size_t)iy * side + ix) * p * p;
    double w1 = q[j];
    for (int a1 = 0; a1 < p; ++a1) {
        double w2 = w1;
        for (int a2 = 0; a2 < p; ++a2) {
            atomicAdd(&Ab[a1 * p + a2], (float)w2);
            w2 = w2 * t2 / (double)(a2 + 1);
        }
        w1 = w1 * t1 / (double)(a1 + 1);
    }
}

int launch_fgt_p2h(int g, int p, double sigma, const double* x, const double* q, int64_t n, float* A, bool acc,
                   cudaStream_t st)
{
    const size_t bytes = ((size_t)1 << (2 * g)) * (size_t)p * p * sizeof(float);
    if (!acc) FMM_CUDA_TRY(cudaMemsetAsync(A, 0, bytes, st));
    if (n == 0) return FMM_OK;
    fgt_p2h_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, p, 1.0 / (sqrt(2.0) * sigma), x, q, n, A);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

int launch_p2m(int level, int p, const double* xy, const double* c, int64_t n, float2* M, bool acc, cudaStream_t st)
{
    const size_t bytes = ((size_t)1 << (2 * level)) * (size_t)p * sizeof(float2);
    if (!acc) FMM_CUDA_TRY(cudaMemsetAsync(M, 0, bytes, st));
    if (n == 0) return FMM_OK;
    const int64_t blocks = (n + 255) / 256;
    p2m_kernel<<<(unsigned)blocks, 256, 0, st>>>(level, p, xy, c, n, M);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

int launch_m2m_adjoint(int child_level, int p, const float2* Wp, float2* Wc, bool acc, cudaStream_t st)
{
    const int64_t side = (int64_t)1 << child_level;
    const int64_t total = side * side * p;
    m2m_adjoint_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(child_level, p, Wp, Wc, acc ? 1 : 0);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

int launch_m2m(int child_level, int p, const float2* Mc, float2* Mp, bool acc, cudaStream_t st)
{
    const int64_t np = (int64_t)1 << (child_level - 1);
    const int64_t total = np * np * p;
    m2m_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(child_level, p, Mc, Mp, acc ? 1 : 0);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

}  // namespace fmmgb
