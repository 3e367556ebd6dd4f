// farfield.cu -- the far-field stages around the M2L path on the device, in
// radius-scaled units (Sec. 2.1 stages 3-4), with the adjoints that carry a
// gradient back through them:
//   L2L   L~c[j] = sum_{n>=j} C(n,j) u^(n-j) 2^-(j+1) L~p[n],  u = (x_c - x_P) / r_P = (+-1/4, +-1/4)
//   L2P   phi(z) = (1/r) sum_n L~[leaf][n] w^n,  w = (z - x_leaf) / r
//   P2M^T grad of sum_k <G_k, M~_k(y)> in the point positions, M~_k = sum_i c_i d_i^k, d = (y - x_b)/r
// The L2L entries (binomials, powers of (+-1 +- i)/4, powers of 2) are exact
// in FP32; L2P forms w in FP64 and evaluates in FP32.  Adjoints are conjugate transposes (the
// gradient of a real objective in PyTorch's convention for complex tensors).
#include "common.cuh"

namespace fmmgb {

// One thread per (child box, j): Lc[child][j] (+)= sum_n T_c[j][n] Lp[parent][n]; the
// binomials from the compile-time table.
__global__ void l2l_kernel(int child_level, int p, const float2* __restrict__ Lp, float2* __restrict__ Lc,
                           int accumulate)
{
    const int side = 1 << child_level, ps = side >> 1;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)side * side * p) return;
    const int j = (int)(idx % p);
    const int64_t b = idx / p;
    const int ix = (int)(b % side), iy = (int)(b / side);
    const float ur = (ix & 1) ? 0.25f : -0.25f, ui = (iy & 1) ? 0.25f : -0.25f;
    const float2* lp = Lp + ((size_t)(iy >> 1) * ps + (ix >> 1)) * p;
    // n from j upward: C(n, j) u^(n-j)
    float sr = 0.f, si = 0.f, pr = 1.f, pim = 0.f;
    for (int n = j; n < p; ++n) {
        const float2 v = lp[n];
        const float binom = kBinom.v[n * 64 + j];
        const float tr = pr * v.x - pim * v.y, ti = pr * v.y + pim * v.x;
        sr = fmaf(binom, tr, sr);
        si = fmaf(binom, ti, si);
        const float nr = pr * ur - pim * ui;
        pim = pr * ui + pim * ur;
        pr = nr;
    }
    const float sc = pow2_neg(j + 1);
    float2* out = Lc + (size_t)b * p + j;
    float2 o = make_float2(sc * sr, sc * si);
    if (accumulate) {
        o.x += out->x;
        o.y += out->y;
    }
    *out = o;
}

// Conjugate transpose: one thread per (parent box, n):
//   Wp[parent][n] (+)= sum_{children c} sum_{j<=n} conj(T_c[j][n]) Wc[child][j].
__global__ void l2l_adjoint_kernel(int child_level, int p, const float2* __restrict__ Wc, float2* __restrict__ Wp,
                                   int accumulate)
{
    const int side = 1 << child_level, ps = side >> 1;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)ps * ps * p) return;
    const int n = (int)(idx % p);
    const int64_t pb = idx / p;
    const int px = (int)(pb % ps), py = (int)(pb / ps);
    float sr = 0.f, si = 0.f;
    for (int cy = 0; cy < 2; ++cy)
        for (int cx = 0; cx < 2; ++cx) {
            const float ur = cx ? 0.25f : -0.25f, ui = cy ? 0.25f : -0.25f;
            const float2* wc = Wc + ((size_t)(2 * py + cy) * side + (2 * px + cx)) * p;
            // j from n down to 0: entry C(n, j) u^(n-j) 2^-(j+1), conjugated
            const float* brow = kBinom.v + n * 64;
            float pr = 1.f, pim = 0.f;  // u^(n-j)
            for (int j = n; j >= 0; --j) {
                const float sc = brow[j] * pow2_neg(j + 1);
                const float2 w = wc[j];
                // conj(u^(n-j)) * w
                const float tr = pr * w.x + pim * w.y, ti = pr * w.y - pim * w.x;
                sr = fmaf(sc, tr, sr);
                si = fmaf(sc, ti, si);
                const float nr = pr * ur - pim * ui;
                pim = pr * ui + pim * ur;
                pr = nr;
            }
        }
    float2* out = Wp + (size_t)pb * p + n;
    float2 o = make_float2(sr, si);
    if (accumulate) {
        o.x += out->x;
        o.y += out->y;
    }
    *out = o;
}

struct LevelPtrs {
    const float2* L[FMM_MAX_LEVEL + 1];
};
struct LevelOutPtrs {
    float2* G[FMM_MAX_LEVEL + 1];
};

// One thread per point: phi_j (+)= (1/r) sum_n L~[leaf][n] w^n, w formed in FP64 and the
// Horner recurrence in FP32 (|w| <= 1/sqrt(2) in radius-scaled units, so it is stable).
// A point's (level, box) must address an existing array; otherwise it is
// skipped and the device error word records the failed check.
__device__ __forceinline__ bool leaf_ok(int l, int64_t b, const void* const* tab, int max_level, int* err)
{
    const bool ok = l >= 0 && l <= max_level && b >= 0 && b < ((int64_t)1 << (2 * l)) && tab[l] != nullptr;
    if (!ok && l >= 2) atomicOr(err, DEV_ERR_CHECK);
    return ok;
}

__global__ void l2p_kernel(int p, int64_t n, const double* __restrict__ z, const int32_t* __restrict__ lev,
                           const int64_t* __restrict__ box, LevelPtrs Ls, int max_level, float2* __restrict__ phi,
                           int accumulate, int* err)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int l = lev[i];
    float ar = 0.f, ai = 0.f;
    if (l >= 2 && leaf_ok(l, box[i], (const void* const*)Ls.L, max_level, err)) {
        const int side = 1 << l;
        const int64_t b = box[i];
        const int bx = (int)(b & (side - 1)), by = (int)(b >> l);
        const double x = z[2 * i], y = z[2 * i + 1];
        long long X, Y;
        float wr, wi;  // offset from the leaf's centre in leaf sides
        if (grid_fixed31(x, l, X) && grid_fixed31(y, l, Y) && (int)(X >> 31) == bx && (int)(Y >> 31) == by) {
            wr = cell_offset31(X);  // no FP64 arithmetic for a point inside its leaf
            wi = cell_offset31(Y);
        } else {
            wr = (float)(x * side - (bx + 0.5));
            wi = (float)(y * side - (by + 0.5));
        }
        const float2* lb = Ls.L[l] + (size_t)b * p;
        for (int k = p - 1; k >= 0; --k) {
            const float2 v = lb[k];
            const float tr = fmaf(ar, wr, fmaf(-ai, wi, v.x));
            ai = fmaf(ar, wi, fmaf(ai, wr, v.y));
            ar = tr;
        }
        ar *= (float)side;
        ai *= (float)side;
    }
    float2 o = make_float2(ar, ai);
    if (accumulate) {
        o.x += phi[i].x;
        o.y += phi[i].y;
    }
    phi[i] = o;
}

// Conjugate transpose of L2P: G[leaf][n] += conj(w^n / r) c_j (FP32 atomic additions).
__global__ void l2p_adjoint_kernel(int p, int64_t n, const double* __restrict__ z, const int32_t* __restrict__ lev,
                                   const int64_t* __restrict__ box, const float2* __restrict__ cot, LevelOutPtrs Gs,
                                   int max_level, int* err)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int l = lev[i];
    if (l < 2 || !leaf_ok(l, box[i], (const void* const*)Gs.G, max_level, err)) return;
    const int side = 1 << l;
    const int64_t b = box[i];
    const double wr = z[2 * i] * side - ((double)(b % side) + 0.5);
    const double wi = -(z[2 * i + 1] * side - ((double)(b / side) + 0.5));  // conj(w)
    const double cr = (double)cot[i].x * side, ci = (double)cot[i].y * side;
    double pr = cr, pi = ci;  // conj(w)^k c side
    float2* gb = Gs.G[l] + (size_t)b * p;
    for (int k = 0; k < p; ++k) {
        atomicAdd(&gb[k].x, (float)pr);
        atomicAdd(&gb[k].y, (float)pi);
        const double t = pr * wr - pi * wi;
        pi = pr * wi + pi * wr;
        pr = t;
    }
}

// P2M adjoint in the positions: grad_i (+)= sum_k G[b][k] conj(c_i k d^(k-1) / r),
// returned as (d/dx, d/dy) = (Re, Im) of that sum.  d (in box sides, |d| <= 1/sqrt 2)
// is read off the bits of the FP64 coordinates (points outside the unit square: the
// clamped box, in FP64) and the series runs in FP32, like the FP32 G it reads.
__global__ void p2m_adjoint_kernel(int level, int p, const double* __restrict__ xy, const double* __restrict__ c,
                                   int64_t n, const float2* __restrict__ G, double* __restrict__ grad, int accumulate)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int side = 1 << level;
    const double x = xy[2 * i], y = xy[2 * i + 1];
    int ix, iy;
    float dr, di;  // conj(d)
    long long X, Y;
    if (grid_fixed31(x, level, X) && grid_fixed31(y, level, Y)) {
        ix = (int)(X >> 31);
        iy = (int)(Y >> 31);
        dr = cell_offset31(X);
        di = -cell_offset31(Y);
    } else {
        const double xs = x * side, ys = y * side;
        ix = (int)floor(xs);
        iy = (int)floor(ys);
        ix = ix < 0 ? 0 : (ix > side - 1 ? side - 1 : ix);
        iy = iy < 0 ? 0 : (iy > side - 1 ? side - 1 : iy);
        dr = (float)(xs - (ix + 0.5));
        di = (float)-(ys - (iy + 0.5));
    }
    const float2* gb = G + ((size_t)iy * side + ix) * p;
    // sum_k G_k k conj(d)^(k-1)
    float sr = 0.f, si = 0.f, pr = 1.f, pi = 0.f;
    for (int k = 1; k < p; ++k) {
        const float2 g = gb[k];
        const float gr = g.x * (float)k, gi = g.y * (float)k;
        sr = fmaf(gr, pr, fmaf(-gi, pi, sr));
        si = fmaf(gr, pi, fmaf(gi, pr, si));
        const float t = pr * dr - pi * di;
        pi = pr * di + pi * dr;
        pr = t;
    }
    const double f = c[i] * side;  // c_i / r
    if (accumulate) {
        grad[2 * i] += f * (double)sr;
        grad[2 * i + 1] += f * (double)si;
    } else {
        grad[2 * i] = f * (double)sr;
        grad[2 * i + 1] = f * (double)si;
    }
}

int launch_l2l(int child_level, int p, const float2* Lp, float2* Lc, bool acc, bool adjoint, cudaStream_t st)
{
    const int64_t side = (int64_t)1 << child_level;
    const int64_t total = (adjoint ? side * side / 4 : side * side) * p;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    if (adjoint)
        l2l_adjoint_kernel<<<blocks, 256, 0, st>>>(child_level, p, Lp, Lc, acc ? 1 : 0);
    else
        l2l_kernel<<<blocks, 256, 0, st>>>(child_level, p, Lp, Lc, acc ? 1 : 0);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

// L2P at points binned by box (fmm_bin_points): one block per box keeps the box's
// LE in shared memory and evaluates it at each of the box's points.  The
// per-point kernel above reads a random box's LE per thread (16 scattered
// 8-byte loads, the SM's L1 serving one line per lane); here the LE is one
// coalesced read per box and every point's Horner loop runs from shared memory.
constexpr int kL2pThreads = 64;

__global__ void __launch_bounds__(kL2pThreads) l2p_binned_kernel(int level, int p, const double* __restrict__ z,
                                                                 int n, const int* __restrict__ perm,
                                                                 const int* __restrict__ box_start,
                                                                 const float2* __restrict__ L, float2* __restrict__ phi,
                                                                 int accumulate, int* err)
{
    __shared__ float2 s_l[64];
    const int side = 1 << level;
    const int b = blockIdx.x, tid = threadIdx.x;
    const int bx = b & (side - 1), by = b >> level;
    int first = box_start[b], end = box_start[b + 1];
    if (first < 0 || end > n || first > end) {
        if (tid == 0) atomicOr(err, DEV_ERR_CHECK);
        return;
    }
    if (first == end) return;
    for (int k = tid; k < p; k += kL2pThreads) s_l[k] = level >= 2 ? L[(size_t)b * p + k] : make_float2(0.f, 0.f);
    __syncthreads();
    for (int q = first + tid; q < end; q += kL2pThreads) {
        const int j = perm[q];
        if ((unsigned)j >= (unsigned)n) {
            atomicOr(err, DEV_ERR_CHECK);
            continue;
        }
        const double x = z[2 * (size_t)j], y = z[2 * (size_t)j + 1];
        long long X, Y;
        float wr, wi;  // offset from the box centre in box sides
        if (grid_fixed31(x, level, X) && grid_fixed31(y, level, Y) && (int)(X >> 31) == bx && (int)(Y >> 31) == by) {
            wr = cell_offset31(X);
            wi = cell_offset31(Y);
        } else {
            wr = (float)(x * side - (bx + 0.5));
            wi = (float)(y * side - (by + 0.5));
        }
        float ar = 0.f, ai = 0.f;
        for (int k = p - 1; k >= 0; --k) {
            const float2 v = s_l[k];
            const float tr = fmaf(ar, wr, fmaf(-ai, wi, v.x));
            ai = fmaf(ar, wi, fmaf(ai, wr, v.y));
            ar = tr;
        }
        float2 o = make_float2(ar * (float)side, ai * (float)side);
        if (accumulate) {
            o.x += phi[j].x;
            o.y += phi[j].y;
        }
        phi[j] = o;
    }
}

int launch_l2p(int p, int64_t n, const double* z, const int32_t* lev, const int64_t* box, const void* const* L,
               int max_level, void* phi, bool acc, bool adjoint, cudaStream_t st)
{
    if (n == 0) return FMM_OK;
    int* err = nullptr;
    int rc = device_error_word(&err);
    if (rc) return rc;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (!adjoint) {
        LevelPtrs Ls{};
        for (int l = 0; l <= max_level; ++l) Ls.L[l] = (const float2*)L[l];
        l2p_kernel<<<blocks, 256, 0, st>>>(p, n, z, lev, box, Ls, max_level, (float2*)phi, acc ? 1 : 0, err);
    } else {
        LevelOutPtrs Gs{};
        for (int l = 0; l <= max_level; ++l) Gs.G[l] = (float2*)L[l];
        l2p_adjoint_kernel<<<blocks, 256, 0, st>>>(p, n, z, lev, box, (const float2*)phi, Gs, max_level, err);
    }
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

int launch_p2m_adjoint(int level, int p, const double* xy, const double* c, int64_t n, const float2* G, double* grad,
                       bool acc, cudaStream_t st)
{
    if (n == 0) return FMM_OK;
    p2m_adjoint_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(level, p, xy, c, n, G, grad, acc ? 1 : 0);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

// Deepest existing box holding each point: the box of level l is
// (floor(x 2^l), floor(y 2^l)) clamped to the level (reading R5), read off the
// bits of the FP64 coordinates; levels without an existence mask have every box.
struct LeafLevelMasks {
    const uint8_t* ex[FMM_MAX_LEVEL + 1];
};

__global__ void leaf_boxes_kernel(int max_level, LeafLevelMasks m, const double* __restrict__ xy, int64_t n,
                                  int32_t* __restrict__ lev, int64_t* __restrict__ box)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = xy[2 * i], y = xy[2 * i + 1];
    int bl = 0;
    int64_t bb = 0;
    for (int l = 0; l <= max_level; ++l) {
        const int64_t b = ((int64_t)grid_cell(y, l) << l) | grid_cell(x, l);
        if (!m.ex[l] || m.ex[l][b]) {
            bl = l;
            bb = b;
        }
    }
    lev[i] = bl;
    box[i] = bb;
}

}  // namespace fmmgb

using namespace fmmgb;

static int far_common(const char* who, int32_t p, const void* a, const void* b)
{
    if (p < 1 || p > 64) return fail(FMM_EINVAL, "%s: p = %d outside 1..64", who, p);
    if (!a || !b) return fail(FMM_EINVAL, "%s: NULL pointer", who);
    if (((uintptr_t)a & 7) || ((uintptr_t)b & 7)) return fail(FMM_EINVAL, "%s: pointers must be 8-byte aligned", who);
    return FMM_OK;
}

extern "C" {

int fmm_l2l(int32_t child_level, int32_t p, const void* Lp, void* Lc, int32_t flags, void* stream)
{
    clear_error();
    if (child_level < 1 || child_level > FMM_MAX_LEVEL)
        return fail(FMM_EINVAL, "fmm_l2l: child_level %d outside 1..%d", child_level, FMM_MAX_LEVEL);
    if (int rc = far_common("fmm_l2l", p, Lp, Lc)) return rc;
    if (flags & ~FMM_ACCUMULATE) return fail(FMM_EINVAL, "fmm_l2l: unknown flags 0x%x", flags);
    return launch_l2l(child_level, p, (const float2*)Lp, (float2*)Lc, (flags & FMM_ACCUMULATE) != 0, false,
                      (cudaStream_t)stream);
}

int fmm_l2l_adjoint(int32_t child_level, int32_t p, const void* Wc, void* Wp, int32_t flags, void* stream)
{
    clear_error();
    if (child_level < 1 || child_level > FMM_MAX_LEVEL)
        return fail(FMM_EINVAL, "fmm_l2l_adjoint: child_level %d outside 1..%d", child_level, FMM_MAX_LEVEL);
    if (int rc = far_common("fmm_l2l_adjoint", p, Wc, Wp)) return rc;
    if (flags & ~FMM_ACCUMULATE) return fail(FMM_EINVAL, "fmm_l2l_adjoint: unknown flags 0x%x", flags);
    return launch_l2l(child_level, p, (const float2*)Wc, (float2*)Wp, (flags & FMM_ACCUMULATE) != 0, true,
                      (cudaStream_t)stream);
}

static int l2p_common(const char* who, int32_t p, int64_t n, const double* z, const int32_t* lev, const int64_t* box,
                      const void* const* L, int32_t max_level, const void* phi)
{
    if (p < 1 || p > 64) return fail(FMM_EINVAL, "%s: p = %d outside 1..64", who, p);
    if (n < 0) return fail(FMM_EINVAL, "%s: n < 0", who);
    if (max_level < 0 || max_level > FMM_MAX_LEVEL)
        return fail(FMM_EINVAL, "%s: max_level %d outside 0..%d", who, max_level, FMM_MAX_LEVEL);
    if (!L) return fail(FMM_EINVAL, "%s: NULL level array", who);
    if (n > 0 && (!z || !lev || !box || !phi)) return fail(FMM_EINVAL, "%s: NULL pointer", who);
    if (((uintptr_t)z & 7) || ((uintptr_t)phi & 7) || ((uintptr_t)box & 7) || ((uintptr_t)lev & 3))
        return fail(FMM_EINVAL, "%s: misaligned pointer", who);
    for (int l = 0; l <= max_level; ++l)
        if ((uintptr_t)L[l] & 7) return fail(FMM_EINVAL, "%s: level %d array misaligned", who, l);
    return FMM_OK;
}

int fmm_l2p(int32_t p, int64_t n, const double* z, const int32_t* lev, const int64_t* box, const void* const* L_levels,
            int32_t max_level, void* phi, int32_t flags, void* stream)
{
    clear_error();
    if (int rc = l2p_common("fmm_l2p", p, n, z, lev, box, L_levels, max_level, phi)) return rc;
    if (flags & ~FMM_ACCUMULATE) return fail(FMM_EINVAL, "fmm_l2p: unknown flags 0x%x", flags);
    return launch_l2p(p, n, z, lev, box, L_levels, max_level, phi, (flags & FMM_ACCUMULATE) != 0, false,
                      (cudaStream_t)stream);
}

int fmm_l2p_binned(int32_t level, int32_t p, const double* z, int64_t n, const int32_t* perm,
                   const int32_t* box_start, const void* L, void* phi, int32_t flags, void* stream)
{
    clear_error();
    if (level < 0 || level > 10) return fail(FMM_EINVAL, "fmm_l2p_binned: level %d outside 0..10", level);
    if (p < 1 || p > 64) return fail(FMM_EINVAL, "fmm_l2p_binned: p = %d outside 1..64", p);
    if (n < 0 || n > INT32_MAX) return fail(FMM_EINVAL, "fmm_l2p_binned: n = %lld outside 0..2^31-1", (long long)n);
    if (!box_start || (n > 0 && (!z || !perm || !phi || (level >= 2 && !L))))
        return fail(FMM_EINVAL, "fmm_l2p_binned: NULL pointer");
    if (((uintptr_t)z & 7) || ((uintptr_t)phi & 7) || ((uintptr_t)L & 7) || ((uintptr_t)perm & 3) ||
        ((uintptr_t)box_start & 3))
        return fail(FMM_EINVAL, "fmm_l2p_binned: misaligned pointer");
    if (flags & ~FMM_ACCUMULATE) return fail(FMM_EINVAL, "fmm_l2p_binned: unknown flags 0x%x", flags);
    if (n == 0) return FMM_OK;
    int* err = nullptr;
    if (int rc = device_error_word(&err)) return rc;
    l2p_binned_kernel<<<1u << (2 * level), kL2pThreads, 0, (cudaStream_t)stream>>>(
        level, p, z, (int)n, perm, box_start, (const float2*)L, (float2*)phi, (flags & FMM_ACCUMULATE) ? 1 : 0, err);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

int fmm_l2p_adjoint(int32_t p, int64_t n, const double* z, const int32_t* lev, const int64_t* box, const void* cot,
                    void* const* G_levels, int32_t max_level, void* stream)
{
    clear_error();
    if (int rc = l2p_common("fmm_l2p_adjoint", p, n, z, lev, box, (const void* const*)G_levels, max_level, cot))
        return rc;
    return launch_l2p(p, n, z, lev, box, (const void* const*)G_levels, max_level, const_cast<void*>(cot), true, true,
                      (cudaStream_t)stream);
}

int fmm_p2m_adjoint(int32_t level, int32_t p, const double* xy, const double* c, int64_t n, const void* G,
                    double* grad, int32_t flags, void* stream)
{
    clear_error();
    if (level < 0 || level > FMM_MAX_LEVEL)
        return fail(FMM_EINVAL, "fmm_p2m_adjoint: level %d outside 0..%d", level, FMM_MAX_LEVEL);
    if (p < 1 || p > 64) return fail(FMM_EINVAL, "fmm_p2m_adjoint: p = %d outside 1..64", p);
    if (n < 0) return fail(FMM_EINVAL, "fmm_p2m_adjoint: n < 0");
    if (!G || (n > 0 && (!xy || !c || !grad))) return fail(FMM_EINVAL, "fmm_p2m_adjoint: NULL pointer");
    if (((uintptr_t)G & 7) || ((uintptr_t)xy & 7) || ((uintptr_t)c & 7) || ((uintptr_t)grad & 7))
        return fail(FMM_EINVAL, "fmm_p2m_adjoint: misaligned pointer");
    if (flags & ~FMM_ACCUMULATE) return fail(FMM_EINVAL, "fmm_p2m_adjoint: unknown flags 0x%x", flags);
    return launch_p2m_adjoint(level, p, xy, c, n, (const float2*)G, grad, (flags & FMM_ACCUMULATE) != 0,
                              (cudaStream_t)stream);
}

int fmm_leaf_boxes(const fmm_tree* tree, const double* xy, int64_t n, int32_t* level, int64_t* box, void* stream)
{
    clear_error();
    if (!tree) return fail(FMM_EINVAL, "fmm_leaf_boxes: NULL tree");
    if (n < 0) return fail(FMM_EINVAL, "fmm_leaf_boxes: n < 0");
    if (n > 0 && (!xy || !level || !box)) return fail(FMM_EINVAL, "fmm_leaf_boxes: NULL pointer");
    if (((uintptr_t)xy & 7) || ((uintptr_t)box & 7) || ((uintptr_t)level & 3))
        return fail(FMM_EINVAL, "fmm_leaf_boxes: misaligned pointer");
    if (n == 0) return FMM_OK;
    const int L = tree_max_level(tree);
    LeafLevelMasks m = {};
    for (int l = 0; l <= L; ++l) {
        const int32_t* tiles = nullptr;
        int ntiles = 0;
        if (int rc = tree_device_level(tree, l, &m.ex[l], &tiles, &ntiles)) return rc;
    }
    leaf_boxes_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(L, m, xy, n, level, box);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

}  // extern "C"
