// p2p.cu -- the near field of a uniform quadtree at its finest level
// (Sec. 2.1 stage 5: Eq. n_body restricted to each target's own and adjacent
// boxes, the complement of the interaction lists of every level):
//
//   phi(z) (+)= sum_{i : box(y_i) adjacent to or equal box(z), y_i != z} c_i / (z - y_i).
//
// Targets and sources are binned by box (fmm_bin_points); a pre-pass copies the
// sources into box order, each as its position relative to its own box's
// centre in box sides (read off the bits of the FP64 position, kept in FP32)
// and strength, so a box's sources are one contiguous range and staging adds
// only the exact offset between box centres (-1, 0 or 1) -- no FP64
// arithmetic per staged source or per claim.  Persistent CTAs of 128 threads claim runs of up to 96 targets of
// one box from a claim table (a finest-level box holds a few dozen points, so
// nearly every box is one claim), gather the sources of the 3 x 3
// neighbourhood into shared memory in batches -- position relative to the
// target box's centre and strength -- and each warp sums the run's targets
// (one to three rows of 32, as many as the run fills, one target per lane and
// row) against a quarter of every batch; the four partial sums of a target
// meet in shared memory.  In FP32:
//   1/(dx + i dy) = (dx - i dy) / r2 with one approximate reciprocal per pair,
// dx, dy in box sides, and the sums scaled by 2^level (exact) at the end.
// Positions relative to the target box keep |dx|, |dy| <= 1.5 box sides, so
// FP32 carries the difference of two nearby points to ~2^-24 of a box side.
// A source at the target's position (the point itself, when targets are the
// sources) contributes nothing: r^2 carries a 1e-30 offset and dx = dy = 0.
#include <mutex>

#include "fgt_hermite.cuh"

namespace fmmgb {

constexpr int kP2pThreads = 128;
constexpr int kP2pWarps = kP2pThreads / 32;     // each takes a quarter of the sources
constexpr int kP2pR = 3;                        // targets per lane (rows of 32 targets per claim)
constexpr int kP2pRun = 32 * kP2pR;             // targets per claim
constexpr int kP2pBatch = 1024;                 // sources per shared-memory batch
constexpr int kP2pSharedCtas = 8;               // resident CTAs per SM with FMM_P2P_SHARE_SM
// added to every r^2 (in box sides squared): a source at the target's position
// (dx = dy = 0) then contributes exactly 0 -- c / 1e-30 is finite for |c| < 3e8 -- and
// any other pair changes by a relative 1e-30 / r^2 (below FP32 rounding for distances
// above 1e-11 box sides; positions resolve 2^-31 of a side, 4.7e-10)
constexpr float kP2pTiny = 1e-30f;

struct P2pArgs {
    int level, n, nz, accumulate;
    const double* xy;
    const double* c;
    const float4* src;  // sources in box order: x, y relative to their own box's centre, c (p2p_sort_kernel)
    const int* sperm;
    const int* sstart;
    const double* z;
    const int* tperm;
    const int* tstart;
    const int* claims;
    const int4* tab;  // claim table (p2p_claim_table_kernel), ntab entries
    int ntab;
    float2* phi;
    int* cursor;  // [0] next claim index, [1] CTAs finished
    int* err;
};

// sources in box order, so that a box's sources are one contiguous range; positions relative to
// the centre of their own box in box sides, read off the bits of the FP64 coordinates and kept
// in FP32 (|x - c| <= 1/2)
__global__ void p2p_sort_kernel(int level, const double* __restrict__ xy, const double* __restrict__ c,
                                const int* __restrict__ perm, int n, float4* __restrict__ out, int* err)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = __ldg(perm + k);
    if ((unsigned)i >= (unsigned)n) {
        atomicOr(err, DEV_ERR_CHECK);
        out[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const double x = __ldg(xy + 2 * (size_t)i), y = __ldg(xy + 2 * (size_t)i + 1);
    const float cf = (float)__ldg(c + i);
    long long X, Y;
    if (grid_fixed31(x, level, X) && grid_fixed31(y, level, Y)) {
        out[k] = make_float4(cell_offset31(X), cell_offset31(Y), cf, 0.f);  // offset in box sides
        return;
    }
    // outside the unit square: the clamped box, offset in FP64 (x 2^level is exact)
    const int side = 1 << level;
    const double px = x * side, py = y * side;
    const int ix = !(px >= 0.0) ? 0 : (px >= side ? side - 1 : (int)px);
    const int iy = !(py >= 0.0) ? 0 : (py >= side ? side - 1 : (int)py);
    out[k] = make_float4((float)(px - (ix + 0.5)), (float)(py - (iy + 0.5)), cf, 0.f);
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Packed two-lane FP32 (PTX f32x2): two targets of a lane in one 64-bit register pair.
__device__ __forceinline__ unsigned long long p2_pk(float a, float b)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 p2_upk(unsigned long long v)
{
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ unsigned long long p2_sub(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long p2_mul(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long p2_fma(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// One warp's share of a staged batch (sources warp, warp + 4, ...) against the
// claim's NR occupied rows of 32 targets (NR warp-uniform: empty rows cost nothing).
// Rows 0 and 1 run as one packed pair (dx, dy, r^2, the weight and both sums in
// f32x2 operations; the two reciprocals stay scalar), row 2 alone.
template <int NR>
__device__ __forceinline__ void p2p_batch(const float4* __restrict__ s_src, int cnt, int warp, const float* zx,
                                          const float* zy, float* re, float* im)
{
    if constexpr (NR >= 2) {
        const unsigned long long zx01 = p2_pk(zx[0], zx[1]), zy01 = p2_pk(zy[0], zy[1]);
        const unsigned long long tiny = p2_pk(kP2pTiny, kP2pTiny);
        unsigned long long re01 = p2_pk(re[0], re[1]), im01 = p2_pk(-im[0], -im[1]);  // im01 sums +w dy
        float re2 = NR > 2 ? re[2] : 0.f, im2 = NR > 2 ? im[2] : 0.f;
#pragma unroll 8
        for (int i = warp; i < cnt; i += kP2pWarps) {
            const float4 v = s_src[i];
            const unsigned long long dx = p2_sub(zx01, p2_pk(v.x, v.x)), dy = p2_sub(zy01, p2_pk(v.y, v.y));
            const float2 r2 = p2_upk(p2_fma(dx, dx, p2_fma(dy, dy, tiny)));
            const unsigned long long w = p2_mul(p2_pk(v.z, v.z), p2_pk(rcp_approx(r2.x), rcp_approx(r2.y)));
            re01 = p2_fma(w, dx, re01);
            im01 = p2_fma(w, dy, im01);
            if constexpr (NR > 2) {
                const float ex = zx[2] - v.x, ey = zy[2] - v.y;
                const float q2 = fmaf(ex, ex, fmaf(ey, ey, kP2pTiny));
                const float u = v.z * rcp_approx(q2);
                re2 = fmaf(u, ex, re2);
                im2 = fmaf(-u, ey, im2);
            }
        }
        const float2 a = p2_upk(re01), b = p2_upk(im01);
        re[0] = a.x;
        re[1] = a.y;
        im[0] = -b.x;
        im[1] = -b.y;
        if constexpr (NR > 2) {
            re[2] = re2;
            im[2] = im2;
        }
    } else {
#pragma unroll 4
        for (int i = warp; i < cnt; i += kP2pWarps) {
            const float4 v = s_src[i];
            const float dx = zx[0] - v.x, dy = zy[0] - v.y;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, kP2pTiny));
            const float w = v.z * rcp_approx(r2);
            re[0] = fmaf(w, dx, re[0]);
            im[0] = fmaf(-w, dy, im[0]);
        }
    }
}

// Claim table: entry k = (first, end, box) of the k-th run of at most kP2pRun
// targets of one box (the runs of box b are claims[b] .. claims[b+1]-1), so a
// CTA finds its claim with one load instead of a binary search over the boxes.
// Runs past `cap` entries, or a box_start that does not bin [0, nz), set the
// error word (the kernel then skips those runs).
__global__ void p2p_claim_table_kernel(int nbox, const int* __restrict__ claims, const int* __restrict__ tstart,
                                       int nz, int cap, int4* __restrict__ tab, int* err)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    const int c0 = claims[b], c1 = claims[b + 1];
    const int f0 = tstart[b], e0 = min(tstart[b + 1], nz);
    for (int k = c0; k < c1; ++k) {
        if (k < 0 || k >= cap) {
            atomicOr(err, DEV_ERR_CHECK);
            return;
        }
        const int f = f0 + (k - c0) * kP2pRun, e = min(f + kP2pRun, e0);
        const bool ok = 0 <= f && f < e;
        if (!ok) atomicOr(err, DEV_ERR_CHECK);
        tab[k] = ok ? make_int4(f, e, b, 0) : make_int4(0, 0, b, 0);
    }
}

__global__ void __launch_bounds__(kP2pThreads) fmm_p2p_kernel(P2pArgs a)
{
    __shared__ float4 s_src[kP2pBatch];  // position relative to the target box's centre (box sides), c
    __shared__ int4 s_claim;
    __shared__ int s_box[9], s_cnt[9];  // first sorted source and source count of each neighbour box
    __shared__ float s_ox[9], s_oy[9];  // centre of each neighbour box minus the target box's (box sides)
    __shared__ float2 s_part[kP2pWarps - 1][kP2pRun];  // partial sums of warps 1..3

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int side = 1 << a.level;
    const int total = min(__ldg(a.claims + (side * side)), a.ntab);
    // thread 0 fetches the index of the CTA's next claim one claim ahead
    int knext = tid == 0 ? atomicAdd(a.cursor, 1) : 0;

    for (;;) {
        if (tid == 0) {
            const int k = knext;
            s_claim = k < total ? __ldg(a.tab + k) : make_int4(-1, -1, 0, 0);
            if (k < total) knext = atomicAdd(a.cursor, 1);
        }
        __syncthreads();
        const int4 cl = s_claim;
        const int first = cl.x, end = cl.y, box = cl.z;
        if (first < 0) break;
        const int nrow = (end - first + 31) >> 5;  // occupied rows of 32 targets (0..kP2pR)
        const int tx = box & (side - 1), ty = box >> a.level;
        if (tid < 9) {  // the 3 x 3 neighbourhood, one box per thread
            const int sx = tx + tid % 3 - 1, sy = ty + tid / 3 - 1;
            s_ox[tid] = (float)(tid % 3 - 1);
            s_oy[tid] = (float)(tid / 3 - 1);
            int b0 = -1, m = 0;
            if (sx >= 0 && sy >= 0 && sx < side && sy < side) {
                const int b = sy * side + sx;
                b0 = __ldg(a.sstart + b);
                m = __ldg(a.sstart + b + 1) - b0;
                if (m <= 0 || b0 < 0 || b0 + m > a.n) {
                    b0 = -1;
                    m = 0;
                }
            }
            s_box[tid] = b0;
            s_cnt[tid] = m;
        }

        int tj[kP2pR];
        float zx[kP2pR], zy[kP2pR], re[kP2pR], im[kP2pR];
#pragma unroll
        for (int r = 0; r < kP2pR; ++r) {
            const int pos = first + r * 32 + lane;
            tj[r] = -1;
            zx[r] = zy[r] = re[r] = im[r] = 0.f;
            if (pos < end) {
                const int j = __ldg(a.tperm + pos);
                if ((unsigned)j < (unsigned)a.nz) {
                    tj[r] = j;
                    const double x = __ldg(a.z + 2 * (size_t)j), y = __ldg(a.z + 2 * (size_t)j + 1);
                    long long X, Y;
                    if (grid_fixed31(x, a.level, X) && grid_fixed31(y, a.level, Y) && (int)(X >> 31) == tx &&
                        (int)(Y >> 31) == ty) {
                        zx[r] = cell_offset31(X);  // in the claimed box: no FP64 arithmetic
                        zy[r] = cell_offset31(Y);
                    } else {  // outside it (coordinates outside the unit square): FP64, x 2^level exact
                        zx[r] = (float)(x * side - (tx + 0.5));
                        zy[r] = (float)(y * side - (ty + 0.5));
                    }
                } else if (warp == 0) {
                    atomicOr(a.err, DEV_ERR_CHECK);
                }
            }
        }
        __syncthreads();
        int pre[10];  // prefix of the neighbour boxes' source counts
        pre[0] = 0;
#pragma unroll
        for (int q = 0; q < 9; ++q) pre[q + 1] = pre[q] + s_cnt[q];
        const int S = pre[9];

        for (int base = 0; base < S; base += kP2pBatch) {
            const int cnt = min(kP2pBatch, S - base);
            for (int i = tid; i < cnt; i += kP2pThreads) {
                const int g = base + i;
                int q = 0;
#pragma unroll
                for (int t = 1; t < 9; ++t) q += pre[t] <= g;  // the neighbour box holding source g
                const int b0 = s_box[q];
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (b0 >= 0) {
                    int off = 0;  // pre[q], with registers indexed by constants only
#pragma unroll
                    for (int t = 1; t < 9; ++t) off = t == q ? pre[t] : off;
                    const float4 u = a.src[b0 + (g - off)];
                    v.x = u.x + s_ox[q];
                    v.y = u.y + s_oy[q];
                    v.z = u.z;
                }
                s_src[i] = v;
            }
            __syncthreads();
            switch (nrow) {
                case 0: break;  // a run the claim table flagged (error word set)
                case 1: p2p_batch<1>(s_src, cnt, warp, zx, zy, re, im); break;
                case 2: p2p_batch<2>(s_src, cnt, warp, zx, zy, re, im); break;
                default: p2p_batch<3>(s_src, cnt, warp, zx, zy, re, im); break;
            }
            __syncthreads();  // the batch buffer is refilled next
        }
        if (warp > 0) {
#pragma unroll
            for (int r = 0; r < kP2pR; ++r)
                if (r < nrow) s_part[warp - 1][r * 32 + lane] = make_float2(re[r], im[r]);
        }
        __syncthreads();
        if (warp > 0) continue;  // warp 0 writes; every warp is back at the claim's barrier next
#pragma unroll
        for (int r = 0; r < kP2pR; ++r) {
            if (tj[r] < 0) continue;
            float2 o = make_float2(re[r], im[r]);
#pragma unroll
            for (int q = 0; q < kP2pWarps - 1; ++q) {
                o.x += s_part[q][r * 32 + lane].x;
                o.y += s_part[q][r * 32 + lane].y;
            }
            o.x *= (float)side;  // 1/(z - y) = 2^level / ((z - y) in box sides): exact scaling
            o.y *= (float)side;
            if (a.accumulate) {
                const float2 old = a.phi[tj[r]];
                o.x += old.x;
                o.y += old.y;
            }
            a.phi[tj[r]] = o;
        }
    }
    // the last CTA to finish returns the cursor slot to zero for its next use
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(a.cursor + 1, 1) == (int)gridDim.x - 1) {
            atomicExch(a.cursor, 0);
            atomicExch(a.cursor + 1, 0);
        }
    }
}

// Per-device buffer of sorted sources (grown on demand).
static std::mutex g_src_mu;
static float4* g_src[64];
static size_t g_src_bytes[64];

static int p2p_source_buffer(size_t bytes, float4** out)
{
    int dev = 0;
    FMM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(FMM_EUNSUPPORTED, "fmm_p2p: device ordinal %d above 63", dev);
    std::lock_guard<std::mutex> lk(g_src_mu);
    if (g_src_bytes[dev] < bytes) {
        if (g_src[dev]) {
            FMM_CUDA_TRY(cudaDeviceSynchronize());
            cudaFree(g_src[dev]);
            g_src[dev] = nullptr;
            g_src_bytes[dev] = 0;
        }
        FMM_CUDA_TRY(cudaMalloc(&g_src[dev], bytes));
        g_src_bytes[dev] = bytes;
    }
    *out = g_src[dev];
    return FMM_OK;
}

}  // namespace fmmgb

using namespace fmmgb;

extern "C" int fmm_p2p(int32_t level, const double* xy, const double* c, int64_t n, const int32_t* src_perm,
                       const int32_t* src_start, const double* z, int64_t nz, const int32_t* tgt_perm,
                       const int32_t* tgt_start, void* phi, int32_t flags, void* stream)
{
    clear_error();
    if (level < 0 || level > 10) return fail(FMM_EINVAL, "fmm_p2p: level %d outside 0..10", level);
    if (n < 0 || n > INT32_MAX || nz < 0 || nz > INT32_MAX)
        return fail(FMM_EINVAL, "fmm_p2p: point counts must lie in 0..2^31-1");
    if (!src_start || !tgt_start || (n > 0 && (!xy || !c || !src_perm)) || (nz > 0 && (!z || !tgt_perm || !phi)))
        return fail(FMM_EINVAL, "fmm_p2p: NULL pointer");
    if (((uintptr_t)xy & 7) || ((uintptr_t)c & 7) || ((uintptr_t)z & 7) || ((uintptr_t)phi & 7) ||
        ((uintptr_t)src_perm & 3) || ((uintptr_t)src_start & 3) || ((uintptr_t)tgt_perm & 3) ||
        ((uintptr_t)tgt_start & 3))
        return fail(FMM_EINVAL, "fmm_p2p: misaligned pointer (xy, c, z, phi 8 bytes; int32 arrays 4)");
    if (flags & ~(FMM_ACCUMULATE | FMM_P2P_SHARE_SM)) return fail(FMM_EINVAL, "fmm_p2p: unknown flags 0x%x", flags);
    if (nz == 0) return FMM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    P2pArgs args;
    args.level = level;
    args.n = (int)n;
    args.nz = (int)nz;
    args.accumulate = (flags & FMM_ACCUMULATE) ? 1 : 0;
    args.xy = xy;
    args.c = c;
    args.sperm = src_perm;
    args.sstart = src_start;
    args.z = z;
    args.tperm = tgt_perm;
    args.tstart = tgt_start;
    args.phi = reinterpret_cast<float2*>(phi);
    if (int rc = tile_counter(&args.cursor, st)) return rc;
    if (int rc = device_error_word(&args.err)) return rc;
    unsigned char* scratch = nullptr;
    if (int rc = fgt_flag_buffer(&scratch)) return rc;
    int* claims = reinterpret_cast<int*>(scratch + kFgtFlagBytes);
    args.claims = claims;
    const int nbox = 1 << (2 * level);
    if (int rc = launch_h2p_claims(nbox, tgt_start, kP2pRun, claims, args.err, st)) return rc;
    // one buffer: the sources in box order, then the claim table
    const int64_t most = nz / kP2pRun + nbox;  // claims can be no more
    float4* src = nullptr;
    if (int rc = p2p_source_buffer((size_t)(n + most) * sizeof(float4), &src)) return rc;
    int4* tab = reinterpret_cast<int4*>(src + n);
    p2p_claim_table_kernel<<<(unsigned)((nbox + 255) / 256), 256, 0, st>>>(nbox, claims, tgt_start, (int)nz, (int)most,
                                                                          tab, args.err);
    FMM_CUDA_TRY(cudaGetLastError());
    if (n > 0) {
        p2p_sort_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(level, xy, c, src_perm, (int)n, src, args.err);
        FMM_CUDA_TRY(cudaGetLastError());
    }
    args.src = src;
    args.tab = tab;
    args.ntab = (int)most;
    static int occ;
    static std::mutex mu;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!occ) {
            FMM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fmm_p2p_kernel, kP2pThreads, 0));
            if (occ < 1) occ = 1;
        }
    }
    int sms = 0;
    if (int rc = device_sm_count(&sms)) return rc;
    // sharing the SMs with kernels of other streams: 8 CTAs (132 KB of shared memory, 1,024
    // threads) per SM measured 1.5 % slower alone than the occupancy limit, and left room for
    // the far field of the same FMM beside it (fewer starved the near field itself)
    const int per_sm = (flags & FMM_P2P_SHARE_SM) ? std::min(occ, kP2pSharedCtas) : occ;
    const int grid = (int)std::min<int64_t>((int64_t)per_sm * sms, most);
    fmm_p2p_kernel<<<grid, kP2pThreads, 0, st>>>(args);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}
