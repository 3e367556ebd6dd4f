// fgt_hermite.cu -- the fast Gauss transform evaluated directly from Hermite
// series at target points (Sec. 4.2, Eq. hermite), over the n_cut
// neighbourhood of each target's box on the uniform 2^g x 2^g grid:
//
//   G(y) (+)= sum_{B : max(|sx-tx|,|sy-ty|) <= n_cut}
//               sum_{a1,a2 < p} A_B[a1][a2] h_a1((y1 - sB1)/(sqrt2 sigma)) h_a2((y2 - sB2)/(sqrt2 sigma)),
//
// h_n(t) = exp(-t^2) H_n(t).  Targets are first binned by box (a counting
// sort on the device), so that one CTA serves a run of targets of one box and
// stages each source box's p x p coefficients in shared memory once for all
// of them -- the paper's design point of keeping the series coefficients in
// shared memory for a block of targets, without its per-call size limits.
// The same binning gives a P2H (Eq. A_alpha) without contended atomics.
//
// Evaluation kernel (FP32, CUDA cores; no dense contraction here that tensor
// cores could take without forming an m x p^2 operand per box):
//   - persistent CTAs of 128 threads claim runs of up to 128 R targets of one
//     box by an atomic claim index and a per-box claim table built just
//     before (a scan of ceil(targets / run) over the boxes);
//   - the neighbourhood is walked one source row at a time: the row's boxes
//     are contiguous in A and are copied to shared memory with cp.async,
//     double-buffered, while the previous row is evaluated;
//   - per thread R targets; per row h_b(t2) is formed once by the three-term
//     recurrence h_{n+1} = 2t h_n - 2n h_{n-1}; per box
//     acc += sum_a h_a(t1) sum_b A[a][b] h_b(t2), the outer sum by Clenshaw's
//     backward recurrence (p^2 + 2p multiply-adds, the A rows read as broadcast
//     float4 from shared memory);
//   - t = u + k d with u = (y - t_C)/(sqrt2 sigma) formed once per target in
//     FP64 and k d (k = tx - sx, d = side/(sqrt2 sigma)) from a small table,
//     so no FP64 arithmetic runs per box;
//   - boxes whose coefficients are all zero (no sources) are skipped.
#include <mutex>

#include "fgt_hermite.cuh"

namespace fmmgb {

// ---------------------------------------------------------------------------
// binning of points by grid box
// ---------------------------------------------------------------------------
constexpr int kBinThreads = 256;
constexpr int kScanThreads = 1024;

__device__ __forceinline__ int fgt_grid_box(double x, double y, int g)
{
    // floor(v 2^g) per coordinate, clamped to the grid; NaN and negatives to cell 0
    return grid_cell(y, g) * (1 << g) + grid_cell(x, g);
}

// Warp-aggregated counting: the lanes of a warp whose points share a box make
// one atomic between them (clustered inputs put many points of a warp in one
// box), and each lane learns its rank among them.  Every lane of the warp calls
// it (key < 0: no point); returns the box's count before the warp's additions
// plus the lane's rank, or -1 without a point.
__device__ __forceinline__ int warp_box_claim(int* __restrict__ counter, int key)
{
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    int base = 0;
    if (key >= 0 && lane == leader) base = atomicAdd(&counter[key], __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    return key >= 0 ? base + __popc(peers & ((1u << lane) - 1u)) : -1;
}

// grid-stride over warps: all 32 lanes of a warp take part in every round
__global__ void bin_count_kernel(int g, const double* __restrict__ y, int64_t n, int* __restrict__ counts)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = w0; 32 * w < n; w += nw) {
        const int64_t i = 32 * w + lane;
        const int key = i < n ? fgt_grid_box(__ldg(y + 2 * i), __ldg(y + 2 * i + 1), g) : -1;
        warp_box_claim(counts, key);
    }
}

// One CTA: exclusive scan of v(0..nbox-1) into out[0..nbox] (out[nbox] = total); put(i, prefix)
// also receives each prefix.
template <class Load, class Put>
__device__ void block_exclusive_scan(int nbox, Load v, Put put, int* out)
{
    __shared__ int s_warp[kScanThreads / 32];
    __shared__ int s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < nbox; base += kScanThreads) {
        const int i = base + tid;
        const int c = i < nbox ? v(i) : 0;
        int x = c;  // inclusive warp scan
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = s_warp[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        const int excl = s_carry + (warp ? s_warp[warp - 1] : 0) + x - c;
        if (i < nbox) {
            out[i] = excl;
            put(i, excl);
        }
        __syncthreads();
        if (tid == kScanThreads - 1) s_carry = excl + c;
        __syncthreads();
    }
    if (tid == 0) out[nbox] = s_carry;
}

// box_start[0..nbox] = exclusive scan of counts; counts becomes the scatter cursor (the same prefix)
__global__ void __launch_bounds__(kScanThreads) bin_scan_kernel(int nbox, int* counts, int* __restrict__ box_start)
{
    block_exclusive_scan(
        nbox, [&](int i) { return counts[i]; }, [&](int i, int e) { counts[i] = e; }, box_start);
}

__global__ void bin_scatter_kernel(int g, const double* __restrict__ y, int64_t n, int* __restrict__ cursor,
                                   int* __restrict__ perm)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = w0; 32 * w < n; w += nw) {
        const int64_t i = 32 * w + lane;
        const int key = i < n ? fgt_grid_box(__ldg(y + 2 * i), __ldg(y + 2 * i + 1), g) : -1;
        const int slot = warp_box_claim(cursor, key);
        if (slot >= 0) perm[slot] = (int)i;
    }
}

// Small grids (up to 4^7 boxes): a block counts its contiguous chunk of points in a
// shared-memory histogram, so contended boxes (clustered points) cost shared-memory
// atomics, and the global counters see one addition per box a block touches.
constexpr int kBinSmemMaxLog2 = 7;

__global__ void __launch_bounds__(kBinThreads) bin_count_smem_kernel(int g, const double* __restrict__ y, int64_t n,
                                                                     int64_t chunk, int* __restrict__ counts)
{
    extern __shared__ int s_cnt[];
    const int nbox = 1 << (2 * g);
    for (int b = threadIdx.x; b < nbox; b += kBinThreads) s_cnt[b] = 0;
    __syncthreads();
    const int64_t i0 = (int64_t)blockIdx.x * chunk, i1 = i0 + chunk < n ? i0 + chunk : n;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += kBinThreads)
        atomicAdd(&s_cnt[fgt_grid_box(__ldg(y + 2 * i), __ldg(y + 2 * i + 1), g)], 1);
    __syncthreads();
    for (int b = threadIdx.x; b < nbox; b += kBinThreads)
        if (s_cnt[b]) atomicAdd(&counts[b], s_cnt[b]);
}

// The scatter over the same kind of chunks: recount the chunk, reserve each
// touched box's range with one global atomic, then place the points with
// shared-memory atomics.
__global__ void __launch_bounds__(kBinThreads) bin_scatter_smem_kernel(int g, const double* __restrict__ y, int64_t n,
                                                                       int64_t chunk, int* __restrict__ cursor,
                                                                       int* __restrict__ perm)
{
    extern __shared__ int s_cnt[];
    const int nbox = 1 << (2 * g);
    for (int b = threadIdx.x; b < nbox; b += kBinThreads) s_cnt[b] = 0;
    __syncthreads();
    const int64_t i0 = (int64_t)blockIdx.x * chunk, i1 = i0 + chunk < n ? i0 + chunk : n;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += kBinThreads)
        atomicAdd(&s_cnt[fgt_grid_box(__ldg(y + 2 * i), __ldg(y + 2 * i + 1), g)], 1);
    __syncthreads();
    for (int b = threadIdx.x; b < nbox; b += kBinThreads)
        if (s_cnt[b]) s_cnt[b] = atomicAdd(&cursor[b], s_cnt[b]);  // this block's first slot in box b
    __syncthreads();
    for (int64_t i = i0 + threadIdx.x; i < i1; i += kBinThreads)
        perm[atomicAdd(&s_cnt[fgt_grid_box(__ldg(y + 2 * i), __ldg(y + 2 * i + 1), g)], 1)] = (int)i;
}

static int bin_grid(int64_t n)
{
    int sms = 0;
    if (device_sm_count(&sms) || sms <= 0) sms = 148;
    const int64_t want = (n + kBinThreads - 1) / kBinThreads;
    return (int)(want < 8LL * sms ? (want > 0 ? want : 1) : 8LL * sms);
}

// ---------------------------------------------------------------------------
// P2H from binned sources (Eq. A_alpha): a CTA takes 256 consecutive binned
// points, forms q t1^a1 / a1! and t2^a2 / a2! for each in shared memory, and
// thread (a1, a2) sums their products over each run of points of one box,
// adding the run's sum to A with one atomic per coefficient.
// ---------------------------------------------------------------------------
constexpr int kP2hPoints = 256;

template <int P>
__global__ void __launch_bounds__(kP2hPoints) fgt_p2h_binned_kernel(int g, double inv_c, float dcell,
                                                                    const double* __restrict__ x,
                                                                    const double* __restrict__ q, int n,
                                                                    const int* __restrict__ perm,
                                                                    float* __restrict__ A, int* err)
{
    __shared__ float s_w1[kP2hPoints][P + 1];
    __shared__ float s_w2[kP2hPoints][P + 1];
    __shared__ int s_box[kP2hPoints];
    const int tid = threadIdx.x;
    const int base = blockIdx.x * kP2hPoints;
    const int cnt = min(kP2hPoints, n - base);
    if (tid < cnt) {
        const int j = perm[base + tid];
        if ((unsigned)j < (unsigned)n) {
            const double x0 = x[2 * (size_t)j], x1 = x[2 * (size_t)j + 1];
            const int side = 1 << g;
            int b;
            float t1, t2;
            long long X0, X1;
            if (grid_fixed31(x0, g, X0) && grid_fixed31(x1, g, X1)) {
                // offsets from the box centre in box sides, times side / (sqrt2 sigma)
                b = (int)(X1 >> 31) * side + (int)(X0 >> 31);
                t1 = cell_offset31(X0) * dcell;
                t2 = cell_offset31(X1) * dcell;
            } else {  // outside the unit square: clamped box, offset in FP64
                b = fgt_grid_box(x0, x1, g);
                t1 = (float)((x0 * side - ((b & (side - 1)) + 0.5)) / side * inv_c);
                t2 = (float)((x1 * side - ((b >> g) + 0.5)) / side * inv_c);
            }
            float w1 = (float)q[j], w2 = 1.f;
#pragma unroll
            for (int a = 0; a < P; ++a) {
                s_w1[tid][a] = w1;
                s_w2[tid][a] = w2;
                w1 = w1 * t1 * (1.f / (float)(a + 1));
                w2 = w2 * t2 * (1.f / (float)(a + 1));
            }
            s_box[tid] = b;
        } else {
            atomicOr(err, DEV_ERR_CHECK);
            s_box[tid] = -1;
        }
    }
    __syncthreads();
    if (tid >= P * P) return;
    const int a1 = tid / P, a2 = tid % P;
    float acc = 0.f;
    int cur = -1;
    for (int k = 0; k < cnt; ++k) {
        const int b = s_box[k];
        if (b != cur) {
            if (cur >= 0) atomicAdd(&A[(size_t)cur * P * P + tid], acc);
            acc = 0.f;
            cur = b;
        }
        if (b >= 0) acc = fmaf(s_w1[k][a1], s_w2[k][a2], acc);
    }
    if (cur >= 0) atomicAdd(&A[(size_t)cur * P * P + tid], acc);
}

// ---------------------------------------------------------------------------
// Hermite evaluation at binned targets
// ---------------------------------------------------------------------------
constexpr int kH2pThreads = 128;
constexpr int kH2pWarps = kH2pThreads / 32;
constexpr int kH2pMaxCut = 16;
constexpr int kH2pMaxBoxes = (2 * kH2pMaxCut + 1) * (2 * kH2pMaxCut + 1);
constexpr int kH2pBatch = 8;                  // source boxes per shared-memory stage
constexpr int kH2pStages = 3;                 // ring depth (two batches in flight)

template <int P>
struct H2pCfg {
    // 4 targets per thread: each broadcast 16-byte load of A feeds 16 FMAs; 64-thread CTAs at
    // p >= 12 keep a claim at 256 targets (a box's last claim is partly idle)
    static constexpr int R = 4;                        // targets per thread
    static constexpr int THREADS = P >= 12 ? 64 : 128;
    static constexpr int WARPS = THREADS / 32;
    static constexpr int CH = THREADS * R;             // targets per claim
    static constexpr int PP = P * P;
    static constexpr size_t smem = (size_t)kH2pStages * kH2pBatch * PP * sizeof(float);
};

struct H2pArgs {
    int g, ncut, n;
    double d;  // box side / (sqrt2 sigma)
    const float* A;
    const double* y;
    const int* perm;
    const int* box_start;
    const unsigned char* nz;  // per source box: any non-zero coefficient
    const int* claims;        // [nbox + 1] claim-index prefix over the boxes in `order`
    const int* order;         // [nbox] the boxes, heaviest neighbourhood first (h2p_order_*)
    float* G;
    int accumulate;
    int* cursor;  // [0] next claim index, [1] CTAs finished
    int* err;
};

// flag[b] = any coefficient of box b is non-zero (one warp per box)
__global__ void fgt_box_flags_kernel(const float* __restrict__ A, int nbox, int pp, unsigned char* __restrict__ flag)
{
    const int b = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (b >= nbox) return;
    bool nz = false;
    for (int i = lane; i < pp; i += 32) nz |= A[(size_t)b * pp + i] != 0.f;
    nz = __any_sync(0xffffffffu, nz);
    if (lane == 0) flag[b] = nz ? 1 : 0;
}

__device__ __forceinline__ void cp_async_16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }


// claims[0..nbox]: exclusive scan of ceil(targets of box b / ch), the table that maps a claim
// index to its box; a box_start that decreases counts as empty and is reported.
__global__ void __launch_bounds__(kScanThreads) h2p_claims_kernel(int nbox, const int* __restrict__ box_start, int ch,
                                                                  int* __restrict__ claims, int* err)
{
    block_exclusive_scan(
        nbox,
        [&](int i) {
            const int m = box_start[i + 1] - box_start[i];
            if (m < 0) atomicOr(err, DEV_ERR_CHECK);
            return m > 0 ? (m + ch - 1) / ch : 0;
        },
        [](int, int) {}, claims);
}

// ---------------------------------------------------------------------------
// Claim order.  A claim's work is its targets times the non-empty source boxes of
// its box's n_cut neighbourhood, and a claim is large (a few hundred microseconds
// of one CTA), so claims handed out in box order leave SMs idle at the end of the
// launch.  The boxes are counting-sorted by that count, heaviest first (longest
// processing time first), and the claim table runs over that order.  Only the order
// in which claims are taken changes: every target is still evaluated by one thread
// with the same arithmetic.
// ---------------------------------------------------------------------------
constexpr int kH2pKeys = kH2pMaxBoxes + 2;  // neighbourhood counts 0..kH2pMaxBoxes, and "no targets"

// rp[y][x] = nz[y][0] + ... + nz[y][x]: one warp per grid row, 32 columns per step
__global__ void h2p_row_prefix_kernel(const unsigned char* __restrict__ nz, int g, int* __restrict__ rp)
{
    const int side = 1 << g, lane = threadIdx.x & 31;
    const int y = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (y >= side) return;
    int carry = 0;
    for (int x0 = 0; x0 < side; x0 += 32) {
        const int x = x0 + lane;
        int v = x < side ? (int)(nz[(size_t)y * side + x] != 0) : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (x < side) rp[(size_t)y * side + x] = carry + v;
        carry += __shfl_sync(0xffffffffu, v, 31);
    }
}

// key[b] = kH2pMaxBoxes - (non-empty source boxes within n_cut of b), or kH2pKeys - 1 for a box
// without targets; hist[key] counts the boxes of each key
__global__ void h2p_order_keys_kernel(const int* __restrict__ rp, const int* __restrict__ box_start, int g, int ncut,
                                      int* __restrict__ key, int* __restrict__ hist)
{
    const int side = 1 << g, nbox = side * side;
    const int b = (int)(blockIdx.x * (size_t)blockDim.x + threadIdx.x);
    if (b >= nbox) return;
    int k = kH2pKeys - 1;
    if (box_start[b + 1] > box_start[b]) {
        const int tx = b & (side - 1), ty = b >> g;
        const int x0 = max(tx - ncut, 0), x1 = min(tx + ncut, side - 1);
        const int y0 = max(ty - ncut, 0), y1 = min(ty + ncut, side - 1);
        int w = 0;
        for (int yy = y0; yy <= y1; ++yy) {
            const int* r = rp + (size_t)yy * side;
            w += r[x1] - (x0 > 0 ? r[x0 - 1] : 0);
        }
        k = kH2pMaxBoxes - w;
    }
    key[b] = k;
    atomicAdd(hist + k, 1);
}

// the boxes in key order (within a key in no particular order): a counting sort's scatter
__global__ void h2p_order_scatter_kernel(const int* __restrict__ key, int nbox, int* __restrict__ cursor,
                                         int* __restrict__ order)
{
    const int b = (int)(blockIdx.x * (size_t)blockDim.x + threadIdx.x);
    if (b >= nbox) return;
    order[atomicAdd(cursor + key[b], 1)] = b;
}

// cursor[0..kH2pKeys]: exclusive scan of the key histogram, the scatter cursors (one CTA)
__global__ void __launch_bounds__(kScanThreads) h2p_order_scan_kernel(const int* __restrict__ hist,
                                                                      int* __restrict__ cursor)
{
    block_exclusive_scan(
        kH2pKeys, [&](int i) { return hist[i]; }, [](int, int) {}, cursor);
}

// claims[0..nbox]: exclusive scan over the boxes in `order` of ceil(targets / ch)
__global__ void __launch_bounds__(kScanThreads) h2p_claims_ordered_kernel(int nbox, const int* __restrict__ box_start,
                                                                          const int* __restrict__ order, int ch,
                                                                          int* __restrict__ claims, int* err)
{
    block_exclusive_scan(
        nbox,
        [&](int i) {
            const int b = order[i];
            const int m = box_start[b + 1] - box_start[b];
            if (m < 0) atomicOr(err, DEV_ERR_CHECK);
            return m > 0 ? (m + ch - 1) / ch : 0;
        },
        [](int, int) {}, claims);
}

// The same for grids of up to kH2pOrderSmall boxes in one CTA (one launch instead of five):
// row prefix and key histogram in shared memory, then order and claims.
constexpr int kH2pOrderSmall = 4096;
constexpr int kH2pOrderPer = kH2pOrderSmall / kScanThreads;  // boxes per thread
__global__ void __launch_bounds__(kScanThreads) h2p_order_small_kernel(const unsigned char* __restrict__ nz,
                                                                       const int* __restrict__ box_start, int g,
                                                                       int ncut, int ch, int* __restrict__ order,
                                                                       int* __restrict__ claims, int* err)
{
    __shared__ int s_rp[kH2pOrderSmall];
    __shared__ int s_hist[kH2pKeys];
    __shared__ int s_cur[kH2pKeys + 1];
    const int tid = threadIdx.x, side = 1 << g, nbox = side * side;
    for (int b = tid; b < nbox; b += kScanThreads) s_rp[b] = nz[b] != 0;
    for (int k = tid; k < kH2pKeys; k += kScanThreads) s_hist[k] = 0;
    __syncthreads();
    if (tid < side) {
        int c = 0;
        for (int x = 0; x < side; ++x) s_rp[tid * side + x] = (c += s_rp[tid * side + x]);
    }
    __syncthreads();
    int key[kH2pOrderPer];
#pragma unroll
    for (int j = 0; j < kH2pOrderPer; ++j) {
        const int b = tid + j * kScanThreads;
        key[j] = -1;
        if (b >= nbox) continue;
        int k = kH2pKeys - 1;
        if (box_start[b + 1] > box_start[b]) {
            const int tx = b & (side - 1), ty = b >> g;
            const int x0 = max(tx - ncut, 0), x1 = min(tx + ncut, side - 1);
            const int y0 = max(ty - ncut, 0), y1 = min(ty + ncut, side - 1);
            int w = 0;
            for (int yy = y0; yy <= y1; ++yy) w += s_rp[yy * side + x1] - (x0 > 0 ? s_rp[yy * side + x0 - 1] : 0);
            k = kH2pMaxBoxes - w;
        }
        key[j] = k;
        atomicAdd(s_hist + k, 1);
    }
    __syncthreads();
    block_exclusive_scan(
        kH2pKeys, [&](int i) { return s_hist[i]; }, [](int, int) {}, s_cur);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kH2pOrderPer; ++j)
        if (key[j] >= 0) order[atomicAdd(s_cur + key[j], 1)] = tid + j * kScanThreads;
    __syncthreads();  // the order, written by this block, is visible to it
    block_exclusive_scan(
        nbox,
        [&](int i) {
            const int b = order[i];
            const int m = box_start[b + 1] - box_start[b];
            if (m < 0) atomicOr(err, DEV_ERR_CHECK);
            return m > 0 ? (m + ch - 1) / ch : 0;
        },
        [](int, int) {}, claims);
}

// Claim k = the next unclaimed index: run [first, end) of at most ch binned targets of one box
// (the claim table runs over the boxes in a.order).  Returns false when no claim is left.
__device__ bool h2p_claim(const H2pArgs& a, int nbox, int ch, int* first, int* end, int* box)
{
    const int total = __ldg(a.claims + nbox);
    const int k = atomicAdd(a.cursor, 1);
    if (k >= total) return false;
    h2p_claim_range_ordered(a.claims, a.order, a.box_start, nbox, a.n, ch, k, first, end, box);
    if (*first >= *end) atomicOr(a.err, DEV_ERR_CHECK);  // box_start does not bin [0, n)
    return true;
}

template <int P>
__global__ void __launch_bounds__(H2pCfg<P>::THREADS) fgt_h2p_kernel(H2pArgs a)
{
    using C = H2pCfg<P>;
    constexpr int R = C::R;
    constexpr int PP = C::PP;
    constexpr int NT = C::THREADS;
    extern __shared__ float4 h2p_smem[];
    float* sA = reinterpret_cast<float*>(h2p_smem);  // [kH2pStages][kH2pBatch][P][P]
    __shared__ float s_off[2 * kH2pMaxCut + 1];       // k d, k = -ncut .. ncut
    __shared__ short s_list[kH2pMaxBoxes];            // non-empty source boxes, row-major, as (dy + ncut) * 64 + dx + ncut
    __shared__ int s_warp_cnt[C::WARPS];
    __shared__ int s_claim[4];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int side = 1 << a.g, nbox = side * side;
    const int wmax = 2 * a.ncut + 1;
    if (tid < wmax) s_off[tid] = (float)((double)(tid - a.ncut) * a.d);

    for (;;) {
        if (tid == 0) {
            int f = 0, e = 0, b = 0;
            if (!h2p_claim(a, nbox, C::CH, &f, &e, &b)) f = e = -1;
            s_claim[0] = f;
            s_claim[1] = e;
            s_claim[2] = b;
        }
        __syncthreads();
        const int first = s_claim[0], end = s_claim[1], box = s_claim[2];
        if (first < 0) break;
        if (first >= end) {  // an inconsistent claim (reported); keep s_claim stable until all have read it
            __syncthreads();
            continue;
        }
        const int tx = box & (side - 1), ty = box >> a.g;
        const int x0 = max(tx - a.ncut, 0), x1 = min(tx + a.ncut, side - 1);
        const int y0 = max(ty - a.ncut, 0), y1 = min(ty + a.ncut, side - 1);
        const int w = x1 - x0 + 1, nb = w * (y1 - y0 + 1);

        // ordered compaction of the neighbourhood's non-empty source boxes (row-major)
        int total = 0;
        for (int base = 0; base < nb; base += NT) {
            const int i = base + tid;
            bool keep = false;
            int code = 0;
            if (i < nb) {
                const int sx = x0 + i % w, sy = y0 + i / w;
                keep = __ldg(a.nz + sy * side + sx) != 0;
                code = (sy - ty + a.ncut) * 64 + (sx - tx + a.ncut);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (lane == 0) s_warp_cnt[warp] = __popc(bal);
            __syncthreads();
            int off = total;
            for (int q = 0; q < warp; ++q) off += s_warp_cnt[q];
            if (keep) s_list[off + __popc(bal & ((1u << lane) - 1))] = (short)code;
            for (int q = 0; q < C::WARPS; ++q) total += s_warp_cnt[q];
            __syncthreads();
        }

        // this thread's targets and their offsets u within the box
        int tj[R];
        float u1[R], u2[R], acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int pos = first + warp * 32 * R + r * 32 + lane;  // a warp's 32 R targets
            tj[r] = -1;
            u1[r] = u2[r] = acc[r] = 0.f;
            if (pos < end) {
                const int j = __ldg(a.perm + pos);
                if ((unsigned)j < (unsigned)a.n) {
                    tj[r] = j;
                    u1[r] = (float)((__ldg(a.y + 2 * (size_t)j) * side - (tx + 0.5)) * a.d);
                    u2[r] = (float)((__ldg(a.y + 2 * (size_t)j + 1) * side - (ty + 0.5)) * a.d);
                } else {
                    atomicOr(a.err, DEV_ERR_CHECK);
                }
            }
        }
        const bool active = first + warp * 32 * R < end;  // warp-uniform

        const int nbatch = (total + kH2pBatch - 1) / kH2pBatch;
        auto stage = [&](int k) {
            if (k < nbatch) {
                float4* dst = reinterpret_cast<float4*>(sA + (size_t)(k % kH2pStages) * kH2pBatch * PP);
                const int cnt = min(kH2pBatch, total - k * kH2pBatch) * (PP / 4);
                for (int i = tid; i < cnt; i += NT) {
                    const int code = s_list[k * kH2pBatch + i / (PP / 4)];
                    const int sx = tx + (code & 63) - a.ncut, sy = ty + (code >> 6) - a.ncut;
                    cp_async_16(dst + i, reinterpret_cast<const float4*>(a.A + ((size_t)sy * side + sx) * PP) +
                                             i % (PP / 4));
                }
            }
            cp_async_commit();  // an empty group past the end keeps the wait counts uniform
        };
        stage(0);
        stage(1);
        int cur_dy = -1;
        float h2[R][P];
        for (int k = 0; k < nbatch; ++k) {
            cp_async_wait<1>();
            __syncthreads();  // batch k landed; everyone is done with batch k - 1's stage
            stage(k + 2);
            if (active) {
                const float* sb = sA + (size_t)(k % kH2pStages) * kH2pBatch * PP;
                const int nk = min(kH2pBatch, total - k * kH2pBatch);
#pragma unroll 1
                for (int e = 0; e < nk; ++e) {
                    const int code = s_list[k * kH2pBatch + e];
                    const int dy = code >> 6, dx = code & 63;  // source offset + ncut
                    if (dy != cur_dy) {
                        cur_dy = dy;
#pragma unroll
                        for (int r = 0; r < R; ++r) hermite_functions<P>(u2[r] + s_off[2 * a.ncut - dy], h2[r]);
                    }
                    // sum_a1 h_a1(t1) T[a1], T[a1] = sum_a2 A[a1][a2] h_a2(t2), by Clenshaw's backward
                    // recurrence for h_{a+1} = 2t h_a - 2a h_{a-1}:
                    //   c_a = T[a] + 2t c_{a+1} - 2(a+1) c_{a+2},  c_p = c_{p+1} = 0,  sum = h_0(t1) c_0,
                    // two multiply-adds per a1 beside the p of T[a1] (the forward recurrence and the
                    // accumulation take three)
                    float c1[R], c2[R], tt[R], e0[R];
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const float t = u1[r] + s_off[2 * a.ncut - dx];
                        tt[r] = t + t;
                        e0[r] = __expf(-t * t);
                        c1[r] = c2[r] = 0.f;
                    }
                    const float4* Ab = reinterpret_cast<const float4*>(sb + e * PP);
#pragma unroll
                    for (int a1 = P - 1; a1 >= 0; --a1) {
                        float t[R];
#pragma unroll
                        for (int r = 0; r < R; ++r) t[r] = fmaf(tt[r], c1[r], -(float)(2 * (a1 + 1)) * c2[r]);
#pragma unroll
                        for (int qd = 0; qd < P / 4; ++qd) {
                            const float4 v = Ab[a1 * (P / 4) + qd];
#pragma unroll
                            for (int r = 0; r < R; ++r) {
                                t[r] = fmaf(v.x, h2[r][4 * qd], t[r]);
                                t[r] = fmaf(v.y, h2[r][4 * qd + 1], t[r]);
                                t[r] = fmaf(v.z, h2[r][4 * qd + 2], t[r]);
                                t[r] = fmaf(v.w, h2[r][4 * qd + 3], t[r]);
                            }
                        }
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            c2[r] = c1[r];
                            c1[r] = t[r];
                        }
                    }
#pragma unroll
                    for (int r = 0; r < R; ++r) acc[r] = fmaf(e0[r], c1[r], acc[r]);
                }
            }
        }
        cp_async_wait<0>();
        __syncthreads();  // the ring and the list are free for the next claim
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (tj[r] >= 0) a.G[tj[r]] = a.accumulate ? a.G[tj[r]] + acc[r] : acc[r];
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

int launch_h2p_claims(int nbox, const int* box_start, int ch, int* claims, int* err, cudaStream_t st)
{
    h2p_claims_kernel<<<1, kScanThreads, 0, st>>>(nbox, box_start, ch, claims, err);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

// The claim order and the claim table over it, runs of ch targets: one CTA for grids of up to
// kH2pOrderSmall boxes, else row prefix, keys, histogram scan, scatter and claims as five
// launches.  nz: the source boxes' non-empty flags (already set); order points at the scratch
// words after the claims array.
static int h2p_order_claims(const unsigned char* nz, const int* box_start, int g, int ncut, int ch, int* order, int* claims,
                     int* err, cudaStream_t st)
{
    const int nbox = 1 << (2 * g), side = 1 << g;
    if (nbox <= kH2pOrderSmall) {
        h2p_order_small_kernel<<<1, kScanThreads, 0, st>>>(nz, box_start, g, ncut, ch, order, claims, err);
        FMM_CUDA_TRY(cudaGetLastError());
        return FMM_OK;
    }
    int* rp = order + nbox;               // [nbox] row prefix of the flags
    int* hist = rp + nbox;                // [kH2pKeys] key histogram
    int* cursor = hist + kH2pKeys;        // [kH2pKeys + 1] scatter cursors (their scan, total last)
    int* key = cursor + kH2pKeys + 1;     // [nbox]
    FMM_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(int) * kH2pKeys, st));
    h2p_row_prefix_kernel<<<(side * 32 + 255) / 256, 256, 0, st>>>(nz, g, rp);
    FMM_CUDA_TRY(cudaGetLastError());
    h2p_order_keys_kernel<<<(nbox + 255) / 256, 256, 0, st>>>(rp, box_start, g, ncut, key, hist);
    FMM_CUDA_TRY(cudaGetLastError());
    h2p_order_scan_kernel<<<1, kScanThreads, 0, st>>>(hist, cursor);
    FMM_CUDA_TRY(cudaGetLastError());
    h2p_order_scatter_kernel<<<(nbox + 255) / 256, 256, 0, st>>>(key, nbox, cursor, order);
    FMM_CUDA_TRY(cudaGetLastError());
    h2p_claims_ordered_kernel<<<1, kScanThreads, 0, st>>>(nbox, box_start, order, ch, claims, err);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

template <int P>
static int h2p_launch(const H2pArgs& args, cudaStream_t st)
{
    using C = H2pCfg<P>;
    static unsigned long long opted;
    static int occ;
    static std::mutex mu;
    if (int rc = smem_opt_in((const void*)fgt_h2p_kernel<P>, (int)C::smem, &opted)) return rc;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!occ) {
            FMM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fgt_h2p_kernel<P>, C::THREADS, C::smem));
            if (occ < 1) occ = 1;
        }
    }
    int sms = 0;
    if (int rc = device_sm_count(&sms)) return rc;
    const int nbox = 1 << (2 * args.g);
    fgt_box_flags_kernel<<<(nbox + 7) / 8, 256, 0, st>>>(args.A, nbox, C::PP, const_cast<unsigned char*>(args.nz));
    FMM_CUDA_TRY(cudaGetLastError());
    // the claim order (heaviest neighbourhood first), then the claim table over it
    if (int rc = h2p_order_claims(args.nz, args.box_start, args.g, args.ncut, C::CH, const_cast<int*>(args.order),
                                  const_cast<int*>(args.claims), args.err, st))
        return rc;
    const int64_t most = (int64_t)args.n / C::CH + nbox;  // claims can be no more
    const int grid = (int)std::min<int64_t>((int64_t)occ * sms, most > 0 ? most : 1);
    fgt_h2p_kernel<P><<<grid, C::THREADS, C::smem, st>>>(args);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

}  // namespace fmmgb

using namespace fmmgb;

extern "C" int fgt_bin_points(int32_t grid_log2, const double* y, int64_t n, int32_t* perm, int32_t* box_start,
                              int32_t* work, void* stream)
{
    clear_error();
    if (grid_log2 < 0 || grid_log2 > 10) return fail(FMM_EINVAL, "fgt_bin_points: grid_log2 %d outside 0..10", grid_log2);
    if (n < 0 || n > INT32_MAX) return fail(FMM_EINVAL, "fgt_bin_points: n = %lld outside 0..2^31-1", (long long)n);
    if (!box_start || !work || (n > 0 && (!y || !perm))) return fail(FMM_EINVAL, "fgt_bin_points: NULL pointer");
    if (((uintptr_t)y & 7) || ((uintptr_t)perm & 3) || ((uintptr_t)box_start & 3) || ((uintptr_t)work & 3))
        return fail(FMM_EINVAL, "fgt_bin_points: misaligned pointer (y 8 bytes, int32 arrays 4)");
    const int nbox = 1 << (2 * grid_log2);
    if ((const void*)work < (const void*)(box_start + nbox + 1) && (const void*)box_start < (const void*)(work + nbox))
        return fail(FMM_EINVAL, "fgt_bin_points: work overlaps box_start");
    cudaStream_t st = (cudaStream_t)stream;
    FMM_CUDA_TRY(cudaMemsetAsync(work, 0, sizeof(int) * (size_t)nbox, st));
    const bool smem = grid_log2 <= kBinSmemMaxLog2;
    const int smem_bytes = smem ? (int)sizeof(int) * nbox : 0;
    int grid = bin_grid(n);
    int64_t chunk = 0;
    if (smem && n > 0) {
        static unsigned long long opted[2];  // opted in once per device, for the largest such grid
        constexpr int kMaxBytes = (int)sizeof(int) << (2 * kBinSmemMaxLog2);
        if (int rc = smem_opt_in((const void*)bin_count_smem_kernel, kMaxBytes, &opted[0])) return rc;
        if (int rc = smem_opt_in((const void*)bin_scatter_smem_kernel, kMaxBytes, &opted[1])) return rc;
        int sms = 0;
        if (device_sm_count(&sms) || sms <= 0) sms = 148;
        grid = (int)std::min<int64_t>(2LL * sms, (n + kBinThreads - 1) / kBinThreads);
        chunk = (n + grid - 1) / grid;
    }
    if (n > 0) {
        if (smem)
            bin_count_smem_kernel<<<grid, kBinThreads, smem_bytes, st>>>(grid_log2, y, n, chunk, work);
        else
            bin_count_kernel<<<grid, kBinThreads, 0, st>>>(grid_log2, y, n, work);
        FMM_CUDA_TRY(cudaGetLastError());
    }
    bin_scan_kernel<<<1, kScanThreads, 0, st>>>(nbox, work, box_start);
    FMM_CUDA_TRY(cudaGetLastError());
    if (n > 0) {
        if (smem)
            bin_scatter_smem_kernel<<<grid, kBinThreads, smem_bytes, st>>>(grid_log2, y, n, chunk, work, perm);
        else
            bin_scatter_kernel<<<grid, kBinThreads, 0, st>>>(grid_log2, y, n, work, perm);
        FMM_CUDA_TRY(cudaGetLastError());
    }
    return FMM_OK;
}

extern "C" int fmm_bin_points(int32_t level, const double* y, int64_t n, int32_t* perm, int32_t* box_start,
                              int32_t* work, void* stream)
{
    // the boxes of quadtree level l are the cells of the 2^l x 2^l grid (reading R5)
    return fgt_bin_points(level, y, n, perm, box_start, work, stream);
}

extern "C" int fgt_p2h_binned(int32_t grid_log2, int32_t p, double sigma, const double* x, const double* q, int64_t n,
                              const int32_t* perm, float* A, int32_t flags, void* stream)
{
    clear_error();
    if (grid_log2 < 0 || grid_log2 > 10) return fail(FMM_EINVAL, "fgt_p2h_binned: grid_log2 %d outside 0..10", grid_log2);
    if (!fgt_supported(p)) return fail(FMM_EINVAL, "fgt_p2h_binned: unsupported p = %d (4, 8, 12, 16)", p);
    if (!(sigma > 0.0) || !(sigma < 1e300)) return fail(FMM_EINVAL, "fgt_p2h_binned: sigma must be positive and finite");
    if (n < 0 || n > INT32_MAX) return fail(FMM_EINVAL, "fgt_p2h_binned: n = %lld outside 0..2^31-1", (long long)n);
    if (!A || (n > 0 && (!x || !q || !perm))) return fail(FMM_EINVAL, "fgt_p2h_binned: NULL pointer");
    if (((uintptr_t)x & 7) || ((uintptr_t)q & 7) || ((uintptr_t)perm & 3) || ((uintptr_t)A & 3))
        return fail(FMM_EINVAL, "fgt_p2h_binned: misaligned pointer");
    if (flags & ~FMM_ACCUMULATE) return fail(FMM_EINVAL, "fgt_p2h_binned: unknown flags 0x%x", flags);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = ((size_t)1 << (2 * grid_log2)) * (size_t)p * p * sizeof(float);
    if (!(flags & FMM_ACCUMULATE)) FMM_CUDA_TRY(cudaMemsetAsync(A, 0, bytes, st));
    if (n == 0) return FMM_OK;
    int* err = nullptr;
    if (int rc = device_error_word(&err)) return rc;
    const unsigned grid = (unsigned)((n + kP2hPoints - 1) / kP2hPoints);
    const double inv_c = 1.0 / (sqrt(2.0) * sigma);
    const float dcell = (float)(ldexp(1.0, -grid_log2) * inv_c);  // box side / (sqrt2 sigma)
    const int nn = (int)n;
    switch (p) {
        case 4: fgt_p2h_binned_kernel<4><<<grid, kP2hPoints, 0, st>>>(grid_log2, inv_c, dcell, x, q, nn, perm, A, err); break;
        case 8: fgt_p2h_binned_kernel<8><<<grid, kP2hPoints, 0, st>>>(grid_log2, inv_c, dcell, x, q, nn, perm, A, err); break;
        case 12: fgt_p2h_binned_kernel<12><<<grid, kP2hPoints, 0, st>>>(grid_log2, inv_c, dcell, x, q, nn, perm, A, err); break;
        default: fgt_p2h_binned_kernel<16><<<grid, kP2hPoints, 0, st>>>(grid_log2, inv_c, dcell, x, q, nn, perm, A, err); break;
    }
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

extern "C" int fgt_h2p(int32_t grid_log2, int32_t n_cut, int32_t p, int32_t prec, double sigma, const float* A,
                       const double* y, int64_t n, const int32_t* perm, const int32_t* box_start, float* G,
                       int32_t flags, void* stream)
{
    clear_error();
    if (prec == FMM_TC_TF32X3) return fail(FMM_EUNSUPPORTED, "fgt_h2p: FMM_TC_TF32X3 is an M2L precision");
    if (prec != FMM_FP32 && prec != FMM_TC_BF16X3 && prec != FMM_TC_BF16)
        return fail(FMM_EINVAL, "fgt_h2p: unknown precision %d", prec);
    if (prec != FMM_FP32 && p != 16)
        return fail(FMM_EUNSUPPORTED, "fgt_h2p: the tensor-core forms take p = 16 (got %d)", p);
    if (prec != FMM_FP32 && n_cut > 15)
        return fail(FMM_EUNSUPPORTED, "fgt_h2p: the tensor-core forms take n_cut <= 15 (got %d)", n_cut);
    if (grid_log2 < 0 || grid_log2 > 10) return fail(FMM_EINVAL, "fgt_h2p: grid_log2 %d outside 0..10", grid_log2);
    if (n_cut < 0 || n_cut > kH2pMaxCut) return fail(FMM_EINVAL, "fgt_h2p: n_cut %d outside 0..%d", n_cut, kH2pMaxCut);
    if (!fgt_supported(p)) return fail(FMM_EINVAL, "fgt_h2p: unsupported p = %d (4, 8, 12, 16)", p);
    if (!(sigma > 0.0) || !(sigma < 1e300)) return fail(FMM_EINVAL, "fgt_h2p: sigma must be positive and finite");
    if (n < 0 || n > INT32_MAX) return fail(FMM_EINVAL, "fgt_h2p: n = %lld outside 0..2^31-1", (long long)n);
    if (!A || !box_start || (n > 0 && (!y || !perm || !G))) return fail(FMM_EINVAL, "fgt_h2p: NULL pointer");
    if (((uintptr_t)A & 15) || ((uintptr_t)y & 7) || ((uintptr_t)perm & 3) || ((uintptr_t)box_start & 3) ||
        ((uintptr_t)G & 3))
        return fail(FMM_EINVAL, "fgt_h2p: misaligned pointer (A 16 bytes, y 8, the rest 4)");
    if (flags & ~FMM_ACCUMULATE) return fail(FMM_EINVAL, "fgt_h2p: unknown flags 0x%x", flags);
    if (n == 0) return FMM_OK;
    H2pArgs args;
    args.g = grid_log2;
    args.ncut = n_cut;
    args.n = (int)n;
    args.d = ldexp(1.0, -grid_log2) / (sqrt(2.0) * sigma);
    args.A = A;
    args.y = y;
    args.perm = perm;
    args.box_start = box_start;
    args.G = G;
    args.accumulate = (flags & FMM_ACCUMULATE) ? 1 : 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = tile_counter(&args.cursor, st)) return rc;
    if (int rc = device_error_word(&args.err)) return rc;
    unsigned char* nzbuf = nullptr;
    if (int rc = fgt_flag_buffer(&nzbuf)) return rc;
    args.nz = nzbuf;
    args.claims = reinterpret_cast<const int*>(nzbuf + kFgtFlagBytes);
    args.order = args.claims + ((size_t)1 << 20) + 1;
    if (prec != FMM_FP32) {
        const int nbox = 1 << (2 * grid_log2);
        if (int rc = launch_h2p_claims(nbox, box_start, 128, const_cast<int*>(args.claims), args.err, st)) return rc;
        return launch_fgt_h2p_tc(grid_log2, n_cut, args.d, prec == FMM_TC_BF16X3, A, y, args.n, perm, box_start,
                                 args.claims, G, args.accumulate != 0, args.err, st);
    }
    switch (p) {
        case 4: return h2p_launch<4>(args, st);
        case 8: return h2p_launch<8>(args, st);
        case 12: return h2p_launch<12>(args, st);
        default: return h2p_launch<16>(args, st);
    }
}
