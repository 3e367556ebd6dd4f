// fgt_hermite_tc.cu -- FGT Hermite evaluation (Sec. 4.2, Eq. hermite) on the
// 5th-generation tensor cores (tcgen05, TMEM accumulator), p = 16.
//
// Recasting.  For the targets y_m of one box T and the source boxes of its
// n_cut neighbourhood (columns sx = x0..x1, rows sy = y0..y1),
//
//   G(y_m) = sum_{sx, a1} hx[m][sx, a1] D[m][sx, a1],
//   D[m][sx, a1] = sum_{sy, a2} hy[m][sy, a2] A_{sx,sy}[a1][a2],
//
// hx[m][sx, a1] = h_a1((y_m1 - c_sx)/(sqrt2 sigma)), hy[m][sy, a2] = h_a2((y_m2 - c_sy)/(sqrt2 sigma)).
// D is a dense product [targets x (rows p)] x [(rows p) x (columns p)]:
//   M = 128 targets of one box (one claim of the binned targets),
//   N = w p (source column, a1) pairs -- w p <= 496 FP32 columns of TMEM,
//       issued as MMAs of up to 16 boxes (256 columns),
//   K = 16 (a2) per source row; the rows stream through a shared-memory ring.
// The B operand of a row (the row's w boxes, 512 bytes each per precision
// plane) is one contiguous bulk copy per plane from a BF16 image of A that a
// pre-pass lays out in the MMA's canonical K-major layout.  The A operand
// (hy of the 128 targets for that row) is generated in shared memory by four
// warps, one target per thread.  The epilogue forms hx per source column and
// reduces each TMEM row against it: one dot product of w p per target.
//
// Precision: BF16 keeps 8 significant bits.  With x = hi + lo (both BF16) the
// three products hy_hi B_hi + hy_lo B_hi + hy_hi B_lo recover ~16 bits per
// product, accumulated in FP32 (FMM_TC_BF16X3); FMM_TC_BF16 issues hy_hi B_hi only.
//
// Roles (23 warps, one CTA per SM): warp 0 lane 0 issues the B copies; warp 1
// owns TMEM; lane 0 of warps 1 and 2 issue the MMAs for the first and second
// half of the source columns (TMEM columns from 0 and from 256), so that one
// issuer's wait for a stage overlaps the other's MMAs; warps 3-6 generate hy;
// warps 7-22 drain the accumulator in four groups of four (one warp per TMEM
// lane quarter, warp % 4), each group over a quarter of the source columns,
// groups 1-3 handing their partial sums to group 0 through shared memory.  A ring stage holds two source rows (K = 32),
// one mbarrier completes when its copies have landed and its hy is written:
// each wait of the MMA thread costs several hundred cycles even when the
// phase has long completed, so a stage carries twice the MMAs of one row.
// The ring has as many stages as shared memory holds (3 at n_cut = 10).
// Tiles (claims) go to CTAs round-robin.  Every wait is bounded: on timeout the CTA records
// FMM_ETIMEOUT in the device error word, waits (bounded) for its own copies,
// frees its TMEM and returns.
#include <cuda_bf16.h>

#include <mutex>

#include "fgt_hermite.cuh"
#include "tc_ptx.cuh"

namespace fmmgb {

constexpr int kTcP = 16;
constexpr int kTcRows = 128;                   // targets per tile (= claim size)
constexpr int kTcMaxStages = 8;                // ring depth: as many stages as shared memory holds, up to 8
constexpr int kTcMmaWarp = 1, kTcMma2Warp = 2, kTcHyWarp0 = 3, kTcEpiWarp0 = 7;
constexpr int kTcEpiGroups = 4, kTcEpiWarps = 4 * kTcEpiGroups;  // four warps (one per TMEM lane quarter) per group
constexpr int kTcThreads = 32 * (kTcEpiWarp0 + kTcEpiWarps);
constexpr int kTcBoxBytes = 512;               // one box, one plane: 16 x 16 BF16, canonical K-major
constexpr int kTcHyBytes = kTcRows * 32;       // one hy plane: 128 rows x 16 BF16
constexpr int kTcMaxCut = 15;                  // (2 n_cut + 1) p <= 512 TMEM columns
constexpr int kTcMinSmem = 120 * 1024;         // keeps one CTA per SM (the CTA allocates all of TMEM)
constexpr int kTcSmemCap = 227 * 1024;         // opt-in shared memory per CTA
constexpr int kTcRps = 2;                      // source rows per ring stage (K = 32 per stage)

__host__ __device__ constexpr int tc_stage_bytes(int ncut) { return kTcRps * (2 * (2 * ncut + 1) * kTcBoxBytes + 2 * kTcHyBytes); }
__host__ __device__ constexpr int tc_bar_bytes() { return 4096; }

struct H2pTcArgs {
    int g, ncut, n, split, accumulate, stages, max_claims;
    double d;  // box side / (sqrt2 sigma)
    const double* y;
    const int* perm;
    const int* box_start;
    const int* claims;
    const int4* tiles;         // per claim: first, end, box (h2p_tiles_kernel)
    const unsigned char* img;  // [2][nbox][512]: hi plane, then lo plane
    float* G;
    int* err;
};

// A (FP32 [nbox][16][16]) -> BF16 hi and lo planes, each box 512 bytes in the
// canonical no-swizzle K-major layout of 8-row x 16-byte core matrices:
//   offset(a1, a2) = (a1 / 8) 256 + (a2 / 8) 128 + (a1 % 8) 16 + (a2 % 8) 2
// (rows a1 form N, columns a2 form K), so the boxes of a grid row are
// consecutive N rows of the MMA's B operand.
__global__ void fgt_tc_image_kernel(const float* __restrict__ A, int nbox, unsigned char* __restrict__ img)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nbox * 256) return;
    const int64_t b = i >> 8;
    const int a1 = (int)(i >> 4) & 15, a2 = (int)i & 15;
    const float v = A[i];
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    const size_t off = (size_t)b * kTcBoxBytes + (a1 >> 3) * 256 + (a2 >> 3) * 128 + (a1 & 7) * 16 + (a2 & 7) * 2;
    *reinterpret_cast<__nv_bfloat16*>(img + off) = hi;
    *reinterpret_cast<__nv_bfloat16*>(img + (size_t)nbox * kTcBoxBytes + off) = lo;
}

// per claim k < claims[nbox]: its run of targets and its box, so that each role
// reads one 16-byte entry per tile instead of searching the claim table
__global__ void h2p_tiles_kernel(const int* __restrict__ claims, const int* __restrict__ box_start, int nbox, int n,
                                 int max_claims, int4* __restrict__ tiles)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= max_claims || k >= __ldg(claims + nbox)) return;
    int f, e, b;
    h2p_claim_range(claims, box_start, nbox, n, kTcRows, k, &f, &e, &b);
    tiles[k] = make_int4(f, e, b, 0);
}

struct TcH2pTile {
    int first, end, tx, ty, x0, x1, y0, y1;
};

__device__ __forceinline__ TcH2pTile tc_h2p_tile(const H2pTcArgs& a, int4 ti)
{
    const int side = 1 << a.g;
    TcH2pTile t;
    t.first = ti.x;
    t.end = ti.y;
    const int box = ti.z;
    t.tx = box & (side - 1);
    t.ty = box >> a.g;
    t.x0 = max(t.tx - a.ncut, 0);
    t.x1 = min(t.tx + a.ncut, side - 1);
    t.y0 = max(t.ty - a.ncut, 0);
    t.y1 = min(t.ty + a.ncut, side - 1);
    return t;
}

// one lane waits, the warp follows its outcome (all lanes leave together); the
// __syncwarp orders the other lanes' later accesses after lane 0's acquire
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, int lane, uint32_t sleep_ns = 128)
{
    int ok = 0;
    if (lane == 0) ok = mbar_wait(bar, parity, sleep_ns) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok != 0;
}

__global__ void __launch_bounds__(kTcThreads, 1) fgt_h2p_tc_kernel(H2pTcArgs a)
{
    extern __shared__ __align__(1024) unsigned char tsm[];
    const int wmax = 2 * a.ncut + 1;
    const int stage_bytes = tc_stage_bytes(a.ncut);
    const int brow = wmax * kTcBoxBytes;   // one source row of one precision plane
    const int bplane = kTcRps * brow;      // a stage's rows of one plane
    const int hyoff = 2 * bplane;          // hy planes: [hi: kTcRps rows][lo: kTcRps rows] x kTcHyBytes
    const int S = a.stages;
    unsigned char* bars = tsm + (size_t)S * stage_bytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(bars);   // B copies landed (tx) and hy written (4 warps)
    uint64_t* sempty = full + kTcMaxStages;               // stage read by the MMAs (commit)
    uint64_t* dfull = sempty + kTcMaxStages;              // [2] accumulator half e holds a tile (issuer e's commit)
    uint64_t* dempty = dfull + 2;                         // [2] accumulator half e drained (16 warps)
    uint64_t* pfull = dempty + 2;                         // partial sums of groups 1.. written (12 warps)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(pfull + 1);
    float* s_off = reinterpret_cast<float*>(tmem_slot + 4);  // k d, k = -ncut .. ncut
    float* s_part = s_off + 2 * kTcMaxCut + 3;               // [groups - 1][128] partial sums

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int side = 1 << a.g, nbox = side * side;
    const int total = min(__ldg(a.claims + nbox), a.max_claims);  // tiles[] holds max_claims entries

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1 + 4);
            mbar_init(&sempty[s], 2);  // one commit per MMA issuer
        }
        for (int e = 0; e < 2; ++e) {
            mbar_init(&dfull[e], 1);
            mbar_init(&dempty[e], kTcEpiWarps);
        }
        mbar_init(pfull, kTcEpiWarps - 4);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < wmax) s_off[tid] = (float)((double)(tid - a.ncut) * a.d);
    if (warp == kTcMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- B producer ----------------
        if (lane == 0) {
            int gs = 0;
            bool ok = true;
            for (int k = blockIdx.x; k < total && ok; k += gridDim.x) {
                const TcH2pTile t = tc_h2p_tile(a, __ldg(a.tiles + k));
                const uint32_t bytes = (uint32_t)(t.x1 - t.x0 + 1) * kTcBoxBytes;
                for (int r0 = t.y0; r0 <= t.y1; r0 += kTcRps, ++gs) {
                    const int s = gs % S, nr = min(kTcRps, t.y1 - r0 + 1);
                    if (gs >= S && !mbar_wait(&sempty[s], (uint32_t)(((gs / S) - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    unsigned char* st = tsm + (size_t)s * stage_bytes;
                    mbar_expect_tx(&full[s], 2 * nr * bytes);
                    for (int j = 0; j < nr; ++j) {
                        const size_t src = ((size_t)(r0 + j) * side + t.x0) * kTcBoxBytes;
                        bulk_load(st + j * brow, a.img + src, bytes, &full[s]);
                        bulk_load(st + bplane + j * brow, a.img + (size_t)nbox * kTcBoxBytes + src, bytes, &full[s]);
                    }
                }
            }
            if (!ok) atomicOr(a.err, DEV_ERR_TIMEOUT);
            // do not leave while copies are in flight: the last min(gs, stages) fills must have landed
            for (int q = (gs > S ? gs - S : 0); q < gs; ++q)
                if (!mbar_wait(&full[q % S], (uint32_t)((q / S) & 1))) atomicOr(a.err, DEV_ERR_TIMEOUT);
        }
    } else if (warp == kTcMmaWarp || warp == kTcMma2Warp) {
        // ---------------- MMA issuers: warp 1 the first ceil(w/2) source columns
        // (TMEM columns from 0), warp 2 the rest (TMEM columns from 256); each
        // one's wait for a stage overlaps the other's MMAs ----------------
        const int hsel = warp - kTcMmaWarp;
        if (lane == 0) {
            int gs = 0, i = 0;
            bool ok = true;
            int4 next = (int)blockIdx.x < total ? __ldg(a.tiles + blockIdx.x) : make_int4(0, 0, 0, 0);
            for (int k = blockIdx.x; k < total && ok; k += gridDim.x, ++i) {
                const TcH2pTile t = tc_h2p_tile(a, next);
                if (k + (int)gridDim.x < total) next = __ldg(a.tiles + k + gridDim.x);  // in flight during this tile
                const int w = t.x1 - t.x0 + 1;
                if (i > 0 && !mbar_spin(&dempty[hsel], (uint32_t)((i - 1) & 1))) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                for (int r0 = t.y0; r0 <= t.y1; r0 += kTcRps, ++gs) {
                    const int s = gs % S, nr = min(kTcRps, t.y1 - r0 + 1);
                    if (!mbar_spin(&full[s], (uint32_t)((gs / S) & 1))) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t st = su32(tsm + (size_t)s * stage_bytes);
                    const int c0 = (w + 1) >> 1;  // boxes of the first half
                    const int nb = hsel ? w - c0 : c0;
                    if (nb > 0) {
                        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(nb * 16 >> 3) << 17) |
                                               ((uint32_t)(kTcRows >> 4) << 24);
                        const uint32_t d = tmem + (uint32_t)(256 * hsel);
                        for (int j = 0; j < nr; ++j) {
                            const uint32_t boff = (uint32_t)(j * brow + hsel * c0 * kTcBoxBytes);
                            const uint64_t bhi = umma_desc(st + boff, 128, 256);
                            const uint64_t blo = umma_desc(st + bplane + boff, 128, 256);
                            const uint64_t ahi = umma_desc(st + hyoff + j * kTcHyBytes, 128, 256);
                            const uint64_t alo = umma_desc(st + hyoff + (kTcRps + j) * kTcHyBytes, 128, 256);
                            const uint32_t acc0 = (r0 > t.y0 || j > 0) ? 1u : 0u;
                            umma_bf16(d, ahi, bhi, idesc, acc0);
                            if (a.split) {
                                umma_bf16(d, alo, bhi, idesc, 1u);
                                umma_bf16(d, ahi, blo, idesc, 1u);
                            }
                        }
                    }
                    umma_commit(&sempty[s]);  // the stage is free once these MMAs have read it
                }
                if (!ok) break;
                umma_commit(&dfull[hsel]);  // this half of the accumulator holds tile k
            }
            if (!ok) atomicOr(a.err, DEV_ERR_TIMEOUT);
        }
    } else if (warp < kTcEpiWarp0) {
        // ---------------- hy generators: one target row per thread ----------------
        const int m = tid - 32 * kTcHyWarp0;
        int gs = 0;
        bool ok = true;
        for (int k = blockIdx.x; k < total && ok; k += gridDim.x) {
            const TcH2pTile t = tc_h2p_tile(a, __ldg(a.tiles + k));
            const bool valid = m < t.end - t.first;
            float u2 = 0.f;
            if (valid) {
                const int j = __ldg(a.perm + t.first + m);
                if ((unsigned)j < (unsigned)a.n)
                    u2 = (float)((__ldg(a.y + 2 * (size_t)j + 1) * side - (t.ty + 0.5)) * a.d);
            }
            for (int r0 = t.y0; r0 <= t.y1; r0 += kTcRps, ++gs) {
                const int s = gs % S, nr = min(kTcRps, t.y1 - r0 + 1);
                if (gs >= S && !warp_wait(&sempty[s], (uint32_t)(((gs / S) - 1) & 1), lane)) {
                    ok = false;
                    break;
                }
                for (int j = 0; j < nr; ++j) {
                    float h[kTcP];
                    if (valid) {
                        hermite_functions<kTcP>(u2 + s_off[t.ty - (r0 + j) + a.ncut], h);
                    } else {
#pragma unroll
                        for (int q = 0; q < kTcP; ++q) h[q] = 0.f;
                    }
                    uint32_t hi[8], lo[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const __nv_bfloat162 hv = __floats2bfloat162_rn(h[2 * q], h[2 * q + 1]);
                        const float2 hf = __bfloat1622float2(hv);
                        hi[q] = *reinterpret_cast<const uint32_t*>(&hv);
                        lo[q] = pack_bf16(h[2 * q] - hf.x, h[2 * q + 1] - hf.y);
                    }
                    unsigned char* hy =
                        tsm + (size_t)s * stage_bytes + hyoff + j * kTcHyBytes + (m >> 3) * 256 + (m & 7) * 16;
                    unsigned char* hyl = hy + kTcRps * kTcHyBytes;
                    *reinterpret_cast<uint4*>(hy) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                    *reinterpret_cast<uint4*>(hy + 128) = make_uint4(hi[4], hi[5], hi[6], hi[7]);
                    *reinterpret_cast<uint4*>(hyl) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                    *reinterpret_cast<uint4*>(hyl + 128) = make_uint4(lo[4], lo[5], lo[6], lo[7]);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor cores
                __syncwarp();
                if (lane == 0) mbar_arrive(&full[s]);
            }
        }
        if (!ok && lane == 0) atomicOr(a.err, DEV_ERR_TIMEOUT);
    } else {
        // ---------------- epilogue: TMEM row m against hx, group e over a quarter of the columns ----------------
        const int q4 = warp & 3;  // TMEM lane quarter
        const int grp = (warp - kTcEpiWarp0) >> 2;
        const int m = q4 * 32 + lane;
        const uint32_t lanes = (uint32_t)(q4 * 32) << 16;
        int i = 0;
        for (int k = blockIdx.x; k < total; k += gridDim.x, ++i) {
            const TcH2pTile t = tc_h2p_tile(a, __ldg(a.tiles + k));
            const int w = t.x1 - t.x0 + 1;
            const bool valid = m < t.end - t.first;
            int j = -1;
            float u1 = 0.f;
            if (valid) {
                j = __ldg(a.perm + t.first + m);
                if ((unsigned)j < (unsigned)a.n) {
                    u1 = (float)((__ldg(a.y + 2 * (size_t)j) * side - (t.tx + 0.5)) * a.d);
                } else {
                    atomicOr(a.err, DEV_ERR_CHECK);
                    j = -1;
                }
            }
            if (t.first >= t.end && grp == 0 && q4 == 0 && lane == 0) atomicOr(a.err, DEV_ERR_CHECK);  // box_start does not bin [0, n)
            // the first half of the columns, then the second: issuer 0 starts the next
            // tile as soon as the first half is drained
            float acc = 0.f;
            const int c0 = (w + 1) >> 1;  // source columns of the first half (TMEM columns from 0)
            bool ok = true;
#pragma unroll 1
            for (int e = 0; e < 2 && ok; ++e) {
                if (!warp_wait(&dfull[e], (uint32_t)(i & 1), lane, 32)) {
                    if (lane == 0) atomicOr(a.err, DEV_ERR_TIMEOUT);
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int cb = e ? c0 : 0, ce = e ? w : c0;      // this half's source columns
                const int qw = (ce - cb + kTcEpiGroups - 1) / kTcEpiGroups;
#pragma unroll 1
                for (int c = cb + grp * qw; c < min(ce, cb + (grp + 1) * qw); ++c) {
                    uint32_t v[16];
                    tmem_ld16_async(tmem + lanes + (uint32_t)(256 * e + 16 * (c - cb)), v);
                    float h[kTcP];
                    hermite_functions<kTcP>(u1 + s_off[t.tx - (t.x0 + c) + a.ncut], h);
                    tmem_wait_ld();
#pragma unroll
                    for (int q = 0; q < kTcP; ++q) acc = fmaf(h[q], __uint_as_float(v[q]), acc);
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                if (e == 0 || grp) {
                    if (e == 1) s_part[(grp - 1) * kTcRows + m] = acc;
                    __syncwarp();
                    if (lane == 0) {
                        if (e == 1) mbar_arrive(pfull);
                        mbar_arrive(&dempty[e]);
                    }
                }
            }
            if (!ok) break;
            if (grp) continue;
            // group 0: the other groups' partial sums of tile i, read before this warp's
            // arrival on the second half's dempty lets the next tile (and its s_part) proceed
            if (!warp_wait(pfull, (uint32_t)(i & 1), lane, 32)) {
                if (lane == 0) atomicOr(a.err, DEV_ERR_TIMEOUT);
                break;
            }
#pragma unroll
            for (int e = 1; e < kTcEpiGroups; ++e) acc += s_part[(e - 1) * kTcRows + m];
            __syncwarp();
            if (lane == 0) mbar_arrive(&dempty[1]);
            if (j >= 0) a.G[j] = a.accumulate ? a.G[j] + acc : acc;
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == kTcMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
}

// Per-device BF16 image of A (grown on demand).
static std::mutex g_img_mu;
static unsigned char* g_img[64];
static size_t g_img_bytes[64];

static int tc_image_buffer(size_t bytes, unsigned char** out)
{
    int dev = 0;
    FMM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(FMM_EUNSUPPORTED, "fgt_h2p: device ordinal %d above 63", dev);
    std::lock_guard<std::mutex> lk(g_img_mu);
    if (g_img_bytes[dev] < bytes) {
        if (g_img[dev]) {
            FMM_CUDA_TRY(cudaDeviceSynchronize());
            cudaFree(g_img[dev]);
            g_img[dev] = nullptr;
            g_img_bytes[dev] = 0;
        }
        FMM_CUDA_TRY(cudaMalloc(&g_img[dev], bytes));
        g_img_bytes[dev] = bytes;
    }
    *out = g_img[dev];
    return FMM_OK;
}

// Per-device tile table (grown on demand).
static unsigned char* g_tiles[64];
static size_t g_tiles_bytes[64];

static int tc_tile_buffer(size_t bytes, int4** out)
{
    int dev = 0;
    FMM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(FMM_EUNSUPPORTED, "fgt_h2p: device ordinal %d above 63", dev);
    std::lock_guard<std::mutex> lk(g_img_mu);
    if (g_tiles_bytes[dev] < bytes) {
        if (g_tiles[dev]) {
            FMM_CUDA_TRY(cudaDeviceSynchronize());
            cudaFree(g_tiles[dev]);
            g_tiles[dev] = nullptr;
            g_tiles_bytes[dev] = 0;
        }
        FMM_CUDA_TRY(cudaMalloc(&g_tiles[dev], bytes));
        g_tiles_bytes[dev] = bytes;
    }
    *out = reinterpret_cast<int4*>(g_tiles[dev]);
    return FMM_OK;
}

int launch_fgt_h2p_tc(int g, int ncut, double d, bool split, const float* A, const double* y, int n, const int* perm,
                      const int* box_start, const int* claims, float* G, bool accumulate, int* err, cudaStream_t st)
{
    if (ncut > kTcMaxCut) return fail(FMM_EUNSUPPORTED, "fgt_h2p: tensor-core form needs n_cut <= %d", kTcMaxCut);
    const int nbox = 1 << (2 * g);
    unsigned char* img = nullptr;
    if (int rc = tc_image_buffer((size_t)nbox * 2 * kTcBoxBytes, &img)) return rc;
    const int64_t elems = (int64_t)nbox * 256;
    fgt_tc_image_kernel<<<(unsigned)((elems + 255) / 256), 256, 0, st>>>(A, nbox, img);
    FMM_CUDA_TRY(cudaGetLastError());
    static unsigned long long opted;
    if (int rc = smem_opt_in((const void*)fgt_h2p_tc_kernel, kTcSmemCap, &opted)) return rc;
    // as many stages as fit, released in groups of 3 (2 when fewer than 6 fit, 4 when 8 fit)
    const int stages = std::min(kTcMaxStages, (kTcSmemCap - tc_bar_bytes()) / tc_stage_bytes(ncut));
    int smem = stages * tc_stage_bytes(ncut) + tc_bar_bytes();
    if (smem < kTcMinSmem) smem = kTcMinSmem;
    const int max_claims = (int)std::min<int64_t>((int64_t)n / kTcRows + nbox, INT32_MAX);
    int4* tiles = nullptr;
    if (int rc = tc_tile_buffer((size_t)max_claims * sizeof(int4), &tiles)) return rc;
    h2p_tiles_kernel<<<(max_claims + 255) / 256, 256, 0, st>>>(claims, box_start, nbox, n, max_claims, tiles);
    FMM_CUDA_TRY(cudaGetLastError());
    int sms = 0;
    if (int rc = device_sm_count(&sms)) return rc;
    H2pTcArgs args;
    args.g = g;
    args.ncut = ncut;
    args.n = n;
    args.split = split ? 1 : 0;
    args.accumulate = accumulate ? 1 : 0;
    args.stages = stages;
    args.d = d;
    args.y = y;
    args.perm = perm;
    args.box_start = box_start;
    args.claims = claims;
    args.tiles = tiles;
    args.max_claims = max_claims;
    args.img = img;
    args.G = G;
    args.err = err;
    fgt_h2p_tc_kernel<<<sms, kTcThreads, smem, st>>>(args);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

}  // namespace fmmgb
