// m2l_tc.cu -- M2L + reduction on the 5th-generation tensor cores (tcgen05,
// TMEM accumulators), BF16 inputs with an optional hi/lo split, FP32
// accumulation (Sec. 4.1 steps 2-3, Eq. M2Lmat recast as a dense contraction).
//
// Recasting.  In radius-scaled units the M2L operator of a list entry depends
// only on the box offset.  Group a level's boxes by parent: a target of child
// class c under parent P receives, for each parent offset e in the 3x3
// neighbourhood (e != 0: siblings are all adjacent) and each source child
// class c', the translation T(delta) with delta = 2e + c' - c, or nothing when
// delta is adjacent.  So for one parent P
//
//   out[c, n, re/im](P) = sum_{e, c'} W[(c,n,re/im)][(e,c'), (k,re/im)] in[c'](P + e)[k, re/im]
//
// -- a 3x3 convolution over the parent grid whose "channels" are the 4 child
// classes x 2p real coefficients.  With D[rows][parents] in TMEM:
//   M rows  = 4 classes x 2p       (128 at p = 16; 192 -> two M=128 tiles at p = 24)
//   N       = the 8 x TPY parents of a tile
//   K       = 32 blocks (e, c') x 2p, processed 16 at a time.
// A (the operator blocks) streams from an L2-resident image through a ring
// of shared-memory stages (cp.async.bulk, mbarrier transaction counts).  B
// (the source MEs) is the tile's halo, staged once: for block (e, c') the B
// operand is the class-c' plane seen through a descriptor whose start is
// shifted by e -- the 8 parents of one tile row are 8 consecutive 16-byte
// rows, and the stride to the next tile row is the halo row pitch (SBO).
//
// Precision.  BF16 keeps 8 significant bits.  With the hi/lo split
// x = hi + lo (both BF16), the three products A_hi B_hi + A_hi B_lo +
// A_lo B_hi recover ~16 bits per product, accumulated in FP32.
//
// Schedule.  A persistent CTA per SM takes tiles round-robin and runs four
// roles concurrently: producer warps (eight at p = 16, three at p = 24; one
// bulk copy in flight per warp, one ring stage each) stream the 32 operator
// blocks of every tile through a ring of shared-memory stages; an MMA thread
// (warp 8) issues the tcgen05 products into a TMEM accumulator; three staging
// warps (9-11) load the next tile's halo (TMA tensor-map copies of the BF16
// hi/lo planes that a pre-pass writes, or bulk copies where a level is too
// small for the tensor map); four epilogue warps (12-15) drain the
// accumulator.
// Hand-overs use mbarriers; every wait is bounded: on timeout the CTA records
// FMM_ETIMEOUT in the device error word, waits (bounded) for its own copies,
// frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace fmmgb {

constexpr int kTcTileX = 8;               // parents per tile row (one core-matrix group)

template <int P>
struct TcCfg {
    static constexpr int K2 = 2 * P;                  // real K per block
    static constexpr int KCH = K2 / 8;                // 16-byte BF16 chunks per block row
    static constexpr int KSTEP = K2 / 16;             // MMA K steps of 16 per block
    static constexpr int MT = (8 * P + 127) / 128;    // M tiles of 128 rows
    static constexpr int TPY = P <= 16 ? 16 : 8;      // parent rows per tile
    static constexpr int N = kTcTileX * TPY;          // parents per tile (the split MMA has N = 2 x this)
    static constexpr int HX = kTcTileX + 2, HY = TPY + 2;
    static constexpr int NPOS = HX * HY;              // halo parent positions
    // one (class, chunk) plane of a halo buffer: 2 HY rows (halo row, hi/lo interleaved) x HX x 16 B
    static constexpr int ROWB = HX * 16;
    static constexpr int IPLANE = 2 * HY * ROWB;
    static constexpr int BBUF = 4 * KCH * IPLANE;     // bytes of one halo buffer (hi and lo)
    static constexpr int APART = MT * 128 * K2 * 2;   // bytes of one block's hi (or lo) operator image
    static constexpr int NBUF = 1;                    // halo buffers
    // Producer warps, one ring stage each.  A stage is refilled only after the
    // MMAs that read it complete, so the operator stream is bound by the ring
    // depth over that round trip (completion, wake-up, one bulk-copy latency):
    // as many stages as shared memory holds (8 x 16 KB at p = 16, 3 x 48 KB at
    // p = 24, beside the halo buffer).
    static constexpr int NPROD = P <= 16 ? 8 : 3;
    static constexpr int SP = 1;                      // ring stages per producer
    static constexpr int STAGES = NPROD * SP;         // operator ring depth
    // Stages are released in groups of G by one tcgen05.commit: the arrival
    // of a commit on its mbarrier comes ~600 cycles after the previous one
    // (measured), so a commit per 16 KB block caps the stream below the
    // tensor pipe's rate at p = 16.  Blocks per CTA (32 per tile) are a
    // multiple of G.
    static constexpr int G = P <= 16 ? 2 : 1;
    static_assert(STAGES % G == 0 && 32 % G == 0, "stage groups");
    // TMEM: per M tile a 2N-column accumulator (A_hi x [B_hi|B_lo] interleaved) + an N-column one (A_lo x B_hi)
    static constexpr int SETCOLS = MT * 3 * N;
    static constexpr int NACC = 2 * SETCOLS <= 512 ? 2 : 1;
    static constexpr int TMEM_COLS = 512;
    static constexpr size_t smem = (size_t)NBUF * BBUF + (size_t)STAGES * 2 * APART + 1024;
};

constexpr int kTcBlocks = 32;   // (e != 0) x 4 source classes
constexpr int kTcReplicas = 4;  // copies of the operator image in global memory

// block index b = pe * 4 + c', pe = 0..7 enumerating the 8 non-central parent offsets
__host__ __device__ inline void tc_block(int b, int& ex, int& ey, int& cs)
{
    cs = b & 3;
    int pe = b >> 2;
    if (pe >= 4) ++pe;  // skip the centre (ex, ey) = (0, 0)
    ex = pe % 3 - 1;
    ey = pe / 3 - 1;
}

// ---------------------------------------------------------------------------
// operator image: W[(c, n, r_out)][(k, r_in)] per block, BF16 hi and lo, in
// the canonical K-major no-swizzle layout (8-row x 16-byte core matrices):
//   byte offset of (row R, real column q) = (R / 8) * (KCH * 128) + (q / 8) * 128 + (R % 8) * 16 + (q % 8) * 2
// built in FP64 on the GPU from a(D) = (-1)^n C(n+k,k) D^-(n+k+1).
// ---------------------------------------------------------------------------
template <int P>
__global__ void build_tc_image_kernel(double s, int variant, unsigned char* __restrict__ img)
{
    using C = TcCfg<P>;
    const int rows = C::MT * 128;
    const int64_t total = (int64_t)kTcBlocks * rows * C::K2;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int q = (int)(idx % C::K2);
    const int R = (int)((idx / C::K2) % rows);
    const int b = (int)(idx / ((int64_t)C::K2 * rows));
    double w = 0.0;
    if (R < 8 * P) {
        const int c = R / (2 * P), n = (R % (2 * P)) / 2, ro = R & 1;
        const int k = q / 2, ri = q & 1;
        int ex, ey, cs;
        tc_block(b, ex, ey, cs);
        const int dx = 2 * ex + (cs & 1) - (c & 1), dy = 2 * ey + (cs >> 1) - (c >> 1);
        const int adx = dx < 0 ? -dx : dx, ady = dy < 0 ? -dy : dy;
        if ((adx > ady ? adx : ady) >= 2) {
            // T[n][k] = a_n h_D[n+k] b_k with the balanced factors of the FP32 path, in FP64
            const double Dr = -(double)dx, Di = -(double)dy, den = Dr * Dr + Di * Di;
            const double ir = Dr / den, ii = -Di / den;
            double hr = ir, hi = ii;
            for (int i = 1; i <= n + k; ++i) {
                const double f = (double)i * s;
                const double nr = (hr * ir - hi * ii) * f;
                const double ni = (hr * ii + hi * ir) * f;
                hr = nr;
                hi = ni;
            }
            double fa = 1.0, fb = 1.0;
            for (int i = 1; i <= n; ++i) fa *= (double)i * s;
            for (int i = 1; i <= k; ++i) fb *= (double)i * s;
            const double scale = ((n & 1) ? -1.0 : 1.0) / (fa * fb);
            // variant 0: T (forward); 1: -T (plain adjoint); 2: -conj T (conjugate adjoint),
            // by a(D)^T = -a(-D) on the symmetric lists
            const double tr = (variant ? -hr : hr) * scale, ti = (variant == 1 ? -hi : hi) * scale;
            // out_re = Re T in_re - Im T in_im;  out_im = Im T in_re + Re T in_im
            w = ro == 0 ? (ri == 0 ? tr : -ti) : (ri == 0 ? ti : tr);
        }
    }
    const __nv_bfloat16 whi = __double2bfloat16(w);
    const __nv_bfloat16 wlo = __double2bfloat16(w - (double)__bfloat162float(whi));
    const size_t off = (size_t)(R / 8) * (C::KCH * 128) + (size_t)(q / 8) * 128 + (R % 8) * 16 + (q % 8) * 2;
    unsigned char* blk = img + (size_t)b * 2 * C::APART;
    *reinterpret_cast<__nv_bfloat16*>(blk + off) = whi;
    *reinterpret_cast<__nv_bfloat16*>(blk + C::APART + off) = wlo;
}

// tensor-map load (the other PTX helpers are in tc_ptx.cuh)
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(
            su32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(su32(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// pre-pass: every level's MEs -> BF16 hi/lo planes laid out so that a tile's
// halo is one TMA box that lands in exactly the shared-memory layout the MMAs
// read: [cc = class * KCH + chunk][parent row qy][part: hi, lo][parent column qx]
// x 16 bytes (a chunk = 8 consecutive real coefficients of a box)
// ---------------------------------------------------------------------------
template <int P>
__global__ void me_planes_kernel(M2LLaunch job, int split)
{
    // one thread per 16-byte unit of a plane row, consecutive threads along qx: the
    // stores are coalesced, each thread reads one 32-byte chunk of one box
    using C = TcCfg<P>;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int li = 0;
    for (; li < job.nlev; ++li) {
        const int64_t n = ((int64_t)1 << (2 * job.lv[li].level)) * C::KCH;
        if (idx < n) break;
        idx -= n;
    }
    if (li >= job.nlev) return;
    const M2LLevel& lv = job.lv[li];
    const int side = 1 << lv.level, np = side >> 1;
    const int qx = (int)(idx % np);
    const int64_t t = idx / np;
    const int qy = (int)(t % np), cc = (int)(t / np);  // cc = class * KCH + chunk
    const int c = cc / C::KCH, ch = cc % C::KCH;
    const int ix = 2 * qx + (c & 1), iy = 2 * qy + (c >> 1);
    const float4* src = reinterpret_cast<const float4*>(lv.M) + ((int64_t)iy * side + ix) * (P / 2) + 2 * ch;
    const float4 v0 = __ldg(src), v1 = __ldg(src + 1);
    const float f[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
    uint32_t h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        __nv_bfloat162 hv = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
        const float2 hf = __bfloat1622float2(hv);
        h[j] = *reinterpret_cast<uint32_t*>(&hv);
        l[j] = pack_bf16(f[2 * j] - hf.x, f[2 * j + 1] - hf.y);
    }
    const size_t row = (size_t)np * 16;  // one (cc, qy, part) row of np positions
    const size_t off = ((size_t)cc * np + qy) * 2 * row + (size_t)qx * 16;
    *reinterpret_cast<uint4*>(lv.planes + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(lv.planes + off + row) = make_uint4(l[0], l[1], l[2], l[3]);
    (void)split;
}


// ---------------------------------------------------------------------------
// the kernel: persistent, one CTA per SM, warp-specialised
//   warps 0-2, lane 0  producers: operator block g of the continuous stream
//                   (32 per tile) comes from producer g % 3 into that
//                   producer's share of the ring; each issuing thread keeps
//                   one bulk copy in flight, so three producers triple the rate
//   warp 4, lane 0  MMA issuer (warp 4 also owns the TMEM allocation)
//   warps 5-7       halo staging: one TMA tensor load of the tile's halo from
//                   the BF16 hi/lo planes written by me_planes_kernel (cp.async
//                   when the halo is larger than the level or lists are periodic)
//   warps 8-11      epilogue: TMEM -> registers -> coalesced LE stores; two
//                   TMEM accumulators so tile i's epilogue overlaps tile i+1's MMAs
// Tiles are handed out round-robin (tile = blockIdx.x + i * gridDim.x); all
// tiles cost the same.
// ---------------------------------------------------------------------------
// warps 0-7 producers (NPROD of them active), 8 MMA issuer, 9-11 halo staging,
// 12-15 epilogue (a multiple of 4, so that warp % 4 is its TMEM lane quarter)
constexpr int kTcCtaThreads = 512;
constexpr int kMmaWarp = 8, kStageWarp0 = 9, kStageWarps = 3, kEpiWarp0 = 12;

struct TcTile {
    const unsigned char* planes;
    float2* L;
    int side, np, PX0, PY0, li;
};

template <int P>
__device__ __forceinline__ TcTile tc_tile(const M2LLaunch& job, int tile)
{
    using C = TcCfg<P>;
    int li = 0;
    while (li + 1 < job.nlev && tile >= job.lv[li + 1].tile_begin) ++li;
    const M2LLevel& lv = job.lv[li];
    TcTile g;
    g.planes = lv.planes;
    g.L = lv.L;
    g.side = 1 << lv.level;
    g.np = g.side >> 1;
    const int t = tile - lv.tile_begin;
    const int tpr = (g.np + kTcTileX - 1) / kTcTileX;
    g.PX0 = (t % tpr) * kTcTileX;
    g.PY0 = (t / tpr) * C::TPY;
    g.li = li;
    return g;
}


struct TcMaps {
    CUtensorMap map[kMaxLaunchLevels];  // per launch level: 5-D map over its planes (when use_tma)
    int use_tma[kMaxLaunchLevels];
};

template <int P>
__global__ void __launch_bounds__(kTcCtaThreads, 1) m2l_tc_kernel(M2LLaunch job, const __grid_constant__ TcMaps maps,
                                                                   const unsigned char* __restrict__ img, int split,
                                                                   int total_tiles, int* __restrict__ err)
{
    using C = TcCfg<P>;
    extern __shared__ __align__(1024) unsigned char tsm[];
    unsigned char* bbuf = tsm;                                 // NBUF halo buffers
    unsigned char* astage = tsm + (size_t)C::NBUF * C::BBUF;   // STAGES x (hi APART, lo APART)
    uint64_t* afull = reinterpret_cast<uint64_t*>(astage + (size_t)C::STAGES * 2 * C::APART);
    uint64_t* aempty = afull + C::STAGES;
    uint64_t* bfull = aempty + C::STAGES;
    uint64_t* bfree = bfull + 2;
    uint64_t* dfull = bfree + 2;
    uint64_t* dfree = dfull + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(dfree + 2);
    uint32_t* boff16 = tmem_slot + 4;  // [32] B-operand offset of each (e, c') block, in 16-byte units

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = blockIdx.x < (unsigned)total_tiles ? (total_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const uint32_t abytes = split ? 2u * C::APART : (uint32_t)C::APART;
    // Every CTA walks the same operator blocks; starting at a CTA-dependent
    // block and reading one of kTcReplicas copies of the image spreads the
    // simultaneous reads of all SMs over many L2 lines.
    const int rot = (int)(blockIdx.x % kTcBlocks);
    const unsigned char* rimg = img + (size_t)(blockIdx.x % kTcReplicas) * kTcBlocks * 2 * C::APART;

    if (tid == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(&afull[s], 1);
            if (s % C::G == 0) mbar_init(&aempty[s / C::G], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bfull[i], 1);
            mbar_init(&bfree[i], 1);
            mbar_init(&dfull[i], 1);
            mbar_init(&dfree[i], 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < kTcBlocks) {
        int ex, ey, cs;
        tc_block(tid, ex, ey, cs);
        boff16[tid] = (uint32_t)((cs * C::KCH * C::IPLANE + 2 * (ey + 1) * C::ROWB + (ex + 1) * 16) >> 4);
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"((uint32_t)C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp < C::NPROD) {
        // ---------------- producer `warp` ----------------
        if (lane == 0) {
            const int pr = warp;
            const int total_blocks = ntiles * kTcBlocks;
            int k = 0;  // local fill index of this producer
            bool ok = true;
            for (int g = pr; g < total_blocks; g += C::NPROD, ++k) {
                const int s = pr * C::SP + k % C::SP;
                if (k >= C::SP && !mbar_wait(&aempty[s / C::G], (uint32_t)(((k / C::SP) - 1) & 1))) {
                    ok = false;
                    break;
                }
                const int b = (g % kTcBlocks + rot) % kTcBlocks;
                mbar_expect_tx(&afull[s], abytes);
                bulk_load(astage + (size_t)s * 2 * C::APART, rimg + (size_t)b * 2 * C::APART, abytes, &afull[s]);
            }
            if (!ok) atomicOr(err, DEV_ERR_TIMEOUT);
            // do not leave while copies are in flight: this producer's last min(k, SP) fills must have landed
            for (int q = (k > C::SP ? k - C::SP : 0); q < k; ++q)
                if (!mbar_wait(&afull[pr * C::SP + q % C::SP], (uint32_t)((q / C::SP) & 1))) atomicOr(err, DEV_ERR_TIMEOUT);
        }
    } else if (warp == kMmaWarp && lane == 0) {
        // ---------------- MMA issuer ----------------
        // per K step of 16: D1 (2N cols) += A_hi x [B_hi | B_lo] (rows interleaved, N = 2 x 64),
        //                   D2 (N cols)  += A_lo x B_hi; result = D1 hi cols + D1 lo cols + D2.
        // Without the split: D2 += A_hi x B_hi only.
        const uint32_t id2n = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((2 * C::N) >> 3) << 17) | ((128u >> 4) << 24);
        const uint32_t idn = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(C::N >> 3) << 17) | ((128u >> 4) << 24);
        const uint64_t a0 = umma_desc(su32(astage), 128, C::KCH * 128);  // stage 0, hi part
        constexpr uint64_t alo_off = (uint64_t)(C::APART >> 4);
        int g = 0;
        bool ok = true;
        for (int i = 0; i < ntiles && ok; ++i) {
            const int ts = i % C::NBUF, td = i % C::NACC;
            if (!mbar_spin(&bfull[ts], (uint32_t)((i / C::NBUF) & 1))) ok = false;
            if (ok && i >= C::NACC && !mbar_spin(&dfree[td], (uint32_t)(((i / C::NACC) - 1) & 1))) ok = false;
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t bb = su32(bbuf + (size_t)ts * C::BBUF);
            const uint64_t bint0 = umma_desc(bb, C::IPLANE, C::ROWB);     // hi/lo rows interleaved
            const uint64_t bhi0 = umma_desc(bb, C::IPLANE, 2 * C::ROWB);  // hi rows only
            const uint32_t dset = tmem + (uint32_t)(td * C::SETCOLS);
            for (int bi = 0; bi < kTcBlocks; ++bi, ++g) {
                const int b = (bi + rot) % kTcBlocks;
                const int pk = g / C::NPROD;  // fill index within producer g % NPROD
                const int s = (g % C::NPROD) * C::SP + pk % C::SP;
                if (!mbar_spin(&afull[s], (uint32_t)((pk / C::SP) & 1))) {
                    ok = false;
                    break;
                }
                const uint64_t boff = (uint64_t)boff16[b];
#pragma unroll
                for (int kk = 0; kk < C::KSTEP; ++kk) {
                    const uint64_t kb = (uint64_t)((2 * kk * C::IPLANE) >> 4);
                    const uint64_t dbi = bint0 + boff + kb, dbh = bhi0 + boff + kb;
#pragma unroll
                    for (int mt = 0; mt < C::MT; ++mt) {
                        const uint64_t da = a0 + (uint64_t)(((size_t)s * 2 * C::APART + mt * 16 * C::KCH * 128 + 2 * kk * 128) >> 4);
                        const uint32_t d1 = dset + (uint32_t)(mt * 3 * C::N), d2 = d1 + (uint32_t)(2 * C::N);
                        const uint32_t acc = (bi | kk) ? 1u : 0u;
                        if (split) {
                            umma_bf16(d1, da, dbi, id2n, acc);
                            umma_bf16(d2, da + alo_off, dbh, idn, acc);
                        } else {
                            umma_bf16(d2, da, dbh, idn, acc);
                        }
                    }
                }
                if (s % C::G == C::G - 1) umma_commit(&aempty[s / C::G]);  // the group's stages are free once read
            }
            umma_commit(&dfull[td]);  // accumulator set td holds tile i
            umma_commit(&bfree[ts]);  // halo buffer ts may be restaged
        }
        if (!ok) atomicOr(err, DEV_ERR_TIMEOUT);
    } else if (warp >= kStageWarp0 && warp < kStageWarp0 + kStageWarps) {
        // ---------------- halo staging ----------------
        constexpr int NST = 32 * kStageWarps;
        const int st = tid - 32 * kStageWarp0;
        for (int i = 0; i < ntiles; ++i) {
            const int ts = i % C::NBUF;
            if (i >= C::NBUF && !mbar_wait(&bfree[ts], (uint32_t)(((i / C::NBUF) - 1) & 1), 256)) {
                atomicOr(err, DEV_ERR_TIMEOUT);
                break;
            }
            const TcTile g = tc_tile<P>(job, (int)blockIdx.x + i * (int)gridDim.x);
            unsigned char* bb = bbuf + (size_t)ts * C::BBUF;
            if (maps.use_tma[g.li]) {
                // one TMA box: {HX columns x 8 bf16 (160 contiguous bytes), 2 parts, HY rows, 4 KCH planes},
                // zero-filled outside the level; x = 8 (PX0 - 1) elements is a multiple of 16 bytes
                if (st == 0) {
                    mbar_expect_tx(&bfull[ts], (uint32_t)C::BBUF);
                    tma_load_4d(bb, &maps.map[g.li], 8 * (g.PX0 - 1), 0, g.PY0 - 1, 0, &bfull[ts]);
                }
                continue;
            }
            const size_t row = (size_t)g.np * 16;
            const int units = 2 * 4 * C::KCH * C::NPOS;  // 16-byte halo units
            for (int it = st; it < units; it += NST) {
                const int pos = it % C::NPOS;
                const int pc = it / C::NPOS;  // (part, cc)
                const int part = pc / (4 * C::KCH), cc = pc % (4 * C::KCH);
                const int hx = pos % C::HX, hy = pos / C::HX;
                int qx = g.PX0 - 1 + hx, qy = g.PY0 - 1 + hy;  // source parent
                bool in = qx >= 0 && qy >= 0 && qx < g.np && qy < g.np;
                if (job.periodic) {
                    qx = (qx + g.np) % g.np;
                    qy = (qy + g.np) % g.np;
                    in = true;
                }
                const unsigned char* src =
                    in ? g.planes + (((size_t)cc * g.np + qy) * 2 + part) * row + (size_t)qx * 16 : g.planes;
                cp_async16(bb + (size_t)cc * C::IPLANE + (size_t)(2 * hy + part) * C::ROWB + (size_t)hx * 16, src, in);
            }
            asm volatile("cp.async.commit_group;\n" ::: "memory");
            asm volatile("cp.async.wait_all;\n" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("bar.sync 1, %0;" ::"n"(NST) : "memory");
            if (st == 0) mbar_arrive(&bfull[ts]);
        }
    } else if (warp >= kEpiWarp0) {
        // ---------------- epilogue ----------------
        const int q4 = warp - kEpiWarp0;  // TMEM lane quarter (= warp % 4)
        for (int i = 0; i < ntiles; ++i) {
            const int td = i % C::NACC;
            const bool fin = mbar_wait(&dfull[td], (uint32_t)((i / C::NACC) & 1), 256);
            if (!fin) {
                if (lane == 0) atomicOr(err, DEV_ERR_TIMEOUT);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const TcTile g = tc_tile<P>(job, (int)blockIdx.x + i * (int)gridDim.x);
            const uint32_t lanes = (uint32_t)(q4 * 32) << 16;
#pragma unroll 1
            for (int mt = 0; mt < C::MT; ++mt) {
                const int R = mt * 128 + q4 * 32 + lane;  // output row (c, n, re/im)
                const bool valid_row = R < 8 * P;
                const int c = R / (2 * P), q = R % (2 * P);
                const uint32_t d1 = tmem + lanes + (uint32_t)(td * C::SETCOLS + mt * 3 * C::N);
                const uint32_t d2 = d1 + (uint32_t)(2 * C::N);
#pragma unroll 1
                for (int y2 = 0; y2 < C::TPY / 2; ++y2) {  // two tile rows = 16 parents per round
                    uint32_t a0[16], a1[16], b[16];
                    tmem_ld16_async(d2 + (uint32_t)(16 * y2), b);  // D2 columns of tile rows 2y2, 2y2+1
                    if (split) {
                        tmem_ld16_async(d1 + (uint32_t)(32 * y2), a0);       // row 2y2: hi cols 0-7, lo cols 8-15
                        tmem_ld16_async(d1 + (uint32_t)(32 * y2 + 16), a1);  // row 2y2+1
                    }
                    tmem_wait_ld();
                    if (!valid_row) continue;
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) {
                        const int yy = 2 * y2 + (jj >> 3), xx = jj & 7;
                        float v = __uint_as_float(b[jj]);
                        if (split) {
                            const uint32_t* a = (jj >> 3) ? a1 : a0;
                            v += __uint_as_float(a[xx]) + __uint_as_float(a[8 + xx]);
                        }
                        const int px = g.PX0 + xx, py = g.PY0 + yy;
                        if (px >= g.np || py >= g.np) continue;
                        const int ix = 2 * px + (c & 1), iy = 2 * py + (c >> 1);
                        float* dst = reinterpret_cast<float*>(g.L + ((size_t)iy * g.side + ix) * P) + q;
                        if (job.accumulate) v += *dst;
                        *dst = v;
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&dfree[td]);
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == kMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)C::TMEM_COLS)
                     : "memory");
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
bool m2l_tc_supported(int p) { return p == 16 || p == 24; }

size_t m2l_tc_image_bytes(int p)
{
    switch (p) {
        case 16: return (size_t)kTcReplicas * kTcBlocks * 2 * TcCfg<16>::APART;
        case 24: return (size_t)kTcReplicas * kTcBlocks * 2 * TcCfg<24>::APART;
        default: return 0;
    }
}

template <int P>
static int build_image_p(double s, int variant, unsigned char* img, cudaStream_t st)
{
    using C = TcCfg<P>;
    const int64_t total = (int64_t)kTcBlocks * C::MT * 128 * C::K2;
    build_tc_image_kernel<P><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(s, variant, img);
    FMM_CUDA_TRY(cudaGetLastError());
    const size_t one = (size_t)kTcBlocks * 2 * C::APART;
    for (int r = 1; r < kTcReplicas; ++r) FMM_CUDA_TRY(cudaMemcpyAsync(img + r * one, img, one, cudaMemcpyDeviceToDevice, st));
    return FMM_OK;
}

int launch_build_tc_image(int p, double s, int variant, void* img, cudaStream_t st)
{
    switch (p) {
        case 16: return build_image_p<16>(s, variant, (unsigned char*)img, st);
        case 24: return build_image_p<24>(s, variant, (unsigned char*)img, st);
        default: return fail(FMM_EINVAL, "M2L TC: unsupported p = %d", p);
    }
}

// cuTensorMapEncodeTiled from the driver, looked up once (no link against libcuda)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            (void)cudaGetLastError();
    });
    return fn;
}

template <int P>
static int launch_tc_p(M2LLaunch& job, const void* img, bool split, int* err, cudaStream_t st)
{
    using C = TcCfg<P>;
    int total = 0;
    for (int i = 0; i < job.nlev; ++i) {
        job.lv[i].tile_begin = total;
        const int np = 1 << (job.lv[i].level - 1);
        total += ((np + kTcTileX - 1) / kTcTileX) * ((np + C::TPY - 1) / C::TPY);
    }
    if (total == 0) return FMM_OK;
    int sms = 0;
    int rc = device_sm_count(&sms);
    if (rc) return rc;
    // BF16 hi/lo planes of every level's MEs (library scratch), then the main kernel
    size_t bytes = 0;
    int64_t items = 0;
    for (int i = 0; i < job.nlev; ++i) {
        bytes += ((size_t)1 << (2 * job.lv[i].level)) * (size_t)P * 8;
        items += ((int64_t)1 << (2 * job.lv[i].level)) * C::KCH;
    }
    unsigned char* ws = nullptr;
    if ((rc = tc_plane_workspace(bytes, &ws))) return rc;
    for (int i = 0; i < job.nlev; ++i) {
        job.lv[i].planes = ws;
        ws += ((size_t)1 << (2 * job.lv[i].level)) * (size_t)P * 8;
    }
    me_planes_kernel<P><<<(unsigned)((items + 255) / 256), 256, 0, st>>>(job, split ? 1 : 0);
    FMM_CUDA_TRY(cudaGetLastError());
    TcMaps maps;
    memset(&maps, 0, sizeof(maps));
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    for (int i = 0; i < job.nlev; ++i) {
        const int np = 1 << (job.lv[i].level - 1);
        if (!encode || job.periodic || np < C::HX || np < C::HY) continue;  // halo larger than the level: cp.async path
        // planes [cc][qy][part][qx][8 bf16]: (qx, 8) merge into one contiguous dimension of 8 np elements
        const cuuint64_t dims[4] = {(cuuint64_t)np * 8, 2, (cuuint64_t)np, (cuuint64_t)(4 * C::KCH)};
        const cuuint64_t strides[3] = {(cuuint64_t)np * 16, (cuuint64_t)np * 32, (cuuint64_t)np * np * 32};
        const cuuint32_t box[4] = {(cuuint32_t)(8 * C::HX), 2, (cuuint32_t)C::HY, (cuuint32_t)(4 * C::KCH)};
        const cuuint32_t estr[4] = {1, 1, 1, 1};
        const CUresult r = encode(&maps.map[i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)job.lv[i].planes, dims,
                                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(FMM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
        maps.use_tma[i] = 1;
    }
    static unsigned long long opted;
    if ((rc = smem_opt_in((const void*)m2l_tc_kernel<P>, (int)C::smem, &opted))) return rc;
    const int grid = total < sms ? total : sms;
    m2l_tc_kernel<P><<<grid, kTcCtaThreads, C::smem, st>>>(job, maps, (const unsigned char*)img, split ? 1 : 0, total,
                                                            err);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

int launch_m2l_tc(M2LLaunch& job, int p, const void* img, bool split, cudaStream_t st)
{
    int* err = nullptr;
    int rc = device_error_word(&err);
    if (rc) return rc;
    switch (p) {
        case 16: return launch_tc_p<16>(job, img, split, err, st);
        case 24: return launch_tc_p<24>(job, img, split, err, st);
        default: return fail(FMM_EINVAL, "M2L TC: unsupported p = %d", p);
    }
}

}  // namespace fmmgb
