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
//   N       = the 8 x 32 = 256 parents of a tile
//   K       = 32 blocks (e, c') x 2p, processed 16 at a time.
// A (the operator block of (e, c')) streams from an L2-resident image
// through a ring of shared-memory stages (cp.async.bulk).  B (the source MEs)
// is the class-c' halo of the tile, 10 x 34 parents, seen through a
// descriptor whose start is shifted by e: the 8 parents of one tile row are
// 8 consecutive 16-byte rows, and the stride to the next tile row is the halo
// row pitch (SBO).
//
// Precision.  BF16 keeps 8 significant bits.  With the hi/lo split
// x = hi + lo (both BF16), the three products A_hi B_hi + A_hi B_lo +
// A_lo B_hi recover ~16 bits, all accumulated into the same FP32 TMEM
// columns.
//
// Why N = 256.  A tcgen05 MMA reads its operands from shared memory at about
// 128 B per cycle: an M = 128, K = 16 product reads 4 KB of A and N/16 KB of
// B and executes in N/2 cycles, so N = 128 products are bound by the
// shared-memory port (64 cycles either way) with no room for the operator
// stream, while N = 256 products (128 cycles for 96 cycles of operand reads)
// leave the port time the 16 KB ring refill of each block needs.  One
// 256-column accumulator holds the three products, so two accumulators fit in
// TMEM at p = 16 and a segment's epilogue overlaps the next one's MMAs.
//
// Work split (stream-K).  The U = tiles x 32 units (tile, block) are cut into
// equal contiguous ranges, one per CTA, so every SM does the same number of
// MMAs whatever the tile count.  A CTA walks its range's tiles from last to
// first.  For a tile cut between CTAs, the part holding its first unit (the
// head) is the first segment its CTA processes: it stores into L and then
// publishes the tile's flag; every other part of the tile, held by higher
// CTAs, waits for that flag (long published when the waiting CTA gets there)
// and adds its sums with fire-and-forget reductions.  No CTA waits on a
// higher one, every wait is bounded, and the kernel's last CTA to finish
// clears the flags for the next launch.
//
// Schedule.  One CTA per SM (grid = min(SMs, U / 8)), four roles: producer
// warps (six at p = 16, two at p = 24, one ring stage and one bulk copy in
// flight each) stream the operator blocks of the range; an MMA thread (warp
// 8, which also owns the TMEM allocation) issues the products; the staging
// warps (the rest of warps 0-7 and warps 9-11: five at p = 16, nine at p = 24)
// build the class halos in shared memory, converting the FP32 MEs that a
// tensor copy lands into their BF16 hi/lo parts in the layout the MMAs read
// (no pre-pass, no copy of the MEs in global memory); four epilogue warps
// (12-15) drain the accumulators.  The first operator fills and the first halo
// copy are issued before the TMEM allocation.  Every mbarrier and flag wait is bounded:
// on timeout the waiting role records FMM_ETIMEOUT in the device error word
// and stops; producers wait (bounded) for their own copies in flight, the
// MMA thread for its own MMAs, and the TMEM is freed before the CTA exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace fmmgb {

constexpr int kTcTileX = 8;     // parents per tile row (one core-matrix group of the N operand)
constexpr int kTcTileY = 32;    // parent rows per tile
constexpr int kTcBlocks = 32;   // (e != 0) x 4 source classes
constexpr int kTcReplicas = 1;  // copies of the operator image in global memory (1, 2 and 4 measured alike)
constexpr int kTcMinUnits = 8;  // fewest units per CTA: a tile is cut between at most 5 CTAs

// TF: TF32 operands (hi/lo in 32-bit containers, K = 8 per MMA) instead of BF16 (K = 16)
template <int P, bool TF = false>
struct TcCfg {
    static constexpr int ES = TF ? 4 : 2;             // operand element bytes
    static constexpr int EPC = 16 / ES;               // elements per 16-byte chunk
    static constexpr int K2 = 2 * P;                  // real K per block
    static constexpr int KCH = K2 / EPC;              // 16-byte chunks per block row
    static constexpr int KSTEP = K2 * ES / 32;        // MMA K steps (32 bytes of K each) per block
    static constexpr int MT = (8 * P + 127) / 128;    // M tiles of 128 rows
    static constexpr int N = kTcTileX * kTcTileY;     // parents per tile = MMA N
    static constexpr int HX = kTcTileX + 2, HY = kTcTileY + 2;
    static constexpr int NPOS = HX * HY;              // halo parent positions
    // one chunk plane of a class halo: HY rows x (hi, lo) x HX positions x 16 B
    static constexpr int ROWB = HX * 16;
    static constexpr int IPLANE = 2 * HY * ROWB;
    static constexpr int HBUF = KCH * IPLANE;         // one class halo (hi and lo)
    static constexpr int APART = MT * 128 * K2 * ES;  // one block's hi (or lo) operator image
    static constexpr int STAGE = 2 * APART;           // a ring stage: hi then lo
    static constexpr int NHB = (P <= 16 && !TF) ? 2 : 1;  // class halo buffers (hi/lo)
    static constexpr int LBUF = NPOS * K2 * 4;        // the FP32 landing buffer of one class halo
    // ring stages, one producer warp each: as many as shared memory holds
    // beside the halo buffers (6 x 16 KB at p = 16, 2 x 48 KB at p = 24; TF32 at p = 16: 3 x 32 KB)
    static constexpr int STAGES = TF ? 3 : (P <= 16 ? 6 : 2);
    static constexpr int DCOLS = MT * N;              // TMEM columns of one accumulator
    static constexpr int NACC = 2 * DCOLS <= 512 ? 2 : 1;
    static constexpr int TMEM_COLS = 512;
    static constexpr size_t smem = (size_t)NHB * HBUF + (size_t)LBUF + (size_t)STAGES * STAGE + 1024;
    static_assert(STAGES <= 8, "producer warps 0-7");
    static_assert(smem <= 232448, "dynamic shared memory");
    static_assert(DCOLS * NACC <= TMEM_COLS, "TMEM");
};

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
// operator image: W[(c, n, r_out)][(k, r_in)] per block, hi and lo (BF16, or TF32
// in 32-bit containers), in the canonical K-major no-swizzle layout (8-row x
// 16-byte core matrices of EPC elements of ES bytes):
//   byte offset of (row R, real column q) = (R / 8) * (KCH * 128) + (q / EPC) * 128 + (R % 8) * 16 + (q % EPC) * ES
// built in FP64 on the GPU from a(D) = (-1)^n C(n+k,k) D^-(n+k+1).
// ---------------------------------------------------------------------------
template <int P, bool TF>
__global__ void build_tc_image_kernel(double s, int variant, unsigned char* __restrict__ img)
{
    using C = TcCfg<P, TF>;
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
    const size_t off =
        (size_t)(R / 8) * (C::KCH * 128) + (size_t)(q / C::EPC) * 128 + (R % 8) * 16 + (q % C::EPC) * C::ES;
    unsigned char* blk = img + (size_t)b * 2 * C::APART;
    if constexpr (TF) {
        const uint32_t whi = f32_to_tf32((float)w);
        const uint32_t wlo = f32_to_tf32((float)(w - (double)__uint_as_float(whi)));
        *reinterpret_cast<uint32_t*>(blk + off) = whi;
        *reinterpret_cast<uint32_t*>(blk + C::APART + off) = wlo;
    } else {
        const __nv_bfloat16 whi = __double2bfloat16(w);
        const __nv_bfloat16 wlo = __double2bfloat16(w - (double)__bfloat162float(whi));
        *reinterpret_cast<__nv_bfloat16*>(blk + off) = whi;
        *reinterpret_cast<__nv_bfloat16*>(blk + C::APART + off) = wlo;
    }
}

// unit order within a tile: u & 31 = c' * 8 + pe (class-major, so a class
// halo serves 8 consecutive units); the image stores block b = pe * 4 + c'
__host__ __device__ inline int tc_image_block(int blk) { return (blk & 7) * 4 + (blk >> 3); }

// ---------------------------------------------------------------------------
// the kernel: persistent, one CTA per SM, warp-specialised, stream-K ranges
// ---------------------------------------------------------------------------
// warps 0-7 producers (the first STAGES of them; the others join the staging),
// 8 MMA issuer, 9-11 halo staging, 12-15 epilogue (a multiple of 4, so that
// warp % 4 is its TMEM lane quarter)
constexpr int kTcCtaThreads = 512;
constexpr int kMmaWarp = 8, kStageWarp0 = 9, kStageWarps = 3, kEpiWarp0 = 12;
constexpr int kStageBatch = 5;  // halo items in flight per staging thread (global-load path)
// named barriers: staging warps (wait outcome; cp.async completion), epilogue warps (wait outcome;
// publish; the target-existence mask of an adaptive tile)
constexpr int kStageBar = 1, kStageCopyBar = 2, kEpiBar = 3, kPubBar = 4, kMaskBar = 5;

struct TcTile {
    const float4* M;
    float2* L;
    const uint8_t* ex;  // adaptive level: box existence, NULL = every box exists
    int side, np, PX0, PY0, li;
};

__device__ __forceinline__ TcTile tc_tile(const M2LLaunch& job, int tile)
{
    int li = 0;
    while (li + 1 < job.nlev && tile >= job.lv[li + 1].tile_begin) ++li;
    const M2LLevel& lv = job.lv[li];
    TcTile g;
    g.M = reinterpret_cast<const float4*>(lv.M);
    g.L = lv.L;
    g.ex = lv.exists;
    g.side = 1 << lv.level;
    g.np = g.side >> 1;
    int t = tile - lv.tile_begin;
    if (lv.tc_tiles) t = __ldg(lv.tc_tiles + t);  // adaptive level: the active tiles only
    const int tpr = (g.np + kTcTileX - 1) / kTcTileX;
    g.PX0 = (t % tpr) * kTcTileX;
    g.PY0 = (t / tpr) * kTcTileY;
    g.li = li;
    return g;
}

// Per launch level: a 5-D tensor map over its FP32 MEs, [qy][cy][qx][cx][2p floats]
// (box (2 qx + cx, 2 qy + cy)), so that one box {2p, 1, 10, 1, 34} at (0, c'x,
// PX0 - 1, c'y, PY0 - 1) is the class-c' halo of a tile, zero outside the level
// (also for levels smaller than the box).
struct TcMaps {
    CUtensorMap map[kMaxLaunchLevels];
    int use_tma[kMaxLaunchLevels];  // 0: the level is smaller than the box, or the lists are periodic
};

// tensor-map load into this CTA's shared memory, completion on an mbarrier
__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];" ::"r"(su32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(su32(bar))
        : "memory");
}

// first unit of CTA j's range: the U units in `grid` equal contiguous shares
__device__ __forceinline__ int tc_range_begin(int j, int grid, int units)
{
    return (int)(((long long)units * j) / grid);
}

// A CTA's range [u0, u1) is walked tile by tile from its last tile to its first
// (segment i = the units of tile t1 - i inside the range), units in order
// within a segment.  Every role runs this walk.
struct TcSeg {
    int t, sa, sb;  // tile, units [sa, sb)
};
__device__ __forceinline__ TcSeg tc_seg(int u0, int u1, int i)
{
    TcSeg s;
    s.t = ((u1 - 1) >> 5) - i;
    s.sa = max(u0, s.t * kTcBlocks);
    s.sb = min(u1, (s.t + 1) * kTcBlocks);
    return s;
}
__device__ __forceinline__ int tc_nseg(int u0, int u1) { return u1 > u0 ? ((u1 - 1) >> 5) - (u0 >> 5) + 1 : 0; }

// the unit at walk position g (0 <= g < u1 - u0) of the range [u0, u1)
__device__ __forceinline__ int tc_walk_unit(int u0, int u1, int g)
{
    const int nseg = tc_nseg(u0, u1);
    for (int i = 0; i < nseg; ++i) {
        const TcSeg sg = tc_seg(u0, u1, i);
        if (g < sg.sb - sg.sa) return sg.sa + g;
        g -= sg.sb - sg.sa;
    }
    return u0;
}

// class group k (0-based, in walk order) of the range [u0, u1): its tile and source class
__device__ __forceinline__ bool tc_group(int u0, int u1, int k, int& t, int& cls)
{
    const int nseg = tc_nseg(u0, u1);
    for (int i = 0; i < nseg; ++i) {
        const TcSeg sg = tc_seg(u0, u1, i);
        const int c0 = (sg.sa & 31) >> 3, c1 = ((sg.sb - 1) & 31) >> 3;
        if (k <= c1 - c0) {
            t = sg.t;
            cls = c0 + k;
            return true;
        }
        k -= c1 - c0 + 1;
    }
    return false;
}


// One chunk (4 complex = 8 floats) of a source ME -> its BF16 hi part at dst and lo part at dst + lo_off.
__device__ __forceinline__ void tc_stage_chunk(const float4* a, const float4* b, unsigned char* dst, int lo_off)
{
    const float4 v0 = *a, v1 = *b;
    const float f[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
    uint32_t h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        __nv_bfloat162 hv = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
        const float2 hf = __bfloat1622float2(hv);
        h[j] = *reinterpret_cast<uint32_t*>(&hv);
        l[j] = pack_bf16(f[2 * j] - hf.x, f[2 * j + 1] - hf.y);
    }
    *reinterpret_cast<uint4*>(dst) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(dst + lo_off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// One TF32 chunk (2 complex = 4 floats) -> its TF32 hi part at dst and lo part at dst + lo_off.
__device__ __forceinline__ void tc_stage_chunk_tf32(const float4 v, unsigned char* dst, int lo_off)
{
    const uint32_t h0 = f32_to_tf32(v.x), h1 = f32_to_tf32(v.y), h2 = f32_to_tf32(v.z), h3 = f32_to_tf32(v.w);
    *reinterpret_cast<uint4*>(dst) = make_uint4(h0, h1, h2, h3);
    *reinterpret_cast<uint4*>(dst + lo_off) =
        make_uint4(f32_to_tf32(v.x - __uint_as_float(h0)), f32_to_tf32(v.y - __uint_as_float(h1)),
                   f32_to_tf32(v.z - __uint_as_float(h2)), f32_to_tf32(v.w - __uint_as_float(h3)));
}

// A class halo that a tensor copy landed as FP32 [parent][2p] -> its hi/lo parts in the
// layout the MMAs read, by NT threads (this one is `st`).  TF32: thread st converts parents
// st, st + NT, ..., each one's chunks from (st + s) % KCH on (8 consecutive threads read 8
// different 16-byte bank groups and write 8 consecutive parents of a halo row).  BF16:  Thread st converts parents st,
// st + NT, ..., each one's chunks in the order (st + s) % KCH and the two 16-byte halves of a
// chunk in the order set by bit 2 of st, so that 8 consecutive threads read 8 different
// 16-byte bank groups of the landing buffer and write 8 consecutive parents of a halo row.
template <int P, int NT, bool TF = false>
__device__ __forceinline__ void tc_convert_landed(const unsigned char* lbuf, unsigned char* buf, int st, uint32_t keep)
{
    using C = TcCfg<P, TF>;
    const int h = (st >> 2) & 1, c0 = st % C::KCH;
    int j = 0;
#pragma unroll 1
    for (int pos = st; pos < C::NPOS; pos += NT, ++j) {
        if (!((keep >> j) & 1)) {  // an absent source box (adaptive level): zero
            unsigned char* dst = buf + (size_t)(2 * (pos / C::HX)) * C::ROWB + (size_t)(pos % C::HX) * 16;
#pragma unroll
            for (int s = 0; s < C::KCH; ++s) {
                *reinterpret_cast<uint4*>(dst + (size_t)s * C::IPLANE) = make_uint4(0u, 0u, 0u, 0u);
                *reinterpret_cast<uint4*>(dst + (size_t)s * C::IPLANE + C::ROWB) = make_uint4(0u, 0u, 0u, 0u);
            }
            continue;
        }
        const float4* src = reinterpret_cast<const float4*>(lbuf + (size_t)pos * (C::K2 * 4));
        unsigned char* dst = buf + (size_t)(2 * (pos / C::HX)) * C::ROWB + (size_t)(pos % C::HX) * 16;
        if constexpr (TF) {
            float4 x[C::KCH];
#pragma unroll
            for (int s = 0; s < C::KCH; ++s) x[s] = src[c0 + s < C::KCH ? c0 + s : c0 + s - C::KCH];
#pragma unroll
            for (int s = 0; s < C::KCH; ++s) {
                const int ch = c0 + s < C::KCH ? c0 + s : c0 + s - C::KCH;
                tc_stage_chunk_tf32(x[s], dst + (size_t)ch * C::IPLANE, C::ROWB);
            }
            continue;
        }
        float4 x[C::KCH], y[C::KCH];
#pragma unroll
        for (int s = 0; s < C::KCH; ++s) {
            const int ch = c0 + s < C::KCH ? c0 + s : c0 + s - C::KCH;
            x[s] = src[2 * ch + h];
            y[s] = src[2 * ch + 1 - h];
        }
#pragma unroll
        for (int s = 0; s < C::KCH; ++s) {
            const int ch = c0 + s < C::KCH ? c0 + s : c0 + s - C::KCH;
            const float4 f0 = h ? y[s] : x[s], f1 = h ? x[s] : y[s];
            tc_stage_chunk(&f0, &f1, dst + (size_t)ch * C::IPLANE, C::ROWB);
        }
    }
}

// Bit j: the source box at halo position st + j NT of class `cls` exists (adaptive levels; every
// bit set on a level where every box exists, and for positions outside the level, which the
// tensor copy zero-fills).  Read before the copy is waited for, so the loads overlap it.
template <int P, int NT>
__device__ __forceinline__ uint32_t tc_halo_keep(const TcTile& tl, int cls, int st)
{
    using C = TcCfg<P>;
    uint32_t keep = ~0u;
    if (!tl.ex) return keep;
    constexpr int NJ = (C::NPOS + NT - 1) / NT;
    static_assert(NJ <= 32, "keep mask");
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int pos = st + j * NT;
        if (pos >= C::NPOS) break;
        const int qx = tl.PX0 - 1 + pos % C::HX, qy = tl.PY0 - 1 + pos / C::HX;
        if (qx < 0 || qy < 0 || qx >= tl.np || qy >= tl.np) continue;
        if (!__ldg(tl.ex + (size_t)(2 * qy + (cls >> 1)) * tl.side + 2 * qx + (cls & 1))) keep &= ~(1u << j);
    }
    return keep;
}

// AND of `v` over the `n` threads of named barrier `id` (uniform control flow after a bounded wait)
__device__ __forceinline__ bool bar_and(int id, int n, bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.and.pred p, %2, %3, q;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}

// bounded wait for a flag that another CTA of this launch publishes with release semantics
__device__ __forceinline__ bool wait_flag(const int* f)
{
    for (uint32_t it = 0; it < kWaitCap; ++it) {
        int v;
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
        if (v) return true;
        __nanosleep(128);
    }
    return false;
}

template <int P, bool TF>
__global__ void __launch_bounds__(kTcCtaThreads, 1)
    m2l_tc_kernel(M2LLaunch job, const __grid_constant__ TcMaps maps, const unsigned char* __restrict__ img, int split,
                  int units, int* __restrict__ flags, int* __restrict__ done, int* __restrict__ err)
{
    using C = TcCfg<P, TF>;
    extern __shared__ __align__(1024) unsigned char tsm[];
    unsigned char* hbuf = tsm;                                   // NHB class halos
    unsigned char* lbuf = tsm + (size_t)C::NHB * C::HBUF;        // FP32 landing buffer of a class halo
    unsigned char* astage = lbuf + C::LBUF;                      // STAGES x (hi APART, lo APART)
    uint64_t* afull = reinterpret_cast<uint64_t*>(astage + (size_t)C::STAGES * C::STAGE);
    uint64_t* aempty = afull + C::STAGES;
    uint64_t* hfull = aempty + C::STAGES;
    uint64_t* hfree = hfull + C::NHB;
    uint64_t* dfull = hfree + C::NHB;
    uint64_t* dfree = dfull + 2;
    uint64_t* mdone = dfree + 2;  // the MMA thread's final commit: every issued MMA has completed
    uint64_t* lfull = mdone + 1;  // a tensor copy into the landing buffer has landed
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(lfull + 1);
    uint8_t* s_tmask = reinterpret_cast<uint8_t*>(tmem_slot + 1);  // [4 classes][32 tile rows]: bit x, target exists

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cta = (int)blockIdx.x, grid = (int)gridDim.x;
    const int u0 = tc_range_begin(cta, grid, units), u1 = tc_range_begin(cta + 1, grid, units);
    const int nseg = tc_nseg(u0, u1);
    const uint32_t abytes = split ? (uint32_t)C::STAGE : (uint32_t)C::APART;
    // CTAs read one of kTcReplicas copies of the image, spreading the
    // simultaneous reads of all SMs over more L2 lines
    const unsigned char* rimg = img + (size_t)(cta % kTcReplicas) * kTcBlocks * C::STAGE;

    const int nunits = u1 - u0;
    // halo staging: the producer warps beyond STAGES, then warps 9-11; stw = index among them (-1: other role)
    constexpr int NST = 32 * (8 - C::STAGES + kStageWarps);
    const int stw = (warp >= C::STAGES && warp < 8) ? warp - C::STAGES
                    : (warp >= kStageWarp0 && warp < kStageWarp0 + kStageWarps) ? 8 - C::STAGES + warp - kStageWarp0
                                                                                : -1;
    const int st = stw * 32 + lane;
    int ngrp = 0;  // class groups of the walk
    for (int i = 0; i < nseg; ++i) {
        const TcSeg sg = tc_seg(u0, u1, i);
        ngrp += (((sg.sb - 1) & 31) >> 3) - ((sg.sa & 31) >> 3) + 1;
    }
    // the next tensor copy into the landing buffer: the first group at or after `from` on the
    // tensor-copy path, issued by staging thread 0; every staging thread returns that group (-1: none)
    auto issue_tma = [&](int from) -> int {
        for (int k = from; k < ngrp; ++k) {
            int t, cls;
            tc_group(u0, u1, k, t, cls);
            const TcTile tl = tc_tile(job, t);
            if (!maps.use_tma[tl.li]) continue;
            if (st == 0) {
                mbar_expect_tx(lfull, (uint32_t)C::LBUF);
                tma_load_5d(lbuf, &maps.map[tl.li], 0, cls & 1, tl.PX0 - 1, cls >> 1, tl.PY0 - 1, lfull);
            }
            return k;
        }
        return -1;
    };
    int pending = -1;  // staging: the group whose tensor copy is in flight

    if (tid == 0) {
        for (int i = 0; i < C::NHB; ++i) {
            mbar_init(&hfull[i], 1);
            mbar_init(&hfree[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&dfull[i], 1);
            mbar_init(&dfree[i], 4);
        }
        mbar_init(mdone, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // The first operator fill of every stage and the first halo copy leave before the setup
    // barrier (the TMEM allocation): each issuing thread initialises the barrier its copy
    // completes on, and the setup barrier orders that before any wait on it.
    if (warp < C::STAGES && lane == 0) {
        mbar_init(&afull[warp], 1);
        mbar_init(&aempty[warp], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (warp < nunits) {
            mbar_expect_tx(&afull[warp], abytes);
            bulk_load(astage + (size_t)warp * C::STAGE,
                      rimg + (size_t)tc_image_block(tc_walk_unit(u0, u1, warp) & 31) * C::STAGE, abytes, &afull[warp]);
        }
    }
    if (stw >= 0) {
        if (st == 0) {
            mbar_init(lfull, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        pending = issue_tma(0);
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

    // No MMA can start before the first class halo: when it comes by tensor copy, the whole CTA
    // converts it.  If that copy does not land in time, the staging warps take the group over.
    bool first_done = false;
    if (ngrp > 0) {
        int t, cls;
        tc_group(u0, u1, 0, t, cls);
        const TcTile tl0 = tc_tile(job, t);
        if (maps.use_tma[tl0.li]) {
            const uint32_t keep = tc_halo_keep<P, kTcCtaThreads>(tl0, cls, tid);
            const bool landed = mbar_wait(lfull, 0, 64);
            if (__syncthreads_and(landed ? 1 : 0)) {
                tc_convert_landed<P, kTcCtaThreads, TF>(lbuf, hbuf, tid, keep);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                first_done = true;
            }
            __syncthreads();
            if (first_done && tid == 0) mbar_arrive(&hfull[0]);
        }
    }

    if (warp < C::STAGES) {
        // ---------------- producer `warp`: units g = warp, warp + STAGES, ... of the walk ----------------
        if (lane == 0) {
            const int s = warp;
            int k = s < nunits ? 1 : 0;  // fills issued into stage s (the first left before the setup barrier)
            bool ok = true;
            for (int g = s + C::STAGES; g < nunits; g += C::STAGES) {
                if (!mbar_wait(&aempty[s], (uint32_t)((k - 1) & 1))) {
                    ok = false;
                    break;
                }
                const int b = tc_image_block(tc_walk_unit(u0, u1, g) & 31);
                mbar_expect_tx(&afull[s], abytes);
                bulk_load(astage + (size_t)s * C::STAGE, rimg + (size_t)b * C::STAGE, abytes, &afull[s]);
                ++k;
            }
            if (!ok) atomicOr(err, DEV_ERR_TIMEOUT);
            // do not leave while a copy is in flight: the last fill of stage s must have landed
            if (k > 0 && !mbar_wait(&afull[s], (uint32_t)((k - 1) & 1))) atomicOr(err, DEV_ERR_TIMEOUT);
        }
    } else if (warp == kMmaWarp && lane == 0) {
        // ---------------- MMA issuer ----------------
        // per K step (32 bytes of K: 16 BF16 or 8 TF32) and M tile: D += A_hi B_hi (+ A_hi B_lo +
        // A_lo B_hi with the split), all N = 256 products into the same accumulator columns;
        // instruction descriptor: D F32, A and B BF16 (1) or TF32 (2), K-major, N, M = 128
        constexpr uint32_t kFmt = TF ? 2u : 1u;
        const uint32_t idesc =
            (1u << 4) | (kFmt << 7) | (kFmt << 10) | ((uint32_t)(C::N >> 3) << 17) | ((128u >> 4) << 24);
        const uint32_t abase = su32(astage), hbase = su32(hbuf);
        constexpr uint64_t alo_off = (uint64_t)(C::APART >> 4);
        int g = 0, hg = 0;
        bool ok = true;
        for (int i = 0; i < nseg && ok; ++i) {
            const TcSeg sg = tc_seg(u0, u1, i);
            const int d = i % C::NACC;
            if (i >= C::NACC && !mbar_spin(&dfree[d], (uint32_t)(((i / C::NACC) - 1) & 1))) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t dset = tmem + (uint32_t)(d * C::DCOLS);
            bool first = true;
            for (int u = sg.sa; u < sg.sb && ok;) {
                const int cls = (u & 31) >> 3;
                const int grp_end = min(sg.sb, sg.t * kTcBlocks + (cls + 1) * 8);
                const int hb = hg % C::NHB;
                if (!mbar_spin(&hfull[hb], (uint32_t)((hg / C::NHB) & 1))) {
                    ok = false;
                    break;
                }
                const uint32_t hbb = hbase + (uint32_t)(hb * C::HBUF);
                for (; u < grp_end; ++u, ++g) {
                    const int s = g % C::STAGES;
                    if (!mbar_spin(&afull[s], (uint32_t)((g / C::STAGES) & 1))) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    int ex, ey, cs;
                    tc_block(tc_image_block(u & 31), ex, ey, cs);
                    const uint32_t bst = hbb + (uint32_t)((ey + 1) * 2 * C::ROWB + (ex + 1) * 16);
                    const uint64_t bhi = umma_desc(bst, C::IPLANE, 2 * C::ROWB);
                    const uint64_t blo = umma_desc(bst + C::ROWB, C::IPLANE, 2 * C::ROWB);
                    const uint64_t ahi = umma_desc(abase + (uint32_t)(s * C::STAGE), 128, C::KCH * 128);
#pragma unroll
                    for (int kk = 0; kk < C::KSTEP; ++kk) {
                        const uint64_t kb = (uint64_t)((2 * kk * C::IPLANE) >> 4);
#pragma unroll
                        for (int mt = 0; mt < C::MT; ++mt) {
                            const uint64_t da = ahi + (uint64_t)((mt * 16 * C::KCH * 128 + 2 * kk * 128) >> 4);
                            const uint32_t dm = dset + (uint32_t)(mt * C::N);
                            if constexpr (TF) {
                                umma_tf32(dm, da, bhi + kb, idesc, (first && kk == 0) ? 0u : 1u);
                                umma_tf32(dm, da, blo + kb, idesc, 1u);
                                umma_tf32(dm, da + alo_off, bhi + kb, idesc, 1u);
                            } else {
                                umma_bf16(dm, da, bhi + kb, idesc, (first && kk == 0) ? 0u : 1u);
                                if (split) {
                                    umma_bf16(dm, da, blo + kb, idesc, 1u);
                                    umma_bf16(dm, da + alo_off, bhi + kb, idesc, 1u);
                                }
                            }
                        }
                    }
                    first = false;
                    umma_commit(&aempty[s]);  // stage s is free once these MMAs have read it
                }
                if (!ok) break;
                umma_commit(&hfree[hb]);  // the class halo may be restaged
                ++hg;
            }
            if (!ok) break;
            umma_commit(&dfull[d]);  // accumulator d holds segment i
        }
        if (!ok) atomicOr(err, DEV_ERR_TIMEOUT);
        // before the TMEM is freed, every MMA issued here must have completed (also after a timeout)
        umma_commit(mdone);
        if (!mbar_wait(mdone, 0)) atomicOr(err, DEV_ERR_TIMEOUT);
    } else if (stw >= 0) {
        // ---------------- class-halo staging ----------------
        // The halo of source class c' for a tile: the MEs of boxes (2 qx + c'x, 2 qy + c'y) for the
        // 10 x 34 parents (qx, qy) around it, zero outside the level (periodic lists wrap), as BF16
        // hi and lo in the layout the MMAs read: [chunk of 4 complex][halo row][hi, lo][halo
        // column] x 16 bytes.  A halo arrives as FP32 by one tensor copy into the landing buffer
        // (prefetched while the previous class is converted and translated) and is converted
        // shared-to-shared; periodic lists (which wrap) are read from global memory (an item is
        // one (parent, chunk): 32 bytes in, 2 x 16 out).
        constexpr int NIT = C::KCH * C::NPOS;
        int nlanded = first_done ? 1 : 0;  // tensor copies consumed so far (landing-buffer phase)
        if (first_done) pending = issue_tma(1);
        bool ok = true;
        for (int k = first_done ? 1 : 0; k < ngrp && ok; ++k) {
            int t, cls;
            tc_group(u0, u1, k, t, cls);
            const TcTile tl = tc_tile(job, t);
            const int hb = k % C::NHB;
            bool w = true;
            const uint32_t keep = pending == k ? tc_halo_keep<P, NST>(tl, cls, st) : ~0u;
            if (k >= C::NHB) w = mbar_wait(&hfree[hb], (uint32_t)(((k / C::NHB) - 1) & 1), 256);
            if (pending == k) w = mbar_wait(lfull, (uint32_t)(nlanded & 1), 128) && w;
            if (!bar_and(kStageBar, NST, w)) {
                ok = false;
                break;
            }
            unsigned char* buf = hbuf + (size_t)hb * C::HBUF;
            if (pending == k) {
                tc_convert_landed<P, NST, TF>(lbuf, buf, st, keep);
                ++nlanded;
            } else {
#pragma unroll 1
                for (int it0 = st; it0 < NIT; it0 += NST * kStageBatch) {
                    float4 v[kStageBatch][2];
#pragma unroll
                    for (int b = 0; b < kStageBatch; ++b) {
                        const int it = it0 + b * NST;
                        v[b][0] = v[b][1] = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (it >= NIT) continue;
                        const int pos = it / C::KCH, ch = it % C::KCH;
                        int qx = tl.PX0 - 1 + pos % C::HX, qy = tl.PY0 - 1 + pos / C::HX;  // source parent
                        if (job.periodic) {
                            qx = (qx + tl.np) % tl.np;
                            qy = (qy + tl.np) % tl.np;
                        } else if (qx < 0 || qy < 0 || qx >= tl.np || qy >= tl.np) {
                            continue;
                        }
                        const int ix = 2 * qx + (cls & 1), iy = 2 * qy + (cls >> 1);
                        if (tl.ex && !__ldg(tl.ex + (size_t)iy * tl.side + ix)) continue;  // absent source
                        const float4* src = tl.M + ((size_t)iy * tl.side + ix) * (P / 2) + (TF ? ch : 2 * ch);
                        v[b][0] = __ldg(src);
                        if (!TF) v[b][1] = __ldg(src + 1);
                    }
#pragma unroll
                    for (int b = 0; b < kStageBatch; ++b) {
                        const int it = it0 + b * NST;
                        if (it >= NIT) break;
                        const int pos = it / C::KCH, ch = it % C::KCH;
                        float4 f0 = v[b][0], f1 = v[b][1];
                        unsigned char* dst = buf + (size_t)ch * C::IPLANE + (size_t)(2 * (pos / C::HX)) * C::ROWB +
                                             (size_t)(pos % C::HX) * 16;
                        if constexpr (TF) tc_stage_chunk_tf32(f0, dst, C::ROWB);
                        else tc_stage_chunk(&f0, &f1, dst, C::ROWB);
                    }
                }
            }
            // generic-proxy writes (and, for the landing buffer, reads), next touched by the async
            // proxy: the MMAs read the halo, the next tensor copy overwrites the landing buffer
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("bar.sync %0, %1;" ::"n"(kStageCopyBar), "n"(NST) : "memory");
            if (pending == k) pending = issue_tma(k + 1);
            if (st == 0) mbar_arrive(&hfull[hb]);
        }
        if (!ok && st == 0) atomicOr(err, DEV_ERR_TIMEOUT);
        // do not leave while a tensor copy is in flight (after a timeout one may be)
        if (pending >= 0 && st == 0 && !mbar_wait(lfull, (uint32_t)(nlanded & 1))) atomicOr(err, DEV_ERR_TIMEOUT);
    } else if (warp >= kEpiWarp0) {
        // ---------------- epilogue ----------------
        // A tile cut between CTAs: the part holding its first unit (the head, always the
        // first segment its CTA processes) stores into L and then publishes the tile's flag;
        // every other part waits for that flag (published early by a lower CTA) and adds
        // its sums with fire-and-forget reductions.
        const int q4 = warp - kEpiWarp0;  // TMEM lane quarter (= warp % 4)
        const uint32_t lanes = (uint32_t)(q4 * 32) << 16;
        for (int i = 0; i < nseg; ++i) {
            const TcSeg sg = tc_seg(u0, u1, i);
            const int d = i % C::NACC;
            const bool fin = mbar_wait(&dfull[d], (uint32_t)((i / C::NACC) & 1), 256);
            if (!bar_and(kEpiBar, 128, fin)) {
                if (q4 == 0 && lane == 0) atomicOr(err, DEV_ERR_TIMEOUT);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const TcTile tl = tc_tile(job, sg.t);
            const bool head = sg.sa == sg.t * kTcBlocks;
            const bool whole = head && sg.sb == (sg.t + 1) * kTcBlocks;
            // adaptive level: which of the tile's targets exist (absent ones are left untouched)
            const bool adapt = tl.ex != nullptr;
            if (adapt) {
                const int e = tid - 32 * kEpiWarp0, ce = e >> 5, py = tl.PY0 + (e & 31);
                uint32_t m = 0;
                if (py < tl.np)
#pragma unroll
                    for (int x = 0; x < kTcTileX; ++x) {
                        const int px = tl.PX0 + x;
                        if (px < tl.np && __ldg(tl.ex + (size_t)(2 * py + (ce >> 1)) * tl.side + 2 * px + (ce & 1)))
                            m |= 1u << x;
                    }
                s_tmask[e] = (uint8_t)m;
                asm volatile("bar.sync %0, %1;" ::"n"(kMaskBar), "n"(128) : "memory");
            }
            if (!head) {
                bool got = true;
                if (lane == 0) got = wait_flag(flags + sg.t);
                got = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
                if (got) {  // every lane's own acquire of the published flag
                    int v;
                    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(flags + sg.t) : "memory");
                    (void)v;
                } else if (lane == 0) {
                    atomicOr(err, DEV_ERR_TIMEOUT);
                }
            }
            // a tile row (8 parents) of one output row lands in 8 boxes 2 apart: one base pointer per
            // tile row, the columns at constant offsets; rows and columns outside the level are clipped
            const int xlim = min(kTcTileX, tl.np - tl.PX0), ylim = min(kTcTileY, tl.np - tl.PY0);
            const size_t ystride = (size_t)4 * tl.side * P;  // floats between tile rows (two box rows)
            constexpr int XS = 4 * P;                         // floats between neighbouring parents' boxes
#pragma unroll 1
            for (int mt = 0; mt < C::MT; ++mt) {
                const int R = mt * 128 + q4 * 32 + lane;  // output row (c, n, re/im)
                const bool valid_row = R < 8 * P;
                const int c = valid_row ? R / (2 * P) : 0, q = R % (2 * P);
                float* base = reinterpret_cast<float*>(tl.L + ((size_t)(2 * tl.PY0 + (c >> 1)) * tl.side +
                                                               2 * tl.PX0 + (c & 1)) * P) + q;
                const uint32_t dcol = tmem + lanes + (uint32_t)(d * C::DCOLS + mt * C::N);
#pragma unroll 1
                for (int j0 = 0; j0 < C::N && j0 / kTcTileX < ylim; j0 += 32) {
                    uint32_t r[32];
                    tmem_ld16_async(dcol + (uint32_t)j0, *reinterpret_cast<uint32_t(*)[16]>(&r[0]));
                    tmem_ld16_async(dcol + (uint32_t)(j0 + 16), *reinterpret_cast<uint32_t(*)[16]>(&r[16]));
                    tmem_wait_ld();
                    if (!valid_row) continue;
#pragma unroll
                    for (int yy = 0; yy < 4; ++yy) {
                        const int y = j0 / kTcTileX + yy;
                        if (y >= ylim) break;
                        float* b = base + (size_t)y * ystride;
                        if (xlim == kTcTileX && !adapt) {
                            if (head) {
                                if (job.accumulate) {
                                    float old[kTcTileX];
#pragma unroll
                                    for (int x = 0; x < kTcTileX; ++x) old[x] = b[x * XS];
#pragma unroll
                                    for (int x = 0; x < kTcTileX; ++x) b[x * XS] = old[x] + __uint_as_float(r[8 * yy + x]);
                                } else {
#pragma unroll
                                    for (int x = 0; x < kTcTileX; ++x) b[x * XS] = __uint_as_float(r[8 * yy + x]);
                                }
                            } else {
#pragma unroll
                                for (int x = 0; x < kTcTileX; ++x) atomicAdd(b + x * XS, __uint_as_float(r[8 * yy + x]));
                            }
                        } else {
                            const uint32_t tm = adapt ? s_tmask[c * 32 + y] : 0xFFu;
#pragma unroll
                            for (int x = 0; x < kTcTileX; ++x) {
                                if (x >= xlim) break;
                                if (!((tm >> x) & 1u)) continue;  // absent target (adaptive level)
                                const float o = __uint_as_float(r[8 * yy + x]);
                                if (!head) atomicAdd(b + x * XS, o);
                                else b[x * XS] = job.accumulate ? o + b[x * XS] : o;
                            }
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&dfree[d]);
            if (head && !whole) {
                // publish the head: every writer's stores, then one release of the tile's flag
                __threadfence();
                asm volatile("bar.sync %0, %1;" ::"n"(kPubBar), "n"(128) : "memory");
                if (q4 == 0 && lane == 0)
                    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(flags + sg.t), "r"(1) : "memory");
            }
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == kMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)C::TMEM_COLS)
                     : "memory");
    // the last CTA to finish clears the flags and the counter for the next launch
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(done, 1) == grid - 1) {
            for (int j = 0; j < (units >> 5); ++j) flags[j] = 0;
            __threadfence();
            atomicExch(done, 0);
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
bool m2l_tc_supported(int p) { return p == 16 || p == 24; }

// TF32 operands double the halo and operator bytes: they fit shared memory at p = 16 only
bool m2l_tc_tf32_supported(int p) { return p == 16; }

size_t m2l_tc_image_bytes(int p, bool tf32)
{
    if (tf32) return p == 16 ? (size_t)kTcReplicas * kTcBlocks * 2 * TcCfg<16, true>::APART : 0;
    switch (p) {
        case 16: return (size_t)kTcReplicas * kTcBlocks * 2 * TcCfg<16>::APART;
        case 24: return (size_t)kTcReplicas * kTcBlocks * 2 * TcCfg<24>::APART;
        default: return 0;
    }
}

template <int P, bool TF>
static int build_image_p(double s, int variant, unsigned char* img, cudaStream_t st)
{
    using C = TcCfg<P, TF>;
    const int64_t total = (int64_t)kTcBlocks * C::MT * 128 * C::K2;
    build_tc_image_kernel<P, TF><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(s, variant, img);
    FMM_CUDA_TRY(cudaGetLastError());
    const size_t one = (size_t)kTcBlocks * 2 * C::APART;
    for (int r = 1; r < kTcReplicas; ++r) FMM_CUDA_TRY(cudaMemcpyAsync(img + r * one, img, one, cudaMemcpyDeviceToDevice, st));
    return FMM_OK;
}

int launch_build_tc_image(int p, double s, int variant, bool tf32, void* img, cudaStream_t st)
{
    if (tf32) {
        if (p == 16) return build_image_p<16, true>(s, variant, (unsigned char*)img, st);
        return fail(FMM_EUNSUPPORTED, "M2L TC TF32x3: unsupported p = %d (16)", p);
    }
    switch (p) {
        case 16: return build_image_p<16, false>(s, variant, (unsigned char*)img, st);
        case 24: return build_image_p<24, false>(s, variant, (unsigned char*)img, st);
        default: return fail(FMM_EINVAL, "M2L TC: unsupported p = %d", p);
    }
}

// cuTensorMapEncodeTiled from the CUDA driver API, looked up once (no link against libcuda)
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

template <int P, bool TF>
static int launch_tc_p(M2LLaunch& job, const void* img, bool split, int* err, cudaStream_t st)
{
    using C = TcCfg<P, TF>;
    int total = 0;
    for (int i = 0; i < job.nlev; ++i) {
        job.lv[i].tile_begin = total;
        const int np = 1 << (job.lv[i].level - 1);
        total += job.lv[i].tc_tiles ? job.lv[i].tc_ntiles
                                    : ((np + kTcTileX - 1) / kTcTileX) * ((np + kTcTileY - 1) / kTcTileY);
    }
    if (total == 0) return FMM_OK;
    int sms = 0;
    int rc = device_sm_count(&sms);
    if (rc) return rc;
    const int units = total * kTcBlocks;
    int grid = units / kTcMinUnits;
    grid = grid < 1 ? 1 : (grid > sms ? sms : grid);
    int* flags = nullptr;
    if ((rc = tc_flag_workspace(total, &flags))) return rc;
    int* ctr = nullptr;
    if ((rc = tile_counter(&ctr, st))) return rc;
    TcMaps maps;
    memset(&maps, 0, sizeof(maps));
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    for (int i = 0; i < job.nlev; ++i) {
        const int np = 1 << (job.lv[i].level - 1);
        const int side = 2 * np;
        if (!encode || job.periodic) continue;  // periodic lists wrap: global loads
        // MEs [iy][ix][2p floats] read as [qy][cy][qx][cx][2p]: box (2 qx + cx, 2 qy + cy)
        const cuuint64_t dims[5] = {(cuuint64_t)(2 * P), 2, (cuuint64_t)np, 2, (cuuint64_t)np};
        const cuuint64_t rowb = (cuuint64_t)side * 2 * P * 4;  // bytes per box row
        const cuuint64_t strides[4] = {(cuuint64_t)2 * P * 4, (cuuint64_t)4 * P * 4, rowb, 2 * rowb};
        const cuuint32_t box[5] = {(cuuint32_t)(2 * P), 1, (cuuint32_t)C::HX, 1, (cuuint32_t)C::HY};
        const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
        const CUresult r = encode(&maps.map[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, (void*)job.lv[i].M, dims, strides,
                                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            // a level smaller than the box may be refused: its halos are then read from global memory
            if (np < C::HX || np < C::HY) continue;
            return fail(FMM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
        }
        maps.use_tma[i] = 1;
    }
    static unsigned long long opted;
    if ((rc = smem_opt_in((const void*)m2l_tc_kernel<P, TF>, (int)C::smem, &opted))) return rc;
    m2l_tc_kernel<P, TF><<<grid, kTcCtaThreads, C::smem, st>>>(job, maps, (const unsigned char*)img, split ? 1 : 0,
                                                                units, flags, ctr + 1, err);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

int launch_m2l_tc(M2LLaunch& job, int p, const void* img, bool split, bool tf32, cudaStream_t st)
{
    int* err = nullptr;
    int rc = device_error_word(&err);
    if (rc) return rc;
    if (tf32) {
        if (p == 16) return launch_tc_p<16, true>(job, img, true, err, st);
        return fail(FMM_EUNSUPPORTED, "M2L TC TF32x3: unsupported p = %d (16)", p);
    }
    switch (p) {
        case 16: return launch_tc_p<16, false>(job, img, split, err, st);
        case 24: return launch_tc_p<24, false>(job, img, split, err, st);
        default: return fail(FMM_EINVAL, "M2L TC: unsupported p = %d", p);
    }
}

}  // namespace fmmgb
