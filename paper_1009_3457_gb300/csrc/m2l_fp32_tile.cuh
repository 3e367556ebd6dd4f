// m2l_fp32_tile.cuh -- the FP32 M2L work unit shared by the per-level stencil
// kernel (m2l_fp32.cu) and the batched persistent kernel (m2l_batched.cu):
// one CTA translates and reduces every interaction list of the 64 target boxes
// of a 4 x 4 tile of parent boxes of one uniform level (Sec. 4.1 steps 2-3,
// Eq. M2Lmat).
//
// Formulation (radius-scaled units, D = (x_t - x_s)/r a complex integer):
//   L~_t[n] = sum_{s in IL(t)} sum_k a_n h_D[n+k] b_k M~_s[k]
//           = a_n * sum_{s} sum_k h_D[n+k] (b_k M~_s[k])
// so each translation is a Hankel matrix-vector product between two diagonal
// scalings that do not depend on the offset: b_k is applied once per source
// box while it is staged into shared memory, a_n once per target box at the
// store.  Because the matrix is Hankel, a thread that owns RN consecutive
// rows n0..n0+RN-1 needs one new operator value h[n0+RN+k] per k (a sliding
// register window) instead of a column of the p x p matrix.
//
// Work unit (GB300-first; replaces the paper's thread-per-row, source-centric
// kernel and its separate reduction kernel, Sec. 4.1.1):
//   - the parent halo (tile + 1 on each side) holds every source any of the
//     64 targets needs; each source ME is read once per tile (coalesced
//     16-byte loads), scaled by b_k and reused by up to 27 targets;
//   - the halo is stored in shared memory split by child class
//     c' = (ix & 1) + 2 (iy & 1) and transposed to [c'][k][hy][hx], so that
//     for a target class c every interaction-list entry is a constant shift
//     (ex, ey) inside one class plane;
//   - warp w handles the 16 targets of child class c = w, whose 27 list
//     offsets are therefore warp-uniform; lane = (half, target): for p <= 16
//     a lane keeps all p rows of its target and the two half-warps take 14
//     and 13 of the 27 list entries (one shuffle adds the halves), so each k
//     step costs two shared loads per 4p FFMA; for p = 24 the halves split
//     the rows instead (register budget);
//   - the reduction over the list is a register accumulation, written once
//     per target (no separate reduction kernel, no atomics: deterministic).
#pragma once

#include "common.cuh"

namespace fmmgb {

constexpr int kThreads = 128;  // 4 warps, one per target child class
constexpr int kTile = 4;       // parent boxes per tile side
constexpr int kHalo = kTile + 2;
constexpr int kPlane = kHalo * kHalo + 1;  // float2 stride between k-planes

template <int P>
struct M2LCfg {
    // packed two-lane FP32 (f32x2) multiply-adds, the half-warps split the rows
    static constexpr bool PACKED = P >= 6 && P <= 24;
    static constexpr bool SPLIT_ROWS = P > 16 || PACKED;
    static constexpr int RN = SPLIT_ROWS ? P / 2 : P;  // rows per lane
    static constexpr int NH = 2 * P - 1;           // Hankel diagonals
    static constexpr int CS = P * kPlane;          // float2 stride between class planes
    static constexpr int HALO = 4 * CS;            // float2 per halo buffer
    static constexpr int MIN_CTAS = P == 16 ? 7 : 1;  // p = 16: 7 resident CTAs per SM (<= 72 registers)
    // halo loads a thread keeps in flight while staging a tile (register budget of the order)
    static constexpr int LOADS = P <= 6 ? 2 : (P <= 8 ? 3 : 4);
    static constexpr size_t smem = sizeof(float2) * (HALO + kOffsetSlots * NH) + sizeof(float) * 2 * P +
                                   sizeof(int2) * 4 * 27;
};

__device__ __forceinline__ void cmac(float2& acc, const float2 w, const float2 m)
{
    acc.x = fmaf(w.x, m.x, acc.x);
    acc.x = fmaf(-w.y, m.y, acc.x);
    acc.y = fmaf(w.x, m.y, acc.y);
    acc.y = fmaf(w.y, m.x, acc.y);
}

// Packed two-lane FP32 (PTX f32x2): a complex number is one 64-bit register
// pair (re, im), so acc += w m is two packed multiply-adds,
//   acc += (w.x, w.y) (m.x, m.x) + (-w.y, w.x) (m.y, m.y),
// each issuing the work of two FFMAs in one slot.
__device__ __forceinline__ unsigned long long pk2(float a, float b)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long v)
{
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Number of 4 x 4-parent tiles of a level (levels 0 and 1 have no lists).
__host__ __device__ inline int m2l_tiles(int level)
{
    if (level < 2) return 0;
    const int np = 1 << (level - 1);
    const int t = (np + kTile - 1) / kTile;
    return t * t;
}

// One tile of one level: its coefficient arrays, its first parent box and,
// on an adaptive level, which boxes exist (NULL: all of them).
struct TileGeom {
    const float2* M;
    float2* L;
    const uint8_t* exists;
    int side, np, PX0, PY0;
};

__device__ __forceinline__ TileGeom tile_geom_of(const float2* M, float2* L, const uint8_t* exists, int level, int t)
{
    TileGeom g;
    g.M = M;
    g.L = L;
    g.exists = exists;
    g.side = 1 << level;
    g.np = g.side >> 1;
    const int tpr = (g.np + kTile - 1) / kTile;
    g.PX0 = (t % tpr) * kTile;
    g.PY0 = (t / tpr) * kTile;
    return g;
}

// Shared-memory layout of the work unit for order P.
template <int P>
struct TileSmem {
    float2* buf;  // [4][P][kPlane] class-split halo
    float2* hs;   // [49][NH] Hankel operator values
    float* as;    // [P] post-scale
    float* bs;    // [P] pre-scale
    int2* lst;    // [4][27]: (Hankel row offset, halo offset) per target class
    __device__ __forceinline__ explicit TileSmem(unsigned char* raw)
    {
        using C = M2LCfg<P>;
        buf = reinterpret_cast<float2*>(raw);
        hs = buf + C::HALO;
        as = reinterpret_cast<float*>(hs + kOffsetSlots * C::NH);
        bs = as + P;
        lst = reinterpret_cast<int2*>(bs + P);
    }
};

// Load the operator tables of order P and the per-class list stencils into
// shared memory.  The caller synchronises before the next m2l_tile.
template <int P>
__device__ __forceinline__ void m2l_load_operator(unsigned char* raw, const float2* __restrict__ hsel,
                                                  const float* __restrict__ ascale, const float* __restrict__ bscale)
{
    using C = M2LCfg<P>;
    constexpr int NH = C::NH;
    const TileSmem<P> s(raw);
    const int tid = threadIdx.x;
    // 16-byte copies, several in flight per thread (the table and the shared-memory
    // copy are 16-byte aligned): the copy is on every launch's critical path
    constexpr int N4 = kOffsetSlots * NH / 2;
    const float4* h4 = reinterpret_cast<const float4*>(hsel);
    float4* d4 = reinterpret_cast<float4*>(s.hs);
#pragma unroll 4
    for (int i = tid; i < N4; i += kThreads) d4[i] = __ldg(h4 + i);
    if ((kOffsetSlots * NH) & 1)
        if (tid == 0) s.hs[kOffsetSlots * NH - 1] = hsel[kOffsetSlots * NH - 1];
    for (int i = tid; i < P; i += kThreads) {
        s.as[i] = ascale[i];
        s.bs[i] = bscale[i];
    }
    if (tid < 4) {  // the 27 interaction-list entries of child class tid, in (ey, ex, c') order
        const int cx = tid & 1, cy = tid >> 1;
        int n = 0;
        for (int e = 0; e < 36; ++e) {
            const int sx = e & 1, sy = (e >> 1) & 1, pe = e >> 2;
            const int ex = pe % 3 - 1, ey = pe / 3 - 1;
            const int dx = 2 * ex + sx - cx, dy = 2 * ey + sy - cy;
            const int adx = dx < 0 ? -dx : dx, ady = dy < 0 ? -dy : dy;
            if ((adx > ady ? adx : ady) < 2) continue;  // adjacent: near field
            s.lst[tid * 27 + n++] = make_int2(offset_slot(dx, dy) * NH, (sx + 2 * sy) * C::CS + (ey + 1) * kHalo + (ex + 1));
        }
    }
}

// How a warp's lanes share the work of its 16 targets (two lanes per target):
//   kFormRowsPacked  each lane p/2 rows, all 27 list entries, packed f32x2 multiply-adds;
//   kFormEntries     each lane all p rows, 14 or 13 of the 27 entries, one shuffle adds the halves;
//   kFormRows        each lane p/2 rows, all 27 entries, scalar FFMAs;
//   kFormRowsPacked2 as kFormRowsPacked, with the sums of w m.re and of w m.im in separate
//                    packed accumulators (no (-w.im, w.re) copy of the operator window);
//   kFormAuto        the order's default: packed rows with separate sums at p = 12, 16, 24
//                    (measured faster there, slower at p = 8), packed rows at p = 6, 8.
enum : int { kFormAuto = -1, kFormRowsPacked = 0, kFormEntries = 1, kFormRows = 2, kFormRowsPacked2 = 3 };

// Translate and reduce one tile (ADAPTIVE and g.exists set: only existing
// sources are read and existing targets written).  Requires the operator of order P in shared
// memory (m2l_load_operator + a barrier) and no thread still reading the halo
// buffer of a previous tile (a barrier).  All 128 threads call it.
template <int P, bool ADAPTIVE = false, int UMAX = M2LCfg<P>::LOADS, int FORM = kFormAuto>
__device__ __forceinline__ void m2l_tile(unsigned char* raw, const TileGeom& g, int periodic, int accumulate)
{
    using C = M2LCfg<P>;
    constexpr int F = FORM != kFormAuto ? FORM
                                        : (C::PACKED ? (P >= 12 ? kFormRowsPacked2 : kFormRowsPacked)
                                                     : (C::SPLIT_ROWS ? kFormRows : kFormEntries));
    constexpr bool SPLIT = F != kFormEntries;
    constexpr int RN = SPLIT ? P / 2 : P, Q = P / 2;
    const TileSmem<P> s(raw);
    const int tid = threadIdx.x;

    // Stage the 2 kHalo x 2 kHalo halo boxes, pre-scaled by b_k, into the
    // class-split transposed layout; consecutive threads read consecutive
    // 16-byte chunks of a row of boxes (coalesced); zero outside the level.
    // Each thread first issues up to U (<= UMAX, a register budget) loads, then scales
    // and stores them, so that a tile's staging costs a memory round trip or two
    // instead of one per chunk.
    const float4* M4 = reinterpret_cast<const float4*>(g.M);
    constexpr int NCH = (2 * kHalo) * (2 * kHalo) * Q;  // 16-byte chunks of the halo
    constexpr int U = (NCH + kThreads - 1) / kThreads < UMAX ? (NCH + kThreads - 1) / kThreads : UMAX;
    for (int i0 = tid; i0 < NCH; i0 += U * kThreads) {
        float4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * kThreads;
            v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i >= NCH) continue;
            const int q = i % Q, bxy = i / Q;
            const int hxb = bxy % (2 * kHalo), hyb = bxy / (2 * kHalo);
            int ix = 2 * g.PX0 - 2 + hxb, iy = 2 * g.PY0 - 2 + hyb;
            bool in = ix >= 0 && iy >= 0 && ix < g.side && iy < g.side;
            if (periodic) {
                ix = (ix + 2 * g.side) % g.side;
                iy = (iy + 2 * g.side) % g.side;
                in = true;
            }
            if constexpr (ADAPTIVE)
                if (in && g.exists) in = g.exists[(size_t)iy * g.side + ix] != 0;  // V-list: existing sources only
            if (in) v[u] = __ldg(M4 + ((size_t)iy * g.side + ix) * Q + q);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * kThreads;
            if (i >= NCH) continue;
            const int q = i % Q, bxy = i / Q;
            const int hxb = bxy % (2 * kHalo), hyb = bxy / (2 * kHalo);
            float2* dst = s.buf + ((hxb & 1) + 2 * (hyb & 1)) * C::CS + (hyb >> 1) * kHalo + (hxb >> 1);
            const float b0 = s.bs[2 * q], b1 = s.bs[2 * q + 1];
            dst[(2 * q) * kPlane] = make_float2(v[u].x * b0, v[u].y * b0);
            dst[(2 * q + 1) * kPlane] = make_float2(v[u].z * b1, v[u].w * b1);
        }
    }
    __syncthreads();

    const int warp = tid >> 5, lane = tid & 31;
    const int cls = warp, cx = warp & 1, cy = warp >> 1;
    const int half = lane >> 4, t = lane & 15;
    const int tpx = t & 3, tpy = t >> 2;
    const int2* mylist = s.lst + cls * 27;

    // On an adaptive level a warp (one child class, 16 targets) whose targets
    // are all absent skips the translation; the vote is warp-uniform.
    const int px = g.PX0 + tpx, py = g.PY0 + tpy;
    bool target = px < g.np && py < g.np;
    if constexpr (ADAPTIVE)
        if (target && g.exists) target = g.exists[(size_t)(2 * py + cy) * g.side + 2 * px + cx] != 0;
    bool work = true;
    if constexpr (ADAPTIVE) work = __any_sync(0xffffffffu, target);

    // ---- translate and reduce ----
    float2 acc[RN];
#pragma unroll
    for (int i = 0; i < RN; ++i) acc[i] = make_float2(0.f, 0.f);
    const float2* tbase = s.buf + tpy * kHalo + tpx;
    if (!work) {
        // nothing to store for this warp
    } else if constexpr (!SPLIT) {
        // half-warp `half` takes list entries [14 half, 14 half + 14) of 27; all p rows
#pragma unroll 1
        for (int j = 0; j < 14; ++j) {
            const int e = half * 14 + j;
            if (e >= 27) break;
            const int2 ent = mylist[e];
            const float2* hrow = s.hs + ent.x;
            const float2* src = tbase + ent.y;
            float2 w[RN];
#pragma unroll
            for (int i = 0; i < RN; ++i) w[i] = hrow[i];
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const float2 m = src[k * kPlane];
#pragma unroll
                for (int i = 0; i < RN; ++i) cmac(acc[i], w[i], m);
                if (k + 1 < P) {
#pragma unroll
                    for (int i = 0; i + 1 < RN; ++i) w[i] = w[i + 1];
                    w[RN - 1] = hrow[RN + k];
                }
            }
        }
    } else if constexpr (F == kFormRowsPacked) {
        // half-warp `half` takes rows [RN half, RN half + RN); all 27 entries; packed
        // accumulators and operator window (w and i w), m broadcast per k
        const int n0 = half * RN;
        unsigned long long pacc[RN];
#pragma unroll
        for (int i = 0; i < RN; ++i) pacc[i] = 0ull;
#pragma unroll 1
        for (int e = 0; e < 27; ++e) {
            const int2 ent = mylist[e];
            const float2* hrow = s.hs + ent.x + n0;
            const float2* src = tbase + ent.y;
            unsigned long long w[RN], wr[RN];
#pragma unroll
            for (int i = 0; i < RN; ++i) {
                const float2 h = hrow[i];
                w[i] = pk2(h.x, h.y);
                wr[i] = pk2(-h.y, h.x);
            }
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const float2 m = src[k * kPlane];
                const unsigned long long mx = pk2(m.x, m.x), my = pk2(m.y, m.y);
#pragma unroll
                for (int i = 0; i < RN; ++i) pacc[i] = fma2(wr[i], my, fma2(w[i], mx, pacc[i]));
                if (k + 1 < P) {
#pragma unroll
                    for (int i = 0; i + 1 < RN; ++i) {
                        w[i] = w[i + 1];
                        wr[i] = wr[i + 1];
                    }
                    const float2 h = hrow[RN + k];
                    w[RN - 1] = pk2(h.x, h.y);
                    wr[RN - 1] = pk2(-h.y, h.x);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < RN; ++i) acc[i] = upk2(pacc[i]);
    } else if constexpr (F == kFormRowsPacked2) {
        // as above; acc = sum w m.re + i sum w m.im, the two sums in separate packed accumulators
        const int n0 = half * RN;
        unsigned long long pa[RN], pb[RN];
#pragma unroll
        for (int i = 0; i < RN; ++i) pa[i] = pb[i] = 0ull;
        // two list entries per iteration: the next entry's list item and operator window load
        // while the current one's multiply-adds run (measured ~3 % at p = 12 and 16)
#pragma unroll 2
        for (int e = 0; e < 27; ++e) {
            const int2 ent = mylist[e];
            const float2* hrow = s.hs + ent.x + n0;
            const float2* src = tbase + ent.y;
            unsigned long long w[RN];
#pragma unroll
            for (int i = 0; i < RN; ++i) {
                const float2 h = hrow[i];
                w[i] = pk2(h.x, h.y);
            }
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const float2 m = src[k * kPlane];
                const unsigned long long mx = pk2(m.x, m.x), my = pk2(m.y, m.y);
#pragma unroll
                for (int i = 0; i < RN; ++i) {
                    pa[i] = fma2(w[i], mx, pa[i]);
                    pb[i] = fma2(w[i], my, pb[i]);
                }
                if (k + 1 < P) {
#pragma unroll
                    for (int i = 0; i + 1 < RN; ++i) w[i] = w[i + 1];
                    const float2 h = hrow[RN + k];
                    w[RN - 1] = pk2(h.x, h.y);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < RN; ++i) {
            const float2 a = upk2(pa[i]), b = upk2(pb[i]);
            acc[i] = make_float2(a.x - b.y, a.y + b.x);
        }
    } else {
        // half-warp `half` takes rows [RN half, RN half + RN); all 27 entries
        const int n0 = half * RN;
#pragma unroll 1
        for (int e = 0; e < 27; ++e) {
            const int2 ent = mylist[e];
            const float2* hrow = s.hs + ent.x + n0;
            const float2* src = tbase + ent.y;
            float2 w[RN];
#pragma unroll
            for (int i = 0; i < RN; ++i) w[i] = hrow[i];
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const float2 m = src[k * kPlane];
#pragma unroll
                for (int i = 0; i < RN; ++i) cmac(acc[i], w[i], m);
                if (k + 1 < P) {
#pragma unroll
                    for (int i = 0; i + 1 < RN; ++i) w[i] = w[i + 1];
                    w[RN - 1] = hrow[RN + k];
                }
            }
        }
    }

    // ---- combine the half-warps: each lane ends with p/2 finished rows ----
    constexpr int HR = P / 2;
    float2 res[HR];
    if constexpr (!SPLIT) {
#pragma unroll
        for (int i = 0; i < HR; ++i) {
            const float2 send = half ? acc[i] : acc[HR + i];
            const float2 mine = half ? acc[HR + i] : acc[i];
            float2 r;
            r.x = __shfl_xor_sync(0xffffffffu, send.x, 16);
            r.y = __shfl_xor_sync(0xffffffffu, send.y, 16);
            res[i] = make_float2(mine.x + r.x, mine.y + r.y);
        }
    } else {
#pragma unroll
        for (int i = 0; i < HR; ++i) res[i] = acc[i];
    }

    // ---- store L~[n] = a_n * res (rows [HR half, HR half + HR)) ----
    if (target) {
        const int ix = 2 * px + cx, iy = 2 * py + cy;
        const int n0 = half * HR;
        float2* dst = g.L + ((size_t)iy * g.side + ix) * P + n0;
        if constexpr (HR % 2 == 0) {
            float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
            for (int i = 0; i < HR; i += 2) {
                const float s0 = s.as[n0 + i], s1 = s.as[n0 + i + 1];
                float4 o = make_float4(s0 * res[i].x, s0 * res[i].y, s1 * res[i + 1].x, s1 * res[i + 1].y);
                if (accumulate) {
                    const float4 old = d4[i / 2];
                    o.x += old.x;
                    o.y += old.y;
                    o.z += old.z;
                    o.w += old.w;
                }
                d4[i / 2] = o;
            }
        } else {
#pragma unroll
            for (int i = 0; i < HR; ++i) {
                const float s0 = s.as[n0 + i];
                float2 o = make_float2(s0 * res[i].x, s0 * res[i].y);
                if (accumulate) {
                    const float2 old = dst[i];
                    o.x += old.x;
                    o.y += old.y;
                }
                dst[i] = o;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// stencil kernel: every requested level in one launch, tiles ordered heaviest
// level first.  Persistent when `counter` is set: each resident CTA (6 per SM
// at p = 16) loads the operator once, takes its first tile by blockIdx and
// claims the next from the work counter (counter[0]; counter[1] counts the
// CTAs that finished, and the last one resets both), so the operator table is staged
// once per CTA instead of once per tile and no second round of CTAs leaves
// SMs half empty at the end.  With counter == NULL the grid covers every
// tile, one CTA each.
// ---------------------------------------------------------------------------
template <int P, bool ADAPTIVE>
__global__ void __launch_bounds__(kThreads, M2LCfg<P>::MIN_CTAS)
    m2l_fp32_kernel(M2LLaunch job, const float2* __restrict__ hsel, const float* __restrict__ ascale,
                    const float* __restrict__ bscale, int total, int* __restrict__ counter)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_next;
    m2l_load_operator<P>(smem_raw, hsel, ascale, bscale);
    int tile = blockIdx.x;
    while (tile < total) {
        int li = 0;
        while (li + 1 < job.nlev && tile >= job.lv[li + 1].tile_begin) ++li;
        const M2LLevel& lv = job.lv[li];
        int t = tile - lv.tile_begin;
        if constexpr (ADAPTIVE)
            if (lv.tiles) t = lv.tiles[t];  // the level's tiles that hold an existing box
        const TileGeom g = tile_geom_of(lv.M, lv.L, ADAPTIVE ? lv.exists : nullptr, lv.level, t);
        __syncthreads();  // operator visible; the previous tile is done with the halo buffer
        m2l_tile<P, ADAPTIVE>(smem_raw, g, job.periodic, job.accumulate);
        if (!counter) break;
        // every thread read s_next of the previous claim before the barrier inside m2l_tile
        if (threadIdx.x == 0) s_next = (int)gridDim.x + atomicAdd(counter, 1);
        __syncthreads();
        tile = s_next;
    }
    // the last CTA to finish returns the counter slot to zero for its next use
    if (counter && threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(counter + 1, 1) == (int)gridDim.x - 1) {
            atomicExch(counter, 0);
            atomicExch(counter + 1, 0);
        }
    }
}

}  // namespace fmmgb
