// m2l_fp32.cu -- FP32 M2L with the reduction fused in, over one or several
// levels of a uniform quadtree in one launch (Sec. 4.1 steps 2-3, Eq. M2Lmat),
// plus the FP64 operator-table builder.
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
// Work decomposition (GB300-first; replaces the paper's thread-per-row,
// source-centric kernel and its separate reduction kernel, Sec. 4.1.1):
//   - a CTA owns an 8 x 4 tile of parent boxes = 128 target boxes of one level
//     (4 x 4 tile for p = 24); one launch covers every tile of every requested
//     level (heaviest level first), so the ~680 CTAs of the level 2..8 pass are
//     resident in one wave (5 CTAs per SM at p = 16) and one CTA's staging
//     overlaps the others' arithmetic;
//   - the parent halo (tile + 1 on each side) holds every source any target
//     needs; each source ME is read once per tile and reused by up to 27
//     targets;
//   - the halo is stored in shared memory split by child class
//     c' = (ix & 1) + 2 (iy & 1) and transposed to [c'][k][hy][hx], so that
//     for a target class c every interaction-list entry is a constant shift
//     (ex, ey) inside one class plane;
//   - warp w handles the targets of child class c = w, whose 27 list offsets
//     are therefore warp-uniform (no divergence); a lane owns all p rows of
//     one target (two lanes of p/2 rows each for p = 24), so each k step costs
//     two shared loads (one ME value, one new Hankel value) per 4p FFMA;
//   - the reduction over the list is a register accumulation, written once
//     per target (no separate reduction kernel, no atomics: deterministic).
#include "common.cuh"

namespace fmmgb {

// ---------------------------------------------------------------------------
// operator tables, computed in FP64 on the GPU, stored as FP32
// ---------------------------------------------------------------------------
__global__ void build_m2l_tables_kernel(int p, double s, float2* __restrict__ hf, float2* __restrict__ ha,
                                        float2* __restrict__ hac, float* __restrict__ a, float* __restrict__ b)
{
    const int nh = 2 * p - 1;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < kOffsetSlots * nh) {
        const int slot = idx / nh, j = idx % nh;
        const int dx = slot % 7 - 3, dy = slot / 7 - 3;
        const int adx = dx < 0 ? -dx : dx, ady = dy < 0 ? -dy : dy;
        float2 v = make_float2(0.f, 0.f);
        if ((adx > ady ? adx : ady) >= 2) {
            // D = x_t - x_s in box units = -(dx + i dy);  h = j! s^j D^-(j+1)
            const double Dr = -(double)dx, Di = -(double)dy;
            const double den = Dr * Dr + Di * Di;
            const double ir = Dr / den, ii = -Di / den;  // 1/D
            double hr = ir, hi = ii;
            for (int i = 1; i <= j; ++i) {
                const double f = (double)i * s;
                const double nr = (hr * ir - hi * ii) * f;
                const double ni = (hr * ii + hi * ir) * f;
                hr = nr;
                hi = ni;
            }
            v = make_float2((float)hr, (float)hi);
        }
        hf[idx] = v;
        ha[idx] = make_float2(-v.x, -v.y);
        hac[idx] = make_float2(-v.x, v.y);
    }
    if (idx < p) {
        double fact = 1.0, sp = 1.0;
        for (int i = 1; i <= idx; ++i) {
            fact *= (double)i;
            sp *= s;
        }
        b[idx] = (float)(1.0 / (fact * sp));
        a[idx] = (float)(((idx & 1) ? -1.0 : 1.0) / (fact * sp));
    }
}

int launch_build_m2l_tables(const M2LTables& t, cudaStream_t st)
{
    const int n = kOffsetSlots * (2 * t.p - 1);
    build_m2l_tables_kernel<<<(n + 127) / 128, 128, 0, st>>>(t.p, t.s, t.h_fwd, t.h_adj, t.h_adjc, t.a, t.b);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

// ---------------------------------------------------------------------------
// stencil kernel
// ---------------------------------------------------------------------------
constexpr int kThreads = 128;  // 4 warps, one per target child class
constexpr int kTileY = 4;      // parent rows per tile

// NB = row blocks per target: NB = 1 (one lane = all p rows of one target,
// 8 x 4 parent tile, 32 targets per class) for p <= 16; NB = 2 (two lanes per
// target, 4 x 4 tile) for p = 24 to bound registers.
template <int P>
struct M2LCfg {
    static constexpr int NB = P <= 16 ? 1 : 2;
    static constexpr int TX = 8 / NB;                  // parent columns per tile
    static constexpr int HX = TX + 2, HY = kTileY + 2;  // halo parents
    static constexpr int PL = HX * HY + 1;            // float2 stride between k-planes
    static constexpr int RN = P / NB;                 // rows per lane
    static constexpr int NH = 2 * P - 1;              // Hankel diagonals
    static constexpr int CS = P * PL;                 // float2 stride between class planes
    static constexpr int Q = P / 2;                   // float4 per box
    static constexpr size_t smem = sizeof(float2) * (4 * CS + kOffsetSlots * NH) + sizeof(float) * 2 * P;
};

__device__ __forceinline__ void cmac(float2& acc, const float2 w, const float2 m)
{
    acc.x = fmaf(w.x, m.x, acc.x);
    acc.x = fmaf(-w.y, m.y, acc.x);
    acc.y = fmaf(w.x, m.y, acc.y);
    acc.y = fmaf(w.y, m.x, acc.y);
}

template <int P>
__host__ __device__ constexpr int m2l_tiles_p(int level)
{
    using C = M2LCfg<P>;
    if (level < 2) return 0;
    const int np = 1 << (level - 1);
    return ((np + C::TX - 1) / C::TX) * ((np + kTileY - 1) / kTileY);
}

template <int P>
__global__ void __launch_bounds__(kThreads) m2l_fp32_kernel(M2LLaunch job, const float2* __restrict__ hsel,
                                                            const float* __restrict__ ascale,
                                                            const float* __restrict__ bscale)
{
    using C = M2LCfg<P>;
    constexpr int NB = C::NB, TX = C::TX, HX = C::HX, HY = C::HY, PL = C::PL;
    constexpr int RN = C::RN, NH = C::NH, CS = C::CS, Q = C::Q;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* halo = reinterpret_cast<float2*>(smem_raw);  // [4][P][PL]
    float2* hs = halo + 4 * CS;                            // [49][NH]
    float* as = reinterpret_cast<float*>(hs + kOffsetSlots * NH);
    float* bs = as + P;

    // which level / tile this CTA owns (levels are listed heaviest first)
    int li = 0;
    while (li + 1 < job.nlev && (int)blockIdx.x >= job.lv[li + 1].tile_begin) ++li;
    const M2LLevel lv = job.lv[li];
    const int tile = (int)blockIdx.x - lv.tile_begin;
    const int side = 1 << lv.level;
    const int np = side >> 1;
    const int tpr = (np + TX - 1) / TX;  // tiles per row
    const int PX0 = (tile % tpr) * TX, PY0 = (tile / tpr) * kTileY;
    const int bx0 = 2 * PX0 - 2, by0 = 2 * PY0 - 2;  // first halo box (even)

    const int tid = threadIdx.x;
    for (int i = tid; i < kOffsetSlots * NH; i += kThreads) hs[i] = hsel[i];
    for (int i = tid; i < P; i += kThreads) {
        as[i] = ascale[i];
        bs[i] = bscale[i];
    }
    __syncthreads();

    // Stage the 2 HX x 2 HY halo boxes, pre-scaled by b_k, into the class-split
    // transposed layout.  Consecutive threads read consecutive 16-byte chunks of
    // a row of boxes (coalesced).
    const float4* M4 = reinterpret_cast<const float4*>(lv.M);
    for (int i = tid; i < (2 * HX) * (2 * HY) * Q; i += kThreads) {
        const int q = i % Q;
        const int bxy = i / Q;
        const int hxb = bxy % (2 * HX), hyb = bxy / (2 * HX);
        int ix = bx0 + hxb, iy = by0 + hyb;
        bool inside = ix >= 0 && iy >= 0 && ix < side && iy < side;
        if (job.periodic) {
            ix = (ix + 2 * side) % side;
            iy = (iy + 2 * side) % side;
            inside = true;
        }
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (inside) v = __ldg(M4 + ((size_t)iy * side + ix) * Q + q);
        const int cls = (hxb & 1) + 2 * (hyb & 1);
        float2* dst = halo + cls * CS + (hyb >> 1) * HX + (hxb >> 1);
        const float b0 = bs[2 * q], b1 = bs[2 * q + 1];
        dst[(2 * q) * PL] = make_float2(v.x * b0, v.y * b0);
        dst[(2 * q + 1) * PL] = make_float2(v.z * b1, v.w * b1);
    }
    __syncthreads();

    const int warp = tid >> 5, lane = tid & 31;
    const int cx = warp & 1, cy = warp >> 1;  // target child class
    const int i_n = lane % NB, i_t = lane / NB;
    const int n0 = i_n * RN;
    const int tpx = i_t % TX, tpy = i_t / TX;  // target parent within the tile

    float2 acc[RN];
#pragma unroll
    for (int i = 0; i < RN; ++i) acc[i] = make_float2(0.f, 0.f);

#pragma unroll 1
    for (int e = 0; e < 36; ++e) {
        // (parent offset, source child class): e = ((ey+1)*3 + (ex+1))*4 + sy*2 + sx
        const int sx = e & 1, sy = (e >> 1) & 1;
        const int pe = e >> 2;
        const int ex = pe % 3 - 1, ey = pe / 3 - 1;
        const int dx = 2 * ex + sx - cx, dy = 2 * ey + sy - cy;
        const int adx = dx < 0 ? -dx : dx, ady = dy < 0 ? -dy : dy;
        if ((adx > ady ? adx : ady) < 2) continue;  // adjacent: not in the interaction list (warp-uniform)

        const float2* hrow = hs + offset_slot(dx, dy) * NH + n0;
        const float2* src = halo + (sx + 2 * sy) * CS + (tpy + ey + 1) * HX + (tpx + ex + 1);
        float2 w[RN];
#pragma unroll
        for (int i = 0; i < RN; ++i) w[i] = hrow[i];
#pragma unroll
        for (int k = 0; k < P; ++k) {
            const float2 m = src[k * PL];
#pragma unroll
            for (int i = 0; i < RN; ++i) cmac(acc[i], w[i], m);
            if (k + 1 < P) {
#pragma unroll
                for (int i = 0; i + 1 < RN; ++i) w[i] = w[i + 1];
                w[RN - 1] = hrow[RN + k];
            }
        }
    }

    // store L~[n] = a_n * acc (the fused reduction's result)
    const int px = PX0 + tpx, py = PY0 + tpy;
    if (px >= np || py >= np) return;
    const int ix = 2 * px + cx, iy = 2 * py + cy;
    float2* dst = lv.L + ((size_t)iy * side + ix) * P + n0;
    if constexpr (RN % 2 == 0) {
        float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
        for (int i = 0; i < RN; i += 2) {
            const float s0 = as[n0 + i], s1 = as[n0 + i + 1];
            float4 o = make_float4(s0 * acc[i].x, s0 * acc[i].y, s1 * acc[i + 1].x, s1 * acc[i + 1].y);
            if (job.accumulate) {
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
        for (int i = 0; i < RN; ++i) {
            const float s0 = as[n0 + i];
            float2 o = make_float2(s0 * acc[i].x, s0 * acc[i].y);
            if (job.accumulate) {
                const float2 old = dst[i];
                o.x += old.x;
                o.y += old.y;
            }
            dst[i] = o;
        }
    }
}

bool m2l_fp32_supported(int p) { return p == 6 || p == 8 || p == 12 || p == 16 || p == 24; }

template <int P>
static int launch_p(M2LLaunch& job, const float2* h, const float* a, const float* b, cudaStream_t st)
{
    using C = M2LCfg<P>;
    int total = 0;
    for (int i = 0; i < job.nlev; ++i) {
        job.lv[i].tile_begin = total;
        total += m2l_tiles_p<P>(job.lv[i].level);
    }
    if (total == 0) return FMM_OK;
    FMM_CUDA_TRY(cudaFuncSetAttribute(m2l_fp32_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem));
    m2l_fp32_kernel<P><<<total, kThreads, C::smem, st>>>(job, h, a, b);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

int launch_m2l_fp32(M2LLaunch& job, int p, const float2* h, const float* a, const float* b, cudaStream_t st)
{
    switch (p) {
        case 6: return launch_p<6>(job, h, a, b, st);
        case 8: return launch_p<8>(job, h, a, b, st);
        case 12: return launch_p<12>(job, h, a, b, st);
        case 16: return launch_p<16>(job, h, a, b, st);
        case 24: return launch_p<24>(job, h, a, b, st);
        default: return fail(FMM_EINVAL, "M2L FP32: unsupported p = %d", p);
    }
}

}  // namespace fmmgb
