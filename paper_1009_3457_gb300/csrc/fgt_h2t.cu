// fgt_h2t.cu -- FGT Hermite-to-Taylor translation over a uniform box grid
// (Sec. 2.2, Eq. C_beta with the factor (-1)^|beta| / beta!):
//
//   C_t[b1][b2] = sum_{s : max(|sx-tx|, |sy-ty|) <= n_cut}
//                 ((-1)^(b1+b2) / (b1! b2!)) sum_{a1,a2} A_s[a1][a2] h_{a1+b1}(u1) h_{a2+b2}(u2),
//   u = (t_C - s_B) / (sqrt(2) sigma),  h_n(t) = exp(-t^2) H_n(t).
//
// In 2-D with tensor truncation the kernel factorises: h_{a+b}(u) is a Hankel
// matrix H(u) per axis, and the neighbourhood is a square, so the sum over
// source boxes splits into two 1-D stencils along x and y:
//
//   Y[x,y]  = S H-pass along x:  Y[b1][a2] = s_b1 sum_{dx} sum_{a1} h_{a1+b1}(u(dx)) A[x+dx, y][a1][a2]
//   C[x,y]  = S H-pass along y:  C[b1][b2] = s_b2 sum_{dy} sum_{a2} h_{a2+b2}(u(dy)) Y[x, y+dy][b1][a2]
//
// (s_b = (-1)^b / b!), which costs 2 (2 n_cut + 1) p^3 multiply-adds per box
// instead of (2 n_cut + 1)^2 2 p^3 for the box-pair form -- the same result up
// to rounding order.  Both passes run the same stencil kernel: out[box] =
// diag(s) sum_d H_d^T in[box + d e_axis], written transposed so that the second
// pass contracts the other Hermite index.  The Hermite-function values of the
// 2 n_cut + 1 offsets are computed once per (p, n_cut, sigma, grid) by an FP64
// kernel and cached per device (the allocation-free entry point computes them
// in every CTA instead).  The intermediate Y is library-owned
// scratch (one [4^g][p][p] float buffer per device, grown on demand).
#include <math.h>

#include <cooperative_groups.h>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace fmmgb {

constexpr int kFgtMaxCut = 16;   // largest n_cut accepted

// Thread mapping: (tap group, box of the segment, 4-row block, 4-column block);
// a thread accumulates a 4 x 4 block of one box's output over its group's share
// of the taps, and the groups' partial sums are reduced in shared memory.
// p = 16 runs segments of 8 boxes with 3 tap groups (384 threads): the halo of
// 2 n_cut boxes is staged once per 8 outputs.  Smaller p keep 4 boxes and 7
// groups, which give them enough warps per SM (at sigma = 0.05, 32 x 32 boxes,
// a pass of p = 8 is 256 CTAs of 112 threads).  Both shapes were timed on the
// sigma = 0.05 grid (n_cut = 10) against 2-32 boxes and 1-11 groups.
template <int P>
struct FgtCfg {
    static constexpr int SEG = P == 16 ? 8 : 4;     // boxes per CTA along the pass axis
    static constexpr int GROUPS = P == 16 ? 3 : 7;  // tap groups per box
    static constexpr int RB = 4;                // output rows (b) per thread
    static constexpr int RBLK = P / RB;         // row blocks per box
    static constexpr int CB = P / 4;            // column blocks of 4 per box
    static constexpr int TPB = RBLK * CB;       // threads per box and tap group
    static constexpr int THREADS = GROUPS * SEG * TPB;
    static constexpr int NH = 2 * P - 1;
    static constexpr int BS = P * P + 16;       // padded float stride between boxes in shared memory
    static_assert(P % 4 == 0 && BS % 4 == 0, "16-byte aligned float4 rows");
};

template <int P>
size_t fgt_smem_bytes(int ncut)
{
    using C = FgtCfg<P>;
    return sizeof(float) * ((size_t)(C::SEG + 2 * ncut) * C::BS + (size_t)(2 * ncut + 1) * C::NH + P +
                            (size_t)(C::GROUPS - 1) * C::SEG * P * P);
}

// Hermite-function values h_j(u_d), j < nh, u_d = -(d - ncut) * ustep (source
// offset d - ncut), by the recurrence h_{j+1} = 2u h_j - 2j h_{j-1}, in FP64.
__device__ __forceinline__ void fgt_hermite_row(int d, int ncut, int nh, double ustep, float* row)
{
    const double u = -(double)(d - ncut) * ustep;
    double hm = exp(-u * u), h = 2.0 * u * hm;
    row[0] = (float)hm;
    if (nh > 1) row[1] = (float)h;
    for (int j = 1; j + 1 < nh; ++j) {
        const double hn = 2.0 * u * h - 2.0 * (double)j * hm;
        hm = h;
        h = hn;
        row[j + 1] = (float)h;
    }
}

// The table of one (p, n_cut, step): [2 n_cut + 1][2p - 1], cached per device.
__global__ void fgt_table_kernel(int nh, int ncut, double ustep, float* __restrict__ tab)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d < 2 * ncut + 1) fgt_hermite_row(d, ncut, nh, ustep, tab + (size_t)d * nh);
}

template <int P>
__global__ void __launch_bounds__(FgtCfg<P>::THREADS) fgt_pass_kernel(int g, int ncut, double ustep, int axis,
                                                                      const float* __restrict__ in,
                                                                      float* __restrict__ out, int accumulate,
                                                                      const float* __restrict__ htab)
{
    using C = FgtCfg<P>;
    constexpr int RB = C::RB, NH = C::NH, BS = C::BS, SEG = C::SEG, GROUPS = C::GROUPS;
    extern __shared__ __align__(16) float fsm[];
    const int taps = 2 * ncut + 1;
    // float4-accessed arrays first: BS and P * P are multiples of 4 floats, so
    // halo and part start on 16-byte boundaries; the scalar tables follow
    float* halo = fsm;                                      // [SEG + 2 ncut][BS]
    float* part = halo + (size_t)(SEG + 2 * ncut) * BS;     // [GROUPS - 1][SEG][P][P]
    float* hs = part + (size_t)(GROUPS - 1) * SEG * P * P;  // [taps][NH]
    float* ss = hs + taps * NH;                                     // [P]

    const int side = 1 << g;
    const int seg0 = blockIdx.x * SEG;
    const int other = blockIdx.y;
    const int tid = threadIdx.x;
    // the second pass may be scheduled now: it prepares its tables and waits for this grid
    // (griddepcontrol.wait) before it reads what this pass writes
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    // Hermite-function table: the cached copy, or computed here (allocation-free entry point)
    if (htab) {
        for (int i = tid; i < taps * NH; i += blockDim.x) hs[i] = __ldg(htab + i);
    } else {
        for (int d = tid; d < taps; d += blockDim.x) fgt_hermite_row(d, ncut, NH, ustep, hs + d * NH);
    }
    for (int b = tid; b < P; b += blockDim.x) {
        double f = 1.0;
        for (int i = 2; i <= b; ++i) f *= (double)i;
        ss[b] = (float)(((b & 1) ? -1.0 : 1.0) / f);
    }
    // the input may come from the grid launched just before (the first pass): wait for it
    // (a no-op unless this grid was launched as its programmatic dependent)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // stage the boxes [seg0 - ncut, seg0 + SEG + ncut) of this row/column, zero outside the grid
    const int nhb = SEG + 2 * ncut;
    const float4* in4 = reinterpret_cast<const float4*>(in);
    for (int i = tid; i < nhb * (P * P / 4); i += blockDim.x) {  // every copy in flight before any wait
        const int q = i % (P * P / 4), hb = i / (P * P / 4);
        const int pos = seg0 - ncut + hb;
        const bool inside = pos >= 0 && pos < side;
        const size_t box = axis == 0 ? (size_t)other * side + pos : (size_t)pos * side + other;
        cp_async16(halo + (size_t)hb * BS + 4 * q, inside ? (const void*)(in4 + box * (P * P / 4) + q) : in, inside);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();

    const int grp = tid / (SEG * C::TPB);
    const int rem = tid % (SEG * C::TPB);
    const int j = rem / C::TPB;                  // box within the segment
    const int r = rem % C::TPB;
    const int b0 = (r % C::RBLK) * RB;           // first output row
    const int c0 = (r / C::RBLK) * 4;            // first of 4 columns
    const int pos = seg0 + j;
    const int per = (taps + GROUPS - 1) / GROUPS;
    const int d0 = grp * per, d1 = min(taps, d0 + per);

    float acc[RB][4];
#pragma unroll
    for (int i = 0; i < RB; ++i)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) acc[i][cc] = 0.f;

    if (pos < side) {
        for (int d = d0; d < d1; ++d) {
            const int spos = pos + d - ncut;
            if (spos < 0 || spos >= side) continue;
            const float* hrow = hs + d * NH + b0;
            const float* src = halo + (size_t)(j + d) * BS + c0;
            float w[RB];
#pragma unroll
            for (int i = 0; i < RB; ++i) w[i] = hrow[i];
#pragma unroll
            for (int a = 0; a < P; ++a) {
                const float4 v = *reinterpret_cast<const float4*>(src + a * P);
#pragma unroll
                for (int i = 0; i < RB; ++i) {
                    acc[i][0] = fmaf(w[i], v.x, acc[i][0]);
                    acc[i][1] = fmaf(w[i], v.y, acc[i][1]);
                    acc[i][2] = fmaf(w[i], v.z, acc[i][2]);
                    acc[i][3] = fmaf(w[i], v.w, acc[i][3]);
                }
                if (a + 1 < P) {
#pragma unroll
                    for (int i = 0; i + 1 < RB; ++i) w[i] = w[i + 1];
                    w[RB - 1] = hrow[RB + a];
                }
            }
        }
    }
    // tap groups 1.. hand their partial sums to group 0 through shared memory
    if (grp > 0) {
        float* pp = part + ((size_t)(grp - 1) * SEG + j) * (P * P);
#pragma unroll
        for (int i = 0; i < RB; ++i)
            *reinterpret_cast<float4*>(pp + (b0 + i) * P + c0) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    }
    __syncthreads();
    if (grp != 0 || pos >= side) return;
#pragma unroll
    for (int q = 0; q < GROUPS - 1; ++q) {
        const float* pp = part + ((size_t)q * SEG + j) * (P * P);
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            const float4 v = *reinterpret_cast<const float4*>(pp + (b0 + i) * P + c0);
            acc[i][0] += v.x;
            acc[i][1] += v.y;
            acc[i][2] += v.z;
            acc[i][3] += v.w;
        }
    }
    // transposed store: out[box][c][b] = s_b acc[b][c]
    const size_t box = axis == 0 ? (size_t)other * side + pos : (size_t)pos * side + other;
    float* dst = out + box * (P * P);
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
        float* row = dst + (size_t)(c0 + cc) * P + b0;
        float4 o = make_float4(ss[b0] * acc[0][cc], ss[b0 + 1] * acc[1][cc], ss[b0 + 2] * acc[2][cc],
                               ss[b0 + 3] * acc[3][cc]);
        if (accumulate) {
            const float4 old = *reinterpret_cast<const float4*>(row);
            o.x += old.x;
            o.y += old.y;
            o.z += old.z;
            o.w += old.w;
        }
        *reinterpret_cast<float4*>(row) = o;
    }
}

bool fgt_supported(int p) { return p == 4 || p == 8 || p == 12 || p == 16; }

// Per-device cache of Hermite tables, keyed by (device, p, n_cut, step bits).
static std::mutex g_tab_mu;
static std::map<std::tuple<int, int, int, uint64_t>, float*> g_tabs;

static int fgt_table(int p, int ncut, double ustep, const float** out)
{
    int dev = 0;
    FMM_CUDA_TRY(cudaGetDevice(&dev));
    uint64_t bits;
    memcpy(&bits, &ustep, sizeof bits);
    const auto key = std::make_tuple(dev, p, ncut, bits);
    std::lock_guard<std::mutex> lk(g_tab_mu);
    auto it = g_tabs.find(key);
    if (it != g_tabs.end()) {
        *out = it->second;
        return FMM_OK;
    }
    const int nh = 2 * p - 1, taps = 2 * ncut + 1;
    float* tab = nullptr;
    FMM_CUDA_TRY(cudaMalloc(&tab, sizeof(float) * (size_t)taps * nh));
    cudaStream_t st;
    FMM_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    fgt_table_kernel<<<1, 64, 0, st>>>(nh, ncut, ustep, tab);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (e != cudaSuccess) {
        cudaFree(tab);
        return cuda_fail(e, "building the FGT Hermite table");
    }
    g_tabs[key] = tab;
    *out = tab;
    return FMM_OK;
}

template <int P>
static int fgt_launch(int g, int ncut, double ustep, const float* A, float* Y, float* Cout, bool acc,
                      bool cached_table, cudaStream_t st)
{
    using C = FgtCfg<P>;
    const int side = 1 << g;
    const size_t smem = fgt_smem_bytes<P>(ncut);
    static unsigned long long opted;  // opted in once for the largest neighbourhood, so every n_cut fits
    if (int rc = smem_opt_in((const void*)fgt_pass_kernel<P>, (int)fgt_smem_bytes<P>(kFgtMaxCut), &opted)) return rc;
    const float* htab = nullptr;
    if (cached_table)
        if (int rc = fgt_table(P, ncut, ustep, &htab)) return rc;
    const dim3 grid((side + C::SEG - 1) / C::SEG, side);
    fgt_pass_kernel<P><<<grid, C::THREADS, smem, st>>>(g, ncut, ustep, 0, A, Y, 0, htab);
    FMM_CUDA_TRY(cudaGetLastError());
    // the second pass as the first's programmatic dependent: its set-up overlaps the first pass
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(C::THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    FMM_CUDA_TRY(cudaLaunchKernelEx(&cfg, fgt_pass_kernel<P>, g, ncut, ustep, 1, (const float*)Y, Cout, acc ? 1 : 0,
                                    htab));
    return FMM_OK;
}

int launch_fgt_h2t(int g, int ncut, int p, double sigma, const float* A, float* Y, float* Cout, bool acc,
                   bool cached_table, cudaStream_t st)
{
    const double ustep = ldexp(1.0, -g) / (sqrt(2.0) * sigma);
    switch (p) {
        case 4: return fgt_launch<4>(g, ncut, ustep, A, Y, Cout, acc, cached_table, st);
        case 8: return fgt_launch<8>(g, ncut, ustep, A, Y, Cout, acc, cached_table, st);
        case 12: return fgt_launch<12>(g, ncut, ustep, A, Y, Cout, acc, cached_table, st);
        case 16: return fgt_launch<16>(g, ncut, ustep, A, Y, Cout, acc, cached_table, st);
        default: return fail(FMM_EINVAL, "fgt_h2t: unsupported p = %d", p);
    }
}

// ---------------------------------------------------------------------------
// One launch for grids up to 32 x 32 boxes (every bandwidth down to
// sigma = 0.05 with the grid of reading R9): a thread-block cluster owns C
// columns of the grid and all of its rows, its CTA of rank r the rows
// [r R, r R + R).  The x-pass writes the CTA's own boxes of Y into its
// shared memory; after a cluster barrier each CTA copies the Y boxes its
// y-pass needs (its columns, rows within n_cut of its own) from the other
// CTAs' shared memory (distributed shared memory), and a second barrier
// lets every CTA leave once nobody reads its memory.  Y never goes to
// global memory and there is no second launch.
// ---------------------------------------------------------------------------
constexpr int kFusedMaxLog2 = 4;  // 32 x 32: only 8 clusters of 8 are resident at once, two passes are faster
constexpr int kFusedCluster = 8;    // CTAs per cluster (portable size: a cluster always fits a GPC)
constexpr int kFusedCopyBatch = 8;  // remote float4 loads in flight per thread
constexpr size_t kFusedMaxSmem = 232448;  // dynamic shared memory a CTA may opt into (227 KB)

struct FusedShape {
    int R, C, CS, TG;  // rows and columns per CTA, CTAs per cluster, tap groups
};

template <int P>
struct FusedSmem {
    // float offsets: own Y [R C][BS], staging [max(R (C + 2 ncut), C (R + 2 ncut))][BS],
    // partial sums [TG - 1][R C][P P], Hermite table [taps][NH], s_b [P]
    size_t own, stage, part, hs, ss, total;
    __host__ __device__ FusedSmem(const FusedShape& f, int ncut)
    {
        using Cf = FgtCfg<P>;
        const int nst1 = f.R * (f.C + 2 * ncut), nst2 = f.C * (f.R + 2 * ncut);
        own = 0;
        stage = own + (size_t)f.R * f.C * Cf::BS;
        part = stage + (size_t)(nst1 > nst2 ? nst1 : nst2) * Cf::BS;
        hs = part + (size_t)(f.TG - 1) * f.R * f.C * P * P;
        ss = hs + (size_t)(2 * ncut + 1) * Cf::NH;
        total = ss + P;
    }
};

// acc[b][c] = sum over taps d in [d0, d1) of sum_a h_{a+b}(u_d) src(d)[a][c], the 4 x 4 block
// (b0.., c0..) of one box; src(d) is a shared-memory box or NULL (outside the grid)
template <int P, typename SrcFn>
__device__ __forceinline__ void fgt_taps(const float* hs, int b0, int c0, int d0, int d1, SrcFn src, float (&acc)[4][4])
{
    using Cf = FgtCfg<P>;
    constexpr int NH = Cf::NH;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) acc[i][cc] = 0.f;
    for (int d = d0; d < d1; ++d) {
        const float* box = src(d);
        if (!box) continue;
        const float* hrow = hs + d * NH + b0;
        const float* in = box + c0;
        float w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i] = hrow[i];
#pragma unroll
        for (int a = 0; a < P; ++a) {
            const float4 v = *reinterpret_cast<const float4*>(in + a * P);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                acc[i][0] = fmaf(w[i], v.x, acc[i][0]);
                acc[i][1] = fmaf(w[i], v.y, acc[i][1]);
                acc[i][2] = fmaf(w[i], v.z, acc[i][2]);
                acc[i][3] = fmaf(w[i], v.w, acc[i][3]);
            }
            if (a + 1 < P) {
#pragma unroll
                for (int i = 0; i < 3; ++i) w[i] = w[i + 1];
                w[3] = hrow[4 + a];
            }
        }
    }
}

template <int P>
__global__ void __launch_bounds__(512) fgt_fused_kernel(int g, int ncut, FusedShape f, const float* __restrict__ A,
                                                         float* __restrict__ Cout, int accumulate,
                                                         const float* __restrict__ htab)
{
    namespace cg = cooperative_groups;
    using Cf = FgtCfg<P>;
    constexpr int BS = Cf::BS, NH = Cf::NH, TPB = Cf::TPB;
    extern __shared__ __align__(16) float fsm[];
    cg::cluster_group cl = cg::this_cluster();
    const FusedSmem<P> L(f, ncut);
    float* own = fsm + L.own;
    float* stage = fsm + L.stage;
    float* part = fsm + L.part;
    float* hs = fsm + L.hs;
    float* ss = fsm + L.ss;

    const int n = 1 << g, taps = 2 * ncut + 1;
    const int rank = (int)cl.block_rank();
    const int y0 = rank * f.R, x0 = (int)(blockIdx.x / f.CS) * f.C;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int nbox = f.R * f.C;

    // x-pass inputs: rows [y0, y0 + R), columns [x0 - ncut, x0 + C + ncut), zero outside the grid;
    // every copy is issued before anything waits on one
    const int w1 = f.C + 2 * ncut;
    const float4* A4 = reinterpret_cast<const float4*>(A);
    for (int i = tid; i < f.R * w1 * (P * P / 4); i += nthr) {
        const int q = i % (P * P / 4), hb = i / (P * P / 4);
        const int yy = y0 + hb / w1, xx = x0 - ncut + hb % w1;
        const bool in = xx >= 0 && xx < n;
        cp_async16(stage + (size_t)hb * BS + 4 * q, in ? (const void*)(A4 + ((size_t)yy * n + xx) * (P * P / 4) + q) : A,
                   in);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    for (int i = tid; i < taps * NH; i += nthr) hs[i] = __ldg(htab + i);
    for (int b = tid; b < P; b += nthr) {
        float fct = 1.f;
        for (int i = 2; i <= b; ++i) fct *= (float)i;  // b! exact in FP32 for b <= 13, to 1 ulp beyond
        ss[b] = ((b & 1) ? -1.f : 1.f) / fct;
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();

    // thread -> (tap group, box of the CTA, 4 x 4 output block)
    const int grp = tid / (nbox * TPB), rem = tid % (nbox * TPB);
    const int j = rem / TPB, r = rem % TPB;
    const int jr = j / f.C, jc = j % f.C;
    const int b0 = (r % Cf::RBLK) * 4, c0 = (r / Cf::RBLK) * 4;
    const int per = (taps + f.TG - 1) / f.TG;
    const int d0 = grp * per, d1 = min(taps, d0 + per);
    const bool active = grp < f.TG;
    float acc[4][4];

    // ---- x-pass: Y[box][c][b] = s_b sum_dx sum_a h_{a+b} A[box + dx][a][c] ----
    const int x = x0 + jc;
    if (active) {
        fgt_taps<P>(hs, b0, c0, d0, d1,
                    [&](int d) -> const float* {
                        const int sx = x + d - ncut;
                        return (sx >= 0 && sx < n) ? stage + (size_t)(jr * w1 + jc + d) * BS : nullptr;
                    },
                    acc);
        if (grp > 0) {
            float* pp = part + ((size_t)(grp - 1) * nbox + j) * (P * P);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                *reinterpret_cast<float4*>(pp + (b0 + i) * P + c0) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        }
    }
    __syncthreads();
    if (active && grp == 0) {
        for (int q = 0; q < f.TG - 1; ++q) {
            const float* pp = part + ((size_t)q * nbox + j) * (P * P);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 v = *reinterpret_cast<const float4*>(pp + (b0 + i) * P + c0);
                acc[i][0] += v.x;
                acc[i][1] += v.y;
                acc[i][2] += v.z;
                acc[i][3] += v.w;
            }
        }
        float* dst = own + (size_t)j * BS;
#pragma unroll
        for (int cc = 0; cc < 4; ++cc)
            *reinterpret_cast<float4*>(dst + (c0 + cc) * P + b0) =
                make_float4(ss[b0] * acc[0][cc], ss[b0 + 1] * acc[1][cc], ss[b0 + 2] * acc[2][cc], ss[b0 + 3] * acc[3][cc]);
    }
    cl.sync();  // every CTA's Y is in its shared memory

    // ---- y-pass inputs: columns [x0, x0 + C), rows [y0 - ncut, y0 + R + ncut) of Y, from their owners ----
    const int h2 = f.R + 2 * ncut;
    const int n2 = f.C * h2 * (P * P / 4);
    for (int i0 = tid; i0 < n2; i0 += nthr * kFusedCopyBatch) {
        float4 v[kFusedCopyBatch];  // a batch of remote loads in flight before any store
#pragma unroll
        for (int k = 0; k < kFusedCopyBatch; ++k) {
            const int i = i0 + k * nthr;
            v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i >= n2) continue;
            const int q = i % (P * P / 4), hb = i / (P * P / 4);
            const int yy = y0 - ncut + hb / f.C, cc = hb % f.C;
            if (yy >= 0 && yy < n) {
                const float* peer = cl.map_shared_rank(own, (unsigned)(yy / f.R));
                v[k] = *reinterpret_cast<const float4*>(peer + (size_t)((yy % f.R) * f.C + cc) * BS + 4 * q);
            }
        }
#pragma unroll
        for (int k = 0; k < kFusedCopyBatch; ++k) {
            const int i = i0 + k * nthr;
            if (i >= n2) break;
            const int q = i % (P * P / 4), hb = i / (P * P / 4);
            *reinterpret_cast<float4*>(stage + (size_t)hb * BS + 4 * q) = v[k];
        }
    }
    cl.sync();  // nobody reads another CTA's shared memory after this

    // ---- y-pass: C[box][b1][b2] = s_b2 sum_dy sum_a2 h_{a2+b2} Y[box + dy][a2][b1] ----
    const int y = y0 + jr;
    if (active) {
        fgt_taps<P>(hs, b0, c0, d0, d1,
                    [&](int d) -> const float* {
                        const int sy = y + d - ncut;
                        return (sy >= 0 && sy < n) ? stage + (size_t)((jr + d) * f.C + jc) * BS : nullptr;
                    },
                    acc);
        if (grp > 0) {
            float* pp = part + ((size_t)(grp - 1) * nbox + j) * (P * P);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                *reinterpret_cast<float4*>(pp + (b0 + i) * P + c0) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        }
    }
    __syncthreads();
    if (active && grp == 0) {
        for (int q = 0; q < f.TG - 1; ++q) {
            const float* pp = part + ((size_t)q * nbox + j) * (P * P);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 v = *reinterpret_cast<const float4*>(pp + (b0 + i) * P + c0);
                acc[i][0] += v.x;
                acc[i][1] += v.y;
                acc[i][2] += v.z;
                acc[i][3] += v.w;
            }
        }
        float* dst = Cout + ((size_t)y * n + x) * (P * P);
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            float* row = dst + (size_t)(c0 + cc) * P + b0;
            float4 o = make_float4(ss[b0] * acc[0][cc], ss[b0 + 1] * acc[1][cc], ss[b0 + 2] * acc[2][cc],
                                   ss[b0 + 3] * acc[3][cc]);
            if (accumulate) {
                const float4 old = *reinterpret_cast<const float4*>(row);
                o.x += old.x;
                o.y += old.y;
                o.z += old.z;
                o.w += old.w;
            }
            *reinterpret_cast<float4*>(row) = o;
        }
    }
}

bool fgt_fused_supported(int g) { return g <= kFusedMaxLog2; }

template <int P>
static int fused_launch(int g, int ncut, double ustep, const float* A, float* Cout, bool acc, cudaStream_t st)
{
    using Cf = FgtCfg<P>;
    const int n = 1 << g, taps = 2 * ncut + 1;
    const float* htab = nullptr;
    if (int rc = fgt_table(P, ncut, ustep, &htab)) return rc;
    // opted into the most a CTA may use; each launch asks for its own shape's need, which the
    // shape selection below keeps within that limit
    static unsigned long long opted;
    if (int rc = smem_opt_in((const void*)fgt_fused_kernel<P>, (int)kFusedMaxSmem, &opted)) return rc;
    // shape: the cluster holds every row (R rows per CTA); C columns per cluster, the fewest that
    // let every cluster be resident at once (about 128 CTAs when they fit)
    FusedShape f;
    f.R = n > kFusedCluster ? n / kFusedCluster : 1;
    f.CS = n / f.R;
    for (f.C = n >= 32 ? 2 : 1;; f.C *= 2) {
        const int pt = f.R * f.C * Cf::TPB;
        f.TG = 512 / pt;
        if (f.TG > taps) f.TG = taps;
        if (f.TG < 1) f.TG = 1;
        if (f.C >= n) break;
        {  // a wider shape must still fit the shared memory of an SM
            FusedShape w = f;
            w.C *= 2;
            w.TG = 512 / (w.R * w.C * Cf::TPB);
            w.TG = w.TG > taps ? taps : (w.TG < 1 ? 1 : w.TG);
            if (sizeof(float) * FusedSmem<P>(w, ncut).total > kFusedMaxSmem) break;
        }
        cudaLaunchConfig_t q = {};
        q.gridDim = dim3((unsigned)(f.CS * (n / f.C)));
        q.blockDim = dim3((unsigned)(f.TG * pt));
        q.dynamicSmemBytes = sizeof(float) * FusedSmem<P>(f, ncut).total;
        cudaLaunchAttribute qa[1];
        qa[0].id = cudaLaunchAttributeClusterDimension;
        qa[0].val.clusterDim.x = (unsigned)f.CS;
        qa[0].val.clusterDim.y = 1;
        qa[0].val.clusterDim.z = 1;
        q.attrs = qa;
        q.numAttrs = 1;
        int active = 0;
        if (cudaOccupancyMaxActiveClusters(&active, (const void*)fgt_fused_kernel<P>, &q) != cudaSuccess) {
            (void)cudaGetLastError();
            break;
        }
        if (active >= n / f.C) break;
    }
    const int per_tg = f.R * f.C * Cf::TPB;
    const FusedSmem<P> L(f, ncut);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(f.CS * (n / f.C)));
    cfg.blockDim = dim3((unsigned)(f.TG * per_tg));
    cfg.dynamicSmemBytes = sizeof(float) * L.total;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)f.CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    FMM_CUDA_TRY(cudaLaunchKernelEx(&cfg, fgt_fused_kernel<P>, g, ncut, f, A, Cout, acc ? 1 : 0, htab));
    return FMM_OK;
}

int launch_fgt_h2t_fused(int g, int ncut, int p, double sigma, const float* A, float* Cout, bool acc, cudaStream_t st)
{
    const double ustep = ldexp(1.0, -g) / (sqrt(2.0) * sigma);
    switch (p) {
        case 4: return fused_launch<4>(g, ncut, ustep, A, Cout, acc, st);
        case 8: return fused_launch<8>(g, ncut, ustep, A, Cout, acc, st);
        case 12: return fused_launch<12>(g, ncut, ustep, A, Cout, acc, st);
        case 16: return fused_launch<16>(g, ncut, ustep, A, Cout, acc, st);
        default: return fail(FMM_EINVAL, "fgt_h2t: unsupported p = %d", p);
    }
}

int fgt_max_cut() { return kFgtMaxCut; }

// ---------------------------------------------------------------------------
// Allocation-free variant: the intermediate Y lives in a fixed device array
// that is part of the loaded module, so no call ever allocates device memory.
// Every GPU that loads the library holds this array until the process exits.
// ---------------------------------------------------------------------------
constexpr size_t kFgtStaticScratchFloats = (size_t)1 << 18;  // 1 MiB: 4^g p^2 <= 262,144 (32 x 32 boxes at p = 16)
static __device__ __align__(256) float g_fgt_static_scratch[kFgtStaticScratchFloats];

constexpr int kMaxDevices = 64;
static std::mutex g_static_mu;
static float* g_static_scratch_dev[kMaxDevices] = {};

// Device address of g_fgt_static_scratch on the current device.  In host code
// the symbol is only a host-side stand-in, so the address is fetched once per
// device (with that device current) and cached.
static int static_scratch(float** out)
{
    int dev = 0;
    FMM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(FMM_EUNSUPPORTED, "fgt_h2t_noalloc: device %d >= %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_scratch_dev[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_fgt_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_fgt_static_scratch)");
        g_static_scratch_dev[dev] = static_cast<float*>(ptr);
    }
    *out = g_static_scratch_dev[dev];
    return FMM_OK;
}

}  // namespace fmmgb

extern "C" int fgt_h2t_noalloc(int32_t grid_log2, int32_t n_cut, int32_t p, double sigma, const float* A, float* C,
                               int32_t flags, void* stream)
{
    using namespace fmmgb;
    clear_error();
    int rc = fgt_check_args("fgt_h2t_noalloc", grid_log2, n_cut, p, sigma, A, C, nullptr, flags);
    if (rc) return rc;
    const size_t need = ((size_t)1 << (2 * grid_log2)) * (size_t)p * p;
    if (need > kFgtStaticScratchFloats)
        return fail(FMM_EINVAL,
                    "fgt_h2t_noalloc: a 2^%d x 2^%d grid at p = %d needs %zu floats of scratch; the built-in scratch "
                    "holds %zu (4^g p^2 <= %zu, e.g. 32 x 32 boxes at p = 16); use fgt_h2t for larger grids",
                    grid_log2, grid_log2, p, need, kFgtStaticScratchFloats, kFgtStaticScratchFloats);
    float* Y = nullptr;
    if ((rc = static_scratch(&Y))) return rc;
    // A or C inside the built-in array would be overwritten by the first pass
    if ((rc = fgt_check_args("fgt_h2t_noalloc", grid_log2, n_cut, p, sigma, A, C, Y, flags))) return rc;
    // The first pass writes every element of Y before the second pass reads
    // it, so the scratch needs no clearing between calls.
    return launch_fgt_h2t(grid_log2, n_cut, p, sigma, A, Y, C, (flags & FMM_ACCUMULATE) != 0, false,
                          (cudaStream_t)stream);
}
