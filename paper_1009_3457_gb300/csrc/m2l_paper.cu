// m2l_paper.cu -- the paper's own M2L data flow (Sec. 4.1.1-4.1.2), kept as a
// comparison for the fused target-centric stencil:
//   1. translate: one thread block per source ME, one thread per LE row n of
//      each translation; the block translates its ME to every target whose
//      interaction list holds it and writes one LE per translation to global
//      memory;
//   2. reduce: a separate kernel sums the (up to 27) translated LEs of each
//      target (the paper's "Reduction" column).
// The arithmetic is the library's: the scaled Hankel operator h_D of each
// offset from the per-device tables (rows l_n = a_n sum_k h_D[n+k] b_k m_k),
// where the paper forms the powers of the offset in every thread.  What the
// comparison measures is the data flow: 27 LEs written and read back per
// target (p complex each) instead of one store per target.
#include "common.cuh"

namespace fmmgb {

// per child class: for each of the 49 offset slots (source - target), its position in the
// class's 27-entry stencil or -1; and per stencil position its parent offset
struct PaperStencil {
    int8_t pos[4][kOffsetSlots];
    int8_t ex[4][27], ey[4][27];
};

template <int P>
__global__ void __launch_bounds__(32 * P) m2l_paper_translate_kernel(const float2* __restrict__ M, int level,
                                                                     const float2* __restrict__ h,
                                                                     const float* __restrict__ a,
                                                                     const float* __restrict__ b, PaperStencil st,
                                                                     float2* __restrict__ T)
{
    constexpr int NH = 2 * P - 1;
    __shared__ float2 s_m[P];
    __shared__ float2 s_h[kOffsetSlots * NH];
    const int side = 1 << level;
    const int s = blockIdx.x, sx = s & (side - 1), sy = s >> level;
    const int tid = threadIdx.x;
    if (tid < P) {
        const float2 v = M[(size_t)s * P + tid];
        s_m[tid] = make_float2(v.x * b[tid], v.y * b[tid]);
    }
    for (int i = tid; i < kOffsetSlots * NH; i += blockDim.x) s_h[i] = h[i];
    __syncthreads();
    const int n = tid % P, w = tid / P;  // row n of the translations w, w + 32
    const float an = a[n];
    for (int o = w; o < kOffsetSlots; o += 32) {
        const int dx = o % 7 - 3, dy = o / 7 - 3;  // source - target
        const int tx = sx - dx, ty = sy - dy;
        if (tx < 0 || ty < 0 || tx >= side || ty >= side) continue;
        const int cls = (tx & 1) + 2 * (ty & 1);
        const int j = st.pos[cls][o];
        if (j < 0) continue;
        const float2* hr = s_h + o * NH + n;
        float re = 0.f, im = 0.f;
#pragma unroll
        for (int k = 0; k < P; ++k) {
            const float2 hv = hr[k], m = s_m[k];
            re = fmaf(hv.x, m.x, fmaf(-hv.y, m.y, re));
            im = fmaf(hv.x, m.y, fmaf(hv.y, m.x, im));
        }
        T[(((size_t)ty * side + tx) * 27 + j) * P + n] = make_float2(an * re, an * im);
    }
}

template <int P>
__global__ void m2l_paper_reduce_kernel(int level, PaperStencil st, const float2* __restrict__ T,
                                        float2* __restrict__ L, int accumulate)
{
    const int side = 1 << level, np = side >> 1;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)side * side * P) return;
    const int n = (int)(i % P);
    const int t = (int)(i / P), tx = t & (side - 1), ty = t >> level;
    const int cls = (tx & 1) + 2 * (ty & 1);
    float2 acc = accumulate ? L[i] : make_float2(0.f, 0.f);
    for (int j = 0; j < 27; ++j) {
        const int qx = (tx >> 1) + st.ex[cls][j], qy = (ty >> 1) + st.ey[cls][j];
        if (qx < 0 || qy < 0 || qx >= np || qy >= np) continue;  // no such source: never written
        const float2 v = T[((size_t)t * 27 + j) * P + n];
        acc.x += v.x;
        acc.y += v.y;
    }
    L[i] = acc;
}

template <int P>
static int paper_launch(int level, const M2LTables* tab, PaperStencil st, const float2* M, float2* L, float2* T,
                        bool acc, cudaStream_t s)
{
    const int nbox = 1 << (2 * level);
    m2l_paper_translate_kernel<P><<<nbox, 32 * P, 0, s>>>(M, level, tab->h_fwd, tab->a, tab->b, st, T);
    FMM_CUDA_TRY(cudaGetLastError());
    const int64_t total = (int64_t)nbox * P;
    m2l_paper_reduce_kernel<P><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(level, st, T, L, acc ? 1 : 0);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

}  // namespace fmmgb

using namespace fmmgb;

extern "C" int fmm_m2l_paper_design(const fmm_tree* tree, int32_t level, int32_t p, const void* M, void* L,
                                    void* work, int32_t flags, void* stream)
{
    clear_error();
    if (!tree) return fail(FMM_EINVAL, "fmm_m2l_paper_design: tree is NULL");
    if (tree_adaptive(tree) || tree_periodic(tree))
        return fail(FMM_EUNSUPPORTED, "fmm_m2l_paper_design: uniform, non-periodic trees only");
    if (level < 2 || level > tree_max_level(tree))
        return fail(FMM_EINVAL, "fmm_m2l_paper_design: level %d outside 2..%d", level, tree_max_level(tree));
    if (p != 8 && p != 12 && p != 16) return fail(FMM_EINVAL, "fmm_m2l_paper_design: p = %d (8, 12, 16)", p);
    if (!M || !L || !work) return fail(FMM_EINVAL, "fmm_m2l_paper_design: NULL pointer");
    if (((uintptr_t)M & 15) || ((uintptr_t)L & 15) || ((uintptr_t)work & 15))
        return fail(FMM_EINVAL, "fmm_m2l_paper_design: pointers must be 16-byte aligned");
    if (flags & ~FMM_ACCUMULATE) return fail(FMM_EINVAL, "fmm_m2l_paper_design: unknown flags 0x%x", flags);
    const M2LTables* tab = nullptr;
    if (int rc = get_m2l_tables(p, &tab)) return rc;
    PaperStencil st;
    for (int c = 0; c < 4; ++c) {
        StencilEntry e[27];
        class_stencil(c, e);
        for (int o = 0; o < kOffsetSlots; ++o) st.pos[c][o] = -1;
        for (int j = 0; j < 27; ++j) {
            st.pos[c][(int)e[j].slot] = (int8_t)j;
            st.ex[c][j] = e[j].ex;
            st.ey[c][j] = e[j].ey;
        }
    }
    const float2* Mp = (const float2*)M;
    float2* Lp = (float2*)L;
    float2* T = (float2*)work;
    const bool acc = (flags & FMM_ACCUMULATE) != 0;
    cudaStream_t s = (cudaStream_t)stream;
    switch (p) {
        case 8: return paper_launch<8>(level, tab, st, Mp, Lp, T, acc, s);
        case 12: return paper_launch<12>(level, tab, st, Mp, Lp, T, acc, s);
        default: return paper_launch<16>(level, tab, st, Mp, Lp, T, acc, s);
    }
}
