// m2l_fp32.cu -- FP32 M2L with the reduction fused in, over one or several
// levels of a uniform quadtree in one launch (Sec. 4.1 steps 2-3, Eq. M2Lmat),
// plus the FP64 operator-table builder.
//
// The work unit (a 4 x 4 tile of parent boxes, the Hankel factorisation of the
// operator and the class-split shared-memory halo) and the stencil kernel are
// in m2l_fp32_tile.cuh; this file holds the operator-table builder and the
// launcher.
#include "m2l_fp32_tile.cuh"

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

bool m2l_fp32_supported(int p) { return p == 6 || p == 8 || p == 12 || p == 16 || p == 24; }

template <int P>
static int launch_p(M2LLaunch& job, const float2* h, const float* a, const float* b, cudaStream_t st)
{
    using C = M2LCfg<P>;
    int total = 0;
    for (int i = 0; i < job.nlev; ++i) {
        job.lv[i].tile_begin = total;
        total += job.lv[i].tiles ? job.lv[i].ntiles : m2l_tiles(job.lv[i].level);
    }
    if (total == 0) return FMM_OK;
    bool adaptive = false;
    for (int i = 0; i < job.nlev; ++i) adaptive |= job.lv[i].exists != nullptr;
    auto kern = adaptive ? m2l_fp32_kernel<P, true> : m2l_fp32_kernel<P, false>;
    // persistent grid: resident CTAs x SMs, tiles claimed from a zeroed counter
    int sms = 0, occ = 0;
    int rc = device_sm_count(&sms);
    if (rc) return rc;
    static unsigned long long opted[2];
    if ((rc = smem_opt_in((const void*)kern, (int)C::smem, &opted[adaptive]))) return rc;
    static int occ_cache[2];  // resident CTAs per SM (same on every device of one model)
    if (!(occ = __atomic_load_n(&occ_cache[adaptive], __ATOMIC_ACQUIRE))) {
        FMM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, C::smem));
        __atomic_store_n(&occ_cache[adaptive], occ, __ATOMIC_RELEASE);
    }
    int grid = total, *counter = nullptr;
    if (occ > 0 && (int64_t)occ * sms < total) {
        grid = occ * sms;
        if ((rc = tile_counter(&counter, st))) return rc;
    }
    kern<<<grid, kThreads, C::smem, st>>>(job, h, a, b, total, counter);
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
