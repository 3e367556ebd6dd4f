// host_stream.cu -- the M2L stage (Sec. 4.1) over a stream of problems whose
// multipole and local expansions live in host memory (fmm_host_stream_*).
//
// A step is: copy the MEs of every level in, fmm_m2l_levels, copy the LEs of
// every level out.  Three non-blocking streams carry the three parts and
// `depth` device buffer sets rotate between the steps, so that step i's
// translation overlaps step i+1's copy in and step i-1's copy out.  Events
// order a buffer set's reuse: its MEs are overwritten only after the
// translation that read them (translated[b]), its LEs only after they have
// been copied out (returned[b]).  Inside a buffer set the levels are back to
// back, so a caller whose host buffer is laid out the same way
// (FMM_HOST_CONTIGUOUS) moves a step in one copy per direction.
#include <new>
#include <vector>

#include "common.cuh"

namespace {

constexpr int kMaxDepth = 8;

enum { kH2D = 0, kComp = 1, kD2H = 2 };

}  // namespace

struct fmm_host_stream {
    const fmm_tree* tree = nullptr;
    int32_t lmin = 0, lmax = 0, p = 0, prec = 0, depth = 0;
    int64_t entries = 0;            // complex64 values per step and direction
    std::vector<int64_t> off;       // first value of each level inside a buffer set
    std::vector<int64_t> len;       // values of each level
    cudaStream_t st[3] = {nullptr, nullptr, nullptr};
    float2* Md[kMaxDepth] = {};
    float2* Ld[kMaxDepth] = {};
    cudaEvent_t arrived[kMaxDepth] = {}, translated[kMaxDepth] = {}, returned[kMaxDepth] = {};
    std::vector<const void*> Mp[kMaxDepth];  // per-level device pointers of each set
    std::vector<void*> Lp[kMaxDepth];
    int64_t steps = 0;
};

using namespace fmmgb;

namespace {

void release(fmm_host_stream* hs)
{
    for (cudaStream_t s : hs->st)
        if (s) cudaStreamSynchronize(s);
    for (int b = 0; b < kMaxDepth; ++b) {
        if (hs->Md[b]) cudaFree(hs->Md[b]);
        if (hs->Ld[b]) cudaFree(hs->Ld[b]);
        if (hs->arrived[b]) cudaEventDestroy(hs->arrived[b]);
        if (hs->translated[b]) cudaEventDestroy(hs->translated[b]);
        if (hs->returned[b]) cudaEventDestroy(hs->returned[b]);
    }
    for (cudaStream_t s : hs->st)
        if (s) cudaStreamDestroy(s);
    delete hs;
}

int create(const fmm_tree* tree, int32_t lmin, int32_t lmax, int32_t p, int32_t prec, int32_t depth,
           fmm_host_stream* hs)
{
    hs->tree = tree;
    hs->lmin = lmin;
    hs->lmax = lmax;
    hs->p = p;
    hs->prec = prec;
    hs->depth = depth;
    for (int l = lmin; l <= lmax; ++l) {
        hs->off.push_back(hs->entries);
        hs->len.push_back(((int64_t)1 << (2 * l)) * p);
        hs->entries += hs->len.back();
    }
    for (int i = 0; i < 3; ++i) FMM_CUDA_TRY(cudaStreamCreateWithFlags(&hs->st[i], cudaStreamNonBlocking));
    const size_t bytes = (size_t)hs->entries * sizeof(float2);
    for (int b = 0; b < depth; ++b) {
        if (cudaMalloc(&hs->Md[b], bytes) != cudaSuccess || cudaMalloc(&hs->Ld[b], bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(FMM_ENOMEM, "fmm_host_stream_create: %zu bytes of device buffers", 2 * depth * bytes);
        }
        FMM_CUDA_TRY(cudaEventCreateWithFlags(&hs->arrived[b], cudaEventDisableTiming));
        FMM_CUDA_TRY(cudaEventCreateWithFlags(&hs->translated[b], cudaEventDisableTiming));
        FMM_CUDA_TRY(cudaEventCreateWithFlags(&hs->returned[b], cudaEventDisableTiming));
        for (size_t i = 0; i < hs->off.size(); ++i) {
            hs->Mp[b].push_back(hs->Md[b] + hs->off[i]);
            hs->Lp[b].push_back(hs->Ld[b] + hs->off[i]);
        }
    }
    // tables, operator images and flags of this (p, prec) now, not inside the first step
    return fmm_prepare(p, prec);
}

// Copies of one direction for the levels of a step: one per level, or one for
// a caller's buffer that holds them all back to back.  (Levels are not merged
// because their addresses happen to be adjacent: separate page-locked
// allocations can be neighbours, and a copy may not span two.)
int copy_levels(const fmm_host_stream* hs, char* dev, const void* const* host, bool contiguous, bool to_device,
                cudaStream_t st)
{
    const int nlev = contiguous ? 1 : (int)hs->off.size();
    for (int i = 0; i < nlev; ++i) {
        const size_t bytes = (size_t)(contiguous ? hs->entries : hs->len[i]) * sizeof(float2);
        char* d = dev + (size_t)hs->off[i] * sizeof(float2);
        if (to_device)
            FMM_CUDA_TRY(cudaMemcpyAsync(d, host[i], bytes, cudaMemcpyHostToDevice, st));
        else
            FMM_CUDA_TRY(cudaMemcpyAsync(const_cast<void*>(host[i]), d, bytes, cudaMemcpyDeviceToHost, st));
    }
    return FMM_OK;
}

}  // namespace

extern "C" {

int fmm_host_stream_create(const fmm_tree* tree, int32_t lmin, int32_t lmax, int32_t p, int32_t prec, int32_t depth,
                           fmm_host_stream** out)
{
    clear_error();
    if (!out) return fail(FMM_EINVAL, "fmm_host_stream_create: out is NULL");
    *out = nullptr;
    if (depth < 1 || depth > kMaxDepth)
        return fail(FMM_EINVAL, "fmm_host_stream_create: depth %d outside 1..%d", depth, kMaxDepth);
    int rc = m2l_levels_check("fmm_host_stream_create", tree, lmin, lmax, p, prec, nullptr, nullptr);
    if (rc) return rc;
    fmm_host_stream* hs = new (std::nothrow) fmm_host_stream;
    if (!hs) return fail(FMM_ENOMEM, "fmm_host_stream_create: host allocation");
    if ((rc = create(tree, lmin, lmax, p, prec, depth, hs))) {
        release(hs);
        return rc;
    }
    *out = hs;
    return FMM_OK;
}

int fmm_host_stream_submit(fmm_host_stream* hs, const void* const* M_host, void* const* L_host, int32_t flags)
{
    clear_error();
    if (!hs || !M_host || !L_host) return fail(FMM_EINVAL, "fmm_host_stream_submit: NULL argument");
    if (flags & ~FMM_HOST_CONTIGUOUS) return fail(FMM_EINVAL, "fmm_host_stream_submit: unknown flags 0x%x", flags);
    const bool contiguous = (flags & FMM_HOST_CONTIGUOUS) != 0;
    // the host ranges of the step: one per level, or one buffer of all levels
    const int nr = contiguous ? 1 : (int)hs->off.size();
    auto bytes = [&](int i) { return (size_t)(contiguous ? hs->entries : hs->len[i]) * sizeof(float2); };
    for (int i = 0; i < nr; ++i)
        if (!M_host[i] || !L_host[i]) return fail(FMM_EINVAL, "fmm_host_stream_submit: NULL level pointer");
    for (int i = 0; i < nr; ++i)
        for (int j = 0; j < nr; ++j) {
            const char* m = (const char*)M_host[i];
            const char* o = (const char*)L_host[j];
            if (m < o + bytes(j) && o < m + bytes(i))
                return fail(FMM_EINVAL, "fmm_host_stream_submit: the MEs overlap the LEs (ranges %d and %d)", i, j);
        }
    const int b = (int)(hs->steps % hs->depth);
    cudaStream_t h2d = hs->st[kH2D], comp = hs->st[kComp], d2h = hs->st[kD2H];
    if (hs->steps >= hs->depth) {
        FMM_CUDA_TRY(cudaStreamWaitEvent(h2d, hs->translated[b], 0));
        FMM_CUDA_TRY(cudaStreamWaitEvent(comp, hs->returned[b], 0));
    }
    int rc = copy_levels(hs, (char*)hs->Md[b], M_host, contiguous, true, h2d);
    if (rc) return rc;
    FMM_CUDA_TRY(cudaEventRecord(hs->arrived[b], h2d));
    FMM_CUDA_TRY(cudaStreamWaitEvent(comp, hs->arrived[b], 0));
    if ((rc = fmm_m2l_levels(hs->tree, hs->lmin, hs->lmax, hs->p, hs->prec, hs->Mp[b].data(), hs->Lp[b].data(), 0,
                             comp)))
        return rc;
    FMM_CUDA_TRY(cudaEventRecord(hs->translated[b], comp));
    FMM_CUDA_TRY(cudaStreamWaitEvent(d2h, hs->translated[b], 0));
    if ((rc = copy_levels(hs, (char*)hs->Ld[b], (const void* const*)L_host, contiguous, false, d2h))) return rc;
    FMM_CUDA_TRY(cudaEventRecord(hs->returned[b], d2h));
    ++hs->steps;
    return FMM_OK;
}

int fmm_host_stream_sync(fmm_host_stream* hs)
{
    clear_error();
    if (!hs) return fail(FMM_EINVAL, "fmm_host_stream_sync: NULL handle");
    FMM_CUDA_TRY(cudaStreamSynchronize(hs->st[kH2D]));
    FMM_CUDA_TRY(cudaStreamSynchronize(hs->st[kD2H]));
    return fmm_sync_status(hs->st[kComp]);
}

int fmm_host_stream_info(const fmm_host_stream* hs, fmm_host_stream_info_t* out)
{
    clear_error();
    if (!hs || !out) return fail(FMM_EINVAL, "fmm_host_stream_info: NULL argument");
    out->entries = hs->entries;
    out->bytes_in = hs->entries * (int64_t)sizeof(float2);
    out->bytes_out = out->bytes_in;
    out->steps = hs->steps;
    out->depth = hs->depth;
    out->lmin = hs->lmin;
    out->lmax = hs->lmax;
    out->p = hs->p;
    out->prec = hs->prec;
    out->h2d_stream = hs->st[kH2D];
    out->compute_stream = hs->st[kComp];
    out->d2h_stream = hs->st[kD2H];
    return FMM_OK;
}

void fmm_host_stream_destroy(fmm_host_stream* hs)
{
    if (hs) release(hs);
}

}  // extern "C"
