// m2l_batched.cu -- many independent uniform-tree M2L problems (each with its
// own depth and p) in ONE persistent launch (Sec. 4.1 steps 2-3, Eq. M2Lmat,
// per problem).
//
// Work items are the FP32 work unit of m2l_fp32_tile.cuh: a 4 x 4 tile of
// parent boxes of one level of one problem.  The host orders them heaviest
// first (p^2 x translations per tile of the level) and uploads the list once
// per plan.  Each resident CTA takes its first chunk of items by blockIdx and
// then claims further chunks from a work counter, so a greedy
// longest-processing-time schedule balances problems whose sizes differ by
// four orders of magnitude.  A CTA keeps the operator tables of its current p
// in shared memory and reloads them only when the p of its next item differs
// (items are grouped by p, so that happens a few times per CTA).
//
// A run is a 4-byte counter reset plus one kernel launch: the plan holds an
// instantiated CUDA graph of the two, and a caller's stream capture records
// them as they are.  The autotuner times, on the plan itself with every output
// pointer redirected to library scratch, first the grid sizes (resident CTAs
// per SM) and claim chunks, then the work-unit variants (how a warp's lanes
// share a target's rows and list entries, and the halo loads a thread keeps in
// flight) at the best of those; the choice is cached per GPU and workload
// signature in memory and in a JSON file that later processes reload.
#include "m2l_fp32_tile.cuh"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <sys/stat.h>
#include <unistd.h>

namespace fmmgb {

// One (problem, level) pair of the batch.
struct BatchDesc {
    const float2* M;
    float2* L;
    int level;
    int p;
    int periodic;
    int pad;
};

// Operator tables per batched order, indexed by batch_p_index(p).
constexpr int kBatchOrders = 4;
struct BatchTables {
    const float2* h[kBatchOrders];
    const float* a[kBatchOrders];
    const float* b[kBatchOrders];
};

static inline int batch_p_index(int p)
{
    switch (p) {
        case 6: return 0;
        case 8: return 1;
        case 12: return 2;
        case 16: return 3;
        default: return -1;
    }
}

constexpr size_t kBatchSmem = M2LCfg<16>::smem;  // the largest batched order
constexpr int kBatchMinCtas = 6;

// Work-unit variants the autotuner chooses between: the lane form of the work unit
// (m2l_fp32_tile.cuh) and the halo loads a thread keeps in flight while staging (the
// one kernel holds every order's code, so its register budget is the largest order's).
struct BatchVariant {
    int form, loads;
};
constexpr BatchVariant kBatchVariants[] = {
    {kFormAuto, 3}, {kFormRowsPacked, 3}, {kFormRowsPacked, 2}, {kFormEntries, 3}, {kFormRows, 3}};
constexpr int kBatchNumVariants = 5;

template <int FORM, int LOADS>
__global__ void __launch_bounds__(kThreads, kBatchMinCtas)
    m2l_batched_kernel(const BatchDesc* __restrict__ desc, const int2* __restrict__ items, int nitems,
                       int* __restrict__ counter, int chunk, int accumulate, BatchTables tabs)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_next;
    int cur_p = 0;
    int base = blockIdx.x * chunk;
    while (base < nitems) {
        const int end = min(base + chunk, nitems);
        for (int it = base; it < end; ++it) {
            const int2 item = items[it];
            const BatchDesc d = desc[item.x];
            if (d.p != cur_p) {
                __syncthreads();  // no thread still reads the previous operator
                switch (d.p) {
                    case 6: m2l_load_operator<6>(smem_raw, tabs.h[0], tabs.a[0], tabs.b[0]); break;
                    case 8: m2l_load_operator<8>(smem_raw, tabs.h[1], tabs.a[1], tabs.b[1]); break;
                    case 12: m2l_load_operator<12>(smem_raw, tabs.h[2], tabs.a[2], tabs.b[2]); break;
                    default: m2l_load_operator<16>(smem_raw, tabs.h[3], tabs.a[3], tabs.b[3]); break;
                }
                cur_p = d.p;
            }
            const TileGeom g = tile_geom_of(d.M, d.L, nullptr, d.level, item.y);
            __syncthreads();  // operator visible; previous tile done with the halo buffer
            switch (d.p) {
                case 6: m2l_tile<6, false, LOADS, FORM>(smem_raw, g, d.periodic, accumulate); break;
                case 8: m2l_tile<8, false, LOADS, FORM>(smem_raw, g, d.periodic, accumulate); break;
                case 12: m2l_tile<12, false, LOADS, FORM>(smem_raw, g, d.periodic, accumulate); break;
                default: m2l_tile<16, false, LOADS, FORM>(smem_raw, g, d.periodic, accumulate); break;
            }
        }
        if (!counter) break;  // one chunk per CTA (grid covers every item)
        // Every thread read s_next of the previous claim before the barrier
        // inside the tile loop above, so thread 0 may overwrite it.
        if (threadIdx.x == 0) s_next = gridDim.x * chunk + atomicAdd(counter, chunk);
        __syncthreads();
        base = s_next;
    }
}

// the kernel of variant v (kBatchVariants order)
static const void* batch_kernel(int v)
{
    switch (v) {
        case 1: return (const void*)m2l_batched_kernel<kFormRowsPacked, 3>;
        case 2: return (const void*)m2l_batched_kernel<kFormRowsPacked, 2>;
        case 3: return (const void*)m2l_batched_kernel<kFormEntries, 3>;
        case 4: return (const void*)m2l_batched_kernel<kFormRows, 3>;
        default: return (const void*)m2l_batched_kernel<kFormAuto, 3>;
    }
}

}  // namespace fmmgb

using namespace fmmgb;

struct fmm_batch {
    int dev = 0;
    int64_t nitems = 0;
    int64_t ntr = 0;
    int accumulate = 0;
    void* block = nullptr;  // one stream-ordered allocation: counter | descriptors | items
    int* counter = nullptr;
    BatchDesc* desc = nullptr;
    int2* items = nullptr;
    std::vector<BatchDesc> host_desc;
    BatchTables tabs{};
    int grid = 0, chunk = 1, persistent = 1, tuned = 0, variant = 0, from_cache = 0;
    float tuned_ms = 0.f;
    size_t max_level_bytes = 0;
    std::string signature;
    cudaGraphExec_t exec = nullptr;
};

namespace {

struct TuneChoice {
    int grid, chunk, persistent, variant;
    float ms;
};
std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune_cache;
bool g_tune_loaded = false;

// The persistent cache: $FMMGB_TUNE_CACHE, else $HOME/.cache/fmmgb/m2l_batched_tune.json (no file
// when neither is set).  One JSON object, one entry per line:
//   "<gpu name>|<SMs>|fp32|<workload signature>": {"grid": G, "chunk": C, "persistent": P, "variant": V, "ms": T},
std::string tune_cache_path()
{
    if (const char* e = getenv("FMMGB_TUNE_CACHE")) return e;
    if (const char* h = getenv("HOME")) {
        const std::string dir = std::string(h) + "/.cache/fmmgb";
        mkdir((std::string(h) + "/.cache").c_str(), 0755);
        mkdir(dir.c_str(), 0755);
        return dir + "/m2l_batched_tune.json";
    }
    return "";
}

// under g_tune_mu
void tune_cache_load()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const std::string path = tune_cache_path();
    if (path.empty()) return;
    FILE* f = fopen(path.c_str(), "r");
    if (!f) return;
    char line[2048], key[1024];
    while (fgets(line, sizeof line, f)) {
        TuneChoice c{};
        if (sscanf(line, " \"%1023[^\"]\": {\"grid\": %d, \"chunk\": %d, \"persistent\": %d, \"variant\": %d, \"ms\": %f}",
                   key, &c.grid, &c.chunk, &c.persistent, &c.variant, &c.ms) == 6 &&
            c.grid > 0 && c.chunk > 0 && c.variant >= 0 && c.variant < kBatchNumVariants)
            g_tune_cache.emplace(key, c);
    }
    fclose(f);
}

// under g_tune_mu: rewrite the whole file (written aside, then renamed into place)
void tune_cache_store()
{
    const std::string path = tune_cache_path();
    if (path.empty()) return;
    const std::string tmp = path + ".tmp" + std::to_string((long)getpid());
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return;
    fprintf(f, "{\n");
    size_t i = 0;
    for (const auto& kv : g_tune_cache) {
        const TuneChoice& c = kv.second;
        fprintf(f, "\"%s\": {\"grid\": %d, \"chunk\": %d, \"persistent\": %d, \"variant\": %d, \"ms\": %.6f}%s\n",
                kv.first.c_str(), c.grid, c.chunk, c.persistent, c.variant, c.ms, ++i < g_tune_cache.size() ? "," : "");
    }
    fprintf(f, "}\n");
    const bool ok = fclose(f) == 0;
    if (ok) rename(tmp.c_str(), path.c_str());
    else remove(tmp.c_str());
}

// the cache key of a plan: the GPU (name and SM count), the precision and the workload signature
int tune_key(const fmm_batch* b, std::string* key)
{
    cudaDeviceProp prop;
    FMM_CUDA_TRY(cudaGetDeviceProperties(&prop, b->dev));
    std::string name = prop.name;
    for (char& ch : name)
        if (ch == '"' || ch == '|' || ch == '\\') ch = '_';
    *key = name + "|" + std::to_string(prop.multiProcessorCount) + "|fp32|" + b->signature;
    return FMM_OK;
}

int batch_occupancy(int v, int* occ)
{
    FMM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, batch_kernel(v), kThreads, kBatchSmem));
    if (*occ < 1) return fail(FMM_ECUDA, "batched M2L: kernel variant %d cannot be resident (occupancy 0)", v);
    return FMM_OK;
}

int launch_batch(const fmm_batch* b, const BatchDesc* desc, int grid, int chunk, int persistent, int variant,
                 cudaStream_t st)
{
    FMM_CUDA_TRY(cudaMemsetAsync(b->counter, 0, sizeof(int), st));
    const int2* items = b->items;
    int nitems = (int)b->nitems;
    int* ctr = persistent ? b->counter : nullptr;
    int acc = b->accumulate;
    BatchTables tabs = b->tabs;
    void* args[] = {(void*)&desc, (void*)&items, (void*)&nitems, (void*)&ctr, (void*)&chunk, (void*)&acc, (void*)&tabs};
    FMM_CUDA_TRY(cudaLaunchKernel(batch_kernel(variant), dim3((unsigned)grid), dim3(kThreads), args, kBatchSmem, st));
    return FMM_OK;
}

int build_graph(fmm_batch* b)
{
    cudaGraph_t g = nullptr;
    FMM_CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaMemsetParams mp{};
    mp.dst = b->counter;
    mp.value = 0;
    mp.elementSize = sizeof(int);
    mp.width = 1;
    mp.height = 1;
    mp.pitch = sizeof(int);
    cudaGraphNode_t nset = nullptr, nker = nullptr;
    cudaError_t e = cudaGraphAddMemsetNode(&nset, g, nullptr, 0, &mp);
    const BatchDesc* desc = b->desc;
    const int2* items = b->items;
    int nitems = (int)b->nitems;
    int* ctr = b->persistent ? b->counter : nullptr;
    int chunk = b->chunk, acc = b->accumulate;
    BatchTables tabs = b->tabs;
    void* args[] = {(void*)&desc, (void*)&items, (void*)&nitems, (void*)&ctr, (void*)&chunk, (void*)&acc, (void*)&tabs};
    if (e == cudaSuccess) {
        cudaKernelNodeParams kp{};
        kp.func = const_cast<void*>(batch_kernel(b->variant));
        kp.gridDim = dim3((unsigned)b->grid);
        kp.blockDim = dim3(kThreads);
        kp.sharedMemBytes = (unsigned)kBatchSmem;
        kp.kernelParams = args;
        e = cudaGraphAddKernelNode(&nker, g, &nset, 1, &kp);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        return cuda_fail(e, "building the batched M2L graph");
    }
    return FMM_OK;
}

// Time the candidate configurations on the plan with outputs redirected to scratch:
// first the grid sizes and claim chunks with the default work unit, then every work-unit
// variant at the best of those; keep the fastest.  A choice stored for this GPU and
// workload (in memory or in the cache file) is reused without timing.  Synchronous.
int autotune(fmm_batch* b, cudaStream_t st)
{
    std::string key;
    int rc = tune_key(b, &key);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_cache_load();
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            b->grid = it->second.grid;
            b->chunk = it->second.chunk;
            b->persistent = it->second.persistent;
            b->variant = it->second.variant;
            b->tuned = 1;
            b->from_cache = 1;
            b->tuned_ms = it->second.ms;
            return FMM_OK;
        }
    }
    int sms = 0, occ = 0;
    if ((rc = device_sm_count(&sms)) || (rc = batch_occupancy(0, &occ))) return rc;
    const int64_t n = b->nitems;
    float2* scratch = nullptr;
    BatchDesc* sdesc = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<BatchDesc> hd = b->host_desc;
    cudaError_t e = cudaMalloc(&scratch, b->max_level_bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, b->max_level_bytes, st);
    if (e == cudaSuccess) e = cudaMalloc(&sdesc, hd.size() * sizeof(BatchDesc));
    for (auto& d : hd) d.L = scratch;
    if (e == cudaSuccess) e = cudaMemcpyAsync(sdesc, hd.data(), hd.size() * sizeof(BatchDesc), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    rc = (e == cudaSuccess) ? FMM_OK : cuda_fail(e, "batched M2L autotuner setup");
    auto time_one = [&](TuneChoice& c) {
        if (rc) return;
        if ((rc = launch_batch(b, sdesc, c.grid, c.chunk, c.persistent, c.variant, st))) return;  // warm-up
        float t = 1e30f;
        for (int rep = 0; rep < 3 && !rc; ++rep) {
            float ms = 0.f;
            if ((e = cudaEventRecord(e0, st)) != cudaSuccess) { rc = cuda_fail(e, "cudaEventRecord"); return; }
            if ((rc = launch_batch(b, sdesc, c.grid, c.chunk, c.persistent, c.variant, st))) return;
            if ((e = cudaEventRecord(e1, st)) != cudaSuccess) { rc = cuda_fail(e, "cudaEventRecord"); return; }
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { rc = cuda_fail(e, "cudaEventSynchronize"); return; }
            cudaEventElapsedTime(&ms, e0, e1);
            t = std::min(t, ms);
        }
        c.ms = t;
    };
    // stage 1: launch configurations with the default work unit
    std::vector<TuneChoice> cand;
    cand.push_back({(int)n, 1, 0, 0, 0.f});  // one CTA per item, hardware scheduling
    for (int r = 1; r <= occ; ++r)
        for (int c : {1, 2, 4}) {
            const int64_t g = std::min<int64_t>((int64_t)r * sms, (n + c - 1) / c);
            if (g >= 1) cand.push_back({(int)g, c, 1, 0, 0.f});
        }
    TuneChoice best{0, 0, 0, 0, 1e30f};
    for (auto& c : cand) {
        time_one(c);
        if (!rc && c.ms < best.ms) best = c;
    }
    // stage 2: the other work-unit variants at that configuration (a persistent grid is
    // clamped to what the variant keeps resident)
    for (int v = 1; v < kBatchNumVariants && !rc; ++v) {
        int occ_v = 0;
        if ((rc = batch_occupancy(v, &occ_v))) break;
        TuneChoice c = best;
        c.variant = v;
        if (c.persistent) c.grid = (int)std::min<int64_t>(c.grid, (int64_t)occ_v * sms);
        time_one(c);
        if (!rc && c.ms < best.ms) best = c;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    cudaFree(sdesc);
    cudaFree(scratch);
    if (rc) return rc;
    b->grid = best.grid;
    b->chunk = best.chunk;
    b->persistent = best.persistent;
    b->variant = best.variant;
    b->tuned = 1;
    b->from_cache = 0;
    b->tuned_ms = best.ms;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_cache_load();
    g_tune_cache[key] = best;
    tune_cache_store();
    return FMM_OK;
}

void free_batch(fmm_batch* b, cudaStream_t st)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->block) cudaFreeAsync(b->block, st);
    delete b;
}

int create_batch(const fmm_tree* const* trees, const int32_t* p, int32_t nprob, const void* const* M_levels,
                 void* const* L_levels, int32_t prec, int32_t flags, cudaStream_t st, bool sync, fmm_batch** out)
{
    const char* who = "fmm_batch_create";
    if (!out) return fail(FMM_EINVAL, "%s: out is NULL", who);
    *out = nullptr;
    if (!trees || !p || !M_levels || !L_levels) return fail(FMM_EINVAL, "%s: NULL array argument", who);
    if (nprob < 1 || nprob > 65536) return fail(FMM_EINVAL, "%s: nprob %d outside 1..65536", who, nprob);
    if (flags & ~(FMM_ACCUMULATE | FMM_BATCH_AUTOTUNE)) return fail(FMM_EINVAL, "%s: unknown flags 0x%x", who, flags);
    if (prec != FMM_FP32) {
        if (prec == FMM_TC_BF16X3 || prec == FMM_TC_BF16 || prec == FMM_TC_TF32X3)
            return fail(FMM_EUNSUPPORTED, "%s: the batched path computes in FMM_FP32 only", who);
        return fail(FMM_EINVAL, "%s: unknown precision %d", who, prec);
    }
    fmm_batch* b = new (std::nothrow) fmm_batch();
    if (!b) return fail(FMM_ENOMEM, "%s: out of host memory", who);
    b->accumulate = (flags & FMM_ACCUMULATE) ? 1 : 0;
    int64_t k = 0;
    std::map<std::string, int64_t> sig;
    for (int i = 0; i < nprob; ++i) {
        const fmm_tree* t = trees[i];
        if (!t) { delete b; return fail(FMM_EINVAL, "%s: trees[%d] is NULL", who, i); }
        const int pi = p[i];
        if (batch_p_index(pi) < 0) {
            delete b;
            return fail(pi == 24 ? FMM_EUNSUPPORTED : FMM_EINVAL,
                        "%s: p[%d] = %d outside the batched set 6, 8, 12, 16", who, i, pi);
        }
        if (tree_adaptive(t)) {
            delete b;
            return fail(FMM_EUNSUPPORTED, "%s: trees[%d] is adaptive; the batched path takes uniform trees", who, i);
        }
        const int lmax = tree_max_level(t), per = tree_periodic(t);
        for (int l = 2; l <= lmax; ++l, ++k) {
            const void* M = M_levels[k];
            void* L = L_levels[k];
            if (!M || !L) { delete b; return fail(FMM_EINVAL, "%s: NULL coefficient pointer (problem %d level %d)", who, i, l); }
            if (((uintptr_t)M & 15) || ((uintptr_t)L & 15)) {
                delete b;
                return fail(FMM_EINVAL, "%s: coefficient pointers must be 16-byte aligned (problem %d level %d)", who, i, l);
            }
            const size_t bytes = ((size_t)1 << (2 * l)) * (size_t)pi * 8;
            const char* a = (const char*)M;
            const char* c = (const char*)L;
            if (a < c + bytes && c < a + bytes) {
                delete b;
                return fail(FMM_EINVAL, "%s: input and output overlap (problem %d level %d)", who, i, l);
            }
            b->host_desc.push_back(BatchDesc{(const float2*)M, (float2*)L, l, pi, per, 0});
            b->max_level_bytes = std::max(b->max_level_bytes, bytes);
            b->ntr += fmm_tree_translations(t, l);
            char key[48];
            snprintf(key, sizeof key, "%d/%d/%d;", pi, l, per);
            sig[key] += 1;
        }
    }
    for (auto& kv : sig) b->signature += kv.first + std::to_string(kv.second) + ",";
    b->signature += b->accumulate ? "acc" : "set";
    // Heaviest first: p^2 x interaction entries per tile of the level.
    std::vector<int> order(b->host_desc.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    auto cost = [&](int i) {
        const BatchDesc& d = b->host_desc[i];
        const double side = (double)(1 << d.level);
        const double ntr = d.periodic ? 27.0 * side * side
                                      : (6 * side - 8) * (6 * side - 8) - (3 * side - 2) * (3 * side - 2);
        return (double)d.p * d.p * ntr / m2l_tiles(d.level);
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
    std::vector<BatchDesc> sorted;
    sorted.reserve(order.size());
    for (int i : order) sorted.push_back(b->host_desc[i]);
    b->host_desc.swap(sorted);
    std::vector<int2> items;
    for (size_t i = 0; i < b->host_desc.size(); ++i) {
        const int nt = m2l_tiles(b->host_desc[i].level);
        for (int t = 0; t < nt; ++t) items.push_back(make_int2((int)i, t));
    }
    if (items.size() > (size_t)0x7fffffff / 4) { delete b; return fail(FMM_EINVAL, "%s: too many work items", who); }
    b->nitems = (int64_t)items.size();
    for (int pv : {6, 8, 12, 16}) {
        bool used = false;
        for (int i = 0; i < nprob; ++i) used |= p[i] == pv;
        if (!used) continue;
        const M2LTables* t = nullptr;
        int rc = get_m2l_tables(pv, &t);
        if (rc) { delete b; return rc; }
        const int j = batch_p_index(pv);
        b->tabs.h[j] = t->h_fwd;
        b->tabs.a[j] = t->a;
        b->tabs.b[j] = t->b;
    }
    int sms = 0, occ = 0, rc;
    FMM_CUDA_TRY(cudaGetDevice(&b->dev));
    if ((rc = device_sm_count(&sms)) || (rc = batch_occupancy(0, &occ))) { delete b; return rc; }
    b->persistent = 1;
    b->chunk = 1;
    b->grid = (int)std::min<int64_t>((int64_t)occ * sms, b->nitems);
    // device arrays: counter (256 B) | descriptors | items, stream-ordered
    const size_t dbytes = b->host_desc.size() * sizeof(BatchDesc), ibytes = items.size() * sizeof(int2);
    const size_t doff = 256, ioff = doff + ((dbytes + 255) / 256) * 256;
    cudaError_t e = cudaMallocAsync(&b->block, ioff + ibytes, st);
    if (e != cudaSuccess) { delete b; return cuda_fail(e, "cudaMallocAsync(batch plan)"); }
    b->counter = (int*)b->block;
    b->desc = (BatchDesc*)((char*)b->block + doff);
    b->items = (int2*)((char*)b->block + ioff);
    if ((e = cudaMemsetAsync(b->counter, 0, sizeof(int), st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(b->desc, b->host_desc.data(), dbytes, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(b->items, items.data(), ibytes, cudaMemcpyHostToDevice, st)) != cudaSuccess) {
        free_batch(b, st);
        return cuda_fail(e, "uploading the batch plan");
    }
    if (sync || (flags & FMM_BATCH_AUTOTUNE)) {
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) {
            free_batch(b, st);
            return cuda_fail(e, "uploading the batch plan");
        }
    }
    if (flags & FMM_BATCH_AUTOTUNE) {
        if ((rc = autotune(b, st))) {
            free_batch(b, st);
            return rc;
        }
    }
    *out = b;
    return FMM_OK;
}

}  // namespace

extern "C" {

int fmm_batch_create(const fmm_tree* const* trees, const int32_t* p, int32_t nprob, const void* const* M_levels,
                     void* const* L_levels, int32_t prec, int32_t flags, void* stream, fmm_batch** out)
{
    clear_error();
    return create_batch(trees, p, nprob, M_levels, L_levels, prec, flags, (cudaStream_t)stream, true, out);
}

int fmm_batch_run(fmm_batch* b, void* stream)
{
    clear_error();
    if (!b) return fail(FMM_EINVAL, "fmm_batch_run: batch is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (b->nitems == 0) return FMM_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    FMM_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone)  // the caller's capture records the two operations
        return launch_batch(b, b->desc, b->grid, b->chunk, b->persistent, b->variant, st);
    if (!b->exec) {
        int rc = build_graph(b);
        if (rc) return rc;
    }
    FMM_CUDA_TRY(cudaGraphLaunch(b->exec, st));
    return FMM_OK;
}

int fmm_batch_info(const fmm_batch* b, fmm_batch_info_t* out)
{
    clear_error();
    if (!b || !out) return fail(FMM_EINVAL, "fmm_batch_info: NULL argument");
    out->items = b->nitems;
    out->translations = b->ntr;
    out->grid = b->grid;
    out->chunk = b->chunk;
    out->persistent = b->persistent;
    out->tuned = b->tuned;
    out->tuned_ms = b->tuned_ms;
    out->variant = b->variant;
    out->form = kBatchVariants[b->variant].form;
    out->loads = kBatchVariants[b->variant].loads;
    out->from_cache = b->from_cache;
    return FMM_OK;
}

void fmm_batch_destroy(fmm_batch* b, void* stream) { free_batch(b, (cudaStream_t)stream); }

int fmm_m2l_batched(const fmm_tree* const* trees, const int32_t* p, int32_t nprob, const void* const* M_levels,
                    void* const* L_levels, int32_t prec, int32_t flags, void* stream)
{
    clear_error();
    if (flags & FMM_BATCH_AUTOTUNE) return fail(FMM_EINVAL, "fmm_m2l_batched: FMM_BATCH_AUTOTUNE needs fmm_batch_create");
    cudaStream_t st = (cudaStream_t)stream;
    fmm_batch* b = nullptr;
    int rc = create_batch(trees, p, nprob, M_levels, L_levels, prec, flags, st, false, &b);
    if (rc) return rc;
    rc = b->nitems ? launch_batch(b, b->desc, b->grid, b->chunk, b->persistent, b->variant, st) : FMM_OK;
    free_batch(b, st);
    return rc;
}

}  // extern "C"
