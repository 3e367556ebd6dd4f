// api.cu -- C ABI of libfmmgb: argument checks, tree handles, per-device
// operator tables and dispatch to the kernels.  All arithmetic of the method
// runs in the kernels of m2l_fp32.cu, m2l_tc.cu, fgt_h2t.cu and upward.cu.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace fmmgb {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local char g_msg[512] = "";

int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(e == cudaErrorMemoryAllocation ? FMM_ENOMEM : FMM_ECUDA, "%s: %s (%s)", what,
                cudaGetErrorString(e), cudaGetErrorName(e));
}

void clear_error() { g_msg[0] = 0; }

// ---------------------------------------------------------------------------
// interaction-list stencil per child class (Sec. 4.1 step 1)
// ---------------------------------------------------------------------------
void class_stencil(int cls, StencilEntry out[27])
{
    const int cx = cls & 1, cy = cls >> 1;
    int n = 0;
    for (int ey = -1; ey <= 1; ++ey)
        for (int ex = -1; ex <= 1; ++ex)
            for (int sy = 0; sy < 2; ++sy)
                for (int sx = 0; sx < 2; ++sx) {
                    const int dx = 2 * ex + sx - cx, dy = 2 * ey + sy - cy;
                    const int adx = dx < 0 ? -dx : dx, ady = dy < 0 ? -dy : dy;
                    if ((adx > ady ? adx : ady) < 2) continue;  // adjacent: near field
                    out[n].ex = (int8_t)ex;
                    out[n].ey = (int8_t)ey;
                    out[n].csrc = (int8_t)(sx + 2 * sy);
                    out[n].slot = (int8_t)offset_slot(dx, dy);
                    ++n;
                }
}

// ---------------------------------------------------------------------------
// per-device state
// ---------------------------------------------------------------------------
struct DeviceState {
    int* err_word = nullptr;
    std::map<int, M2LTables*> m2l;
    float* fgt_ws = nullptr;  // FGT H2T intermediate (grown on demand)
    size_t fgt_ws_bytes = 0;
    int* tc_flags = nullptr;  // tensor-core M2L: one flag per tile, zero between launches (grown on demand)
    int tc_flag_count = 0;
    int sm_count = 0;
    int* counters = nullptr;  // ring of persistent-launch work counters
    unsigned next_counter = 0;
    unsigned char* fgt_flags = nullptr;  // FGT Hermite evaluation: non-empty flag per grid box
};
constexpr int kCounterRing = 256;
static std::mutex g_mu;
static std::map<int, DeviceState*> g_dev;

static int current_state(DeviceState** out)
{
    int dev = 0;
    FMM_CUDA_TRY(cudaGetDevice(&dev));
    auto it = g_dev.find(dev);
    if (it != g_dev.end()) {
        *out = it->second;
        return FMM_OK;
    }
    DeviceState* s = new DeviceState();
    cudaError_t e = cudaMalloc(&s->err_word, sizeof(int));
    if (e != cudaSuccess) {
        delete s;
        return cuda_fail(e, "cudaMalloc(error word)");
    }
    e = cudaMemset(s->err_word, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(error word)");
    g_dev[dev] = s;
    *out = s;
    return FMM_OK;
}

int device_error_word(int** out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState* s = nullptr;
    int rc = current_state(&s);
    if (rc) return rc;
    *out = s->err_word;
    return FMM_OK;
}

int device_sm_count(int* out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState* s = nullptr;
    int rc = current_state(&s);
    if (rc) return rc;
    if (!s->sm_count) {
        int dev = 0;
        FMM_CUDA_TRY(cudaGetDevice(&dev));
        FMM_CUDA_TRY(cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, dev));
    }
    *out = s->sm_count;
    return FMM_OK;
}

int smem_opt_in(const void* func, int bytes, unsigned long long* done)
{
    int dev = 0;
    FMM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(FMM_EUNSUPPORTED, "device ordinal %d above 63", dev);
    const unsigned long long bit = 1ull << dev;
    if (__atomic_load_n(done, __ATOMIC_ACQUIRE) & bit) return FMM_OK;
    FMM_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    __atomic_fetch_or(done, bit, __ATOMIC_RELEASE);
    return FMM_OK;
}

int tile_counter(int** out, cudaStream_t st)
{
    (void)st;  // nothing is enqueued: the slot is zero on allocation and the kernel resets it
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState* s = nullptr;
    int rc = current_state(&s);
    if (rc) return rc;
    if (!s->counters) {
        FMM_CUDA_TRY(cudaMalloc(&s->counters, kCounterRing * 2 * sizeof(int)));
        FMM_CUDA_TRY(cudaMemset(s->counters, 0, kCounterRing * 2 * sizeof(int)));
    }
    *out = s->counters + 2 * (s->next_counter++ % kCounterRing);
    return FMM_OK;
}

int fgt_flag_buffer(unsigned char** out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState* s = nullptr;
    int rc = current_state(&s);
    if (rc) return rc;
    if (!s->fgt_flags) FMM_CUDA_TRY(cudaMalloc(&s->fgt_flags, kFgtScratchBytes));
    *out = s->fgt_flags;
    return FMM_OK;
}

int tc_flag_workspace(int ntiles, int** flags)
{
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState* s = nullptr;
    int rc = current_state(&s);
    if (rc) return rc;
    if (s->tc_flag_count < ntiles) {
        if (s->tc_flags) {
            FMM_CUDA_TRY(cudaDeviceSynchronize());
            cudaFree(s->tc_flags);
            s->tc_flags = nullptr;
            s->tc_flag_count = 0;
        }
        FMM_CUDA_TRY(cudaMalloc(&s->tc_flags, (size_t)ntiles * sizeof(int)));
        FMM_CUDA_TRY(cudaMemset(s->tc_flags, 0, (size_t)ntiles * sizeof(int)));
        s->tc_flag_count = ntiles;
    }
    *flags = s->tc_flags;
    return FMM_OK;
}

int fgt_workspace(size_t bytes, float** out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState* s = nullptr;
    int rc = current_state(&s);
    if (rc) return rc;
    if (s->fgt_ws_bytes < bytes) {
        if (s->fgt_ws) {
            FMM_CUDA_TRY(cudaDeviceSynchronize());
            cudaFree(s->fgt_ws);
            s->fgt_ws = nullptr;
            s->fgt_ws_bytes = 0;
        }
        FMM_CUDA_TRY(cudaMalloc(&s->fgt_ws, bytes));
        s->fgt_ws_bytes = bytes;
    }
    *out = s->fgt_ws;
    return FMM_OK;
}

double m2l_balance(int p)
{
    // s = 2e / (2p - 2) balances j! s^j |D|^-(j+1) (|D| >= 2) against
    // 1 / (n! s^n) over the index ranges j <= 2p-2, n <= p-1.
    const double jmax = (p > 1) ? 2.0 * p - 2.0 : 1.0;
    return 2.0 * 2.718281828459045 / jmax;
}

int get_m2l_tables(int p, const M2LTables** out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState* s = nullptr;
    int rc = current_state(&s);
    if (rc) return rc;
    auto it = s->m2l.find(p);
    if (it != s->m2l.end()) {
        *out = it->second;
        return FMM_OK;
    }
    M2LTables* t = new M2LTables();
    t->p = p;
    t->s = m2l_balance(p);
    const size_t nh = (size_t)kOffsetSlots * (2 * p - 1);
    cudaError_t e;
    if ((e = cudaMalloc(&t->h_fwd, nh * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc(&t->h_adj, nh * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc(&t->h_adjc, nh * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc(&t->a, p * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&t->b, p * sizeof(float))) != cudaSuccess) {
        cudaFree(t->h_fwd);
        cudaFree(t->h_adj);
        cudaFree(t->h_adjc);
        cudaFree(t->a);
        cudaFree(t->b);
        delete t;
        return cuda_fail(e, "cudaMalloc(M2L operator tables)");
    }
    cudaStream_t st;
    FMM_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    rc = launch_build_m2l_tables(*t, st);
    cudaError_t es = cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (rc) return rc;
    if (es != cudaSuccess) return cuda_fail(es, "building M2L operator tables");
    s->m2l[p] = t;
    *out = t;
    return FMM_OK;
}

int get_tc_image(int p, int variant, bool tf32, const void** out)
{
    if (!m2l_tc_supported(p)) return fail(FMM_EUNSUPPORTED, "tensor-core M2L is provided for p = 16 and 24, not %d", p);
    if (tf32 && !m2l_tc_tf32_supported(p))
        return fail(FMM_EUNSUPPORTED, "tensor-core M2L with TF32 operands is provided for p = 16, not %d", p);
    const int f = tf32 ? 1 : 0;
    const M2LTables* tc = nullptr;
    int rc = get_m2l_tables(p, &tc);
    if (rc) return rc;
    M2LTables* t = const_cast<M2LTables*>(tc);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!t->tc_ready[f][variant]) {
        const size_t bytes = m2l_tc_image_bytes(p, tf32);
        cudaError_t e = cudaMalloc(&t->tc_w[f][variant], bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(tensor-core operator image)");
        cudaStream_t st;
        FMM_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        rc = launch_build_tc_image(p, t->s, variant, tf32, t->tc_w[f][variant], st);
        cudaError_t es = cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
        if (rc) return rc;
        if (es != cudaSuccess) return cuda_fail(es, "building the tensor-core operator image");
        t->tc_ready[f][variant] = 1;
    }
    *out = t->tc_w[f][variant];
    return FMM_OK;
}

}  // namespace fmmgb

using namespace fmmgb;

// ---------------------------------------------------------------------------
// tree handle
// ---------------------------------------------------------------------------
struct fmm_tree {
    int32_t max_level = 0;
    int32_t periodic = 0;
    int32_t leaf_cap = 0;  // 0: uniform tree
    struct Level {
        bool built = false;
        int64_t ntr = 0;
        std::vector<int32_t> list;
        std::vector<int8_t> code;
        int32_t* list_dev = nullptr;
        int8_t* code_dev = nullptr;
        // adaptive trees: box existence (empty vector: every box of the level exists)
        std::vector<uint8_t> exists;
        int64_t nexist = 0;
        bool dev_ready = false;
        uint8_t* exists_dev = nullptr;
        int32_t* tiles_dev = nullptr;  // 4 x 4-parent tiles holding at least one existing box
        int32_t ntiles = 0;
        bool tc_ready = false;
        int32_t* tc_tiles_dev = nullptr;  // 8 x 32-parent tiles (tensor-core M2L) holding an existing box
        int32_t tc_ntiles = 0;
    };
    Level levels[FMM_MAX_LEVEL + 1];
    std::mutex mu;
};

int fmmgb::tree_max_level(const fmm_tree* t) { return t->max_level; }
int fmmgb::tree_periodic(const fmm_tree* t) { return t->periodic; }
int fmmgb::tree_adaptive(const fmm_tree* t) { return t->leaf_cap > 0; }

static int64_t translations_closed_form(int level, bool periodic)
{
    if (level < 2) return 0;
    const int64_t n = (int64_t)1 << level;
    if (periodic) return 27 * n * n;
    return (6 * n - 8) * (6 * n - 8) - (3 * n - 2) * (3 * n - 2);
}

static inline bool box_exists(const fmm_tree::Level& L, int64_t b) { return L.exists.empty() || L.exists[b]; }

// Calls fn(source box, offset code) for every list entry of target (tx, ty):
// the class stencil of the target, cut at the domain edge (or wrapped), and
// for an adaptive tree restricted to existing sources (V-list).
template <class F>
static void for_each_entry(const fmm_tree* t, int level, int64_t tx, int64_t ty, const StencilEntry* st, F fn)
{
    const int64_t side = (int64_t)1 << level;
    const fmm_tree::Level& L = t->levels[level];
    for (int e = 0; e < 27; ++e) {
        const int code = st[e].slot;
        int64_t sx = tx + (code % 7 - 3), sy = ty + (code / 7 - 3);
        if (t->periodic) {
            sx = ((sx % side) + side) % side;
            sy = ((sy % side) + side) % side;
        } else if (sx < 0 || sy < 0 || sx >= side || sy >= side) {
            continue;
        }
        if (!box_exists(L, sy * side + sx)) continue;
        fn(sy * side + sx, code);
    }
}

// Adaptive subdivision: the root exists; an existing box of level l <
// max_level holding more than q points is split and its non-empty children
// exist.  Then the per-level V-list counts.
static int build_adaptive(fmm_tree* t, const double* xy, int64_t n, int q)
{
    std::vector<int64_t> cnt_parent;
    for (int l = 0; l <= t->max_level; ++l) {
        const int64_t side = (int64_t)1 << l;
        std::vector<int64_t> cnt((size_t)(side * side), 0);
        for (int64_t i = 0; i < n; ++i) {
            double fx = std::floor(xy[2 * i] * (double)side), fy = std::floor(xy[2 * i + 1] * (double)side);
            int64_t ix = fx < 0.0 || fx != fx ? 0 : (fx > (double)(side - 1) ? side - 1 : (int64_t)fx);
            int64_t iy = fy < 0.0 || fy != fy ? 0 : (fy > (double)(side - 1) ? side - 1 : (int64_t)fy);
            cnt[(size_t)(iy * side + ix)] += 1;
        }
        auto& L = t->levels[l];
        L.exists.assign((size_t)(side * side), 0);
        if (l == 0) {
            L.exists[0] = 1;
        } else {
            const int64_t pside = side / 2;
            const auto& P = t->levels[l - 1];
            for (int64_t iy = 0; iy < side; ++iy)
                for (int64_t ix = 0; ix < side; ++ix) {
                    const int64_t pb = (iy / 2) * pside + ix / 2;
                    if (P.exists[(size_t)pb] && cnt_parent[(size_t)pb] > q && cnt[(size_t)(iy * side + ix)] > 0)
                        L.exists[(size_t)(iy * side + ix)] = 1;
                }
        }
        L.nexist = 0;
        for (uint8_t e : L.exists) L.nexist += e;
        cnt_parent.swap(cnt);
    }
    StencilEntry st[4][27];
    for (int c = 0; c < 4; ++c) class_stencil(c, st[c]);
    for (int l = 0; l <= t->max_level; ++l) {
        auto& L = t->levels[l];
        const int64_t side = (int64_t)1 << l;
        L.ntr = 0;
        if (l >= 2)
            for (int64_t ty = 0; ty < side; ++ty)
                for (int64_t tx = 0; tx < side; ++tx) {
                    if (!L.exists[(size_t)(ty * side + tx)]) continue;
                    for_each_entry(t, l, tx, ty, st[(tx & 1) + 2 * (ty & 1)], [&](int64_t, int) { ++L.ntr; });
                }
    }
    // Levels where every box exists take the uniform fast path.
    for (int l = 0; l <= t->max_level; ++l) {
        auto& L = t->levels[l];
        if (L.nexist == ((int64_t)1 << (2 * l))) std::vector<uint8_t>().swap(L.exists);
    }
    return FMM_OK;
}

int fmmgb::tree_device_level(const fmm_tree* ctree, int level, const uint8_t** exists, const int32_t** tiles,
                             int* ntiles)
{
    fmm_tree* t = const_cast<fmm_tree*>(ctree);
    auto& L = t->levels[level];
    *exists = nullptr;
    *tiles = nullptr;
    *ntiles = -1;  // every tile of the level
    if (L.exists.empty()) return FMM_OK;
    std::lock_guard<std::mutex> lk(t->mu);
    if (!L.dev_ready) {
        const int64_t side = (int64_t)1 << level, np = side / 2;
        const int64_t tpr = (np + 3) / 4;
        std::vector<int32_t> tl;
        for (int64_t tt = 0; tt < tpr * tpr; ++tt) {
            const int64_t x0 = (tt % tpr) * 8, y0 = (tt / tpr) * 8;
            bool any = false;
            for (int64_t y = y0; y < y0 + 8 && y < side && !any; ++y)
                for (int64_t x = x0; x < x0 + 8 && x < side; ++x)
                    if (L.exists[(size_t)(y * side + x)]) {
                        any = true;
                        break;
                    }
            if (any) tl.push_back((int32_t)tt);
        }
        FMM_CUDA_TRY(cudaMalloc(&L.exists_dev, L.exists.size()));
        FMM_CUDA_TRY(cudaMemcpy(L.exists_dev, L.exists.data(), L.exists.size(), cudaMemcpyHostToDevice));
        if (!tl.empty()) {
            FMM_CUDA_TRY(cudaMalloc(&L.tiles_dev, tl.size() * sizeof(int32_t)));
            FMM_CUDA_TRY(cudaMemcpy(L.tiles_dev, tl.data(), tl.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        }
        L.ntiles = (int32_t)tl.size();
        L.dev_ready = true;
    }
    *exists = L.exists_dev;
    *tiles = L.tiles_dev;
    *ntiles = L.ntiles;
    return FMM_OK;
}

// The 8 x 32-parent tiles of an adaptive level (tensor-core M2L, tile t = ty * ceil(np / 8) + tx)
// that hold at least one existing box, uploaded on first use; NULL, -1 for a level where every
// box exists.
int fmmgb::tree_device_tc_tiles(const fmm_tree* ctree, int level, const int32_t** tiles, int* ntiles)
{
    fmm_tree* t = const_cast<fmm_tree*>(ctree);
    auto& L = t->levels[level];
    *tiles = nullptr;
    *ntiles = -1;
    if (L.exists.empty()) return FMM_OK;
    std::lock_guard<std::mutex> lk(t->mu);
    if (!L.tc_ready) {
        const int64_t side = (int64_t)1 << level, np = side / 2;
        const int64_t tpr = (np + 7) / 8, rows = (np + 31) / 32;
        std::vector<int32_t> tl;
        for (int64_t tt = 0; tt < tpr * rows; ++tt) {
            const int64_t x0 = (tt % tpr) * 16, y0 = (tt / tpr) * 64;  // boxes of the tile's parents
            bool any = false;
            for (int64_t y = y0; y < y0 + 64 && y < side && !any; ++y)
                for (int64_t x = x0; x < x0 + 16 && x < side; ++x)
                    if (L.exists[(size_t)(y * side + x)]) {
                        any = true;
                        break;
                    }
            if (any) tl.push_back((int32_t)tt);
        }
        if (!tl.empty()) {
            FMM_CUDA_TRY(cudaMalloc(&L.tc_tiles_dev, tl.size() * sizeof(int32_t)));
            FMM_CUDA_TRY(cudaMemcpy(L.tc_tiles_dev, tl.data(), tl.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        }
        L.tc_ntiles = (int32_t)tl.size();
        L.tc_ready = true;
    }
    *tiles = L.tc_tiles_dev;
    *ntiles = L.tc_ntiles;
    return FMM_OK;
}

extern "C" {

const char* fmm_last_error(void) { return g_msg; }

const char* fmm_version(void) { return "fmmgb 0.1 (sm_103a)"; }

int fmm_build_lists(const double* xy, int64_t n, int32_t max_level, int32_t leaf_cap, int32_t flags,
                    fmm_tree** out)
{
    clear_error();
    if (!out) return fail(FMM_EINVAL, "fmm_build_lists: out is NULL");
    *out = nullptr;
    if (n < 0) return fail(FMM_EINVAL, "fmm_build_lists: n = %lld < 0", (long long)n);
    if (n > 0 && !xy && leaf_cap != 0) return fail(FMM_EINVAL, "fmm_build_lists: xy is NULL");
    if (max_level < 2 || max_level > FMM_MAX_LEVEL)
        return fail(FMM_EINVAL, "fmm_build_lists: max_level %d outside 2..%d", max_level, FMM_MAX_LEVEL);
    if (leaf_cap < 0) return fail(FMM_EINVAL, "fmm_build_lists: leaf_cap %d < 0", leaf_cap);
    if (flags & ~FMM_TREE_PERIODIC) return fail(FMM_EINVAL, "fmm_build_lists: unknown flags 0x%x", flags);
    if (leaf_cap > 0 && (flags & FMM_TREE_PERIODIC))
        return fail(FMM_EINVAL, "fmm_build_lists: periodic lists need a uniform tree (leaf_cap = 0)");
    fmm_tree* t = new (std::nothrow) fmm_tree();
    if (!t) return fail(FMM_ENOMEM, "fmm_build_lists: out of host memory");
    t->max_level = max_level;
    t->periodic = (flags & FMM_TREE_PERIODIC) ? 1 : 0;
    t->leaf_cap = leaf_cap;
    if (leaf_cap > 0) {
        int rc = build_adaptive(t, xy, n, leaf_cap);
        if (rc) {
            delete t;
            return rc;
        }
    } else {
        for (int l = 0; l <= max_level; ++l) {
            t->levels[l].ntr = translations_closed_form(l, t->periodic);
            t->levels[l].nexist = (int64_t)1 << (2 * l);
        }
    }
    *out = t;
    return FMM_OK;
}

int64_t fmm_tree_translations(const fmm_tree* tree, int32_t level)
{
    if (!tree || level < 0 || level > tree->max_level) return -1;
    return tree->levels[level].ntr;
}

int fmm_tree_level_info(const fmm_tree* ctree, int32_t level, fmm_level_info* out)
{
    clear_error();
    if (!ctree || !out) return fail(FMM_EINVAL, "fmm_tree_level_info: NULL argument");
    fmm_tree* tree = const_cast<fmm_tree*>(ctree);
    if (level < 0 || level > tree->max_level)
        return fail(FMM_EINVAL, "fmm_tree_level_info: level %d outside 0..%d", level, tree->max_level);
    std::lock_guard<std::mutex> lk(tree->mu);
    auto& L = tree->levels[level];
    const int64_t side = (int64_t)1 << level, nbox = side * side;
    if (!L.built) {
        if (nbox * 27 > ((int64_t)1 << 31)) return fail(FMM_EINVAL, "fmm_tree_level_info: level %d lists too large", level);
        L.list.assign((size_t)nbox * 27, -1);
        L.code.assign((size_t)nbox * 27, (int8_t)-1);
        int64_t cnt = 0;
        if (level >= 2) {
            StencilEntry st[4][27];
            for (int c = 0; c < 4; ++c) class_stencil(c, st[c]);
            for (int64_t ty = 0; ty < side; ++ty)
                for (int64_t tx = 0; tx < side; ++tx) {
                    const int64_t t = ty * side + tx;
                    if (!box_exists(L, t)) continue;  // absent box: empty V-list
                    int slot = 0;
                    for_each_entry(tree, level, tx, ty, st[(tx & 1) + 2 * (ty & 1)], [&](int64_t s, int code) {
                        L.list[(size_t)t * 27 + slot] = (int32_t)s;
                        L.code[(size_t)t * 27 + slot] = (int8_t)code;
                        ++slot;
                        ++cnt;
                    });
                }
        }
        if (cnt != L.ntr) return fail(FMM_EDEVICE, "fmm_tree_level_info: list count %lld != %lld", (long long)cnt, (long long)L.ntr);
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
            (void)cudaGetLastError();  // host-only use: device copies stay NULL
        } else {
            cudaError_t e = cudaMalloc(&L.list_dev, L.list.size() * sizeof(int32_t));
            if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(list)");
            e = cudaMalloc(&L.code_dev, L.code.size());
            if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(offset codes)");
            e = cudaMemcpy(L.list_dev, L.list.data(), L.list.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(list)");
            e = cudaMemcpy(L.code_dev, L.code.data(), L.code.size(), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(offset codes)");
        }
        L.built = true;
    }
    out->nbox = nbox;
    out->side = (int32_t)side;
    out->list_stride = 27;
    out->ntranslations = L.ntr;
    out->list_host = L.list.data();
    out->offcode_host = L.code.data();
    out->list_dev = L.list_dev;
    out->offcode_dev = L.code_dev;
    out->nexist = L.nexist;
    out->exists_host = L.exists.empty() ? nullptr : L.exists.data();
    return FMM_OK;
}

void fmm_tree_destroy(fmm_tree* tree)
{
    if (!tree) return;
    for (auto& L : tree->levels) {
        if (L.list_dev) cudaFree(L.list_dev);
        if (L.code_dev) cudaFree(L.code_dev);
        if (L.exists_dev) cudaFree(L.exists_dev);
        if (L.tiles_dev) cudaFree(L.tiles_dev);
        if (L.tc_tiles_dev) cudaFree(L.tc_tiles_dev);
    }
    delete tree;
}

static bool valid_p(int p) { return m2l_fp32_supported(p); }

static bool m2l_prec_known(int prec)
{
    return prec == FMM_FP32 || prec == FMM_TC_BF16X3 || prec == FMM_TC_BF16 || prec == FMM_TC_TF32X3;
}

int fmm_prepare(int32_t p, int32_t prec)
{
    clear_error();
    if (!valid_p(p)) return fail(FMM_EINVAL, "fmm_prepare: unsupported p = %d (6, 8, 12, 16, 24)", p);
    if (!m2l_prec_known(prec)) return fail(FMM_EINVAL, "fmm_prepare: unknown precision %d", prec);
    const M2LTables* t = nullptr;
    int rc = get_m2l_tables(p, &t);
    if (rc) return rc;
    if (prec != FMM_FP32) {
        const void* img = nullptr;
        if ((rc = get_tc_image(p, 0, prec == FMM_TC_TF32X3, &img))) return rc;
    }
    int* ctr = nullptr;
    if ((rc = tile_counter(&ctr, nullptr))) return rc;
    unsigned char* flags = nullptr;
    if ((rc = fgt_flag_buffer(&flags))) return rc;
    return cudaStreamSynchronize(nullptr) == cudaSuccess ? FMM_OK : fail(FMM_ECUDA, "fmm_prepare: sync failed");
}

static int m2l_common(const char* who, const fmm_tree* tree, int32_t level, int32_t p, int32_t prec,
                      const void* in, void* out, int32_t flags, int32_t allowed_flags)
{
    if (!tree) return fail(FMM_EINVAL, "%s: tree is NULL", who);
    if (level < 0 || level > tree->max_level)
        return fail(FMM_EINVAL, "%s: level %d outside 0..%d", who, level, tree->max_level);
    if (!valid_p(p)) return fail(FMM_EINVAL, "%s: unsupported p = %d (6, 8, 12, 16, 24)", who, p);
    if (!m2l_prec_known(prec)) return fail(FMM_EINVAL, "%s: unknown precision %d", who, prec);
    if (!in || !out) return fail(FMM_EINVAL, "%s: NULL coefficient pointer", who);
    if (((uintptr_t)in & 15) || ((uintptr_t)out & 15))
        return fail(FMM_EINVAL, "%s: coefficient pointers must be 16-byte aligned", who);
    if (flags & ~allowed_flags) return fail(FMM_EINVAL, "%s: unknown flags 0x%x", who, flags);
    const size_t bytes = ((size_t)1 << (2 * level)) * (size_t)p * 8;
    const char* a = (const char*)in;
    const char* b = (const char*)out;
    if (a < b + bytes && b < a + bytes) return fail(FMM_EINVAL, "%s: input and output overlap", who);
    return FMM_OK;
}

// One launch over levels lmin..lmax (heaviest first) of the forward or adjoint stencil.
static int m2l_dispatch(const char* who, const fmm_tree* tree, int32_t lmin, int32_t lmax, int32_t p, int32_t prec,
                        const void* const* in, void* const* out, int32_t flags, bool adjoint, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    const bool acc = (flags & FMM_ACCUMULATE) != 0;
    for (int l = lmin; l <= lmax && l < 2; ++l)
        if (!acc) FMM_CUDA_TRY(cudaMemsetAsync(out[l - lmin], 0, ((size_t)1 << (2 * l)) * (size_t)p * 8, st));
    if (lmax < 2) return FMM_OK;
    if (prec != FMM_FP32 && !m2l_tc_supported(p))
        return fail(FMM_EUNSUPPORTED, "%s: tensor-core precision %d is provided at p = 16, 24", who, prec);
    if (prec == FMM_TC_TF32X3 && !m2l_tc_tf32_supported(p))
        return fail(FMM_EUNSUPPORTED, "%s: FMM_TC_TF32X3 is provided at p = 16", who);
    const M2LTables* t = nullptr;
    int rc = get_m2l_tables(p, &t);
    if (rc) return rc;
    M2LLaunch job{};
    job.periodic = tree->periodic;
    job.accumulate = acc ? 1 : 0;
    for (int l = lmax; l >= lmin && l >= 2; --l) {
        const uint8_t* ex = nullptr;
        const int32_t* tiles = nullptr;
        int ntiles = -1;
        if ((rc = tree_device_level(tree, l, &ex, &tiles, &ntiles))) return rc;
        if (ntiles == 0) continue;  // no existing box at this level
        const int32_t* tc_tiles = nullptr;
        int tc_ntiles = -1;
        if (ex && prec != FMM_FP32 && (rc = tree_device_tc_tiles(tree, l, &tc_tiles, &tc_ntiles))) return rc;
        M2LLevel& d = job.lv[job.nlev++];
        d.M = (const float2*)in[l - lmin];
        d.L = (float2*)out[l - lmin];
        d.level = l;
        d.exists = ex;
        d.tiles = tiles;
        d.ntiles = ntiles;
        d.tc_tiles = tc_tiles;
        d.tc_ntiles = tc_ntiles;
    }
    if (job.nlev == 0) return FMM_OK;
    // The adjoint is the forward stencil with the table of -a(D) (plain) or
    // -conj a(D) (FMM_CONJ): a(D)^T = -a(-D) on symmetric lists.
    if (prec != FMM_FP32) {
        const int variant = !adjoint ? 0 : ((flags & FMM_CONJ) ? 2 : 1);
        const void* img = nullptr;
        const bool tf32 = prec == FMM_TC_TF32X3;
        if ((rc = get_tc_image(p, variant, tf32, &img))) return rc;
        return launch_m2l_tc(job, p, img, prec != FMM_TC_BF16, tf32, st);
    }
    const float2* h = !adjoint ? t->h_fwd : ((flags & FMM_CONJ) ? t->h_adjc : t->h_adj);
    return launch_m2l_fp32(job, p, h, t->a, t->b, st);
}

static int levels_common(const char* who, const fmm_tree* tree, int32_t lmin, int32_t lmax, int32_t p, int32_t prec,
                         const void* const* in, void* const* out, int32_t flags, int32_t allowed)
{
    if (!tree) return fail(FMM_EINVAL, "%s: tree is NULL", who);
    if (!in || !out) return fail(FMM_EINVAL, "%s: NULL pointer array", who);
    if (lmin < 0 || lmax > tree->max_level || lmin > lmax)
        return fail(FMM_EINVAL, "%s: levels %d..%d outside 0..%d", who, lmin, lmax, tree->max_level);
    for (int l = lmin; l <= lmax; ++l) {
        int rc = m2l_common(who, tree, l, p, prec, in[l - lmin], out[l - lmin], flags, allowed);
        if (rc) return rc;
    }
    return FMM_OK;
}

int fmm_m2l(const fmm_tree* tree, int32_t level, int32_t p, int32_t prec, const void* M, void* L, int32_t flags,
            void* stream)
{
    clear_error();
    int rc = m2l_common("fmm_m2l", tree, level, p, prec, M, L, flags, FMM_ACCUMULATE);
    if (rc) return rc;
    const void* in[1] = {M};
    void* out[1] = {L};
    return m2l_dispatch("fmm_m2l", tree, level, level, p, prec, in, out, flags, false, stream);
}

int fmm_m2l_levels(const fmm_tree* tree, int32_t lmin, int32_t lmax, int32_t p, int32_t prec, const void* const* M,
                   void* const* L, int32_t flags, void* stream)
{
    clear_error();
    int rc = levels_common("fmm_m2l_levels", tree, lmin, lmax, p, prec, M, L, flags, FMM_ACCUMULATE);
    if (rc) return rc;
    return m2l_dispatch("fmm_m2l_levels", tree, lmin, lmax, p, prec, M, L, flags, false, stream);
}

int fmm_m2l_adjoint(const fmm_tree* tree, int32_t level, int32_t p, int32_t prec, const void* W, void* G,
                    int32_t flags, void* stream)
{
    clear_error();
    int rc = m2l_common("fmm_m2l_adjoint", tree, level, p, prec, W, G, flags, FMM_ACCUMULATE | FMM_CONJ);
    if (rc) return rc;
    const void* in[1] = {W};
    void* out[1] = {G};
    return m2l_dispatch("fmm_m2l_adjoint", tree, level, level, p, prec, in, out, flags, true, stream);
}

int fmm_m2l_adjoint_levels(const fmm_tree* tree, int32_t lmin, int32_t lmax, int32_t p, int32_t prec,
                           const void* const* W, void* const* G, int32_t flags, void* stream)
{
    clear_error();
    int rc = levels_common("fmm_m2l_adjoint_levels", tree, lmin, lmax, p, prec, W, G, flags,
                           FMM_ACCUMULATE | FMM_CONJ);
    if (rc) return rc;
    return m2l_dispatch("fmm_m2l_adjoint_levels", tree, lmin, lmax, p, prec, W, G, flags, true, stream);
}

int fmm_p2m(int32_t level, int32_t p, const double* xy, const double* c, int64_t n, void* M, int32_t flags,
            void* stream)
{
    clear_error();
    if (level < 0 || level > FMM_MAX_LEVEL) return fail(FMM_EINVAL, "fmm_p2m: level %d outside 0..%d", level, FMM_MAX_LEVEL);
    if (p < 1 || p > 64) return fail(FMM_EINVAL, "fmm_p2m: p = %d outside 1..64", p);
    if (n < 0) return fail(FMM_EINVAL, "fmm_p2m: n < 0");
    if (!M || (n > 0 && (!xy || !c))) return fail(FMM_EINVAL, "fmm_p2m: NULL pointer");
    if (flags & ~FMM_ACCUMULATE) return fail(FMM_EINVAL, "fmm_p2m: unknown flags 0x%x", flags);
    return launch_p2m(level, p, xy, c, n, (float2*)M, (flags & FMM_ACCUMULATE) != 0, (cudaStream_t)stream);
}

int fmm_p2m_binned(int32_t level, int32_t p, const double* xy, const double* c, int64_t n, const int32_t* perm,
                   const int32_t* box_start, void* M, int32_t flags, void* stream)
{
    clear_error();
    if (level < 0 || level > 10) return fail(FMM_EINVAL, "fmm_p2m_binned: level %d outside 0..10", level);
    if (p != 6 && p != 8 && p != 12 && p != 16 && p != 24)
        return fail(FMM_EINVAL, "fmm_p2m_binned: unsupported p = %d (6, 8, 12, 16, 24)", p);
    if (n < 0 || n > INT32_MAX) return fail(FMM_EINVAL, "fmm_p2m_binned: n = %lld outside 0..2^31-1", (long long)n);
    if (!M || !box_start || (n > 0 && (!xy || !c || !perm))) return fail(FMM_EINVAL, "fmm_p2m_binned: NULL pointer");
    if (((uintptr_t)M & 7) || ((uintptr_t)xy & 7) || ((uintptr_t)c & 7) || ((uintptr_t)perm & 3) ||
        ((uintptr_t)box_start & 3))
        return fail(FMM_EINVAL, "fmm_p2m_binned: misaligned pointer");
    if (flags & ~FMM_ACCUMULATE) return fail(FMM_EINVAL, "fmm_p2m_binned: unknown flags 0x%x", flags);
    int* err = nullptr;
    if (int rc = device_error_word(&err)) return rc;
    return launch_p2m_binned(level, p, xy, c, (int)n, perm, box_start, (float2*)M, (flags & FMM_ACCUMULATE) != 0,
                             err, (cudaStream_t)stream);
}

int fmm_m2m_adjoint(int32_t child_level, int32_t p, const void* Wp, void* Wc, int32_t flags, void* stream)
{
    clear_error();
    if (child_level < 1 || child_level > FMM_MAX_LEVEL)
        return fail(FMM_EINVAL, "fmm_m2m_adjoint: child_level %d outside 1..%d", child_level, FMM_MAX_LEVEL);
    if (p < 1 || p > 64) return fail(FMM_EINVAL, "fmm_m2m_adjoint: p = %d outside 1..64", p);
    if (!Wp || !Wc) return fail(FMM_EINVAL, "fmm_m2m_adjoint: NULL pointer");
    if (((uintptr_t)Wp & 7) || ((uintptr_t)Wc & 7)) return fail(FMM_EINVAL, "fmm_m2m_adjoint: misaligned pointer");
    if (flags & ~FMM_ACCUMULATE) return fail(FMM_EINVAL, "fmm_m2m_adjoint: unknown flags 0x%x", flags);
    return launch_m2m_adjoint(child_level, p, (const float2*)Wp, (float2*)Wc, (flags & FMM_ACCUMULATE) != 0,
                              (cudaStream_t)stream);
}

int fmm_m2m(int32_t child_level, int32_t p, const void* Mc, void* Mp, int32_t flags, void* stream)
{
    clear_error();
    if (child_level < 1 || child_level > FMM_MAX_LEVEL)
        return fail(FMM_EINVAL, "fmm_m2m: child_level %d outside 1..%d", child_level, FMM_MAX_LEVEL);
    if (p < 1 || p > 64) return fail(FMM_EINVAL, "fmm_m2m: p = %d outside 1..64", p);
    if (!Mc || !Mp) return fail(FMM_EINVAL, "fmm_m2m: NULL pointer");
    if (flags & ~FMM_ACCUMULATE) return fail(FMM_EINVAL, "fmm_m2m: unknown flags 0x%x", flags);
    return launch_m2m(child_level, p, (const float2*)Mc, (float2*)Mp, (flags & FMM_ACCUMULATE) != 0,
                      (cudaStream_t)stream);
}

}  // extern "C"

int fmmgb::m2l_levels_check(const char* who, const fmm_tree* tree, int32_t lmin, int32_t lmax, int32_t p,
                            int32_t prec, const void* const* in, void* const* out)
{
    if (in || out) {
        int rc = levels_common(who, tree, lmin, lmax, p, prec, in, out, 0, 0);
        if (rc) return rc;
    } else {  // the arguments alone, before the caller allocates its buffers
        if (!tree) return fail(FMM_EINVAL, "%s: tree is NULL", who);
        if (lmin < 0 || lmax > tree->max_level || lmin > lmax)
            return fail(FMM_EINVAL, "%s: levels %d..%d outside 0..%d", who, lmin, lmax, tree->max_level);
        if (!valid_p(p)) return fail(FMM_EINVAL, "%s: unsupported p = %d (6, 8, 12, 16, 24)", who, p);
        if (!m2l_prec_known(prec)) return fail(FMM_EINVAL, "%s: unknown precision %d", who, prec);
    }
    if (lmax >= 2 && prec != FMM_FP32 && !m2l_tc_supported(p))
        return fail(FMM_EUNSUPPORTED, "%s: tensor-core precision %d is provided at p = 16, 24", who, prec);
    if (lmax >= 2 && prec == FMM_TC_TF32X3 && !m2l_tc_tf32_supported(p))
        return fail(FMM_EUNSUPPORTED, "%s: FMM_TC_TF32X3 is provided at p = 16", who);
    return FMM_OK;
}

int fmmgb::fgt_check_args(const char* who, int g, int n_cut, int p, double sigma, const float* A, const float* C,
                          const float* work, int flags)
{
    if (g < 0 || g > 12) return fail(FMM_EINVAL, "%s: grid_log2 %d outside 0..12", who, g);
    if (n_cut < 0 || n_cut > fgt_max_cut()) return fail(FMM_EINVAL, "%s: n_cut %d outside 0..%d", who, n_cut, fgt_max_cut());
    if (!fgt_supported(p)) return fail(FMM_EINVAL, "%s: unsupported p = %d (4, 8, 12, 16)", who, p);
    if (!(sigma > 0.0) || !(sigma < 1e300)) return fail(FMM_EINVAL, "%s: sigma must be positive and finite", who);
    if (!A || !C) return fail(FMM_EINVAL, "%s: NULL coefficient pointer", who);
    if (((uintptr_t)A & 15) || ((uintptr_t)C & 15) || ((uintptr_t)work & 15))
        return fail(FMM_EINVAL, "%s: pointers must be 16-byte aligned", who);
    if (flags & ~FMM_ACCUMULATE) return fail(FMM_EINVAL, "%s: unknown flags 0x%x", who, flags);
    const size_t bytes = ((size_t)1 << (2 * g)) * (size_t)p * p * sizeof(float);
    const char* a = (const char*)A;
    const char* c = (const char*)C;
    if (a < c + bytes && c < a + bytes) return fail(FMM_EINVAL, "%s: A and C overlap", who);
    if (work) {
        const char* w = (const char*)work;
        if ((w < a + bytes && a < w + bytes) || (w < c + bytes && c < w + bytes))
            return fail(FMM_EINVAL, "%s: work overlaps A or C", who);
    }
    return FMM_OK;
}

extern "C" {

int fgt_h2t(int32_t grid_log2, int32_t n_cut, int32_t p, int32_t prec, double sigma, const float* A, float* C,
            float* work, int32_t flags, void* stream)
{
    clear_error();
    int rc = fgt_check_args("fgt_h2t", grid_log2, n_cut, p, sigma, A, C, work, flags);
    if (rc) return rc;
    if (prec == FMM_TC_TF32X3) return fail(FMM_EUNSUPPORTED, "fgt_h2t: FMM_TC_TF32X3 is an M2L precision");
    if (prec != FMM_FP32 && prec != FMM_TC_BF16X3 && prec != FMM_TC_BF16)
        return fail(FMM_EINVAL, "fgt_h2t: unknown precision %d", prec);
    if (prec != FMM_FP32) {
        if (!fgt_h2t_tc_supported(grid_log2, n_cut, p))
            return fail(FMM_EUNSUPPORTED, "fgt_h2t: tensor-core precisions take p = 16, grid_log2 >= 3, n_cut <= 16");
        float* Y = work;
        if (!Y) {
            const size_t bytes = ((size_t)1 << (2 * grid_log2)) * (size_t)p * p * sizeof(float);
            if ((rc = fgt_workspace(bytes, &Y))) return rc;
        }
        return launch_fgt_h2t_tc(grid_log2, n_cut, sigma, prec == FMM_TC_BF16X3, A, Y, C, (flags & FMM_ACCUMULATE) != 0,
                                 (cudaStream_t)stream);
    }
    if (fgt_fused_supported(grid_log2))
        return launch_fgt_h2t_fused(grid_log2, n_cut, p, sigma, A, C, (flags & FMM_ACCUMULATE) != 0, (cudaStream_t)stream);
    float* Y = work;
    if (!Y) {
        const size_t bytes = ((size_t)1 << (2 * grid_log2)) * (size_t)p * p * sizeof(float);
        if ((rc = fgt_workspace(bytes, &Y))) return rc;
    }
    return launch_fgt_h2t(grid_log2, n_cut, p, sigma, A, Y, C, (flags & FMM_ACCUMULATE) != 0, true,
                          (cudaStream_t)stream);
}

int fgt_p2h(int32_t grid_log2, int32_t p, double sigma, const double* x, const double* q, int64_t n, float* A,
            int32_t flags, void* stream)
{
    clear_error();
    if (grid_log2 < 0 || grid_log2 > 12) return fail(FMM_EINVAL, "fgt_p2h: grid_log2 %d outside 0..12", grid_log2);
    if (p < 1 || p > 32) return fail(FMM_EINVAL, "fgt_p2h: p = %d outside 1..32", p);
    if (!(sigma > 0.0) || !(sigma < 1e300)) return fail(FMM_EINVAL, "fgt_p2h: sigma must be positive and finite");
    if (n < 0) return fail(FMM_EINVAL, "fgt_p2h: n < 0");
    if (!A || (n > 0 && (!x || !q))) return fail(FMM_EINVAL, "fgt_p2h: NULL pointer");
    if (flags & ~FMM_ACCUMULATE) return fail(FMM_EINVAL, "fgt_p2h: unknown flags 0x%x", flags);
    return launch_fgt_p2h(grid_log2, p, sigma, x, q, n, A, (flags & FMM_ACCUMULATE) != 0, (cudaStream_t)stream);
}

int fmm_sync_status(void* stream)
{
    clear_error();
    FMM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    int* w = nullptr;
    int rc = device_error_word(&w);
    if (rc) return rc;
    int h = 0;
    FMM_CUDA_TRY(cudaMemcpy(&h, w, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) FMM_CUDA_TRY(cudaMemset(w, 0, sizeof(int)));
    if (h & DEV_ERR_TIMEOUT) return fail(FMM_ETIMEOUT, "a bounded device-side wait timed out");
    if (h & DEV_ERR_CHECK) return fail(FMM_EDEVICE, "a device-side argument check failed");
    return FMM_OK;
}

}  // extern "C"
