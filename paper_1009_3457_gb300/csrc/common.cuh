// common.cuh -- internal declarations shared by the translation units of libfmmgb.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fmmgb.h"

namespace fmmgb {

// ---------------------------------------------------------------------------
// error reporting (thread-local message, status codes of fmmgb.h)
// ---------------------------------------------------------------------------
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
void clear_error();

#define FMM_CUDA_TRY(expr)                                  \
    do {                                                    \
        cudaError_t e__ = (expr);                           \
        if (e__ != cudaSuccess) return cuda_fail(e__, #expr); \
    } while (0)

// ---------------------------------------------------------------------------
// device error word: bit 0 = a device-side check failed, bit 1 = a bounded
// wait timed out.  One word per device, library-owned.
// ---------------------------------------------------------------------------
enum : int { DEV_ERR_CHECK = 1, DEV_ERR_TIMEOUT = 2 };
int device_error_word(int** out);

// ---------------------------------------------------------------------------
// Placing points in the 2^g x 2^g grid over [0, 1)^2 without FP64 arithmetic.
// FP64 runs at a small fraction of the FP32 rate on this part, so a handful of
// FP64 operations per point sets the time of the kernels that only locate
// points (binning, P2M, L2P, the near-field sort).  A v in [0, 1) is
// m 2^(e - 52) with m its 53-bit significand and e < 0, so
//   X = floor(v 2^(g + 31)) = m >> (21 - e - g)
// exactly; X >> 31 = floor(v 2^g) is v's cell and the low 31 bits are its
// place in the cell in units of 2^-31 of a side.
// ---------------------------------------------------------------------------
// X for v in [0, 1) (g <= 20); false for v outside it (negative, -0, >= 1, infinite, NaN).
__device__ __forceinline__ bool grid_fixed31(double v, int g, long long& X)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    if (u >= 0x3FF0000000000000ull) return false;  // sign bit set, or v >= 1, inf, NaN
    const int e = (int)(u >> 52) - 1023;            // -1023 for 0 and subnormals: X = 0 below
    const int sh = 21 - e - g;
    const unsigned long long m = (u & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    X = sh >= 64 ? 0ll : (long long)(m >> sh);
    return true;
}

// floor(v 2^g) clamped to 0..2^g-1, NaN to 0 (the cell of a coordinate).
__device__ __forceinline__ int grid_cell(double v, int g)
{
    long long X;
    if (grid_fixed31(v, g, X)) return (int)(X >> 31);
    return v >= 1.0 ? (1 << g) - 1 : 0;
}

// v's offset from the centre of its cell, in cell sides, from X (|result| <= 1/2;
// truncated to 2^-31 of a side, then rounded to FP32).
__device__ __forceinline__ float cell_offset31(long long X)
{
    return (float)((int)(X & 0x7FFFFFFFll) - (1 << 30)) * 4.656612873077393e-10f;  // 2^-31
}

// Binomials C(n, k), n, k < 64, as a table in device memory built at compile time
// (Pascal's rule in FP64, exact up to 2^53, then rounded to FP32: exact while
// C(n, k) < 2^24, every n < 25), row n at kBinom.v[64 n], zero for k > n.  The
// M2M / L2L kernels and their adjoints read it instead of a per-step recurrence
// with an FP32 division.
struct BinomTable64 {
    float v[64 * 64];
};
constexpr BinomTable64 make_binom_table64()
{
    BinomTable64 t{};
    double row[64] = {1.0};
    for (int n = 0; n < 64; ++n) {
        if (n > 0)
            for (int k = n; k > 0; --k) row[k] += row[k - 1];
        for (int k = 0; k < 64; ++k) t.v[n * 64 + k] = k <= n ? (float)row[k] : 0.f;
    }
    return t;
}
__device__ constexpr BinomTable64 kBinom = make_binom_table64();

// 2^-k as an FP32 bit pattern (0 <= k <= 126).
__device__ __forceinline__ float pow2_neg(int k) { return __int_as_float((127 - k) << 23); }

// Number of SMs of the current device (cached).
int device_sm_count(int* out);

// Opt `func` into `bytes` of dynamic shared memory on the current device,
// once per device (`done` is a per-kernel bitmask of device ordinals 0..63;
// higher ordinals are refused with FMM_EUNSUPPORTED): the attribute
// persists, so later launches, including those inside a stream capture,
// make no runtime call besides the launch itself.
int smem_opt_in(const void* func, int bytes, unsigned long long* done);

// A work counter for one persistent launch: a slot of two ints (claimed
// work, CTAs finished) from a per-device ring of 256, zero when allocated.
// The kernel's last CTA to finish sets both back to zero, so no reset is
// enqueued per launch and a captured graph replays with the same slot.
// Launches that overlap on the GPU use different slots unless 256 or more
// are in flight at once.
int tile_counter(int** out, cudaStream_t st);

// A per-device scratch for the FGT Hermite evaluation (grids up to 1024 x
// 1024 boxes): 4^10 bytes of non-empty flags, one per box, then 4^10 + 1
// ints of the claim table; refilled before each evaluation, allocated on
// first use (or by fmm_prepare).
constexpr size_t kFgtFlagBytes = (size_t)1 << 20;
// flags [2^20 bytes], claims [2^20 + 1], then the Hermite evaluation's claim order: order [2^20],
// row prefix [2^20], key histogram [1091], cursors [1092], keys [2^20] (ints)
constexpr size_t kFgtScratchBytes = kFgtFlagBytes + (((size_t)1 << 20) + 1) * sizeof(int) +
                                    (3 * ((size_t)1 << 20) + 2 * 1091 + 1) * sizeof(int);
int fgt_flag_buffer(unsigned char** out);

// ---------------------------------------------------------------------------
// offset codes: box offset (dx, dy) = source - target, |dx|,|dy| <= 3
// ---------------------------------------------------------------------------
constexpr int kOffsetSlots = 49;  // 7 x 7 grid; the 9 central slots are never used
__host__ __device__ constexpr int offset_slot(int dx, int dy) { return (dy + 3) * 7 + (dx + 3); }

// Per child class c = (tx & 1) + 2 (ty & 1): the 27 interaction-list offsets,
// as (parent offset ex, ey in -1..1, source child class c').  Filled on the
// host by class_stencil(); the kernels get a copy in constant memory.
struct StencilEntry {
    int8_t ex, ey;   // parent offset
    int8_t csrc;     // source child class
    int8_t slot;     // offset_slot(dx, dy)
};
void class_stencil(int cls, StencilEntry out[27]);

// ---------------------------------------------------------------------------
// M2L operator tables (per device, per p), built by a GPU FP64 kernel.
//
// Scaled operator of offset D = (x_t - x_s)/r (a complex integer):
//   T[n][k] = (-1)^n C(n+k,k) D^-(n+k+1) = a_n h_D[n+k] b_k,
//   a_n = (-1)^n / (n! s^n),  b_k = 1 / (k! s^k),  h_D[j] = j! s^j D^-(j+1),
// a Hankel matrix between two diagonal scalings.  The balance factor s keeps
// every factor well inside FP32 range for p <= 32.
// ---------------------------------------------------------------------------
struct M2LTables {
    int p = 0;
    double s = 0.0;
    float2* h_fwd = nullptr;   // [49][2p-1] complex: forward M2L
    float2* h_adj = nullptr;   // [49][2p-1]: plain adjoint  (= -h_fwd)
    float2* h_adjc = nullptr;  // [49][2p-1]: conjugate adjoint (= -conj h_fwd)
    float* a = nullptr;        // [p] post-scale
    float* b = nullptr;        // [p] pre-scale
    // dense scaled operators for the tensor-core path, built on demand:
    // [0] forward, [1] plain adjoint (-T), [2] conjugate adjoint (-conj T)
    // [0] BF16 hi/lo, [1] TF32 hi/lo operands
    void* tc_w[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    int tc_ready[2][3] = {{0, 0, 0}, {0, 0, 0}};
};
int get_m2l_tables(int p, const M2LTables** out);
double m2l_balance(int p);

// One launch of the M2L stencil over several uniform levels (kernel parameter).
struct M2LLevel {
    const float2* M;          // [4^level][p] scaled MEs
    float2* L;                // [4^level][p] scaled LEs
    int level;
    int tile_begin;           // first CTA of this level (filled by the launcher)
    const uint8_t* exists;    // adaptive level: [4^level] box existence, NULL = every box exists
    const int32_t* tiles;     // adaptive level: the tiles to run (ntiles of them), NULL = all
    int ntiles;
    const int32_t* tc_tiles;  // adaptive level, tensor cores: the 8 x 32-parent tiles to run, NULL = all
    int tc_ntiles;
};
constexpr int kMaxLaunchLevels = FMM_MAX_LEVEL + 1;
struct M2LLaunch {
    M2LLevel lv[kMaxLaunchLevels];
    int nlev;
    int periodic;
    int accumulate;
};

// tree handle accessors (api.cu)
int tree_max_level(const fmm_tree* t);
int tree_periodic(const fmm_tree* t);
int tree_adaptive(const fmm_tree* t);
// Device data of an adaptive level: box existence [4^level] and the list of
// 4 x 4-parent tiles that hold an existing box (uploaded on first use,
// synchronously).  For a level where every box exists: NULL, NULL, -1.
int tree_device_level(const fmm_tree* t, int level, const uint8_t** exists, const int32_t** tiles, int* ntiles);
int tree_device_tc_tiles(const fmm_tree* t, int level, const int32_t** tiles, int* ntiles);

// launchers (m2l_fp32.cu)
int launch_build_m2l_tables(const M2LTables& t, cudaStream_t st);
bool m2l_fp32_supported(int p);
int launch_m2l_fp32(M2LLaunch& job, int p, const float2* hsel, const float* a, const float* b, cudaStream_t st);

// launchers (m2l_tc.cu)
bool m2l_tc_supported(int p);
bool m2l_tc_tf32_supported(int p);
size_t m2l_tc_image_bytes(int p, bool tf32);
int launch_build_tc_image(int p, double s, int variant, bool tf32, void* img, cudaStream_t st);
int launch_m2l_tc(M2LLaunch& job, int p, const void* img, bool split, bool tf32, cudaStream_t st);
int get_tc_image(int p, int variant, bool tf32, const void** out);
// Every check fmm_m2l_levels makes before it launches (flags 0), for a caller
// that validates its buffers once; with in = out = NULL the arguments other
// than the buffers (api.cu).
int m2l_levels_check(const char* who, const fmm_tree* tree, int32_t lmin, int32_t lmax, int32_t p, int32_t prec,
                     const void* const* in, void* const* out);
// Per-device flags of the tensor-core M2L, one per tile (zero between
// launches; grown on demand, zeroed when allocated).
int tc_flag_workspace(int ntiles, int** flags);

// launchers (fgt_h2t.cu)
bool fgt_supported(int p);
int fgt_max_cut();
// one launch (thread-block clusters, Y in distributed shared memory) for grids up to 32 x 32
bool fgt_fused_supported(int g);
int launch_fgt_h2t_fused(int g, int ncut, int p, double sigma, const float* A, float* C, bool acc, cudaStream_t st);
int launch_fgt_h2t(int g, int ncut, int p, double sigma, const float* A, float* Y, float* C, bool acc,
                   bool cached_table, cudaStream_t st);
int fgt_workspace(size_t bytes, float** out);
int fgt_check_args(const char* who, int g, int ncut, int p, double sigma, const float* A, const float* C,
                   const float* work, int flags);

// launchers (upward.cu)
int launch_p2m_binned(int level, int p, const double* xy, const double* c, int n, const int* perm,
                      const int* box_start, float2* M, bool acc, int* err, cudaStream_t st);
int launch_p2m(int level, int p, const double* xy, const double* c, int64_t n, float2* M, bool accumulate,
               cudaStream_t st);
int launch_m2m(int child_level, int p, const float2* Mc, float2* Mp, bool accumulate, cudaStream_t st);
// FGT H2T on the tensor cores (fgt_h2t_tc.cu): p = 16, grid_log2 >= 3, n_cut <= 16
bool fgt_h2t_tc_supported(int g, int ncut, int p);
int launch_fgt_h2t_tc(int g, int ncut, double sigma, bool split, const float* A, float* Y, float* C, bool acc,
                      cudaStream_t st);
int launch_m2m_adjoint(int child_level, int p, const float2* Wp, float2* Wc, bool accumulate, cudaStream_t st);
int launch_fgt_p2h(int g, int p, double sigma, const double* x, const double* q, int64_t n, float* A, bool acc,
                   cudaStream_t st);

}  // namespace fmmgb
