// fgt_h2t_tc.cu -- FGT Hermite-to-Taylor translation (Sec. 2.2, Eq. C_beta with
// the factor (-1)^|beta| / beta!) on the 5th-generation tensor cores (tcgen05,
// TMEM accumulator), p = 16.
//
// Recasting.  With tensor truncation the neighbourhood sum separates into a
// pass along x and a pass along y, each a sum over 2 n_cut + 1 source offsets of
// p x p products with the Hankel matrix H_d[a][b] = h_{a+b}(u_d):
//   x pass  Y_(tx,sy)[b1][a2] = f(b1) sum_{sx} sum_{a1} h_{a1+b1}(u(tx - sx)) A_(sx,sy)[a1][a2]
//   y pass  C_(tx,ty)[b1][b2] = f(b2) sum_{sy} sum_{a2} h_{a2+b2}(u(ty - sy)) Y_(tx,sy)[b1][a2]
// with f(b) = (-1)^b / b!.  For 8 consecutive target boxes t0..t0+7 of one
// line (a row in the x pass, a column in the y pass) each pass is one dense
// product D[(i, r)][n] = sum_{(d, k)} W[(i + d, r)][k] H_d[k][n]:
//   M = 8 boxes x 16 rows r (a2 in the x pass, b1 in the y pass) = 128,
//   N = 16 (b1, b2),  K = (2 n_cut + 1) x 16 (source offset d, a1 or a2),
// where W is the line's window of 8 + 2 n_cut source boxes staged in shared
// memory as BF16 in the canonical K-major layout: the A operand of offset d is
// the window seen from box d on (a descriptor start shifted by 512 bytes per
// box), and H_d (the B operand) comes from a per-device BF16 image.  The y pass
// reads Y in transposed box order, so a column's boxes are contiguous.
//
// Precision: the BF16 hi/lo split, three products (W_hi H_hi + W_hi H_lo +
// W_lo H_hi) accumulated in FP32 (FMM_TC_BF16X3), or W_hi H_hi alone
// (FMM_TC_BF16).
//
// Schedule: one cooperative launch.  Every CTA (256 threads) takes line
// segments of the x pass round-robin, all CTAs meet at a grid barrier (Y is
// complete), then the same for the y pass.  Per segment: all threads stage the
// window (FP32 loads, all in flight at once, BF16 hi/lo stores); two threads
// issue the MMAs, one the even source offsets and one the odd, into two
// accumulators (a thread issues an MMA only every ~60 cycles, and these MMAs
// are short), each committing to its own mbarrier; with the split, the hi and
// lo planes of H_d form one N = 32 B operand, so W_hi H_hi and W_hi H_lo are
// one MMA and W_lo H_hi a second; warps 0-3 (one per TMEM lane quarter) sum the
// accumulators' column blocks.  The H_d image is copied by cp.async while the
// first window is staged.  Every wait is bounded: on timeout the CTA records
// FMM_ETIMEOUT in the device error word, waits (bounded) for its own MMAs,
// frees its TMEM and returns.
#include <cuda_bf16.h>

#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace fmmgb {

constexpr int kH2tTcP = 16;
constexpr int kH2tTcSeg = 8;           // target boxes per segment (M = 8 x 16 = 128)
constexpr int kH2tTcThreads = 256;
constexpr int kH2tTcMaxCut = 16;
constexpr int kH2tTcBox = 512;         // one box, one plane: 16 x 16 BF16, canonical K-major
constexpr int kH2tTcTmemCols = 64;     // two accumulators of 32 columns (one per MMA issuer)
// 16-byte words of a window per thread: every load of a window is issued before any is used
constexpr int kH2tTcLoads = (kH2tTcSeg + 2 * kH2tTcMaxCut) * 64 / kH2tTcThreads;

// byte offset of element (row r, column k) of a 16 x 16 K-major BF16 block:
// 8-row x 16-byte core matrices, 128 bytes between K chunks, 256 between row groups
__host__ __device__ __forceinline__ int h2t_tc_off(int r, int k)
{
    return (r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// The BF16 image of H_d for d = 0 .. 2 n_cut (source offset d - n_cut):
// [d][hi, lo][n][k] with value h_{k+n}(u), u = -(d - n_cut) ustep, from the
// recurrence h_{j+1} = 2u h_j - 2j h_{j-1} in FP64.  The hi and lo blocks of one
// d are one 32-row B operand [hi; lo], so W_hi H_hi and W_hi H_lo are one MMA.
__global__ void h2t_tc_image_kernel(int ncut, double ustep, unsigned char* __restrict__ img)
{
    const int d = blockIdx.x;
    const int idx = threadIdx.x;  // (n, k), 256 threads
    const int n = idx >> 4, k = idx & 15;
    const double u = -(double)(d - ncut) * ustep;
    double hm = exp(-u * u), h = 2.0 * u * hm;  // h_0, h_1
    const int j = n + k;
    double v = j == 0 ? hm : h;
    for (int i = 1; i < j; ++i) {
        const double hn = 2.0 * u * h - 2.0 * (double)i * hm;
        hm = h;
        h = hn;
        v = h;
    }
    const __nv_bfloat16 hi = __double2bfloat16(v);
    const __nv_bfloat16 lo = __double2bfloat16(v - (double)__bfloat162float(hi));
    unsigned char* blk = img + (size_t)d * 2 * kH2tTcBox;
    *reinterpret_cast<__nv_bfloat16*>(blk + h2t_tc_off(n, k)) = hi;
    *reinterpret_cast<__nv_bfloat16*>(blk + kH2tTcBox + h2t_tc_off(n, k)) = lo;
}

struct H2tTcArgs {
    const float* A;            // [4^g][16][16] Hermite coefficients A[box][a1][a2]
    float* Y;                  // [4^g][16][16] x-pass result, box index tx * 2^g + sy
    float* C;                  // [4^g][16][16] Taylor coefficients C[box][b1][b2]
    const unsigned char* img;  // BF16 image of H_d, (2 n_cut + 1) x 1 KB
    int* bar;                  // [2]: grid-barrier arrivals, CTAs finished (zero between launches)
    int* err;
    int g, ncut, split, accumulate;
};

__device__ __forceinline__ bool h2t_tc_grid_wait(const int* bar, int target)
{
    for (uint32_t it = 0; it < kSpinCap; ++it) {
        int v;
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
        if (v >= target) return true;
    }
    return false;
}

__global__ void __launch_bounds__(kH2tTcThreads) fgt_h2t_tc_kernel(H2tTcArgs a)
{
    extern __shared__ __align__(1024) unsigned char hsm[];
    const int taps = 2 * a.ncut + 1, nw = kH2tTcSeg + 2 * a.ncut;
    unsigned char* win_hi = hsm;                                  // [nw] boxes
    unsigned char* win_lo = hsm + (size_t)nw * kH2tTcBox;         // [nw] boxes
    unsigned char* himg = win_lo + (size_t)nw * kH2tTcBox;        // [taps][hi, lo]
    uint64_t* mbar = reinterpret_cast<uint64_t*>(himg + (size_t)taps * 2 * kH2tTcBox);  // [2], one per issuer
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = 1 << a.g, segs = N / kH2tTcSeg, nseg = N * segs;

    // a window's FP32 words into registers, every load in flight at once: boxes t0 - ncut ..
    // t0 + 7 + ncut of line `line` of `src` (x pass: A, a row; y pass: Y, a column), zero outside
    float4 vin[kH2tTcLoads];
    auto load_window = [&](const float* src, int line, int t0) {
#pragma unroll
        for (int j = 0; j < kH2tTcLoads; ++j) {
            const int e = tid + j * kH2tTcThreads;
            const int w = e >> 6, q = e & 63;  // window box, float4 of the box
            const int pos = t0 - a.ncut + w;
            vin[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (e < nw * 64 && pos >= 0 && pos < N)
                vin[j] = __ldg(reinterpret_cast<const float4*>(src + ((size_t)line * N + pos) * 256) + q);
        }
    };
    // the first segment's window is requested before the set-up
    if ((int)blockIdx.x < nseg) load_window(a.A, (int)blockIdx.x / segs, ((int)blockIdx.x % segs) * kH2tTcSeg);

    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"((uint32_t)kH2tTcTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the H_d image into shared memory by cp.async, in flight while the first window is staged
    {
        const unsigned char* src = a.img;
        const int nimg = taps * 2 * kH2tTcBox / 16;
        for (int i = tid; i < nimg; i += kH2tTcThreads) cp_async16(himg + (size_t)i * 16, src + (size_t)i * 16, true);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    // (-1)^n / n!, n = 0..15 (FP32 constants: no FP64 arithmetic in the kernel)
    constexpr float fac[kH2tTcP] = {1.0f,
                                    -1.0f,
                                    1.0f / 2,
                                    -1.0f / 6,
                                    1.0f / 24,
                                    -1.0f / 120,
                                    1.0f / 720,
                                    -1.0f / 5040,
                                    1.0f / 40320,
                                    -1.0f / 362880,
                                    1.0f / 3628800,
                                    -1.0f / 39916800,
                                    1.0f / 479001600,
                                    -1.0f / 6227020800.0f,
                                    1.0f / 87178291200.0f,
                                    -1.0f / 1307674368000.0f};
    // M = 128; N = 16 (one plane of H_d) or 32 ([hi; lo] of H_d)
    const uint32_t idesc16 = (1u << 4) | (1u << 7) | (1u << 10) | (2u << 17) | ((128u >> 4) << 24);
    const uint32_t idesc32 = (1u << 4) | (1u << 7) | (1u << 10) | (4u << 17) | ((128u >> 4) << 24);
    bool ok = true;
    int phase = 0;  // MMA commits waited on so far (per issuer)
    bool img_waited = false;

    for (int pass = 0; pass < 2 && ok; ++pass) {
        const float* src = pass ? a.Y : a.A;
        for (int s = blockIdx.x; s < nseg && ok; s += gridDim.x) {
            const int line = s / segs, t0 = (s % segs) * kH2tTcSeg;
            // ---- stage the window: boxes t0 - ncut .. t0 + 7 + ncut of the line, zero outside the grid.
            // x pass: box (sx, sy = line) of A, rows r = a2, columns k = a1 (a transpose);
            // y pass: box (tx = line, sy) of Y, rows r = b1, columns k = a2.
            if (pass > 0 || s != (int)blockIdx.x) load_window(src, line, t0);
#pragma unroll
            for (int j = 0; j < kH2tTcLoads; ++j) {
                const int e = tid + j * kH2tTcThreads;
                if (e >= nw * 64) break;
                const int w = e >> 6, q = e & 63;
                const float4 v = vin[j];
                const int o = q >> 2, i0 = (q & 3) * 4;  // element (o, i0 .. i0 + 3) of the box
                unsigned char* bh = win_hi + (size_t)w * kH2tTcBox;
                unsigned char* bl = win_lo + (size_t)w * kH2tTcBox;
                const float f[4] = {v.x, v.y, v.z, v.w};
                if (pass == 0) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const __nv_bfloat16 hi = __float2bfloat16_rn(f[j]);
                        const __nv_bfloat16 lo = __float2bfloat16_rn(f[j] - __bfloat162float(hi));
                        *reinterpret_cast<__nv_bfloat16*>(bh + h2t_tc_off(i0 + j, o)) = hi;
                        *reinterpret_cast<__nv_bfloat16*>(bl + h2t_tc_off(i0 + j, o)) = lo;
                    }
                } else {
                    uint32_t hw[2], lw[2];
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const __nv_bfloat162 hv = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
                        const float2 hf = __bfloat1622float2(hv);
                        hw[j] = *reinterpret_cast<const uint32_t*>(&hv);
                        lw[j] = pack_bf16(f[2 * j] - hf.x, f[2 * j + 1] - hf.y);
                    }
                    *reinterpret_cast<uint2*>(bh + h2t_tc_off(o, i0)) = make_uint2(hw[0], hw[1]);
                    *reinterpret_cast<uint2*>(bl + h2t_tc_off(o, i0)) = make_uint2(lw[0], lw[1]);
                }
            }
            if (!img_waited) {
                asm volatile("cp.async.wait_all;" ::: "memory");
                img_waited = true;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();

            // ---- D = sum_d W(from box d) H_d: two threads issue the MMAs, issuer j the offsets
            // d = j, j + 2, ... into accumulator j (TMEM columns 32 j ..); with the split, per d one
            // N = 32 product W_hi [H_hi; H_lo] (columns 0-15 and 16-31) and one N = 16 product
            // W_lo H_hi into columns 0-15 ----
            if (lane == 0 && warp < 2) {
                const int j = warp;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t wh = su32(win_hi), wl = su32(win_lo), hb = su32(himg);
                const uint32_t acc = tmem + (uint32_t)(32 * j);
                for (int d = j; d < taps; d += 2) {
                    const uint64_t ahi = umma_desc(wh + (uint32_t)(d * kH2tTcBox), 128, 256);
                    const uint64_t bhl = umma_desc(hb + (uint32_t)(d * 2 * kH2tTcBox), 128, 256);
                    const uint32_t first = d > j ? 1u : 0u;
                    if (a.split) {
                        const uint64_t alo = umma_desc(wl + (uint32_t)(d * kH2tTcBox), 128, 256);
                        umma_bf16(acc, ahi, bhl, idesc32, first);
                        umma_bf16(acc, alo, bhl, idesc16, 1u);
                    } else {
                        umma_bf16(acc, ahi, bhl, idesc16, first);
                    }
                }
                if (j < taps) umma_commit(&mbar[j]);
                else mbar_arrive(&mbar[j]);  // no offset for this issuer (n_cut = 0)
            }
            const bool done = mbar_wait(&mbar[0], (uint32_t)(phase & 1), 32) && mbar_wait(&mbar[1], (uint32_t)(phase & 1), 32);
            ++phase;
            if (!__syncthreads_and(done ? 1 : 0)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

            // ---- epilogue: warp q drains TMEM lanes 32 q .. 32 q + 31 = rows (i, r) ----
            if (warp < 4) {
                // the sum of the used column blocks: accumulator 0 (and 1 when n_cut > 0), each
                // columns 0-15 (and 16-31, W_hi H_lo, with the split)
                uint32_t rv[16], tv[16];
                const uint32_t lanes = (uint32_t)(warp * 32) << 16;
                tmem_ld16(tmem + lanes, rv);
                const int nblk = (a.split ? 2 : 1) * (taps > 1 ? 2 : 1);
                for (int b = 1; b < nblk; ++b) {
                    const uint32_t col = a.split ? (uint32_t)(32 * (b >> 1) + 16 * (b & 1)) : (uint32_t)(32 * b);
                    tmem_ld16(tmem + lanes + col, tv);
#pragma unroll
                    for (int n = 0; n < kH2tTcP; ++n) rv[n] = __float_as_uint(__uint_as_float(rv[n]) + __uint_as_float(tv[n]));
                }
                const int row = warp * 32 + lane, i = row >> 4, r = row & 15;
                if (pass == 0) {
                    // Y at box (tx, sy) stored as tx * N + sy: [b1 = n][a2 = r]
                    float* dst = a.Y + ((size_t)(t0 + i) * N + line) * 256 + r;
#pragma unroll
                    for (int n = 0; n < kH2tTcP; ++n) dst[n * 16] = __uint_as_float(rv[n]) * fac[n];
                } else {
                    // C at box (tx = line, ty = t0 + i): [b1 = r][b2 = n]
                    float4* dst = reinterpret_cast<float4*>(a.C + ((size_t)(t0 + i) * N + line) * 256 + r * 16);
#pragma unroll
                    for (int n4 = 0; n4 < 4; ++n4) {
                        float4 o = make_float4(__uint_as_float(rv[4 * n4]) * fac[4 * n4],
                                               __uint_as_float(rv[4 * n4 + 1]) * fac[4 * n4 + 1],
                                               __uint_as_float(rv[4 * n4 + 2]) * fac[4 * n4 + 2],
                                               __uint_as_float(rv[4 * n4 + 3]) * fac[4 * n4 + 3]);
                        if (a.accumulate) {
                            const float4 c = dst[n4];
                            o.x += c.x;
                            o.y += c.y;
                            o.z += c.z;
                            o.w += c.w;
                        }
                        dst[n4] = o;
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();  // the window and the accumulator are free for the next segment
        }
        if (pass == 0 && ok) {
            // grid barrier: every CTA's Y is written (all CTAs are resident: cooperative launch)
            bool got = true;
            if (tid == 0) {
                __threadfence();
                atomicAdd(a.bar, 1);
                got = h2t_tc_grid_wait(a.bar, (int)gridDim.x);
            }
            if (!__syncthreads_and(got ? 1 : 0)) ok = false;
        }
    }
    if (!ok && tid == 0) {
        atomicOr(a.err, DEV_ERR_TIMEOUT);
        // commits may be outstanding: wait (bounded) for them before the TMEM is freed
        if (phase > 0) {
            mbar_wait(&mbar[0], (uint32_t)((phase - 1) & 1));
            mbar_wait(&mbar[1], (uint32_t)((phase - 1) & 1));
        }
    }
    if (!img_waited) asm volatile("cp.async.wait_all;" ::: "memory");  // no copy left in flight
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)kH2tTcTmemCols)
                     : "memory");
    // the last CTA to finish returns the barrier words to zero for the next launch
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(a.bar + 1, 1) == (int)gridDim.x - 1) {
            atomicExch(a.bar, 0);
            atomicExch(a.bar + 1, 0);
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
bool fgt_h2t_tc_supported(int g, int ncut, int p) { return p == kH2tTcP && g >= 3 && ncut <= kH2tTcMaxCut; }

static size_t h2t_tc_smem(int ncut)
{
    const int taps = 2 * ncut + 1, nw = kH2tTcSeg + 2 * ncut;
    return (size_t)2 * nw * kH2tTcBox + (size_t)taps * 2 * kH2tTcBox + 64;  // + two mbarriers and the TMEM slot
}

// Per-device cache of H_d images, keyed by (device, n_cut, step bits).
static std::mutex g_img_mu;
static std::map<std::tuple<int, int, uint64_t>, unsigned char*> g_imgs;

static int h2t_tc_image(int ncut, double ustep, const unsigned char** out)
{
    int dev = 0;
    FMM_CUDA_TRY(cudaGetDevice(&dev));
    uint64_t bits;
    memcpy(&bits, &ustep, sizeof bits);
    const auto key = std::make_tuple(dev, ncut, bits);
    std::lock_guard<std::mutex> lk(g_img_mu);
    auto it = g_imgs.find(key);
    if (it != g_imgs.end()) {
        *out = it->second;
        return FMM_OK;
    }
    const int taps = 2 * ncut + 1;
    unsigned char* img = nullptr;
    FMM_CUDA_TRY(cudaMalloc(&img, (size_t)taps * 2 * kH2tTcBox));
    cudaStream_t st;
    FMM_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    h2t_tc_image_kernel<<<taps, 256, 0, st>>>(ncut, ustep, img);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (e != cudaSuccess) {
        cudaFree(img);
        return cuda_fail(e, "building the FGT H2T tensor-core image");
    }
    g_imgs[key] = img;
    *out = img;
    return FMM_OK;
}

int launch_fgt_h2t_tc(int g, int ncut, double sigma, bool split, const float* A, float* Y, float* C, bool acc,
                      cudaStream_t st)
{
    int* err = nullptr;
    int rc = device_error_word(&err);
    if (rc) return rc;
    const double ustep = ldexp(1.0, -g) / (sqrt(2.0) * sigma);
    const unsigned char* img = nullptr;
    if ((rc = h2t_tc_image(ncut, ustep, &img))) return rc;
    int* bar = nullptr;
    if ((rc = tile_counter(&bar, st))) return rc;
    const size_t smem = h2t_tc_smem(ncut);
    static unsigned long long opted;
    if ((rc = smem_opt_in((const void*)fgt_h2t_tc_kernel, (int)h2t_tc_smem(kH2tTcMaxCut), &opted))) return rc;
    int sms = 0, occ = 0;
    if ((rc = device_sm_count(&sms))) return rc;
    FMM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fgt_h2t_tc_kernel, kH2tTcThreads, smem));
    if (occ < 1) return fail(FMM_ECUDA, "fgt_h2t (tensor cores): the kernel cannot be resident");
    const int N = 1 << g, nseg = N * (N / kH2tTcSeg);
    const int grid = nseg < sms * occ ? nseg : sms * occ;
    H2tTcArgs args;
    args.A = A;
    args.Y = Y;
    args.C = C;
    args.img = img;
    args.bar = bar;
    args.err = err;
    args.g = g;
    args.ncut = ncut;
    args.split = split ? 1 : 0;
    args.accumulate = acc ? 1 : 0;
    // one cooperative launch: every CTA is resident, so the grid barrier between the passes completes
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kH2tTcThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    FMM_CUDA_TRY(cudaLaunchKernelEx(&cfg, fgt_h2t_tc_kernel, args));
    return FMM_OK;
}

}  // namespace fmmgb
