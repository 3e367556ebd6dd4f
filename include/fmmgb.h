/*
 * fmmgb.h -- C ABI of libfmmgb, the GB300 (sm_103a) M2L / FGT translation engine.
 *
 * The operations follow Cruz, Layton & Barba, "How to obtain efficient GPU
 * kernels: an illustration using FMM & FGT algorithms" (arXiv:1009.3457):
 *   - the downward sweep of the FMM: build interaction lists, translate every
 *     multipole expansion (ME) of a list into a local expansion (LE) about the
 *     target centre, and reduce (sum) them into the target's LE (Sec. 4.1,
 *     steps 1-3), with the M2L matrix of Eq. (M2Lmat);
 *   - the Hermite-to-Taylor translation of the fast Gauss transform
 *     (Sec. 2.2, Eq. C_beta).
 *
 * Conventions shared by every call
 * --------------------------------
 *   Kernel.  2-D Cauchy kernel 1/(z - y) on the complex plane: ME
 *     phi(z) = sum_{k<p} m_k (z - x_s)^-(k+1),  LE  phi(z) = sum_{n<p} l_n (z - x_t)^n,
 *     and M2L  l_n = sum_k (-1)^n C(n+k,k) (x_t - x_s)^-(n+k+1) m_k  (Eq. M2Lmat,
 *     x_t = target centre = the paper's x_i, x_s = source centre = x_j).
 *   Boxes.  Level l of the quadtree on [0,1)^2 has 2^l x 2^l boxes of side
 *     r_l = 2^-l; box (ix, iy) has index b = iy * 2^l + ix and centre
 *     ((ix + 1/2) r_l, (iy + 1/2) r_l).
 *   Coefficient units.  Coefficients cross this boundary radius-scaled:
 *     M~[b][k] = m_{b,k} / r_l^k,   L~[b][n] = l_{b,n} * r_l^(n+1).
 *     Scaled values stay O(1) at every depth, while physical FP32 values
 *     overflow (l_n ~ r^-(n+1)) below about level 7 at p = 16.  In these units
 *     the M2L operator depends only on the integer box offset.
 *   Layout.  An expansion array is [nbox][p] complex64 (interleaved re, im,
 *     8 bytes per coefficient, box-major), 16-byte aligned, on the device.
 *   Memory.  The caller owns every coefficient buffer.  The library owns the
 *     tree handle and its per-device operator tables (built by a GPU FP64
 *     kernel on first use of an order p on a device: call fmm_prepare() before
 *     stream capture to keep allocation out of the captured region).
 *   Streams.  `stream` is a cudaStream_t (NULL = legacy default stream).
 *     Calls enqueue work and return without synchronising.
 *   Errors.  Every call returns an fmm_status; FMM_OK is 0.  Arguments are
 *     checked on the host before any launch, and a failed check launches
 *     nothing.  fmm_last_error() returns a message for the calling thread's
 *     last failure.  Kernels never trap: a device-side check that fails sets a
 *     device error word that fmm_sync_status() reports.
 */
#ifndef FMMGB_H
#define FMMGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FMM_OK = 0,
    FMM_EINVAL = -1,        /* bad argument (null pointer, size, level, order) */
    FMM_ENOMEM = -2,        /* device or host allocation failed */
    FMM_ECUDA = -3,         /* a CUDA runtime call failed */
    FMM_ETIMEOUT = -4,      /* a bounded device-side wait gave up */
    FMM_EUNSUPPORTED = -5,  /* valid request the library does not implement */
    FMM_EDEVICE = -6        /* a device-side check failed (see fmm_last_error) */
} fmm_status;

typedef enum {
    FMM_FP32 = 0,           /* FP32 FFMA path (Hankel-structured stencil kernel) */
    FMM_TC_BF16X3 = 1,      /* tcgen05 tensor cores, BF16 hi/lo split, 3 products, FP32 accumulate */
    FMM_TC_BF16 = 2,        /* tcgen05 tensor cores, plain BF16 inputs, FP32 accumulate */
    FMM_TC_TF32X3 = 3       /* tcgen05 tensor cores, TF32 hi/lo split, 3 products, FP32 accumulate (M2L, p = 16) */
} fmm_prec;

/* flags for fmm_m2l / fmm_m2l_adjoint / fgt_h2t */
#define FMM_ACCUMULATE 1    /* add into the output instead of overwriting it */
#define FMM_CONJ 2          /* adjoint only: conjugate transpose instead of plain transpose */

/* flags for fmm_build_lists */
#define FMM_TREE_PERIODIC 1 /* wrap parent neighbours modulo 2^(l-1): every box has 27 entries */

/* Largest quadtree level accepted by fmm_build_lists. */
#define FMM_MAX_LEVEL 14

typedef struct fmm_tree fmm_tree; /* opaque, library-owned */

/* ---------------------------------------------------------------------------
 * fmm_build_lists -- quadtree decomposition and interaction lists
 * (Sec. 2.1 "Initialization"; Sec. 4.1 step 1).
 *
 * Interaction list of a box t at level l >= 2: the children of the parent's
 * neighbours (Chebyshev distance <= 1 at level l-1) that are not adjacent to
 * t (Chebyshev distance >= 2 at level l).  Levels 0 and 1 have none.  Each
 * entry carries an offset code  (dy + 3) * 7 + (dx + 3)  of the box offset
 * (dx, dy) = source - target, one of 40 values.
 *
 * Adaptive tree (leaf_cap = q > 0): the root exists; an existing box of
 * level l < max_level holding more than q points is split, and each of its
 * children holding at least one point exists (empty children are not
 * created).  Its lists are V-lists: the interaction-list rule above applied
 * to existing boxes only (the existing children of the parent's colleagues
 * that are not adjacent to t); a box that does not exist has an empty list.
 * Coefficient arrays stay dense, [4^level][p] per level: the translation
 * reads only existing sources and writes only existing targets (entries of
 * absent boxes are ignored on input and left untouched on output).
 *
 *   xy        host, n interleaved (x, y) points; a point goes to box
 *             floor(x 2^l) of each level, clamped to 0 .. 2^l - 1.  May be
 *             NULL when leaf_cap == 0 (a uniform tree does not depend on the
 *             points).
 *   n         number of points (>= 0).
 *   max_level deepest level, 2 .. FMM_MAX_LEVEL.
 *   leaf_cap  0: uniform tree with every level down to max_level.
 *             q > 0: adaptive tree with at most q points per leaf above
 *             max_level.
 *   flags     FMM_TREE_PERIODIC or 0 (periodic lists: uniform trees only).
 *   out       receives the handle; release it with fmm_tree_destroy().
 * Host-side and synchronous.  Lists are materialised on demand by
 * fmm_tree_level_info().  Returns FMM_EINVAL on a bad argument.
 * ------------------------------------------------------------------------- */
int fmm_build_lists(const double* xy, int64_t n, int32_t max_level, int32_t leaf_cap,
                    int32_t flags, fmm_tree** out);

typedef struct {
    int64_t nbox;              /* 4^level */
    int32_t side;              /* 2^level */
    int32_t list_stride;       /* 27 */
    int64_t ntranslations;     /* number of valid list entries at this level */
    const int32_t* list_host;  /* [nbox][27] source box index, -1 = empty slot */
    const int8_t* offcode_host;/* [nbox][27] offset code 0..48, -1 = empty slot */
    const int32_t* list_dev;   /* device copies of the two arrays above */
    const int8_t* offcode_dev;
    int64_t nexist;            /* boxes of the level that exist (nbox for a uniform tree) */
    const uint8_t* exists_host;/* [nbox] 1 = box exists; NULL when every box of the level exists */
} fmm_level_info;

/* Materialise (once) and return the interaction lists of one level.
 * Pointers stay valid until fmm_tree_destroy().  Allocates host and device
 * memory on first call for a level (synchronous).  On a machine without a
 * CUDA device the host arrays are still built and the device pointers are
 * NULL. */
int fmm_tree_level_info(const fmm_tree* tree, int32_t level, fmm_level_info* out);

/* Number of interaction-list entries at a level (no allocation). */
int64_t fmm_tree_translations(const fmm_tree* tree, int32_t level);

void fmm_tree_destroy(fmm_tree* tree);

/* Build the operator tables for order p on the current device (FP64 GPU
 * kernel, then FP32 copies, and the BF16 or TF32 tensor-core image for a
 * tensor-core prec).  Optional: fmm_m2l does it on first use.  Synchronous. */
int fmm_prepare(int32_t p, int32_t prec);

/* ---------------------------------------------------------------------------
 * fmm_m2l -- M2L translation of every interaction-list entry of one level,
 * fused with the reduction into each target's LE (Sec. 4.1 steps 2-3,
 * Eq. M2Lmat):
 *     L~_t[n] (+)= sum_{s in IL(t)} sum_{k<p} (-1)^n C(n+k,k) D^-(n+k+1) M~_s[k],
 *     D = (x_t - x_s) / r_l  (a complex integer: minus the box offset).
 *
 *   tree   handle from fmm_build_lists (uniform or adaptive tree).
 *   level  0 .. max_level; levels 0 and 1 have empty lists (the output is
 *          zeroed, or left unchanged with FMM_ACCUMULATE).
 *   p      number of terms: 6, 8, 12, 16 or 24.
 *   prec   FMM_FP32, FMM_TC_BF16X3, FMM_TC_BF16 or FMM_TC_TF32X3 (tensor-core
 *          forms: p = 16 or 24, FMM_TC_TF32X3 p = 16 only, FMM_EUNSUPPORTED
 *          otherwise; on an adaptive level they run the 8 x 32-parent tiles that
 *          hold an existing box, with absent sources read as zero and absent
 *          targets left untouched).  FMM_TC_TF32X3 splits operator and MEs into
 *          TF32 hi + lo (~21 significant bits each) and issues three products:
 *          close to FP32 accuracy, at twice the MMA count of FMM_TC_BF16X3.
 *   M      device, const, [4^level][p] complex64 scaled MEs (input).
 *   L      device, [4^level][p] complex64 scaled LEs (output; must not
 *          overlap M).
 *   flags  FMM_ACCUMULATE or 0.
 * ------------------------------------------------------------------------- */
int fmm_m2l(const fmm_tree* tree, int32_t level, int32_t p, int32_t prec,
            const void* M, void* L, int32_t flags, void* stream);

/* fmm_m2l_levels -- fmm_m2l for every level lmin..lmax in ONE launch (the
 * levels are independent given their MEs).  M[i], L[i] are the arrays of
 * level lmin + i (host array of device pointers, read during the call).
 * Equivalent to lmax - lmin + 1 calls of fmm_m2l.
 * Host-resident problems: fmm_host_stream_* (below) runs this call over a
 * stream of problems in host memory with the transfers overlapped.
 * Tensor-core precisions: one kernel per call; calls on different streams
 * must not overlap on the GPU (they share the library's per-device flags). */
int fmm_m2l_levels(const fmm_tree* tree, int32_t lmin, int32_t lmax, int32_t p, int32_t prec,
                   const void* const* M, void* const* L, int32_t flags, void* stream);

/* ---------------------------------------------------------------------------
 * fmm_m2l_adjoint -- transpose of fmm_m2l on the same lists:
 *     G~_s[k] (+)= sum_{t : s in IL(t)} sum_n a_nk W~_t[n]       (plain transpose)
 *     G~_s[k] (+)= sum_{t : s in IL(t)} sum_n conj(a_nk) W~_t[n] (flags & FMM_CONJ)
 * with a_nk the scaled entries of Eq. (M2Lmat) for the pair (t, s).  The
 * conjugate form is the gradient of a real objective with respect to the
 * multipole coefficients (PyTorch's convention for complex tensors).
 * Arguments as fmm_m2l with W (input, [nbox][p] complex64) in place of M and
 * G (output) in place of L; prec as fmm_m2l (the tensor-core forms run the
 * forward kernel with the operator image of -T or -conj T).
 * ------------------------------------------------------------------------- */
int fmm_m2l_adjoint(const fmm_tree* tree, int32_t level, int32_t p, int32_t prec,
                    const void* W, void* G, int32_t flags, void* stream);

/* fmm_m2l_adjoint over levels lmin..lmax in one launch (as fmm_m2l_levels). */

int fmm_m2l_adjoint_levels(const fmm_tree* tree, int32_t lmin, int32_t lmax, int32_t p, int32_t prec,
                           const void* const* W, void* const* G, int32_t flags, void* stream);

/* ---------------------------------------------------------------------------
 * Host-resident problems (Sec. 4.1's M2L stage served from host memory):
 * fmm_m2l_levels over a stream of problems whose MEs and LEs live in host
 * memory, each problem's copy in, translation and copy out overlapped with
 * its neighbours'.  The pipeline owns `depth` device buffer sets (MEs and LEs
 * of every level) and three non-blocking CUDA streams on the device current
 * at creation: host-to-device copies, translations, device-to-host copies.
 * Step i uses buffer set i mod depth.  Its MEs are copied in once the
 * translation that last read that set has finished; its translation waits
 * for its MEs and for the copy out of the LEs last written to that set; its
 * LEs are copied out once it has finished.  With depth >= 2 step i's
 * translation runs while step i+1's MEs arrive and step i-1's LEs leave.
 *
 * fmm_host_stream_create
 *   tree        uniform, periodic or adaptive tree handle; must outlive the
 *               pipeline.
 *   lmin, lmax  levels translated per step (as fmm_m2l_levels).
 *   p, prec     as fmm_m2l_levels (FMM_EUNSUPPORTED where it is).
 *   depth       device buffer sets, 1..8.
 *   out         receives the handle.
 * Allocates 2 * depth * entries * 8 bytes of device memory, entries =
 * p * sum_{l = lmin..lmax} 4^l complex64 values per direction and step.
 * Errors: FMM_EINVAL (tree, levels, order, depth, NULL out), FMM_EUNSUPPORTED,
 * FMM_ENOMEM / FMM_ECUDA (allocation, stream or event creation; nothing is
 * left allocated).
 * ------------------------------------------------------------------------- */
typedef struct fmm_host_stream fmm_host_stream; /* opaque, library-owned */
int fmm_host_stream_create(const fmm_tree* tree, int32_t lmin, int32_t lmax, int32_t p, int32_t prec,
                           int32_t depth, fmm_host_stream** out);

/* fmm_host_stream_submit -- enqueue one step and return.
 *   M_host  host array [lmax - lmin + 1] of HOST pointers: entry i is level
 *           lmin + i's const complex64 [4^l][p] scaled MEs.
 *   L_host  the same layout for the scaled LEs (output, overwritten).
 *   flags   0: one copy per level and direction.
 *           FMM_HOST_CONTIGUOUS: M_host[0] and L_host[0] each address ONE
 *           buffer (one allocation) holding all levels back to back, level
 *           lmin first; one copy per direction; the other entries are not
 *           read.  (Adjacent addresses alone do not make one buffer: two
 *           page-locked allocations can be neighbours, and a copy may not
 *           span them.)
 * The host buffers must stay valid, M_host unmodified and L_host
 * unread, until fmm_host_stream_sync() returns.  Page-locked buffers
 * (cudaHostAlloc, cudaHostRegister) let the copies run asynchronously;
 * pageable ones are accepted, and their copies then return only after the
 * data has been staged (no overlap on the host side).  A NULL entry, an
 * unknown flag, or an M level overlapping an L level is FMM_EINVAL, and
 * nothing is enqueued. */
#define FMM_HOST_CONTIGUOUS 8
int fmm_host_stream_submit(fmm_host_stream* hs, const void* const* M_host, void* const* L_host, int32_t flags);

/* Wait for every submitted step; returns what fmm_sync_status() returns for
 * the translation stream (device-side checks and timeouts included).
 * A pipeline is used by one host thread at a time (its calls are not
 * serialised against each other). */
int fmm_host_stream_sync(fmm_host_stream* hs);

/* Sizes, progress and streams of a pipeline.  The stream handles
 * (cudaStream_t) let a caller record events around submitted steps. */
typedef struct {
    int64_t entries;       /* complex64 values per step and direction */
    int64_t bytes_in;      /* host-to-device bytes per step (entries * 8) */
    int64_t bytes_out;     /* device-to-host bytes per step */
    int64_t steps;         /* steps submitted so far */
    int32_t depth;
    int32_t lmin, lmax, p, prec;
    void* h2d_stream;
    void* compute_stream;
    void* d2h_stream;
} fmm_host_stream_info_t;
int fmm_host_stream_info(const fmm_host_stream* hs, fmm_host_stream_info_t* out);

/* Wait for the pipeline's work, then free its buffers, events and streams. */
void fmm_host_stream_destroy(fmm_host_stream* hs);

/* ---------------------------------------------------------------------------
 * Batched M2L: many independent uniform-tree problems (each with its own
 * depth and p) translated in ONE persistent launch.  Each problem's levels
 * 2..max_level are split into work items (a 4 x 4 tile of parent boxes of one
 * level of one problem, the unit of fmm_m2l), ordered heaviest first
 * (p^2 x translations per tile); resident CTAs claim items from a work counter,
 * so the launch load-balances across problems of very different sizes.  The
 * per-problem semantics are exactly fmm_m2l_levels(trees[i], 2, max_level_i,
 * p[i], FMM_FP32, ...): levels 0 and 1 have no interaction lists and are not
 * passed.  (Sec. 4.1 steps 2-3, Eq. M2Lmat, applied per problem.)
 *
 * A plan (fmm_batch) owns the device copy of the item list and the launch
 * configuration; running it launches one kernel after a 4-byte counter reset,
 * both of which a CUDA stream capture can record, so a plan replays inside a
 * CUDA graph.
 *
 * fmm_batch_create
 *   trees     host array [nprob] of tree handles (uniform trees); must outlive
 *             the call only.
 *   p         host array [nprob]: 6, 8, 12 or 16 per problem.
 *   nprob     number of problems, 1..65536.
 *   M_levels  host array of device pointers: problem 0's levels 2..max_level_0,
 *             then problem 1's levels 2..max_level_1, and so on (sum over
 *             problems of max_level_i - 1 entries); level l of problem i is
 *             const complex64 [4^l][p_i] scaled MEs.  Pointers are copied into
 *             the plan: the buffers must stay allocated while the plan runs.
 *   L_levels  the same layout for the outputs (scaled LEs), each [4^l][p_i],
 *             none overlapping its own level's input.
 *   prec      FMM_FP32 (the only precision of the batched path).
 *   flags     FMM_ACCUMULATE (add into L), FMM_BATCH_AUTOTUNE (time the
 *             candidate launch configurations -- grid size, claim chunk -- and
 *             then the work-unit variants -- rows per lane, packed or scalar
 *             multiply-adds, halo loads in flight -- on this plan before
 *             returning, writing only library scratch, never L).  The choice
 *             is cached per GPU (name, SM count), precision and workload
 *             signature (p, level, periodicity and count of every (problem,
 *             level), accumulate) in memory and in a JSON file that later
 *             processes reload without timing: $FMMGB_TUNE_CACHE, else
 *             $HOME/.cache/fmmgb/m2l_batched_tune.json (none when neither
 *             is set).
 *   stream    the plan's device arrays are uploaded on this stream; the call
 *             returns after they are resident (it synchronises the stream).
 *   out       receives the plan.
 * Errors: FMM_EINVAL (bad argument; nothing allocated), FMM_EUNSUPPORTED (p or
 * prec outside the batched set), FMM_ENOMEM / FMM_ECUDA.
 * ------------------------------------------------------------------------- */
typedef struct fmm_batch fmm_batch; /* opaque, library-owned */
#define FMM_BATCH_AUTOTUNE 4

int fmm_batch_create(const fmm_tree* const* trees, const int32_t* p, int32_t nprob,
                     const void* const* M_levels, void* const* L_levels, int32_t prec, int32_t flags,
                     void* stream, fmm_batch** out);

/* Launch the plan on `stream` (asynchronous; no host synchronisation, no
 * allocation).  Runs of one plan must be ordered (same stream, or events):
 * they share the plan's work counter. */
int fmm_batch_run(fmm_batch* batch, void* stream);

/* Launch configuration and size of a plan. */
typedef struct {
    int64_t items;         /* work items (tiles) */
    int64_t translations;  /* interaction-list entries over all problems and levels */
    int32_t grid;          /* CTAs launched */
    int32_t chunk;         /* items claimed per work-counter update */
    int32_t persistent;    /* 1: grid < items, CTAs loop over claimed items */
    int32_t tuned;         /* 1: configuration chosen by timing (FMM_BATCH_AUTOTUNE) */
    float tuned_ms;        /* best timed run of the autotuner, 0 if not tuned */
    int32_t variant;       /* work-unit variant: index into the tuned set */
    int32_t form;          /* -1: each order's default (p/2 rows per lane, packed multiply-adds, the
                              sums of w Re m and w Im m apart at p = 12, 16); 0: p/2 rows per lane,
                              packed multiply-adds; 1: p rows per lane, half the list entries each;
                              2: p/2 rows per lane, scalar multiply-adds */
    int32_t loads;         /* halo loads a thread keeps in flight while staging a tile */
    int32_t from_cache;    /* 1: the tuned choice was reused (memory or cache file), not timed */
} fmm_batch_info_t;
int fmm_batch_info(const fmm_batch* batch, fmm_batch_info_t* out);

/* Free the plan's device arrays in stream order on `stream` (the plan may
 * still be running there) and the plan itself. */
void fmm_batch_destroy(fmm_batch* batch, void* stream);

/* One-shot form: create (without autotuning), run and destroy on `stream`,
 * fully stream-ordered (no host synchronisation after the upload). */
int fmm_m2l_batched(const fmm_tree* const* trees, const int32_t* p, int32_t nprob,
                    const void* const* M_levels, void* const* L_levels, int32_t prec, int32_t flags,
                    void* stream);

/* ---------------------------------------------------------------------------
 * fgt_h2t -- Hermite-to-Taylor translation of the fast Gauss transform over
 * a uniform grid of 2^g x 2^g boxes on [0,1)^2 (Sec. 2.2, Eq. C_beta, with
 * the factor (-1)^|beta| / beta! that the printed equation omits):
 *   C_t[b1][b2] (+)= sum_{s : max(|sx-tx|,|sy-ty|) <= n_cut}
 *        ((-1)^(b1+b2) / (b1! b2!)) sum_{a1,a2 < p} A_s[a1][a2] h_{a1+b1}(u1) h_{a2+b2}(u2),
 *   u = (t_C - s_B) / (sqrt(2) sigma),  h_n(t) = exp(-t^2) H_n(t)  (Hermite
 *   functions, Sec. 2.2), tensor truncation a_i, b_i < p.
 *
 *   grid_log2  g, 0..12; box b = iy * 2^g + ix, centre ((ix+1/2) 2^-g, (iy+1/2) 2^-g).
 *   n_cut      neighbourhood half-width in boxes, 0..16.
 *   p          Hermite order per dimension: 4, 8, 12 or 16.
 *   prec       FMM_FP32 (CUDA cores), or FMM_TC_BF16X3 / FMM_TC_BF16 (tcgen05
 *              tensor cores: each separable pass as a dense product of 8 target
 *              boxes x 16 rows by (2 n_cut + 1) x 16 over the BF16 hi/lo split,
 *              three products or one, FP32 accumulation; p = 16, grid_log2 >= 3,
 *              one cooperative launch; FMM_EUNSUPPORTED otherwise, also for
 *              FMM_TC_TF32X3).  Any other value: FMM_EINVAL.
 *   sigma      Gaussian width (exp(-|x-y|^2 / (2 sigma^2))), > 0.
 *   A          device, const, [4^g][p][p] float32 Hermite coefficients
 *              A[b][a1][a2] (a1: x order, a2: y order), Eq. A_alpha.
 *   C          device, [4^g][p][p] float32 Taylor coefficients C[b][b1][b2].
 *   work       device scratch of 4^g p^2 floats, or NULL to use a
 *              library-owned per-device buffer (allocated on first use of a
 *              size; concurrent calls on different streams must then not
 *              overlap on the GPU).  Must not overlap A or C.
 *   flags      FMM_ACCUMULATE or 0.
 * All pointers 16-byte aligned; A and C must not overlap.
 * ------------------------------------------------------------------------- */
int fgt_h2t(int32_t grid_log2, int32_t n_cut, int32_t p, int32_t prec, double sigma, const float* A, float* C,
            float* work, int32_t flags, void* stream);

/* ---------------------------------------------------------------------------
 * fgt_h2t_noalloc -- fgt_h2t that never allocates device memory.
 *
 * The paper has no counterpart.  Some callers cannot call cudaMalloc and
 * cannot hand the library a `work` buffer either: a host application whose
 * caching allocator or fixed memory pool owns all of the device's memory, a
 * plugin that is not allowed to allocate behind its host's back, or a
 * latency-critical loop in which an allocation (which may synchronise the
 * whole device) is not acceptable.  For them the intermediate of the two
 * passes lives in a fixed 1 MiB array compiled into the library:
 * 4^g * p^2 must not exceed 262,144 floats (for example grids up to 32 x 32
 * boxes at p = 16, 64 x 64 at p = 8); larger requests are rejected with
 * FMM_EINVAL and a message, and fgt_h2t serves them.  Every GPU that loads the
 * library keeps that array for the life of the process.
 *
 * Arguments and results are those of fgt_h2t (FMM_FP32) without `prec` and `work`; A and C must not
 * lie inside the built-in array (FMM_EINVAL).  Set-up on first use, none of it
 * an allocation: the first call on a device looks up the array's device
 * address, and the first call of each p on a device sets that kernel's
 * shared-memory limit.  Make those first calls before any stream capture.
 * All calls share the one array and each overwrites it completely before
 * reading it, so nothing needs clearing; calls that overlap on the GPU
 * (different streams, or a graph replay running beside another call) race on
 * it and must be serialised by the caller.
 * ------------------------------------------------------------------------- */
int fgt_h2t_noalloc(int32_t grid_log2, int32_t n_cut, int32_t p, double sigma, const float* A, float* C,
                    int32_t flags, void* stream);

/* ---------------------------------------------------------------------------
 * Support for building M2L inputs on the device (upward sweep, Sec. 2.1
 * stage 2; not the translation path itself).
 *
 * fmm_p2m: M~_b[k] (+)= sum_{i in box b} c_i ((y_i - x_b) / r_l)^k for every
 *   box of `level`; a point goes to box floor(x 2^l) clamped to 2^l - 1.
 *   xy: device float64 [n][2]; c: device float64 [n]; M: device complex64
 *   [4^level][p].  Uses FP32 atomic additions (result order-dependent in the
 *   last bits).  flags: FMM_ACCUMULATE or 0.
 * fmm_m2m: parent MEs from child MEs, M_j = sum_{k<=j} C(j,k)(x_c - x_P)^(j-k) m_k,
 *   in scaled units (FP32; the scaled entries are exact in FP32).
 *   Mc: [4^child_level][p], Mp: [4^(child_level-1)][p].
 * ------------------------------------------------------------------------- */
int fmm_p2m(int32_t level, int32_t p, const double* xy, const double* c, int64_t n,
            void* M, int32_t flags, void* stream);
int fmm_m2m(int32_t child_level, int32_t p, const void* Mc, void* Mp, int32_t flags, void* stream);
/* fmm_m2m_adjoint: conjugate transpose of fmm_m2m:
 *   Wc[child][k] (+)= sum_{j>=k} conj(C(j,k) z^(j-k) 2^-k) Wp[parent][j],
 *   z = (x_child - x_parent) / r_parent.  Wp: [4^(child_level-1)][p], Wc: [4^child_level][p].
 *   flags: FMM_ACCUMULATE. */
int fmm_m2m_adjoint(int32_t child_level, int32_t p, const void* Wp, void* Wc, int32_t flags, void* stream);

/* ---------------------------------------------------------------------------
 * Far-field stages around the M2L path (Sec. 2.1 stages 3-4), scaled units,
 * with the conjugate transposes that carry the gradient of a real objective
 * back through them (PyTorch's convention for complex tensors).  p: 1..64.
 * Coefficient arrays complex64, 8-byte aligned.  Support for the gradient
 * chain of the translation path, not part of the translation itself.
 *
 * fmm_l2l: L~c[j] (+)= sum_{n>=j} C(n,j) u^(n-j) 2^-(j+1) L~p[n] for every box
 *   of child_level, u = (x_child - x_parent) / r_parent = (+-1/4, +-1/4).
 *   Lp: [4^(child_level-1)][p]; Lc: [4^child_level][p].  flags: FMM_ACCUMULATE.
 * fmm_l2l_adjoint: Wp[parent] (+)= sum_{its 4 children} T_c^H Wc[child]
 *   (Wc: [4^child_level][p], Wp: [4^(child_level-1)][p]).
 * ------------------------------------------------------------------------- */
int fmm_l2l(int32_t child_level, int32_t p, const void* Lp, void* Lc, int32_t flags, void* stream);
int fmm_l2l_adjoint(int32_t child_level, int32_t p, const void* Wc, void* Wp, int32_t flags, void* stream);

/* fmm_leaf_boxes: for each of n points, the deepest existing box of `tree`
 *   that contains it (the leaf a point's far field is evaluated from, Sec. 2.1
 *   stage 4): level[j] = the largest l <= max_level whose box
 *   (floor(x 2^l), floor(y 2^l)), each clamped to 0..2^l - 1 (a point goes to
 *   box floor(x 2^l), reading of Sec. 2.1), exists; box[j] = iy * 2^l + ix.
 *   Every box exists on a uniform tree, so there level[j] = max_level.
 *   Coordinates are read exactly (no rounding); a NaN coordinate goes to
 *   cell 0.  xy: device float64 [n][2]; level: device int32 [n]; box: device
 *   int64 [n].  The first call on an adaptive tree uploads its existence
 *   masks (synchronously).  FMM_EINVAL for a NULL tree or pointer, n < 0, or
 *   misaligned pointers.
 */
int fmm_leaf_boxes(const fmm_tree* tree, const double* xy, int64_t n, int32_t* level, int64_t* box,
                   void* stream);

/* fmm_l2p: far field at n points from the LE of each point's box:
 *     phi_j (+)= (1/r_l) sum_n L~_l[b][n] ((z_j - x_b) / r_l)^n,  l = lev[j], b = box[j],
 *   phi_j = 0 where lev[j] < 2.
 *   z: device float64 [n][2]; lev: device int32 [n]; box: device int64 [n]
 *   (b = iy * 2^l + ix); L_levels: host array of max_level + 1 device pointers,
 *   entry l = level l's [4^l][p] LEs (NULL for levels no point uses);
 *   phi: device complex64 [n].  flags: FMM_ACCUMULATE.  A point whose
 *   (level, box) does not address a given array is skipped and reported by
 *   fmm_sync_status (FMM_EDEVICE).
 * fmm_l2p_adjoint: G_l[b][n] += conj(((z_j - x_b) / r_l)^n / r_l) cot_j for every
 *   point (FP32 atomic additions, order-dependent in the last bits); cot:
 *   device complex64 [n]; G_levels like L_levels (accumulated into). */
int fmm_l2p(int32_t p, int64_t n, const double* z, const int32_t* lev, const int64_t* box,
            const void* const* L_levels, int32_t max_level, void* phi, int32_t flags, void* stream);
int fmm_l2p_adjoint(int32_t p, int64_t n, const double* z, const int32_t* lev, const int64_t* box,
                    const void* cot, void* const* G_levels, int32_t max_level, void* stream);

/* fmm_l2p_binned: fmm_l2p for the n points z of a uniform tree's `level`, binned
 *   by fmm_bin_points(level, z, n, perm, box_start, ...) (Sec. 2.1 stage 4):
 *     phi_j (+)= (1/r) sum_n L~[b][n] ((z_j - x_b) / r)^n,  b the box of z_j,
 *   phi_j = 0 at levels 0 and 1 (no lists there).  One thread block per box
 *   keeps the box's LE in shared memory; a point's offset from its box centre is
 *   read off the bits of its FP64 coordinates.  z: device float64 [n][2];
 *   perm, box_start: device int32 [n], [4^level + 1]; L: device complex64
 *   [4^level][p] (may be NULL at levels 0, 1); phi: device complex64 [n].
 *   p 1..64; level 0..10; flags FMM_ACCUMULATE.  A perm entry or box start out
 *   of range sets the device error word's check bit and is skipped. */
int fmm_l2p_binned(int32_t level, int32_t p, const double* z, int64_t n, const int32_t* perm,
                   const int32_t* box_start, const void* L, void* phi, int32_t flags, void* stream);

/* fmm_p2m_binned: fmm_p2m for points binned by fmm_bin_points(level, xy, n, ...)
 *   (perm, box_start): one thread block per box sums its points (powers in FP32
 *   of d read off the bits of the FP64 coordinates), one store per coefficient --
 *   no atomics, the same result on every run.  p 6, 8, 12, 16 or 24; level
 *   0..10; flags FMM_ACCUMULATE.  A perm entry or box start out of range sets the
 *   device error word's check bit and is skipped. */
int fmm_p2m_binned(int32_t level, int32_t p, const double* xy, const double* c, int64_t n, const int32_t* perm,
                   const int32_t* box_start, void* M, int32_t flags, void* stream);

/* fmm_p2m_adjoint: for the P2M of fmm_p2m at `level` (M~_b[k] = sum_i c_i d_i^k,
 *   d_i = (y_i - x_b) / r_l) and G = dJ/dM~ of a real objective J, the gradient
 *   in the point positions:
 *     grad[i] (+)= (Re, Im) of sum_k G[b_i][k] conj(c_i k d_i^(k-1) / r_l) = (dJ/dx_i, dJ/dy_i).
 *   xy, c: device float64 as fmm_p2m; G: device complex64 [4^level][p];
 *   grad: device float64 [n][2].  flags: FMM_ACCUMULATE. */
int fmm_p2m_adjoint(int32_t level, int32_t p, const double* xy, const double* c, int64_t n,
                    const void* G, double* grad, int32_t flags, void* stream);

/* fgt_p2h: FGT Hermite coefficients of every box of a 2^g grid (Eq. A_alpha),
 *   A_b[a1][a2] (+)= sum_{j in box b} q_j t1^a1 t2^a2 / (a1! a2!),
 *   t = (x_j - s_b) / (sqrt(2) sigma), s_b the box centre, a1, a2 < p.
 *   x: device float64 [n][2]; q: device float64 [n]; A: device float32
 *   [4^g][p][p].  FP32 atomic additions.  flags: FMM_ACCUMULATE or 0. */
int fgt_p2h(int32_t grid_log2, int32_t p, double sigma, const double* x, const double* q, int64_t n,
            float* A, int32_t flags, void* stream);

/* fgt_t2p: the transform at n targets from the Taylor coefficients of each
 *   target's box (Sec. 2.2, Eq. taylor):
 *     G(y_j) (+)= sum_{b1,b2 < p} C[b][b1][b2] t1^b1 t2^b2,  t = (y_j - t_C) / (sqrt(2) sigma),
 *   b = the box floor(y 2^g) (clamped) of the 2^g grid, t_C its centre.
 *   C: device float32 [4^g][p][p] (fgt_h2t's output, 16-byte aligned); y: device
 *   float64 [n][2]; G: device float32 [n].  p: 4, 8, 12 or 16.  flags: FMM_ACCUMULATE.
 *   With fgt_p2h and fgt_h2t this is the whole transform on the device. */
int fgt_t2p(int32_t grid_log2, int32_t p, double sigma, const float* C, const double* y, int64_t n,
            float* G, int32_t flags, void* stream);

/* fgt_t2p_binned: fgt_t2p (Sec. 2.2, Eq. taylor) at targets binned by
 *   fgt_bin_points(grid_log2, y, n, perm, box_start, ...): one thread block per
 *   box holds its p x p coefficients in shared memory and evaluates them at the
 *   box's targets (a target's offset from the box centre read off the bits of
 *   its FP64 coordinates).  Same
 *   arguments as fgt_t2p plus perm, box_start (device int32 [n], [4^g + 1]);
 *   grid_log2 0..10; C 4-byte aligned.  A perm entry or box start out of range
 *   sets the device error word's check bit and is skipped. */
int fgt_t2p_binned(int32_t grid_log2, int32_t p, double sigma, const float* C, const double* y, int64_t n,
                   const int32_t* perm, const int32_t* box_start, float* G, int32_t flags, void* stream);

/* ---------------------------------------------------------------------------
 * FGT Hermite-series evaluation at targets (Sec. 4.2, Eq. hermite), the
 * paper's own FGT GPU kernel, on the uniform 2^g x 2^g grid:
 *
 * fgt_bin_points -- counting sort of n points by box of the grid (box
 *   floor(y 2^g), clamped to the grid; NaN coordinates go to box 0).
 *   y: device float64 [n][2]; perm: device int32 [n], written with the point
 *   indices box by box (order within a box unspecified); box_start: device
 *   int32 [4^g + 1], box b's points are perm[box_start[b] .. box_start[b+1]);
 *   work: device int32 [4^g] scratch (not overlapping box_start).
 *   grid_log2 0..10, n < 2^31.  No allocation, no synchronisation.
 *
 * fgt_p2h_binned -- fgt_p2h (Eq. A_alpha) for sources binned by
 *   fgt_bin_points(grid_log2, x, ...): one atomic addition per coefficient per
 *   run of a box's points within a block of 256, instead of one per point.
 *   Summation order within a box follows the binning, so the FP32 result
 *   varies by rounding from run to run.  p: 4, 8, 12 or 16.
 *
 * fgt_h2p -- for every target y_j,
 *   G(y_j) (+)= sum_{B : max(|sx-tx|,|sy-ty|) <= n_cut}
 *                sum_{a1,a2 < p} A_B[a1][a2] h_a1((y_j1 - sB1)/(sqrt2 sigma)) h_a2((y_j2 - sB2)/(sqrt2 sigma)),
 *   (tx, ty) the box of y_j, s_B the centre of source box B, h_n(t) = exp(-t^2) H_n(t).
 *   A: device float32 [4^g][p][p] Hermite coefficients (fgt_p2h), 16-byte
 *   aligned; y: device float64 [n][2]; perm, box_start: fgt_bin_points(grid_log2,
 *   y, n, ...) of these targets; G: device float32 [n], indexed like y.
 *   n_cut 0..16, p 4, 8, 12 or 16, flags FMM_ACCUMULATE or 0.
 *   prec FMM_FP32: CUDA cores.  Source boxes whose coefficients are all zero
 *   are skipped: a first kernel writes one flag per box.  The targets are
 *   taken in runs of up to 256 of one box, the boxes with the most non-empty
 *   source boxes within n_cut first (an order built on the device in every
 *   call; G does not depend on it).  Flags, claim order and claim table live
 *   in a ~17 MiB per-device scratch that the library allocates on the first
 *   call (or in fmm_prepare; make one of them before any stream capture);
 *   calls that overlap on the GPU (different streams) share it and must be
 *   serialised by the caller.  A perm
 *   entry outside [0, n) or a box_start that does not bin [0, n) sets the
 *   device error word's check bit (fmm_sync_status returns FMM_EDEVICE); the
 *   affected targets are skipped.
 *   prec FMM_TC_BF16X3 / FMM_TC_BF16: tensor cores, p = 16 and n_cut <= 15
 *   only (else FMM_EUNSUPPORTED; FMM_TC_TF32X3 is FMM_EUNSUPPORTED here).  Per target box the evaluation is the
 *   product of the targets' y-direction Hermite values with the
 *   neighbourhood's coefficients, reduced against the x-direction values;
 *   FP32 accumulation, BF16 operands split into hi + lo (three products,
 *   ~16 significant bits each) or hi only.  Every box of the neighbourhood
 *   is evaluated (no skipping).  A BF16 copy of A (1 KiB per box) lives in a
 *   per-device buffer grown on demand (the first call of a grid size
 *   allocates: make it before any stream capture).
 * ------------------------------------------------------------------------- */
int fgt_bin_points(int32_t grid_log2, const double* y, int64_t n, int32_t* perm, int32_t* box_start, int32_t* work,
                   void* stream);
int fgt_p2h_binned(int32_t grid_log2, int32_t p, double sigma, const double* x, const double* q, int64_t n,
                   const int32_t* perm, float* A, int32_t flags, void* stream);
int fgt_h2p(int32_t grid_log2, int32_t n_cut, int32_t p, int32_t prec, double sigma, const float* A, const double* y,
            int64_t n, const int32_t* perm, const int32_t* box_start, float* G, int32_t flags, void* stream);

/* ---------------------------------------------------------------------------
 * Near field of a uniform quadtree at its finest level (Sec. 2.1 stage 5,
 * Eq. n_body restricted to the own and adjacent boxes):
 *
 * fmm_bin_points -- fgt_bin_points on the 2^level x 2^level boxes of a
 *   quadtree level (box floor(x 2^l), clamped): the same counting sort.
 *
 * fmm_p2p -- for every target z_j,
 *     phi_j (+)= sum_{i : max(|sx - tx|, |sy - ty|) <= 1, y_i != z_j} c_i / (z_j - y_i),
 *   (tx, ty) the level-`level` box of z_j, (sx, sy) that of source y_i.  With
 *   fmm_m2l over levels 2..level, L2L down and L2P at level `level`, this is
 *   the whole FMM potential at the targets.
 *   xy: device float64 [n][2] source positions; c: device float64 [n]
 *   strengths; src_perm, src_start: fmm_bin_points(level, xy, n, ...);
 *   z: device float64 [nz][2] targets; tgt_perm, tgt_start:
 *   fmm_bin_points(level, z, nz, ...); phi: device complex64 [nz], indexed
 *   like z.  level 0..10, n and nz < 2^31.
 *   flags   FMM_ACCUMULATE; FMM_P2P_SHARE_SM: size the persistent grid for
 *           at most 8 resident CTAs per SM instead of the occupancy limit,
 *           leaving each SM room for kernels that other streams run at the
 *           same time (the far field of the same FMM: 1.39 -> 1.28 ms for the
 *           whole potential at 2^22 points; alone the call is ~1.5 % slower).
 *   FP32 arithmetic on positions taken relative to the target box's centre;
 *   1e-30 is added to every squared distance, so a source at exactly a
 *   target's position (e.g. the points themselves) contributes nothing
 *   (strengths |c| < 3e8) and other pairs change by a relative 1e-30 / r^2.  Uses the per-device scratch of
 *   fgt_h2p (calls that overlap on the GPU must be serialised).  A
 *   permutation entry outside range or inconsistent box starts set the device
 *   error word's check bit; the affected pairs are skipped.
 * ------------------------------------------------------------------------- */
int fmm_bin_points(int32_t level, const double* y, int64_t n, int32_t* perm, int32_t* box_start, int32_t* work,
                   void* stream);
#define FMM_P2P_SHARE_SM 16
int fmm_p2p(int32_t level, const double* xy, const double* c, int64_t n, const int32_t* src_perm,
            const int32_t* src_start, const double* z, int64_t nz, const int32_t* tgt_perm, const int32_t* tgt_start,
            void* phi, int32_t flags, void* stream);

/* ---------------------------------------------------------------------------
 * fmm_m2l_paper_design -- the paper's own M2L data flow (Sec. 4.1.1-4.1.2),
 * for comparison with fmm_m2l: a thread block per source ME translates it to
 * every target whose interaction list holds it, one thread per LE row, and
 * writes one LE per translation to `work`; a second kernel sums each
 * target's translated LEs (the paper's separate reduction).  Same result as
 * fmm_m2l (FP32, up to summation order) at one level of a uniform,
 * non-periodic tree; p 8, 12 or 16.  work: device, 4^level * 27 * p complex64
 * (16-byte aligned), overwritten.  flags: FMM_ACCUMULATE.
 * ------------------------------------------------------------------------- */
int fmm_m2l_paper_design(const fmm_tree* tree, int32_t level, int32_t p, const void* M, void* L, void* work,
                         int32_t flags, void* stream);

/* ---------------------------------------------------------------------------
 * fmm_wait_probe -- run the library's bounded device-side wait on purpose.
 *
 * The paper has no counterpart.  Every hand-over between warps in the
 * tensor-core kernels waits on a shared-memory mbarrier with a poll limit;
 * a wait that reaches it records a timeout in the device error word (read
 * by fmm_sync_status as FMM_ETIMEOUT) and the kernel returns instead of
 * hanging.  This call launches one 64-thread CTA in which thread 0 waits on
 * a one-arrival barrier with both wait forms those kernels use (sleeping
 * poll and busy spin).
 *   polls   1..4,194,304: the poll limit of each wait; 0 = the limits the
 *           kernels use.
 *   arrive  1: a second warp completes the barrier, so the waits return
 *           normally; 0: nothing arrives, so each wait gives up after
 *           `polls` polls and the error word records a timeout.
 * Asynchronous on `stream`; nothing is allocated after the first call on a
 * device (which creates the error word).  Errors: FMM_EINVAL for arguments
 * out of range.
 * ------------------------------------------------------------------------- */
int fmm_wait_probe(int32_t polls, int32_t arrive, void* stream);

/* Read and clear the device error word after synchronising `stream`.
 * Returns FMM_OK, FMM_ETIMEOUT or FMM_EDEVICE. */
int fmm_sync_status(void* stream);

/* Message for the calling thread's most recent failure ("" if none). */
const char* fmm_last_error(void);

/* Library version string. */
const char* fmm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FMMGB_H */
