// wait_probe.cu -- a one-CTA kernel that runs the library's bounded mbarrier
// waits (mbar_wait, mbar_spin of tc_ptx.cuh, the ones every tensor-core kernel
// uses) on a barrier that is, or is not, completed, so the give-up path and
// its report through the device error word can be exercised on purpose
// without faulting or hanging the GPU.  No counterpart in the paper.
#include "common.cuh"
#include "tc_ptx.cuh"

namespace fmmgb {

// Thread 0 waits on a one-arrival barrier with both wait forms; when `arrive`
// is set, thread 32 (another warp) makes that arrival.  A wait that gives up
// records DEV_ERR_TIMEOUT and the kernel returns.  Nothing else is touched:
// no copy is in flight and no tensor memory is held, so giving up is safe.
__global__ void __launch_bounds__(64) wait_probe_kernel(uint32_t wait_cap, uint32_t spin_cap, int arrive, int* err)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (arrive && threadIdx.x == 32) mbar_arrive(&bar);
    if (threadIdx.x == 0) {
        const bool waited = mbar_wait(&bar, 0, 64, wait_cap);
        const bool spun = mbar_spin(&bar, 0, spin_cap);
        if (!waited || !spun) atomicOr(err, DEV_ERR_TIMEOUT);
    }
}

}  // namespace fmmgb

extern "C" int fmm_wait_probe(int32_t polls, int32_t arrive, void* stream)
{
    using namespace fmmgb;
    clear_error();
    if (polls < 0) return fail(FMM_EINVAL, "fmm_wait_probe: polls %d < 0", polls);
    if ((uint32_t)polls > kWaitCap)
        return fail(FMM_EINVAL, "fmm_wait_probe: polls %d above the library's cap %u", polls, kWaitCap);
    if (arrive != 0 && arrive != 1) return fail(FMM_EINVAL, "fmm_wait_probe: arrive must be 0 or 1");
    int* err = nullptr;
    if (int rc = device_error_word(&err)) return rc;
    const uint32_t wait_cap = polls ? (uint32_t)polls : kWaitCap;
    const uint32_t spin_cap = polls ? (uint32_t)polls : kSpinCap;
    wait_probe_kernel<<<1, 64, 0, (cudaStream_t)stream>>>(wait_cap, spin_cap, arrive, err);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}
