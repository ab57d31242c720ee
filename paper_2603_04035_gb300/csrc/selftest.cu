// Self-test of the bounded device-side wait that every tensor-core kernel of
// the library uses (mbar_wait): one thread waits on an mbarrier that nothing
// arrives at (or, as a control, one it arrives at first), with a given limit.
// When the limit passes, the wait raises the CTA's abort flag, reports
// DRGB_ERR_TIMEOUT in the context's status word and returns, and the kernel
// exits; no copy or tensor-core operation is in flight, so nothing is left
// pending on the device.
#include "common.cuh"
#include "tc_ptx.cuh"

namespace drgb {

__global__ void wait_selftest_kernel(int* status, unsigned long long limit_ns, int arrive) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (arrive) mbar_arrive(&bar);  // the phase completes: no timeout
        mbar_wait(&bar, 0, &abort_flag, status, limit_ns);
    }
}

}  // namespace drgb

using namespace drgb;

extern "C" int drgb_wait_selftest(drgb_ctx* c, int64_t limit_us, int32_t arrive, void* stream) {
    if (!c) return DRGB_ERR_INVALID;
    if (limit_us < 1 || limit_us > 10000000)
        return set_error(c, DRGB_ERR_INVALID, "wait_selftest: limit must be 1 us .. 10 s");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    wait_selftest_kernel<<<1, 32, 0, st>>>(c->d_status, static_cast<unsigned long long>(limit_us) * 1000ull,
                                           arrive ? 1 : 0);
    DRGB_CHECK_LAUNCH(c);
    return drgb_sync(c, stream);
}
