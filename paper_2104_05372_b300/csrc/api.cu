// Library-wide entry points of the C ABI: status names, version, and the
// check of the device's bounded waits.
#include "common.cuh"
#include "trace.cuh"

extern "C" const char* gpa_status_string(int status) {
    switch (status) {
        case GPA_OK: return "GPA_OK";
        case GPA_ERR_ARG: return "GPA_ERR_ARG: null pointer or size out of range";
        case GPA_ERR_INDEX: return "GPA_ERR_INDEX: an index outside its index set";
        case GPA_ERR_CUDA: return "GPA_ERR_CUDA: a CUDA launch or runtime call failed";
        case GPA_ERR_WORKSPACE: return "GPA_ERR_WORKSPACE: workspace smaller than required";
        case GPA_ERR_TIMEOUT: return "GPA_ERR_TIMEOUT: a bounded device wait gave up";
        case GPA_ERR_UNSUPPORTED: return "GPA_ERR_UNSUPPORTED: shape, precision or strategy not provided";
        case GPA_ERR_ALIGN: return "GPA_ERR_ALIGN: pointer lacks the required alignment";
    }
    return "unknown gpa_status";
}

extern "C" int gpa_version(void) { return 100; }

namespace gpa {
// One CTA of two warps waits on an mbarrier that expects one arrival which never
// comes: warp 0 with the per-thread wait, warp 1 with the warp-uniform wait
// used before .sync.aligned instructions. Both give up after limit_ns and
// report GPA_ERR_TIMEOUT; nothing else happens (no copies, no tensor memory).
__global__ void __launch_bounds__(64) wait_timeout_kernel(unsigned long long limit_ns, int32_t* status,
                                                          int32_t* gave_up) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool ok = threadIdx.x < 32 ? mbar_wait(&bar, 0, status, limit_ns)
                                     : mbar_wait_warp(&bar, 0, status, limit_ns);
    if (!ok) atomicAdd(gave_up, 1);
}
}  // namespace gpa

extern "C" int gpa_check_bounded_wait(int64_t limit_ns, int32_t* dev_status, int32_t* gave_up,
                                      gpa_stream_t stream) {
    if (!dev_status || !gave_up) return GPA_ERR_ARG;
    if (limit_ns < 1 || limit_ns > (int64_t)gpa::kWaitLimitNs) return GPA_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    GPA_LAUNCH("wait_timeout_check", s,
               gpa::wait_timeout_kernel<<<1, 64, 0, s>>>((unsigned long long)limit_ns, dev_status, gave_up));
    return GPA_OK;
}
