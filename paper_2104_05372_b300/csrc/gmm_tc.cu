// Tensor-core GMM path placeholder: reports GPA_ERR_UNSUPPORTED until built.
#include "common.cuh"
#include "gmm_internal.cuh"

namespace gpa {
bool gmm_tc_supported(int) { return false; }
size_t gmm_tc_extra_bytes(int64_t, int, int) { return 0; }
int gmm_tc_objective_run(const GmmArgs&, const GmmLayout&, char*, size_t, cudaStream_t) {
    return GPA_ERR_UNSUPPORTED;
}
int gmm_tc_vjp_run(const GmmArgs&, const GmmLayout&, char*, size_t, cudaStream_t) {
    return GPA_ERR_UNSUPPORTED;
}
}  // namespace gpa
