// Tensor-core (tcgen05) auxiliary-problem solver: not built yet.
#include "dpm_internal.cuh"

namespace dpm {

bool tc_supported(int N) {
    (void)N;
    return false;
}

int ap_solve_tc(const ApParams &p, const ApRhs<float> *rhs_dev, float *work, cudaStream_t s) {
    (void)p; (void)rhs_dev; (void)work; (void)s;
    set_error("tensor-core AP solve is not available in this build");
    return DPM_EUNSUPPORTED;
}

}  // namespace dpm
