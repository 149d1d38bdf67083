// qa_soft_fwd.cu -- soft occupation forward pass (instantiations).
#include "qa_soft.cuh"

namespace qa {

cudaError_t launch_soft_forward(const SoftLaunch& a, cudaStream_t st) {
  return dispatch_soft<false>(a, st);
}

size_t soft_partials_floats(int n, long long P, const SearchCfg& cfg) {
  return soft_partials_floats_impl(n, P, cfg);
}

}  // namespace qa
