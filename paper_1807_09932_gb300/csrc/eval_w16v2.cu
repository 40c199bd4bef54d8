// Evaluator instantiations for 16-bit ranks with 2 row group(s) per slab.
#include "eval_kernel.cuh"

namespace ebic {
cudaError_t launch_eval_w16v2(const EvalConfig& c, const CUtensorMap* t, const EvalArgs& a,
                           cudaStream_t s) {
  return launch_eval_layout<16, 2>(c, t, a, s);
}
cudaError_t ready_eval_w16v2() { return ready_eval_layout<16, 2>(); }
}  // namespace ebic
