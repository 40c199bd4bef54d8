// Evaluator instantiations for 8-bit ranks with 4 row group(s) per slab.
#include "eval_kernel.cuh"

namespace ebic {
cudaError_t launch_eval_w8v4(const EvalConfig& c, const CUtensorMap* t, const EvalArgs& a,
                           cudaStream_t s) {
  return launch_eval_layout<8, 4>(c, t, a, s);
}
cudaError_t ready_eval_w8v4() { return ready_eval_layout<8, 4>(); }
}  // namespace ebic
