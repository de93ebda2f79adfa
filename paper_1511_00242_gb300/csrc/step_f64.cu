// Step kernels with FP64 storage and arithmetic (the parity path).
#include "step_kernel.cuh"

namespace dvbe {
cudaError_t launch_step_f64(int scheme, const CaseArgs &a, int blocks, int wpb, const StepStreams &s) {
  return launch_step_impl<ST_F64>(scheme, a, blocks, wpb, s);
}
cudaError_t launch_batch_f64(int scheme, const CaseArgs *c, const long long *p, int n, long long ni,
                             unsigned long long *q, int blocks, int wpb, cudaStream_t s) {
  return launch_batch_impl<ST_F64>(scheme, c, p, n, ni, q, blocks, wpb, s);
}
int inner_blocks_per_sm_f64(int scheme, int wpb) { return inner_blocks_per_sm_impl<ST_F64>(scheme, wpb); }
} // namespace dvbe
