// Step kernels with FP32 arithmetic and FP32 storage (absolute or deviation).
#include "step_kernel.cuh"

namespace dvbe {
cudaError_t launch_step_f32(int store, int scheme, const CaseArgs &a, int blocks, int wpb,
                            const StepStreams &s) {
  if (store == ST_F32) return launch_step_impl<ST_F32>(scheme, a, blocks, wpb, s);
  return launch_step_impl<ST_F32_DEV>(scheme, a, blocks, wpb, s);
}
cudaError_t launch_batch_f32(int store, int scheme, const CaseArgs *c, const long long *p, int n,
                             long long ni, unsigned long long *q, int blocks, int wpb,
                             cudaStream_t s) {
  if (store == ST_F32) return launch_batch_impl<ST_F32>(scheme, c, p, n, ni, q, blocks, wpb, s);
  return launch_batch_impl<ST_F32_DEV>(scheme, c, p, n, ni, q, blocks, wpb, s);
}
int inner_blocks_per_sm_f32(int store, int scheme, int wpb) {
  if (store == ST_F32) return inner_blocks_per_sm_impl<ST_F32>(scheme, wpb);
  return inner_blocks_per_sm_impl<ST_F32_DEV>(scheme, wpb);
}
} // namespace dvbe
