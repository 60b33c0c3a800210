// Kernel instantiations for the ProbHumanoid36Hull problem class (CoM on the
// support polygon): the FP32 path
// runs the group-cooperative kernel (the cyclic form: the warp kernel), the plain FP64 path and the collision
// check the thread-per-configuration kernels.
#include "mcp_group.cuh"

namespace mcp {

template <>
cudaError_t launch_project<ProbHumanoid36Hull>(const HostModel &hm, const ProjCall &c, int *launches) {
  if (c.precision == 1) {
    if (c.total <= 0) return cudaSuccess;
    if (c.segments) return cudaErrorNotSupported;
    cudaError_t e =
        launch_plain64_any<ProbHumanoid36Hull>(hm, c, BatchSrc<double>{static_cast<const double *>(c.q_in), c.ld_in});
    *launches += 1;
    if (e == cudaSuccess && c.fused_check) e = check_outputs<ProbHumanoid36Hull>(hm, c, launches);
    return e;
  }
  // stacked form: four lanes per configuration; the cyclic form's masked
  // sub-steps run on the warp-per-configuration kernel
  cudaError_t e = c.cyclic ? launch_project_warp<ProbHumanoid36Hull>(hm, c, launches)
                           : launch_project_group<ProbHumanoid36Hull>(hm, c, launches);
  if (e == cudaSuccess && c.fused_check) e = check_outputs<ProbHumanoid36Hull>(hm, c, launches);
  return e;
}

template <>
cudaError_t launch_check<ProbHumanoid36Hull>(const HostModel &hm, const CheckCall &c, int *launches) {
  return launch_check_impl<ProbHumanoid36Hull>(hm, c, launches);
}

template <>
cudaError_t launch_vjp<ProbHumanoid36Hull>(const HostModel &, const VjpCall &, int *) {
  return cudaErrorNotSupported;
}

MCP_NO_EXTEND(ProbHumanoid36Hull)

}  // namespace mcp
