// Kernel instantiations for the ProbDual14Rel problem class.  The FP32
// projection has two kernels: one thread per configuration (k_project_f32)
// and one lane per arm (k_project_pair); the tuning's threads per
// configuration selects.
#include "mcp_extend.cuh"
#include "mcp_pair.cuh"

namespace mcp {

template <>
cudaError_t launch_project<ProbDual14Rel>(const HostModel &hm, const ProjCall &c, int *launches) {
  using P = ProbDual14Rel;
  static_assert(has_pair_kernel<P>() && PairOf<P>::ok, "pair kernel traits disagree");
  if (c.precision != 0 || c.tune.tpc != 2 || c.outer || c.total <= 0) return launch_project_impl<P>(hm, c, launches);
  cudaError_t err = cudaMemsetAsync(c.counter, 0, sizeof(unsigned long long), c.stream);
  if (err != cudaSuccess) return err;
  if (c.segments) {
    const SegSrc<float> src{static_cast<const float *>(c.start), static_cast<const float *>(c.delta), c.ld_seg,
                            c.seg_off, c.n_seg};
    err = c.fused_check ? launch_pair<P, SegSrc<float>, true>(hm, c, src)
                        : launch_pair<P, SegSrc<float>, false>(hm, c, src);
  } else {
    const BatchSrc<float> src{static_cast<const float *>(c.q_in), c.ld_in};
    err = c.fused_check ? launch_pair<P, BatchSrc<float>, true>(hm, c, src)
                        : launch_pair<P, BatchSrc<float>, false>(hm, c, src);
  }
  *launches += 1;
  return err;
}

template <>
cudaError_t launch_check<ProbDual14Rel>(const HostModel &hm, const CheckCall &c, int *launches) {
  return launch_check_impl<ProbDual14Rel>(hm, c, launches);
}

template <>
cudaError_t launch_vjp<ProbDual14Rel>(const HostModel &hm, const VjpCall &c, int *launches) {
  return launch_vjp_impl<ProbDual14Rel>(hm, c, launches);
}

}  // namespace mcp
MCP_INSTANTIATE_EXTEND(ProbDual14Rel)
