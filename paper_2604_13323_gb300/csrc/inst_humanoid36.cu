// Kernel instantiations for the ProbHumanoid36 problem class (collision check;
// projection of this class runs in the warp-cooperative kernels).
#include "mcp_kernels.cuh"

namespace mcp {
MCP_INSTANTIATE_CHECK_ONLY(ProbHumanoid36)
}  // namespace mcp
