// Kernel instantiations for the ProbArm7Pose problem class.
#include "mcp_kernels.cuh"

namespace mcp {
MCP_INSTANTIATE(ProbArm7Pose)
MCP_NO_EXTEND(ProbArm7Pose)
}  // namespace mcp
