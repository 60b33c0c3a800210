// Kernel instantiations for the ProbArm7Axis problem class.
#include "mcp_kernels.cuh"

namespace mcp {
MCP_INSTANTIATE(ProbArm7Axis)
}  // namespace mcp
