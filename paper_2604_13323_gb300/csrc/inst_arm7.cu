// Kernel instantiations for the ProbArm7Axis problem class.
#include "mcp_extend.cuh"

namespace mcp {
MCP_INSTANTIATE(ProbArm7Axis)
}  // namespace mcp
MCP_INSTANTIATE_EXTEND(ProbArm7Axis)
