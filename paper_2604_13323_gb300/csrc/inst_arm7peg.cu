// Kernel instantiations for the ProbArm7Peg problem class (the arm with a line and an axis constraint).
#include "mcp_kernels.cuh"

namespace mcp {
MCP_INSTANTIATE(ProbArm7Peg)
MCP_NO_EXTEND(ProbArm7Peg)
}  // namespace mcp
