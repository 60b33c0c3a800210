// Kernel instantiations for the ProbArm7Tsr problem class (the arm with a bounded TSR).
#include "mcp_kernels.cuh"

namespace mcp {
MCP_INSTANTIATE(ProbArm7Tsr)
MCP_NO_EXTEND(ProbArm7Tsr)
}  // namespace mcp
