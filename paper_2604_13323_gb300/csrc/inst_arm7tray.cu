// Kernel instantiations for the ProbArm7Tray problem class (the arm with a plane and an axis constraint).
#include "mcp_kernels.cuh"

namespace mcp {
MCP_INSTANTIATE(ProbArm7Tray)
MCP_NO_EXTEND(ProbArm7Tray)
}  // namespace mcp
