// Kernel instantiations for the ProbDual14Rod problem class (the dual arm carrying a rod on a plane).
#include "mcp_kernels.cuh"

namespace mcp {
MCP_INSTANTIATE(ProbDual14Rod)
MCP_NO_EXTEND(ProbDual14Rod)
}  // namespace mcp
