// Kernel instantiations for the ProbDual14Rel problem class.
#include "mcp_kernels.cuh"

namespace mcp {
MCP_INSTANTIATE(ProbDual14Rel)
}  // namespace mcp
