// Kernel instantiations for the ProbSphere3 problem class.
#include "mcp_kernels.cuh"

namespace mcp {
MCP_INSTANTIATE(ProbSphere3)
}  // namespace mcp
