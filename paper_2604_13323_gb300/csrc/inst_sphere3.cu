// Kernel instantiations for the ProbSphere3 problem class.
#include "mcp_extend.cuh"

namespace mcp {
MCP_INSTANTIATE(ProbSphere3)
}  // namespace mcp
MCP_INSTANTIATE_EXTEND(ProbSphere3)
