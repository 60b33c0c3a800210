// Kernel instantiations for the ProbDual14Rel problem class.
#include "mcp_extend.cuh"

namespace mcp {
MCP_INSTANTIATE(ProbDual14Rel)
}  // namespace mcp
MCP_INSTANTIATE_EXTEND(ProbDual14Rel)
