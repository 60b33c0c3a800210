// Kernel instantiations for the Cartesian-point problem classes (ProbSphere3,
// ProbPoint3Planes4).
#include "mcp_extend.cuh"

namespace mcp {
MCP_INSTANTIATE(ProbSphere3)
MCP_INSTANTIATE(ProbPoint3Planes4)
MCP_NO_EXTEND(ProbPoint3Planes4)
}  // namespace mcp
MCP_INSTANTIATE_EXTEND(ProbSphere3)
