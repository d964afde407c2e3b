// Step kernels instantiated for triangles (D = 2).
#include "lmood_ops_impl.cuh"
namespace lmood {
const Ops &ops_dim2() { LMOOD_OPS_TABLE(2) }
}  // namespace lmood
