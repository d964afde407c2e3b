// Step kernels instantiated for tetrahedra (D = 3).
#include "lmood_ops_impl.cuh"
namespace lmood {
const Ops &ops_dim3() { LMOOD_OPS_TABLE(3) }
}  // namespace lmood
