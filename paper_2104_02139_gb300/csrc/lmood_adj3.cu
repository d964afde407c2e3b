// Reverse-pass kernels instantiated for tetrahedra (D = 3).
#include "lmood_adj_ops_impl.cuh"
namespace lmood {
const AdjOps &adj_ops_dim3() { LMOOD_ADJ_OPS_TABLE(3) }
}  // namespace lmood
