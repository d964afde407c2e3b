// Reverse-pass kernels instantiated for triangles (D = 2).
#include "lmood_adj_ops_impl.cuh"
namespace lmood {
const AdjOps &adj_ops_dim2() { LMOOD_ADJ_OPS_TABLE(2) }
}  // namespace lmood
