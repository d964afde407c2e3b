// lmood_adj_ops_impl.cuh -- launchers of the reverse-pass kernels for one dimension.
#pragma once
#include "lmood_adjoint_kernels.cuh"

namespace lmood {
namespace {

constexpr int kAdjCellBlock = 128, kAdjNodeBlock = 128;
inline int adj_blocks(int n, int b) { return (n + b - 1) / b; }

template <int D> void adj_update(const Geo &g, const Fld &f, const Prm &p, const AdjBuf &a, cudaStream_t s) {
    if (a.lE1) k_adj_update<D, true><<<adj_blocks(g.N, kAdjCellBlock), kAdjCellBlock, 0, s>>>(g, f, p, a);
    else k_adj_update<D, false><<<adj_blocks(g.N, kAdjCellBlock), kAdjCellBlock, 0, s>>>(g, f, p, a);
}
template <int D> void adj_nodes(const Geo &g, const Fld &f, const AdjBuf &a, int init_mode, cudaStream_t s) {
    k_adj_nodes<D, false><<<adj_blocks(g.Np, kAdjNodeBlock), kAdjNodeBlock, 0, s>>>(g, f, a, init_mode);
    if (a.bf) k_adj_nodes<D, true><<<adj_blocks(g.Np, kAdjNodeBlock), kAdjNodeBlock, 0, s>>>(g, f, a, init_mode);
}
template <int D, int MAT>
void adj_predict_m(const Geo &g, const Fld &f, const Prm &p, const AdjBuf &a, int force_p0, cudaStream_t s) {
    if (!force_p0) {
        const int nc = (D + 1) * g.N;
        k_adj_pred_fw<D, MAT, false><<<adj_blocks(g.N, kAdjCellBlock), kAdjCellBlock, 0, s>>>(g, f, p, a);
        if (a.bj) k_adj_pred_fw<D, MAT, true><<<adj_blocks(g.N, kAdjCellBlock), kAdjCellBlock, 0, s>>>(g, f, p, a);
        k_adj_pred_c2<D, MAT><<<adj_blocks(nc, kAdjCellBlock), kAdjCellBlock, 0, s>>>(g, f, p, a);
        k_adj_pred_c1<D, MAT><<<adj_blocks(nc, kAdjCellBlock), kAdjCellBlock, 0, s>>>(g, f, p, a);
        constexpr int MF = MAT == 2 ? 2 : 0;
        k_adj_pred_fin<D, MF, false><<<adj_blocks(g.N, kAdjCellBlock), kAdjCellBlock, 0, s>>>(g, f, p, a);
        if (a.bj) k_adj_pred_fin<D, MF, true><<<adj_blocks(g.N, kAdjCellBlock), kAdjCellBlock, 0, s>>>(g, f, p, a);
        // (the second-order cells' corner-matrix and geometry part runs in k_adj_cells)
    }
    k_adj_predict<D, MAT><<<adj_blocks(g.N, kAdjCellBlock), kAdjCellBlock, 0, s>>>(g, f, p, a, force_p0);
}
template <int D>
void adj_predict(const Geo &g, const Fld &f, const Prm &p, const AdjBuf &a, int force_p0, cudaStream_t s) {
    if (p.eos) adj_predict_m<D, 2>(g, f, p, a, force_p0, s);
    else if (p.shear_a == -1.0) adj_predict_m<D, 0>(g, f, p, a, force_p0, s);
    else adj_predict_m<D, 1>(g, f, p, a, force_p0, s);
}
template <int D> void adj_momsum(const Geo &g, const Fld &f, const AdjBuf &a, cudaStream_t s) {
    (void)f;
    k_adj_momsum<D><<<adj_blocks(g.Np, kAdjNodeBlock), kAdjNodeBlock, 0, s>>>(g, a);
}
template <int D> void adj_cells(const Geo &g, const Fld &f, const Prm &p, const AdjBuf &a, int tail, cudaStream_t s) {
    if (p.eos) k_adj_cells<D, true><<<adj_blocks(g.N, kAdjCellBlock), kAdjCellBlock, 0, s>>>(g, f, p, a, tail);
    else k_adj_cells<D, false><<<adj_blocks(g.N, kAdjCellBlock), kAdjCellBlock, 0, s>>>(g, f, p, a, tail);
}
template <int D> void adj_gather(const Geo &g, const AdjBuf &a, cudaStream_t s) {
    k_adj_gather<D><<<adj_blocks(g.Np, kAdjNodeBlock), kAdjNodeBlock, 0, s>>>(g, a);
}
template <int D> void adj_faces(const Geo &g, const Fld &f, const AdjBuf &a, cudaStream_t s) {
    if (a.bf && g.nbf > 0) k_adj_faces<D><<<adj_blocks(g.nbf, kAdjNodeBlock), kAdjNodeBlock, 0, s>>>(g, f, a);
}
template <int D> void adj_bj_gather(const Geo &g, const Fld &f, const AdjBuf &a, cudaStream_t s) {
    if (a.bj) k_adj_bj_gather<D><<<adj_blocks(g.N, kAdjCellBlock), kAdjCellBlock, 0, s>>>(g, f, a);
}
template <int D> void adj_e0(const Geo &g, const Fld &f, const Prm &p, const AdjBuf &a, cudaStream_t s) {
    if (a.lE0) k_adj_e0<D><<<adj_blocks(g.N, kAdjCellBlock), kAdjCellBlock, 0, s>>>(g, f, p, a);
}
template <int D> void adj_z0(const Geo &g, const Fld &f, const Prm &p, const AdjBuf &a, cudaStream_t s) {
    k_adj_z0<D><<<adj_blocks(g.N, kAdjCellBlock), kAdjCellBlock, 0, s>>>(g, f, p, a);
}

}  // namespace

#define LMOOD_ADJ_OPS_TABLE(D)                                                                              \
    static const AdjOps table = {D, adj_update<D>, adj_nodes<D>, adj_predict<D>, adj_momsum<D>, adj_cells<D>, \
                                 adj_faces<D>, adj_gather<D>, adj_z0<D>, adj_bj_gather<D>, adj_e0<D>};       \
    return table;

}  // namespace lmood
