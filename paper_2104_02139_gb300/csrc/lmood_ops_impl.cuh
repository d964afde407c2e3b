// lmood_ops_impl.cuh -- launchers of the step kernels for one dimension D (LMOOD_DIM).
#pragma once
#include "lmood_kernels.cuh"
#include "lmood_ops.h"

namespace lmood {
namespace {

inline int blocks(int n, int b) { return (n + b - 1) / b; }

template <int D>
void predict(const Geo &g, const Fld &f, const Prm &p, const int *list, const int *cnt, int n, cudaStream_t s) {
    if (n > 0) k_predict<D><<<blocks(n, kCellBlock), kCellBlock, 0, s>>>(g, f, p, list, cnt, n);
}
template <int D>
void nodes(const Geo &g, const Fld &f, const int *list, const int *cnt, int n, int init_mode, cudaStream_t s) {
    if (n > 0) k_nodes<D><<<blocks(n, kNodeBlock), kNodeBlock, 0, s>>>(g, f, list, cnt, n, init_mode);
}
template <int D>
void update(const Geo &g, const Fld &f, const Prm &p, const int *list, const int *cnt, int n, int *tlist, int *tcnt,
            cudaStream_t s) {
    if (n > 0) k_update<D><<<blocks(n, kCellBlock), kCellBlock, 0, s>>>(g, f, p, list, cnt, n, tlist, tcnt);
}
template <int D>
void mark_nodes(const Geo &g, const Fld &f, const int *tlist, const int *tcnt, int n, int *node_mark, int stamp,
                int *nlist, cudaStream_t s) {
    if (n > 0) k_mark_nodes<D><<<blocks(n, 256), 256, 0, s>>>(g, f, tlist, tcnt, node_mark, stamp, nlist);
}
void mark_cells(const Geo &g, const Fld &f, const int *nlist, int n, int *cell_mark, int stamp, int *clist,
                cudaStream_t s) {
    if (n > 0) k_mark_cells<<<blocks(n, 256), 256, 0, s>>>(g, f, nlist, cell_mark, stamp, clist);
}
void dt_init(const Fld &f, const Prm &p, int n_inst, int first, cudaStream_t s) {
    k_dt_init<<<blocks(n_inst, 128), 128, 0, s>>>(f, p, n_inst, first);
}
void finalize(const Geo &g, const Fld &f, const Prm &p, cudaStream_t s) {
    k_finalize<<<blocks(g.N, 256), 256, 0, s>>>(g, f, p);
}
template <int D>
void init_cells(const Geo &g, const Fld &f, const Prm &p, double rho0, double *m, double *im, int f_given,
                cudaStream_t s) {
    k_init_cells<D><<<blocks(g.N, kCellBlock), kCellBlock, 0, s>>>(g, f, p, rho0, m, im, f_given);
}
template <int D> void refresh(const Geo &g, const Fld &f, const Prm &p, cudaStream_t s) {
    k_refresh<D><<<blocks(g.N, kCellBlock), kCellBlock, 0, s>>>(g, f, p);
}
template <int D> void totals(const Geo &g, const Fld &f, double *out, cudaStream_t s) {
    k_totals<D><<<blocks(g.N, 256), 256, 0, s>>>(g, f, out);
}

}  // namespace

#define LMOOD_OPS_TABLE(D)                                                                                  \
    static const Ops table = {D,          predict<D>,  nodes<D>,   update<D>, mark_nodes<D>, mark_cells, \
                              dt_init,    finalize,    init_cells<D>, refresh<D>, totals<D>};            \
    return table;

}  // namespace lmood
