// lmood_adj_ops.h -- buffers and per-dimension launch table of the reverse-pass kernels (the
// adjoint of one step with its MOOD order mask and dt frozen; kernels in
// lmood_adjoint_kernels.cuh, one translation unit per dimension).
#pragma once
#include "lmood_dev.cuh"

namespace lmood {

// Device buffers of the reverse pass. "1" = adjoint of the t^{n+1} state (input of the
// reverse of step n), "0" = adjoint of the t^n state (its output); the host swaps the pairs
// between steps. Corner arrays are [component][(D+1) N], corner id k N + c.
struct AdjBuf {
    double *lv1, *lF1, *lv0, *lF0;  // cells: [D][N], [D*D][N]
    double *lz0;                    // cells: adjoint of z^n (scratch of one step)
    double *lmu;                    // cells: d/d mu, accumulated over the steps
    double *lx1, *lvp1, *lx0, *lvp0;  // nodes: [D][Np]
    double *pkM, *pkR;              // corners: packet adjoints [NS], [D]
    double *ca;                     // corners: update products lvs, lx0, lx1, lvp0, lvp1 [5 D];
                                    //          later the moment products lxc, lq [D + D + D*D]
    double *cb;                     // corners: predictor products lxs [D], lmom [NMOM]
    double *cd;                     // corners: centroid / measure products lx [D] (aliases pkM)
};

struct AdjOps {
    int dim;
    // cells: reverse of the cell update (with z^{n+1} treated as derived, so no adjoint of it)
    void (*update)(const Geo &, const Fld &, const Prm &, const AdjBuf &, cudaStream_t);
    // nodes: reverse of node motion and nodal solve; init_mode: the t^0 solve v_p^0 = v*_p
    void (*nodes)(const Geo &, const Fld &, const AdjBuf &, int init_mode, cudaStream_t);
    // cells: reverse of geometry, least squares, predictor and packets (force_p0: all cells P0)
    void (*predict)(const Geo &, const Fld &, const Prm &, const AdjBuf &, int force_p0, cudaStream_t);
    // nodes: reverse of the node moments
    void (*moments)(const Geo &, const Fld &, const AdjBuf &, cudaStream_t);
    // cells: gathers of the moment products, centroid and impedance of the t^n state
    void (*cells)(const Geo &, const Fld &, const Prm &, const AdjBuf &, cudaStream_t);
    // nodes: gather of the per-corner position adjoints
    void (*gather)(const Geo &, const AdjBuf &, cudaStream_t);
    // cells: impedance of the initial state (after the t^0 predictor's reverse)
    void (*z0)(const Geo &, const Fld &, const Prm &, const AdjBuf &, cudaStream_t);
};

const AdjOps &adj_ops_dim2();
const AdjOps &adj_ops_dim3();

}  // namespace lmood
