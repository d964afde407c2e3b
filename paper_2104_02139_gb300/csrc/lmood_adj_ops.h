// lmood_adj_ops.h -- buffers and per-dimension launch table of the reverse-pass kernels (the
// adjoint of one step with its MOOD order mask and dt frozen; kernels in
// lmood_adjoint_kernels.cuh, one translation unit per dimension).
#pragma once
#include "lmood_dev.cuh"

namespace lmood {

// Device buffers of the reverse pass. "1" = adjoint of the t^{n+1} state (input of the
// reverse of step n), "0" = adjoint of the t^n state (its output); the host swaps the pairs
// between steps. Cell and node adjoints of the state are structure-of-arrays ([comp][n]);
// the records the reverse kernels pass to one another are arrays of structures (one
// contiguous record per corner, cell or node), so that the node-side gathers read whole
// sectors. Corner id k N + c.
template <int D> struct AdjRec {
    static constexpr int NS = D * (D + 1) / 2, NQ = D + D * D, NMOM = 1 + D + NS + NQ + NQ * D;
    // corner record of the update and nodal solve: packet adjoints lM [NS], lR [D], then the
    // update's products lvs, lx0, lx1, lvp0, lvp1 [D] each
    static constexpr int CR = NS + D + 5 * D, CR_M = 0, CR_R = NS, CR_U = NS + D;
    // corner record of the predictor: lxs [D], then the per-corner moment adjoints lU [NQ],
    // lS1 [D], ln
    static constexpr int CP = D + NQ + D + 1, CP_X = 0, CP_U = D, CP_S1 = D + NQ, CP_N = D + NQ + D;
    // cell record of the predictor: the moment adjoints equal at all its corners, lT [NQ][D],
    // lS2 [NS]
    static constexpr int CC = NQ * D + NS, CC_T = 0, CC_S2 = NQ * D;
};

struct AdjBuf {
    double *lv1, *lF1, *lv0, *lF0;    // cells: [D][N], [D*D][N]
    double *lE1, *lE0;                // cells: adjoints of e (NULL: not carried -- the
                                      // neo-Hookean volumetric law with no energy term in J)
    double *lz0;                      // cells: adjoint of z^n (scratch of one step)
    double *lmu;                      // cells: d/d mu, accumulated over the steps
    double *lx1, *lvp1, *lx0, *lvp0;  // nodes: [D][Np]
    double *cr;                       // corner records of update and nodal solve [NC][CR]
    double *cp;                       // corner records of the predictor [NC][CP]
    double *cc;                       // cell records of the predictor [N][CC]
    double *lm;                       // node moment adjoints [Np][NMOM]
    double *cd;                       // corner records of the cell gather: lx [NC][D]
    // the reverse predictor of the second-order cells in four kernels (adj::PredRec): the cell's
    // forward intermediates [N][F_LEN], each corner's [NC][K_LEN], the corners' pass-2 and
    // pass-1 products [NC][Q2_LEN], [NC][Q1_LEN]
    double *pf, *pk, *q2, *q1;
    // boundary faces of traction, pressure or velocity kind [nbf][D][D]: per node of the face
    // (slot i for its node i) the adjoint of the face's area vector from that node's solve,
    // then (k_adj_faces) the adjoint of that node's position; NULL when the mesh has none
    double *bf;
    // cells at the limited (Barth-Jespersen) level of this step: their records [N][B_LEN]
    // (adj::PredRec<D>::B_*); NULL when the step has none
    double *bj;
};

struct AdjOps {
    int dim;
    // cells: reverse of the cell update (with z^{n+1} treated as derived, so no adjoint of it)
    void (*update)(const Geo &, const Fld &, const Prm &, const AdjBuf &, cudaStream_t);
    // nodes: reverse of node motion and nodal solve; init_mode: the t^0 solve v_p^0 = v*_p
    void (*nodes)(const Geo &, const Fld &, const AdjBuf &, int init_mode, cudaStream_t);
    // cells: reverse of geometry, least squares, predictor and packets (force_p0: all cells P0)
    void (*predict)(const Geo &, const Fld &, const Prm &, const AdjBuf &, int force_p0, cudaStream_t);
    // nodes: adjoints of the node moments, summed over the corners around each node
    void (*momsum)(const Geo &, const Fld &, const AdjBuf &, cudaStream_t);
    // cells: reverse of the node moments (per corner of the cell), centroid and impedance of t^n;
    // tail: first the second-order cells' corner-matrix and geometry part of the predictor's
    // reverse (after predict without force_p0)
    void (*cells)(const Geo &, const Fld &, const Prm &, const AdjBuf &, int tail, cudaStream_t);
    // boundary faces: the area-vector adjoints left by the nodal solves -> the face nodes'
    // position adjoints (no launch when AdjBuf::bf is NULL)
    void (*faces)(const Geo &, const Fld &, const AdjBuf &, cudaStream_t);
    // nodes: gather of the per-corner (and per-face) position adjoints
    void (*gather)(const Geo &, const AdjBuf &, cudaStream_t);
    // cells: impedance of the initial state (after the t^0 predictor's reverse)
    void (*z0)(const Geo &, const Fld &, const Prm &, const AdjBuf &, cudaStream_t);
    // cells: the adjoints of the stencil bounds that set the limited cells' factors, gathered
    // into the cells that hold those bounds (no launch when AdjBuf::bj is NULL)
    void (*bj_gather)(const Geo &, const Fld &, const AdjBuf &, cudaStream_t);
    // cells: the adjoint of the initial energy e^0 (a function of v, F, mu) moved to v, F, mu
    void (*e0)(const Geo &, const Fld &, const Prm &, const AdjBuf &, cudaStream_t);
};

const AdjOps &adj_ops_dim2();
const AdjOps &adj_ops_dim3();

}  // namespace lmood
