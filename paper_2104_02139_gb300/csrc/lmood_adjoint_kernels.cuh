// lmood_adjoint_kernels.cuh -- kernels of the reverse pass of one step (adjoint with the
// MOOD order mask and dt frozen), templated on the dimension. They read the t^n state, the
// t^{n+1} node positions and velocities and the step's products (corner packets, v*_p, node
// moments) -- from the state's buffers after a replay of the step, or from a tape that kept
// them -- and, with the adjoints of the t^{n+1} state (lam x, lam v_p per node; lam v, lam F
// per cell; the impedance z of a state is a function of its F and x, so its adjoint is
// applied where the state is read), produce those of t^n:
//   k_adj_update   cells : reverse of the cell update -> corner records: packet adjoints and
//                          the update's products for the node adjoints
//   k_adj_nodes    nodes : reverse of node motion and nodal solve with BCs -> packet adjoints
//   k_adj_predict  cells : reverse of predictor, least squares, geometry -> position adjoints
//                          per corner, node-moment adjoints (per corner and per cell)
//   k_adj_momsum   nodes : node-moment adjoints summed over the corners around each node
//   k_adj_cells    cells : reverse of the node moments at the cell's corners, of the centroid
//                          and of the impedance of t^n
//   k_adj_gather   nodes : position adjoints of t^n
// Contributions are written per corner (corner id k N + c, one writer each) and gathered
// through the node -> corner CSR or the cell's own corners: no atomics, deterministic. The
// stored masses m_c stay fixed: the position adjoints are those of the map at fixed m.
#pragma once
#include "lmood_adj_ops.h"
#include "lmood_adjoint.cuh"

namespace lmood {

template <int D> __device__ __forceinline__ int cell_of_corner(int cid, int N) {
#pragma unroll
    for (int k = 0; k < D; ++k) cid -= cid >= N ? N : 0;
    return cid;
}

template <int D> __device__ __forceinline__ double kappa_mu_factor(const Prm &prm) {
    return prm.vol_coeff ? 1.0 : 2.0 / 3.0;  // d kappa / d mu
}

// ---------------------------------------------------------------------------------------
// E: the energy adjoint is carried (a.lE1, a.lE0): the energy equation's terms join the force part
template <int D, bool E> __global__ void __launch_bounds__(128) k_adj_update(Geo g, Fld f, Prm prm, AdjBuf a) {
    using Q = adj::Sz<D>;
    using R = AdjRec<D>;
    constexpr int NV = Q::NV, DD = Q::DD, NS = Q::NS, NX = NV * D;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    const int N = g.N, Np = g.Np, NC = NV * N;
    const double mu = f.mu[c], kap = kappa_of(prm, mu), dt = f.dt[g.cell_inst ? g.cell_inst[c] : 0];
    const int ord = f.order[c];
    // the velocity part first: its adjoints go to the corner records and lv0 at once, so that
    // none of its values is live in the deformation part
    {
        double vs[NX], M[NV * NS], lv1[D], lvs[NX] = {}, lv[D] = {}, lM[NV * NS] = {}, lR[NX] = {}, Rk[E ? NX : 1];
        for (int k = 0; k < NV; ++k) {
            const int p = g.c2n[k * N + c];
            for (int b = 0; b < D; ++b) vs[k * D + b] = f.vs[b * Np + p];
            for (int s = 0; s < NS; ++s) M[k * NS + s] = f.pkM[s * NC + k * N + c];
            if (E)
                for (int b = 0; b < D; ++b) Rk[k * D + b] = f.pkR[b * NC + k * N + c];
        }
        for (int b = 0; b < D; ++b) lv1[b] = a.lv1[b * N + c];
        if (E) {
            const double le1 = a.lE1[c];
            adj::update_force_vjp<D>(vs, M, f.im[c], dt, lv1, lvs, lM, lR, lv, le1, Rk);
            a.lE0[c] = le1;  // e^{n+1} = e^n + ...
        } else {
            adj::update_force_vjp<D>(vs, M, f.im[c], dt, lv1, lvs, lM, lR, lv);
        }
        for (int k = 0; k < NV; ++k) {
            double *r = a.cr + (size_t)(k * N + c) * R::CR;
            for (int s = 0; s < NS; ++s) r[R::CR_M + s] = lM[k * NS + s];
            for (int b = 0; b < D; ++b) {
                r[R::CR_R + b] = lR[k * D + b];
                r[R::CR_U + b] = lvs[k * D + b];
            }
        }
        for (int b = 0; b < D; ++b) a.lv0[b * N + c] = lv[b];
    }
    int pn[NV];
    for (int k = 0; k < NV; ++k) pn[k] = g.c2n[k * N + c];
    double lF[DD] = {}, lmu = 0.0, lkap = 0.0;
    // nodal inputs read at their use; nodal adjoints stored as they are formed (record slot i
    // of CR_U; the deformation part's lvs added to the velocity part's, stored above)
    auto ld = [&](int i, double *u) {
        const double *src = i == 0 ? f.vs : i == 1 ? f.x : i == 2 ? f.x1 : i == 3 ? f.vp : f.vp1;
        for (int k = 0; k < NV; ++k)
            for (int b = 0; b < D; ++b) u[k * D + b] = src[b * Np + pn[k]];
    };
    auto out = [&](int i, const double *l) {
        for (int k = 0; k < NV; ++k) {
            double *r = a.cr + (size_t)(k * N + c) * R::CR + R::CR_U + i * D;
            for (int b = 0; b < D; ++b) r[b] = i == 0 ? r[b] + l[k * D + b] : l[k * D + b];
        }
    };
    // F^n, the adjoint of F^{n+1} and F^{n+1} of the recorded step read where they are used
    adj::update_deform_vjp<D>(ld, out, f.F + c, f.m[c], mu, kap, dt, ord, a.lF1 + c, 0.0, lF, lmu, lkap, f.F1 + c,
                              (long)N);
    for (int q = 0; q < DD; ++q) a.lF0[q * N + c] = lF[q];
    a.lmu[c] += lmu + lkap * kappa_mu_factor<D>(prm);
}

// ---------------------------------------------------------------------------------------
// init_mode: the t^0 nodal solve v_p^0 = v*_p (no motion); lam v*_p = lam v_p^0. BC: the
// nodes with traction / pressure / velocity faces or contact walls (a second launch, only on
// meshes that have them), else the others (the first keeps the common kernel's registers low).
template <int D, bool BC>
__global__ void __launch_bounds__(128) k_adj_nodes(Geo g, Fld f, AdjBuf a, int init_mode) {
    using R = AdjRec<D>;
    constexpr int NV = D + 1;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.Np) return;
    const unsigned char ndf = g.bc_ndof[p];
    if (((ndf & (BC_EXT | BC_CONTACT)) != 0) != BC) return;
    const int N = g.N, Np = g.Np, NC = NV * N;
    double M[D * D] = {}, b[D] = {}, lvs[D] = {}, lx0[D] = {}, lx1[D] = {}, lvp0[D] = {}, lvp1[D] = {};
    const int j0 = g.n2c_off[p], j1 = g.n2c_off[p + 1];
    for (int j = j0; j < j1; ++j) {
        const int cid = g.n2c[j];
        for (int r = 0; r < D; ++r)
            for (int s = 0; s < D; ++s) M[r * D + s] += f.pkM[adj::sym<D>(r, s) * NC + cid];
        for (int r = 0; r < D; ++r) b[r] += f.pkR[r * NC + cid];
        if (!init_mode) {
            const double *rc = a.cr + (size_t)cid * R::CR + R::CR_U;
            for (int r = 0; r < D; ++r) {
                lvs[r] += rc[0 * D + r];
                lx0[r] += rc[1 * D + r];
                lx1[r] += rc[2 * D + r];
                lvp0[r] += rc[3 * D + r];
                lvp1[r] += rc[4 * D + r];
            }
        }
    }
    double lb[D], lM[D * D] = {}, tv[6];
    for (int i = 0; i < 6; ++i) tv[i] = g.bc_t[i * Np + p];
    if (init_mode) {
        for (int r = 0; r < D; ++r) lvs[r] = a.lvp1[r * Np + p];
    } else {
        const double dt = f.dt[g.node_inst ? g.node_inst[p] : 0];
        for (int r = 0; r < D; ++r) {
            const double lx1t = a.lx1[r * Np + p] + lx1[r];   // x^{n+1} = x^n + dt v*
            const double lvp1t = a.lvp1[r * Np + p] + lvp1[r]; // v_p^{n+1} = 2 v* - v_p^n
            lvs[r] += dt * lx1t + 2.0 * lvp1t;
            a.lx0[r * Np + p] = lx1t + lx0[r];
            a.lvp0[r * Np + p] = -lvp1t + lvp0[r];
        }
    }
    if constexpr (!BC) {
        adj::node_solve_vjp<D>(M, b, ndf & BC_NDOF, tv, lvs, lb, lM);
    } else {
        // traction / pressure / velocity faces and contact walls: the faces' area-vector
        // adjoints go to the node's slot of each face record (summed and moved to the face's
        // nodes by k_adj_faces)
        const int jb0 = g.nbf_off[p], nf = g.nbf_off[p + 1] - jb0, nb = g.nbf;
        auto fc = [&](int j, int &tag, double *N, double *val) {
            const int fid = g.nbf_idx[jb0 + j];
            tag = g.bf_tag[fid];
            if (tag < TAG_TRACTION || tag > TAG_VELOCITY) return;
            double xq[D * D];
            for (int i = 0; i < D; ++i)
                for (int c = 0; c < D; ++c) xq[i * D + c] = f.x[c * Np + g.bf_nodes[i * nb + fid]];
            adj::bface_area<D>(xq, N);
            for (int c = 0; c < D; ++c) val[c] = g.bf_val[c * nb + fid];
        };
        auto ln = [&](int j, const double *lN) {
            const int fid = g.nbf_idx[jb0 + j], tag = g.bf_tag[fid];
            if (tag < TAG_TRACTION || tag > TAG_VELOCITY) return;
            int i = 0;
            while (i < D - 1 && g.bf_nodes[i * nb + fid] != p) ++i;
            for (int c = 0; c < D; ++c) a.bf[((size_t)fid * D + i) * D + c] = lN[c];
        };
        double xp[D];
        for (int c = 0; c < D; ++c) xp[c] = f.x[c * Np + p];
        const int nw = (ndf & BC_CONTACT) ? (int)g.contact[0] : 0;
        adj::node_solve_bc_vjp<D>(M, b, ndf & BC_NDOF, tv, (ndf & BC_EXT) != 0, nf, fc, nw, g.contact + 2,
                                  g.contact[1], xp, lvs, lb, lM, ln);
    }
    for (int j = j0; j < j1; ++j) {
        double *r = a.cr + (size_t)g.n2c[j] * R::CR;
        for (int q = 0; q < D; ++q) r[R::CR_R + q] = (init_mode ? 0.0 : r[R::CR_R + q]) + lb[q];
        for (int q = 0; q < D; ++q)
            for (int s = q; s < D; ++s) {
                const double l = q == s ? lM[q * D + q] : lM[q * D + s] + lM[s * D + q];
                double &m = r[R::CR_M + adj::sym<D>(q, s)];
                m = (init_mode ? 0.0 : m) + l;
            }
    }
}

// ---------------------------------------------------------------------------------------
// Reverse of geometry, least squares, predictor and packets. A first-order cell's product is
// small and stays whole (k_adj_predict); a second-order cell's runs as four kernels, so that
// no thread holds the cell's forward intermediates and all its adjoint accumulators at once:
//   k_adj_pred_fw  cells   : forward intermediates -> records pf (cell), pk (corners)
//   k_adj_pred_c2  corners : reverse of the packet R_k (one stress product) -> q2, lM_k
//   k_adj_pred_c1  corners : reverse of the corner's term of dv (one stress product) -> q1
//   k_adj_predict  cells   : the rest (slopes, least squares, corner matrices, geometry), and
//                            the whole product of the first-order cells
// force_p0: the t^0 packets (every cell first order; only k_adj_predict runs).
// ---------------------------------------------------------------------------------------
template <int D> __device__ __forceinline__ bool second_order(const Fld &f, int c, int force_p0) {
    return !force_p0 && f.order[c] != 1;
}

// MAT: 0 the neo-Hookean law, 1 the shear energy family (a = prm.shear_a), 2 the stiffened gas
// (with that shear energy); the neo-Hookean instances compile no code of the others
template <int MAT> __device__ __forceinline__ double mat_a(const Prm &prm) { return MAT ? prm.shear_a : -1.0; }

// BJ: the cells at the limited level (order 3) alone, else the other second-order cells
template <int D, int MAT, bool BJ>
__global__ void __launch_bounds__(128) k_adj_pred_fw(Geo g, Fld f, Prm prm, AdjBuf a) {
    using Q = adj::Sz<D>;
    using P = adj::PredRec<D>;
    constexpr int NV = Q::NV, DD = Q::DD, NX = NV * D, NQ = Q::NQ;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N || !second_order<D>(f, c, 0) || (f.order[c] == 3) != BJ) return;
    const int N = g.N, Np = g.Np;
    double xs[NX], vc[D], Fc[DD];
    adj::Mom<D> mom;
    mom.stride = Np;
    for (int k = 0; k < NV; ++k) {
        const int p = g.c2n[k * N + c];
        mom.p[k] = f.mom + p;
        for (int b = 0; b < D; ++b) xs[k * D + b] = f.x[b * Np + p];
    }
    for (int b = 0; b < D; ++b) vc[b] = f.v[b * N + c];
    for (int q = 0; q < DD; ++q) Fc[q] = f.F[q * N + c];
    const double mu = f.mu[c], kap = kappa_of(prm, mu), dt = f.dt[g.cell_inst ? g.cell_inst[c] : 0];
    const adj::SgMat sgm{prm.gamma, prm.pinf, prm.rho0};
    double lo[BJ ? NQ : 1], hi[BJ ? NQ : 1];
    int tlo[BJ ? NQ : 1], thi[BJ ? NQ : 1];
    double *bjr = nullptr;
    if constexpr (BJ) {
        // each field's range over the cells around the cell's nodes and the cell, and the cells
        // that hold its ends: on a tie the cell itself, else the smallest cell id (the choice of
        // a derivative where the range is not differentiable; the oracle's, whose stencil is in
        // ascending order)
        for (int q = 0; q < NQ; ++q) {
            lo[q] = hi[q] = q < D ? vc[q] : Fc[q - D];
            tlo[q] = thi[q] = c;
        }
        for (int k = 0; k < NV; ++k) {
            const int p = g.c2n[k * N + c];
            for (int j = g.n2c_off[p]; j < g.n2c_off[p + 1]; ++j) {
                const int o = cell_of_corner<D>(g.n2c[j], N);
                for (int q = 0; q < NQ; ++q) {
                    const double qo = q < D ? f.v[q * N + o] : f.F[(q - D) * N + o];
                    if (qo < lo[q] || (qo == lo[q] && tlo[q] != c && o < tlo[q])) {
                        lo[q] = qo;
                        tlo[q] = o;
                    }
                    if (qo > hi[q] || (qo == hi[q] && thi[q] != c && o < thi[q])) {
                        hi[q] = qo;
                        thi[q] = o;
                    }
                }
            }
        }
        bjr = a.bj + (size_t)c * P::B_LEN;
    }
    adj::predict_fw_rec<D>(xs, mom, vc, Fc, f.z[c], mu, kap, f.im[c], dt, a.pf + (size_t)c * P::F_LEN,
                           a.pk + (size_t)c * P::K_LEN, (long)N * P::K_LEN, mat_a<MAT>(prm), MAT == 2 ? &sgm : nullptr,
                           f.e[c], bjr, BJ ? lo : nullptr, BJ ? hi : nullptr, f.dvs ? f.dvs + c : nullptr, (long)N);
    if constexpr (BJ)
        for (int q = 0; q < NQ; ++q) {
            const int sel = (int)bjr[P::B_SEL + q], t = sel > 0 ? thi[q] : sel < 0 ? tlo[q] : -1;
            bjr[P::B_T + q] = t == c ? -1 : t;
            if (t == c) bjr[P::B_SEL + q] = 2 * sel;  // the cell's own value: phi = 0 identically
        }
}

template <int D, int MAT> __global__ void __launch_bounds__(128) k_adj_pred_c2(Geo g, Fld f, Prm prm, AdjBuf a) {
    using R = AdjRec<D>;
    using P = adj::PredRec<D>;
    constexpr int NS = R::NS;
    const int N = g.N;
    const int cid = blockIdx.x * blockDim.x + threadIdx.x;
    if (cid >= (D + 1) * N) return;
    const int c = cell_of_corner<D>(cid, N), k = (cid - c) / N;
    if (!second_order<D>(f, c, 0)) return;
    const double mu = f.mu[c], kap = kappa_of(prm, mu), dt = f.dt[g.cell_inst ? g.cell_inst[c] : 0];
    const adj::SgMat sgm{prm.gamma, prm.pinf, prm.rho0};
    double *cr = a.cr + (size_t)cid * R::CR;
    double lR[D], lM[NS];
    for (int b = 0; b < D; ++b) lR[b] = cr[R::CR_R + b];
    for (int s2 = 0; s2 < NS; ++s2) lM[s2] = cr[R::CR_M + s2];
    adj::predict_corner2_vjp<D>(a.pf + (size_t)c * P::F_LEN, a.pk + (size_t)cid * P::K_LEN, k, mu, kap, dt, lR, lM,
                                a.q2 + (size_t)cid * P::Q2_LEN, mat_a<MAT>(prm), MAT == 2 ? &sgm : nullptr);
    for (int s2 = 0; s2 < NS; ++s2) cr[R::CR_M + s2] = lM[s2];
}

template <int D, int MAT> __global__ void __launch_bounds__(128) k_adj_pred_c1(Geo g, Fld f, Prm prm, AdjBuf a) {
    using P = adj::PredRec<D>;
    const int N = g.N;
    const int cid = blockIdx.x * blockDim.x + threadIdx.x;
    if (cid >= (D + 1) * N) return;
    const int c = cell_of_corner<D>(cid, N), k = (cid - c) / N;
    if (!second_order<D>(f, c, 0)) return;
    const double mu = f.mu[c], kap = kappa_of(prm, mu), dt = f.dt[g.cell_inst ? g.cell_inst[c] : 0];
    const adj::SgMat sgm{prm.gamma, prm.pinf, prm.rho0};
    // the adjoint of dv = hv sum_k T(F_h,k) N_k is the sum of the corners' lv*
    double lacc[D] = {};
    for (int kk = 0; kk <= D; ++kk)
        for (int b = 0; b < D; ++b) lacc[b] += a.q2[(size_t)(kk * N + c) * P::Q2_LEN + P::Q2_LV + b];
    const double hv = -0.5 * dt * f.im[c] * (1.0 / D);
    for (int b = 0; b < D; ++b) lacc[b] *= hv;
    adj::predict_corner1_vjp<D>(a.pf + (size_t)c * P::F_LEN, a.pk + (size_t)cid * P::K_LEN, k, mu, kap, lacc,
                                a.q1 + (size_t)cid * P::Q1_LEN, mat_a<MAT>(prm), MAT == 2 ? &sgm : nullptr);
}

// node-moment adjoint writer of cell c: the parts equal at every corner (lT, lS2) into the
// cell record (stored once, at k = 0), the others into the corner records
template <int D> struct MomOut {
    double *cp, *ccr;
    int N, c;
    __device__ void operator()(int k, int j, double v) const {
        using Q = adj::Sz<D>;
        using R = AdjRec<D>;
        double *cpr = cp + (size_t)(k * N + c) * R::CP;
        if (j >= Q::M_T) {
            if (k == 0) ccr[R::CC_T + (j - Q::M_T)] = v;
        } else if (j >= Q::M_U) {
            cpr[R::CP_U + (j - Q::M_U)] = v;
        } else if (j >= Q::M_S2) {
            if (k == 0) ccr[R::CC_S2 + (j - Q::M_S2)] = v;
        } else if (j >= Q::M_S1) {
            cpr[R::CP_S1 + (j - Q::M_S1)] = v;
        } else {
            cpr[R::CP_N] = v;
        }
    }
};

template <int D>
__device__ __forceinline__ void adj_predict_out(const AdjBuf &a, const Prm &prm, int N, int c, const double *lxs,
                                                const double *lvc, const double *lF, double lz, double lmu,
                                                double lkap) {
    using R = AdjRec<D>;
    for (int k = 0; k <= D; ++k)
        for (int b = 0; b < D; ++b) a.cp[(size_t)(k * N + c) * R::CP + R::CP_X + b] = lxs[k * D + b];
    for (int b = 0; b < D; ++b) a.lv0[b * N + c] += lvc[b];
    for (int q = 0; q < D * D; ++q) a.lF0[q * N + c] += lF[q];
    a.lz0[c] = lz;
    a.lmu[c] += lmu + lkap * kappa_mu_factor<D>(prm);
}

// the rest of a second-order cell's product (after k_adj_pred_c1) but the corner matrices and
// the geometry: the slopes, dF/dt and the least squares; writes the position adjoints of
// d_k = x_k - x_c (the corner records) and x_c (lxcc, into the pass-1 records' spare room:
// the pass-1 records are consumed here)
template <int D, int MAT, bool BJ>
__global__ void __launch_bounds__(128) k_adj_pred_fin(Geo g, Fld f, Prm prm, AdjBuf a) {
    using Q = adj::Sz<D>;
    using R = AdjRec<D>;
    using P = adj::PredRec<D>;
    constexpr int NV = Q::NV, DD = Q::DD, NX = NV * D;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N || !second_order<D>(f, c, 0) || (f.order[c] == 3) != BJ) return;
    const int N = g.N, Np = g.Np;
    adj::Mom<D> mom;
    mom.stride = Np;
    for (int k = 0; k < NV; ++k) mom.p[k] = f.mom + g.c2n[k * N + c];
    const double dt = f.dt[g.cell_inst ? g.cell_inst[c] : 0];
    double lxs[NX] = {}, lxcc[D] = {}, lvc[D] = {}, lF[DD] = {}, lmu = 0.0, lkap = 0.0, le = 0.0;
    for (int k = 0; k < NV; ++k) {
        const double *q2 = a.q2 + (size_t)(k * N + c) * P::Q2_LEN, *q1 = a.q1 + (size_t)(k * N + c) * P::Q1_LEN;
        lmu += q2[P::Q2_MU] + q1[P::Q1_MU];
        lkap += q2[P::Q2_KAP] + q1[P::Q1_KAP];
    }
    const adj::SgMat sgm{prm.gamma, prm.pinf, prm.rho0};
    adj::predict_finish_vjp<D>(
        mom, f.v + c, f.F + c, dt, a.pf + (size_t)c * P::F_LEN,
        [&](int k) { return (const double *)(a.q2 + (size_t)(k * N + c) * P::Q2_LEN); },
        [&](int k) { return (const double *)(a.q1 + (size_t)(k * N + c) * P::Q1_LEN); }, lxs, lxcc,
        MomOut<D>{a.cp, a.cc + (size_t)c * R::CC, N, c}, lvc, lF, MAT == 2 ? &sgm : nullptr, f.mu[c],
        mat_a<MAT>(prm), f.im[c], &lmu, &le, BJ ? a.bj + (size_t)c * P::B_LEN : nullptr, (long)N);
    if (MAT == 2) a.lE0[c] += le;
    for (int k = 0; k < NV; ++k)
        for (int b = 0; b < D; ++b) a.cp[(size_t)(k * N + c) * R::CP + R::CP_X + b] = lxs[k * D + b];
    // lxcc for the tail, in the first corner's pass-1 record (its lF_h is consumed)
    for (int b = 0; b < D; ++b) a.q1[(size_t)c * P::Q1_LEN + P::Q1_LF + b] = lxcc[b];
    for (int b = 0; b < D; ++b) a.lv0[b * N + c] += lvc[b];
    for (int q = 0; q < DD; ++q) a.lF0[q * N + c] += lF[q];
    a.lmu[c] += lmu + lkap * kappa_mu_factor<D>(prm);
}

// the whole product of a first-order cell (force_p0: every cell, the t^0 packets)
template <int D, int MAT>
__global__ void __launch_bounds__(128) k_adj_predict(Geo g, Fld f, Prm prm, AdjBuf a, int force_p0) {
    using Q = adj::Sz<D>;
    using R = AdjRec<D>;
    constexpr int NV = Q::NV, DD = Q::DD, NS = Q::NS, NX = NV * D;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N || second_order<D>(f, c, force_p0)) return;
    const int N = g.N, Np = g.Np;
    double xs[NX], vc[D], Fc[DD], lM[NV * NS], lR[NX];
    for (int k = 0; k < NV; ++k) {
        const int p = g.c2n[k * N + c];
        for (int b = 0; b < D; ++b) xs[k * D + b] = f.x[b * Np + p];
        const double *r = a.cr + (size_t)(k * N + c) * R::CR;
        for (int b = 0; b < D; ++b) lR[k * D + b] = r[R::CR_R + b];
        for (int s = 0; s < NS; ++s) lM[k * NS + s] = r[R::CR_M + s];
    }
    for (int b = 0; b < D; ++b) vc[b] = f.v[b * N + c];
    for (int q = 0; q < DD; ++q) Fc[q] = f.F[q * N + c];
    const double mu = f.mu[c], kap = kappa_of(prm, mu);
    const adj::SgMat sgm{prm.gamma, prm.pinf, prm.rho0};
    double lxs[NX] = {}, lvc[D] = {}, lF[DD] = {}, lz = 0.0, lmu = 0.0, lkap = 0.0, le = 0.0;
    adj::predict_p0_vjp<D>(xs, vc, Fc, f.z[c], mu, kap, lM, lR, lxs, MomOut<D>{a.cp, a.cc + (size_t)c * R::CC, N, c},
                           lvc, lF, lz, lmu, lkap, mat_a<MAT>(prm), MAT == 2 ? &sgm : nullptr, f.e[c], &le);
    adj_predict_out<D>(a, prm, N, c, lxs, lvc, lF, lz, lmu, lkap);
    if (MAT == 2) a.lE0[c] += le;
}

// ---------------------------------------------------------------------------------------
// node-moment adjoints of node p: the corner parts of its corners and the cell parts of the
// cells around it, in the corners' CSR order
template <int D> __global__ void __launch_bounds__(128) k_adj_momsum(Geo g, AdjBuf a) {
    using Q = adj::Sz<D>;
    using R = AdjRec<D>;
    constexpr int NQ = Q::NQ, NS = Q::NS, NM = Q::NMOM;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.Np) return;
    const int N = g.N;
    double lm[NM];
    for (int j = 0; j < NM; ++j) lm[j] = 0.0;
    for (int j = g.n2c_off[p]; j < g.n2c_off[p + 1]; ++j) {
        const int cid = g.n2c[j];
        const double *cp = a.cp + (size_t)cid * R::CP;
        const double *cc = a.cc + (size_t)cell_of_corner<D>(cid, N) * R::CC;
        lm[Q::M_N] += cp[R::CP_N];
        for (int b = 0; b < D; ++b) lm[Q::M_S1 + b] += cp[R::CP_S1 + b];
        for (int s = 0; s < NS; ++s) lm[Q::M_S2 + s] += cc[R::CC_S2 + s];
        for (int q = 0; q < NQ; ++q) lm[Q::M_U + q] += cp[R::CP_U + q];
        for (int i = 0; i < NQ * D; ++i) lm[Q::M_T + i] += cc[R::CC_T + i];
    }
    double *o = a.lm + (size_t)p * NM;
    for (int j = 0; j < NM; ++j) o[j] = lm[j];
}

// ---------------------------------------------------------------------------------------
// per cell: the reverse of the node moments at its corners (the cell as a neighbour of each
// of its nodes), of its centroid x_c = mean of its nodes, and of the impedance
// z^n = Z(F^n, m / V(x^n), mu)
// SG: the stiffened gas (its impedance depends on the energy)
template <int D, bool SG> __global__ void __launch_bounds__(128) k_adj_cells(Geo g, Fld f, Prm prm, AdjBuf a, int tail) {
    using Q = adj::Sz<D>;
    using R = AdjRec<D>;
    using P = adj::PredRec<D>;
    constexpr int NV = Q::NV, DD = Q::DD, NQ = Q::NQ, NX = NV * D, NM = Q::NMOM;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    const int N = g.N, Np = g.Np;
    double xs[NX], xc[D], q[NQ], lxc[D] = {}, lq[NQ] = {}, lxp[NX] = {};
    for (int k = 0; k < NV; ++k) {
        const int p = g.c2n[k * N + c];
        for (int b = 0; b < D; ++b) xs[k * D + b] = f.x[b * Np + p];
    }
    // a second-order cell's predictor product ends here: its corner matrices and geometry
    // (lz^n, and position adjoints into lxp); lxcc was left in the first corner's pass-1 record
    if (tail && second_order<D>(f, c, 0)) {
        double lxcc[D], lz = 0.0;
        for (int b = 0; b < D; ++b) lxcc[b] = a.q1[(size_t)c * P::Q1_LEN + P::Q1_LF + b];
        adj::predict_tail_p1_vjp<D>(
            xs, f.z[c], a.pf + (size_t)c * P::F_LEN,
            [&](int k) { return (const double *)(a.cr + (size_t)(k * N + c) * R::CR + R::CR_M); },
            [&](int k) { return (const double *)(a.q2 + (size_t)(k * N + c) * P::Q2_LEN); },
            [&](int k) { return (const double *)(a.q1 + (size_t)(k * N + c) * P::Q1_LEN); }, lxcc, lxp, lz);
        a.lz0[c] = lz;
    }
    for (int b = 0; b < D; ++b) xc[b] = f.xc[b * N + c];
    for (int i = 0; i < NQ; ++i) q[i] = i < D ? f.v[i * N + c] : f.F[(i - D) * N + c];
    for (int k = 0; k < NV; ++k) {
        const int p = g.c2n[k * N + c];
        const double *lm = a.lm + (size_t)p * NM;
        adj::moments_corner_vjp<D>([&](int j) { return lm[j]; }, xc, xs + k * D, q, lxc, lq, lxp + k * D);
    }
    for (int b = 0; b < D; ++b) a.lv0[b * N + c] += lq[b];
    // z^n
    double F[DD], lF[DD] = {}, lrho = 0.0, lmu = 0.0, lkap = 0.0;
    for (int i = 0; i < DD; ++i) F[i] = q[D + i];
    double V, Nf[NX];
    adj::faces<D>(xs, V, Nf);
    const double mu = f.mu[c], kap = kappa_of(prm, mu);
    if (SG) {  // z = z(F, rho, mu, eps), eps = e - |v|^2 / 2
        const adj::SgMat sgm{prm.gamma, prm.pinf, prm.rho0};
        double eps = f.e[c], leps = 0.0;
        for (int b = 0; b < D; ++b) eps -= 0.5 * q[b] * q[b];
        adj::impedance_sg_a_vjp<D>(F, f.m[c] / V, mu, prm.shear_a, sgm, eps, a.lz0[c], lF, lrho, lmu, leps);
        a.lE0[c] += leps;
        for (int b = 0; b < D; ++b) a.lv0[b * N + c] -= leps * q[b];
    } else {
        adj::impedance_vjp<D>(F, f.m[c] / V, mu, kap, a.lz0[c], lF, lrho, lmu, lkap);
    }
    for (int i = 0; i < DD; ++i) a.lF0[i * N + c] += lF[i] + lq[D + i];
    a.lmu[c] += lmu + lkap * kappa_mu_factor<D>(prm);
    const double lV = lrho * (-f.m[c] / (V * V));
    double lxs[NX] = {}, lN0[NX] = {};
    adj::faces_vjp<D>(xs, lV, lN0, lxs);
    for (int k = 0; k < NV; ++k)
        for (int b = 0; b < D; ++b)
            a.cd[(size_t)(k * N + c) * D + b] = lxs[k * D + b] + lxc[b] * (1.0 / NV) + lxp[k * D + b];
}

template <int D> __global__ void __launch_bounds__(128) k_adj_gather(Geo g, AdjBuf a) {
    using R = AdjRec<D>;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.Np) return;
    const int Np = g.Np;
    double l[D] = {};
    for (int j = g.n2c_off[p]; j < g.n2c_off[p + 1]; ++j) {
        const size_t cid = g.n2c[j];
        for (int b = 0; b < D; ++b) l[b] += a.cp[cid * R::CP + R::CP_X + b] + a.cd[cid * D + b];
    }
    if (a.bf && (g.bc_ndof[p] & BC_EXT))  // the node's share of its boundary faces' products
        for (int j = g.nbf_off[p]; j < g.nbf_off[p + 1]; ++j) {
            const int fid = g.nbf_idx[j], tag = g.bf_tag[fid];
            if (tag < TAG_TRACTION || tag > TAG_VELOCITY) continue;
            int i = 0;
            while (i < D - 1 && g.bf_nodes[i * g.nbf + fid] != p) ++i;
            for (int b = 0; b < D; ++b) l[b] += a.bf[((size_t)fid * D + i) * D + b];
        }
    for (int b = 0; b < D; ++b) a.lx0[b * Np + p] += l[b];
}

// boundary faces of traction, pressure or velocity kind: the area-vector adjoints the face's
// D nodes left in its record (k_adj_nodes) summed, and their product with respect to the
// face's node positions written back into the same record, slot i for the face's node i
template <int D> __global__ void __launch_bounds__(128) k_adj_faces(Geo g, Fld f, AdjBuf a) {
    const int fid = blockIdx.x * blockDim.x + threadIdx.x;
    if (fid >= g.nbf) return;
    const int tag = g.bf_tag[fid];
    if (tag < TAG_TRACTION || tag > TAG_VELOCITY) return;
    const int nb = g.nbf, Np = g.Np;
    double *r = a.bf + (size_t)fid * D * D;
    double lN[D] = {}, xq[D * D], lxq[D * D] = {};
    for (int i = 0; i < D; ++i)
        for (int c = 0; c < D; ++c) {
            lN[c] += r[i * D + c];
            xq[i * D + c] = f.x[c * Np + g.bf_nodes[i * nb + fid]];
        }
    adj::bface_area_vjp<D>(xq, lN, lxq);
    for (int i = 0; i < D * D; ++i) r[i] = lxq[i];
}

// impedance of the initial state only (the t^0 packets' z): lmu and lF from lz0
template <int D> __global__ void __launch_bounds__(128) k_adj_z0(Geo g, Fld f, Prm prm, AdjBuf a) {
    using Q = adj::Sz<D>;
    constexpr int NV = Q::NV, DD = Q::DD, NX = NV * D;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    const int N = g.N, Np = g.Np;
    double xs[NX], F[DD], lF[DD] = {}, lrho = 0.0, lmu = 0.0, lkap = 0.0, V, Nf[NX];
    for (int k = 0; k < NV; ++k)
        for (int b = 0; b < D; ++b) xs[k * D + b] = f.x[b * Np + g.c2n[k * N + c]];
    for (int q = 0; q < DD; ++q) F[q] = f.F[q * N + c];
    adj::faces<D>(xs, V, Nf);
    const double mu = f.mu[c], kap = kappa_of(prm, mu);
    if (prm.eos) {  // the stiffened gas: z depends on eps = e - |v|^2 / 2
        const adj::SgMat sgm{prm.gamma, prm.pinf, prm.rho0};
        double eps = f.e[c], leps = 0.0;
        for (int b = 0; b < D; ++b) eps -= 0.5 * f.v[b * N + c] * f.v[b * N + c];
        adj::impedance_sg_a_vjp<D>(F, f.m[c] / V, mu, prm.shear_a, sgm, eps, a.lz0[c], lF, lrho, lmu, leps);
        a.lE0[c] += leps;
        for (int b = 0; b < D; ++b) a.lv0[b * N + c] -= leps * f.v[b * N + c];
    } else {
        adj::impedance_vjp<D>(F, f.m[c] / V, mu, kap, a.lz0[c], lF, lrho, lmu, lkap);
    }
    for (int q = 0; q < DD; ++q) a.lF0[q * N + c] += lF[q];
    a.lmu[c] += lmu + lkap * kappa_mu_factor<D>(prm);
    // rho = m / V at fixed m: the positions' part, added to the corners' records of the t^0
    // packets' product (k_adj_predict wrote them)
    using R = AdjRec<D>;
    double lxs[NX] = {}, lN0[NX] = {};
    adj::faces_vjp<D>(xs, -lrho * f.m[c] / (V * V), lN0, lxs);
    for (int k = 0; k < NV; ++k)
        for (int b = 0; b < D; ++b) a.cp[(size_t)(k * N + c) * R::CP + R::CP_X + b] += lxs[k * D + b];
}

// the adjoints of the bounds that set the limited cells' factors: cell o adds those of the
// limited cells around its nodes that name it (each such cell once: it is skipped at a node
// of o when it also holds one of o's earlier nodes); no atomics, a fixed order
template <int D> __global__ void __launch_bounds__(128) k_adj_bj_gather(Geo g, Fld f, AdjBuf a) {
    using P = adj::PredRec<D>;
    constexpr int NV = D + 1, NQ = D + D * D;
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= g.N) return;
    const int N = g.N;
    double l[NQ];
    for (int q = 0; q < NQ; ++q) l[q] = 0.0;
    bool any = false;
    for (int k = 0; k < NV; ++k) {
        const int p = g.c2n[k * N + o];
        for (int j = g.n2c_off[p]; j < g.n2c_off[p + 1]; ++j) {
            const int c = cell_of_corner<D>(g.n2c[j], N);
            if (f.order[c] != 3) continue;
            bool seen = false;
            for (int kk = 0; kk < k; ++kk) {
                const int pk = g.c2n[kk * N + o];
                for (int jj = 0; jj < NV; ++jj) seen |= g.c2n[jj * N + c] == pk;
            }
            if (seen) continue;
            const double *r = a.bj + (size_t)c * P::B_LEN;
            for (int q = 0; q < NQ; ++q)
                if ((int)r[P::B_T + q] == o) {
                    l[q] += r[P::B_LE + q];
                    any = true;
                }
        }
    }
    if (!any) return;
    for (int b = 0; b < D; ++b) a.lv0[b * N + o] += l[b];
    for (int q = 0; q < D * D; ++q) a.lF0[q * N + o] += l[D + q];
}

// the initial energy e^0 = |v|^2 / 2 + Psi(F) (Eq. EOS_neoHook with the family's shear energy)
// or, for the stiffened gas, |v|^2 / 2 + eps_v(F) + Psi_s(F) with eps_v the volumetric energy of
// the pressure p0 at rho0 / det F: its adjoint (lE0) moved to v, F, mu
template <int D> __global__ void __launch_bounds__(128) k_adj_e0(Geo g, Fld f, Prm prm, AdjBuf a) {
    constexpr int DD = D * D;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    const int N = g.N;
    const double le = a.lE0[c];
    double F[DD], lF[DD] = {}, lmu = 0.0;
    for (int q = 0; q < DD; ++q) F[q] = f.F[q * N + c];
    const double mu = f.mu[c];
    for (int b = 0; b < D; ++b) a.lv0[b * N + c] += le * f.v[b * N + c];
    adj::shear_energy_a_vjp<D>(F, prm.rho0, mu, prm.shear_a, le, lF, lmu);
    double C[DD];
    adj::cofactor<D>(F, C);
    const double J = adj::det<D>(F);
    double lJ;
    if (prm.eos) {  // eps_v = (p0 + gam pinf) J / ((gam - 1) rho0)
        lJ = le * (prm.p0 + prm.gamma * prm.pinf) / ((prm.gamma - 1.0) * prm.rho0);
    } else {  // Psi_v = kap / (4 rho0) ((J - 1)^2 + log^2 J)
        const double kap = kappa_of(prm, mu), lj = adj::adj_log(J);
        lJ = le * kap / (4.0 * prm.rho0) * (2.0 * (J - 1.0) + 2.0 * lj / J);
        lmu += le * ((J - 1.0) * (J - 1.0) + lj * lj) / (4.0 * prm.rho0) * kappa_mu_factor<D>(prm);
    }
    for (int q = 0; q < DD; ++q) a.lF0[q * N + c] += lF[q] + lJ * C[q];
    a.lmu[c] += lmu;
}

}  // namespace lmood
