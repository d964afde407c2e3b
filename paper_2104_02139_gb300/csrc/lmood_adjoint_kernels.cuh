// lmood_adjoint_kernels.cuh -- kernels of the reverse pass of one step (adjoint with the
// MOOD order mask and dt frozen), templated on the dimension. The forward step is first
// replayed from the stored state t^n (same kernels, recorded mask and dt), so that the
// packets, v*_p and the state t^{n+1} are in the state's buffers; then, with the adjoints of
// the t^{n+1} state (lam x, lam v_p per node; lam v, lam F per cell; the impedance z of a
// state is a function of its F and x, so its adjoint is applied where the state is read):
//   k_adj_update   cells : product of the cell update -> packet adjoints and per-corner
//                          contributions to the node adjoints
//   k_adj_nodes    nodes : node motion and nodal solve with BCs -> packet adjoints
//   k_adj_predict  cells : predictor, least squares, geometry -> node-moment adjoints
//   k_adj_moments  nodes : node moments -> per-corner adjoints of the cells' x_c, v, F
//   k_adj_cells    cells : gather of those, centroid and impedance of the t^n state
//   k_adj_gather   nodes : node adjoints of t^n
// The stored masses m_c stay fixed: the position adjoints are those of the map at fixed m.
// Contributions are written per corner (corner id k N + c, one writer each) and gathered
// through the node -> corner CSR or the cell's own corners: no atomics, deterministic.
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
template <int D> __global__ void __launch_bounds__(128) k_adj_update(Geo g, Fld f, Prm prm, AdjBuf a) {
    using Q = adj::Sz<D>;
    constexpr int NV = Q::NV, DD = Q::DD, NS = Q::NS, NX = NV * D;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    const int N = g.N, Np = g.Np, NC = NV * N;
    double xs0[NX], xs1[NX], vs[NX], vp0[NX], vp1[NX], M[NV * NS], R[NX], v[D], F[DD];
    for (int k = 0; k < NV; ++k) {
        const int p = g.c2n[k * N + c];
        for (int b = 0; b < D; ++b) {
            xs0[k * D + b] = f.x[b * Np + p];
            xs1[k * D + b] = f.x1[b * Np + p];
            vs[k * D + b] = f.vs[b * Np + p];
            vp0[k * D + b] = f.vp[b * Np + p];
            vp1[k * D + b] = f.vp1[b * Np + p];
            R[k * D + b] = f.pkR[b * NC + k * N + c];
        }
        for (int s = 0; s < NS; ++s) M[k * NS + s] = f.pkM[s * NC + k * N + c];
    }
    for (int b = 0; b < D; ++b) v[b] = f.v[b * N + c];
    for (int q = 0; q < DD; ++q) F[q] = f.F[q * N + c];
    double lv1[D], lF1[DD];
    for (int b = 0; b < D; ++b) lv1[b] = a.lv1[b * N + c];
    for (int q = 0; q < DD; ++q) lF1[q] = a.lF1[q * N + c];
    const double mu = f.mu[c], kap = kappa_of(prm, mu), dt = f.dt[g.cell_inst ? g.cell_inst[c] : 0];
    const int ord = f.order[c];
    double l0[NX] = {}, l1[NX] = {}, lvs[NX] = {}, lp0[NX] = {}, lp1[NX] = {}, lM[NV * NS] = {}, lR[NX] = {},
           lv[D] = {}, lF[DD] = {}, lmu = 0.0, lkap = 0.0;
    adj::update_vjp<D>(xs0, xs1, vs, vp0, vp1, M, R, v, F, f.m[c], f.im[c], mu, kap, dt, ord, lv1, lF1, 0.0, l0,
                       l1, lvs, lp0, lp1, lM, lR, lv, lF, lmu, lkap);
    for (int k = 0; k < NV; ++k) {
        const int cid = k * N + c;
        for (int s = 0; s < NS; ++s) a.pkM[s * NC + cid] = lM[k * NS + s];
        for (int b = 0; b < D; ++b) {
            a.pkR[b * NC + cid] = lR[k * D + b];
            a.ca[(0 * D + b) * NC + cid] = lvs[k * D + b];
            a.ca[(1 * D + b) * NC + cid] = l0[k * D + b];
            a.ca[(2 * D + b) * NC + cid] = l1[k * D + b];
            a.ca[(3 * D + b) * NC + cid] = lp0[k * D + b];
            a.ca[(4 * D + b) * NC + cid] = lp1[k * D + b];
        }
    }
    for (int b = 0; b < D; ++b) a.lv0[b * N + c] = lv[b];
    for (int q = 0; q < DD; ++q) a.lF0[q * N + c] = lF[q];
    a.lmu[c] += lmu + lkap * kappa_mu_factor<D>(prm);
}

// ---------------------------------------------------------------------------------------
// init_mode: the t^0 nodal solve v_p^0 = v*_p (no motion); lam v*_p = lam v_p^0.
template <int D> __global__ void __launch_bounds__(128) k_adj_nodes(Geo g, Fld f, AdjBuf a, int init_mode) {
    constexpr int NV = adj::Sz<D>::NV;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.Np) return;
    const int N = g.N, Np = g.Np, NC = NV * N;
    double M[D * D] = {}, b[D] = {}, lvs[D] = {}, lx0[D] = {}, lx1[D] = {}, lvp0[D] = {}, lvp1[D] = {};
    const int j0 = g.n2c_off[p], j1 = g.n2c_off[p + 1];
    for (int j = j0; j < j1; ++j) {
        const int cid = g.n2c[j];
        for (int r = 0; r < D; ++r)
            for (int s = 0; s < D; ++s) M[r * D + s] += f.pkM[adj::sym<D>(r, s) * NC + cid];
        for (int r = 0; r < D; ++r) {
            b[r] += f.pkR[r * NC + cid];
            if (!init_mode) {
                lvs[r] += a.ca[(0 * D + r) * NC + cid];
                lx0[r] += a.ca[(1 * D + r) * NC + cid];
                lx1[r] += a.ca[(2 * D + r) * NC + cid];
                lvp0[r] += a.ca[(3 * D + r) * NC + cid];
                lvp1[r] += a.ca[(4 * D + r) * NC + cid];
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
    adj::node_solve_vjp<D>(M, b, g.bc_ndof[p], tv, lvs, lb, lM);
    for (int j = j0; j < j1; ++j) {
        const int cid = g.n2c[j];
        for (int r = 0; r < D; ++r) a.pkR[r * NC + cid] = (init_mode ? 0.0 : a.pkR[r * NC + cid]) + lb[r];
        for (int r = 0; r < D; ++r)
            for (int s = r; s < D; ++s) {
                const double l = r == s ? lM[r * D + r] : lM[r * D + s] + lM[s * D + r];
                const int sx = adj::sym<D>(r, s) * NC + cid;
                a.pkM[sx] = (init_mode ? 0.0 : a.pkM[sx]) + l;
            }
    }
}

// ---------------------------------------------------------------------------------------
// force_p0: the t^0 packets (every cell first order)
#ifndef LMOOD_ADJ_PREDICT_MINB
#define LMOOD_ADJ_PREDICT_MINB 1  // resident blocks of 128 asked of the compiler (2D)
#endif
template <int D>
__global__ void __launch_bounds__(128, D == 2 ? LMOOD_ADJ_PREDICT_MINB : 1) k_adj_predict(Geo g, Fld f, Prm prm, AdjBuf a, int force_p0) {
    using Q = adj::Sz<D>;
    constexpr int NV = Q::NV, DD = Q::DD, NS = Q::NS, NX = NV * D;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    const int N = g.N, Np = g.Np, NC = NV * N;
    double xs[NX], vc[D], Fc[DD], lM[NV * NS], lR[NX];
    adj::Mom<D> mom;
    mom.stride = Np;
    for (int k = 0; k < NV; ++k) {
        const int p = g.c2n[k * N + c];
        mom.p[k] = f.mom + p;
        for (int b = 0; b < D; ++b) {
            xs[k * D + b] = f.x[b * Np + p];
            lR[k * D + b] = a.pkR[b * NC + k * N + c];
        }
        for (int s = 0; s < NS; ++s) lM[k * NS + s] = a.pkM[s * NC + k * N + c];
    }
    for (int b = 0; b < D; ++b) vc[b] = f.v[b * N + c];
    for (int q = 0; q < DD; ++q) Fc[q] = f.F[q * N + c];
    const double mu = f.mu[c], kap = kappa_of(prm, mu), dt = f.dt[g.cell_inst ? g.cell_inst[c] : 0];
    const int ord = force_p0 ? 1 : f.order[c];
    double lxs[NX] = {}, lvc[D] = {}, lF[DD] = {}, lz = 0.0, lmu = 0.0, lkap = 0.0;
    double *cbm = a.cb + (size_t)D * NC + c;  // moment adjoints of corner (k, c): cbm[j NC + k N]
    adj::predict_vjp<D>(xs, mom, vc, Fc, f.z[c], mu, kap, f.im[c], dt, ord, lM, lR, lxs,
                        [&](int k, int j, double v) { cbm[(size_t)j * NC + k * N] = v; }, lvc, lF, lz, lmu, lkap);
    for (int k = 0; k < NV; ++k)
        for (int b = 0; b < D; ++b) a.cb[b * NC + k * N + c] = lxs[k * D + b];
    for (int b = 0; b < D; ++b) a.lv0[b * N + c] += lvc[b];
    for (int q = 0; q < DD; ++q) a.lF0[q * N + c] += lF[q];
    a.lz0[c] = lz;
    a.lmu[c] += lmu + lkap * kappa_mu_factor<D>(prm);
}

// ---------------------------------------------------------------------------------------
template <int D> __global__ void __launch_bounds__(128) k_adj_moments(Geo g, Fld f, AdjBuf a) {
    using Q = adj::Sz<D>;
    constexpr int NV = Q::NV, NQ = Q::NQ, NM = Q::NMOM;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.Np) return;
    const int N = g.N, Np = g.Np, NC = NV * N;
    double lmom[NM] = {}, xp[D], lxp[D] = {};
    const int j0 = g.n2c_off[p], j1 = g.n2c_off[p + 1];
    for (int j = j0; j < j1; ++j) {
        const int cid = g.n2c[j];
        for (int m = 0; m < NM; ++m) lmom[m] += a.cb[(D + m) * NC + cid];
    }
    for (int b = 0; b < D; ++b) xp[b] = f.x[b * Np + p];
    for (int j = j0; j < j1; ++j) {
        const int cid = g.n2c[j];
        const int c = cell_of_corner<D>(cid, N);
        double xc[D], q[NQ], lxc[D] = {}, lq[NQ] = {};
        for (int b = 0; b < D; ++b) xc[b] = f.xc[b * N + c];
        for (int i = 0; i < NQ; ++i) q[i] = i < D ? f.v[i * N + c] : f.F[(i - D) * N + c];
        adj::moments_corner_vjp<D>(lmom, xc, xp, q, lxc, lq, lxp);
        for (int b = 0; b < D; ++b) a.ca[b * NC + cid] = lxc[b];
        for (int i = 0; i < NQ; ++i) a.ca[(D + i) * NC + cid] = lq[i];
    }
    for (int b = 0; b < D; ++b) a.lx0[b * Np + p] += lxp[b];
}

// ---------------------------------------------------------------------------------------
// gather of the moment products at the cell; the centroid x_c = mean of its nodes; the
// impedance z^n = Z(F^n, m / V(x^n), mu) (has_z: z^n was produced by the previous update or
// by the initialisation from F^n and x^n)
template <int D> __global__ void __launch_bounds__(128) k_adj_cells(Geo g, Fld f, Prm prm, AdjBuf a) {
    using Q = adj::Sz<D>;
    constexpr int NV = Q::NV, DD = Q::DD, NQ = Q::NQ, NX = NV * D;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    const int N = g.N, Np = g.Np, NC = NV * N;
    double lxc[D] = {}, xs[NX];
    for (int k = 0; k < NV; ++k) {
        const int cid = k * N + c;
        const int p = g.c2n[k * N + c];
        for (int b = 0; b < D; ++b) {
            lxc[b] += a.ca[b * NC + cid];
            xs[k * D + b] = f.x[b * Np + p];
        }
        for (int i = 0; i < NQ; ++i) {
            const double l = a.ca[(D + i) * NC + cid];
            if (i < D) a.lv0[i * N + c] += l;
            else a.lF0[(i - D) * N + c] += l;
        }
    }
    // z^n
    double F[DD], lF[DD] = {}, lrho = 0.0, lmu = 0.0, lkap = 0.0;
    for (int q = 0; q < DD; ++q) F[q] = f.F[q * N + c];
    double V, Nf[NX];
    adj::faces<D>(xs, V, Nf);
    const double mu = f.mu[c], kap = kappa_of(prm, mu);
    adj::impedance_vjp<D>(F, f.m[c] / V, mu, kap, a.lz0[c], lF, lrho, lmu, lkap);
    for (int q = 0; q < DD; ++q) a.lF0[q * N + c] += lF[q];
    a.lmu[c] += lmu + lkap * kappa_mu_factor<D>(prm);
    const double lV = lrho * (-f.m[c] / (V * V));
    double lxs[NX] = {}, lN0[NX] = {};
    adj::faces_vjp<D>(xs, lV, lN0, lxs);
    for (int k = 0; k < NV; ++k)
        for (int b = 0; b < D; ++b) a.cd[b * NC + k * N + c] = lxs[k * D + b] + lxc[b] / NV;
}

template <int D> __global__ void __launch_bounds__(128) k_adj_gather(Geo g, AdjBuf a) {
    constexpr int NV = D + 1;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.Np) return;
    const int NC = NV * g.N, Np = g.Np;
    double l[D] = {};
    for (int j = g.n2c_off[p]; j < g.n2c_off[p + 1]; ++j) {
        const int cid = g.n2c[j];
        for (int b = 0; b < D; ++b) l[b] += a.cb[b * NC + cid] + a.cd[b * NC + cid];
    }
    for (int b = 0; b < D; ++b) a.lx0[b * Np + p] += l[b];
}

// impedance of the initial state only (the t^0 packets' z): lmu from lz0
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
    adj::impedance_vjp<D>(F, f.m[c] / V, mu, kap, a.lz0[c], lF, lrho, lmu, lkap);
    for (int q = 0; q < DD; ++q) a.lF0[q * N + c] += lF[q];
    a.lmu[c] += lmu + lkap * kappa_mu_factor<D>(prm);
}

}  // namespace lmood
