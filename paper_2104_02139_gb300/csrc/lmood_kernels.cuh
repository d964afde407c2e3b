// lmood_kernels.cuh -- the kernels of one explicit Lagrangian ADER-MOOD step, templated
// on the space dimension. Included by one translation unit per dimension.
//
// Per step (all cells / all nodes, then MOOD rounds over compacted lists):
//   k_moments  nodes : moments of the cells around each node (the least-squares sums)
//   k_predict  cells : geometry at x^n, least-squares slopes of v and F, ADER predictor,
//                      corner packets (M_cp, rhs_cp)
//   k_nodes    nodes : ordered gather of the packets around the node, Eucclhyd solve with
//                      boundary conditions, node motion
//   k_update   cells : subcell forces, update of v, e, tau, F, detection, dt candidate
//   k_mark_*         : troubled cells -> their nodes -> the cells around those nodes
//   k_finalize       : next dt (exact min over cells) and the per-step counters
// The whole-mesh node kernels take the nodes of each window of 256 in order of their cell
// count (Geo::node_perm), so that the lanes of a warp run loops of one length.
#pragma once
#include "lmood_dev.cuh"

namespace lmood {

constexpr int kCellBlock = 128;
constexpr int kNodeBlock = 256;

// list launches use at most this many blocks and loop over the device-counted list
constexpr int kListBlocks = 152 * 8;

// ---------------------------------------------------------------------------------------
// k_predict: corner packets of a cell (Sect. "Space-Time discretization --- ADER
// methodology", Eqs. Mcp^n, nodal_solver^n, subforce^n).
//   P1: v and F reconstructed by least squares (sums from the node moments), then the predictor
//       v*_cp = v_h(x_p) + dt/2 (1/m_c) sum_q T(F_h(x_q)) ln_q,  F*_cp = F_h(x_p) + dt/2 L^ F_c
//   P0: v*_cp = v_c, F*_cp = F_c.
//   M_cp = z_c sum_{f containing p} |ln_f| n_f (x) n_f, rhs_cp = M_cp v*_cp - T(F*_cp) ln_p.
// With a list, only the listed cells (troubled ones, already marked P0) are recomputed.
// (predict_cell and k_predict follow the node moments they read.)
// ---------------------------------------------------------------------------------------
// ---------------------------------------------------------------------------------------
// k_moments: per node p, moments of the cells c' around it (positions relative to x_p):
//   n_p, S1 = sum dx, S2 = sum dx dx^t, U = sum q, T = sum dx (x) q,  dx = x_c' - x_p,
// q = (v, F). A cell's least-squares sums over the (node, neighbour) pairs follow from the
// moments of its D+1 nodes (reading of Sect. "Algorithm": stencil = cells sharing a node,
// each neighbour weighted by the number of nodes it shares with the cell).
// ---------------------------------------------------------------------------------------
// B: threads per block (a launch-shape variant chosen by the autotuner; same arithmetic)
template <int D> __device__ __forceinline__ void moments_node(const Geo &g, const Fld &f, int p) {
    using Q = Dim<D>;
    constexpr int NS = Q::NS, NQ = Q::NQ, DD = D * D;
    const int N = g.N, Np = g.Np;
    double xp[D], S1[D], S2[NS], U[NQ], T[NQ][D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        xp[a] = f.x[a * Np + p];
        S1[a] = 0.0;
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) S2[s] = 0.0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        U[q] = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) T[q][a] = 0.0;
    }
    const int j1 = __ldg(g.n2c_off + p + 1);
    for (int j = __ldg(g.n2c_off + p); j < j1; ++j) {
        int c = __ldg(g.n2c + j);  // corner id k N + c -> cell c (k <= D)
#pragma unroll
        for (int k = 0; k < D; ++k) c -= c >= N ? N : 0;
        double dx[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            dx[a] = f.xc[a * N + c] - xp[a];
            S1[a] += dx[a];
        }
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = a; b < D; ++b) S2[sidx<D>(a, b)] = fma(dx[a], dx[b], S2[sidx<D>(a, b)]);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const double qv = q < D ? f.v[q * N + c] : f.F[(q - D) * N + c];
            U[q] += qv;
#pragma unroll
            for (int a = 0; a < D; ++a) T[q][a] = fma(dx[a], qv, T[q][a]);
        }
    }
    (void)DD;
    double *m = f.mom + p;
    m[Q::M_N * Np] = (double)(j1 - __ldg(g.n2c_off + p));  // the node's cell count
#pragma unroll
    for (int a = 0; a < D; ++a) m[(Q::M_S1 + a) * Np] = S1[a];
#pragma unroll
    for (int s = 0; s < NS; ++s) m[(Q::M_S2 + s) * Np] = S2[s];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        m[(Q::M_U + q) * Np] = U[q];
#pragma unroll
        for (int a = 0; a < D; ++a) m[(Q::M_T + q * D + a) * Np] = T[q][a];
    }
}

template <int D, int B = kNodeBlock> __global__ void __launch_bounds__(B) k_moments(Geo g, Fld f) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < g.Np) moments_node<D>(g, f, g.node_perm[t]);
}

// MAT: 0 neo-Hookean, 1 another shear energy of the family, 2 stiffened gas (separate
// instances, so the neo-Hookean kernels are compiled as if the other materials did not exist)
template <int D, int MAT>
__device__ __forceinline__ void cell_stress(const Prm &prm, const double (&F)[D * D], double mu, double kappa,
                                            double eps, double (&T)[D * D]) {
    if constexpr (MAT == 2) stress_sg<D>(prm, F, mu, eps, T);
    else if constexpr (MAT == 1) stress_family<D>(F, mu, kappa, prm.shear_a, T);
    else stress<D>(F, mu, kappa, T);
}

template <int D, bool LISTED, int MAT = 0>
__device__ __forceinline__ void predict_cell(const Geo &g, const Fld &f, const Prm &prm, int c) {
    constexpr int NV = D + 1, DD = D * D, NS = D * (D + 1) / 2, NQ = D + DD;
    const int N = g.N, Np = g.Np, NC = NV * N;
    int ord;
    if constexpr (LISTED) {
        ord = f.order[c];
    } else if (prm.base_order == 0) {
        ord = f.order[c];  // replay of a recorded step: the cells' orders are given
    } else {
        ord = prm.base_order;
        f.order[c] = (unsigned char)ord;
    }
    int nod[NV];
    double xs[NV][D];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        nod[k] = __ldg(g.c2n + k * N + c);
#pragma unroll
        for (int a = 0; a < D; ++a) xs[k][a] = f.x[a * Np + nod[k]];
    }
    // the geometry at x^n, as the previous step's update (or init / refresh) left it
    double V, Nf[NV][D];
    load_cell_geo<D>(f.gf, N, c, Nf, V);
    double vc[D], Fc[DD];
#pragma unroll
    for (int a = 0; a < D; ++a) vc[a] = f.v[a * N + c];
#pragma unroll
    for (int q = 0; q < DD; ++q) Fc[q] = f.F[q * N + c];
    const double muc = f.mu[c], kap = kappa_of(prm, muc);
    double eps_c = 0.0;  // specific internal energy (the stiffened gas's pressure depends on it)
    if constexpr (MAT == 2) {
        eps_c = f.e[c];
#pragma unroll
        for (int a = 0; a < D; ++a) eps_c -= 0.5 * vc[a] * vc[a];
    }
    // face matrices W_f = z |l n_f| n_f (x) n_f with l n_f = N_f / D; M_cp = sum_{f != p} W_f
    // (filled just before the packets are emitted, so that they are not live through the
    // reconstruction and the predictor)
    double W[NV][NS];
    auto face_matrices = [&]() {
        const double z = f.z[c];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            // with u = N_f / D: z / |u| u u^t = (z / (D |N_f|)) N_f N_f^t
            const double w = z * f.gf[(CellGeo<D>::RS + k) * N + c] * (1.0 / D);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const double wa = w * Nf[k][a];
#pragma unroll
                for (int b = a; b < D; ++b) W[k][sidx<D>(a, b)] = wa * Nf[k][b];
            }
        }
    };
    // T* N_k, the stress part of corner k's packet
    auto stress_normal = [&](int k, const double(&Tst)[DD], double(&tn)[D]) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
            double s = 0.0;
#pragma unroll
            for (int b = 0; b < D; ++b) s += Tst[a * D + b] * Nf[k][b];
            tn[a] = s;
        }
    };
    // packet of corner k: M_cp and rhs_cp = M_cp v* - T* l n_p, with l n_p = -N_p / D
    auto emit = [&](int k, const double(&vst)[D], const double(&tn)[D]) {
        double M[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            double acc = 0.0;
#pragma unroll
            for (int fq = 0; fq < NV; ++fq)
                if (fq != k) acc += W[fq][s];
            M[s] = acc;
            f.pkM[s * NC + k * N + c] = acc;
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
            double mv = 0.0;
#pragma unroll
            for (int b = 0; b < D; ++b) mv += M[sidx<D>(a, b)] * vst[b];
            f.pkR[a * NC + k * N + c] = fma(tn[a], 1.0 / D, mv);
        }
    };
    if (ord != 1) {
        // least-squares sums over the (node, neighbour) pairs from the node moments:
        // with d = x_p - x_c, dx' = (x_c' - x_p) + d, so
        //   G += S2 + S1 d^t + d S1^t + n d d^t,   r_q += T_q + d U_q - (S1 + n d) q_c
        // (the cell itself is one of the node's cells and contributes zero); the q_c terms of
        // the D+1 nodes are gathered into one: r_q = sum_p (T_q + d U_q) - (sum_p w) q_c
        using Q = Dim<D>;
        double xcc[D];
#pragma unroll
        for (int a = 0; a < D; ++a) xcc[a] = f.xc[a * N + c];
        double G[NS], r[NQ][D], wsum[D], npair = -NV;  // (node, other cell) pairs of the stencil
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const double *m = f.mom + nod[k];
            double d[D], S1[D], w[D];
            const double nn = m[Q::M_N * Np];
            npair += nn;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                d[a] = xs[k][a] - xcc[a];
                S1[a] = m[(Q::M_S1 + a) * Np];
                w[a] = fma(nn, d[a], S1[a]);
                wsum[a] = k == 0 ? w[a] : wsum[a] + w[a];
            }
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int b = a; b < D; ++b) {
                    const int sb = sidx<D>(a, b);
                    const double s2 = m[(Q::M_S2 + sb) * Np];
                    G[sb] = fma(S1[a], d[b], fma(d[a], w[b], k == 0 ? s2 : G[sb] + s2));
                }
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const double uq = m[(Q::M_U + q) * Np];
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    const double tq = m[(Q::M_T + q * D + a) * Np];
                    r[q][a] = k == 0 ? fma(d[a], uq, tq) : fma(d[a], uq, r[q][a] + tq);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const double qc = q < D ? vc[q] : Fc[q - D];
#pragma unroll
            for (int a = 0; a < D; ++a) r[q][a] = fma(-wsum[a], qc, r[q][a]);
        }
        double Gf[DD], Gi[DD];
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = 0; b < D; ++b) Gf[a * D + b] = G[sidx<D>(a, b)];
        double tr = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) tr += Gf[a * D + a];
        const double t = tr * (1.0 / D);
        // an empty stencil gives G = 0 up to the rounding of the moment sums: no slopes
        const bool ok = npair > 0.0 && det<D>(Gf) > 1e-12 * (D == 2 ? t * t : t * t * t);
        inverse<D>(Gf, Gi);
        double dxs[NV][D];
#pragma unroll
        for (int k = 0; k < NV; ++k)
#pragma unroll
            for (int a = 0; a < D; ++a) dxs[k][a] = xs[k][a] - xcc[a];
        // The reconstruction at corner k is q_c + g_q . dx_k with the slopes g_q = G^-1 r_q.
        // The whole-mesh launch evaluates it as q_c + r_q . y_k with y_k = G^-1 dx_k (the same
        // value; D^2 products per corner instead of D^2 per field), and forms the slopes of v
        // alone (for dF/dt); a listed cell may limit its slopes (Barth-Jespersen), so there the
        // slopes are formed and y_k = dx_k. rr holds r_q or g_q accordingly.
        double rr[NQ][D], yk[NV][D], gv[DD];
        if (!LISTED) {
#pragma unroll
            for (int k = 0; k < NV; ++k)
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    double s = 0.0;
#pragma unroll
                    for (int b = 0; b < D; ++b) s += Gi[a * D + b] * dxs[k][b];
                    yk[k][a] = ok ? s : 0.0;
                }
#pragma unroll
            for (int q = 0; q < NQ; ++q)
#pragma unroll
                for (int a = 0; a < D; ++a) rr[q][a] = r[q][a];
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    double s = 0.0;
#pragma unroll
                    for (int b = 0; b < D; ++b) s += Gi[a * D + b] * r[i][b];
                    gv[i * D + a] = ok ? s : 0.0;
                }
        } else {
#pragma unroll
            for (int q = 0; q < NQ; ++q)
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    double s = 0.0;
#pragma unroll
                    for (int b = 0; b < D; ++b) s += Gi[a * D + b] * r[q][b];
                    rr[q][a] = ok ? s : 0.0;
                }
            // cells reach level 3 only through a MOOD decrement, i.e. in list launches
            if (ord == 3) {
                // Barth-Jespersen: scale each field's slope by the largest phi <= 1 that keeps
                // its values at the cell's nodes within its range over the stencil and the cell
                double lo[NQ], hi[NQ];
#pragma unroll
                for (int q = 0; q < NQ; ++q) lo[q] = hi[q] = q < D ? vc[q] : Fc[q - D];
                for (int k = 0; k < NV; ++k) {
                    const int j1 = __ldg(g.n2c_off + nod[k] + 1);
                    for (int j = __ldg(g.n2c_off + nod[k]); j < j1; ++j) {
                        int o = __ldg(g.n2c + j);
#pragma unroll
                        for (int kk = 0; kk < D; ++kk) o -= o >= N ? N : 0;
#pragma unroll
                        for (int q = 0; q < NQ; ++q) {
                            const double qo = q < D ? f.v[q * N + o] : f.F[(q - D) * N + o];
                            lo[q] = fmin(lo[q], qo);
                            hi[q] = fmax(hi[q], qo);
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const double qc = q < D ? vc[q] : Fc[q - D];
                    double phi = 1.0;
#pragma unroll
                    for (int k = 0; k < NV; ++k) {
                        double delta = 0.0;
#pragma unroll
                        for (int a = 0; a < D; ++a) delta += rr[q][a] * dxs[k][a];
                        if (delta > 0.0) phi = fmin(phi, (hi[q] - qc) / delta);
                        if (delta < 0.0) phi = fmin(phi, (lo[q] - qc) / delta);
                    }
#pragma unroll
                    for (int a = 0; a < D; ++a) rr[q][a] *= phi;
                }
            }
#pragma unroll
            for (int k = 0; k < NV; ++k)
#pragma unroll
                for (int a = 0; a < D; ++a) yk[k][a] = dxs[k][a];
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int a = 0; a < D; ++a) gv[i * D + a] = rr[i][a];
        }
        // half step of F: dt/2 dF/dt with dF/dt = L^ F_c (Eq. GCLL)
        const double dt = f.dt[g.cell_inst ? __ldg(g.cell_inst + c) : 0];
        double dFdt[DD];
        matmul<D>(gv, Fc, dFdt);
        // stiffened gas: the internal energy at the half step, d eps/dt = T_c : L^ / rho
        double eps_h = eps_c;
        if constexpr (MAT == 2) {
            double Tc[DD], pw = 0.0;
            cell_stress<D, MAT>(prm, Fc, muc, kap, eps_c, Tc);
#pragma unroll
            for (int q = 0; q < DD; ++q) pw += Tc[q] * gv[q];
            eps_h = eps_c + 0.5 * dt * pw * V / f.m[c];
        }
        // per corner k, from the reconstructed value F_h(x_k): the stress T(F_h) of
        // dv/dt = (1/m) sum_q T(F_h(x_q)) l n_q, and the stress T* = T(F_h + dt/2 dF/dt) at
        // t^{n+1/2}, of which the packet needs T* N_k (F_h is formed once per corner)
        double dvdt[D], tn[NV][D];
#pragma unroll
        for (int a = 0; a < D; ++a) dvdt[a] = 0.0;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double Fh[DD], Fs[DD], T[DD];
#pragma unroll
            for (int q = 0; q < DD; ++q) {
                double s = Fc[q];
#pragma unroll
                for (int a = 0; a < D; ++a) s += rr[D + q][a] * yk[k][a];
                Fh[q] = s;
                Fs[q] = fma(0.5 * dt, dFdt[q], s);
            }
            cell_stress<D, MAT>(prm, Fh, muc, kap, eps_c, T);
#pragma unroll
            for (int i = 0; i < D; ++i) {
#pragma unroll
                for (int b = 0; b < D; ++b) dvdt[i] = fma(T[i * D + b], Nf[k][b], dvdt[i]);
            }
            cell_stress<D, MAT>(prm, Fs, muc, kap, eps_h, T);
            stress_normal(k, T, tn[k]);
        }
        // half step of v: dt/2 dv/dt, added to the cell value once
        const double hv = -0.5 * dt * f.im[c] * (1.0 / D);
        if (f.dvs) {  // the sum itself (its scaling by hv stays fused into v_c + dv below)
#pragma unroll
            for (int a = 0; a < D; ++a) f.dvs[a * N + c] = dvdt[a];
        }
#pragma unroll
        for (int a = 0; a < D; ++a) dvdt[a] *= hv;
        face_matrices();
        double vch[D];
#pragma unroll
        for (int i = 0; i < D; ++i) vch[i] = vc[i] + dvdt[i];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double vst[D];
#pragma unroll
            for (int i = 0; i < D; ++i) {
                double s = vch[i];
#pragma unroll
                for (int a = 0; a < D; ++a) s += rr[i][a] * yk[k][a];
                vst[i] = s;
            }
            emit(k, vst, tn[k]);
        }
    } else {
        double T[DD];
        cell_stress<D, MAT>(prm, Fc, muc, kap, eps_c, T);
        face_matrices();
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double tn[D];
            stress_normal(k, T, tn);
            emit(k, vc, tn);
        }
    }
}

// LISTED = false: one thread per cell of the whole mesh; true: a grid-stride loop over a
// device-counted list (separate instances, so each gets its own register allocation)
// (the 2D bound keeps the register cap at 128 per thread for every block size B)
template <int D, bool LISTED, int B = kCellBlock, int MAT = 0>
__global__ void __launch_bounds__(B, D == 2 ? 512 / B : 1) k_predict(Geo g, Fld f, Prm prm, const int *__restrict__ list,
                                                        const int *__restrict__ cnt, int n) {
    if constexpr (!LISTED) {
        const int c = blockIdx.x * blockDim.x + threadIdx.x;
        if (c < n) predict_cell<D, false, MAT>(g, f, prm, c);
    } else {
        const int nn = *cnt;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x)
            predict_cell<D, true, MAT>(g, f, prm, list[i]);
    }
}

// ---------------------------------------------------------------------------------------
// k_nodes: Eucclhyd nodal solver (Eqs. nodal_solver^n, Mcp^n) with the BCs of Appendix B:
// M_p = sum_c M_cp, b_p = sum_c rhs_cp in ascending cell id (plus the forces of traction and
// pressure faces, Eq. pBC), v*_p the Galerkin solution of M_p v = b_p on the node's free
// directions (Eq. sBC1), corrected along d_p to meet a prescribed normal velocity (Eqs. vBC1,
// vBC); then x^{n+1} = x^n + dt v*_p and v_p^{n+1} = 2 v*_p - v_p^n. init_mode stores v*_p as
// v_p^0 and moves nothing.
// ---------------------------------------------------------------------------------------
// Galerkin solve of M v = rhs on the node's free subspace (Eq. sBC1): nd = D free, 0 clamped,
// else the span of the node's nd tangent vectors
// the Galerkin solve on the node's ND free directions t_i (ND a compile-time count, so that the
// small arrays stay in registers)
template <int D, int ND>
__device__ __forceinline__ void solve_K_proj(const Geo &g, const double (&M)[D * D], int p, const double (&rhs)[D],
                                             double (&v)[D]) {
    const int Np = g.Np;
    double t[ND][D], A[ND * ND], r[ND], al[ND];
#pragma unroll
    for (int i = 0; i < ND; ++i)
#pragma unroll
        for (int a = 0; a < D; ++a) t[i][a] = g.bc_t[(i * 3 + a) * Np + p];
#pragma unroll
    for (int i = 0; i < ND; ++i) {
        double s = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) s += t[i][a] * rhs[a];
        r[i] = s;
#pragma unroll
        for (int j = 0; j < ND; ++j) {
            double q = 0.0;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                double mt = 0.0;
#pragma unroll
                for (int c = 0; c < D; ++c) mt += M[a * D + c] * t[j][c];
                q += t[i][a] * mt;
            }
            A[i * ND + j] = q;
        }
    }
    if constexpr (ND == 1) {
        al[0] = r[0] / A[0];
    } else {
        const double dA = A[0] * A[3] - A[1] * A[2];
        const double idA = 1.0 / dA;
        al[0] = (A[3] * idA) * r[0] + (-A[1] * idA) * r[1];
        al[1] = (-A[2] * idA) * r[0] + (A[0] * idA) * r[1];
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < ND; ++i) s += al[i] * t[i][a];
        v[a] = s;
    }
}

template <int D>
__device__ __forceinline__ void solve_K(const Geo &g, const double (&M)[D * D], int nd, int p, const double (&rhs)[D],
                                        double (&v)[D]) {
    constexpr int DD = D * D;
    const int Np = g.Np;
    if (nd == D) {
        double Mi[DD];
        inverse<D>(M, Mi);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            double s = 0.0;
#pragma unroll
            for (int c = 0; c < D; ++c) s += Mi[a * D + c] * rhs[c];
            v[a] = s;
        }
    } else if (nd == 0) {
#pragma unroll
        for (int a = 0; a < D; ++a) v[a] = 0.0;
    } else if (nd == 1) {
        solve_K_proj<D, 1>(g, M, p, rhs, v);
    } else {
        solve_K_proj<D, 2>(g, M, p, rhs, v);
    }
}

// outward area vector of boundary face fid at positions x: 2D edge (q0, q1): (y1 - y0,
// x0 - x1); 3D triangle: (1/2) (x1 - x0) x (x2 - x0)
template <int D>
__device__ __forceinline__ void face_area_vector(const Geo &g, const double *x, int fid, double (&N)[D]) {
    const int Np = g.Np, nb = g.nbf;
    if constexpr (D == 2) {
        const int q0 = g.bf_nodes[fid], q1 = g.bf_nodes[nb + fid];
        N[0] = x[Np + q1] - x[Np + q0];
        N[1] = x[q0] - x[q1];
    } else {
        const int q0 = g.bf_nodes[fid], q1 = g.bf_nodes[nb + fid], q2 = g.bf_nodes[2 * nb + fid];
        double u[3], w[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            u[a] = x[a * Np + q1] - x[a * Np + q0];
            w[a] = x[a * Np + q2] - x[a * Np + q0];
        }
        N[0] = 0.5 * (u[1] * w[2] - u[2] * w[1]);
        N[1] = 0.5 * (u[2] * w[0] - u[0] * w[2]);
        N[2] = 0.5 * (u[0] * w[1] - u[1] * w[0]);
    }
}

template <int D>
__device__ __forceinline__ void node_solve(const Geo &g, const Fld &f, int p, int init_mode) {
    constexpr int NV = D + 1, NS = D * (D + 1) / 2, DD = D * D;
    const int Np = g.Np, NC = NV * g.N;
    double Ms[NS], b[D];
#pragma unroll
    for (int s = 0; s < NS; ++s) Ms[s] = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) b[a] = 0.0;
    // also the range of rho^n over the cells around the node (RDMP bounds, Eq. RDMP: the
    // union over a cell's nodes is its stencil plus the cell itself)
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    long long klo = order_key(inf), khi = order_key(-inf);
    const int j1 = __ldg(g.n2c_off + p + 1);
    for (int j = __ldg(g.n2c_off + p); j < j1; ++j) {
        const int cid = __ldg(g.n2c + j);
#pragma unroll
        for (int s = 0; s < NS; ++s) Ms[s] += f.pkM[s * NC + cid];
#pragma unroll
        for (int a = 0; a < D; ++a) b[a] += f.pkR[a * NC + cid];
        int cc = cid;  // corner id k N + c -> cell c (k < 4)
        cc -= cc >= g.N ? g.N : 0;
        cc -= cc >= g.N ? g.N : 0;
        cc -= cc >= g.N ? g.N : 0;
        const long long kr = order_key(f.rho[cc]);
        klo = min(klo, kr);
        khi = max(khi, kr);
    }
    f.rlo[p] = key_value(klo);
    f.rhi[p] = key_value(khi);
    double M[DD];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int c = 0; c < D; ++c) M[a * D + c] = Ms[sidx<D>(a, c)];
    const int ndf = g.bc_ndof[p];
    const int nd = ndf & BC_NDOF;
    double v[D];
    if (!(ndf & BC_EXT)) {
        solve_K<D>(g, M, nd, p, b, v);
    } else {
        // traction, pressure and prescribed-velocity faces around the node (Eqs. pBC, vBC1,
        // vBC): N_f = outward area vector at x^n, the node's share N_f / D
        double dv[D], gsum = 0.0;
        int nvel = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) dv[a] = 0.0;
        for (int j = g.nbf_off[p]; j < g.nbf_off[p + 1]; ++j) {
            const int fid = g.nbf_idx[j];
            const int tag = g.bf_tag[fid];
            if (tag < TAG_TRACTION) continue;
            double N[D];
            face_area_vector<D>(g, f.x, fid, N);
            if (tag == TAG_TRACTION) {
                double ar = 0.0;
#pragma unroll
                for (int a = 0; a < D; ++a) ar += N[a] * N[a];
                ar = sqrt(ar) * (1.0 / D);
#pragma unroll
                for (int a = 0; a < D; ++a) b[a] += ar * g.bf_val[a * g.nbf + fid];
            } else if (tag == TAG_PRESSURE) {
                const double pr = g.bf_val[fid];
#pragma unroll
                for (int a = 0; a < D; ++a) b[a] -= pr * N[a] * (1.0 / D);
            } else if (tag == TAG_VELOCITY) {
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    dv[a] += N[a] * (1.0 / D);
                    gsum += g.bf_val[a * g.nbf + fid] * N[a] * (1.0 / D);
                }
                ++nvel;
            }
        }
        solve_K<D>(g, M, nd, p, b, v);
        if (nvel > 0) {  // v = K b - T K d with v . d = g
            double w[D], wd = 0.0, vd = 0.0;
            solve_K<D>(g, M, nd, p, dv, w);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                wd += w[a] * dv[a];
                vd += v[a] * dv[a];
            }
            if (wd > 0.0) {
                const double T = (vd - gsum) / wd;
#pragma unroll
                for (int a = 0; a < D; ++a) v[a] -= T * w[a];
            }
        }
    }
    if (ndf & BC_CONTACT) {
        // contact walls (Sect. "Boundary condition treatments"): within the distance threshold
        // of a wall and moving into it, the node gets v . n = 0 (the multiplier above, g = 0)
        const int nw = (int)g.contact[0];
        const double eps = g.contact[1];
        for (int k = 0; k < nw; ++k) {
            const double *P = g.contact + 2 + 2 * D * k, *nrm = P + D;
            double dist = 0.0, vn = 0.0, n[D];
#pragma unroll
            for (int a = 0; a < D; ++a) {
                n[a] = nrm[a];
                dist += n[a] * (f.x[a * Np + p] - P[a]);
                vn += n[a] * v[a];
            }
            if (!(dist < eps && vn < 0.0)) continue;
            double w[D], wn = 0.0;
            solve_K<D>(g, M, nd, p, n, w);
#pragma unroll
            for (int a = 0; a < D; ++a) wn += w[a] * n[a];
            if (wn > 0.0) {
                const double T = vn / wn;
#pragma unroll
                for (int a = 0; a < D; ++a) v[a] -= T * w[a];
            }
        }
    }
#pragma unroll
    for (int a = 0; a < D; ++a) f.vs[a * Np + p] = v[a];
    if (init_mode) {
#pragma unroll
        for (int a = 0; a < D; ++a) f.vp[a * Np + p] = v[a];
        return;
    }
    const double dt = f.dt[g.node_inst ? __ldg(g.node_inst + p) : 0];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        f.x1[a * Np + p] = f.x[a * Np + p] + dt * v[a];
        f.vp1[a * Np + p] = 2.0 * v[a] - f.vp[a * Np + p];
    }
}

template <int D, bool LISTED, int B = kNodeBlock>
__global__ void __launch_bounds__(B) k_nodes(Geo g, Fld f, const int *__restrict__ list,
                                                      const int *__restrict__ cnt, int n, int init_mode) {
    if constexpr (!LISTED) {  // every node (n = Np); in 3D in order of their cell count
        const int t = blockIdx.x * blockDim.x + threadIdx.x;
        if (t < n) node_solve<D>(g, f, kNodesByCount<D> ? g.node_perm[t] : t, init_mode);
    } else {
        const int nn = *cnt;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x)
            node_solve<D>(g, f, list[i], init_mode);
    }
}

// velocity gradient L_ij = (1/|w_c|) sum_p v_{p,i} ln_{p,j} (Eq. div_grad_v, read so that
// dF/dt = L F), with ln_p = -N_p / D: L = -(1 / (D |w_c|)) sum_p v_p (x) N_p
template <int D>
__device__ __forceinline__ void vel_gradient(const double (&vn)[D + 1][D], const double (&Nf)[D + 1][D], double iV,
                                             double (&L)[D * D]) {
    const double s0 = iV * (-1.0 / D);  // iV = 1 / |w_c|
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < D + 1; ++k) s += vn[k][i] * Nf[k][j];
            L[i * D + j] = s * s0;
        }
}

// ---------------------------------------------------------------------------------------
// k_update: subcell forces f_cp = M_cp v*_p - rhs_cp and the cell update (Eqs. tau_c^n,
// v_c^n, e_c^n, firstB, CN_B): tau^{n+1} = |w_c(x^{n+1})| / m_c; F by Crank-Nicolson (P1)
// or explicit Euler (P0). Then detection (Eqs. PAD, RDMP), the dt candidate (Eq. CFL2) and
// the impedance of the candidate (used by the next step's packets). P1 cells that fail are
// appended to tlist.
// ---------------------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void update_cell(const Geo &g, const Fld &f, const Prm &prm, int c, int *tlist, int *tcnt) {
    constexpr int NV = D + 1, DD = D * D, NS = D * (D + 1) / 2;
    const int N = g.N, Np = g.Np, NC = NV * N;
    const int ord = f.order[c];
    const double dt = f.dt[g.cell_inst ? __ldg(g.cell_inst + c) : 0];
    int nod[NV];
    double xs1[NV][D], vsn[NV][D];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        nod[k] = __ldg(g.c2n + k * N + c);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            xs1[k][a] = f.x1[a * Np + nod[k]];
            vsn[k][a] = f.vs[a * Np + nod[k]];
        }
    }
    double sf[D], sfv = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) sf[a] = 0.0;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double M[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) M[s] = f.pkM[s * NC + k * N + c];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            double fa = -f.pkR[a * NC + k * N + c];  // f_cp = M_cp v*_p - rhs_cp
#pragma unroll
            for (int b = 0; b < D; ++b) fa = fma(M[sidx<D>(a, b)], vsn[k][b], fa);
            sf[a] += fa;
            sfv = fma(fa, vsn[k][a], sfv);
        }
    }
    const double mc = f.m[c], im = f.im[c], muc = f.mu[c], kap = kappa_of(prm, muc);
    const double dtm = dt * im;
    double v1[D];
#pragma unroll
    for (int a = 0; a < D; ++a) v1[a] = fma(dtm, sf[a], f.v[a * N + c]);
    const double e1 = fma(dtm, sfv, f.e[c]);
    // the geometry at x^n as the previous step left it; that of x^{n+1} computed and kept for
    // the next step
    const double V0 = f.gf[CellGeo<D>::VOL * N + c];
    double V1, Nf1[NV][D], rs1[NV], ss1[NV];
    simplex_faces<D>(xs1, V1, Nf1);
    face_rnorms<D>(Nf1, rs1, ss1);
    store_cell_geo<D>(f.gf1, N, c, Nf1, V1, rs1);
    const double iV1 = 1.0 / V1;
    double Fn[DD], F1[DD];
#pragma unroll
    for (int q = 0; q < DD; ++q) Fn[q] = f.F[q * N + c];
    // the velocity gradient of v_p^{n+1} at x^{n+1}: this step's L^{n+1}, kept as the next
    // step's L^n
    double L1[DD];
    {
        double vn[NV][D];
#pragma unroll
        for (int k = 0; k < NV; ++k)
#pragma unroll
            for (int a = 0; a < D; ++a) vn[k][a] = f.vp1[a * Np + nod[k]];
        vel_gradient<D>(vn, Nf1, iV1, L1);
        store_cell_grad<D>(f.gf1, N, c, L1);
    }
    if (ord != 1) {
        double L0[DD], A[DD], Bm[DD], Ai[DD], R[DD];
        load_cell_grad<D>(f.gf, N, c, L0);  // L^n, as the previous update (or a refresh) left it
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const double id = i == j ? 1.0 : 0.0;
                A[i * D + j] = fma(-0.5 * dt, L1[i * D + j], id);
                Bm[i * D + j] = fma(0.5 * dt, L0[i * D + j], id);
            }
        matmul<D>(Bm, Fn, R);
        inverse<D>(A, Ai);
        matmul<D>(Ai, R, F1);
    } else {
        // 1 / |w_c| at x^n is rho^n / m_c (rho^n = m_c / |w_c(x^n)| is stored)
        double Nf0[NV][D], V0g, Ls[DD], LF[DD];
        load_cell_geo<D>(f.gf, N, c, Nf0, V0g);
        vel_gradient<D>(vsn, Nf0, f.rho[c] * im, Ls);
        matmul<D>(Ls, Fn, LF);
#pragma unroll
        for (int q = 0; q < DD; ++q) F1[q] = fma(dt, LF[q], Fn[q]);
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
        f.v1[a * N + c] = v1[a];
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < NV; ++k) s += xs1[k][a];
        f.xc1[a * N + c] = s * (1.0 / NV);
    }
    f.e1[c] = e1;
#pragma unroll
    for (int q = 0; q < DD; ++q) f.F1[q * N + c] = F1[q];
    const double rho1 = mc * iV1;
    f.rho1[c] = rho1;
    f.tau1[c] = V1 * im;
    double area1 = 0.0;  // sum of the face measures at x^{n+1} (in-sphere diameter 2 D V / area)
#pragma unroll
    for (int k = 0; k < NV; ++k) area1 += ss1[k] * rs1[k];  // |N_f| = |N_f|^2 / |N_f|
    if (prm.mood) {
        int ps = pad_state<D>(v1, e1, F1, V1, a0sq_of(prm, muc, kap));
        if (prm.eos && ps == 0) {  // stiffened gas: p + p_inf > 0 (a real sound speed)
            double eps1 = e1, Fg[DD];
#pragma unroll
            for (int a = 0; a < D; ++a) eps1 -= 0.5 * v1[a] * v1[a];
            // a copy: the shear energy of the family takes its argument's address, which would
            // put F1 in local memory on every path
#pragma unroll
            for (int q = 0; q < DD; ++q) Fg[q] = F1[q];
            if (!(sg_pressure<D>(prm, Fg, muc, eps1) + prm.pinf > 0.0)) ps = 1;
        }
        if (ord != 1) {
            bool bad = ps != 0;
            if (!bad) {
                long long klo = order_key(f.rlo[nod[0]]), khi = order_key(f.rhi[nod[0]]);
#pragma unroll
                for (int k = 1; k < NV; ++k) {
                    klo = min(klo, order_key(f.rlo[nod[k]]));
                    khi = max(khi, order_key(f.rhi[nod[k]]));
                }
                const double lo = key_value(klo), hi = key_value(khi);
                const long long kd = max(order_key(prm.delta0), order_key(prm.delta1 * (hi - lo)));
                const double delta = key_value(kd);
                const long long kr = order_key(rho1);  // finite: PAD passed
                bad = !(kr >= order_key(lo - delta) && kr <= order_key(hi + delta));
            }
            if (bad) tlist[atomicAdd(tcnt, 1)] = c;
        } else {
            f.pflag[c] = (unsigned char)ps;
        }
    }
    // next impedance and dt candidate: C_CFL L_c / a = C_CFL (2 D V / area) (m / V) / z
    double z1;
    if (prm.eos) {
        double eps1 = e1, Fg[DD];
#pragma unroll
        for (int a = 0; a < D; ++a) eps1 -= 0.5 * v1[a] * v1[a];
#pragma unroll
        for (int q = 0; q < DD; ++q) Fg[q] = F1[q];  // (a copy, as above)
        z1 = impedance_sg<D>(prm, Fg, rho1, muc, eps1);
    } else {
        z1 = impedance<D>(F1, rho1, muc, kap);
    }
    f.z1[c] = z1;
    // min(A / B, C / |dV|) with one division: compare A |dV| with C B (B, |dV| > 0; a NaN
    // quotient A / B loses, as in fmin)
    const double A = prm.cfl * (2.0 * D) * mc, B = area1 * z1;
    const double dV = fabs(V1 - V0), C = prm.Cv * dt * V0;
    const bool vol = dV != 0.0 && !(A * dV <= C * B);
    f.dtc[c] = vol ? C / dV : A / B;
}

template <int D, bool LISTED, int B = kCellBlock>
__global__ void __launch_bounds__(B) k_update(Geo g, Fld f, Prm prm, const int *__restrict__ list,
                                                       const int *__restrict__ cnt, int n, int *tlist, int *tcnt) {
    if constexpr (!LISTED) {
        const int c = blockIdx.x * blockDim.x + threadIdx.x;
        if (c < n) update_cell<D>(g, f, prm, c, tlist, tcnt);
    } else {
        const int nn = *cnt;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x)
            update_cell<D>(g, f, prm, list[i], tlist, tcnt);
    }
}

// MOOD round bookkeeping on the device (one thread): the round consumes the troubled list
// counted in cnt[in]; a new mark stamp, the output counters cleared, the iteration bound
// checked (exceeding it sets ctl->err and empties the round).
static __global__ void k_round_begin(Fld f, Ctl *ctl, int in, int out, int max_iters) {
    const int n = f.cnt[in];
    if (n > 0) {
        if (ctl->iters >= max_iters) {
            ctl->err = 1;
            f.cnt[in] = 0;
        } else {
            ctl->iters += 1;
            ctl->troubled += n;
            ctl->stamp += 1;
        }
    }
    f.cnt[out] = 0;
    f.cnt[CNT_NODES] = 0;
    f.cnt[CNT_CELLS] = 0;
}

static __global__ void k_ctl_reset(Ctl *ctl) {
    ctl->iters = 0;
    ctl->troubled = 0;
    ctl->err = 0;
}

// append item to list[*cnt] when take is set, one atomicAdd per converged group of lanes
// (the lanes that take share one slot range; the order within it follows the lanes)
__device__ __forceinline__ void append_aggregated(bool take, int item, int *list, int *cnt) {
    const unsigned m = __activemask();
    const unsigned b = __ballot_sync(m, take);
    if (!take) return;  // the lanes of b alone take part in the broadcast below
    const int lane = threadIdx.x & 31, leader = __ffs(b) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(cnt, __popc(b));
    base = __shfl_sync(b, base, leader);
    list[base + __popc(b & ((1u << lane) - 1u))] = item;
}

// troubled cells become P0 (or P1 with limited slopes); their nodes are appended (once) to
// the node list. Work item i is the pair (troubled cell i / (D+1), its vertex i % (D+1)).
template <int D>
__device__ __forceinline__ void mark_nodes_range(const Geo &g, const Fld &f, const Prm &prm, const int *tlist, int n,
                                                 int *node_mark, int stamp, int *nlist, int i0, int di) {
    const long long items = (long long)n * (D + 1);
    for (long long i = i0; i < items; i += di) {
        const int c = tlist[i / (D + 1)], k = (int)(i % (D + 1));
        if (k == 0) f.order[c] = (f.order[c] == 2 && prm.cascade == 3) ? 3 : 1;  // one level down the cascade
        const int p = __ldg(g.c2n + k * g.N + c);
        append_aggregated(atomicExch(node_mark + p, stamp) != stamp, p, nlist, f.cnt + CNT_NODES);
    }
}

template <int D>
__global__ void k_mark_nodes(Geo g, Fld f, Prm prm, const int *__restrict__ tlist, const int *__restrict__ tcnt,
                             int *node_mark, const Ctl *ctl, int *nlist) {
    mark_nodes_range<D>(g, f, prm, tlist, *tcnt, node_mark, ctl->stamp, nlist, blockIdx.x * blockDim.x + threadIdx.x,
                        gridDim.x * blockDim.x);
}

// every cell around a listed node is appended (once) to the cell list; G consecutive lanes
// (G divides 32, the caller's indices keep lanes of a warp consecutive) share a node and
// take its cells in parallel
template <int G>
__device__ __forceinline__ void mark_cells_range(const Geo &g, const Fld &f, const int *nlist, int n, int *cell_mark,
                                                 int stamp, int *clist, int i0, int di) {
    const int sub = i0 % G;
    for (int i = i0 / G; i < n; i += di / G) {
        const int p = nlist[i];
        const int j1 = g.n2c_off[p + 1];
        for (int j = g.n2c_off[p] + sub; j < j1; j += G) {
            const int c = g.n2c[j] % g.N;
            append_aggregated(atomicExch(cell_mark + c, stamp) != stamp, c, clist, f.cnt + CNT_CELLS);
        }
    }
}

// lanes per node when marking cells: about the node degree (2D ~6, 3D Kuhn meshes ~24)
template <int D> constexpr int kMarkLanes = D == 2 ? 8 : 32;

template <int D>
__global__ void k_mark_cells(Geo g, Fld f, const int *__restrict__ nlist, int *cell_mark, const Ctl *ctl, int *clist) {
    mark_cells_range<kMarkLanes<D>>(g, f, nlist, f.cnt[CNT_NODES], cell_mark, ctl->stamp, clist,
                                    blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// while-loop condition of a graph-captured step: another MOOD round is needed
static __global__ void k_loop_cond(cudaGraphConditionalHandle h, Fld f, const Ctl *ctl) {
    cudaGraphSetConditional(h, (f.cnt[CNT_T0] > 0 && ctl->err == 0) ? 1u : 0u);
}

static __global__ void k_report(Fld f, const Ctl *ctl, Report *r) {
    r->n_troubled = ctl->troubled;
    r->mood_iters = ctl->iters;
    r->err = ctl->err;
    r->n_p0 = f.cnt[CNT_P0];
    r->n_para = f.cnt[CNT_PARA];
    r->n_eps = f.cnt[CNT_EPS];
    r->n_lim = f.cnt[CNT_LIM];
    r->dt_used = f.dt[0];
    r->dt_next = __longlong_as_double((long long)f.dtn[0]);
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    return v;
}

__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// dtn[inst] = (1 + C_i) dt[inst] (or dt_fixed, or +inf when ci < 0: initial acoustic dt)
static __global__ void k_dt_init(Fld f, Prm prm, int n_inst, int first) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_inst) return;
    double d;
    if (prm.dt_fixed > 0) d = prm.dt_fixed;
    else if (first) d = __longlong_as_double(0x7ff0000000000000LL);
    else d = (1.0 + prm.Ci) * f.dt[i];
    f.dtn[i] = (unsigned long long)__double_as_longlong(d);
}

// min of the dt candidates per instance (positive doubles compare as their bit patterns, so
// the result is exact and independent of the order) and the P0 / parachute counters
// the block's cells c0 .. c0 + blockDim.x - 1 (at most 256 threads); every thread of the block calls it
__device__ __forceinline__ void finalize_block(const Geo &g, const Fld &f, const Prm &prm, int c0) {
    const int c = c0 + threadIdx.x;
    const bool in = c < g.N;
    unsigned long long bits = ~0ull;
    int p0 = 0, para = 0, eps = 0, lim = 0;
    int inst = 0;
    if (in) {
        if (!(prm.dt_fixed > 0)) bits = (unsigned long long)__double_as_longlong(f.dtc[c]);
        const int o = f.order[c];
        p0 = o == 1;
        lim = o == 3;
        const int pf = f.pflag[c];
        para = p0 && pf == 2;
        eps = p0 && pf == 1;
        inst = g.cell_inst ? g.cell_inst[c] : 0;
    }
    // blocks whose cells all belong to one instance reduce before the atomic
    const int c1 = min(g.N, c0 + (int)blockDim.x) - 1;
    const bool uniform = !g.cell_inst || g.cell_inst[c0] == g.cell_inst[c1];
    __shared__ unsigned long long sb[8];
    __shared__ int si[8][4];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    p0 = warp_sum_i(p0);
    para = warp_sum_i(para);
    eps = warp_sum_i(eps);
    lim = warp_sum_i(lim);
    if (lane == 0) {
        si[w][0] = p0;
        si[w][1] = para;
        si[w][2] = eps;
        si[w][3] = lim;
    }
    if (uniform) {
        const unsigned long long m = warp_min_u64(bits);
        if (lane == 0) sb[w] = m;
    } else if (in && bits != ~0ull) {
        atomicMin(f.dtn + inst, bits);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int a = 0, b = 0, e = 0, l = 0;
        unsigned long long m = ~0ull;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            a += si[q][0];
            b += si[q][1];
            e += si[q][2];
            l += si[q][3];
            if (uniform) m = sb[q] < m ? sb[q] : m;
        }
        if (a) atomicAdd(f.cnt + CNT_P0, a);
        if (b) atomicAdd(f.cnt + CNT_PARA, b);
        if (e) atomicAdd(f.cnt + CNT_EPS, e);
        if (l) atomicAdd(f.cnt + CNT_LIM, l);
        if (uniform && m != ~0ull) atomicMin(f.dtn + (g.cell_inst ? g.cell_inst[c0] : 0), m);
    }
}

static __global__ void __launch_bounds__(256) k_finalize(Geo g, Fld f, Prm prm) {
    finalize_block(g, f, prm, blockIdx.x * blockDim.x);
}

// initial cell state: m = rho0 |w_c|, 1/m, centroid, rho, tau, F (identity when not given),
// e = |v|^2/2 + Psi(F), impedance, acoustic dt candidate
// the velocity gradient of the current v_p on the cell's geometry at the current x, kept in the
// geometry record as the update keeps its L^{n+1} (the same arithmetic: one division for 1/|w_c|)
template <int D>
__device__ __forceinline__ void cell_grad_current(const Geo &g, const Fld &f, int c, const double (&Nf)[D + 1][D],
                                                  double V) {
    double vn[D + 1][D], L[D * D];
#pragma unroll
    for (int k = 0; k < D + 1; ++k) {
        const int p = g.c2n[k * g.N + c];
#pragma unroll
        for (int a = 0; a < D; ++a) vn[k][a] = f.vp[a * g.Np + p];
    }
    vel_gradient<D>(vn, Nf, 1.0 / V, L);
    store_cell_grad<D>(f.gf, g.N, c, L);
}

template <int D>
__global__ void __launch_bounds__(kCellBlock) k_init_cells(Geo g, Fld f, Prm prm, double rho0, double *m_out,
                                                           double *im_out, int f_given) {
    constexpr int NV = D + 1, DD = D * D;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    const int N = g.N, Np = g.Np;
    double xs[NV][D];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const int p = g.c2n[k * N + c];
#pragma unroll
        for (int a = 0; a < D; ++a) xs[k][a] = f.x[a * Np + p];
    }
    double V, Nf[NV][D], rs[NV], ss[NV];
    simplex_faces<D>(xs, V, Nf);
    face_rnorms<D>(Nf, rs, ss);
    store_cell_geo<D>(f.gf, N, c, Nf, V, rs);
    const double mc = rho0 * V, imc = 1.0 / mc;
    m_out[c] = mc;
    im_out[c] = imc;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < NV; ++k) s += xs[k][a];
        f.xc[a * N + c] = s * (1.0 / NV);
    }
    const double rho = mc * (1.0 / V);  // as the update and a refresh compute rho and tau
    f.rho[c] = rho;
    f.tau1[c] = V * imc;
    double F[DD];
#pragma unroll
    for (int q = 0; q < DD; ++q) {
        F[q] = f_given ? f.F[q * N + c] : ((q % (D + 1)) == 0 ? 1.0 : 0.0);
        f.F[q * N + c] = F[q];
    }
    const double muc = f.mu[c], kap = kappa_of(prm, muc);
    double ke = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const double va = f.v[a * N + c];
        ke += 0.5 * va * va;
    }
    double z;
    if (prm.eos) {  // stiffened gas: eps_v from the initial pressure p0 at rho0 / det F
        const double eps_v = (prm.p0 + prm.gamma * prm.pinf) / ((prm.gamma - 1.0) * rho0 / det<D>(F));
        const double eps = eps_v + shear_energy<D>(prm, F, muc);
        f.e[c] = ke + eps;
        z = impedance_sg<D>(prm, F, rho, muc, eps);
    } else {
        f.e[c] = ke + (prm.shear_a == -1.0 ? free_energy<D>(F, rho0, muc, kap)
                                           : free_energy_family<D>(F, rho0, muc, kap, prm.shear_a));
        z = impedance<D>(F, rho, muc, kap);
    }
    f.order[c] = 1;
    f.pflag[c] = 0;
    f.z[c] = z;
    f.dtc[c] = prm.cfl * insphere<D>(V, Nf) * rho / z;
}

// derived quantities of the current positions, v_p and F: the cell geometry record (with the
// velocity gradient of v_p), centroid, rho = m / |w_c|, tau = |w_c| / m, impedance z
template <int D> __global__ void __launch_bounds__(kCellBlock) k_refresh(Geo g, Fld f, Prm prm) {
    constexpr int NV = D + 1, DD = D * D;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    double xs[NV][D];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const int p = g.c2n[k * g.N + c];
#pragma unroll
        for (int a = 0; a < D; ++a) xs[k][a] = f.x[a * g.Np + p];
    }
    double V, Nf[NV][D], rs[NV], ss[NV];
    simplex_faces<D>(xs, V, Nf);
    face_rnorms<D>(Nf, rs, ss);
    store_cell_geo<D>(f.gf, g.N, c, Nf, V, rs);  // as the update stores it
    cell_grad_current<D>(g, f, c, Nf, V);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < NV; ++k) s += xs[k][a];
        f.xc[a * g.N + c] = s * (1.0 / NV);
    }
    const double rho = f.m[c] * (1.0 / V);  // as the update computes it, so that a restart is bitwise
    f.rho[c] = rho;
    f.tau1[c] = V * f.im[c];
    double F[DD];
#pragma unroll
    for (int q = 0; q < DD; ++q) F[q] = f.F[q * g.N + c];
    const double muc = f.mu[c];
    if (prm.eos) {
        double eps = f.e[c];
#pragma unroll
        for (int a = 0; a < D; ++a) eps -= 0.5 * f.v[a * g.N + c] * f.v[a * g.N + c];
        f.z[c] = impedance_sg<D>(prm, F, rho, muc, eps);
    } else {
        f.z[c] = impedance<D>(F, rho, muc, kappa_of(prm, muc));
    }
}

// the cells' geometry at the current positions and the velocity gradient of the current v_p
// alone (the initial state once v_p^0 is known, or a view of a recorded state, whose x^n
// record no update has left)
template <int D> __global__ void __launch_bounds__(kCellBlock) k_geometry(Geo g, Fld f) {
    constexpr int NV = D + 1;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    double xs[NV][D];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const int p = g.c2n[k * g.N + c];
#pragma unroll
        for (int a = 0; a < D; ++a) xs[k][a] = f.x[a * g.Np + p];
    }
    double V, Nf[NV][D], rs[NV], ss[NV];
    simplex_faces<D>(xs, V, Nf);
    face_rnorms<D>(Nf, rs, ss);
    store_cell_geo<D>(f.gf, g.N, c, Nf, V, rs);
    cell_grad_current<D>(g, f, c, Nf, V);
}

// sums of m, m v, m e (diagnostic; atomics, so the last bits depend on scheduling)
template <int D> __global__ void __launch_bounds__(256) k_totals(Geo g, Fld f, double *out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    double q[5] = {0, 0, 0, 0, 0};
    if (c < g.N) {
        const double m = f.m[c];
        q[0] = m;
#pragma unroll
        for (int a = 0; a < D; ++a) q[1 + a] = m * f.v[a * g.N + c];
        q[4] = m * f.e[c];
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        double v = q[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(out + i, v);
    }
}

}  // namespace lmood
