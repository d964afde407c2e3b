// lmood_adjoint.cuh -- per-entity functions of the step written as pure functions of their
// gathered inputs, and their hand-written vector-Jacobian products (reverse mode), for the
// adjoint of the whole step with the MOOD order mask and the time step frozen. They compile
// for host and device, so that each product can be checked against finite differences of its
// forward function on the CPU. The forward kernels keep their own FP64-lean arithmetic; these
// functions recompute intermediates for the reverse pass (a linearisation, where a last-bit
// difference in an intermediate does not matter).
#pragma once
#include <math.h>

#include "lmood_dev.cuh"

#ifdef __CUDACC__
#define LMOOD_HD __host__ __device__ __forceinline__
#else
#define LMOOD_HD inline
#endif

namespace lmood {
namespace adj {

// J^{-1/3} and log J: on the device the forward kernels' own FP64 evaluations (rcbrt_j,
// log_j: a few ulp, far fewer instructions than pow / log), on the host the C library's
LMOOD_HD double adj_rcbrt(double J) {
#ifdef __CUDA_ARCH__
    return rcbrt_j(J);
#else
    return 1.0 / cbrt(J);
#endif
}

LMOOD_HD double adj_log(double J) {
#ifdef __CUDA_ARCH__
    return log_j(J);
#else
    return log(J);
#endif
}

template <int D> struct Sz {
    static constexpr int NV = D + 1, DD = D * D, NS = D * (D + 1) / 2, NQ = D + D * D;
    static constexpr int M_N = 0, M_S1 = 1, M_S2 = 1 + D, M_U = 1 + D + NS, M_T = 1 + D + NS + NQ;
    static constexpr int NMOM = 1 + D + NS + NQ + NQ * D;
};

template <int D> LMOOD_HD int sym(int a, int b) {
    if (D == 2) return a + b;
    if (a > b) {
        const int t = a;
        a = b;
        b = t;
    }
    return a == 0 ? b : (a == 1 ? 2 + b : 5);
}

template <int D> LMOOD_HD double det(const double *A) {
    if constexpr (D == 2) return A[0] * A[3] - A[1] * A[2];
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) + A[2] * (A[3] * A[7] - A[4] * A[6]);
}

// cofactor matrix d(det A)/dA
template <int D> LMOOD_HD void cofactor(const double *A, double *C) {
    if constexpr (D == 2) {
        C[0] = A[3]; C[1] = -A[2];
        C[2] = -A[1]; C[3] = A[0];
    } else {
        C[0] = A[4] * A[8] - A[5] * A[7]; C[1] = A[5] * A[6] - A[3] * A[8]; C[2] = A[3] * A[7] - A[4] * A[6];
        C[3] = A[2] * A[7] - A[1] * A[8]; C[4] = A[0] * A[8] - A[2] * A[6]; C[5] = A[1] * A[6] - A[0] * A[7];
        C[6] = A[1] * A[5] - A[2] * A[4]; C[7] = A[2] * A[3] - A[0] * A[5]; C[8] = A[0] * A[4] - A[1] * A[3];
    }
}

template <int D> LMOOD_HD void inverse(const double *A, double *Ai) {
    double C[D * D];
    cofactor<D>(A, C);
    const double r = 1.0 / det<D>(A);
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) Ai[i * D + j] = C[j * D + i] * r;
}

template <int D> LMOOD_HD void mm(const double *A, const double *B, double *C) {  // C = A B
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            double s = 0.0;
            for (int k = 0; k < D; ++k) s += A[i * D + k] * B[k * D + j];
            C[i * D + j] = s;
        }
}

template <int D> LMOOD_HD void mtm(const double *A, const double *B, double *C) {  // C = A^t B
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            double s = 0.0;
            for (int k = 0; k < D; ++k) s += A[k * D + i] * B[k * D + j];
            C[i * D + j] = s;
        }
}

template <int D> LMOOD_HD void mmt(const double *A, const double *B, double *C) {  // C = A B^t
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            double s = 0.0;
            for (int k = 0; k < D; ++k) s += A[i * D + k] * B[j * D + k];
            C[i * D + j] = s;
        }
}

// ---------------------------------------------------------------------------------------
// Neo-Hookean stress T(F) (plane strain in 2D) and its product lamT -> (lamF, lam_mu, lam_kappa).
// ---------------------------------------------------------------------------------------
template <int D> LMOOD_HD void stress(const double *F, double mu, double kap, double *T) {
    const double J = det<D>(F), lJ = adj_log(J), rc = adj_rcbrt(J), Jm23 = rc * rc, invJ = Jm23 * rc;
    const double cj = mu * invJ * Jm23;
    const double p = -0.5 * kap * (J - 1.0 + lJ * invJ);
    double B[D * D];
    mmt<D>(F, F, B);
    double tr = D == 2 ? 1.0 : 0.0;
    for (int i = 0; i < D; ++i) tr += B[i * D + i];
    const double diag = -p - cj * tr * (1.0 / 3.0);
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) T[i * D + j] = cj * B[i * D + j] + (i == j ? diag : 0.0);
}

// T_out (may be NULL) receives T(F) itself, sharing the scalar functions of J.
template <int D>
LMOOD_HD void stress_vjp(const double *F, double mu, double kap, const double *lT, double *lF, double &lmu,
                         double &lkap, double *T_out = nullptr) {
    const double J = det<D>(F), lJ = adj_log(J), rc = adj_rcbrt(J), Jm23 = rc * rc, invJ = Jm23 * rc;
    const double J53 = invJ * Jm23;
    const double cj = mu * J53;
    double B[D * D];
    mmt<D>(F, F, B);
    double tr = D == 2 ? 1.0 : 0.0;
    for (int i = 0; i < D; ++i) tr += B[i * D + i];
    if (T_out) {
        const double p = -0.5 * kap * (J - 1.0 + lJ * invJ);
        const double diag = -p - cj * tr * (1.0 / 3.0);
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) T_out[i * D + j] = cj * B[i * D + j] + (i == j ? diag : 0.0);
    }
    double lcj = 0.0, ldiag = 0.0, lB[D * D];
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            lcj += lT[i * D + j] * B[i * D + j];
            lB[i * D + j] = cj * lT[i * D + j];
        }
    for (int i = 0; i < D; ++i) ldiag += lT[i * D + i];
    // diag = -p - cj tr / 3
    const double lp = -ldiag;
    lcj += -ldiag * tr * (1.0 / 3.0);
    const double ltr = -ldiag * cj * (1.0 / 3.0);
    for (int i = 0; i < D; ++i) lB[i * D + i] += ltr;
    // cj = mu J^{-5/3};  p = -(kap/2)(J - 1 + log J / J)
    lmu += lcj * J53;
    double lJv = lcj * (-5.0 / 3.0) * cj * invJ;
    lkap += lp * (-0.5) * (J - 1.0 + lJ * invJ);
    lJv += lp * (-0.5 * kap) * (1.0 + (1.0 - lJ) * invJ * invJ);
    // B = F F^t: lF = (lB + lB^t) F;  J = det F: lF += lJ cof(F)
    double C[D * D];
    cofactor<D>(F, C);
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            double s = 0.0;
            for (int k = 0; k < D; ++k) s += (lB[i * D + k] + lB[k * D + i]) * F[k * D + j];
            lF[i * D + j] += s + lJv * C[i * D + j];
        }
}

// impedance z = sqrt(rho (K + 4 mu / (3 J))), K = (kap/2)(J + (1 - log J)/J)
template <int D> LMOOD_HD double impedance(const double *F, double rho, double mu, double kap) {
    const double J = det<D>(F), invJ = 1.0 / J;
    const double K = 0.5 * kap * (J + (1.0 - adj_log(J)) * invJ);
    return sqrt(rho * (K + (4.0 / 3.0) * mu * invJ));
}

template <int D>
LMOOD_HD void impedance_vjp(const double *F, double rho, double mu, double kap, double lz, double *lF, double &lrho,
                            double &lmu, double &lkap) {
    const double J = det<D>(F), invJ = 1.0 / J, lJ = adj_log(J);
    const double K = 0.5 * kap * (J + (1.0 - lJ) * invJ);
    const double inner = K + (4.0 / 3.0) * mu * invJ;
    const double z = sqrt(rho * inner), h = 0.5 / z;
    const double linner = lz * rho * h;
    lrho += lz * inner * h;
    lmu += linner * (4.0 / 3.0) * invJ;
    lkap += linner * 0.5 * (J + (1.0 - lJ) * invJ);
    const double lJv = linner * (0.5 * kap * (1.0 + (lJ - 2.0) * invJ * invJ) - (4.0 / 3.0) * mu * invJ * invJ);
    double C[D * D];
    cofactor<D>(F, C);
    for (int i = 0; i < D * D; ++i) lF[i] += lJv * C[i];
}

// ---------------------------------------------------------------------------------------
// Simplex geometry: measure V and outward face area vectors N_k (face opposite vertex k);
// dV/dx_k = -N_k / D (the corner vector).
// ---------------------------------------------------------------------------------------
template <int D> LMOOD_HD void faces(const double *xs, double &V, double *N) {  // xs [NV][D], N [NV][D]
    if constexpr (D == 2) {
        V = 0.5 * ((xs[2] - xs[0]) * (xs[5] - xs[1]) - (xs[3] - xs[1]) * (xs[4] - xs[0]));
        for (int k = 0; k < 3; ++k) {
            const int a = (k + 1) % 3, b = (k + 2) % 3;
            N[k * 2 + 0] = xs[b * 2 + 1] - xs[a * 2 + 1];
            N[k * 2 + 1] = xs[a * 2 + 0] - xs[b * 2 + 0];
        }
    } else {
        double e[3][3];
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) e[k][a] = xs[(k + 1) * 3 + a] - xs[a];
        V = (e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) + e[0][1] * (e[1][2] * e[2][0] - e[1][0] * e[2][2]) +
             e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0])) / 6.0;
        for (int k = 0; k < 4; ++k) {
            const int fa = (k + 1) & 3, fb = (k + 2) & 3, fc = (k + 3) & 3;
            double u[3], w[3];
            for (int a = 0; a < 3; ++a) {
                u[a] = xs[fb * 3 + a] - xs[fa * 3 + a];
                w[a] = xs[fc * 3 + a] - xs[fa * 3 + a];
            }
            const double s = (k & 1) ? -0.5 : 0.5;
            N[k * 3 + 0] = s * (u[1] * w[2] - u[2] * w[1]);
            N[k * 3 + 1] = s * (u[2] * w[0] - u[0] * w[2]);
            N[k * 3 + 2] = s * (u[0] * w[1] - u[1] * w[0]);
        }
    }
}

template <int D> LMOOD_HD void faces_vjp(const double *xs, double lV, const double *lN, double *lxs) {
    double V, N[(D + 1) * D];
    faces<D>(xs, V, N);
    for (int k = 0; k < D + 1; ++k)
        for (int a = 0; a < D; ++a) lxs[k * D + a] += lV * (N[k * D + a] * (-1.0 / D));
    if constexpr (D == 2) {
        for (int k = 0; k < 3; ++k) {
            const int a = (k + 1) % 3, b = (k + 2) % 3;
            lxs[b * 2 + 1] += lN[k * 2 + 0];
            lxs[a * 2 + 1] -= lN[k * 2 + 0];
            lxs[a * 2 + 0] += lN[k * 2 + 1];
            lxs[b * 2 + 0] -= lN[k * 2 + 1];
        }
    } else {
        for (int k = 0; k < 4; ++k) {
            const int fa = (k + 1) & 3, fb = (k + 2) & 3, fc = (k + 3) & 3;
            double u[3], w[3], l[3];
            const double s = (k & 1) ? -0.5 : 0.5;
            for (int a = 0; a < 3; ++a) {
                u[a] = xs[fb * 3 + a] - xs[fa * 3 + a];
                w[a] = xs[fc * 3 + a] - xs[fa * 3 + a];
                l[a] = s * lN[k * 3 + a];
            }
            // d(u x w) = du x w + u x dw:  lu = w x l,  lw = l x u
            const double lu[3] = {w[1] * l[2] - w[2] * l[1], w[2] * l[0] - w[0] * l[2], w[0] * l[1] - w[1] * l[0]};
            const double lw[3] = {l[1] * u[2] - l[2] * u[1], l[2] * u[0] - l[0] * u[2], l[0] * u[1] - l[1] * u[0]};
            for (int a = 0; a < 3; ++a) {
                lxs[fb * 3 + a] += lu[a];
                lxs[fc * 3 + a] += lw[a];
                lxs[fa * 3 + a] -= lu[a] + lw[a];
            }
        }
    }
}

// velocity gradient L = -(1/(D V)) sum_k v_k (x) N_k and its product; the _iv forms take
// iV = 1 / V (shared by the callers that also need it), the product also L itself
template <int D> LMOOD_HD void velgrad_iv(const double *vn, const double *N, double iV, double *L) {
    const double s0 = iV * (-1.0 / D);
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            double s = 0.0;
            for (int k = 0; k < D + 1; ++k) s += vn[k * D + i] * N[k * D + j];
            L[i * D + j] = s * s0;
        }
}

template <int D> LMOOD_HD void velgrad(const double *vn, const double *N, double V, double *L) {
    velgrad_iv<D>(vn, N, 1.0 / V, L);
}

template <int D>
LMOOD_HD void velgrad_vjp_iv(const double *vn, const double *N, double iV, const double *L, const double *lL,
                             double *lvn, double *lN, double &lV) {
    const double s0 = iV * (-1.0 / D);
    for (int k = 0; k < D + 1; ++k)
        for (int i = 0; i < D; ++i) {
            double a = 0.0, b = 0.0;
            for (int j = 0; j < D; ++j) {
                a += lL[i * D + j] * N[k * D + j];
                b += lL[j * D + i] * vn[k * D + j];
            }
            lvn[k * D + i] += s0 * a;
            lN[k * D + i] += s0 * b;
        }
    double s = 0.0;
    for (int i = 0; i < D * D; ++i) s += lL[i] * L[i];
    lV -= s * iV;  // L is proportional to 1 / V
}

template <int D>
LMOOD_HD void velgrad_vjp(const double *vn, const double *N, double V, const double *lL, double *lvn, double *lN,
                          double &lV) {
    const double iV = 1.0 / V;
    double L[D * D];
    velgrad_iv<D>(vn, N, iV, L);
    velgrad_vjp_iv<D>(vn, N, iV, L, lL, lvn, lN, lV);
}

// ---------------------------------------------------------------------------------------
// Nodal solve with a projector: v = K b, K = P (P^t M P)^{-1} P^t (free: M^{-1}; clamped: 0).
// Product: lb = K lv, lM = -lb (x) v (full matrix).
// ---------------------------------------------------------------------------------------
template <int D>
LMOOD_HD void node_solve(const double *M, const double *b, int nd, const double *t /*[2][3]*/, double *v) {
    if (nd == D) {
        double Mi[D * D];
        inverse<D>(M, Mi);
        for (int a = 0; a < D; ++a) {
            double s = 0.0;
            for (int c = 0; c < D; ++c) s += Mi[a * D + c] * b[c];
            v[a] = s;
        }
    } else if (nd == 0) {
        for (int a = 0; a < D; ++a) v[a] = 0.0;
    } else {
        double A[4], r[2], al[2] = {0.0, 0.0};
        for (int i = 0; i < nd; ++i) {
            double s = 0.0;
            for (int a = 0; a < D; ++a) s += t[i * 3 + a] * b[a];
            r[i] = s;
            for (int j = 0; j < nd; ++j) {
                double q = 0.0;
                for (int a = 0; a < D; ++a)
                    for (int c = 0; c < D; ++c) q += t[i * 3 + a] * M[a * D + c] * t[j * 3 + c];
                A[i * nd + j] = q;
            }
        }
        if (nd == 1) {
            al[0] = r[0] / A[0];
        } else {
            const double dA = A[0] * A[3] - A[1] * A[2];
            al[0] = (A[3] * r[0] - A[1] * r[1]) / dA;
            al[1] = (-A[2] * r[0] + A[0] * r[1]) / dA;
        }
        for (int a = 0; a < D; ++a) {
            double s = 0.0;
            for (int i = 0; i < nd; ++i) s += al[i] * t[i * 3 + a];
            v[a] = s;
        }
    }
}

template <int D>
LMOOD_HD void node_solve_vjp(const double *M, const double *b, int nd, const double *t, const double *lv, double *lb,
                             double *lM /* full D x D, accumulated */) {
    double v[D];
    node_solve<D>(M, b, nd, t, v);
    node_solve<D>(M, lv, nd, t, lb);  // K is symmetric: lb = K lv
    for (int a = 0; a < D; ++a)
        for (int c = 0; c < D; ++c) lM[a * D + c] += -lb[a] * v[c];
}


// ---------------------------------------------------------------------------------------
// Cell predictor and corner packets (pure form of k_predict for orders 1 and 2).
// Inputs: xs [NV][D] node positions at t^n; mom(k, j) = moment j of node k (accessor with a
// stride); vc, Fc, z, mu, kappa, 1/m, dt; ord. Outputs: M [NV][NS] (symmetric storage),
// R [NV][D].
// ---------------------------------------------------------------------------------------
template <int D> struct Mom {
    const double *p[D + 1];
    int stride;
    LMOOD_HD double operator()(int k, int j) const { return p[k][j * stride]; }
};

template <int D>
LMOOD_HD void predict_fw(const double *xs, const Mom<D> &mom, const double *vc, const double *Fc, double z, double mu,
                         double kap, double im, double dt, int ord, double *Mo, double *Ro) {
    using Q = Sz<D>;
    constexpr int NV = Q::NV, DD = Q::DD, NS = Q::NS, NQ = Q::NQ;
    double V, N[NV * D], xcc[D], W[NV][NS];
    faces<D>(xs, V, N);
    for (int a = 0; a < D; ++a) {
        double s = 0.0;
        for (int k = 0; k < NV; ++k) s += xs[k * D + a];
        xcc[a] = s * (1.0 / NV);
    }
    for (int f = 0; f < NV; ++f) {
        double u[D], ss = 0.0;
        for (int a = 0; a < D; ++a) {
            u[a] = N[f * D + a] * (1.0 / D);
            ss += u[a] * u[a];
        }
        const double w = z / sqrt(ss);
        for (int a = 0; a < D; ++a)
            for (int b = a; b < D; ++b) W[f][sym<D>(a, b)] = w * u[a] * u[b];
    }
    for (int k = 0; k < NV; ++k)
        for (int s = 0; s < NS; ++s) {
            double acc = 0.0;
            for (int f = 0; f < NV; ++f)
                if (f != k) acc += W[f][s];
            Mo[k * NS + s] = acc;
        }
    auto Mfull = [&](int k, int a, int b) { return Mo[k * NS + sym<D>(a, b)]; };
    if (ord == 1) {
        double T[DD];
        stress<D>(Fc, mu, kap, T);
        for (int k = 0; k < NV; ++k)
            for (int a = 0; a < D; ++a) {
                double s = 0.0;
                for (int b = 0; b < D; ++b) s += Mfull(k, a, b) * vc[b] + T[a * D + b] * N[k * D + b] * (1.0 / D);
                Ro[k * D + a] = s;
            }
        return;
    }
    // least squares from the node moments
    double G[DD] = {}, r[NQ][D] = {}, npair = -NV;  // (node, other cell) pairs of the stencil
    double qc[NQ];
    for (int q = 0; q < NQ; ++q) qc[q] = q < D ? vc[q] : Fc[q - D];
    for (int k = 0; k < NV; ++k) {
        double d[D], S1[D], w[D];
        const double n = mom(k, Q::M_N);
        npair += n;
        for (int a = 0; a < D; ++a) {
            d[a] = xs[k * D + a] - xcc[a];
            S1[a] = mom(k, Q::M_S1 + a);
            w[a] = S1[a] + n * d[a];
        }
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b) G[a * D + b] += mom(k, Q::M_S2 + sym<D>(a, b)) + S1[a] * d[b] + d[a] * w[b];
        for (int q = 0; q < NQ; ++q)
            for (int a = 0; a < D; ++a)
                r[q][a] += mom(k, Q::M_T + q * D + a) + d[a] * mom(k, Q::M_U + q) - w[a] * qc[q];
    }
    double tr = 0.0;
    for (int a = 0; a < D; ++a) tr += G[a * D + a];
    const double t = tr * (1.0 / D);
    const bool ok = npair > 0.0 && det<D>(G) > 1e-12 * (D == 2 ? t * t : t * t * t);
    double Gi[DD], gs[NQ][D];
    inverse<D>(G, Gi);
    for (int q = 0; q < NQ; ++q)
        for (int a = 0; a < D; ++a) {
            double s = 0.0;
            for (int b = 0; b < D; ++b) s += Gi[a * D + b] * r[q][b];
            gs[q][a] = ok ? s : 0.0;
        }
    double dv[D] = {}, dFdt[DD], gv[DD];
    const double hv = -0.5 * dt * im * (1.0 / D);
    for (int k = 0; k < NV; ++k) {
        double Fh[DD], T[DD];
        for (int q = 0; q < DD; ++q) {
            double s = Fc[q];
            for (int a = 0; a < D; ++a) s += gs[D + q][a] * (xs[k * D + a] - xcc[a]);
            Fh[q] = s;
        }
        stress<D>(Fh, mu, kap, T);
        for (int i = 0; i < D; ++i)
            for (int b = 0; b < D; ++b) dv[i] += T[i * D + b] * N[k * D + b];
    }
    for (int a = 0; a < D; ++a) dv[a] *= hv;
    for (int i = 0; i < D; ++i)
        for (int a = 0; a < D; ++a) gv[i * D + a] = gs[i][a];
    mm<D>(gv, Fc, dFdt);
    for (int k = 0; k < NV; ++k) {
        double vst[D], Fs[DD], T[DD];
        for (int i = 0; i < D; ++i) {
            double s = vc[i];
            for (int a = 0; a < D; ++a) s += gs[i][a] * (xs[k * D + a] - xcc[a]);
            vst[i] = s + dv[i];
        }
        for (int q = 0; q < DD; ++q) {
            double s = Fc[q];
            for (int a = 0; a < D; ++a) s += gs[D + q][a] * (xs[k * D + a] - xcc[a]);
            Fs[q] = s + 0.5 * dt * dFdt[q];
        }
        stress<D>(Fs, mu, kap, T);
        for (int a = 0; a < D; ++a) {
            double s = 0.0;
            for (int b = 0; b < D; ++b) s += Mfull(k, a, b) * vst[b] + T[a * D + b] * N[k * D + b] * (1.0 / D);
            Ro[k * D + a] = s;
        }
    }
}

// Product of predict_fw: (lM [NV][NS], lR [NV][D]) -> accumulates lxs [NV][D], lvc [D],
// lFc [DD], lz, lmu, lkap, and stores the adjoints of the node moments through
// mout(k, j, value) (every (k, j) exactly once; zero where the packets do not depend on them).
template <int D, class MO>
LMOOD_HD void predict_vjp(const double *xs, const Mom<D> &mom, const double *vc, const double *Fc, double z, double mu,
                          double kap, double im, double dt, int ord, const double *lM_in, const double *lR, double *lxs,
                          MO &&mout, double *lvc, double *lFc, double &lz, double &lmu, double &lkap) {
    using Q = Sz<D>;
    constexpr int NV = Q::NV, DD = Q::DD, NS = Q::NS, NQ = Q::NQ, NM = Q::NMOM;
    double V, N[NV * D], xcc[D];
    faces<D>(xs, V, N);
    for (int a = 0; a < D; ++a) {
        double s = 0.0;
        for (int k = 0; k < NV; ++k) s += xs[k * D + a];
        xcc[a] = s * (1.0 / NV);
    }
    // M_k = sum_{f != k} W_f, W_f = (z / |u_f|) u_f u_f^t, u_f = N_f / D
    double Mo[NV * NS], inu[NV];  // inu = 1 / |u_f|
    {
        double W[NV][NS];
        for (int f = 0; f < NV; ++f) {
            double ss = 0.0;
            for (int a = 0; a < D; ++a) ss += N[f * D + a] * N[f * D + a];
            inu[f] = D / sqrt(ss);
            const double w = z * inu[f] * (1.0 / (D * D));
            for (int a = 0; a < D; ++a)
                for (int b = a; b < D; ++b) W[f][sym<D>(a, b)] = w * N[f * D + a] * N[f * D + b];
        }
        for (int k = 0; k < NV; ++k)
            for (int s2 = 0; s2 < NS; ++s2) {
                double acc = 0.0;
                for (int f = 0; f < NV; ++f)
                    if (f != k) acc += W[f][s2];
                Mo[k * NS + s2] = acc;
            }
    }
    auto Mfull = [&](int k, int a, int b) { return Mo[k * NS + sym<D>(a, b)]; };
    double lM[NV * NS], lN[NV * D] = {}, lxcc[D] = {};
    for (int i = 0; i < NV * NS; ++i) lM[i] = lM_in[i];
    // R_k = M_k vst_k + (1/D) T_k N_k: the parts that do not need T_k (lvst, lM, lT)
    auto packet_rhs_vjp = [&](int k, const double *vst, double *lvst, double *lT) {
        for (int a = 0; a < D; ++a) {
            const double l = lR[k * D + a];
            for (int b = 0; b < D; ++b) {
                lvst[b] += Mfull(k, a, b) * l;
                lM[k * NS + sym<D>(a, b)] += l * vst[b];
                lT[a * D + b] += l * N[k * D + b] * (1.0 / D);
            }
        }
    };
    // ... and the part that does: lN_k += (1/D) T_k^t lR_k
    auto packet_rhs_vjp_T = [&](int k, const double *T) {
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b) lN[k * D + b] += lR[k * D + a] * T[a * D + b] * (1.0 / D);
    };
    auto zero_moments = [&]() {
        for (int k = 0; k < NV; ++k)
            for (int j = 0; j < NM; ++j) mout(k, j, 0.0);
    };
    if (ord == 1) {
        double T[DD], lT[DD] = {}, lF[DD] = {};
        for (int k = 0; k < NV; ++k) {
            double lvst[D] = {};
            packet_rhs_vjp(k, vc, lvst, lT);
            for (int a = 0; a < D; ++a) lvc[a] += lvst[a];
        }
        stress_vjp<D>(Fc, mu, kap, lT, lF, lmu, lkap, T);
        for (int k = 0; k < NV; ++k) packet_rhs_vjp_T(k, T);
        for (int q = 0; q < DD; ++q) lFc[q] += lF[q];
        zero_moments();
    } else {
        // ---- recompute the forward intermediates
        double G[DD] = {}, r[NQ][D] = {}, qc[NQ], dk[NV][D], npair = -NV;
        for (int q = 0; q < NQ; ++q) qc[q] = q < D ? vc[q] : Fc[q - D];
        for (int k = 0; k < NV; ++k) {
            const double nk = mom(k, Q::M_N);
            npair += nk;
            double S1[D], w[D];
            for (int a = 0; a < D; ++a) {
                dk[k][a] = xs[k * D + a] - xcc[a];
                S1[a] = mom(k, Q::M_S1 + a);
                w[a] = S1[a] + nk * dk[k][a];
            }
            for (int a = 0; a < D; ++a)
                for (int b = 0; b < D; ++b) G[a * D + b] += mom(k, Q::M_S2 + sym<D>(a, b)) + S1[a] * dk[k][b] + dk[k][a] * w[b];
            for (int q = 0; q < NQ; ++q)
                for (int a = 0; a < D; ++a)
                    r[q][a] += mom(k, Q::M_T + q * D + a) + dk[k][a] * mom(k, Q::M_U + q) - w[a] * qc[q];
        }
        double tr = 0.0;
        for (int a = 0; a < D; ++a) tr += G[a * D + a];
        const double t = tr * (1.0 / D);
        const bool ok = npair > 0.0 && det<D>(G) > 1e-12 * (D == 2 ? t * t : t * t * t);
        double Gi[DD], gs[NQ][D];
        inverse<D>(G, Gi);
        for (int q = 0; q < NQ; ++q)
            for (int a = 0; a < D; ++a) {
                double s = 0.0;
                for (int b = 0; b < D; ++b) s += Gi[a * D + b] * r[q][b];
                gs[q][a] = ok ? s : 0.0;
            }
        auto Fh_of = [&](int k, double *Fh) {
            for (int q = 0; q < DD; ++q) {
                double s = Fc[q];
                for (int a = 0; a < D; ++a) s += gs[D + q][a] * dk[k][a];
                Fh[q] = s;
            }
        };
        double gv[DD], dFdt[DD], dvraw[D] = {};
        const double hv = -0.5 * dt * im * (1.0 / D);
        for (int k = 0; k < NV; ++k) {
            double Fh[DD], T[DD];
            Fh_of(k, Fh);
            stress<D>(Fh, mu, kap, T);
            for (int i = 0; i < D; ++i)
                for (int b = 0; b < D; ++b) dvraw[i] += T[i * D + b] * N[k * D + b];
        }
        for (int i = 0; i < D; ++i)
            for (int a = 0; a < D; ++a) gv[i * D + a] = gs[i][a];
        mm<D>(gv, Fc, dFdt);
        // ---- reverse of pass 2 (the corner predictor and packets)
        double lgs[NQ][D] = {}, ldk[NV][D] = {}, ldv[D] = {}, ldFdt[DD] = {}, lFh[NV][DD] = {};
        for (int k = 0; k < NV; ++k) {
            double vst[D], Fs[DD], T[DD], lvst[D] = {}, lT[DD] = {}, lFs[DD] = {};
            for (int i = 0; i < D; ++i) {
                double s = vc[i];
                for (int a = 0; a < D; ++a) s += gs[i][a] * dk[k][a];
                vst[i] = s + hv * dvraw[i];
            }
            Fh_of(k, Fs);
            for (int q = 0; q < DD; ++q) Fs[q] += 0.5 * dt * dFdt[q];
            packet_rhs_vjp(k, vst, lvst, lT);
            stress_vjp<D>(Fs, mu, kap, lT, lFs, lmu, lkap, T);
            packet_rhs_vjp_T(k, T);
            for (int q = 0; q < DD; ++q) {
                lFh[k][q] += lFs[q];
                ldFdt[q] += 0.5 * dt * lFs[q];
            }
            for (int i = 0; i < D; ++i) {
                lvc[i] += lvst[i];
                ldv[i] += lvst[i];
                for (int a = 0; a < D; ++a) {
                    lgs[i][a] += lvst[i] * dk[k][a];
                    ldk[k][a] += lvst[i] * gs[i][a];
                }
            }
        }
        // dFdt = gv Fc
        double lgv[DD];
        mmt<D>(ldFdt, Fc, lgv);  // lgv = ldFdt Fc^t
        {
            double t2[DD];
            mtm<D>(gv, ldFdt, t2);  // lFc += gv^t ldFdt
            for (int q = 0; q < DD; ++q) lFc[q] += t2[q];
        }
        for (int i = 0; i < D; ++i)
            for (int a = 0; a < D; ++a) lgs[i][a] += lgv[i * D + a];
        // ---- reverse of pass 1: dv = hv sum_k T(Fh_k) N_k
        double lacc[D];
        for (int i = 0; i < D; ++i) lacc[i] = hv * ldv[i];
        for (int k = 0; k < NV; ++k) {
            double Fh[DD], T[DD], lT[DD], lF[DD] = {};
            Fh_of(k, Fh);
            for (int i = 0; i < D; ++i)
                for (int b = 0; b < D; ++b) lT[i * D + b] = lacc[i] * N[k * D + b];
            stress_vjp<D>(Fh, mu, kap, lT, lF, lmu, lkap, T);
            for (int i = 0; i < D; ++i)
                for (int b = 0; b < D; ++b) lN[k * D + b] += lacc[i] * T[i * D + b];
            for (int q = 0; q < DD; ++q) lFh[k][q] += lF[q];
        }
        // Fh_k = Fc + gsF dk
        for (int k = 0; k < NV; ++k)
            for (int q = 0; q < DD; ++q) {
                lFc[q] += lFh[k][q];
                for (int a = 0; a < D; ++a) {
                    lgs[D + q][a] += lFh[k][q] * dk[k][a];
                    ldk[k][a] += lFh[k][q] * gs[D + q][a];
                }
            }
        // ---- least squares: gs = Gi r
        if (ok) {
            // gs_q = G^{-1} r_q, G symmetric: lr_q = G^{-1} lgs_q, lG = -sum_q lr_q gs_q^t
            double lr[NQ][D], lG[DD] = {};
            for (int q = 0; q < NQ; ++q)
                for (int a = 0; a < D; ++a) {
                    double s = 0.0;
                    for (int b = 0; b < D; ++b) s += Gi[a * D + b] * lgs[q][b];
                    lr[q][a] = s;
                }
            for (int q = 0; q < NQ; ++q)
                for (int a = 0; a < D; ++a)
                    for (int b = 0; b < D; ++b) lG[a * D + b] -= lr[q][a] * gs[q][b];
            // the -w_k q_c terms of r summed over k: lw_k += lwq (the same for every k), and
            // lq_c -= lr_q . sum_k w_k
            double lwq[D] = {}, wsum[D] = {};
            for (int q = 0; q < NQ; ++q)
                for (int a = 0; a < D; ++a) lwq[a] -= lr[q][a] * qc[q];
            for (int k = 0; k < NV; ++k) {
                const double nk = mom(k, Q::M_N);
                double S1[D], w[D], lS1[D] = {}, lw[D] = {}, lS2[NS] = {}, ln_ = 0.0;
                for (int a = 0; a < D; ++a) {
                    S1[a] = mom(k, Q::M_S1 + a);
                    w[a] = S1[a] + nk * dk[k][a];
                }
                // G += S2 + S1 d^t + d w^t
                for (int a = 0; a < D; ++a)
                    for (int b = 0; b < D; ++b) {
                        const double l = lG[a * D + b];
                        lS2[sym<D>(a, b)] += l;
                        lS1[a] += l * dk[k][b];
                        ldk[k][b] += l * S1[a];
                        ldk[k][a] += l * w[b];
                        lw[b] += l * dk[k][a];
                    }
                // r_q += T_q + d U_q - w q_c
                for (int q = 0; q < NQ; ++q) {
                    const double Uq = mom(k, Q::M_U + q);
                    double lU = 0.0;
                    for (int a = 0; a < D; ++a) {
                        const double l = lr[q][a];
                        mout(k, Q::M_T + q * D + a, l);
                        ldk[k][a] += l * Uq;
                        lU += l * dk[k][a];
                    }
                    mout(k, Q::M_U + q, lU);
                }
                for (int a = 0; a < D; ++a) {
                    lw[a] += lwq[a];
                    wsum[a] += w[a];
                }
                // w = S1 + n d
                for (int a = 0; a < D; ++a) {
                    lS1[a] += lw[a];
                    ldk[k][a] += nk * lw[a];
                    ln_ += lw[a] * dk[k][a];
                }
                for (int a = 0; a < D; ++a) mout(k, Q::M_S1 + a, lS1[a]);
                for (int s2 = 0; s2 < NS; ++s2) mout(k, Q::M_S2 + s2, lS2[s2]);
                mout(k, Q::M_N, ln_);
            }
            for (int q = 0; q < NQ; ++q) {
                double lq = 0.0;
                for (int a = 0; a < D; ++a) lq -= lr[q][a] * wsum[a];
                if (q < D) lvc[q] += lq;
                else lFc[q - D] += lq;
            }
        } else {
            zero_moments();
        }
        // d_k = xs_k - xcc
        for (int k = 0; k < NV; ++k)
            for (int a = 0; a < D; ++a) {
                lxs[k * D + a] += ldk[k][a];
                lxcc[a] -= ldk[k][a];
            }
    }
    // ---- M_k = sum_{f != k} W_f;  W_f = (z / |u_f|) u_f u_f^t, u_f = N_f / D
    for (int f = 0; f < NV; ++f) {
        double lW[NS] = {}, u[D];
        for (int k = 0; k < NV; ++k)
            if (k != f)
                for (int s2 = 0; s2 < NS; ++s2) lW[s2] += lM[k * NS + s2];
        for (int a = 0; a < D; ++a) u[a] = N[f * D + a] * (1.0 / D);
        // full symmetric lW: stored entry s = (a <= b) used once
        double uWu = 0.0, lWu[D] = {};
        for (int a = 0; a < D; ++a)
            for (int b = a; b < D; ++b) {
                const double l = lW[sym<D>(a, b)];
                uWu += l * u[a] * u[b];
                lWu[a] += l * u[b];
                lWu[b] += l * u[a];
            }
        lz += uWu * inu[f];
        const double c1 = z * inu[f], c3 = c1 * inu[f] * inu[f];
        for (int a = 0; a < D; ++a) lN[f * D + a] += (c1 * lWu[a] - c3 * uWu * u[a]) * (1.0 / D);
    }
    // ---- geometry: N(xs), xcc = mean(xs)
    faces_vjp<D>(xs, 0.0, lN, lxs);
    for (int k = 0; k < NV; ++k)
        for (int a = 0; a < D; ++a) lxs[k * D + a] += lxcc[a] * (1.0 / NV);
}

// ---------------------------------------------------------------------------------------
// Cell update (pure form of k_update for orders 1 and 2): inputs xs0, xs1, vs, vp0, vp1
// [NV][D] at the cell's nodes, packets M [NV][NS], R [NV][D], v [D], F [DD], m, 1/m, mu,
// kappa, dt, ord. Outputs v1 [D], F1 [DD], z1 (impedance of the new state).
// ---------------------------------------------------------------------------------------
template <int D>
LMOOD_HD void update_fw(const double *xs0, const double *xs1, const double *vs, const double *vp0, const double *vp1,
                        const double *M, const double *R, const double *v, const double *F, double m, double im,
                        double mu, double kap, double dt, int ord, double *v1, double *F1, double &z1) {
    using Q = Sz<D>;
    constexpr int NV = Q::NV, DD = Q::DD, NS = Q::NS;
    double sf[D] = {};
    for (int k = 0; k < NV; ++k)
        for (int a = 0; a < D; ++a) {
            double s = -R[k * D + a];
            for (int b = 0; b < D; ++b) s += M[k * NS + sym<D>(a, b)] * vs[k * D + b];
            sf[a] += s;
        }
    for (int a = 0; a < D; ++a) v1[a] = v[a] + dt * im * sf[a];
    double V0, N0[NV * D], V1, N1[NV * D];
    faces<D>(xs0, V0, N0);
    faces<D>(xs1, V1, N1);
    if (ord != 1) {
        double L0[DD], L1[DD], A[DD], Bm[DD], Ai[DD], Rm[DD];
        velgrad<D>(vp0, N0, V0, L0);
        velgrad<D>(vp1, N1, V1, L1);
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) {
                A[i * D + j] = (i == j ? 1.0 : 0.0) - 0.5 * dt * L1[i * D + j];
                Bm[i * D + j] = (i == j ? 1.0 : 0.0) + 0.5 * dt * L0[i * D + j];
            }
        mm<D>(Bm, F, Rm);
        inverse<D>(A, Ai);
        mm<D>(Ai, Rm, F1);
    } else {
        double Ls[DD], LF[DD];
        velgrad<D>(vs, N0, V0, Ls);
        mm<D>(Ls, F, LF);
        for (int q = 0; q < DD; ++q) F1[q] = F[q] + dt * LF[q];
    }
    z1 = impedance<D>(F1, m / V1, mu, kap);
}

// Product of update_fw: (lv1, lF1, lz1) -> accumulates lxs0, lxs1, lvs, lvp0, lvp1 [NV][D],
// lM [NV][NS], lR [NV][D], lv [D], lF [DD], lmu, lkap. Recomputes only what the product
// needs (F1 and the impedance term only where used; lz1 = 0 drops the impedance).
template <int D>
LMOOD_HD void update_vjp(const double *xs0, const double *xs1, const double *vs, const double *vp0, const double *vp1,
                         const double *M, const double *R, const double *v, const double *F, double m, double im,
                         double mu, double kap, double dt, int ord, const double *lv1, const double *lF1_in, double lz1,
                         double *lxs0, double *lxs1, double *lvs, double *lvp0, double *lvp1, double *lM, double *lR,
                         double *lv, double *lF, double &lmu, double &lkap) {
    using Q = Sz<D>;
    constexpr int NV = Q::NV, DD = Q::DD, NS = Q::NS;
    (void)R;
    (void)v;
    double V0, N0[NV * D], V1, N1[NV * D], lN0[NV * D] = {}, lN1[NV * D] = {}, lV0 = 0.0, lV1 = 0.0;
    faces<D>(xs0, V0, N0);
    faces<D>(xs1, V1, N1);
    const double iV0 = 1.0 / V0, iV1 = 1.0 / V1;
    double lF1[DD];
    for (int q = 0; q < DD; ++q) lF1[q] = lF1_in[q];
    if (ord != 1) {
        double L0[DD], L1[DD], A[DD], Bm[DD], Ai[DD], Rm[DD], F1[DD];
        velgrad_iv<D>(vp0, N0, iV0, L0);
        velgrad_iv<D>(vp1, N1, iV1, L1);
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) {
                A[i * D + j] = (i == j ? 1.0 : 0.0) - 0.5 * dt * L1[i * D + j];
                Bm[i * D + j] = (i == j ? 1.0 : 0.0) + 0.5 * dt * L0[i * D + j];
            }
        mm<D>(Bm, F, Rm);
        inverse<D>(A, Ai);
        mm<D>(Ai, Rm, F1);
        if (lz1 != 0.0) {  // z1 = Z(F1, m / V1)
            double lrho = 0.0;
            impedance_vjp<D>(F1, m * iV1, mu, kap, lz1, lF1, lrho, lmu, lkap);
            lV1 -= lrho * m * iV1 * iV1;
        }
        // F1 = Ai Rm, Rm = Bm F
        double lRm[DD], lA[DD], lBm[DD], t[DD], lL0[DD], lL1[DD];
        mtm<D>(Ai, lF1, lRm);       // lRm = Ai^t lF1
        mmt<D>(lRm, F1, lA);        // lA = -lRm F1^t
        mmt<D>(lRm, F, lBm);        // lBm = lRm F^t
        mtm<D>(Bm, lRm, t);         // lF += Bm^t lRm
        for (int q = 0; q < DD; ++q) {
            lF[q] += t[q];
            lL1[q] = 0.5 * dt * lA[q];  // A = I - dt/2 L1, lA was -(...) -> +dt/2
            lL0[q] = 0.5 * dt * lBm[q];
        }
        velgrad_vjp_iv<D>(vp1, N1, iV1, L1, lL1, lvp1, lN1, lV1);
        velgrad_vjp_iv<D>(vp0, N0, iV0, L0, lL0, lvp0, lN0, lV0);
    } else {
        double Ls[DD], t[DD], lLs[DD];
        velgrad_iv<D>(vs, N0, iV0, Ls);
        if (lz1 != 0.0) {
            double LF[DD], F1[DD], lrho = 0.0;
            mm<D>(Ls, F, LF);
            for (int q = 0; q < DD; ++q) F1[q] = F[q] + dt * LF[q];
            impedance_vjp<D>(F1, m * iV1, mu, kap, lz1, lF1, lrho, lmu, lkap);
            lV1 -= lrho * m * iV1 * iV1;
        }
        mtm<D>(Ls, lF1, t);
        for (int q = 0; q < DD; ++q) lF[q] += lF1[q] + dt * t[q];
        mmt<D>(lF1, F, lLs);
        for (int q = 0; q < DD; ++q) lLs[q] *= dt;
        velgrad_vjp_iv<D>(vs, N0, iV0, Ls, lLs, lvs, lN0, lV0);
    }
    faces_vjp<D>(xs0, lV0, lN0, lxs0);
    faces_vjp<D>(xs1, lV1, lN1, lxs1);
    // v1 = v + dt im sum_k (M_k vs_k - R_k)
    for (int a = 0; a < D; ++a) lv[a] += lv1[a];
    for (int k = 0; k < NV; ++k)
        for (int a = 0; a < D; ++a) {
            const double lf = dt * im * lv1[a];
            lR[k * D + a] -= lf;
            for (int b = 0; b < D; ++b) {
                lM[k * NS + sym<D>(a, b)] += lf * vs[k * D + b];
                lvs[k * D + b] += M[k * NS + sym<D>(a, b)] * lf;
            }
        }
}

// Node moments: product for one corner (node p, cell c'): with dx = x_c' - x_p, accumulate
// the adjoints of x_c' (lxc), of (v, F) of c' (lq [NQ]) and of x_p (lxp) from the adjoints of
// node p's moments, read through lmom(j), j < NMOM.
template <int D, class LM>
LMOOD_HD void moments_corner_vjp(LM &&lmom, const double *xc, const double *xp, const double *q, double *lxc,
                                 double *lq, double *lxp) {
    using Q = Sz<D>;
    constexpr int NQ = Q::NQ;
    double dx[D], ldx[D];
    for (int a = 0; a < D; ++a) {
        dx[a] = xc[a] - xp[a];
        ldx[a] = lmom(Q::M_S1 + a);
    }
    for (int a = 0; a < D; ++a)
        for (int b = a; b < D; ++b) {
            const double l = lmom(Q::M_S2 + sym<D>(a, b));
            ldx[a] += l * dx[b];
            ldx[b] += l * dx[a];
        }
    for (int qi = 0; qi < NQ; ++qi) {
        double lqq = lmom(Q::M_U + qi);
        for (int a = 0; a < D; ++a) {
            const double l = lmom(Q::M_T + qi * D + a);
            lqq += l * dx[a];
            ldx[a] += l * q[qi];
        }
        lq[qi] += lqq;
    }
    for (int a = 0; a < D; ++a) {
        lxc[a] += ldx[a];
        lxp[a] -= ldx[a];
    }
}

}  // namespace adj
}  // namespace lmood
