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

// The same product for a rank-one adjoint lT = l n^t, the form in which the predictor's
// packets and dv/dt use the stress (T n): with u = F^t n and v = F^t l, lT : B = u . v and
// (lB + lB^t) F = cj (l u^t + n v^t) for lB = cj l n^t, so B = F F^t is never formed
// (tr B = |F|^2, plus 1 for the plane-strain F33). Tl_out (may be NULL) receives T l (= l^t T,
// T symmetric).
template <int D>
LMOOD_HD void stress_vjp_r1(const double *F, double mu, double kap, const double *l, const double *n, double *lF,
                            double &lmu, double &lkap, double *Tl_out = nullptr) {
    double C[D * D];
    cofactor<D>(F, C);
    double J = 0.0;
    for (int b = 0; b < D; ++b) J += F[b] * C[b];  // det F along the first row
    const double lJ = adj_log(J), rc = adj_rcbrt(J), Jm23 = rc * rc, invJ = Jm23 * rc;
    const double J53 = invJ * Jm23, cj = mu * J53;
    double u[D], v[D], tr = D == 2 ? 1.0 : 0.0, ln = 0.0, uv = 0.0;
    for (int j = 0; j < D; ++j) {
        double su = 0.0, sv = 0.0;
        for (int i = 0; i < D; ++i) {
            su += F[i * D + j] * n[i];
            sv += F[i * D + j] * l[i];
        }
        u[j] = su;
        v[j] = sv;
        uv += su * sv;
        ln += l[j] * n[j];
    }
    for (int q = 0; q < D * D; ++q) tr += F[q] * F[q];
    const double p0 = J - 1.0 + lJ * invJ;  // p = -(kap/2) p0
    if (Tl_out) {
        const double diag = 0.5 * kap * p0 - cj * tr * (1.0 / 3.0);
        for (int i = 0; i < D; ++i) {
            double s = 0.0;
            for (int j = 0; j < D; ++j) s += F[i * D + j] * v[j];  // (B l)_i
            Tl_out[i] = cj * s + diag * l[i];
        }
    }
    // T = cj B + diag I, diag = -p - cj tr / 3: lcj = u . v - (l . n) tr / 3, lp = -(l . n),
    // ltr = -(l . n) cj / 3
    const double lcj = uv - ln * tr * (1.0 / 3.0), ltr2 = -ln * cj * (2.0 / 3.0);
    lmu += lcj * J53;
    lkap += ln * 0.5 * p0;
    const double lJv = lcj * (-5.0 / 3.0) * cj * invJ + ln * 0.5 * kap * (1.0 + (1.0 - lJ) * invJ * invJ);
    for (int i = 0; i < D; ++i) {
        const double cl = cj * l[i], cn = cj * n[i];
        for (int j = 0; j < D; ++j)
            lF[i * D + j] += cl * u[j] + cn * v[j] + ltr2 * F[i * D + j] + lJv * C[i * D + j];
    }
}

// ---------------------------------------------------------------------------------------
// Stress of the shear energy family (Eq. familiy_energies with the volumetric part of Eq.
// EOS_neoHook; a = -1 is the neo-Hookean law above): with Bbar = J^{-2/3} F F^t (plane strain
// in 2D), I1 = tr Bbar, I2 = (I1^2 - tr Bbar^2) / 2,
//   T = -p I + (mu / J) dev(c1 Bbar - c2 Bbar^2),  c1 = -a + (1 + a) I1 I2 / 3,
//   c2 = (1 + a) I2 / 3,  p = -(kap/2)(J - 1 + log J / J),
// and its product lamT -> (lamF, lam_mu, lam_kappa). Worked in 3 x 3 (2D: F33 = 1, the
// in-plane block of T and of lamT).
// ---------------------------------------------------------------------------------------
struct FamStress {
    double J, invJ, lJ, Jm23, B[9], B2[9], I1, I2, c1, c2, X[9], trX, p;
};

template <int D> LMOOD_HD void family_parts(const double *F, double mu, double kap, double a, FamStress &q) {
    double F3[9];
    for (int i = 0; i < 9; ++i) F3[i] = 0.0;
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) F3[i * 3 + j] = F[i * D + j];
    if (D == 2) F3[8] = 1.0;
    q.J = det<3>(F3);
    const double rc = adj_rcbrt(q.J);
    q.Jm23 = rc * rc;
    q.invJ = q.Jm23 * rc;
    q.lJ = adj_log(q.J);
    double C[9];
    mmt<3>(F3, F3, C);
    for (int i = 0; i < 9; ++i) q.B[i] = q.Jm23 * C[i];
    mm<3>(q.B, q.B, q.B2);
    q.I1 = q.B[0] + q.B[4] + q.B[8];
    q.I2 = 0.5 * (q.I1 * q.I1 - (q.B2[0] + q.B2[4] + q.B2[8]));
    q.c1 = -a + (1.0 + a) * q.I1 * q.I2 * (1.0 / 3.0);
    q.c2 = (1.0 + a) * q.I2 * (1.0 / 3.0);
    for (int i = 0; i < 9; ++i) q.X[i] = q.c1 * q.B[i] - q.c2 * q.B2[i];
    q.trX = q.X[0] + q.X[4] + q.X[8];
    q.p = -0.5 * kap * (q.J - 1.0 + q.lJ * q.invJ);
    (void)mu;
}

template <int D> LMOOD_HD void stress_family_fw(const double *F, double mu, double kap, double a, double *T) {
    FamStress q;
    family_parts<D>(F, mu, kap, a, q);
    const double s = mu * q.invJ;
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j)
            T[i * D + j] = (i == j ? -q.p - s * q.trX * (1.0 / 3.0) : 0.0) + s * q.X[i * 3 + j];
}

template <int D>
LMOOD_HD void stress_family_vjp(const double *F, double mu, double kap, double a, const double *lT, double *lF,
                                double &lmu, double &lkap, double *T_out = nullptr) {
    FamStress q;
    family_parts<D>(F, mu, kap, a, q);
    const double s = mu * q.invJ;
    if (T_out)
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j)
                T_out[i * D + j] = (i == j ? -q.p - s * q.trX * (1.0 / 3.0) : 0.0) + s * q.X[i * 3 + j];
    // lamT in 3 x 3 (zero outside the in-plane block in 2D); Y = dev(lamT)
    double Y[9], tr = 0.0;
    for (int i = 0; i < 9; ++i) Y[i] = 0.0;
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) Y[i * 3 + j] = lT[i * D + j];
    for (int i = 0; i < 3; ++i) tr += Y[i * 4];
    const double lp = -tr;  // T = -p I + ...
    for (int i = 0; i < 3; ++i) Y[i * 4] -= tr * (1.0 / 3.0);
    double YX = 0.0;
    for (int i = 0; i < 9; ++i) YX += Y[i] * q.X[i];
    // s dev(X): lX = s Y, ls = <Y, X>, s = mu / J
    lmu += YX * q.invJ;
    double lJv = -s * YX * q.invJ;
    // p = -(kap/2)(J - 1 + log J / J)
    lkap += lp * (-0.5) * (q.J - 1.0 + q.lJ * q.invJ);
    lJv += lp * (-0.5 * kap) * (1.0 + (1.0 - q.lJ) * q.invJ * q.invJ);
    // X = c1 B - c2 B^2 (B symmetric)
    double lc1 = 0.0, lc2 = 0.0, lB[9], lXB[9], BlX[9];
    for (int i = 0; i < 9; ++i) {
        lc1 += s * Y[i] * q.B[i];
        lc2 -= s * Y[i] * q.B2[i];
    }
    double lX[9];
    for (int i = 0; i < 9; ++i) lX[i] = s * Y[i];
    mm<3>(lX, q.B, lXB);
    mm<3>(q.B, lX, BlX);
    for (int i = 0; i < 9; ++i) lB[i] = q.c1 * lX[i] - q.c2 * (lXB[i] + BlX[i]);
    // c1 = -a + (1+a) I1 I2 / 3, c2 = (1+a) I2 / 3; I2 = (I1^2 - tr B^2) / 2; I1 = tr B
    const double ap = (1.0 + a) * (1.0 / 3.0);
    const double lI2 = lc1 * ap * q.I1 + lc2 * ap;
    const double lI1 = lc1 * ap * q.I2 + lI2 * q.I1;
    for (int i = 0; i < 9; ++i) lB[i] -= lI2 * q.B[i];
    for (int i = 0; i < 3; ++i) lB[i * 4] += lI1;
    // B = J^{-2/3} F F^t: lC = J^{-2/3} lB, lJ -= (2 / (3 J)) <lB, B>
    double lBB = 0.0;
    for (int i = 0; i < 9; ++i) lBB += lB[i] * q.B[i];
    lJv -= (2.0 / 3.0) * q.invJ * lBB;
    // lF3 = J^{-2/3} (lB + lB^t) F3 + lJ cof(F3); the in-plane block in 2D
    double F3[9], Cf[9];
    for (int i = 0; i < 9; ++i) F3[i] = 0.0;
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) F3[i * 3 + j] = F[i * D + j];
    if (D == 2) F3[8] = 1.0;
    cofactor<3>(F3, Cf);
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            double t = 0.0;
            for (int k = 0; k < 3; ++k) t += (lB[i * 3 + k] + lB[k * 3 + i]) * F3[k * 3 + j];
            lF[i * D + j] += q.Jm23 * t + lJv * Cf[i * 3 + j];
        }
}

// the material's stress and product: the neo-Hookean law (a = -1) or the family
template <int D> LMOOD_HD void stress_m(const double *F, double mu, double kap, double a, double *T) {
    if (a == -1.0) stress<D>(F, mu, kap, T);
    else stress_family_fw<D>(F, mu, kap, a, T);
}

template <int D>
LMOOD_HD void stress_m_vjp(const double *F, double mu, double kap, double a, const double *lT, double *lF, double &lmu,
                           double &lkap, double *T_out = nullptr) {
    if (a == -1.0) stress_vjp<D>(F, mu, kap, lT, lF, lmu, lkap, T_out);
    else stress_family_vjp<D>(F, mu, kap, a, lT, lF, lmu, lkap, T_out);
}

// ---------------------------------------------------------------------------------------
// Stiffened gas (Eq. EOS_stiffened_gas, incomplete form): p = (gam - 1) (rho0 / J)
// (eps - Psi_s(F)) - gam pinf with Psi_s the shear energy of the family (a = -1: the
// neo-Hookean one) and eps the specific internal energy; T = -p I + the shear stress
// (kappa = 0); impedance z = sqrt(rho (gam (p + pinf) + 4 mu / (3 J))). With their products.
// ---------------------------------------------------------------------------------------
struct SgMat {
    double gam, pinf, rho0;
};

// Psi_s = mu / (4 rho0) (-2a (I1 - 3) + (1 + a)/3 (I2^2 - 9)) of Bbar (a = -1: mu / (2 rho0)
// (I1 - 3)); the product l -> lF, lmu
template <int D> LMOOD_HD double shear_energy_a(const double *F, double rho0, double mu, double a) {
    FamStress q;
    family_parts<D>(F, mu, 0.0, a, q);
    return mu / (4.0 * rho0) * (-2.0 * a * (q.I1 - 3.0) + (1.0 + a) * (1.0 / 3.0) * (q.I2 * q.I2 - 9.0));
}

template <int D>
LMOOD_HD void shear_energy_a_vjp(const double *F, double rho0, double mu, double a, double l, double *lF, double &lmu) {
    FamStress q;
    family_parts<D>(F, mu, 0.0, a, q);
    const double g = -2.0 * a * (q.I1 - 3.0) + (1.0 + a) * (1.0 / 3.0) * (q.I2 * q.I2 - 9.0);
    lmu += l * g / (4.0 * rho0);
    const double lg = l * mu / (4.0 * rho0);
    const double lI2 = lg * (2.0 / 3.0) * (1.0 + a) * q.I2;
    const double lI1 = lg * (-2.0 * a) + lI2 * q.I1;
    double lB[9], lBB = 0.0;
    for (int i = 0; i < 9; ++i) lB[i] = -lI2 * q.B[i];
    for (int i = 0; i < 3; ++i) lB[i * 4] += lI1;
    for (int i = 0; i < 9; ++i) lBB += lB[i] * q.B[i];
    const double lJv = -(2.0 / 3.0) * q.invJ * lBB;
    double F3[9], Cf[9];
    for (int i = 0; i < 9; ++i) F3[i] = 0.0;
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) F3[i * 3 + j] = F[i * D + j];
    if (D == 2) F3[8] = 1.0;
    cofactor<3>(F3, Cf);
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            double t = 0.0;
            for (int k = 0; k < 3; ++k) t += (lB[i * 3 + k] + lB[k * 3 + i]) * F3[k * 3 + j];
            lF[i * D + j] += q.Jm23 * t + lJv * Cf[i * 3 + j];
        }
}

template <int D>
LMOOD_HD double sg_pressure_a(const double *F, double mu, double a, const SgMat &sg, double eps) {
    return (sg.gam - 1.0) * (sg.rho0 / det<D>(F)) * (eps - shear_energy_a<D>(F, sg.rho0, mu, a)) - sg.gam * sg.pinf;
}

// product of p: lp -> lF, lmu, leps
template <int D>
LMOOD_HD void sg_pressure_a_vjp(const double *F, double mu, double a, const SgMat &sg, double eps, double lp,
                                double *lF, double &lmu, double &leps) {
    const double J = det<D>(F), iJ = 1.0 / J, k = (sg.gam - 1.0) * sg.rho0 * iJ;
    const double psi = shear_energy_a<D>(F, sg.rho0, mu, a);
    leps += lp * k;
    shear_energy_a_vjp<D>(F, sg.rho0, mu, a, -lp * k, lF, lmu);
    const double lJ = -lp * k * (eps - psi) * iJ;
    double C[D * D];
    cofactor<D>(F, C);
    for (int i = 0; i < D * D; ++i) lF[i] += lJ * C[i];
}

template <int D>
LMOOD_HD void stress_sg_a(const double *F, double mu, double a, const SgMat &sg, double eps, double *T) {
    stress_m<D>(F, mu, 0.0, a, T);
    const double p = sg_pressure_a<D>(F, mu, a, sg, eps);
    for (int i = 0; i < D; ++i) T[i * D + i] -= p;
}

template <int D>
LMOOD_HD void stress_sg_a_vjp(const double *F, double mu, double a, const SgMat &sg, double eps, const double *lT,
                              double *lF, double &lmu, double &leps, double *T_out = nullptr) {
    double lkap = 0.0;
    stress_m_vjp<D>(F, mu, 0.0, a, lT, lF, lmu, lkap, T_out);
    double lp = 0.0;
    for (int i = 0; i < D; ++i) lp -= lT[i * D + i];
    sg_pressure_a_vjp<D>(F, mu, a, sg, eps, lp, lF, lmu, leps);
    if (T_out) {
        const double p = sg_pressure_a<D>(F, mu, a, sg, eps);
        for (int i = 0; i < D; ++i) T_out[i * D + i] -= p;
    }
}

template <int D>
LMOOD_HD double impedance_sg_a(const double *F, double rho, double mu, double a, const SgMat &sg, double eps) {
    const double p = sg_pressure_a<D>(F, mu, a, sg, eps);
    return sqrt(rho * (sg.gam * (p + sg.pinf) + (4.0 / 3.0) * mu / det<D>(F)));
}

// product of z: lz -> lF, lrho, lmu, leps
template <int D>
LMOOD_HD void impedance_sg_a_vjp(const double *F, double rho, double mu, double a, const SgMat &sg, double eps,
                                 double lz, double *lF, double &lrho, double &lmu, double &leps) {
    const double J = det<D>(F), iJ = 1.0 / J;
    const double p = sg_pressure_a<D>(F, mu, a, sg, eps);
    const double Y = sg.gam * (p + sg.pinf) + (4.0 / 3.0) * mu * iJ;
    const double z = sqrt(rho * Y), lX = lz * 0.5 / z;
    lrho += lX * Y;
    const double lY = lX * rho;
    lmu += lY * (4.0 / 3.0) * iJ;
    const double lJ = -lY * (4.0 / 3.0) * mu * iJ * iJ;
    double C[D * D];
    cofactor<D>(F, C);
    for (int i = 0; i < D * D; ++i) lF[i] += lJ * C[i];
    sg_pressure_a_vjp<D>(F, mu, a, sg, eps, lY * sg.gam, lF, lmu, leps);
}

// the material's stress with the energy: the stiffened gas when sg is given, else stress_m
template <int D>
LMOOD_HD void stress_x(const double *F, double mu, double kap, double a, const SgMat *sg, double eps, double *T) {
    if (sg) stress_sg_a<D>(F, mu, a, *sg, eps, T);
    else stress_m<D>(F, mu, kap, a, T);
}

template <int D>
LMOOD_HD void stress_x_vjp(const double *F, double mu, double kap, double a, const SgMat *sg, double eps,
                           const double *lT, double *lF, double &lmu, double &lkap, double &leps,
                           double *T_out = nullptr) {
    if (sg) stress_sg_a_vjp<D>(F, mu, a, *sg, eps, lT, lF, lmu, leps, T_out);
    else stress_m_vjp<D>(F, mu, kap, a, lT, lF, lmu, lkap, T_out);
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

// product of faces at xs, with N = faces(xs) already formed by the caller
template <int D> LMOOD_HD void faces_vjp_n(const double *xs, const double *N, double lV, const double *lN, double *lxs) {
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

template <int D> LMOOD_HD void faces_vjp(const double *xs, double lV, const double *lN, double *lxs) {
    double V, N[(D + 1) * D];
    faces<D>(xs, V, N);
    faces_vjp_n<D>(xs, N, lV, lN, lxs);
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
// the Galerkin solve on ND free directions t_i: v = sum_i al_i t_i, (t_i . M t_j) al = t_i . b
// (ND a compile-time count, so that the small arrays stay in registers)
template <int D, int ND>
LMOOD_HD void node_solve_proj(const double *M, const double *b, const double *t /*[2][3]*/, double *v) {
    double A[ND * ND], r[ND], al[ND];
    for (int i = 0; i < ND; ++i) {
        double s = 0.0;
        for (int a = 0; a < D; ++a) s += t[i * 3 + a] * b[a];
        r[i] = s;
        for (int j = 0; j < ND; ++j) {
            double q = 0.0;
            for (int a = 0; a < D; ++a)
                for (int c = 0; c < D; ++c) q += t[i * 3 + a] * M[a * D + c] * t[j * 3 + c];
            A[i * ND + j] = q;
        }
    }
    if constexpr (ND == 1) {
        al[0] = r[0] / A[0];
    } else {
        const double dA = A[0] * A[3] - A[1] * A[2];
        al[0] = (A[3] * r[0] - A[1] * r[1]) / dA;
        al[1] = (-A[2] * r[0] + A[0] * r[1]) / dA;
    }
    for (int a = 0; a < D; ++a) {
        double s = 0.0;
        for (int i = 0; i < ND; ++i) s += al[i] * t[i * 3 + a];
        v[a] = s;
    }
}

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
    } else if (nd == 1) {
        node_solve_proj<D, 1>(M, b, t, v);
    } else {
        node_solve_proj<D, 2>(M, b, t, v);
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
// Boundary faces of the nodal solve. bface_area: the outward area vector of a boundary face
// from its D nodes xq [D][D] (2D edge (q0, q1): (y1 - y0, x0 - x1); 3D triangle:
// (1/2) (x1 - x0) x (x2 - x0)); bface_area_vjp accumulates lxq from lN.
// ---------------------------------------------------------------------------------------
template <int D> LMOOD_HD void bface_area(const double *xq, double *N) {
    if constexpr (D == 2) {
        N[0] = xq[3] - xq[1];
        N[1] = xq[0] - xq[2];
    } else {
        double u[3], w[3];
        for (int a = 0; a < 3; ++a) {
            u[a] = xq[3 + a] - xq[a];
            w[a] = xq[6 + a] - xq[a];
        }
        N[0] = 0.5 * (u[1] * w[2] - u[2] * w[1]);
        N[1] = 0.5 * (u[2] * w[0] - u[0] * w[2]);
        N[2] = 0.5 * (u[0] * w[1] - u[1] * w[0]);
    }
}

template <int D> LMOOD_HD void bface_area_vjp(const double *xq, const double *lN, double *lxq) {
    if constexpr (D == 2) {
        lxq[3] += lN[0];
        lxq[1] -= lN[0];
        lxq[0] += lN[1];
        lxq[2] -= lN[1];
    } else {
        double u[3], w[3];
        for (int a = 0; a < 3; ++a) {
            u[a] = xq[3 + a] - xq[a];
            w[a] = xq[6 + a] - xq[a];
        }
        // N = (1/2) u x w: lu = (1/2) w x lN, lw = (1/2) lN x u
        const double lu[3] = {0.5 * (w[1] * lN[2] - w[2] * lN[1]), 0.5 * (w[2] * lN[0] - w[0] * lN[2]),
                              0.5 * (w[0] * lN[1] - w[1] * lN[0])};
        const double lw[3] = {0.5 * (lN[1] * u[2] - lN[2] * u[1]), 0.5 * (lN[2] * u[0] - lN[0] * u[2]),
                              0.5 * (lN[0] * u[1] - lN[1] * u[0])};
        for (int a = 0; a < 3; ++a) {
            lxq[3 + a] += lu[a];
            lxq[6 + a] += lw[a];
            lxq[a] -= lu[a] + lw[a];
        }
    }
}

// ---------------------------------------------------------------------------------------
// Nodal solve with traction, pressure and prescribed-velocity faces and contact walls (Eqs.
// pBC, vBC1, vBC; Sect. "Boundary condition treatments"), pure form. b0: the corners' sum;
// the node's boundary faces j < nf are read through fc(j, tag, N, val) (N [D] the face's
// outward area vector at x^n, val [D] its value: traction vector, pressure in val[0],
// prescribed velocity; faces of other tags are skipped) when ext; walls: nw planes (point,
// unit normal into the body) [nw][2D], threshold eps, the node's position xp. v = K b with
// b = b0 + the traction and pressure forces (each face's share N / D), then the multiplier
// step v -= T K d, T = (v . d - g) / (d . K d) of the velocity faces (d = sum N / D, g = sum
// val . N / D), then the same step with d = n, g = 0 for each wall the node is within eps of
// and moving into.
// ---------------------------------------------------------------------------------------
template <int D> struct BcSolve {
    double b[D], v0[D], dv[D], gsum, w1[D], wd, T1, v[D];
    bool p1;
    bool act[kMaxContact];
    double vb[kMaxContact][D], ww[kMaxContact][D], Tw[kMaxContact], wn[kMaxContact];
};

template <int D, class FC>
LMOOD_HD void node_solve_bc_fw(const double *M, const double *b0, int nd, const double *t, bool ext, int nf, FC &&fc,
                               int nw, const double *planes, double eps, const double *xp, BcSolve<D> &r) {
    int nvel = 0;
    r.gsum = 0.0;
    for (int a = 0; a < D; ++a) {
        r.b[a] = b0[a];
        r.dv[a] = 0.0;
    }
    if (ext)
        for (int j = 0; j < nf; ++j) {
            int tag;
            double N[D], val[D];
            fc(j, tag, N, val);
            if (tag == TAG_TRACTION) {
                double ar = 0.0;
                for (int a = 0; a < D; ++a) ar += N[a] * N[a];
                ar = sqrt(ar) * (1.0 / D);
                for (int a = 0; a < D; ++a) r.b[a] += ar * val[a];
            } else if (tag == TAG_PRESSURE) {
                for (int a = 0; a < D; ++a) r.b[a] -= val[0] * N[a] * (1.0 / D);
            } else if (tag == TAG_VELOCITY) {
                for (int a = 0; a < D; ++a) {
                    r.dv[a] += N[a] * (1.0 / D);
                    r.gsum += val[a] * N[a] * (1.0 / D);
                }
                ++nvel;
            }
        }
    node_solve<D>(M, r.b, nd, t, r.v0);
    for (int a = 0; a < D; ++a) r.v[a] = r.v0[a];
    r.p1 = false;
    if (nvel > 0) {
        node_solve<D>(M, r.dv, nd, t, r.w1);
        double wd = 0.0, vd = 0.0;
        for (int a = 0; a < D; ++a) {
            wd += r.w1[a] * r.dv[a];
            vd += r.v0[a] * r.dv[a];
        }
        if (wd > 0.0) {
            r.p1 = true;
            r.wd = wd;
            r.T1 = (vd - r.gsum) / wd;
            for (int a = 0; a < D; ++a) r.v[a] -= r.T1 * r.w1[a];
        }
    }
    for (int k = 0; k < kMaxContact; ++k) {
        r.act[k] = false;
        if (k >= nw) continue;
        const double *P = planes + 2 * D * k, *n = P + D;
        double dist = 0.0, vn = 0.0;
        for (int a = 0; a < D; ++a) {
            dist += n[a] * (xp[a] - P[a]);
            vn += n[a] * r.v[a];
        }
        if (!(dist < eps && vn < 0.0)) continue;
        double w[D], wn = 0.0;
        node_solve<D>(M, n, nd, t, w);
        for (int a = 0; a < D; ++a) wn += w[a] * n[a];
        if (wn > 0.0) {
            r.act[k] = true;
            r.wn[k] = wn;
            r.Tw[k] = vn / wn;
            for (int a = 0; a < D; ++a) {
                r.vb[k][a] = r.v[a];
                r.ww[k][a] = w[a];
                r.v[a] -= r.Tw[k] * w[a];
            }
        }
    }
}

template <int D, class FC>
LMOOD_HD void node_solve_bc(const double *M, const double *b0, int nd, const double *t, bool ext, int nf, FC &&fc,
                            int nw, const double *planes, double eps, const double *xp, double *v) {
    BcSolve<D> r;
    node_solve_bc_fw<D>(M, b0, nd, t, ext, nf, fc, nw, planes, eps, xp, r);
    for (int a = 0; a < D; ++a) v[a] = r.v[a];
}

// Product: lv -> lb [D] (the adjoint of b0), lM (full D x D, accumulated), and ln(j, lN) for
// every face j < nf (lN [D] the adjoint of its area vector; zero for faces of other tags).
// The walls a node is in contact with, and whether each multiplier step applies, are those
// of the forward evaluation (a frozen active set, like the MOOD mask).
template <int D, class FC, class LN>
LMOOD_HD void node_solve_bc_vjp(const double *M, const double *b0, int nd, const double *t, bool ext, int nf, FC &&fc,
                                int nw, const double *planes, double eps, const double *xp, const double *lv_in,
                                double *lb, double *lM, LN &&ln) {
    BcSolve<D> r;
    node_solve_bc_fw<D>(M, b0, nd, t, ext, nf, fc, nw, planes, eps, xp, r);
    double lv[D], kl[D];
    for (int a = 0; a < D; ++a) lv[a] = lv_in[a];
    // v' = v - T w, T = (v . d - g) / (w . d), w = K d: lT = -lv' . w, lw = -T lv', then through
    // T to v, w (and d, g); through w = K d to M (-(K lw) (x) w) and d (K lw)
    for (int k = kMaxContact - 1; k >= 0; --k) {
        if (!r.act[k]) continue;
        const double *n = planes + 2 * D * k + D;
        double lT = 0.0, lw[D];
        for (int a = 0; a < D; ++a) lT -= lv[a] * r.ww[k][a];
        const double lvn = lT / r.wn[k], lwn = -lT * r.Tw[k] / r.wn[k];
        for (int a = 0; a < D; ++a) {
            lw[a] = -r.Tw[k] * lv[a] + lwn * n[a];
            lv[a] += lvn * n[a];
        }
        node_solve<D>(M, lw, nd, t, kl);
        for (int a = 0; a < D; ++a)
            for (int c = 0; c < D; ++c) lM[a * D + c] -= kl[a] * r.ww[k][c];
    }
    double ldv[D] = {}, lgsum = 0.0;
    if (r.p1) {
        double lT = 0.0, lw[D];
        for (int a = 0; a < D; ++a) lT -= lv[a] * r.w1[a];
        const double lvd = lT / r.wd, lwd = -lT * r.T1 / r.wd;
        lgsum = -lT / r.wd;
        for (int a = 0; a < D; ++a) {
            lw[a] = -r.T1 * lv[a] + lwd * r.dv[a];
            ldv[a] += lvd * r.v0[a] + lwd * r.w1[a];
            lv[a] += lvd * r.dv[a];
        }
        node_solve<D>(M, lw, nd, t, kl);
        for (int a = 0; a < D; ++a) {
            ldv[a] += kl[a];
            for (int c = 0; c < D; ++c) lM[a * D + c] -= kl[a] * r.w1[c];
        }
    }
    node_solve<D>(M, lv, nd, t, lb);  // v0 = K b: lb = K lv, lM -= lb (x) v0
    for (int a = 0; a < D; ++a)
        for (int c = 0; c < D; ++c) lM[a * D + c] -= lb[a] * r.v0[c];
    if (!ext) return;
    for (int j = 0; j < nf; ++j) {
        int tag;
        double N[D], val[D], lN[D] = {};
        fc(j, tag, N, val);
        if (tag == TAG_TRACTION) {
            double nn = 0.0, lbt = 0.0;
            for (int a = 0; a < D; ++a) {
                nn += N[a] * N[a];
                lbt += lb[a] * val[a];
            }
            const double s = lbt / (sqrt(nn) * D);
            for (int a = 0; a < D; ++a) lN[a] = s * N[a];
        } else if (tag == TAG_PRESSURE) {
            for (int a = 0; a < D; ++a) lN[a] = -val[0] * lb[a] * (1.0 / D);
        } else if (tag == TAG_VELOCITY) {
            for (int a = 0; a < D; ++a) lN[a] = (ldv[a] + lgsum * val[a]) * (1.0 / D);
        }
        ln(j, lN);
    }
}

// the reverse predictor's records (see the product of predict_fw below)
template <int D> struct PredRec {
    static constexpr int NV = D + 1, DD = D * D, NS = D * (D + 1) / 2, NQ = D + DD;
    // cell record: slopes gs [NQ][D], G^-1 [DD], d_k = x_k - x_c [NV][D], dF/dt [DD], face
    // area vectors N [NV][D], D / |N_f| [NV], slopes taken (1) or not (0), the volume, and for
    // the stiffened gas the specific internal energy at t^n and at the half step
    static constexpr int F_GS = 0, F_GI = F_GS + NQ * D, F_DK = F_GI + DD, F_DFDT = F_DK + NV * D, F_N = F_DFDT + DD,
                         F_INU = F_N + NV * D, F_OK = F_INU + NV, F_V = F_OK + 1, F_EPS = F_V + 1, F_EPH = F_EPS + 1,
                         F_LEN = F_EPH + 1;
    // corner record: F_h [DD], v* [D], M_k [NS]
    static constexpr int K_FH = 0, K_VST = DD, K_M = DD + D, K_LEN = DD + D + NS;
    // pass-2 products of a corner: lv* [D], lF* [DD], lN_k [D], lmu, lkappa, leps (half step)
    static constexpr int Q2_LV = 0, Q2_LF = D, Q2_LN = D + DD, Q2_MU = 2 * D + DD, Q2_KAP = Q2_MU + 1,
                         Q2_EPS = Q2_KAP + 1, Q2_LEN = Q2_EPS + 1;
    // pass-1 products of a corner: lF_h [DD], lN_k [D], lmu, lkappa, leps (t^n)
    static constexpr int Q1_LF = 0, Q1_LN = DD, Q1_MU = DD + D, Q1_KAP = Q1_MU + 1, Q1_EPS = Q1_KAP + 1,
                         Q1_LEN = Q1_EPS + 1;
    // Barth-Jespersen record of a cell at the limited level: the unlimited slopes [NQ][D], per
    // field the factor phi, the corner that set it (-1: phi = 1), which bound (+1 the
    // stencil's maximum, -1 its minimum, 0 none; +-2 when the cell itself holds it), the cell
    // that holds that bound (filled by the kernel), and the adjoint of that bound (the reverse
    // pass's output)
    static constexpr int B_G = 0, B_PHI = NQ * D, B_K = B_PHI + NQ, B_SEL = B_K + NQ, B_T = B_SEL + NQ,
                         B_LE = B_T + NQ, B_LEN = B_LE + NQ;
};

// Barth-Jespersen limiter of a cell at the limited level (the cascade's middle level): each
// field's slopes gs [NQ][D] scaled by the largest phi <= 1 that keeps its values at the cell's
// nodes (d_k = x_k - x_c, dk [NV][D]) within [lo, hi], the field's range over the stencil and
// the cell; the unlimited slopes, phi and the choice that set it go to the record bjr, the
// limited slopes to gs and gs_out
template <int D>
LMOOD_HD void bj_limit(const double *vc, const double *Fc, const double (&dk)[D + 1][D], const double *lo,
                       const double *hi, double (&gs)[D + D * D][D], double *gs_out, double *bjr) {
    using P = PredRec<D>;
    constexpr int NV = D + 1, NQ = D + D * D;
    for (int q = 0; q < NQ; ++q) {
        const double qc = q < D ? vc[q] : Fc[q - D];
        double phi = 1.0;
        int ks = -1, sel = 0;
        for (int k = 0; k < NV; ++k) {
            double delta = 0.0;
            for (int a = 0; a < D; ++a) delta += gs[q][a] * dk[k][a];
            if (delta > 0.0) {
                const double cnd = (hi[q] - qc) / delta;
                if (cnd < phi) {
                    phi = cnd;
                    ks = k;
                    sel = 1;
                }
            }
            if (delta < 0.0) {
                const double cnd = (lo[q] - qc) / delta;
                if (cnd < phi) {
                    phi = cnd;
                    ks = k;
                    sel = -1;
                }
            }
        }
        bjr[P::B_PHI + q] = phi;
        bjr[P::B_K + q] = ks;
        bjr[P::B_SEL + q] = sel;
        for (int a = 0; a < D; ++a) {
            bjr[P::B_G + q * D + a] = gs[q][a];
            gs[q][a] *= phi;
            gs_out[q * D + a] = gs[q][a];
        }
    }
}

// reverse of bj_limit: lgs [NQ][D] the adjoint of the limited slopes in, of the unlimited ones
// out; accumulates the adjoints of the cell's values (lvc, lFc) and of d_k (lxs, lxcc as in
// predict_finish_vjp); the adjoint of the bound that set phi goes to bjr[B_LE + q]
template <int D>
LMOOD_HD void bj_limit_vjp(const double *dk, double (&lgs)[D + D * D][D], double *lvc, double *lFc, double *lxs,
                           double *lxcc, double *bjr) {
    using P = PredRec<D>;
    constexpr int NQ = D + D * D;
    for (int q = 0; q < NQ; ++q) {
        const double phi = bjr[P::B_PHI + q], *g = bjr + P::B_G + q * D;
        const int ks = (int)bjr[P::B_K + q];
        double lphi = 0.0;
        for (int a = 0; a < D; ++a) {
            lphi += lgs[q][a] * g[a];
            lgs[q][a] *= phi;
        }
        double lb = 0.0;
        // phi = (bound - q_c) / delta, delta = g . d_ks; a bound held by the cell itself
        // (|sel| = 2) is q_c: phi = 0 whatever q_c and delta, no adjoint (the products through
        // q_c and the bound would cancel, each ~ 1 / delta with delta at rounding level in a
        // uniform region)
        if (ks >= 0 && (int)bjr[P::B_SEL + q] * (int)bjr[P::B_SEL + q] == 1) {
            double delta = 0.0;
            for (int a = 0; a < D; ++a) delta += g[a] * dk[ks * D + a];
            lb = lphi / delta;
            if (q < D) lvc[q] -= lb;
            else lFc[q - D] -= lb;
            const double ld = -lphi * phi / delta;
            for (int a = 0; a < D; ++a) {
                lgs[q][a] += ld * dk[ks * D + a];
                lxs[ks * D + a] += ld * g[a];
                lxcc[a] -= ld * g[a];
            }
        }
        bjr[P::B_LE + q] = lb;
    }
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
                         double kap, double im, double dt, int ord, double *Mo, double *Ro, double sa = -1.0,
                         const SgMat *sg = nullptr, double ec = 0.0, const double *bjlo = nullptr,
                         const double *bjhi = nullptr) {
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
    double eps = 0.0;  // the stiffened gas: eps = e - |v|^2 / 2
    if (sg) {
        eps = ec;
        for (int a = 0; a < D; ++a) eps -= 0.5 * vc[a] * vc[a];
    }
    if (ord == 1) {
        double T[DD];
        stress_x<D>(Fc, mu, kap, sa, sg, eps, T);
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
    if (bjlo) {  // the limited level
        double dkk[NV][D], rec[PredRec<D>::B_LEN], gso[NQ * D];
        for (int k = 0; k < NV; ++k)
            for (int a = 0; a < D; ++a) dkk[k][a] = xs[k * D + a] - xcc[a];
        bj_limit<D>(vc, Fc, dkk, bjlo, bjhi, gs, gso, rec);
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
        stress_x<D>(Fh, mu, kap, sa, sg, eps, T);
        for (int i = 0; i < D; ++i)
            for (int b = 0; b < D; ++b) dv[i] += T[i * D + b] * N[k * D + b];
    }
    for (int a = 0; a < D; ++a) dv[a] *= hv;
    for (int i = 0; i < D; ++i)
        for (int a = 0; a < D; ++a) gv[i * D + a] = gs[i][a];
    mm<D>(gv, Fc, dFdt);
    double eps_h = eps;  // the stiffened gas: eps at the half step
    if (sg) {
        double Tc[DD], pw = 0.0;
        stress_x<D>(Fc, mu, kap, sa, sg, eps, Tc);
        for (int q = 0; q < DD; ++q) pw += Tc[q] * gv[q];
        eps_h = eps + 0.5 * dt * pw * V * im;
    }
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
        stress_x<D>(Fs, mu, kap, sa, sg, eps_h, T);
        for (int a = 0; a < D; ++a) {
            double s = 0.0;
            for (int b = 0; b < D; ++b) s += Mfull(k, a, b) * vst[b] + T[a * D + b] * N[k * D + b] * (1.0 / D);
            Ro[k * D + a] = s;
        }
    }
}

// ---------------------------------------------------------------------------------------
// Product of predict_fw, in pieces that the reverse pass runs as separate kernels for the
// second-order (P1) cells, so that none of them holds the whole cell's forward intermediates
// and adjoint accumulators at once:
//   predict_fw_rec      (cell)   the forward intermediates: record PF of the cell and PK of
//                                each corner (the reconstructed F_h, v*, M_k)
//   predict_corner2_vjp (corner) reverse of the packet R_k = M_k v*_k + (1/D) T(F*_k) N_k,
//                                F*_k = F_h,k + dt/2 dF/dt: record Q2 of the corner
//   predict_corner1_vjp (corner) reverse of dv = hv sum_k T(F_h,k) N_k, given the adjoint of
//                                dv (sum over the cell's corners of Q2's lv*): record Q1
//   predict_finish_vjp  (cell)   the rest: v* and F_h of the slopes, dF/dt, least squares,
//                                corner matrices, geometry
// predict_vjp below composes them (and keeps the first-order cells' product whole).
// ---------------------------------------------------------------------------------------

LMOOD_HD double adj_rsqrt(double x) {
#ifdef __CUDA_ARCH__
    return rsqrt(x);
#else
    return 1.0 / sqrt(x);
#endif
}

#ifdef __CUDA_ARCH__
#define LMOOD_UNROLL _Pragma("unroll")
#else
#define LMOOD_UNROLL
#endif

// forward intermediates of a P1 cell: pf [F_LEN]; corner k's record at pk + k * kstride. The
// least-squares sums follow the forward kernel's grouping (G symmetric; the q_c terms of the
// D+1 nodes gathered into one): the same values up to rounding. dvk (may be NULL): the stress
// sum sum_k T(F_h,k) N_k of the half-step velocity increment dv = hv sum_k T(F_h,k) N_k as the
// forward step formed it, component i at dvk[i * dvs]; given, it is taken instead of
// re-evaluating its D+1 stresses.
template <int D>
LMOOD_HD void predict_fw_rec(const double *xs, const Mom<D> &mom, const double *vc, const double *Fc, double z,
                             double mu, double kap, double im, double dt, double *pf, double *pk, long kstride,
                             double sa = -1.0, const SgMat *sg = nullptr, double ec = 0.0, double *bjr = nullptr,
                             const double *bjlo = nullptr, const double *bjhi = nullptr,
                             const double *dvk = nullptr, long dvs = 0) {
    using Q = Sz<D>;
    using P = PredRec<D>;
    constexpr int NV = Q::NV, DD = Q::DD, NS = Q::NS, NQ = Q::NQ;
    double V, xcc[D], N[NV * D];
    faces<D>(xs, V, N);
    LMOOD_UNROLL
    for (int i = 0; i < NV * D; ++i) pf[P::F_N + i] = N[i];
    pf[P::F_V] = V;
    double eps_c = 0.0;  // the stiffened gas: eps = e - |v|^2 / 2
    if (sg) {
        eps_c = ec;
        for (int a = 0; a < D; ++a) eps_c -= 0.5 * vc[a] * vc[a];
    }
    pf[P::F_EPS] = eps_c;
    LMOOD_UNROLL
    for (int a = 0; a < D; ++a) {
        double s = 0.0;
        LMOOD_UNROLL
        for (int k = 0; k < NV; ++k) s += xs[k * D + a];
        xcc[a] = s * (1.0 / NV);
    }
    double dk[NV][D];
    LMOOD_UNROLL
    for (int k = 0; k < NV; ++k)
        LMOOD_UNROLL
        for (int a = 0; a < D; ++a) {
            dk[k][a] = xs[k * D + a] - xcc[a];
            pf[P::F_DK + k * D + a] = dk[k][a];
        }
    // least squares from the node moments: G = sum_k (S2 + S1 d^t + d w^t), w = S1 + n d,
    // r_q = sum_k (T_q + d U_q) - (sum_k w) q_c
    double Gs[NS], r[NQ][D], wsum[D], npair = -NV;  // (node, other cell) pairs of the stencil
    LMOOD_UNROLL
    for (int k = 0; k < NV; ++k) {
        const double nk = mom(k, Q::M_N);
        npair += nk;
        double S1[D], w[D];
        LMOOD_UNROLL
        for (int a = 0; a < D; ++a) {
            S1[a] = mom(k, Q::M_S1 + a);
            w[a] = S1[a] + nk * dk[k][a];
            wsum[a] = k == 0 ? w[a] : wsum[a] + w[a];
        }
        LMOOD_UNROLL
        for (int a = 0; a < D; ++a)
            LMOOD_UNROLL
            for (int b = a; b < D; ++b) {
                const int sb = sym<D>(a, b);
                const double g = mom(k, Q::M_S2 + sb) + S1[a] * dk[k][b] + dk[k][a] * w[b];
                Gs[sb] = k == 0 ? g : Gs[sb] + g;
            }
        LMOOD_UNROLL
        for (int q = 0; q < NQ; ++q) {
            const double uq = mom(k, Q::M_U + q);
            LMOOD_UNROLL
            for (int a = 0; a < D; ++a) {
                const double t = mom(k, Q::M_T + q * D + a) + dk[k][a] * uq;
                r[q][a] = k == 0 ? t : r[q][a] + t;
            }
        }
    }
    LMOOD_UNROLL
    for (int q = 0; q < NQ; ++q) {
        const double qc = q < D ? vc[q] : Fc[q - D];
        LMOOD_UNROLL
        for (int a = 0; a < D; ++a) r[q][a] -= wsum[a] * qc;
    }
    double G[DD];
    LMOOD_UNROLL
    for (int a = 0; a < D; ++a)
        LMOOD_UNROLL
        for (int b = 0; b < D; ++b) G[a * D + b] = Gs[sym<D>(a, b)];
    double tr = 0.0;
    LMOOD_UNROLL
    for (int a = 0; a < D; ++a) tr += G[a * D + a];
    const double t = tr * (1.0 / D);
    const bool ok = npair > 0.0 && det<D>(G) > 1e-12 * (D == 2 ? t * t : t * t * t);
    pf[P::F_OK] = ok ? 1.0 : 0.0;
    double Gi[DD];
    inverse<D>(G, Gi);
    LMOOD_UNROLL
    for (int i = 0; i < DD; ++i) pf[P::F_GI + i] = Gi[i];
    double gs[NQ][D];
    LMOOD_UNROLL
    for (int q = 0; q < NQ; ++q)
        LMOOD_UNROLL
        for (int a = 0; a < D; ++a) {
            double s = 0.0;
            LMOOD_UNROLL
            for (int b = 0; b < D; ++b) s += Gi[a * D + b] * r[q][b];
            gs[q][a] = ok ? s : 0.0;
            pf[P::F_GS + q * D + a] = gs[q][a];
        }
    if (bjr) bj_limit<D>(vc, Fc, dk, bjlo, bjhi, gs, pf + P::F_GS, bjr);
    // corner matrices M_k = sum_{f != k} W_f, W_f = (z / |u_f|) u_f u_f^t, u_f = N_f / D
    double W[NV][NS];
    LMOOD_UNROLL
    for (int f = 0; f < NV; ++f) {
        double ss = 0.0;
        LMOOD_UNROLL
        for (int a = 0; a < D; ++a) ss += N[f * D + a] * N[f * D + a];
        const double inu = D * adj_rsqrt(ss);
        pf[P::F_INU + f] = inu;
        const double w = z * inu * (1.0 / (D * D));
        LMOOD_UNROLL
        for (int a = 0; a < D; ++a)
            LMOOD_UNROLL
            for (int b = a; b < D; ++b) W[f][sym<D>(a, b)] = w * N[f * D + a] * N[f * D + b];
    }
    // F_h at the corners and dv = hv sum_k T(F_h,k) N_k
    double dv[D] = {};
    LMOOD_UNROLL
    for (int k = 0; k < NV; ++k) {
        double *rk = pk + k * kstride;
        LMOOD_UNROLL
        for (int s2 = 0; s2 < NS; ++s2) {
            double acc = 0.0;
            LMOOD_UNROLL
            for (int f = 0; f < NV; ++f)
                if (f != k) acc += W[f][s2];
            rk[P::K_M + s2] = acc;
        }
        double T[DD], Fh[DD];
        LMOOD_UNROLL
        for (int q = 0; q < DD; ++q) {
            double s = Fc[q];
            LMOOD_UNROLL
            for (int a = 0; a < D; ++a) s += gs[D + q][a] * dk[k][a];
            Fh[q] = s;
            rk[P::K_FH + q] = s;
        }
        if (!dvk) {
            stress_x<D>(Fh, mu, kap, sa, sg, eps_c, T);
            LMOOD_UNROLL
            for (int i = 0; i < D; ++i)
                LMOOD_UNROLL
                for (int b = 0; b < D; ++b) dv[i] += T[i * D + b] * N[k * D + b];
        }
    }
    const double hv = -0.5 * dt * im * (1.0 / D);
    LMOOD_UNROLL
    for (int i = 0; i < D; ++i) dv[i] = hv * (dvk ? dvk[i * dvs] : dv[i]);
    LMOOD_UNROLL
    for (int k = 0; k < NV; ++k) {
        double *rk = pk + k * kstride;
        LMOOD_UNROLL
        for (int i = 0; i < D; ++i) {
            double s = vc[i];
            LMOOD_UNROLL
            for (int a = 0; a < D; ++a) s += gs[i][a] * dk[k][a];
            rk[P::K_VST + i] = s + dv[i];
        }
    }
    double gv[DD], dFdt[DD];
    LMOOD_UNROLL
    for (int i = 0; i < D; ++i)
        LMOOD_UNROLL
        for (int a = 0; a < D; ++a) gv[i * D + a] = gs[i][a];
    mm<D>(gv, Fc, dFdt);
    LMOOD_UNROLL
    for (int i = 0; i < DD; ++i) pf[P::F_DFDT + i] = dFdt[i];
    // the stiffened gas: eps at the half step, eps_h = eps + dt/2 (T_c : gv) V / m
    double eps_h = eps_c;
    if (sg) {
        double Tc[DD], pw = 0.0;
        stress_x<D>(Fc, mu, kap, sa, sg, eps_c, Tc);
        for (int i = 0; i < DD; ++i) pw += Tc[i] * gv[i];
        eps_h = eps_c + 0.5 * dt * pw * V * im;
    }
    pf[P::F_EPH] = eps_h;
}

// reverse of corner k's packet R_k = M_k v*_k + (1/D) T(F*_k) N_k, F*_k = F_h,k + dt/2 dF/dt,
// from lR_k [D]; adds lR_k (x) v*_k to lM_k [NS] and writes q2 [Q2_LEN]
template <int D>
LMOOD_HD void predict_corner2_vjp(const double *pf, const double *rk, int k, double mu, double kap, double dt,
                                  const double *lR_k, double *lM_k, double *q2, double sa = -1.0,
                                  const SgMat *sg = nullptr) {
    using P = PredRec<D>;
    constexpr int DD = D * D;
    const double *N = pf + P::F_N + k * D, *vst = rk + P::K_VST;
    double Fs[DD], lFs[DD] = {}, lvst[D] = {}, lmu = 0.0, lkap = 0.0, leps = 0.0;
    for (int q = 0; q < DD; ++q) Fs[q] = rk[P::K_FH + q] + 0.5 * dt * pf[P::F_DFDT + q];
    for (int a = 0; a < D; ++a) {
        const double l = lR_k[a];
        for (int b = 0; b < D; ++b) {
            lvst[b] += rk[P::K_M + sym<D>(a, b)] * l;
            lM_k[sym<D>(a, b)] += l * vst[b];
        }
    }
    if (!sg && sa == -1.0) {  // neo-Hookean: the rank-one product, lT = lR_k (N_k / D)^t
        double n[D], Tl[D];
        for (int b = 0; b < D; ++b) n[b] = N[b] * (1.0 / D);
        stress_vjp_r1<D>(Fs, mu, kap, lR_k, n, lFs, lmu, lkap, Tl);
        for (int b = 0; b < D; ++b) q2[P::Q2_LN + b] = Tl[b] * (1.0 / D);
    } else {
        double lT[DD], T[DD];
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b) lT[a * D + b] = lR_k[a] * N[b] * (1.0 / D);
        stress_x_vjp<D>(Fs, mu, kap, sa, sg, sg ? pf[P::F_EPH] : 0.0, lT, lFs, lmu, lkap, leps, T);
        for (int b = 0; b < D; ++b) {
            double s = 0.0;
            for (int a = 0; a < D; ++a) s += lR_k[a] * T[a * D + b];
            q2[P::Q2_LN + b] = s * (1.0 / D);
        }
    }
    for (int a = 0; a < D; ++a) q2[P::Q2_LV + a] = lvst[a];
    for (int q = 0; q < DD; ++q) q2[P::Q2_LF + q] = lFs[q];
    q2[P::Q2_MU] = lmu;
    q2[P::Q2_KAP] = lkap;
    q2[P::Q2_EPS] = leps;
}

// reverse of corner k's term of dv = hv sum_k T(F_h,k) N_k, given lacc = hv * (adjoint of dv);
// writes q1 [Q1_LEN]
template <int D>
LMOOD_HD void predict_corner1_vjp(const double *pf, const double *rk, int k, double mu, double kap,
                                  const double *lacc, double *q1, double sa = -1.0, const SgMat *sg = nullptr) {
    using P = PredRec<D>;
    constexpr int DD = D * D;
    const double *N = pf + P::F_N + k * D;
    double lF[DD] = {}, lmu = 0.0, lkap = 0.0, leps = 0.0;
    if (!sg && sa == -1.0) {  // neo-Hookean: the rank-one product, lT = lacc N_k^t
        stress_vjp_r1<D>(rk + P::K_FH, mu, kap, lacc, N, lF, lmu, lkap, q1 + P::Q1_LN);
    } else {
        double lT[DD], T[DD];
        for (int i = 0; i < D; ++i)
            for (int b = 0; b < D; ++b) lT[i * D + b] = lacc[i] * N[b];
        stress_x_vjp<D>(rk + P::K_FH, mu, kap, sa, sg, sg ? pf[P::F_EPS] : 0.0, lT, lF, lmu, lkap, leps, T);
        for (int b = 0; b < D; ++b) {
            double s = 0.0;
            for (int i = 0; i < D; ++i) s += lacc[i] * T[i * D + b];
            q1[P::Q1_LN + b] = s;
        }
    }
    for (int q = 0; q < DD; ++q) q1[P::Q1_LF + q] = lF[q];
    q1[P::Q1_MU] = lmu;
    q1[P::Q1_KAP] = lkap;
    q1[P::Q1_EPS] = leps;
}

// reverse of the corner matrices M_k = sum_{f != k} W_f (lmk(k): the final adjoint of M_k,
// NS values) and of the geometry (faces N, centroid): accumulates lz and lxs, given
// lN [NV][D] and lxcc [D]
template <int D, class LMK>
LMOOD_HD void predict_tail_vjp(const double *xs, const double *N, const double *inu, double z, LMK &&lmk,
                               double *lN, const double *lxcc, double *lxs, double &lz) {
    constexpr int NV = D + 1, NS = D * (D + 1) / 2;
    for (int f = 0; f < NV; ++f) {
        double lW[NS] = {}, u[D];
        for (int k = 0; k < NV; ++k)
            if (k != f)
                for (int s2 = 0; s2 < NS; ++s2) lW[s2] += lmk(k)[s2];
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
    faces_vjp<D>(xs, 0.0, lN, lxs);
    for (int k = 0; k < NV; ++k)
        for (int a = 0; a < D; ++a) lxs[k * D + a] += lxcc[a] * (1.0 / NV);
}

// the rest of a P1 cell's product, from the corner products: q2k(k) and q1k(k) give the
// records Q2, Q1 of corner k, lmk(k) the final adjoint of the corner matrix M_k (NS values).
// Accumulates lxs, lvc, lFc, lz and stores the node-moment adjoints through mout. (The loops
// run field by field, reading the slopes and the corner products as they go, so that few of
// them are live at once.)
template <int D, class Q2K, class Q1K, class MO>
LMOOD_HD void predict_finish_vjp(const Mom<D> &mom, const double *vc, const double *Fc, double dt, const double *pf,
                                 Q2K &&q2k, Q1K &&q1k, double *lxs, double *lxcc, MO &&mout, double *lvc,
                                 double *lFc, const SgMat *sg = nullptr, double mu = 0.0, double sa = -1.0,
                                 double im = 0.0, double *lmu = nullptr, double *le = nullptr,
                                 double *bjr = nullptr, long qs = 1) {
    // (vc, Fc: component i at [i * qs], read where they are used)
    using Q = Sz<D>;
    using P = PredRec<D>;
    constexpr int NV = Q::NV, DD = Q::DD, NS = Q::NS, NQ = Q::NQ;
    const double *gs = pf + P::F_GS, *Gi = pf + P::F_GI, *dk = pf + P::F_DK;
    // lxs collects the adjoints of d_k = x_k - x_c directly; lxcc gets their negated sum once,
    // at the end (lx0: what lxs held on entry)
    double lgs[NQ][D], ldFdt[DD], lx0[D];
    LMOOD_UNROLL
    for (int a = 0; a < D; ++a) {
        double s = 0.0;
        LMOOD_UNROLL
        for (int k = 0; k < NV; ++k) s += lxs[k * D + a];
        lx0[a] = s;
    }
    // v*_k = v_c + gs_v d_k + dv
    LMOOD_UNROLL
    for (int i = 0; i < D; ++i) {
        double l[NV], ls = 0.0;
        LMOOD_UNROLL
        for (int k = 0; k < NV; ++k) {
            l[k] = q2k(k)[P::Q2_LV + i];
            ls += l[k];
        }
        lvc[i] += ls;
        LMOOD_UNROLL
        for (int a = 0; a < D; ++a) {
            const double g = gs[i * D + a];
            double s = 0.0;
            LMOOD_UNROLL
            for (int k = 0; k < NV; ++k) {
                s += l[k] * dk[k * D + a];
                lxs[k * D + a] += l[k] * g;
            }
            lgs[i][a] = s;
        }
    }
    // F*_k = F_h,k + dt/2 dF/dt, F_h,k = F_c + gs_F d_k
    LMOOD_UNROLL
    for (int q = 0; q < DD; ++q) {
        double l[NV], sfs = 0.0, ls = 0.0;
        LMOOD_UNROLL
        for (int k = 0; k < NV; ++k) {
            const double lfs = q2k(k)[P::Q2_LF + q];
            sfs += lfs;
            l[k] = lfs + q1k(k)[P::Q1_LF + q];
            ls += l[k];
        }
        lFc[q] += ls;
        ldFdt[q] = 0.5 * dt * sfs;
        LMOOD_UNROLL
        for (int a = 0; a < D; ++a) {
            const double g = gs[(D + q) * D + a];
            double s = 0.0;
            LMOOD_UNROLL
            for (int k = 0; k < NV; ++k) {
                s += l[k] * dk[k * D + a];
                lxs[k * D + a] += l[k] * g;
            }
            lgs[D + q][a] = s;
        }
    }
    // dF/dt = gv F_c: lgv = ldFdt F_c^t, lF_c += gv^t ldFdt
    LMOOD_UNROLL
    for (int i = 0; i < D; ++i)
        LMOOD_UNROLL
        for (int j = 0; j < D; ++j) {
            double s = 0.0, u = 0.0;
            LMOOD_UNROLL
            for (int k = 0; k < D; ++k) {
                s += ldFdt[i * D + k] * Fc[(j * D + k) * qs];
                u += gs[k * D + i] * ldFdt[k * D + j];
            }
            lgs[i][j] += s;
            lFc[i * D + j] += u;
        }
    // the stiffened gas: eps_h = eps + dt/2 (T_c : gv) V / m, the corners' stresses at eps
    // (pass 1) and eps_h (pass 2); eps = e - |v|^2 / 2
    double lVsg = 0.0;
    if (sg) {
        const double V = pf[P::F_V], c = 0.5 * dt * V * im;
        double leh = 0.0, lec = 0.0;
        LMOOD_UNROLL
        for (int k = 0; k < NV; ++k) {
            leh += q2k(k)[P::Q2_EPS];
            lec += q1k(k)[P::Q1_EPS];
        }
        lec += leh;
        double lTc[DD], Tc[DD], lk = 0.0, Fcc[DD];
        LMOOD_UNROLL
        for (int i = 0; i < DD; ++i) {
            lTc[i] = c * leh * gs[i];  // gs [0..D)[D] is gv
            Fcc[i] = Fc[i * qs];
        }
        stress_x_vjp<D>(Fcc, mu, 0.0, sa, sg, pf[P::F_EPS], lTc, lFc, *lmu, lk, lec, Tc);
        double pw = 0.0;
        LMOOD_UNROLL
        for (int i = 0; i < DD; ++i) pw += Tc[i] * gs[i];
        LMOOD_UNROLL
        for (int i = 0; i < D; ++i)
            LMOOD_UNROLL
            for (int a = 0; a < D; ++a) lgs[i][a] += c * leh * Tc[i * D + a];
        lVsg = 0.5 * dt * pw * im * leh;  // dV / dx_k = -N_k / D, applied at the end
        *le += lec;
        LMOOD_UNROLL
        for (int a = 0; a < D; ++a) lvc[a] -= lec * vc[a * qs];
    }
    if (bjr) {  // the limited level (its centroid part is taken with the others at the end)
        double lxcc_bj[D] = {};
        bj_limit_vjp<D>(dk, lgs, lvc, lFc, lxs, lxcc_bj, bjr);
    }
    const double *gu = bjr ? bjr + P::B_G : gs;                   // the least squares' own slopes
    // least squares: gs = Gi r
    if (pf[P::F_OK] != 0.0) {
        // r_q = sum_k (T_q,k + d_k U_q,k) - (sum_k w_k) q_c with w_k = S1_k + n_k d_k; taken field
        // by field, so that one field's adjoint lr_q is live at a time: wsum first
        double wsum[D] = {};
        LMOOD_UNROLL
        for (int k = 0; k < NV; ++k) {
            const double nk = mom(k, Q::M_N);
            LMOOD_UNROLL
            for (int a = 0; a < D; ++a) wsum[a] += mom(k, Q::M_S1 + a) + nk * dk[k * D + a];
        }
        // gs_q = G^{-1} r_q, G symmetric: lr_q = G^{-1} lgs_q; G = G^t is formed from its upper
        // triangle Gs: lGs_ab = lG_ab + lG_ba (a < b), lG_aa, with lG = -sum_q lr_q gu_q^t; the
        // -w_k q_c terms: lw_k += lwq (the same for every k) and lq_c -= lr_q . wsum
        double lGs[NS] = {}, lwq[D] = {}, ldkr[NV][D] = {};
        LMOOD_UNROLL
        for (int q = 0; q < NQ; ++q) {
            double lr[D];
            LMOOD_UNROLL
            for (int a = 0; a < D; ++a) {
                double s = 0.0;
                LMOOD_UNROLL
                for (int b = 0; b < D; ++b) s += Gi[a * D + b] * lgs[q][b];
                lr[a] = s;
            }
            LMOOD_UNROLL
            for (int a = 0; a < D; ++a)
                LMOOD_UNROLL
                for (int b = a; b < D; ++b) {
                    double t = lr[a] * gu[q * D + b];
                    if (b != a) t += lr[b] * gu[q * D + a];
                    lGs[sym<D>(a, b)] -= t;
                }
            const double qc = q < D ? vc[q * qs] : Fc[(q - D) * qs];
            double lq = 0.0;
            LMOOD_UNROLL
            for (int a = 0; a < D; ++a) {
                lwq[a] -= lr[a] * qc;
                lq -= lr[a] * wsum[a];
            }
            if (q < D) lvc[q] += lq;
            else lFc[q - D] += lq;
            // r_q += T_q,k + d_k U_q,k at each node k
            LMOOD_UNROLL
            for (int k = 0; k < NV; ++k) {
                const double Uq = mom(k, Q::M_U + q);
                double lU = 0.0;
                LMOOD_UNROLL
                for (int a = 0; a < D; ++a) {
                    mout(k, Q::M_T + q * D + a, lr[a]);
                    ldkr[k][a] += lr[a] * Uq;
                    lU += lr[a] * dk[k * D + a];
                }
                mout(k, Q::M_U + q, lU);
            }
        }
        LMOOD_UNROLL
        for (int k = 0; k < NV; ++k) {
            const double nk = mom(k, Q::M_N);
            double S1[D], w[D], lS1[D] = {}, lw[D] = {}, lS2[NS] = {}, ln_ = 0.0, ldk[D];
            LMOOD_UNROLL
            for (int a = 0; a < D; ++a) {
                S1[a] = mom(k, Q::M_S1 + a);
                w[a] = S1[a] + nk * dk[k * D + a];
                ldk[a] = ldkr[k][a];
            }
            // Gs_ab += S2_ab + S1_a d_b + d_a w_b (a <= b)
            LMOOD_UNROLL
            for (int a = 0; a < D; ++a)
                LMOOD_UNROLL
                for (int b = a; b < D; ++b) {
                    const double l = lGs[sym<D>(a, b)];
                    lS2[sym<D>(a, b)] += l;
                    lS1[a] += l * dk[k * D + b];
                    ldk[b] += l * S1[a];
                    ldk[a] += l * w[b];
                    lw[b] += l * dk[k * D + a];
                }
            // w = S1 + n d
            LMOOD_UNROLL
            for (int a = 0; a < D; ++a) {
                lw[a] += lwq[a];
                lS1[a] += lw[a];
                ldk[a] += nk * lw[a];
                ln_ += lw[a] * dk[k * D + a];
            }
            LMOOD_UNROLL
            for (int a = 0; a < D; ++a) {
                mout(k, Q::M_S1 + a, lS1[a]);
                lxs[k * D + a] += ldk[a];
            }
            LMOOD_UNROLL
            for (int s2 = 0; s2 < NS; ++s2) mout(k, Q::M_S2 + s2, lS2[s2]);
            mout(k, Q::M_N, ln_);
        }
    } else {
        for (int k = 0; k < NV; ++k)
            for (int j = 0; j < Q::NMOM; ++j) mout(k, j, 0.0);
    }
    // x_c = mean of the x_k: the d_k adjoints' negated sum
    LMOOD_UNROLL
    for (int a = 0; a < D; ++a) {
        double s = 0.0;
        LMOOD_UNROLL
        for (int k = 0; k < NV; ++k) s += lxs[k * D + a];
        lxcc[a] -= s - lx0[a];
    }
    if (sg) {
        const double *N = pf + P::F_N;
        LMOOD_UNROLL
        for (int k = 0; k < NV; ++k)
            LMOOD_UNROLL
            for (int a = 0; a < D; ++a) lxs[k * D + a] -= lVsg * N[k * D + a] * (1.0 / D);
    }
}

// the corner matrices' and the geometry's part of a P1 cell's product (predict_tail_vjp with
// the face vectors of the record and lN from the corner products)
template <int D, class LMK, class Q2K, class Q1K>
LMOOD_HD void predict_tail_p1_vjp(const double *xs, double z, const double *pf, LMK &&lmk, Q2K &&q2k, Q1K &&q1k,
                                  const double *lxcc, double *lxs, double &lz) {
    using P = PredRec<D>;
    constexpr int NV = D + 1;
    double lN[NV * D];
    LMOOD_UNROLL
    for (int k = 0; k < NV; ++k)
        LMOOD_UNROLL
        for (int b = 0; b < D; ++b) lN[k * D + b] = q2k(k)[P::Q2_LN + b] + q1k(k)[P::Q1_LN + b];
    predict_tail_vjp<D>(xs, pf + P::F_N, pf + P::F_INU, z, lmk, lN, lxcc, lxs, lz);
}

template <int D, class MO>
LMOOD_HD void predict_p0_vjp(const double *xs, const double *vc, const double *Fc, double z, double mu, double kap,
                             double *lM, const double *lR, double *lxs, MO &&mout, double *lvc, double *lFc,
                             double &lz, double &lmu, double &lkap, double sa = -1.0, const SgMat *sg = nullptr,
                             double ec = 0.0, double *le = nullptr);

// Product of predict_fw: (lM [NV][NS], lR [NV][D]) -> accumulates lxs [NV][D], lvc [D],
// lFc [DD], lz, lmu, lkap, and stores the adjoints of the node moments through
// mout(k, j, value) (every (k, j) exactly once; zero where the packets do not depend on them).
template <int D, class MO>
LMOOD_HD void predict_vjp(const double *xs, const Mom<D> &mom, const double *vc, const double *Fc, double z, double mu,
                          double kap, double im, double dt, int ord, const double *lM_in, const double *lR, double *lxs,
                          MO &&mout, double *lvc, double *lFc, double &lz, double &lmu, double &lkap,
                          double sa = -1.0, const SgMat *sg = nullptr, double ec = 0.0, double *le = nullptr,
                          const double *bjlo = nullptr, const double *bjhi = nullptr, double *bjr = nullptr) {
    using Q = Sz<D>;
    using P = PredRec<D>;
    constexpr int NV = Q::NV, DD = Q::DD, NS = Q::NS, NM = Q::NMOM;
    double lM[NV * NS];
    for (int i = 0; i < NV * NS; ++i) lM[i] = lM_in[i];
    if (ord != 1) {
        double pf[P::F_LEN], pk[NV * P::K_LEN], q2[NV][P::Q2_LEN], q1[NV][P::Q1_LEN];
        predict_fw_rec<D>(xs, mom, vc, Fc, z, mu, kap, im, dt, pf, pk, P::K_LEN, sa, sg, ec, bjlo ? bjr : nullptr,
                          bjlo, bjhi);
        double ldv[D] = {};
        for (int k = 0; k < NV; ++k) {
            predict_corner2_vjp<D>(pf, pk + k * P::K_LEN, k, mu, kap, dt, lR + k * D, lM + k * NS, q2[k], sa, sg);
            for (int a = 0; a < D; ++a) ldv[a] += q2[k][P::Q2_LV + a];
        }
        const double hv = -0.5 * dt * im * (1.0 / D);
        double lacc[D];
        for (int a = 0; a < D; ++a) lacc[a] = hv * ldv[a];
        for (int k = 0; k < NV; ++k) predict_corner1_vjp<D>(pf, pk + k * P::K_LEN, k, mu, kap, lacc, q1[k], sa, sg);
        for (int k = 0; k < NV; ++k) {
            lmu += q2[k][P::Q2_MU] + q1[k][P::Q1_MU];
            lkap += q2[k][P::Q2_KAP] + q1[k][P::Q1_KAP];
        }
        double lxcc[D] = {};
        auto q2k = [&](int k) { return (const double *)q2[k]; };
        auto q1k = [&](int k) { return (const double *)q1[k]; };
        predict_finish_vjp<D>(mom, vc, Fc, dt, pf, q2k, q1k, lxs, lxcc, mout, lvc, lFc, sg, mu, sa, im, &lmu, le,
                              bjlo ? bjr : nullptr);
        predict_tail_p1_vjp<D>(xs, z, pf, [&](int k) { return (const double *)(lM + k * NS); }, q2k, q1k, lxcc, lxs,
                               lz);
        return;
    }
    predict_p0_vjp<D>(xs, vc, Fc, z, mu, kap, lM, lR, lxs, mout, lvc, lFc, lz, lmu, lkap, sa, sg, ec, le);
}

// the product for a first-order cell: R_k = M_k v_c + (1/D) T(F_c) N_k (lM [NV][NS] is
// updated in place; the node moments do not enter)
template <int D, class MO>
LMOOD_HD void predict_p0_vjp(const double *xs, const double *vc, const double *Fc, double z, double mu, double kap,
                             double *lM, const double *lR, double *lxs, MO &&mout, double *lvc, double *lFc,
                             double &lz, double &lmu, double &lkap, double sa, const SgMat *sg, double ec,
                             double *le) {
    using Q = Sz<D>;
    constexpr int NV = Q::NV, DD = Q::DD, NS = Q::NS, NM = Q::NMOM;
    double V, N[NV * D], inu[NV], lN[NV * D] = {}, lxcc[D] = {};
    faces<D>(xs, V, N);
    double Mo[NV * NS];
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
    double T[DD], lT[DD] = {}, lF[DD] = {};
    for (int k = 0; k < NV; ++k)
        for (int a = 0; a < D; ++a) {
            const double l = lR[k * D + a];
            for (int b = 0; b < D; ++b) {
                lvc[b] += Mo[k * NS + sym<D>(a, b)] * l;
                lM[k * NS + sym<D>(a, b)] += l * vc[b];
                lT[a * D + b] += l * N[k * D + b] * (1.0 / D);
            }
        }
    double eps = 0.0, leps = 0.0;  // the stiffened gas: eps = e - |v|^2 / 2
    if (sg) {
        eps = ec;
        for (int a = 0; a < D; ++a) eps -= 0.5 * vc[a] * vc[a];
    }
    stress_x_vjp<D>(Fc, mu, kap, sa, sg, eps, lT, lF, lmu, lkap, leps, T);
    if (sg) {
        *le += leps;
        for (int a = 0; a < D; ++a) lvc[a] -= leps * vc[a];
    }
    for (int k = 0; k < NV; ++k)
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b) lN[k * D + b] += lR[k * D + a] * T[a * D + b] * (1.0 / D);
    for (int q = 0; q < DD; ++q) lFc[q] += lF[q];
    for (int k = 0; k < NV; ++k)
        for (int j = 0; j < NM; ++j) mout(k, j, 0.0);
    predict_tail_vjp<D>(xs, N, inu, z, [&](int k) { return (const double *)(lM + k * NS); }, lN, lxcc, lxs, lz);
}

// ---------------------------------------------------------------------------------------
// Cell update (pure form of k_update for orders 1 and 2): inputs xs0, xs1, vs, vp0, vp1
// [NV][D] at the cell's nodes, packets M [NV][NS], R [NV][D], v [D], F [DD], m, 1/m, mu,
// kappa, dt, ord. Outputs v1 [D], F1 [DD], z1 (impedance of the new state).
// ---------------------------------------------------------------------------------------
template <int D>
LMOOD_HD void update_fw(const double *xs0, const double *xs1, const double *vs, const double *vp0, const double *vp1,
                        const double *M, const double *R, const double *v, const double *F, double m, double im,
                        double mu, double kap, double dt, int ord, double *v1, double *F1, double &z1,
                        double e = 0.0, double *e1 = nullptr) {
    using Q = Sz<D>;
    constexpr int NV = Q::NV, DD = Q::DD, NS = Q::NS;
    double sf[D] = {}, sfv = 0.0;
    for (int k = 0; k < NV; ++k)
        for (int a = 0; a < D; ++a) {
            double s = -R[k * D + a];
            for (int b = 0; b < D; ++b) s += M[k * NS + sym<D>(a, b)] * vs[k * D + b];
            sf[a] += s;
            sfv += s * vs[k * D + a];
        }
    for (int a = 0; a < D; ++a) v1[a] = v[a] + dt * im * sf[a];
    if (e1) *e1 = e + dt * im * sfv;  // e^{n+1} = e^n + dt/m sum_k f_k . v*_k
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

// Product of update_fw in two parts. The velocity part, v1 = v + dt im sum_k f_k with
// f_k = M_k vs_k - R_k, and (R given) the energy e1 = e + dt im sum_k f_k . vs_k:
// accumulates lvs [NV][D], lM [NV][NS], lR [NV][D] and lv [D] from lv1 and le1 (the
// adjoint of e^n is le1 itself).
template <int D>
LMOOD_HD void update_force_vjp(const double *vs, const double *M, double im, double dt, const double *lv1,
                               double *lvs, double *lM, double *lR, double *lv, double le1 = 0.0,
                               const double *R = nullptr) {
    constexpr int NV = D + 1, NS = D * (D + 1) / 2;
    for (int a = 0; a < D; ++a) lv[a] += lv1[a];
    const double dtm = dt * im;
    for (int k = 0; k < NV; ++k) {
        double fk[D];
        if (R)
            for (int a = 0; a < D; ++a) {
                double s = -R[k * D + a];
                for (int b = 0; b < D; ++b) s += M[k * NS + sym<D>(a, b)] * vs[k * D + b];
                fk[a] = s;
            }
        for (int a = 0; a < D; ++a) {
            const double lf = dtm * (R ? lv1[a] + le1 * vs[k * D + a] : lv1[a]);
            lR[k * D + a] -= lf;
            for (int b = 0; b < D; ++b) {
                lM[k * NS + sym<D>(a, b)] += lf * vs[k * D + b];
                lvs[k * D + b] += M[k * NS + sym<D>(a, b)] * lf;
            }
            if (R) lvs[k * D + a] += dtm * le1 * fk[a];
        }
    }
}

// The deformation part (F^{n+1} from the velocity gradients at both levels, or the first-order
// step with v*, and the impedance of F^{n+1}): (lF1, lz1) -> accumulates lF [DD], lmu, lkap.
// The corners' nodal values are read when needed through ld(i, u) (u [NV][D] <- 0 v*, 1 x^n,
// 2 x^{n+1}, 3 v_p^n, 4 v_p^{n+1}), and each nodal adjoint is handed over once, whole, through
// out(i, l) (l [NV][D]: 0 lvs, 1 lxs0, 2 lxs1, 3 lvp0, 4 lvp1; zeros where it has no term), so
// that a caller holds neither all inputs nor all outputs at once. Recomputes only what the
// product needs (F1 and the impedance term only where used; lz1 = 0 drops the impedance).
// F1_in (may be NULL): F^{n+1} as the forward step produced it, used instead of recomputing it.
// F, lF1_in and F1_in hold component q at [q * fs] (a cell's column of structure-of-arrays
// fields, or fs = 1), and are read where they are used.
template <int D, class LD, class OUT>
LMOOD_HD void update_deform_vjp(LD &&ld, OUT &&out, const double *F, double m, double mu, double kap, double dt,
                                int ord, const double *lF1_in, double lz1, double *lF, double &lmu, double &lkap,
                                const double *F1_in = nullptr, long fs = 1) {
    using Q = Sz<D>;
    constexpr int NV = Q::NV, DD = Q::DD, NX = NV * D;
    double lF1[DD], xs[NX], u[NX], N0[NX], V0, l[NX], lN[NX];
    auto get = [&](const double *p, double *o) {
        for (int q = 0; q < DD; ++q) o[q] = p[q * fs];
    };
    ld(1, xs);
    faces<D>(xs, V0, N0);
    const double iV0 = 1.0 / V0;
    if (ord != 1) {
        double N1[NX], V1, L0[DD], L1[DD], lL0[DD], lL1[DD], lV1 = 0.0, lV0 = 0.0;
        ld(2, xs);
        faces<D>(xs, V1, N1);
        const double iV1 = 1.0 / V1;
        ld(3, u);
        velgrad_iv<D>(u, N0, iV0, L0);
        ld(4, u);
        velgrad_iv<D>(u, N1, iV1, L1);
        {
            double A[DD], Bm[DD], Ai[DD], F1[DD], Fn[DD];
            for (int i = 0; i < D; ++i)
                for (int j = 0; j < D; ++j) {
                    A[i * D + j] = (i == j ? 1.0 : 0.0) - 0.5 * dt * L1[i * D + j];
                    Bm[i * D + j] = (i == j ? 1.0 : 0.0) + 0.5 * dt * L0[i * D + j];
                }
            inverse<D>(A, Ai);
            get(F, Fn);
            if (F1_in) {
                get(F1_in, F1);
            } else {
                double Rm[DD];
                mm<D>(Bm, Fn, Rm);
                mm<D>(Ai, Rm, F1);
            }
            get(lF1_in, lF1);
            if (lz1 != 0.0) {  // z1 = Z(F1, m / V1)
                double lrho = 0.0;
                impedance_vjp<D>(F1, m * iV1, mu, kap, lz1, lF1, lrho, lmu, lkap);
                lV1 -= lrho * m * iV1 * iV1;
            }
            // F1 = Ai Rm, Rm = Bm F
            double lRm[DD], lA[DD], lBm[DD], t[DD];
            mtm<D>(Ai, lF1, lRm);  // lRm = Ai^t lF1
            mmt<D>(lRm, F1, lA);   // lA = -lRm F1^t
            mmt<D>(lRm, Fn, lBm);  // lBm = lRm F^t
            mtm<D>(Bm, lRm, t);    // lF += Bm^t lRm
            for (int q = 0; q < DD; ++q) {
                lF[q] += t[q];
                lL1[q] = 0.5 * dt * lA[q];  // A = I - dt/2 L1, lA was -(...) -> +dt/2
                lL0[q] = 0.5 * dt * lBm[q];
            }
        }
        // level n+1: u holds v_p^{n+1}, xs holds x^{n+1}
        for (int i = 0; i < NX; ++i) l[i] = lN[i] = 0.0;
        velgrad_vjp_iv<D>(u, N1, iV1, L1, lL1, l, lN, lV1);
        out(4, l);
        for (int i = 0; i < NX; ++i) l[i] = 0.0;
        faces_vjp_n<D>(xs, N1, lV1, lN, l);
        out(2, l);
        // level n
        for (int i = 0; i < NX; ++i) l[i] = lN[i] = 0.0;
        ld(3, u);
        velgrad_vjp_iv<D>(u, N0, iV0, L0, lL0, l, lN, lV0);
        out(3, l);
        for (int i = 0; i < NX; ++i) l[i] = 0.0;
        ld(1, xs);
        faces_vjp_n<D>(xs, N0, lV0, lN, l);
        out(1, l);
        for (int i = 0; i < NX; ++i) l[i] = 0.0;
        out(0, l);
    } else {
        double Ls[DD], t[DD], lLs[DD], lV1 = 0.0, lV0 = 0.0, Fn[DD];
        ld(0, u);
        velgrad_iv<D>(u, N0, iV0, Ls);
        get(F, Fn);
        get(lF1_in, lF1);
        if (lz1 != 0.0) {
            double LF[DD], F1[DD], lrho = 0.0, V1, N1[NX];
            ld(2, xs);
            faces<D>(xs, V1, N1);
            const double iV1 = 1.0 / V1;
            mm<D>(Ls, Fn, LF);
            for (int q = 0; q < DD; ++q) F1[q] = Fn[q] + dt * LF[q];
            impedance_vjp<D>(F1, m * iV1, mu, kap, lz1, lF1, lrho, lmu, lkap);
            lV1 -= lrho * m * iV1 * iV1;
            for (int i = 0; i < NX; ++i) l[i] = lN[i] = 0.0;
            faces_vjp_n<D>(xs, N1, lV1, lN, l);
            out(2, l);
            ld(1, xs);
        } else {
            for (int i = 0; i < NX; ++i) l[i] = 0.0;
            out(2, l);
        }
        mtm<D>(Ls, lF1, t);
        for (int q = 0; q < DD; ++q) lF[q] += lF1[q] + dt * t[q];
        mmt<D>(lF1, Fn, lLs);
        for (int q = 0; q < DD; ++q) lLs[q] *= dt;
        for (int i = 0; i < NX; ++i) l[i] = lN[i] = 0.0;
        velgrad_vjp_iv<D>(u, N0, iV0, Ls, lLs, l, lN, lV0);
        out(0, l);
        for (int i = 0; i < NX; ++i) l[i] = 0.0;
        faces_vjp_n<D>(xs, N0, lV0, lN, l);
        out(1, l);
        for (int i = 0; i < NX; ++i) l[i] = 0.0;
        out(3, l);
        out(4, l);
    }
}

// Product of update_fw: (lv1, lF1, lz1) -> accumulates lxs0, lxs1, lvs, lvp0, lvp1 [NV][D],
// lM [NV][NS], lR [NV][D], lv [D], lF [DD], lmu, lkap.
template <int D>
LMOOD_HD void update_vjp(const double *xs0, const double *xs1, const double *vs, const double *vp0, const double *vp1,
                         const double *M, const double *R, const double *v, const double *F, double m, double im,
                         double mu, double kap, double dt, int ord, const double *lv1, const double *lF1, double lz1,
                         double *lxs0, double *lxs1, double *lvs, double *lvp0, double *lvp1, double *lM, double *lR,
                         double *lv, double *lF, double &lmu, double &lkap, double le1 = 0.0) {
    (void)v;
    update_force_vjp<D>(vs, M, im, dt, lv1, lvs, lM, lR, lv, le1, R);
    const double *in[5] = {vs, xs0, xs1, vp0, vp1};
    double *acc[5] = {lvs, lxs0, lxs1, lvp0, lvp1};
    update_deform_vjp<D>([&](int i, double *u) { for (int j = 0; j < (D + 1) * D; ++j) u[j] = in[i][j]; },
                         [&](int i, const double *l) { for (int j = 0; j < (D + 1) * D; ++j) acc[i][j] += l[j]; }, F,
                         m, mu, kap, dt, ord, lF1, lz1, lF, lmu, lkap);
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
