// Host-side check of the adjoint's vector-Jacobian products against central finite
// differences of their forward functions (no GPU needed: the functions are host+device).
// For random inputs x, a random output weight l and a random direction d it prints
//   name  <l, (f(x + h d) - f(x - h d)) / 2h>  <vjp(l), d>
// and the test compares the two numbers.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "lmood_adjoint.cuh"

using namespace lmood::adj;

static std::mt19937_64 rng(12345);
static double U(double a, double b) { return std::uniform_real_distribution<double>(a, b)(rng); }

static void report(const char *name, double fd, double an) { std::printf("%s %.17g %.17g\n", name, fd, an); }

template <int D> void randF(double *F, double amp) {
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) F[i * D + j] = (i == j ? 1.0 : 0.0) + U(-amp, amp);
}

// a random positively oriented simplex of size ~h around the origin
template <int D> void rand_simplex(double *xs, double h) {
    for (;;) {
        for (int k = 0; k < D + 1; ++k)
            for (int a = 0; a < D; ++a) xs[k * D + a] = (k == a + 1 ? h : 0.0) + U(-0.25 * h, 0.25 * h);
        double V, N[(D + 1) * D];
        faces<D>(xs, V, N);
        if (V > 0.05 * (D == 2 ? h * h : h * h * h)) return;
    }
}

template <int D> void check_stress() {
    constexpr int DD = D * D;
    for (int t = 0; t < 5; ++t) {
        double F[DD], lT[DD], dF[DD], mu = U(0.5, 2), kap = U(1, 4), dmu = U(-1, 1), dk = U(-1, 1);
        randF<D>(F, 0.2);
        for (int i = 0; i < DD; ++i) {
            lT[i] = U(-1, 1);
            dF[i] = U(-1, 1);
        }
        const double h = 1e-6;
        double Fp[DD], Fm[DD], Tp[DD], Tm[DD];
        for (int i = 0; i < DD; ++i) {
            Fp[i] = F[i] + h * dF[i];
            Fm[i] = F[i] - h * dF[i];
        }
        stress<D>(Fp, mu + h * dmu, kap + h * dk, Tp);
        stress<D>(Fm, mu - h * dmu, kap - h * dk, Tm);
        double fd = 0.0;
        for (int i = 0; i < DD; ++i) fd += lT[i] * (Tp[i] - Tm[i]) / (2 * h);
        double lF[DD] = {}, lmu = 0, lkap = 0;
        stress_vjp<D>(F, mu, kap, lT, lF, lmu, lkap);
        double an = lmu * dmu + lkap * dk;
        for (int i = 0; i < DD; ++i) an += lF[i] * dF[i];
        report(D == 2 ? "stress2" : "stress3", fd, an);
    }
}

// the rank-one form (lT = l n^t): its product against central differences of l^t T(F) n, and
// its T l against the forward stress
template <int D> void check_stress_r1() {
    constexpr int DD = D * D;
    for (int t = 0; t < 5; ++t) {
        double F[DD], l[D], n[D], dF[DD], mu = U(0.5, 2), kap = U(1, 4), dmu = U(-1, 1), dk = U(-1, 1);
        randF<D>(F, 0.2);
        for (int i = 0; i < D; ++i) {
            l[i] = U(-1, 1);
            n[i] = U(-1, 1);
        }
        for (int i = 0; i < DD; ++i) dF[i] = U(-1, 1);
        const double h = 1e-6;
        double Fp[DD], Fm[DD], Tp[DD], Tm[DD], T[DD];
        for (int i = 0; i < DD; ++i) {
            Fp[i] = F[i] + h * dF[i];
            Fm[i] = F[i] - h * dF[i];
        }
        stress<D>(Fp, mu + h * dmu, kap + h * dk, Tp);
        stress<D>(Fm, mu - h * dmu, kap - h * dk, Tm);
        double fd = 0.0;
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) fd += l[i] * (Tp[i * D + j] - Tm[i * D + j]) / (2 * h) * n[j];
        double lF[DD] = {}, lmu = 0, lkap = 0, Tl[D];
        stress_vjp_r1<D>(F, mu, kap, l, n, lF, lmu, lkap, Tl);
        double an = lmu * dmu + lkap * dk;
        for (int i = 0; i < DD; ++i) an += lF[i] * dF[i];
        report(D == 2 ? "stressr1_2" : "stressr1_3", fd, an);
        stress<D>(F, mu, kap, T);
        for (int i = 0; i < D; ++i) {
            double s = 0.0;
            for (int j = 0; j < D; ++j) s += T[i * D + j] * l[j];
            report(D == 2 ? "stressr1T_2" : "stressr1T_3", s, Tl[i]);
        }
    }
}

// the shear energy family (a != -1), and a = -1 through the dispatch against the neo-Hookean
// routine itself
template <int D> void check_stress_family() {
    constexpr int DD = D * D;
    const double as[4] = {0.0, 0.5, -0.5, 1.0};
    for (int t = 0; t < 4; ++t) {
        const double a = as[t];
        double F[DD], lT[DD], dF[DD], mu = U(0.5, 2), kap = U(1, 4), dmu = U(-1, 1), dk = U(-1, 1);
        randF<D>(F, 0.2);
        for (int i = 0; i < DD; ++i) {
            lT[i] = U(-1, 1);
            dF[i] = U(-1, 1);
        }
        const double h = 1e-6;
        double Fp[DD], Fm[DD], Tp[DD], Tm[DD];
        for (int i = 0; i < DD; ++i) {
            Fp[i] = F[i] + h * dF[i];
            Fm[i] = F[i] - h * dF[i];
        }
        stress_m<D>(Fp, mu + h * dmu, kap + h * dk, a, Tp);
        stress_m<D>(Fm, mu - h * dmu, kap - h * dk, a, Tm);
        double fd = 0.0;
        for (int i = 0; i < DD; ++i) fd += lT[i] * (Tp[i] - Tm[i]) / (2 * h);
        double lF[DD] = {}, lmu = 0, lkap = 0, T[DD], T2[DD];
        stress_m_vjp<D>(F, mu, kap, a, lT, lF, lmu, lkap, T);
        stress_m<D>(F, mu, kap, a, T2);
        double an = lmu * dmu + lkap * dk, dT = 0.0;
        for (int i = 0; i < DD; ++i) {
            an += lF[i] * dF[i];
            dT = fmax(dT, fabs(T[i] - T2[i]));
        }
        report(D == 2 ? "stressfam2" : "stressfam3", fd, an);
        report(D == 2 ? "stressfamT2" : "stressfamT3", 1.0, 1.0 + dT);  // T_out equals the forward
    }
    // the family's formula at a = -1 (not the dispatch) is the neo-Hookean stress
    for (int t = 0; t < 2; ++t) {
        double F[DD], T1[DD], T2[DD], mu = U(0.5, 2), kap = U(1, 4), dT = 0.0;
        randF<D>(F, 0.2);
        stress<D>(F, mu, kap, T1);
        stress_family_fw<D>(F, mu, kap, -1.0, T2);
        for (int i = 0; i < DD; ++i) dT = fmax(dT, fabs(T1[i] - T2[i]));
        report(D == 2 ? "stressfamNH2" : "stressfamNH3", 1.0, 1.0 + dT);
    }
}

// the stiffened gas: its stress and impedance with the energy (a = -1 and a = 0.3), and the
// shear energy of the family
template <int D> void check_stiffened_gas() {
    constexpr int DD = D * D;
    const SgMat sg{2.2, 1.5, 1.1};
    const double as[2] = {-1.0, 0.3};
    for (int t = 0; t < 6; ++t) {
        const double a = as[t & 1];
        double F[DD], dF[DD], lT[DD], mu = U(0.5, 2), dmu = U(-1, 1), eps = U(4, 6), de = U(-1, 1);  // p + pinf > 0
        double rho = U(0.5, 2), dr = U(-1, 1);
        randF<D>(F, 0.2);
        for (int i = 0; i < DD; ++i) {
            dF[i] = U(-1, 1);
            lT[i] = U(-1, 1);
        }
        const double h = 1e-6;
        double Fp[DD], Fm[DD];
        for (int i = 0; i < DD; ++i) {
            Fp[i] = F[i] + h * dF[i];
            Fm[i] = F[i] - h * dF[i];
        }
        // shear energy
        {
            const double fd = (shear_energy_a<D>(Fp, sg.rho0, mu + h * dmu, a) -
                               shear_energy_a<D>(Fm, sg.rho0, mu - h * dmu, a)) / (2 * h);
            double lF[DD] = {}, lmu = 0.0;
            shear_energy_a_vjp<D>(F, sg.rho0, mu, a, 1.0, lF, lmu);
            double an = lmu * dmu;
            for (int i = 0; i < DD; ++i) an += lF[i] * dF[i];
            report(D == 2 ? "sgpsi2" : "sgpsi3", fd, an);
        }
        // stress
        {
            double Tp[DD], Tm[DD];
            stress_sg_a<D>(Fp, mu + h * dmu, a, sg, eps + h * de, Tp);
            stress_sg_a<D>(Fm, mu - h * dmu, a, sg, eps - h * de, Tm);
            double fd = 0.0;
            for (int i = 0; i < DD; ++i) fd += lT[i] * (Tp[i] - Tm[i]) / (2 * h);
            double lF[DD] = {}, lmu = 0.0, le = 0.0, T[DD], T2[DD], dT = 0.0;
            stress_sg_a_vjp<D>(F, mu, a, sg, eps, lT, lF, lmu, le, T);
            stress_sg_a<D>(F, mu, a, sg, eps, T2);
            double an = lmu * dmu + le * de;
            for (int i = 0; i < DD; ++i) {
                an += lF[i] * dF[i];
                dT = fmax(dT, fabs(T[i] - T2[i]));
            }
            report(D == 2 ? "sgstress2" : "sgstress3", fd, an);
            report(D == 2 ? "sgstressT2" : "sgstressT3", 1.0, 1.0 + dT);
        }
        // impedance
        {
            const double fd = (impedance_sg_a<D>(Fp, rho + h * dr, mu + h * dmu, a, sg, eps + h * de) -
                               impedance_sg_a<D>(Fm, rho - h * dr, mu - h * dmu, a, sg, eps - h * de)) / (2 * h);
            double lF[DD] = {}, lr = 0.0, lmu = 0.0, le = 0.0;
            impedance_sg_a_vjp<D>(F, rho, mu, a, sg, eps, 1.0, lF, lr, lmu, le);
            double an = lr * dr + lmu * dmu + le * de;
            for (int i = 0; i < DD; ++i) an += lF[i] * dF[i];
            report(D == 2 ? "sgimp2" : "sgimp3", fd, an);
        }
    }
}

template <int D> void check_impedance() {
    constexpr int DD = D * D;
    for (int t = 0; t < 5; ++t) {
        double F[DD], dF[DD], rho = U(0.5, 2), mu = U(0.5, 2), kap = U(1, 4), dr = U(-1, 1), dmu = U(-1, 1),
                              dk = U(-1, 1);
        randF<D>(F, 0.2);
        for (int i = 0; i < DD; ++i) dF[i] = U(-1, 1);
        const double h = 1e-6;
        double Fp[DD], Fm[DD];
        for (int i = 0; i < DD; ++i) {
            Fp[i] = F[i] + h * dF[i];
            Fm[i] = F[i] - h * dF[i];
        }
        const double fd = (impedance<D>(Fp, rho + h * dr, mu + h * dmu, kap + h * dk) -
                           impedance<D>(Fm, rho - h * dr, mu - h * dmu, kap - h * dk)) / (2 * h);
        double lF[DD] = {}, lr = 0, lmu = 0, lk = 0;
        impedance_vjp<D>(F, rho, mu, kap, 1.0, lF, lr, lmu, lk);
        double an = lr * dr + lmu * dmu + lk * dk;
        for (int i = 0; i < DD; ++i) an += lF[i] * dF[i];
        report(D == 2 ? "impedance2" : "impedance3", fd, an);
    }
}

template <int D> void check_faces_velgrad() {
    constexpr int NV = D + 1;
    for (int t = 0; t < 5; ++t) {
        double xs[NV * D], dx[NV * D], lN[NV * D], lV = U(-1, 1);
        rand_simplex<D>(xs, 1.0);
        for (int i = 0; i < NV * D; ++i) {
            dx[i] = U(-1, 1);
            lN[i] = U(-1, 1);
        }
        const double h = 1e-6;
        double xp[NV * D], xm[NV * D], Vp, Vm, Np[NV * D], Nm[NV * D];
        for (int i = 0; i < NV * D; ++i) {
            xp[i] = xs[i] + h * dx[i];
            xm[i] = xs[i] - h * dx[i];
        }
        faces<D>(xp, Vp, Np);
        faces<D>(xm, Vm, Nm);
        double fd = lV * (Vp - Vm) / (2 * h);
        for (int i = 0; i < NV * D; ++i) fd += lN[i] * (Np[i] - Nm[i]) / (2 * h);
        double lxs[NV * D] = {};
        faces_vjp<D>(xs, lV, lN, lxs);
        double an = 0.0;
        for (int i = 0; i < NV * D; ++i) an += lxs[i] * dx[i];
        report(D == 2 ? "faces2" : "faces3", fd, an);
        // velocity gradient
        double vn[NV * D], dvn[NV * D], N[NV * D], dN[NV * D], V = U(0.5, 2), dV = U(-1, 1), lL[D * D];
        for (int i = 0; i < NV * D; ++i) {
            vn[i] = U(-1, 1);
            dvn[i] = U(-1, 1);
            N[i] = U(-1, 1);
            dN[i] = U(-1, 1);
        }
        for (int i = 0; i < D * D; ++i) lL[i] = U(-1, 1);
        double vp_[NV * D], vm_[NV * D], Np_[NV * D], Nm_[NV * D], Lp[D * D], Lm[D * D];
        for (int i = 0; i < NV * D; ++i) {
            vp_[i] = vn[i] + h * dvn[i];
            vm_[i] = vn[i] - h * dvn[i];
            Np_[i] = N[i] + h * dN[i];
            Nm_[i] = N[i] - h * dN[i];
        }
        velgrad<D>(vp_, Np_, V + h * dV, Lp);
        velgrad<D>(vm_, Nm_, V - h * dV, Lm);
        fd = 0.0;
        for (int i = 0; i < D * D; ++i) fd += lL[i] * (Lp[i] - Lm[i]) / (2 * h);
        double lvn[NV * D] = {}, lNn[NV * D] = {}, lVv = 0.0;
        velgrad_vjp<D>(vn, N, V, lL, lvn, lNn, lVv);
        an = lVv * dV;
        for (int i = 0; i < NV * D; ++i) an += lvn[i] * dvn[i] + lNn[i] * dN[i];
        report(D == 2 ? "velgrad2" : "velgrad3", fd, an);
    }
}

template <int D> void check_node_solve() {
    for (int nd = 0; nd <= D; ++nd)
        for (int t = 0; t < 3; ++t) {
            double M[D * D], dM[D * D], b[D], db[D], lv[D], tv[6] = {0, 0, 0, 0, 0, 0};
            // SPD M, symmetric perturbation
            double A[D * D];
            for (int i = 0; i < D * D; ++i) A[i] = U(-1, 1);
            for (int i = 0; i < D; ++i)
                for (int j = 0; j < D; ++j) {
                    double s = (i == j ? 2.0 : 0.0);
                    for (int k = 0; k < D; ++k) s += A[i * D + k] * A[j * D + k];
                    M[i * D + j] = s;
                }
            for (int i = 0; i < D; ++i)
                for (int j = i; j < D; ++j) dM[i * D + j] = dM[j * D + i] = U(-1, 1);
            for (int a = 0; a < D; ++a) {
                b[a] = U(-1, 1);
                db[a] = U(-1, 1);
                lv[a] = U(-1, 1);
            }
            // orthonormal tangents (first nd axes rotated)
            const double th = U(0, 3.14);
            if (D == 2) {
                tv[0] = cos(th); tv[1] = sin(th);
            } else {
                tv[0] = cos(th); tv[1] = sin(th); tv[2] = 0;
                tv[3] = 0; tv[4] = 0; tv[5] = 1;
            }
            const int nuse = nd == D ? D : nd;
            const double h = 1e-6;
            double Mp[D * D], Mm[D * D], bp[D], bm[D], vp_[D], vm_[D];
            for (int i = 0; i < D * D; ++i) {
                Mp[i] = M[i] + h * dM[i];
                Mm[i] = M[i] - h * dM[i];
            }
            for (int a = 0; a < D; ++a) {
                bp[a] = b[a] + h * db[a];
                bm[a] = b[a] - h * db[a];
            }
            node_solve<D>(Mp, bp, nuse, tv, vp_);
            node_solve<D>(Mm, bm, nuse, tv, vm_);
            double fd = 0.0;
            for (int a = 0; a < D; ++a) fd += lv[a] * (vp_[a] - vm_[a]) / (2 * h);
            double lb[D], lM[D * D] = {};
            node_solve_vjp<D>(M, b, nuse, tv, lv, lb, lM);
            double an = 0.0;
            for (int a = 0; a < D; ++a) an += lb[a] * db[a];
            for (int i = 0; i < D * D; ++i) an += lM[i] * dM[i];
            report(D == 2 ? "nodesolve2" : "nodesolve3", fd, an);
        }
}

// a random cell with node moments built from random cells around each node
template <int D> struct Patch {
    using Q = Sz<D>;
    double xs[(D + 1) * D], mom[(D + 1) * Q::NMOM], vc[D], Fc[D * D], z, mu, kap, im, dt;
    void make() {
        const double hcell = 0.05;
        rand_simplex<D>(xs, hcell);
        for (int a = 0; a < D; ++a) vc[a] = U(-0.1, 0.1);
        randF<D>(Fc, 0.05);
        z = U(1, 3);
        mu = U(0.5, 2);
        kap = U(1, 4);
        im = U(100, 400);
        dt = U(0.001, 0.005);
        for (int k = 0; k < D + 1; ++k) {
            double *m = mom + k * Q::NMOM;
            for (int j = 0; j < Q::NMOM; ++j) m[j] = 0.0;
            const int nc = 4 + (int)U(0, 4);
            for (int i = 0; i < nc; ++i) {
                double dx[D], q[Q::NQ];
                for (int a = 0; a < D; ++a) dx[a] = U(-hcell, hcell);
                for (int qi = 0; qi < Q::NQ; ++qi)
                    q[qi] = (qi < D ? vc[qi] : Fc[qi - D]) + 0.3 * U(-hcell, hcell);
                m[Q::M_N] += 1.0;
                for (int a = 0; a < D; ++a) m[Q::M_S1 + a] += dx[a];
                for (int a = 0; a < D; ++a)
                    for (int b = a; b < D; ++b) m[Q::M_S2 + sym<D>(a, b)] += dx[a] * dx[b];
                for (int qi = 0; qi < Q::NQ; ++qi) {
                    m[Q::M_U + qi] += q[qi];
                    for (int a = 0; a < D; ++a) m[Q::M_T + qi * D + a] += dx[a] * q[qi];
                }
            }
        }
    }
    Mom<D> acc(const double *mm) const {
        Mom<D> r;
        for (int k = 0; k < D + 1; ++k) r.p[k] = mm + k * Q::NMOM;
        r.stride = 1;
        return r;
    }
};

template <int D> void check_predict(int ord, double sa = -1.0, const SgMat *sg = nullptr) {
    using Q = Sz<D>;
    constexpr int NV = D + 1, NS = Q::NS, DD = D * D, NM = Q::NMOM;
    for (int t = 0; t < 4; ++t) {
        Patch<D> P;
        P.make();
        double lM[NV * NS], lR[NV * D];
        for (int i = 0; i < NV * NS; ++i) lM[i] = U(-1, 1);
        for (int i = 0; i < NV * D; ++i) lR[i] = U(-1, 1);
        // direction
        double dxs[NV * D], dmom[NV * NM], dvc[D], dF[DD], dz = U(-1, 1), dmu = U(-1, 1), dk = U(-1, 1);
        const double ec = U(1, 3), dec = U(-1, 1);  // the stiffened gas's specific total energy
        for (int i = 0; i < NV * D; ++i) dxs[i] = U(-1, 1) * 0.05;
        for (int i = 0; i < NV * NM; ++i) dmom[i] = U(-1, 1) * 0.01;
        for (int a = 0; a < D; ++a) dvc[a] = U(-1, 1);
        for (int q = 0; q < DD; ++q) dF[q] = U(-1, 1);
        const double h = 1e-7;
        auto eval = [&](double s, double *Mo, double *Ro) {
            Patch<D> Q2 = P;
            for (int i = 0; i < NV * D; ++i) Q2.xs[i] += s * dxs[i];
            for (int i = 0; i < NV * NM; ++i) Q2.mom[i] += s * dmom[i];
            for (int a = 0; a < D; ++a) Q2.vc[a] += s * dvc[a];
            for (int q = 0; q < DD; ++q) Q2.Fc[q] += s * dF[q];
            predict_fw<D>(Q2.xs, Q2.acc(Q2.mom), Q2.vc, Q2.Fc, P.z + s * dz, P.mu + s * dmu, P.kap + s * dk, P.im, P.dt,
                          ord, Mo, Ro, sa, sg, ec + s * dec);
        };
        double Mp[NV * NS], Rp[NV * D], Mm[NV * NS], Rm[NV * D];
        eval(h, Mp, Rp);
        eval(-h, Mm, Rm);
        double fd = 0.0;
        for (int i = 0; i < NV * NS; ++i) fd += lM[i] * (Mp[i] - Mm[i]) / (2 * h);
        for (int i = 0; i < NV * D; ++i) fd += lR[i] * (Rp[i] - Rm[i]) / (2 * h);
        double lxs[NV * D] = {}, lmom[NV * NM] = {}, lvc[D] = {}, lF[DD] = {}, lz = 0, lmu = 0, lkap = 0, le = 0;
        for (int i = 0; i < NV * NM; ++i) lmom[i] = 1e300;  // every entry must be stored exactly once
        predict_vjp<D>(P.xs, P.acc(P.mom), P.vc, P.Fc, P.z, P.mu, P.kap, P.im, P.dt, ord, lM, lR, lxs,
                       [&](int k, int j, double v) { lmom[k * NM + j] = v; }, lvc, lF, lz, lmu, lkap, sa, sg, ec,
                       &le);
        double an = lz * dz + lmu * dmu + lkap * dk + le * dec;
        for (int i = 0; i < NV * D; ++i) an += lxs[i] * dxs[i];
        for (int i = 0; i < NV * NM; ++i) an += lmom[i] * dmom[i];
        for (int a = 0; a < D; ++a) an += lvc[a] * dvc[a];
        for (int q = 0; q < DD; ++q) an += lF[q] * dF[q];
        char name[32];
        if (sg) std::snprintf(name, sizeof name, "predictsg%d_ord%d", D, ord);
        else if (sa == -1.0) std::snprintf(name, sizeof name, "predict%d_ord%d", D, ord);
        else std::snprintf(name, sizeof name, "predictfam%d_ord%d", D, ord);
        report(name, fd, an);
    }
}

// the Barth-Jespersen level: the stencil's bounds placed so that several fields are limited,
// and perturbed too (the adjoint of the bound that set each field's phi)
template <int D> void check_predict_bj() {
    using Q = Sz<D>;
    using P = PredRec<D>;
    constexpr int NV = D + 1, NS = Q::NS, DD = D * D, NM = Q::NMOM, NQ = Q::NQ;
    for (int t = 0; t < 4; ++t) {
        Patch<D> Pt;
        Pt.make();
        double lM[NV * NS], lR[NV * D], lo[NQ], hi[NQ], dlo[NQ], dhi[NQ];
        for (int i = 0; i < NV * NS; ++i) lM[i] = U(-1, 1);
        for (int i = 0; i < NV * D; ++i) lR[i] = U(-1, 1);
        for (int q = 0; q < NQ; ++q) {  // bounds close to the cell's value: most fields limited
            const double qc = q < D ? Pt.vc[q] : Pt.Fc[q - D];
            lo[q] = qc - U(0.001, 0.02) * 0.05;  // (0.05: the patch's cell size)
            hi[q] = qc + U(0.001, 0.02) * 0.05;
            dlo[q] = U(-1, 1) * 0.01;
            dhi[q] = U(-1, 1) * 0.01;
        }
        double dxs[NV * D], dmom[NV * NM], dvc[D], dF[DD], dz = U(-1, 1), dmu = U(-1, 1), dk = U(-1, 1);
        for (int i = 0; i < NV * D; ++i) dxs[i] = U(-1, 1) * 0.05;
        for (int i = 0; i < NV * NM; ++i) dmom[i] = U(-1, 1) * 0.01;
        for (int a = 0; a < D; ++a) dvc[a] = U(-1, 1) * 0.01;
        for (int q = 0; q < DD; ++q) dF[q] = U(-1, 1) * 0.01;
        const double h = 1e-7;
        auto eval = [&](double s, double *Mo, double *Ro) {
            Patch<D> Q2 = Pt;
            double lo2[NQ], hi2[NQ];
            for (int i = 0; i < NV * D; ++i) Q2.xs[i] += s * dxs[i];
            for (int i = 0; i < NV * NM; ++i) Q2.mom[i] += s * dmom[i];
            for (int a = 0; a < D; ++a) Q2.vc[a] += s * dvc[a];
            for (int q = 0; q < DD; ++q) Q2.Fc[q] += s * dF[q];
            for (int q = 0; q < NQ; ++q) {
                lo2[q] = lo[q] + s * dlo[q];
                hi2[q] = hi[q] + s * dhi[q];
            }
            predict_fw<D>(Q2.xs, Q2.acc(Q2.mom), Q2.vc, Q2.Fc, Pt.z + s * dz, Pt.mu + s * dmu, Pt.kap + s * dk, Pt.im,
                          Pt.dt, 2, Mo, Ro, -1.0, nullptr, 0.0, lo2, hi2);
        };
        double Mp[NV * NS], Rp[NV * D], Mm[NV * NS], Rm[NV * D];
        eval(h, Mp, Rp);
        eval(-h, Mm, Rm);
        double fd = 0.0;
        for (int i = 0; i < NV * NS; ++i) fd += lM[i] * (Mp[i] - Mm[i]) / (2 * h);
        for (int i = 0; i < NV * D; ++i) fd += lR[i] * (Rp[i] - Rm[i]) / (2 * h);
        double lxs[NV * D] = {}, lmom[NV * NM] = {}, lvc[D] = {}, lF[DD] = {}, lz = 0, lmu = 0, lkap = 0, le = 0;
        double rec[P::B_LEN];
        predict_vjp<D>(Pt.xs, Pt.acc(Pt.mom), Pt.vc, Pt.Fc, Pt.z, Pt.mu, Pt.kap, Pt.im, Pt.dt, 2, lM, lR, lxs,
                       [&](int k, int j, double v) { lmom[k * NM + j] = v; }, lvc, lF, lz, lmu, lkap, -1.0, nullptr,
                       0.0, &le, lo, hi, rec);
        double an = lz * dz + lmu * dmu + lkap * dk;
        int limited = 0;
        for (int i = 0; i < NV * D; ++i) an += lxs[i] * dxs[i];
        for (int i = 0; i < NV * NM; ++i) an += lmom[i] * dmom[i];
        for (int a = 0; a < D; ++a) an += lvc[a] * dvc[a];
        for (int q = 0; q < DD; ++q) an += lF[q] * dF[q];
        for (int q = 0; q < NQ; ++q) {
            const int sel = (int)rec[P::B_SEL + q];
            an += rec[P::B_LE + q] * (sel > 0 ? dhi[q] : sel < 0 ? dlo[q] : 0.0);
            limited += sel != 0;
        }
        report(D == 2 ? "predictbj2" : "predictbj3", fd, an);
        report(D == 2 ? "predictbjlimited2" : "predictbjlimited3", 1.0, limited > 0 ? 1.0 : 0.0);
    }
}

template <int D> void check_update(int ord) {
    using Q = Sz<D>;
    constexpr int NV = D + 1, NS = Q::NS, DD = D * D, NX = NV * D;
    for (int t = 0; t < 4; ++t) {
        double xs0[NX], xs1[NX], vs[NX], vp0[NX], vp1[NX], M[NV * NS], R[NX], v[D], F[DD];
        rand_simplex<D>(xs0, 0.05);
        for (int i = 0; i < NX; ++i) {
            vs[i] = U(-0.1, 0.1);
            vp0[i] = U(-0.1, 0.1);
            vp1[i] = 2 * vs[i] - vp0[i];
            R[i] = U(-1, 1);
        }
        const double dt = U(0.001, 0.004), m = U(0.001, 0.003), mu = U(0.5, 2), kap = U(1, 4);
        for (int i = 0; i < NX; ++i) xs1[i] = xs0[i] + dt * vs[i];
        for (int i = 0; i < NV * NS; ++i) M[i] = U(0.5, 1.5);
        for (int a = 0; a < D; ++a) v[a] = U(-0.1, 0.1);
        randF<D>(F, 0.05);
        double lv1[D], lF1[DD], lz1 = U(-1, 1);
        for (int a = 0; a < D; ++a) lv1[a] = U(-1, 1);
        for (int q = 0; q < DD; ++q) lF1[q] = U(-1, 1);
        double d0[NX], d1[NX], dvs[NX], dp0[NX], dp1[NX], dM[NV * NS], dR[NX], dv[D], dF[DD], dmu = U(-1, 1),
            dk = U(-1, 1);
        for (int i = 0; i < NX; ++i) {
            d0[i] = U(-1, 1) * 0.01;
            d1[i] = U(-1, 1) * 0.01;
            dvs[i] = U(-1, 1);
            dp0[i] = U(-1, 1);
            dp1[i] = U(-1, 1);
            dR[i] = U(-1, 1);
        }
        for (int i = 0; i < NV * NS; ++i) dM[i] = U(-1, 1);
        for (int a = 0; a < D; ++a) dv[a] = U(-1, 1);
        for (int q = 0; q < DD; ++q) dF[q] = U(-1, 1);
        const double h = 1e-7, e0 = U(0.5, 2), de = U(-1, 1), le1 = U(-1, 1);  // the energy equation too
        auto eval = [&](double s, double *v1, double *F1, double &z1, double &e1) {
            double a0[NX], a1[NX], avs[NX], ap0[NX], ap1[NX], aM[NV * NS], aR[NX], av[D], aF[DD];
            for (int i = 0; i < NX; ++i) {
                a0[i] = xs0[i] + s * d0[i];
                a1[i] = xs1[i] + s * d1[i];
                avs[i] = vs[i] + s * dvs[i];
                ap0[i] = vp0[i] + s * dp0[i];
                ap1[i] = vp1[i] + s * dp1[i];
                aR[i] = R[i] + s * dR[i];
            }
            for (int i = 0; i < NV * NS; ++i) aM[i] = M[i] + s * dM[i];
            for (int a = 0; a < D; ++a) av[a] = v[a] + s * dv[a];
            for (int q = 0; q < DD; ++q) aF[q] = F[q] + s * dF[q];
            update_fw<D>(a0, a1, avs, ap0, ap1, aM, aR, av, aF, m, 1.0 / m, mu + s * dmu, kap + s * dk, dt, ord, v1, F1,
                         z1, e0 + s * de, &e1);
        };
        double v1p[D], F1p[DD], z1p, e1p, v1m[D], F1m[DD], z1m, e1m;
        eval(h, v1p, F1p, z1p, e1p);
        eval(-h, v1m, F1m, z1m, e1m);
        double fd = lz1 * (z1p - z1m) / (2 * h) + le1 * (e1p - e1m) / (2 * h);
        for (int a = 0; a < D; ++a) fd += lv1[a] * (v1p[a] - v1m[a]) / (2 * h);
        for (int q = 0; q < DD; ++q) fd += lF1[q] * (F1p[q] - F1m[q]) / (2 * h);
        double l0[NX] = {}, l1[NX] = {}, lvs[NX] = {}, lp0[NX] = {}, lp1[NX] = {}, lM[NV * NS] = {}, lR[NX] = {},
               lv[D] = {}, lF[DD] = {}, lmu = 0, lkap = 0;
        update_vjp<D>(xs0, xs1, vs, vp0, vp1, M, R, v, F, m, 1.0 / m, mu, kap, dt, ord, lv1, lF1, lz1, l0, l1, lvs, lp0,
                      lp1, lM, lR, lv, lF, lmu, lkap, le1);
        double an = lmu * dmu + lkap * dk + le1 * de;  // e^n's adjoint is le1
        for (int i = 0; i < NX; ++i)
            an += l0[i] * d0[i] + l1[i] * d1[i] + lvs[i] * dvs[i] + lp0[i] * dp0[i] + lp1[i] * dp1[i] + lR[i] * dR[i];
        for (int i = 0; i < NV * NS; ++i) an += lM[i] * dM[i];
        for (int a = 0; a < D; ++a) an += lv[a] * dv[a];
        for (int q = 0; q < DD; ++q) an += lF[q] * dF[q];
        char name[32];
        std::snprintf(name, sizeof name, "update%d_ord%d", D, ord);
        report(name, fd, an);
        // the deformation part given F^{n+1} as the forward produced it equals the one that
        // recomputes it (the same linearisation point)
        double v1z[D], F1z[DD], z1z, e1z;
        eval(0.0, v1z, F1z, z1z, e1z);
        const double *in[5] = {vs, xs0, xs1, vp0, vp1};
        double w[5][NX];
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < NX; ++j) w[i][j] = U(-1, 1);
        // pass 2: the same inputs as pass 1 read with a stride (a cell's column of SoA fields)
        double Fs2[2 * DD], lF1s2[2 * DD], F1s2[2 * DD];
        for (int q = 0; q < DD; ++q) {
            Fs2[2 * q] = F[q];
            lF1s2[2 * q] = lF1[q];
            F1s2[2 * q] = F1z[q];
            Fs2[2 * q + 1] = lF1s2[2 * q + 1] = F1s2[2 * q + 1] = 1e300;  // never read
        }
        double sum[3];
        for (int pass = 0; pass < 3; ++pass) {
            double lFd[DD] = {}, lmud = 0, lkapd = 0, acc = 0.0;
            update_deform_vjp<D>([&](int i, double *u) { for (int j = 0; j < NX; ++j) u[j] = in[i][j]; },
                                 [&](int i, const double *l) { for (int j = 0; j < NX; ++j) acc += w[i][j] * l[j]; },
                                 pass == 2 ? Fs2 : F, m, mu, kap, dt, ord, pass == 2 ? lF1s2 : lF1, lz1, lFd, lmud,
                                 lkapd, pass == 2 ? F1s2 : pass ? F1z : nullptr, pass == 2 ? 2 : 1);
            acc += lmud * dmu + lkapd * dk;
            for (int q = 0; q < DD; ++q) acc += lFd[q] * dF[q];
            sum[pass] = acc;
        }
        std::snprintf(name, sizeof name, "updateF1in%d_ord%d", D, ord);
        report(name, sum[0], sum[1]);
        std::snprintf(name, sizeof name, "updatestride%d_ord%d", D, ord);
        report(name, sum[1], sum[2]);
    }
}

// nodal solve with traction / pressure / velocity faces and two active contact walls (one
// more wall out of reach), free or with one direction fixed; perturbs M, b and the faces' node
// positions
template <int D> void check_node_solve_bc() {
    constexpr int NF = 5;  // traction, pressure, velocity, velocity, slip (skipped)
    const int tags[NF] = {lmood::TAG_TRACTION, lmood::TAG_PRESSURE, lmood::TAG_VELOCITY, lmood::TAG_VELOCITY,
                          lmood::TAG_SLIP};
    for (int nd = D - 1; nd <= D; ++nd)
        for (int t = 0; t < 3; ++t) {
            double M[D * D], dM[D * D], b[D], db[D], lv[D], tv[6] = {0, 0, 0, 0, 0, 0}, A[D * D];
            for (int i = 0; i < D * D; ++i) A[i] = U(-1, 1);
            for (int i = 0; i < D; ++i)
                for (int j = 0; j < D; ++j) {
                    double s = (i == j ? 2.0 : 0.0);
                    for (int k = 0; k < D; ++k) s += A[i * D + k] * A[j * D + k];
                    M[i * D + j] = s;
                }
            for (int i = 0; i < D; ++i)
                for (int j = i; j < D; ++j) dM[i * D + j] = dM[j * D + i] = U(-1, 1);
            for (int a = 0; a < D; ++a) {
                b[a] = U(-1, 1);
                db[a] = U(-1, 1);
                lv[a] = U(-1, 1);
            }
            const double th = U(0, 3.14);
            tv[0] = cos(th);
            tv[1] = sin(th);
            if (D == 3) tv[5] = 1.0;
            double xq[NF][D * D], dxq[NF][D * D], val[NF][D], xp[D];
            for (int j = 0; j < NF; ++j) {
                for (int i = 0; i < D * D; ++i) {
                    xq[j][i] = U(-1, 1);
                    dxq[j][i] = U(-1, 1);
                }
                for (int a = 0; a < D; ++a) val[j][a] = U(-1, 1);
            }
            for (int a = 0; a < D; ++a) xp[a] = U(-1, 1);
            auto fc_of = [&](double (*x)[D * D]) {
                return [x, &tags, &val](int j, int &tag, double *N, double *v) {
                    tag = tags[j];
                    bface_area<D>(x[j], N);
                    for (int a = 0; a < D; ++a) v[a] = val[j][a];
                };
            };
            // walls: normals against the velocity each meets, the node 0.5 eps from them (as
            // many as leave the node a free direction), then one out of reach
            const double eps = 0.1;
            const int n_act = nd == D ? 2 : nd - 1;
            double planes[3 * 2 * D], v[D];
            int nw = 0;
            for (int k = 0; k <= n_act; ++k) {
                node_solve_bc<D>(M, b, nd, tv, true, NF, fc_of(xq), nw, planes, eps, xp, v);
                double n[D], nn = 0.0;
                for (int a = 0; a < D; ++a) {
                    n[a] = -v[a] + 0.3 * U(-1, 1);
                    nn += n[a] * n[a];
                }
                nn = sqrt(nn);
                const double dist = k == n_act ? 3.0 * eps : 0.5 * eps;
                for (int a = 0; a < D; ++a) {
                    planes[2 * D * k + D + a] = n[a] / nn;
                    planes[2 * D * k + a] = xp[a] - dist * n[a] / nn;
                }
                ++nw;
            }
            const double h = 1e-6;
            double Mp[D * D], Mm[D * D], bp[D], bm[D], vp_[D], vm_[D], xqp[NF][D * D], xqm[NF][D * D];
            for (int i = 0; i < D * D; ++i) {
                Mp[i] = M[i] + h * dM[i];
                Mm[i] = M[i] - h * dM[i];
            }
            for (int a = 0; a < D; ++a) {
                bp[a] = b[a] + h * db[a];
                bm[a] = b[a] - h * db[a];
            }
            for (int j = 0; j < NF; ++j)
                for (int i = 0; i < D * D; ++i) {
                    xqp[j][i] = xq[j][i] + h * dxq[j][i];
                    xqm[j][i] = xq[j][i] - h * dxq[j][i];
                }
            node_solve_bc<D>(Mp, bp, nd, tv, true, NF, fc_of(xqp), nw, planes, eps, xp, vp_);
            node_solve_bc<D>(Mm, bm, nd, tv, true, NF, fc_of(xqm), nw, planes, eps, xp, vm_);
            double fd = 0.0;
            for (int a = 0; a < D; ++a) fd += lv[a] * (vp_[a] - vm_[a]) / (2 * h);
            double lb[D], lM[D * D] = {}, an = 0.0;
            node_solve_bc_vjp<D>(M, b, nd, tv, true, NF, fc_of(xq), nw, planes, eps, xp, lv, lb, lM,
                                 [&](int j, const double *lN) {
                                     double lx[D * D] = {};
                                     bface_area_vjp<D>(xq[j], lN, lx);
                                     for (int i = 0; i < D * D; ++i) an += lx[i] * dxq[j][i];
                                 });
            for (int a = 0; a < D; ++a) an += lb[a] * db[a];
            for (int i = 0; i < D * D; ++i) an += lM[i] * dM[i];
            report(D == 2 ? "nodesolvebc2" : "nodesolvebc3", fd, an);
        }
}

template <int D> void check_moments() {
    using Q = Sz<D>;
    constexpr int NM = Q::NMOM, NQ = Q::NQ;
    for (int t = 0; t < 4; ++t) {
        double lmom[NM], xc[D], xp[D], q[NQ], dxc[D], dxp[D], dq[NQ];
        for (int j = 0; j < NM; ++j) lmom[j] = U(-1, 1);
        for (int a = 0; a < D; ++a) {
            xc[a] = U(-1, 1);
            xp[a] = U(-1, 1);
            dxc[a] = U(-1, 1);
            dxp[a] = U(-1, 1);
        }
        for (int i = 0; i < NQ; ++i) {
            q[i] = U(-1, 1);
            dq[i] = U(-1, 1);
        }
        auto mom_of = [&](double s, double *m) {
            for (int j = 0; j < NM; ++j) m[j] = 0.0;
            double dx[D], qq[NQ];
            for (int a = 0; a < D; ++a) dx[a] = (xc[a] + s * dxc[a]) - (xp[a] + s * dxp[a]);
            for (int i = 0; i < NQ; ++i) qq[i] = q[i] + s * dq[i];
            m[Q::M_N] = 1.0;
            for (int a = 0; a < D; ++a) m[Q::M_S1 + a] = dx[a];
            for (int a = 0; a < D; ++a)
                for (int b = a; b < D; ++b) m[Q::M_S2 + sym<D>(a, b)] = dx[a] * dx[b];
            for (int i = 0; i < NQ; ++i) {
                m[Q::M_U + i] = qq[i];
                for (int a = 0; a < D; ++a) m[Q::M_T + i * D + a] = dx[a] * qq[i];
            }
        };
        const double h = 1e-6;
        double mp[NM], mm_[NM];
        mom_of(h, mp);
        mom_of(-h, mm_);
        double fd = 0.0;
        for (int j = 0; j < NM; ++j) fd += lmom[j] * (mp[j] - mm_[j]) / (2 * h);
        double lxc[D] = {}, lq[NQ] = {}, lxp[D] = {};
        moments_corner_vjp<D>([&](int j) { return lmom[j]; }, xc, xp, q, lxc, lq, lxp);
        double an = 0.0;
        for (int a = 0; a < D; ++a) an += lxc[a] * dxc[a] + lxp[a] * dxp[a];
        for (int i = 0; i < NQ; ++i) an += lq[i] * dq[i];
        report(D == 2 ? "moments2" : "moments3", fd, an);
    }
}

int main() {
    check_stress<2>();
    check_stress<3>();
    check_stress_r1<2>();
    check_stress_r1<3>();
    check_stress_family<2>();
    check_stress_family<3>();
    check_stiffened_gas<2>();
    check_stiffened_gas<3>();
    check_impedance<2>();
    check_impedance<3>();
    check_faces_velgrad<2>();
    check_faces_velgrad<3>();
    check_node_solve<2>();
    check_node_solve<3>();
    check_node_solve_bc<2>();
    check_node_solve_bc<3>();
    check_moments<2>();
    check_predict_bj<2>();
    check_predict_bj<3>();
    check_moments<3>();
    for (int ord = 1; ord <= 2; ++ord) {
        check_predict<2>(ord);
        check_predict<3>(ord);
        check_predict<2>(ord, 0.0);
        check_predict<3>(ord, 0.5);
        const SgMat sg{2.2, 1.5, 1.1};
        check_predict<2>(ord, -1.0, &sg);
        check_predict<3>(ord, 0.3, &sg);
        check_update<2>(ord);
        check_update<3>(ord);
    }
    return 0;
}
