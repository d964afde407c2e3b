/*
 * lmood_tangent.cpp -- the oracle's step differentiated in forward mode: the CPU reference
 * for the library's adjoint.
 *
 * TEST INFRASTRUCTURE ONLY (like lmood_oracle.c, which it compiles): only the test-suite may
 * load it. It shares nothing with the CUDA path.
 *
 * How: lmood_oracle.c writes every quantity of the scheme in the scalar type `real`. Here that
 * type is a dual number, a value v and a directional derivative d, whose arithmetic and
 * elementary functions propagate d by the chain rule (sum, product and quotient rules;
 * sqrt, log, pow, fabs, fmin, fmax), and the oracle's source is compiled unchanged with it.
 * Every comparison looks at the value only, so the branches -- the MOOD decisions, the
 * boundary-condition cases, the log and cbrt-free paths of the oracle -- are exactly those of
 * the plain oracle, and the value parts are bitwise the plain oracle's (same operations, no FP
 * contraction). Seeding the derivative parts of the initial data (v per cell, mu per cell, F
 * per cell) with a direction delta gives, after n steps, J(state^N) delta exactly (up to
 * rounding), where J is the Jacobian of the n-step map with every step's order mask and dt
 * held at the values the run takes (and, with boundary faces, every contact and multiplier
 * decision, which are comparisons too): the derivative parts of dt are dropped after every step,
 * which is what "dt frozen" means (the adjoint of the library differentiates the same map;
 * its readings A1 and A2: the masses are fixed, and the initial first-order nodal solve of
 * v_p^0 is differentiated through).
 */
#include <cmath>

struct Dual {
    double v, d;
    Dual() = default;  // like double: uninitialised unless initialised
    Dual(double x) : v(x), d(0.0) {}
    Dual(double x, double dx) : v(x), d(dx) {}
    Dual &operator+=(const Dual &b) {
        v += b.v;
        d += b.d;
        return *this;
    }
    Dual &operator-=(const Dual &b) {
        v -= b.v;
        d -= b.d;
        return *this;
    }
    Dual &operator*=(const Dual &b) {
        d = d * b.v + v * b.d;
        v *= b.v;
        return *this;
    }
    Dual &operator/=(const Dual &b) {
        const double q = v / b.v;
        d = (d - q * b.d) / b.v;
        v = q;
        return *this;
    }
};

static inline Dual operator+(Dual a, const Dual &b) { return a += b; }
static inline Dual operator-(Dual a, const Dual &b) { return a -= b; }
static inline Dual operator*(Dual a, const Dual &b) { return a *= b; }
static inline Dual operator/(Dual a, const Dual &b) { return a /= b; }
static inline Dual operator-(const Dual &a) { return Dual(-a.v, -a.d); }
static inline Dual operator+(const Dual &a) { return a; }
static inline bool operator<(const Dual &a, const Dual &b) { return a.v < b.v; }
static inline bool operator>(const Dual &a, const Dual &b) { return a.v > b.v; }
static inline bool operator<=(const Dual &a, const Dual &b) { return a.v <= b.v; }
static inline bool operator>=(const Dual &a, const Dual &b) { return a.v >= b.v; }
static inline bool operator==(const Dual &a, const Dual &b) { return a.v == b.v; }
static inline bool operator!=(const Dual &a, const Dual &b) { return a.v != b.v; }

static inline Dual sqrt(const Dual &a) {
    const double r = std::sqrt(a.v);
    return Dual(r, a.d / (2.0 * r));
}
static inline Dual log(const Dual &a) { return Dual(std::log(a.v), a.d / a.v); }
static inline Dual pow(const Dual &a, double p) { return Dual(std::pow(a.v, p), p * std::pow(a.v, p - 1.0) * a.d); }
static inline Dual fabs(const Dual &a) { return a.v < 0.0 ? -a : a; }
static inline Dual fmin(const Dual &a, const Dual &b) {
    if (std::isnan(a.v)) return b;
    if (std::isnan(b.v)) return a;
    return b.v < a.v ? b : a;
}
static inline Dual fmax(const Dual &a, const Dual &b) {
    if (std::isnan(a.v)) return b;
    if (std::isnan(b.v)) return a;
    return b.v > a.v ? b : a;
}
static inline bool isfinite(const Dual &a) { return std::isfinite(a.v); }

#define ORC_REAL_DEFINED 1
typedef Dual real;

#include "lmood_oracle.c"

namespace {

real *dual_array(long n, const double *val, const double *dir) {
    real *a = ORC_NEW(real, n > 0 ? n : 1);
    for (long i = 0; i < n; ++i) a[i] = Dual(val[i], dir ? dir[i] : 0.0);
    return a;
}

// SoA [k][n] output of an AoS [n][k] real array: values and derivatives
void split_soa(const real *a, long n, int k, double *val, double *dir) {
    for (long i = 0; i < n; ++i)
        for (int c = 0; c < k; ++c) {
            if (val) val[c * n + i] = a[i * k + c].v;
            if (dir) dir[c * n + i] = a[i * k + c].d;
        }
}

}  // namespace

/*
 * Run n_steps oracle steps from the initial data (v [d][nc], mu [nc], F [d*d][nc] or NULL = I)
 * with derivative parts (dv, dmu, dF, and dx [d][np] of the node positions; each may be
 * NULL = 0), dt's derivative dropped at initialisation and after every step. The mesh's
 * boundary values bcval [d][nb] (NULL: zero) and contact walls (n_planes planes [n][2d],
 * threshold eps) are constants. A direction dx of the positions is taken at fixed cell masses:
 * the masses and the mesh's own data (slip directions) are those of x, the run starts from the
 * positions x + x_shift dx with derivative part dx, and the initial first-order nodal solve of
 * v_p^0 is done again there (x_shift != 0 gives the values of a displaced start, whose central
 * differences pin the derivative part). Outputs (each may be NULL): the
 * final state's values and derivatives, SoA like the oracle's orc_get (x, vp [d][np]; v [d][nc];
 * F [d*d][nc]; e [nc]), the order mask of every step masks [n_steps][nc] and its dt dts [n_steps].
 * Returns the oracle's status (0 ok; the first failing step stops the run).
 */
extern "C" int orct_run(int d, long np, const double *x_soa, const double *dx_soa, double x_shift, long nc,
                        const int *c2n_soa,
                        long nb, const int *bf_soa, const int *btag, const double *bcval_soa, int n_planes,
                        const double *planes, double contact_eps, double rho0, double lam, const double *mu,
                        const double *dmu, const double *v_soa, const double *dv_soa, const double *F_soa,
                        const double *dF_soa, const OrcParams *prm, long n_steps, double *x_out, double *dx_out,
                        double *vp_out, double *dvp_out, double *v_out, double *dv_out, double *F_out,
                        double *dF_out, double *e_out, double *de_out, signed char *masks, double *dts) {
    if ((d != 2 && d != 3) || !x_soa || !c2n_soa || !mu || !v_soa || !prm || n_steps < 0) return ORC_ERR_ARG;
    const int dd = d * d;
    real *xr = dual_array(np * d, x_soa, nullptr);
    OrcMesh *M = nullptr;
    int st = orc_mesh_new(d, np, xr, nc, c2n_soa, nb, bf_soa, btag, &M);
    free(xr);
    if (st) return st;
    if (bcval_soa && nb > 0) {
        real *bv = dual_array(nb * d, bcval_soa, nullptr);
        st = orc_mesh_set_bc_values(M, bv);
        free(bv);
    }
    if (st == ORC_OK && n_planes > 0) {
        real *pl = dual_array(n_planes * 2 * d, planes, nullptr);
        st = orc_mesh_set_contact(M, n_planes, pl, contact_eps);
        free(pl);
    }
    if (st) {
        orc_mesh_free(M);
        return st;
    }
    real *mur = dual_array(nc, mu, dmu);
    real *vr = dual_array(nc * d, v_soa, dv_soa);
    real *Fr = F_soa ? dual_array(nc * dd, F_soa, dF_soa) : nullptr;
    OrcState *S = nullptr;
    st = orc_state_new(M, rho0, lam, mur, vr, Fr, prm, &S);
    free(mur);
    free(vr);
    free(Fr);
    if (st) {
        orc_mesh_free(M);
        return st;
    }
    if (dx_soa) {
        for (long p = 0; p < np; ++p)
            for (int a = 0; a < d; ++a)
                S->x[p * d + a] = Dual(S->x[p * d + a].v + x_shift * dx_soa[a * np + p], dx_soa[a * np + p]);
        // the initial first-order nodal solve again, at the positions with their derivative
        // and the masses held (the oracle's own initialisation steps, in its order)
        Work w = work_new(M);
        phase_geometry(S, S->x, &w);
        for (long c = 0; c < nc; ++c) S->tau[c] = w.V[c] / S->m[c];
        phase_packets(S, S->order, 0.0, &w);
        for (long p = 0; p < np; ++p) node_solve_one(M, S->x, w.pkM, w.pkR, p, S->vp + p * d);
        work_free(&w);
    }
    S->dt = Dual(S->dt.v);  // dt frozen
    for (long s = 0; s < n_steps && st == ORC_OK; ++s) {
        st = orc_step(S, nullptr);
        if (masks)
            for (long c = 0; c < nc; ++c) masks[s * nc + c] = (signed char)S->order[c];
        if (dts) dts[s] = S->last.dt_used.v;
        S->dt = Dual(S->dt.v);
    }
    if (st == ORC_OK) {
        split_soa(S->x, np, d, x_out, dx_out);
        split_soa(S->vp, np, d, vp_out, dvp_out);
        split_soa(S->v, nc, d, v_out, dv_out);
        split_soa(S->F, nc, dd, F_out, dF_out);
        split_soa(S->e, nc, 1, e_out, de_out);
    }
    orc_state_free(S);
    orc_mesh_free(M);
    return st;
}
