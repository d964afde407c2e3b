// lmood_dev.cuh -- device-side data views and per-entity arithmetic of the Lagrangian
// ADER-MOOD step (arXiv 2104.02139), templated on the space dimension D (2 or 3).
//
// Layout in HBM (all FP64 unless noted, structure of arrays, "[k][n]" = k runs of n):
//   nodes : x, v_p^n, x^{n+1}, v_p^{n+1}, v*_p            [D][Np]
//   cells : v [D][N], e [N], F [D*D][N] (row-major), and the same for the candidate;
//           centroid x_c [D][N], rho, tau and impedance z [N] of the current and the
//           candidate state; m, 1/m, mu [N]; order, pad flag (u8) [N]; dt candidate [N]
//   corner packets (corner id = k*N + c, k = local vertex):
//           M_cp symmetric [D(D+1)/2][D+1][N], rhs_cp [D][D+1][N]
//   node moments of the least-squares sums [NMOM][Np] (see k_moments)
//   adjacency (int32): c2n [D+1][N]; node -> corner CSR (ascending cell id)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lmood {

struct Prm {
    double cfl, Cv, Ci, delta0, delta1, dt_fixed, lam;
    double irho0;    // 1 / rho0
    double shear_a;  // a of the shear energy family (Eq. familiy_energies); -1: neo-Hookean
    int eos;         // volumetric law: 0 Eq. EOS_neoHook, 1 stiffened gas (Eq. EOS_stiffened_gas)
    double gamma, pinf, p0, rho0;  // stiffened gas: gamma, p_infinity, initial pressure; rho0
    int base_order;  // order every cell starts the step with (2: P1, 1: P0; 0: keep f.order)
    int mood;        // detection on/off
    int vol_coeff;   // 0: kappa = lambda + 2 mu / 3; 1: kappa = mu
    int cascade;     // 2: P1 -> P0; 3: P1 -> P1 with Barth-Jespersen slopes -> P0
};

// threads per block of the full-mesh launches (autotuned per mesh; the arithmetic per cell or
// node does not depend on it)
struct Blk {
    int predict = 128, update = 128, nodes = 256, moments = 256;
};

struct Geo {
    int N, Np, n_inst, nbf;
    Blk blk;
    const int *c2n;
    const int *n2c_off, *n2c;
    const int *node_perm;          // the nodes of each window of 256 in order of their cell count
                                   // (whole-mesh node loops)
    const unsigned char *bc_ndof;  // free directions per node (D = free, 0 = clamped), | BC_EXT
                                   // when a traction / pressure / velocity face touches the node
    const double *bc_t;            // tangent vectors [2][3][Np]
    const int *cell_inst, *node_inst;  // NULL for one instance
    // boundary faces (NULL when the mesh has none): nodes [D][nbf] ordered so that the area
    // vector points outward, tag [nbf], values [D][nbf], the faces around each node
    // (ascending face id)
    const int *bf_nodes;
    const unsigned char *bf_tag;
    const double *bf_val;
    const int *nbf_off, *nbf_idx;
    // contact walls (device, updatable in place): [0] count n <= 4, [1] distance threshold,
    // then n planes of 2 D values (a point, the unit normal from the wall into the body)
    const double *contact;
};

// the whole-mesh nodal solve takes the nodes in the permuted order (cell count within
// windows of 256) in both dimensions
template <int D> constexpr bool kNodesByCount = true;

constexpr unsigned char BC_EXT = 0x80;      // node has traction / pressure / velocity faces
constexpr unsigned char BC_CONTACT = 0x40;  // node has contact faces
constexpr unsigned char BC_NDOF = 0x3f;     // the free directions
enum { TAG_FREE = 0, TAG_SLIP = 1, TAG_CLAMPED = 2, TAG_TRACTION = 3, TAG_PRESSURE = 4, TAG_VELOCITY = 5,
       TAG_CONTACT = 6 };
constexpr int kMaxContact = 4;

struct Fld {
    const double *m, *mu;
    double *x, *vp, *x1, *vp1, *vs;
    double *v, *e, *F, *v1, *e1, *F1;
    double *xc, *xc1, *rho, *rho1, *tau1;
    double *z, *z1;              // acoustic impedance rho a of the current / candidate state
    double *rlo, *rhi;           // [Np] range of rho^n over the cells around each node
    double *mom;                 // [NMOM][Np] least-squares moments of the cells around each node
    const double *im;            // 1 / m_c
    double *pkM, *pkR;
    double *dvs;                 // [D][N] or NULL: the predictor's stress sum sum_q T(F_h(x_q)) N_q of
                                 // the second-order cells (its half-step velocity increment is
                                 // -dt/2 (1/(D m)) times it), written when set (a tape's record of the
                                 // step: the reverse pass reads it instead of re-evaluating the D+1
                                 // stresses it takes)
    double *gf, *gf1;            // [CellGeo<D>::LEN][N] the cells' geometry at x^n / x^{n+1} (face area
                                 // vectors, volume, 1 / |N_f|, velocity gradient): the update writes that
                                 // of x^{n+1}, which the next step's predictor and update read
    unsigned char *order, *pflag;
    double *dtc;
    const double *dt;            // [n_inst] dt of this step
    unsigned long long *dtn;     // [n_inst] bit pattern of the next dt (positive doubles order as integers)
    int *cnt;                    // device counters, see CNT_*
};

// MOOD control block (device): mark stamp, rounds taken, troubled cells, error flag
struct Ctl {
    int stamp, iters, troubled, err;
};

// per-step report written by the last kernel of a step and copied to the host
struct Report {
    int n_troubled, mood_iters, err, n_p0, n_para, n_eps, n_lim, pad1;
    double dt_used, dt_next;
};

enum { CNT_T0 = 0, CNT_T1 = 1, CNT_NODES = 2, CNT_CELLS = 3, CNT_P0 = 4, CNT_PARA = 5, CNT_EPS = 6, CNT_LIM = 7,
       CNT_N = 8 };

template <int D> struct Dim {
    static constexpr int NV = D + 1, DD = D * D, NS = D * (D + 1) / 2, NQ = D + D * D;
    // node moments: count, S1 [D], S2 [NS], U [NQ], T [NQ][D]
    static constexpr int M_N = 0, M_S1 = 1, M_S2 = 1 + D, M_U = 1 + D + NS, M_T = 1 + D + NS + NQ;
    static constexpr int NMOM = 1 + D + NS + NQ + NQ * D;
};

// index of (a,b) in symmetric storage: 2D (xx,xy,yy), 3D (xx,xy,xz,yy,yz,zz)
template <int D> __host__ __device__ constexpr int sidx(int a, int b) {
    return D == 2 ? a + b
                  : (a <= b ? (a == 0 ? b : (a == 1 ? 2 + b : 5)) : (b == 0 ? a : (b == 1 ? 2 + a : 5)));
}

// ---------------------------------------------------------------------------------------
// Simplex geometry (Sect. "Mesh and notation", Eq. def_lcpncp): outward area vector N_k of
// the face opposite vertex k and the measure |w_c|. The corner vector is
// l n_p = sum_{f != p} N_f / D = -N_p / D (the face vectors of a closed simplex sum to zero).
// ---------------------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void simplex_faces(const double (&xs)[D + 1][D], double &V, double (&Nf)[D + 1][D]) {
    if constexpr (D == 2) {
        const double e1x = xs[1][0] - xs[0][0], e1y = xs[1][1] - xs[0][1];
        const double e2x = xs[2][0] - xs[0][0], e2y = xs[2][1] - xs[0][1];
        V = 0.5 * (e1x * e2y - e1y * e2x);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int a = (k + 1) % 3, b = (k + 2) % 3;
            Nf[k][0] = xs[b][1] - xs[a][1];
            Nf[k][1] = xs[a][0] - xs[b][0];
        }
    } else {
        double e[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int a = 0; a < 3; ++a) e[k][a] = xs[k + 1][a] - xs[0][a];
        const double c0 = e[1][1] * e[2][2] - e[1][2] * e[2][1];
        const double c1 = e[1][2] * e[2][0] - e[1][0] * e[2][2];
        const double c2 = e[1][0] * e[2][1] - e[1][1] * e[2][0];
        V = (e[0][0] * c0 + e[0][1] * c1 + e[0][2] * c2) * (1.0 / 6.0);
        // For a positively oriented tet the face opposite k, taken as (k+1, k+2, k+3) mod 4
        // in this order, has normal (x_b - x_a) x (x_c - x_a) pointing outward for even k
        // and inward for odd k.
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int fa = (k + 1) & 3, fb = (k + 2) & 3, fc = (k + 3) & 3;
            const double u0 = xs[fb][0] - xs[fa][0], u1 = xs[fb][1] - xs[fa][1], u2 = xs[fb][2] - xs[fa][2];
            const double w0 = xs[fc][0] - xs[fa][0], w1 = xs[fc][1] - xs[fa][1], w2 = xs[fc][2] - xs[fa][2];
            const double s = (k & 1) ? -0.5 : 0.5;
            Nf[k][0] = s * (u1 * w2 - u2 * w1);
            Nf[k][1] = s * (u2 * w0 - u0 * w2);
            Nf[k][2] = s * (u0 * w1 - u1 * w0);
        }
    }
}

// A cell's geometry at one set of node positions, kept per cell from the kernel that computes it
// (the update, at x^{n+1}; init and refresh at the current positions) for the next ones that
// need it: face area vectors N_f [D+1][D], volume |w_c|, 1 / |N_f| [D+1], and the velocity
// gradient L = (1/|w_c|) sum_p v_p (x) (l n)_cp [D*D] of the node velocities at the same time
// level (the next update's L^n). Component i of cell c at gf[i * N + c].
template <int D> struct CellGeo {
    static constexpr int NV = D + 1, NF = 0, VOL = NV * D, RS = NV * D + 1, LG = NV * D + 1 + NV,
                         LEN = NV * D + 1 + NV + D * D;
};
inline int cell_geo_len(int D) { return D == 2 ? CellGeo<2>::LEN : CellGeo<3>::LEN; }

// 1 / |N_f| of each face, and |N_f|^2
template <int D>
__device__ __forceinline__ void face_rnorms(const double (&Nf)[D + 1][D], double (&rs)[D + 1], double (&ss)[D + 1]) {
#pragma unroll
    for (int k = 0; k < D + 1; ++k) {
        double s = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) s += Nf[k][a] * Nf[k][a];
        ss[k] = s;
        rs[k] = rsqrt(s);
    }
}

template <int D>
__device__ __forceinline__ void store_cell_geo(double *gf, int N, int c, const double (&Nf)[D + 1][D], double V,
                                               const double (&rs)[D + 1]) {
    using G = CellGeo<D>;
#pragma unroll
    for (int k = 0; k < D + 1; ++k) {
#pragma unroll
        for (int a = 0; a < D; ++a) gf[(G::NF + k * D + a) * N + c] = Nf[k][a];
        gf[(G::RS + k) * N + c] = rs[k];
    }
    gf[G::VOL * N + c] = V;
}

template <int D> __device__ __forceinline__ void store_cell_grad(double *gf, int N, int c, const double (&L)[D * D]) {
#pragma unroll
    for (int q = 0; q < D * D; ++q) gf[(CellGeo<D>::LG + q) * N + c] = L[q];
}

template <int D> __device__ __forceinline__ void load_cell_grad(const double *gf, int N, int c, double (&L)[D * D]) {
#pragma unroll
    for (int q = 0; q < D * D; ++q) L[q] = gf[(CellGeo<D>::LG + q) * N + c];
}

template <int D>
__device__ __forceinline__ void load_cell_geo(const double *gf, int N, int c, double (&Nf)[D + 1][D], double &V) {
    using G = CellGeo<D>;
#pragma unroll
    for (int k = 0; k < D + 1; ++k)
#pragma unroll
        for (int a = 0; a < D; ++a) Nf[k][a] = gf[(G::NF + k * D + a) * N + c];
    V = gf[G::VOL * N + c];
}

template <int D>
__device__ __forceinline__ void corner_vectors(const double (&Nf)[D + 1][D], double (&ln)[D + 1][D]) {
#pragma unroll
    for (int p = 0; p < D + 1; ++p)
#pragma unroll
        for (int a = 0; a < D; ++a) ln[p][a] = Nf[p][a] * (-1.0 / D);
}

template <int D>
__device__ __forceinline__ void simplex_geometry(const double (&xs)[D + 1][D], double &V, double (&Nf)[D + 1][D],
                                                 double (&ln)[D + 1][D]) {
    simplex_faces<D>(xs, V, Nf);
    corner_vectors<D>(Nf, ln);
}

// in-sphere diameter 2 D |w_c| / sum_f |N_f| (the characteristic length L_c of Eq. CFL2)
template <int D> __device__ __forceinline__ double insphere(double V, const double (&Nf)[D + 1][D]) {
    double area = 0.0;
#pragma unroll
    for (int k = 0; k < D + 1; ++k) {
        double s = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) s += Nf[k][a] * Nf[k][a];
        area += sqrt(s);
    }
    return 2.0 * D * V / area;
}

template <int D> __device__ __forceinline__ double det(const double (&A)[D * D]) {
    if constexpr (D == 2) return A[0] * A[3] - A[1] * A[2];
    else
        return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
               A[2] * (A[3] * A[7] - A[4] * A[6]);
}

// adjugate times the reciprocal of the determinant
template <int D> __device__ __forceinline__ void inverse(const double (&A)[D * D], double (&Ai)[D * D]) {
    const double r = 1.0 / det<D>(A);
    if constexpr (D == 2) {
        Ai[0] = A[3] * r; Ai[1] = -A[1] * r;
        Ai[2] = -A[2] * r; Ai[3] = A[0] * r;
    } else {
        Ai[0] = (A[4] * A[8] - A[5] * A[7]) * r;
        Ai[1] = (A[2] * A[7] - A[1] * A[8]) * r;
        Ai[2] = (A[1] * A[5] - A[2] * A[4]) * r;
        Ai[3] = (A[5] * A[6] - A[3] * A[8]) * r;
        Ai[4] = (A[0] * A[8] - A[2] * A[6]) * r;
        Ai[5] = (A[2] * A[3] - A[0] * A[5]) * r;
        Ai[6] = (A[3] * A[7] - A[4] * A[6]) * r;
        Ai[7] = (A[1] * A[6] - A[0] * A[7]) * r;
        Ai[8] = (A[0] * A[4] - A[1] * A[3]) * r;
    }
}

template <int D>
__device__ __forceinline__ void matmul(const double (&A)[D * D], const double (&B)[D * D], double (&C)[D * D]) {
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) s += A[i * D + k] * B[k * D + j];
            C[i * D + j] = s;
        }
}

// ---------------------------------------------------------------------------------------
// Scalar functions of J = det F with few FP64 instructions (the FP64 pipe bounds the step).
// ---------------------------------------------------------------------------------------
// J^{-1/3}: single-precision seed y, then one third-order correction in FP64,
// y (1 - e)^{-1/3} = y (1 + e/3 + 2 e^2/9 + O(e^3)) with e = 1 - J y^3. The seed is good to
// ~1e-7, so the truncation is ~1e-20 and the result is within a couple of ulp.
__device__ __forceinline__ double rcbrt_j(double J) {
    const double y = (double)rcbrtf((float)J);
    const double y3 = y * y * y;
    const double e = fma(-J, y3, 1.0);
    const double q = e * fma(e, 2.0 / 9.0, 1.0 / 3.0);
    return fma(y, q, y);
}

// log J with few FP64 operations (d = J - 1), the range chosen from the exponent of d with
// integer operations:
//  |d| < 2^-12 : Taylor series ln(1 + d) = d - d^2/2 + ... + d^5/5 (tail < 1e-22 relative; the
//                weakly strained cells of an elastic body);
//  |d| < 2^-6  : the series to d^10/10 (tail < 1e-20 relative);
//  |d| < 2^-3  : ln J = 2 atanh(s) = 2 (s + s^3/3 + ... + s^13/13), s = d/(J + 1), |s| < 1/15
//                (tail below 2e-17 relative);
//  elsewhere (large strains, and J <= 0 which gives NaN / -inf): the CUDA log.
__device__ __forceinline__ double log_j(double J) {
    const double d = J - 1.0;
    const int E = (__double2hiint(d) >> 20) & 0x7ff;  // biased exponent of |d|
    if (E <= 1023 - 13) {
        double p = 1.0 / 5.0;
        p = fma(p, d, -1.0 / 4.0);
        p = fma(p, d, 1.0 / 3.0);
        p = fma(p, d, -1.0 / 2.0);
        p = fma(p, d, 1.0);
        return d * p;
    }
    if (E <= 1023 - 7) {
        double p = -1.0 / 10.0;
        p = fma(p, d, 1.0 / 9.0);
        p = fma(p, d, -1.0 / 8.0);
        p = fma(p, d, 1.0 / 7.0);
        p = fma(p, d, -1.0 / 6.0);
        p = fma(p, d, 1.0 / 5.0);
        p = fma(p, d, -1.0 / 4.0);
        p = fma(p, d, 1.0 / 3.0);
        p = fma(p, d, -1.0 / 2.0);
        p = fma(p, d, 1.0);
        return d * p;
    }
    if (E > 1023 - 4) return log(J);
    const double s = d / (J + 1.0);
    const double s2 = s * s;
    double p = 1.0 / 13.0;
    p = fma(p, s2, 1.0 / 11.0);
    p = fma(p, s2, 1.0 / 9.0);
    p = fma(p, s2, 1.0 / 7.0);
    p = fma(p, s2, 1.0 / 5.0);
    p = fma(p, s2, 1.0 / 3.0);
    p = fma(p, s2, 1.0);
    return 2.0 * s * p;
}

// ---------------------------------------------------------------------------------------
// Neo-Hookean Cauchy stress (Eqs. T_psi, EOS_neoHook, cstnh): T = -p I + (mu/J) dev(Bbar),
// p = -(kappa/2)(J - 1 + log J / J), Bbar = J^{-2/3} F F^t. 2D is plane strain (F33 = 1).
// ---------------------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void stress(const double (&F)[D * D], double mu, double kappa, double (&T)[D * D]) {
    const double J = det<D>(F);
    const double rc = rcbrt_j(J);
    const double Jm23 = rc * rc;
    const double invJ = Jm23 * rc;
    const double p = -0.5 * kappa * (J - 1.0 + log_j(J) * invJ);
    const double coef = mu * invJ;
    double B[D * D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = i; j < D; ++j) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) s += F[i * D + k] * F[j * D + k];
            B[i * D + j] = s;
            B[j * D + i] = s;
        }
    const double tr = (D == 2) ? B[0] + B[3] + 1.0 : B[0] + B[4] + B[8];
    const double cj = coef * Jm23;
    const double diag = -p - cj * tr * (1.0 / 3.0);
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) T[i * D + j] = cj * B[i * D + j] + (i == j ? diag : 0.0);
}

// Cauchy stress of the shear energy family (Eq. familiy_energies) for a != -1, with the
// volumetric part of Eq. EOS_neoHook: T = -p I + (mu/J) dev(c1 Bbar - c2 Bbar^2),
// c1 = -a + (1+a) I1 I2 / 3, c2 = (1+a) I2 / 3, I1 = tr Bbar, I2 = (I1^2 - tr Bbar^2) / 2,
// evaluated on the 3x3 embedding (2D plane strain, F33 = 1).
template <int D>
__device__ __forceinline__ void stress_family(const double (&F)[D * D], double mu, double kappa, double a,
                                           double (&T)[D * D]) {
    double F3[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) F3[i * 3 + j] = (i < D && j < D) ? F[i * D + j] : (i == j ? 1.0 : 0.0);
    const double J = F3[0] * (F3[4] * F3[8] - F3[5] * F3[7]) - F3[1] * (F3[3] * F3[8] - F3[5] * F3[6]) +
                     F3[2] * (F3[3] * F3[7] - F3[4] * F3[6]);
    const double rc = rcbrt_j(J), Jm23 = rc * rc, invJ = Jm23 * rc;
    double B[9], B2[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) s += F3[i * 3 + k] * F3[j * 3 + k];
            B[i * 3 + j] = Jm23 * s;
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) s += B[i * 3 + k] * B[k * 3 + j];
            B2[i * 3 + j] = s;
        }
    const double I1 = B[0] + B[4] + B[8], I2 = 0.5 * (I1 * I1 - (B2[0] + B2[4] + B2[8]));
    const double c1 = -a + (1.0 + a) * I1 * I2 * (1.0 / 3.0), c2 = (1.0 + a) * I2 * (1.0 / 3.0);
    double X[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) X[i] = c1 * B[i] - c2 * B2[i];
    const double trX = X[0] + X[4] + X[8];
    const double p = -0.5 * kappa * (J - 1.0 + log_j(J) * invJ);
    const double coef = mu * invJ;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) T[i * D + j] = coef * (X[i * 3 + j] - (i == j ? trX * (1.0 / 3.0) : 0.0)) - (i == j ? p : 0.0);
}

// acoustic impedance z = rho a with a^2 = (K + 4 mu / (3 J)) / rho, K = -J dp/dJ =
// (kappa/2)(J + (1 - log J)/J): z = sqrt(rho (K + 4 mu / (3 J)))
template <int D>
__device__ __forceinline__ double impedance(const double (&F)[D * D], double rho, double mu, double kappa) {
    const double J = det<D>(F);
    const double invJ = 1.0 / J;
    const double K = 0.5 * kappa * (J + (1.0 - log_j(J)) * invJ);
    return sqrt(rho * (K + (4.0 / 3.0) * mu * invJ));
}

// specific free energy Psi = kappa/(4 rho0)((J-1)^2 + log^2 J) + mu/(2 rho0)(I1(Bbar) - 3)
template <int D>
__device__ __forceinline__ double free_energy(const double (&F)[D * D], double rho0, double mu, double kappa) {
    const double J = det<D>(F);
    const double lJ = log_j(J);
    double trB = (D == 2) ? 1.0 : 0.0;
#pragma unroll
    for (int i = 0; i < D * D; ++i) trB += F[i] * F[i];
    const double rc = rcbrt_j(J);
    const double I1bar = rc * rc * trB;
    return kappa / (4.0 * rho0) * ((J - 1.0) * (J - 1.0) + lJ * lJ) + mu / (2.0 * rho0) * (I1bar - 3.0);
}

// the same with the shear energy of the family (a != -1)
template <int D>
__device__ __noinline__ double free_energy_family(const double (&F)[D * D], double rho0, double mu, double kappa,
                                                  double a) {
    double F3[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) F3[i * 3 + j] = (i < D && j < D) ? F[i * D + j] : (i == j ? 1.0 : 0.0);
    const double J = F3[0] * (F3[4] * F3[8] - F3[5] * F3[7]) - F3[1] * (F3[3] * F3[8] - F3[5] * F3[6]) +
                     F3[2] * (F3[3] * F3[7] - F3[4] * F3[6]);
    const double rc = rcbrt_j(J), Jm23 = rc * rc;
    double B[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) s += F3[i * 3 + k] * F3[j * 3 + k];
            B[i * 3 + j] = Jm23 * s;
        }
    double I1 = B[0] + B[4] + B[8], trB2 = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) trB2 += B[i] * B[i];
    const double I2 = 0.5 * (I1 * I1 - trB2), lJ = log_j(J);
    return kappa / (4.0 * rho0) * ((J - 1.0) * (J - 1.0) + lJ * lJ) +
           mu / (4.0 * rho0) * (-2.0 * a * (I1 - 3.0) + (1.0 + a) * (1.0 / 3.0) * (I2 * I2 - 9.0));
}

__device__ __forceinline__ double kappa_of(const Prm &prm, double mu) {
    return prm.vol_coeff ? mu : prm.lam + mu * (2.0 / 3.0);
}

// A double's bits as a signed integer whose order is the numeric order (NaN aside): min / max
// of densities on the integer pipe instead of the FP64 one
__device__ __forceinline__ long long order_key(double x) {
    const long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double key_value(long long k) {
    return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}

// physical admissibility (Eq. PAD): 0 admissible, 1 only eps < -tol, 2 not computable;
// tol = 1e-10 max(|e|, |v|^2/2, a0sq) with a0sq the material's energy scale
// (kappa + 4 mu / 3) / rho0, the squared P-wave speed at rest: in a cell at rest e and
// |v|^2/2 are at rounding level and the sign of eps is noise
template <int D>
__device__ __forceinline__ int pad_state(const double (&v)[D], double e, const double (&F)[D * D], double V,
                                         double a0sq) {
    // finite: exponent field below all ones, tested on the high words with integer operations
    auto expo = [](double x) { return (unsigned)__double2hiint(x) & 0x7ff00000u; };
    unsigned inf = (expo(e) + 0x00100000u) | (expo(V) + 0x00100000u);
#pragma unroll
    for (int i = 0; i < D; ++i) inf |= expo(v[i]) + 0x00100000u;
#pragma unroll
    for (int i = 0; i < D * D; ++i) inf |= expo(F[i]) + 0x00100000u;
    // V finite here: V > 0 exactly when its bits are a positive integer
    if ((inf & 0x80000000u) || __double_as_longlong(V) <= 0 || !(det<D>(F) > 0.0)) return 2;
    double ke = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) ke += 0.5 * v[i] * v[i];
    const double eps = e - ke;
    // finite operands: the comparisons on order keys (integer pipe) equal the FP64 ones
    const double scale = key_value(max(max(order_key(fabs(e)), order_key(ke)), order_key(a0sq)));
    return order_key(eps) >= order_key(-1e-10 * scale) ? 0 : 1;
}

// ---------------------------------------------------------------------------------------
// Stiffened gas (Eq. EOS_stiffened_gas, incomplete form): p = (gamma - 1) rho eps_v -
// gamma p_inf with rho = rho0 / det F and eps_v = eps - Psi_s(F), eps the specific internal
// energy and Psi_s the shear energy of the family; T = -p I + the family's shear stress;
// sound speed a^2 = (gamma (p + p_inf) + 4 mu / (3 J)) / rho.
// ---------------------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ double shear_energy(const Prm &prm, const double (&F)[D * D], double mu) {
    return prm.shear_a == -1.0 ? free_energy<D>(F, prm.rho0, mu, 0.0)
                               : free_energy_family<D>(F, prm.rho0, mu, 0.0, prm.shear_a);
}

template <int D>
__device__ __forceinline__ double sg_pressure(const Prm &prm, const double (&F)[D * D], double mu, double eps) {
    const double J = det<D>(F);
    return (prm.gamma - 1.0) * (prm.rho0 / J) * (eps - shear_energy<D>(prm, F, mu)) - prm.gamma * prm.pinf;
}

template <int D>
__device__ __forceinline__ void stress_sg(const Prm &prm, const double (&F)[D * D], double mu, double eps,
                                          double (&T)[D * D]) {
    if (prm.shear_a == -1.0) stress<D>(F, mu, 0.0, T);  // shear part alone
    else stress_family<D>(F, mu, 0.0, prm.shear_a, T);
    const double p = sg_pressure<D>(prm, F, mu, eps);
#pragma unroll
    for (int i = 0; i < D; ++i) T[i * D + i] -= p;
}

template <int D>
__device__ __forceinline__ double impedance_sg(const Prm &prm, const double (&F)[D * D], double rho, double mu,
                                               double eps) {
    const double J = det<D>(F);
    const double p = sg_pressure<D>(prm, F, mu, eps);
    return sqrt(rho * (prm.gamma * (p + prm.pinf) + (4.0 / 3.0) * mu / J));
}

// the material's energy scale at rest for the PAD tolerance: the squared P-wave speed
__device__ __forceinline__ double a0sq_of(const Prm &prm, double mu, double kappa) {
    return prm.eos ? (prm.gamma * (prm.p0 + prm.pinf) + (4.0 / 3.0) * mu) * prm.irho0
                   : (kappa + (4.0 / 3.0) * mu) * prm.irho0;
}

}  // namespace lmood
