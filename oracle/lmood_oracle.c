/*
 * lmood_oracle.c -- plain, slow, FP64 CPU reference of one explicit time step of the
 * cell-centered Lagrangian ADER-MOOD scheme for neo-Hookean hyper-elasticity
 * (Boscheri, Loubere, Maire, arXiv 2104.02139) on triangle (d=2) and tetrahedral (d=3)
 * meshes.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the oracle that the CUDA library is checked
 * against. Only the test-suite, the smoke check and the CPU-baseline leg of the benchmark
 * may load it. It shares no code, header, table or helper with the CUDA path.
 *
 * Style: one function per passage of the paper, in the paper's order and notation,
 * plain loops, arrays of structures, no fusion, sums in a fixed order (ascending cell id
 * around a node), compiled with -ffp-contract=off. Per-entity loops carry an OpenMP
 * pragma; every iteration writes only its own entity, so the result does not depend on
 * the thread count.
 *
 * Readings of passages that are garbled, ambiguous or deferred to another paper (each is
 * also listed in the design notes):
 *  R1  the state stores the deformation gradient F (d x d; 2D is plane strain, F33 = 1);
 *      B = F F^t. The Crank-Nicolson update of B (Eq. CN_B) is applied to F:
 *      (I - dt/2 L^{n+1}) F^{n+1} = (I + dt/2 L^n) F^n, with the dt/2 on the left that the
 *      printed second line drops.
 *  R2  L_c is the velocity gradient with L_ij = dv_i/dx_j, i.e. (1/|w_c|) sum_p v_p (x) l n
 *      (the transpose of the printed ln (x) v_p, which is what dF/dt = L F needs).
 *  R3  volumetric coefficient: Psi_v = kappa/(4 rho0) ((J-1)^2 + (log J)^2) with
 *      kappa = lambda + 2 mu / 3 (small-strain bulk modulus), so the scheme reduces to
 *      Lame (lambda, mu) linear elasticity at small strain; vol_coeff = 1 selects the
 *      printed kappa = mu (Eq. EOS_neoHook).
 *  R4  sound speed a^2 = (K(J) + 4 mu / (3 J)) / rho with K = -J dp/dJ; z_c = rho_c a_c at t^n.
 *  R5  M_cp = z_c sum_{f in F(c) cap F(p)} l_cpf n_cpf (x) n_cpf (the printed extra sum over
 *      C(p) in Eq. Mcp is dropped); l_cpf n_cpf = (1/d) x outward area vector of face f.
 *  R6  the stress term of Eq. nodal_solver^n is summed over C(p); x^{n+1} = x^n + dt v*_p.
 *  R7  tau^{n+1} = |w_c(x^{n+1})| / m_c: the GCL-exact form of Eq. tau_c^n (equal to
 *      tau^n + dt/m sum (ln)(x^{n+1/2}) . v*_p in 2D).
 *  R8  ADER predictor (details are deferred to another paper): cell-local second-order
 *      Cauchy-Kowalevski step on the P1 reconstruction with frozen geometry:
 *      v*_cp = v_h(x_p) + dt/2 (1/m_c) sum_q T(F_h(x_q)) (ln)_cq,
 *      F*_cp = F_h(x_p) + dt/2 L^_c F_c with L^_c the reconstructed velocity gradient,
 *      T*_cp = T(F*_cp). First-order (P0) cells use v*_cp = v_c^n, T*_cp = T(F_c^n).
 *      The paper gives no formula to compare with; the form is pinned by what the method must
 *      do (tests/test_oracle_predictor.py): reproduce to round-off the exact homogeneous
 *      motion x = (I + t L) F0 X (uniform stress, constant particle velocities), and approach
 *      small-amplitude elastic P and S waves at (x_p, t^{n+1/2}) at second order in h.
 *  R9  reconstruction: least squares about cell centroids over the stencil V_c = all cells
 *      sharing a node with c (the "Voronoi neighbours" of Sect. "Algorithm"; the same set
 *      bounds the RDMP), each neighbour weighted by the number of nodes it shares with c
 *      (i.e. unweighted over the (node, neighbour) pairs), for v and F only; a near-singular
 *      normal matrix gives zero slopes. Face neighbours alone give an observed order near 1.3
 *      on irregular meshes, below the table of Sect. "2D swinging plate"; this stencil gives
 *      about 2 with or without the weights (the paper gives none).
 *  R10 v_p^n is stored per node; v_p^{n+1} = 2 v*_p - v_p^n; v_p^0 is the first-order
 *      nodal solution at t^0.
 *  R11 MOOD (the detection thresholds of Eqs. PAD and RDMP are pinned by closed-form cases
 *      in the tests; the CUDA path's masks are compared with these at every step): cascade P1 -> P0
 *      (default) or, as in Sect. "Limiting: a posteriori MOOD loop",
 *      P1 -> P1 with Barth-Jespersen limited slopes -> P0 (order codes 2, 3, 1). The limiter
 *      scales each field's slope by the largest factor <= 1 that keeps its values at the
 *      cell's nodes within the field's range over the stencil and the cell (at t^n).
 *      Troubled cells move one level down; the step is recomputed
 *      from t^n with the new order mask (neighbours keep their order but see the new node
 *      velocities); repeat until no new troubled cell. A P0 candidate that cannot be
 *      advanced further (non-finite value, tau <= 0 or det F <= 0) is a parachute failure;
 *      a P0 candidate whose only defect is eps < 0 is accepted and counted (eps does not
 *      enter the stress of this model).
 *  R12 PAD: finite values, tau > 0, det F > 0, eps = e - |v|^2/2 >= -1e-10 max(|e|, |v|^2/2,
 *      a0^2) with a0^2 = (kappa + 4 mu / 3) / rho0 the squared P-wave speed at rest (the
 *      material's energy scale: in a cell at rest e and |v|^2/2 are both at rounding level,
 *      and eps's sign is noise); theta is not modelled. RDMP on rho over V_c and c at t^n,
 *      delta0 absolute.
 *  R13 dt^{n+1} = min(C_CFL min L_c/a_c, C_v dt^n min V^n/|V^{n+1}-V^n|, (1+C_i) dt^n),
 *      evaluated on the accepted state; dt^0 is the acoustic bound.
 *  R14 BCs: per node, clamped > slip > free; k independent slip planes leave the
 *      intersection subspace; the node velocity is the Galerkin solution of
 *      M_p v_p = b_p on that subspace (Eq. sBC1).
 *  R17 boundary conditions that change type by a distance function (Sect. "Boundary
 *      condition treatments"): faces tagged 6 are traction-free, but a node of such a face
 *      whose distance to a contact wall (a plane) is below eps at x^n and whose nodal
 *      velocity (after the other conditions) points into the wall gets v*_p . n = 0 for the
 *      step, with the multiplier of R15 (d = n, g = 0): the wall does no work; the node
 *      detaches when its velocity points away from the wall again.
 *  R18 stiffened gas (Eq. EOS_stiffened_gas, the incomplete form): p = (gamma - 1) rho eps_v -
 *      gamma p_inf, rho = rho0 / det F, eps_v = e - |v|^2/2 - Psi_s(F) (the volumetric part of
 *      the specific internal energy; Psi_s the shear energy of the family); T = -p I + the
 *      family's shear stress. The predictor evaluates it with the cell's eps at t^n (pass 1)
 *      and eps advanced half a step by T_c : L^ / rho (pass 2); sound speed a^2 = (gamma
 *      (p + p_inf) + 4 mu / (3 J)) / rho; PAD also asks p + p_inf > 0; the initial eps_v
 *      comes from an initial pressure p0.
 *  R16 shear energy family (Eq. familiy_energies, any a; a = -1 neo-Hookean, the default):
 *      T = -p I + (mu/J) dev(c1 Bbar - c2 Bbar^2), c1 = -a + (1+a) I1 I2 / 3,
 *      c2 = (1+a) I2 / 3 (the Cauchy stress of an isotropic energy of Bbar's invariants);
 *      every member has shear modulus mu at small strain, so the impedance keeps the sound
 *      speed of R4.
 *  R15 traction, pressure and prescribed-velocity faces (Eqs. pBC, vBC1, vBC), with N_f
 *      the face's outward area vector at x^n and each of its d nodes taking N_f / d:
 *      a traction vector t_f adds |N_f| t_f / d to b_p, a pressure p_f adds -p_f N_f / d
 *      (the external force on the node's share of the face); prescribed-velocity faces
 *      give d_p = sum N_f / d and g_p = sum V_f . N_f / d, and v*_p = K b_p - T K d_p with
 *      T = (K b_p . d_p - g_p) / (K d_p . d_p), K the solve of R14 (so v*_p . d_p = g_p;
 *      skipped when K d_p . d_p = 0, e.g. at clamped nodes). Hierarchy: clamped >
 *      prescribed velocity > slip > free; traction and pressure forces add at any node.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

/* The scalar type of every quantity the scheme computes. This file is the oracle as a plain C
 * program with real = double. The tangent build (lmood_tangent.cpp) compiles the same file as
 * C++ with real a dual number (a value and a directional derivative), so that the oracle's own
 * step also gives the exact derivative of its map: the CPU reference for the library's
 * adjoint. The parameters of the scheme (OrcParams) stay double. */
#ifndef ORC_REAL_DEFINED
typedef double real;
#endif

/* typed allocations (valid C and C++) */
#define ORC_NEW(T, n) ((T *)malloc(sizeof(T) * (size_t)(n)))
#define ORC_ZNEW(T, n) ((T *)calloc((size_t)(n), sizeof(T)))

#define MAXD 3
#define MAXV 4

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_MESH = 2, ORC_ERR_PARACHUTE = 5, ORC_ERR_MOOD_ITERS = 6 };

typedef struct {
    double cfl, Cv, Ci, delta0, delta1, dt_fixed;
    int max_mood_iters; /* MOOD iterations allowed per step                          */
    int order;          /* 2: P1 with MOOD cascade to P0; 1: first order everywhere  */
    int mood;           /* 1: detection on; 0: unlimited (no detection)              */
    int vol_coeff;      /* 0: kappa = lambda + 2 mu / 3; 1: kappa = mu (printed)      */
    int cascade;        /* 2: P1 -> P0; 3: P1 -> P1 with Barth-Jespersen slopes -> P0     */
    double shear_a;     /* a of the shear energy family (Eq. familiy_energies); -1: neo-Hookean */
    int eos;            /* volumetric law: 0 Eq. EOS_neoHook, 1 stiffened gas (reading R18) */
    double gamma, p_inf, p0; /* stiffened gas: gamma, p_infinity, initial pressure          */
} OrcParams;

typedef struct {
    real t, dt_used, dt_next;
    long step;
    int n_troubled, n_p0, mood_iters, n_parachute, n_p0_eps, n_lim;
    real mass, mom[3], energy;
} OrcInfo;

typedef struct {
    int d, nv;
    long np, nc;
    int *c2n;              /* [nc][nv]                                                */
    long *n2c_off;         /* [np+1]                                                  */
    long *n2c_cell;        /* corners around a node, ascending cell id                */
    int *n2c_k;            /* local vertex index of the node in that cell             */
    long *st_off, *st_idx; /* reconstruction stencil V_c                              */
    int *bc_ndof;          /* per node: number of free velocity directions (d = free) */
    real *bc_t;          /* per node: [2][3] tangent vectors spanning the free space */
    real *x0;            /* [np][d] initial positions                                */
    long nb;               /* boundary faces                                          */
    int *bf_nodes;         /* [nb][d] face nodes, ordered so that the face's area vector
                              points out of the mesh (reading R15)                     */
    int *bf_tag;           /* [nb] 0 free, 1 slip, 2 clamped, 3 traction, 4 pressure,
                              5 prescribed velocity, 6 contact (free until it touches a
                              contact wall)                                             */
    real *bf_val;        /* [nb][d] traction vector / pressure (first entry) /
                              prescribed velocity vector; zero until set               */
    long *nbf_off, *nbf_idx; /* boundary faces around each node, ascending face id     */
    int n_contact;         /* contact walls for faces tagged 6 (reading R17)          */
    real contact[4][6];  /* point, unit normal from the wall into the body          */
    real contact_eps;    /* distance threshold                                      */
} OrcMesh;

typedef struct {
    OrcMesh *M;
    OrcParams prm;
    real rho0, lam;
    real *mu;                   /* [nc]                                         */
    real *m;                    /* [nc] constant cell masses                    */
    real *x, *vp;               /* [np][d] positions and v_p^n                  */
    real *v, *e, *F, *tau;      /* [nc][d], [nc], [nc][d*d], [nc]               */
    real t, dt;
    long step;
    /* last accepted step's intermediates (for kernel-level parity) */
    int *order;                   /* [nc] 1 or 2                                  */
    real *pkM, *pkR;            /* [nc][nv][d*d], [nc][nv][d]                   */
    real *vstar;                /* [np][d]                                      */
    OrcInfo last;
} OrcState;

/* --------------------------------------------------------------------------------------
 * small dense algebra
 * ------------------------------------------------------------------------------------ */
static real det_n(int d, const real *A) {
    if (d == 2) return A[0] * A[3] - A[1] * A[2];
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}

/* inverse by adjugate / determinant; returns the determinant */
static real inv_n(int d, const real *A, real *Ai) {
    real det = det_n(d, A);
    if (d == 2) {
        Ai[0] = A[3] / det; Ai[1] = -A[1] / det;
        Ai[2] = -A[2] / det; Ai[3] = A[0] / det;
    } else {
        Ai[0] = (A[4] * A[8] - A[5] * A[7]) / det;
        Ai[1] = (A[2] * A[7] - A[1] * A[8]) / det;
        Ai[2] = (A[1] * A[5] - A[2] * A[4]) / det;
        Ai[3] = (A[5] * A[6] - A[3] * A[8]) / det;
        Ai[4] = (A[0] * A[8] - A[2] * A[6]) / det;
        Ai[5] = (A[2] * A[3] - A[0] * A[5]) / det;
        Ai[6] = (A[3] * A[7] - A[4] * A[6]) / det;
        Ai[7] = (A[1] * A[6] - A[0] * A[7]) / det;
        Ai[8] = (A[0] * A[4] - A[1] * A[3]) / det;
    }
    return det;
}

static void matmul_n(int d, const real *A, const real *B, real *C) {
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            real s = 0.0;
            for (int k = 0; k < d; ++k) s += A[i * d + k] * B[k * d + j];
            C[i * d + j] = s;
        }
}

static void matvec_n(int d, const real *A, const real *x, real *y) {
    for (int i = 0; i < d; ++i) {
        real s = 0.0;
        for (int k = 0; k < d; ++k) s += A[i * d + k] * x[k];
        y[i] = s;
    }
}

/* --------------------------------------------------------------------------------------
 * Geometry of one simplex (Sect. "Mesh and notation", Eq. def_lcpncp).
 *   xs[k][d]   vertex positions, positively oriented
 *   V          measure |w_c|
 *   xc         centroid (vertex average)
 *   N[k][d]    outward area vector of the face opposite vertex k
 *   ln[k][d]   corner vector l_cp n_cp = sum over faces f containing p of l_cpf n_cpf,
 *              with l_cpf n_cpf = N_f / d (each face is split evenly among its d vertices)
 *   Lc         in-sphere diameter 2 d |w_c| / sum_f |N_f|
 * ------------------------------------------------------------------------------------ */
void orc_cell_geometry(int d, const real *xs, real *V, real *xc, real *N, real *ln, real *Lc) {
    int nv = d + 1;
    for (int a = 0; a < d; ++a) {
        real s = 0.0;
        for (int k = 0; k < nv; ++k) s += xs[k * d + a];
        xc[a] = s / nv;
    }
    if (d == 2) {
        real e1x = xs[2] - xs[0], e1y = xs[3] - xs[1];
        real e2x = xs[4] - xs[0], e2y = xs[5] - xs[1];
        *V = 0.5 * (e1x * e2y - e1y * e2x);
        for (int k = 0; k < 3; ++k) {
            /* face opposite k is the edge a -> b traversed counter-clockwise */
            int a = (k + 1) % 3, b = (k + 2) % 3;
            N[k * 2 + 0] = xs[b * 2 + 1] - xs[a * 2 + 1];
            N[k * 2 + 1] = xs[a * 2 + 0] - xs[b * 2 + 0];
        }
    } else {
        real e[3][3];
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) e[k][a] = xs[(k + 1) * 3 + a] - xs[a];
        real cr[3] = {e[1][1] * e[2][2] - e[1][2] * e[2][1], e[1][2] * e[2][0] - e[1][0] * e[2][2],
                        e[1][0] * e[2][1] - e[1][1] * e[2][0]};
        *V = (e[0][0] * cr[0] + e[0][1] * cr[1] + e[0][2] * cr[2]) / 6.0;
        for (int k = 0; k < 4; ++k) {
            int f[3], q = 0;
            for (int j = 0; j < 4; ++j)
                if (j != k) f[q++] = j;
            real u[3], w[3], n[3];
            for (int a = 0; a < 3; ++a) {
                u[a] = xs[f[1] * 3 + a] - xs[f[0] * 3 + a];
                w[a] = xs[f[2] * 3 + a] - xs[f[0] * 3 + a];
            }
            n[0] = 0.5 * (u[1] * w[2] - u[2] * w[1]);
            n[1] = 0.5 * (u[2] * w[0] - u[0] * w[2]);
            n[2] = 0.5 * (u[0] * w[1] - u[1] * w[0]);
            /* outward: away from the opposite vertex k */
            real s = 0.0;
            for (int a = 0; a < 3; ++a) s += n[a] * (xs[k * 3 + a] - xs[f[0] * 3 + a]);
            if (s > 0)
                for (int a = 0; a < 3; ++a) n[a] = -n[a];
            for (int a = 0; a < 3; ++a) N[k * 3 + a] = n[a];
        }
    }
    real area = 0.0;
    for (int k = 0; k < nv; ++k) {
        real s = 0.0;
        for (int a = 0; a < d; ++a) s += N[k * d + a] * N[k * d + a];
        area += sqrt(s);
    }
    *Lc = 2.0 * d * (*V) / area;
    for (int p = 0; p < nv; ++p)
        for (int a = 0; a < d; ++a) {
            real s = 0.0;
            for (int f = 0; f < nv; ++f)
                if (f != p) s += N[f * d + a] / d;
            ln[p * d + a] = s;
        }
}

/* --------------------------------------------------------------------------------------
 * Constitutive law (Sect. "Volumetric shear strain decomposition", "Examples of
 * constitutive laws"): T = -p I + T_0 with
 *   p   = -(kappa/2) (J - 1 + log J / J)                 (Eq. EOS_neoHook, reading R3)
 *   T_0 = (mu / J) dev(Bbar),  Bbar = J^{-2/3} F F^t     (Eq. cstnh)
 * 2D is plane strain: F is embedded as diag(F, 1) and the in-plane block of T returned.
 * ------------------------------------------------------------------------------------ */
static void embed3(int d, const real *F, real *F3) {
    if (d == 3) {
        memcpy(F3, F, 9 * sizeof(real));
        return;
    }
    F3[0] = F[0]; F3[1] = F[1]; F3[2] = 0.0;
    F3[3] = F[2]; F3[4] = F[3]; F3[5] = 0.0;
    F3[6] = 0.0;  F3[7] = 0.0;  F3[8] = 1.0;
}

void orc_stress(int d, const real *F, real mu, real kappa, real *T) {
    real F3[9], B[9], T3[9];
    embed3(d, F, F3);
    real J = det_n(3, F3);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            real s = 0.0;
            for (int k = 0; k < 3; ++k) s += F3[i * 3 + k] * F3[j * 3 + k];
            B[i * 3 + j] = s;
        }
    real Jm23 = pow(J, -2.0 / 3.0);
    real trBbar = Jm23 * (B[0] + B[4] + B[8]);
    real p = -0.5 * kappa * (J - 1.0 + log(J) / J);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            real Bbar0 = Jm23 * B[i * 3 + j] - (i == j ? trBbar / 3.0 : 0.0);
            T3[i * 3 + j] = (i == j ? -p : 0.0) + mu / J * Bbar0;
        }
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) T[i * d + j] = T3[i * 3 + j];
}

/* Cauchy stress of the shear energy family of Eq. familiy_energies (reading R16),
 *   rho0 Psi_s = (mu/4) (-2a (I1 - 3) + (1+a)/3 (I2^2 - 9)),  I1, I2 the invariants of Bbar,
 * with the volumetric part of Eq. EOS_neoHook: for an isotropic W(I1, I2) of Bbar,
 * T = -p I + (2/J) dev((W_1 + I1 W_2) Bbar - W_2 Bbar^2), W_1 = -a mu/2, W_2 = (1+a) mu I2/6,
 * i.e. T = -p I + (mu/J) dev(c1 Bbar - c2 Bbar^2), c1 = -a + (1+a) I1 I2/3, c2 = (1+a) I2/3.
 * a = -1 is the neo-Hookean law of orc_stress. 2D is plane strain (F33 = 1). */
void orc_stress_a(int d, const real *F, real mu, real kappa, real a, real *T) {
    if (a == -1.0) {
        orc_stress(d, F, mu, kappa, T);
        return;
    }
    real F3[9], B[9], B2[9], T3[9];
    embed3(d, F, F3);
    real J = det_n(3, F3);
    real Jm23 = pow(J, -2.0 / 3.0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            real s = 0.0;
            for (int k = 0; k < 3; ++k) s += F3[i * 3 + k] * F3[j * 3 + k];
            B[i * 3 + j] = Jm23 * s;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            real s = 0.0;
            for (int k = 0; k < 3; ++k) s += B[i * 3 + k] * B[k * 3 + j];
            B2[i * 3 + j] = s;
        }
    real I1 = B[0] + B[4] + B[8], trB2 = B2[0] + B2[4] + B2[8];
    real I2 = 0.5 * (I1 * I1 - trB2);
    real c1 = -a + (1.0 + a) * I1 * I2 / 3.0, c2 = (1.0 + a) * I2 / 3.0;
    real X[9], trX = 0.0;
    for (int i = 0; i < 9; ++i) X[i] = c1 * B[i] - c2 * B2[i];
    trX = X[0] + X[4] + X[8];
    real p = -0.5 * kappa * (J - 1.0 + log(J) / J);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            T3[i * 3 + j] = (i == j ? -p : 0.0) + mu / J * (X[i * 3 + j] - (i == j ? trX / 3.0 : 0.0));
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) T[i * d + j] = T3[i * 3 + j];
}

/* specific free energy Psi = Psi_v + Psi_s (Eqs. EOS_neoHook and familiy_energies with
 * a = -1): Psi_v = kappa/(4 rho0) ((J-1)^2 + log^2 J), Psi_s = mu/(2 rho0) (I1(Bbar) - 3) */
real orc_free_energy(int d, const real *F, real rho0, real mu, real kappa) {
    real F3[9];
    embed3(d, F, F3);
    real J = det_n(3, F3);
    real trB = 0.0;
    for (int i = 0; i < 9; ++i) trB += F3[i] * F3[i];
    real I1bar = pow(J, -2.0 / 3.0) * trB;
    real lj = log(J);
    return kappa / (4.0 * rho0) * ((J - 1.0) * (J - 1.0) + lj * lj) + mu / (2.0 * rho0) * (I1bar - 3.0);
}

/* the same with the shear energy of Eq. familiy_energies for any a (reading R16) */
real orc_free_energy_a(int d, const real *F, real rho0, real mu, real kappa, real a) {
    if (a == -1.0) return orc_free_energy(d, F, rho0, mu, kappa);
    real F3[9], B[9];
    embed3(d, F, F3);
    real J = det_n(3, F3);
    real Jm23 = pow(J, -2.0 / 3.0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            real s = 0.0;
            for (int k = 0; k < 3; ++k) s += F3[i * 3 + k] * F3[j * 3 + k];
            B[i * 3 + j] = Jm23 * s;
        }
    real I1 = B[0] + B[4] + B[8], trB2 = 0.0;
    for (int i = 0; i < 9; ++i) trB2 += B[i] * B[i];  /* B symmetric: tr(B^2) = sum B_ij^2 */
    real I2 = 0.5 * (I1 * I1 - trB2);
    real lj = log(J);
    return kappa / (4.0 * rho0) * ((J - 1.0) * (J - 1.0) + lj * lj) +
           mu / (4.0 * rho0) * (-2.0 * a * (I1 - 3.0) + (1.0 + a) / 3.0 * (I2 * I2 - 9.0));
}

/* sound speed, reading R4: a^2 = (K + 4 mu / (3 J)) / rho, K = (kappa/2)(J + (1 - log J)/J) */
real orc_sound_speed(int d, const real *F, real rho, real mu, real kappa) {
    real F3[9];
    embed3(d, F, F3);
    real J = det_n(3, F3);
    real K = 0.5 * kappa * (J + (1.0 - log(J)) / J);
    return sqrt((K + 4.0 * mu / (3.0 * J)) / rho);
}

static real kappa_of(const OrcState *S, long c) {
    return S->prm.vol_coeff == 1 ? S->mu[c] : S->lam + 2.0 * S->mu[c] / 3.0;
}

/* stiffened gas (Eq. EOS_stiffened_gas; reading R18): p = (gamma - 1) rho eps_v - gamma p_inf
 * with rho = rho0 / det F and eps_v = eps - Psi_s(F) the volumetric part of the specific
 * internal energy eps = e - |v|^2/2 (Psi_s the shear energy of Eq. familiy_energies) */
static real sg_pressure(const OrcState *S, long c, const real *F, real eps) {
    int d = S->M->d;
    real F3[9];
    embed3(d, F, F3);
    real J = det_n(3, F3);
    real eps_s = orc_free_energy_a(d, F, S->rho0, S->mu[c], 0.0, S->prm.shear_a);
    return (S->prm.gamma - 1.0) * (S->rho0 / J) * (eps - eps_s) - S->prm.gamma * S->prm.p_inf;
}

/* the material's Cauchy stress at F with specific internal energy eps (used by the stiffened
 * gas only): Eqs. EOS_neoHook + familiy_energies, or the stiffened-gas pressure plus the
 * family's shear stress */
static void stress_state(const OrcState *S, long c, const real *F, real eps, real *T) {
    int d = S->M->d;
    if (S->prm.eos == 0) {
        orc_stress_a(d, F, S->mu[c], kappa_of(S, c), S->prm.shear_a, T);
        return;
    }
    orc_stress_a(d, F, S->mu[c], 0.0, S->prm.shear_a, T);  /* shear part (no volumetric term) */
    real p = sg_pressure(S, c, F, eps);
    for (int i = 0; i < d; ++i) T[i * d + i] -= p;
}

/* sound speed of the material (readings R4, R18): stiffened gas a^2 = (gamma (p + p_inf) +
 * 4 mu / (3 J)) / rho */
static real sound_speed_state(const OrcState *S, long c, const real *F, real rho, real eps) {
    int d = S->M->d;
    if (S->prm.eos == 0) return orc_sound_speed(d, F, rho, S->mu[c], kappa_of(S, c));
    real F3[9];
    embed3(d, F, F3);
    real J = det_n(3, F3);
    real p = sg_pressure(S, c, F, eps);
    return sqrt((S->prm.gamma * (p + S->prm.p_inf) + 4.0 / 3.0 * S->mu[c] / J) / rho);
}

/* the material's energy scale at rest (PAD tolerance, reading R12): the squared P-wave speed */
static real a0sq_of(const OrcState *S, long c) {
    if (S->prm.eos == 0) return (kappa_of(S, c) + 4.0 / 3.0 * S->mu[c]) / S->rho0;
    return (S->prm.gamma * (S->prm.p0 + S->prm.p_inf) + 4.0 / 3.0 * S->mu[c]) / S->rho0;
}

/* --------------------------------------------------------------------------------------
 * Mesh set-up: corners around nodes, face neighbours, stencils, BC resolution
 * ------------------------------------------------------------------------------------ */
static int cmp_long(const void *a, const void *b) {
    long x = *(const long *)a, y = *(const long *)b;
    return (x > y) - (x < y);
}

/* the cells sharing at least one node with c, other than c, sorted and unique, into tmp */
static int stencil_of(const OrcMesh *M, long c, long *tmp) {
    int n = 0;
    for (int k = 0; k < M->nv; ++k) {
        int p = M->c2n[c * M->nv + k];
        for (long j = M->n2c_off[p]; j < M->n2c_off[p + 1]; ++j)
            if (M->n2c_cell[j] != c && n < 8192) tmp[n++] = M->n2c_cell[j];
    }
    qsort(tmp, n, sizeof(long), cmp_long);
    int u = 0;
    for (int i = 0; i < n; ++i)
        if (u == 0 || tmp[i] != tmp[u - 1]) tmp[u++] = tmp[i];
    return u;
}

void orc_mesh_free(OrcMesh *M) {
    if (!M) return;
    free(M->c2n); free(M->n2c_off); free(M->n2c_cell); free(M->n2c_k);
    free(M->st_off); free(M->st_idx); free(M->bc_ndof); free(M->bc_t); free(M->x0);
    free(M->bf_nodes); free(M->bf_tag); free(M->bf_val); free(M->nbf_off); free(M->nbf_idx);
    free(M);
}

/* area vector of boundary face b at positions x ([np][d]): 2D edge (q0, q1):
 * (y1 - y0, x0 - x1); 3D triangle: (1/2) (x1 - x0) x (x2 - x0); its length is the face measure */
static void face_area_vector(const OrcMesh *M, const real *x, long b, real *N) {
    int d = M->d;
    const int *q = M->bf_nodes + b * d;
    if (d == 2) {
        N[0] = x[q[1] * 2 + 1] - x[q[0] * 2 + 1];
        N[1] = x[q[0] * 2 + 0] - x[q[1] * 2 + 0];
    } else {
        real u[3], w[3];
        for (int a = 0; a < 3; ++a) {
            u[a] = x[q[1] * 3 + a] - x[q[0] * 3 + a];
            w[a] = x[q[2] * 3 + a] - x[q[0] * 3 + a];
        }
        N[0] = 0.5 * (u[1] * w[2] - u[2] * w[1]);
        N[1] = 0.5 * (u[2] * w[0] - u[0] * w[2]);
        N[2] = 0.5 * (u[0] * w[1] - u[1] * w[0]);
    }
}

/* per-node boundary conditions from the face tags (Appendix B; hierarchy clamped > slip >
 * free for the velocity subspace, reading R14; traction, pressure and prescribed velocity
 * faces act in the nodal solve, reading R15) */
static void resolve_bcs(OrcMesh *M) {
    int d = M->d;
    long np = M->np, nb = M->nb;
    int *clamped = ORC_ZNEW(int, np);
    int *nplanes = ORC_ZNEW(int, np);
    real *planes = ORC_ZNEW(real, np * 9);
    memset(M->bc_t, 0, sizeof(real) * np * 6);
    for (long b = 0; b < nb; ++b) {
        const int *fn = M->bf_nodes + b * d;
        real n[3] = {0, 0, 0};
        face_area_vector(M, M->x0, b, n);
        real nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        for (int a = 0; a < 3; ++a) n[a] /= nn;
        for (int a = 0; a < d; ++a) {
            int p = fn[a];
            if (M->bf_tag[b] == 2) clamped[p] = 1;
            if (M->bf_tag[b] == 1) {
                int dup = 0;
                for (int q = 0; q < nplanes[p]; ++q) {
                    real dot = 0.0;
                    for (int i = 0; i < 3; ++i) dot += planes[p * 9 + q * 3 + i] * n[i];
                    if (fabs(dot) > 1.0 - 1e-12) dup = 1;
                }
                if (!dup && nplanes[p] < 3) {
                    for (int i = 0; i < 3; ++i) planes[p * 9 + nplanes[p] * 3 + i] = n[i];
                    nplanes[p]++;
                }
            }
        }
    }
    for (long p = 0; p < np; ++p) {
        real *t = M->bc_t + p * 6;
        const real *n1 = planes + p * 9, *n2 = planes + p * 9 + 3;
        int k = clamped[p] ? d : nplanes[p];
        if (k >= d) {
            M->bc_ndof[p] = 0;
        } else if (k == 0) {
            M->bc_ndof[p] = d;
        } else if (d == 2) {
            M->bc_ndof[p] = 1;
            t[0] = -n1[1]; t[1] = n1[0];
        } else if (k == 1) {
            /* tangent basis of the plane: t1 = e x n normalised (e = axis least aligned with n), t2 = n x t1 */
            int ax = 0;
            for (int a = 1; a < 3; ++a)
                if (fabs(n1[a]) < fabs(n1[ax])) ax = a;
            real e[3] = {0, 0, 0};
            e[ax] = 1.0;
            real t1[3] = {e[1] * n1[2] - e[2] * n1[1], e[2] * n1[0] - e[0] * n1[2], e[0] * n1[1] - e[1] * n1[0]};
            real l1 = sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
            for (int a = 0; a < 3; ++a) t1[a] /= l1;
            real t2[3] = {n1[1] * t1[2] - n1[2] * t1[1], n1[2] * t1[0] - n1[0] * t1[2], n1[0] * t1[1] - n1[1] * t1[0]};
            real l2 = sqrt(t2[0] * t2[0] + t2[1] * t2[1] + t2[2] * t2[2]);
            for (int a = 0; a < 3; ++a) { t[a] = t1[a]; t[3 + a] = t2[a] / l2; }
            M->bc_ndof[p] = 2;
        } else {
            real l[3] = {n1[1] * n2[2] - n1[2] * n2[1], n1[2] * n2[0] - n1[0] * n2[2], n1[0] * n2[1] - n1[1] * n2[0]};
            real ll = sqrt(l[0] * l[0] + l[1] * l[1] + l[2] * l[2]);
            for (int a = 0; a < 3; ++a) t[a] = l[a] / ll;
            M->bc_ndof[p] = 1;
        }
    }
    free(clamped); free(nplanes); free(planes);
}

/* x_soa [d][np], c2n_soa [d+1][nc], bf_soa [d][nb], btag [nb] (0 free, 1 slip, 2 clamped) */
int orc_mesh_new(int d, long np, const real *x_soa, long nc, const int *c2n_soa, long nb,
                 const int *bf_soa, const int *btag, OrcMesh **out) {
    if ((d != 2 && d != 3) || np <= 0 || nc <= 0 || !out) return ORC_ERR_ARG;
    OrcMesh *M = ORC_ZNEW(OrcMesh, 1);
    int nv = d + 1;
    M->d = d; M->nv = nv; M->np = np; M->nc = nc;
    M->c2n = ORC_NEW(int, nc * nv);
    M->x0 = ORC_NEW(real, np * d);
    for (long p = 0; p < np; ++p)
        for (int a = 0; a < d; ++a) M->x0[p * d + a] = x_soa[a * np + p];
    for (long c = 0; c < nc; ++c)
        for (int k = 0; k < nv; ++k) {
            int p = c2n_soa[k * nc + c];
            if (p < 0 || p >= np) { orc_mesh_free(M); return ORC_ERR_MESH; }
            M->c2n[c * nv + k] = p;
        }
    /* positive orientation */
    for (long c = 0; c < nc; ++c) {
        real xs[MAXV * MAXD], V, xc[MAXD], N[MAXV * MAXD], ln[MAXV * MAXD], Lc;
        for (int k = 0; k < nv; ++k)
            for (int a = 0; a < d; ++a) xs[k * d + a] = M->x0[M->c2n[c * nv + k] * d + a];
        orc_cell_geometry(d, xs, &V, xc, N, ln, &Lc);
        if (!(V > 0)) { orc_mesh_free(M); return ORC_ERR_MESH; }
    }
    /* C(p): corners around each node, ascending cell id */
    M->n2c_off = ORC_ZNEW(long, np + 1);
    for (long c = 0; c < nc; ++c)
        for (int k = 0; k < nv; ++k) M->n2c_off[M->c2n[c * nv + k] + 1]++;
    for (long p = 0; p < np; ++p) M->n2c_off[p + 1] += M->n2c_off[p];
    M->n2c_cell = ORC_NEW(long, nc * nv);
    M->n2c_k = ORC_NEW(int, nc * nv);
    long *fill = ORC_NEW(long, np);
    for (long p = 0; p < np; ++p) fill[p] = M->n2c_off[p];
    for (long c = 0; c < nc; ++c)
        for (int k = 0; k < nv; ++k) {
            int p = M->c2n[c * nv + k];
            M->n2c_cell[fill[p]] = c;
            M->n2c_k[fill[p]] = k;
            fill[p]++;
        }
    free(fill);
    /* stencil V_c (reading R9): every other cell sharing at least one node with c,
     * ascending cell id (two passes: sizes, then entries; cells are independent) */
    M->st_off = ORC_ZNEW(long, nc + 1);
#pragma omp parallel
    {
        long *tmp = ORC_NEW(long, 8192);
#pragma omp for schedule(static)
        for (long c = 0; c < nc; ++c) M->st_off[c + 1] = stencil_of(M, c, tmp);
        free(tmp);
    }
    for (long c = 0; c < nc; ++c) M->st_off[c + 1] += M->st_off[c];
    M->st_idx = ORC_NEW(long, (M->st_off[nc] > 0 ? M->st_off[nc] : 1));
#pragma omp parallel
    {
        long *tmp = ORC_NEW(long, 8192);
#pragma omp for schedule(static)
        for (long c = 0; c < nc; ++c) {
            int u = stencil_of(M, c, tmp);
            memcpy(M->st_idx + M->st_off[c], tmp, sizeof(long) * u);
        }
        free(tmp);
    }
    /* boundary faces: nodes oriented outward (the face's area vector points away from the
     * vertex of its cell that is not on the face), tags, values, node -> face CSR */
    M->nb = nb;
    M->bf_nodes = ORC_NEW(int, (nb > 0 ? nb : 1) * d);
    M->bf_tag = ORC_NEW(int, (nb > 0 ? nb : 1));
    M->bf_val = ORC_ZNEW(real, (nb > 0 ? nb : 1) * d);
    for (long b = 0; b < nb; ++b) {
        int *fn = M->bf_nodes + b * d;
        for (int a = 0; a < d; ++a) {
            fn[a] = bf_soa[a * nb + b];
            if (fn[a] < 0 || fn[a] >= np) { orc_mesh_free(M); return ORC_ERR_MESH; }
        }
        if (btag[b] < 0 || btag[b] > 6) { orc_mesh_free(M); return ORC_ERR_ARG; }
        M->bf_tag[b] = btag[b];
        long owner = -1;
        int opp = -1;
        for (long j = M->n2c_off[fn[0]]; j < M->n2c_off[fn[0] + 1] && owner < 0; ++j) {
            long c = M->n2c_cell[j];
            int hits = 0, other = -1;
            for (int k = 0; k < nv; ++k) {
                int q = M->c2n[c * nv + k], on = 0;
                for (int a = 0; a < d; ++a) on |= q == fn[a];
                if (on) hits++;
                else other = q;
            }
            if (hits == d) { owner = c; opp = other; }
        }
        if (owner < 0) { orc_mesh_free(M); return ORC_ERR_MESH; }
        real N[3] = {0, 0, 0}, dot = 0.0;
        face_area_vector(M, M->x0, b, N);
        for (int a = 0; a < d; ++a) {
            real xf = 0.0;
            for (int i = 0; i < d; ++i) xf += M->x0[fn[i] * d + a];
            dot += N[a] * (xf / d - M->x0[opp * d + a]);
        }
        if (dot < 0.0) { int tmp = fn[0]; fn[0] = fn[1]; fn[1] = tmp; }
        real nn = 0.0;
        face_area_vector(M, M->x0, b, N);
        for (int a = 0; a < d; ++a) nn += N[a] * N[a];
        if (!(nn > 0.0)) { orc_mesh_free(M); return ORC_ERR_MESH; }
    }
    M->nbf_off = ORC_ZNEW(long, np + 1);
    for (long b = 0; b < nb; ++b)
        for (int a = 0; a < d; ++a) M->nbf_off[M->bf_nodes[b * d + a] + 1]++;
    for (long p = 0; p < np; ++p) M->nbf_off[p + 1] += M->nbf_off[p];
    M->nbf_idx = ORC_NEW(long, (nb > 0 ? nb * d : 1));
    {
        long *fill = ORC_NEW(long, np);
        for (long p = 0; p < np; ++p) fill[p] = M->nbf_off[p];
        for (long b = 0; b < nb; ++b)
            for (int a = 0; a < d; ++a) M->nbf_idx[fill[M->bf_nodes[b * d + a]]++] = b;
        free(fill);
    }
    M->bc_ndof = ORC_NEW(int, np);
    M->bc_t = ORC_ZNEW(real, np * 6);
    resolve_bcs(M);
    *out = M;
    return ORC_OK;
}

/* --------------------------------------------------------------------------------------
 * The step
 * ------------------------------------------------------------------------------------ */
typedef struct {
    /* geometry at x^n */
    real *V, *xc, *ln, *N, *Lc;
    /* slopes */
    real *gv, *gF;
    /* packets */
    real *pkM, *pkR;
    /* nodes */
    real *vs, *x1, *vp1;
    /* candidate */
    real *v1, *e1, *F1, *V1;
} Work;

static Work work_new(const OrcMesh *M) {
    int d = M->d, nv = M->nv;
    long nc = M->nc, np = M->np;
    Work w;
    w.V = ORC_NEW(real, nc);
    w.xc = ORC_NEW(real, nc * d);
    w.ln = ORC_NEW(real, nc * nv * d);
    w.N = ORC_NEW(real, nc * nv * d);
    w.Lc = ORC_NEW(real, nc);
    w.gv = ORC_NEW(real, nc * d * d);
    w.gF = ORC_NEW(real, nc * d * d * d);
    w.pkM = ORC_NEW(real, nc * nv * d * d);
    w.pkR = ORC_NEW(real, nc * nv * d);
    w.vs = ORC_NEW(real, np * d);
    w.x1 = ORC_NEW(real, np * d);
    w.vp1 = ORC_NEW(real, np * d);
    w.v1 = ORC_NEW(real, nc * d);
    w.e1 = ORC_NEW(real, nc);
    w.F1 = ORC_NEW(real, nc * d * d);
    w.V1 = ORC_NEW(real, nc);
    return w;
}

static void work_free(Work *w) {
    free(w->V); free(w->xc); free(w->ln); free(w->N); free(w->Lc); free(w->gv); free(w->gF);
    free(w->pkM); free(w->pkR); free(w->vs); free(w->x1); free(w->vp1); free(w->v1); free(w->e1);
    free(w->F1); free(w->V1);
}

static void gather_xs(const OrcMesh *M, const real *x, long c, real *xs) {
    for (int k = 0; k < M->nv; ++k)
        for (int a = 0; a < M->d; ++a) xs[k * M->d + a] = x[M->c2n[c * M->nv + k] * M->d + a];
}

/* 1. geometry of every cell at x^n */
static void phase_geometry(const OrcState *S, const real *x, Work *w) {
    const OrcMesh *M = S->M;
    int d = M->d, nv = M->nv;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < M->nc; ++c) {
        real xs[MAXV * MAXD];
        gather_xs(M, x, c, xs);
        orc_cell_geometry(d, xs, &w->V[c], &w->xc[c * d], &w->N[c * nv * d], &w->ln[c * nv * d], &w->Lc[c]);
    }
}

/* 2. piecewise-linear reconstruction of v and F by least squares (reading R9):
 *    G = sum_k w_k dx_k dx_k^t, slope = G^{-1} sum_k w_k dx_k (q_k - q_c), dx_k = x_k - x_c,
 *    w_k = number of nodes neighbour k shares with c */
static void phase_slopes(const OrcState *S, const int *order, Work *w) {
    const OrcMesh *M = S->M;
    int d = M->d, nq = d + d * d;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < M->nc; ++c) {
        real *gv = w->gv + c * d * d, *gF = w->gF + c * d * d * d;
        memset(gv, 0, sizeof(real) * d * d);
        memset(gF, 0, sizeof(real) * d * d * d);
        if (order[c] == 1) continue;
        real G[9] = {0}, r[12][3];
        memset(r, 0, sizeof(r));
        for (long j = M->st_off[c]; j < M->st_off[c + 1]; ++j) {
            long o = M->st_idx[j];
            /* weight: number of nodes o shares with c (sum over the (node, neighbour) pairs) */
            real wt = 0.0;
            for (int k = 0; k < M->nv; ++k)
                for (int kk = 0; kk < M->nv; ++kk)
                    if (M->c2n[c * M->nv + k] == M->c2n[o * M->nv + kk]) wt += 1.0;
            real dx[3], dq[12];
            for (int a = 0; a < d; ++a) dx[a] = w->xc[o * d + a] - w->xc[c * d + a];
            for (int i = 0; i < d; ++i) dq[i] = S->v[o * d + i] - S->v[c * d + i];
            for (int i = 0; i < d * d; ++i) dq[d + i] = S->F[o * d * d + i] - S->F[c * d * d + i];
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) G[a * d + b] += wt * dx[a] * dx[b];
            for (int q = 0; q < nq; ++q)
                for (int a = 0; a < d; ++a) r[q][a] += wt * dx[a] * dq[q];
        }
        real tr = 0.0;
        for (int a = 0; a < d; ++a) tr += G[a * d + a];
        real det = det_n(d, G);
        if (!(det > 1e-12 * pow(tr / d, d))) continue; /* degenerate stencil: first order slopes */
        real Gi[9];
        inv_n(d, G, Gi);
        for (int q = 0; q < nq; ++q) {
            real g[3];
            matvec_n(d, Gi, r[q], g);
            if (order[c] == 3) {
                /* Barth-Jespersen: largest phi <= 1 keeping q_c + phi g.(x_p - x_c) in [lo, hi] */
                real qc = q < d ? S->v[c * d + q] : S->F[c * d * d + q - d], lo = qc, hi = qc;
                for (long j = M->st_off[c]; j < M->st_off[c + 1]; ++j) {
                    long o = M->st_idx[j];
                    real qo = q < d ? S->v[o * d + q] : S->F[o * d * d + q - d];
                    lo = fmin(lo, qo);
                    hi = fmax(hi, qo);
                }
                real phi = 1.0;
                for (int k = 0; k < M->nv; ++k) {
                    int p = M->c2n[c * M->nv + k];
                    real delta = 0.0;
                    for (int a = 0; a < d; ++a) delta += g[a] * (S->x[p * d + a] - w->xc[c * d + a]);
                    if (delta > 0.0) phi = fmin(phi, (hi - qc) / delta);
                    if (delta < 0.0) phi = fmin(phi, (lo - qc) / delta);
                }
                for (int a = 0; a < d; ++a) g[a] *= phi;
            }
            real *dst = q < d ? gv + q * d : gF + (q - d) * d;
            for (int a = 0; a < d; ++a) dst[a] = g[a];
        }
    }
}

/* 3. predictor and corner packets (Sect. "Space-Time discretization --- ADER methodology",
 *    reading R8; Eqs. Mcp^n, nodal_solver^n):
 *    M_cp   = z_c sum_{f containing p} |l n|_cpf n_cpf (x) n_cpf
 *    rhs_cp = M_cp v*_cp - T*_cp (l n)_cp         so that f_cp = M_cp v*_p - rhs_cp */
/* the predictor of cell c (reading R8): v*_cp, F*_cp and T*_cp = T(F*_cp) at the cell's
 * corners for its order (P0: v*_cp = v_c, F*_cp = F_c); eps: the cell's specific internal
 * energy at t^n */
static void predict_cell(const OrcState *S, const Work *w, long c, int order_c, real dt, real eps,
                         real vstar[MAXV][MAXD], real Fstar[MAXV][9], real Tstar[MAXV][9]) {
    const OrcMesh *M = S->M;
    int d = M->d, nv = M->nv, dd = d * d;
    const real *ln = w->ln + c * nv * d;
    const real *vc = S->v + c * d, *Fc = S->F + c * dd;
    real rho = S->m[c] / w->V[c];
    if (order_c != 1) {
        const real *gv = w->gv + c * dd, *gF = w->gF + c * dd * d;
        real vh[MAXV][MAXD], Fh[MAXV][9], dvdt[MAXD] = {0, 0, 0}, dFdt[9];
        for (int k = 0; k < nv; ++k) {
            int p = M->c2n[c * nv + k];
            real dx[3];
            for (int a = 0; a < d; ++a) dx[a] = S->x[p * d + a] - w->xc[c * d + a];
            for (int i = 0; i < d; ++i) {
                real s = vc[i];
                for (int a = 0; a < d; ++a) s += gv[i * d + a] * dx[a];
                vh[k][i] = s;
            }
            for (int i = 0; i < dd; ++i) {
                real s = Fc[i];
                for (int a = 0; a < d; ++a) s += gF[i * d + a] * dx[a];
                Fh[k][i] = s;
            }
            real Tk[9], Tn[3];
            stress_state(S, c, Fh[k], eps, Tk);
            matvec_n(d, Tk, ln + k * d, Tn);
            for (int i = 0; i < d; ++i) dvdt[i] += Tn[i];
        }
        for (int i = 0; i < d; ++i) dvdt[i] /= S->m[c];
        matmul_n(d, gv, Fc, dFdt); /* dF/dt = L^ F (Eq. GCLL) with L^ the reconstructed gradient */
        /* stiffened gas: the internal energy at the half step, d eps/dt = T : L^ / rho with
         * the cell's stress (reading R18) */
        real eps_h = eps;
        if (S->prm.eos != 0) {
            real Tc[9], pw = 0.0;
            stress_state(S, c, Fc, eps, Tc);
            for (int i = 0; i < dd; ++i) pw += Tc[i] * gv[i];
            eps_h = eps + 0.5 * dt * pw / rho;
        }
        for (int k = 0; k < nv; ++k) {
            real *Fs = Fstar[k];
            for (int i = 0; i < d; ++i) vstar[k][i] = vh[k][i] + 0.5 * dt * dvdt[i];
            for (int i = 0; i < dd; ++i) Fs[i] = Fh[k][i] + 0.5 * dt * dFdt[i];
            stress_state(S, c, Fs, eps_h, Tstar[k]);
        }
    } else {
        real T0[9];
        stress_state(S, c, Fc, eps, T0);
        for (int k = 0; k < nv; ++k) {
            for (int i = 0; i < d; ++i) vstar[k][i] = vc[i];
            memcpy(Fstar[k], Fc, sizeof(real) * dd);
            memcpy(Tstar[k], T0, sizeof(real) * dd);
        }
    }
}

static void phase_packets(const OrcState *S, const int *order, real dt, Work *w) {
    const OrcMesh *M = S->M;
    int d = M->d, nv = M->nv, dd = d * d;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < M->nc; ++c) {
        const real *ln = w->ln + c * nv * d, *N = w->N + c * nv * d;
        const real *vc = S->v + c * d, *Fc = S->F + c * dd;
        real rho = S->m[c] / w->V[c];
        real eps = S->e[c];  /* specific internal energy (enters the stiffened gas only) */
        for (int i = 0; i < d; ++i) eps -= 0.5 * vc[i] * vc[i];
        real z = rho * sound_speed_state(S, c, Fc, rho, eps);
        real vstar[MAXV][MAXD], Fstar[MAXV][9], Tstar[MAXV][9];
        predict_cell(S, w, c, order[c], dt, eps, vstar, Fstar, Tstar);
        for (int k = 0; k < nv; ++k) {
            real *Mk = w->pkM + (c * nv + k) * dd, *Rk = w->pkR + (c * nv + k) * d;
            memset(Mk, 0, sizeof(real) * dd);
            for (int f = 0; f < nv; ++f) {
                if (f == k) continue;
                real lnf[3], l = 0.0;
                for (int a = 0; a < d; ++a) { lnf[a] = N[f * d + a] / d; l += lnf[a] * lnf[a]; }
                l = sqrt(l);
                for (int a = 0; a < d; ++a)
                    for (int b = 0; b < d; ++b) Mk[a * d + b] += z * lnf[a] * lnf[b] / l;
            }
            real Mv[3], Tn[3];
            matvec_n(d, Mk, vstar[k], Mv);
            matvec_n(d, Tstar[k], ln + k * d, Tn);
            for (int i = 0; i < d; ++i) Rk[i] = Mv[i] - Tn[i];
        }
    }
}

/* 4. nodal solver with BCs (Eqs. nodal_solver^n, sBC1, pBC, vBC1, vBC; readings R6, R10,
 *    R14, R15): M_p = sum_c M_cp, b_p = sum_c rhs_cp + the forces of the traction and
 *    pressure faces around p; v*_p = K b_p with K the Galerkin solve on the node's free
 *    subspace; with prescribed-velocity faces around p, v*_p = K b_p - T_p K d_p with T_p
 *    chosen so that v*_p . d_p = g_p; x^{n+1} = x^n + dt v*_p, v_p^{n+1} = 2 v*_p - v_p^n */
static void solve_K(const OrcMesh *M, const real *Mp, long p, const real *rhs, real *out) {
    int d = M->d;
    int nf = M->bc_ndof[p];
    if (nf == d) {
        real Mi[9];
        inv_n(d, Mp, Mi);
        matvec_n(d, Mi, rhs, out);
    } else if (nf == 0) {
        for (int i = 0; i < d; ++i) out[i] = 0.0;
    } else {
        const real *t = M->bc_t + p * 6;
        real A[4], r[2], al[2];
        for (int i = 0; i < nf; ++i) {
            r[i] = 0.0;
            for (int a = 0; a < d; ++a) r[i] += t[3 * i + a] * rhs[a];
            for (int j = 0; j < nf; ++j) {
                real Mtj[3], s = 0.0;
                matvec_n(d, Mp, t + 3 * j, Mtj);
                for (int a = 0; a < d; ++a) s += t[3 * i + a] * Mtj[a];
                A[i * nf + j] = s;
            }
        }
        if (nf == 1) {
            al[0] = r[0] / A[0];
        } else {
            real Ai[4];
            inv_n(2, A, Ai);
            al[0] = Ai[0] * r[0] + Ai[1] * r[1];
            al[1] = Ai[2] * r[0] + Ai[3] * r[1];
        }
        for (int a = 0; a < d; ++a) {
            real s = 0.0;
            for (int i = 0; i < nf; ++i) s += al[i] * t[3 * i + a];
            out[a] = s;
        }
    }
}

static void node_solve_one(const OrcMesh *M, const real *x, const real *pkM, const real *pkR, long p,
                           real *vs) {
    int d = M->d, nv = M->nv, dd = d * d;
    real Mp[9] = {0}, bp[3] = {0, 0, 0};
    for (long j = M->n2c_off[p]; j < M->n2c_off[p + 1]; ++j) {
        long c = M->n2c_cell[j];
        int k = M->n2c_k[j];
        for (int i = 0; i < dd; ++i) Mp[i] += pkM[(c * nv + k) * dd + i];
        for (int i = 0; i < d; ++i) bp[i] += pkR[(c * nv + k) * d + i];
    }
    /* faces around p with a prescribed traction, pressure or normal velocity (reading R15) */
    real dp[3] = {0, 0, 0}, gp = 0.0;
    int nvel = 0;
    for (long j = M->nbf_off[p]; j < M->nbf_off[p + 1]; ++j) {
        long b = M->nbf_idx[j];
        int tag = M->bf_tag[b];
        if (tag < 3) continue;
        real N[3] = {0, 0, 0};
        face_area_vector(M, x, b, N);
        const real *val = M->bf_val + b * d;
        if (tag == 3) {
            real area = 0.0;
            for (int a = 0; a < d; ++a) area += N[a] * N[a];
            area = sqrt(area);
            for (int a = 0; a < d; ++a) bp[a] += area / d * val[a];
        } else if (tag == 4) {
            for (int a = 0; a < d; ++a) bp[a] -= val[0] * N[a] / d;
        } else if (tag == 5) {
            for (int a = 0; a < d; ++a) {
                dp[a] += N[a] / d;
                gp += val[a] * N[a] / d;
            }
            nvel++;
        }
    }
    solve_K(M, Mp, p, bp, vs);
    if (nvel > 0) {
        real w[3];
        solve_K(M, Mp, p, dp, w);
        real wd = 0.0, vd = 0.0;
        for (int a = 0; a < d; ++a) {
            wd += w[a] * dp[a];
            vd += vs[a] * dp[a];
        }
        if (wd > 0.0) {
            real T = (vd - gp) / wd;
            for (int a = 0; a < d; ++a) vs[a] -= T * w[a];
        }
    }
    /* contact walls (reading R17): a node of a contact face closer than eps to a wall and
     * moving into it gets v . n = 0 for the step, through the same multiplier as above */
    int contact = 0;
    for (long j = M->nbf_off[p]; j < M->nbf_off[p + 1]; ++j) contact |= M->bf_tag[M->nbf_idx[j]] == 6;
    if (contact) {
        for (int k = 0; k < M->n_contact; ++k) {
            const real *P = M->contact[k], *n = M->contact[k] + d;
            real dist = 0.0, vn = 0.0;
            for (int a = 0; a < d; ++a) {
                dist += n[a] * (x[p * d + a] - P[a]);
                vn += n[a] * vs[a];
            }
            if (!(dist < M->contact_eps && vn < 0.0)) continue;
            real w[3], wn = 0.0;
            solve_K(M, Mp, p, n, w);
            for (int a = 0; a < d; ++a) wn += w[a] * n[a];
            if (wn > 0.0) {
                real T = vn / wn;
                for (int a = 0; a < d; ++a) vs[a] -= T * w[a];
            }
        }
    }
}

static void phase_nodes(const OrcState *S, real dt, Work *w) {
    const OrcMesh *M = S->M;
    int d = M->d;
#pragma omp parallel for schedule(static)
    for (long p = 0; p < M->np; ++p) {
        node_solve_one(M, S->x, w->pkM, w->pkR, p, w->vs + p * d);
        for (int a = 0; a < d; ++a) {
            w->x1[p * d + a] = S->x[p * d + a] + dt * w->vs[p * d + a];
            w->vp1[p * d + a] = 2.0 * w->vs[p * d + a] - S->vp[p * d + a];
        }
    }
}

/* velocity gradient of a cell from node velocities (Eq. div_grad_v, reading R2) */
static void vel_gradient(int d, int nv, const real *ln, real V, const real *vnodes, real *L) {
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            real s = 0.0;
            for (int k = 0; k < nv; ++k) s += vnodes[k * d + i] * ln[k * d + j];
            L[i * d + j] = s / V;
        }
}

/* 5. subcell forces and cell update (Eqs. subforce^n, tau_c^n, v_c^n, e_c^n, firstB, CN_B;
 *    readings R1, R7) */
static void phase_update(const OrcState *S, const int *order, real dt, Work *w) {
    const OrcMesh *M = S->M;
    int d = M->d, nv = M->nv, dd = d * d;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < M->nc; ++c) {
        real sf[3] = {0, 0, 0}, sfv = 0.0;
        real vsn[MAXV * MAXD], vpn[MAXV * MAXD], vp1n[MAXV * MAXD];
        for (int k = 0; k < nv; ++k) {
            int p = M->c2n[c * nv + k];
            const real *Mk = w->pkM + (c * nv + k) * dd, *Rk = w->pkR + (c * nv + k) * d;
            real f[3];
            matvec_n(d, Mk, w->vs + p * d, f);
            for (int i = 0; i < d; ++i) f[i] -= Rk[i];
            for (int i = 0; i < d; ++i) {
                sf[i] += f[i];
                sfv += f[i] * w->vs[p * d + i];
            }
            for (int a = 0; a < d; ++a) {
                vsn[k * d + a] = w->vs[p * d + a];
                vpn[k * d + a] = S->vp[p * d + a];
                vp1n[k * d + a] = w->vp1[p * d + a];
            }
        }
        real m = S->m[c];
        for (int i = 0; i < d; ++i) w->v1[c * d + i] = S->v[c * d + i] + dt / m * sf[i];
        w->e1[c] = S->e[c] + dt / m * sfv;
        /* volume at x^{n+1} */
        real xs[MAXV * MAXD], V1, xc1[MAXD], N1[MAXV * MAXD], ln1[MAXV * MAXD], Lc1;
        gather_xs(M, w->x1, c, xs);
        orc_cell_geometry(d, xs, &V1, xc1, N1, ln1, &Lc1);
        w->V1[c] = V1;
        const real *Fn = S->F + c * dd;
        real *F1 = w->F1 + c * dd;
        if (order[c] != 1) {
            /* Crank-Nicolson: (I - dt/2 L^{n+1}) F^{n+1} = (I + dt/2 L^n) F^n */
            real L0[9], L1[9], A[9], Bm[9], Ai[9], R[9];
            vel_gradient(d, nv, w->ln + c * nv * d, w->V[c], vpn, L0);
            vel_gradient(d, nv, ln1, V1, vp1n, L1);
            for (int i = 0; i < d; ++i)
                for (int j = 0; j < d; ++j) {
                    real id = i == j ? 1.0 : 0.0;
                    A[i * d + j] = id - 0.5 * dt * L1[i * d + j];
                    Bm[i * d + j] = id + 0.5 * dt * L0[i * d + j];
                }
            matmul_n(d, Bm, Fn, R);
            inv_n(d, A, Ai);
            matmul_n(d, Ai, R, F1);
        } else {
            /* first order: F^{n+1} = F^n + dt L* F^n, L* from v*_p on the x^n geometry */
            real Ls[9], LF[9];
            vel_gradient(d, nv, w->ln + c * nv * d, w->V[c], vsn, Ls);
            matmul_n(d, Ls, Fn, LF);
            for (int i = 0; i < dd; ++i) F1[i] = Fn[i] + dt * LF[i];
        }
    }
}

/* 6. detection (Eqs. PAD and RDMP; reading R12).
 * pad_state: 0 admissible; 1 only eps < -tol; 2 not computable (non-finite, tau <= 0, det F <= 0) */
static int pad_state(int d, const real *v, real e, const real *F, real V, real a0sq) {
    int dd = d * d;
    if (!isfinite(e) || !isfinite(V)) return 2;
    for (int i = 0; i < d; ++i)
        if (!isfinite(v[i])) return 2;
    for (int i = 0; i < dd; ++i)
        if (!isfinite(F[i])) return 2;
    if (!(V > 0.0)) return 2;
    if (!(det_n(d, F) > 0.0)) return 2;
    real ke = 0.0;
    for (int i = 0; i < d; ++i) ke += 0.5 * v[i] * v[i];
    real eps = e - ke;
    real tol = 1e-10 * fmax(fmax(fabs(e), ke), a0sq);
    return eps >= -tol ? 0 : 1;
}

/* Eq. RDMP: the range [lo, hi] of the density at t^n over the stencil V_c and the cell c
 * itself (reading R12), from the volumes Vn at x^n */
static void rdmp_range(const OrcState *S, const real *Vn, long c, real *lo, real *hi) {
    const OrcMesh *M = S->M;
    *lo = S->m[c] / Vn[c];
    *hi = *lo;
    for (long j = M->st_off[c]; j < M->st_off[c + 1]; ++j) {
        long o = M->st_idx[j];
        real r = S->m[o] / Vn[o];
        *lo = fmin(*lo, r);
        *hi = fmax(*hi, r);
    }
}

/* Eq. RDMP: a candidate density is admissible when it lies in [lo - delta, hi + delta],
 * delta = max(delta0, delta1 (hi - lo)) with delta0 absolute (reading R12) */
static int rdmp_admits(const OrcState *S, real rho_new, real lo, real hi) {
    real delta = fmax(S->prm.delta0, S->prm.delta1 * (hi - lo));
    return rho_new >= lo - delta && rho_new <= hi + delta;
}

static int rdmp_ok(const OrcState *S, const Work *w, long c) {
    real lo, hi;
    rdmp_range(S, w->V, c, &lo, &hi);
    return rdmp_admits(S, S->m[c] / w->V1[c], lo, hi);
}

static void candidate(const OrcState *S, const int *order, real dt, Work *w) {
    phase_geometry(S, S->x, w);
    phase_slopes(S, order, w);
    phase_packets(S, order, dt, w);
    phase_nodes(S, dt, w);
    phase_update(S, order, dt, w);
}

/* 7. time step (Eqs. CFL, CFL2; reading R13) */
static real dt_acoustic_cell(const OrcState *S, long c, const real *F, real V, real Lc, real eps) {
    real rho = S->m[c] / V;
    return S->prm.cfl * Lc / sound_speed_state(S, c, F, rho, eps);
}

static real eps_of(int d, const real *v, real e) {
    real ke = 0.0;
    for (int i = 0; i < d; ++i) ke += 0.5 * v[i] * v[i];
    return e - ke;
}

static void totals(const OrcState *S, OrcInfo *info) {
    int d = S->M->d;
    info->mass = 0; info->energy = 0;
    info->mom[0] = info->mom[1] = info->mom[2] = 0;
    for (long c = 0; c < S->M->nc; ++c) {
        info->mass += S->m[c];
        info->energy += S->m[c] * S->e[c];
        for (int i = 0; i < d; ++i) info->mom[i] += S->m[c] * S->v[c * d + i];
    }
}

int orc_step(OrcState *S, OrcInfo *info) {
    const OrcMesh *M = S->M;
    int d = M->d, dd = d * d, nv = M->nv;
    long nc = M->nc;
    real dt = S->dt;
    Work w = work_new(M);
    int *order = S->order;
    for (long c = 0; c < nc; ++c) order[c] = S->prm.order == 1 ? 1 : 2;
    int iters = 0, n_troubled = 0, n_para = 0, n_eps = 0, status = ORC_OK;
    for (;;) {
        candidate(S, order, dt, &w);
        int fresh = 0;
        n_para = 0;
        n_eps = 0;
        if (S->prm.mood) {
            /* new troubled cells are decided on this candidate before any mask change */
            int *flag = ORC_ZNEW(int, nc);
#pragma omp parallel for schedule(static) reduction(+ : fresh, n_para, n_eps)
            for (long c = 0; c < nc; ++c) {
                int ps = pad_state(d, w.v1 + c * d, w.e1[c], w.F1 + c * dd, w.V1[c], a0sq_of(S, c));
                /* stiffened gas: p + p_inf > 0 (real sound speed; reading R18) */
                if (ps == 0 && S->prm.eos != 0 &&
                    !(sg_pressure(S, c, w.F1 + c * dd, eps_of(d, w.v1 + c * d, w.e1[c])) + S->prm.p_inf > 0.0))
                    ps = 1;
                if (order[c] != 1) {
                    if (ps != 0 || !rdmp_ok(S, &w, c)) { flag[c] = 1; fresh++; }
                } else if (ps == 2) {
                    n_para++;
                } else if (ps == 1) {
                    n_eps++;
                }
            }
            for (long c = 0; c < nc; ++c)
                if (flag[c]) order[c] = (order[c] == 2 && S->prm.cascade == 3) ? 3 : 1;
            free(flag);
        }
        if (fresh == 0) break;
        n_troubled += fresh;
        if (++iters > S->prm.max_mood_iters) { status = ORC_ERR_MOOD_ITERS; break; }
    }
    if (status == ORC_OK && n_para > 0) status = ORC_ERR_PARACHUTE;
    if (status == ORC_OK) {
        /* accept the candidate */
        real dtn = S->prm.dt_fixed > 0 ? S->prm.dt_fixed : (1.0 + S->prm.Ci) * dt;
        if (!(S->prm.dt_fixed > 0)) {
            for (long c = 0; c < nc; ++c) {
                real xs[MAXV * MAXD], V1, xc1[MAXD], N1[MAXV * MAXD], ln1[MAXV * MAXD], Lc1;
                gather_xs(M, w.x1, c, xs);
                orc_cell_geometry(d, xs, &V1, xc1, N1, ln1, &Lc1);
                real dtc = dt_acoustic_cell(S, c, w.F1 + c * dd, V1, Lc1, eps_of(d, w.v1 + c * d, w.e1[c]));
                real dV = V1 - w.V[c];
                if (dV != 0.0) dtc = fmin(dtc, S->prm.Cv * dt * w.V[c] / fabs(dV));
                dtn = fmin(dtn, dtc);
            }
        }
        memcpy(S->x, w.x1, sizeof(real) * M->np * d);
        memcpy(S->vp, w.vp1, sizeof(real) * M->np * d);
        memcpy(S->v, w.v1, sizeof(real) * nc * d);
        memcpy(S->e, w.e1, sizeof(real) * nc);
        memcpy(S->F, w.F1, sizeof(real) * nc * dd);
        for (long c = 0; c < nc; ++c) S->tau[c] = w.V1[c] / S->m[c];
        memcpy(S->pkM, w.pkM, sizeof(real) * nc * nv * dd);
        memcpy(S->pkR, w.pkR, sizeof(real) * nc * nv * d);
        memcpy(S->vstar, w.vs, sizeof(real) * M->np * d);
        S->t += dt;
        S->step += 1;
        S->last.dt_used = dt;
        S->dt = dtn;
    }
    int np0 = 0, nlim = 0;
    for (long c = 0; c < nc; ++c) {
        np0 += order[c] == 1;
        nlim += order[c] == 3;
    }
    S->last.n_lim = nlim;
    S->last.t = S->t;
    S->last.dt_next = S->dt;
    S->last.step = S->step;
    S->last.n_troubled = n_troubled;
    S->last.n_p0 = np0;
    S->last.mood_iters = iters;
    S->last.n_parachute = n_para;
    S->last.n_p0_eps = n_eps;
    totals(S, &S->last);
    if (info) *info = S->last;
    work_free(&w);
    return status;
}

/* --------------------------------------------------------------------------------------
 * State initialisation (Sect. "2D and 3D test problems"): m_c = rho0 |w_c(x^0)|,
 * e = |v|^2/2 + Psi(F), v_p^0 = first-order nodal solution, dt^0 = acoustic bound.
 * ------------------------------------------------------------------------------------ */
void orc_state_free(OrcState *S) {
    if (!S) return;
    free(S->mu); free(S->m); free(S->x); free(S->vp); free(S->v); free(S->e); free(S->F);
    free(S->tau); free(S->order); free(S->pkM); free(S->pkR); free(S->vstar);
    free(S);
}

int orc_state_new(OrcMesh *M, real rho0, real lam, const real *mu_cell, const real *v_soa,
                  const real *F_soa, const OrcParams *prm, OrcState **out) {
    if (!M || !prm || !mu_cell || !v_soa || !out) return ORC_ERR_ARG;
    if (prm->eos != 0 && !(prm->eos == 1 && prm->gamma > 1.0 && prm->p0 + prm->p_inf > 0.0)) return ORC_ERR_ARG;
    int d = M->d, nv = M->nv, dd = d * d;
    long nc = M->nc, np = M->np;
    OrcState *S = ORC_ZNEW(OrcState, 1);
    S->M = M; S->prm = *prm; S->rho0 = rho0; S->lam = lam;
    S->mu = ORC_NEW(real, nc);
    S->m = ORC_NEW(real, nc);
    S->x = ORC_NEW(real, np * d);
    S->vp = ORC_ZNEW(real, np * d);
    S->v = ORC_NEW(real, nc * d);
    S->e = ORC_NEW(real, nc);
    S->F = ORC_NEW(real, nc * dd);
    S->tau = ORC_NEW(real, nc);
    S->order = ORC_NEW(int, nc);
    S->pkM = ORC_ZNEW(real, nc * nv * dd);
    S->pkR = ORC_ZNEW(real, nc * nv * d);
    S->vstar = ORC_ZNEW(real, np * d);
    memcpy(S->x, M->x0, sizeof(real) * np * d);
    for (long c = 0; c < nc; ++c) {
        S->mu[c] = mu_cell[c];
        for (int i = 0; i < d; ++i) S->v[c * d + i] = v_soa[i * nc + c];
        for (int i = 0; i < dd; ++i) S->F[c * dd + i] = F_soa ? F_soa[i * nc + c] : ((i % (d + 1)) == 0 ? 1.0 : 0.0);
        S->order[c] = 1;
    }
    Work w = work_new(M);
    phase_geometry(S, S->x, &w);
    real dt0 = INFINITY;
    for (long c = 0; c < nc; ++c) {
        S->m[c] = rho0 * w.V[c];
        S->tau[c] = w.V[c] / S->m[c];
        real ke = 0.0;
        for (int i = 0; i < d; ++i) ke += 0.5 * S->v[c * d + i] * S->v[c * d + i];
        if (S->prm.eos == 0) {
            S->e[c] = ke + orc_free_energy_a(d, S->F + c * dd, rho0, S->mu[c], kappa_of(S, c), S->prm.shear_a);
        } else {  /* eps_v from the initial pressure p0 at rho = rho0 / det F (reading R18) */
            real F3[9];
            embed3(d, S->F + c * dd, F3);
            real J = det_n(3, F3);
            real eps_v = (S->prm.p0 + S->prm.gamma * S->prm.p_inf) / ((S->prm.gamma - 1.0) * rho0 / J);
            S->e[c] = ke + eps_v + orc_free_energy_a(d, S->F + c * dd, rho0, S->mu[c], 0.0, S->prm.shear_a);
        }
        dt0 = fmin(dt0, dt_acoustic_cell(S, c, S->F + c * dd, w.V[c], w.Lc[c], eps_of(d, S->v + c * d, S->e[c])));
    }
    /* v_p^0: first-order nodal solve at t^0 */
    phase_packets(S, S->order, 0.0, &w);
    for (long p = 0; p < np; ++p) node_solve_one(M, S->x, w.pkM, w.pkR, p, S->vp + p * d);
    work_free(&w);
    S->dt = prm->dt_fixed > 0 ? prm->dt_fixed : dt0;
    S->t = 0.0;
    S->step = 0;
    *out = S;
    return ORC_OK;
}

/* field ids for orc_get (SoA [ncomp][n] output) */
enum { F_X = 0, F_VP = 1, F_VSTAR = 2, F_V = 3, F_E = 4, F_F = 5, F_TAU = 6, F_ORDER = 7,
       F_MASS = 8, F_PKM = 9, F_PKR = 10 };

int orc_get(const OrcState *S, int field, real *dst) {
    const OrcMesh *M = S->M;
    int d = M->d, dd = d * d, nv = M->nv;
    long nc = M->nc, np = M->np;
    switch (field) {
    case F_X: for (long p = 0; p < np; ++p) for (int a = 0; a < d; ++a) dst[a * np + p] = S->x[p * d + a]; break;
    case F_VP: for (long p = 0; p < np; ++p) for (int a = 0; a < d; ++a) dst[a * np + p] = S->vp[p * d + a]; break;
    case F_VSTAR: for (long p = 0; p < np; ++p) for (int a = 0; a < d; ++a) dst[a * np + p] = S->vstar[p * d + a]; break;
    case F_V: for (long c = 0; c < nc; ++c) for (int a = 0; a < d; ++a) dst[a * nc + c] = S->v[c * d + a]; break;
    case F_E: for (long c = 0; c < nc; ++c) dst[c] = S->e[c]; break;
    case F_F: for (long c = 0; c < nc; ++c) for (int a = 0; a < dd; ++a) dst[a * nc + c] = S->F[c * dd + a]; break;
    case F_TAU: for (long c = 0; c < nc; ++c) dst[c] = S->tau[c]; break;
    case F_ORDER: for (long c = 0; c < nc; ++c) dst[c] = S->order[c]; break;
    case F_MASS: for (long c = 0; c < nc; ++c) dst[c] = S->m[c]; break;
    /* packets: [comp][k][c] with M as full d x d row-major comps and rhs d comps */
    case F_PKM:
        for (long c = 0; c < nc; ++c)
            for (int k = 0; k < nv; ++k)
                for (int a = 0; a < dd; ++a) dst[(a * nv + k) * nc + c] = S->pkM[(c * nv + k) * dd + a];
        break;
    case F_PKR:
        for (long c = 0; c < nc; ++c)
            for (int k = 0; k < nv; ++k)
                for (int a = 0; a < d; ++a) dst[(a * nv + k) * nc + c] = S->pkR[(c * nv + k) * d + a];
        break;
    default: return ORC_ERR_ARG;
    }
    return ORC_OK;
}

real orc_get_dt(const OrcState *S) { return S->dt; }
real orc_get_t(const OrcState *S) { return S->t; }

/* Set the dynamic state (used to replay a state on both sides): SoA arrays, NULL = keep. */
int orc_set_state(OrcState *S, const real *x, const real *vp, const real *v, const real *e,
                  const real *F, real dt) {
    const OrcMesh *M = S->M;
    int d = M->d, dd = d * d;
    long nc = M->nc, np = M->np;
    if (x) for (long p = 0; p < np; ++p) for (int a = 0; a < d; ++a) S->x[p * d + a] = x[a * np + p];
    if (vp) for (long p = 0; p < np; ++p) for (int a = 0; a < d; ++a) S->vp[p * d + a] = vp[a * np + p];
    if (v) for (long c = 0; c < nc; ++c) for (int a = 0; a < d; ++a) S->v[c * d + a] = v[a * nc + c];
    if (e) for (long c = 0; c < nc; ++c) S->e[c] = e[c];
    if (F) for (long c = 0; c < nc; ++c) for (int a = 0; a < dd; ++a) S->F[c * dd + a] = F[a * nc + c];
    if (dt > 0) S->dt = dt;
    return ORC_OK;
}

/* The predictor of every cell at the given level (1 first order, 2 unlimited, 3
 * Barth-Jespersen) from the current state with the time step dt: v*_cp out_v [nc][nv][d] and
 * F*_cp out_F [nc][nv][d*d] (the values the corner packets are built from). Used by tests. */
int orc_debug_predictor(const OrcState *S, int level, real dt, real *out_v, real *out_F) {
    const OrcMesh *M = S->M;
    if (level < 1 || level > 3) return ORC_ERR_ARG;
    int d = M->d, nv = M->nv, dd = d * d;
    Work w = work_new(M);
    int *order = ORC_NEW(int, M->nc);
    for (long i = 0; i < M->nc; ++i) order[i] = level;
    phase_geometry(S, S->x, &w);
    phase_slopes(S, order, &w);
#pragma omp parallel for schedule(static)
    for (long c = 0; c < M->nc; ++c) {
        real eps = S->e[c];
        for (int i = 0; i < d; ++i) eps -= 0.5 * S->v[c * d + i] * S->v[c * d + i];
        real vstar[MAXV][MAXD], Fstar[MAXV][9], Tstar[MAXV][9];
        predict_cell(S, &w, c, level, dt, eps, vstar, Fstar, Tstar);
        for (int k = 0; k < nv; ++k) {
            for (int i = 0; i < d; ++i) out_v[(c * nv + k) * d + i] = vstar[k][i];
            for (int i = 0; i < dd; ++i) out_F[(c * nv + k) * dd + i] = Fstar[k][i];
        }
    }
    free(order);
    work_free(&w);
    return ORC_OK;
}

/* Reconstructed values of v and F at the nodes of cell c from the current state with the
 * given level (2 unlimited, 3 Barth-Jespersen), and each field's range over the stencil and
 * the cell: out [nv][nq], lo [nq], hi [nq]. Used by tests. */
int orc_debug_corner_values(const OrcState *S, long c, int level, real *out, real *lo, real *hi) {
    const OrcMesh *M = S->M;
    int d = M->d, nq = d + d * d, nv = M->nv;
    Work w = work_new(M);
    int *order = ORC_NEW(int, M->nc);
    for (long i = 0; i < M->nc; ++i) order[i] = 1;
    order[c] = level;
    phase_geometry(S, S->x, &w);
    phase_slopes(S, order, &w);
    for (int q = 0; q < nq; ++q) {
        real qc = q < d ? S->v[c * d + q] : S->F[c * d * d + q - d];
        lo[q] = hi[q] = qc;
        for (long j = M->st_off[c]; j < M->st_off[c + 1]; ++j) {
            long o = M->st_idx[j];
            real qo = q < d ? S->v[o * d + q] : S->F[o * d * d + q - d];
            lo[q] = fmin(lo[q], qo);
            hi[q] = fmax(hi[q], qo);
        }
        const real *g = q < d ? w.gv + c * d * d + q * d : w.gF + c * d * d * d + (q - d) * d;
        for (int k = 0; k < nv; ++k) {
            int p = M->c2n[c * nv + k];
            real val = qc;
            for (int a = 0; a < d; ++a) val += g[a] * (S->x[p * d + a] - w.xc[c * d + a]);
            out[k * nq + q] = val;
        }
    }
    free(order);
    work_free(&w);
    return ORC_OK;
}

/* The detection of Eqs. PAD and RDMP as the step applies it, for the tests that pin its
 * thresholds: orc_debug_rdmp gives the density range of cell c at the state's current
 * positions (lo, hi, may be NULL) and whether a candidate density rho_new passes the RDMP;
 * orc_debug_pad classifies a candidate (v [d], e, F [d*d] row-major, volume V) of cell c
 * with the cell's material: 0 admissible, 1 only eps below the tolerance, 2 not computable. */
int orc_debug_rdmp(const OrcState *S, long c, real rho_new, real *lo, real *hi) {
    const OrcMesh *M = S->M;
    if (c < 0 || c >= M->nc) return -1;
    Work w = work_new(M);
    phase_geometry(S, S->x, &w);
    real l, h;
    rdmp_range(S, w.V, c, &l, &h);
    int ok = rdmp_admits(S, rho_new, l, h);
    if (lo) *lo = l;
    if (hi) *hi = h;
    work_free(&w);
    return ok;
}

int orc_debug_pad(const OrcState *S, long c, const real *v, real e, const real *F, real V) {
    if (c < 0 || c >= S->M->nc) return -1;
    return pad_state(S->M->d, v, e, F, V, a0sq_of(S, c));
}

/* threads the oracle's OpenMP loops run on */
int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Mesh queries used by tests (stencil and BC resolution). */
long orc_mesh_stencil(const OrcMesh *M, long c, long *dst, long cap) {
    long n = M->st_off[c + 1] - M->st_off[c];
    for (long j = 0; j < n && j < cap; ++j) dst[j] = M->st_idx[M->st_off[c] + j];
    return n;
}
int orc_mesh_bc_ndof(const OrcMesh *M, long p) { return M->bc_ndof[p]; }

/* values of the boundary faces, [d][nb] (traction vectors; pressures in the first row;
 * prescribed velocities), applied from the next nodal solve on */
int orc_mesh_set_bc_values(OrcMesh *M, const real *val_soa) {
    if (!M || !val_soa) return ORC_ERR_ARG;
    for (long b = 0; b < M->nb; ++b)
        for (int a = 0; a < M->d; ++a) M->bf_val[b * M->d + a] = val_soa[a * M->nb + b];
    return ORC_OK;
}

/* contact walls for the faces tagged 6: n (<= 4) planes [n][2d] (a point, then the unit
 * normal pointing from the wall into the body) and the distance threshold eps */
int orc_mesh_set_contact(OrcMesh *M, int n, const real *planes, real eps) {
    if (!M || n < 0 || n > 4 || (n > 0 && !planes) || !(eps >= 0.0)) return ORC_ERR_ARG;
    int d = M->d;
    M->n_contact = n;
    M->contact_eps = eps;
    for (int k = 0; k < n; ++k)
        for (int i = 0; i < 2 * d; ++i) M->contact[k][i] = planes[k * 2 * d + i];
    return ORC_OK;
}

/* new tags of the boundary faces [nb] (a boundary condition that changes type during the
 * run, Sect. "Boundary condition treatments"); the per-node conditions are re-derived */
int orc_mesh_set_btag(OrcMesh *M, const int *btag) {
    if (!M || !btag) return ORC_ERR_ARG;
    for (long b = 0; b < M->nb; ++b)
        if (btag[b] < 0 || btag[b] > 6) return ORC_ERR_ARG;
    for (long b = 0; b < M->nb; ++b) M->bf_tag[b] = btag[b];
    resolve_bcs(M);
    return ORC_OK;
}
