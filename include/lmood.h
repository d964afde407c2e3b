/*
 * lmood.h -- C ABI of the GB300 (sm_103a) library that advances the cell-centered
 * Lagrangian ADER-MOOD scheme for neo-Hookean hyper-elasticity of Boscheri, Loubere and
 * Maire (arXiv 2104.02139) on unstructured triangle (dim 2) or tetrahedral (dim 3) meshes,
 * in FP64.
 *
 * Conventions shared by every entry point
 *  - Arrays are structure-of-arrays: a field with k components over n entities is k
 *    contiguous runs of n values ("[k][n]").
 *  - Host input pointers are borrowed for the duration of the call only; the library copies
 *    what it needs. It owns every device buffer it allocates and frees them in the matching
 *    destroy call.
 *  - Nothing is thrown across the ABI. Every call returns an lmood_status; on failure
 *    lmood_last_error() returns a message (thread-local, valid until the next call on that
 *    thread). A failed lmood_step leaves the state as it was before the call.
 *  - All device work of a mesh and its states is ordered on the CUDA stream given to
 *    lmood_mesh_create (NULL = legacy default stream). Calls that return data to the host
 *    synchronise that stream.
 *  - Cells must be positively oriented simplices (counter-clockwise triangles, tetrahedra
 *    with (x1-x0).((x2-x0)x(x3-x0)) > 0); the library renumbers nothing.
 */
#ifndef LMOOD_H
#define LMOOD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lmood_mesh_s *lmood_mesh;
typedef struct lmood_state_s *lmood_state;

typedef enum {
    LMOOD_OK = 0,
    LMOOD_ERR_ARG = 1,        /* NULL pointer, bad dimension, bad size or field id          */
    LMOOD_ERR_MESH = 2,       /* node index out of range, non-positive simplex volume       */
    LMOOD_ERR_CUDA = 3,       /* a CUDA runtime call failed (message names it)               */
    LMOOD_ERR_OOM = 4,        /* device allocation failed                                    */
    LMOOD_ERR_PARACHUTE = 5,  /* a first-order (P0) candidate is not computable: non-finite,
                                 tau <= 0 or det F <= 0 (Sect. "Limiting: a posteriori MOOD
                                 loop", the parachute scheme); the state is left unchanged   */
    LMOOD_ERR_MOOD_ITERS = 6, /* troubled cells remain after max_mood_iters iterations      */
    LMOOD_ERR_TIMEOUT = 7,    /* a bounded device-side wait gave up (graph = 2); state unchanged */
    LMOOD_ERR_STATE = 8       /* the handle is unusable after an earlier CUDA failure        */
} lmood_status;

/* Material constants (Sect. "Examples of constitutive laws"). The shear modulus mu is given
 * per cell to lmood_state_init. Volumetric free energy
 *   Psi_v = kappa / (4 rho0) ((J - 1)^2 + (log J)^2)          (Eq. EOS_neoHook)
 * with kappa = lambda + 2 mu / 3 when vol_coeff = 0 (small-strain bulk modulus), or
 * kappa = mu when vol_coeff = 1 (the coefficient as printed). Shear free energy of the family
 *   Psi_s = mu / (4 rho0) (-2a (I1 - 3) + (1+a)/3 (I2^2 - 9))   (Eq. familiy_energies)
 * with I1, I2 the invariants of J^{-2/3} F F^t; a = -1 (neo-Hookean) is the default and the
 * fastest path; a must lie in [-1, 1/2], where the paper states the system is hyperbolic.
 * eos = 1 replaces the volumetric law by the stiffened gas (Eq. EOS_stiffened_gas, incomplete
 * form): p = (gamma - 1) rho eps_v - gamma p_inf with rho = rho0 / det F and eps_v the
 * volumetric part e - |v|^2/2 - Psi_s of the specific internal energy; the initial eps_v is
 * that of the pressure p0 (gamma > 1, p0 + p_inf > 0). lambda and vol_coeff are then unused. */
typedef struct {
    double rho0;     /* initial density (> 0)                 */
    double lambda;   /* first Lame coefficient                */
    int32_t vol_coeff;
    int32_t eos;     /* 0: Eq. EOS_neoHook (default); 1: stiffened gas */
    double shear_a;  /* a of the shear energy family (-1: neo-Hookean) */
    double gamma, p_inf, p0;  /* stiffened gas parameters and initial pressure */
} lmood_material;

/* Scheme parameters (Sect. "Time-step monitoring", "Limiting: a posteriori MOOD loop"). */
typedef struct {
    double cfl;             /* C_CFL: 0.4 in 2D, 0.25 in 3D                               */
    double Cv;              /* C_v = 0.2: volume-change bound of Eq. CFL2                  */
    double Ci;              /* C_i = 0.1: dt^{n+1} <= (1 + C_i) dt^n                       */
    double delta0;          /* 1e-4: absolute RDMP relaxation (Eq. RDMP)                   */
    double delta1;          /* 1e-3: relative RDMP relaxation                              */
    double dt_fixed;        /* > 0: use this dt for every step instead of Eq. CFL           */
    int32_t max_mood_iters; /* MOOD rounds allowed per step (default 100000; a first step from
                               F = I can cascade over a whole mesh)               */
    int32_t order;          /* 2: second order with the P1 -> P0 cascade; 1: first order    */
    int32_t mood;           /* 1: a-posteriori detection on (default); 0: unlimited         */
    int32_t graph;          /* 1: each step is one CUDA graph with the MOOD loop as a device-side
                               conditional while node (default); 0: host-driven MOOD rounds;
                               2: each step is one persistent cooperative launch whose stages
                               are separated by grid-wide barriers with bounded waits (a wait
                               that gives up returns LMOOD_ERR_TIMEOUT, state unchanged;
                               neo-Hookean material only; fastest for small meshes, where
                               launch latency dominates); 3: as 1 with the MOOD loop as one
                               cooperative kernel node with such barriers instead of the
                               conditional while node (a timeout also returns
                               LMOOD_ERR_TIMEOUT). Results are identical.                    */
    int32_t cascade;        /* 2: P1 -> P0 (default); 3: P1 -> P1 with Barth-Jespersen limited
                               slopes -> P0, the three-scheme cascade of Sect. "Limiting: a
                               posteriori MOOD loop" (order codes 2, 3, 1)                    */
    int32_t barrier_polls;  /* graph = 2: polls (~0.1 us each) one grid-barrier wait may take
                               before the launch gives up with LMOOD_ERR_TIMEOUT; <= 0: the
                               default 1e8 (~10 s, far above any stage's duration)          */
} lmood_params;

/* Per-step report. */
typedef struct {
    double t;            /* time after the step                               */
    double dt_used;      /* dt of the step (instance 0 for batches)            */
    double dt_next;      /* dt of the next step (instance 0 for batches)       */
    int64_t step;        /* steps taken so far                                */
    int32_t n_troubled;  /* cells decremented to P0 during the step            */
    int32_t n_p0;        /* cells advanced with the first-order scheme         */
    int32_t mood_iters;  /* MOOD iterations the step needed                    */
    int32_t n_parachute; /* P0 candidates that were not computable (then the status is an error) */
    int32_t n_p0_eps;    /* P0 cells accepted with a negative specific internal energy */
    int32_t n_lim;       /* cells advanced with Barth-Jespersen limited slopes (cascade 3) */
    int32_t syncs;       /* host synchronisations of the mesh stream the call made (lmood_run:
                            for all its steps; 1 when its steps were chained on the device) */
} lmood_step_info;

/* Field ids for lmood_get / lmood_set (layout, entity count n, components k). */
enum {
    LMOOD_FIELD_X = 0,     /* node positions x_p                 [dim][n_nodes]            */
    LMOOD_FIELD_VP = 1,    /* node velocities v_p^n              [dim][n_nodes]            */
    LMOOD_FIELD_VSTAR = 2, /* last step's nodal-solver velocity  [dim][n_nodes]   get only */
    LMOOD_FIELD_V = 3,     /* cell velocities v_c                [dim][n_cells]            */
    LMOOD_FIELD_E = 4,     /* specific total energy e_c          [n_cells]                 */
    LMOOD_FIELD_F = 5,     /* deformation gradient F_c, row-major [dim*dim][n_cells]       */
    LMOOD_FIELD_TAU = 6,   /* specific volume tau_c = |w_c| / m_c [n_cells]       get only */
    LMOOD_FIELD_ORDER = 7, /* last step's scheme per cell as double [n_cells] get only: 2 P1,
                              3 P1 with limited slopes, 1 first order (P0) */
    LMOOD_FIELD_MASS = 8,  /* cell masses m_c                    [n_cells]        get only */
    LMOOD_FIELD_PKM = 9,   /* last step's corner matrices M_cp, symmetric storage
                              [dim(dim+1)/2][dim+1][n_cells] (xx,xy,yy | xx,xy,xz,yy,yz,zz) get only */
    LMOOD_FIELD_PKR = 10,  /* last step's corner right-hand sides M_cp v*_cp - T*_cp l_cp n_cp
                              [dim][dim+1][n_cells]                                get only */
    LMOOD_FIELD_DT = 11    /* dt of the next step per instance   [n_instances]             */
};

/* Fill *p with the paper's defaults for dim (2: cfl 0.4, 3: cfl 0.25). */
lmood_status lmood_params_default(int dim, lmood_params *p);

/*
 * Build a mesh on the device (Sect. "Mesh and notation").
 *   dim            2 or 3
 *   x              host, [dim][n_nodes] initial node positions
 *   c2n            host, [dim+1][n_cells] node ids of each simplex (positively oriented)
 *   bface, btag    host, [dim][n_bfaces] node ids and [n_bfaces] tags of boundary faces that
 *                  carry a condition (Appendix B): 0 free traction, 1 slip wall (symmetry
 *                  plane through the face), 2 clamped (symmetry point, v = 0), 3 prescribed
 *                  traction vector t_f, 4 prescribed pressure p_f, 5 prescribed velocity V_f
 *                  (its normal component is imposed; Eqs. pBC, vBC1, vBC), 6 contact (free,
 *                  until it meets a contact wall, see lmood_mesh_set_contact). The values of
 *                  tags 3-5 are set with lmood_mesh_set_bc_values (zero until then). Faces not
 *                  listed are traction-free. Each face must be a face of one cell; the library
 *                  orders its nodes so that its area vector N_f points out of the mesh. Per
 *                  node: clamped > prescribed velocity > slip > free for the velocity (several
 *                  distinct slip planes leave their intersection; a prescribed velocity
 *                  imposes v_p . d_p = g_p with d_p = sum N_f / dim, g_p = sum V_f . N_f / dim
 *                  over the node's velocity faces, on top of the slip / free solve); traction
 *                  faces add |N_f| t_f / dim and pressure faces -p_f N_f / dim to the node's
 *                  force balance, with N_f at the current positions. May be NULL when
 *                  n_bfaces = 0.
 *   cell_inst      host, [n_cells] instance id of each cell for a batch of independent meshes
 *                  concatenated into one (cells of different instances share no node), or
 *                  NULL for a single instance. Each instance keeps its own dt.
 *   n_inst         number of instances (1 when cell_inst is NULL)
 *   stream         cudaStream_t on which every device operation of this mesh is ordered
 * Builds the node-to-corner adjacency and the per-node boundary conditions. Errors:
 * LMOOD_ERR_ARG (also for a mesh beyond the kernels' 32-bit indexing: at most 238,609,294
 * cells and 89,478,485 nodes in 2D, 89,478,485 cells and 37,025,580 nodes in 3D, checked
 * before anything is read), LMOOD_ERR_MESH (index out of range, |w_c| <= 0, a boundary face
 * that is not the face of exactly one cell, a face listed twice (in any node order),
 * instances of a batch sharing a node; all checked
 * on the host before any device call), LMOOD_ERR_OOM (device memory), LMOOD_ERR_CUDA (any
 * other CUDA failure, e.g. no usable device).
 */
lmood_status lmood_mesh_create(int dim, int64_t n_nodes, const double *x, int64_t n_cells,
                               const int32_t *c2n, int64_t n_bfaces, const int32_t *bface,
                               const int32_t *btag, const int32_t *cell_inst, int32_t n_inst,
                               void *stream, lmood_mesh *out);
lmood_status lmood_mesh_destroy(lmood_mesh m);

/* Values of the boundary faces, [dim][n_bfaces] in the order given to lmood_mesh_create:
 * traction vectors (tag 3), pressures in row 0 (tag 4), prescribed velocities (tag 5); other
 * faces' values are ignored. Host (is_device = 0, the call synchronises) or device pointer.
 * They act from the next nodal solve on (set them before lmood_state_init for the initial
 * one); all states on the mesh see them. */
lmood_status lmood_mesh_set_bc_values(lmood_mesh m, const double *values, int is_device);

/* Contact walls for the faces tagged 6 (Sect. "Boundary condition treatments": a condition
 * that changes type with a distance function): n_planes (0-4) planes, [n_planes][2 dim] on
 * the host (a point, then the unit normal pointing from the wall into the body), and the
 * distance threshold eps. In a nodal solve, a node of a contact face whose distance to a wall
 * at x^n is below eps and whose velocity (after its other conditions) points into the wall
 * gets v . n = 0 for that step (the wall does no work); it is free again once its velocity
 * points away. Synchronises. Errors: LMOOD_ERR_ARG (count, eps < 0, non-unit normal). */
lmood_status lmood_mesh_set_contact(lmood_mesh m, int n_planes, const double *planes, double eps);

/* New tags [n_bfaces] (host) for the mesh's boundary faces, e.g. a wall that becomes free at
 * a given time (Sect. "Boundary condition treatments"); the per-node conditions are re-derived
 * and take effect from the next nodal solve. Synchronises. Errors: LMOOD_ERR_ARG for a tag
 * outside 0-6. */
lmood_status lmood_mesh_set_btag(lmood_mesh m, const int32_t *btag);

/*
 * Create a state at t = 0 on mesh m (initialisation of Sect. "2D and 3D test problems"):
 * m_c = rho0 |w_c(x^0)|, v_c = v_cell, F_c = F_cell (NULL: identity), e_c = |v_c|^2 / 2 +
 * Psi(F_c), node velocities v_p^0 = first-order nodal solution, dt^0 = acoustic bound of
 * Eq. CFL2 (or prm->dt_fixed).
 *   mu_cell  host, [n_cells] shear modulus per cell (> 0)
 *   v_cell   host, [dim][n_cells]
 *   F_cell   host, [dim*dim][n_cells] row-major, or NULL
 * The state keeps a reference to m: destroy the state before the mesh.
 */
lmood_status lmood_state_init(lmood_mesh m, const lmood_material *mat, const double *mu_cell,
                              const double *v_cell, const double *F_cell, const lmood_params *prm,
                              lmood_state *out);
/* The same with mu_cell, v_cell and F_cell (NULL: identity) in device memory, read in order on
 * the mesh's stream (the caller makes them ready there); mu > 0 is checked on the device
 * (LMOOD_ERR_ARG). Nothing of the inputs goes through host memory. */
lmood_status lmood_state_init_device(lmood_mesh m, const lmood_material *mat, const double *mu_cell,
                                     const double *v_cell, const double *F_cell, const lmood_params *prm,
                                     lmood_state *out);
lmood_status lmood_state_destroy(lmood_state s);

/*
 * Advance one full explicit step t^n -> t^{n+1} (Sects. "Space-Time discretization ---
 * ADER methodology", "Limiting: a posteriori MOOD loop", "Time-step monitoring"): corner
 * geometry, least-squares reconstruction of v and F, ADER predictor and corner matrices,
 * Eucclhyd nodal solver with boundary conditions, subcell forces and update of tau, v, e, F,
 * node motion, MOOD detection and first-order recomputation of troubled cells, next dt.
 * info may be NULL. Synchronises the stream (the MOOD loop reads the troubled count).
 * Errors: LMOOD_ERR_PARACHUTE, LMOOD_ERR_MOOD_ITERS (state unchanged), LMOOD_ERR_CUDA.
 */
lmood_status lmood_step(lmood_state s, lmood_step_info *info);

/* nsteps steps, exactly as nsteps calls of lmood_step (bitwise the same state and reports);
 * stops at the first error, which it returns with the state after the last accepted step.
 * last (may be NULL) gets the report of the last step taken (on an error: of the failing
 * step). With params.graph = 1 and timing off, the steps are chained on the device: each
 * step's graph runs behind a device-side gate that skips it once a step of the run has
 * failed, all nsteps are launched back to back and the call synchronises once, at the end
 * (last->syncs = 1); otherwise (and where the device cannot build the chained graph) it calls
 * lmood_step nsteps times. */
lmood_status lmood_run(lmood_state s, int64_t nsteps, lmood_step_info *last);

/*
 * Copy a field out of (get) or into (set) the state. dst/src is a device pointer when
 * is_device != 0 (ordered on the mesh's stream), else a host pointer (the call
 * synchronises). Sizes and layouts are those of the field ids above; set accepts X, VP, V,
 * E, F and DT (replacing the dynamic state, e.g. to restart from a checkpoint; setting X,
 * VP or F also refreshes the derived cell geometry (with the velocity gradient of v_p that
 * the next update uses as L^n), density and impedance, and with the stiffened gas so does
 * setting V or E, on which its impedance depends).
 * Errors: LMOOD_ERR_ARG for an unknown or read-only field id.
 */
lmood_status lmood_get(lmood_state s, int field, void *dst, int is_device);
lmood_status lmood_set(lmood_state s, int field, const void *src, int is_device);

/*
 * Several fields in one call: the n copies are queued on the mesh's stream back to back and,
 * for host pointers, the call synchronises once at the end (set: the derived cell geometry
 * is refreshed once, after the last copy, when X, VP or F is among the fields, or with the
 * stiffened gas V or E). fields[i] and
 * dst[i] / src[i] as for lmood_get / lmood_set; all host or all device (is_device).
 * Errors: LMOOD_ERR_ARG for a NULL pointer, an unknown or (set) read-only field id, or ORDER
 * requested twice in one get; every argument is checked before the first copy.
 */
lmood_status lmood_get_fields(lmood_state s, int n, const int *fields, void *const *dst, int is_device);
lmood_status lmood_set_fields(lmood_state s, int n, const int *fields, const void *const *src, int is_device);

/* Sums over cells of m_c, m_c v_c and m_c e_c (out: mass, mom[dim], energy; 5 doubles). */
lmood_status lmood_totals(lmood_state s, double *out5);

/* Counts of the mesh: out[0] n_nodes, [1] n_cells, [2] dim, [3] (node, neighbour) pairs of the
 * least-squares sums, i.e. sum over nodes of deg (deg - 1),
 * [4] largest number of corners around a node, [5] instances. */
lmood_status lmood_mesh_info(lmood_mesh m, int64_t *out6);

/* Kernel timing with CUDA events on the mesh's stream, for profiling the step.
 * lmood_timing(s, 1) resets and starts the per-class accumulators, lmood_timing(s, 0) stops.
 * lmood_timing_read fills ms[LMOOD_NK] (summed device time per class) and launches[LMOOD_NK]
 * (kernel launches per class since the last reset; counted whether or not timing is on). */
/* Autotuning of the launch shapes: times the full-mesh kernels of the step with each
 * candidate block size on the state's current fields (moments and nodes: 128, 256, 512
 * threads; predictor and update: 64, 128, 256), reps launches each (<= 0: 5), with detection
 * off, and keeps the fastest for the mesh (every state on it launches with them from then on;
 * this state's captured step graphs are re-captured at its next step). The state's fields are
 * not changed (only per-step scratch and the diagnostic fields VSTAR, PKM, PKR); results of
 * later steps are bitwise the same as without tuning. ms12 (may be NULL) gets the mean
 * times [4][3] (moments, predict, nodes, update x the candidates in the order above);
 * chosen4 (may be NULL) the chosen sizes in the same kernel order. Synchronises. */
lmood_status lmood_autotune(lmood_state s, int reps, double *ms12, int32_t *chosen4);

/* Autotuning of the step's schedule beyond the block sizes (the paper has no counterpart:
 * launch shapes of this implementation; the per-cell and per-node arithmetic is the same in
 * every schedule, so later steps are bitwise the same as without tuning):
 *  - the order in which the whole-mesh node kernels (moments, nodal solve) take the nodes: the
 *    nodes of each window of W consecutive ones in order of their cell count (a warp's lanes
 *    then run loops of one length while a block still reads one neighbourhood), W = 32, 256
 *    (the order lmood_mesh_create sets), 2048, or 0 (the nodes in their own order); timed by
 *    reps launches of the two kernels (<= 0: 5) and the fastest kept for the mesh (every
 *    state on it);
 *  - the step form, when the state was created with graph 1 or 2 and its material allows the
 *    persistent form (neo-Hookean): reps lmood_step calls in each form (host synchronisation
 *    included) from the state as it is, the state copied aside on the device before and
 *    restored after each trial (fields, time, step count and report unchanged), and the state
 *    switched to the faster form.
 * ms_window4 (may be NULL): mean ms of one moments + nodal-solve pass per candidate W in the
 * order above; window (may be NULL): the chosen W; ms_form2 (may be NULL): ms per step of
 * graph 1 and graph 2 (-1 when not timed); form (may be NULL): the chosen graph, -1 when the
 * form was not tuned. Errors: LMOOD_ERR_ARG with timing on; LMOOD_ERR_OOM (the state copy);
 * a trial step's own error (the state is then that of the failed trial's start). Synchronises. */
lmood_status lmood_autotune_schedule(lmood_state s, int reps, double *ms_window4, int32_t *window,
                                     double *ms_form2, int32_t *form);

enum { LMOOD_K_PREDICT = 0, LMOOD_K_NODES = 1, LMOOD_K_UPDATE = 2, LMOOD_K_MOOD = 3, LMOOD_K_FINALIZE = 4,
       LMOOD_K_MOMENTS = 5, LMOOD_NK = 6 };
lmood_status lmood_timing(lmood_state s, int enable);
lmood_status lmood_timing_read(lmood_state s, double *ms, int64_t *launches);

/*
 * Conserved totals of caller-owned cell arrays without any device allocation (the paper has
 * no counterpart: this is a service for host applications that own all device memory and do
 * not let libraries call cudaMalloc after start-up, e.g. codes that carve the GPU into one
 * pool at initialisation or real-time loops where an allocation could synchronise or fail).
 *   m [n_cells], v [dim][n_cells], e [n_cells]: device arrays (masses, velocities, specific
 *   total energies, e.g. filled by lmood_get with is_device = 1); out5: device array of 5
 *   doubles receiving sum m, sum m v (3; z = 0 in 2D), sum m e. Ordered on stream; returns
 *   without synchronising. Sums are taken in a fixed order, so repeated calls agree bitwise.
 * Scratch is a fixed file-scope device array of 256 KiB (per GPU, held until exit), so
 * n_cells is limited to 16,777,216: larger sizes return LMOOD_ERR_ARG. The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress), and so does the first
 * call after the device's context changed (e.g. after cudaDeviceReset, which drops the array
 * and its contents); make those calls outside any stream capture. All calls share the array: calls whose work overlaps on the GPU
 * race and must be ordered by the caller. Allocates nothing (no cudaMalloc / cudaFree).
 */
lmood_status lmood_totals_noalloc(int dim, int64_t n_cells, const double *m, const double *v, const double *e,
                                  double *out5, void *stream);

/*
 * Adjoint (reverse-mode gradients) of a stretch of steps, with every step's MOOD order mask
 * and time step frozen at their recorded values. Each step is then a smooth map of the state
 * (x, v_p per node; v, F per cell) and of the per-cell mu; the adjoint is the exact transpose
 * of its linearisation, written by hand kernel by kernel (no atomics, deterministic).
 * Both cascades are differentiated: at the limited level (P1 with Barth-Jespersen slopes) each
 * field's factor phi is differentiated with the corner and the stencil bound that set it
 * frozen (the bound's adjoint goes to the cell that holds it). Every material is differentiated: the neo-Hookean law,
 * every a of the shear energy family (Eq. familiy_energies) and the stiffened gas (whose
 * pressure depends on the internal energy e, which then carries an adjoint: see
 * lmood_tape_backward_e). Boundary faces of every kind are differentiated: slip and
 * clamped nodes, traction and pressure faces (their forces depend on the faces' area vectors,
 * hence on the positions), prescribed-velocity faces and contact walls (their multiplier
 * steps, with the set of walls a node is in contact with, and whether each multiplier step
 * applies, frozen like the order mask); the boundary values and contact walls themselves are
 * constants. lmood_tape_backward returns LMOOD_ERR_STATE if the mesh's boundary values, tags or
 * contact walls were changed after the recording. With the volumetric law of Eq. EOS_neoHook
 * the energy e has no influence on the other fields; lmood_tape_backward takes no adjoint of
 * it, lmood_tape_backward_e does.
 *
 * lmood_tape_record: runs n_steps ordinary lmood_step calls on s (the forward pass, with the
 *   MOOD loop and the dt rule as configured) and records what the reverse pass needs: the dt
 *   and the final order mask of every step, and
 *     checkpoint_every = 0 (store mode): every state and every step's corner packets, the
 *       predictor's stress sums, nodal solver velocities and node moments (while recording,
 *       the steps also write the stress sums, which ordinary steps skip); the reverse pass
 *       reads them in place (fastest). Device memory: about n_steps + 1 states plus n_steps
 *       step products (a state is (4 dim + dim^2 + 3) doubles per cell-or-node; the products
 *       (dim+1)(dim(dim+1)/2 + dim) + dim doubles per cell and
 *       dim + 1 + dim + dim(dim+1)/2 + (dim + dim^2)(dim + 1) per node);
 *     checkpoint_every = C >= 1: a checkpoint of the state every C steps; the reverse pass
 *       rebuilds each segment from its checkpoint (one replay of each step, keeping the
 *       segment's states and products) and runs its reverse kernels on them. Device memory:
 *       about ceil(n_steps / C) + C states plus C step products.
 *   Both modes also hold n_steps (n_cells + 8 n_inst) bytes of masks and dts, and the adjoint
 *   work arrays (about 5 states). last (may be NULL) gets the last step's report. If a step
 *   fails, its status is returned, no tape is made (*out = NULL), and the state has taken the
 *   steps before it. If s was just initialised (no step and no lmood_set since
 *   lmood_state_init), v_p at the start is the initial nodal solve of (v, F, mu) and the
 *   reverse pass differentiates through it.
 * lmood_tape_backward: given the adjoints of the final state (lam_x, lam_vp [dim][n_nodes],
 *   lam_v [dim][n_cells], lam_F [dim*dim][n_cells]; NULL = zero), computes the gradients with
 *   respect to the state at the start of the tape: grad_x, grad_vp [dim][n_nodes] (at fixed
 *   cell masses), grad_v [dim][n_cells], grad_F [dim*dim][n_cells], and grad_mu [n_cells]
 *   (accumulated over the steps; mu enters the stress, the impedance and kappa). When the tape
 *   starts from a just-initialised state, grad_v, grad_F and grad_mu are the gradients with
 *   respect to the inputs of lmood_state_init, grad_x includes the positions' part of the
 *   initial nodal solve (at the same fixed masses), and grad_vp is zero. Any output may be NULL.
 *   Pointers are device pointers when is_device != 0 (ordered on the mesh's stream), else
 *   host pointers (the call synchronises). s's fields are left as they are, except the
 *   diagnostic fields PKM and PKR when the tape starts from a just-initialised state. Results
 *   are bitwise the same in both modes and for every C. May be called repeatedly.
 * lmood_tape_replay: advances the state s2 (any state on a mesh of the same sizes, e.g. one
 *   initialised from perturbed data) by the first n_steps recorded steps, from its current
 *   fields, with the recorded orders and dt and no MOOD detection or dt rule: the smooth map
 *   whose gradient lmood_tape_backward computes. s2's next dt is then set by the usual rule,
 *   so it can go on with lmood_step. Synchronises once per step.
 * lmood_tape_info: out4[0] steps, [1] checkpoint interval (0: store mode), [2] 1 if the tape
 *   starts from a just-initialised state, [3] device bytes held.
 * Destroy the tape before its state. (Destroyed out of order -- a mesh before its states, a
 * state before its tapes, as a garbage collector may do -- the dependent handles stay
 * destroyable and every other call on them returns an error.)
 */
typedef struct lmood_tape_s *lmood_tape;
lmood_status lmood_tape_record(lmood_state s, int64_t n_steps, int64_t checkpoint_every, lmood_tape *out,
                               lmood_step_info *last);
lmood_status lmood_tape_backward(lmood_tape t, const double *lam_x, const double *lam_vp, const double *lam_v,
                                 const double *lam_F, double *grad_x, double *grad_vp, double *grad_v,
                                 double *grad_F, double *grad_mu, int is_device);
/* The same with the energy: lam_e [n_cells] the adjoint of the final e (NULL = 0) and grad_e
 * [n_cells] the gradient with respect to the starting e (NULL: not wanted; zero when the tape
 * starts from a just-initialised state, whose e is a function of v, F and mu, through which
 * the gradient then goes). With the stiffened gas e enters the pressure, so it always carries
 * an adjoint; with the volumetric law of Eq. EOS_neoHook it has none unless lam_e is given. */
lmood_status lmood_tape_backward_e(lmood_tape t, const double *lam_x, const double *lam_vp, const double *lam_v,
                                   const double *lam_F, const double *lam_e, double *grad_x, double *grad_vp,
                                   double *grad_v, double *grad_F, double *grad_e, double *grad_mu, int is_device);
lmood_status lmood_tape_replay(lmood_tape t, lmood_state s2, int64_t n_steps);
lmood_status lmood_tape_info(lmood_tape t, int64_t *out4);
lmood_status lmood_tape_destroy(lmood_tape t);

const char *lmood_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LMOOD_H */
