// lmood_ops.h -- per-dimension launch table of the step kernels (one translation unit per
// dimension fills it).
#pragma once
#include "lmood_dev.cuh"

namespace lmood {

// arguments of the persistent step (lmood_persistent.cuh)
struct PersistArgs {
    int *tl0, *tl1;                 // troubled lists of the two round parities
    int *nlist, *clist, *node_mark, *cell_mark;
    Ctl *ctl;
    Report *report;
    unsigned int *bar;              // [0] arrivals, [1] generation, [2] timeout flag (zero at launch)
    int max_iters, n_inst;
    long long max_spin;             // barrier wait bound in polls of ~0.1 us
};

struct Ops {
    int dim;
    int nmom;  // node moments per node
    void (*moments)(const Geo &, const Fld &, cudaStream_t);
    void (*predict)(const Geo &, const Fld &, const Prm &, const int *list, const int *cnt, int n, cudaStream_t);
    void (*nodes)(const Geo &, const Fld &, const int *list, const int *cnt, int n, int init_mode, cudaStream_t);
    void (*update)(const Geo &, const Fld &, const Prm &, const int *list, const int *cnt, int n, int *tlist,
                   int *tcnt, cudaStream_t);
    void (*mark_nodes)(const Geo &, const Fld &, const Prm &, const int *tlist, const int *tcnt, int n, int *node_mark,
                       const Ctl *ctl, int *nlist, cudaStream_t);
    void (*mark_cells)(const Geo &, const Fld &, const int *nlist, int n, int *cell_mark, const Ctl *ctl,
                       int *clist, cudaStream_t);
    void (*round_begin)(const Fld &, Ctl *ctl, int in, int out, int max_iters, cudaStream_t);
    void (*ctl_reset)(Ctl *ctl, cudaStream_t);
    void (*loop_cond)(cudaGraphConditionalHandle h, const Fld &, const Ctl *ctl, cudaStream_t);
    void (*report)(const Fld &, const Ctl *ctl, Report *r, cudaStream_t);
    void (*dt_init)(const Fld &, const Prm &, int n_inst, int first, cudaStream_t);
    void (*finalize)(const Geo &, const Fld &, const Prm &, cudaStream_t);
    void (*init_cells)(const Geo &, const Fld &, const Prm &, double rho0, double *m, double *im, int f_given,
                       cudaStream_t);
    void (*refresh)(const Geo &, const Fld &, const Prm &, cudaStream_t);
    // the cells' geometry at the current positions into f.gf (views of recorded states)
    void (*geometry)(const Geo &, const Fld &, cudaStream_t);
    void (*totals)(const Geo &, const Fld &, double *out, cudaStream_t);
    // the whole step as one cooperative launch (neo-Hookean material)
    cudaError_t (*persistent)(const Geo &, const Fld &, const Prm &, const PersistArgs &, cudaStream_t);
    // the MOOD loop alone as one cooperative launch (capturable in a graph)
    cudaError_t (*mood_persistent)(const Geo &, const Fld &, const Prm &, const PersistArgs &, cudaStream_t);
};

const Ops &ops_dim2();
const Ops &ops_dim3();

}  // namespace lmood
