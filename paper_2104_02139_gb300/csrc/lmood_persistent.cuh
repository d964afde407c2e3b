// lmood_persistent.cuh -- the whole step t^n -> t^{n+1} as one cooperative (persistent)
// launch: every block loops over cells or nodes of each stage (moments, predictor, nodal
// solve, update, then the MOOD rounds over their compacted lists, then the next dt and the
// step report), with a grid-wide barrier between stages. It runs the same per-cell and
// per-node functions as the per-stage kernels, so the results are bitwise the same; what it
// saves is the launch and graph-node latency of the ~10 + 6-per-MOOD-round stages, which
// dominates the step of small meshes.
//
// The barrier's waits are bounded: a block that has waited max_spin polls (each ~0.1 us) sets
// the timeout flag bar[2] and returns, and every block that sees the flag returns too, so a
// launch always ends; the host then reports LMOOD_ERR_TIMEOUT and keeps the state at t^n.
// Co-residency of all blocks is guaranteed by the cooperative launch (the grid is sized from
// the occupancy of this kernel).
#pragma once
#include "lmood_kernels.cuh"
#include "lmood_ops.h"

namespace lmood {

// grid-wide barrier with bounded waits; false when the launch must end (a timeout here or in
// another block)
__device__ __forceinline__ bool grid_sync(unsigned int *bar, long long max_spin) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *gen = bar + 1, *flag = bar + 2;
        const unsigned int g0 = *gen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);  // every block has arrived: reset, then release
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long i = 0;
            while (*gen == g0) {
                if (*flag) {
                    ok = 0;
                    break;
                }
                if (++i > max_spin) {
                    atomicExch(bar + 2, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        s_ok = ok && *flag == 0;
    }
    __syncthreads();
    return s_ok;
}

__device__ __forceinline__ int vload(const int *p) { return *(const volatile int *)p; }

// The MOOD rounds (as k_round_begin, k_mark_nodes, k_mark_cells and the list launches of
// the predictor, nodal solver and update) over the troubled list left in tl0 / cnt[CNT_T0];
// tid / nth: this thread's spread index and the grid's thread count. False when a barrier
// gave up.
template <int D, int MAT>
__device__ __forceinline__ bool mood_rounds(const Geo &g, const Fld &f, const Prm &prm, const PersistArgs &a, int tid,
                                            int nth) {
    for (int cur = 0;; cur ^= 1) {
        const int in = CNT_T0 + cur, out = CNT_T0 + (cur ^ 1);
        const int n_in = vload(f.cnt + in);  // written before the last barrier: the same in every block
        if (n_in == 0) return true;
        if (tid == 0) {
            if (a.ctl->iters >= a.max_iters) {
                a.ctl->err = 1;
            } else {
                a.ctl->iters += 1;
                a.ctl->troubled += n_in;
                a.ctl->stamp += 1;
            }
            f.cnt[out] = 0;
            f.cnt[CNT_NODES] = 0;
            f.cnt[CNT_CELLS] = 0;
        }
        if (!grid_sync(a.bar, a.max_spin)) return false;
        if (vload(&a.ctl->err)) return true;
        const int stamp = vload(&a.ctl->stamp);
        int *tin = cur ? a.tl1 : a.tl0, *tout = cur ? a.tl0 : a.tl1;
        mark_nodes_range<D>(g, f, prm, tin, n_in, a.node_mark, stamp, a.nlist, tid, nth);
        if (!grid_sync(a.bar, a.max_spin)) return false;
        const int nn = vload(f.cnt + CNT_NODES);
        mark_cells_range<kMarkLanes<D>>(g, f, a.nlist, nn, a.cell_mark, stamp, a.clist, tid, nth);
        if (!grid_sync(a.bar, a.max_spin)) return false;
        for (int i = tid; i < n_in; i += nth) predict_cell<D, true, MAT>(g, f, prm, tin[i]);
        if (!grid_sync(a.bar, a.max_spin)) return false;
        for (int i = tid; i < nn; i += nth) node_solve<D>(g, f, a.nlist[i], 0);
        if (!grid_sync(a.bar, a.max_spin)) return false;
        const int nc = vload(f.cnt + CNT_CELLS);
        for (int i = tid; i < nc; i += nth) update_cell<D>(g, f, prm, a.clist[i], tout, f.cnt + out);
        if (!grid_sync(a.bar, a.max_spin)) return false;
    }
}

// work item i goes to warp i / 32 of the grid counted block-fastest (warp w of block b is
// warp w * gridDim.x + b), so that a small mesh's cells spread over all SMs and their
// sub-partitions instead of filling the first blocks' warps
__device__ __forceinline__ int spread_index() {
    return ((threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32 + (threadIdx.x & 31);
}

#ifndef LMOOD_PERSIST_MINB2
#define LMOOD_PERSIST_MINB2 2
#endif

template <int D>
__global__ void __launch_bounds__(kCellBlock, D == 2 ? LMOOD_PERSIST_MINB2 : 1)
    k_step_persistent(Geo g, Fld f, Prm prm, PersistArgs a) {
    const int nth = gridDim.x * blockDim.x, tid = spread_index();
    const int N = g.N, Np = g.Np;
    // step set-up: counters, MOOD control, next-dt initial value (as k_ctl_reset, k_dt_init)
    if (tid == 0) {
        for (int i = 0; i < CNT_N; ++i) f.cnt[i] = 0;
        a.ctl->iters = 0;
        a.ctl->troubled = 0;
        a.ctl->err = 0;
    }
    for (int i = tid; i < a.n_inst; i += nth) {
        const double d = prm.dt_fixed > 0 ? prm.dt_fixed : (1.0 + prm.Ci) * f.dt[i];
        f.dtn[i] = (unsigned long long)__double_as_longlong(d);
    }
    if (!grid_sync(a.bar, a.max_spin)) return;
    for (int p = tid; p < Np; p += nth) moments_node<D>(g, f, g.node_perm[p]);
    if (!grid_sync(a.bar, a.max_spin)) return;
    for (int c = tid; c < N; c += nth) predict_cell<D, false, 0>(g, f, prm, c);
    if (!grid_sync(a.bar, a.max_spin)) return;
    for (int p = tid; p < Np; p += nth) node_solve<D>(g, f, kNodesByCount<D> ? g.node_perm[p] : p, 0);
    if (!grid_sync(a.bar, a.max_spin)) return;
    for (int c = tid; c < N; c += nth) update_cell<D>(g, f, prm, c, a.tl0, f.cnt + CNT_T0);
    if (!grid_sync(a.bar, a.max_spin)) return;
    if (!mood_rounds<D, 0>(g, f, prm, a, tid, nth)) return;
    // next dt and counters (as k_finalize), then the report (as k_report)
    for (int c0 = blockIdx.x * blockDim.x; c0 < N; c0 += nth) {
        finalize_block(g, f, prm, c0);
        __syncthreads();  // the block's shared partial sums are reused by the next chunk
    }
    if (!grid_sync(a.bar, a.max_spin)) return;
    if (tid == 0) {
        Report *r = a.report;
        r->n_troubled = a.ctl->troubled;
        r->mood_iters = a.ctl->iters;
        r->err = a.ctl->err;
        r->n_p0 = f.cnt[CNT_P0];
        r->n_para = f.cnt[CNT_PARA];
        r->n_eps = f.cnt[CNT_EPS];
        r->n_lim = f.cnt[CNT_LIM];
        r->dt_used = f.dt[0];
        r->dt_next = __longlong_as_double((long long)f.dtn[0]);
    }
}

// the MOOD loop alone as one cooperative launch (a node of the captured step graph, after
// the full-mesh update); a barrier that gives up marks the step with ctl->err = 2
template <int D, int MAT>
__global__ void __launch_bounds__(kCellBlock, D == 2 ? LMOOD_PERSIST_MINB2 : 1)
    k_mood_persistent(Geo g, Fld f, Prm prm, PersistArgs a) {
    const int nth = gridDim.x * blockDim.x, tid = spread_index();
    if (!mood_rounds<D, MAT>(g, f, prm, a, tid, nth) && threadIdx.x == 0) atomicExch(&a.ctl->err, 2);
}

}  // namespace lmood
