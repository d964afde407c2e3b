// lmood_ops_impl.cuh -- launchers of the step kernels for one dimension D (LMOOD_DIM).
#pragma once
#include "lmood_kernels.cuh"
#include "lmood_ops.h"
#include "lmood_persistent.cuh"

namespace lmood {
namespace {

inline int blocks(int n, int b) { return (n + b - 1) / b; }

// a full launch covers n entities one per thread; a list launch (list != NULL) uses at most
// kListBlocks blocks and loops over the device-counted list (n only bounds the grid)
inline int grid_for(const int *list, int n, int b) {
    const int g = blocks(n, b);
    return list && g > kListBlocks ? kListBlocks : g;
}

// full-mesh launches take the mesh's autotuned block size (g.blk); list launches keep the default
template <int D> void moments(const Geo &g, const Fld &f, cudaStream_t s) {
    switch (g.blk.moments) {
    case 128: k_moments<D, 128><<<blocks(g.Np, 128), 128, 0, s>>>(g, f); break;
    case 512: k_moments<D, 512><<<blocks(g.Np, 512), 512, 0, s>>>(g, f); break;
    default: k_moments<D, 256><<<blocks(g.Np, 256), 256, 0, s>>>(g, f); break;
    }
}
template <int D>
void predict(const Geo &g, const Fld &f, const Prm &p, const int *list, const int *cnt, int n, cudaStream_t s) {
    if (n <= 0) return;
    if (p.eos) {  // stiffened gas: its own instances
        if (list) k_predict<D, true, kCellBlock, 2><<<grid_for(list, n, kCellBlock), kCellBlock, 0, s>>>(g, f, p, list, cnt, n);
        else k_predict<D, false, kCellBlock, 2><<<blocks(n, kCellBlock), kCellBlock, 0, s>>>(g, f, p, list, cnt, n);
        return;
    }
    if (p.shear_a != -1.0) {  // another member of the shear energy family: its own instances
        if (list) k_predict<D, true, kCellBlock, 1><<<grid_for(list, n, kCellBlock), kCellBlock, 0, s>>>(g, f, p, list, cnt, n);
        else k_predict<D, false, kCellBlock, 1><<<blocks(n, kCellBlock), kCellBlock, 0, s>>>(g, f, p, list, cnt, n);
        return;
    }
    if (list) {
        k_predict<D, true><<<grid_for(list, n, kCellBlock), kCellBlock, 0, s>>>(g, f, p, list, cnt, n);
        return;
    }
    switch (g.blk.predict) {
    case 64: k_predict<D, false, 64><<<blocks(n, 64), 64, 0, s>>>(g, f, p, list, cnt, n); break;
    case 256: k_predict<D, false, 256><<<blocks(n, 256), 256, 0, s>>>(g, f, p, list, cnt, n); break;
    default: k_predict<D, false, 128><<<blocks(n, 128), 128, 0, s>>>(g, f, p, list, cnt, n); break;
    }
}
template <int D>
void nodes(const Geo &g, const Fld &f, const int *list, const int *cnt, int n, int init_mode, cudaStream_t s) {
    if (n <= 0) return;
    if (list) {
        k_nodes<D, true><<<grid_for(list, n, kNodeBlock), kNodeBlock, 0, s>>>(g, f, list, cnt, n, init_mode);
        return;
    }
    switch (g.blk.nodes) {
    case 128: k_nodes<D, false, 128><<<blocks(n, 128), 128, 0, s>>>(g, f, list, cnt, n, init_mode); break;
    case 512: k_nodes<D, false, 512><<<blocks(n, 512), 512, 0, s>>>(g, f, list, cnt, n, init_mode); break;
    default: k_nodes<D, false, 256><<<blocks(n, 256), 256, 0, s>>>(g, f, list, cnt, n, init_mode); break;
    }
}
template <int D>
void update(const Geo &g, const Fld &f, const Prm &p, const int *list, const int *cnt, int n, int *tlist, int *tcnt,
            cudaStream_t s) {
    if (n <= 0) return;
    if (list) {
        k_update<D, true><<<grid_for(list, n, kCellBlock), kCellBlock, 0, s>>>(g, f, p, list, cnt, n, tlist, tcnt);
        return;
    }
    switch (g.blk.update) {
    case 64: k_update<D, false, 64><<<blocks(n, 64), 64, 0, s>>>(g, f, p, list, cnt, n, tlist, tcnt); break;
    case 256: k_update<D, false, 256><<<blocks(n, 256), 256, 0, s>>>(g, f, p, list, cnt, n, tlist, tcnt); break;
    default: k_update<D, false, 128><<<blocks(n, 128), 128, 0, s>>>(g, f, p, list, cnt, n, tlist, tcnt); break;
    }
}
template <int D>
void mark_nodes(const Geo &g, const Fld &f, const Prm &p, const int *tlist, const int *tcnt, int n, int *node_mark,
                const Ctl *ctl, int *nlist, cudaStream_t s) {
    if (n > 0)
        k_mark_nodes<D><<<grid_for(tlist, (int)std::min<long long>((long long)n * (D + 1), 1 << 30), 256), 256, 0, s>>>(
            g, f, p, tlist, tcnt, node_mark, ctl, nlist);
}
template <int D>
void mark_cells(const Geo &g, const Fld &f, const int *nlist, int n, int *cell_mark, const Ctl *ctl, int *clist,
                cudaStream_t s) {
    if (n > 0)
        k_mark_cells<D><<<grid_for(nlist, (int)std::min<long long>((long long)n * kMarkLanes<D>, 1 << 30), 256), 256, 0, s>>>(
            g, f, nlist, cell_mark, ctl, clist);
}
void round_begin(const Fld &f, Ctl *ctl, int in, int out, int max_iters, cudaStream_t s) {
    k_round_begin<<<1, 1, 0, s>>>(f, ctl, in, out, max_iters);
}
void ctl_reset(Ctl *ctl, cudaStream_t s) { k_ctl_reset<<<1, 1, 0, s>>>(ctl); }
void loop_cond(cudaGraphConditionalHandle h, const Fld &f, const Ctl *ctl, cudaStream_t s) {
    k_loop_cond<<<1, 1, 0, s>>>(h, f, ctl);
}
void report(const Fld &f, const Ctl *ctl, Report *r, cudaStream_t s) { k_report<<<1, 1, 0, s>>>(f, ctl, r); }
void dt_init(const Fld &f, const Prm &p, int n_inst, int first, cudaStream_t s) {
    k_dt_init<<<blocks(n_inst, 128), 128, 0, s>>>(f, p, n_inst, first);
}
void finalize(const Geo &g, const Fld &f, const Prm &p, cudaStream_t s) {
    k_finalize<<<blocks(g.N, 256), 256, 0, s>>>(g, f, p);
}
template <int D>
void init_cells(const Geo &g, const Fld &f, const Prm &p, double rho0, double *m, double *im, int f_given,
                cudaStream_t s) {
    k_init_cells<D><<<blocks(g.N, kCellBlock), kCellBlock, 0, s>>>(g, f, p, rho0, m, im, f_given);
}
template <int D> void geometry(const Geo &g, const Fld &f, cudaStream_t s) {
    k_geometry<D><<<blocks(g.N, kCellBlock), kCellBlock, 0, s>>>(g, f);
}
template <int D> void refresh(const Geo &g, const Fld &f, const Prm &p, cudaStream_t s) {
    k_refresh<D><<<blocks(g.N, kCellBlock), kCellBlock, 0, s>>>(g, f, p);
}
template <int D> void totals(const Geo &g, const Fld &f, double *out, cudaStream_t s) {
    k_totals<D><<<blocks(g.N, 256), 256, 0, s>>>(g, f, out);
}
// cooperative launch of a persistent kernel: as many blocks as can be resident at once, or
// max_blocks if fewer (work is spread one warp per block first, so a small mesh needs no more
// blocks than it has warps of work, and fewer blocks make the grid barriers cheaper)
template <typename K>
static cudaError_t launch_cooperative(K kern, const Geo &g, const Fld &f, const Prm &p, const PersistArgs &a,
                                      cudaStream_t s, long long max_blocks) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCellBlock, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::max(1LL, std::min<long long>((long long)per_sm * sms, max_blocks)));
    cfg.blockDim = dim3(kCellBlock);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, g, f, p, a);
}
template <int D> cudaError_t persistent(const Geo &g, const Fld &f, const Prm &p, const PersistArgs &a, cudaStream_t s) {
    const long long items = std::max<long long>(std::max(g.N, g.Np), a.n_inst);
    return launch_cooperative(k_step_persistent<D>, g, f, p, a, s, (items + 31) / 32);
}
template <int D> cudaError_t mood_persistent(const Geo &g, const Fld &f, const Prm &p, const PersistArgs &a, cudaStream_t s) {
    const long long all = 1LL << 40;  // the lists' lengths are known on the device only
    if (p.eos) return launch_cooperative(k_mood_persistent<D, 2>, g, f, p, a, s, all);
    if (p.shear_a != -1.0) return launch_cooperative(k_mood_persistent<D, 1>, g, f, p, a, s, all);
    return launch_cooperative(k_mood_persistent<D, 0>, g, f, p, a, s, all);
}

}  // namespace

#define LMOOD_OPS_TABLE(D)                                                                                  \
    static const Ops table = {D, Dim<D>::NMOM, moments<D>, predict<D>, nodes<D>,  update<D>,     mark_nodes<D>, mark_cells<D>, \
                              round_begin, ctl_reset,  loop_cond, report,        dt_init,       finalize,   \
                              init_cells<D>, refresh<D>, geometry<D>, totals<D>, persistent<D>, mood_persistent<D>};                                      \
    return table;

}  // namespace lmood
