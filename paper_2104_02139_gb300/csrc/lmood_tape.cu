// lmood_tape.cu -- recording of a stretch of steps and its reverse pass (lmood_tape_* in
// include/lmood.h): the adjoint of the step with the MOOD order mask and dt frozen.
//
// Record: ordinary steps; before each, the dt it will use; after each, its final order mask;
// every C steps, a checkpoint of the state (x, v_p, v, F, e, z, rho, x_c).
// Reverse, per segment of C steps from the last: the segment is rebuilt from its checkpoint by
// replaying its steps (the step kernels with the recorded dt and orders given, no detection),
// each replay writing the next state and the step's products (corner packets, v*_p, node
// moments) straight into segment storage; then the reverse kernels of the segment's steps run,
// last step first, reading that storage in place. Store mode (C = 0): the recording keeps
// every state and every step's products, and the reverse kernels read them in place: no
// replay. In both modes the state's own fields are left as they are.
#include <algorithm>
#include <string>

#include "lmood_adj_ops.h"
#include "lmood_adjoint.cuh"
#include "lmood_internal.h"

using namespace lmood;

struct lmood_tape_s {
    lmood_state s = nullptr;
    const AdjOps *aop = nullptr;
    int64_t n = 0, C = 1, n_ck = 0, bytes = 0, pd = 0;
    uint64_t bc_version = 0;        // the mesh's boundary data the steps were taken with
    bool at_init = false, store = false;
    double *prod = nullptr;         // store mode: [n] products of each step (pkM, pkR, the
                                    // predictor's stress sums, the nodal v*_p, moments); checkpoint
                                    // mode: [C] products of the segment's steps
    double *dvb = nullptr;          // store mode: the predictor's stress sums the recorded steps write
    double *dts = nullptr;          // [n][n_inst]
    unsigned char *masks = nullptr; // [n][N]
    double *ck = nullptr;           // [n_ck] snapshots of the states at steps 0, C, 2C, ...
    double *seg = nullptr;          // checkpoint mode: [C] snapshots of a segment's states after
                                    // its first (the first is its checkpoint)
    unsigned char *tmp_order = nullptr;  // [N] scratch orders of the initial packets
    double *gf = nullptr, *gf1 = nullptr;  // the views' cell geometry at x^n, x^{n+1} (the state's
                                           // own buffers carry its current geometry)
    std::vector<char> bjs;          // [n] 1 if step j has cells at the limited (Barth-Jespersen) level
    double *bj = nullptr;           // their reverse records [N][B_LEN] (allocated when some step has)
    int *bjl = nullptr, *bjn = nullptr;  // the list of those cells in a replay, and its length
    AdjBuf a{};
    DevAllocs mem;
};

namespace {

// a snapshot of the t^n fields, one contiguous block
struct Snap {
    double *x, *vp, *v, *F, *e, *z, *rho, *xc;
};

int64_t snap_doubles(int D, int64_t N, int64_t Np) { return 2 * D * Np + (2 * D + D * D + 3) * N; }

Snap snap_at(double *base, int D, int64_t N, int64_t Np) {
    Snap q;
    q.x = base;
    q.vp = q.x + D * Np;
    q.v = q.vp + D * Np;
    q.F = q.v + D * N;
    q.e = q.F + D * D * N;
    q.z = q.e + N;
    q.rho = q.z + N;
    q.xc = q.rho + N;
    return q;
}

Snap cur_of(const Fld &f) { return Snap{f.x, f.vp, f.v, f.F, f.e, f.z, f.rho, f.xc}; }

// the products of one step the reverse kernels read, one contiguous block
struct Prod {
    double *pkM, *pkR, *dvs, *vs, *mom;
};

// a step's products: the corner packets, the second-order cells' predictor stress sums (of
// their half-step velocity increments), the nodal solver's v*_p and the node moments
int64_t prod_doubles(int D, int nmom, int64_t N, int64_t Np) {
    return (int64_t)(D * (D + 1) / 2 + D) * (D + 1) * N + (int64_t)D * N + (int64_t)(D + nmom) * Np;
}

Prod prod_at(double *base, int D, int64_t N, int64_t Np) {
    const int64_t NC = (int64_t)(D + 1) * N;
    Prod q;
    q.pkM = base;
    q.pkR = q.pkM + (int64_t)D * (D + 1) / 2 * NC;
    q.dvs = q.pkR + D * NC;
    q.vs = q.dvs + D * N;
    q.mom = q.vs + D * Np;
    return q;
}

cudaError_t copy_snap(const Snap &dst, const Snap &src, int D, int64_t N, int64_t Np, cudaStream_t st) {
    const size_t nd = sizeof(double);
    const std::pair<double *, const double *> ps[8] = {{dst.x, src.x}, {dst.vp, src.vp}, {dst.v, src.v},
                                                       {dst.F, src.F}, {dst.e, src.e},   {dst.z, src.z},
                                                       {dst.rho, src.rho}, {dst.xc, src.xc}};
    const int64_t len[8] = {D * Np, D * Np, D * N, D * D * N, N, N, N, D * N};
    for (int i = 0; i < 8; ++i) {
        cudaError_t e = cudaMemcpyAsync(ps[i].first, ps[i].second, len[i] * nd, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// one step of the forward scheme on the state's buffers with the recorded dt and orders
// (t^n in the current buffers -> packets, v*_p and t^{n+1} in the candidate buffers)
// the cells at the limited level (order 3) into a list
__global__ static void k_order3_list(const unsigned char *order, int n, int *list, int *cnt) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n && order[c] == 3) list[atomicAdd(cnt, 1)] = c;
}

// a replay's predictor: every cell in one launch (its orders given), then the cells at the
// limited level again with their limited slopes (a list launch, as the MOOD loop computed them)
void replay_predict(lmood_tape t, int64_t j, const Ops &op, const Geo &geo, const Fld &f, const Prm &kr, int N,
                    cudaStream_t st) {
    op.predict(geo, f, kr, nullptr, nullptr, N, st);
    if (!t->bjs[j]) return;
    cudaMemsetAsync(t->bjn, 0, sizeof(int), st);
    k_order3_list<<<(N + 255) / 256, 256, 0, st>>>(f.order, N, t->bjl, t->bjn);
    op.predict(geo, f, kr, t->bjl, t->bjn, N, st);
}

lmood_status replay_step(lmood_tape t, int64_t j, lmood_state s) {
    lmood_mesh M = s->M;
    const Ops &op = *M->ops;
    const Fld &f = s->f;
    cudaStream_t st = M->st;
    const int N = (int)M->nc, Np = (int)M->np;
    LM_CUDA(cudaMemcpyAsync(const_cast<double *>(f.dt), t->dts + j * M->n_inst, M->n_inst * sizeof(double),
                            cudaMemcpyDeviceToDevice, st));
    LM_CUDA(cudaMemcpyAsync(f.order, t->masks + j * (int64_t)N, N, cudaMemcpyDeviceToDevice, st));
    Prm kr = s->kp;
    kr.base_order = 0;  // orders as recorded
    kr.mood = 0;        // no detection: the mask is frozen
    op.moments(M->geo, f, st);
    replay_predict(t, j, op, M->geo, f, kr, N, st);
    op.nodes(M->geo, f, nullptr, nullptr, Np, 0, st);
    op.update(M->geo, f, kr, nullptr, nullptr, N, s->tl[0], f.cnt + CNT_T0, st);
    return LMOOD_OK;
}

// a view of the state's fields with t^n = cur, t^{n+1} = nxt, the step's products in q and
// the recorded dt and orders of step j (fields outside these stay the state's own scratch)
Fld view(lmood_tape t, const Fld &base, const Snap &cur, const Snap &nxt, const Prod &q, int64_t j) {
    const lmood_mesh M = t->s->M;
    Fld fr = base;
    fr.x = cur.x;
    fr.vp = cur.vp;
    fr.v = cur.v;
    fr.F = cur.F;
    fr.e = cur.e;
    fr.z = cur.z;
    fr.rho = cur.rho;
    fr.xc = cur.xc;
    fr.x1 = nxt.x;
    fr.vp1 = nxt.vp;
    fr.v1 = nxt.v;
    fr.F1 = nxt.F;
    fr.e1 = nxt.e;
    fr.z1 = nxt.z;
    fr.rho1 = nxt.rho;
    fr.xc1 = nxt.xc;
    fr.pkM = q.pkM;
    fr.pkR = q.pkR;
    fr.dvs = q.dvs;  // a replay's predictor writes them, the reverse pass reads them
    fr.vs = q.vs;
    fr.mom = q.mom;
    fr.dt = t->dts + j * M->n_inst;
    fr.order = t->masks + j * M->nc;
    fr.gf = t->gf;
    fr.gf1 = t->gf1;
    return fr;
}

// the step kernels through a view (orders as recorded, no detection): t^n -> products, t^{n+1}.
// geo: compute the view's x^n geometry first (else f.gf already holds it: the previous replay's
// update wrote it, as the recorded step read it)
void replay_view(lmood_tape t, const Fld &fr, bool geo, int64_t j) {
    lmood_state s = t->s;
    lmood_mesh M = s->M;
    const Ops &op = *M->ops;
    cudaStream_t st = M->st;
    Prm kr = s->kp;
    kr.base_order = 0;
    kr.mood = 0;
    if (geo) op.geometry(M->geo, fr, st);  // the state's own geometry is of another time
    op.moments(M->geo, fr, st);
    replay_predict(t, j, op, M->geo, fr, kr, (int)M->nc, st);
    op.nodes(M->geo, fr, nullptr, nullptr, (int)M->np, 0, st);
    op.update(M->geo, fr, kr, nullptr, nullptr, (int)M->nc, s->tl[0], fr.cnt + CNT_T0, st);
}

// the reverse kernels of one step, reading t^n, t^{n+1} and the step's products through f
void reverse_step(lmood_tape t, AdjBuf &a, const Fld &f, int64_t j) {
    lmood_state s = t->s;
    lmood_mesh M = s->M;
    const AdjOps &ao = *t->aop;
    cudaStream_t st = M->st;
    Prm kr = s->kp;
    kr.base_order = 0;
    kr.mood = 0;
    a.bj = t->bjs[j] ? t->bj : nullptr;
    ao.update(M->geo, f, kr, a, st);
    ao.nodes(M->geo, f, a, 0, st);
    ao.predict(M->geo, f, kr, a, 0, st);
    ao.bj_gather(M->geo, f, a, st);
    ao.momsum(M->geo, f, a, st);
    ao.cells(M->geo, f, kr, a, 1, st);
    ao.faces(M->geo, f, a, st);
    ao.gather(M->geo, a, st);
    std::swap(a.lv0, a.lv1);
    std::swap(a.lF0, a.lF1);
    std::swap(a.lE0, a.lE1);
    std::swap(a.lx0, a.lx1);
    std::swap(a.lvp0, a.lvp1);
}

lmood_status copy_in(double *dst, const double *src, int64_t n, int is_device, cudaStream_t st) {
    if (!src) LM_CUDA(cudaMemsetAsync(dst, 0, n * sizeof(double), st));
    else
        LM_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                st));
    return LMOOD_OK;
}

lmood_status copy_out(double *dst, const double *src, int64_t n, int is_device, cudaStream_t st) {
    if (dst)
        LM_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                st));
    return LMOOD_OK;
}

void tape_free(lmood_tape t) {
    if (t->s) {
        if (t->s->M) cudaStreamSynchronize(t->s->M->st);
        auto &v = t->s->tapes;
        v.erase(std::remove(v.begin(), v.end(), t), v.end());
    }
    t->mem.release();
    delete t;
}

}  // namespace

void lmood::tapes_orphan(lmood_state_s *s) {
    for (lmood_tape t : s->tapes) t->s = nullptr;
    s->tapes.clear();
}

extern "C" lmood_status lmood_tape_record(lmood_state s, int64_t n_steps, int64_t checkpoint_every, lmood_tape *out,
                                          lmood_step_info *last) {
    if (!out) return fail(LMOOD_ERR_ARG, "lmood_tape_record: out is NULL");
    *out = nullptr;
    if (!s) return fail(LMOOD_ERR_ARG, "lmood_tape_record: NULL state");
    if (s->broken) return fail(LMOOD_ERR_STATE, "lmood_tape_record: state unusable after an earlier CUDA error");
    if (n_steps < 1 || checkpoint_every < 0)
        return fail(LMOOD_ERR_ARG, "lmood_tape_record: n_steps must be >= 1 and checkpoint_every >= 0");
    lmood_mesh M = s->M;
    const int D = M->dim, NV = D + 1, NS = D * (D + 1) / 2, DD = D * D;
    const int64_t N = M->nc, Np = M->np, NC = NV * N;
    const int nmom = M->ops->nmom;
    auto *t = new lmood_tape_s();
    t->s = s;
    t->aop = D == 2 ? &adj_ops_dim2() : &adj_ops_dim3();
    t->n = n_steps;
    t->bjs.assign((size_t)n_steps, 0);
    t->store = checkpoint_every == 0;
    t->C = t->store ? 1 : std::min(checkpoint_every, n_steps);
    t->n_ck = t->store ? n_steps + 1 : (n_steps + t->C - 1) / t->C;
    t->at_init = s->at_init;
    t->bc_version = M->bc_version;
    const int64_t sd = snap_doubles(D, N, Np);
    t->pd = prod_doubles(D, nmom, N, Np);
    const size_t nd = sizeof(double);
    lmood_status r = LMOOD_OK;
    auto A = [&](void **p, size_t bytes) {
        if (r == LMOOD_OK) {
            r = t->mem.alloc(p, bytes);
            t->bytes += (int64_t)bytes;
        }
    };
    A((void **)&t->dts, n_steps * M->n_inst * nd);
    A((void **)&t->masks, (size_t)(n_steps * N));
    A((void **)&t->ck, t->n_ck * sd * nd);
    if (t->store) {
        A((void **)&t->prod, n_steps * t->pd * nd);
        A((void **)&t->dvb, (size_t)D * N * nd);
    } else {
        A((void **)&t->prod, t->C * t->pd * nd);
        A((void **)&t->seg, t->C * sd * nd);
    }
    A((void **)&t->tmp_order, (size_t)N);
    A((void **)&t->gf, (size_t)cell_geo_len(D) * N * nd);
    A((void **)&t->gf1, (size_t)cell_geo_len(D) * N * nd);
    AdjBuf &a = t->a;
    A((void **)&a.lv1, D * N * nd);
    A((void **)&a.lv0, D * N * nd);
    A((void **)&a.lF1, DD * N * nd);
    A((void **)&a.lF0, DD * N * nd);
    A((void **)&a.lz0, N * nd);
    A((void **)&a.lE1, N * nd);
    A((void **)&a.lE0, N * nd);
    A((void **)&a.lmu, N * nd);
    A((void **)&a.lx1, D * Np * nd);
    A((void **)&a.lx0, D * Np * nd);
    A((void **)&a.lvp1, D * Np * nd);
    A((void **)&a.lvp0, D * Np * nd);
    const int CR = NS + D + 5 * D, CP = D + (D + DD) + D + 1, CC = (D + DD) * D + NS;
    A((void **)&a.cr, (size_t)CR * NC * nd);
    A((void **)&a.cp, (size_t)CP * NC * nd);
    A((void **)&a.cc, (size_t)CC * N * nd);
    A((void **)&a.cd, (size_t)D * NC * nd);
    {
        const int FL = D == 2 ? adj::PredRec<2>::F_LEN : adj::PredRec<3>::F_LEN;
        const int KL = D == 2 ? adj::PredRec<2>::K_LEN : adj::PredRec<3>::K_LEN;
        const int Q2L = D == 2 ? adj::PredRec<2>::Q2_LEN : adj::PredRec<3>::Q2_LEN;
        const int Q1L = D == 2 ? adj::PredRec<2>::Q1_LEN : adj::PredRec<3>::Q1_LEN;
        A((void **)&a.pf, (size_t)FL * N * nd);
        A((void **)&a.pk, (size_t)KL * NC * nd);
        A((void **)&a.q2, (size_t)Q2L * NC * nd);
        A((void **)&a.q1, (size_t)Q1L * NC * nd);
    }
    // (its own buffer: the cell kernel after the moment sums still reads the corner records)
    A((void **)&a.lm, (size_t)nmom * Np * nd);
    if (M->has_ext && M->nb > 0) A((void **)&a.bf, (size_t)M->nb * DD * nd);
    if (r) {
        tape_free(t);
        return r;
    }
    cudaStream_t st = M->st;
    Fld &f = s->f;
    // while the whole trajectory is recorded, the steps also write the second-order cells'
    // predictor stress sums (into dvb, copied into each step's products); the state's
    // step graphs are re-captured with and again without them
    struct DvOn {
        lmood_state s;
        bool on;
        DvOn(lmood_state s_, double *buf) : s(s_), on(buf != nullptr) {
            if (on) {
                s->f.dvs = buf;
                graphs_reset(s);
            }
        }
        ~DvOn() {
            if (on) {
                s->f.dvs = nullptr;
                graphs_reset(s);
            }
        }
    } dv_on(s, t->dvb);
    for (int64_t j = 0; j < n_steps; ++j) {
        cudaError_t e = cudaSuccess;
        if (j % t->C == 0) e = copy_snap(snap_at(t->ck + (j / t->C) * sd, D, N, Np), cur_of(f), D, N, Np, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(t->dts + j * M->n_inst, f.dt, M->n_inst * nd, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) {
            tape_free(t);
            return fail(LMOOD_ERR_CUDA, std::string("lmood_tape_record: ") + cudaGetErrorString(e));
        }
        lmood_step_info info{};
        r = lmood_step(s, &info);
        if (last) *last = info;
        if (r) {
            tape_free(t);
            return r;
        }
        t->bjs[j] = info.n_lim > 0;
        if (info.n_lim > 0 && !t->bj) {  // the first step with limited cells: their buffers
            const size_t BL = D == 2 ? adj::PredRec<2>::B_LEN : adj::PredRec<3>::B_LEN;
            lmood_status ra = t->mem.alloc((void **)&t->bj, BL * N * nd);
            if (!ra) ra = t->mem.alloc((void **)&t->bjl, N * sizeof(int));
            if (!ra) ra = t->mem.alloc((void **)&t->bjn, sizeof(int));
            if (ra) {
                tape_free(t);
                return ra;
            }
            t->bytes += (int64_t)(BL * N * nd + N * sizeof(int) + sizeof(int));
        }
        e = cudaMemcpyAsync(t->masks + j * N, f.order, N, cudaMemcpyDeviceToDevice, st);
        if (t->store && e == cudaSuccess) {
            const Prod q = prod_at(t->prod + j * t->pd, D, N, Np);
            const std::pair<double *, const double *> cp[5] = {{q.pkM, f.pkM}, {q.pkR, f.pkR}, {q.dvs, f.dvs},
                                                               {q.vs, f.vs}, {q.mom, f.mom}};
            const int64_t len[5] = {NS * NC, D * NC, D * N, D * Np, nmom * Np};
            for (int i = 0; i < 5 && e == cudaSuccess; ++i)
                e = cudaMemcpyAsync(cp[i].first, cp[i].second, len[i] * nd, cudaMemcpyDeviceToDevice, st);
        }
        if (e != cudaSuccess) {
            tape_free(t);
            return fail(LMOOD_ERR_CUDA, std::string("lmood_tape_record: ") + cudaGetErrorString(e));
        }
    }
    if (t->store) {  // the final state, t^{n+1} of the last step
        cudaError_t e = copy_snap(snap_at(t->ck + n_steps * sd, D, N, Np), cur_of(f), D, N, Np, st);
        if (e != cudaSuccess) {
            tape_free(t);
            return fail(LMOOD_ERR_CUDA, std::string("lmood_tape_record: ") + cudaGetErrorString(e));
        }
    }
    r = sync_check(s, "lmood_tape_record");
    if (r) {
        tape_free(t);
        return r;
    }
    s->tapes.push_back(t);
    *out = t;
    return LMOOD_OK;
}

extern "C" lmood_status lmood_tape_backward(lmood_tape t, const double *lam_x, const double *lam_vp,
                                            const double *lam_v, const double *lam_F, double *grad_x,
                                            double *grad_vp, double *grad_v, double *grad_F, double *grad_mu,
                                            int is_device) {
    return lmood_tape_backward_e(t, lam_x, lam_vp, lam_v, lam_F, nullptr, grad_x, grad_vp, grad_v, grad_F, nullptr,
                                 grad_mu, is_device);
}

extern "C" lmood_status lmood_tape_backward_e(lmood_tape t, const double *lam_x, const double *lam_vp,
                                              const double *lam_v, const double *lam_F, const double *lam_e,
                                              double *grad_x, double *grad_vp, double *grad_v, double *grad_F,
                                              double *grad_e, double *grad_mu, int is_device) {
    if (!t || !t->s) return fail(LMOOD_ERR_ARG, "lmood_tape_backward: NULL tape, or its state was destroyed");
    lmood_state s = t->s;
    if (s->broken) return fail(LMOOD_ERR_STATE, "lmood_tape_backward: state unusable after an earlier CUDA error");
    if (s->M->bc_version != t->bc_version)
        return fail(LMOOD_ERR_STATE, "lmood_tape_backward: the mesh's boundary values, tags or contact walls changed "
                                     "after the tape was recorded");
    lmood_mesh M = s->M;
    const int D = M->dim;
    const int64_t N = M->nc, Np = M->np, sd = snap_doubles(D, N, Np);
    cudaStream_t st = M->st;
    Fld &f = s->f;
    const Ops &op = *M->ops;
    const AdjOps &ao = *t->aop;
    // adjoints of the final state; the energy's only when it is given or has influence (the
    // stiffened gas's pressure depends on it)
    AdjBuf a = t->a;
    const bool with_e = lam_e || s->mat.eos != 0;
    if (!with_e) a.lE0 = a.lE1 = nullptr;
    lmood_status r;
    if ((r = copy_in(a.lx1, lam_x, D * Np, is_device, st)) || (r = copy_in(a.lvp1, lam_vp, D * Np, is_device, st)) ||
        (r = copy_in(a.lv1, lam_v, D * N, is_device, st)) || (r = copy_in(a.lF1, lam_F, D * D * N, is_device, st)) ||
        (with_e && (r = copy_in(a.lE1, lam_e, N, is_device, st))))
        return r;
    LM_CUDA(cudaMemsetAsync(a.lmu, 0, N * sizeof(double), st));
    auto ck = [&](int64_t i) { return snap_at(t->ck + i * sd, D, N, Np); };
    // store mode: step j reads states j, j+1 and products j of the tape
    auto stored = [&](int64_t j) { return view(t, f, ck(j), ck(j + 1), prod_at(t->prod + j * t->pd, D, N, Np), j); };
    if (t->store) {
        for (int64_t j = t->n - 1; j >= 0; --j) reverse_step(t, a, stored(j), j);
    } else {
        // the segment's states: S(0) = its checkpoint, S(i) = seg[i - 1]; products P(i) = prod[i]
        for (int64_t k = t->n_ck - 1; k >= 0; --k) {
            const int64_t b = k * t->C, len = std::min(t->C, t->n - b);
            auto S = [&](int64_t i) { return i == 0 ? ck(k) : snap_at(t->seg + (i - 1) * sd, D, N, Np); };
            auto P = [&](int64_t i) { return prod_at(t->prod + i * t->pd, D, N, Np); };
            for (int64_t i = 0; i < len; ++i) {
                replay_view(t, view(t, f, S(i), S(i + 1), P(i), b + i), i == 0, b + i);
                std::swap(t->gf, t->gf1);  // the update's x^{n+1} geometry is the next replay's x^n
            }
            for (int64_t i = len - 1; i >= 0; --i) reverse_step(t, a, view(t, f, S(i), S(i + 1), P(i), b + i), b + i);
        }
    }
    if (t->at_init) {
        // v_p^0 = v* of the first-order packets of the initial state (read from the tape's
        // first checkpoint): the packets are rebuilt into the state's packet buffers, the
        // orders into a scratch array
        Fld f0 = view(t, f, ck(0), ck(0), prod_at(t->prod, D, N, Np), 0);
        f0.pkM = f.pkM;
        f0.pkR = f.pkR;
        f0.order = t->tmp_order;
        Prm p0 = s->kp;
        p0.base_order = 1;
        op.geometry(M->geo, f0, st);
        op.predict(M->geo, f0, p0, nullptr, nullptr, (int)N, st);
        AdjBuf ai = a;
        ai.lv0 = a.lv1;
        ai.lF0 = a.lF1;
        ai.lx0 = a.lx1;
        ai.lE0 = a.lE1;
        ai.bj = nullptr;  // the t^0 packets are first order
        ao.nodes(M->geo, f0, ai, 1, st);
        ao.predict(M->geo, f0, p0, ai, 1, st);
        ao.z0(M->geo, f0, p0, ai, st);
        ao.e0(M->geo, f0, p0, ai, st);  // e^0 is a function of v, F, mu
        // the positions' part of the initial solve (packets, impedance, boundary faces; the
        // corners' records of the cell gather carry nothing here)
        LM_CUDA(cudaMemsetAsync(a.cd, 0, (size_t)D * (D + 1) * N * sizeof(double), st));
        ao.faces(M->geo, f0, ai, st);
        ao.gather(M->geo, ai, st);
        LM_CUDA(cudaMemsetAsync(a.lvp1, 0, D * Np * sizeof(double), st));
    }
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) {
        s->broken = true;
        return fail(LMOOD_ERR_CUDA, std::string("lmood_tape_backward: ") + cudaGetErrorString(le));
    }
    if (grad_e && (!with_e || t->at_init)) {  // e has no influence, or the start's e is derived
        LM_CUDA(cudaMemsetAsync(t->a.lE1, 0, N * sizeof(double), st));
        a.lE1 = t->a.lE1;
    }
    if ((r = copy_out(grad_x, a.lx1, D * Np, is_device, st)) || (r = copy_out(grad_vp, a.lvp1, D * Np, is_device, st)) ||
        (r = copy_out(grad_v, a.lv1, D * N, is_device, st)) || (r = copy_out(grad_F, a.lF1, D * D * N, is_device, st)) ||
        (r = copy_out(grad_e, a.lE1, N, is_device, st)) || (r = copy_out(grad_mu, a.lmu, N, is_device, st)))
        return r;
    if (!is_device) return sync_check(s, "lmood_tape_backward");
    return LMOOD_OK;
}

extern "C" lmood_status lmood_tape_replay(lmood_tape t, lmood_state s2, int64_t n_steps) {
    if (!t || !t->s || !s2) return fail(LMOOD_ERR_ARG, "lmood_tape_replay: NULL argument, or the tape's state was destroyed");
    if (s2->broken || !t->s->M)
        return fail(LMOOD_ERR_STATE, "lmood_tape_replay: a state is unusable (an earlier CUDA error, or its mesh was "
                                     "destroyed)");
    const lmood_mesh M = s2->M, Mt = t->s->M;
    if (M->dim != Mt->dim || M->nc != Mt->nc || M->np != Mt->np || M->n_inst != Mt->n_inst)
        return fail(LMOOD_ERR_ARG, "lmood_tape_replay: the state's mesh differs in size from the tape's");
    if (n_steps < 0 || n_steps > t->n) return fail(LMOOD_ERR_ARG, "lmood_tape_replay: n_steps out of range");
    const Ops &op = *M->ops;
    cudaStream_t st = M->st;
    for (int64_t j = 0; j < n_steps; ++j) {
        lmood_status r = replay_step(t, j, s2);
        if (r) return r;
        // next dt from the candidates, as after an ordinary step, so that s2 can step on
        LM_CUDA(cudaMemsetAsync(s2->f.cnt, 0, CNT_N * sizeof(int), st));
        op.dt_init(s2->f, s2->kp, M->n_inst, 0, st);
        op.finalize(M->geo, s2->f, s2->kp, st);
        LM_CUDA(cudaMemcpyAsync(s2->h_dt, s2->f.dt, sizeof(double), cudaMemcpyDeviceToHost, st));
        lmood_status rs = sync_check(s2, "lmood_tape_replay");
        if (rs) return rs;
        swap_state(s2);
        s2->t += s2->h_dt[0];
        s2->step += 1;
        s2->at_init = false;
    }
    return LMOOD_OK;
}

extern "C" lmood_status lmood_tape_info(lmood_tape t, int64_t *out4) {
    if (!t || !out4) return fail(LMOOD_ERR_ARG, "lmood_tape_info: NULL argument");
    out4[0] = t->n;
    out4[1] = t->store ? 0 : t->C;
    out4[2] = t->at_init ? 1 : 0;
    out4[3] = t->bytes;
    return LMOOD_OK;
}

extern "C" lmood_status lmood_tape_destroy(lmood_tape t) {
    if (!t) return fail(LMOOD_ERR_ARG, "lmood_tape_destroy: NULL");
    tape_free(t);
    return LMOOD_OK;
}
