// lmood_tape.cu -- recording of a stretch of steps and its reverse pass (lmood_tape_* in
// include/lmood.h): the adjoint of the step with the MOOD order mask and dt frozen.
//
// Record: ordinary steps; before each, the dt it will use; after each, its final order mask;
// every C steps, a checkpoint of the state (x, v_p, v, F, e, z, rho, x_c).
// Reverse, per segment of C steps from the last: the segment's states are rebuilt from its
// checkpoint by replaying the steps (the step kernels with the recorded dt and orders given,
// no detection), then for each step from the last, the state t^n is loaded, the step replayed
// once more (packets, v*_p, t^{n+1} in the state's buffers) and the reverse kernels run.
// Store mode (C = 0): every state and every step's products (corner packets, v*_p, node
// moments) are kept, and the reverse kernels read them in place: no replay, no copies.
#include <algorithm>
#include <string>

#include "lmood_adj_ops.h"
#include "lmood_internal.h"

using namespace lmood;

struct lmood_tape_s {
    lmood_state s = nullptr;
    const AdjOps *aop = nullptr;
    int64_t n = 0, C = 1, n_ck = 0, bytes = 0, pd = 0;
    bool at_init = false, store = false;
    double *prod = nullptr;         // store mode: [n] products of each step (pkM, pkR, v*, moments)
    double *dts = nullptr;          // [n][n_inst]
    unsigned char *masks = nullptr; // [n][N]
    double *ck = nullptr;           // [n_ck] snapshots of the states at steps 0, C, 2C, ...
    double *seg = nullptr;          // [C - 1] snapshots of a segment's inner states
    double *tmp = nullptr;          // snapshot of the state's current fields during a reverse pass
    double *tmp_dt = nullptr;       // [n_inst]
    unsigned char *tmp_order = nullptr;  // [N]
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
Snap next_of(const Fld &f) { return Snap{f.x1, f.vp1, f.v1, f.F1, f.e1, f.z1, f.rho1, f.xc1}; }

// the products of one step the reverse kernels read, one contiguous block
struct Prod {
    double *pkM, *pkR, *vs, *mom;
};

int64_t prod_doubles(int D, int nmom, int64_t N, int64_t Np) {
    return (int64_t)(D * (D + 1) / 2 + D) * (D + 1) * N + (int64_t)(D + nmom) * Np;
}

Prod prod_at(double *base, int D, int64_t N, int64_t Np) {
    const int64_t NC = (int64_t)(D + 1) * N;
    Prod q;
    q.pkM = base;
    q.pkR = q.pkM + (int64_t)D * (D + 1) / 2 * NC;
    q.vs = q.pkR + D * NC;
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
    op.predict(M->geo, f, kr, nullptr, nullptr, N, st);
    op.nodes(M->geo, f, nullptr, nullptr, Np, 0, st);
    op.update(M->geo, f, kr, nullptr, nullptr, N, s->tl[0], f.cnt + CNT_T0, st);
    return LMOOD_OK;
}

// the reverse kernels of one step, reading t^n, t^{n+1} and the step's products through f
void reverse_step(lmood_tape t, AdjBuf &a, const Fld &f) {
    lmood_state s = t->s;
    lmood_mesh M = s->M;
    const AdjOps &ao = *t->aop;
    cudaStream_t st = M->st;
    Prm kr = s->kp;
    kr.base_order = 0;
    kr.mood = 0;
    ao.update(M->geo, f, kr, a, st);
    ao.nodes(M->geo, f, a, 0, st);
    ao.predict(M->geo, f, kr, a, 0, st);
    ao.momsum(M->geo, f, a, st);
    ao.cells(M->geo, f, kr, a, st);
    ao.gather(M->geo, a, st);
    std::swap(a.lv0, a.lv1);
    std::swap(a.lF0, a.lF1);
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
    if (t->s && t->s->M) cudaStreamSynchronize(t->s->M->st);
    t->mem.release();
    delete t;
}

}  // namespace

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
    t->store = checkpoint_every == 0;
    t->C = t->store ? 1 : std::min(checkpoint_every, n_steps);
    t->n_ck = t->store ? n_steps + 1 : (n_steps + t->C - 1) / t->C;
    t->at_init = s->at_init;
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
    } else {
        A((void **)&t->seg, (t->C - 1) * sd * nd);
        A((void **)&t->tmp, sd * nd);
    }
    A((void **)&t->tmp_dt, M->n_inst * nd);
    A((void **)&t->tmp_order, (size_t)N);
    AdjBuf &a = t->a;
    A((void **)&a.lv1, D * N * nd);
    A((void **)&a.lv0, D * N * nd);
    A((void **)&a.lF1, DD * N * nd);
    A((void **)&a.lF0, DD * N * nd);
    A((void **)&a.lz0, N * nd);
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
    if ((int64_t)nmom * Np <= (int64_t)CR * NC) a.lm = a.cr;  // written after the corner records are consumed
    else A((void **)&a.lm, (size_t)nmom * Np * nd);          // (meshes with unreferenced nodes)
    if (r) {
        tape_free(t);
        return r;
    }
    cudaStream_t st = M->st;
    Fld &f = s->f;
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
        if (info.n_lim > 0) {
            tape_free(t);
            return fail(LMOOD_ERR_ARG, "lmood_tape_record: step " + std::to_string(info.step) +
                                           " used the limited (Barth-Jespersen) level, which has no adjoint");
        }
        e = cudaMemcpyAsync(t->masks + j * N, f.order, N, cudaMemcpyDeviceToDevice, st);
        if (t->store && e == cudaSuccess) {
            const Prod q = prod_at(t->prod + j * t->pd, D, N, Np);
            const std::pair<double *, const double *> cp[4] = {{q.pkM, f.pkM}, {q.pkR, f.pkR}, {q.vs, f.vs},
                                                               {q.mom, f.mom}};
            const int64_t len[4] = {NS * NC, D * NC, D * Np, nmom * Np};
            for (int i = 0; i < 4 && e == cudaSuccess; ++i)
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
    *out = t;
    return LMOOD_OK;
}

extern "C" lmood_status lmood_tape_backward(lmood_tape t, const double *lam_x, const double *lam_vp,
                                            const double *lam_v, const double *lam_F, double *grad_x,
                                            double *grad_vp, double *grad_v, double *grad_F, double *grad_mu,
                                            int is_device) {
    if (!t || !t->s) return fail(LMOOD_ERR_ARG, "lmood_tape_backward: NULL tape");
    lmood_state s = t->s;
    if (s->broken) return fail(LMOOD_ERR_STATE, "lmood_tape_backward: state unusable after an earlier CUDA error");
    lmood_mesh M = s->M;
    const int D = M->dim;
    const int64_t N = M->nc, Np = M->np, sd = snap_doubles(D, N, Np);
    cudaStream_t st = M->st;
    Fld &f = s->f;
    const Ops &op = *M->ops;
    const AdjOps &ao = *t->aop;
    const Snap tmp = t->store ? Snap{} : snap_at(t->tmp, D, N, Np);
    if (!t->store) {  // keep the state's current fields (the replays run on its buffers)
        LM_CUDA(copy_snap(tmp, cur_of(f), D, N, Np, st));
        LM_CUDA(cudaMemcpyAsync(t->tmp_dt, f.dt, M->n_inst * sizeof(double), cudaMemcpyDeviceToDevice, st));
        LM_CUDA(cudaMemcpyAsync(t->tmp_order, f.order, N, cudaMemcpyDeviceToDevice, st));
    }
    // adjoints of the final state
    AdjBuf a = t->a;
    lmood_status r;
    if ((r = copy_in(a.lx1, lam_x, D * Np, is_device, st)) || (r = copy_in(a.lvp1, lam_vp, D * Np, is_device, st)) ||
        (r = copy_in(a.lv1, lam_v, D * N, is_device, st)) || (r = copy_in(a.lF1, lam_F, D * D * N, is_device, st)))
        return r;
    LM_CUDA(cudaMemsetAsync(a.lmu, 0, N * sizeof(double), st));
    const Snap cur = cur_of(f), nxt = next_of(f);
    // store mode: a view of step j's recorded data (state fields not read stay the state's own)
    auto stored = [&](int64_t j) {
        Fld fr = f;
        const Snap s0 = snap_at(t->ck + j * sd, D, N, Np), s1 = snap_at(t->ck + (j + 1) * sd, D, N, Np);
        const Prod q = prod_at(t->prod + j * t->pd, D, N, Np);
        fr.x = s0.x;
        fr.vp = s0.vp;
        fr.v = s0.v;
        fr.F = s0.F;
        fr.e = s0.e;
        fr.z = s0.z;
        fr.rho = s0.rho;
        fr.xc = s0.xc;
        fr.x1 = s1.x;
        fr.vp1 = s1.vp;
        fr.pkM = q.pkM;
        fr.pkR = q.pkR;
        fr.vs = q.vs;
        fr.mom = q.mom;
        fr.dt = t->dts + j * M->n_inst;
        fr.order = t->masks + j * N;
        return fr;
    };
    if (t->store)
        for (int64_t j = t->n - 1; j >= 0; --j) reverse_step(t, a, stored(j));
    for (int64_t k = t->store ? -1 : t->n_ck - 1; k >= 0; --k) {
        const int64_t b = k * t->C, len = std::min(t->C, t->n - b);
        const Snap ck = snap_at(t->ck + k * sd, D, N, Np);
        LM_CUDA(copy_snap(cur, ck, D, N, Np, st));
        for (int64_t i = 0; i + 1 < len; ++i) {  // states b+1 .. b+len-1 into seg[0 ..]
            if ((r = replay_step(t, b + i, s))) return r;
            LM_CUDA(copy_snap(snap_at(t->seg + i * sd, D, N, Np), nxt, D, N, Np, st));
            LM_CUDA(copy_snap(cur, nxt, D, N, Np, st));
        }
        for (int64_t i = len - 1; i >= 0; --i) {
            if (i < len - 1) LM_CUDA(copy_snap(cur, i == 0 ? ck : snap_at(t->seg + (i - 1) * sd, D, N, Np), D, N, Np, st));
            if ((r = replay_step(t, b + i, s))) return r;
            reverse_step(t, a, f);
        }
    }
    if (t->at_init) {
        // v_p^0 = v* of the first-order packets of the initial state: the packets are rebuilt
        // into the state's packet buffers (replay mode: the state's buffers hold t^0; store
        // mode: t^0 is read from the tape, the orders written to a scratch array)
        Fld f0 = f;
        if (t->store) {
            f0 = stored(0);
            f0.pkM = f.pkM;
            f0.pkR = f.pkR;
            f0.order = t->tmp_order;
        }
        Prm p0 = s->kp;
        p0.base_order = 1;
        op.predict(M->geo, f0, p0, nullptr, nullptr, (int)N, st);
        AdjBuf ai = a;
        ai.lv0 = a.lv1;
        ai.lF0 = a.lF1;
        ao.nodes(M->geo, f0, ai, 1, st);
        ao.predict(M->geo, f0, p0, ai, 1, st);
        ao.z0(M->geo, f0, p0, ai, st);
        LM_CUDA(cudaMemsetAsync(a.lvp1, 0, D * Np * sizeof(double), st));
    }
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) {
        s->broken = true;
        return fail(LMOOD_ERR_CUDA, std::string("lmood_tape_backward: ") + cudaGetErrorString(le));
    }
    if ((r = copy_out(grad_x, a.lx1, D * Np, is_device, st)) || (r = copy_out(grad_vp, a.lvp1, D * Np, is_device, st)) ||
        (r = copy_out(grad_v, a.lv1, D * N, is_device, st)) || (r = copy_out(grad_F, a.lF1, D * D * N, is_device, st)) ||
        (r = copy_out(grad_mu, a.lmu, N, is_device, st)))
        return r;
    if (!t->store) {  // the state's current fields back
        LM_CUDA(copy_snap(cur, tmp, D, N, Np, st));
        LM_CUDA(cudaMemcpyAsync(const_cast<double *>(f.dt), t->tmp_dt, M->n_inst * sizeof(double),
                                cudaMemcpyDeviceToDevice, st));
        LM_CUDA(cudaMemcpyAsync(f.order, t->tmp_order, N, cudaMemcpyDeviceToDevice, st));
    }
    if (!is_device) return sync_check(s, "lmood_tape_backward");
    return LMOOD_OK;
}

extern "C" lmood_status lmood_tape_replay(lmood_tape t, lmood_state s2, int64_t n_steps) {
    if (!t || !t->s || !s2) return fail(LMOOD_ERR_ARG, "lmood_tape_replay: NULL argument");
    if (s2->broken) return fail(LMOOD_ERR_STATE, "lmood_tape_replay: state unusable after an earlier CUDA error");
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
